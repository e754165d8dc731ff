"""The N > 1 host path on CPU ranks (gloo, world size 2): the bench's
whole-job timing takes the slowest rank and counts every rank's units, and
under torchrun only rank 0 runs and prints the reference arm.  The data
path has no collective (replicas only), so this is all there is to test
without GPUs."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r is slower on the first value and faster on the second
        got = bench.reduce_max_over_ranks([10.0 + rank, 5.0 - rank, 2.5], ws)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(got, f)
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    for r in range(ws):
        assert json.load(open(tmp_path / f"rank{r}.json")) == [11.0, 5.0, 2.5]
    sys.path.insert(0, ROOT)
    import bench
    # every rank ran its own 1e7 histories; the job took the slowest 20 ms
    assert bench.job_throughput(2, 10_000_000, 20.0) == pytest.approx(1.0e9)
    assert bench.reduce_max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]


@pytest.mark.slow
def test_reference_arm_prints_once_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--reference-seconds", "0.3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
