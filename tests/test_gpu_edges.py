"""Edge and degenerate cases of the whole path on the GPU, each against the
oracle or an exact invariant: spots with no protons, histories fewer than
spots, beams that miss the grid, one-voxel and one-voxel-thick grids, the
spot limit, one-subvoxel accumulation on one voxel, a one-voxel
registration grid and a one-spot delivery."""
import numpy as np
import pytest
import torch

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _plan(xs, ys, es, protons, sigma=0.0):
    n = len(xs)
    return W.Plan(np.array(xs, float), np.array(ys, float), np.array(es, float), np.full(n, sigma),
                  np.array(protons, np.uint64), np.zeros(n, np.int32), np.zeros(n, np.int32))


def _ledger_balanced(led):
    dep, esc, rem, inc, steps = [int(v) for v in led[:5]]
    return abs(dep + esc + rem - inc) <= steps + inc * 2.0 ** -22


def test_spots_without_protons_and_fewer_histories_than_spots(gpu, orc):
    ph = W.water_phantom(16, 16, 40)
    plan = _plan([0, 2, -2, 4, 0], [0, 0, 1, -3, 2], [100, 90, 110, 80, 120], [0, 5, 0, 3, 1], sigma=1.0)
    for n in (1, 3, 9):
        r = H.gpu_run(gpu, ph, plan, n, 2)
        assert _ledger_balanced(r["ledger"]) and int(r["ledger"][5]) == n
        alloc = orc.allocate(plan.protons, n)
        assert alloc[0] == 0 and alloc[2] == 0
        # matched streams, no scattering: the same few histories on both sides
        g = H.gpu_run(gpu, ph, plan, n, 2, physics=5)["dose"]
        o, _ = H.oracle_batches(orc, ph, plan, n, 2, physics=5)
        assert np.max(np.abs(g - o)) <= 2e-3 * max(o.max(), 1e-30)


def test_plan_with_no_protons_gives_zero_dose(gpu):
    ph = W.water_phantom(8, 8, 8)
    r = H.gpu_run(gpu, ph, _plan([0, 1], [0, 1], [100, 120], [0, 0]), 1000, 1)
    assert r["dose"].max() == 0.0 and int(r["tally"].sum()) == 0
    assert int(r["ledger"][3]) == 0 and int(r["ledger"][7]) == 0


def test_beam_that_misses_the_grid_escapes_whole(gpu):
    ph = W.water_phantom(16, 16, 16)          # lateral extent [-16, 16] mm
    plan = _plan([40.0, -50.0], [0.0, 30.0], [150.0, 100.0], [1_000_000, 1_000_000])
    r = H.gpu_run(gpu, ph, plan, 20_000, 3)
    led = [int(v) for v in r["ledger"]]
    assert r["dose"].max() == 0.0
    assert led[0] == 0 and led[2] == 0 and led[1] == led[3] > 0


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 60), (40, 1, 40)])
def test_tiny_and_one_voxel_thick_grids(gpu, orc, shape):
    nx, ny, nz = shape
    ph = W.Phantom(np.zeros((nz, ny, nx), np.int16), (2.0, 2.0, 2.0), (-nx, -ny, 0.0), 2, 1)
    plan = _plan([0.0], [0.0], [120.0], [1_000_000], sigma=0.5)
    n = 20_000
    r = H.gpu_run(gpu, ph, plan, n, 4, physics=5)
    assert _ledger_balanced(r["ledger"])
    o, _ = H.oracle_batches(orc, ph, plan, n, 4, physics=5)
    assert np.max(np.abs(r["dose"] - o)) <= 2e-3 * o.max()


def test_spot_limit(gpu):
    """16384 spots (the largest plan a context takes) on a small phantom;
    one more is refused."""
    ph = W.water_phantom(32, 32, 64)
    rng = np.random.default_rng(5)
    n = 16384
    plan = _plan(rng.uniform(-20, 20, n), rng.uniform(-20, 20, n), rng.uniform(70, 130, n),
                 rng.integers(1, 1000, n), sigma=2.0)
    r = H.gpu_run(gpu, ph, plan, 200_000, 6)
    assert _ledger_balanced(r["ledger"]) and r["dose"].max() > 0
    big = _plan(np.zeros(n + 1), np.zeros(n + 1), np.full(n + 1, 100.0), np.ones(n + 1))
    ctx = H.make_ctx(gpu, ph)
    try:
        with pytest.raises(gpu.DoseError):
            gpu.dose_add_spots(ctx, gpu.spots_array(big), None)
    finally:
        gpu.dose_destroy(ctx)


def test_accumulation_on_one_voxel(gpu, orc):
    """EMTM and DIM with one subvoxel on a one-voxel, three-phase grid:
    every phase maps onto the voxel, so both give the phase sum."""
    P = 3
    hu = np.zeros((P, 1, 1, 1), np.int16)
    ctx = gpu.dose_create_grid(1, 1, 1, 2.0, 2.0, 2.0, (0.0, 0.0, 0.0), P, hu, (0.0, 0.0, 1.0))
    doses = np.array([0.5, 1.25, 2.0], np.float32).reshape(P, 1, 1, 1)
    try:
        for p in range(P):
            gpu.dose_set_phase_dose(ctx, p, np.ascontiguousarray(doses[p]))
        for method in (gpu.ACCUM_EMTM, gpu.ACCUM_DIM):
            gpu.dose_accumulate_subvoxel(ctx, 1, (1, 1, 1), method=method)
            acc = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros((1, 1, 1), np.float32))
            assert acc[0, 0, 0] == np.float32(3.75), method
    finally:
        gpu.dose_destroy(ctx)
    assert orc.dim(doses, (2.0, 2.0, 2.0), 1, (1, 1, 1))[0, 0, 0] == 3.75


def test_one_voxel_registration_grid(gpu, orc):
    """A registration grid of one voxel is defined only at its centre: the
    CT voxel whose centre it is gets its translation, every other voxel is
    outside."""
    nx, ny, nz = 5, 4, 3
    hu = np.zeros((1, nz, ny, nx), np.int16)
    ctx = gpu.dose_create_grid(nx, ny, nz, 2.0, 2.0, 2.0, (0.0, 0.0, 0.0), 1, hu, (0.0, 0.0, 1.0))
    g = dict(n=(1, 1, 1), start_mm=(5.0, 3.0, 1.0), spacing_mm=(1.0, 1.0, 1.0), row_cos=(1, 0, 0),
             col_cos=(0, 1, 0))
    delta = np.array([[[[0.25, -0.5, 1.0]]]], np.float32)
    try:
        out = torch.zeros(3 * nx * ny * nz, dtype=torch.float32, device="cuda")
        mask = torch.ones(nx * ny * nz, dtype=torch.uint8, device="cuda")
        gpu.dose_decode_dvf(ctx, g, delta, out, mask=mask)
        got = out.cpu().numpy().reshape(3, nz, ny, nx)
        m = mask.cpu().numpy().reshape(nz, ny, nx)
    finally:
        gpu.dose_destroy(ctx)
    want, inside = orc.dvf_decode(g, delta, (nx, ny, nz), (2.0, 2.0, 2.0), (0.0, 0.0, 0.0))
    np.testing.assert_array_equal(m, inside)          # exact values: the single centre is inside
    assert m.sum() == 1 and m[0, 1, 2] == 1                 # centre (5, 3, 1) is voxel (2, 1, 0)
    np.testing.assert_allclose(got[:, 0, 1, 2], [0.25, -0.5, 1.0], atol=1e-6)
    np.testing.assert_allclose(got, want, atol=1e-6)


def test_one_spot_delivery(gpu, orc):
    """One spot whose spill crosses several phase boundaries."""
    plan = _plan([0.0], [0.0], [100.0], [7_777_777])
    dlv = W.Delivery(n_phases=4, start_phase=1, period_ns=8_000_000, rate_protons_per_s=1_000_000_000)
    ph = W.water_phantom(8, 8, 8)
    hu = np.repeat(ph.hu[None], 4, axis=0)
    ctx = gpu.dose_create_grid(8, 8, 8, 2.0, 2.0, 2.0, ph.origin, 4, hu, (0.0, 0.0, 1.0))
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(plan), gpu.delivery_struct(dlv))
        pp = gpu.dose_read(ctx, gpu.DOSE_SUBPLAN, 0, np.zeros((4, 1), np.uint64))
    finally:
        gpu.dose_destroy(ctx)
    opp, _, _ = orc.timeline(plan, dlv)
    np.testing.assert_array_equal(pp, opp)
    assert np.count_nonzero(pp) == 4 and int(pp.sum()) == 7_777_777


def test_host_wait_gives_up_while_the_kernel_finishes(gpu):
    """Failure detection on the host (no GPU fault): with a 1 ms wait limit,
    reading a 1e8-history run's tally into pinned host memory returns
    DOSE_ETIMEOUT while the transport is still running; the work itself is
    untouched, so after waiting normally the tally is the untimed run's, bit
    for bit, and the context keeps working."""
    D = gpu
    ph = W.slab_phantom(n=64)
    pl = W.slab_plan(n_layers=4, nx=3, ny=2)
    n, seed = 100_000_000, 31
    ref = H.gpu_run(D, ph, pl, n, seed)["tally"]
    ctx = H.make_ctx(D, ph)
    try:
        D.dose_add_spots(ctx, D.spots_array(pl), None)
        D.dose_set_option(ctx, D.DOSE_OPT_TIMEOUT_MS, 1)
        out = torch.zeros(ph.hu.shape, dtype=torch.int64).pin_memory()
        D.dose_run_phase(ctx, 0, n, seed)
        with pytest.raises(D.DoseError) as e:
            D.dose_read(ctx, D.DOSE_TALLY_I64, 0, out)
        assert e.value.code == D.DOSE_ETIMEOUT and "did not finish" in str(e.value)
        torch.cuda.synchronize()                      # the copy the read enqueued lands here
        np.testing.assert_array_equal(out.numpy().view(np.uint64), ref)
        D.dose_set_option(ctx, D.DOSE_OPT_TIMEOUT_MS, 600_000)
        again = D.dose_read(ctx, D.DOSE_TALLY_I64, 0, np.zeros(ph.hu.shape, np.uint64))
        np.testing.assert_array_equal(again, ref)
    finally:
        D.dose_destroy(ctx)
