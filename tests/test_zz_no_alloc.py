"""The allocation-free entry point, dose_run_phase_noalloc, against the
regular one.

It is meant for callers that cannot call cudaMalloc, such as code running
inside a framework or service whose allocator owns the device memory.  Its
scratch lives in one static device array shared by every call, so two
calls in a row must each give the regular entry point's dose, bit for bit:
the second call must clear what the first left behind.  This file is
collected last so that a run stopping at the first failure has run every
other test.
"""
import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _case():
    ph = W.slab_phantom(n=64)
    pl = W.slab_plan(n_layers=4, nx=3, ny=2)
    return ph, pl, 200_000, 5


def test_noalloc_matches_regular_entry_point_twice(gpu):
    import torch
    D = gpu
    ph, pl, n, seed = _case()
    ref = H.gpu_run(D, ph, pl, n, seed)
    hu = torch.from_numpy(np.ascontiguousarray(ph.hu)).cuda()
    out = torch.empty(ph.hu.shape, dtype=torch.float32, device="cuda")
    spots = D.spots_array(pl)
    free = []
    for _ in range(2):
        out.fill_(-1.0)
        torch.cuda.synchronize()
        led = D.dose_run_phase_noalloc(hu, *ph.n, *ph.d, ph.origin, ph.beam_dir, spots, n, seed, out)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        np.testing.assert_array_equal(out.cpu().numpy(), ref["dose"])
        np.testing.assert_array_equal(led, ref["ledger"])
    # after the first call's set-up, a call takes no device memory
    assert free[1] == free[0]


def test_noalloc_on_a_side_stream_without_ledger(gpu):
    """Two calls in a row on a non-default stream with no ledger buffer: the
    call returns once the dose is written, and each dose is the regular
    entry point's, bit for bit."""
    import torch
    D = gpu
    ph, pl, n, seed = _case()
    ref = H.gpu_run(D, ph, pl, n, seed + 1)
    s = torch.cuda.Stream()
    hu = torch.from_numpy(np.ascontiguousarray(ph.hu)).cuda()
    outs = [torch.full(ph.hu.shape, -1.0, dtype=torch.float32, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for out in outs:
            assert D.dose_run_phase_noalloc(hu, *ph.n, *ph.d, ph.origin, ph.beam_dir, D.spots_array(pl), n,
                                            seed + 1, out, stream=s, ledger=False) is None
    s.synchronize()
    for out in outs:
        np.testing.assert_array_equal(out.cpu().numpy(), ref["dose"])


def test_noalloc_rejects_inputs_beyond_its_limits(gpu):
    import torch
    D = gpu
    pl = W.pencil_plan(100.0, 4.0)
    hu = torch.zeros(8, dtype=torch.int16, device="cuda")
    out = torch.zeros(8, dtype=torch.float32, device="cuda")
    big = 256 * 128 * 128
    with pytest.raises(D.DoseError) as e:
        D.dose_run_phase_noalloc(torch.zeros(big, dtype=torch.int16, device="cuda"), 256, 128, 128, 2.0, 2.0,
                                 2.0, (0, 0, 0), (0, 0, 1), D.spots_array(pl), 1000, 1,
                                 torch.zeros(big, dtype=torch.float32, device="cuda"))
    assert e.value.code == D.DOSE_EINVAL and "MAX_VOXELS" in str(e.value)
    with pytest.raises(D.DoseError) as e:
        D.dose_run_phase_noalloc(hu, 2, 2, 2, 2.0, 2.0, 2.0, (0, float("nan"), 0), (0, 0, 1),
                                 D.spots_array(pl), 1000, 1, out)
    assert e.value.code == D.DOSE_EINVAL and "origin" in str(e.value)
    two = W.Plan(*(np.concatenate([a, a]) for a in (pl.x, pl.y, pl.energy, pl.sigma, pl.protons, pl.layer)),
                 np.array([0, 1], np.int32))
    with pytest.raises(D.DoseError) as e:
        D.dose_run_phase_noalloc(hu, 2, 2, 2, 2.0, 2.0, 2.0, (0, 0, 0), (0, 0, 1), D.spots_array(two), 1000, 1, out)
    assert e.value.code == D.DOSE_EINVAL and "field 0" in str(e.value)


def test_noalloc_binding_checks_types_sizes_and_device(gpu):
    """The C call cannot check raw pointers; the binding refuses tensors of
    the wrong type, too few elements or host memory before calling it."""
    import torch
    D = gpu
    pl = D.spots_array(W.pencil_plan(100.0, 4.0))
    hu = torch.zeros(8, dtype=torch.int16, device="cuda")
    out = torch.zeros(8, dtype=torch.float32, device="cuda")
    args = (2, 2, 2, 2.0, 2.0, 2.0, (0, 0, 0), (0, 0, 1), pl, 1000, 1)
    with pytest.raises(ValueError, match="int16"):
        D.dose_run_phase_noalloc(hu.float(), *args, out)
    with pytest.raises(ValueError, match="float32"):
        D.dose_run_phase_noalloc(hu, *args, out.double())
    with pytest.raises(ValueError, match="elements"):
        D.dose_run_phase_noalloc(hu[:7], *args, out)
    with pytest.raises(ValueError, match="elements"):
        D.dose_run_phase_noalloc(hu, *args, out[:4])
    with pytest.raises(ValueError, match="CUDA"):
        D.dose_run_phase_noalloc(hu.cpu(), *args, out)
