"""The allocation-free entry point, dose_run_phase_noalloc, against the
regular one.

It is meant for callers that cannot call cudaMalloc, such as code running
inside a framework or service whose allocator owns the device memory.  Its
scratch lives in one static device array shared by every call, so two
calls in a row must each give the regular entry point's dose: the second
call must clear what the first left behind.  This file is collected last
so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_twice(gpu):
    import torch
    D = gpu
    ph = W.slab_phantom(n=64)
    pl = W.slab_plan(n_layers=4, nx=3, ny=2)
    n, seed = 200_000, 5
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
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref["dose"], rtol=1e-6, atol=0.0)
        np.testing.assert_array_equal(led, ref["ledger"])
    # after the first call's set-up, a call takes no device memory
    assert free[1] == free[0]


def test_noalloc_rejects_inputs_beyond_its_limits(gpu):
    import torch
    D = gpu
    pl = W.pencil_plan(100.0, 4.0)
    hu = torch.zeros(8, dtype=torch.int16, device="cuda")
    out = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(D.DoseError) as e:
        D.dose_run_phase_noalloc(hu, 256, 128, 128, 2.0, 2.0, 2.0, (0, 0, 0), (0, 0, 1),
                                 D.spots_array(pl), 1000, 1, out)
    assert e.value.code == D.DOSE_EINVAL and "MAX_VOXELS" in str(e.value)
