"""Dose-interpolation accumulation (Sec. 2.D.2, Eqs. 2-3) on the GPU against
the oracle's or_dim.

Tolerance.  The kernel interpolates in FP32 where the oracle uses FP64.  A
carried point t (index units, |t| < 256 here) is off by at most a few ulp,
about 3e-5 voxel, which moves an interpolated dose by at most its change
over one voxel times that (<= 3e-5 max D); the FP32 lerps and the FP32 sum
of at most 125 subvoxels add a few 1e-7 relative.  Over up to 9 source
phases the bound is 9 x 3e-5 max D plus 1e-5 relative, so the tests use
|gpu - oracle| <= 3e-4 max|D| + 1e-5 |D|.
"""
import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

D3 = (2.0, 1.5, 2.5)


def _close(acc, want):
    tol = 3e-4 * np.abs(want).max() + 1e-5 * np.abs(want)
    bad = np.abs(acc.astype(np.float64) - want) > tol
    assert not bad.any(), (int(bad.sum()), float(np.abs(acc - want).max()), float(np.abs(want).max()))


def _water_ctx(gpu, shape, n_phases, d=D3):
    nz, ny, nx = shape
    hu = np.zeros((n_phases, nz, ny, nx), np.int16)
    return gpu.dose_create_grid(nx, ny, nz, *d, (0.0, 0.0, 0.0), n_phases, hu, (0.0, 0.0, 1.0))


def _smooth_field(rng, n_phases, shape, d, amp_vox):
    """A smooth displacement field (mm): a few random plane waves per
    component, up to amp_vox voxels."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.zeros((n_phases, 3) + shape, np.float64)
    for p in range(1, n_phases):
        for c in range(3):
            for _ in range(3):
                k = rng.uniform(-0.3, 0.3, 3)
                f[p, c] += rng.uniform(-1, 1) * np.sin(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, 6.3))
            f[p, c] *= amp_vox / 3.0 * d[c]
    return f.astype(np.float32)


def _gpu_dim(gpu, doses, ref, nsub, dvf=None, mask=None, d=D3):
    P = doses.shape[0]
    ctx = _water_ctx(gpu, doses.shape[1:], P, d)
    try:
        for p in range(P):
            gpu.dose_set_phase_dose(ctx, p, np.ascontiguousarray(doses[p]))
        gpu.dose_accumulate_subvoxel(ctx, ref, nsub, dvf=dvf, mask=mask, method=1)
        acc = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros(doses.shape[1:], np.float32))
        with pytest.raises(gpu.DoseError):
            gpu.dose_read(ctx, gpu.DOSE_EMTM_STATS, 0, np.zeros(4, np.uint64))
    finally:
        gpu.dose_destroy(ctx)
    return acc


SHAPE = (23, 29, 37)        # 24,679 voxels: 97 blocks of 256, the last one ragged


@pytest.mark.parametrize("case,nsub", [
    ("identity", (2, 2, 5)), ("dvf", (1, 1, 1)), ("dvf", (2, 2, 5)), ("dvf", (3, 3, 3)),
    ("dvf_mask", (2, 2, 2)), ("ref2", (2, 3, 4)), ("large", (2, 2, 5))])
def test_dim_parity(gpu, orc, case, nsub):
    rng = np.random.default_rng(sum(map(ord, case)) + 10 * sum(nsub))
    P = 4
    doses = rng.gamma(2.0, 0.5, size=(P,) + SHAPE).astype(np.float32)
    amp = 6.0 if case == "large" else 1.5        # "large" carries points past the grid edges
    dvf = None if case == "identity" else _smooth_field(rng, P, SHAPE, D3, amp)
    mask = (rng.random(SHAPE) > 0.3).astype(np.uint8) if case == "dvf_mask" else None
    ref = 2 if case == "ref2" else 0
    acc = _gpu_dim(gpu, doses, ref, nsub, dvf=dvf, mask=mask)
    want = orc.dim(doses, D3, ref, nsub, dvf=dvf, mask=mask)
    _close(acc, want)
    if mask is not None:
        assert np.all(acc[mask == 0] == 0.0)


@pytest.mark.parametrize("case", ["blob", "corner", "empty_phase", "far_field"])
def test_dim_sparse_dose_reach(gpu, orc, case):
    """Doses with compact support: reference voxels out of a phase's reach
    skip it, and the pull still matches the oracle's DIM of every voxel."""
    rng = np.random.default_rng(sum(map(ord, case)))
    P = 4
    doses = rng.gamma(2.0, 0.5, size=(P,) + SHAPE).astype(np.float32)
    keep = np.zeros(doses.shape, bool)
    if case == "corner":
        keep[:, -3:, :4, -2:] = True
    elif case == "empty_phase":
        keep[:, 5:12, 8:16, 10:20] = True
        keep[3] = False
    else:
        keep[:, 5:12, 8:16, 10:20] = True
    doses = np.where(keep, doses, np.float32(0.0)).astype(np.float32)
    dvf = _smooth_field(rng, P, SHAPE, D3, 30.0 if case == "far_field" else 1.5)
    acc = _gpu_dim(gpu, doses, 0, (2, 2, 5), dvf=dvf)
    want = orc.dim(doses, D3, 0, (2, 2, 5), dvf=dvf)
    _close(acc, want)
    assert acc.max() > 0
    # the phase sum reaches beyond the reference phase's own dose
    assert np.count_nonzero(acc) > np.count_nonzero(doses[0])


def test_dim_identity_n1_is_the_exact_phase_sum(gpu):
    """At n = 1 with no field every subvoxel centre is a voxel centre, so
    the interpolation returns the voxel value exactly and the accumulated
    dose is the FP64 phase sum (reference first) rounded once."""
    rng = np.random.default_rng(2)
    doses = rng.gamma(2.0, 0.5, size=(5,) + SHAPE).astype(np.float32)
    acc = _gpu_dim(gpu, doses, 0, (1, 1, 1))
    want = doses[0].astype(np.float64)
    for p in range(1, 5):
        want = want + doses[p].astype(np.float64)
    np.testing.assert_array_equal(acc, want.astype(np.float32))


def test_dim_integer_shift_is_exact(gpu):
    """A field of whole voxels at n = 1 reads source voxels exactly: the
    reference voxel (z, y, x) takes the source value at (z - 1, y, x + 2),
    clamped at the grid edge."""
    rng = np.random.default_rng(3)
    doses = rng.gamma(2.0, 0.5, size=(2,) + SHAPE).astype(np.float32)
    dvf = np.zeros((2, 3) + SHAPE, np.float32)
    dvf[1, 0] = 2 * D3[0]
    dvf[1, 2] = -D3[2]
    acc = _gpu_dim(gpu, doses, 0, (1, 1, 1), dvf=dvf)
    nz, ny, nx = SHAPE
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    want = doses[0].astype(np.float64) + doses[1][np.clip(z - 1, 0, nz - 1), y, np.clip(x + 2, 0, nx - 1)]
    np.testing.assert_array_equal(acc, want.astype(np.float32))


def test_dim_on_transported_4d_doses(gpu, orc):
    """The pull after a whole 4D Monte Carlo: the phase doses the engine
    computed, accumulated with the reference-to-phase field of the same
    breathing model, against the oracle's DIM of those doses."""
    ph, dvf, geo = H.small_4dct(n_phases=4)
    plan = W.tumour_plan(geo, ph.origin, n_layers=3, per_layer=12, e_lo=70.0, e_hi=100.0)
    dlv = W.Delivery(n_phases=4, start_phase=-1, seed=21, period_ns=20_000_000,
                     spot_switch_ns=200_000, layer_switch_ns=3_000_000)
    pull = W.reference_to_phase_field(dvf)
    ctx = H.make_ctx(gpu, ph)
    shape = ph.hu.shape[1:]
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(plan), gpu.delivery_struct(dlv))
        gpu.dose_run_4d(ctx, 20_000, 5, 0, (2, 2, 5), dvf=dvf)
        doses = np.stack([gpu.dose_read(ctx, gpu.DOSE_PHASE_DOSE, p, np.zeros(shape, np.float32))
                          for p in range(ph.n_phases)])
        gpu.dose_accumulate_subvoxel(ctx, 0, (2, 2, 5), dvf=pull, method=1)
        acc = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros(shape, np.float32))
    finally:
        gpu.dose_destroy(ctx)
    assert doses.max() > 0
    _close(acc, orc.dim(doses, ph.d, 0, (2, 2, 5), dvf=pull))


def test_dim_full_size_sampled(gpu, orc):
    """The 10-phase 256 x 256 x 160 4DCT at 1 x 1 x 2.5 mm with (2, 2, 5)
    subvoxels.  The pull is local, so each sampled voxel is recomputed by
    the oracle on a crop around it wider than the largest displacement (the
    crop clamps only where the full grid does)."""
    ph, dvf, geo = W.phantom_4dct()
    pull = W.reference_to_phase_field(dvf)
    P = ph.n_phases
    shape = ph.hu.shape[1:]
    rng = np.random.default_rng(11)
    doses = rng.gamma(2.0, 0.5, size=(P,) + shape).astype(np.float32)
    nsub = (2, 2, 5)
    acc = _gpu_dim(gpu, doses, 0, nsub, dvf=pull, d=ph.d)
    reach = [int(np.ceil(np.abs(pull[:, c]).max() / ph.d[c])) + 2 for c in range(3)]
    nz, ny, nx = shape
    picks = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, 0, nx - 1)]
    picks += [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(100)]
    moving = np.argwhere(np.abs(pull[1:, 2]).max(axis=0) > 1.0)       # inside the breathing region
    picks += [tuple(int(v) for v in moving[k]) for k in rng.choice(len(moving), 100, replace=False)]
    mz, my, mx = reach[2], reach[1], reach[0]
    for (z, y, x) in picks:
        sz = slice(max(0, z - mz), min(nz, z + mz + 1))
        sy = slice(max(0, y - my), min(ny, y + my + 1))
        sx = slice(max(0, x - mx), min(nx, x + mx + 1))
        want = orc.dim(doses[:, sz, sy, sx], ph.d, 0, nsub, dvf=pull[:, :, sz, sy, sx])
        w = want[z - sz.start, y - sy.start, x - sx.start]
        got = float(acc[z, y, x])
        assert abs(got - w) <= 3e-4 * np.abs(want).max() + 1e-5 * abs(w), ((z, y, x), got, w)
