"""Registration-grid decode (App. B, Eqs. 7-8) on the GPU against the
oracle's or_dvf_decode.

The hull mask is an integer decided by floating point: the oracle decides
it in FP64 and flags the CT voxels whose grid index lies within its tie
tolerance of a hull face, where either decision is correct; every other
voxel must match bit for bit (and where every quantity is exactly
representable, as on the grids of CT voxel centres below, so must those).
The displacement is FP32 on the GPU (grid displacement e = r_f - r0 formed
with the rigid parts folded, then interpolated) and FP64 in the oracle; with
|r0| < 100 mm and |e| < 20 mm the FP32 rounding is below 1e-5 mm, so the
test allows 1e-4 mm + 1e-5 relative where both sides call the voxel inside.
"""
import numpy as np
import pytest
import torch

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

N = (37, 29, 23)                 # CT nx, ny, nz: 24,679 voxels, ragged against 256-thread blocks
D = (1.5, 2.0, 2.5)
ORIGIN = (-27.0, -29.0, -28.0)


def _ctx(gpu, n_phases=1):
    nx, ny, nz = N
    hu = np.zeros((n_phases, nz, ny, nx), np.int16)
    return gpu.dose_create_grid(nx, ny, nz, *D, ORIGIN, n_phases, hu, (0.0, 0.0, 1.0))


def _rot_z(deg):
    t = np.deg2rad(deg)
    return np.array([[np.cos(t), -np.sin(t), 0], [np.sin(t), np.cos(t), 0], [0, 0, 1.0]])


def _rigid(R, t):
    m = np.eye(4)
    m[:3, :3] = R
    m[:3, 3] = t
    return m


def _grids():
    th = np.deg2rad(30.0)
    return {
        "axis_coarse": dict(n=(20, 16, 11), start_mm=(-26.0, -28.0, -26.0), spacing_mm=(3.0, 4.0, 5.0),
                            row_cos=(1, 0, 0), col_cos=(0, 1, 0)),
        "axis_partial": dict(n=(9, 7, 5), start_mm=(-12.0, -14.0, -10.0), spacing_mm=(3.0, 4.0, 5.0),
                             row_cos=(1, 0, 0), col_cos=(0, 1, 0)),
        "turned_90": dict(n=(16, 20, 11), start_mm=(28.0, -28.0, -26.0), spacing_mm=(4.0, 3.0, 5.0),
                          row_cos=(0, 1, 0), col_cos=(-1, 0, 0)),
        "oblique": dict(n=(18, 12, 14), start_mm=(-24.0, -6.0, -26.0), spacing_mm=(3.0, 4.0, 3.5),
                        row_cos=(np.cos(th), np.sin(th), 0.0), col_cos=(0, 0, 1)),
        "rigid": dict(n=(20, 16, 11), start_mm=(-26.0, -28.0, -26.0), spacing_mm=(3.0, 4.0, 5.0),
                      row_cos=(1, 0, 0), col_cos=(0, 1, 0),
                      pre=_rigid(_rot_z(5.0), (1.0, -2.0, 0.5)), post=_rigid(np.eye(3), (-0.25, 0.75, 3.0))),
    }


def _translations(rng, g, amp=6.0):
    """Smooth random translations (mm) on the registration grid."""
    nx, ny, nz = g["n"]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    t = np.zeros((nz, ny, nx, 3))
    for c in range(3):
        for _ in range(3):
            w = rng.uniform(-0.4, 0.4, 3)
            t[..., c] += rng.uniform(-1, 1) * np.sin(w[0] * i + w[1] * j + w[2] * k + rng.uniform(0, 6.3))
    return (amp / 3.0 * t).astype(np.float32)


def _gpu_decode(gpu, ctx, g, delta, on_device=False, mask=None):
    nvox = int(np.prod(N))
    out = torch.full((3 * nvox,), np.nan, dtype=torch.float32, device="cuda")
    src = torch.from_numpy(delta).cuda() if on_device else delta
    gpu.dose_decode_dvf(ctx, g, src, out, mask=mask)
    torch.cuda.synchronize()
    nx, ny, nz = N
    return out.cpu().numpy().reshape(3, nz, ny, nx)


@pytest.mark.parametrize("name", list(_grids()))
def test_decode_parity(gpu, orc, name):
    g = _grids()[name]
    rng = np.random.default_rng(sum(map(ord, name)))
    delta = _translations(rng, g)
    nx, ny, nz = N
    ctx = _ctx(gpu)
    try:
        mask = torch.ones(nx * ny * nz, dtype=torch.uint8, device="cuda")
        got = _gpu_decode(gpu, ctx, g, delta, on_device=(name == "oblique"), mask=mask)
        gmask = mask.cpu().numpy().reshape(nz, ny, nx)
    finally:
        gpu.dose_destroy(ctx)
    want, inside, amb = orc.dvf_decode(g, delta, N, D, ORIGIN, return_ambiguous=True)
    if name == "oblique":
        # cosines of 30 degrees: the hull test is rounded on both sides, and
        # only voxels within the tie tolerance of a hull face may differ
        sure = amb == 0
        np.testing.assert_array_equal(gmask[sure], inside[sure])
        assert amb.sum() <= 0.01 * amb.size, int(amb.sum())
    else:
        # axis-aligned grids with binary-exact start, spacing and CT centres:
        # the hull test is exact on both sides, faces included (these grids
        # have a hull face through a row of CT voxel centres)
        np.testing.assert_array_equal(gmask, inside)
    assert inside.sum() > 500
    assert np.all(got[:, gmask == 0] == 0.0)
    both = (gmask == 1) & (inside == 1)
    tol = 1e-4 + 1e-5 * np.abs(want)
    bad = (np.abs(got - want) > tol) & both[None]
    assert not bad.any(), (int(bad.sum()), float(np.abs(got - want)[:, both].max()))


def test_decode_masks_intersect_over_phases(gpu, orc):
    """Decoding two registrations into one mask leaves the voxels both grids
    cover (the report mask of Sec. 2.D.2)."""
    gs = _grids()
    nx, ny, nz = N
    ctx = _ctx(gpu)
    try:
        mask = torch.ones(nx * ny * nz, dtype=torch.uint8, device="cuda")
        for name in ("axis_partial", "oblique"):
            _gpu_decode(gpu, ctx, gs[name], np.zeros(tuple(gs[name]["n"][::-1]) + (3,), np.float32), mask=mask)
        gmask = mask.cpu().numpy().reshape(nz, ny, nx)
    finally:
        gpu.dose_destroy(ctx)
    _, a, amb_a = orc.dvf_decode(gs["axis_partial"], np.zeros(tuple(gs["axis_partial"]["n"][::-1]) + (3,),
                                                             np.float32), N, D, ORIGIN, return_ambiguous=True)
    _, b, amb_b = orc.dvf_decode(gs["oblique"], np.zeros(tuple(gs["oblique"]["n"][::-1]) + (3,), np.float32),
                                 N, D, ORIGIN, return_ambiguous=True)
    sure = (amb_a == 0) & (amb_b == 0)
    np.testing.assert_array_equal(gmask[sure], (a & b)[sure])
    assert 0 < gmask.sum() < min(a.sum(), b.sum())


def test_decode_rejects_bad_input(gpu):
    g = dict(_grids()["axis_coarse"])
    ctx = _ctx(gpu)
    nvox = int(np.prod(N))
    out = torch.zeros(3 * nvox, dtype=torch.float32, device="cuda")
    delta = np.zeros(tuple(g["n"][::-1]) + (3,), np.float32)
    try:
        with pytest.raises(gpu.DoseError):
            gpu.dose_decode_dvf(ctx, dict(g, col_cos=(0.5, 0.5, 0.0)), delta, out)
        with pytest.raises(gpu.DoseError):
            gpu.dose_decode_dvf(ctx, dict(g, spacing_mm=(3.0, 0.0, 5.0)), delta, out)
        with pytest.raises(ValueError):
            gpu.dose_decode_dvf(ctx, g, delta, np.zeros(3 * nvox, np.float32))
    finally:
        gpu.dose_destroy(ctx)


def test_decoded_field_drives_the_accumulation(gpu, orc):
    """The 4DCT's own phase->reference field, stored as a registration grid
    on the CT voxel centres, decodes back to itself; the decoded fields of
    all phases then drive the EMTM on the device, which matches the
    oracle's EMTM given the same decoded field."""
    ph, dvf, geo = H.small_4dct(n_phases=3, nx=40, ny=36, nz=24)
    P = ph.n_phases
    nx, ny, nz = ph.n
    nvox = nx * ny * nz
    rng = np.random.default_rng(5)
    doses = rng.gamma(2.0, 0.5, size=(P, nz, ny, nx)).astype(np.float32)
    start = tuple(ph.origin[k] + 0.5 * ph.d[k] for k in range(3))
    ctx = H.make_ctx(gpu, ph)
    try:
        field = torch.zeros(P * 3 * nvox, dtype=torch.float32, device="cuda")
        mask = torch.ones(nvox, dtype=torch.uint8, device="cuda")
        for p in range(P):
            g = dict(n=(nx, ny, nz), start_mm=start, spacing_mm=ph.d, row_cos=(1, 0, 0), col_cos=(0, 1, 0))
            delta = np.ascontiguousarray(np.moveaxis(dvf[p], 0, -1))
            gpu.dose_decode_dvf(ctx, g, delta, field[p * 3 * nvox:(p + 1) * 3 * nvox], mask=mask)
        for p in range(P):
            gpu.dose_set_phase_dose(ctx, p, np.ascontiguousarray(doses[p]))
        gpu.dose_accumulate_subvoxel(ctx, 0, (2, 2, 5), dvf=field, mask=mask)
        acc = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros((nz, ny, nx), np.float32))
        dec = field.cpu().numpy().reshape(P, 3, nz, ny, nx)
        gmask = mask.cpu().numpy().reshape(nz, ny, nx)
    finally:
        gpu.dose_destroy(ctx)
    assert gmask.all()
    np.testing.assert_allclose(dec, dvf, rtol=0, atol=2e-5)
    rho = np.stack([orc.density(ph, p) for p in range(P)]).astype(np.float32)
    _, inside = orc.dvf_decode(g, np.ascontiguousarray(np.moveaxis(dvf[P - 1], 0, -1)), ph.n, ph.d, ph.origin)
    assert inside.all()                  # grid on the CT voxel centres: exact, hull faces included
    want, _, B = orc.emtm(doses, rho, ph.d, 0, (2, 2, 5), dvf=dec, mask=gmask, bounds=True)
    H.check_emtm(acc, want, B)
