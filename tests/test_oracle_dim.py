"""Pins of the oracle's dose-interpolation accumulation (Sec. 2.D.2, Eqs. 2
and 3) against closed forms: trilinear interpolation reproduces linear
fields exactly and misses a quadratic by phi (1 - phi) in each cell, the
subvoxel centres of a voxel sit symmetrically about its centre, and a
uniform field of whole voxels pulls the source dose from the shifted voxel
(reference-to-source direction)."""
import numpy as np
import pytest

D3 = (2.0, 1.5, 3.0)            # dx, dy, dz in mm


def _centres(n):
    """Offsets of the n subvoxel centres from the voxel centre (voxels)."""
    return (np.arange(n) + 0.5) / n - 0.5


def _interp_sq(t):
    """Linear interpolation of x^2 between the integers around t, the
    closed form t^2 + phi (1 - phi), phi = t - floor(t)."""
    phi = t - np.floor(t)
    return t * t + phi * (1.0 - phi)


def test_dim_identity_n1_is_the_static_sum(orc):
    rng = np.random.default_rng(1)
    shape = (4, 5, 6)
    dose = rng.uniform(0.0, 2.0, (3,) + shape).astype(np.float32)
    want = dose.astype(np.float64).sum(axis=0)
    for dvf in (None, np.zeros((3, 3) + shape, np.float32)):
        acc = orc.dim(dose, D3, 1, (1, 1, 1), dvf=dvf)
        np.testing.assert_allclose(acc, want, rtol=1e-12, atol=0)


def test_dim_linear_dose_is_reproduced(orc):
    """A dose linear in position is interpolated exactly, and the mean over
    subvoxel centres placed symmetrically in a voxel is its centre value
    (interior voxels: no edge clamping)."""
    nz, ny, nx = 7, 6, 8
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lin = (0.5 + 0.03 * x - 0.02 * y + 0.07 * z).astype(np.float32)
    dose = np.stack([np.zeros_like(lin), lin])
    acc = orc.dim(dose, D3, 0, (2, 3, 5))
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(acc[inner], lin.astype(np.float64)[inner], rtol=0, atol=1e-6)


@pytest.mark.parametrize("nsub", [(1, 1, 1), (2, 2, 2), (3, 4, 5), (2, 2, 5)])
def test_dim_quadratic_dose_closed_form(orc, nsub):
    """D = x^2 + y^2 + z^2 (voxel indices).  At subvoxel offset delta from
    the centre of voxel i the interpolant is (i + delta)^2 + |delta| -
    delta^2, so D_i^S = |i|^2 + sum over axes of mean |delta| (interior)."""
    nz, ny, nx = 7, 7, 7
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    quad = (x * x + y * y + z * z).astype(np.float32)
    dose = np.stack([np.zeros_like(quad), quad])
    acc = orc.dim(dose, (1.0, 1.0, 1.0), 0, nsub)
    extra = sum(np.abs(_centres(n)).mean() for n in nsub)
    want = quad.astype(np.float64) + extra
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(acc[inner], want[inner], rtol=0, atol=1e-9)
    # the same correction from the counted sums: n even -> 1/4, n odd -> (n^2 - 1) / (4 n^2)
    assert extra == pytest.approx(sum(0.25 if n % 2 == 0 else (n * n - 1) / (4.0 * n * n) for n in nsub))


def test_dim_integer_translation_pulls_from_the_shifted_voxel(orc):
    """u = (+1 voxel in x, -1 voxel in z): reference voxel (z, y, x) takes
    the source dose at (z - 1, y, x + 1), clamped at the grid edge."""
    rng = np.random.default_rng(3)
    shape = (4, 5, 6)
    nz, ny, nx = shape
    dose = rng.uniform(0.0, 2.0, (2,) + shape).astype(np.float32)
    dvf = np.zeros((2, 3) + shape, np.float32)
    dvf[1, 0] = D3[0]
    dvf[1, 2] = -D3[2]
    acc = orc.dim(dose, D3, 0, (1, 1, 1), dvf=dvf)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    src = dose[1][np.clip(z - 1, 0, nz - 1), y, np.clip(x + 1, 0, nx - 1)]
    np.testing.assert_allclose(acc, dose[0].astype(np.float64) + src, rtol=1e-12, atol=0)


def test_dim_linear_field_on_a_quadratic_dose(orc):
    """u_x = beta (x - c) dx mm is linear, so it is interpolated exactly at
    every subvoxel centre q, which lands at t = q + beta (q - c); the dose
    x^2 is then read through the interpolation closed form at t.  A sampler
    that read the field at the voxel centre, or forgot the mm -> voxel
    conversion, moves t and fails."""
    nz, ny, nx = 3, 3, 16
    beta, c = 0.15, 7.3
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dose = np.stack([np.zeros((nz, ny, nx), np.float32), (x * x).astype(np.float32)])
    dvf = np.zeros((2, 3, nz, ny, nx), np.float32)
    dvf[1, 0] = (beta * (x - c) * D3[0]).astype(np.float32)
    nsub = (4, 1, 1)
    acc = orc.dim(dose, D3, 0, nsub, dvf=dvf)
    checked = 0
    for i in range(1, nx - 1):
        q = i + _centres(nsub[0])
        t = q + beta * (q - c)
        if t.min() < 0.0 or t.max() > nx - 1:
            continue                          # the edge clamp would apply
        want = _interp_sq(t).mean()
        assert acc[1, 1, i] == pytest.approx(want, rel=1e-6, abs=1e-5)
        checked += 1
    assert checked >= 10


def test_dim_matches_emtm_for_inverse_whole_voxel_shifts(orc):
    """Pull (DIM, reference-to-source +1 voxel in y) and push (EMTM,
    source-to-reference -1 voxel in y) give the same voxel shift at n = 1
    away from the edge the push drops and the pull clamps."""
    rng = np.random.default_rng(5)
    shape = (3, 6, 4)
    dose = rng.uniform(0.0, 2.0, (2,) + shape).astype(np.float32)
    rho = rng.uniform(0.5, 1.5, (2,) + shape).astype(np.float32)
    pull = np.zeros((2, 3) + shape, np.float32)
    pull[1, 1] = D3[1]
    acc_dim = orc.dim(dose, D3, 0, (1, 1, 1), dvf=pull)
    acc_emtm, _ = orc.emtm(dose, rho, D3, 0, (1, 1, 1), dvf=-pull)
    np.testing.assert_allclose(acc_dim[:, :-1, :], acc_emtm[:, :-1, :], rtol=1e-12)


def test_dim_reference_phase_and_mask(orc):
    rng = np.random.default_rng(6)
    shape = (3, 4, 5)
    dose = rng.uniform(0.0, 2.0, (3,) + shape).astype(np.float32)
    mask = (rng.uniform(size=shape) > 0.3).astype(np.uint8)
    acc = orc.dim(dose, D3, 2, (1, 1, 1), mask=mask)
    want = np.where(mask > 0, dose.astype(np.float64).sum(axis=0), 0.0)
    np.testing.assert_allclose(acc, want, rtol=1e-12)
    with pytest.raises(ValueError):
        orc.dim(dose, D3, 3, (1, 1, 1))
    with pytest.raises(ValueError):
        orc.dim(dose, D3, 0, (0, 1, 1))


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_dim_half_voxel_shift_and_edge_clamp(orc, sign):
    """u = +-1/2 voxel in x at n = 1: each reference voxel takes the mean of
    the two source voxels around the carried point; past the outermost
    voxel centre the dose is that voxel's (edge clamp)."""
    rng = np.random.default_rng(7)
    shape = (2, 3, 6)
    dose = rng.uniform(0.0, 2.0, (2,) + shape).astype(np.float32)
    dvf = np.zeros((2, 3) + shape, np.float32)
    dvf[1, 0] = sign * 0.5 * D3[0]
    acc = orc.dim(dose, D3, 0, (1, 1, 1), dvf=dvf) - dose[0]
    d1 = dose[1].astype(np.float64)
    if sign > 0:
        want = np.concatenate([0.5 * (d1[:, :, :-1] + d1[:, :, 1:]), d1[:, :, -1:]], axis=2)
    else:
        want = np.concatenate([d1[:, :, :1], 0.5 * (d1[:, :, :-1] + d1[:, :, 1:])], axis=2)
    np.testing.assert_allclose(acc, want, rtol=1e-6, atol=1e-7)
