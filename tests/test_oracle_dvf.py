"""Pins of the oracle's registration-grid decode (App. B, Eqs. 7-8; positions
between grid voxels interpolate trilinearly) against closed forms: a
trilinear interpolant reproduces affine fields exactly, so uniform and
affine translations, rotated grid axes, the depth axis W = U x V and rigid
pre/post transforms all have displacements written by hand."""
import numpy as np
import pytest

N = (20, 16, 12)                      # CT nx, ny, nz
D = (1.5, 2.0, 2.5)
ORIGIN = (-15.0, -16.0, -15.0)        # CT grid corner, patient frame


def _ct_centres():
    nx, ny, nz = N
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (ORIGIN[0] + (x + 0.5) * D[0], ORIGIN[1] + (y + 0.5) * D[1], ORIGIN[2] + (z + 0.5) * D[2])


def _grid(n, start, spacing, U=(1, 0, 0), V=(0, 1, 0), **kw):
    g = {"n": n, "start_mm": start, "spacing_mm": spacing, "row_cos": U, "col_cos": V}
    g.update(kw)
    return g


def _grid_positions(g):
    """r0 of every grid voxel (Eq. 8), shape (N_Z, N_Y, N_X, 3)."""
    U, V = np.array(g["row_cos"], float), np.array(g["col_cos"], float)
    W = np.cross(U, V)
    nx, ny, nz = g["n"]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sp = g["spacing_mm"]
    return (np.array(g["start_mm"], float) + i[..., None] * sp[0] * U + j[..., None] * sp[1] * V
            + k[..., None] * sp[2] * W)


AXIS = _grid((8, 7, 5), (-12.0, -14.0, -10.0), (3.0, 4.0, 5.0))


def _axis_box():
    X, Y, Z = _ct_centres()
    lo = np.array(AXIS["start_mm"])
    hi = lo + (np.array(AXIS["n"]) - 1) * np.array(AXIS["spacing_mm"])
    return ((X >= lo[0]) & (X <= hi[0]) & (Y >= lo[1]) & (Y <= hi[1]) & (Z >= lo[2]) & (Z <= hi[2]))


def test_uniform_translation_and_hull_mask(orc):
    c = np.array([1.25, -0.5, 2.0], np.float32)
    delta = np.broadcast_to(c, (5, 7, 8, 3)).copy()
    disp, inside = orc.dvf_decode(AXIS, delta, N, D, ORIGIN)
    box = _axis_box()
    assert box.sum() > 100 and (~box).sum() > 100
    np.testing.assert_array_equal(inside.astype(bool), box)
    for k in range(3):
        np.testing.assert_allclose(disp[k][box], c[k], rtol=0, atol=1e-12)
        assert np.all(disp[k][~box] == 0.0)


def test_affine_translation_is_reproduced(orc):
    """Delta(r0) = A r0 + b gives r_f = r0 + A r0 + b, affine in the grid
    index, so the trilinear interpolant is exact: u(p) = A p + b."""
    rng = np.random.default_rng(1)
    A = rng.uniform(-0.05, 0.05, (3, 3))
    b = rng.uniform(-2, 2, 3)
    r0 = _grid_positions(AXIS)
    delta = (r0 @ A.T + b).astype(np.float32)
    disp, inside = orc.dvf_decode(AXIS, delta, N, D, ORIGIN)
    X, Y, Z = _ct_centres()
    P = np.stack([X, Y, Z], axis=-1)
    want = P @ A.T + b
    box = inside.astype(bool)
    for k in range(3):
        np.testing.assert_allclose(disp[k][box], want[..., k][box], rtol=0, atol=2e-5)


def test_rotated_grid_axes(orc):
    """U = +y, V = -x (W = +z): grid index i runs along +y and j along -x,
    so i = (p_y - s_y)/dX, j = (s_x - p_x)/dY, k = (p_z - s_z)/dZ; with
    Delta = 0.1 (i, 2 j, 3 k) mm the displacement follows by hand."""
    g = _grid((7, 9, 5), (10.0, -13.0, -9.0), (4.0, 3.0, 5.0), U=(0, 1, 0), V=(-1, 0, 0))
    nz_, ny_, nx_ = 5, 9, 7
    k, j, i = np.meshgrid(np.arange(nz_), np.arange(ny_), np.arange(nx_), indexing="ij")
    delta = (0.1 * np.stack([i, 2 * j, 3 * k], axis=-1)).astype(np.float32)
    disp, inside = orc.dvf_decode(g, delta, N, D, ORIGIN)
    X, Y, Z = _ct_centres()
    gi, gj, gk = (Y + 13.0) / 4.0, (10.0 - X) / 3.0, (Z + 9.0) / 5.0
    box = (gi >= 0) & (gi <= 6) & (gj >= 0) & (gj <= 8) & (gk >= 0) & (gk <= 4)
    assert box.sum() > 100
    np.testing.assert_array_equal(inside.astype(bool), box)
    want = 0.1 * np.stack([gi, 2 * gj, 3 * gk])
    for c in range(3):
        np.testing.assert_allclose(disp[c][box], want[c][box], rtol=0, atol=1e-5)


def test_depth_axis_is_row_cross_column(orc):
    """U = +x, V = +z gives W = U x V = -y: grid index k grows toward -y."""
    g = _grid((6, 5, 4), (-10.0, 8.0, -8.0), (3.0, 4.0, 5.0), U=(1, 0, 0), V=(0, 0, 1))
    k = np.arange(4)[:, None, None, None] * np.ones((4, 5, 6, 1))
    delta = np.concatenate([np.zeros((4, 5, 6, 2)), 0.3 * k], axis=-1).astype(np.float32)
    disp, inside = orc.dvf_decode(g, delta, N, D, ORIGIN)
    X, Y, Z = _ct_centres()
    gk = (8.0 - Y) / 5.0
    gi, gj = (X + 10.0) / 3.0, (Z + 8.0) / 4.0
    box = (gi >= 0) & (gi <= 5) & (gj >= 0) & (gj <= 4) & (gk >= 0) & (gk <= 3)
    assert box.sum() > 50
    np.testing.assert_array_equal(inside.astype(bool), box)
    np.testing.assert_allclose(disp[2][box], 0.3 * gk[box], rtol=0, atol=1e-5)
    np.testing.assert_allclose(disp[0][box], 0.0, atol=1e-5)


def test_rigid_pre_and_post_transforms(orc):
    """M_pre = 90 degrees about z plus t1, M_post = translation t2, Delta =
    c: r_f = R r0 + t1 + c + t2, so u(p) = R p + t1 + c + t2 - p."""
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    t1, t2, c = np.array([1.0, -2.0, 0.5]), np.array([-0.25, 0.75, 3.0]), np.array([0.5, 0.25, -1.0])
    pre = np.eye(4); pre[:3, :3] = R; pre[:3, 3] = t1
    post = np.eye(4); post[:3, 3] = t2
    g = dict(AXIS, pre=pre, post=post)
    delta = np.broadcast_to(c.astype(np.float32), (5, 7, 8, 3)).copy()
    disp, inside = orc.dvf_decode(g, delta, N, D, ORIGIN)
    X, Y, Z = _ct_centres()
    P = np.stack([X, Y, Z], axis=-1)
    want = P @ R.T + t1 + c + t2 - P
    box = _axis_box()
    np.testing.assert_array_equal(inside.astype(bool), box)
    for k in range(3):
        np.testing.assert_allclose(disp[k][box], want[..., k][box], rtol=0, atol=1e-9)


def test_rejects_bad_grid(orc):
    delta = np.zeros((5, 7, 8, 3), np.float32)
    with pytest.raises(ValueError):
        orc.dvf_decode(dict(AXIS, spacing_mm=(0.0, 4.0, 5.0)), delta, N, D, ORIGIN)


def test_oblique_grid_affine(orc):
    """A grid turned 30 degrees about z with its columns along z (U =
    (cos, sin, 0), V = +z, so W = U x V = (sin, -cos, 0) has no zero
    component but z): an affine translation is still reproduced exactly,
    and the mask is the grid's hull of voxel centres."""
    th = np.deg2rad(30.0)
    U, V = (np.cos(th), np.sin(th), 0.0), (0.0, 0.0, 1.0)
    g = _grid((9, 6, 7), (-14.0, -4.0, -12.0), (3.0, 4.0, 3.5), U=U, V=V)
    rng = np.random.default_rng(2)
    A = rng.uniform(-0.05, 0.05, (3, 3))
    b = rng.uniform(-2, 2, 3)
    r0 = _grid_positions(g)
    disp, inside = orc.dvf_decode(g, (r0 @ A.T + b).astype(np.float32), N, D, ORIGIN)
    X, Y, Z = _ct_centres()
    P = np.stack([X, Y, Z], axis=-1)
    W = np.cross(U, V)
    assert np.all(np.abs(W[:2]) > 0.4)
    rel = P - np.array(g["start_mm"])
    q = [rel @ np.array(ax) / sp for ax, sp in zip((U, V, W), g["spacing_mm"])]
    hi = np.array(g["n"]) - 1
    eps = 1e-4
    surely_in = np.all([(q[a] >= eps) & (q[a] <= hi[a] - eps) for a in range(3)], axis=0)
    surely_out = np.any([(q[a] < -eps) | (q[a] > hi[a] + eps) for a in range(3)], axis=0)
    assert surely_in.sum() > 100 and surely_out.sum() > 100
    assert np.all(inside[surely_in] == 1) and np.all(inside[surely_out] == 0)
    want = P @ A.T + b
    box = inside.astype(bool)
    for k in range(3):
        np.testing.assert_allclose(disp[k][box], want[..., k][box], rtol=0, atol=2e-5)
