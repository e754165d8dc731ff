"""Pins of the oracle's delivery timeline (Sec. 2.B, App. A), history
allocation and energy/mass-transfer accumulation (Sec. 2.D.2, Eqs. 2, 4-6).

Timeline: hand-worked examples (tests/golden), proton conservation, the
clock total, the one-phase test of Sec. 2.E and gating/repainting
invariants.  Allocation: exhaustive search on tiny plans.  EMTM: the
identity-DVF test of Sec. 2.E, integer and half-voxel translations
(closed forms), conservation, masking and the convergence in n reported in
Sec. 3.B.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- timeline
def _hand_cases():
    g = json.load(open(os.path.join(GOLDEN, "timeline_hand_examples.json")))
    plan = W.Plan(np.zeros(3), np.zeros(3), np.full(3, 100.0), np.zeros(3),
                  np.array(g["plan"]["protons"], np.uint64), np.array(g["plan"]["layer"], np.int32),
                  np.array(g["plan"]["field"], np.int32))
    out = []
    for c in g["cases"]:
        kw = dict(g["common"])
        kw.update({k: v for k, v in c.items() if k in W.Delivery.__dataclass_fields__})
        out.append((c["name"], plan, W.Delivery(**kw), c["expect"], c["end_ns"]))
    return out


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: c[0])
def test_timeline_hand_examples(orc, case):
    name, plan, dlv, expect, end_ns = case
    pp, fe, sp = orc.timeline(plan, dlv)
    want = np.zeros_like(pp)
    for s, d in expect.items():
        for ph, v in d.items():
            want[int(ph), int(s)] = v
    np.testing.assert_array_equal(pp, want)
    assert int(fe[0]) == end_ns and int(sp[0]) == dlv.start_phase


def _tumour_plan(n_layers=5, per_layer=30):
    ph, _, geo = W.phantom_4dct(64, 64, 40, with_dvf=False)
    return W.tumour_plan(geo, ph.origin, n_layers=n_layers, per_layer=per_layer)


def test_timeline_conserves_protons_and_clock(orc):
    plan = _tumour_plan()
    dlv = W.Delivery(start_phase=-1, seed=11)
    pp, fe, sp = orc.timeline(plan, dlv)
    np.testing.assert_array_equal(pp.sum(axis=0), plan.protons)
    # ungated: clock = spill time + (spots - layers) spot switches + (layers - 1) layer switches
    n = len(plan)
    n_layers = len(np.unique(plan.layer))
    spill = int(np.sum(plan.protons))          # rate 1e9 p/s: 1 ns per proton
    want = spill + (n - n_layers) * dlv.spot_switch_ns + (n_layers - 1) * dlv.layer_switch_ns
    assert int(fe[0]) == want
    assert 0 <= sp[0] < dlv.n_phases


def test_timeline_single_phase_puts_everything_on_phase_0(orc):
    """Sec. 2.E, second test: one phase -> the whole plan lands on it."""
    plan = _tumour_plan()
    pp, _, sp = orc.timeline(plan, W.Delivery(n_phases=1, start_phase=-1, seed=5))
    assert pp.shape[0] == 1 and sp[0] == 0
    np.testing.assert_array_equal(pp[0], plan.protons)


def test_timeline_short_delivery_stays_in_one_phase(orc):
    plan = W.Plan(np.zeros(3), np.zeros(3), np.full(3, 100.0), np.zeros(3),
                  np.array([10, 20, 30], np.uint64), np.zeros(3, np.int32), np.zeros(3, np.int32))
    dlv = W.Delivery(start_phase=7, spot_switch_ns=0, layer_switch_ns=0)
    pp, fe, _ = orc.timeline(plan, dlv)
    assert int(fe[0]) == 60
    np.testing.assert_array_equal(pp[7], plan.protons)
    assert pp.sum() == 60


def test_timeline_gating(orc):
    plan = _tumour_plan()
    g = W.Delivery(start_phase=2, gated=1, gate_first=4, gate_last=6)
    pp, fe, _ = orc.timeline(plan, g)
    np.testing.assert_array_equal(pp.sum(axis=0), plan.protons)
    off = [p for p in range(10) if not 4 <= p <= 6]
    assert pp[off].sum() == 0
    free, fe_free, _ = orc.timeline(plan, W.Delivery(start_phase=2))
    assert fe[0] > fe_free[0]
    # a window covering every phase is the same as free breathing
    allon, fe_all, _ = orc.timeline(plan, W.Delivery(start_phase=2, gated=1, gate_first=0, gate_last=9))
    np.testing.assert_array_equal(allon, free)
    assert fe_all[0] == fe_free[0]


def test_timeline_repainting(orc):
    plan = _tumour_plan()
    one, _, _ = orc.timeline(plan, W.Delivery(start_phase=0, repaints=1))
    plain, _, _ = orc.timeline(plan, W.Delivery(start_phase=0))
    np.testing.assert_array_equal(one, plain)
    four, fe4, _ = orc.timeline(plan, W.Delivery(start_phase=0, repaints=4))
    np.testing.assert_array_equal(four.sum(axis=0), plan.protons)
    # repainting spreads each spot over more phases on average
    assert np.mean((four > 0).sum(axis=0)) > np.mean((plain > 0).sum(axis=0))


def test_timeline_multi_field_independent_clocks(orc):
    plan = _tumour_plan(n_layers=3, per_layer=10)
    two = W.Plan(np.concatenate([plan.x, plan.x]), np.concatenate([plan.y, plan.y]),
                 np.concatenate([plan.energy, plan.energy]), np.concatenate([plan.sigma, plan.sigma]),
                 np.concatenate([plan.protons, plan.protons]), np.concatenate([plan.layer, plan.layer]),
                 np.concatenate([np.zeros(len(plan), np.int32), np.ones(len(plan), np.int32)]))
    pp2, fe2, _ = orc.timeline(two, W.Delivery(start_phase=3))
    pp1, fe1, _ = orc.timeline(plan, W.Delivery(start_phase=3))
    n = len(plan)
    np.testing.assert_array_equal(pp2[:, :n], pp1)
    np.testing.assert_array_equal(pp2[:, n:], pp1)
    assert fe2[0] == fe1[0] == fe2[1]


def test_timeline_random_start_phase(orc):
    plan = _tumour_plan(n_layers=2, per_layer=5)
    seen = set()
    for seed in range(60):
        _, _, sp = orc.timeline(plan, W.Delivery(start_phase=-1, seed=seed))
        seen.add(int(sp[0]))
    assert seen == set(range(10))
    a = orc.timeline(plan, W.Delivery(start_phase=-1, seed=9))
    b = orc.timeline(plan, W.Delivery(start_phase=-1, seed=9))
    np.testing.assert_array_equal(a[0], b[0])


def test_timeline_rejects_bad_input(orc):
    plan = _tumour_plan(n_layers=1, per_layer=3)
    for bad in (dict(n_phases=0), dict(repaints=0), dict(period_ns=0), dict(rate_protons_per_s=0),
                dict(gated=1, gate_first=5, gate_last=3), dict(start_phase=10),
                dict(gated=1, gate_first=4, gate_last=4, discard_ns=400_000_000)):
        with pytest.raises(ValueError):
            orc.timeline(plan, W.Delivery(**bad))


# -------------------------------------------------------------- allocation
def _alloc_exhaustive(p, n):
    """Largest-remainder allocation by exhaustive search: among the sets of
    spots given floor(q)+1, take the one whose chosen remainders are the
    largest (sorted descending, compared lexicographically), ties broken by
    the lexicographically smallest index set."""
    w = sum(p)
    q = [Fraction(n * v, w) for v in p]
    base = [int(x) for x in q]
    left = n - sum(base)
    best = None
    for combo in itertools.combinations(range(len(p)), left):
        key = (sorted([q[i] - base[i] for i in combo], reverse=True), [-i for i in combo])
        if best is None or key > best[0]:
            best = (key, combo)
    out = list(base)
    for i in best[1]:
        out[i] += 1
    return out


def test_allocation_exhaustive(orc):
    rng = np.random.default_rng(0)
    for _ in range(60):
        k = int(rng.integers(1, 8))
        p = [int(v) for v in rng.integers(0, 20, size=k)]
        if sum(p) == 0:
            p[0] = 1
        n = int(rng.integers(0, 40))
        got = [int(v) for v in orc.allocate(np.array(p, np.uint64), n)]
        assert got == _alloc_exhaustive(p, n), (p, n)


def test_allocation_large_invariants(orc):
    rng = np.random.default_rng(1)
    p = rng.integers(500_000, 1_500_000, size=3000).astype(np.uint64)
    n = 100_000_000
    a = orc.allocate(p, n)
    assert int(a.sum()) == n
    q = n * p.astype(np.float64) / p.astype(np.float64).sum()
    assert np.all(np.abs(a - q) < 1.0 + 1e-6)
    # equal weights: ties go to the lower spot index
    a = orc.allocate(np.full(7, 3, np.uint64), 10)
    assert list(a) == [2, 2, 2, 1, 1, 1, 1]


# -------------------------------------------------------------------- EMTM
def _fields(rng, n_phases, shape):
    dose = rng.gamma(2.0, 1.0, size=(n_phases,) + shape).astype(np.float32)
    rho = rng.choice(np.array([0.2, 1.0, 1.04, 1.7], np.float32), size=(n_phases,) + shape)
    return dose, rho.astype(np.float32)


def test_emtm_identity_reproduces_static_sum(orc):
    """Sec. 2.E, first test: the same geometry for every phase and an identity
    DVF give back the plain sum of the phase doses."""
    rng = np.random.default_rng(2)
    shape = (5, 6, 7)
    dose, rho = _fields(rng, 4, shape)
    rho[:] = rho[0]
    acc, dropped = orc.emtm(dose, rho, (1.0, 1.0, 2.5), 0, (2, 2, 5))
    assert dropped == 0
    np.testing.assert_allclose(acc, dose.astype(np.float64).sum(axis=0), rtol=1e-12)
    zero = np.zeros((4, 3) + shape, np.float32)
    acc0, _ = orc.emtm(dose, rho, (1.0, 1.0, 2.5), 0, (2, 2, 5), dvf=zero)
    np.testing.assert_array_equal(acc0, acc)


def test_emtm_integer_translation(orc):
    rng = np.random.default_rng(3)
    shape = (4, 5, 6)                         # nz, ny, nx
    dose, rho = _fields(rng, 2, shape)
    dvf = np.zeros((2, 3) + shape, np.float32)
    dvf[1, 0] = 2.0                           # +1 voxel in x (dx = 2 mm)
    dvf[1, 2] = -3.0                          # -1 voxel in z (dz = 3 mm)
    acc, dropped = orc.emtm(dose, rho, (2.0, 1.5, 3.0), 0, (2, 3, 2), dvf=dvf)
    want = dose[0].astype(np.float64).copy()
    shifted = np.zeros(shape)
    shifted[:-1, :, 1:] = dose[1][1:, :, :-1]
    want += shifted
    np.testing.assert_allclose(acc, want, rtol=1e-12)
    nz, ny, nx = shape
    lost = ny * (nz * 1 + nx * 1 - 1)         # source voxels with x = nx-1 or z = 0
    assert dropped == lost * 12


def test_emtm_half_voxel_translation_closed_form(orc):
    """Shift of half a voxel in x with two subvoxels along x: each reference
    voxel i takes one half of source voxel i and one of i-1, so
    D_i = (rho_i D_i + rho_{i-1} D_{i-1}) / (rho_i + rho_{i-1})."""
    rng = np.random.default_rng(4)
    shape = (3, 4, 8)
    dose, rho = _fields(rng, 2, shape)
    dvf = np.zeros((2, 3) + shape, np.float32)
    dvf[1, 0] = 0.5                            # dx = 1 mm
    acc, _ = orc.emtm(dose, rho, (1.0, 1.0, 1.0), 0, (2, 1, 1), dvf=dvf)
    d1 = dose[1].astype(np.float64); r1 = rho[1].astype(np.float64)
    want = dose[0].astype(np.float64).copy()
    want[:, :, 1:] += (r1[:, :, 1:] * d1[:, :, 1:] + r1[:, :, :-1] * d1[:, :, :-1]) / (
        r1[:, :, 1:] + r1[:, :, :-1])
    want[:, :, 0] += d1[:, :, 0]              # x = 0 receives only the left half of source voxel 0
    np.testing.assert_allclose(acc, want, rtol=1e-12)


def test_emtm_conserves_energy_and_mass(orc):
    rng = np.random.default_rng(5)
    shape = (8, 9, 10)
    dose, rho = _fields(rng, 3, shape)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    bump = np.sin(np.pi * (x + 0.5) / nx) * np.sin(np.pi * (y + 0.5) / ny) * np.sin(np.pi * (z + 0.5) / nz)
    dvf = np.zeros((3, 3) + shape, np.float32)
    for p in (1, 2):
        for a in range(3):
            dvf[p, a] = (0.7 * p * (a - 1) * bump * (bump > 0.2)).astype(np.float32)
    nsub = (2, 2, 3)
    acc, es, ms, dropped = orc.emtm(dose, rho, (1.0, 1.0, 1.0), 0, nsub, dvf=dvf, return_sums=True)
    assert dropped == 0
    k = nsub[0] * nsub[1] * nsub[2]
    r = rho[1:].astype(np.float64)
    d = dose[1:].astype(np.float64)
    np.testing.assert_allclose(ms.sum(), k * r.sum(), rtol=1e-12)
    np.testing.assert_allclose(es.sum(), k * (r * d).sum(), rtol=1e-12)


def test_emtm_mask(orc):
    rng = np.random.default_rng(6)
    shape = (3, 3, 3)
    dose, rho = _fields(rng, 2, shape)
    mask = (rng.random(shape) > 0.5).astype(np.uint8)
    full, _ = orc.emtm(dose, rho, (1, 1, 1), 0, (1, 1, 1))
    masked, _ = orc.emtm(dose, rho, (1, 1, 1), 0, (1, 1, 1), mask=mask)
    np.testing.assert_array_equal(masked, np.where(mask > 0, full, 0.0))


def test_emtm_converges_in_n(orc):
    """Sec. 3.B: EMTM with n = 1 differs visibly, while n = 2 already agrees
    closely with a fine subdivision."""
    n = 24
    shape = (n, n, n)
    c = (np.arange(n) + 0.5)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    dose1 = np.exp(-((x - 12) ** 2 + (y - 12) ** 2 + (z - 12) ** 2) / 30.0).astype(np.float32)
    dose = np.stack([np.zeros_like(dose1), dose1])
    rho = np.ones((2,) + shape, np.float32)
    dvf = np.zeros((2, 3) + shape, np.float32)
    dvf[1, 0] = (2.3 * np.sin(2 * np.pi * y / n) + 0.4 * np.cos(2 * np.pi * z / n)).astype(np.float32)
    dvf[1, 2] = (1.7 * np.cos(2 * np.pi * x / n)).astype(np.float32)
    res = {k: orc.emtm(dose, rho, (1, 1, 1), 0, (k, k, k), dvf=dvf)[0] for k in (1, 2, 6)}
    err1 = np.abs(res[1] - res[6]).mean()
    err2 = np.abs(res[2] - res[6]).mean()
    assert err2 < 0.5 * err1


def _emtm_numpy(dose, rho, d, nsub, u_x, flip_ties):
    """An independent restatement of Eqs. 2, 4-6 for a field that moves every
    point by the constant u_x (mm) along x: the subvoxel centre at cell
    coordinate t = j + (k + 1/2)/n lands in floor(t + u_x/d_x).  With
    ``flip_ties`` a point exactly on a cell face goes to the cell below it
    instead (the other legitimate decision).  Returns (accumulated dose,
    dropped count)."""
    P, nz, ny, nx = dose.shape
    dose, rho = dose.astype(np.float64), rho.astype(np.float64)
    acc = dose[0].copy()
    dropped = 0
    for S in range(1, P):
        E = np.zeros((nz, ny, nx))
        M = np.zeros((nz, ny, nx))
        for kz in range(nsub[2]):
            for ky in range(nsub[1]):
                for kx in range(nsub[0]):
                    t = np.arange(nx) + (kx + 0.5) / nsub[0] + u_x / d[0]
                    i = np.floor(t).astype(int)
                    if flip_ties:
                        i = np.where(t == np.floor(t), i - 1, i)
                    ok = (i >= 0) & (i < nx)
                    dropped += int((~ok).sum()) * nz * ny
                    for jx in np.nonzero(ok)[0]:
                        E[:, :, i[jx]] += rho[S, :, :, jx] * dose[S, :, :, jx]
                        M[:, :, i[jx]] += rho[S, :, :, jx]
        acc += np.where(M > 0, E / np.where(M > 0, M, 1.0), 0.0)
    return acc, dropped


def test_emtm_bounds_cover_either_decision_of_points_on_faces(orc):
    """A field of a quarter voxel along x with two subvoxels along x puts every
    second subvoxel centre exactly on a cell face (t = j + 1).  The oracle
    flags those points, decides them itself (floor: the upper cell), and
    bounds what any decision gives: an independent implementation deciding
    every tie the other way (the lower cell) gives another dose, inside the
    bounds, and a dropped count inside the reported range; an implementation
    deciding like the oracle gives the oracle's dose; voxels no tied point
    can reach have lo = hi = the oracle's dose."""
    rng = np.random.default_rng(11)
    shape = (3, 4, 7)
    dose, rho = _fields(rng, 3, shape)
    d = (2.0, 1.0, 1.0)
    dvf = np.zeros((3, 3) + shape, np.float32)
    dvf[1:, 0] = 0.5                                   # u/d = 1/4 exactly
    nsub = (2, 1, 1)
    acc, dropped, B = orc.emtm(dose, rho, d, 0, nsub, dvf=dvf, bounds=True)
    same, drop_same = _emtm_numpy(dose, rho, d, nsub, 0.5, flip_ties=False)
    other, drop_other = _emtm_numpy(dose, rho, d, nsub, 0.5, flip_ties=True)
    np.testing.assert_allclose(acc, same, rtol=1e-12)
    assert dropped == drop_same
    assert B["ambiguous"] == 2 * 3 * 4 * 7             # half of the subvoxels of two source phases
    assert not np.allclose(other, acc, rtol=1e-6)
    for a in (acc, other):
        assert np.all(a >= B["lo"] * (1 - 1e-12)) and np.all(a <= B["hi"] * (1 + 1e-12))
    assert B["dropped_min"] <= min(dropped, drop_other) and max(dropped, drop_other) <= B["dropped_max"]
    # no field: no ties, the bounds collapse onto the result
    acc0, _, B0 = orc.emtm(dose, rho, d, 0, nsub, bounds=True)
    assert B0["ambiguous"] == 0
    np.testing.assert_array_equal(B0["lo"], acc0)
    np.testing.assert_array_equal(B0["hi"], acc0)


def test_decode_flags_voxels_on_the_hull_faces(orc):
    """A registration grid whose hull faces pass through CT voxel centres:
    those voxels are flagged (either decision is correct there), the ones
    strictly inside or outside are not, and the FP64 decision puts the faces
    inside (the hull is closed)."""
    g = dict(n=(5, 4, 3), start_mm=(1.0, 1.0, 1.0), spacing_mm=(2.0, 2.0, 2.0), row_cos=(1, 0, 0),
             col_cos=(0, 1, 0))
    delta = np.zeros((3, 4, 5, 3), np.float32)
    n = (12, 10, 8)
    _, inside, amb = orc.dvf_decode(g, delta, n, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), return_ambiguous=True)
    # CT centres i + 1/2 never meet the grid points 1 + 2 m: nothing is on a face
    assert amb.sum() == 0 and inside.sum() > 0
    g2 = dict(g, start_mm=(0.5, 0.5, 0.5))                # grid points on CT centres 0, 2, 4, ...
    _, inside2, amb2 = orc.dvf_decode(g2, delta, n, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), return_ambiguous=True)
    k, j, i = np.meshgrid(np.arange(8), np.arange(10), np.arange(12), indexing="ij")
    want_in = (i <= 8) & (j <= 6) & (k <= 4)
    np.testing.assert_array_equal(inside2.astype(bool), want_in)
    face = want_in & ((i == 0) | (i == 8) | (j == 0) | (j == 6) | (k == 0) | (k == 4))
    np.testing.assert_array_equal(amb2.astype(bool), face)
