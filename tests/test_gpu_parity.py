"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact where the method is integer or decided by integers (Philox,
delivery timeline, history allocation, EMTM target voxels, tallies across
runs, launch shapes and batching); within the stated tolerances where it is
floating point (lookup tables) or statistical (Monte Carlo dose):

* per-voxel |D_gpu - D_oracle| <= 3 sigma_comb for >= 99.5 % of voxels above
  10 % Dmax (independent seeds; sigma from oracle batches scaled to both
  history counts);
* |D_gpu - D_oracle| <= 1 % Dmax for >= 99 % of voxels above 10 % Dmax and
  global gamma(1 %, 1 mm) >= 99 %, against 1e7-history oracle references
  (tests/golden, written by make_oracle_reference.py) so that Monte Carlo
  noise stays well below 1 % of Dmax;
* matched random streams (same seed) agree voxel by voxel to 0.2 % of Dmax
  whenever multiple scattering is off.
"""
import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------------ random
def test_philox_bit_exact(gpu, orc):
    import os
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(v, 16) for v in line.split()])
    rng = np.random.default_rng(0)
    ctr = np.array([r[0:4] for r in rows] + list(rng.integers(0, 2 ** 32, size=(500, 4))), np.uint32)
    key = np.array([r[4:6] for r in rows] + list(rng.integers(0, 2 ** 32, size=(500, 2))), np.uint32)
    w, u = gpu.dose_debug_philox(ctr, key)
    for i in range(3):
        assert [int(v) for v in w[i]] == rows[i][6:10]
    for i in range(len(ctr)):
        assert np.array_equal(w[i], orc.philox4x32_10(ctr[i], key[i]))
    # the transport's uniforms of (block, history, stream) under seed
    for h in (0, 1, 12345, (1 << 32) + 7):
        for block in (0, 1, 99):
            seed = 0x1234_5678_9ABC_DEF0
            c = np.array([[block, h & 0xFFFFFFFF, h >> 32, 3]], np.uint32)
            k = np.array([[seed & 0xFFFFFFFF, seed >> 32]], np.uint32)
            _, uu = gpu.dose_debug_philox(c, k)
            np.testing.assert_array_equal(uu[0].astype(np.float64), orc.block_uniforms(seed, h, 3, block))


def test_lookup_tables_vs_fp64(gpu, orc):
    e = np.concatenate([np.linspace(0.6, 250.0, 997), [1.0, 7.5, 70.0, 150.0, 200.0]]).astype(np.float32)
    t = gpu.dose_debug_tables(e)
    for i, ei in enumerate(e.astype(np.float64)):
        r = orc.range_mm(ei)
        assert abs(t[i, 0] - r) <= 2e-5 * r + 2e-4, ei        # mm; largest near the cut-off
        assert abs(t[i, 1] - ei) <= 1e-4 * ei + 2e-3, ei       # MeV; largest in the last micrometres
        assert abs(t[i, 2] - orc.bohr_var(ei, 1.0)) <= 1e-5 * orc.bohr_var(ei, 1.0)
        hl = (13.6 / orc.pv(ei)) ** 2
        assert abs(t[i, 3] - hl) <= 2e-4 * hl, ei
        s = orc.sigma_nuc(ei) / 10.0
        assert abs(t[i, 4] - s) <= 1e-4 * 0.00123 + 1e-5 * s


# --------------------------------------------------------------- timeline
def _timeline_gpu(D, plan, dlv, n_phases):
    ph = W.water_phantom(8, 8, 8)
    hu = np.repeat(ph.hu[None], n_phases, axis=0)
    ctx = D.dose_create_grid(8, 8, 8, 2, 2, 2, ph.origin, n_phases, hu, (0, 0, 1))
    try:
        D.dose_add_spots(ctx, D.spots_array(plan), D.delivery_struct(dlv))
        pp = D.dose_read(ctx, D.DOSE_SUBPLAN, 0, np.zeros((n_phases, len(plan)), np.uint64))
        nf = int(np.max(plan.field)) + 1
        sp = D.dose_read(ctx, D.DOSE_START_PHASE, 0, np.zeros(nf, np.int32))
        fe = D.dose_read(ctx, D.DOSE_FIELD_END_NS, 0, np.zeros(nf, np.int64))
        return pp, fe, sp
    finally:
        D.dose_destroy(ctx)


@pytest.mark.parametrize("variant", ["free", "random_start", "gated", "repaint4", "gated_discard",
                                     "slow_rate", "two_fields"])
def test_timeline_bit_exact(gpu, orc, variant):
    ph, _, geo = H.small_4dct(n_phases=10)
    plan = W.tumour_plan(geo, ph.origin, n_layers=20, per_layer=150)
    dlv = {"free": W.Delivery(start_phase=3),
           "random_start": W.Delivery(start_phase=-1, seed=77),
           "gated": W.Delivery(start_phase=1, gated=1, gate_first=4, gate_last=6),
           "repaint4": W.Delivery(start_phase=-1, seed=5, repaints=4),
           "gated_discard": W.Delivery(start_phase=8, gated=1, gate_first=3, gate_last=7,
                                       discard_ns=70_000_000),
           "slow_rate": W.Delivery(start_phase=0, rate_protons_per_s=333_333_333),
           "two_fields": W.Delivery(start_phase=-1, seed=9)}[variant]
    if variant == "two_fields":
        f = np.zeros(len(plan), np.int32)
        f[len(plan) // 2:] = 1
        plan = W.Plan(plan.x, plan.y, plan.energy, plan.sigma, plan.protons, plan.layer, f)
    pp, fe, sp = _timeline_gpu(gpu, plan, dlv, 10)
    opp, ofe, osp = orc.timeline(plan, dlv)
    np.testing.assert_array_equal(pp, opp)
    np.testing.assert_array_equal(fe, ofe)
    np.testing.assert_array_equal(sp, osp)
    np.testing.assert_array_equal(pp.sum(axis=0), plan.protons)


def test_timeline_one_phase(gpu):
    """Sec. 2.E: with one phase the whole plan lands on it."""
    ph, _, geo = H.small_4dct(n_phases=10)
    plan = W.tumour_plan(geo, ph.origin, n_layers=5, per_layer=30)
    pp, _, sp = _timeline_gpu(gpu, plan, W.Delivery(n_phases=1, start_phase=-1), 1)
    np.testing.assert_array_equal(pp[0], plan.protons)
    assert sp[0] == 0


# ------------------------------------------------------------- allocation
@pytest.mark.parametrize("n_hist", [1, 7, 399, 400, 401, 123457, 10_000_000])
def test_allocation_bit_exact(gpu, orc, n_hist):
    ph = W.slab_phantom(n=32)
    plan = W.slab_plan()
    ctx = H.make_ctx(gpu, ph)
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(plan), None)
        gpu.dose_set_option(ctx, gpu.DOSE_OPT_PHYSICS, 0)
        gpu.dose_run_phase(ctx, 0, n_hist, 1)
        pre = gpu.dose_read(ctx, gpu.DOSE_HIST_PREFIX, 0, np.zeros(len(plan) + 1, np.uint64))
        led = gpu.dose_read(ctx, gpu.DOSE_ENERGY_LEDGER, 0, np.zeros(8, np.uint64))
    finally:
        gpu.dose_destroy(ctx)
    np.testing.assert_array_equal(np.diff(pre), orc.allocate(plan.protons, n_hist))
    assert int(led[5]) == n_hist and int(led[7]) == int(plan.protons.sum())


# --------------------------------------------------------------- transport
def test_csda_deterministic_depth_dose(gpu, orc):
    """Straggling, scattering and nuclear removal off, zero-width pencil:
    every history is identical on both sides, so the per-voxel doses must
    agree to table/FP32 accuracy."""
    ph = W.water_phantom(nx=8, ny=8, nz=100)
    pl = W.pencil_plan(energy=150.0, sigma=0.0)
    g = H.gpu_run(gpu, ph, pl, 1000, 1, physics=0)
    o, _ = H.oracle_batches(orc, ph, pl, 1000, 1, physics=0)
    dmax = o.max()
    assert np.max(np.abs(g["dose"] - o)) <= 1e-3 * dmax
    np.testing.assert_array_equal(g["dose"] > 0, o > 0)


def _config1(n=64, nz=160):
    return W.water_phantom(nx=n, ny=n, nz=nz), W.pencil_plan(energy=150.0, sigma=4.0)


@pytest.mark.parametrize("physics", [0, 1, 4, 5])
def test_matched_streams_without_scattering(gpu, orc, physics):
    """Without multiple scattering the step sequence of a history does not
    depend on rounding, so with the same seed the GPU (FP32) and the oracle
    (FP64) follow the same histories and agree voxel by voxel.  (With
    scattering on, rounding changes which voxel face a step ends on and the
    same random numbers then drive different paths: the oracle rounded to
    float after every step decorrelates from itself just as much, so the
    scattering physics is compared statistically below.)"""
    ph, pl = _config1(n=32, nz=100)
    n = 100_000
    g = H.gpu_run(gpu, ph, pl, n, 1, physics=physics)
    o, _ = H.oracle_batches(orc, ph, pl, n, 1, physics=physics)
    assert np.max(np.abs(g["dose"] - o)) <= 0.002 * o.max()


def _lateral_sigma(d, axis_sum, spacing):
    p = d.sum(axis=axis_sum)
    x = (np.arange(p.shape[-1]) + 0.5) * spacing
    w = p.sum(axis=-1)
    safe = np.where(w > 0, w, 1.0)                 # depths the beam never reaches: nan
    m = np.where(w > 0, (p * x).sum(axis=-1) / safe, np.nan)
    return np.where(w > 0, np.sqrt((p * (x - m[:, None]) ** 2).sum(axis=-1) / safe), np.nan), m


def _comb(sg, so):
    return np.sqrt(sg * sg + so * so)


def test_dose_parity_independent_streams(gpu, orc):
    """Config-1 geometry, equal history counts on both sides, independent
    seeds, standard errors estimated on both sides (100 batches each): 3
    sigma per voxel; depth-dose within 1 % of its maximum; lateral spread per
    depth within 1 %."""
    ph, pl = _config1()
    n = 200_000
    g, sg = H.gpu_batches(gpu, ph, pl, n, 12345, 100)
    o, so = H.oracle_batches(orc, ph, pl, n, 777, n_batches=100)
    dmax = o.max()
    frac, nsel = H.sigma_pass(g, o, _comb(sg, so), dmax)
    assert nsel > 1000 and frac >= 0.995, frac
    dg, do = g.sum(axis=(1, 2)), o.sum(axis=(1, 2))
    assert np.max(np.abs(dg - do)) <= 0.01 * do.max()
    sgl, _ = _lateral_sigma(g, 1, 2.0)
    sol, _ = _lateral_sigma(o, 1, 2.0)
    zs = do > 0.2 * do.max()
    assert np.max(np.abs(sgl[zs] - sol[zs]) / sol[zs]) < 0.02


def _golden(name):
    import os
    f = np.load(os.path.join(os.path.dirname(__file__), "golden", f"oracle_{name}.npz"))
    lo = f["lo"]
    box = tuple(slice(int(a), int(a) + s) for a, s in zip(lo, f["mean"].shape))
    return box, f["mean"].astype(np.float64), f["sem"].astype(np.float64), float(f["dmax"]), int(f["n_hist"])


def test_high_statistics_pencil_beam(gpu):
    """Config 1 (150 MeV pencil, sigma 4 mm, water 64x64x160 at 2 mm): 1e8
    GPU histories (20 independent batches) against the 1e7-history oracle
    reference: 3 sigma, 1 % Dmax and gamma(1 %/1 mm)."""
    box, mean, sem, dmax, n_o = _golden("pencil_1e7")
    ph, pl = _config1()
    g, sg = H.gpu_batches(gpu, ph, pl, 100_000_000, 4242, 20)
    g, sg = g[box], sg[box]
    frac, nsel = H.sigma_pass(g, mean, _comb(sg, sem), dmax)
    assert nsel > 500 and frac >= 0.995, frac
    assert H.dmax_pass(g, mean, dmax) >= 0.99
    assert H.gamma_pass(mean, g, ph.d) >= 0.99


def test_full_size_slab_workload(gpu, orc):
    """The benchmark workload at full size (slab phantom 128^3, 400 spots) in
    the benchmark's launch configuration: at 1e7 histories the allocation is
    bit-exact, the energy ledger balances and a rerun is bit-identical; then
    1e9 histories (100 independent runs of 1e7) against the 2e8-history
    oracle reference at the full criteria, over the voxels above 10 % of
    Dmax: within 3 combined standard errors (>= 99.5 %), within 1 % of Dmax
    (>= 99 %), and gamma(1 %/1 mm, global) >= 99 %."""
    box, mean, sem, dmax, n_o = _golden("slab_2e8")
    assert n_o == 200_000_000
    ph, pl = W.slab_phantom(128), W.slab_plan(seed=2)
    n = 10_000_000
    ctx = H.make_ctx(gpu, ph)
    try:
        a = H.gpu_run(gpu, ph, pl, n, 2, ctx=ctx)
        pre = gpu.dose_read(ctx, gpu.DOSE_HIST_PREFIX, 0, np.zeros(len(pl) + 1, np.uint64))
        b = H.gpu_run(gpu, ph, pl, n, 2, ctx=ctx)
    finally:
        gpu.dose_destroy(ctx)
    np.testing.assert_array_equal(np.diff(pre), orc.allocate(pl.protons, n))
    np.testing.assert_array_equal(a["tally"], b["tally"])
    dep, esc, rem, inc, steps = [int(v) for v in a["ledger"][:5]]
    assert abs(dep + esc + rem - inc) <= steps + inc * 2.0 ** -22
    g, sg = H.gpu_batches_on_device(gpu, ph, pl, 1_000_000_000, 77, 100)
    g, sg = g[box], sg[box]
    frac, nsel = H.sigma_pass(g, mean, _comb(sg, sem), dmax)
    one = H.dmax_pass(g, mean, dmax)
    gam = H.gamma_pass(mean, g, ph.d)
    print(f"slab 1e9 vs oracle 2e8: {nsel} voxels, 3 sigma {frac:.4f}, 1 % Dmax {one:.4f}, gamma {gam:.4f}")
    assert nsel > 500 and frac >= 0.995, frac
    assert one >= 0.99, one
    assert gam >= 0.99, gam


def _blocks(a, b):
    """Sums of a (z, y, x) array over blocks of b voxels (trailing partial blocks dropped)."""
    nz, ny, nx = a.shape
    bz, by, bx = b
    a = a[:nz - nz % bz, :ny - ny % by, :nx - nx % bx]
    return a.reshape(a.shape[0] // bz, bz, a.shape[1] // by, by, a.shape[2] // bx, bx).sum(axis=(1, 3, 5))


def test_full_size_4dct_phase(gpu, orc):
    """Phase 0 of the 10-phase 256x256x160 4DCT at 1x1x2.5 mm with the whole
    3000-spot plan (20 layers, 70-180 MeV) along +y: 1e9 histories (100
    independent runs of 1e7) against the 1e8-history oracle reference, inside
    the body contour.

    In these 2.5 mm^3 voxels a single dose is heavy-tailed: the local deposit
    of a nuclear removal puts 60 % of a proton's energy into one voxel (five
    times the dose per MeV in lung), so at 1e8 oracle histories the batch
    estimate of a voxel's standard error is itself unreliable (median 1 % of
    Dmax).  Measured on the oracle against itself (an independent 1e7-history
    run against this reference) only 93.6 % of the voxels fall within 3
    estimated combined errors.  The criteria are therefore: per voxel above
    10 % of Dmax, within 3 combined errors for >= 98 %; the deposited energy
    along the beam and across it (dose x density summed over the other two
    axes, noise ~0.03 % of the maximum) within 1 % of its maximum; the dose of
    2x4x4-voxel blocks (5 x 4 x 4 mm, energy over mass) within 1 % of the
    block Dmax for >= 99 % of the blocks above 10 %; and gamma(1 %/1 mm) >= 99 %
    on the voxels whose combined error is at most a third of 1 % of Dmax."""
    box, mean, sem, dmax, n_o = _golden("4dct_p0_1e8")
    assert n_o == 100_000_000
    ph, _, geo = W.phantom_4dct(with_dvf=False)
    ph = W.Phantom(np.ascontiguousarray(ph.hu[0]), ph.d, ph.origin, ph.beam_axis, ph.beam_sign)
    plan = W.tumour_plan(geo, ph.origin)
    g, sg = H.gpu_batches_on_device(gpu, ph, plan, 1_000_000_000, 101, 100)
    rho = orc.density(ph)[box]
    body = rho >= 0.1
    g, sg = np.where(body, g[box], 0.0), np.where(body, sg[box], 0.0)
    mean, sem = np.where(body, mean, 0.0), np.where(body, sem, 0.0)
    comb = _comb(sg, sem)
    frac, nsel = H.sigma_pass(g, mean, comb, dmax)
    profiles = []
    for axes in ((0, 2), (0, 1), (1, 2)):                 # along y (the beam), along z, along x
        pg, po = (g * rho).sum(axis=axes), (mean * rho).sum(axis=axes)
        keep = po >= 0.1 * po.max()
        profiles.append(float(np.max(np.abs(pg - po)[keep]) / po.max()))
    mass = _blocks(rho, (2, 4, 4))
    bg = _blocks(g * rho, (2, 4, 4)) / np.maximum(mass, 1e-30)
    bo = _blocks(mean * rho, (2, 4, 4)) / np.maximum(mass, 1e-30)
    bsel = bo >= 0.1 * bo.max()
    blocks1 = float(np.mean((np.abs(bg - bo) <= 0.01 * bo.max())[bsel]))
    sel = mean >= 0.1 * dmax
    resolved = sel & (comb <= dmax * 0.01 / 3.0)
    gam = H.gamma_pass(mean, g, ph.d, dmax=dmax, select=resolved)
    print(f"4DCT phase 1e9 vs oracle 1e8: {nsel} voxels, 3 sigma {frac:.4f}; energy profiles (y, z, x) max "
          f"|diff| {profiles[0]:.4f} {profiles[1]:.4f} {profiles[2]:.4f} of their maxima; {int(bsel.sum())} blocks "
          f"within 1 % of Dmax {blocks1:.4f}; gamma on {int(resolved.sum())} resolved voxels {gam:.4f}")
    assert nsel > 100_000 and frac >= 0.98, frac
    assert max(profiles) <= 0.01, profiles
    assert bsel.sum() > 5000 and blocks1 >= 0.99, blocks1
    assert resolved.sum() >= 5000 and gam >= 0.99, gam


def test_slab_parity(gpu, orc):
    ph = W.slab_phantom(n=64)
    pl = W.slab_plan(n_layers=4, nx=3, ny=2)
    n = 100_000
    g, sg = H.gpu_batches(gpu, ph, pl, n, 99, 100)
    o, so = H.oracle_batches(orc, ph, pl, n, 7, n_batches=100)
    frac, _ = H.sigma_pass(g, o, _comb(sg, so), o.max())
    assert frac >= 0.995, frac


def test_4dct_phase_parity_beam_along_y(gpu, orc):
    """AP beam through air, body, lung and tumour; voxels inside the body."""
    ph, _, geo = H.small_4dct(n_phases=3)
    plan = W.tumour_plan(geo, ph.origin, n_layers=3, per_layer=12, e_lo=70.0, e_hi=110.0)
    n = 100_000
    for phase in (0, 2):
        body = H.body_mask(orc, ph, phase)
        g, sg = H.gpu_batches(gpu, ph, plan, n, 3, 100, phase=phase)
        o, so = H.oracle_batches(orc, ph, plan, n, 13, phase=phase, stream=phase, n_batches=100)
        g, o = np.where(body, g, 0.0), np.where(body, o, 0.0)
        frac, nsel = H.sigma_pass(g, o, _comb(sg, so), o.max())
        assert nsel > 1000 and frac >= 0.995, (phase, frac)


def test_spr_scale_and_shift(gpu, orc):
    ph, pl = _config1(n=32, nz=100)
    n = 100_000
    kw = dict(spr_scale=1.035, shift=(3.0, -3.0, 3.0))
    g, sg = H.gpu_batches(gpu, ph, pl, n, 8, 100, **kw)
    o, so = H.oracle_batches(orc, ph, pl, n, 18, n_batches=100, **kw)
    frac, _ = H.sigma_pass(g, o, _comb(sg, so), o.max())
    assert frac >= 0.995, frac
    # the setup shift moves the dose by -shift laterally
    g1 = H.gpu_run(gpu, ph, pl, 2_000_000, 8, **kw)["dose"]
    g0 = H.gpu_run(gpu, ph, pl, 2_000_000, 8, spr_scale=1.035)["dose"]
    _, mx = _lateral_sigma(g1, 1, 2.0)
    _, mx0 = _lateral_sigma(g0, 1, 2.0)
    dd = g0.sum(axis=(1, 2))
    zs = dd > 0.3 * dd.max()
    assert np.all(np.abs((mx - mx0)[zs] + 3.0) < 0.1)


def test_energy_balance(gpu):
    ph = W.slab_phantom(n=64)
    pl = W.slab_plan(n_layers=4, nx=3, ny=2)
    g = H.gpu_run(gpu, ph, pl, 500_000, 2)
    dep, esc, rem, inc, steps, hist, flags, w = [int(v) for v in g["ledger"]]
    assert dep == int(g["tally"].sum(dtype=np.uint64))
    # per deposit: half a unit of rounding plus the FP32 product e * w (2^-24 relative)
    assert abs(dep + esc + rem - inc) <= steps + inc * 2.0 ** -22
    assert hist == 500_000 and flags == 0 and esc > 0 and rem > 0


# ---------------------------------------------------- determinism, batching
def test_bit_reproducible_across_runs_and_launch_shapes(gpu):
    ph = W.slab_phantom(n=48)
    pl = W.slab_plan(n_layers=3, nx=3, ny=2)
    ref = H.gpu_run(gpu, ph, pl, 300_000, 4)["tally"]
    again = H.gpu_run(gpu, ph, pl, 300_000, 4)["tally"]
    np.testing.assert_array_equal(ref, again)
    for opts in ({gpu.DOSE_OPT_BLOCK: 128}, {gpu.DOSE_OPT_BLOCK: 512, gpu.DOSE_OPT_CHUNK: 7},
                 {gpu.DOSE_OPT_BLOCKS_PER_SM: 1, gpu.DOSE_OPT_CHUNK: 1000},
                 {gpu.DOSE_OPT_REGISTERS: 0, gpu.DOSE_OPT_BLOCK: 256, gpu.DOSE_OPT_CHUNK: 64},
                 {gpu.DOSE_OPT_REGISTERS: 0, gpu.DOSE_OPT_BLOCK: 512, gpu.DOSE_OPT_MATERIAL_GRID: 1},
                 {gpu.DOSE_OPT_REGISTERS: 1, gpu.DOSE_OPT_BLOCK: 256, gpu.DOSE_OPT_CHUNK: 32}):
        np.testing.assert_array_equal(H.gpu_run(gpu, ph, pl, 300_000, 4, options=opts)["tally"], ref)


def test_history_slices_equal_one_run(gpu):
    ph = W.slab_phantom(n=48)
    pl = W.slab_plan(n_layers=3, nx=3, ny=2)
    n = 300_000
    ref = H.gpu_run(gpu, ph, pl, n, 4)
    ctx = H.make_ctx(gpu, ph)
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(pl), None)
        cuts = [0, 1, 99_999, 250_000, n]
        for i in range(4):
            flags = (gpu.DOSE_JOB_CLEAR if i == 0 else 0) | (gpu.DOSE_JOB_FINISH if i == 3 else 0)
            gpu.dose_run_batch(gpu.make_jobs([dict(ctx=ctx, phase=0, n_histories=n, flags=flags,
                                                   hist_begin=cuts[i], hist_end=cuts[i + 1], seed=4)]))
        shape = ph.hu.shape
        tally = gpu.dose_read(ctx, gpu.DOSE_TALLY_I64, 0, np.zeros(shape, np.uint64))
        dose = gpu.dose_read(ctx, gpu.DOSE_PHASE_DOSE, 0, np.zeros(shape, np.float32))
    finally:
        gpu.dose_destroy(ctx)
    np.testing.assert_array_equal(tally, ref["tally"])
    np.testing.assert_array_equal(dose, ref["dose"])


def test_ragged_batch_equals_jobs_alone(gpu):
    rng = np.random.default_rng(11)
    specs = []
    for side, n in ((32, 50_000), (48, 200_000), (40, 10_000)):
        ph = W.random_phantom(rng, side)
        pl = W.random_plan(rng, int(rng.integers(20, 60)), side * 0.6)
        specs.append((ph, pl, n))
    alone = [H.gpu_run(gpu, ph, pl, n, 21 + i)["tally"] for i, (ph, pl, n) in enumerate(specs)]
    ctxs = [H.make_ctx(gpu, ph) for ph, _, _ in specs]
    try:
        for c, (ph, pl, n) in zip(ctxs, specs):
            gpu.dose_add_spots(c, gpu.spots_array(pl), None)
        gpu.dose_run_batch(gpu.make_jobs([dict(ctx=c, phase=0, n_histories=n, seed=21 + i)
                                          for i, (c, (_, _, n)) in enumerate(zip(ctxs, specs))]))
        for c, (ph, _, _), ref in zip(ctxs, specs, alone):
            t = gpu.dose_read(c, gpu.DOSE_TALLY_I64, 0, np.zeros(ph.hu.shape, np.uint64))
            np.testing.assert_array_equal(t, ref)
    finally:
        for c in ctxs:
            gpu.dose_destroy(c)


def test_specialised_and_generic_builds_agree(gpu):
    """The transport is built generic and for all-physics jobs with either
    material source; the launcher picks the build from the jobs.  A job run
    alone (its specialised build) and the same job in a batch whose jobs
    mix physics masks and material sources (the generic build) give the
    same tally bits, as does a batch of only all-physics grid jobs."""
    rng = np.random.default_rng(17)
    specs = []   # (phantom, plan, histories, physics, material grid)
    for side, n, phys, grid in ((32, 60_000, 7, 1), (40, 80_000, 7, 0), (36, 50_000, 3, 1), (32, 40_000, 6, 0)):
        specs.append((W.random_phantom(rng, side), W.random_plan(rng, int(rng.integers(20, 50)), side * 0.6),
                      n, phys, grid))
    alone = [H.gpu_run(gpu, ph, pl, n, 40 + i, physics=phys, options={gpu.DOSE_OPT_MATERIAL_GRID: grid})["tally"]
             for i, (ph, pl, n, phys, grid) in enumerate(specs)]

    def batch(idx):
        ctxs = [H.make_ctx(gpu, specs[i][0]) for i in idx]
        try:
            for c, i in zip(ctxs, idx):
                gpu.dose_set_option(c, gpu.DOSE_OPT_PHYSICS, specs[i][3])
                gpu.dose_set_option(c, gpu.DOSE_OPT_MATERIAL_GRID, specs[i][4])
                gpu.dose_add_spots(c, gpu.spots_array(specs[i][1]), None)
            gpu.dose_run_batch(gpu.make_jobs([dict(ctx=c, phase=0, n_histories=specs[i][2], seed=40 + i)
                                              for c, i in zip(ctxs, idx)]))
            for c, i in zip(ctxs, idx):
                t = gpu.dose_read(c, gpu.DOSE_TALLY_I64, 0, np.zeros(specs[i][0].hu.shape, np.uint64))
                np.testing.assert_array_equal(t, alone[i])
        finally:
            for c in ctxs:
                gpu.dose_destroy(c)

    batch([0, 1, 2, 3])      # mixed masks and sources: the generic build
    batch([2, 0])            # a partial mask first
    batch([0, 0])            # all physics, all grids: the specialised table build


def test_batch_of_large_jobs_equals_jobs_alone(gpu):
    """Jobs of at least 2^25 histories each run as consecutive single-job
    launches within the batch (each with its own work counter); the tallies
    are those of the jobs run alone, including a job that is a later slice
    of a run (its history range starts past zero)."""
    ph = W.water_phantom(24, 24, 60)
    pl = W.pencil_plan(120.0, 3.0)
    n = 1 << 25
    alone = [H.gpu_run(gpu, ph, pl, n, 60 + i, physics=7 if i else 3)["tally"] for i in range(2)]
    ctxs = [H.make_ctx(gpu, ph) for _ in range(3)]
    try:
        for i, c in enumerate(ctxs):
            gpu.dose_set_option(c, gpu.DOSE_OPT_PHYSICS, 3 if i == 0 else 7)
            gpu.dose_add_spots(c, gpu.spots_array(pl), None)
        # ctx 2: the second run in two slices, the first alone, the second in the batch
        gpu.dose_run_batch(gpu.make_jobs([dict(ctx=ctxs[2], phase=0, n_histories=2 * n, seed=61,
                                               hist_begin=0, hist_end=n, flags=gpu.DOSE_JOB_CLEAR)]))
        gpu.dose_run_batch(gpu.make_jobs([dict(ctx=ctxs[0], phase=0, n_histories=n, seed=60),
                                          dict(ctx=ctxs[1], phase=0, n_histories=n, seed=61),
                                          dict(ctx=ctxs[2], phase=0, n_histories=2 * n, seed=61,
                                               hist_begin=n, hist_end=2 * n, flags=gpu.DOSE_JOB_FINISH)]))
        for i in range(2):
            t = gpu.dose_read(ctxs[i], gpu.DOSE_TALLY_I64, 0, np.zeros(ph.hu.shape, np.uint64))
            np.testing.assert_array_equal(t, alone[i])
        whole = H.gpu_run(gpu, ph, pl, 2 * n, 61)["tally"]
        t = gpu.dose_read(ctxs[2], gpu.DOSE_TALLY_I64, 0, np.zeros(ph.hu.shape, np.uint64))
        np.testing.assert_array_equal(t, whole)
    finally:
        for c in ctxs:
            gpu.dose_destroy(c)


def test_view_shares_grid(gpu):
    ph = W.slab_phantom(n=32)
    pl = W.slab_plan(n_layers=2, nx=2, ny=2)
    base = H.make_ctx(gpu, ph)
    try:
        view = gpu.dose_create_view(base)
        try:
            a = H.gpu_run(gpu, ph, pl, 50_000, 3, ctx=base)["tally"]
            b = H.gpu_run(gpu, ph, pl, 50_000, 3, ctx=view)["tally"]
            np.testing.assert_array_equal(a, b)
        finally:
            gpu.dose_destroy(view)
        rho = gpu.dose_read(base, gpu.DOSE_DENSITY, 0, np.zeros(ph.hu.shape, np.float32))
        assert rho.min() > 0
    finally:
        gpu.dose_destroy(base)


# ---------------------------------------------------------- failure paths
def test_step_limit_reported(gpu, orc):
    """A history that reaches the step limit stops after that many steps with
    its energy counted as escaped, and the run reports DOSE_ESTEPLIMIT; with
    matched streams (no scattering) the deposits of the first steps are the
    oracle's, whose histories stop at the same step."""
    ph, pl = _config1(n=16, nz=100)
    g = H.gpu_run(gpu, ph, pl, 1000, 1, options={gpu.DOSE_OPT_MAX_STEPS: 5})
    assert g["status"] == gpu.DOSE_ESTEPLIMIT
    dep, esc, rem, inc = [int(v) for v in g["ledger"][:4]]
    assert abs(dep + esc + rem - inc) <= 6000
    ok = H.gpu_run(gpu, ph, pl, 1000, 1)
    assert ok["status"] == gpu.DOSE_OK
    phys = orc.PHYS_STRAGGLING | orc.PHYS_NUCLEAR
    m = H.gpu_run(gpu, ph, pl, 20_000, 3, physics=phys, options={gpu.DOSE_OPT_MAX_STEPS: 7})
    o = orc.dose(ph, pl, 20_000, 3, physics=phys, max_steps=7)
    assert o["status"] == orc.ESTEP and m["status"] == gpu.DOSE_ESTEPLIMIT
    assert np.max(np.abs(m["dose"] - o["dose"])) <= 0.002 * o["dose"].max()
    assert int(m["ledger"][4]) == o["steps"]


def test_errors_leave_context_usable(gpu):
    ph, pl = _config1(n=16, nz=40)
    ctx = H.make_ctx(gpu, ph)
    try:
        with pytest.raises(gpu.DoseError) as e:
            gpu.dose_run_phase(ctx, 0, 100, 1)
        assert e.value.code == gpu.DOSE_ESTATE
        gpu.dose_add_spots(ctx, gpu.spots_array(pl), None)
        with pytest.raises(gpu.DoseError) as e:
            gpu.dose_run_phase(ctx, 1, 100, 1)
        assert e.value.code == gpu.DOSE_EINVAL
        with pytest.raises(gpu.DoseError) as e:
            gpu.dose_read(ctx, gpu.DOSE_PHASE_DOSE, 0, np.zeros(3, np.float32))
        assert e.value.code == gpu.DOSE_ESTATE
        gpu.dose_set_option(ctx, gpu.DOSE_OPT_FAIL_ALLOC_AFTER, 0)
        with pytest.raises(gpu.DoseError) as e:
            gpu.dose_run_phase(ctx, 0, 100, 1)
        assert e.value.code == gpu.DOSE_ENOMEM
        gpu.dose_set_option(ctx, gpu.DOSE_OPT_FAIL_ALLOC_AFTER, -1)
        gpu.dose_run_phase(ctx, 0, 1000, 1)
        d = gpu.dose_read(ctx, gpu.DOSE_PHASE_DOSE, 0, np.zeros(ph.hu.shape, np.float32))
        assert d.max() > 0
    finally:
        gpu.dose_destroy(ctx)


# -------------------------------------------------------------------- EMTM
def _emtm_inputs(orc, n_phases=4):
    ph, dvf, geo = H.small_4dct(n_phases=n_phases)
    rng = np.random.default_rng(17)
    shape = ph.hu.shape[1:]
    doses = rng.gamma(2.0, 0.5, size=(n_phases,) + shape).astype(np.float32)
    rho = np.stack([orc.density(ph, p) for p in range(n_phases)]).astype(np.float32)
    return ph, dvf, doses, rho


@pytest.mark.parametrize("case", ["identity", "dvf", "dvf_mask", "ref2"])
def test_emtm_parity(gpu, orc, case):
    ph, dvf, doses, rho = _emtm_inputs(orc)
    nsub = (2, 2, 5)
    ref = 2 if case == "ref2" else 0
    use_dvf = None if case == "identity" else dvf
    mask = None
    if case == "dvf_mask":
        mask = (np.random.default_rng(1).random(doses.shape[1:]) > 0.3).astype(np.uint8)
    ctx = H.make_ctx(gpu, ph)
    try:
        grho = gpu.dose_read(ctx, gpu.DOSE_DENSITY, 1, np.zeros(doses.shape[1:], np.float32))
        np.testing.assert_array_equal(grho, rho[1])
        for p in range(doses.shape[0]):
            gpu.dose_set_phase_dose(ctx, p, np.ascontiguousarray(doses[p]))
        gpu.dose_accumulate_subvoxel(ctx, ref, nsub, dvf=use_dvf, mask=mask)
        acc = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros(doses.shape[1:], np.float32))
        stats = gpu.dose_read(ctx, gpu.DOSE_EMTM_STATS, 0, np.zeros(4, np.uint64))
    finally:
        gpu.dose_destroy(ctx)
    want, dropped, B = orc.emtm(doses, rho, ph.d, ref, nsub, dvf=use_dvf, mask=mask, bounds=True)
    tied = H.check_emtm(acc, want, B)
    nvox = doses[0].size
    assert int(stats[0]) == (doses.shape[0] - 1) * nvox * 20
    assert B["dropped_min"] <= int(stats[1]) <= B["dropped_max"]
    # subvoxels on a cell face are rare: a few per ten thousand pushed
    assert B["ambiguous"] <= 1e-3 * int(stats[0]), B["ambiguous"]
    print(f"{case}: {B['ambiguous']} of {int(stats[0])} subvoxels within the tie tolerance, {tied} voxels affected")
    if case == "identity":
        np.testing.assert_allclose(acc, doses.astype(np.float64).sum(axis=0), rtol=2e-6)


@pytest.mark.parametrize("case", ["blob", "corner", "empty_phase", "far_field", "identity"])
def test_emtm_sparse_dose_reach(gpu, orc, case):
    """Doses with compact support, as a Monte Carlo gives them: the kernel
    pushes only the source voxels within reach of dose (the header's reach
    box), and the accumulated dose is still the oracle's push of every
    voxel; the pushed count is the reach boxes' volume times the subvoxels."""
    ph, dvf, doses, rho = _emtm_inputs(orc)
    P = doses.shape[0]
    keep = np.zeros(doses.shape, bool)                       # (phase, z, y, x)
    if case == "corner":
        keep[:, :3, -4:, :2] = True
    elif case == "empty_phase":
        keep[:, 15:22, 30:40, 5:12] = True
        keep[2] = False
    else:
        keep[:, 10:20, 20:35, 25:40] = True
    doses = np.where(keep, doses, np.float32(0.0)).astype(np.float32)
    field = None if case == "identity" else (dvf * np.float32(12.0) if case == "far_field" else dvf)
    nsub = (2, 2, 5)
    ctx = H.make_ctx(gpu, ph)
    try:
        for p in range(P):
            gpu.dose_set_phase_dose(ctx, p, np.ascontiguousarray(doses[p]))
        gpu.dose_accumulate_subvoxel(ctx, 0, nsub, dvf=field)
        acc = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros(doses.shape[1:], np.float32))
        stats = gpu.dose_read(ctx, gpu.DOSE_EMTM_STATS, 0, np.zeros(4, np.uint64))
    finally:
        gpu.dose_destroy(ctx)
    want, dropped, B = orc.emtm(doses, rho, ph.d, 0, nsub, dvf=field, bounds=True)
    H.check_emtm(acc, want, B)
    assert acc.max() > 0 and int(stats[1]) <= B["dropped_max"]
    boxes = [H.reach_box((rho[p] > 0) & (doses[p] > 0), None if field is None else field[p], ph.d, 2)
             for p in range(1, P)]
    assert int(stats[0]) == 20 * sum(H.box_voxels(b) for b in boxes)
    nvox = doses[0].size
    if case == "far_field":                                 # motion past the grid: the whole z axis
        assert all(b[2] == (0, doses.shape[1] - 1) for b in boxes)
    else:
        assert int(stats[0]) < (P - 1) * nvox * 20 // 2
    if case == "empty_phase":
        assert boxes[1] is None


def test_emtm_after_a_dense_accumulation(gpu, orc):
    """E and M are cleared only where a pushed subvoxel can land: a sparse
    accumulation after a dense one on the same context (stale sums
    everywhere) still equals the oracle, and so does the dense one again."""
    ph, dvf, dense, rho = _emtm_inputs(orc)
    keep = np.zeros(dense.shape, bool)
    keep[:, 12:18, 25:33, 30:38] = True
    sparse = np.where(keep, dense, np.float32(0.0)).astype(np.float32)
    ctx = H.make_ctx(gpu, ph)
    got = []
    try:
        for doses in (dense, sparse, dense):
            for p in range(doses.shape[0]):
                gpu.dose_set_phase_dose(ctx, p, np.ascontiguousarray(doses[p]))
            gpu.dose_accumulate_subvoxel(ctx, 0, (2, 2, 5), dvf=dvf)
            got.append(gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros(dense.shape[1:], np.float32)))
    finally:
        gpu.dose_destroy(ctx)
    for acc, doses in zip(got, (dense, sparse, dense)):
        want, _, B = orc.emtm(doses, rho, ph.d, 0, (2, 2, 5), dvf=dvf, bounds=True)
        H.check_emtm(acc, want, B)
    np.testing.assert_array_equal(got[0], got[2])


def test_autotune_keeps_results(gpu):
    """The autotuner only picks a launch shape: tallies are bit-identical."""
    ph = W.slab_phantom(n=48)
    pl = W.slab_plan(n_layers=3, nx=3, ny=2)
    ref = H.gpu_run(gpu, ph, pl, 300_000, 4)["tally"]
    ctx = H.make_ctx(gpu, ph)
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(pl), None)
        regs, block, chunk, us = gpu.dose_autotune(ctx, 0, 300_000, 100_000, 4)
        assert regs in (0, 1) and block in (128, 256, 512, 1024) and chunk in (32, 64, 128, 256) and us > 0
        t = H.gpu_run(gpu, ph, pl, 300_000, 4, ctx=ctx)["tally"]
    finally:
        gpu.dose_destroy(ctx)
    np.testing.assert_array_equal(t, ref)


def test_autotune_batch_keeps_results(gpu):
    """The batch autotuner times a sample of a ragged batch (two grids, two
    seeds: the job-table kernel) and only picks its launch shape: the
    batch's tallies are bit-identical before and after tuning, and every
    context of the batch gets the picked shape."""
    ph, pl = W.slab_phantom(n=48), W.slab_plan(n_layers=3, nx=3, ny=2)
    ph2, pl2 = W.water_phantom(32, 32, 60), W.pencil_plan(120.0, 3.0)
    ctxs = [H.make_ctx(gpu, ph), H.make_ctx(gpu, ph2)]
    try:
        gpu.dose_add_spots(ctxs[0], gpu.spots_array(pl), None)
        gpu.dose_add_spots(ctxs[1], gpu.spots_array(pl2), None)
        jobs = gpu.make_jobs([dict(ctx=ctxs[0], phase=0, n_histories=200_000, seed=3),
                              dict(ctx=ctxs[1], phase=0, n_histories=100_000, seed=4)])

        def tallies():
            gpu.dose_run_batch(jobs)
            return [gpu.dose_read(c, gpu.DOSE_TALLY_I64, 0, np.zeros(p.hu.shape, np.uint64))
                    for c, p in zip(ctxs, (ph, ph2))]

        ref = tallies()
        regs, block, chunk, us = gpu.dose_autotune_batch(jobs, 60_000)
        assert regs in (0, 1) and block in (128, 256, 512, 1024) and chunk in (32, 64, 128, 256) and us > 0
        for c in ctxs:
            assert gpu.dose_get_option(c, gpu.DOSE_OPT_BLOCK) == block
            assert gpu.dose_get_option(c, gpu.DOSE_OPT_CHUNK) == chunk
        got = tallies()
    finally:
        for c in ctxs:
            gpu.dose_destroy(c)
    for a, b in zip(ref, got):
        assert a.sum() > 0
        np.testing.assert_array_equal(a, b)


def test_material_grid_gives_the_same_tallies(gpu):
    """The per-voxel (density, SPR) grid holds the table's values, so the
    transport's results do not depend on DOSE_OPT_MATERIAL_GRID (checked on
    phase 2 of a 4DCT so the phase offset of the grid is exercised)."""
    ph, _, geo = H.small_4dct(n_phases=3, nx=40, ny=40, nz=24)
    plan = W.tumour_plan(geo, ph.origin, n_layers=3, per_layer=10, e_lo=70.0, e_hi=100.0)
    dlv = H.whole_plan_on(2, 3)
    out = []
    for mat in (0, 1):
        ctx = H.make_ctx(gpu, ph)
        try:
            gpu.dose_set_option(ctx, gpu.DOSE_OPT_MATERIAL_GRID, mat)
            gpu.dose_add_spots(ctx, gpu.spots_array(plan), gpu.delivery_struct(dlv))
            gpu.dose_run_phase(ctx, 2, 200_000, 6)
            out.append(gpu.dose_read(ctx, gpu.DOSE_TALLY_I64, 2, np.zeros(ph.hu.shape[1:], np.uint64)))
        finally:
            gpu.dose_destroy(ctx)
    assert out[0].sum() > 0
    np.testing.assert_array_equal(out[0], out[1])


def test_normalisation_matches_fp64_division(gpu):
    """D_i = tally_i x (W/N) x 1.602176634e-10 / (2^24 V) / rho_i in FP64,
    rounded once to FP32: the device's Newton-Raphson quotient gives the
    correctly rounded FP64 division's float in every voxel (at most 1 ulp
    off, and only in a vanishing fraction)."""
    ph = W.slab_phantom(n=64)
    pl = W.slab_plan(n_layers=4, nx=3, ny=2)
    r = H.gpu_run(gpu, ph, pl, 400_000, 12)
    ctx = H.make_ctx(gpu, ph)
    try:
        rho = gpu.dose_read(ctx, gpu.DOSE_DENSITY, 0, np.zeros(ph.hu.shape, np.float32))
    finally:
        gpu.dose_destroy(ctx)
    W_, N = int(r["ledger"][7]), int(r["ledger"][5])
    v = float(np.float32(ph.d[0])) * float(np.float32(ph.d[1])) * float(np.float32(ph.d[2])) / 1000.0
    factor = W_ / N * 1.602176634e-10 / (16777216.0 * v)
    want = (r["tally"].astype(np.float64) * factor / rho.astype(np.float64)).astype(np.float32)
    got = r["dose"]
    ulp = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1
    assert (ulp > 0).mean() <= 1e-4
    assert np.count_nonzero(want) > 1000
