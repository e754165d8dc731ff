"""The whole 4D dose (Sec. 2.A): delivery timeline -> per-phase Monte Carlo
-> energy/mass-transfer accumulation, through dose_run_4d, against the
oracle's pipeline (or_timeline -> or_transport per phase -> or_emtm)."""
import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

NSUB = (2, 2, 5)


def _case():
    ph, dvf, geo = W.phantom_4dct(48, 48, 32, (1.0, 1.0, 2.5), n_phases=4, motion_pp=8.0)
    plan = W.tumour_plan(geo, ph.origin, n_layers=3, per_layer=12, e_lo=70.0, e_hi=100.0)
    # a delivery that spreads the plan over all four phases
    dlv = W.Delivery(n_phases=4, start_phase=-1, seed=21, period_ns=20_000_000,
                     spot_switch_ns=200_000, layer_switch_ns=3_000_000)
    return ph, dvf, plan, dlv


def _gpu_4d(D, ph, dvf, plan, dlv, n, seed):
    ctx = H.make_ctx(D, ph)
    try:
        D.dose_add_spots(ctx, D.spots_array(plan), D.delivery_struct(dlv))
        D.dose_run_4d(ctx, n, seed, 0, NSUB, dvf=dvf)
        acc = D.dose_read(ctx, D.DOSE_ACCUM, 0, np.zeros(ph.hu.shape[1:], np.float32))
        doses = np.stack([D.dose_read(ctx, D.DOSE_PHASE_DOSE, p, np.zeros(ph.hu.shape[1:], np.float32))
                          for p in range(ph.n_phases)])
        pp = D.dose_read(ctx, D.DOSE_SUBPLAN, 0, np.zeros((ph.n_phases, len(plan)), np.uint64))
    finally:
        D.dose_destroy(ctx)
    return acc, doses, pp


def _oracle_4d(orc, ph, dvf, plan, dlv, n, seed):
    pp, _, _ = orc.timeline(plan, dlv)
    rho = np.stack([orc.density(ph, p) for p in range(ph.n_phases)]).astype(np.float32)
    doses = np.zeros((ph.n_phases,) + ph.hu.shape[1:], np.float32)
    for p in range(ph.n_phases):
        if pp[p].sum() == 0:
            continue
        doses[p] = orc.dose(ph, plan.with_protons(pp[p]), n, seed, stream=p, phase=p)["dose"]
    acc, _ = orc.emtm(doses, rho, ph.d, 0, NSUB, dvf=dvf)
    return acc


def test_4d_pipeline_parity(gpu, orc):
    ph, dvf, plan, dlv = _case()
    pp, _, _ = orc.timeline(plan, dlv)
    assert np.count_nonzero(pp.sum(axis=1)) == 4
    B, n = 64, 1_500
    g = np.stack([_gpu_4d(gpu, ph, dvf, plan, dlv, n, 1000 + b)[0] for b in range(B)]).astype(np.float64)
    o = np.stack([_oracle_4d(orc, ph, dvf, plan, dlv, n, 5000 + b) for b in range(B)])
    body = H.body_mask(orc, ph, 0)
    gm, gs = g.mean(axis=0), g.std(axis=0, ddof=1) / np.sqrt(B)
    om, os_ = o.mean(axis=0), o.std(axis=0, ddof=1) / np.sqrt(B)
    gm, om = np.where(body, gm, 0.0), np.where(body, om, 0.0)
    frac, nsel = H.sigma_pass(gm, om, np.sqrt(gs ** 2 + os_ ** 2), om.max())
    assert nsel > 500 and frac >= 0.995, frac


def test_4d_equals_phases_run_separately(gpu):
    """One launch over all phases gives the per-phase tallies of separate
    runs bit for bit, and the accumulation of those doses."""
    ph, dvf, plan, dlv = _case()
    n, seed = 50_000, 9
    acc, doses, pp = _gpu_4d(gpu, ph, dvf, plan, dlv, n, seed)
    ctx = H.make_ctx(gpu, ph)
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(plan), gpu.delivery_struct(dlv))
        sep = []
        for p in range(ph.n_phases):
            gpu.dose_run_phase(ctx, p, n, seed)
            sep.append(gpu.dose_read(ctx, gpu.DOSE_PHASE_DOSE, p, np.zeros(ph.hu.shape[1:], np.float32)))
        gpu.dose_accumulate_subvoxel(ctx, 0, NSUB, dvf=dvf)
        acc2 = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros(ph.hu.shape[1:], np.float32))
    finally:
        gpu.dose_destroy(ctx)
    np.testing.assert_array_equal(np.stack(sep), doses)
    np.testing.assert_array_equal(acc2, acc)


def test_4d_gated_skips_empty_phases(gpu, orc):
    ph, dvf, plan, _ = _case()
    dlv = W.Delivery(n_phases=4, start_phase=0, seed=1, period_ns=20_000_000, gated=1,
                     gate_first=1, gate_last=2, spot_switch_ns=200_000, layer_switch_ns=3_000_000)
    acc, doses, pp = _gpu_4d(gpu, ph, dvf, plan, dlv, 20_000, 3)
    opp, _, _ = orc.timeline(plan, dlv)
    np.testing.assert_array_equal(pp, opp)
    assert doses[0].max() == 0.0 and doses[3].max() == 0.0
    assert doses[1].max() > 0.0 and doses[2].max() > 0.0
    assert acc.max() > 0.0


def test_readme_example_runs(gpu):
    """The usage example of the README, as written."""
    import re
    readme = open(__import__("os").path.join(__import__("os").path.dirname(__file__), "..", "README.md")).read()
    code = re.search(r"```python\n(.*?)```", readme, re.S).group(1)
    scope = {}
    exec(compile(code, "README.md", "exec"), scope)
    assert scope["acc"].max() > 0


def test_emtm_full_size_properties(gpu, orc):
    """The EMTM on the 10-phase 256 x 256 x 160 4DCT with (2, 2, 5)
    subvoxels, properties that hold at any size: with no field the
    accumulation is the phase sum; with the breathing field, voxels whose
    whole neighbourhood stays still in every phase keep the phase sum, every
    subvoxel is pushed once, and the moving region changes the dose.  Then
    the oracle's EMTM on a crop through the right lung and the tumour, wider
    than the largest displacement (15 mm = 6 voxels, along z only): inside
    the crop's interior (8 voxels from its z faces, 1 from the others) every
    subvoxel that lands comes from the crop and sees the same field, so the
    full-size device result there is the oracle's."""
    import torch
    ph, dvf, geo = W.phantom_4dct()
    P = ph.n_phases
    nx, ny, nz = ph.n
    rng = np.random.default_rng(3)
    doses = rng.gamma(2.0, 0.5, size=(P, nz, ny, nx)).astype(np.float32)
    total = doses.astype(np.float64).sum(axis=0)
    ctx = H.make_ctx(gpu, ph)
    try:
        for p in range(P):
            gpu.dose_set_phase_dose(ctx, p, np.ascontiguousarray(doses[p]))
        gpu.dose_accumulate_subvoxel(ctx, 0, NSUB)
        ident = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros((nz, ny, nx), np.float32))
        gpu.dose_accumulate_subvoxel(ctx, 0, NSUB, dvf=torch.from_numpy(dvf).cuda())
        moved = gpu.dose_read(ctx, gpu.DOSE_ACCUM, 0, np.zeros((nz, ny, nx), np.float32))
        stats = gpu.dose_read(ctx, gpu.DOSE_EMTM_STATS, 0, np.zeros(4, np.uint64))
    finally:
        gpu.dose_destroy(ctx)
    np.testing.assert_allclose(ident, total, rtol=2e-6)
    still = np.abs(dvf).max(axis=(0, 1)) == 0.0
    # a voxel is safe when it and its 26 neighbours never move
    pad = np.pad(still, 1, constant_values=True)
    safe = np.ones_like(still)
    for dz in (0, 1, 2):
        for dy in (0, 1, 2):
            for dx in (0, 1, 2):
                safe &= pad[dz:dz + nz, dy:dy + ny, dx:dx + nx]
    assert safe.mean() > 0.5 and (~safe).sum() > 10_000
    np.testing.assert_allclose(moved[safe], total[safe], rtol=2e-6)
    assert not np.allclose(moved[~safe], total[~safe], rtol=1e-3)
    assert int(stats[0]) == (P - 1) * nx * ny * nz * 20
    assert np.abs(dvf[:, :2]).max() == 0.0 and np.abs(dvf).max() <= 15.0
    z0, z1, y0, y1, x0, x1 = 30, 130, 90, 150, 50, 100
    rho = np.stack([orc.density(ph, p)[z0:z1, y0:y1, x0:x1] for p in range(P)]).astype(np.float32)
    sub = np.ascontiguousarray(doses[:, z0:z1, y0:y1, x0:x1])
    field = np.ascontiguousarray(dvf[:, :, z0:z1, y0:y1, x0:x1])
    want, _, B = orc.emtm(sub, rho, ph.d, 0, NSUB, dvf=field, bounds=True)
    inner = np.zeros(want.shape, bool)
    inner[8:-8, 1:-1, 1:-1] = True
    crop = moved[z0:z1, y0:y1, x0:x1]
    H.check_emtm(crop, want, B, where=inner)
    assert not np.allclose(crop[inner], sub.astype(np.float64).sum(axis=0)[inner], rtol=1e-3)
