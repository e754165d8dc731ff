"""The delivery simulation's extensions on the GPU (Sec. 2.B, App. A):
synchrotron fills with charge and extraction-time limits, gate holds,
irregular breathing, capped repainting and the uncertainty trials, bit for
bit against the oracle's or_timeline / or_trial_delivery (all integer)."""
import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

S = 1_000_000_000        # ns per second

VARIANTS = {
    "synchrotron_charge": dict(start_phase=2, synchrotron=1, fill_protons=20_000_000, discard_ns=70_000_000,
                               layer_switch_ns=2 * S),
    "synchrotron_time": dict(start_phase=-1, seed=8, synchrotron=1, extraction_limit_ns=50_000_000,
                             discard_ns=70_000_000),
    "synchrotron_gated": dict(start_phase=-1, seed=12, synchrotron=1, gated=1, gate_first=3, gate_last=7,
                              discard_ns=70_000_000, fill_protons=500_000_000, extraction_limit_ns=8 * S,
                              period_sigma_ns=400_000_000),
    "irregular": dict(start_phase=-1, seed=21, period_sigma_ns=500_000_000),
    "irregular_gated": dict(start_phase=4, gated=1, gate_first=4, gate_last=6, discard_ns=70_000_000,
                            period_sigma_ns=300_000_000),
    "capped": dict(start_phase=0, max_protons_per_paint=300_000, period_sigma_ns=200_000_000),
    "capped_synchrotron": dict(start_phase=-1, seed=3, synchrotron=1, max_protons_per_paint=400_000,
                               fill_protons=60_000_000, gated=1, gate_first=2, gate_last=6,
                               discard_ns=70_000_000),
    "two_fields": dict(start_phase=-1, seed=9, synchrotron=1, extraction_limit_ns=200_000_000,
                       period_sigma_ns=600_000_000),
}


def _grid(D, n_phases):
    ph = W.water_phantom(8, 8, 8)
    hu = np.repeat(ph.hu[None], n_phases, axis=0)
    return D.dose_create_grid(8, 8, 8, 2, 2, 2, ph.origin, n_phases, hu, (0, 0, 1))


def _read(D, ctx, plan, n_phases):
    pp = D.dose_read(ctx, D.DOSE_SUBPLAN, 0, np.zeros((n_phases, len(plan)), np.uint64))
    nf = int(np.max(plan.field)) + 1
    sp = D.dose_read(ctx, D.DOSE_START_PHASE, 0, np.zeros(nf, np.int32))
    fe = D.dose_read(ctx, D.DOSE_FIELD_END_NS, 0, np.zeros(nf, np.int64))
    return pp, fe, sp


def _plan(n_layers=20, per_layer=150, two_fields=False):
    ph, _, geo = H.small_4dct(n_phases=10)
    plan = W.tumour_plan(geo, ph.origin, n_layers=n_layers, per_layer=per_layer)
    if two_fields:
        f = np.zeros(len(plan), np.int32)
        f[len(plan) // 2:] = 1
        plan = W.Plan(plan.x, plan.y, plan.energy, plan.sigma, plan.protons, plan.layer, f)
    return plan


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_delivery_extensions_bit_exact(gpu, orc, variant):
    plan = _plan(two_fields=variant == "two_fields")
    dlv = W.Delivery(**VARIANTS[variant])
    ctx = _grid(gpu, 10)
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(plan), gpu.delivery_struct(dlv))
        pp, fe, sp = _read(gpu, ctx, plan, 10)
        used = gpu.read_delivery(ctx)
    finally:
        gpu.dose_destroy(ctx)
    opp, ofe, osp = orc.timeline(plan, dlv)
    np.testing.assert_array_equal(pp, opp)
    np.testing.assert_array_equal(fe, ofe)
    np.testing.assert_array_equal(sp, osp)
    np.testing.assert_array_equal(pp.sum(axis=0), plan.protons)
    assert all(used[k] == int(getattr(dlv, k)) for k in used)


def test_delivery_rejected_on_the_host(gpu):
    plan = _plan(n_layers=2, per_layer=10)
    ctx = _grid(gpu, 10)
    try:
        for bad in (dict(synchrotron=1, extraction_limit_ns=1, rate_protons_per_s=1000),
                    dict(max_protons_per_paint=10, repaints=2),
                    dict(period_sigma_ns=700_000_000)):
            with pytest.raises(gpu.DoseError):
                gpu.dose_add_spots(ctx, gpu.spots_array(plan), gpu.delivery_struct(W.Delivery(**bad)))
    finally:
        gpu.dose_destroy(ctx)


MEAN = dict(seed=77, spot_switch_ns=2_000_000, layer_switch_ns=2 * S, discard_ns=70_000_000,
            rate_protons_per_s=1_000_000_000, fill_protons=2_000_000_000, extraction_limit_ns=8 * S,
            synchrotron=1, start_phase=-1)
SPREAD = W.DeliverySpread(period_min_ns=3 * S, period_max_ns=7 * S, period_step_ns=S,
                          spot_switch_sigma_ns=200_000, layer_switch_sigma_ns=100_000_000,
                          discard_sigma_ns=10_000_000, rate_sigma=50_000_000, fill_protons_sigma=100_000_000,
                          extraction_limit_sigma_ns=500_000_000)


@pytest.mark.parametrize("gated", [0, 1])
def test_trials_bit_exact(gpu, orc, gated):
    """25 trials in one launch: each trial's sampled delivery and subplan
    equal the oracle's or_trial_delivery followed by or_timeline."""
    plan = _plan(n_layers=10, per_layer=60)
    mean = W.Delivery(**MEAN, gated=gated, gate_first=3, gate_last=7)
    base = _grid(gpu, 10)
    views = []
    try:
        views = [gpu.dose_create_view(base) for _ in range(25)]
        gpu.dose_add_spots_trials(views, gpu.spots_array(plan), gpu.delivery_struct(mean),
                                  gpu.spread_struct(SPREAD), first_trial=100)
        for k, v in enumerate(views):
            sampled = orc.trial_delivery(mean, SPREAD, 100 + k)
            used = gpu.read_delivery(v)
            assert used == sampled, k
            pp, fe, sp = _read(gpu, v, plan, 10)
            opp, ofe, osp = orc.timeline(plan, W.Delivery(**sampled))
            np.testing.assert_array_equal(pp, opp)
            np.testing.assert_array_equal(fe, ofe)
            np.testing.assert_array_equal(sp, osp)
        periods = {gpu.read_delivery(v)["period_ns"] for v in views}
        assert len(periods) >= 3 and periods <= {p * S for p in range(3, 8)}
    finally:
        for v in views:
            gpu.dose_destroy(v)
        gpu.dose_destroy(base)


def test_trial_that_cannot_progress_is_reported(gpu):
    """A discard spread wide enough to fill a gate window for some trial."""
    plan = _plan(n_layers=2, per_layer=10)
    mean = W.Delivery(**dict(MEAN, gated=1, gate_first=4, gate_last=4, discard_ns=300_000_000))
    spread = W.DeliverySpread(discard_sigma_ns=200_000_000)
    base = _grid(gpu, 10)
    views = []
    try:
        views = [gpu.dose_create_view(base) for _ in range(16)]
        with pytest.raises(gpu.DoseError, match="trial"):
            gpu.dose_add_spots_trials(views, gpu.spots_array(plan), gpu.delivery_struct(mean),
                                      gpu.spread_struct(spread))
    finally:
        for v in views:
            gpu.dose_destroy(v)
        gpu.dose_destroy(base)


def test_trials_transport_as_one_ragged_batch(gpu):
    """The trials' phase subplans transported in one persistent launch give
    each trial the tallies of its own phase-by-phase runs."""
    ph, _, geo = H.small_4dct(n_phases=4, nx=48, ny=48, nz=32)
    plan = W.tumour_plan(geo, ph.origin, n_layers=3, per_layer=12, e_lo=70.0, e_hi=100.0)
    mean = W.Delivery(**dict(MEAN, layer_switch_ns=50_000_000), n_phases=4)
    spread = W.DeliverySpread(period_min_ns=S // 10, period_max_ns=S // 5, period_step_ns=S // 20,
                              spot_switch_sigma_ns=100_000)
    base = H.make_ctx(gpu, ph)
    views = []
    n = 20_000
    try:
        views = [gpu.dose_create_view(base) for _ in range(5)]
        gpu.dose_add_spots_trials(views, gpu.spots_array(plan), gpu.delivery_struct(mean), gpu.spread_struct(spread))
        jobs = []
        for k, v in enumerate(views):
            pp = gpu.dose_read(v, gpu.DOSE_SUBPLAN, 0, np.zeros((4, len(plan)), np.uint64))
            for p in range(4):
                if pp[p].sum():
                    jobs.append(dict(ctx=v, phase=p, n_histories=n, seed=40 + k))
        assert len(jobs) > 5
        gpu.dose_run_batch(gpu.make_jobs(jobs))
        batched = [gpu.dose_read(j["ctx"], gpu.DOSE_TALLY_I64, j["phase"], np.zeros(ph.hu.shape[1:], np.uint64))
                   for j in jobs]
        for j, t in zip(jobs, batched):
            gpu.dose_run_phase(j["ctx"], j["phase"], n, j["seed"])
            alone = gpu.dose_read(j["ctx"], gpu.DOSE_TALLY_I64, j["phase"], np.zeros(ph.hu.shape[1:], np.uint64))
            np.testing.assert_array_equal(t, alone)
    finally:
        for v in views:
            gpu.dose_destroy(v)
        gpu.dose_destroy(base)
