"""Pins of the oracle's delivery extensions (Sec. 2.B, App. A): synchrotron
fills with charge and extraction-time limits, gate holds, capped
isolayered repainting, irregular breathing and the uncertainty-trial
sampler.  Hand-worked examples (tests/golden/synchrotron_hand_examples.json),
the reduction of the synchrotron model to the simple clock when nothing
limits it, an independent re-implementation of the breathing clock for a
long spill, conservation invariants and the moments of the deviates."""
import json
import os

import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _plan(protons, layer, field=None):
    n = len(protons)
    return W.Plan(np.zeros(n), np.zeros(n), np.full(n, 100.0), np.zeros(n), np.array(protons, np.uint64),
                  np.array(layer, np.int32), np.zeros(n, np.int32) if field is None else np.array(field, np.int32))


def _cases():
    g = json.load(open(os.path.join(GOLDEN, "synchrotron_hand_examples.json")))
    return [(c["name"], c) for c in g["cases"]]


@pytest.mark.parametrize("name,case", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_hand_examples(orc, name, case):
    plan = _plan(case["plan"]["protons"], case["plan"]["layer"])
    dlv = W.Delivery(**case["delivery"])
    pp, fe, sp = orc.timeline(plan, dlv)
    want = np.zeros_like(pp)
    for s, d in case["expect"].items():
        for ph, v in d.items():
            want[int(ph), int(s)] = v
    np.testing.assert_array_equal(pp, want)
    assert int(fe[0]) == case["end_ns"]


def _random_plan(rng, n_fields=2, n_layers=4, per_layer=7):
    prot, lay, fld = [], [], []
    for f in range(n_fields):
        for l in range(n_layers):
            for _ in range(per_layer):
                prot.append(int(rng.integers(1, 4_000_000)))
                lay.append(l)
                fld.append(f)
    return _plan(prot, lay, fld)


@pytest.mark.parametrize("sigma,cap,repaints", [(0, 0, 1), (0, 0, 3), (300_000_000, 0, 1), (0, 1_000_000, 1),
                                                (500_000_000, 700_000, 1)])
def test_unlimited_synchrotron_is_the_simple_clock(orc, sigma, cap, repaints):
    """Without charge or time limits, discard or gating, every layer takes
    one fill whose reset is the layer switch: the two clocks agree."""
    rng = np.random.default_rng(7 + repaints)
    plan = _random_plan(rng)
    base = dict(n_phases=10, start_phase=-1, seed=11, period_ns=4_000_000_000, period_sigma_ns=sigma,
                spot_switch_ns=2_000_000, layer_switch_ns=1_000_000_000, max_protons_per_paint=cap,
                repaints=repaints)
    a = orc.timeline(plan, W.Delivery(**base))
    b = orc.timeline(plan, W.Delivery(**base, synchrotron=1))
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_breathing_deviate_is_irwin_hall_of_the_cycle_blocks(orc):
    """2^21 Z_c is the sum of the twelve 21-bit fields of Philox blocks
    (f, c, 1, 0) and (f, c, 2, 0) under the seed, minus 6 (2^21 - 1)."""
    seed = 0x1234_5678_9ABC_DEF0
    for f, c in [(0, 0), (1, 5), (3, 1000)]:
        k = 0
        for blk in (1, 2):
            w = orc.philox4x32_10([f, c, blk, 0], [seed & 0xFFFFFFFF, seed >> 32])
            v = int(w[0]) | (int(w[1]) << 32) | (int(w[2]) << 64) | (int(w[3]) << 96)
            k += sum((v >> (21 * i)) & 0x1FFFFF for i in range(6))
        assert orc.breathing_deviate(seed, f, c) == k - 6 * 0x1FFFFF


def test_breathing_deviate_moments_and_bounds(orc):
    z = np.array([orc.breathing_deviate(99, 0, c) for c in range(20000)], np.float64) / 2.0 ** 21
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1.0) < 0.04
    assert np.abs(z).max() <= 6.0
    # the Irwin-Hall sum has kurtosis 3 - 1.2 / 12 = 2.9
    kurt = ((z - z.mean()) ** 4).mean() / z.var() ** 2
    assert abs(kurt - 2.9) < 0.1


def test_irregular_breathing_clock_by_hand(orc):
    """One long spill under sigma > 0, re-derived here: cycle c lasts N t_c
    with t_c = max(N, mu + round(sigma Z_c)) // N; the clock starts at the
    beginning of phase p0 of cycle 0; protons go by time share."""
    N, mu, sigma, p0, seed = 4, 4000, 600, 2, 5
    w = 1_000_003                                    # ns at 1e9 protons/s
    plan = _plan([w], [0])
    pp, fe, _ = orc.timeline(plan, W.Delivery(n_phases=N, start_phase=p0, period_ns=mu, period_sigma_ns=sigma,
                                              seed=seed, rate_protons_per_s=1_000_000_000))
    segs, t, c = [], 0, 0
    while t < w:
        zk = orc.breathing_deviate(seed, 0, c)
        T = max(N, mu + ((sigma * zk + (1 << 20)) >> 21))
        tc = T // N
        for j in range(p0 if c == 0 else 0, N):
            e = min(t + tc, w)
            if e > t:
                segs.append((j, e - t))
            t = e
        c += 1
    want = np.zeros(N, np.int64)
    given = 0
    for i, (j, d) in enumerate(segs):
        pj = w - given if i == len(segs) - 1 else (w * d) // w
        want[j] += pj
        given += pj
    np.testing.assert_array_equal(pp[:, 0].astype(np.int64), want)
    assert int(fe[0]) == w
    assert len({d for _, d in segs[:-1]}) > 3        # the phase length really varies


@pytest.mark.parametrize("kw", [
    dict(synchrotron=1, fill_protons=3_000_000),
    dict(synchrotron=1, extraction_limit_ns=5_000_000, discard_ns=70_000_000),
    dict(synchrotron=1, gated=1, gate_first=3, gate_last=7, discard_ns=70_000_000, fill_protons=20_000_000,
         extraction_limit_ns=8_000_000_000, period_sigma_ns=400_000_000),
    dict(gated=1, gate_first=4, gate_last=6, discard_ns=70_000_000, max_protons_per_paint=500_000,
         period_sigma_ns=300_000_000),
])
def test_conservation_and_gating(orc, kw):
    rng = np.random.default_rng(3)
    plan = _random_plan(rng)
    dlv = W.Delivery(n_phases=10, start_phase=-1, seed=4, period_ns=4_000_000_000, **kw)
    pp, fe, sp = orc.timeline(plan, dlv)
    np.testing.assert_array_equal(pp.sum(axis=0), plan.protons)
    if dlv.gated:
        off = [p for p in range(10) if not (dlv.gate_first <= p <= dlv.gate_last)]
        assert pp[off].sum() == 0
    # a field takes at least its spill time plus its layer switches
    for f in range(2):
        sel = plan.field == f
        assert int(fe[f]) >= int(plan.protons[sel].sum()) + 3 * dlv.layer_switch_ns


def test_limits_take_more_fills_and_time(orc):
    rng = np.random.default_rng(9)
    plan = _random_plan(rng)
    base = dict(n_phases=10, start_phase=0, period_ns=4_000_000_000, synchrotron=1, discard_ns=70_000_000)
    _, free, _ = orc.timeline(plan, W.Delivery(**base))
    _, charged, _ = orc.timeline(plan, W.Delivery(**base, fill_protons=2_000_000))
    _, timed, _ = orc.timeline(plan, W.Delivery(**base, extraction_limit_ns=3_000_000))
    assert np.all(charged > free) and np.all(timed > free)


def test_rejects_deliveries_that_cannot_progress(orc):
    plan = _plan([1000], [0])
    base = dict(n_phases=10, start_phase=0, period_ns=4_000_000_000, synchrotron=1)
    for bad in (dict(extraction_limit_ns=1, rate_protons_per_s=1000),          # limit below one proton
                dict(gated=1, gate_first=2, gate_last=2, discard_ns=399_999_999, rate_protons_per_s=1000),
                dict(max_protons_per_paint=10, repaints=2),
                dict(period_sigma_ns=700_000_000)):                              # mu - 6 sigma < N
        with pytest.raises(ValueError):
            orc.timeline(plan, W.Delivery(**dict(base, **bad)))


def test_trial_sampler(orc):
    """Periods from the discrete uniform set {3, ..., 7} s; Gaussian
    synchrotron parameters with the requested moments, clamped at 0; the
    trial seed advances by the 64-bit golden ratio."""
    mean = W.Delivery(seed=77, spot_switch_ns=2_000_000, layer_switch_ns=2_000_000_000, discard_ns=70_000_000,
                      rate_protons_per_s=1_000_000_000, fill_protons=12_500_000_000,
                      extraction_limit_ns=8_000_000_000, synchrotron=1)
    spread = W.DeliverySpread(period_min_ns=3_000_000_000, period_max_ns=7_000_000_000,
                              period_step_ns=1_000_000_000, spot_switch_sigma_ns=200_000,
                              layer_switch_sigma_ns=100_000_000, discard_sigma_ns=50_000_000,
                              rate_sigma=50_000_000, fill_protons_sigma=1_000_000_000,
                              extraction_limit_sigma_ns=500_000_000)
    n = 4000
    tr = [orc.trial_delivery(mean, spread, k) for k in range(n)]
    per = np.array([t["period_ns"] for t in tr])
    vals, counts = np.unique(per, return_counts=True)
    np.testing.assert_array_equal(vals, np.arange(3, 8) * 1_000_000_000)
    assert np.all(np.abs(counts / n - 0.2) < 0.03)
    for name, mu, sd in (("spot_switch_ns", 2e6, 2e5), ("layer_switch_ns", 2e9, 1e8),
                         ("rate_protons_per_s", 1e9, 5e7), ("fill_protons", 12.5e9, 1e9),
                         ("extraction_limit_ns", 8e9, 5e8)):
        x = np.array([t[name] for t in tr], np.float64)
        assert abs(x.mean() - mu) < 4 * sd / np.sqrt(n), name
        assert abs(x.std() / sd - 1.0) < 0.05, name
    disc = np.array([t["discard_ns"] for t in tr])
    assert disc.min() >= 0                     # 70 ms +- 50 ms is clamped at 0
    assert all(t["seed"] == (77 + k * 0x9E3779B97F4A7C15) % 2 ** 64 for k, t in enumerate(tr[:50]))
    # no spread: the mean delivery comes back (but for its trial seed)
    same = orc.trial_delivery(mean, W.DeliverySpread(), 5)
    assert same["period_ns"] == mean.period_ns and same["fill_protons"] == mean.fill_protons
