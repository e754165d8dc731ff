"""Continuous-batching server: requests that arrive while others run are
admitted at the next step and share launches; each result must be the same
bits as the request served alone (histories are keyed by seed, history and
phase, and slicing a run does not change its tally)."""
import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

NSUB = (2, 2, 5)


def _setup(D):
    import torch
    ph, dvf, geo = W.phantom_4dct(48, 48, 32, (1.0, 1.0, 2.5), n_phases=4, motion_pp=8.0)
    plan = W.tumour_plan(geo, ph.origin, n_layers=3, per_layer=12, e_lo=70.0, e_hi=100.0)
    dlv = D.delivery_struct(W.Delivery(n_phases=4, start_phase=-1, seed=21, period_ns=20_000_000,
                                       spot_switch_ns=200_000, layer_switch_ns=3_000_000))
    base = H.make_ctx(D, ph)
    return ph, torch.from_numpy(dvf).cuda(), D.spots_array(plan), dlv, base


REQUESTS = [  # (histories, seed, spr scale, shift)
    (40_000, 1, 1.0, (0.0, 0.0, 0.0)),
    (8_000, 2, 1.035, (0.0, 0.0, 0.0)),
    (120_000, 3, 1.0, (3.0, 0.0, 0.0)),
    (4_000, 4, 0.965, (0.0, -3.0, 0.0)),
    (60_000, 5, 1.0, (0.0, 0.0, 3.0)),
]


def _serve(D, base, spots, dlv, dvf, arrivals, shape, **kw):
    """Serve REQUESTS; request k is submitted before step arrivals[k]."""
    srv = D.dose_server_create(base, 1 << 34, kw.get("step", 30_000), spots, dlv, min_slice=kw.get("min_slice", 50),
                               max_active=kw.get("max_active", 0), nsub=NSUB, dvf=dvf,
                               policy=kw.get("policy", D.DOSE_SERVE_FAIR), max_wait_steps=kw.get("max_wait", 0))
    out, ids, done_step, step, pending = {}, {}, {}, 0, list(range(len(REQUESTS)))
    try:
        while len(out) < len(REQUESTS):
            for k in list(pending):
                if arrivals[k] <= step:
                    n, seed, spr, sh = REQUESTS[k]
                    ids[D.dose_server_submit(srv, n, seed, spr, sh)] = k
                    pending.remove(k)
            for rid in D.dose_server_step(srv):
                acc = D.dose_server_result(srv, rid, D.DOSE_ACCUM, 0, np.zeros(shape, np.float32))
                ph2 = D.dose_server_result(srv, rid, D.DOSE_PHASE_DOSE, 2, np.zeros(shape, np.float32))
                out[ids[rid]] = (acc, ph2)
                done_step[ids[rid]] = step
                D.dose_server_release(srv, rid)
            step += 1
            assert step < 10_000
        stats = D.dose_server_stats(srv)
        stats["done_step"] = done_step
    finally:
        D.dose_server_destroy(srv)
    return out, stats


@pytest.mark.parametrize("policy", ["fair", "shortest_first"])
def test_served_results_equal_alone(gpu, policy):
    """Under either sharing policy (equal shares, or the step's budget to
    the requests with the fewest histories left) the slices differ but the
    results are the bits of each request alone."""
    D = gpu
    ph, dvf, spots, dlv, base = _setup(D)
    shape = ph.hu.shape[1:]
    pol = D.DOSE_SERVE_FAIR if policy == "fair" else D.DOSE_SERVE_SHORTEST_FIRST
    try:
        mixed, stats = _serve(D, base, spots, dlv, dvf, [0, 1, 1, 3, 6], shape, policy=pol)
        assert stats["completed"] == len(REQUESTS) and stats["queued"] == 0 and stats["active"] == 0
        assert stats["steps"] > 3 and stats["slots"] >= 2
        # each request alone: dose_run_4d with the server's even split over the phases
        view = D.dose_create_view(base)
        try:
            D.dose_add_spots(view, spots, dlv)
            for k, (n, seed, spr, sh) in enumerate(REQUESTS):
                D.dose_run_4d(view, n // 4, seed, 0, NSUB, dvf=dvf, spr_scale=spr, shift_mm=sh)
                acc = D.dose_read(view, D.DOSE_ACCUM, 0, np.zeros(shape, np.float32))
                ph2 = D.dose_read(view, D.DOSE_PHASE_DOSE, 2, np.zeros(shape, np.float32))
                np.testing.assert_array_equal(mixed[k][0], acc)
                np.testing.assert_array_equal(mixed[k][1], ph2)
        finally:
            D.dose_destroy(view)
    finally:
        D.dose_destroy(base)


def test_shortest_first_finishes_small_requests_first(gpu):
    """All requests submitted together: with the budget going to the fewest
    histories left, requests complete in order of size and the two smallest
    in the first step, while the whole batch takes no more steps than equal
    shares (the same histories go through each step)."""
    D = gpu
    ph, dvf, spots, dlv, base = _setup(D)
    shape = ph.hu.shape[1:]
    try:
        _, fair = _serve(D, base, spots, dlv, dvf, [0] * len(REQUESTS), shape, policy=D.DOSE_SERVE_FAIR)
        _, srpt = _serve(D, base, spots, dlv, dvf, [0] * len(REQUESTS), shape,
                         policy=D.DOSE_SERVE_SHORTEST_FIRST)
        by_size = sorted(range(len(REQUESTS)), key=lambda k: REQUESTS[k][0])
        steps = [srpt["done_step"][k] for k in by_size]
        assert steps == sorted(steps)
        assert srpt["done_step"][by_size[0]] == 0 and srpt["done_step"][by_size[1]] == 0
        assert max(srpt["done_step"].values()) <= max(fair["done_step"].values())
        for k in by_size[:-1]:
            assert srpt["done_step"][k] <= fair["done_step"][k]
    finally:
        D.dose_destroy(base)


def _completion_steps(sizes, nph, step, min_slice, bound):
    """Completion step of each request (all submitted before step 0) under
    shortest-first with a wait bound, from the policy's definition: requests
    that have waited `bound` steps first, then fewest histories left (ties
    in submission order); each takes min(left per phase, max(min_slice,
    budget // nph)) per phase while budget remains, an overdue one at least
    min(left, min_slice) after it is spent."""
    per = [n // nph for n in sizes]
    nxt, waited, done, st = [0] * len(sizes), [0] * len(sizes), {}, 0
    while len(done) < len(sizes):
        act = [i for i in range(len(sizes)) if i not in done]
        over = {i: bound > 0 and waited[i] >= bound for i in act}
        order = sorted(act, key=lambda i: (0 if over[i] else 1, (per[i] - nxt[i]) * nph))
        budget, take = step, {}
        for i in order:
            if budget == 0 and not over[i]:
                take[i] = 0
                continue
            take[i] = min(per[i] - nxt[i], max(min_slice, budget // nph))
            budget = max(0, budget - take[i] * nph)
        for i in act:
            waited[i] = waited[i] + 1 if take[i] == 0 else 0
            nxt[i] += take[i]
            if nxt[i] == per[i]:
                done[i] = st
        st += 1
    return done


def test_shortest_first_wait_bound(gpu):
    """With max_wait_steps the largest request is not held back until the
    others finish: the completion steps follow the policy's definition for
    the bound (computed here from it) and differ from those without one."""
    D = gpu
    ph, dvf, spots, dlv, base = _setup(D)
    shape = ph.hu.shape[1:]
    sizes = [r[0] for r in REQUESTS]
    try:
        got = {}
        for bound in (0, 1):
            _, st = _serve(D, base, spots, dlv, dvf, [0] * len(REQUESTS), shape,
                           policy=D.DOSE_SERVE_SHORTEST_FIRST, max_wait=bound)
            nph = [k for k in range(1, 5) if sum(n // k * k for n in sizes) == st["histories"]]
            assert len(nph) >= 1
            want = _completion_steps(sizes, nph[0], 30_000, 50, bound)
            assert st["done_step"] == want, (bound, st["done_step"], want)
            got[bound] = st["done_step"]
        assert got[0] != got[1]
        with pytest.raises(D.DoseError):
            D.dose_server_create(base, 1 << 34, 30_000, spots, dlv, dvf=dvf,
                                 policy=D.DOSE_SERVE_SHORTEST_FIRST, max_wait_steps=-1)
    finally:
        D.dose_destroy(base)


def test_served_two_field_plan_equals_alone(gpu):
    """A second field entering along +x (dose_set_field_beam on the base
    before the server is created): slots copy the template's plan with its
    field beams, and each request equals the same request computed alone on
    a view of the base."""
    D = gpu
    ph, dvf, spots0, dlv, base = _setup(D)
    shape = ph.hu.shape[1:]
    geo = W.phantom_4dct(48, 48, 32, (1.0, 1.0, 2.5), n_phases=4, motion_pp=8.0, with_dvf=False)[2]
    plan = W.tumour_plan(geo, ph.origin, n_layers=3, per_layer=12, e_lo=70.0, e_hi=100.0)
    two = W.Plan(np.concatenate([plan.x, plan.x]), np.concatenate([plan.y, plan.y]),
                 np.concatenate([plan.energy, plan.energy]), np.concatenate([plan.sigma, plan.sigma]),
                 np.concatenate([plan.protons, plan.protons]), np.concatenate([plan.layer, plan.layer]),
                 np.concatenate([np.zeros(len(plan), np.int32), np.ones(len(plan), np.int32)]))
    spots = D.spots_array(two)
    reqs = [(30_000, 7, 1.0, (0.0, 0.0, 0.0)), (20_000, 8, 1.035, (2.0, 0.0, 0.0))]
    try:
        D.dose_set_field_beam(base, 1, (1.0, 0.0, 0.0))
        srv = D.dose_server_create(base, 1 << 34, 20_000, spots, dlv, min_slice=50, nsub=NSUB, dvf=dvf)
        out, ids = {}, {}
        try:
            for k, (n, seed, spr, sh) in enumerate(reqs):
                ids[D.dose_server_submit(srv, n, seed, spr, sh)] = k
            steps = 0
            while len(out) < len(reqs):
                for rid in D.dose_server_step(srv):
                    out[ids[rid]] = D.dose_server_result(srv, rid, D.DOSE_ACCUM, 0, np.zeros(shape, np.float32))
                    D.dose_server_release(srv, rid)
                steps += 1
                assert steps < 10_000
        finally:
            D.dose_server_destroy(srv)
        view = D.dose_create_view(base)
        try:
            D.dose_add_spots(view, spots, dlv)
            pp = D.dose_read(view, D.DOSE_SUBPLAN, 0, np.zeros((4, len(two)), np.uint64)).sum(axis=1)
            reached = int(np.count_nonzero(pp))
            for k, (n, seed, spr, sh) in enumerate(reqs):
                D.dose_run_4d(view, n // reached, seed, 0, NSUB, dvf=dvf, spr_scale=spr, shift_mm=sh)
                alone = D.dose_read(view, D.DOSE_ACCUM, 0, np.zeros(shape, np.float32))
                np.testing.assert_array_equal(out[k], alone)
                assert alone.max() > 0
        finally:
            D.dose_destroy(view)
    finally:
        D.dose_destroy(base)


def test_slot_cap_and_reuse(gpu):
    """With one slot, requests run one at a time and reuse it; results are
    unchanged."""
    D = gpu
    ph, dvf, spots, dlv, base = _setup(D)
    shape = ph.hu.shape[1:]
    try:
        capped, stats = _serve(D, base, spots, dlv, dvf, [0] * len(REQUESTS), shape, max_active=1)
        assert stats["slots"] == 1
        free, _ = _serve(D, base, spots, dlv, dvf, [0] * len(REQUESTS), shape, step=1_000_000)
        for k in range(len(REQUESTS)):
            np.testing.assert_array_equal(capped[k][0], free[k][0])
    finally:
        D.dose_destroy(base)


def test_server_rejects_bad_input(gpu):
    D = gpu
    ph, dvf, spots, dlv, base = _setup(D)
    try:
        with pytest.raises(D.DoseError):
            D.dose_server_create(base, 1000, 30_000, spots, dlv, dvf=dvf)       # budget below one slot
        with pytest.raises(D.DoseError):
            D.dose_server_create(base, 1 << 34, 30_000, spots, dlv, dvf=dvf, policy=2)   # no such policy
        srv = D.dose_server_create(base, 1 << 34, 30_000, spots, dlv, dvf=dvf)
        try:
            with pytest.raises(D.DoseError):
                D.dose_server_submit(srv, 0, 1)
            with pytest.raises(D.DoseError):
                D.dose_server_result(srv, 12345, D.DOSE_ACCUM, 0, np.zeros(ph.hu.shape[1:], np.float32))
        finally:
            D.dose_server_destroy(srv)
    finally:
        D.dose_destroy(base)


@pytest.mark.parametrize("policy", ["fair", "shortest_first"])
def test_requests_with_their_own_delivery(gpu, policy):
    """Gating and repainting variants served next to nominal requests: each
    request's result equals that request computed alone with its delivery
    (the even split over the phases its delivery reaches)."""
    D = gpu
    ph, dvf, spots, dlv, base = _setup(D)
    shape = ph.hu.shape[1:]
    common = dict(n_phases=4, start_phase=-1, seed=21, period_ns=20_000_000, spot_switch_ns=200_000,
                  layer_switch_ns=3_000_000)
    gated = D.delivery_struct(W.Delivery(**dict(common, gated=1, gate_first=1, gate_last=2, start_phase=0)))
    repaint = D.delivery_struct(W.Delivery(**dict(common, max_protons_per_paint=300_000)))
    late = D.delivery_struct(W.Delivery(**dict(common, gated=1, gate_first=3, gate_last=3, start_phase=0)))
    reqs = [(30_000, 11, None), (20_000, 12, gated), (24_000, 13, repaint), (10_000, 14, None),
            (16_000, 15, gated), (8_000, 16, late)]
    srv = D.dose_server_create(base, 1 << 34, 25_000, spots, dlv, min_slice=50, max_active=3, nsub=NSUB, dvf=dvf,
                               policy=D.DOSE_SERVE_FAIR if policy == "fair" else D.DOSE_SERVE_SHORTEST_FIRST)
    out, ids = {}, {}
    try:
        for k, (n, seed, d) in enumerate(reqs):
            ids[D.dose_server_submit(srv, n, seed, delivery=d)] = k
        steps = 0
        while len(out) < len(reqs):
            for rid in D.dose_server_step(srv):
                out[ids[rid]] = D.dose_server_result(srv, rid, D.DOSE_ACCUM, 0, np.zeros(shape, np.float32))
                D.dose_server_release(srv, rid)
            steps += 1
            assert steps < 10_000
    finally:
        D.dose_server_destroy(srv)
    view = D.dose_create_view(base)
    try:
        for k, (n, seed, d) in enumerate(reqs):
            D.dose_add_spots(view, spots, d if d is not None else dlv)
            pp = D.dose_read(view, D.DOSE_SUBPLAN, 0, np.zeros((4, len(spots)), np.uint64)).sum(axis=1)
            reached = int(np.count_nonzero(pp))
            D.dose_run_4d(view, max(1, n // reached), seed, 0, NSUB, dvf=dvf)
            alone = D.dose_read(view, D.DOSE_ACCUM, 0, np.zeros(shape, np.float32))
            np.testing.assert_array_equal(out[k], alone)
            assert alone.max() > 0
    finally:
        D.dose_destroy(view)
        D.dose_destroy(base)
