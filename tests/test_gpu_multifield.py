"""Multi-field plans whose fields enter along different grid axes
(dose_set_field_beam): one launch transports every field's histories with
its own beam, bit for bit the sum of the fields' parts, and matches the
oracle run field by field over the same history ranges."""
import dataclasses

import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

# field -> (beam_dir, beam_axis, beam_sign); spots' (x_mm, y_mm) are on the
# field's lateral axes, lower axis first
FIELDS = {0: ((0.0, 0.0, 1.0), 2, 1), 1: ((-1.0, 0.0, 0.0), 0, -1), 2: ((0.0, 1.0, 0.0), 1, 1)}


def _setup():
    ph = W.water_phantom(nx=48, ny=48, nz=48, d=2.0)          # x, y in [-48, 48], z in [0, 96] mm
    xs, ys, es, fs = [], [], [], []
    for x, y, e in ((-5.0, 0.0, 100.0), (5.0, 0.0, 120.0)):            # field 0 (+z): (x, y)
        xs.append(x); ys.append(y); es.append(e); fs.append(0)
    for y, z, e in ((0.0, 40.0, 90.0), (0.0, 56.0, 110.0)):            # field 1 (-x): (y, z)
        xs.append(y); ys.append(z); es.append(e); fs.append(1)
    for x, z, e in ((-10.0, 48.0, 80.0), (10.0, 48.0, 100.0)):         # field 2 (+y): (x, z)
        xs.append(x); ys.append(z); es.append(e); fs.append(2)
    n = len(xs)
    plan = W.Plan(np.array(xs), np.array(ys), np.array(es), np.full(n, 3.0),
                  np.array([1_000_000, 1_300_000, 900_000, 1_100_000, 1_000_000, 1_200_000], np.uint64),
                  np.arange(n, dtype=np.int32) // 2, np.array(fs, np.int32))
    return ph, plan


def _ctx(gpu, ph, physics, beams):
    ctx = H.make_ctx(gpu, ph)
    gpu.dose_set_option(ctx, gpu.DOSE_OPT_PHYSICS, physics)
    for f, d in beams.items():
        gpu.dose_set_field_beam(ctx, f, d)
    return ctx


def _field_ranges(prefix, plan):
    out = {}
    for f in FIELDS:
        idx = np.nonzero(plan.field == f)[0]
        out[f] = (int(prefix[idx[0]]), int(prefix[idx[-1] + 1]))
    return out


def test_multifield_is_the_sum_of_its_field_parts(gpu):
    ph, plan = _setup()
    n, seed = 300_000, 3
    shape = ph.hu.shape
    ctx = _ctx(gpu, ph, 7, {f: v[0] for f, v in FIELDS.items()})
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(plan), None)
        gpu.dose_run_phase(ctx, 0, n, seed)
        whole = gpu.dose_read(ctx, gpu.DOSE_TALLY_I64, 0, np.zeros(shape, np.uint64))
        prefix = gpu.dose_read(ctx, gpu.DOSE_HIST_PREFIX, 0, np.zeros(len(plan) + 1, np.uint64))
    finally:
        gpu.dose_destroy(ctx)
    ranges = _field_ranges(prefix, plan)
    parts = np.zeros(shape, np.uint64)
    for f, (d, _, _) in FIELDS.items():
        # every field enters along field f's beam; only field f's histories run
        c = _ctx(gpu, ph, 7, {g: d for g in FIELDS})
        try:
            gpu.dose_add_spots(c, gpu.spots_array(plan), None)
            h0, h1 = ranges[f]
            gpu.dose_run_batch(gpu.make_jobs([dict(ctx=c, phase=0, n_histories=n, hist_begin=h0, hist_end=h1,
                                                   seed=seed)]))
            parts += gpu.dose_read(c, gpu.DOSE_TALLY_I64, 0, np.zeros(shape, np.uint64))
        finally:
            gpu.dose_destroy(c)
    np.testing.assert_array_equal(whole, parts)
    # the three beams really deposit along three axes
    for axis in range(3):
        prof = whole.sum(axis=tuple(a for a in range(3) if a != axis))
        assert np.count_nonzero(prof) > 20


def test_multifield_matched_streams_against_the_oracle(gpu, orc):
    """Without scattering the same seed gives the same histories on both
    sides; the oracle runs each field's history range with that field's
    beam and the doses add up."""
    ph, plan = _setup()
    n, seed, physics = 200_000, 5, 5
    ctx = _ctx(gpu, ph, physics, {f: v[0] for f, v in FIELDS.items()})
    try:
        gpu.dose_add_spots(ctx, gpu.spots_array(plan), None)
        gpu.dose_run_phase(ctx, 0, n, seed)
        dose = gpu.dose_read(ctx, gpu.DOSE_PHASE_DOSE, 0, np.zeros(ph.hu.shape, np.float32))
        prefix = gpu.dose_read(ctx, gpu.DOSE_HIST_PREFIX, 0, np.zeros(len(plan) + 1, np.uint64))
    finally:
        gpu.dose_destroy(ctx)
    alloc = orc.allocate(plan.protons, n)
    np.testing.assert_array_equal(np.diff(prefix.astype(np.int64)), alloc.astype(np.int64))
    edep = np.zeros(ph.hu.shape)
    for f, (_, axis, sign), in FIELDS.items():
        phf = dataclasses.replace(ph, beam_axis=axis, beam_sign=sign)
        edep += orc.transport(phf, plan, n, seed, hist_range=_field_ranges(prefix, plan)[f], physics=physics)["edep"]
    w_bar = float(plan.protons.astype(np.float64).sum()) / n
    want = orc.normalise(edep, orc.density(ph), w_bar, ph.d[0] * ph.d[1] * ph.d[2] / 1000.0)
    assert np.max(np.abs(dose - want)) <= 0.002 * want.max()


def test_field_beam_after_loading_and_in_views(gpu):
    ph, plan = _setup()
    n, seed = 100_000, 9
    a = _ctx(gpu, ph, 7, {f: v[0] for f, v in FIELDS.items()})
    b = _ctx(gpu, ph, 7, {})
    v = None
    try:
        gpu.dose_add_spots(a, gpu.spots_array(plan), None)
        gpu.dose_run_phase(a, 0, n, seed)
        ta = gpu.dose_read(a, gpu.DOSE_TALLY_I64, 0, np.zeros(ph.hu.shape, np.uint64))
        # set after the plan is loaded
        gpu.dose_add_spots(b, gpu.spots_array(plan), None)
        for f, d in FIELDS.items():
            gpu.dose_set_field_beam(b, f, d[0])
        gpu.dose_run_phase(b, 0, n, seed)
        np.testing.assert_array_equal(gpu.dose_read(b, gpu.DOSE_TALLY_I64, 0, np.zeros(ph.hu.shape, np.uint64)), ta)
        # a view starts with its base's beams
        v = gpu.dose_create_view(a)
        gpu.dose_add_spots(v, gpu.spots_array(plan), None)
        gpu.dose_run_phase(v, 0, n, seed)
        np.testing.assert_array_equal(gpu.dose_read(v, gpu.DOSE_TALLY_I64, 0, np.zeros(ph.hu.shape, np.uint64)), ta)
        # back to the grid's beam for every field: a different dose
        for f in FIELDS:
            gpu.dose_set_field_beam(b, f, None)
        gpu.dose_run_phase(b, 0, n, seed)
        assert not np.array_equal(gpu.dose_read(b, gpu.DOSE_TALLY_I64, 0, np.zeros(ph.hu.shape, np.uint64)), ta)
        with pytest.raises(gpu.DoseError):
            gpu.dose_set_field_beam(b, 0, (0.6, 0.8, 0.0))
        with pytest.raises(gpu.DoseError):
            gpu.dose_set_field_beam(b, 64, (1.0, 0.0, 0.0))
    finally:
        if v is not None:
            gpu.dose_destroy(v)
        gpu.dose_destroy(a)
        gpu.dose_destroy(b)
