"""Helpers shared by the GPU tests: run the CUDA engine through the C-ABI
binding, run the CPU oracle in batches, and compare doses (per-voxel
sigma test, fraction of Dmax, global gamma index)."""
from __future__ import annotations

import numpy as np

from paper_1809_03927_gb300 import workloads as W


# ------------------------------------------------------------------ engine
def make_ctx(D, phantom):
    hu = np.ascontiguousarray(phantom.hu, np.int16)
    nx, ny, nz = phantom.n
    ctx = D.dose_create_grid(nx, ny, nz, *phantom.d, phantom.origin, phantom.n_phases, hu,
                             phantom.beam_dir)
    return ctx


def gpu_run(D, phantom, plan, n_hist, seed, phase=0, physics=7, spr_scale=1.0,
            shift=(0.0, 0.0, 0.0), delivery=None, ctx=None, options=None):
    """Dose, tally and ledger of one phase; the context is destroyed unless
    one was passed in."""
    own = ctx is None
    if own:
        ctx = make_ctx(D, phantom)
    try:
        D.dose_set_option(ctx, D.DOSE_OPT_PHYSICS, physics)
        for k, v in (options or {}).items():
            D.dose_set_option(ctx, k, v)
        D.dose_add_spots(ctx, D.spots_array(plan),
                         D.delivery_struct(delivery) if delivery is not None else None)
        D.dose_run_phase(ctx, phase, n_hist, seed, spr_scale, shift)
        shape = phantom.hu.shape[-3:]
        dose = D.dose_read(ctx, D.DOSE_PHASE_DOSE, phase, np.zeros(shape, np.float32))
        tally = D.dose_read(ctx, D.DOSE_TALLY_I64, phase, np.zeros(shape, np.uint64))
        led = D.dose_read(ctx, D.DOSE_ENERGY_LEDGER, phase, np.zeros(8, np.uint64))
        st = np.zeros(1, np.int32)
        D.dose_read(ctx, D.DOSE_STATUS, phase, st)
        return dict(dose=dose, tally=tally, ledger=led, status=int(st[0]))
    finally:
        if own:
            D.dose_destroy(ctx)


def whole_plan_on(phase, n_phases):
    """Delivery that puts the whole plan on one phase: start there with a
    breathing period far longer than the delivery."""
    return W.Delivery(n_phases=n_phases, start_phase=phase, period_ns=n_phases * 10 ** 15)


def gpu_batches(D, phantom, plan, n_hist, seed, n_batches, phase=0, physics=7, **kw):
    """GPU estimate of an n_hist-history dose of the whole plan on `phase`
    as the mean of n_batches independent runs (seed + 7919 b, n_hist /
    n_batches histories each); returns (mean dose, its standard error)."""
    ctx = make_ctx(D, phantom)
    try:
        D.dose_set_option(ctx, D.DOSE_OPT_PHYSICS, physics)
        dl = None if phase == 0 else D.delivery_struct(whole_plan_on(phase, phantom.n_phases))
        D.dose_add_spots(ctx, D.spots_array(plan), dl)
        shape = phantom.hu.shape[-3:]
        nb = n_hist // n_batches
        doses = []
        for b in range(n_batches):
            D.dose_run_phase(ctx, phase, nb, seed + 7919 * b, kw.get("spr_scale", 1.0),
                             kw.get("shift", (0.0, 0.0, 0.0)))
            doses.append(D.dose_read(ctx, D.DOSE_PHASE_DOSE, phase, np.zeros(shape, np.float32)))
    finally:
        D.dose_destroy(ctx)
    doses = np.stack(doses).astype(np.float64)
    return doses.mean(axis=0), doses.std(axis=0, ddof=1) / np.sqrt(n_batches)


def gpu_batches_on_device(D, phantom, plan, n_hist, seed, n_batches, phase=0):
    """As gpu_batches, with the batch doses summed on the device (a large
    grid's 100 doses are not copied to the host): mean dose and its
    standard error, float64 on the host."""
    import torch
    ctx = make_ctx(D, phantom)
    shape = phantom.hu.shape[-3:]
    try:
        dl = None if phase == 0 else D.delivery_struct(whole_plan_on(phase, phantom.n_phases))
        D.dose_add_spots(ctx, D.spots_array(plan), dl)
        nb = n_hist // n_batches
        d = torch.empty(shape, dtype=torch.float32, device="cuda")
        s1 = torch.zeros(shape, dtype=torch.float64, device="cuda")
        s2 = torch.zeros(shape, dtype=torch.float64, device="cuda")
        for b in range(n_batches):
            D.dose_run_phase(ctx, phase, nb, seed + 7919 * b)
            D.dose_read(ctx, D.DOSE_PHASE_DOSE, phase, d)
            x = d.double()
            s1 += x
            s2 += x * x
        torch.cuda.synchronize()
    finally:
        D.dose_destroy(ctx)
    mean = (s1 / n_batches).cpu().numpy()
    var = np.maximum((s2 / n_batches).cpu().numpy() - mean * mean, 0.0) * n_batches / (n_batches - 1)
    return mean, np.sqrt(var / n_batches)


def body_mask(orc, phantom, phase=None, rho_min=0.1):
    """Voxels inside the patient (density above air); dose outside the
    external contour is not evaluated (Sec. 2.A: the MC is limited to it)."""
    return orc.density(phantom, phase) >= rho_min


# ------------------------------------------------------------------ oracle
def oracle_batches(orc, phantom, plan, n_hist, seed, n_batches=1, phase=None, **kw):
    """Oracle dose of an n_hist run as the mean over n_batches interleaved
    batches (batch b = histories h with h mod n_batches == b, so every batch
    samples every spot); returns (mean dose, standard error of the mean)."""
    rho = orc.density(phantom, phase)
    w_bar = float(np.sum(plan.protons.astype(np.float64))) / float(n_hist)
    v = phantom.d[0] * phantom.d[1] * phantom.d[2] / 1000.0
    doses, counts = [], []
    for b in range(n_batches):
        r = orc.transport(phantom, plan, n_hist, seed, phase=phase, batch=(b, n_batches), **kw)
        frac = r["histories"] / n_hist
        counts.append(r["histories"])
        doses.append(orc.normalise(r["edep"], rho, w_bar, v) / frac)
    doses = np.stack(doses)
    mean = np.average(doses, axis=0, weights=counts)
    if n_batches > 1:
        sem = doses.std(axis=0, ddof=1) / np.sqrt(n_batches)
    else:
        sem = np.zeros_like(mean)
    return mean, sem


# ----------------------------------------------------------------- compare
def sigma_pass(dg, do, sem_comb, dmax, threshold=0.1, k=3.0):
    sel = do >= threshold * dmax
    ok = np.abs(dg - do)[sel] <= k * sem_comb[sel]
    return float(np.mean(ok)), int(sel.sum())


def dmax_pass(dg, do, dmax, threshold=0.1, frac=0.01):
    sel = do >= threshold * dmax
    return float(np.mean(np.abs(dg - do)[sel] <= frac * dmax))


def _trilinear(a, k, j, i):
    nz, ny, nx = a.shape
    k0 = np.floor(k).astype(int); j0 = np.floor(j).astype(int); i0 = np.floor(i).astype(int)
    fk, fj, fi = k - k0, j - j0, i - i0
    def at(kk, jj, ii):
        return a[np.clip(kk, 0, nz - 1), np.clip(jj, 0, ny - 1), np.clip(ii, 0, nx - 1)]
    out = 0.0
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                w = (fk if dk else 1 - fk) * (fj if dj else 1 - fj) * (fi if di else 1 - fi)
                out = out + w * at(k0 + dk, j0 + dj, i0 + di)
    return out


def gamma_pass(ref, evl, spacing, dd=0.01, dta=1.0, threshold=0.1, step=0.25, dmax=None, select=None):
    """Global gamma index (Low, Harms, Mutic, Purdy, Med. Phys. 25, 1998):
    for each reference voxel with dose >= threshold * max, gamma^2 is the
    minimum over evaluated points r' within dta of |r'-r|^2/dta^2 +
    (D_e(r') - D_r(r))^2/(dd * max)^2, the evaluated dose interpolated
    trilinearly between voxel centres on a `step`-mm sub-grid.  Returns the
    fraction of voxels with gamma <= 1.  ``dmax`` overrides the maximum
    (global normalisation); ``select`` restricts the reference voxels."""
    dmax = float(ref.max()) if dmax is None else float(dmax)
    sel = ref >= threshold * dmax
    if select is not None:
        sel &= select
    idx = np.argwhere(sel)
    dr = ref[tuple(idx.T)]
    r = np.arange(-dta, dta + 1e-9, step)
    best = np.full(len(idx), np.inf)
    for ox in r:
        for oy in r:
            for oz in r:
                d2 = ox * ox + oy * oy + oz * oz
                if d2 > dta * dta + 1e-12:
                    continue
                de = _trilinear(evl, idx[:, 0] + oz / spacing[2], idx[:, 1] + oy / spacing[1],
                                idx[:, 2] + ox / spacing[0])
                best = np.minimum(best, d2 / dta ** 2 + ((de - dr) / (dd * dmax)) ** 2)
    return float(np.mean(best <= 1.0))


def check_emtm(got, want, bounds, rtol=2e-6, atol=1e-9, where=None):
    """The device's energy/mass-transfer accumulation against the oracle's
    (Sec. 2.D.2, Eqs. 2, 4-6).  A subvoxel whose mapped point lies within the
    tie tolerance of a cell face may be decided either way by any
    finite-precision implementation; every other subvoxel must land where
    the oracle puts it.  So: where no such subvoxel can land (the oracle's
    bounds coincide) the doses agree within the tolerance of the fixed-point
    sums; elsewhere the device's dose lies within the oracle's bounds.
    ``where`` restricts the check to a boolean region.  Returns the number of
    voxels an ambiguous subvoxel can reach (to report)."""
    lo, hi = bounds["lo"], bounds["hi"]
    sel = np.ones(got.shape, bool) if where is None else where
    exact = (lo == hi) & sel
    np.testing.assert_allclose(got[exact], want[exact], rtol=rtol, atol=atol)
    tied = (lo != hi) & sel
    g = got[tied].astype(np.float64)
    ok = (g >= lo[tied] * (1 - rtol) - atol) & (g <= hi[tied] * (1 + rtol) + atol)
    assert ok.all(), (int((~ok).sum()), int(tied.sum()))
    return int(tied.sum())


def small_4dct(n_phases=4, nx=64, ny=64, nz=40, motion_pp=15.0):
    ph, dvf, geo = W.phantom_4dct(nx, ny, nz, (1.0, 1.0, 2.5), n_phases=n_phases, motion_pp=motion_pp)
    return ph, dvf, geo


def reach_box(carries, field, d, mult):
    """The voxel box an accumulation of one source phase visits, as the
    engine's header defines it: the (x, y, z) box of the voxels that carry
    dose grown by mult x (ceil(max|u| / d) + 2) per axis in FP32, clipped to
    the grid; None when no voxel carries dose.  carries is (nz, ny, nx)
    bool, field (3, nz, ny, nx) mm or None."""
    if not carries.any():
        return None
    n = carries.shape[::-1]
    box = []
    for ax in range(3):
        other = tuple(a for a in range(3) if a != 2 - ax)
        idx = np.nonzero(carries.any(axis=other))[0]
        v = np.float32(np.abs(field[ax]).max()) if field is not None else np.float32(0.0)
        dm = np.float32(v * (np.float32(1.0) / np.float32(d[ax])))
        r = int(np.ceil(dm)) + 2 if dm < n[ax] else n[ax]
        box.append((max(int(idx[0]) - mult * r, 0), min(int(idx[-1]) + mult * r, n[ax] - 1)))
    return box


def box_voxels(box):
    return 0 if box is None else int(np.prod([hi - lo + 1 for lo, hi in box]))
