"""Python access to the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may
import this package.  The CUDA product path never imports it; the two share
no code.  ``build()`` compiles ``oracle.c`` with gcc (plus OpenMP when
available) into ``liboracle.so`` next to this file.

Each wrapper names the paper passage its C function follows; see the header
of ``oracle.c`` for the model and for what pins each function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

PHYS_STRAGGLING, PHYS_MCS, PHYS_NUCLEAR = 1, 2, 4
PHYS_ALL = 7
OK, EINVAL, ENOMEM, ESTEP = 0, -1, -2, -5


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` -> ``liboracle.so`` (no-op if up to date)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class RunParams(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 3), ("d", C.c_double * 3), ("origin", C.c_double * 3),
        ("hu", C.c_void_p), ("beam_axis", C.c_int32), ("beam_sign", C.c_int32),
        ("n_spots", C.c_int64), ("spot_x", C.c_void_p), ("spot_y", C.c_void_p),
        ("spot_e", C.c_void_p), ("spot_sigma", C.c_void_p), ("spot_protons", C.c_void_p),
        ("n_hist", C.c_uint64), ("hist_begin", C.c_uint64), ("hist_end", C.c_uint64),
        ("seed", C.c_uint64), ("stream", C.c_uint32), ("physics", C.c_uint32),
        ("spr_scale", C.c_double), ("shift", C.c_double * 3), ("max_steps", C.c_int64),
        ("nthreads", C.c_int32), ("n_depth_bins", C.c_int32), ("depth_bin_mm", C.c_double),
        ("n_planes", C.c_int32), ("plane_mm", C.c_double),
        ("batch_count", C.c_uint64), ("batch_index", C.c_uint64),
    ]


class RunOut(C.Structure):
    _fields_ = [
        ("edep", C.c_void_p), ("depth_dose", C.c_void_p), ("plane_w", C.c_void_p),
        ("plane_m1", C.c_void_p), ("plane_m2", C.c_void_p), ("ledger", C.c_double * 4),
        ("steps", C.c_uint64), ("histories", C.c_uint64), ("status", C.c_int32),
        ("end_depth", C.c_double * 3),
    ]


class DeliveryC(C.Structure):
    _fields_ = [
        ("n_phases", C.c_int32), ("start_phase", C.c_int32), ("gated", C.c_int32),
        ("gate_first", C.c_int32), ("gate_last", C.c_int32), ("repaints", C.c_int32),
        ("period_ns", C.c_int64), ("period_sigma_ns", C.c_int64), ("spot_switch_ns", C.c_int64),
        ("layer_switch_ns", C.c_int64), ("discard_ns", C.c_int64),
        ("rate_protons_per_s", C.c_uint64), ("seed", C.c_uint64),
        ("synchrotron", C.c_int32), ("reserved", C.c_int32), ("fill_protons", C.c_uint64),
        ("extraction_limit_ns", C.c_int64), ("max_protons_per_paint", C.c_uint64),
    ]


class SpreadC(C.Structure):
    _fields_ = [
        ("period_min_ns", C.c_int64), ("period_max_ns", C.c_int64), ("period_step_ns", C.c_int64),
        ("spot_switch_sigma_ns", C.c_int64), ("layer_switch_sigma_ns", C.c_int64),
        ("discard_sigma_ns", C.c_int64), ("rate_sigma", C.c_int64), ("fill_protons_sigma", C.c_int64),
        ("extraction_limit_sigma_ns", C.c_int64),
    ]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_block_uniforms.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, P]
        for name in ("or_rho", "or_spr"):
            getattr(L, name).argtypes = [C.c_int]
            getattr(L, name).restype = C.c_double
        for name in ("or_bethe_sw", "or_range", "or_energy_from_range", "or_sigma_nuc", "or_pv"):
            getattr(L, name).argtypes = [C.c_double]
            getattr(L, name).restype = C.c_double
        L.or_init_tables.argtypes = []
        L.or_highland_theta2.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_highland_theta2.restype = C.c_double
        L.or_bohr_var.argtypes = [C.c_double, C.c_double]
        L.or_bohr_var.restype = C.c_double
        L.or_allocate.argtypes = [C.c_int64, P, C.c_uint64, P]
        L.or_transport.argtypes = [C.POINTER(RunParams), C.POINTER(RunOut)]
        L.or_single_step.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_uint64,
                                     C.c_uint64, C.c_uint32, C.c_uint32, P]
        L.or_step_theta2.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
        L.or_step_theta2.restype = C.c_double
        L.or_step_tau.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_step_tau.restype = C.c_double
        L.or_frame.argtypes = [P, P, P]
        L.or_normalise.argtypes = [C.c_int64, P, P, C.c_double, C.c_double, P]
        L.or_timeline.argtypes = [C.c_int64, P, P, P, C.POINTER(DeliveryC), P, P, P, C.c_int32]
        L.or_trial_delivery.argtypes = [C.POINTER(DeliveryC), C.POINTER(SpreadC), C.c_uint64,
                                        C.POINTER(DeliveryC)]
        L.or_breathing_deviate.argtypes = [C.c_uint64, C.c_int32, C.c_uint64]
        L.or_breathing_deviate.restype = C.c_int64
        L.or_emtm.argtypes = [P, P, C.c_int32, C.c_int32, P, P, P, P, P, C.c_double, P, P, P, P, P, P]
        L.or_dim.argtypes = [P, P, C.c_int32, C.c_int32, P, P, P, P, P]
        L.or_dvf_decode.argtypes = [P] * 11 + [C.c_double] + [P] * 3
        L.or_init_tables()
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------- random
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11); cuRAND's generator in Sec. 2.B."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def block_uniforms(seed, h, stream, block):
    out = np.zeros(6, dtype=np.float64)
    lib().or_block_uniforms(seed, h, stream, block, _ptr(out))
    return out


# ---------------------------------------------------------------- physics
def rho(hu):
    return lib().or_rho(int(hu))


def spr(hu):
    return lib().or_spr(int(hu))


def bethe_sw(e):
    """Water mass stopping power, MeV cm^2/g."""
    return lib().or_bethe_sw(float(e))


def range_mm(e):
    """CSDA range in water, mm."""
    return lib().or_range(float(e))


def energy_from_range(r_mm):
    return lib().or_energy_from_range(float(r_mm))


def sigma_nuc(e):
    return lib().or_sigma_nuc(float(e))


def pv(e):
    return lib().or_pv(float(e))


def highland_theta2(e, u0, du):
    return lib().or_highland_theta2(float(e), float(u0), float(du))


def bohr_var(e, sw_mm):
    return lib().or_bohr_var(float(e), float(sw_mm))


def step_theta2(hu, e, u0, s):
    """Highland theta0^2 of one step of the transport (step-mean energy)."""
    return lib().or_step_theta2(int(hu), float(e), float(u0), float(s))


def step_tau(hu, e, s):
    """Nuclear optical depth of one step of the transport (step-mean energy)."""
    return lib().or_step_tau(int(hu), float(e), float(s))


def frame(d):
    """Transverse orthonormal pair (e1, e2) used to scatter direction d."""
    d = np.ascontiguousarray(d, np.float64)
    e1 = np.zeros(3); e2 = np.zeros(3)
    lib().or_frame(_ptr(d), _ptr(e1), _ptr(e2))
    return e1, e2


def single_step(hu, e, u0, s, seed, h, stream=0, step=0):
    out = np.zeros(6, dtype=np.float64)
    lib().or_single_step(int(hu), float(e), float(u0), float(s), seed, h, stream, step, _ptr(out))
    return out


# ---------------------------------------------------------------- plan
def allocate(protons, n_hist):
    """Histories per spot: floor + largest remainder (ties -> lower index)."""
    p = np.ascontiguousarray(protons, dtype=np.uint64)
    out = np.zeros(p.shape[0], dtype=np.uint64)
    rc = lib().or_allocate(p.shape[0], _ptr(p), int(n_hist), _ptr(out))
    if rc:
        raise ValueError(f"or_allocate failed: {rc}")
    return out


def transport(phantom, plan, n_hist, seed, stream=0, phase=None, hist_range=None,
              physics=PHYS_ALL, spr_scale=1.0, shift=(0.0, 0.0, 0.0), max_steps=20_000,
              nthreads=None, depth_bin_mm=0.0, n_depth_bins=0, plane_mm=0.0, n_planes=0,
              batch=None):
    """Run histories ``hist_range`` (default all) of an ``n_hist``-history run;
    ``batch=(b, B)`` keeps only the histories h with h mod B == b.

    Returns a dict: ``edep`` (nz, ny, nx) MeV x history weight, ``ledger``
    (deposited, escaped, removed, incident), ``steps``, ``status`` and, if
    requested, ``depth_dose``, ``plane_w``, ``plane_m1``, ``plane_m2``.
    """
    hu = phantom.hu if phase is None else phantom.hu[phase]
    hu = np.ascontiguousarray(hu, dtype=np.int16)
    nz, ny, nx = hu.shape
    sx = np.ascontiguousarray(plan.x, np.float64)
    sy = np.ascontiguousarray(plan.y, np.float64)
    se = np.ascontiguousarray(plan.energy, np.float64)
    ss = np.ascontiguousarray(plan.sigma, np.float64)
    sp = np.ascontiguousarray(plan.protons, np.uint64)
    h0, h1 = (0, n_hist) if hist_range is None else hist_range
    P = RunParams()
    P.n[:] = (nx, ny, nz)
    P.d[:] = tuple(float(v) for v in phantom.d)
    P.origin[:] = tuple(float(v) for v in phantom.origin)
    P.hu = hu.ctypes.data
    P.beam_axis, P.beam_sign = phantom.beam_axis, phantom.beam_sign
    P.n_spots = len(plan)
    P.spot_x, P.spot_y, P.spot_e, P.spot_sigma, P.spot_protons = (
        sx.ctypes.data, sy.ctypes.data, se.ctypes.data, ss.ctypes.data, sp.ctypes.data)
    P.n_hist, P.hist_begin, P.hist_end = int(n_hist), int(h0), int(h1)
    P.seed, P.stream, P.physics = int(seed), int(stream), int(physics)
    P.spr_scale = float(spr_scale)
    P.shift[:] = tuple(float(v) for v in shift)
    P.max_steps = int(max_steps)
    P.nthreads = int(nthreads or os.cpu_count() or 1)
    P.n_depth_bins, P.depth_bin_mm = int(n_depth_bins), float(depth_bin_mm)
    P.n_planes, P.plane_mm = int(n_planes), float(plane_mm)
    if batch is not None:
        P.batch_index, P.batch_count = int(batch[0]), int(batch[1])
    edep = np.zeros((nz, ny, nx), dtype=np.float64)
    dd = np.zeros(n_depth_bins, np.float64) if n_depth_bins else None
    pw = np.zeros(n_planes, np.float64) if n_planes else None
    pm1 = np.zeros(2 * n_planes, np.float64) if n_planes else None
    pm2 = np.zeros(2 * n_planes, np.float64) if n_planes else None
    O = RunOut()
    O.edep, O.depth_dose, O.plane_w, O.plane_m1, O.plane_m2 = (
        edep.ctypes.data, _ptr(dd), _ptr(pw), _ptr(pm1), _ptr(pm2))
    rc = lib().or_transport(C.byref(P), C.byref(O))
    if rc not in (OK, ESTEP):
        raise ValueError(f"or_transport failed: {rc}")
    out = dict(edep=edep, ledger=np.array(O.ledger[:]), steps=int(O.steps),
               histories=int(O.histories), status=int(O.status),
               end_depth=(O.end_depth[0] / O.end_depth[1]) if O.end_depth[1] > 0 else float("nan"),
               end_depth_sd=(np.sqrt(max(O.end_depth[2] / O.end_depth[1]
                                         - (O.end_depth[0] / O.end_depth[1]) ** 2, 0.0))
                             if O.end_depth[1] > 0 else float("nan")),
               end_weight=float(O.end_depth[1]))
    if dd is not None:
        out["depth_dose"] = dd
    if pw is not None:
        out.update(plane_w=pw, plane_m1=pm1.reshape(2, n_planes), plane_m2=pm2.reshape(2, n_planes))
    return out


def density(phantom, phase=None):
    """FP64 mass density of every voxel (Sec. 2.C)."""
    hu = phantom.hu if phase is None else phantom.hu[phase]
    uniq = np.unique(hu)
    table = {int(v): rho(int(v)) for v in uniq}
    out = np.empty(hu.shape, dtype=np.float64)
    for v, r in table.items():
        out[hu == v] = r
    return out


def normalise(edep, rho_arr, w_bar, voxel_cm3):
    e = np.ascontiguousarray(edep, np.float64).ravel()
    r = np.ascontiguousarray(rho_arr, np.float64).ravel()
    out = np.zeros_like(e)
    lib().or_normalise(e.shape[0], _ptr(e), _ptr(r), float(w_bar), float(voxel_cm3), _ptr(out))
    return out.reshape(np.shape(edep))


def dose(phantom, plan, n_hist, seed, stream=0, phase=None, **kw):
    """Dose [Gy] of a run: transport then normalisation with W/N protons per history."""
    r = transport(phantom, plan, n_hist, seed, stream=stream, phase=phase, **kw)
    w_bar = float(np.sum(plan.protons.astype(np.float64))) / float(n_hist)
    v = phantom.d[0] * phantom.d[1] * phantom.d[2] / 1000.0
    r["dose"] = normalise(r["edep"], density(phantom, phase), w_bar, v)
    return r


def timeline(plan, delivery, n_fields=None):
    """Per-phase protons of every spot (Sec. 2.B, App. A).

    Returns ``(pp, field_end_ns, start_phase)`` with ``pp`` of shape
    ``(n_phases, n_spots)`` uint64.
    """
    n = len(plan)
    if n_fields is None:
        n_fields = int(np.max(plan.field)) + 1
    D = _delivery_c(delivery)
    p = np.ascontiguousarray(plan.protons, np.uint64)
    la = np.ascontiguousarray(plan.layer, np.int32)
    fi = np.ascontiguousarray(plan.field, np.int32)
    pp = np.zeros((delivery.n_phases, n), dtype=np.uint64)
    fe = np.zeros(n_fields, dtype=np.int64)
    sp = np.zeros(n_fields, dtype=np.int32)
    rc = lib().or_timeline(n, _ptr(p), _ptr(la), _ptr(fi), C.byref(D), _ptr(pp), _ptr(fe),
                           _ptr(sp), n_fields)
    if rc:
        raise ValueError(f"or_timeline failed: {rc}")
    return pp, fe, sp


def _delivery_c(delivery):
    D = DeliveryC()
    for name, _ in DeliveryC._fields_:
        setattr(D, name, int(getattr(delivery, name, 0)))
    return D


def trial_delivery(mean, spread, trial):
    """Trial ``trial``'s delivery parameters (the uncertainty trials of Sec.
    2.B), drawn from ``mean`` and the ``spread`` (object with the SpreadC
    field names).  Returns a dict of the sampled delivery's fields."""
    S = SpreadC()
    for name, _ in SpreadC._fields_:
        setattr(S, name, int(getattr(spread, name, 0)))
    out = DeliveryC()
    rc = lib().or_trial_delivery(C.byref(_delivery_c(mean)), C.byref(S), int(trial), C.byref(out))
    if rc:
        raise ValueError(f"or_trial_delivery failed: {rc}")
    return {name: getattr(out, name) for name, _ in DeliveryC._fields_}


def breathing_deviate(seed, field, cycle):
    """2^21 times the Irwin-Hall deviate of breathing cycle ``cycle``."""
    return int(lib().or_breathing_deviate(int(seed), int(field), int(cycle)))


# Tie tolerance of the accumulation's and the decode's integer decisions, in
# cell / grid-index units: a single-precision implementation on grids of up
# to a few hundred voxels per axis rounds the mapped coordinate by less than
# about 3e-5 (a few units in the last place at 256).
TIE_EPS = 1e-4


def emtm(dose_phases, rho_phases, d, ref_phase, nsub, dvf=None, mask=None, return_sums=False,
         bounds=False, eps=TIE_EPS):
    """Energy/mass-transfer accumulation onto ``ref_phase`` plus Eq. 2 sum
    (Sec. 2.D.2, Eqs. 2, 4-6), in FP64.

    ``dose_phases``/``rho_phases``: float32 (P, nz, ny, nx); ``dvf`` float32
    (P, 3, nz, ny, nx) mm (None = identity); ``mask`` uint8 (nz, ny, nx).
    Returns the FP64 accumulated dose (and the per-voxel E, M sums in units
    of the subvoxel volume when ``return_sums``) and the dropped count.
    With ``bounds`` a dict follows: ``lo``/``hi`` bound the accumulated dose
    of any decision of the subvoxels within ``eps`` of a cell face,
    ``dropped_min``/``dropped_max`` the dropped count, ``ambiguous`` counts
    those subvoxels.
    """
    ds = np.ascontiguousarray(dose_phases, np.float32)
    rs = np.ascontiguousarray(rho_phases, np.float32)
    P_, nz, ny, nx = ds.shape
    n = np.array([nx, ny, nz], np.int32)
    dm = np.array(d, np.float32)
    ns = np.array(nsub, np.int32)
    dv = None if dvf is None else np.ascontiguousarray(dvf, np.float32)
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    acc = np.zeros((nz, ny, nx), np.float64)
    es = np.zeros((nz, ny, nx), np.float64) if return_sums else None
    ms = np.zeros((nz, ny, nx), np.float64) if return_sums else None
    lo = np.zeros((nz, ny, nx), np.float64) if bounds else None
    hi = np.zeros((nz, ny, nx), np.float64) if bounds else None
    counts = np.zeros(4, np.uint64)
    rc = lib().or_emtm(_ptr(n), _ptr(dm), P_, int(ref_phase), _ptr(ns), _ptr(ds), _ptr(rs),
                       _ptr(dv), _ptr(mk), float(eps), _ptr(acc), _ptr(es), _ptr(ms), _ptr(lo), _ptr(hi),
                       _ptr(counts))
    if rc:
        raise ValueError(f"or_emtm failed: {rc}")
    out = [acc] + ([es, ms] if return_sums else []) + [int(counts[0])]
    if bounds:
        out.append(dict(lo=lo, hi=hi, dropped_min=int(counts[1]), dropped_max=int(counts[2]),
                        ambiguous=int(counts[3])))
    return tuple(out)


def dim(dose_phases, d, ref_phase, nsub, dvf=None, mask=None):
    """Dose-interpolation accumulation (Eq. 3) onto ``ref_phase`` plus Eq. 2.

    ``dose_phases``: float32 (P, nz, ny, nx) Gy; ``dvf`` float32
    (P, 3, nz, ny, nx) mm, the displacement carrying a reference-phase point
    to phase p, given at the reference voxel centres (None = identity);
    ``mask`` uint8 (nz, ny, nx).  Returns the FP64 accumulated dose.
    """
    ds = np.ascontiguousarray(dose_phases, np.float32)
    P_, nz, ny, nx = ds.shape
    n = np.array([nx, ny, nz], np.int32)
    dm = np.array(d, np.float32)
    ns = np.array(nsub, np.int32)
    dv = None if dvf is None else np.ascontiguousarray(dvf, np.float32)
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    acc = np.zeros((nz, ny, nx), np.float64)
    rc = lib().or_dim(_ptr(n), _ptr(dm), P_, int(ref_phase), _ptr(ns), _ptr(ds), _ptr(dv), _ptr(mk),
                      _ptr(acc))
    if rc:
        raise ValueError(f"or_dim failed: {rc}")
    return acc


def dvf_decode(grid, delta, n, d, origin, eps=TIE_EPS, return_ambiguous=False):
    """Decode a registration's vector grid (App. B, Eqs. 7-8) onto a CT grid,
    in FP64.

    ``grid``: dict with ``n`` (N_X, N_Y, N_Z), ``start_mm`` (centre of grid
    voxel 0), ``spacing_mm``, ``row_cos`` (U), ``col_cos`` (V) and optional
    ``pre``/``post`` row-major 4x4 rigid transforms; ``delta`` float32
    (N_Z, N_Y, N_X, 3) mm; the CT grid is ``n`` = (nx, ny, nz) voxels of
    size ``d`` with corner ``origin``.  Returns the FP64 displacement
    (3, nz, ny, nx) in mm and the uint8 inside mask (nz, ny, nx), and with
    ``return_ambiguous`` the uint8 flags of the voxels whose grid index lies
    within ``eps`` of a hull face (either decision is then correct).
    """
    f32 = lambda v: np.ascontiguousarray(np.asarray(v, np.float32).ravel())
    eye = np.eye(4, dtype=np.float32)
    gn = np.array(grid["n"], np.int32)
    args = [gn, f32(grid["start_mm"]), f32(grid["spacing_mm"]), f32(grid["row_cos"]), f32(grid["col_cos"]),
            f32(grid.get("pre", eye)), f32(grid.get("post", eye))]
    dl = np.ascontiguousarray(delta, np.float32)
    assert dl.shape == (gn[2], gn[1], gn[0], 3), dl.shape
    nx, ny, nz = (int(v) for v in n)
    disp = np.zeros((3, nz, ny, nx), np.float64)
    inside = np.zeros((nz, ny, nx), np.uint8)
    amb = np.zeros((nz, ny, nx), np.uint8)
    args += [dl, np.array(n, np.int32), f32(d), f32(origin)]                # kept alive for the call
    ptrs = [_ptr(a) for a in args]
    rc = lib().or_dvf_decode(*ptrs, float(eps), _ptr(disp), _ptr(inside), _ptr(amb))
    if rc:
        raise ValueError(f"or_dvf_decode failed: {rc}")
    if return_ambiguous:
        return disp, inside, amb
    return disp, inside
