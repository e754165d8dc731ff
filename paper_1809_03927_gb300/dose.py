"""Thin ctypes binding of ``libdose`` (``include/dose.h``).

Argument marshalling only: every function below has the name of the C entry
point it calls, converts arrays/tensors to pointers and raises ``DoseError``
on a negative status.  All computation happens in the CUDA kernels of the
library.  Importing this module fails loudly if ``libdose.so`` has not been
built (``python -m paper_1809_03927_gb300.build``); there is no fallback.

Arrays may be numpy arrays (host memory) or torch tensors (host or device);
the ``*_on_device`` flags of the C ABI are derived from them.  ``stream``
defaults to torch's current CUDA stream when torch has CUDA, else NULL.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libdose.so")

DOSE_OK, DOSE_EINVAL, DOSE_ENOMEM, DOSE_ECUDA, DOSE_ETIMEOUT, DOSE_ESTEPLIMIT, DOSE_ESTATE = \
    0, -1, -2, -3, -4, -5, -6
(DOSE_PHASE_DOSE, DOSE_DENSITY, DOSE_ACCUM, DOSE_TALLY_I64, DOSE_SUBPLAN, DOSE_ENERGY_LEDGER,
 DOSE_STATUS, DOSE_START_PHASE, DOSE_FIELD_END_NS, DOSE_EMTM_STATS, DOSE_HIST_PREFIX,
 DOSE_DELIVERY) = range(12)
DOSE_PHYS_STRAGGLING, DOSE_PHYS_MCS, DOSE_PHYS_NUCLEAR, DOSE_PHYS_ALL = 1, 2, 4, 7
(DOSE_OPT_PHYSICS, DOSE_OPT_MAX_STEPS, DOSE_OPT_BLOCK, DOSE_OPT_BLOCKS_PER_SM, DOSE_OPT_CHUNK,
 DOSE_OPT_TIMEOUT_MS, DOSE_OPT_FAIL_ALLOC_AFTER, DOSE_OPT_REGISTERS, DOSE_OPT_MATERIAL_GRID) = range(9)
DOSE_JOB_CLEAR, DOSE_JOB_FINISH = 1, 2
DOSE_SERVE_FAIR, DOSE_SERVE_SHORTEST_FIRST = 0, 1
LEDGER = ("deposited", "escaped", "removed", "incident", "steps", "histories", "flags", "protons")


class DoseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdose error {code}: {msg}")
        self.code = code


class dose_spot(C.Structure):
    _fields_ = [("x_mm", C.c_float), ("y_mm", C.c_float), ("energy_MeV", C.c_float),
                ("sigma_mm", C.c_float), ("protons", C.c_uint64), ("layer", C.c_int32),
                ("field", C.c_int32)]


class dose_delivery(C.Structure):
    _fields_ = [("n_phases", C.c_int32), ("start_phase", C.c_int32), ("gated", C.c_int32),
                ("gate_first", C.c_int32), ("gate_last", C.c_int32), ("repaints", C.c_int32),
                ("period_ns", C.c_int64), ("period_sigma_ns", C.c_int64),
                ("spot_switch_ns", C.c_int64), ("layer_switch_ns", C.c_int64),
                ("discard_ns", C.c_int64), ("rate_protons_per_s", C.c_uint64), ("seed", C.c_uint64),
                ("synchrotron", C.c_int32), ("reserved", C.c_int32), ("fill_protons", C.c_uint64),
                ("extraction_limit_ns", C.c_int64), ("max_protons_per_paint", C.c_uint64)]


class dose_delivery_spread(C.Structure):
    _fields_ = [("period_min_ns", C.c_int64), ("period_max_ns", C.c_int64), ("period_step_ns", C.c_int64),
                ("spot_switch_sigma_ns", C.c_int64), ("layer_switch_sigma_ns", C.c_int64),
                ("discard_sigma_ns", C.c_int64), ("rate_sigma", C.c_int64), ("fill_protons_sigma", C.c_int64),
                ("extraction_limit_sigma_ns", C.c_int64)]


class dose_job(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("phase", C.c_int32), ("flags", C.c_uint32),
                ("n_histories", C.c_uint64), ("hist_begin", C.c_uint64), ("hist_end", C.c_uint64),
                ("seed", C.c_uint64), ("spr_scale", C.c_float), ("shift_mm", C.c_float * 3)]


class dose_server_config(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_uint64), ("step_histories", C.c_uint64),
                ("min_slice", C.c_uint64), ("max_active", C.c_int32), ("ref_phase", C.c_int32),
                ("nsub", C.c_int32 * 3), ("accumulate", C.c_int32), ("dvf", C.c_void_p),
                ("policy", C.c_int32), ("max_wait_steps", C.c_int32)]


class dose_request(C.Structure):
    _fields_ = [("n_histories", C.c_uint64), ("seed", C.c_uint64), ("spr_scale", C.c_float),
                ("shift_mm", C.c_float * 3), ("delivery", C.c_void_p)]


class dose_dvf_grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("start_mm", C.c_float * 3), ("spacing_mm", C.c_float * 3),
                ("row_cos", C.c_float * 3), ("col_cos", C.c_float * 3), ("pre", C.c_float * 16),
                ("post", C.c_float * 16)]


assert C.sizeof(dose_spot) == 32 and C.sizeof(dose_job) == 64 and C.sizeof(dose_delivery) == 112
assert C.sizeof(dose_server_config) == 64 and C.sizeof(dose_request) == 40


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libdose.so is not built ({_LIB_PATH}); run "
                          "`python -m paper_1809_03927_gb300.build` (needs nvcc)")
    L = C.CDLL(_LIB_PATH)
    P, I, U64, I64, F = C.c_void_p, C.c_int, C.c_uint64, C.c_int64, C.c_float
    sig = {
        "dose_create_grid": ([C.POINTER(P), I, I, I, F, F, F, P, I, P, I, P, P], I),
        "dose_create_view": ([P, C.POINTER(P)], I),
        "dose_add_spots": ([P, P, I64, P, P], I),
        "dose_run_phase": ([P, I, U64, U64, F, P, P], I),
        "dose_run_batch": ([P, I, P], I),
        "dose_run_4d": ([P, U64, U64, F, P, I, P, P, I, P, I, P], I),
        "dose_set_phase_dose": ([P, I, P, I, P], I),
        "dose_accumulate_subvoxel": ([P, I, P, P, I, P, I, I, P], I),
        "dose_read": ([P, I, I, P, C.c_size_t, I, P], I),
        "dose_set_option": ([P, I, I64], I),
        "dose_destroy": ([P], None),
        "dose_last_error": ([P], C.c_char_p),
        "dose_version": ([], I),
        "dose_debug_philox": ([P, P, P, I, P], I),
        "dose_autotune": ([P, I, U64, U64, U64, P, P], I),
        "dose_server_create": ([P, P, P, I64, P, C.POINTER(P)], I),
        "dose_server_submit": ([P, P, C.POINTER(I64)], I),
        "dose_server_step": ([P, P, P, I, C.POINTER(I)], I),
        "dose_server_result": ([P, I64, I, I, P, C.c_size_t, I, P], I),
        "dose_server_release": ([P, I64], I),
        "dose_server_stats": ([P, P], I),
        "dose_server_destroy": ([P], None),
        "dose_run_phase_noalloc": ([P, I, I, I, F, F, F, P, P, P, I, U64, U64, P, P, P], I),
        "dose_debug_tables": ([P, I, P, P], I),
        "dose_decode_dvf": ([P, P, P, I, P, P, P], I),
        "dose_add_spots_trials": ([P, I, P, I64, P, P, U64, P], I),
        "dose_set_field_beam": ([P, I, P], I),
        "dose_get_option": ([P, I, C.POINTER(I64)], I),
        "dose_measure_peaks": ([P, P], I),
        "dose_autotune_batch": ([P, I, U64, P, P], I),
        "dose_server_timing": ([P, P], I),
        "dose_debug_spread": ([U64, C.c_uint32, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


_lib = _load()


def lib():
    return _lib


# ------------------------------------------------------------- marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device) of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), int(x.is_cuda)
    if not (x.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data, 0


def _nbytes(x):
    if _is_torch(x):
        return x.numel() * x.element_size()
    return x.nbytes


def default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _stream(s):
    if s is None:
        return default_stream()
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return s


def _check(rc, ctx=None):
    if rc != DOSE_OK:
        msg = _lib.dose_last_error(ctx)
        raise DoseError(rc, msg.decode() if msg else "")
    return rc


def _f3(v):
    return (C.c_float * 3)(*[float(a) for a in v])


# ------------------------------------------------------------------ API
def dose_version():
    return _lib.dose_version()


def dose_last_error(ctx=None):
    m = _lib.dose_last_error(ctx)
    return m.decode() if m else ""


def dose_create_grid(nx, ny, nz, dx_mm, dy_mm, dz_mm, origin_mm, n_phases, hu, beam_dir,
                     stream=None):
    """HU must be int16 of n_phases*nz*ny*nx elements (x fastest)."""
    if not _is_torch(hu):
        hu = np.ascontiguousarray(hu, dtype=np.int16)
    p, dev = _ptr(hu)
    out = C.c_void_p()
    rc = _lib.dose_create_grid(C.byref(out), int(nx), int(ny), int(nz), float(dx_mm), float(dy_mm),
                               float(dz_mm), _f3(origin_mm), int(n_phases), p, dev, _f3(beam_dir),
                               _stream(stream))
    _check(rc, None)
    return out.value


def dose_create_view(base):
    out = C.c_void_p()
    _check(_lib.dose_create_view(base, C.byref(out)), None)
    return out.value


def dose_add_spots(ctx, spots, delivery=None, stream=None):
    """``spots``: a ``dose_spot`` ctypes array; ``delivery``: ``dose_delivery`` or None."""
    dl = C.byref(delivery) if delivery is not None else None
    _check(_lib.dose_add_spots(ctx, C.cast(spots, C.c_void_p), len(spots), dl, _stream(stream)), ctx)


def dose_get_option(ctx, option):
    v = C.c_int64()
    _check(_lib.dose_get_option(ctx, int(option), C.byref(v)), ctx)
    return int(v.value)


def dose_set_field_beam(ctx, field, beam_dir):
    """Field ``field`` enters along the grid-axis vector ``beam_dir`` (None:
    the grid's beam)."""
    d = _f3(beam_dir) if beam_dir is not None else None
    _check(_lib.dose_set_field_beam(ctx, int(field), d), ctx)


def dose_run_phase(ctx, phase, n_histories, seed, spr_scale=1.0, shift_mm=None, stream=None):
    sh = _f3(shift_mm) if shift_mm is not None else None
    _check(_lib.dose_run_phase(ctx, int(phase), int(n_histories), int(seed), float(spr_scale), sh,
                               _stream(stream)), ctx)


def dose_run_batch(jobs, stream=None):
    """``jobs``: a ``dose_job`` ctypes array (see ``make_jobs``)."""
    rc = _lib.dose_run_batch(C.cast(jobs, C.c_void_p), len(jobs), _stream(stream))
    _check(rc, jobs[0].ctx if len(jobs) else None)


def dose_run_4d(ctx, n_histories_per_phase, seed, ref_phase, nsub, dvf=None, mask=None,
                spr_scale=1.0, shift_mm=None, stream=None):
    ns = (C.c_int * 3)(*[int(v) for v in nsub])
    if dvf is not None and not _is_torch(dvf):
        dvf = np.ascontiguousarray(dvf, dtype=np.float32)
    if mask is not None and not _is_torch(mask):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
    dp, ddev = _ptr(dvf)
    mp, mdev = _ptr(mask)
    sh = _f3(shift_mm) if shift_mm is not None else None
    _check(_lib.dose_run_4d(ctx, int(n_histories_per_phase), int(seed), float(spr_scale), sh,
                            int(ref_phase), ns, dp, ddev, mp, mdev, _stream(stream)), ctx)


def dose_set_phase_dose(ctx, phase, dose, stream=None):
    p, dev = _ptr(dose)
    _check(_lib.dose_set_phase_dose(ctx, int(phase), p, dev, _stream(stream)), ctx)


ACCUM_EMTM = 0      # energy/mass transfer, Eqs. 4-6 (dvf: phase -> reference)
ACCUM_DIM = 1       # dose interpolation, Eq. 3 (dvf: reference -> phase)


def dose_accumulate_subvoxel(ctx, ref_phase, nsub, dvf=None, mask=None, method=ACCUM_EMTM, stream=None):
    """Accumulate every phase's dose onto ``ref_phase`` (Eq. 2) by ``method``;
    ``dvf`` float32 (P, 3, nz, ny, nx) mm in the direction the method needs."""
    ns = (C.c_int * 3)(*[int(v) for v in nsub])
    if dvf is not None and not _is_torch(dvf):
        dvf = np.ascontiguousarray(dvf, dtype=np.float32)
    if mask is not None and not _is_torch(mask):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
    dp, ddev = _ptr(dvf)
    mp, mdev = _ptr(mask)
    _check(_lib.dose_accumulate_subvoxel(ctx, int(ref_phase), ns, dp, ddev, mp, mdev, int(method),
                                         _stream(stream)), ctx)


def dvf_grid_struct(grid):
    """dose_dvf_grid from a dict: n, start_mm, spacing_mm, row_cos, col_cos
    and optional pre/post (row-major 4x4, default identity)."""
    g = dose_dvf_grid()
    for name in ("n", "start_mm", "spacing_mm", "row_cos", "col_cos"):
        getattr(g, name)[:] = [v for v in grid[name]]
    eye = np.eye(4).ravel()
    g.pre[:] = [float(v) for v in np.asarray(grid.get("pre", eye), np.float64).ravel()]
    g.post[:] = [float(v) for v in np.asarray(grid.get("post", eye), np.float64).ravel()]
    return g


def dose_decode_dvf(ctx, grid, translation, dvf_out, mask=None, stream=None):
    """Decode a registration grid (App. B, Eqs. 7-8) into ``dvf_out``, a
    device tensor of 3 x nvox floats (one phase's block); ``mask`` (device
    uint8, nvox) is cleared outside the grid's hull."""
    g = dvf_grid_struct(grid)
    if not _is_torch(translation):
        translation = np.ascontiguousarray(translation, dtype=np.float32)
    tp, tdev = _ptr(translation)
    op, odev = _ptr(dvf_out)
    mp, mdev = _ptr(mask)
    if not odev or (mask is not None and not mdev):
        raise ValueError("dvf_out and mask must be device tensors")
    _check(_lib.dose_decode_dvf(ctx, C.byref(g), tp, tdev, op, mp, _stream(stream)), ctx)
    return dvf_out


def dose_read(ctx, what, phase, dst, stream=None):
    p, dev = _ptr(dst)
    _check(_lib.dose_read(ctx, int(what), int(phase), p, _nbytes(dst), dev, _stream(stream)), ctx)
    return dst


def dose_autotune(ctx, phase, n_histories, sample_histories, seed, stream=None):
    """Returns (register option, block, chunk, microseconds of the best shape)."""
    best = (C.c_int64 * 4)()
    _check(_lib.dose_autotune(ctx, int(phase), int(n_histories), int(sample_histories), int(seed),
                              _stream(stream), best), ctx)
    return tuple(int(v) for v in best)


def dose_autotune_batch(jobs, sample_histories, stream=None):
    """Tune the launch shape of a batch (``make_jobs`` array) on a sample of
    its histories; returns (register option, block, chunk, microseconds).
    The batch's phases are cleared: run the batch afterwards."""
    best = (C.c_int64 * 4)()
    _check(_lib.dose_autotune_batch(jobs, len(jobs), int(sample_histories), _stream(stream), best), None)
    return tuple(int(v) for v in best)


def dose_measure_peaks(stream=None):
    """Measured peaks of the current device: mixed FP32/INT32 issue rate
    and FFMA rate (thread instructions/s), 64-bit atomic additions/s to an
    L2-resident array, SM count."""
    out = (C.c_double * 4)()
    _check(_lib.dose_measure_peaks(out, _stream(stream)), None)
    return dict(issue_mixed=out[0], issue_ffma=out[1], atomic_u64=out[2], sms=int(out[3]))


def dose_run_phase_noalloc(hu, nx, ny, nz, dx_mm, dy_mm, dz_mm, origin_mm, beam_dir, spots,
                           n_histories, seed, dose, stream=None, ledger=True):
    """Allocation-free dose of a static plan: ``hu`` (int16) and ``dose``
    (float32) are contiguous device tensors of at least nx*ny*nz elements on
    the current device, ``spots`` a ``dose_spot`` array; returns the 8-word
    ledger (None with ``ledger=False``, which passes no ledger buffer).  The
    call returns once the dose is written.  The C call cannot check raw
    pointers, so the types, sizes and device are checked here."""
    import torch
    nvox = int(nx) * int(ny) * int(nz)
    for name, t, dt in (("hu", hu, torch.int16), ("dose", dose, torch.float32)):
        if not (_is_torch(t) and t.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if t.numel() < nvox:
            raise ValueError(f"{name} has {t.numel()} elements, needs nx*ny*nz = {nvox}")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is "
                             f"cuda:{torch.cuda.current_device()}")
    hp, _ = _ptr(hu)
    dp, _ = _ptr(dose)
    led = (C.c_uint64 * 8)() if ledger else None
    _check(_lib.dose_run_phase_noalloc(hp, int(nx), int(ny), int(nz), float(dx_mm), float(dy_mm),
                                       float(dz_mm), _f3(origin_mm), _f3(beam_dir),
                                       C.cast(spots, C.c_void_p), len(spots), int(n_histories),
                                       int(seed), dp, led, _stream(stream)), None)
    return np.array(led[:], dtype=np.uint64) if ledger else None


def dose_server_create(base, memory_budget_bytes, step_histories, spots, delivery=None,
                       min_slice=0, max_active=0, ref_phase=0, nsub=(2, 2, 5), accumulate=1,
                       dvf=None, policy=0, max_wait_steps=0):
    """``dvf``: device tensor (n_phases x 3 x nvox) or None (identity);
    ``policy``: DOSE_SERVE_FAIR (0) or DOSE_SERVE_SHORTEST_FIRST (1);
    ``max_wait_steps``: shortest-first's bound on steps in a row without a
    slice (0: none)."""
    cfg = dose_server_config()
    cfg.memory_budget_bytes, cfg.step_histories, cfg.min_slice = (
        int(memory_budget_bytes), int(step_histories), int(min_slice))
    cfg.max_active, cfg.ref_phase, cfg.accumulate = int(max_active), int(ref_phase), int(accumulate)
    cfg.policy, cfg.max_wait_steps = int(policy), int(max_wait_steps)
    cfg.nsub[:] = [int(v) for v in nsub]
    if dvf is not None:
        p, dev = _ptr(dvf)
        if not dev:
            raise ValueError("the server's DVF must be a device tensor")
        cfg.dvf = p
    out = C.c_void_p()
    dl = C.byref(delivery) if delivery is not None else None
    _check(_lib.dose_server_create(base, C.byref(cfg), C.cast(spots, C.c_void_p), len(spots), dl,
                                   C.byref(out)), None)
    return out.value


def dose_server_submit(server, n_histories, seed, spr_scale=1.0, shift_mm=(0.0, 0.0, 0.0), delivery=None):
    """``delivery``: a ``dose_delivery`` for this request (copied), or None
    for the server's."""
    r = dose_request(int(n_histories), int(seed), float(spr_scale), _f3(shift_mm),
                     C.cast(C.pointer(delivery), C.c_void_p) if delivery is not None else None)
    rid = C.c_int64()
    _check(_lib.dose_server_submit(server, C.byref(r), C.byref(rid)), None)
    return rid.value


def dose_server_step(server, stream=None, max_completed=4096):
    ids = (C.c_int64 * max_completed)()
    n = C.c_int()
    _check(_lib.dose_server_step(server, _stream(stream), ids, max_completed, C.byref(n)), None)
    return [int(ids[i]) for i in range(n.value)]


def dose_server_result(server, rid, what, phase, dst, stream=None):
    p, dev = _ptr(dst)
    _check(_lib.dose_server_result(server, int(rid), int(what), int(phase), p, _nbytes(dst), dev,
                                   _stream(stream)), None)
    return dst


def dose_server_release(server, rid):
    _check(_lib.dose_server_release(server, int(rid)), None)


def dose_server_stats(server):
    out = (C.c_uint64 * 8)()
    _check(_lib.dose_server_stats(server, out), None)
    return dict(zip(("queued", "active", "slots", "completed", "histories", "steps", "slot_bytes",
                     "unreleased"), [int(v) for v in out]))


def dose_server_timing(server):
    """Seconds summed over the server's steps: device time of the transport
    batches and of the finishing accumulations, host wall time of the
    steps, and the number of timed steps."""
    out = (C.c_double * 4)()
    _check(_lib.dose_server_timing(server, out), None)
    return dict(batch_s=out[0], accumulate_s=out[1], step_wall_s=out[2], steps=int(out[3]))


def dose_server_destroy(server):
    _lib.dose_server_destroy(server)


def dose_set_option(ctx, option, value):
    _check(_lib.dose_set_option(ctx, int(option), int(value)), ctx)


def dose_destroy(ctx):
    _lib.dose_destroy(ctx)


def dose_debug_philox(ctr, key, stream=None):
    """Device Philox4x32-10 of n counters (n x 4 uint32) under keys (n x 2):
    returns (words n x 4 uint32, uniforms n x 6 float32)."""
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    n = c.shape[0]
    w = np.zeros((n, 4), np.uint32)
    u = np.zeros((n, 6), np.float32)
    _check(_lib.dose_debug_philox(c.ctypes.data, k.ctypes.data, w.ctypes.data, n, u.ctypes.data))
    return w, u


def dose_debug_tables(energies):
    """Device table lookups at the given energies: columns R(E), E(R(E)),
    Bohr variance per mm, Highland coefficient, Sigma per mm (float32)."""
    e = np.ascontiguousarray(energies, np.float32)
    out = np.zeros((e.shape[0], 5), np.float32)
    _check(_lib.dose_debug_tables(e.ctypes.data, e.shape[0], out.ctypes.data, None))
    return out


def dose_debug_spread(n, log2_strides):
    """History index of each of a job's n work items in the transport's
    birth order over 2^log2_strides strides (host arithmetic only)."""
    out = np.zeros(int(n), np.uint64)
    _check(_lib.dose_debug_spread(int(n), int(log2_strides), out.ctypes.data), None)
    return out


# ------------------------------------------------------- plan marshalling
def spots_array(plan):
    """``dose_spot`` array from a plan with x, y, energy, sigma, protons,
    layer, field sequences."""
    n = len(plan)
    arr = (dose_spot * n)()
    for i in range(n):
        arr[i] = dose_spot(float(plan.x[i]), float(plan.y[i]), float(plan.energy[i]),
                           float(plan.sigma[i]), int(plan.protons[i]), int(plan.layer[i]),
                           int(plan.field[i]))
    return arr


def delivery_struct(d):
    s = dose_delivery()
    for name, _ in dose_delivery._fields_:
        setattr(s, name, int(getattr(d, name, 0)))
    return s


def spread_struct(d):
    s = dose_delivery_spread()
    for name, _ in dose_delivery_spread._fields_:
        setattr(s, name, int(getattr(d, name, 0)))
    return s


def dose_add_spots_trials(ctxs, spots, mean, spread, first_trial=0, stream=None):
    """Load ``spots`` into every context of ``ctxs`` and run the delivery
    simulation of trials first_trial.. (one per context) in one launch."""
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    _check(_lib.dose_add_spots_trials(arr, len(ctxs), C.cast(spots, C.c_void_p), len(spots), C.byref(mean),
                                      C.byref(spread), int(first_trial), _stream(stream)), ctxs[0])


def read_delivery(ctx):
    """The delivery the context's timeline ran, as a dict."""
    buf = np.zeros(C.sizeof(dose_delivery), np.uint8)
    dose_read(ctx, DOSE_DELIVERY, 0, buf)
    d = dose_delivery.from_buffer_copy(buf.tobytes())
    return {name: getattr(d, name) for name, _ in dose_delivery._fields_}


def make_jobs(specs):
    """``dose_job`` array from dicts with keys ctx, phase, n_histories and
    optionally flags, hist_begin, hist_end, seed, spr_scale, shift_mm."""
    arr = (dose_job * len(specs))()
    for i, s in enumerate(specs):
        n = int(s["n_histories"])
        arr[i] = dose_job(s["ctx"], int(s["phase"]), int(s.get("flags", DOSE_JOB_CLEAR | DOSE_JOB_FINISH)),
                          n, int(s.get("hist_begin", 0)), int(s.get("hist_end", n)), int(s.get("seed", 1)),
                          float(s.get("spr_scale", 1.0)), _f3(s.get("shift_mm", (0.0, 0.0, 0.0))))
    return arr
