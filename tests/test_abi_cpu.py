"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports
every entry point include/dose.h declares, and rejects bad arguments with
DOSE_EINVAL and a message before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dose.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dose_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dose_create_grid", "dose_add_spots", "dose_run_phase", "dose_accumulate_subvoxel",
              "dose_read", "dose_run_batch", "dose_destroy", "dose_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libdose):
    lib = C.CDLL(libdose._LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert libdose.dose_version() == 1


def test_argument_validation_without_device(libdose):
    D = libdose
    hu = np.zeros(64, np.int16)
    with pytest.raises(D.DoseError) as e:
        D.dose_create_grid(0, 4, 4, 1, 1, 1, (0, 0, 0), 1, hu, (0, 0, 1))
    assert e.value.code == D.DOSE_EINVAL and "positive" in str(e.value)
    for bad in [dict(d=(0, 1, 1)), dict(d=(1, float("nan"), 1)), dict(beam=(0, 0.5, 0.5)),
                dict(beam=(1, 1, 0)), dict(phases=0), dict(origin=(0, float("inf"), 0))]:
        with pytest.raises(D.DoseError) as e:
            D.dose_create_grid(4, 4, 4, *bad.get("d", (1, 1, 1)), bad.get("origin", (0, 0, 0)),
                               bad.get("phases", 1), hu, bad.get("beam", (0, 0, 1)))
        assert e.value.code == D.DOSE_EINVAL
        assert D.dose_last_error(None)
    lib = D.lib()
    assert lib.dose_create_grid(None, 4, 4, 4, 1.0, 1.0, 1.0, None, 1, None, 0, None, None) == D.DOSE_EINVAL
    # voxel indices are 32-bit: a grid of 2^31 voxels is refused before any
    # pointer is read or any device memory is touched
    import ctypes as C
    out = C.c_void_p()
    f3 = (C.c_float * 3)
    rc = lib.dose_create_grid(C.byref(out), 2048, 1024, 1024, 1.0, 1.0, 1.0, f3(0, 0, 0), 1, None, 0,
                              f3(0, 0, 1), None)
    assert rc == D.DOSE_EINVAL and out.value is None
    assert b"2^31" in lib.dose_last_error(None)
    assert lib.dose_run_batch(None, 0, None) == D.DOSE_EINVAL
    assert lib.dose_read(None, 0, 0, None, 0, 0, None) == D.DOSE_EINVAL
    assert lib.dose_set_option(None, 0, 0) == D.DOSE_EINVAL
    assert lib.dose_add_spots(None, None, 0, None, None) == D.DOSE_EINVAL
    assert lib.dose_accumulate_subvoxel(None, 0, None, None, 0, None, 0, 0, None) == D.DOSE_EINVAL
    assert lib.dose_debug_philox(None, None, None, 0, None) == D.DOSE_EINVAL
    assert lib.dose_add_spots_trials(None, 0, None, 0, None, None, 0, None) == D.DOSE_EINVAL
    assert lib.dose_decode_dvf(None, None, None, 0, None, None, None) == D.DOSE_EINVAL
    assert lib.dose_get_option(None, 0, None) == D.DOSE_EINVAL
    assert lib.dose_set_field_beam(None, 0, None) == D.DOSE_EINVAL
    lib.dose_destroy(None)


def test_structs_match_the_header(libdose):
    D = libdose
    assert C.sizeof(D.dose_spot) == 32
    assert C.sizeof(D.dose_delivery) == 6 * 4 + 5 * 8 + 2 * 8 + 2 * 4 + 3 * 8
    assert D.dose_delivery.max_protons_per_paint.offset == 104
    assert C.sizeof(D.dose_delivery_spread) == 9 * 8
    assert C.sizeof(D.dose_dvf_grid) == 3 * 4 + 4 * 3 * 4 + 2 * 16 * 4
    assert C.sizeof(D.dose_job) == 64
    assert C.sizeof(D.dose_server_config) == 64
    assert D.dose_server_config.dvf.offset == 48 and D.dose_server_config.policy.offset == 56
    assert D.dose_server_config.max_wait_steps.offset == 60
    assert (D.DOSE_SERVE_FAIR, D.DOSE_SERVE_SHORTEST_FIRST) == (0, 1)
    assert D.dose_job.shift_mm.offset == 52


def test_birth_order_is_a_round_robin_bijection(libdose):
    """The order in which a job's histories are born (host arithmetic, no
    device): every history exactly once; the last t = min(n/8, 2^18) work
    items take the last t histories in order; before them, with 2^s
    strides, work item w goes to stride w mod 2^s of the first n - t
    histories, inside each stride the histories follow one another, and
    the strides tile that range in order, the first (n - t) mod 2^s one
    history longer; s = 0 and short ranges are plan order."""
    D = libdose
    for n in (0, 1, 5, 63, 64, 65, 1000, 4097, 100_003, 3_000_001):
        for s in (0, 1, 4, 6):
            h = D.dose_debug_spread(n, s).astype(np.int64)
            assert np.array_equal(np.sort(h), np.arange(n))
            if s == 0:
                assert np.array_equal(h, np.arange(n))
                continue
            t = min(n // 8, 1 << 18)
            assert np.array_equal(h[n - t:], np.arange(n - t, n))
            ns, K = n - t, 1 << s
            head = h[:ns]
            if ns <= K:
                assert np.array_equal(head, np.arange(ns))
                continue
            starts = []
            for k in range(K):
                mine = head[k::K]
                assert np.all(np.diff(mine) == 1)              # consecutive inside a stride
                assert len(mine) == ns // K + (1 if k < ns % K else 0)
                starts.append(int(mine[0]))
            lengths = [ns // K + (1 if k < ns % K else 0) for k in range(K)]
            assert starts == list(np.cumsum([0] + lengths[:-1]))
    with pytest.raises(D.DoseError):
        D.dose_debug_spread(10, 17)
