"""The engine's Philox4x32-10 against NVIDIA's: cuRAND's Philox4_32_10
device generator, called (not read) from a small kernel built here, gives
the same 128-bit blocks for the same key and counter.  (The generator is
also pinned to the published known-answer vectors through the oracle.)"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_ref(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    so = tmp_path_factory.mktemp("curand") / "libcurandref.so"
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "curand_philox_ref.cu"), "-o", str(so)], check=True)
    lib = C.CDLL(str(so))
    lib.curand_philox_blocks.argtypes = [C.c_void_p] * 4 + [C.c_int]
    lib.curand_philox_blocks.restype = C.c_int
    return lib


def test_device_philox_equals_curand(gpu, curand_ref):
    rng = np.random.default_rng(11)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    ctr[:, 1] %= 2 ** 30                      # offset = 4 (c0 + 2^32 c1) stays below 2^64
    ctr[:8] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [7, 0, 0, 3], [2 ** 32 - 1, 0, 0, 0],
               [0, 1, 0, 0], [5, 2, 2 ** 32 - 1, 2 ** 32 - 1], [12345, 0, 0, 0]]
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64)
    key[0] = [0, 0]
    seed = np.ascontiguousarray(key[:, 0] | (key[:, 1] << np.uint64(32)), np.uint64)
    subsequence = np.ascontiguousarray(ctr[:, 2] | (ctr[:, 3] << np.uint64(32)), np.uint64)
    offset = np.ascontiguousarray((ctr[:, 0] | (ctr[:, 1] << np.uint64(32))) * np.uint64(4), np.uint64)
    ref = np.zeros((n, 4), np.uint32)
    rc = curand_ref.curand_philox_blocks(seed.ctypes.data, subsequence.ctypes.data, offset.ctypes.data,
                                         ref.ctypes.data, n)
    assert rc == 0
    words, _ = gpu.dose_debug_philox(ctr.astype(np.uint32), key.astype(np.uint32))
    np.testing.assert_array_equal(words, ref)
