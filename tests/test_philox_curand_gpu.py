"""Pins the device Philox4x32-10 (and, through the bit-exact GPU/oracle
parity, the oracle's) to NVIDIA cuRAND's Philox4_32_10 on the same key and
counters, via cuRAND's documented device API in a test-only helper."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                           "-o", out, os.path.join(HERE, "helpers", "curand_philox.cu")])
    lib = ctypes.CDLL(out)
    lib.curand_philox_blocks.restype = ctypes.c_int
    lib.curand_philox_blocks.argtypes = [ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
    return lib


def test_device_philox_equals_curand(curand_lib):
    import paper_1811_04384_gb300 as p
    import oracle
    rng = np.random.default_rng(9)
    n = 4096
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] &= 0x3FFFFFFF            # offset = 4 * (low 64 bits) must fit in 64 bits
    ctr[:8] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
               [0xFFFFFFFF, 0, 0, 0], [5, 7, 0xFFFFFFFF, 3], [2, 3, 4, (1 << 31) | 1]]
    for seed in (0, 1, 7, 0xDEADBEEFCAFEF00D):
        ref = np.empty_like(ctr)
        rc = curand_lib.curand_philox_blocks(seed, ctr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                             ref.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n)
        assert rc == 0
        got = p.philox_blocks(seed, ctr)
        np.testing.assert_array_equal(got, ref)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for k in (0, 1, 5, 6, 7, 100, 4095):
            np.testing.assert_array_equal(oracle.philox4x32_10(ctr[k], key), ref[k])
