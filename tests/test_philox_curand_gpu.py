"""Pins every counter word of the oracle's Philox4x32-10 to cuRAND's device API.

The CPU pin (test_oracle_philox.py) uses cuRAND's host generator, whose counters
never reach word 3.  cuRAND's device API puts a 64-bit subsequence number into
counter words 2-3, so a subsequence >= 2^32 exercises word 3, the word that
carries the high half of the site-group index q in the sweep's counter layout.
The helper is compiled here with nvcc from tests/curand_philox_ref.cu.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_ref():
    out = os.path.join(tempfile.mkdtemp(prefix="curand_ref_"), "libcurand_ref.so")
    subprocess.check_call(["nvcc", "-shared", "-Xcompiler", "-fPIC", "-O2", "-gencode",
                           "arch=compute_103a,code=sm_103a", os.path.join(HERE, "curand_philox_ref.cu"), "-o", out])
    lib = ctypes.CDLL(out)
    lib.curand_philox_blocks.restype = ctypes.c_int
    lib.curand_philox_blocks.argtypes = [ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_uint32)]
    return lib


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_all_counter_words_match_curand_device(curand_ref, seed):
    rng = np.random.default_rng(seed & 0xFFFF)
    # exact Python integers throughout (numpy would route values >= 2^63 through float64)
    subseq_list = [0, 1, 0xFFFFFFFF, 1 << 32, (1 << 32) + 5, 0xFFFFFFFFFFFFFFFF]
    subseq_list += [int(v) for v in rng.integers(0, 2**63, size=26, dtype=np.uint64)]
    block_list = [0, 1, 1 << 32, (1 << 32) + 10, (1 << 62) - 1, 0]
    block_list += [int(v) for v in rng.integers(0, 2**61, size=26, dtype=np.uint64)]
    subseq = np.array(subseq_list, dtype=np.uint64)
    offset = np.array([4 * b for b in block_list], dtype=np.uint64)  # whole blocks: cuRAND starts at word 0
    assert all(int(o) % 4 == 0 for o in offset)
    n = subseq.size
    out = np.zeros(4 * n, dtype=np.uint32)
    rc = curand_ref.curand_philox_blocks(seed, subseq.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                         offset.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert rc == 0
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for k in range(n):
        b, s = int(offset[k]) // 4, int(subseq[k])
        ctr = (b & 0xFFFFFFFF, b >> 32, s & 0xFFFFFFFF, s >> 32)
        assert oracle.philox4x32_10(ctr, key) == tuple(int(v) for v in out[4 * k:4 * k + 4]), (k, ctr)
    assert any(int(s) >> 32 for s in subseq)  # word 3 was non-zero in some cases
