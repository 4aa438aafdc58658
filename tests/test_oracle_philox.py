"""Pins the oracle's Philox4x32-10 to an independent implementation.

The oracle's generator is written from Salmon et al. (SC'11).  cuRAND's host
generator (CURAND_RNG_PSEUDO_PHILOX4_32_10, run on the CPU) is a second,
independently written Philox4x32-10: with seed s it emits, for block b of four
words, Philox(key = (s lo, s hi), counter = (b div 65536 as a 64-bit value in
words 0-1, b mod 65536 in word 2, 0 in word 3)); an output offset of o words
starts at block o/4.  This covers the key and counter words 0-2.  Counter word 3
is covered against cuRAND's device API in test_philox_curand_gpu.py.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", os.path.join("/usr/local/cuda/lib64", "libcurand.so")):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcurand not loadable")


def curand_host_words(seed: int, offset: int, n: int) -> np.ndarray:
    cr = _curand()
    g = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert cr.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        return out
    finally:
        cr.curandDestroyGenerator(g)


def expected_counter(block: int):
    a, s = divmod(block, 65536)
    return (a & 0xFFFFFFFF, a >> 32, s, 0)


@pytest.mark.parametrize("seed", [0, 1, 2, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF, 3_000_017])
@pytest.mark.parametrize("offset", [0, 4 * 65536 * 7 + 4 * 123, 1 << 36, (1 << 50) + 4 * 65536 * 3 + 40])
def test_philox_matches_curand_host(seed, offset):
    n = 64
    got = curand_host_words(seed, offset, n)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for b in range(n // 4):
        block = offset // 4 + b
        words = oracle.philox4x32_10(expected_counter(block), key)
        assert tuple(int(v) for v in got[4 * b:4 * b + 4]) == words, (seed, offset, block)


def test_counter_word1_is_exercised():
    # the (1 << 50) offset above puts a 1 into counter word 1
    assert expected_counter(((1 << 50) + 40) // 4)[1] == 1


def test_philox_output_statistics():
    """Top-byte chi-square and mean of 2^16 oracle words look uniform."""
    key = (0xDEADBEEF, 0x01234567)
    words = np.array([w for q in range(1 << 14) for w in oracle.philox4x32_10((q, 0, 5, 1), key)],
                     dtype=np.uint64)
    assert abs(words.mean() / 2**32 - 0.5) < 5 * (1 / np.sqrt(12 * len(words)))
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    exp = len(words) / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert 150 < chi2 < 380  # 255 dof, far tails only


def test_site_word_keying():
    """Site (i,j) of colour c uses word p & 3 of counter (sweep, q lo, c, q hi), q = p >> 2."""
    seed = 0xABCDEF0123
    key = (seed & 0xFFFFFFFF, seed >> 32)
    cases = [(64, i, j) for (i, j) in [(0, 0), (0, 1), (1, 0), (5, 37), (63, 63), (31, 6)]]
    # L = 2^18: q passes 2^32 in the lower rows, so q's high word is non-zero
    cases += [(1 << 18, 200000, 12345), (1 << 18, (1 << 18) - 1, (1 << 18) - 2)]
    for (L, i, j) in cases:
        c = (i + j) & 1
        p = i * (L // 2) + (j >> 1)
        q = p >> 2
        for sweep in (0, 7, 0xFFFFFFFF):
            want = oracle.philox4x32_10((sweep, q & 0xFFFFFFFF, c, q >> 32), key)[p & 3]
            assert oracle.site_word(L, i, j, seed, sweep, c) == want
    assert (200000 * (1 << 17)) >> 2 >= 1 << 32
