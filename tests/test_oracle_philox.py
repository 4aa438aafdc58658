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


def _uniform_from_philox(p, seed, sweep, c):
    """U of plane index p restated from the definition: bit b = p & 31 of the 32
    random words of plane word g = p >> 5, R_k = output k & 3 of the call with
    counter (sweep, q lo, c, q hi), q = 8g + k // 4; R_0 gives the top bit."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    g, b = p >> 5, p & 31
    u = 0
    for k in range(32):
        q = 8 * g + k // 4
        r = oracle.philox4x32_10((sweep, q & 0xFFFFFFFF, c, q >> 32), key)[k & 3]
        u |= ((r >> b) & 1) << (31 - k)
    return u


def test_site_word_keying():
    """Site (i,j) of colour c, plane index p = i*(L/2) + (j>>1), draws the uniform above."""
    seed = 0xABCDEF0123
    cases = [(64, i, j) for (i, j) in [(0, 0), (0, 1), (1, 0), (5, 37), (63, 63), (31, 6)]]
    # L = 2^18: q passes 2^32 in the lower rows, so q's high word is non-zero
    cases += [(1 << 18, 200000, 12345), (1 << 18, (1 << 18) - 1, (1 << 18) - 2)]
    # L = 72 (not a multiple of 64): plane words straddle rows
    cases += [(72, 0, 70), (72, 1, 0), (72, 1, 1), (72, 13, 44)]
    for (L, i, j) in cases:
        c = (i + j) & 1
        p = i * (L // 2) + (j >> 1)
        for sweep in (0, 7, 0xFFFFFFFF):
            assert oracle.site_word(L, i, j, seed, sweep, c) == _uniform_from_philox(p, seed, sweep, c)
    assert (200000 * (1 << 17)) >> 5 >= 1 << 29


def test_site_uniforms_are_uniform():
    """The transposed uniforms of many sites: each of their 32 bits is a fair coin
    and the top byte is flat (chi-square, 255 degrees of freedom)."""
    L = 64
    u = np.array([oracle.site_word(L, i, j, 99, 3, (i + j) & 1) for i in range(L) for j in range(L)], dtype=np.uint64)
    n = u.size
    for bit in range(32):
        ones = int(((u >> np.uint64(bit)) & np.uint64(1)).sum())
        assert abs(ones - n / 2) < 5 * np.sqrt(n / 4), bit
    counts = np.bincount((u >> np.uint64(24)).astype(np.int64), minlength=256)
    chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
    assert 150 < chi2 < 380


def test_hot_start_is_the_top_bit_of_the_first_random_word():
    """U < 2^31 holds exactly when bit b of R_0 is 0: the hot start needs R_0 only."""
    L, seed = 64, 12
    s = oracle.init(L, seed, oracle.HOT)
    key = (seed, 0)
    for (i, j) in [(0, 0), (3, 9), (40, 41), (63, 0)]:
        c = (i + j) & 1
        p = i * (L // 2) + (j >> 1)
        r0 = oracle.philox4x32_10((0xFFFFFFFF, 8 * (p >> 5), c, 0), key)[0]
        assert s[i, j] == (1 if ((r0 >> (p & 31)) & 1) == 0 else -1)
