"""Pins the 3D oracle (the Sec. 3 Hamiltonian on the cubic lattice, d = 3, with the
checkerboard rules of Sec. 3.1 and Algorithms 1-2) to results that do not come
from the oracle itself: 50-digit thresholds, exact enumeration and exact
stationarity on small tori, deterministic limits against a separately written
numpy rule, and the energy bookkeeping of the chain.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
from oracle import exact

BETA_C3 = 0.2216546  # simple-cubic critical coupling (Monte Carlo literature), for choosing test points


# ------------------------------------------------------------- thresholds
@pytest.mark.parametrize("beta", [0.0, 1e-9, 0.05, 0.1, BETA_C3, 0.3, 0.5, 1.0, 3.0, 200.0])
def test_thresholds3d_match_50_digit_arithmetic(beta):
    got = oracle.thresholds3d(beta)
    with mp.workdps(50):
        for h, T in zip((2, 4, 6), got):
            exact_t = mp.exp(-2 * mp.mpf(beta) * h) * 2**32
            ceil_exact = int(mp.ceil(exact_t))
            frac = exact_t - mp.floor(exact_t)
            if min(frac, 1 - frac) > mp.mpf("1e-6"):
                assert T == min(ceil_exact, 2**32), (beta, h)
            else:  # libm may round across an integer; still within one
                assert abs(T - ceil_exact) <= 1
    assert got[0] >= got[1] >= got[2]


def test_thresholds3d_extend_the_2d_ones():
    for beta in np.linspace(0, 2, 41):
        T2, T4 = oracle.thresholds(float(beta))
        assert oracle.thresholds3d(float(beta))[:2] == (T2, T4)


def test_accept3d_rule():
    T = (1000, 100, 10)
    for h in (-6, -4, -2, 0):
        assert oracle.accept3d(h, 2**32 - 1, T)
    for h, t in ((2, 1000), (4, 100), (6, 10)):
        assert oracle.accept3d(h, t - 1, T) and not oracle.accept3d(h, t, T)


# ------------------------------------------------------------- RNG keying
def _uniform3_from_philox(p, seed, sweep, c):
    key = (seed & 0xFFFFFFFF, seed >> 32)
    g, b = p >> 5, p & 31
    u = 0
    for k in range(32):
        q = 8 * g + k // 4
        u |= ((oracle.philox4x32_10((sweep, q & 0xFFFFFFFF, c, q >> 32), key)[k & 3] >> b) & 1) << (31 - k)
    return u


def test_site_word3d_keying():
    """Site (i,j,k) draws the uniform of plane index p = (i*Y + j)*(Z/2) + (k >> 1):
    bit p & 31 of the random words R_0 .. R_31 of plane word p >> 5, R_0 the top bit."""
    seed = 0x1234_5678_9ABC_DEF0
    cases = [((4, 6, 8), (0, 0, 0)), ((4, 6, 8), (3, 5, 7)), ((8, 8, 8), (1, 2, 5)), ((2, 2, 4), (1, 1, 3)),
             # q passes 2^32: X = Y = 65536, Z = 64
             ((65536, 65536, 64), (65535, 40000, 63)), ((65536, 65536, 64), (33000, 1, 2))]
    for dims, (i, j, k) in cases:
        X, Y, Z = dims
        c = (i + j + k) & 1
        p = (i * Y + j) * (Z // 2) + (k >> 1)
        for sweep in (0, 9, 0xFFFFFFFF):
            assert oracle.site_word3d(dims, i, j, k, seed, sweep, c) == _uniform3_from_philox(p, seed, sweep, c)
    assert 8 * (((65535 * 65536 + 40000) * 32) >> 5) >= 1 << 32  # q = 8 (p >> 5) has a high word


def test_3d_row_keying_matches_2d_rows():
    """A 3D row (i, j) is keyed like 2D row i*Y + j of an (X*Y) x Z lattice."""
    X, Y, Z, seed = 4, 6, 8, 77
    for (i, j, k) in [(0, 0, 0), (1, 2, 3), (3, 5, 7), (2, 0, 6)]:
        r = i * Y + j
        for c in (0, 1):
            for sweep in (0, 5):
                p2 = r * (Z // 2) + (k >> 1)
                assert oracle.site_word3d((X, Y, Z), i, j, k, seed, sweep, c) == _uniform3_from_philox(p2, seed, sweep, c)


# --------------------------------------------------- exact enumeration pins
def test_enumeration3d_limits():
    # beta -> infinity: the two ground states, every bond satisfied (3N bonds)
    cold = exact.enumerate3d_observables((2, 2, 4), 5.0)
    assert cold["e"] == pytest.approx(-3.0, abs=1e-12) and cold["abs_m"] == pytest.approx(1.0, abs=1e-12)
    # beta = 0: uniform over 2^N states, <m^2> = 1/N, <m^4> = (3N^2 - 2N)/N^4
    N = 16
    hot = exact.enumerate3d_observables((2, 2, 4), 0.0)
    assert hot["e"] == pytest.approx(0.0, abs=1e-12)
    assert hot["m2"] == pytest.approx(1.0 / N, rel=1e-12)
    assert hot["m4"] == pytest.approx((3 * N * N - 2 * N) / N**4, rel=1e-12)


@pytest.mark.parametrize("beta", [0.1, 0.2, 0.35])
def test_chain3d_matches_enumeration_2x2x4(beta):
    dims = (2, 2, 4)
    N = 16
    ex = exact.enumerate3d_observables(dims, beta)
    _, M, E, _ = oracle.run3d(dims, beta, seed=int(beta * 1000) + 5, start=oracle.HOT, sweeps=400_000)
    burn = 1000
    e_mean, e_err = exact.binned_error(E[burn:] / N)
    m_mean, m_err = exact.binned_error(np.abs(M[burn:]) / N)
    m2_mean, m2_err = exact.binned_error((M[burn:] / N) ** 2)
    assert abs(e_mean - ex["e"]) < 5 * e_err + 1e-4, (e_mean, ex["e"], e_err)
    assert abs(m_mean - ex["abs_m"]) < 5 * m_err + 1e-4, (m_mean, ex["abs_m"], m_err)
    assert abs(m2_mean - ex["m2"]) < 5 * m2_err + 1e-4, (m2_mean, ex["m2"], m2_err)


def _flip_prob_from_oracle3d(beta):
    """The quantised acceptance actually used: P(flip | h) = (first rejected word) / 2^32."""
    T = oracle.thresholds3d(beta)

    def first_reject(h):
        if oracle.accept3d(h, 2**32 - 1, T):
            return 2**32
        if not oracle.accept3d(h, 0, T):
            return 0
        lo, hi = 0, 2**32 - 1
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if oracle.accept3d(h, mid, T):
                lo = mid
            else:
                hi = mid
        return hi

    table = {h: first_reject(h) / 2**32 for h in (-6, -4, -2, 0, 2, 4, 6)}
    return lambda h: table[int(h)]


@pytest.mark.parametrize("beta", [0.1, BETA_C3, 0.4])
@pytest.mark.parametrize("colour", [0, 1])
def test_half_sweep3d_kernel_is_stationary(beta, colour):
    # quantisation to T/2^32 perturbs detailed balance by <= 2^-32 relative
    res = exact.stationarity_residual3d((2, 2, 4), beta, colour, _flip_prob_from_oracle3d(beta))
    assert res < 1e-8


def test_stationarity3d_detects_planted_mistake():
    beta = BETA_C3
    wrong = lambda h: 1.0 if h <= 0 else math.exp(-beta * h)  # dropped factor 2
    assert exact.stationarity_residual3d((2, 2, 4), beta, 0, wrong) > 1e-3
    too_few = lambda h: 1.0 if h <= 2 else math.exp(-2 * beta * h)  # h = 2 always flips
    assert exact.stationarity_residual3d((2, 2, 4), beta, 1, too_few) > 1e-3


# ---------------------------------------------------- deterministic limits
def _zero_temperature_numpy3d(s, c):
    """Zero-temperature rule written from scratch: flip colour-c sites with h <= 0."""
    s = s.astype(np.int64)
    nn = sum(np.roll(s, d, a) for a in range(3) for d in (1, -1))
    X, Y, Z = s.shape
    colour = (np.arange(X)[:, None, None] + np.arange(Y)[None, :, None] + np.arange(Z)[None, None, :]) & 1
    flip = (colour == c) & (s * nn <= 0)
    return np.where(flip, -s, s).astype(np.int8)


@pytest.mark.parametrize("dims", [(4, 6, 8), (8, 8, 8), (2, 4, 6), (16, 16, 16)])
def test_zero_temperature_dynamics3d(dims):
    s = oracle.init3d(dims, seed=sum(dims), start=oracle.HOT)
    ref = s.copy()
    zeros = np.zeros(dims, dtype=np.uint32)
    for t in range(6):
        c = t & 1
        ref = _zero_temperature_numpy3d(ref, c)
        oracle.half_sweep_words3d(s, c, (0, 0, 0), zeros)
        assert np.array_equal(s, ref), (dims, t)
    # the same through the Philox path: beta large enough that every threshold is 0
    assert oracle.thresholds3d(200.0) == (0, 0, 0)
    s_run, _, _, _ = oracle.run3d(dims, 200.0, seed=sum(dims), start=oracle.HOT, sweeps=3)
    assert np.array_equal(s_run, ref)


def test_beta_zero_negates_each_colour3d():
    dims = (6, 4, 8)
    s0 = oracle.init3d(dims, seed=5, start=oracle.HOT)
    s1, _, _, _ = oracle.run3d(dims, 0.0, seed=5, start=oracle.HOT, sweeps=1)
    assert np.array_equal(s1, -s0)
    s = s0.copy()
    T = (2**32, 2**32, 2**32)
    oracle.half_sweep_words3d(s, 1, T, np.full(dims, 2**32 - 1, dtype=np.uint32))
    X, Y, Z = dims
    colour = (np.arange(X)[:, None, None] + np.arange(Y)[None, :, None] + np.arange(Z)[None, None, :]) & 1
    assert np.array_equal(s, np.where(colour == 1, -s0, s0))


def test_threshold_classes_use_their_own_threshold():
    """Words just below / at T_h flip / keep exactly the sites of class h."""
    dims = (4, 4, 4)
    X, Y, Z = dims
    s0 = oracle.init3d(dims, seed=11, start=oracle.HOT)
    si = s0.astype(np.int64)
    nn = sum(np.roll(si, d, a) for a in range(3) for d in (1, -1))
    h = si * nn
    T = (5000, 500, 50)
    colour = (np.arange(X)[:, None, None] + np.arange(Y)[None, :, None] + np.arange(Z)[None, None, :]) & 1
    for below in (True, False):
        words = np.zeros(dims, dtype=np.uint32)
        for hv, t in ((2, T[0]), (4, T[1]), (6, T[2])):
            words[h == hv] = t - 1 if below else t
        words[h <= 0] = 2**32 - 1
        s = s0.copy()
        oracle.half_sweep_words3d(s, 0, T, words)
        want_flip = (colour == 0) & ((h <= 0) | below)
        assert np.array_equal(s, np.where(want_flip, -s0, s0)), below


# ------------------------------------------------------------- invariants
def _observe_numpy3d(s):
    si = s.astype(np.int64)
    return int(si.sum()), int(-sum((si * np.roll(si, -1, a)).sum() for a in range(3)))


@pytest.mark.parametrize("dims,beta", [((8, 8, 8), 0.15), ((16, 16, 16), BETA_C3), ((4, 6, 8), 0.6), ((8, 8, 8), 0.0)])
def test_incremental_energy_invariant3d(dims, beta):
    s, M, E, mism = oracle.run3d(dims, beta, seed=3, start=oracle.HOT, sweeps=20, check=True)
    assert mism == 0
    assert (int(M[-1]), int(E[-1])) == _observe_numpy3d(s)
    assert set(np.unique(s)) <= {-1, 1}


def test_hot_start_is_balanced3d():
    s = oracle.init3d((64, 64, 64), seed=9, start=oracle.HOT)
    N = s.size
    assert abs(int(s.astype(np.int64).sum())) < 5 * math.sqrt(N)
    assert oracle.observe3d(s) == _observe_numpy3d(s)


def test_cold_start_stays_ordered_at_low_temperature3d():
    _, M, _, _ = oracle.run3d((8, 8, 8), 1.0, seed=1, start=oracle.COLD, sweeps=50)
    assert M.min() > 0.95 * 512


def test_resume_equals_uninterrupted3d():
    dims = (8, 6, 4)
    a, Ma, Ea, _ = oracle.run3d(dims, 0.25, seed=4, sweeps=9)
    b, Mb, Eb, _ = oracle.run3d(dims, 0.25, seed=4, sweeps=4)
    c, Mc, Ec, _ = oracle.run3d(dims, 0.25, seed=4, sweeps=5, sweep0=4, state=b)
    assert np.array_equal(a, c)
    assert np.array_equal(Ma, np.concatenate([Mb, Mc])) and np.array_equal(Ea, np.concatenate([Eb, Ec]))


# ------------------------------------------------ light-cone windows (3D)
@pytest.mark.parametrize("origin,shape", [((0, 0, 0), (3, 4, 5)), ((14, 15, 13), (4, 3, 6)),
                                          ((5, 9, 2), (2, 2, 2)), ((15, 17, 19), (1, 1, 1))])
def test_window3d_matches_full_run(origin, shape):
    # unequal extents, so that a transposed axis or a wrong plane index shows
    dims, sweeps, beta, seed = (16, 18, 20), 3, BETA_C3, 41
    full, _, _, _ = oracle.run3d(dims, beta, seed, oracle.HOT, sweeps)
    win = oracle.window3d(dims, beta, seed, oracle.HOT, sweeps, origin, shape)
    idx = [[(o + a) % n for a in range(s)] for o, s, n in zip(origin, shape, dims)]
    assert np.array_equal(win, full[np.ix_(*idx)])


def test_window3d_larger_than_torus_and_offset_sweeps():
    # margin 2 * 4 = 8 exceeds every extent: the box wraps the torus more than once
    dims, beta, seed = (6, 8, 4), 0.3, 9
    full, _, _, _ = oracle.run3d(dims, beta, seed, oracle.COLD, 4)
    win = oracle.window3d(dims, beta, seed, oracle.COLD, 4, (5, 7, 3), (2, 3, 2))
    idx = [[(o + a) % n for a in range(s)] for o, s, n in zip((5, 7, 3), (2, 3, 2), dims)]
    assert np.array_equal(win, full[np.ix_(*idx)])
    # sweeps numbered from sweep0 = 5 draw other uniforms: the same as resuming the
    # full chain at sweep 5 from the start state
    start = oracle.init3d(dims, seed, oracle.HOT)
    ref, _, _, _ = oracle.run3d(dims, beta, seed, sweeps=2, sweep0=5, state=start)
    win5 = oracle.window3d(dims, beta, seed, oracle.HOT, 2, (0, 0, 0), dims, sweep0=5)
    assert np.array_equal(win5, ref)
