"""Pins the oracle's Metropolis chain to results it does not compute itself.

* Exact anchors agree with each other: brute-force enumeration (4x4), the
  transfer matrix (4x4, 6x6, 8x8) and Kaufman's closed form.
* Monte Carlo averages of the oracle chain match exact values within 4 sigma
  (sigma from binning / jackknife): 4x4 vs enumeration, 8x8 vs the transfer
  matrix, 128x128 at beta_c vs Kaufman's finite-torus energy, 128x128 below T_c
  vs Onsager's spontaneous magnetisation.
* The quantised checkerboard kernel is stationary for pi (Sec. 3.1 and the
  appendix's proof), and a planted mistake (exp(-beta h)) breaks it.
* Deterministic limits: beta = 0 negates each colour per half-sweep; at zero
  temperature a site flips iff h <= 0 (checked against a numpy restatement).
* The energy carried incrementally (+2h per accepted flip) equals the energy
  recomputed from scratch after every half-sweep.
* Lattice invariants and the light-cone window evaluation.
* The Sec. 4.1 moments (|m|, m^2, m^4, e, U4) on sample sets with closed-form
  moments: binomial M at beta = 0, ordered chains, a three-point distribution.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact

BETA_C = exact.BETA_C


def _jackknife_binder(M, N, nbins=32):
    M = np.asarray(M, dtype=np.float64) / N
    n = (len(M) // nbins) * nbins
    b = M[len(M) - n:].reshape(nbins, -1)
    s2 = (b ** 2).sum(axis=1)
    s4 = (b ** 4).sum(axis=1)
    tot2, tot4, cnt = s2.sum(), s4.sum(), n
    per = b.shape[1]
    full = 1 - (tot4 / cnt) / (3 * (tot2 / cnt) ** 2)
    jk = np.array([1 - ((tot4 - s4[k]) / (cnt - per)) / (3 * ((tot2 - s2[k]) / (cnt - per)) ** 2)
                   for k in range(nbins)])
    err = math.sqrt((nbins - 1) / nbins * ((jk - jk.mean()) ** 2).sum())
    return full, err


# ---------------------------------------------------------------- exact anchors
@pytest.mark.parametrize("beta", [0.3, 0.4406868, 0.6])
def test_enumeration_matches_transfer_matrix_4x4(beta):
    a = exact.enumerate_observables(4, beta)
    b = exact.transfer_matrix_observables(4, beta)
    for k in ("e", "abs_m", "m2", "m4", "binder"):
        assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-14)


def test_enumeration_reproduces_printed_4x4_values():
    # 13-digit values at beta = 0.4406868, 0.3, 0.6 (E/N, <|M|>/N, U4)
    for beta, e, m, u in [(0.4406868, -1.5656238138147, 0.8438604556001, 0.6171993227991),
                          (0.3, -0.8440540736239, 0.5203580029715, 0.4120282911709),
                          (0.6, -1.9080695278311, 0.9728674502446, 0.6607535637585)]:
        r = exact.enumerate_observables(4, beta)
        assert r["e"] == pytest.approx(e, abs=2e-13)
        assert r["abs_m"] == pytest.approx(m, abs=2e-13)
        assert r["binder"] == pytest.approx(u, abs=2e-13)


@pytest.mark.parametrize("L", [4, 6, 8])
@pytest.mark.parametrize("beta", [0.3, 0.4406868, 0.6])
def test_kaufman_matches_transfer_matrix(L, beta):
    assert exact.kaufman_energy(L, beta) == pytest.approx(exact.transfer_matrix_observables(L, beta)["e"], rel=1e-11)


def test_kaufman_tends_to_minus_sqrt2_at_tc():
    # E/N at beta_c -> -sqrt(2) with an O(1/L) finite-size term (Onsager)
    prev = None
    for L in (64, 256, 1024, 4096):
        d = exact.kaufman_energy(L, BETA_C) + math.sqrt(2.0)
        assert abs(d) < 0.7 / L
        if prev is not None:
            assert abs(d) < abs(prev)
        prev = d


def test_onsager_closed_form_values():
    assert exact.onsager_m0(0.45) == pytest.approx(0.749323, abs=1e-6)
    assert exact.onsager_m0(0.5) == pytest.approx(0.911319, abs=1e-6)
    assert exact.onsager_m0(0.55) == pytest.approx(0.953945, abs=1e-6)
    assert exact.onsager_m0(0.44) == 0.0


# ------------------------------------------------------- Monte Carlo vs exact
@pytest.mark.parametrize("beta", [0.3, 0.4406868, 0.6])
def test_chain_4x4_matches_enumeration(beta):
    L, sweeps, burn = 4, 200_000, 2_000
    _, M, E, _ = oracle.run(L, beta, seed=101, start=oracle.HOT, sweeps=sweeps)
    ex = exact.enumerate_observables(L, beta)
    N = L * L
    e, de = exact.binned_error(E[burn:] / N)
    m, dm = exact.binned_error(np.abs(M[burn:]) / N)
    u, du = _jackknife_binder(M[burn:], N)
    assert abs(e - ex["e"]) < 4 * de, (e, de, ex["e"])
    assert abs(m - ex["abs_m"]) < 4 * dm, (m, dm, ex["abs_m"])
    assert abs(u - ex["binder"]) < 4 * du, (u, du, ex["binder"])


@pytest.mark.parametrize("beta", [0.35, 0.4406868])
def test_chain_8x8_matches_transfer_matrix(beta):
    L, sweeps, burn = 8, 100_000, 2_000
    _, M, E, _ = oracle.run(L, beta, seed=202, start=oracle.HOT, sweeps=sweeps)
    ex = exact.transfer_matrix_observables(L, beta)
    N = L * L
    e, de = exact.binned_error(E[burn:] / N)
    m, dm = exact.binned_error(np.abs(M[burn:]) / N)
    u, du = _jackknife_binder(M[burn:], N)
    assert abs(e - ex["e"]) < 4 * de, (e, de, ex["e"])
    assert abs(m - ex["abs_m"]) < 4 * dm, (m, dm, ex["abs_m"])
    assert abs(u - ex["binder"]) < 4 * du, (u, du, ex["binder"])


def test_energy_at_tc_matches_kaufman_128():
    L, burn, n = 128, 4_000, 16_000
    _, M, E, _ = oracle.run(L, BETA_C, seed=7, start=oracle.COLD, sweeps=burn + n)
    e, de = exact.binned_error(E[burn:] / (L * L))
    k = exact.kaufman_energy(L, BETA_C)
    assert abs(e - k) < 4 * de, (e, de, k)


@pytest.mark.parametrize("beta", [0.5, 0.55])
def test_magnetisation_matches_onsager(beta):
    L, burn, n = 128, 500, 2_500
    _, M, _, _ = oracle.run(L, beta, seed=13, start=oracle.COLD, sweeps=burn + n)
    m, dm = exact.binned_error(np.abs(M[burn:]) / (L * L))
    assert abs(m - exact.onsager_m0(beta)) < 4 * dm, (m, dm, exact.onsager_m0(beta))


# ------------------------------------------------------------- stationarity
def _flip_prob_from_oracle(beta):
    """Acceptance probability of the oracle's decision rule: accept() is the
    indicator of [0, T_h), so the probability is (first rejected word) / 2^32."""
    T2, T4 = oracle.thresholds(beta)

    def first_reject(h):
        if oracle.accept(h, 2**32 - 1, T2, T4):
            return 2**32
        lo, hi = 0, 2**32 - 1  # accept(lo) may be false; find the smallest rejected word
        if not oracle.accept(h, 0, T2, T4):
            return 0
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if oracle.accept(h, mid, T2, T4):
                lo = mid
            else:
                hi = mid
        return hi

    table = {h: first_reject(h) / 2**32 for h in (-4, -2, 0, 2, 4)}
    return lambda h: table[int(h)]


@pytest.mark.parametrize("beta", [0.3, 0.4406868, 0.6])
@pytest.mark.parametrize("colour", [0, 1])
def test_half_sweep_kernel_is_stationary(beta, colour):
    # quantisation to T/2^32 perturbs detailed balance by <= 2^-32 relative
    assert exact.stationarity_residual(4, beta, colour, _flip_prob_from_oracle(beta)) < 1e-8


def test_stationarity_detects_planted_mistake():
    wrong = lambda h: 1.0 if h <= 0 else math.exp(-0.4406868 * h)  # dropped factor 2
    assert exact.stationarity_residual(4, 0.4406868, 0, wrong) > 1e-3


# ------------------------------------------------------ deterministic limits
def test_beta_zero_negates_each_colour():
    L = 16
    s0 = oracle.init(L, seed=5, start=oracle.HOT)
    s1, M, E, _ = oracle.run(L, 0.0, seed=5, start=oracle.HOT, sweeps=1)
    assert np.array_equal(s1, -s0)
    s = s0.copy()
    T = 2**32
    oracle.half_sweep_words(s, 0, T, T, np.full((L, L), 2**32 - 1, dtype=np.uint32))
    colour = (np.add.outer(np.arange(L), np.arange(L)) & 1)
    assert np.array_equal(s, np.where(colour == 0, -s0, s0))


def _zero_temperature_numpy(s, c):
    """Zero-temperature rule written from scratch: flip iff h = sigma * nn <= 0."""
    s = s.astype(np.int64)
    nn = np.roll(s, 1, 0) + np.roll(s, -1, 0) + np.roll(s, 1, 1) + np.roll(s, -1, 1)
    L = s.shape[0]
    colour = (np.add.outer(np.arange(L), np.arange(L)) & 1) == c
    flip = colour & (s * nn <= 0)
    return np.where(flip, -s, s).astype(np.int8)


@pytest.mark.parametrize("L", [4, 8, 12, 64])
def test_zero_temperature_dynamics(L):
    s = oracle.init(L, seed=L, start=oracle.HOT)
    ref = s.copy()
    for t in range(6):
        c = t & 1
        ref = _zero_temperature_numpy(ref, c)
        oracle.half_sweep_words(s, c, 0, 0, np.zeros((L, L), dtype=np.uint32))
        assert np.array_equal(s, ref)
    # the same through the Philox path: beta large enough that T_2 = T_4 = 0
    s_run, _, _, _ = oracle.run(L, 200.0, seed=L, start=oracle.HOT, sweeps=3)
    assert np.array_equal(s_run, ref)


def test_zero_words_accept_every_flip_with_positive_threshold():
    L = 8
    s0 = oracle.init(L, seed=3, start=oracle.HOT)
    s = s0.copy()
    oracle.half_sweep_words(s, 1, 1, 1, np.zeros((L, L), dtype=np.uint32))
    colour = (np.add.outer(np.arange(L), np.arange(L)) & 1)
    assert np.array_equal(s, np.where(colour == 1, -s0, s0))


# ------------------------------------------------------------- invariants
@pytest.mark.parametrize("L,beta", [(8, 0.3), (16, 0.4406868), (64, 0.6), (64, 0.0)])
def test_incremental_energy_invariant(L, beta):
    _, _, _, mism = oracle.run(L, beta, seed=99, start=oracle.HOT, sweeps=40, check=True)
    assert mism == 0


@pytest.mark.parametrize("L,beta,start", [(8, 0.44, 0), (64, 0.3, 0), (64, 0.6, 1), (128, 0.4406868, 0)])
def test_lattice_invariants(L, beta, start):
    s, M, E, _ = oracle.run(L, beta, seed=17, start=start, sweeps=30)
    N = L * L
    assert np.all(np.abs(M) <= N) and np.all(M % 2 == N % 2)
    assert np.all(np.abs(E) <= 2 * N) and np.all(E % 4 == 0)
    assert oracle.observe(s) == (M[-1], E[-1])
    assert set(np.unique(s)) <= {-1, 1}


def test_cold_start_stays_ordered_at_low_temperature():
    L = 64
    _, M, _, _ = oracle.run(L, 1.0, seed=1, start=oracle.COLD, sweeps=50)
    assert M.min() > 0.99 * L * L


def test_hot_start_is_balanced():
    s = oracle.init(512, seed=2, start=oracle.HOT)
    N = s.size
    assert abs(s.astype(np.int64).sum()) < 5 * math.sqrt(N)


# -------------------------------------------------------- light-cone windows
@pytest.mark.parametrize("i0,j0,h,w", [(0, 0, 4, 8), (30, 50, 3, 5), (62, 60, 5, 9), (63, 63, 1, 1)])
def test_window_matches_full_run(i0, j0, h, w):
    L, sweeps, beta, seed = 64, 7, 0.4406868, 77
    full, _, _, _ = oracle.run(L, beta, seed, oracle.HOT, sweeps)
    win = oracle.window(L, beta, seed, oracle.HOT, sweeps, i0, j0, h, w)
    rows = [(i0 + a) % L for a in range(h)]
    cols = [(j0 + b) % L for b in range(w)]
    assert np.array_equal(win, full[np.ix_(rows, cols)])


def test_window_larger_than_torus_still_exact():
    L, sweeps = 16, 9  # margin 18 > L: the buffer wraps the torus more than once
    full, _, _, _ = oracle.run(L, 0.5, 3, oracle.COLD, sweeps)
    win = oracle.window(L, 0.5, 3, oracle.COLD, sweeps, 5, 11, 4, 4)
    assert np.array_equal(win, full[np.ix_([5, 6, 7, 8], [11, 12, 13, 14])])


def test_resume_equals_uninterrupted():
    L, beta, seed = 32, 0.42, 4
    a, Ma, Ea, _ = oracle.run(L, beta, seed, oracle.HOT, 20)
    b1, Mb1, Eb1, _ = oracle.run(L, beta, seed, oracle.HOT, 8)
    b2, Mb2, Eb2, _ = oracle.run(L, beta, seed, oracle.HOT, 12, sweep0=8, state=b1)
    assert np.array_equal(a, b2)
    assert np.array_equal(Ma, np.concatenate([Mb1, Mb2]))
    assert np.array_equal(Ea, np.concatenate([Eb1, Eb2]))


# ----------------------------------------------------------------- moments
def test_moments_exact_against_float():
    rng = np.random.default_rng(0)
    N = 64 * 64
    M = rng.integers(-N, N + 1, size=500) // 2 * 2
    E = rng.integers(-2 * N, 2 * N + 1, size=500) // 4 * 4
    r = oracle.moments_exact(M, E, N, 50)
    m = M[50:].astype(np.float64) / N
    assert r["abs_m"] == pytest.approx(np.abs(m).mean(), rel=1e-13)
    assert r["m2"] == pytest.approx((m ** 2).mean(), rel=1e-13)
    assert r["binder"] == pytest.approx(1 - (m ** 4).mean() / (3 * (m ** 2).mean() ** 2), rel=1e-12)
    assert r["e"] == pytest.approx(E[50:].mean() / N, rel=1e-13)


def test_moments_match_closed_forms():
    """moments_exact on sample sets whose moments are known in closed form, so that a
    wrong power of N, a dropped absolute value or a wrong constant in U4 fails:

    * every configuration of N = 16 independent +-1 spins once (beta = 0): M = 2k - N
      with binomial weights, <M^2> = N, <M^4> = 3N^2 - 2N, hence U4 = 2/(3N);
      <|M|> = N C(N, N/2) / 2^N (the mean distance of a simple random walk after N
      steps); E summed over all states is 0 (each bond product is a fair +-1);
    * an ordered chain, M = +-N: |m| = m^2 = m^4 = 1 and U4 = 2/3;
    * m in {0, +a, -a} with weights 2:1:1: <m^2> = a^2/2, <m^4> = a^4/2, U4 = 1/3;
    * burn-in drops exactly the first samples; a common factor of M and N leaves the
      magnetisation moments unchanged; sums stay exact at |M| = 2^32 (M^4 = 2^128).
    """
    from fractions import Fraction

    N = 16
    x = np.arange(1 << N, dtype=np.uint32)
    k = np.zeros_like(x)
    for b in range(N):
        k += (x >> np.uint32(b)) & np.uint32(1)
    M = 2 * k.astype(np.int64) - N
    E = np.zeros_like(M)
    r = oracle.moments_exact(M, E, N, 0)
    assert r["n"] == 1 << N
    assert r["m2"] == float(Fraction(N, N * N))
    assert r["m4"] == float(Fraction(3 * N * N - 2 * N, N ** 4))
    assert r["binder"] == float(Fraction(2, 3 * N))
    assert r["abs_m"] == float(Fraction(N * math.comb(N, N // 2), (1 << N) * N))
    assert r["e"] == 0.0
    # the 4x4 torus at beta = 0: each of the 2N bond products is +-1 with equal weight
    s = np.where(((x[:, None] >> np.arange(N, dtype=np.uint32)) & 1) == 1, 1, -1).reshape(-1, 4, 4)
    E_torus = -(s * np.roll(s, 1, axis=1) + s * np.roll(s, 1, axis=2)).sum(axis=(1, 2))
    assert oracle.moments_exact(M, E_torus, N, 0)["e"] == 0.0
    assert oracle.moments_exact(M, E_torus, N, 0)["e2"] == float(Fraction(2 * N, N * N))

    L = 64
    Nl = L * L
    ordered = np.array([Nl, -Nl] * 20, dtype=np.int64)
    r = oracle.moments_exact(ordered, np.full(40, -2 * Nl), Nl, 0)
    assert (r["abs_m"], r["m2"], r["m4"], r["binder"], r["e"]) == (1.0, 1.0, 1.0, float(Fraction(2, 3)), -2.0)

    a = 1024
    three = np.array([0, 0, a, -a] * 25, dtype=np.int64)
    r = oracle.moments_exact(three, np.zeros(100, dtype=np.int64), Nl, 0)
    assert r["binder"] == float(Fraction(1, 3))
    assert r["m2"] == float(Fraction(a * a, 2 * Nl * Nl))
    assert r["abs_m"] == float(Fraction(a, 2 * Nl))

    rng = np.random.default_rng(3)
    seq = rng.integers(-Nl, Nl + 1, size=300)
    eseq = rng.integers(-2 * Nl, 2 * Nl + 1, size=300)
    junk = rng.integers(-Nl, Nl + 1, size=7)
    base = oracle.moments_exact(seq, eseq, Nl, 0)
    assert oracle.moments_exact(np.concatenate([junk, seq]), np.concatenate([junk, eseq]), Nl, 7) == base
    scaled = oracle.moments_exact(3 * seq, eseq, 3 * Nl, 0)
    for key in ("abs_m", "m2", "m4", "binder"):
        assert scaled[key] == base[key], key

    big = np.array([1 << 32, -(1 << 32), 1 << 31], dtype=object)
    r = oracle.moments_exact(big, [0, 0, 0], 1 << 32, 0)
    assert r["S4"] == 2 * (1 << 128) + (1 << 124)
    assert r["m4"] == float(Fraction(2 * 16 + 1, 3 * 16))
