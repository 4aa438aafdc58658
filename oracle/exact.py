"""Exact results for the 2D Ising model on an L x L torus (mu = 0, J = 1, Sec. 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  These are the
independent anchors the Monte Carlo oracle is pinned against:

* ``enumerate_observables`` -- brute force over all 2^(L*L) states (L <= 4).
* ``stationarity_residual`` -- exact pi P_c = pi check of one checkerboard
  half-sweep kernel on the 4x4 torus (the stationarity claim of Sec. 3.1 and its
  proof in the appendix).
* ``transfer_matrix_observables`` -- row-to-row transfer matrix carrying the
  magnetisation distribution and the energy moment (L <= 8).
* ``kaufman_log_z`` / ``kaufman_energy`` -- Kaufman's (1949) closed form of the
  finite-torus partition function; the energy is -d ln Z / d beta.
* ``onsager_m0`` -- Onsager/Yang spontaneous magnetisation (1 - sinh^-4(2 beta))^(1/8)
  for beta > beta_c, beta_c = ln(1 + sqrt 2)/2 (Sec. 4.1).
* ``enumerate3d_observables`` / ``stationarity_residual3d`` -- the same brute
  force and exact pi P_c = pi check on a small X x Y x Z torus (the Sec. 3
  Hamiltonian with d = 3), for the three-dimensional generalisation.
"""
from __future__ import annotations

import math

import numpy as np

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


def _all_states(L: int) -> np.ndarray:
    N = L * L
    if N > 20:
        raise ValueError("enumeration is for L*L <= 20")
    idx = np.arange(1 << N, dtype=np.uint32)
    bits = (idx[:, None] >> np.arange(N, dtype=np.uint32)) & 1
    return (1 - 2 * bits.astype(np.int8)).reshape(-1, L, L)


def _energies(s: np.ndarray) -> np.ndarray:
    s = s.astype(np.int64)
    return -(s * np.roll(s, -1, axis=1)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=2)).sum(axis=(1, 2))


def enumerate_observables(L: int, beta: float) -> dict:
    """<E>/N, <|M|>/N, <m^2>, <m^4>, U4 by summing over every state."""
    s = _all_states(L)
    N = L * L
    E = _energies(s).astype(np.float64)
    M = s.astype(np.int64).sum(axis=(1, 2)).astype(np.float64)
    w = np.exp(-beta * (E - E.min()))
    Z = w.sum()
    m2 = (w * (M / N) ** 2).sum() / Z
    m4 = (w * (M / N) ** 4).sum() / Z
    return {"e": (w * E).sum() / Z / N, "abs_m": (w * np.abs(M)).sum() / Z / N, "m2": m2, "m4": m4,
            "binder": 1.0 - m4 / (3.0 * m2 * m2)}


def stationarity_residual(L: int, beta: float, colour: int, flip_prob) -> float:
    """max |pi P_c - pi| / max pi for one half-sweep of colour `colour`.

    P_c flips each colour-c site independently with probability flip_prob(h),
    h = sigma * nn, keeping the other colour fixed (Sec. 3.1).  pi is the
    Boltzmann distribution exp(-beta H)/Z (Sec. 3).
    """
    s = _all_states(L)
    N = L * L
    E = _energies(s).astype(np.float64)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    ii, jj = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    sites = [(int(i), int(j)) for i, j in zip(ii.ravel(), jj.ravel()) if (i + j) % 2 == colour]
    nsite = len(sites)
    f = np.empty((s.shape[0], nsite))
    for k, (i, j) in enumerate(sites):
        nn = (s[:, (i - 1) % L, j].astype(np.int64) + s[:, (i + 1) % L, j] + s[:, i, (j - 1) % L]
              + s[:, i, (j + 1) % L])
        h = s[:, i, j].astype(np.int64) * nn
        f[:, k] = np.vectorize(flip_prob, otypes=[np.float64])(h)
    bitpos = np.array([i * L + j for i, j in sites], dtype=np.uint32)
    state_idx = np.arange(s.shape[0], dtype=np.uint32)
    out = np.zeros_like(pi)
    for F in range(1 << nsite):
        prob = pi.copy()
        mask = np.uint32(0)
        for k in range(nsite):
            if (F >> k) & 1:
                prob *= f[:, k]
                mask |= np.uint32(1) << bitpos[k]
            else:
                prob *= 1.0 - f[:, k]
        np.add.at(out, state_idx ^ mask, prob)
    return float(np.abs(out - pi).max() / pi.max())


def transfer_matrix_observables(L: int, beta: float) -> dict:
    """Exact <E>/N, <|M|>/N, <m^2>, <m^4>, U4 on the L x L torus (L <= 8).

    Rows of L spins are the transfer states.  The first row s0 is kept as an
    index so the chain can be closed periodically; the magnetisation is carried
    as an explicit axis, the energy as a first-moment companion vector.
    """
    N = L * L
    S = 1 << L
    st = np.arange(S)
    sig = 1 - 2 * ((st[:, None] >> np.arange(L)) & 1)  # (S, L)
    m_row = sig.sum(axis=1)
    e_row = -(sig * np.roll(sig, -1, axis=1)).sum(axis=1)
    e_vert = -(sig @ sig.T)  # (S, S)
    eps = (e_row[:, None] + e_vert).astype(np.float64)  # energy of row t plus bond t -> t'
    w = np.exp(-beta * (eps + 2 * L))  # scaled by exp(-beta * E_min / L) per row
    nM = N + 1  # M index (M + N) / 2 in 0..N
    v = np.zeros((S, nM, S))  # (s0, M index, current row)
    u = np.zeros((S, nM, S))
    v[st, (m_row + N) // 2, st] = 1.0

    def shift(a: np.ndarray) -> np.ndarray:
        # appending row t adds m(t) to M, i.e. m(t)/2 to the M index; partial sums
        # stay inside [-N, N], so the roll never wraps a non-zero entry
        out = np.empty_like(a)
        for t in range(S):
            out[:, :, t] = np.roll(a[:, :, t], int(m_row[t]) // 2, axis=1)
        return out

    for _ in range(L - 1):
        v2 = v.reshape(S * nM, S) @ w
        u2 = u.reshape(S * nM, S) @ w + v.reshape(S * nM, S) @ (w * eps)
        v = shift(v2.reshape(S, nM, S))
        u = shift(u2.reshape(S, nM, S))
    # close the torus: weight of the bond from the last row back to s0
    wc = w[:, st]  # (t, s0)
    ec = eps[:, st]
    ZM = np.einsum("amt,ta->m", v, wc)
    ZE = np.einsum("amt,ta->", u, wc) + np.einsum("amt,ta->", v, wc * ec)
    Mv = np.arange(nM) * 2 - N
    Z = ZM.sum()
    m2 = (ZM * (Mv / N) ** 2).sum() / Z
    m4 = (ZM * (Mv / N) ** 4).sum() / Z
    return {"e": ZE / Z / N, "abs_m": (ZM * np.abs(Mv)).sum() / Z / N, "m2": m2, "m4": m4,
            "binder": 1.0 - m4 / (3.0 * m2 * m2)}


def kaufman_log_z(L: int, beta, dps: int = 50):
    """ln Z of the L x L torus from Kaufman's formula (Phys. Rev. 76, 1232 (1949)).

    Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4) with K = beta (J = 1),
    Z1,2 = prod_{k<L} 2 cosh / 2 sinh (L gamma_{2k+1} / 2),
    Z3,4 = prod_{k<L} 2 cosh / 2 sinh (L gamma_{2k} / 2),
    cosh gamma_l = cosh 2K coth 2K - cos(pi l / L) for l >= 1 and
    gamma_0 = 2K + ln tanh K (signed).
    """
    import mpmath as mp

    with mp.workdps(dps):
        K = mp.mpf(beta)
        n = L
        c = mp.cosh(2 * K) * mp.coth(2 * K)

        def gamma(l):
            if l == 0:
                return 2 * K + mp.log(mp.tanh(K))
            return mp.acosh(c - mp.cos(mp.pi * l / n))

        g_odd = [gamma(2 * k + 1) for k in range(n)]
        g_even = [gamma(2 * k) for k in range(n)]
        Z1 = mp.fprod(2 * mp.cosh(L * g / 2) for g in g_odd)
        Z2 = mp.fprod(2 * mp.sinh(L * g / 2) for g in g_odd)
        Z3 = mp.fprod(2 * mp.cosh(L * g / 2) for g in g_even)
        Z4 = mp.fprod(2 * mp.sinh(L * g / 2) for g in g_even)
        return mp.log(mp.mpf(1) / 2) + (L * L / mp.mpf(2)) * mp.log(2 * mp.sinh(2 * K)) + mp.log(Z1 + Z2 + Z3 + Z4)


def kaufman_energy(L: int, beta: float, dps: int = 50) -> float:
    """Exact <E>/N = -(1/N) d ln Z / d beta on the L x L torus."""
    import mpmath as mp

    # central difference at high precision: truncation O(h^2) ~ 1e-50, cancellation
    # leaves ~dps - 25 significant digits
    with mp.workdps(dps + 20):
        b = mp.mpf(beta)
        h = mp.mpf(10) ** -25
        d = (kaufman_log_z(L, b + h, dps=dps + 20) - kaufman_log_z(L, b - h, dps=dps + 20)) / (2 * h)
        return float(-d / (L * L))


def onsager_m0(beta: float) -> float:
    """Spontaneous magnetisation per spin of the infinite lattice, beta > beta_c."""
    if beta <= BETA_C:
        return 0.0
    return (1.0 - math.sinh(2.0 * beta) ** -4) ** 0.125


def binned_error(x, nbins: int = 32) -> tuple[float, float]:
    """Mean and its standard error from nbins equal bins (binning analysis)."""
    x = np.asarray(x, dtype=np.float64)
    n = (len(x) // nbins) * nbins
    b = x[len(x) - n:].reshape(nbins, -1).mean(axis=1)
    return float(x[len(x) - n:].mean()), float(b.std(ddof=1) / math.sqrt(nbins))


# ------------------------------------------------- three-dimensional torus
def _all_states3d(dims) -> np.ndarray:
    X, Y, Z = dims
    N = X * Y * Z
    if N > 20:
        raise ValueError("enumeration is for X*Y*Z <= 20")
    idx = np.arange(1 << N, dtype=np.uint32)
    bits = (idx[:, None] >> np.arange(N, dtype=np.uint32)) & 1
    return (1 - 2 * bits.astype(np.int8)).reshape(-1, X, Y, Z)


def _energies3d(s: np.ndarray) -> np.ndarray:
    """H = -sum over the bonds (s, s + e_a), a = x, y, z, of every state in s."""
    s = s.astype(np.int64)
    return -sum((s * np.roll(s, -1, axis=a)).sum(axis=(1, 2, 3)) for a in (1, 2, 3))


def enumerate3d_observables(dims, beta: float) -> dict:
    """<E>/N, <|M|>/N, <m^2>, <m^4>, U4 on the X x Y x Z torus by summing over every state."""
    s = _all_states3d(dims)
    N = int(np.prod(dims))
    E = _energies3d(s).astype(np.float64)
    M = s.astype(np.int64).sum(axis=(1, 2, 3)).astype(np.float64)
    w = np.exp(-beta * (E - E.min()))
    Z = w.sum()
    m2 = (w * (M / N) ** 2).sum() / Z
    m4 = (w * (M / N) ** 4).sum() / Z
    return {"e": (w * E).sum() / Z / N, "abs_m": (w * np.abs(M)).sum() / Z / N, "m2": m2, "m4": m4,
            "binder": 1.0 - m4 / (3.0 * m2 * m2)}


def stationarity_residual3d(dims, beta: float, colour: int, flip_prob) -> float:
    """max |pi P_c - pi| / max pi for one colour-c half-sweep on the X x Y x Z torus.

    P_c flips each site of colour (i+j+k) mod 2 = c independently with probability
    flip_prob(h), h = sigma * (sum of the six neighbours), the other colour fixed.
    """
    X, Y, Z = dims
    s = _all_states3d(dims)
    E = _energies3d(s).astype(np.float64)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    sites = [(i, j, k) for i in range(X) for j in range(Y) for k in range(Z) if (i + j + k) % 2 == colour]
    f = np.empty((s.shape[0], len(sites)))
    for n, (i, j, k) in enumerate(sites):
        nn = (s[:, (i - 1) % X, j, k].astype(np.int64) + s[:, (i + 1) % X, j, k]
              + s[:, i, (j - 1) % Y, k] + s[:, i, (j + 1) % Y, k]
              + s[:, i, j, (k - 1) % Z] + s[:, i, j, (k + 1) % Z])
        h = s[:, i, j, k].astype(np.int64) * nn
        f[:, n] = np.vectorize(flip_prob, otypes=[np.float64])(h)
    bitpos = np.array([(i * Y + j) * Z + k for i, j, k in sites], dtype=np.uint32)
    state_idx = np.arange(s.shape[0], dtype=np.uint32)
    out = np.zeros_like(pi)
    for F in range(1 << len(sites)):
        prob = pi.copy()
        mask = np.uint32(0)
        for n in range(len(sites)):
            if (F >> n) & 1:
                prob *= f[:, n]
                mask |= np.uint32(1) << bitpos[n]
            else:
                prob *= 1.0 - f[:, n]
        np.add.at(out, state_idx ^ mask, prob)
    return float(np.abs(out - pi).max() / pi.max())
