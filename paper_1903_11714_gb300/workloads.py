"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Both the CUDA path's tests/benchmark and the CPU oracle draw their inputs from
here.  The paper runs on synthetic lattices only (Sec. 4: square tori from
(20*128)^2 to (640*128)^2 sites, temperature scans around T_c), so there is no
dataset to stand in for; these five workloads fix the sizes, temperatures,
seeds and start states.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, asdict

import numpy as np

HOT, COLD = 0, 1
BETA_TC = 0.4406868  # ln(1 + sqrt 2) / 2 to 7 digits (Sec. 4.1)

_HERE = os.path.dirname(os.path.abspath(__file__))


@dataclass(frozen=True)
class Lattice:
    L: int
    beta: float
    seed: int
    start: int
    sweeps: int

    def as_dict(self):
        return asdict(self)


def single_small() -> Lattice:
    """L = 128 at beta_c, hot start from seed 1, 1000 sweeps."""
    return Lattice(L=128, beta=BETA_TC, seed=1, start=HOT, sweeps=1000)


def single_large() -> Lattice:
    """L = 65,536 (4.3e9 spins) at beta_c, hot start from seed 2, 200 sweeps."""
    return Lattice(L=65536, beta=BETA_TC, seed=2, start=HOT, sweeps=200)


# Simple-cubic critical coupling from the Monte Carlo literature (Ferrenberg, Xu and
# Landau 2018: 0.221654626), rounded; the 3D workloads run at it.
BETA_C3 = 0.2216546


def cubic_large() -> Lattice:
    """3D single lattice: L = 2048 (2^33 sites, 1 GB of planes, larger than L2) at beta_c of
    the cubic lattice, hot start from seed 3, 100 sweeps."""
    return Lattice(L=2048, beta=BETA_C3, seed=3, start=HOT, sweeps=100)


CUBIC_BINDER_LS = (64, 128, 256)
CUBIC_BINDER_BETA_OVER_BC = (0.996, 0.998, 1.000, 1.002, 1.004)
CUBIC_BINDER_SWEEPS = 100_000


def cubic_binder_scan(sweeps: int = CUBIC_BINDER_SWEEPS) -> list[Lattice]:
    """3D Binder-parameter scan: L = 64, 128, 256 at beta = beta_c * (0.996 ... 1.004),
    cold start, seed 7,000,000 + 100 L + k; burn-in 10 %."""
    out = []
    for L in CUBIC_BINDER_LS:
        for k, f in enumerate(CUBIC_BINDER_BETA_OVER_BC):
            out.append(Lattice(L=L, beta=BETA_C3 * f, seed=7_000_000 + 100 * L + k, start=COLD, sweeps=sweeps))
    return out


def temperature_scan(n: int = 64, L: int = 1024) -> list[Lattice]:
    """n replicas of L = 1024, beta evenly spaced in [0.35, 0.55], cold start,
    seed_r = 3,000,000 + r; 5000 sweeps (a 100-sweep graph replayed 50 times),
    burn-in 500."""
    return [Lattice(L=L, beta=0.35 + r * (0.20 / (n - 1)), seed=3_000_000 + r, start=COLD, sweeps=5000)
            for r in range(n)]


TEMPERATURE_SCAN_BURN_IN = 500
TEMPERATURE_SCAN_GRAPH_SWEEPS = 100


# Binder-parameter scan (a reduced form of the paper's Fig. 3): U4 and <|m|> against
# T/T_c for several L; 10^6 samples per point with the first 10^5 discarded, as in
# the figure's caption.
BINDER_LS = (64, 128, 256, 512)
BINDER_T_OVER_TC = (0.90, 0.94, 0.97, 0.99, 1.00, 1.01, 1.03, 1.06, 1.10)
BINDER_SWEEPS = 1_000_000
BINDER_BURN_IN = 100_000
BETA_C_EXACT = 0.5 * math.log(1.0 + math.sqrt(2.0))


def binder_scan(sweeps: int = BINDER_SWEEPS) -> list[Lattice]:
    """One lattice per (L, T/T_c): beta = beta_c / (T/T_c), cold start, seed from (L, k)."""
    out = []
    for L in BINDER_LS:
        for k, t in enumerate(BINDER_T_OVER_TC):
            out.append(Lattice(L=L, beta=BETA_C_EXACT / t, seed=7_000_000 + 100 * L + k, start=COLD, sweeps=sweeps))
    return out


def _uneven_path() -> str:
    return os.path.join(_HERE, "configs", "uneven_batch_200.json")


def make_uneven_batch(n: int = 200) -> list[dict]:
    """Draws for the uneven batch from numpy's default_rng(4): L = 64 * 2^u with
    u uniform on {0..6}, beta uniform in [0.30, 0.60], 63-bit seeds, hot start,
    500 sweeps."""
    rng = np.random.default_rng(4)
    u = rng.integers(0, 7, size=n)
    beta = rng.uniform(0.30, 0.60, size=n)
    seed = rng.integers(0, 2**63 - 1, size=n, dtype=np.int64)
    return [dict(L=int(64 << int(u[k])), beta=float(beta[k]), seed=int(seed[k]), start=HOT, sweeps=500)
            for k in range(n)]


def uneven_batch() -> list[Lattice]:
    """The committed uneven-batch list (written once by make_uneven_batch)."""
    with open(_uneven_path()) as f:
        return [Lattice(**d) for d in json.load(f)["lattices"]]


@dataclass(frozen=True)
class Request:
    rid: int
    arrival: float  # seconds since start
    L: int
    beta: float
    seed: int
    sweeps: int

    @property
    def flips(self) -> int:
        return self.L * self.L * self.sweeps


def serving_requests(n: int, rate_per_s: float, seed: int = 5) -> list[Request]:
    """Poisson arrivals at rate_per_s; L = 64 * round(e^U[ln 4, ln 128]) (log-uniform
    in [256, 8192], multiple of 64), beta ~ U[0.35, 0.55], sweeps = round(e^U[ln 100,
    ln 1e4]), seed = request id."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0, size=n) / rate_per_s
    Lf = np.exp(rng.uniform(math.log(4), math.log(128), size=n))
    beta = rng.uniform(0.35, 0.55, size=n)
    sw = np.exp(rng.uniform(math.log(100), math.log(10_000), size=n))
    t = np.cumsum(gaps) - gaps[0]
    return [Request(rid=k, arrival=float(t[k]), L=int(64 * round(Lf[k])), beta=float(beta[k]), seed=k,
                    sweeps=int(round(sw[k]))) for k in range(n)]


def mean_request_flips(n: int = 100_000, seed: int = 5) -> float:
    """E[L^2 * sweeps] of the request distribution (for sizing the arrival rate)."""
    rs = serving_requests(n, 1.0, seed)
    return float(np.mean([r.flips for r in rs]))


if __name__ == "__main__":
    os.makedirs(os.path.dirname(_uneven_path()), exist_ok=True)
    with open(_uneven_path(), "w") as f:
        json.dump({"source": "numpy default_rng(4): u ~ integers(0,7), beta ~ uniform(0.30,0.60), "
                             "seed ~ integers(0, 2^63-1); L = 64 << u; hot start; 500 sweeps",
                   "lattices": make_uneven_batch()}, f, indent=0)
    print("wrote", _uneven_path())
