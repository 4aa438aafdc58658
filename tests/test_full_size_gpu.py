"""GPU parity at the full single-lattice size: L = 65,536 (4.29e9 spins), 200
sweeps, hot start from seed 2, beta = 0.4406868, in the launch configuration the
benchmark times.

* If tests/golden/single_L65536_200sweeps.json (written by the oracle through
  tests/golden/make_golden.py) is present: the final-lattice SHA-256 and all 200
  integer M and E values must match it exactly.
* Always: exact h x w windows of the final lattice from the oracle's light-cone
  evaluator at several places, including both torus seams; packed and int8
  kernels agree bit for bit; M/E invariants.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising, workloads

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "single_L65536_200sweeps.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


@pytest.fixture(scope="module")
def packed_run():
    cfg = workloads.single_large()
    lat = ising.Lattice(cfg.L, cfg.beta, cfg.seed, cfg.start, ising.PACKED)
    specialized = lat.specialized()
    lat.sweep(cfg.sweeps)
    M, E = lat.history()
    s = lat.get_lattice()
    lat.close()
    return cfg, s, M, E, specialized


def test_the_benchmarked_lattice_runs_the_specialised_kernel(packed_run):
    """The default (automatic) mode compiles this lattice's sweep kernel for its
    thresholds -- the kernel the benchmark times -- and the other tests in this file
    check that kernel's chain."""
    specialized, note = packed_run[4]
    assert specialized, note


def test_windows_match_oracle_light_cone(packed_run):
    cfg, s, M, E = packed_run[:4]
    L = cfg.L
    rng = np.random.default_rng(2024)
    spots = [(0, 0), (L - 3, L - 40), (L // 2, 64 * 511 + 7)] + [
        (int(rng.integers(0, L)), int(rng.integers(0, L))) for _ in range(3)]
    h, w = 6, 48
    for i0, j0 in spots:
        win = oracle.window(L, cfg.beta, cfg.seed, cfg.start, cfg.sweeps, i0, j0, h, w)
        rows = [(i0 + a) % L for a in range(h)]
        cols = [(j0 + b) % L for b in range(w)]
        assert np.array_equal(s[np.ix_(rows, cols)], win), (i0, j0)


def test_invariants(packed_run):
    cfg, s, M, E = packed_run[:4]
    N = cfg.L ** 2
    assert np.all(E % 4 == 0) and np.all(np.abs(E) <= 2 * N)
    assert np.all(M % 2 == 0) and np.all(np.abs(M) <= N)
    assert int(s.astype(np.int64).sum()) == M[-1]


def test_matches_golden(packed_run):
    if not os.path.exists(GOLDEN):
        pytest.skip("golden file for L = 65,536 not generated")
    cfg, s, M, E = packed_run[:4]
    g = json.load(open(GOLDEN))
    assert g["workload"] == cfg.as_dict()
    assert M.tolist() == g["M"] and E.tolist() == g["E"]
    assert oracle.lattice_hash(s) == g["sha256"]


def test_int8_kernel_agrees_at_full_size(packed_run):
    cfg, s, M, E = packed_run[:4]
    lat = ising.Lattice(cfg.L, cfg.beta, cfg.seed, cfg.start, ising.INT8)
    lat.sweep(cfg.sweeps)
    M8, E8 = lat.history()
    assert np.array_equal(M8, M) and np.array_equal(E8, E)
    s8 = lat.get_lattice()
    lat.close()
    assert np.array_equal(s8, s)


def test_moments_at_full_magnetisation_of_the_largest_lattice():
    # cold start deep in the ordered phase: M = N = 2^32, so M^2 = 2^64 and M^4 = 2^128
    L = 65536
    lat = ising.Lattice(L, 200.0, 3, ising.COLD, ising.PACKED).sweep(2)  # T = 0: frozen
    M, E = lat.history()
    assert M.tolist() == [L * L, L * L] and E.tolist() == [-2 * L * L, -2 * L * L]
    got = lat.moments(0)
    ex = oracle.moments_exact(M, E, L * L, 0)
    for k in ("S1", "S2", "S4", "SE", "SE2"):
        assert got[k] == ex[k], k
    assert got["binder"] == pytest.approx(2.0 / 3.0, rel=1e-12)
    lat.close()
