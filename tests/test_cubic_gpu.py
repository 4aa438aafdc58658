"""GPU parity of the three-dimensional sweep (ising_init3d handles) against the 3D
oracle, through the C ABI: lattices and per-sweep (M, E) bit-exact, moments from
exact integer sums, start states, degenerate temperatures, plane layout and
checkpoints.  Sizes span the single-word path (L/64 = 1, 2, 3, 5 words per row)
and the four-word path (L % 256 == 0), up to the benchmark's L = 2048 cube (against
values stored from the oracle) and an L = 1024 cube (against the oracle directly).
"""
import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising

pytestmark = pytest.mark.gpu

BETA_C3 = 0.2216546
REL_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


def run_gpu3d(L, beta, seed, start, sweeps):
    lat = ising.Lattice3D(L, beta, seed, start)
    M0, E0, _ = lat.observables()
    lat.sweep(sweeps)
    M, E = lat.history(0, sweeps)
    s = lat.get_lattice()
    lat.close()
    return s, M, E, (M0, E0)


def assert_chain3d_equal(L, beta, seed, start, sweeps):
    ref, Mr, Er, _ = oracle.run3d((L, L, L), beta, seed, start, sweeps)
    s, M, E, me0 = run_gpu3d(L, beta, seed, start, sweeps)
    assert me0 == oracle.observe3d(oracle.init3d((L, L, L), seed, start))
    assert np.array_equal(M, Mr), f"M differs first at sweep {np.argmax(M != Mr)}"
    assert np.array_equal(E, Er), f"E differs first at sweep {np.argmax(E != Er)}"
    if not np.array_equal(s, ref):
        bad = np.argwhere(s != ref)
        raise AssertionError(f"{len(bad)} sites differ, first {bad[:5].tolist()}")


def test_thresholds3d_match_oracle():
    for beta in np.concatenate([np.linspace(0, 3, 301), [BETA_C3, 200.0]]):
        assert ising.ising_thresholds3d(float(beta)) == oracle.thresholds3d(float(beta))


@pytest.mark.parametrize("L,beta,seed,start,sweeps", [
    (64, BETA_C3, 11, ising.HOT, 12),     # one word per plane row
    (128, 0.18, 12, ising.HOT, 8),        # two words
    (192, 0.3, 13, ising.COLD, 4),        # three words
    (256, BETA_C3, 14, ising.HOT, 4),     # four-word groups
    (320, 0.25, 0xFFFFFFFFFFFFFFFF, ising.HOT, 2),  # five words
    (512, 0.2, 15, ising.HOT, 1),         # eight words
])
def test_cubic_matches_oracle(L, beta, seed, start, sweeps):
    assert_chain3d_equal(L, beta, seed, start, sweeps)


@pytest.mark.parametrize("beta", [0.0, 200.0])
@pytest.mark.parametrize("L", [64, 256])
def test_cubic_degenerate_temperatures(L, beta):
    # beta = 0: T = 2^32, every proposal flips; beta = 200: T = 0, zero-temperature dynamics
    assert_chain3d_equal(L, beta, 5, ising.HOT, 4)


def test_cubic_benchmark_lattice_matches_golden():
    """The benchmark's lattice (L = 2048, 2^33 sites, the launch configuration
    bench.py times): M and E of two sweeps and the final lattice hash, stored by
    tests/golden/make_golden.py from the oracle."""
    import json
    import os

    from paper_1903_11714_gb300 import workloads

    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cubic_L2048_2sweeps.json")))
    cfg = workloads.cubic_large()
    w = g["workload"]
    assert (w["L"], w["beta"], w["seed"], w["start"]) == (cfg.L, cfg.beta, cfg.seed, cfg.start)
    lat = ising.Lattice3D(cfg.L, cfg.beta, cfg.seed, cfg.start).sweep(w["sweeps"])
    M, E = lat.history()
    assert M.tolist() == g["M"] and E.tolist() == g["E"]
    assert oracle.lattice_hash(lat.get_lattice()) == g["sha256"]
    lat.close()


def test_cubic_full_size_one_sweep():
    """An L = 1024 cube (2^30 sites, four-word groups) against the oracle directly."""
    assert_chain3d_equal(1024, BETA_C3, 3, ising.HOT, 1)


def test_cubic_moments_match_oracle():
    L, beta, seed, sweeps, burn = 64, 0.21, 7, 300, 30
    _, Mr, Er, _ = oracle.run3d((L, L, L), beta, seed, oracle.HOT, sweeps)
    ex = oracle.moments_exact(Mr, Er, L ** 3, burn)
    lat = ising.Lattice3D(L, beta, seed, ising.HOT).sweep(sweeps)
    got = lat.moments(burn)
    lat.close()
    for k in ("S1", "S2", "S4", "SE", "SE2"):
        assert got[k] == ex[k], k
    for k in ("abs_m", "m2", "m4", "e", "e2", "binder"):
        assert got[k] == pytest.approx(ex[k], rel=REL_TOL, abs=0), k


def test_cubic_planes_layout_and_restart_from_planes():
    L, beta, seed = 128, 0.2, 8
    lat = ising.Lattice3D(L, beta, seed).sweep(3)
    black, white = lat.get_planes()
    s = lat.get_lattice()
    W = L // 64
    for (i, j, k) in [(0, 0, 0), (0, 0, 1), (1, 0, 0), (5, 77, 3), (127, 127, 127), (64, 3, 100)]:
        c = (i + j + k) & 1
        m = k >> 1
        word = (black if c == 0 else white)[(i * L + j) * W + m // 32]
        assert ((int(word) >> (m % 32)) & 1) == (1 if s[i, j, k] > 0 else 0)
    # a lattice set from these planes continues like the oracle from the same state
    lat2 = ising.Lattice3D(L, beta, seed, ising.COLD)
    lat2.set_planes(black, white)
    assert np.array_equal(lat2.get_lattice(), s)
    M0, E0, n0 = lat2.observables()
    assert (M0, E0, n0) == (*oracle.observe3d(s), 0)
    lat2.sweep(2)
    ref, Mr, Er, _ = oracle.run3d((L, L, L), beta, seed, sweeps=2, state=s)
    M, E = lat2.history()
    assert np.array_equal(lat2.get_lattice(), ref) and np.array_equal(M, Mr) and np.array_equal(E, Er)
    lat.close()
    lat2.close()


def test_cubic_checkpoint_resume_is_bit_exact():
    L, beta, seed = 128, 0.23, 77
    a = ising.Lattice3D(L, beta, seed).sweep(9)
    b = ising.Lattice3D(L, beta, seed).sweep(4)
    blob = b.save()
    b.close()
    c = ising.Lattice.load(blob)
    assert isinstance(c, ising.Lattice3D)
    c.sweep(5)
    assert np.array_equal(a.get_lattice(), c.get_lattice())
    Ma, Ea = a.history()
    Mc, Ec = c.history()
    assert np.array_equal(Ma, Mc) and np.array_equal(Ea, Ec)
    a.close()
    c.close()


def test_cubic_sweep_calls_compose_and_errors():
    L = 64
    a = ising.Lattice3D(L, BETA_C3, 4).sweep(10)
    b = ising.Lattice3D(L, BETA_C3, 4)
    for n in (1, 0, 4, 2, 3):
        b.sweep(n)
    assert np.array_equal(a.get_lattice(), b.get_lattice())
    assert np.array_equal(a.history()[0], b.history()[0])
    with pytest.raises(ising.IsingError) as e:
        b.set_lattice(np.ones((L, L, L), dtype=np.int8))
    assert e.value.code == ising.ISING_EINVAL
    for bad_L in (32, 100, 16384):
        with pytest.raises(ising.IsingError):
            ising.Lattice3D(bad_L, 0.2, 1)
    a.close()
    b.close()


def test_cubic_binder_cumulant_on_either_side_of_beta_c():
    """Physics of the 3D chain: 3 % below beta_c of the cubic lattice (0.2216546) the
    Binder cumulant U4 = 1 - <m^4>/(3<m^2>^2) of L = 64 and 128 is near its disordered
    value 0, 3 % above it near the ordered value 2/3, and there the larger lattice is
    the closer one (2/3 - U4 falls like 1/L^3).  The critical value, ~0.465, lies
    between.  Cold starts, 10^5 sweeps, 10 % burn-in: U4 is known to about +-0.07."""
    sweeps, burn = 100_000, 10_000
    u4 = {}
    for f in (0.97, 1.03):
        for L in (64, 128):
            lat = ising.Lattice3D(L, BETA_C3 * f, 900 + L, ising.COLD).sweep(sweeps)
            u4[(f, L)] = lat.moments(burn)["binder"]
            lat.close()
    assert u4[(0.97, 64)] < 0.3 and u4[(0.97, 128)] < 0.3, u4
    assert u4[(1.03, 128)] > u4[(1.03, 64)] > 0.6, u4
