"""GPU parity: the CUDA path against the CPU oracle, through the C ABI.

The bar is bit-exactness: the chain is integer-valued (spins, Philox words,
integer thresholds, integer M and E), so lattices and per-sweep M/E must be
identical; FP64 moments derived from exact integer sums must agree with the
oracle's exact-rational values to 1e-12 relative.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising, workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BC = workloads.BETA_TC
REL_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


def run_gpu(L, beta, seed, start, sweeps, kernel):
    lat = ising.Lattice(L, beta, seed, start, kernel)
    M0, E0, _ = lat.observables()
    lat.sweep(sweeps)
    M, E = lat.history(0, sweeps)
    s = lat.get_lattice()
    lat.close()
    return s, M, E, (M0, E0)


def assert_chain_equal(L, beta, seed, start, sweeps, kernel):
    ref, Mr, Er, _ = oracle.run(L, beta, seed, start, sweeps)
    s, M, E, (M0, E0) = run_gpu(L, beta, seed, start, sweeps, kernel)
    assert (M0, E0) == oracle.observe(oracle.init(L, seed, start))
    assert np.array_equal(M, Mr), f"M differs first at sweep {np.argmax(M != Mr)}"
    assert np.array_equal(E, Er), f"E differs first at sweep {np.argmax(E != Er)}"
    if not np.array_equal(s, ref):
        bad = np.argwhere(s != ref)
        raise AssertionError(f"{len(bad)} sites differ, first {bad[:5].tolist()}")


# ------------------------------------------------------------------ Philox
def test_device_philox_matches_oracle():
    import torch

    key = 0x0123456789ABCDEF
    for ctr in [(0, 0, 0, 0), (7, 0, 123, 1), (0xFFFFFFF0, 0, 0xFFFFFFFF, 0), (5, 3, 9, 0x80000001)]:
        n = 64
        out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
        ising.ising_dev_philox(key, ctr, n, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        for b in range(n):
            q = ((ctr[1] << 32) | ctr[0]) + b
            want = oracle.philox4x32_10((q & 0xFFFFFFFF, q >> 32, ctr[2], ctr[3]), (key & 0xFFFFFFFF, key >> 32))
            assert tuple(int(v) for v in got[4 * b:4 * b + 4]) == want, (ctr, b)


# ------------------------------------------------------ single lattice, small
def test_single_small_matches_golden():
    g = json.load(open(os.path.join(GOLDEN, "single_L128_1000sweeps.json")))
    w = g["workload"]
    for kernel in (ising.PACKED, ising.INT8):
        s, M, E, _ = run_gpu(w["L"], w["beta"], w["seed"], w["start"], w["sweeps"], kernel)
        assert oracle.lattice_hash(s) == g["sha256"], kernel
        assert M.tolist() == g["M"] and E.tolist() == g["E"], kernel


@pytest.mark.parametrize("L,beta,seed,start,sweeps", [
    (64, BC, 11, 0, 30),          # one word per plane row, halo blocks of 4 rows
    (128, 0.3, 12, 0, 25),
    (192, 0.6, 13, 1, 20),        # W = 3: not a multiple of 4
    (256, BC, 14, 0, 15),         # W = 4: single-row halos
    (320, 0.45, 15, 0, 12),       # W = 5
    (384, 0.41, 18, 0, 10),       # W = 6: word pairs
    (512, 0.5, 16, 1, 10),
    (1024, BC, 17, 0, 6),
    (2048, 0.35, 0xFFFFFFFFFFFFFFFF, 0, 3),
])
def test_packed_matches_oracle(L, beta, seed, start, sweeps):
    assert_chain_equal(L, beta, seed, start, sweeps, ising.PACKED)


@pytest.mark.parametrize("L,beta,seed,start,sweeps", [
    (8, BC, 21, 0, 200),
    (16, 0.3, 22, 0, 100),
    (24, 0.6, 23, 1, 50),
    (64, BC, 24, 0, 30),
    (136, 0.45, 25, 0, 20),
    (1000, BC, 26, 0, 5),
])
def test_int8_matches_oracle(L, beta, seed, start, sweeps):
    assert_chain_equal(L, beta, seed, start, sweeps, ising.INT8)


@pytest.mark.parametrize("kernel", [ising.PACKED, ising.INT8])
@pytest.mark.parametrize("beta", [0.0, 200.0])
def test_degenerate_temperatures(kernel, beta):
    # beta = 0: T = 2^32, every proposal flips; beta = 200: T = 0, zero-temperature dynamics
    assert_chain_equal(128, beta, 5, 0, 8, kernel)


@pytest.mark.parametrize("L", [64, 128, 192, 256])
def test_resident_small_lattice_equals_tiled_batch(L):
    """Single handles of L <= 256 keep the lattice in one CTA's shared memory; the
    batch runs the same lattice through the tiled kernel.  Same chain."""
    beta, seed, sweeps = 0.43, 40 + L, 300
    a = ising.Lattice(L, beta, seed, ising.HOT).sweep(sweeps)
    b = ising.Batch(1, L, L * L // 8 + 16 * sweeps + 4096)
    i = b.add(L, beta, seed, ising.HOT, sweeps)
    b.run(sweeps)
    Ma, Ea = a.history()
    Mb, Eb = b.history(i)
    assert np.array_equal(Ma, Mb) and np.array_equal(Ea, Eb)
    assert np.array_equal(a.get_lattice(), b.get_lattice(i))
    a.close()
    b.close()


def test_packed_and_int8_agree_mid_size():
    a = run_gpu(768, 0.43, 99, 0, 40, ising.PACKED)
    b = run_gpu(768, 0.43, 99, 0, 40, ising.INT8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


# ------------------------------------------------------------ handle features
def test_set_lattice_then_sweep_matches_oracle():
    L, beta, seed = 256, 0.47, 31
    rng = np.random.default_rng(3)
    start = np.where(rng.random((L, L)) < 0.3, 1, -1).astype(np.int8)
    ref, Mr, Er, _ = oracle.run(L, beta, seed, sweeps=9, state=start)
    for kernel in (ising.PACKED, ising.INT8):
        lat = ising.Lattice(L, beta, seed, ising.COLD, kernel)
        lat.set_lattice(start)
        assert np.array_equal(lat.get_lattice(), start)
        M0, E0, n0 = lat.observables()
        assert (M0, E0, n0) == (*oracle.observe(start), 0)
        lat.sweep(9)
        M, E = lat.history()
        assert np.array_equal(lat.get_lattice(), ref) and np.array_equal(M, Mr) and np.array_equal(E, Er)
        lat.close()


def test_set_lattice_rejects_non_spins():
    lat = ising.Lattice(64, 0.4, 1)
    bad = np.ones((64, 64), dtype=np.int8)
    bad[3, 4] = 0
    with pytest.raises(ising.IsingError) as e:
        lat.set_lattice(bad)
    assert e.value.code == ising.ISING_EINVAL
    lat.close()


def test_planes_roundtrip_layout():
    L = 128
    lat = ising.Lattice(L, 0.44, 8)
    lat.sweep(3)
    black, white = lat.get_planes()
    s = lat.get_lattice()
    W = L // 64
    for (i, j) in [(0, 0), (0, 1), (1, 0), (5, 77), (127, 127), (64, 3)]:
        c = (i + j) & 1
        k = j >> 1
        word = (black if c == 0 else white)[i * W + k // 32]
        assert ((int(word) >> (k % 32)) & 1) == (1 if s[i, j] > 0 else 0)
    lat2 = ising.Lattice(L, 0.44, 8, ising.COLD)
    lat2.set_planes(black, white)
    assert np.array_equal(lat2.get_lattice(), s)
    lat.close()
    lat2.close()


@pytest.mark.parametrize("kernel", [ising.PACKED, ising.INT8])
def test_checkpoint_resume_is_bit_exact(kernel):
    L, beta, seed = 256, 0.41, 77
    a = ising.Lattice(L, beta, seed, ising.HOT, kernel).sweep(12)
    b = ising.Lattice(L, beta, seed, ising.HOT, kernel).sweep(5)
    blob = b.save()
    b.close()
    c = ising.Lattice.load(blob)
    c.sweep(7)
    assert np.array_equal(a.get_lattice(), c.get_lattice())
    Ma, Ea = a.history()
    Mc, Ec = c.history()
    assert np.array_equal(Ma, Mc) and np.array_equal(Ea, Ec)
    a.close()
    c.close()


def test_sweep_calls_compose():
    L = 256
    a = ising.Lattice(L, BC, 4).sweep(10)
    b = ising.Lattice(L, BC, 4)
    for n in (1, 0, 4, 2, 3):
        b.sweep(n)
    assert np.array_equal(a.get_lattice(), b.get_lattice())
    assert np.array_equal(a.history()[0], b.history()[0])


def test_history_grows_past_initial_capacity():
    L = 64
    ref, Mr, Er, _ = oracle.run(L, 0.44, 3, oracle.HOT, 2500)
    lat = ising.Lattice(L, 0.44, 3).sweep(2500)
    M, E = lat.history()
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    lat.close()


def test_history_range_errors():
    lat = ising.Lattice(64, 0.44, 3).sweep(5)
    with pytest.raises(ising.IsingError):
        lat.history(3, 5)
    with pytest.raises(ising.IsingError):
        lat.moments(5)
    # ranges and sweep counts whose sums wrap a signed 64-bit integer are refused
    # before any copy or launch
    big = (1 << 63) - 3
    lib = ising.lib()
    assert lib.ising_history(lat.h, big, 5, None, None) == ising.ISING_EINVAL
    assert lib.ising_history(lat.h, 2, big, None, None) == ising.ISING_EINVAL
    assert lib.ising_sweep(lat.h, (1 << 63) - 1) == ising.ISING_EINVAL
    assert lib.ising_sweep(lat.h, 0xFFFFFFFE - 4) == ising.ISING_EINVAL
    assert lat.observables()[2] == 5
    lat.close()


# ------------------------------------------------------------------ moments
@pytest.mark.parametrize("kernel", [ising.PACKED, ising.INT8])
def test_moments_match_oracle(kernel):
    L, beta, seed, sweeps, burn = 128, 0.42, 5, 400, 40
    _, Mr, Er, _ = oracle.run(L, beta, seed, oracle.HOT, sweeps)
    ex = oracle.moments_exact(Mr, Er, L * L, burn)
    lat = ising.Lattice(L, beta, seed, ising.HOT, kernel).sweep(sweeps)
    got = lat.moments(burn)
    lat.close()
    for k in ("S1", "S2", "S4", "SE", "SE2"):
        assert got[k] == ex[k], k
    for k in ("abs_m", "m2", "m4", "e", "e2", "binder"):
        assert got[k] == pytest.approx(ex[k], rel=REL_TOL, abs=0), k


def test_moments_exact_at_full_magnetisation():
    # cold start at large beta: M = N on (almost) every sweep, so M^4 = L^8 tests the wide sums
    L = 1024
    lat = ising.Lattice(L, 3.0, 1, ising.COLD).sweep(20)
    M, E = lat.history()
    got = lat.moments(0)
    ex = oracle.moments_exact(M, E, L * L, 0)
    for k in ("S1", "S2", "S4", "SE", "SE2"):
        assert got[k] == ex[k], k
    assert got["binder"] == pytest.approx(ex["binder"], rel=REL_TOL)
    lat.close()
