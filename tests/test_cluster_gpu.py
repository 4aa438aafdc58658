"""GPU parity of the cluster-resident batch sweep (a batch of lattices of one side
L <= 4096 kept in the shared memory of one thread-block cluster each for a whole run).

Every lattice must reach the chain it reaches on the tiled kernel and alone: the
same lattice, M and E as the same batch with clusters switched off, and as the
oracle where the oracle is quick.
"""
import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


def make(L, betas, seeds, starts, limits, mode):
    arena = sum(L * L // 8 + 16 * n + 4096 for n in limits)
    b = ising.Batch(len(betas), L, arena)
    b.set_cluster(mode)
    idx = [b.add(L, be, s, st, n) for be, s, st, n in zip(betas, seeds, starts, limits)]
    return b, idx


def both(L, betas, seeds, starts, limits, runs):
    """The same batch on the cluster path (forced) and on the tiled kernel."""
    out = []
    for mode in (ising.CLUSTER_ALWAYS, ising.CLUSTER_OFF):
        b, idx = make(L, betas, seeds, starts, limits, mode)
        C = b.cluster_size()
        for n in runs:
            b.run(n)
        b.synchronize()
        res = [(b.history(i), b.get_lattice(i), b.sweeps_done(i)) for i in idx]
        b.close()
        out.append((C, res))
    return out


@pytest.mark.parametrize("L", [64, 128, 192, 320, 512, 1024, 2048, 4096])
def test_cluster_matches_tiled(L):
    n = 4
    betas = [0.0, 0.3, 0.4406868, 1.5][:n]
    seeds = [11 + 7 * k for k in range(n)]
    starts = [ising.HOT, ising.COLD, ising.HOT, ising.HOT][:n]
    limits = [40] * n
    (Cc, rc), (Ct, rt) = both(L, betas, seeds, starts, limits, [7, 13])
    assert Cc > 0 and Ct == 0
    for k in range(n):
        (Mc, Ec), sc, dc = rc[k]
        (Mt, Et), st, dt = rt[k]
        assert dc == dt == 20
        assert np.array_equal(Mc, Mt) and np.array_equal(Ec, Et), k
        assert np.array_equal(sc, st), k


@pytest.mark.parametrize("L", [64, 256])
def test_cluster_matches_oracle(L):
    betas = [0.25, 0.4406868, 0.6]
    seeds = [3, 4, 5]
    starts = [ising.HOT, ising.COLD, ising.HOT]
    b, idx = make(L, betas, seeds, starts, [30, 30, 30], ising.CLUSTER_ALWAYS)
    assert b.cluster_size() > 0
    b.run(9)
    b.run(16)
    b.synchronize()
    for k, i in enumerate(idx):
        ref, Mr, Er, _ = oracle.run(L, betas[k], seeds[k], starts[k], 25)
        M, E = b.history(i)
        assert np.array_equal(M, Mr) and np.array_equal(E, Er), k
        assert np.array_equal(b.get_lattice(i), ref), k
    b.close()


def test_cluster_sweep_limits():
    """Each lattice stops at its own limit inside the one launch; later runs skip it."""
    L = 256
    betas = [0.3, 0.44, 0.5, 0.9]
    seeds = [21, 22, 23, 24]
    starts = [ising.HOT] * 4
    limits = [5, 12, 30, 1]
    (Cc, rc), (_, rt) = both(L, betas, seeds, starts, limits, [8, 8, 8, 8])
    assert Cc > 0
    for k in range(4):
        (Mc, Ec), sc, dc = rc[k]
        (Mt, Et), st, dt = rt[k]
        assert dc == dt == limits[k]
        assert np.array_equal(Mc, Mt) and np.array_equal(Ec, Et) and np.array_equal(sc, st), k
        ref, Mr, Er, _ = oracle.run(L, betas[k], seeds[k], starts[k], limits[k])
        assert np.array_equal(Mc, Mr) and np.array_equal(sc, ref), k


def test_cluster_long_run_in_chunks():
    """A run longer than one launch's 4,096 sweeps continues the chain exactly."""
    L = 64
    b, idx = make(L, [0.44, 0.2], [1, 2], [ising.HOT, ising.COLD], [5000, 5000], ising.CLUSTER_ALWAYS)
    assert b.cluster_size() > 0
    b.run(4100)
    b.synchronize()
    for k, i in enumerate(idx):
        ref, Mr, Er, _ = oracle.run(L, [0.44, 0.2][k], [1, 2][k], [ising.HOT, ising.COLD][k], 4100)
        M, E = b.history(i)
        assert np.array_equal(M, Mr) and np.array_equal(E, Er), k
        assert np.array_equal(b.get_lattice(i), ref), k
    b.close()


def test_cluster_choice_follows_the_table():
    """Mixed sides fall back to the tiled kernel; removing the odd one brings the
    cluster form back, and a removed slot is skipped."""
    b = ising.Batch(4, 512, 4 * (512 * 512 // 8 + 16 * 64 + 4096))
    b.set_cluster(ising.CLUSTER_ALWAYS)
    a0 = b.add(256, 0.4, 1, ising.HOT, 64)
    a1 = b.add(512, 0.4, 2, ising.HOT, 64)
    a2 = b.add(256, 0.5, 3, ising.HOT, 64)
    assert b.cluster_size() == 0
    b.run(3)
    b.remove(a1)
    assert b.cluster_size() > 0
    b.run(6)
    b.synchronize()
    for i, (beta, seed) in ((a0, (0.4, 1)), (a2, (0.5, 3))):
        ref, Mr, Er, _ = oracle.run(256, beta, seed, ising.HOT, 9)
        M, E = b.history(i)
        assert np.array_equal(M, Mr) and np.array_equal(E, Er)
        assert np.array_equal(b.get_lattice(i), ref)
    b.set_cluster(ising.CLUSTER_OFF)
    assert b.cluster_size() == 0
    b.close()


def test_automatic_choice_for_the_scan():
    """The 64-replica scan at L = 1024 takes the cluster form by default, and a
    single lattice of L = 4096 (16 CTAs, far fewer than the SMs) does not."""
    reps = workloads.temperature_scan()
    b = ising.Batch(len(reps), 1024, sum(r.L * r.L // 8 + 16 * 8 + 4096 for r in reps))
    for r in reps:
        b.add(r.L, r.beta, r.seed, r.start, 8)
    assert b.cluster_size() > 0
    b.close()
    b = ising.Batch(1, 4096, 4096 * 4096 // 8 + 16 * 8 + 4096)
    b.add(4096, 0.44, 1, ising.HOT, 8)
    assert b.cluster_size() == 0
    b.close()


@pytest.mark.parametrize("count", [200, 2000])
def test_cluster_packed_and_in_waves(count):
    """More lattices than SMs: 256-thread CTAs several to an SM (200 lattices), and one
    CTA per lattice in waves when not every cluster can be resident (2000)."""
    L = 64
    rng = np.random.default_rng(count)
    betas = list(rng.uniform(0.1, 0.9, count))
    seeds = [1000 + k for k in range(count)]
    starts = [ising.HOT if k % 3 else ising.COLD for k in range(count)]
    (Cc, rc), (_, rt) = both(L, betas, seeds, starts, [12] * count, [5, 4])
    assert Cc > 0
    for k in range(count):
        (Mc, Ec), sc, dc = rc[k]
        (Mt, Et), st, dt = rt[k]
        assert dc == dt == 9
        assert np.array_equal(Mc, Mt) and np.array_equal(Ec, Et) and np.array_equal(sc, st), k
    for k in (0, count - 1):
        ref, Mr, Er, _ = oracle.run(L, betas[k], seeds[k], starts[k], 9)
        assert np.array_equal(rc[k][0][0], Mr) and np.array_equal(rc[k][1], ref), k
