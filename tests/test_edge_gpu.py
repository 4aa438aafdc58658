"""Edge cases of the boundary on a GPU, against the oracle: runs of zero sweeps,
a batch holding no lattice, a batch emptied and filled again, and the smallest
sides each layout allows swept through a batch (Sec. 3.1's schedule on the
smallest tori the bit planes and the tiles can hold).  All through the C ABI.
"""
import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising, workloads

pytestmark = pytest.mark.gpu

BC = workloads.BETA_TC


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


def assert_batch_lattice(b, idx, L, beta, seed, start, sweeps):
    ref, Mr, Er, _ = oracle.run(L, beta, seed, start, sweeps)
    M, E = b.history(idx)
    assert len(M) == sweeps
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    assert np.array_equal(b.get_lattice(idx), ref)


@pytest.mark.parametrize("kernel,L", [(ising.PACKED, 64), (ising.PACKED, 512), (ising.PACKED, 16384),
                                      (ising.INT8, 8), (ising.INT8, 96)])
def test_zero_sweeps_leave_the_start_state(kernel, L):
    """sweep(0) changes nothing: the lattice is the oracle's start state, the
    observables are its M and E, no sweep is counted and the history is empty."""
    lat = ising.Lattice(L, BC, 7, ising.HOT, kernel)
    lat.sweep(0)
    start = oracle.init(L, 7, ising.HOT)
    M0, E0, n = lat.observables()
    assert n == 0
    assert (M0, E0) == oracle.observe(start)
    M, E = lat.history(0, 0)
    assert len(M) == 0 and len(E) == 0
    assert np.array_equal(lat.get_lattice(), start)
    lat.close()


def test_batch_with_no_lattice_runs_and_fills_again():
    """A batch with nothing in it runs (plain launches and a captured graph) without
    error; a lattice added afterwards, removed, and another added in its place each
    follow the oracle's chain from their own start."""
    b = ising.Batch(4, 1024, 1 << 24)
    b.run(3)
    b.run(0)
    b.run(4, graph_sweeps=2)
    i = b.add(128, 0.42, 11, ising.HOT, 5)
    b.run(5)
    assert_batch_lattice(b, i, 128, 0.42, 11, ising.HOT, 5)
    b.remove(i)
    b.run(2)
    j = b.add(256, BC, 12, ising.COLD, 6)
    b.run(6, graph_sweeps=3)
    assert_batch_lattice(b, j, 256, BC, 12, ising.COLD, 6)
    b.close()


def test_zero_sweep_batch_run_changes_nothing():
    b = ising.Batch.from_arrays([64, 320], [0.4, 0.5], [13, 14], [ising.HOT, ising.HOT])
    b.run(0)
    for k, L in enumerate((64, 320)):
        assert b.sweeps_done(k) == 0
        assert np.array_equal(b.get_lattice(k), oracle.init(L, 13 + k, ising.HOT))
    b.run(3)
    assert_batch_lattice(b, 0, 64, 0.4, 13, ising.HOT, 3)
    assert_batch_lattice(b, 1, 320, 0.5, 14, ising.HOT, 3)
    b.close()
