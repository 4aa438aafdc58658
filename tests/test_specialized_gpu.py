"""GPU parity of the sweep kernel compiled for a lattice's thresholds.

A packed single handle can sweep with the tiled kernel compiled (NVRTC, at handle
creation) with its thresholds T_2, T_4 as constants, so that each bit plane of the
uniforms is compared with the logic its threshold bits need.  The chain must not
change: with the mode forced on, lattices of every row-width class (words per row
divisible by 4, odd, 2 mod 4) and the degenerate temperatures (beta = 0, where
T = 2^32 and every site flips; beta = 200, where T = 0 and only h <= 0 flips)
match the oracle's lattice and per-sweep M and E, and the built-in kernel's.
"""
import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising

pytestmark = pytest.mark.gpu

CASES = [(320, 0.4406868, 21, ising.HOT, 12),   # W = 5 (odd): one word per thread group
         (384, 0.30, 22, ising.HOT, 9),          # W = 6 (2 mod 4): two words
         (512, 0.55, 23, ising.COLD, 10),        # W = 8: four words
         (1024, 0.4406868, 24, ising.HOT, 25),
         (576, 0.0, 25, ising.HOT, 4),           # T_2 = T_4 = 2^32: every site flips
         (640, 200.0, 26, ising.HOT, 6)]         # T_2 = T_4 = 0: only h <= 0 flips


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()
    yield
    ising.ising_set_specialize(ising.SPECIALIZE_AUTO)


@pytest.mark.parametrize("L,beta,seed,start,sweeps", CASES)
def test_specialised_kernel_matches_oracle_and_built_in(L, beta, seed, start, sweeps):
    ref, Mr, Er, _ = oracle.run(L, beta, seed, start, sweeps)
    got = {}
    for mode in (ising.SPECIALIZE_ALWAYS, ising.SPECIALIZE_OFF):
        ising.ising_set_specialize(mode)
        lat = ising.Lattice(L, beta, seed, start, ising.PACKED)
        spec, note = lat.specialized()
        assert spec == (mode == ising.SPECIALIZE_ALWAYS), note
        lat.sweep(sweeps)
        M, E = lat.history()
        got[mode] = lat.get_lattice()
        lat.close()
        assert np.array_equal(got[mode], ref), (mode, note)
        assert np.array_equal(M, Mr) and np.array_equal(E, Er), mode
    ising.ising_set_specialize(ising.SPECIALIZE_AUTO)


def test_automatic_mode_leaves_small_lattices_built_in():
    ising.ising_set_specialize(ising.SPECIALIZE_AUTO)
    for L in (128, 1024, 8192):
        lat = ising.Lattice(L, 0.44, 1, ising.HOT, ising.PACKED)
        spec, note = lat.specialized()
        lat.close()
        assert not spec and note.startswith("built-in"), (L, note)


def test_specialised_chain_continues_across_calls_and_checkpoints():
    """Sweeps split over several calls, and a checkpoint taken mid-way and resumed
    in a new (again specialised) handle, give the single run's chain."""
    L, beta, seed, n = 768, 0.47, 31, 14
    ising.ising_set_specialize(ising.SPECIALIZE_ALWAYS)
    ref, Mr, Er, _ = oracle.run(L, beta, seed, ising.HOT, n)
    lat = ising.Lattice(L, beta, seed, ising.HOT, ising.PACKED)
    lat.sweep(3).sweep(4)
    blob = lat.save()
    lat.close()
    lat2 = ising.Lattice.load(blob)
    assert lat2.specialized()[0]
    lat2.sweep(n - 7)
    M, E = lat2.history()
    assert np.array_equal(lat2.get_lattice(), ref)
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    lat2.close()
    ising.ising_set_specialize(ising.SPECIALIZE_AUTO)


def test_large_single_handles_take_512_thread_ctas_and_stay_exact():
    """L = 16,384 is the smallest side swept by one 512-thread CTA per SM with tiles of
    32 rows (8,192 words); both its builds (specialised, built-in) match the oracle."""
    L, beta, seed, n = 16384, 0.4406868, 41, 3
    ref, Mr, Er, _ = oracle.run(L, beta, seed, ising.HOT, n)
    for mode in (ising.SPECIALIZE_AUTO, ising.SPECIALIZE_OFF):
        ising.ising_set_specialize(mode)
        lat = ising.Lattice(L, beta, seed, ising.HOT, ising.PACKED)
        assert lat.specialized()[0] == (mode == ising.SPECIALIZE_AUTO)
        lat.sweep(n)
        M, E = lat.history()
        assert np.array_equal(M, Mr) and np.array_equal(E, Er), mode
        assert np.array_equal(lat.get_lattice(), ref), mode
        lat.close()
    ising.ising_set_specialize(ising.SPECIALIZE_AUTO)


def test_batch_of_one_temperature_specialises_until_another_joins():
    """Three lattices at one beta sweep with the multi-lattice kernel compiled for it;
    a fourth at another beta brings back the built-in kernel mid-run (graphs
    re-captured).  Every chain equals the oracle's."""
    ising.ising_set_specialize(ising.SPECIALIZE_ALWAYS)
    beta, other = 0.4406868, 0.31
    specs = [(256, 51, ising.HOT), (320, 52, ising.COLD), (512, 53, ising.HOT)]
    b = ising.Batch(4, 512, 8 << 20, 0)
    idx = [b.add(L, beta, seed, start, 12) for L, seed, start in specs]
    assert b.specialized()
    b.run(6, graph_sweeps=3)
    j = b.add(384, other, 54, ising.HOT, 12)
    assert not b.specialized()
    b.run(6, graph_sweeps=3)
    b.synchronize()
    for (L, seed, start), i in zip(specs, idx):
        ref, Mr, Er, _ = oracle.run(L, beta, seed, start, 12)
        M, E = b.history(i)
        assert np.array_equal(M, Mr) and np.array_equal(E, Er), L
        assert np.array_equal(b.get_lattice(i), ref), L
    ref, Mr, Er, _ = oracle.run(384, other, 54, ising.HOT, 6)
    M, E = b.history(j)
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    assert np.array_equal(b.get_lattice(j), ref)
    b.remove(j)
    assert b.specialized()  # one temperature again
    b.close()
    ising.ising_set_specialize(ising.SPECIALIZE_AUTO)


def test_automatic_mode_leaves_small_batches_built_in():
    ising.ising_set_specialize(ising.SPECIALIZE_AUTO)
    b = ising.Batch.from_arrays([1024] * 4, [0.44] * 4, [1, 2, 3, 4], [ising.HOT] * 4)
    assert not b.specialized()
    b.close()


@pytest.mark.parametrize("L,beta,seed,sweeps", [(64, 0.2216546, 61, 5),    # one word per row: one-word groups
                                                 (256, 0.2216546, 62, 3),   # four-word groups
                                                 (128, 0.0, 63, 2),         # T = 2^32: every site flips
                                                 (192, 200.0, 64, 3)])      # T = 0: only h <= 0 flips
def test_cubic_specialised_kernel_matches_oracle(L, beta, seed, sweeps):
    """The 3D sweep compiled for its three thresholds gives the oracle's cube and M, E."""
    ising.ising_set_specialize(ising.SPECIALIZE_ALWAYS)
    ref, Mr, Er, _ = oracle.run3d((L, L, L), beta, seed, oracle.HOT, sweeps)
    lat = ising.Lattice3D(L, beta, seed, ising.HOT)
    spec, note = lat.specialized()
    assert spec, note
    lat.sweep(sweeps)
    M, E = lat.history()
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    assert np.array_equal(lat.get_lattice(), ref)
    lat.close()
    ising.ising_set_specialize(ising.SPECIALIZE_AUTO)
