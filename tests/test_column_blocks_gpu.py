"""GPU parity of column-block tiles: tiles of a few rows by CW < W words, each source
row staged with 4 halo words on either side (wrapped round the row at its ends).
Lattices whose rows are too long for whole-row tiles (W = L/64 > 4,264) are swept
this way; here the blocks are also forced on small lattices through
ising_batch_add_tiled, so that the oracle can check whole chains: every block
position (first, inner, last, both at once), several block widths and heights, and
the largest side, L = 2^20 (128 GB of planes), whose windows come from the oracle's
light cones.
"""
import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising

pytestmark = pytest.mark.gpu

BC = 0.4406868


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


# (L, beta, seed, start, sweeps, tile_rows, tile_words)
CASES = [
    (512, BC, 41, ising.HOT, 8, 2, 4),      # W = 8: two blocks, each touching a row end
    (768, 0.3, 42, ising.HOT, 6, 4, 4),     # W = 12: first, inner and last block
    (1024, 0.6, 43, ising.COLD, 5, 8, 8),   # W = 16, taller tiles
    (1024, BC, 44, ising.HOT, 5, 2, 4),     # W = 16: four blocks
    (1280, 0.45, 45, ising.HOT, 4, 16, 4),  # W = 20: five blocks
    (1536, 0.2, 46, ising.HOT, 3, 2, 8),    # W = 24: three blocks
]


def test_column_blocks_match_oracle():
    cases = CASES
    b = ising.Batch(len(cases), 2048, 64 << 20, 0)
    ids = [b.add(L, be, s, st, n, tile_rows=tr, tile_words=cw) for (L, be, s, st, n, tr, cw) in cases]
    b.run(max(c[4] for c in cases))
    b.synchronize()
    for k, (L, be, s, st, n, tr, cw) in zip(ids, cases):
        ref, Mr, Er, _ = oracle.run(L, be, s, st, n)
        M, E = b.history(k, 0, n)
        assert np.array_equal(M, Mr) and np.array_equal(E, Er), (L, tr, cw)
        assert np.array_equal(b.get_lattice(k), ref), (L, tr, cw)
    b.close()


@pytest.mark.parametrize("beta", [0.0, 200.0])
def test_column_blocks_degenerate_temperatures(beta):
    L, n = 512, 4
    b = ising.Batch(1, 512, 8 << 20, 0)
    k = b.add(L, beta, 5, ising.HOT, n, tile_rows=2, tile_words=4)
    b.run(n)
    b.synchronize()
    ref, Mr, Er, _ = oracle.run(L, beta, 5, ising.HOT, n)
    M, E = b.history(k, 0, n)
    assert np.array_equal(b.get_lattice(k), ref) and np.array_equal(M, Mr) and np.array_equal(E, Er)
    b.close()


def test_column_block_requests_are_checked():
    b = ising.Batch(4, 2048, 64 << 20, 0)
    for L, tr, cw in [(1024, 2, 6),      # not a multiple of 4
                      (1024, 2, 12),     # does not divide W = 16
                      (1088, 4, 4),      # W = 17: rows not 16-byte units, no blocks
                      (1024, 3, 8)]:     # tile height not a power of two
        with pytest.raises(ising.IsingError) as e:
            b.add(L, BC, 1, ising.HOT, 2, tile_rows=tr, tile_words=cw)
        assert e.value.code == ising.ISING_EINVAL, (L, tr, cw)
    # whole rows named explicitly are whole-row tiles
    k = b.add(1024, BC, 1, ising.HOT, 2, tile_rows=4, tile_words=16)
    b.run(2)
    b.synchronize()
    ref, _, _, _ = oracle.run(1024, BC, 1, ising.HOT, 2)
    assert np.array_equal(b.get_lattice(k), ref)
    b.close()


def test_get_rows_matches_get_lattice():
    lat = ising.Lattice(256, BC, 3, ising.HOT).sweep(3)
    s = lat.get_lattice()
    assert np.array_equal(lat.get_rows(0, 256), s)
    assert np.array_equal(lat.get_rows(250, 6), s[250:256])
    assert lat.get_rows(17, 0).shape == (0, 256)
    for row0, n in [(-1, 2), (255, 2), (0, 257)]:
        with pytest.raises(ising.IsingError):
            lat.get_rows(row0, n)
    lat.close()
    cube = ising.Lattice3D(64, 0.22, 4, ising.HOT).sweep(1)
    c = cube.get_lattice()
    assert np.array_equal(cube.get_rows(64 * 5 + 7, 3), c.reshape(64 * 64, 64)[64 * 5 + 7: 64 * 5 + 10])
    cube.close()


def window_via_rows(lat, L, i0, j0, h, w):
    rows = lat.get_rows(i0, h) if i0 + h <= L else np.concatenate(
        [lat.get_rows(i0, L - i0), lat.get_rows(0, i0 + h - L)])
    return rows[:, [(j0 + b) % L for b in range(w)]]


@pytest.mark.parametrize("L", [
    273_152,      # the first side beyond whole-row tiles: W = 4268, blocks of 388 words
    1 << 20,      # the largest side: W = 16384, blocks of 1,024 words, 128 GB of planes
])
def test_largest_sides_in_column_blocks(L):
    seed, sweeps = 12, 1
    W = L // 64
    lat = ising.Lattice(L, BC, seed, ising.HOT, ising.PACKED)
    lat.sweep(sweeps)
    M, E = lat.history()
    rng = np.random.default_rng(L)
    # windows over block edges (block widths 388 and 1,024 words are multiples of 4),
    # the torus seams, and the plane words where the Philox call index's high word
    # changes (q = 8 * word)
    cw = 388 if W == 4268 else 1024
    spots = [(0, 0), (L - 3, L - 40), (L // 2, 64 * cw - 24), (1, 64 * (W - cw) - 24)]
    for hi in (1, 2, 7, 31):
        g = (hi << 32) // 8
        if g < L * W:
            spots.append((g // W, 64 * (g % W) - 24))
    spots += [(int(rng.integers(0, L - 6)), int(rng.integers(0, L))) for _ in range(2)]
    for i0, j0 in spots:
        want = oracle.window(L, BC, seed, oracle.HOT, sweeps, i0, j0, 6, 48)
        assert np.array_equal(window_via_rows(lat, L, i0, j0, 6, 48), want), (L, i0, j0)
    assert np.all(E % 4 == 0) and np.all(np.abs(E) <= 2 * L * L) and np.all(np.abs(M) <= L * L)
    if L < (1 << 20):
        # M and E of the sweep by their definitions, from the planes (9.3 GB)
        from test_wide_index_gpu import observables_from_planes
        black, white = lat.get_planes()
        assert observables_from_planes(black, white, L) == (int(M[-1]), int(E[-1]))
    lat.close()
