"""GPU parity where the Philox call index q = 8 * (plane word) passes 2^32, so that
its high word (counter word 3) is not zero and the kernels form the per-word Philox
constants instead of the per-launch ones: 2D lattices above L = 185,363 and cubes
above L = 3,251 (4.3-4.6 GB of planes each).  The oracle cannot sweep lattices this
large, so it evaluates exact windows of the final state from their light cones
(oracle.window, oracle.window3d), placed on the plane word where q's high word
first becomes 1, at the torus seams and at random places; M and E of the last sweep
are recomputed on the host from the planes by their definitions.  In 2D only
L % 256 == 0 reaches such sizes (four-word groups; other widths stop at L = 102,336,
where every call index is below 2^32); in 3D both the four-word groups and the
single-word path (W odd) are covered.
"""
import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising

pytestmark = pytest.mark.gpu

BC = 0.4406868
BC3 = 0.2216546


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


def popcount(a: np.ndarray) -> int:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    if hasattr(np, "bitwise_count"):
        return int(np.bitwise_count(a).sum(dtype=np.int64))
    table = np.array([bin(v).count("1") for v in range(1 << 16)], dtype=np.uint8)
    return int(table[a.view(np.uint16)].sum(dtype=np.int64))


def first_wide_word(words_per_row: int) -> tuple[int, int]:
    """(row, word) of the first plane word whose call index 8 * (row * W + word) >= 2^32."""
    g = (1 << 32) // 8
    return g // words_per_row, g % words_per_row


# ------------------------------------------------------------------------ 2D
def window_from_planes(black, white, L, i0, j0, h, w):
    """h x w window (torus-wrapped) of the 2D state: site (i, j) of colour c = (i+j)&1
    is bit (j>>1) & 31 of word (j>>1) >> 5 in row i of plane c."""
    W = L // 64
    I, J = np.meshgrid((i0 + np.arange(h)) % L, (j0 + np.arange(w)) % L, indexing="ij")
    k = J >> 1
    idx = I * W + (k >> 5)
    word = np.where(((I + J) & 1) == 0, black[idx], white[idx])
    return np.where((word >> (k & 31)) & 1, 1, -1).astype(np.int8)


def observables_from_planes(black, white, L, chunk=4096):
    """(M, E) by definition: M = sum of spins; E = -(sum over the 2N bonds) = 2 * (number
    of anti-aligned bonds) - 2N, the bonds counted once each from the white sites'
    four black neighbours (up, down, same column pair, horizontal neighbour)."""
    W = L // 64
    N = L * L
    b = black.reshape(L, W)
    wt = white.reshape(L, W)
    ups = popcount(black) + popcount(white)
    anti = 0
    for r0 in range(0, L, chunk):
        r1 = min(L, r0 + chunk)
        rows = np.arange(r0, r1)
        t = wt[r0:r1]
        same = b[r0:r1]
        up = b[(rows - 1) % L]
        dn = b[(rows + 1) % L]
        nxt = np.roll(same, -1, axis=1)
        prv = np.roll(same, 1, axis=1)
        # white target at row i: neighbour k+1 when (i + 1) is odd, else k-1
        odd = (((rows + 1) & 1) == 1)[:, None]
        hz = np.where(odd, (same >> np.uint32(1)) | (nxt << np.uint32(31)),
                      (same << np.uint32(1)) | (prv >> np.uint32(31)))
        anti += popcount(t ^ up) + popcount(t ^ dn) + popcount(t ^ same) + popcount(t ^ hz)
    return 2 * ups - N, 2 * anti - 2 * N


@pytest.mark.parametrize("L,check_me", [
    (185_600, True),    # W = 2900: four-word groups, 2-row tiles
    (272_896, True),    # the largest side (9.3 GB of planes): q's high word reaches 2
])
def test_2d_past_32_bit_call_index(L, check_me):
    seed, sweeps = 7, 2
    W = L // 64
    assert (L * L) // 8 > (1 << 32)
    lat = ising.Lattice(L, BC, seed, ising.HOT, ising.PACKED)
    lat.sweep(sweeps)
    M, E = lat.history()
    black, white = lat.get_planes()
    lat.close()
    r, w = first_wide_word(W)
    jb = 64 * w                              # first column of that word
    rng = np.random.default_rng(L)
    spots = [(0, 0), (L - 3, L - 40), (r - 2, jb - 24), (r, L - 30), (L - 4, jb - 8)] + [
        (int(rng.integers(0, L)), int(rng.integers(0, L))) for _ in range(2)]
    g2 = (2 << 32) // 8                      # first plane word with q's high word 2
    if g2 < L * W:
        spots.append((g2 // W - 1, 64 * (g2 % W) - 24))
    h, w_ = 6, 48
    for i0, j0 in spots:
        win = oracle.window(L, BC, seed, oracle.HOT, sweeps, i0, j0, h, w_)
        got = window_from_planes(black, white, L, i0, j0, h, w_)
        assert np.array_equal(got, win), (L, i0, j0)
    assert np.all(E % 4 == 0) and np.all(np.abs(E) <= 2 * L * L)
    if check_me:
        assert observables_from_planes(black, white, L) == (int(M[-1]), int(E[-1]))


def test_2d_largest_width_not_a_multiple_of_four():
    """L = 102,336 (W = 1599, odd): the largest side whose rows are not a whole number
    of 16-byte units (4-row tiles with 4-row halos fill the 100 KB stage to within 64
    bytes); windows at the seams and M/E of the last sweep."""
    L, seed, sweeps = 102_336, 9, 2
    W = L // 64
    assert W % 2 == 1 and (4 + 8 + 4) * W * 4 <= 100 * 1024 < (4 + 8 + 4) * (W + 2) * 4
    lat = ising.Lattice(L, BC, seed, ising.HOT, ising.PACKED)
    lat.sweep(sweeps)
    M, E = lat.history()
    black, white = lat.get_planes()
    lat.close()
    rng = np.random.default_rng(L)
    spots = [(0, 0), (L - 3, L - 40), (L // 2 + 1, 64 * (W - 1) + 40)] + [
        (int(rng.integers(0, L)), int(rng.integers(0, L))) for _ in range(3)]
    for i0, j0 in spots:
        win = oracle.window(L, BC, seed, oracle.HOT, sweeps, i0, j0, 6, 48)
        assert np.array_equal(window_from_planes(black, white, L, i0, j0, 6, 48), win), (i0, j0)
    assert observables_from_planes(black, white, L) == (int(M[-1]), int(E[-1]))


# ------------------------------------------------------------------------ 3D
def box_from_planes(black, white, L, origin, shape):
    """Box of the 3D state: site (i, j, k) of colour (i+j+k)&1 is bit (k>>1) & 31 of
    word (k>>1) >> 5 in row i*L + j of its plane."""
    W = L // 64
    I, J, K = np.meshgrid(*[(o + np.arange(s)) % L for o, s in zip(origin, shape)], indexing="ij")
    m = K >> 1
    idx = (I * L + J) * W + (m >> 5)
    word = np.where(((I + J + K) & 1) == 0, black[idx], white[idx])
    return np.where((word >> (m & 31)) & 1, 1, -1).astype(np.int8)


def observables3d_from_planes(black, white, L, slabs=32):
    """(M, E) of the cube by definition: E = 2 * (anti-aligned bonds) - 3N, counted from
    the white sites' six black neighbours."""
    W = L // 64
    N = L ** 3
    b = black.reshape(L, L, W)
    wt = white.reshape(L, L, W)
    ups = popcount(black) + popcount(white)
    anti = 0
    for i0 in range(0, L, slabs):
        i1 = min(L, i0 + slabs)
        ii = np.arange(i0, i1)
        t = wt[i0:i1]
        same = b[i0:i1]
        up = b[(ii - 1) % L]
        dn = b[(ii + 1) % L]
        no = np.roll(same, 1, axis=1)            # (i, j-1)
        so = np.roll(same, -1, axis=1)           # (i, j+1)
        nxt = np.roll(same, -1, axis=2)
        prv = np.roll(same, 1, axis=2)
        jj = np.arange(L)
        odd = (((ii[:, None] + jj[None, :] + 1) & 1) == 1)[:, :, None]
        hz = np.where(odd, (same >> np.uint32(1)) | (nxt << np.uint32(31)),
                      (same << np.uint32(1)) | (prv >> np.uint32(31)))
        for n in (up, dn, no, so, same, hz):
            anti += popcount(t ^ n)
    return 2 * ups - N, 2 * anti - 3 * N


@pytest.mark.parametrize("L,check_me", [
    (3328, True),    # W = 52: four-word groups
    (3264, False),   # W = 51: single words
])
def test_3d_past_32_bit_call_index(L, check_me):
    seed, sweeps = 8, 1
    W = L // 64
    assert L ** 3 // 8 > (1 << 32)
    lat = ising.Lattice3D(L, BC3, seed, ising.HOT)
    lat.sweep(sweeps)
    M, E = lat.history()
    black, white = lat.get_planes()
    lat.close()
    r, w = first_wide_word(W)                # row r = i*L + j of the first wide word
    i, j = divmod(r, L)
    kb = 64 * w
    rng = np.random.default_rng(L)
    boxes = [((0, 0, 0), (3, 3, 40)), ((i - 1, j - 1, kb - 20), (3, 3, 48)), ((L - 2, L - 2, L - 20), (4, 4, 40)),
             ((i, j, L - 8), (2, 2, 16))] + [
        (tuple(int(v) for v in rng.integers(0, L, 3)), (3, 3, 24)) for _ in range(2)]
    for origin, shape in boxes:
        want = oracle.window3d((L, L, L), BC3, seed, oracle.HOT, sweeps, origin, shape)
        got = box_from_planes(black, white, L, origin, shape)
        assert np.array_equal(got, want), (L, origin)
    assert np.all(E % 2 == 0) and np.all(np.abs(E) <= 3 * L ** 3)
    if check_me:
        assert observables3d_from_planes(black, white, L) == (int(M[-1]), int(E[-1]))
