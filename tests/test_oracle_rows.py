"""Pins the oracle's row-band forms (``init_rows``, ``half_sweep_rows``) to the
whole-lattice chain, which the other oracle tests pin to exact results.

The row-band forms are what the CPU baseline times on a bounded sample of a
lattice too large to sweep on the host, so a mistake in them (a band edge that
does not wrap round the torus, a row offset, a wrong colour or sweep in the
keying) would silently change the work that is timed.  These checks use only
the whole-lattice oracle (``init``, ``run``, ``observe``) as the reference:

* the start state of any band, including bands that start at a negative row or
  run past row L - 1, equals the matching rows of the whole start state;
* a half-sweep of colour c changes only the colour-c sites (Sec. 3.1), so one
  whole sweep of ``run`` gives the expected state after each half: black sites
  from after the sweep, white sites from before it (colour 0), then every site
  from after the sweep (colour 1);
* bands that tile the torus in any order, wrapping ones included, give the
  whole half-sweep, and the returned energy changes add up to the recomputed
  change of H (Sec. 3);
* a single band leaves every row outside it untouched.
"""
import numpy as np
import pytest

import oracle
from oracle import exact

BETA_C = exact.BETA_C


def _colour_mask(L):
    i, j = np.indices((L, L))
    return ((i + j) & 1).astype(np.int8)


def _after_black(before, after_sweep):
    """State after the colour-0 half-sweep: black from after the whole sweep, white unchanged."""
    black = _colour_mask(before.shape[0]) == 0
    return np.where(black, after_sweep, before)


@pytest.mark.parametrize("L", [64, 72, 128])
@pytest.mark.parametrize("start", [oracle.HOT, oracle.COLD])
def test_init_rows_over_all_rows_equals_init(L, start):
    full = oracle.init(L, 11 + L, start)
    s = np.zeros((L, L), dtype=np.int8)
    oracle.init_rows(s, 11 + L, start, 0, L)
    np.testing.assert_array_equal(s, full)


@pytest.mark.parametrize("L", [64, 72, 128])
@pytest.mark.parametrize("row0,nrows", [(-5, 9), (-1, 1), (3, 17), (0, 1)])
def test_init_rows_band_equals_matching_rows(L, row0, nrows):
    seed = 77
    full = oracle.init(L, seed, oracle.HOT)
    s = np.zeros((L, L), dtype=np.int8)
    oracle.init_rows(s, seed, oracle.HOT, row0, nrows)
    rows = [(row0 + a) % L for a in range(nrows)]
    np.testing.assert_array_equal(s[rows], full[rows])
    others = sorted(set(range(L)) - set(rows))
    assert not s[others].any(), "rows outside the band were written"


def test_init_rows_band_past_the_last_row_wraps():
    L, seed = 64, 5
    full = oracle.init(L, seed, oracle.HOT)
    s = np.zeros((L, L), dtype=np.int8)
    oracle.init_rows(s, seed, oracle.HOT, L - 3, 7)
    rows = [61, 62, 63, 0, 1, 2, 3]
    np.testing.assert_array_equal(s[rows], full[rows])


@pytest.mark.parametrize("L", [64, 72, 128])
@pytest.mark.parametrize("sweep0", [0, 3])
def test_two_half_sweeps_over_all_rows_equal_one_sweep(L, sweep0):
    beta, seed = BETA_C, 1000 + L
    before = oracle.run(L, beta, seed, oracle.HOT, sweeps=sweep0)[0] if sweep0 else oracle.init(L, seed)
    after, M, E, _ = oracle.run(L, beta, seed, sweeps=1, sweep0=sweep0, state=before)
    _, e0 = oracle.observe(before)
    s = before.copy()
    d0 = oracle.half_sweep_rows(s, 0, beta, seed, sweep0, 0, L)
    np.testing.assert_array_equal(s, _after_black(before, after))
    _, e_mid = oracle.observe(s)
    assert d0 == e_mid - e0
    d1 = oracle.half_sweep_rows(s, 1, beta, seed, sweep0, 0, L)
    np.testing.assert_array_equal(s, after)
    assert (int(M[0]), int(E[0])) == oracle.observe(s)
    assert d0 + d1 == int(E[0]) - e0


@pytest.mark.parametrize("L", [64, 72, 128])
@pytest.mark.parametrize("cuts", [(0, 20, 41), (-7, 13, 30), (5, 6, 50)])
def test_bands_tiling_the_torus_give_the_whole_sweep(L, cuts):
    """Bands [a_k, a_{k+1}) mod L covering every row once, swept in reverse order."""
    beta, seed, sweep = 0.43, 31 + L, 2
    before, _, _, _ = oracle.run(L, beta, seed, oracle.HOT, sweeps=sweep)
    after, _, E, _ = oracle.run(L, beta, seed, sweeps=1, sweep0=sweep, state=before)
    _, e0 = oracle.observe(before)
    edges = list(cuts) + [cuts[0] + L]
    bands = [(edges[k], edges[k + 1] - edges[k]) for k in range(len(cuts))]
    s = before.copy()
    dE = 0
    for c in (0, 1):
        for row0, n in reversed(bands):
            dE += oracle.half_sweep_rows(s, c, beta, seed, sweep, row0, n)
        if c == 0:
            np.testing.assert_array_equal(s, _after_black(before, after))
    np.testing.assert_array_equal(s, after)
    assert dE == int(E[0]) - e0


@pytest.mark.parametrize("L", [64, 72, 128])
@pytest.mark.parametrize("row0,nrows", [(10, 8), (-3, 6), (60, 9)])
def test_one_band_updates_its_rows_only(L, row0, nrows):
    """Neighbour rows come from the whole chain; the band's rows then match it."""
    beta, seed, sweep = 0.47, 900 + L, 4
    before, _, _, _ = oracle.run(L, beta, seed, oracle.HOT, sweeps=sweep)
    after, _, _, _ = oracle.run(L, beta, seed, sweeps=1, sweep0=sweep, state=before)
    mid = _after_black(before, after)
    rows = [(row0 + a) % L for a in range(nrows)]
    others = sorted(set(range(L)) - set(rows))

    s = before.copy()
    oracle.half_sweep_rows(s, 0, beta, seed, sweep, row0, nrows)
    np.testing.assert_array_equal(s[rows], mid[rows])
    np.testing.assert_array_equal(s[others], before[others])

    s = mid.copy()
    oracle.half_sweep_rows(s, 1, beta, seed, sweep, row0, nrows)
    np.testing.assert_array_equal(s[rows], after[rows])
    np.testing.assert_array_equal(s[others], mid[others])


def test_band_keying_depends_on_sweep_and_colour():
    """A band swept with the wrong sweep number or colour differs from the chain
    (so the checks above would see a keying mistake)."""
    L, beta, seed, sweep = 64, BETA_C, 5, 1
    before, _, _, _ = oracle.run(L, beta, seed, oracle.HOT, sweeps=sweep)
    after, _, _, _ = oracle.run(L, beta, seed, sweeps=1, sweep0=sweep, state=before)
    mid = _after_black(before, after)
    s = before.copy()
    oracle.half_sweep_rows(s, 0, beta, seed, sweep + 1, 0, L)
    assert not np.array_equal(s, mid)
    s = before.copy()
    oracle.half_sweep_rows(s, 1, beta, seed, sweep, 0, L)
    assert not np.array_equal(s, mid)
