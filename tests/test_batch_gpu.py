"""GPU parity of the batched runtime (one persistent launch per half-sweep over
many lattices of uneven L and beta, optionally replayed from a CUDA graph).

Every lattice of a batch must reach exactly the chain it reaches alone: the
same lattice, M and E as a single-lattice handle and as the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising, workloads

pytestmark = pytest.mark.gpu
REL_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


def single(L, beta, seed, start, sweeps):
    lat = ising.Lattice(L, beta, seed, start, ising.PACKED).sweep(sweeps)
    M, E = lat.history()
    s = lat.get_lattice()
    lat.close()
    return s, M, E


def arena_for(lats):
    return sum(l.L * l.L // 8 + 16 * l.sweeps + 4096 for l in lats)


def test_temperature_scan_full_size():
    """64 replicas of L = 1024, beta in [0.35, 0.55], cold start, a 100-sweep graph
    replayed 50 times; per-replica FP64 |m|, e, U4 from exact sums."""
    reps = workloads.temperature_scan()
    b = ising.Batch(len(reps), 1024, arena_for(reps))
    idx = [b.add(r.L, r.beta, r.seed, r.start, r.sweeps) for r in reps]
    b.run(5000, graph_sweeps=workloads.TEMPERATURE_SCAN_GRAPH_SWEEPS)
    b.synchronize()
    burn = workloads.TEMPERATURE_SCAN_BURN_IN
    # one replica against the oracle over the whole 5000-sweep chain
    r = 32
    ref, Mr, Er, _ = oracle.run(reps[r].L, reps[r].beta, reps[r].seed, reps[r].start, reps[r].sweeps)
    M, E = b.history(idx[r])
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    assert np.array_equal(b.get_lattice(idx[r]), ref)
    ex = oracle.moments_exact(Mr, Er, reps[r].L ** 2, burn)
    got = b.moments(idx[r], burn)
    for k in ("abs_m", "e", "binder", "m2", "m4"):
        assert got[k] == pytest.approx(ex[k], rel=REL_TOL, abs=0), k
    # every replica: history exact vs the same lattice swept alone, moments vs exact rationals
    for k in (0, 7, 31, 63):
        s1, M1, E1 = single(reps[k].L, reps[k].beta, reps[k].seed, reps[k].start, reps[k].sweeps)
        Mb, Eb = b.history(idx[k])
        assert np.array_equal(Mb, M1) and np.array_equal(Eb, E1), k
        assert np.array_equal(b.get_lattice(idx[k]), s1), k
    for k, i in enumerate(idx):
        Mb, Eb = b.history(i)
        ex = oracle.moments_exact(Mb, Eb, 1024 * 1024, burn)
        got = b.moments(i, burn)
        for key in ("S1", "S2", "S4", "SE", "SE2"):
            assert got[key] == ex[key], (k, key)
        assert got["binder"] == pytest.approx(ex["binder"], rel=REL_TOL, abs=0)
        N = 1024 * 1024
        assert np.all(Eb % 4 == 0) and np.all(np.abs(Mb) <= N) and np.all(Mb % 2 == 0)
    # physics: below T_c the scan sits on Onsager's spontaneous magnetisation
    from oracle import exact

    for k in (50, 63):
        m = b.moments(idx[k], burn)["abs_m"]
        assert abs(m - exact.onsager_m0(reps[k].beta)) < 0.01, (k, m)
    b.close()


def test_first_graph_replay_matches_oracle():
    reps = workloads.temperature_scan()[:8]
    b = ising.Batch(len(reps), 1024, arena_for(reps))
    idx = [b.add(r.L, r.beta, r.seed, r.start, 100) for r in reps]
    b.run(100, graph_sweeps=100)
    for k in (0, 5):
        ref, Mr, Er, _ = oracle.run(reps[k].L, reps[k].beta, reps[k].seed, reps[k].start, 100)
        M, E = b.history(idx[k])
        assert np.array_equal(M, Mr) and np.array_equal(E, Er)
        assert np.array_equal(b.get_lattice(idx[k]), ref)
    b.close()


def test_uneven_batch_full_size():
    """200 lattices, L in {64..4096}, 500 sweeps each, one launch per half-sweep."""
    lats = workloads.uneven_batch()
    b = ising.Batch(len(lats), 4096, arena_for(lats))
    idx = [b.add(l.L, l.beta, l.seed, l.start, l.sweeps) for l in lats]
    b.run(500)
    b.synchronize()
    for k, l in enumerate(lats):
        if l.L <= 128 or k % 25 == 0:
            ref, Mr, Er, _ = oracle.run(l.L, l.beta, l.seed, l.start, l.sweeps)
            M, E = b.history(idx[k])
            assert np.array_equal(M, Mr) and np.array_equal(E, Er), k
            assert np.array_equal(b.get_lattice(idx[k]), ref), k
    for k in (1, 2, 3, 50, 120, 199):
        l = lats[k]
        s1, M1, E1 = single(l.L, l.beta, l.seed, l.start, l.sweeps)
        Mb, Eb = b.history(idx[k])
        assert np.array_equal(Mb, M1) and np.array_equal(Eb, E1), k
        assert np.array_equal(b.get_lattice(idx[k]), s1), k
    b.close()


@pytest.mark.parametrize("tile_rows", [2, 4, 8, 16, 32, 64, 128, 256])
def test_tile_rows_do_not_change_the_chain(tile_rows):
    L, beta, seed = 512, 0.44, 9
    ref, Mr, Er, _ = oracle.run(L, beta, seed, oracle.HOT, 6)
    for threads in (128, 256, 512):
        b = ising.Batch(1, L, L * L // 8 + 4096, threads)
        i = b.add(L, beta, seed, ising.HOT, 6, tile_rows)
        b.run(6)
        M, E = b.history(i)
        assert np.array_equal(M, Mr) and np.array_equal(E, Er), threads
        assert np.array_equal(b.get_lattice(i), ref), threads
        b.close()


def test_graph_and_plain_launches_agree():
    specs = [(64, 0.3, 1), (256, 0.44, 2), (1024, 0.5, 3), (192, 0.6, 4)]
    out = []
    for graph in (0, 10):
        b = ising.Batch(4, 1024, 10 << 20)
        idx = [b.add(L, beta, seed, ising.HOT, 40) for L, beta, seed in specs]
        b.run(40, graph_sweeps=graph)
        out.append([(b.history(i), b.get_lattice(i)) for i in idx])
        b.close()
    for (h0, s0), (h1, s1) in zip(*out):
        assert np.array_equal(h0[0], h1[0]) and np.array_equal(h0[1], h1[1]) and np.array_equal(s0, s1)


def test_sweep_limits_stop_each_lattice():
    b = ising.Batch(3, 256, 4 << 20)
    i0 = b.add(256, 0.44, 1, ising.HOT, 7)
    i1 = b.add(128, 0.44, 2, ising.HOT, 20)
    b.run(12)
    assert b.sweeps_done(i0) == 7 and b.sweeps_done(i1) == 12
    b.run(30)
    assert b.sweeps_done(i0) == 7 and b.sweeps_done(i1) == 20
    ref, Mr, _, _ = oracle.run(256, 0.44, 1, oracle.HOT, 7)
    assert np.array_equal(b.get_lattice(i0), ref) and np.array_equal(b.history(i0)[0], Mr)
    # history ranges whose end wraps a signed 64-bit integer are refused before any copy
    big = (1 << 63) - 3
    assert ising.lib().ising_batch_history(b.b, i0, big, 5, None, None) == ising.ISING_EINVAL
    assert ising.lib().ising_batch_history(b.b, i0, 2, big, None, None) == ising.ISING_EINVAL
    b.close()


def test_add_remove_and_arena_reuse_keep_results_independent():
    """A lattice's chain is the same alone and in any mix (slots, order, arena reuse)."""
    ref, Mr, Er, _ = oracle.run(512, 0.47, 42, oracle.HOT, 15)
    b = ising.Batch(4, 512, 2 * (512 * 512 // 8 + 16 * 64) + 8192)
    a = b.add(256, 0.3, 1, ising.HOT, 64)
    c = b.add(512, 0.5, 2, ising.COLD, 64)
    b.run(5)
    b.remove(a)
    b.remove(c)
    x = b.add(512, 0.47, 42, ising.HOT, 64)  # reuses freed arena memory
    y = b.add(64, 0.9, 3, ising.HOT, 64)
    b.run(15)
    M, E = b.history(x)
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    assert np.array_equal(b.get_lattice(x), ref)
    b.close()


def test_admission_errors():
    b = ising.Batch(2, 256, 256 * 256 // 8 + 16 * 10 + 512)
    b.add(256, 0.4, 1, ising.HOT, 10)
    with pytest.raises(ising.IsingError) as e:
        b.add(256, 0.4, 2, ising.HOT, 10)
    assert e.value.code == ising.ISING_ENOMEM
    with pytest.raises(ising.IsingError) as e:
        b.add(512, 0.4, 3, ising.HOT, 10)
    assert e.value.code == ising.ISING_EINVAL  # beyond max_L
    b.close()
    b = ising.Batch(1, 256, 1 << 20)
    b.add(64, 0.4, 1, ising.HOT, 10)
    with pytest.raises(ising.IsingError) as e:
        b.add(64, 0.4, 2, ising.HOT, 10)
    assert e.value.code == ising.ISING_EBUSY
    b.close()


def test_autotune_returns_a_valid_tile():
    for L in (64, 1024, 4096):
        tr, th, ms = ising.ising_autotune(L)
        assert tr in (2, 4, 8, 16, 32, 64, 128, 256) and L % tr == 0 and th in (256, 512) and ms > 0


def test_batch_still_runs_after_a_smaller_engine_is_configured():
    """Engines share the sweep kernel's shared-memory limit: a single handle with small
    tiles created after a batch with large ones must not lower it below the batch's
    launches."""
    beta = 0.4406868
    b = ising.Batch(2, 8192, 1 << 30, 0)
    k = b.add(8192, beta, 3, ising.HOT, 8, 64)   # 64-row tiles of 128-word rows: a large stage
    b.run(2)
    b.synchronize()
    small = ising.Lattice(512, beta, 4, ising.HOT).sweep(2)  # configures a small engine
    small.close()
    b.run(2)
    b.synchronize()
    assert b.sweeps_done(k) == 4
    M, E = b.history(k, 0, 4)
    lat = ising.Lattice(8192, beta, 3, ising.HOT).sweep(4)
    Ms, Es = lat.history()
    assert np.array_equal(M, Ms) and np.array_equal(E, Es)
    lat.close()
    b.close()


def test_batch_from_arrays_matches_oracle_through_history_growth():
    """The boundary's array form, through the C ABI: ising_batch_create(count, L[],
    beta[], seed[], start[]) on an uneven three-lattice batch (W % 4 == 0, odd W,
    W = 2 mod 4; hot and cold starts), run as a captured 100-sweep graph replayed
    6 times and then 600 plain sweeps: 1,200 sweeps, past the 1,024-sweep history
    a lattice gets at admission, so every history is grown once between runs.
    Lattices, every sweep's M and E, the current (M, E) and the Sec. 4.1 moments
    (ising_moments' five outputs) equal the oracle's."""
    Ls, betas, seeds, starts = [256, 192, 128], [0.4406868, 0.30, 0.55], [11, 12, 13], [ising.HOT, ising.HOT,
                                                                                          ising.COLD]
    h = ising.ising_batch_create(Ls, betas, seeds, starts)
    b = ising.Batch(0, 0, 0, _handle=h, _Ls=Ls)
    try:
        for k in range(3):  # the start states, before any sweep
            ref0 = oracle.init(Ls[k], seeds[k], starts[k])
            assert ising.ising_batch_observables(h, k) == oracle.observe(ref0), k
        ising.ising_batch_run(h, 600, 100)
        ising.ising_batch_run(h, 600, 0)
        n = 1200
        for k in range(3):
            ref, Mr, Er, _ = oracle.run(Ls[k], betas[k], seeds[k], starts[k], n)
            M, E = b.history(k)
            assert len(M) == n
            assert np.array_equal(M, Mr) and np.array_equal(E, Er), k
            assert np.array_equal(b.get_lattice(k), ref), k
            assert ising.ising_batch_observables(h, k) == (int(Mr[-1]), int(Er[-1])), k
            ex = oracle.moments_exact(Mr, Er, Ls[k] ** 2, n // 10)
            got = b.moments(k, n // 10)
            for key in ("abs_m", "m2", "m4", "e", "binder"):
                assert got[key] == pytest.approx(ex[key], rel=REL_TOL, abs=0), (k, key)
    finally:
        b.close()


def test_array_form_with_tall_tiles_matches_oracle():
    """A batch created from arrays with enough lattices that ising_batch_create gives
    each the tallest whole-row tile of up to 8,192 words (here one tile per L = 128
    lattice and three 64-row tiles per L = 192 lattice, whose odd row width needs
    4-row halos: 1,280 tiles, over two per CTA of the grid), swept as a captured
    graph: every lattice and every sweep's M and E equal the oracle's."""
    n_each, sweeps = 320, 4
    Ls = [128] * n_each + [192] * n_each
    betas = [0.30 + 0.3 * k / (2 * n_each) for k in range(2 * n_each)]
    seeds = [5000 + k for k in range(2 * n_each)]
    starts = [ising.HOT if k % 3 else ising.COLD for k in range(2 * n_each)]
    b = ising.Batch.from_arrays(Ls, betas, seeds, starts)
    try:
        b.run(sweeps, graph_sweeps=2)
        for k in range(2 * n_each):
            ref, Mr, Er, _ = oracle.run(Ls[k], betas[k], seeds[k], starts[k], sweeps)
            M, E = b.history(k)
            assert np.array_equal(M, Mr) and np.array_equal(E, Er), k
            assert np.array_equal(b.get_lattice(k), ref), k
    finally:
        b.close()


def test_single_handle_moments_five_outputs_match_the_extended_form():
    """ising_moments (the boundary's five outputs) equals ising_moments_ex's values."""
    lat = ising.Lattice(256, 0.45, 5, ising.HOT, ising.PACKED).sweep(300)
    five = ising.ising_moments(lat.h, 30)
    ex = lat.moments(30)
    assert five == (ex["abs_m"], ex["m2"], ex["m4"], ex["e"], ex["binder"])
    M, E = lat.history()
    ref = oracle.moments_exact(M, E, 256 * 256, 30)
    for got, key in zip(five, ("abs_m", "m2", "m4", "e", "binder")):
        assert got == pytest.approx(ref[key], rel=REL_TOL, abs=0), key
    lat.close()
