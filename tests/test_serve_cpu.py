"""Host logic of the serving loop and the seeded workloads (CPU, no GPU).

The server only schedules: it admits requests first come, first served while the
batch has a slot and arena memory, keeps up to two quanta in flight, gathers the
lattices that finish in a quantum behind it, and retires them once that quantum is
seen to be done.  Here the batch is a fake with the same calls and error codes
(EBUSY when every slot is taken, ENOMEM when the arena is full) whose work is done
at once, so the admission order, the blocked counters, the quanta, the in-flight
limit, the quantum sizes and the memory returned are checked without a device.  The workload generators are checked against the recipes their
docstrings state.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1903_11714_gb300 import ising, serve, workloads
from paper_1903_11714_gb300.workloads import Request


class FakeBatch:
    """Slots and an arena of `budget` bytes; a lattice advances by the quantum until
    its own sweep count.  Observables identify the request: M = seed, E = -sweeps."""

    instances = []

    def __init__(self, slots, max_L, budget, threads=0, stream=None):
        self.slots, self.max_L, self.budget = slots, max_L, budget
        self.live = {}
        self.adds, self.runs, self.removed, self.ops = [], [], [], []
        self.peak_bytes = 0
        FakeBatch.instances.append(self)

    def usage(self):
        return sum(v["bytes"] for v in self.live.values()), self.budget

    def add(self, L, beta, seed, start, sweeps, tile_rows=0):
        assert start == ising.HOT
        assert tile_rows == serve.tile_rows(L)
        need = serve.Server.request_bytes(L, sweeps)
        if len(self.live) >= self.slots:
            raise ising.IsingError(ising.ISING_EBUSY, "no free slot")
        if self.usage()[0] + need > self.budget:
            raise ising.IsingError(ising.ISING_ENOMEM, "arena full")
        idx = min(set(range(self.slots)) - set(self.live))
        self.live[idx] = {"L": L, "sweeps": sweeps, "done": 0, "bytes": need, "seed": seed}
        self.adds.append(seed)
        self.peak_bytes = max(self.peak_bytes, self.usage()[0])
        return idx

    def run(self, n, graph_sweeps=0):
        assert graph_sweeps == n
        self.runs.append(sorted(v["seed"] for v in self.live.values()))
        self.ops.append(("run", n))
        for v in self.live.values():
            v["done"] = min(v["sweeps"], v["done"] + n)

    def progress(self, count):
        return [self.live[i]["done"] if i in self.live else 0 for i in range(count)]

    def observables(self, idx):
        v = self.live[idx]
        return v["seed"], -v["sweeps"], v["done"]

    def gather(self, idx, ptr):
        """Writes (done, M = seed, E = -sweeps) of each slot into 3 int64 at ptr."""
        out = (ctypes.c_int64 * (3 * len(idx))).from_address(ptr)
        for k, i in enumerate(idx):
            v = self.live[i]
            out[3 * k], out[3 * k + 1], out[3 * k + 2] = v["done"], v["seed"], -v["sweeps"]
        self.ops.append(("gather", tuple(idx)))

    def remove(self, idx):
        self.removed.append(self.live.pop(idx)["seed"])
        self.ops.append(("remove", idx))

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    FakeBatch.instances.clear()
    monkeypatch.setattr(ising, "Batch", FakeBatch)
    return FakeBatch


def req(rid, arrival, L, sweeps):
    return Request(rid=rid, arrival=float(arrival), L=L, beta=0.44, seed=rid, sweeps=sweeps)


def server(**kw):
    return serve.Server(device_events=False, **kw)


def test_first_come_first_served_with_slots(fake):
    srv = server(hbm_budget_bytes=1 << 30, slots=2, max_L=1024, quantum=64)
    reqs = [req(0, 0, 256, 64), req(1, 0, 512, 128), req(2, 0, 256, 64), req(3, 5, 128, 64)]
    results, st = srv.serve(reqs, realtime=False)
    b = fake.instances[0]
    # r0, r1 in, r2 waits for a slot.  Quantum 1 finishes r0, quantum 2 (enqueued before
    # quantum 1 is collected) r1; collecting quantum 1 frees r0's slot for r2, whose
    # quantum 3 runs beside r1 until r1 is collected.  Nothing runs until r3 becomes
    # visible after quantum 5.
    assert b.runs == [[0, 1], [0, 1], [1, 2], [3]]
    assert b.adds == [0, 1, 2, 3] and sorted(b.removed) == [0, 1, 2, 3]
    assert [r.rid for r in results] == [0, 1, 2, 3]
    assert st.completed == 4 and st.quanta == 4 and st.max_active == 2
    assert st.admission_blocked_by_slots == 1 and st.admission_blocked_by_memory == 0
    assert st.flips == sum(r.L * r.L * r.sweeps for r in reqs)
    assert all((r.M, r.E) == (r.seed, -r.sweeps) for r in results)
    assert b.usage()[0] == 0


def test_memory_blocks_the_head_of_the_queue(fake):
    big, small = serve.Server.request_bytes(1024, 64), serve.Server.request_bytes(64, 64)
    srv = server(hbm_budget_bytes=big + small, slots=8, max_L=1024, quantum=64)
    reqs = [req(0, 0, 1024, 64), req(1, 0, 1024, 64), req(2, 0, 64, 64)]
    results, st = srv.serve(reqs, realtime=False)
    b = fake.instances[0]
    # r1 does not fit beside r0, and r2 (which would) stays behind it: arrival order holds
    assert b.adds == [0, 1, 2]
    assert b.runs == [[0], [1, 2]]
    assert st.admission_blocked_by_memory == 1 and st.admission_blocked_by_slots == 0
    assert b.peak_bytes <= big + small and st.max_arena_bytes <= big + small
    assert [r.rid for r in results] == [0, 1, 2]


def test_requests_that_can_never_fit_are_refused(fake):
    srv = server(hbm_budget_bytes=serve.Server.request_bytes(512, 100), slots=4, max_L=512, quantum=64)
    with pytest.raises(ValueError):
        srv.serve([req(0, 0, 1024, 10)], realtime=False)
    srv = server(hbm_budget_bytes=1 << 20, slots=4, max_L=512, quantum=64)
    with pytest.raises(ValueError):
        srv.serve([req(0, 0, 256, 100_000)], realtime=False)


def test_adaptive_quantum_follows_the_fewest_sweeps_left(fake):
    """Quantum = the largest power of two in 8 .. 256 not above the fewest sweeps any
    admitted lattice still has to be enqueued."""
    srv = server(hbm_budget_bytes=1 << 30, slots=4, max_L=1024)
    assert [srv.choose_quantum(n) for n in (1, 7, 8, 15, 16, 100, 256, 257, 10_000)] == \
        [8, 8, 8, 8, 16, 64, 256, 256, 256]
    results, st = srv.serve([req(0, 0, 256, 20), req(1, 0, 256, 1000)], realtime=False)
    b = fake.instances[0]
    sizes = [n for op, n in b.ops if op == "run"]
    # 20 left -> 16, then 4 left -> 8 (r0 done), then r1 alone: 976 left -> 256 x 3, 208 -> 128, 80 -> 64, 16 -> 16
    assert sizes == [16, 8, 256, 256, 256, 128, 64, 16]
    assert sum(sizes) >= 1000 and [r.rid for r in results] == [0, 1]
    assert fixed_sizes(fake, 32) == [32] * 32


def fixed_sizes(fake, q):
    srv = server(hbm_budget_bytes=1 << 30, slots=4, max_L=1024, quantum=q)
    srv.serve([req(0, 0, 256, 1000)], realtime=False)
    return [n for op, n in fake.instances[-1].ops if op == "run"]


def test_at_most_two_quanta_in_flight(fake, monkeypatch):
    """Each quantum's event reports done only on its second query: the server enqueues
    two quanta, then collects before it enqueues a third."""
    class Slow:
        def __init__(self):
            self.asked = 0

        def query(self):
            self.asked += 1
            return self.asked > 1

    srv = server(hbm_budget_bytes=1 << 30, slots=4, max_L=1024, quantum=8)
    monkeypatch.setattr(srv, "_event", Slow)
    results, st = srv.serve([req(k, 0, 128, 8 * (k + 1)) for k in range(3)], realtime=False)
    ops = [op for op in fake.instances[0].ops if op[0] in ("run", "remove")]
    # r0 (8 sweeps) finishes in quantum 1, r1 in quantum 2, r2 in quantum 3
    assert ops == [("run", 8), ("run", 8), ("remove", 0), ("run", 8), ("remove", 1), ("remove", 2)]
    assert [r.rid for r in results] == [0, 1, 2] and st.quanta == 3


def test_request_bytes_and_percentiles():
    assert serve.Server.request_bytes(8192, 100) == 8192 * 8192 // 8 + 1600
    st = serve.ServeStats(completed=101, flips=3 * 10 ** 9, wall_s=2.0, latencies=[float(v) for v in range(101)][::-1])
    s = st.summary()
    assert s["p50_s"] == 50.0 and s["p99_s"] == 99.0 and s["mean_s"] == 50.0
    assert s["flips_per_ns"] == 1.5
    assert serve.ServeStats().summary()["p50_s"] is None


def test_serving_requests_follow_their_recipe():
    rate = 40.0
    rs = workloads.serving_requests(4000, rate)
    L = np.array([r.L for r in rs])
    sw = np.array([r.sweeps for r in rs])
    t = np.array([r.arrival for r in rs])
    assert all(r.seed == r.rid == k for k, r in enumerate(rs))
    assert np.all(L % 64 == 0) and L.min() >= 256 and L.max() <= 8192
    assert sw.min() >= 100 and sw.max() <= 10_000
    assert all(0.35 <= r.beta <= 0.55 for r in rs)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert abs(np.diff(t).mean() * rate - 1.0) < 0.06          # Poisson gaps of mean 1/rate
    # log-uniform L and sweeps: medians near the geometric means of their ranges
    assert abs(math.log(np.median(L / 64.0)) - math.log(math.sqrt(4 * 128))) < 0.15
    assert abs(math.log(np.median(sw)) - math.log(1000.0)) < 0.15
    assert workloads.serving_requests(4000, rate) == rs           # seeded: the same list every time


def test_batch_workloads_follow_their_recipes():
    scan = workloads.temperature_scan()
    assert len(scan) == 64 and {s.L for s in scan} == {1024} and {s.start for s in scan} == {workloads.COLD}
    assert [s.seed for s in scan] == list(range(3_000_000, 3_000_064))
    assert scan[0].beta == 0.35 and abs(scan[-1].beta - 0.55) < 1e-15
    assert np.allclose(np.diff([s.beta for s in scan]), 0.2 / 63, rtol=0, atol=1e-15)
    # the committed uneven list is exactly what its generator draws
    committed = workloads.uneven_batch()
    assert [s.as_dict() for s in committed] == workloads.make_uneven_batch()
    assert {s.L for s in committed} <= {64 << u for u in range(7)} and len(committed) == 200
    assert all(0.30 <= s.beta <= 0.60 and s.sweeps == 500 for s in committed)
    binder = workloads.binder_scan(10)
    assert len(binder) == 36 and len({s.seed for s in binder}) == 36
    assert all(abs(s.beta * t - workloads.BETA_C_EXACT) < 1e-15
               for s, t in zip(binder, workloads.BINDER_T_OVER_TC * len(workloads.BINDER_LS)))


def test_served_tiles_are_the_tallest_that_fit():
    """Whole-row tiles of at most 8,192 words and 256 rows, a power of two dividing L,
    for every side the request recipe can draw (L = 64 k, 4 <= k <= 128); each is a
    shape the library accepts (2-row tiles need W % 4 == 0, 4+ rows any W)."""
    for k in range(4, 129):
        L = 64 * k
        W, tr = L // 64, serve.tile_rows(L)
        assert tr & (tr - 1) == 0 and 2 <= tr <= 256 and L % tr == 0
        assert tr * W <= serve.TILE_WORDS
        assert tr == 256 or 2 * tr * W > serve.TILE_WORDS or L % (2 * tr) != 0
        assert tr >= 4 or W % 4 == 0
        # the stage (the tile's source rows with HB halo rows each side -- 4 when W % 4
        # != 0, so that copies stay 16-byte aligned -- and its target rows) fits the
        # library's 100 KB stage cap
        hb = 1 if W % 4 == 0 else 4
        assert ((tr + 2 * hb) * W + tr * W) * 4 <= 100 * 1024
    assert serve.tile_rows(8192) == 64 and serve.tile_rows(1024) == 256 and serve.tile_rows(64 * 127) == 64
    assert serve.tile_rows(2560) == 128  # W = 40: 256 rows would be 10,240 words
