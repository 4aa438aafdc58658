"""Serving loop: continuous batching of Ising simulation requests on one GPU.

Requests (L, beta, seed, sweeps) arrive over time.  A request is admitted as
soon as a slot is free and its device-resident state (bit-packed planes, L^2/8
bytes, plus 16 bytes of M/E history per sweep) fits in the HBM budget (the
batch arena).  Every scheduling quantum enqueues q sweeps of all admitted
lattices as one persistent launch per half-sweep (replayed from a CUDA graph
captured once per quantum size), so requests that arrive while others run share
the same launches.  A lattice stops at its own sweep count.

The host never waits for the GPU between quanta: up to two quanta are in flight;
a request is admitted (its start state and descriptor enqueued) while earlier
quanta run and sweeps from the next quantum on; for the lattices that finish in a
quantum, their final (M, E) are gathered into page-locked host memory behind that
quantum, and the host polls an event, then returns their slots and memory.  The
quantum is the largest power of two (8 .. 256) not above the fewest sweeps any
admitted lattice has left, so a short request finishes at a quantum boundary
instead of waiting out a long quantum; a fixed quantum can be given instead.
Because the random numbers are keyed by (seed, sweep, colour, site), a request's
result does not depend on what else is in the mix.

All GPU work goes through the C ABI (ising_batch_*); this module only
schedules.
"""
from __future__ import annotations

import statistics
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import ising
from .workloads import Request


@dataclass
class Result:
    rid: int
    L: int
    beta: float
    seed: int
    sweeps: int
    arrival: float
    admitted: float
    finished: float
    M: int
    E: int
    lattice: object = None
    history: object = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class ServeStats:
    completed: int = 0
    flips: int = 0
    wall_s: float = 0.0
    quanta: int = 0
    max_active: int = 0
    max_arena_bytes: int = 0
    admission_blocked_by_memory: int = 0   # requests that waited for arena memory
    admission_blocked_by_slots: int = 0    # requests that waited for a slot
    latencies: list = field(default_factory=list)

    def summary(self) -> dict:
        lat = sorted(self.latencies)

        def pct(p):
            if not lat:
                return None
            k = min(len(lat) - 1, max(0, int(round(p / 100.0 * (len(lat) - 1)))))
            return lat[k]

        return {"completed": self.completed, "flips": self.flips, "wall_s": self.wall_s,
                "flips_per_ns": self.flips / (self.wall_s * 1e9) if self.wall_s > 0 else None,
                "p50_s": pct(50), "p99_s": pct(99), "mean_s": statistics.mean(lat) if lat else None,
                "quanta": self.quanta, "max_active": self.max_active, "max_arena_bytes": self.max_arena_bytes,
                "blocked_by_memory": self.admission_blocked_by_memory,
                "blocked_by_slots": self.admission_blocked_by_slots}


# Tile height of a served lattice: the tallest power of two (at most 256 rows) whose
# whole-row tile holds at most TILE_WORDS words and divides L.  The library's built-in
# tiles stay short (about 4,096 words, at most 64 rows) so that a batch of a few small
# lattices still has a tile for every CTA; a serving batch holds dozens to hundreds of
# lattices, and taller tiles give each warp more words per tile, so the per-tile costs
# (the stage handoff, the last partial drain of each warp's queue) weigh less: 13-15 %
# more throughput on the request mix of the serving workload.
TILE_WORDS = 8192


def tile_rows(L: int) -> int:
    W = L // 64
    tr = 2
    while tr * 2 <= 256 and tr * 2 * W <= TILE_WORDS and L % (tr * 2) == 0:
        tr *= 2
    return tr


class _Done:
    """An event that has already happened (host-side batches, whose work is synchronous)."""

    def record(self, stream=None):
        pass

    def query(self) -> bool:
        return True

    def synchronize(self):
        pass


class Server:
    """Admission by HBM budget and slots, continuous batching, p50/p99 latency."""

    QMIN, QMAX = 8, 256
    IN_FLIGHT = 2

    def __init__(self, hbm_budget_bytes: int, slots: int, max_L: int = 8192, quantum: int = 0, threads: int = 0,
                 stream=None, device_events: bool = True):
        """quantum: 0 = adaptive (see the module notes), else a fixed number of sweeps.
        device_events: poll CUDA events and gather into page-locked memory (False for
        host-side stand-ins of the batch, which finish their work at once)."""
        self.quantum = int(quantum)
        self.slots = int(slots)
        self.budget = int(hbm_budget_bytes)
        self.max_L = int(max_L)
        self.device_events = device_events
        if device_events:
            import torch

            self.stream = stream if stream is not None else torch.cuda.Stream()
            self._pinned = [torch.zeros(3 * self.slots, dtype=torch.int64, pin_memory=True)
                            for _ in range(self.IN_FLIGHT + 1)]
            self._bufs = [t.numpy() for t in self._pinned]
        else:
            self.stream = stream
            self._bufs = [np.zeros(3 * self.slots, dtype=np.int64) for _ in range(self.IN_FLIGHT + 1)]
        self.batch = ising.Batch(self.slots, max_L, self.budget, threads, self.stream)

    @staticmethod
    def request_bytes(L: int, sweeps: int) -> int:
        return L * L // 8 + 16 * sweeps

    def _event(self):
        if not self.device_events:
            return _Done()
        import torch

        ev = torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def choose_quantum(self, fewest_left: int) -> int:
        if self.quantum > 0:
            return self.quantum
        q = self.QMIN
        while q * 2 <= min(fewest_left, self.QMAX):
            q *= 2
        return q

    def serve(self, requests: list[Request], realtime: bool = True, keep_lattices: bool = False,
              keep_history: bool = False) -> tuple[list[Result], ServeStats]:
        """Runs all requests to completion.  realtime=True: arrivals follow the
        wall clock (request.arrival seconds after the start); False: arrival is
        the number of quanta enqueued before the request becomes visible."""
        b = self.batch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque[Request] = deque()
        active: dict[int, list] = {}       # slot -> [request, admitted at, sweeps enqueued]
        inflight: deque = deque()          # (event, [(slot, request, admitted)], buffer index)
        results: list[Result] = []
        st = ServeStats()
        t0 = time.perf_counter()
        quanta = 0
        buf_no = 0
        blocked_mem, blocked_slot = set(), set()

        def clock() -> float:
            return time.perf_counter() - t0

        while pending or waiting or active or inflight:
            now = clock() if realtime else float(quanta)
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission: first come, first served, while a slot and the memory are free
            while waiting:
                r = waiting[0]
                if self.request_bytes(r.L, r.sweeps) > self.budget or r.L > self.max_L:
                    raise ValueError(f"request {r.rid} can never fit: L={r.L}, sweeps={r.sweeps}")
                try:
                    idx = b.add(r.L, r.beta, r.seed, ising.HOT, r.sweeps, tile_rows(r.L))
                except ising.IsingError as e:
                    # requests that had to wait for memory / a slot (each counted once)
                    if e.code == ising.ISING_ENOMEM:
                        blocked_mem.add(r.rid)
                    elif e.code == ising.ISING_EBUSY:
                        blocked_slot.add(r.rid)
                    else:
                        raise
                    break
                waiting.popleft()
                active[idx] = [r, clock(), 0]
                st.max_active = max(st.max_active, len(active))
                st.max_arena_bytes = max(st.max_arena_bytes, b.usage()[0])
            runnable = [i for i, a in active.items() if a[2] < a[0].sweeps]
            if runnable and len(inflight) < self.IN_FLIGHT:
                # enqueue a quantum; the lattices that reach their sweep count in it are
                # gathered behind it
                q = self.choose_quantum(min(active[i][0].sweeps - active[i][2] for i in runnable))
                b.run(q, graph_sweeps=q)
                quanta += 1
                st.quanta += 1
                fin = []
                for i in runnable:
                    active[i][2] += q
                    if active[i][2] >= active[i][0].sweeps:
                        fin.append(i)
                buf = buf_no % len(self._bufs)
                buf_no += 1
                if fin:
                    b.gather(fin, self._bufs[buf].ctypes.data)
                inflight.append((self._event(), [(i, active[i][0], active[i][1]) for i in fin], buf))
                continue
            if inflight and inflight[0][0].query():
                _, fin, buf = inflight.popleft()
                out = self._bufs[buf]
                for k, (i, r, adm) in enumerate(fin):
                    done, M, E = (int(v) for v in out[3 * k:3 * k + 3])
                    assert done >= r.sweeps, (r.rid, done)
                    res = Result(rid=r.rid, L=r.L, beta=r.beta, seed=r.seed, sweeps=r.sweeps,
                                 arrival=r.arrival if realtime else 0.0, admitted=adm, finished=clock(), M=M, E=E)
                    if keep_lattices:
                        res.lattice = b.get_lattice(i)
                    if keep_history:
                        res.history = b.history(i)
                    b.remove(i)
                    del active[i]
                    results.append(res)
                    st.completed += 1
                    st.flips += r.flips
                    if realtime:
                        st.latencies.append(res.latency)
                continue
            # nothing to enqueue or collect yet: wait for the oldest quantum or the next arrival
            if not realtime and not inflight:
                if not pending:
                    break  # only requests that can wait forever are left (handled above)
                quanta = max(quanta, int(np.ceil(pending[0].arrival)))
                continue
            nxt = pending[0].arrival - clock() if (realtime and pending) else 1.0
            if inflight:
                time.sleep(max(0.0, min(2e-4, nxt)))
            elif nxt > 0:
                time.sleep(nxt)
        st.wall_s = clock()
        st.admission_blocked_by_memory = len(blocked_mem)
        st.admission_blocked_by_slots = len(blocked_slot)
        return results, st

    def close(self) -> None:
        self.batch.close()
