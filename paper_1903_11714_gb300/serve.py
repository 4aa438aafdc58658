"""Serving loop: continuous batching of Ising simulation requests on one GPU.

Requests (L, beta, seed, sweeps) arrive over time.  A request is admitted as
soon as a slot is free and its device-resident state (bit-packed planes, L^2/8
bytes, plus 16 bytes of M/E history per sweep) fits in the HBM budget (the
batch arena).  Every scheduling quantum enqueues `quantum` sweeps of all
admitted lattices as one persistent launch per half-sweep (replayed from a
captured CUDA graph), so requests that arrive while others run share the same
launches.  A lattice stops at its own sweep count; finished requests are read
back and their memory returned to the arena.  Because the random numbers are
keyed by (seed, sweep, colour, site), a request's result does not depend on
what else is in the mix.

All GPU work goes through the C ABI (ising_batch_*); this module only
schedules.
"""
from __future__ import annotations

import statistics
import time
from collections import deque
from dataclasses import dataclass, field

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
    admission_blocked_by_memory: int = 0
    admission_blocked_by_slots: int = 0
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


class Server:
    """Admission by HBM budget and slots, continuous batching, p50/p99 latency."""

    def __init__(self, hbm_budget_bytes: int, slots: int, max_L: int = 8192, quantum: int = 64, threads: int = 0,
                 stream=None):
        self.quantum = int(quantum)
        self.slots = int(slots)
        self.budget = int(hbm_budget_bytes)
        self.max_L = int(max_L)
        self.batch = ising.Batch(self.slots, max_L, self.budget, threads, stream)

    @staticmethod
    def request_bytes(L: int, sweeps: int) -> int:
        return L * L // 8 + 16 * sweeps

    def serve(self, requests: list[Request], realtime: bool = True, keep_lattices: bool = False,
              keep_history: bool = False) -> tuple[list[Result], ServeStats]:
        """Runs all requests to completion.  realtime=True: arrivals follow the
        wall clock (request.arrival seconds after the start); False: arrival is
        the scheduling quantum at which the request becomes visible."""
        b = self.batch
        b_max_L = self.max_L
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque[Request] = deque()
        active: dict[int, tuple[Request, float]] = {}
        results: list[Result] = []
        st = ServeStats()
        t0 = time.perf_counter()
        quantum_no = 0

        def clock() -> float:
            return time.perf_counter() - t0

        while pending or waiting or active:
            now = clock() if realtime else float(quantum_no)
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission: first come, first served, while a slot and the memory are free
            while waiting:
                r = waiting[0]
                if self.request_bytes(r.L, r.sweeps) > self.budget or r.L > b_max_L:
                    raise ValueError(f"request {r.rid} can never fit: L={r.L}, sweeps={r.sweeps}")
                try:
                    idx = b.add(r.L, r.beta, r.seed, ising.HOT, r.sweeps)
                except ising.IsingError as e:
                    if e.code == ising.ISING_ENOMEM:
                        st.admission_blocked_by_memory += 1
                    elif e.code == ising.ISING_EBUSY:
                        st.admission_blocked_by_slots += 1
                    else:
                        raise
                    break
                waiting.popleft()
                active[idx] = (r, clock())
            if not active:
                if realtime and pending:
                    time.sleep(max(0.0, pending[0].arrival - clock()))
                else:
                    quantum_no += 1
                continue
            st.max_active = max(st.max_active, len(active))
            st.max_arena_bytes = max(st.max_arena_bytes, b.usage()[0])
            b.run(self.quantum, graph_sweeps=self.quantum)
            quantum_no += 1
            st.quanta += 1
            done = b.progress(max(active) + 1)
            for idx in sorted(active):
                r, adm = active[idx]
                if done[idx] >= r.sweeps:
                    M, E, _ = b.observables(idx)
                    res = Result(rid=r.rid, L=r.L, beta=r.beta, seed=r.seed, sweeps=r.sweeps,
                                 arrival=r.arrival if realtime else 0.0, admitted=adm, finished=clock(), M=M, E=E)
                    if keep_lattices:
                        res.lattice = b.get_lattice(idx)
                    if keep_history:
                        res.history = b.history(idx)
                    b.remove(idx)
                    del active[idx]
                    results.append(res)
                    st.completed += 1
                    st.flips += r.flips
                    if realtime:
                        st.latencies.append(res.latency)
        st.wall_s = clock()
        return results, st

    def close(self) -> None:
        self.batch.close()
