#!/usr/bin/env python
"""Benchmark: spin-flip attempts per ns of the bit-packed checkerboard sweep.

Workload (default): one L = 65,536 lattice (4.29e9 spins, 512 MB bit-packed)
at beta = 0.4406868, hot start from seed 2.  A "step" is one sweep (black plus
white half-sweep with the fused M/E reduction); --steps defaults to the
workload's 200 sweeps.  The planes (512 MB) are larger than the 129 MB L2, so
consecutive sweeps stream from HBM without an explicit flush.

value: K * L^2 / (device time of K sweeps), CUDA events on the lattice's stream,
max over ranks.  With N GPUs (torchrun) every rank sweeps its own replica
(seed + rank): replicas only, no collective on the data path.

--impl reference times the CPU oracle (the plain C checkerboard in oracle/) on
bounded samples of the same lattice instead.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin-flip attempts/ns on 1 GB300 (bit-packed checkerboard sweep, bit-exact)"
UNIT = "flips/ns"
# Roofline.  The sweep is integer work in registers (Philox4x32-10, a bitwise
# neighbour count, bit-sliced threshold tests); memory moves 3/16 byte per site
# update and does not bind.  With bit-sliced uniforms a plane word draws only the
# Philox calls its sites need to be decided (about 2 of 8 on average, more where a
# thread waits for its slowest word and a warp for its slowest thread), so the work
# per site is data-dependent and is counted as executed instructions: ncu's
# smsp__inst_executed.sum of one launch of the same kernel on the same workload,
# committed under profiles/ with a hash of the kernel's sources, times 32 lanes.
# The binding resource is instruction issue: one warp instruction per clock per
# scheduler, 4 schedulers per SM -> 128 thread-instruction slots per clock per SM.
ISSUE_SLOTS_PER_CLK_SM = 128.0
ALU_OPS_PER_CLK_SM = 64.0
N_SMS = 152
KERNEL_SOURCES = {
    "packed_half_sweep": ("sweep_packed_kernel.cuh", "word_update.cuh", "philox.cuh", "ising_device.cuh",
                          "jit.cu"),
    "cubic_half_sweep": ("sweep3d_kernel.cuh", "word_update.cuh", "philox.cuh", "ising_device.cuh", "jit.cu"),
    "int8_half_sweep": ("sweep_int8.cu", "word_update.cuh", "philox.cuh", "ising_device.cuh"),
    "cluster_sweep": ("sweep_cluster.cu", "sweep_packed_kernel.cuh", "word_update.cuh", "philox.cuh",
                      "ising_device.cuh"),
}
# algorithmic bytes per site per sweep (packed): each half-sweep reads the target
# and source planes and writes the target plane, N/2 bits each
BYTES_PER_SITE_SWEEP = 3.0 * 2 * (0.5 / 8.0)
# int8: each half-sweep reads and writes all N bytes for N/2 updated sites
INT8_BYTES_PER_SITE = 4.0


def max_over_ranks(value: float, dist, device: str) -> float:
    """Timing of the slowest rank (the job ends when the last replica does)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def total_over_ranks(value: float, dist, device: str) -> float:
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


_CODE_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|//[^\n]*|/\*.*?\*/', re.S)


def code_only(text: str) -> str:
    """C/CUDA source without comments and with runs of whitespace collapsed (string
    literals, which hold the inline PTX, are kept as they are)."""
    text = _CODE_TOKENS.sub(lambda m: " " if m.group(0).startswith("/") else m.group(0), text)
    return " ".join(text.split())


def kernel_source_hash(kernel: str = "packed_half_sweep") -> str:
    """Hash of the kernel's sources as code: comment-only edits leave it unchanged."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1903_11714_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def committed_counters(kernel: str):
    """Per-site ncu counters of one launch of `kernel` (profiles/<kernel>_counters.json):
    thread-instruction slots and DRAM bytes per updated site.  'current' is False when
    the kernel's sources changed after the capture."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_counters.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    sites = d["sites_per_launch"]
    alu = d.get("alu_warp_inst_per_launch")
    pipes = {name: d[f"{name}_pipe_cycles_per_launch"] / sites for name in ("alu", "fmaheavy")
             if f"{name}_pipe_cycles_per_launch" in d}
    # DRAM bytes per site from a one-pass capture of the full-size workload where the
    # record has one (re-reads depend on the lattice's size), else from the small case
    fs = d.get("full_size")
    dram = ((fs["dram_bytes_read_per_launch"] + fs["dram_bytes_write_per_launch"]) / fs["sites_per_launch"] if fs
            else (d["dram_bytes_read_per_launch"] + d["dram_bytes_write_per_launch"]) / sites)
    return {"current": d.get("kernel_source_hash") == kernel_source_hash(kernel),
            "inst_slots_per_site": 32.0 * d["warp_inst_per_launch"] / sites,
            "alu_ops_per_site": None if alu is None else 32.0 * alu / sites,
            "pipe_cycles_per_site": pipes or None,
            "dram_bytes_per_site": dram,
            "capture": d.get("command")}


# Counted model of the method's own integer work (the algorithmic view of the roofline).
# Per 32-site plane word and half-sweep: E Philox calls (see expected_calls_per_word),
# each 16 site-dependent 32x32->64 products and 18 three-input XORs; 4 logic operations
# per bit plane the comparison reads (4 planes per call); a 15-operation bitwise adder.
PHILOX_PRODUCTS_PER_CALL = 16
PHILOX_XOR3_PER_CALL = 18
COMPARE_OPS_PER_PLANE = 4
ADDER_OPS_PER_WORD = 15


def expected_calls_per_word(n):
    """Expected Philox calls of a 32-site word with n tested sites.  U < T is read from
    U's top bit plane down, four planes per call, and a tested site is decided at the
    first plane where U's bit differs from T's: probability 1/2 per plane, independently
    (T strictly between 0 and 2^32).  So call k (0-based) is needed iff some site is
    still undecided after 4k planes: E = sum_k 1 - (1 - 2^-4k)^n, k = 0..7 (n = 0: no
    call)."""
    import numpy as np

    n = np.asarray(n, dtype=np.float64)
    return sum(1.0 - (1.0 - 2.0 ** (-4 * k)) ** n for k in range(8))


def tested_sites_per_word(rows, test2: bool, test4: bool, first_row: int = 1):
    """Tested sites per plane word for the centre rows of `rows` (R + 2 consecutive rows
    of +-1 bytes, the first and last only as neighbours; the second has global index
    first_row), both colours: a site with one anti-aligned neighbour compares against
    T2 (test2: 0 < T2 < 2^32), with none against T4; bit b of word w of row i of colour
    c is the site (i, 2(32w + b) + ((i + c) & 1))."""
    import numpy as np

    s = np.asarray(rows, dtype=np.int8)
    c = s[1:-1]
    n = ((s[:-2] != c).astype(np.int8) + (s[2:] != c) + (np.roll(c, 1, axis=1) != c)
         + (np.roll(c, -1, axis=1) != c))
    tested = ((n == 1) & test2) | ((n == 0) & test4)
    R, L = c.shape
    out = []
    for i in range(R):
        for colour in (0, 1):
            out.append(tested[i, ((first_row + i + colour) & 1)::2].reshape(L // 64, 32).sum(axis=1))
    return np.concatenate(out)


def algorithmic_view(rows, T2: int, T4: int, sites_per_s: float, sm_max: float) -> dict:
    """The roofline of the counted model: per site, E products x 2 lane-cycles on the
    FMA-heavy pipe (a 32x32->64 product holds a 16-lane pipe 4 cycles per warp) / 32,
    and (18 E + 16 E + 15) one-lane-cycle logic operations on the ALU pipe / 32, against
    64 lanes/clk/SM x 152 SMs x the clock on each pipe."""
    import numpy as np

    n = tested_sites_per_word(rows, 0 < T2 < 2 ** 32, 0 < T4 < 2 ** 32)
    E = float(np.mean(expected_calls_per_word(n)))
    peak = ALU_OPS_PER_CLK_SM * N_SMS * sm_max * 1e6 / 1e12
    fma = E * PHILOX_PRODUCTS_PER_CALL * 2.0 / 32.0
    alu = (E * (PHILOX_XOR3_PER_CALL + 4 * COMPARE_OPS_PER_PLANE) + ADDER_OPS_PER_WORD) / 32.0
    views = {name: {"lane_cycles_per_site": v, "achieved": v * sites_per_s / 1e12,
                    "frac": v * sites_per_s / 1e12 / peak} for name, v in (("fmaheavy", fma), ("alu", alu))}
    bind = max(views, key=lambda k: views[k]["frac"])
    return {"frac": views[bind]["frac"], "pipe": PIPE_NAMES[bind], "calls_per_word": E,
            "tested_sites_per_word": float(np.mean(n)), "words_sampled": int(n.size),
            "views": {PIPE_NAMES[k]: v for k, v in views.items()}, "peak": peak, "unit": "Tops/s",
            "model": "per 32-site word: E Philox calls (16 products, 18 XOR3 each) + 4 logic ops per bit plane "
                     "read (4 per call) + 15 adder ops; E from the tested sites of each word of a sample of the "
                     "final state (expected_calls_per_word); no queue, index or load/store work counted"}


PIPE_NAMES = {"alu": "ALU pipe (logic, shifts, compares)",
              "fmaheavy": "FMA-heavy pipe (integer multiplies: the Philox products)"}


def kernel_roofline(kernel: str, sites_per_launch: float, t_launch_s: float, sm_max: float, peaks: dict,
                    bytes_per_site: float = BYTES_PER_SITE_SWEEP) -> dict:
    """Roofline of one half-sweep launch.  The sweep is integer work on two pipes of 16
    lanes per scheduler (4 per SM): the ALU pipe (the Philox XORs, the bit-plane
    comparison, the neighbour adder) and the FMA-heavy pipe (the Philox 32x32->64
    products, 4 pipe cycles each).  The binding unit is the one with more busy cycles
    per site in the committed ncu record (sm__pipe_*_cycles_active.sum, summed over the
    4 scheduler pipes of every SM, with a hash of the kernel's sources); `achieved` is
    those busy cycles x 16 lanes per site x sites per launch / CUDA-event time per
    launch, against 64 lanes/clk/SM x SMs x the maximum SM clock, i.e. the pipe's
    utilisation during the timed run.  Records without pipe cycles fall back to the
    executed ALU-pipe operations.  The other pipe, the instruction-issue view (128
    thread slots/clk/SM) and the HBM view ride along."""
    c = committed_counters(kernel)
    alu_peak = ALU_OPS_PER_CLK_SM * N_SMS * sm_max * 1e6 / 1e12
    issue_peak = ISSUE_SLOTS_PER_CLK_SM * N_SMS * sm_max * 1e6 / 1e12
    hbm_bytes = bytes_per_site * sites_per_launch
    out = {"bound": "alu", "achieved": None, "peak": alu_peak, "unit": "Tops/s", "frac": None, "traffic": None,
           "peak_basis": f"4 schedulers x 16 lanes = {ALU_OPS_PER_CLK_SM:.0f} lane-operations/clk/SM per integer "
                         f"pipe x {N_SMS} SMs x {sm_max:.0f} MHz (the probe in this line measures the lanes per "
                         f"clock)",
           "hbm_achieved_gbs": hbm_bytes / t_launch_s / 1e9, "hbm_peak_gbs": peaks.get("hbm_gbs", 6800.0)}
    if c is not None:
        out["counters"] = "current" if c["current"] else "stale: kernel source changed after the capture"
        if c["current"]:
            out["traffic"] = c["dram_bytes_per_site"] * sites_per_launch
        if c.get("pipe_cycles_per_site"):
            views = {}
            for name, cyc in c["pipe_cycles_per_site"].items():
                ach = 16.0 * cyc * sites_per_launch / t_launch_s / 1e12
                views[name] = {"achieved": ach, "frac": ach / alu_peak, "busy_cycles_per_site": cyc}
            pipe = max(views, key=lambda k: views[k]["frac"])
            out["pipe"] = PIPE_NAMES[pipe]
            out["achieved"] = views[pipe]["achieved"]
            out["frac"] = views[pipe]["frac"]
            out["pipe_views"] = {PIPE_NAMES[k]: v for k, v in views.items()}
            if c["alu_ops_per_site"] is not None:
                out["alu_ops_per_site"] = c["alu_ops_per_site"]
        elif c["alu_ops_per_site"] is not None:
            out["pipe"] = PIPE_NAMES["alu"] + ", counted as executed operations"
            out["achieved"] = c["alu_ops_per_site"] * sites_per_launch / t_launch_s / 1e12
            out["frac"] = out["achieved"] / alu_peak
            out["alu_ops_per_site"] = c["alu_ops_per_site"]
        issue = c["inst_slots_per_site"] * sites_per_launch / t_launch_s / 1e12
        out["issue_view"] = {"achieved": issue, "peak": issue_peak, "unit": "Tinst/s", "frac": issue / issue_peak,
                             "inst_slots_per_site": c["inst_slots_per_site"],
                             "basis": f"{ISSUE_SLOTS_PER_CLK_SM:.0f} thread-instruction slots/clk/SM (4 schedulers x 32)"}
    return out


def cpu_baseline_sample(L: int, beta: float, seed: int, start: int) -> dict:
    """The oracle as it stands on this host: one full sweep of the same lattice."""
    import numpy as np

    import oracle

    s = np.empty((L, L), dtype=np.int8)
    oracle.init_rows(s, seed, start, 0, L)
    t0 = time.perf_counter()
    oracle.half_sweep_rows(s, 0, beta, seed, 0, 0, L)
    oracle.half_sweep_rows(s, 1, beta, seed, 0, 0, L)
    dt = time.perf_counter() - t0
    return {"value": L * L / (dt * 1e9), "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS",
                                                                                 os.cpu_count() or 1)),
            "kind": "oracle", "sample": f"one full sweep (black + white) of the {L}x{L} lattice, hot start, "
                                        f"{L * L:.3e} flip attempts, {dt:.1f} s"}


def run_reference(args, rank: int, world: int) -> None:
    """--impl reference: the CPU oracle on bounded row-band samples of the lattice."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1903_11714_gb300 import workloads

    cfg = workloads.single_large()
    L = cfg.L
    rows = args.ref_rows
    s = np.empty((L, L), dtype=np.int8)
    oracle.init_rows(s, cfg.seed, cfg.start, -1, rows + 2)

    def step(k):
        oracle.half_sweep_rows(s, 0, cfg.beta, cfg.seed, k, 0, rows)
        oracle.half_sweep_rows(s, 1, cfg.beta, cfg.seed, k, 0, rows)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = time.perf_counter() - t0
    flips = args.steps * rows * L
    value = flips / (dt * 1e9)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"each step: one sweep of rows 0..{rows - 1} ({rows * L:.3e} sites) of the {L}x{L} lattice, "
              f"hot start, beta {cfg.beta}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": f"single lattice L={L}, beta={cfg.beta}, hot start, seed {cfg.seed} "
                               f"(CPU oracle on a {rows}-row band)", "l2": "lattice > L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _events(torch, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    return e0, e1


def run_single_small(args) -> dict:
    """L = 128, 1000 sweeps: packed (one resident CTA for all sweeps, bound by that
    one SM) vs plain int8 (two launches per sweep, launch-latency bound)."""
    import torch

    from paper_1903_11714_gb300 import ising, workloads

    cfg = workloads.single_small()
    out = {}
    for name, kernel in (("packed", ising.PACKED), ("int8", ising.INT8)):
        st = torch.cuda.Stream()
        lat = ising.Lattice(cfg.L, cfg.beta, cfg.seed, cfg.start, kernel, stream=st)
        lat.sweep(args.warmup)
        lat.synchronize()
        e0, e1 = _events(torch, st)
        e0.record(st)
        lat.sweep(cfg.sweeps)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        lat.close()
        out[name] = cfg.sweeps * cfg.L ** 2 / (ms * 1e6)
    return {"metric": "spin-flip attempts/ns, L=128 single lattice", "workload": "single_small",
            "unit": UNIT, "value": out["packed"], "plain_int8_value": out["int8"], "basis": "CUDA events",
            "config": cfg.as_dict(),
            "note": "packed: one single-CTA launch for all sweeps; int8: 2 launches per sweep (launch-latency bound)"}


def run_batched(args, which: str) -> dict:
    """Batched forms (one persistent launch per half-sweep over all lattices, or, for
    lattices of one side L <= 4096, each resident in a thread-block cluster for up to
    4,096 sweeps per launch) against plain launches of the int8 and packed kernels, one
    lattice at a time."""
    import torch

    from paper_1903_11714_gb300 import ising, workloads

    if which == "scan":
        lats = workloads.temperature_scan()
        graph = workloads.TEMPERATURE_SCAN_GRAPH_SWEEPS
        sweeps = lats[0].sweeps
        max_L = 1024
    else:
        lats = workloads.uneven_batch()
        graph = 100
        sweeps = lats[0].sweeps
        max_L = 4096
    warm = graph * 3 if graph else args.warmup
    arena = sum(l.L * l.L // 8 + 16 * (l.sweeps + warm) + 4096 for l in lats)
    st = torch.cuda.Stream()
    # tile rows and CTA size from the autotuner; one CTA size serves the whole batch,
    # that of the side carrying the most flips
    tiles, tuned_threads = {}, {}
    for L in sorted({l.L for l in lats}):
        if args.batch_tile_rows and args.batch_threads:
            tiles[L], tuned_threads[L] = args.batch_tile_rows, args.batch_threads  # pinned (for profiling)
        else:
            tiles[L], tuned_threads[L], _ = ising.ising_autotune(L)
    work = {L: sum(l.L * l.L for l in lats if l.L == L) for L in tiles}
    threads = tuned_threads[max(work, key=work.get)]
    modes = {"auto": ising.CLUSTER_AUTO, "off": ising.CLUSTER_OFF, "always": ising.CLUSTER_ALWAYS}

    def timed(mode: int, nvtx: bool):
        b = ising.Batch(len(lats), max_L, arena, threads, stream=st)
        b.set_cluster(mode)
        for l in lats:
            b.add(l.L, l.beta, l.seed, l.start, l.sweeps + warm, tiles.get(l.L, 0))
        b.run(warm, graph_sweeps=graph)
        b.synchronize()
        e0, e1 = _events(torch, st)
        if nvtx:
            torch.cuda.nvtx.range_push("timed")  # lets a profiler pick this region's launches
        e0.record(st)
        b.run(sweeps, graph_sweeps=graph)
        e1.record(st)
        torch.cuda.synchronize()
        if nvtx:
            torch.cuda.nvtx.range_pop()
        b.synchronize()
        cluster = b.cluster_size()
        b.close()
        return e0.elapsed_time(e1), cluster

    ms, cluster = timed(modes[args.batch_cluster], True)
    flips = sweeps * sum(l.L * l.L for l in lats)
    batched = flips / (ms * 1e6)
    tiled = roofline = None
    if cluster:
        # the cluster kernel's roofline over the timed launches (up to 4,096 sweeps each):
        # its busier pipe against the whole GPU's; HBM carries only each launch's load and
        # store of the planes and the (M, E) pairs
        launches = -(-sweeps // 4096)
        peaks = measured_peaks()
        plane_bytes = 2 * sum(l.L * l.L // 8 for l in lats) + 16 * len(lats) * sweeps / launches
        roofline = kernel_roofline("cluster_sweep", flips / launches, ms * 1e-3 / launches,
                                   float(peaks.get("sm_max_mhz", 2070.0)), peaks,
                                   bytes_per_site=plane_bytes / (flips / launches))
        # the same batch on the tiled kernel, for comparison
        tiled = flips / (timed(ising.CLUSTER_OFF, False)[0] * 1e6)
    # plain: each lattice alone, its own launches, for a shorter run (same per-sweep work)
    plain = {}
    n_plain = min(sweeps, 100)
    for name, kernel in (("int8", ising.INT8), ("packed", ising.PACKED)):
        total_ms = 0.0
        for l in lats:
            lat = ising.Lattice(l.L, l.beta, l.seed, l.start, kernel, stream=st)
            lat.sweep(2)
            lat.synchronize()
            a0, a1 = _events(torch, st)
            a0.record(st)
            lat.sweep(n_plain)
            a1.record(st)
            torch.cuda.synchronize()
            total_ms += a0.elapsed_time(a1)
            lat.close()
        plain[name] = n_plain * sum(l.L * l.L for l in lats) / (total_ms * 1e6)
    return {"metric": f"aggregate spin-flip attempts/ns, {which} batch", "workload": which,
            "unit": UNIT, "value": batched, "plain_int8_value": plain["int8"],
            "plain_packed_value": plain["packed"], "lattices": len(lats), "sweeps": sweeps,
            "graph_sweeps": graph, "ms": ms, "basis": "CUDA events on the batch's stream",
            "tile_rows_by_L": tiles or None, "threads": threads, "cluster_size": cluster,
            "tiled_value": tiled, "roofline": roofline,
            "note": (f"batched = every lattice resident in the shared memory of a cluster of {cluster} CTAs, "
                     "up to 4,096 sweeps per launch" if cluster else
                     f"batched = one persistent launch per half-sweep over all lattices, a CUDA graph of {graph} "
                     "sweeps replayed") + f"; plain = each lattice alone with its own launches, {n_plain} sweeps each"}


def run_cubic(args) -> None:
    """3D checkerboard sweep (the paper's d-dimensional Hamiltonian at d = 3, Sec. 3 and
    Conclusion): one L = 2048 lattice at beta_c of the cubic lattice, CUDA events over
    the timed sweeps on the handle's stream; roofline on the same multiply-pipe peak."""
    import torch

    from paper_1903_11714_gb300 import ising, workloads

    cfg = workloads.cubic_large()
    L = args.L or cfg.L
    N = L ** 3
    steps = args.steps if args.steps != 200 else cfg.sweeps
    st = torch.cuda.Stream()
    lat = ising.Lattice3D(L, cfg.beta, cfg.seed, cfg.start, stream=st)
    lat.sweep(args.warmup)
    lat.synchronize()
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    e0, e1 = _events(torch, st)
    torch.cuda.synchronize()
    e0.record(st)
    lat.sweep(steps)
    e1.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    lat.synchronize()
    ms = e0.elapsed_time(e1)
    lat.close()
    value = steps * N / (ms * 1e6)
    t_launch_s = ms * 1e-3 / (2 * steps)
    roofline = kernel_roofline("cubic_half_sweep", N / 2, t_launch_s, sm_max, peaks)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cubic_cpu_baseline(cfg.beta, cfg.seed)
    print(json.dumps({
        "metric": "spin-flip attempts/ns, 3D cubic lattice (bit-packed checkerboard sweep, bit-exact)",
        "workload": "cubic", "unit": UNIT, "value": value, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms / steps, "higher_is_better": True,
        "config": {**cfg.as_dict(), "l2": "inputs larger than L2 (1 GB planes vs 129 MB L2), no flush"},
        "roofline": roofline,
        "cpu_baseline": cpu, "gpu_launches": 2 * steps, "clocks": clocks}))


def run_binder3d(args) -> None:
    """3D physics check: U4(beta) for L = 64, 128, 256 near beta_c of the cubic lattice;
    curves of consecutive sizes cross at beta_c up to finite-size corrections.  One
    handle per lattice, each on its own stream so that the small lattices overlap."""
    import torch

    from paper_1903_11714_gb300 import ising, workloads

    sweeps = args.binder3d_sweeps
    burn = sweeps // 10
    lats = workloads.cubic_binder_scan(sweeps)
    streams = [torch.cuda.Stream() for _ in lats]
    hs = [ising.Lattice3D(l.L, l.beta, l.seed, l.start, stream=st) for l, st in zip(lats, streams)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chunk = 1000
    for done in range(0, sweeps, chunk):
        for h in hs:
            h.sweep(min(chunk, sweeps - done))
    for h in hs:
        h.synchronize()
    dt = time.perf_counter() - t0
    table = {}
    for l, h in zip(lats, hs):
        m = h.moments(burn)
        table.setdefault(l.L, []).append((l.beta / workloads.BETA_C3, m["binder"], m["abs_m"], m["e"]))
        h.close()
    crossings = {}
    Ls = sorted(table)
    for L1, L2 in zip(Ls, Ls[1:]):
        a, c = sorted(table[L1]), sorted(table[L2])
        d = [(p[0], p[1] - q[1]) for p, q in zip(a, c)]
        for (b0, d0), (b1, d1) in zip(d, d[1:]):
            if d0 * d1 <= 0 and d0 != d1:
                crossings[f"{L1}-{L2}"] = b0 + (b1 - b0) * d0 / (d0 - d1)
                break
    flips = sweeps * sum(l.L ** 3 for l in lats)
    print(json.dumps({"metric": "3D Binder-parameter scan: U4 vs beta/beta_c (cubic lattice)", "workload": "binder3d",
                      "unit": UNIT, "value": flips / (dt * 1e9), "sweeps": sweeps, "burn_in": burn,
                      "beta_c": workloads.BETA_C3, "crossing_beta_over_beta_c": crossings,
                      "U4": {str(L): [[round(b, 4), u] for b, u, _, _ in sorted(v)] for L, v in table.items()},
                      "e": {str(L): [[round(b, 4), e] for b, _, _, e in sorted(v)] for L, v in table.items()},
                      "note": "wall clock over all lattices (separate streams); value is aggregate flips/ns"}))


def cubic_cpu_baseline(beta: float, seed: int, L: int = 256) -> dict:
    """The 3D oracle as it stands: one sweep of an L = 256 cube (1.7e7 sites)."""
    import oracle

    s = oracle.init3d((L, L, L), seed, oracle.HOT)
    t0 = time.perf_counter()
    oracle.run3d((L, L, L), beta, seed, sweeps=1, state=s)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": L ** 3 / (dt * 1e9), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one sweep of a {L}^3 cube at the same beta (3D oracle, OpenMP)"}


def run_binder(args) -> None:
    """Physics validation: U4(T) and <|m|>(T) for L = 64..512 from one batch; the
    curves of different L cross near T_c (the paper's Fig. 3, reduced)."""
    import numpy as np
    import torch

    from paper_1903_11714_gb300 import ising, workloads

    sweeps = args.binder_sweeps
    burn = sweeps // 10
    lats = workloads.binder_scan(sweeps)
    st = torch.cuda.Stream()
    arena = sum(l.L * l.L // 8 + 16 * l.sweeps + 4096 for l in lats)
    b = ising.Batch(len(lats), max(workloads.BINDER_LS), arena, 0, stream=st)
    idx = [b.add(l.L, l.beta, l.seed, l.start, l.sweeps) for l in lats]
    graph = 1000 if sweeps % 1000 == 0 else 0
    e0, e1 = _events(torch, st)
    e0.record(st)
    b.run(sweeps, graph_sweeps=graph)
    e1.record(st)
    torch.cuda.synchronize()
    b.synchronize()
    ms = e0.elapsed_time(e1)
    table = {}
    for l, i in zip(lats, idx):
        m = b.moments(i, burn)
        table.setdefault(l.L, []).append((workloads.BETA_C_EXACT / l.beta, m["binder"], m["abs_m"], m["e"]))
    b.close()
    # crossings of U4(T) between consecutive sizes (linear interpolation of the difference)
    crossings = {}
    Ls = sorted(table)
    for L1, L2 in zip(Ls, Ls[1:]):
        a = sorted(table[L1])
        c = sorted(table[L2])
        d = [(p[0], p[1] - q[1]) for p, q in zip(a, c)]
        for (t0, d0), (t1, d1) in zip(d, d[1:]):
            if d0 * d1 <= 0 and d0 != d1:
                crossings[f"{L1}-{L2}"] = t0 + (t1 - t0) * d0 / (d0 - d1)
                break
    flips = sweeps * sum(l.L * l.L for l in lats)
    print(json.dumps({"metric": "Binder-parameter scan: U4 and <|m|> vs T/Tc", "workload": "binder",
                      "unit": UNIT, "value": flips / (ms * 1e6), "sweeps": sweeps, "burn_in": burn,
                      "crossing_T_over_Tc": crossings,
                      "U4": {str(L): [[round(t, 4), u] for t, u, _, _ in sorted(v)] for L, v in table.items()},
                      "abs_m": {str(L): [[round(t, 4), m] for t, _, m, _ in sorted(v)] for L, v in table.items()}}))


def saturated_capacity(results) -> float:
    """Flip attempts per second of a calibration run whose requests were all admitted
    at its start, counted up to the moment half of them have finished.  Every quantum
    advances every unfinished lattice by the same number of sweeps, so once the
    finished requests' longest run (S sweeps) is done, each request still running has
    done min(S, its sweeps) sweeps too: the work done by then is the finished
    requests' flips plus L^2 min(S, sweeps) for each of the others (a lower bound: the
    quanta may have gone past S).  Stopping at half leaves out the drained tail, where
    a few long requests keep only part of the GPU busy."""
    res = sorted(results, key=lambda r: r.finished)
    half = max(1, len(res) // 2)
    done, rest = res[:half], res[half:]
    s = max(r.sweeps for r in done)
    work = sum(r.L * r.L * r.sweeps for r in done) + sum(r.L * r.L * min(s, r.sweeps) for r in rest)
    return work / done[-1].finished


def run_serve(args) -> dict:
    """Poisson arrivals at ~80 % of measured capacity; p50/p99 latency."""
    import torch

    from paper_1903_11714_gb300 import ising, serve, workloads

    budget = int(args.serve_budget_gb * (1 << 30))
    st = torch.cuda.Stream()
    # CTA size from the autotuner at the largest request side, which carries most flips
    threads = ising.ising_autotune(8192)[1]
    srv = serve.Server(budget, slots=args.serve_slots, max_L=8192, quantum=args.serve_quantum, threads=threads,
                       stream=st)
    # capacity: a sample of the same request distribution, all present at t = 0, while at
    # least half of it is still running (saturated_capacity); the whole run's average,
    # which includes the drained tail, rides along
    calib = [workloads.Request(rid=r.rid, arrival=0.0, L=r.L, beta=r.beta, seed=r.seed, sweeps=r.sweeps)
             for r in workloads.serving_requests(args.serve_calib, 1.0, seed=55)]
    cres, cst = srv.serve(calib, realtime=False)
    capacity = saturated_capacity(cres)
    capacity_whole = cst.flips / cst.wall_s
    mean_flips = workloads.mean_request_flips()
    rate = 0.8 * capacity / mean_flips
    reqs = workloads.serving_requests(args.serve_requests, rate)
    results, st_ = srv.serve(reqs, realtime=True)
    srv.close()
    summ = st_.summary()
    return {"metric": "serving: p50/p99 latency and aggregate spin-flip attempts/ns",
            "workload": "serve", "unit": UNIT, "value": summ["flips_per_ns"], "basis": "wall clock, real-time arrivals",
            "p50_s": summ["p50_s"], "p99_s": summ["p99_s"], "requests": summ["completed"],
            "rate_per_s": rate, "capacity_flips_per_ns": capacity / 1e9,
            "capacity_basis": f"{len(calib)} requests present at t = 0, work done until half of them finished",
            "capacity_whole_run_flips_per_ns": capacity_whole / 1e9,
            "mean_request_flips": mean_flips, "hbm_budget_gb": args.serve_budget_gb,
            "slots": args.serve_slots, "quantum_sweeps": args.serve_quantum or "adaptive (8..256)",
            "threads": threads, "quanta": summ["quanta"],
            "max_active": summ["max_active"], "max_arena_gb": summ["max_arena_bytes"] / 2**30,
            "blocked_by_memory": summ["blocked_by_memory"], "blocked_by_slots": summ["blocked_by_slots"]}


def make_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kernel", choices=["packed", "int8"], default="packed")
    ap.add_argument("--L", type=int, default=0, help="override the lattice side (profiling only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-rows", type=int, default=1024)
    ap.add_argument("--workload", choices=["single_large", "single_small", "scan", "uneven", "serve", "binder",
                                           "cubic", "binder3d"],
                    default="single_large")
    ap.add_argument("--config", type=int, choices=[1, 2, 3, 4, 5], default=0,
                    help="the five benchmark configurations: 1 = L=128 single (single_small), "
                         "2 = L=65,536 single (single_large), 3 = temperature scan (scan), "
                         "4 = uneven batch (uneven), 5 = serving loop (serve)")
    ap.add_argument("--binder-sweeps", type=int, default=1_000_000)
    ap.add_argument("--binder3d-sweeps", type=int, default=100_000)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-calib", type=int, default=150)
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--serve-quantum", type=int, default=0, help="sweeps per quantum; 0 = adaptive")
    ap.add_argument("--batch-tile-rows", type=int, default=0,
                    help="scan / uneven: tile rows for every side instead of the autotuner's (with --batch-threads)")
    ap.add_argument("--batch-threads", type=int, default=0, help="scan / uneven: CTA size instead of the autotuner's")
    ap.add_argument("--batch-cluster", choices=["auto", "off", "always"], default="auto",
                    help="scan / uneven: cluster-resident form of one-side batches (ising_batch_set_cluster)")
    ap.add_argument("--no-sub", action="store_true",
                    help="default run: skip the repeats and the records of configurations 1, 3, 4, 5 and int8")
    ap.add_argument("--repeats", type=int, default=5, help="extra timings of the K timed steps (spread)")
    ap.add_argument("--sub-serve-requests", type=int, default=600,
                    help="requests of the serving record appended to the default run")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    return ap


def main() -> None:
    args = make_parser().parse_args()
    if args.config:
        args.workload = {1: "single_small", 2: "single_large", 3: "scan", 4: "uneven", 5: "serve"}[args.config]
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    from paper_1903_11714_gb300 import build as libbuild
    from paper_1903_11714_gb300 import ising, workloads

    torch.cuda.set_device(local)
    if args.workload != "single_large":
        libbuild.build()
        rec = {"single_small": run_single_small, "serve": run_serve, "binder": run_binder, "cubic": run_cubic,
               "binder3d": run_binder3d}.get(args.workload, lambda a: run_batched(a, args.workload))(args)
        if rec is not None:
            print(json.dumps(rec))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    libbuild.build()
    cfg = workloads.single_large()
    L = args.L or cfg.L
    kernel = ising.PACKED if args.kernel == "packed" else ising.INT8
    seed = cfg.seed + rank
    stream = torch.cuda.Stream()
    t_setup = time.perf_counter()
    lat = ising.Lattice(L, cfg.beta, seed, cfg.start, kernel, stream=stream)
    t_setup = time.perf_counter() - t_setup
    specialized, kernel_note = lat.specialized()
    lat.sweep(args.warmup)
    lat.synchronize()
    N = L * L

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    mul_per_clk, alu_per_clk = ising.ising_probe_int_rates()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lat.sweep(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    lat.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    flips_all = total_over_ranks(float(args.steps * N), dist, "cuda")
    value = flips_all / (ms * 1e6)

    # dominant kernel: the packed half-sweep (2 launches per sweep + 1 counter advance per call)
    launches = 2 * args.steps + 1
    t_launch_s = ms * 1e-3 / (2 * args.steps)
    if kernel == ising.PACKED:
        roofline = kernel_roofline("packed_half_sweep", N / 2, t_launch_s, sm_max, peaks)
    else:
        # the int8 kernel reads and writes every byte of the lattice per half-sweep
        roofline = kernel_roofline("int8_half_sweep", N / 2, t_launch_s, sm_max, peaks, bytes_per_site=INT8_BYTES_PER_SITE)
    roofline["probe_alu_ops_per_clk_sm"] = alu_per_clk
    roofline["probe_mul_xor_steps_per_clk_sm"] = mul_per_clk
    if kernel == ising.PACKED:
        # the counted model's fraction beside the executed one, from 64 rows of the state
        T2, T4 = ising.ising_thresholds(cfg.beta)
        nrow = min(66, L)
        roofline["algorithmic"] = algorithmic_view(lat.get_rows(0, nrow), T2, T4, (N / 2) / t_launch_s, sm_max)
        roofline["algorithmic"]["sample"] = f"rows 1..{nrow - 2} of the state after the timed sweeps"

    # the same K timed steps again, for the run-to-run spread (the lattice continues its chain)
    reps = []
    for _ in range(args.repeats if not args.no_sub else 0):
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        r0.record(stream)
        lat.sweep(args.steps)
        r1.record(stream)
        torch.cuda.synchronize()
        reps.append(args.steps * N / (r0.elapsed_time(r1) * 1e6))
    lat.synchronize()
    repeats = None
    if reps:
        allv = [value] + reps if world == 1 else reps
        repeats = {"timings": len(allv), "values": allv, "median": statistics.median(allv), "min": min(allv),
                   "max": max(allv), "spread_pct": 100.0 * (max(allv) - min(allv)) / statistics.median(allv),
                   "basis": f"the {args.steps} timed steps, then {len(reps)} more timings of {args.steps} steps each "
                            f"(CUDA events, same lattice continuing its chain)"}

    e2e = None
    if not args.no_e2e and kernel == ising.PACKED and rank == 0:
        e2e = measure_e2e(lat, L, cfg, args.steps, stream)
    lat.close()

    # the rest of the metric ("batched vs plain; p50/p99 latency"): records of the other
    # configurations and of the plain int8 kernel on this one, each with its own basis
    sub = None
    if rank == 0 and world == 1 and not args.no_sub and kernel == ising.PACKED and not args.L:
        sub = {"config2_plain_int8": run_plain_int8(cfg, args.steps, args.warmup),
               "config1_single_small": run_single_small(args),
               "config3_scan": run_batched(args, "scan"),
               "config4_uneven": run_batched(args, "uneven")}
        sargs = argparse.Namespace(**vars(args))
        sargs.serve_requests = args.sub_serve_requests
        sub["config5_serve"] = run_serve(sargs)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(L, cfg.beta, cfg.seed, cfg.start)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 bit-packed spins, u32 Philox / integer thresholds",
            "data": "synthetic",
            "config": {"workload": f"single lattice L={L}, beta={cfg.beta}, hot start, seed {cfg.seed}"
                                   f"{' + rank' if world > 1 else ''}, {args.kernel} kernel",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (512 MB planes vs 129 MB L2), no flush"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "repeats": repeats, "sub": sub,
            "kernel": {"specialized": specialized, "note": kernel_note, "handle_setup_s": round(t_setup, 3),
                       "basis": "the sweep kernel compiled for this lattice's thresholds when the handle is "
                                "created (NVRTC, once per threshold pair and process, outside the timed region; "
                                "handle_setup_s includes it)"},
        }))
    if dist:
        dist.destroy_process_group()


def run_plain_int8(cfg, steps: int, warmup: int) -> dict:
    """The plain int8 kernel (row-major bytes, one lattice) on the same lattice and steps."""
    import torch

    from paper_1903_11714_gb300 import ising

    st = torch.cuda.Stream()
    lat = ising.Lattice(cfg.L, cfg.beta, cfg.seed, cfg.start, ising.INT8, stream=st)
    lat.sweep(warmup)
    lat.synchronize()
    e0, e1 = _events(torch, st)
    e0.record(st)
    lat.sweep(steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lat.close()
    N = cfg.L * cfg.L
    peaks = measured_peaks()
    roof = kernel_roofline("int8_half_sweep", N / 2, ms * 1e-3 / (2 * steps), float(peaks.get("sm_max_mhz", 2070.0)),
                           peaks, bytes_per_site=INT8_BYTES_PER_SITE)
    return {"metric": "spin-flip attempts/ns, plain int8 kernel", "workload": "single_large", "unit": UNIT,
            "value": steps * N / (ms * 1e6), "steps": steps, "basis": "CUDA events", "roofline": roof,
            "note": "row-major int8 lattice (4.3 GB), each half-sweep reads and writes every byte"}


E2E_RUNS = 3  # wall-clocked runs of the end-to-end measurement (host copies vary run to run)


def measure_e2e(lat, L, cfg, steps, stream) -> dict:
    """Same metric through the C ABI with host buffers: upload the start planes
    from pinned host memory, sweep, read back the M/E history and the final planes."""
    import numpy as np
    import torch

    from paper_1903_11714_gb300 import ising

    words = L * (L // 64)
    e = ising.Lattice(L, cfg.beta, cfg.seed, cfg.start, ising.PACKED, stream=stream)
    black = torch.empty(words, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    white = torch.empty(words, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    b0, w0 = e.get_planes()
    black[:] = b0
    white[:] = w0
    del b0, w0
    e.close()
    start_b, start_w = black.copy(), white.copy()
    values = []
    for _ in range(E2E_RUNS):
        black[:] = start_b
        white[:] = start_w
        h = ising.Lattice(L, cfg.beta, cfg.seed, ising.COLD, ising.PACKED, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.set_planes(black, white)
        h.sweep(steps)
        M, E = h.history(0, steps)
        h.get_planes(black, white)
        dt = time.perf_counter() - t0
        h.close()
        values.append(steps * L * L / (dt * 1e9))
    h2d = 2 * words * 4
    d2h = 2 * words * 4 + 16 * steps
    return {"value": statistics.median(values), "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps, "runs": values,
            "note": f"median of {E2E_RUNS} runs, each on a fresh handle: start planes host->device, the sweeps, M/E "
                    "history and final planes device->host, all pinned host buffers, wall clock"}


if __name__ == "__main__":
    main()
