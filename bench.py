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
# algorithmic work per site per sweep: 1/4 Philox4x32-10 call = 5 32x32->64 multiplies
MULS_PER_SITE_SWEEP = 5.0
# algorithmic bytes per site per sweep (packed): each half-sweep reads the target
# and source planes and writes the target plane, N/2 bits each
BYTES_PER_SITE_SWEEP = 3.0 * 2 * (0.5 / 8.0)


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


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("sweep_packed.cu", "philox.cuh", "ising_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1903_11714_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(L: int):
    """DRAM bytes per half-sweep launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "packed_half_sweep_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    per_site = d.get("dram_bytes_per_site_per_launch")
    return None if per_site is None else per_site * L * L


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


def main() -> None:
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
    args = ap.parse_args()
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
    lat = ising.Lattice(L, cfg.beta, seed, cfg.start, kernel, stream=stream)
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
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * args.steps * N / (ms * 1e6)

    # dominant kernel: the packed half-sweep (2 launches per sweep + 1 counter advance per call)
    launches = 2 * args.steps + 1
    t_launch_s = ms * 1e-3 / (2 * args.steps)
    muls_per_launch = MULS_PER_SITE_SWEEP * N / 2
    achieved = muls_per_launch / t_launch_s / 1e12
    peak = mul_per_clk * 152 * sm_max * 1e6 / 1e12
    bytes_per_launch = BYTES_PER_SITE_SWEEP * N / 2
    traffic = committed_traffic(L) if kernel == ising.PACKED else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tmul/s", "frac": achieved / peak,
                "traffic": traffic,
                "peak_basis": f"{mul_per_clk:.1f} 32x32->64 multiplies/clk/SM (probe) x 152 SMs x {sm_max:.0f} MHz",
                "hbm_achieved_gbs": bytes_per_launch / t_launch_s / 1e9,
                "hbm_peak_gbs": peaks.get("hbm_gbs", 6800.0),
                "alu_ops_per_clk_sm_probe": alu_per_clk}

    e2e = None
    if not args.no_e2e and kernel == ising.PACKED and rank == 0:
        e2e = measure_e2e(lat, L, cfg, args.steps, stream)
    lat.close()

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
        }))
    if dist:
        dist.destroy_process_group()


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
    h = ising.Lattice(L, cfg.beta, cfg.seed, ising.COLD, ising.PACKED, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.set_planes(black, white)
    h.sweep(steps)
    M, E = h.history(0, steps)
    h.get_planes(black, white)
    dt = time.perf_counter() - t0
    h.close()
    h2d = 2 * words * 4
    d2h = 2 * words * 4 + 16 * steps
    return {"value": steps * L * L / (dt * 1e9), "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps,
            "note": "one run per measurement: start planes host->device, the sweeps, M/E history and final planes "
                    "device->host, all pinned host buffers, wall clock"}


if __name__ == "__main__":
    main()
