"""Writes the stored expected values used by the parity tests.

Every value here comes from the CPU oracle (``oracle/``) and nothing else:
the final-lattice SHA-256 and the per-sweep integer M and E for the L = 128
(1000 sweeps) and L = 65,536 (200 sweeps) single-lattice workloads, and for the
first two sweeps of the 3D workload (L = 2048 cube).

    python tests/golden/make_golden.py small   # seconds
    python tests/golden/make_golden.py large   # about an hour on 8 cores, 4.3 GB RAM
    python tests/golden/make_golden.py cubic   # minutes on 8 cores, 8.6 GB RAM
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1903_11714_gb300 import workloads  # noqa: E402


def make(cfg, name):
    t0 = time.time()
    s, M, E, _ = oracle.run(cfg.L, cfg.beta, cfg.seed, cfg.start, cfg.sweeps)
    dt = time.time() - t0
    out = {
        "source": "oracle/ising_oracle.c via tests/golden/make_golden.py",
        "workload": cfg.as_dict(),
        "sha256": oracle.lattice_hash(s),
        "M": [int(v) for v in M],
        "E": [int(v) for v in E],
        "oracle_seconds": round(dt, 1),
        "oracle_threads": os.environ.get("OMP_NUM_THREADS", str(os.cpu_count())),
    }
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path, out["sha256"], f"{dt:.1f}s")


CUBIC_SWEEPS = 2


def make_cubic(name):
    cfg = workloads.cubic_large()
    t0 = time.time()
    s, M, E, _ = oracle.run3d((cfg.L,) * 3, cfg.beta, cfg.seed, cfg.start, CUBIC_SWEEPS)
    dt = time.time() - t0
    workload = cfg.as_dict()
    workload["sweeps"] = CUBIC_SWEEPS
    out = {
        "source": "oracle/ising3d_oracle.c via tests/golden/make_golden.py",
        "workload": workload,
        "sha256": oracle.lattice_hash(s),
        "M": [int(v) for v in M],
        "E": [int(v) for v in E],
        "oracle_seconds": round(dt, 1),
        "oracle_threads": os.environ.get("OMP_NUM_THREADS", str(os.cpu_count())),
    }
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path, out["sha256"], f"{dt:.1f}s")


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "small"
    if which in ("small", "all"):
        make(workloads.single_small(), "single_L128_1000sweeps.json")
    if which in ("large", "all"):
        make(workloads.single_large(), "single_L65536_200sweeps.json")
    if which in ("cubic", "all"):
        make_cubic("cubic_L2048_2sweeps.json")
