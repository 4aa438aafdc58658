"""The serving loop: continuous batching keeps every request's result identical
to the same request run alone (and to the oracle), while admission respects
the slot count and the HBM budget."""
import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising, serve
from paper_1903_11714_gb300.workloads import Request, serving_requests

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    ising.lib()


def _requests(n=24, seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        # the first four are large and arrive together: the budget below holds three
        L = 512 if k < 4 else int(rng.choice([64, 128, 192, 256, 512]))
        out.append(Request(rid=k, arrival=0.0 if k < 4 else float(k // 3), L=L, beta=float(rng.uniform(0.3, 0.6)),
                           seed=1000 + k, sweeps=int(rng.integers(10, 150))))
    return out


def test_results_identical_alone_and_in_the_mix():
    reqs = _requests()
    # 6 slots and a budget that admits only a few large lattices at once
    srv = serve.Server(hbm_budget_bytes=3 * (512 * 512 // 8 + 16 * 150) + 4096, slots=6, max_L=512, quantum=16)
    results, st = srv.serve(reqs, realtime=False, keep_lattices=True, keep_history=True)
    srv.close()
    assert st.completed == len(reqs)
    assert st.max_active <= 6
    assert st.admission_blocked_by_memory > 0  # the budget, not only the slots, limited admission
    by_id = {r.rid: r for r in results}
    for q in reqs:
        r = by_id[q.rid]
        alone = ising.Lattice(q.L, q.beta, q.seed, ising.HOT).sweep(q.sweeps)
        M, E = alone.history()
        assert np.array_equal(r.history[0], M) and np.array_equal(r.history[1], E), q.rid
        assert np.array_equal(r.lattice, alone.get_lattice()), q.rid
        assert (r.M, r.E) == (int(M[-1]), int(E[-1]))
        alone.close()
    for q in reqs[:4]:
        ref, Mr, Er, _ = oracle.run(q.L, q.beta, q.seed, oracle.HOT, q.sweeps)
        assert np.array_equal(by_id[q.rid].lattice, ref)
        assert np.array_equal(by_id[q.rid].history[0], Mr)


def test_realtime_poisson_arrivals_complete_with_latencies():
    reqs = [Request(rid=r.rid, arrival=r.arrival, L=min(r.L, 1024), beta=r.beta, seed=r.seed,
                    sweeps=min(r.sweeps, 300)) for r in serving_requests(40, rate_per_s=200.0)]
    srv = serve.Server(hbm_budget_bytes=1 << 30, slots=16, max_L=1024, quantum=32)
    results, st = srv.serve(reqs, realtime=True)
    srv.close()
    s = st.summary()
    assert s["completed"] == 40 and s["p50_s"] > 0 and s["p99_s"] >= s["p50_s"]
    assert all(r.finished >= r.arrival for r in results)


def test_request_that_can_never_fit_is_rejected():
    srv = serve.Server(hbm_budget_bytes=1 << 16, slots=2, max_L=1024, quantum=8)
    with pytest.raises(ValueError):
        srv.serve([Request(rid=0, arrival=0.0, L=1024, beta=0.4, seed=1, sweeps=10)], realtime=False)
    srv.close()
