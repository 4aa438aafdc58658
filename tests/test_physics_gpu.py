"""Physics of the GPU chain (beyond bit-exactness): the paper's correctness check
(Sec. 4.1, Fig. 3) in reduced form.  Below T_c the Binder parameter grows with L
towards 2/3 and <|m|> sits near Onsager's spontaneous magnetisation; above T_c
(correlation length ~6 sites at 1.1 T_c) U4 is near 0 for every L -- there its
size ordering is within the statistical noise, so the size trend is checked on
<|m|>, which falls like 1/L once L is much larger than the correlation length."""
import pytest

from oracle import exact
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising, workloads

pytestmark = pytest.mark.gpu


def test_binder_parameter_orders_with_size_on_both_sides_of_tc():
    libbuild.build()
    sweeps, burn = 40_000, 4_000
    bc = workloads.BETA_C_EXACT
    specs = [(L, t) for L in (64, 128, 256) for t in (0.9, 1.1)]
    b = ising.Batch(len(specs), 256, sum(L * L // 8 + 16 * sweeps + 4096 for L, _ in specs))
    idx = {(L, t): b.add(L, bc / t, 1000 + L + int(100 * t), ising.COLD, sweeps) for L, t in specs}
    b.run(sweeps, graph_sweeps=1000)
    u = {k: b.moments(i, burn)["binder"] for k, i in idx.items()}
    m = {k: b.moments(i, burn)["abs_m"] for k, i in idx.items()}
    b.close()
    assert u[(64, 0.9)] < u[(128, 0.9)] < u[(256, 0.9)] < 2 / 3 + 1e-9
    assert all(-0.05 < u[(L, 1.1)] < 0.1 for L in (64, 128, 256)), u
    assert m[(64, 1.1)] > 1.5 * m[(128, 1.1)] > 2.25 * m[(256, 1.1)], m
    assert abs(m[(256, 0.9)] - exact.onsager_m0(bc / 0.9)) < 0.01
