"""Failure detection of the sweep kernel's bounded waits, without a GPU fault.

The self-test launches one half-sweep whose tile barriers expect 16 bytes that
are never sent, with each wait bounded by ~1 ms of SM clocks.  The kernel must
give up, record the timeout in its status word, return, and leave the context
usable (a normal sweep afterwards succeeds).  Nothing traps, faults or spins
without a bound.
"""
import pytest

from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_recovers():
    libbuild.build()
    observed = ising.ising_selftest_timeout(2_000_000)
    assert observed == ising.ISING_ETIMEOUT
    # and a fresh lattice still sweeps correctly afterwards
    lat = ising.Lattice(128, 0.44, 1).sweep(3)
    lat.synchronize()
    lat.close()
