"""Pins the oracle's acceptance thresholds and decision rule (Sec. 3.1).

T_h = min(2^32, ceil(exp(-2 beta h) 2^32)) is checked against 50-digit
arithmetic (mpmath), which shares nothing with the libm exp the oracle uses.
The decision x < T_h is checked at its boundary, so accept() is the indicator
of [0, T_h) and its acceptance probability is exactly T_h / 2^32.
"""
import mpmath as mp
import pytest

import oracle

BETAS = [0.0, 1e-9, 0.1, 0.25, 0.35, 0.4406868, 0.44068679350977151, 0.5, 0.55, 0.6, 1.0, 2.5, 5.0, 20.0]


@pytest.mark.parametrize("beta", BETAS)
def test_thresholds_vs_high_precision(beta):
    T2, T4 = oracle.thresholds(beta)
    with mp.workdps(50):
        for h, T in ((2, T2), (4, T4)):
            exact = mp.exp(-2 * mp.mpf(beta) * h) * 2**32
            ceil_exact = int(mp.ceil(exact))
            frac = exact - mp.floor(exact)
            if min(frac, 1 - frac) > mp.mpf("1e-6"):
                assert T == min(ceil_exact, 2**32), (beta, h)
            else:  # libm may round across an integer; still within one
                assert abs(T - ceil_exact) <= 1
            # the acceptance probability T / 2^32 is within 2^-32 of exp(-2 beta h)
            assert abs(mp.mpf(T) / 2**32 - exact / 2**32) <= mp.mpf(2) ** -32


def test_threshold_special_values():
    assert oracle.thresholds(0.0) == (2**32, 2**32)  # beta = 0: every flip accepted
    assert oracle.thresholds(200.0) == (0, 0)  # exp underflows: zero temperature
    # printed to 14 digits at beta = 0.4406868 from exp(-4 beta), exp(-8 beta)
    assert oracle.thresholds(0.4406868) == (736899869, 126432027)


@pytest.mark.parametrize("beta", [0.2, 0.4406868, 0.7])
def test_accept_is_prefix_indicator(beta):
    T2, T4 = oracle.thresholds(beta)
    for h in (-4, -2, 0):
        for x in (0, 1, T4, T2, 2**31, 2**32 - 1):
            assert oracle.accept(h, x, T2, T4)
    for h, T in ((2, T2), (4, T4)):
        assert oracle.accept(h, 0, T2, T4)
        assert oracle.accept(h, T - 1, T2, T4)
        assert not oracle.accept(h, T, T2, T4)
        assert not oracle.accept(h, 2**32 - 1, T2, T4)


def test_accept_edge_thresholds():
    assert oracle.accept(2, 2**32 - 1, 2**32, 2**32)  # T = 2^32 accepts every word
    assert not oracle.accept(4, 0, 5, 0)  # T = 0 accepts none
