"""Pin the bond probability P = 1 - exp(-2J/T) of Sec. I step 1.

At the critical temperature of the square-lattice Ising model,
T_c = 2J / ln(1 + sqrt 2), the identity 1 - exp(-2J/T_c) = 2 - sqrt 2 holds
exactly, so floor((2 - sqrt 2) 2^32) can be computed in exact integer
arithmetic and the oracle's threshold must land within one unit of it.  A
dropped factor 2, a wrong sign or J/T swapped fails this.
"""
import math

import pytest


def _exact_tc_threshold() -> int:
    # floor((2 - sqrt2) * 2^32) = 2^33 - ceil(sqrt(2^65)); sqrt(2^65) is irrational
    return (1 << 33) - (math.isqrt(1 << 65) + 1)


def test_threshold_at_tc_is_two_minus_sqrt2(orc):
    exact = _exact_tc_threshold()
    assert exact == 2515933592
    tc = 2.0 / math.log1p(math.sqrt(2.0))
    assert abs(orc.threshold_T(1.0, tc) - exact) <= 1
    # J/T enters only as a ratio
    assert abs(orc.threshold_T(2.0, 2.0 * tc) - exact) <= 1
    assert abs(orc.threshold_p(2.0 - math.sqrt(2.0)) - exact) <= 1


def test_threshold_limits(orc):
    assert orc.threshold_p(0.0) == 0
    assert orc.threshold_p(-0.5) == 0
    assert orc.threshold_p(1.0) == 1 << 32
    assert orc.threshold_p(0.5) == 1 << 31
    assert orc.threshold_p(0.25) == 1 << 30
    assert orc.threshold_p(2.0 ** -32) == 1
    assert orc.threshold_p(1.0 - 2.0 ** -53) == (1 << 32) - 1
    assert orc.threshold_T(0.0, 2.0) == 0              # no coupling: no bonds
    assert orc.threshold_T(1.0, math.inf) == 0         # infinite temperature
    assert orc.threshold_T(1.0, 1e-300) == 1 << 32     # zero temperature


def test_threshold_monotone_in_T(orc):
    ts = [orc.threshold_T(1.0, T) for T in (0.5, 1.0, 1.8, 2.0, 2.269185, 2.6, 3.0, 3.2, 10.0)]
    assert all(a > b for a, b in zip(ts, ts[1:]))


@pytest.mark.parametrize("T,expected", [(2.0, 2714937127), (2.269185, 2515933809), (3.0, 2089857560)])
def test_threshold_at_config_temperatures(orc, T, expected):
    """Regression values at the workload temperatures (T = 2.269185 is the
    rounded T_c of the critical configuration; it lies 217 units above the
    exact-T_c threshold)."""
    assert orc.threshold_T(1.0, T) == expected
    # the same value from an independent evaluation of the closed form
    assert math.floor(math.ldexp(-math.expm1(-2.0 / T), 32)) == expected
