"""Pins for the oracle's Boys function F_m(T) = int_0^1 u^{2m} exp(-T u^2) du."""
import math

mpmath = __import__("pytest").importorskip("mpmath")
import numpy as np
import pytest

pytestmark = []


def ref_boys(m, T):
    # definition via the lower incomplete gamma function, 40 significant digits
    mpmath.mp.dps = 40
    if T == 0:
        return 1.0 / (2 * m + 1)
    return float(mpmath.gammainc(m + 0.5, 0, T) / (2 * mpmath.mpf(T) ** (m + 0.5)))


@pytest.mark.parametrize("T", [0.0, 1e-8, 0.3, 1.0, 7.5, 17.2, 29.99, 30.0, 30.01, 45.0, 200.0])
def test_boys_against_incomplete_gamma(oracle, T):
    F = oracle.boys(12, T)
    for m in range(13):
        ref = ref_boys(m, T)
        assert abs(F[m] - ref) <= 2e-15 * abs(ref) + 1e-300, (m, T, F[m], ref)


def test_boys_at_zero_and_erf_form(oracle):
    F = oracle.boys(9, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(10)], rtol=0, atol=1e-16)
    for T in (0.5, 3.0, 25.0, 60.0):
        f0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        assert abs(oracle.boys(0, T)[0] - f0) < 1e-15 * f0


def test_boys_recursion_and_asymptote(oracle):
    for T in (0.2, 4.0, 29.0, 31.0, 80.0):
        F = oracle.boys(10, T)
        for m in range(10):
            lhs = (2 * m + 1) * F[m]
            rhs = 2 * T * F[m + 1] + math.exp(-T)
            assert abs(lhs - rhs) <= 1e-14 * lhs
    T = 400.0
    F = oracle.boys(8, T)
    for m in range(9):
        df = 1.0
        for k in range(2 * m - 1, 0, -2):
            df *= k
        asym = df / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert abs(F[m] - asym) <= 1e-14 * asym
