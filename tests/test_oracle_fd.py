"""Pins of the oracle's finite-difference weights (order-12 central second derivative)."""
from fractions import Fraction
from math import factorial, cos, pi

import numpy as np
import pytest

from oracle.fd import second_derivative_weights


def closed_form(M):
    # Known closed form of the central 2M-order weights (a different derivation
    # from the oracle's moment equations):
    #   w_k = 2 (-1)^(k+1) (M!)^2 / (k^2 (M-k)! (M+k)!),  w_0 = -2 sum_k w_k
    wk = [Fraction(2 * (-1) ** (k + 1) * factorial(M) ** 2, k * k * factorial(M - k) * factorial(M + k))
          for k in range(1, M + 1)]
    return [-2 * sum(wk)] + wk


@pytest.mark.parametrize("M", [1, 2, 3, 6])
def test_weights_equal_closed_form(M):
    assert second_derivative_weights(M) == closed_form(M)


def test_order12_values():
    w = second_derivative_weights(6)
    assert w[0] == Fraction(-5369, 1800)
    assert w[1:] == [Fraction(12, 7), Fraction(-15, 56), Fraction(10, 189), Fraction(-1, 112),
                     Fraction(2, 1925), Fraction(-1, 16632)]


@pytest.mark.parametrize("x0", [Fraction(0), Fraction(3, 7), Fraction(-5, 2)])
def test_exact_on_polynomials_up_to_degree_13(x0):
    w = second_derivative_weights(6)
    for q in range(0, 16):
        approx = w[0] * x0 ** q + sum(w[k] * ((x0 + k) ** q + (x0 - k) ** q) for k in range(1, 7))
        exact = q * (q - 1) * x0 ** (q - 2) if q >= 2 else Fraction(0)
        if q <= 13:
            assert approx == exact, q
    # degree 14 is not exact: the scheme is order 12, not higher
    q = 14
    approx = w[0] * 0 + sum(w[k] * (Fraction(k) ** q * 2) for k in range(1, 7))
    assert approx != 0


def test_symbol():
    w = [float(x) for x in second_derivative_weights(6)]
    sym = lambda t: -(w[0] + 2 * sum(w[k] * cos(k * t) for k in range(1, 7)))
    # consistency: symbol ~ theta^2 with an O(theta^14) error
    for t in [1e-2, 0.1, 0.3]:
        assert abs(sym(t) - t * t) < 1e-12 + 1e-3 * t ** 14
    # maximum at theta = pi equals |w0| + 2 sum |w_k|
    ts = np.linspace(0, pi, 20001)
    vals = np.array([sym(t) for t in ts])
    assert abs(vals.max() - sym(pi)) < 1e-12
    assert abs(sym(pi) - (abs(w[0]) + 2 * sum(abs(x) for x in w[1:]))) < 1e-12
