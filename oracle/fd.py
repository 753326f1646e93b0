"""Central finite-difference weights for the second derivative (oracle).

The paper discretises the Kohn-Sham equations with a high-order finite-difference
approach on a uniform real-space grid (Abstract; Intro, the PARSEC paragraph).  The
order is not printed; order 2M = 12 (M = 6 neighbours per side) is used.

Weights w_0..w_M make  f''(0) ~ h^-2 [ w_0 f(0) + sum_k w_k (f(kh) + f(-kh)) ]
exact for all polynomials of degree <= 2M+1.  They are found here by solving the
moment equations in exact rational arithmetic (even monomials x^{2q}, q = 0..M):
    q = 0 : w_0 + 2 sum_k w_k         = 0
    q = 1 : 2 sum_k w_k k^2           = 2
    q >= 2: 2 sum_k w_k k^{2q}        = 0
(odd monomials are exact by symmetry).
"""
from __future__ import annotations

from fractions import Fraction


def second_derivative_weights(M: int = 6) -> list[Fraction]:
    """[w_0, w_1, ..., w_M] as exact fractions."""
    n = M + 1
    A = [[Fraction(0)] * n for _ in range(n)]
    rhs = [Fraction(0)] * n
    for q in range(n):
        A[q][0] = Fraction(1 if q == 0 else 0)
        for k in range(1, M + 1):
            A[q][k] = Fraction(2 * k ** (2 * q))
        rhs[q] = Fraction(2 if q == 1 else 0)
    # Gauss-Jordan elimination over the rationals
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        rhs[col], rhs[piv] = rhs[piv], rhs[col]
        inv = 1 / A[col][col]
        A[col] = [x * inv for x in A[col]]
        rhs[col] *= inv
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
                rhs[r] -= f * rhs[col]
    return rhs


def weights_float(M: int = 6):
    return [float(w) for w in second_derivative_weights(M)]
