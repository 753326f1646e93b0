"""Lanczos bounds of the spectrum (oracle, float64) -- test infrastructure only.

The filter's upper bound b must lie above the spectrum of H; a few Lanczos steps give a
tighter one than Weyl + Gershgorin (the estimate of Zhou & Li 2011, also used for the
CheFSI filter interval by Zhou, Saad, Tiago & Chelikowsky 2006):
    v_1 = x / |x|,  beta_0 = 0,
    for j = 1..K:  w = H v_j - beta_{j-1} v_{j-1};  alpha_j = <v_j, w>;  w -= alpha_j v_j;
                   beta_j = |w|;  v_{j+1} = w / beta_j
    T = tridiag(beta_{1..K-1}; alpha_{1..K}; beta_{1..K-1}),
    upper = theta_max(T) + beta_K,   lower estimate = theta_min(T).
Inner products use the grid weight h^3.  The start vector x is column 0 of the seeded
initial block (the counter-based generator of the initial subspace).  Eigenvalues of T
by Sturm-sequence bisection (a textbook method; checked against LAPACK in the tests).
"""
from __future__ import annotations

import numpy as np


def sturm_count(alpha, beta, x: float) -> int:
    """Number of eigenvalues of the symmetric tridiagonal T that are < x."""
    count = 0
    d = 1.0
    for j in range(len(alpha)):
        off = beta[j - 1] ** 2 if j > 0 else 0.0
        d = alpha[j] - x - (off / d if j > 0 else 0.0)
        if d == 0.0:
            d = -1e-300
        if d < 0.0:
            count += 1
    return count


def tridiag_eigs_bisect(alpha, beta, iters: int = 200):
    """All eigenvalues of T (ascending) by bisection on the Sturm count."""
    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    n = len(alpha)
    r = np.zeros(n)
    for j in range(n):
        r[j] = (abs(beta[j - 1]) if j > 0 else 0.0) + (abs(beta[j]) if j < n - 1 else 0.0)
    lo0 = float(np.min(alpha - r)) - 1.0
    hi0 = float(np.max(alpha + r)) + 1.0
    out = np.empty(n)
    for i in range(n):                   # i-th smallest: the x where the count passes i
        lo, hi = lo0, hi0
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            if sturm_count(alpha, beta, mid) > i:
                hi = mid
            else:
                lo = mid
        out[i] = 0.5 * (lo + hi)
    return out


def lanczos(H, x0: np.ndarray, K: int):
    """(alpha (K,), beta (K,), upper, lower) for H (oracle Hamiltonian: H.apply, H.h3)."""
    h3 = H.h3
    v = x0 / np.sqrt(h3 * float(x0 @ x0))
    v_prev = np.zeros_like(v)
    alpha = np.zeros(K)
    beta = np.zeros(K)
    b_prev = 0.0
    for j in range(K):
        w = H.apply(v[:, None])[:, 0] - b_prev * v_prev
        alpha[j] = h3 * float(v @ w)
        w = w - alpha[j] * v
        beta[j] = np.sqrt(h3 * float(w @ w))
        v_prev, v = v, w / beta[j]
        b_prev = beta[j]
    theta = tridiag_eigs_bisect(alpha, beta[:-1])
    return alpha, beta, float(theta[-1] + beta[-1]), float(theta[0])
