"""Chebyshev-filtered subspace iteration at fixed potential (oracle, float64).

CheFSI (paper, CheFSI paragraph: filter the subspace with a Chebyshev polynomial
of H that amplifies the wanted low end of the spectrum, then orthonormalise and
perform Rayleigh-Ritz; details delegated to Zhou, Saad, Tiago & Chelikowsky 2006
and Liou et al. 2020).  The steps below follow that scheme in this order:

  chebyshev_filter  degree-m scaled three-term recurrence.  With the cut a, the
                    upper bound b and the lowest estimate a0:
                      e = (b - a)/2, c = (b + a)/2, sigma_1 = e/(a0 - c), tau = 2/sigma_1
                      Y_1 = (sigma_1/e)(H X - c X)
                      sigma_j = 1/(tau - sigma_{j-1})
                      Y_j = (2 sigma_j/e)(H Y_{j-1} - c Y_{j-1}) - sigma_{j-1} sigma_j Y_{j-2}
                    so Y_m = T_m(t(H)) / T_m(t(a0)) X with t(x) = (x - c)/e.
  cholesky_qr       S = h^3 Y^T Y = R^T R,  Y <- Y R^-1   (h^3 Y^T Y = I afterwards)
  rayleigh_ritz     Hs = h^3 Y^T (H Y), symmetrised; Hs = Q Lambda Q^T (ascending);
                    Y <- Y Q
  density           rho_p = sum_i f_i y_{p,i}^2   (f_i = 2 for the occupied states)
  chefsi            CholQR + RR of X0 for the first bounds, then n_iter times
                    (filter with a = Lambda_max, a0 = Lambda_min -> CholQR -> RR)
The upper bound b is a Gershgorin/Weyl bound (see spectral_upper_bound).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .fd import weights_float


def spectral_upper_bound(H) -> float:
    """b >= lambda_max(H) by Weyl's inequality over the three terms:
       kinetic: (3/(2h^2)) (|w_0| + 2 sum_k |w_k|)   (Gershgorin row sum of -1/2 Lap_h)
       local:   max_p V_p
       nonlocal: lambda_max(P E+ P^T h^3) = lambda_max(E+^1/2 G E+^1/2) with the projector
                 Gram G = h^3 P^T P, bounded by its Gershgorin row maximum
                 max_i sum_j sqrt(E+_i E+_j) |G_ij|,  E+ = max(E, 0)"""
    w = weights_float(H.M)
    kin = 3.0 / (2.0 * H.h * H.h) * (abs(w[0]) + 2.0 * sum(abs(x) for x in w[1:]))
    bound = kin + float(H.V.max())
    if H.P is not None:
        G = (H.h3 * (H.PT @ H.P)).toarray()
        se = np.sqrt(np.maximum(H.E, 0.0))
        bound += float((np.abs(G) * se[:, None] * se[None, :]).sum(1).max())
    return bound


def chebyshev_filter(H, X: np.ndarray, m: int, a: float, b: float, a0: float) -> np.ndarray:
    if not (a < b) or not (a0 < a):
        raise ValueError("filter bounds need a0 < a < b")
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    sigma = e / (a0 - c)
    tau = 2.0 / sigma
    Y = (sigma / e) * (H.apply(X) - c * X)
    Yprev = X
    for _ in range(2, m + 1):
        sigma_new = 1.0 / (tau - sigma)
        Ynew = (2.0 * sigma_new / e) * (H.apply(Y) - c * Y) - (sigma * sigma_new) * Yprev
        Yprev, Y = Y, Ynew
        sigma = sigma_new
    return Y


def cholesky_qr(X: np.ndarray, h3: float):
    """Return (X R^-1, R) with S = h^3 X^T X = R^T R, R upper triangular."""
    S = h3 * (X.T @ X)
    L = np.linalg.cholesky(S)          # S = L L^T, R = L^T
    R = L.T
    Xn = solve_triangular(R, X.T, trans="T", lower=False).T   # solves R^T Z = X^T
    return Xn, R


def rayleigh_ritz(H, X: np.ndarray, h3: float):
    """Return (Lambda ascending, X Q, H X Q)."""
    HX = H.apply(X)
    Hs = h3 * (X.T @ HX)
    Hs = 0.5 * (Hs + Hs.T)
    lam, Q = np.linalg.eigh(Hs)
    return lam, X @ Q, HX @ Q


def density(X: np.ndarray, occ: np.ndarray) -> np.ndarray:
    occ = np.asarray(occ, dtype=np.float64)
    return (X[:, :len(occ)] ** 2) @ occ


def residual_norms(X: np.ndarray, HX: np.ndarray, lam: np.ndarray, h3: float) -> np.ndarray:
    """||H x_i - lambda_i x_i|| in the h^3-weighted grid norm."""
    R = HX - X * lam[None, :]
    return np.sqrt(h3 * (R * R).sum(0))


def chefsi(H, X0: np.ndarray, m: int, n_iter: int, b: float | None = None):
    """Fixed-potential CheFSI; returns dict with per-iteration Ritz values and the basis."""
    h3 = H.h3
    if b is None:
        b = spectral_upper_bound(H)
    X, _ = cholesky_qr(np.array(X0, dtype=np.float64), h3)
    lam, X, HX = rayleigh_ritz(H, X, h3)
    history = [lam]
    for _ in range(n_iter):
        Y = chebyshev_filter(H, X, m, a=lam[-1], b=b, a0=lam[0])
        X, _ = cholesky_qr(Y, h3)
        lam, X, HX = rayleigh_ritz(H, X, h3)
        history.append(lam)
    return {"lam": lam, "X": X, "HX": HX, "history": history, "b": b}


def chefsi_converged(H, X0: np.ndarray, m: int, n_want: int, tol: float = 1e-7,
                     max_iter: int = 200, b: float | None = None):
    """Iterate until the n_want lowest residual norms are below tol."""
    h3 = H.h3
    if b is None:
        b = spectral_upper_bound(H)
    X, _ = cholesky_qr(np.array(X0, dtype=np.float64), h3)
    lam, X, HX = rayleigh_ritz(H, X, h3)
    for it in range(1, max_iter + 1):
        Y = chebyshev_filter(H, X, m, a=lam[-1], b=b, a0=lam[0])
        X, _ = cholesky_qr(Y, h3)
        lam, X, HX = rayleigh_ritz(H, X, h3)
        res = residual_norms(X, HX, lam, h3)
        if res[:n_want].max() < tol:
            return {"lam": lam, "X": X, "res": res, "iters": it, "b": b}
    raise RuntimeError("CheFSI did not converge")
