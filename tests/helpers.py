"""Shared test helpers: systems, layout conversion between the oracle's lexicographic
order and the library's slot order (a permutation: no arithmetic of the method)."""
import numpy as np


def small_cluster():
    """Si2H2-like cluster with atoms off the grid points (KB spheres overlap)."""
    pos = np.array([[0.11, -0.07, 0.05], [2.3, 2.2, -2.25], [-1.9, 1.0, 2.8], [-2.6, -2.4, -0.3]])
    z = np.array([14, 14, 1, 1], dtype=np.int32)
    return pos, z


def to_slots(X_lex, lex, dtype=np.float64):
    n_slots = len(lex)
    out = np.zeros((n_slots,) + X_lex.shape[1:], dtype=dtype)
    live = lex >= 0
    out[live] = X_lex[lex[live]]
    return out


def from_slots(X_slots, lex, n_points):
    out = np.zeros((n_points,) + X_slots.shape[1:], dtype=X_slots.dtype)
    live = lex >= 0
    out[lex[live]] = X_slots[live]
    return out


def subspace_gap(A, B, h3):
    """sin of the largest principal angle between span(A) and span(B) (h^3 inner product)."""
    qa, _ = np.linalg.qr(A * np.sqrt(h3))
    qb, _ = np.linalg.qr(B * np.sqrt(h3))
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - s.min() ** 2)))
