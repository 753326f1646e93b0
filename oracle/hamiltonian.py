"""Matrix-free real-space Kohn-Sham Hamiltonian at fixed potential (oracle).

    H = -1/2 Lap_h + V_loc + V_NL            (Hartree atomic units)

Lap_h is the order-12 central finite-difference Laplacian (three 1D second
derivatives, axis-aligned 37-point star), applied with y = 0 outside the domain
(zero Dirichlet).  The paper's Hamiltonian is the sparse matrix that this defines
(Intro: high order finite difference; Method: sparse matrix-vector products).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fd import weights_float


def kinetic_matrix(grid, M: int = 6) -> sp.csr_matrix:
    """Sparse -1/2 Lap_h restricted to the domain."""
    w = weights_float(M)
    h2 = grid.h * grid.h
    n = grid.n
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [np.full(n, -0.5 * 3.0 * w[0] / h2)]
    for axis in range(3):
        for k in range(1, M + 1):
            for sgn in (-1, 1):
                off = np.zeros(3, dtype=np.int64)
                off[axis] = sgn * k
                nb = grid.index_of(grid.ijk + off[None, :])
                ok = nb >= 0
                rows.append(np.nonzero(ok)[0])
                cols.append(nb[ok])
                vals.append(np.full(int(ok.sum()), -0.5 * w[k] / h2))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


class Hamiltonian:
    """H y = T y + V * y + P (E h^3 (P^T y))."""

    def __init__(self, grid, V: np.ndarray, P=None, E=None, M: int = 6):
        self.grid = grid
        self.h = grid.h
        self.h3 = grid.h ** 3
        self.n = grid.n
        self.T = kinetic_matrix(grid, M)
        self.M = M
        self.V = np.asarray(V, dtype=np.float64)
        self.P = P.tocsr() if P is not None and P.shape[1] > 0 else None
        self.PT = self.P.T.tocsr() if self.P is not None else None
        self.E = np.asarray(E, dtype=np.float64) if E is not None else np.zeros(0)

    def apply(self, Y: np.ndarray) -> np.ndarray:
        Y = np.asarray(Y, dtype=np.float64)
        one = Y.ndim == 1
        if one:
            Y = Y[:, None]
        out = self.T @ Y + self.V[:, None] * Y
        if self.P is not None:
            coef = (self.E * self.h3)[:, None] * (self.PT @ Y)
            out = out + self.P @ coef
        return out[:, 0] if one else out

    def dense(self) -> np.ndarray:
        """Dense matrix (tiny grids only)."""
        return self.apply(np.eye(self.n))


def apply_at_rows(grid, rows, V_rows, P, E, Y, M: int = 6):
    """(H Y)[rows] by the definition, for sampled rows of a large grid: the stencil from
    the row's axis neighbours (zero outside the domain), V at the rows, and the nonlocal
    term P[rows] (E h^3 (P^T Y)).  Y holds all grid points (lexicographic) x columns."""
    w = weights_float(M)
    h2 = grid.h * grid.h
    rows = np.asarray(rows, dtype=np.int64)
    Y = np.asarray(Y, dtype=np.float64)
    out = (-0.5 * 3.0 * w[0] / h2) * Y[rows]
    for axis in range(3):
        for k in range(1, M + 1):
            for sgn in (-1, 1):
                off = np.zeros(3, dtype=np.int64)
                off[axis] = sgn * k
                nb = grid.index_of(grid.ijk[rows] + off[None, :])
                ok = nb >= 0
                out[ok] += (-0.5 * w[k] / h2) * Y[nb[ok]]
    out += np.asarray(V_rows, dtype=np.float64)[:, None] * Y[rows]
    if P is not None and P.shape[1] > 0:
        Pc = P.tocsc()
        coef = (np.asarray(E) * grid.h ** 3)[:, None] * (Pc.T @ Y)
        out += P.tocsr()[rows] @ coef
    return out
