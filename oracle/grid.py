"""Real-space grids in lexicographic order (oracle).

Spherical domain (Intro: aperiodic nanoclusters on a finite domain, no supercell;
zero Dirichlet condition outside).  Grid points are center + h*(i, j, k) for integers
(i, j, k); a point belongs to the domain iff  i^2 + j^2 + k^2 <= R^2/h^2 + 1e-9
(the small slack makes exact ties inclusive).  A box domain (all 0 <= i < nx,
0 <= j < ny, 0 <= k < nz) serves the closed-form tests.

Lexicographic order: k slowest, then j, then i fastest.
"""
from __future__ import annotations

import numpy as np


class Grid:
    def __init__(self, ijk: np.ndarray, h: float, center: np.ndarray):
        self.ijk = np.ascontiguousarray(ijk, dtype=np.int64)      # (N, 3) as (i, j, k)
        self.h = float(h)
        self.center = np.asarray(center, dtype=np.float64)
        self.n = len(self.ijk)
        lo = self.ijk.min(0) if self.n else np.zeros(3, np.int64)
        hi = self.ijk.max(0) if self.n else np.zeros(3, np.int64)
        self._lo = lo - 7
        self._ext = (hi - lo) + 15
        self._keys = self._key(self.ijk)
        assert np.all(np.diff(self._keys) > 0), "points must be in lexicographic order"

    def _key(self, ijk):
        s = ijk - self._lo
        return (s[:, 2] * self._ext[1] + s[:, 1]) * self._ext[0] + s[:, 0]

    def index_of(self, ijk: np.ndarray) -> np.ndarray:
        """Lexicographic index of each (i, j, k), or -1 if outside the domain."""
        ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, 3)
        inside_box = np.all((ijk - self._lo >= 0) & (ijk - self._lo < self._ext), axis=1)
        key = np.where(inside_box, self._key(np.where(inside_box[:, None], ijk, self._lo)), -1)
        pos = np.searchsorted(self._keys, key)
        pos = np.minimum(pos, max(self.n - 1, 0))
        hit = inside_box & (self.n > 0) & (self._keys[pos] == key)
        return np.where(hit, pos, -1)

    def points(self) -> np.ndarray:
        """Cartesian coordinates (bohr): center + h * ijk."""
        return self.center[None, :] + self.h * self.ijk.astype(np.float64)


def sphere_grid(center, radius: float, h: float) -> Grid:
    n = int(np.floor(radius / h)) + 1
    lim = radius * radius / (h * h) + 1e-9
    r = np.arange(-n, n + 1, dtype=np.int64)
    k, j, i = np.meshgrid(r, r, r, indexing="ij")          # k slowest, i fastest
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
    n2 = (ijk * ijk).sum(1).astype(np.float64)
    return Grid(ijk[n2 <= lim], h, center)


def box_grid(nx: int, ny: int, nz: int, h: float, center=(0.0, 0.0, 0.0)) -> Grid:
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], 1).astype(np.int64)
    return Grid(ijk, h, center)
