"""Counter-based normal generator for the initial subspace X0.

Generator definition (each side that draws X0 implements it from this text):
  mix64(z)  : SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014):
              z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
              z *= 0x94D049BB133111EB; z ^= z >> 31   (all mod 2^64)
  key       = mix64(seed)
  u64(c)    = mix64(key + (c + 1) * 0x9E3779B97F4A7C15)
  entry n of the (lexicographic point, column) array, n = point * k + col:
      q  = n >> 1
      u1 = ((u64(2q) >> 11) + 1) * 2^-53          in (0, 1]
      u2 = (u64(2q+1) >> 11) * 2^-53              in [0, 1)
      r  = sqrt(-2 ln u1)
      x  = r cos(2 pi u2)  if n even,  r sin(2 pi u2)  if n odd     (Box-Muller)
"""
from __future__ import annotations

import numpy as np

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _u64(seed: int, c: np.ndarray) -> np.ndarray:
    key = _mix64(np.array([seed], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        z = key + (c.astype(np.uint64) + np.uint64(1)) * _GAMMA
    return _mix64(z)


def normal_entries(seed: int, n: np.ndarray) -> np.ndarray:
    """N(0,1) values for flat entry indices n (int64 array), float64."""
    n = np.asarray(n, dtype=np.int64)
    q = n >> 1
    a = _u64(seed, 2 * q)
    b = _u64(seed, 2 * q + 1)
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (b >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return np.where((n & 1) == 0, r * np.cos(ang), r * np.sin(ang))


def random_block_lex(seed: int, n_points: int, k: int, points=None, cols=None) -> np.ndarray:
    """X0[p, j] for lexicographic points p and columns j (all by default), float64."""
    p = np.arange(n_points, dtype=np.int64) if points is None else np.asarray(points, np.int64)
    j = np.arange(k, dtype=np.int64) if cols is None else np.asarray(cols, np.int64)
    n = p[:, None] * np.int64(k) + j[None, :]
    return normal_entries(seed, n.reshape(-1)).reshape(len(p), len(j))
