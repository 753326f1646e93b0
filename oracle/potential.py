"""Synthetic pseudopotential on the grid (oracle).

The paper uses norm-conserving Troullier-Martins pseudopotentials in the separable
Kleinman-Bylander form (Computational details).  Their tables are not available, so a
synthetic set with the same structure stands in (parameters in the workloads JSON):

  local part, per atom a at R_a, r = |p - R_a|:
      v_a(r) = -Z_a erf(r / r_c) / r + A_a exp(-r^2 / r_g^2),     v_a(0) = -2 Z_a/(r_c sqrt(pi)) + A_a
  V_loc(p) = sum over all atoms (no truncation)

  nonlocal part (KB form), for atoms with projectors (s + p):
      chi_s(p)   = exp(-r^2 / (2 r_p^2))
      chi_m(p)   = ((p - R_a)_m / r_p) exp(-r^2 / (2 r_p^2)),   m = x, y, z
      nonzero only where r^2 <= r_cut^2 (hard cutoff) and p in the domain
      V_NL y = sum_i chi_i E_i h^3 <chi_i, y>,   <u, v> = sum_p u_p v_p
  with E = e_s for the s projector and e_p for the three p projectors.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.special import erf


def _species_by_z(species):
    return {int(s["z_number"]): s for s in species}


def local_potential(points: np.ndarray, atom_pos: np.ndarray, atom_z: np.ndarray,
                    species) -> np.ndarray:
    """V_loc at each point (float64)."""
    table = _species_by_z(species)
    V = np.zeros(len(points), dtype=np.float64)
    for pos, z in zip(atom_pos, atom_z):
        s = table[int(z)]
        dx = points[:, 0] - pos[0]
        dy = points[:, 1] - pos[1]
        dz = points[:, 2] - pos[2]
        r2 = dx * dx + dy * dy + dz * dz
        r = np.sqrt(r2)
        Z, rc = s["z_valence"], s["r_c"]
        with np.errstate(divide="ignore", invalid="ignore"):
            coul = np.where(r > 0.0, -Z * erf(r / rc) / np.where(r > 0.0, r, 1.0),
                            -2.0 * Z / (rc * np.sqrt(np.pi)))
        V += coul + s["a_gauss"] * np.exp(-r2 / (s["r_gauss"] ** 2))
    return V


def kb_projectors(grid, atom_pos: np.ndarray, atom_z: np.ndarray, species):
    """Sparse projector matrix P (N x n_proj, CSC), energies E (n_proj,), owning atom per column.

    Columns are ordered atom by atom, each atom contributing (s, p_x, p_y, p_z)."""
    table = _species_by_z(species)
    h = grid.h
    rows, cols, vals, E, owner = [], [], [], [], []
    col = 0
    for a, (pos, z) in enumerate(zip(atom_pos, atom_z)):
        s = table[int(z)]
        if int(s["n_proj"]) == 0:
            continue
        rcut, rp = s["r_cut"], s["r_p"]
        lo = np.floor((pos - grid.center - rcut) / h).astype(np.int64) - 1
        hi = np.ceil((pos - grid.center + rcut) / h).astype(np.int64) + 1
        rk, rj, ri = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1),
                                 np.arange(lo[0], hi[0] + 1), indexing="ij")
        ijk = np.stack([ri.ravel(), rj.ravel(), rk.ravel()], 1)
        idx = grid.index_of(ijk)
        ijk, idx = ijk[idx >= 0], idx[idx >= 0]
        pts = grid.center[None, :] + h * ijk.astype(np.float64)
        dx = pts[:, 0] - pos[0]
        dy = pts[:, 1] - pos[1]
        dz = pts[:, 2] - pos[2]
        r2 = dx * dx + dy * dy + dz * dz
        keep = r2 <= rcut * rcut
        idx, dx, dy, dz, r2 = idx[keep], dx[keep], dy[keep], dz[keep], r2[keep]
        g = np.exp(-r2 / (2.0 * rp * rp))
        for m, chi in enumerate([g, dx / rp * g, dy / rp * g, dz / rp * g]):
            rows.append(idx)
            cols.append(np.full(len(idx), col + m, dtype=np.int64))
            vals.append(chi)
        E += [s["e_s"], s["e_p"], s["e_p"], s["e_p"]]
        owner += [a] * 4
        col += 4
    if col == 0:
        P = sp.csc_matrix((grid.n, 0))
    else:
        P = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(grid.n, col))
    return P, np.array(E, dtype=np.float64), np.array(owner, dtype=np.int64)
