"""Hydrogen-passivated spherical silicon nanoclusters (input geometry).

The paper's systems are spherical Si nanoclusters cut from bulk diamond-structure
silicon with the surface dangling bonds passivated by hydrogen (Computational
details, the paragraph after the SCF criterion; Table I).  The lattice constant used
here is the observed 5.43 A quoted there; the Si-H bond length is 1.48 A.

Construction (one reading of the paper, which gives no recipe):
  1. diamond lattice in quarter-cell integer units, centred on an atom at the origin;
  2. keep Si with |r| <= r_cut;
  3. repeatedly drop Si that have fewer than two Si neighbours;
  4. cap every missing tetrahedral bond of the remaining Si with H at 1.48 A
     along the bond direction.
Positions are returned in bohr.  Atom 0 is the central Si at the origin.
"""
from __future__ import annotations

import numpy as np

ANG2BOHR = 1.0 / 0.529177210903          # CODATA 2018 bohr radius in angstrom
A_SI_ANG = 5.43                           # observed lattice constant (Table I paragraph)
D_SIH_ANG = 1.48                          # Si-H bond length
Z_SI, Z_H = 14, 1

# tetrahedral bond vectors in quarter-cell units for the two fcc sublattices
_BONDS_A = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.int64)
_BONDS_B = -_BONDS_A


def _diamond_sites(r_cut_ang: float, a_ang: float) -> np.ndarray:
    """All diamond sites (quarter-cell integer coords) within r_cut of the origin."""
    n = int(np.ceil(4.0 * r_cut_ang / a_ang)) + 4
    rng = np.arange(-n, n + 1, dtype=np.int64)
    u = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    even = np.all(u % 2 == 0, axis=1) & (u.sum(1) % 4 == 0)          # sublattice A
    odd = np.all(u % 2 != 0, axis=1) & ((u - 1).sum(1) % 4 == 0)     # sublattice B
    u = u[even | odd]
    q2 = (u * u).sum(1).astype(np.float64)
    lim = (4.0 * r_cut_ang / a_ang) ** 2
    return u[q2 <= lim * (1.0 + 1e-12)]


def silicon_cluster(r_cut_ang: float, a_ang: float = A_SI_ANG, d_sih_ang: float = D_SIH_ANG):
    """Return (positions_bohr (n,3) float64, Z (n,) int32); Si first, central Si at index 0."""
    sites = _diamond_sites(r_cut_ang, a_ang)
    keyset = {tuple(s) for s in sites.tolist()}

    def is_a(s):
        return s[0] % 2 == 0

    changed = True
    while changed:
        changed = False
        drop = []
        for s in keyset:
            bonds = _BONDS_A if is_a(s) else _BONDS_B
            nb = sum((s[0] + b[0], s[1] + b[1], s[2] + b[2]) in keyset for b in bonds)
            if nb < 2 and s != (0, 0, 0):
                drop.append(s)
        if drop:
            changed = True
            for s in drop:
                keyset.discard(s)

    si = sorted(keyset, key=lambda s: (s[0] * s[0] + s[1] * s[1] + s[2] * s[2], s))
    si_pos = np.array(si, dtype=np.float64) * (a_ang / 4.0)
    h_pos = []
    for s in si:
        bonds = _BONDS_A if is_a(s) else _BONDS_B
        for b in bonds:
            if (s[0] + b[0], s[1] + b[1], s[2] + b[2]) not in keyset:
                d = b.astype(np.float64) / np.sqrt(3.0)
                h_pos.append(np.array(s, dtype=np.float64) * (a_ang / 4.0) + d_sih_ang * d)
    pos = np.concatenate([si_pos, np.array(h_pos).reshape(-1, 3)], 0) * ANG2BOHR
    z = np.array([Z_SI] * len(si) + [Z_H] * len(h_pos), dtype=np.int32)
    return pos, z


def cluster_for_diameter(d_nm: float):
    """Cluster cut at radius d/2 (diameter in nm)."""
    return silicon_cluster(d_nm * 10.0 / 2.0)


def n_electrons(z: np.ndarray) -> int:
    """Valence electrons: 4 per Si, 1 per H."""
    z = np.asarray(z)
    return int(4 * np.count_nonzero(z == Z_SI) + np.count_nonzero(z == Z_H))


def n_occupied(z: np.ndarray) -> int:
    """Doubly occupied states (spin-degenerate, closed shell)."""
    ne = n_electrons(z)
    return (ne + 1) // 2


def random_rotation(seed: int) -> np.ndarray:
    """A seeded rotation matrix (QR of a Gaussian 3x3 with the signs fixed, det +1)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def training_clusters(n: int = 30, seed0: int = 1000, d_min_nm: float = 1.0, d_max_nm: float = 3.0):
    """Seeded H-passivated Si clusters for training the learned SCF start: diameter drawn
    uniformly in [d_min, d_max] nm, lattice rotated by a seeded rotation about the central
    atom.  Returns a list of (seed, d_nm, positions_bohr, Z)."""
    out = []
    for i in range(n):
        seed = seed0 + i
        rng = np.random.default_rng(seed)
        d = float(rng.uniform(d_min_nm, d_max_nm))
        pos, z = cluster_for_diameter(d)
        out.append((seed, d, pos @ random_rotation(seed).T, z))
    return out
