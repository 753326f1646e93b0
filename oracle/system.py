"""Build the oracle Hamiltonian for a cluster (convenience; plain composition)."""
from __future__ import annotations

import numpy as np

from .grid import sphere_grid
from .hamiltonian import Hamiltonian
from .potential import kb_projectors, local_potential


def cluster_hamiltonian(atom_pos, atom_z, species, radius: float, h: float, center=None):
    atom_pos = np.asarray(atom_pos, dtype=np.float64)
    c = atom_pos[0] if center is None else np.asarray(center, dtype=np.float64)
    g = sphere_grid(c, radius, h)
    V = local_potential(g.points(), atom_pos, atom_z, species)
    P, E, _ = kb_projectors(g, atom_pos, atom_z, species)
    return Hamiltonian(g, V, P, E)
