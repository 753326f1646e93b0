"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds no arithmetic of the method itself (no stencil, no potential,
no filter, no orthonormalisation): only the inputs the method consumes --
hydrogen-passivated silicon nanocluster geometries, the synthetic
pseudopotential parameter set, the initial random subspace X0 drawn from a
counter-based generator, and the named workload sizes.
"""
from .cluster import (ANG2BOHR, silicon_cluster, cluster_for_diameter, n_electrons,
                      n_occupied)
from .rng import normal_entries, random_block_lex
from .configs import WORKLOADS, Workload, pseudo_params, workload

__all__ = [
    "ANG2BOHR", "silicon_cluster", "cluster_for_diameter", "n_electrons", "n_occupied",
    "normal_entries", "random_block_lex", "WORKLOADS", "Workload", "pseudo_params",
    "workload",
]
