"""Density of states and HOMO-LUMO gap (oracle) -- test infrastructure only.

The DOS paragraph and Fig. 1 of the paper: the eigenvalues are shifted so that the highest
occupied state is at zero, histogrammed in 0.1 eV bins, and every DOS is scaled to the
same area below the Fermi level (here: the occupied states integrate to one).  The band
gap of Fig. 3 is the HOMO-LUMO gap.  Energies in eV with the CODATA 2018 Hartree energy.
"""
from __future__ import annotations

import numpy as np

HARTREE_EV = 27.211386245988


def dos(eigvals, n_occ: int, bin_ev: float = 0.1, e_lo_ev: float = -15.0, n_bins: int = 200):
    lam = np.sort(np.asarray(eigvals, dtype=np.float64))
    homo = lam[n_occ - 1]
    gap = (lam[n_occ] - homo) * HARTREE_EV if n_occ < len(lam) else float("nan")
    e = (lam - homo) * HARTREE_EV
    edges = e_lo_ev + bin_ev * np.arange(n_bins + 1)
    counts = np.zeros(n_bins)
    for x in e:                       # bin b holds [edge_b, edge_{b+1})
        b = int(np.floor((x - e_lo_ev) / bin_ev))
        if 0 <= b < n_bins:
            counts[b] += 1
    return counts / (n_occ * bin_ev), edges[:-1], gap
