"""Named synthetic workloads (sizes of the paper's H-passivated Si nanocluster runs).

Each workload is an H-passivated Si cluster, grid spacing h = 0.7 bohr (Table I), a
spherical domain of radius (nominal cluster radius d/2 + 6 bohr) centred on the
central Si atom, the synthetic pseudopotential set in synthetic_pseudo.json, k
subspace vectors and Chebyshev degree m.  The cut radius of each cluster is chosen
so that the cut reproduces the stated formula (Si35H36, Si353H196) or lands nearest
to it (Si1911H604 for ~Si1900H600, Si3325H876 for ~Si3300H900).
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

from .cluster import ANG2BOHR, silicon_cluster

_HERE = os.path.dirname(os.path.abspath(__file__))


@dataclass(frozen=True)
class Workload:
    name: str
    r_cut_ang: float       # cluster cut radius (angstrom)
    d_nm: float            # nominal cluster diameter (nm)
    h: float               # grid spacing (bohr)
    margin: float          # domain radius = d/2 + margin (bohr)
    k: int                 # subspace size (occupied + buffer)
    degree: int            # Chebyshev filter degree m
    block: int             # column block streamed through the filter
    n_iter: int            # outer CheFSI iterations for the parity runs
    dtype: str             # arithmetic of the filter: "f64" or "f32"

    def atoms(self):
        return silicon_cluster(self.r_cut_ang)

    @property
    def radius(self) -> float:
        """Radius of the spherical Dirichlet domain in bohr."""
        return self.d_nm * 10.0 / 2.0 * ANG2BOHR + self.margin


WORKLOADS = {
    # Si35H36 in a ~1 nm sphere: cut 5.7 A keeps the shells 1+4+12+12+6 = 35 Si
    "si35h36": Workload("si35h36", 5.7, 1.0, 0.7, 6.0, 100, 10, 100, 3, "f64"),
    # ~2.2 nm cluster (cut 11.8 A gives exactly Si353H196)
    "si353h196": Workload("si353h196", 11.8, 2.2, 0.7, 6.0, 850, 12, 850, 1, "f32"),
    # ~4 nm cluster (nearest cut to Si1900H600), blocks of 512
    "si1911h604": Workload("si1911h604", 20.9, 4.0, 0.7, 6.0, 4600, 16, 512, 1, "f32"),
    # ~5 nm cluster (nearest cut to Si3300H900), blocks of 1024
    "si3325h876": Workload("si3325h876", 25.2, 5.0, 0.7, 6.0, 7700, 20, 1024, 1, "f32"),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def pseudo_params(path: str | None = None) -> list[dict]:
    """Species parameter dicts of the synthetic pseudopotential set."""
    with open(path or os.path.join(_HERE, "synthetic_pseudo.json")) as f:
        return json.load(f)["species"]


def cluster_scf_config(d_nm: float, z, h: float = 0.7, margin: float = 6.0, degree: int = 12) -> dict:
    """SCF sizes for a cluster of nominal diameter d_nm: domain radius d/2 + margin,
    spacing h, k = occupied states + the larger of 16 and 6 % of them (the 2.2 nm
    workload's 850 = 804 + 46 is the same ratio), Chebyshev degree."""
    from .cluster import n_occupied
    nocc = n_occupied(z)
    return {"radius": d_nm * 10.0 / 2.0 * ANG2BOHR + margin, "h": h,
            "k": nocc + max(16, -(-6 * nocc // 100)), "degree": degree}
