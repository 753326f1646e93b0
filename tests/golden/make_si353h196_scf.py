"""Writes tests/golden/<workload>_scf.json from the FP64 CPU oracle alone.

Default: the 2.2 nm cluster (Si353H196, 234,489 grid points, k = 850, degree 12); with
--workload si35h36 the 1 nm cluster (Si35H36, 45,025 points, k = 100, degree 10).  The oracle's
self-consistent field (Computational details: LDA, Anderson mixing of the input
potential, the 4-then-1 CheFSI schedule, stop at SRE < 1e-4 Ry) from the seeded X0
(seed 1), followed by the converged mode at the final input potential: CheFSI at
fixed potential until every occupied state and the LUMO have residual norm
|H x - lambda x| < 1e-7 Ha.  Stored: the SCF history, the converged Ritz values of the
occupied states and the first unoccupied ones, HOMO, LUMO, gap, the total energy
evaluated with the converged orbitals, and moments of the converged density (charge,
dipole, quadrupole about the domain centre, charge in 1-bohr radial shells, and the
density at 4096 seeded sample points of the lexicographic grid).

Only oracle/ and workloads/ are called.  About two hours on eight cores for the 2.2 nm
cluster, a few minutes for the 1 nm one:
    python tests/golden/make_si353h196_scf.py [--workload NAME] [--checkpoint DIR]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import chefsi as cf                       # noqa: E402
from oracle.hamiltonian import Hamiltonian            # noqa: E402
from oracle.potential import kb_projectors, local_potential  # noqa: E402
from oracle.scf import Poisson, lda_xc, occupations, scf    # noqa: E402
from workloads import n_electrons, pseudo_params, random_block_lex, workload  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
N_SAMPLE = 4096
N_UNOCC = 10
RESID_TOL = 1e-7


def density_moments(grid, rho):
    h3 = grid.h ** 3
    x = grid.h * grid.ijk.astype(np.float64)
    r2 = (x * x).sum(1)
    q = h3 * rho.sum()
    p = h3 * (rho[:, None] * x).sum(0)
    Q = h3 * (3.0 * np.einsum("n,ni,nj->ij", rho, x, x) - np.eye(3) * (rho * r2).sum())
    r = np.sqrt(r2)
    nshell = int(math.ceil(r.max())) + 1
    shells = np.bincount(np.floor(r).astype(np.int64), weights=rho, minlength=nshell) * h3
    idx = np.sort(np.random.default_rng(20230301).choice(grid.n, N_SAMPLE, replace=False))
    return {"charge": q, "dipole": p.tolist(), "quadrupole": [Q[0, 0], Q[1, 1], Q[2, 2], Q[0, 1], Q[0, 2], Q[1, 2]],
            "shell_charge_1bohr": shells.tolist(), "sample_index_lex": idx.tolist(),
            "sample_rho": rho[idx].tolist()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--checkpoint", default=None, help="directory for the post-SCF state (resumable)")
    ap.add_argument("--workload", default="si353h196")
    args = ap.parse_args()
    wl = workload(args.workload)
    out_path = os.path.join(HERE, f"{wl.name}_scf.json")
    pos, z = wl.atoms()
    species = pseudo_params()
    ne = n_electrons(z)
    nocc = ne // 2
    t0 = time.time()
    ck = os.path.join(args.checkpoint, f"{wl.name}_scf_state.npz") if args.checkpoint else None
    if ck and os.path.exists(ck):
        st = np.load(ck, allow_pickle=False)
        X, v_in, lam = st["X"], st["v_in"], st["lam"]
        hist = json.loads(str(st["hist"]))
        from oracle.grid import sphere_grid
        g = sphere_grid(np.asarray(pos[0], dtype=np.float64), wl.radius, wl.h)
    else:
        from oracle.grid import sphere_grid
        g = sphere_grid(np.asarray(pos[0], dtype=np.float64), wl.radius, wl.h)
        X0 = random_block_lex(1, g.n, wl.k)
        res = scf(pos, z, species, wl.radius, wl.h, wl.k, wl.degree, X0, max_steps=80, sre_tol_ry=1e-4)
        X, v_in, lam = res["X"], res["v_in"], res["lam"]
        hist = [{"step": r["step"], "sre_ry": r["sre_ry"], "e_total": r["e_total"], "homo": r["homo"],
                 "lumo": r["lumo"]} for r in res["reports"]]
        print(f"SCF: {len(hist)} steps, SRE {hist[-1]['sre_ry']:.3e} Ry, {time.time() - t0:.0f} s", flush=True)
        if ck:
            os.makedirs(args.checkpoint, exist_ok=True)
            np.savez(ck, X=X, v_in=v_in, lam=lam, hist=json.dumps(hist))
    # the SCF stops after mixing is skipped, so v_in is the potential of the last step
    pts = g.points()
    v_ion = local_potential(pts, pos, z, species)
    P, E, _ = kb_projectors(g, pos, z, species)
    H = Hamiltonian(g, v_in, P, E)
    t1 = time.time()
    conv = cf.chefsi_converged(H, X, wl.degree, nocc + 1, tol=RESID_TOL, max_iter=400)
    lamc = conv["lam"]
    print(f"converged mode: {conv['iters']} iterations, {time.time() - t1:.0f} s", flush=True)
    occ, mu, minus_ts = occupations(lamc, ne, 0.0)
    rho = cf.density(conv["X"], occ)
    vh = Poisson(g).solve(rho)
    eps, _ = lda_xc(rho)
    h3 = g.h ** 3
    e_band = float(np.dot(occ, lamc))
    e_tot = (e_band - h3 * float(np.dot(rho, v_in - v_ion)) + 0.5 * h3 * float(np.dot(rho, vh))
             + h3 * float(np.dot(rho, eps)) + minus_ts)
    out = {
        "what": f"FP64 CPU oracle: SCF of {wl.name} to SRE < 1e-4 Ry, then fixed-potential CheFSI "
                "to residual < 1e-7 Ha (occupied states and the LUMO)",
        "written_by": "tests/golden/make_si353h196_scf.py (oracle/ and workloads/ only)",
        "workload": wl.name, "n_points": int(g.n), "n_atoms": int(len(z)), "k": wl.k, "degree": wl.degree,
        "x0_seed": 1, "mixing": "Anderson alpha 0.3 history 8", "chefsi_schedule": "4 then 1",
        "sre_tol_ry": 1e-4, "n_occ": int(nocc),
        "scf": {"steps": len(hist), "history": hist},
        "converged": {"iters": int(conv["iters"]), "resid_tol_ha": RESID_TOL,
                      "max_resid_wanted": float(conv["res"][:nocc + 1].max()),
                      "lam": lamc[:nocc + N_UNOCC].tolist(), "homo": float(lamc[nocc - 1]),
                      "lumo": float(lamc[nocc]), "gap": float(lamc[nocc] - lamc[nocc - 1]),
                      "e_band": e_band, "e_total": e_tot, "electrons": float(h3 * rho.sum()),
                      "rho": density_moments(g, rho)},
        "seconds": time.time() - t0,
    }
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {out_path} ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
