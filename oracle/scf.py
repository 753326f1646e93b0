"""Self-consistent field loop (oracle, float64) -- test infrastructure only.

Kohn-Sham DFT with the LDA (Computational details: Ceperley-Alder correlation as
parametrised by Perdew & Zunger 1981) at fixed ions:

  V_eff = V_ion + V_H[rho] + V_xc[rho]
  V_H    solves  -Lap_h V_H = 4 pi rho  on the domain (order-12 FD Laplacian); the
         values the stencil needs outside the sphere come from the multipole expansion
         (monopole, dipole, quadrupole) of rho about the grid centre; conjugate
         gradients in float64
  V_xc   Slater exchange + PZ81 correlation (unpolarised, Hartree units)
  mixing Anderson mixing of the input potential (the Broyden-type quasi-Newton scheme;
         history m, linear step alpha), optionally with the Kerker preconditioner
         P = (-Lap_h) (-Lap_h + q0^2)^-1 on the residuals (zero outside the domain):
         P f = f - q0^2 u with (-Lap_h + q0^2) u = f (conjugate gradients)
  SRE    sqrt(h^3 sum_p rho_p (V_out - V_in)_p^2), reported in Ry (x 2); stop below 1e-4 Ry
  CheFSI four filter/Cholesky-QR/Rayleigh-Ritz iterations in the first SCF step, one in
         every later step (the schedule the paper states)
  degree the fixed degree m, or (degree_max > 0) a degree per group of columns from the
         residuals of the current Ritz pairs (the per-vector degrees of ChASE, Winkelmann,
         Springer & Di Napoli 2019): with e = (b - a)/2, c = (b + a)/2, t_i = (c - lambda_i)/e
         and rho_i = 1/(t_i + sqrt(t_i^2 - 1)) the error of vector i shrinks by rho_i per
         degree step, so m_i = ceil(log(tol / r_i) / log(rho_i)) (m_min if r_i <= tol,
         m_max if t_i <= 1), clamped to [m_min, m_max]; a group of `group` columns takes
         its largest m_i.  Each vector is asked for the same reduction of its residual per
         filter, tol_i = max(tol_floor, reduction * r_i); lambda_i = <x_i, H x_i> and
         r_i = |H x_i - lambda_i x_i| with the Hamiltonian of the current step.
  occupations  kT = 0: the n_e/2 lowest Ritz states doubly occupied.  kT > 0: Fermi-Dirac
         occupations 2 f((lambda - mu)/kT) with mu fixed by sum = n_e (bisection), and the
         energy reported is the Mermin free energy E - T S,
         S = -2 sum_i [f_i ln f_i + (1 - f_i) ln(1 - f_i)]

The starting potential is the superposition of neutral atoms: Gaussian valence densities
Z/(pi^{3/2} r_a^3) exp(-r^2/r_a^2) per atom (r_a = the species' r_start), V_in = V_ion + V_H[rho_at] + V_xc[rho_at].
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as spla

from . import chefsi as cf
from .fd import weights_float
from .hamiltonian import Hamiltonian, kinetic_matrix

# Perdew-Zunger 1981 correlation of the Ceperley-Alder gas, unpolarised (Hartree)
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116
RHO_FLOOR = 1e-14


def lda_xc(rho: np.ndarray):
    """(eps_xc, V_xc) per point for density rho (LDA: Slater + PZ81)."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    m = rho > RHO_FLOOR
    r = rho[m]
    rs = (3.0 / (4.0 * math.pi * r)) ** (1.0 / 3.0)
    ex = -0.75 * (3.0 * r / math.pi) ** (1.0 / 3.0)
    vx = (4.0 / 3.0) * ex
    ec = np.empty_like(r)
    vc = np.empty_like(r)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * s + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_BETA1 * s + 4.0 / 3.0 * PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    x = rs[lo]
    lnx = np.log(x)
    ec[lo] = PZ_A * lnx + PZ_B + PZ_C * x * lnx + PZ_D * x
    vc[lo] = PZ_A * lnx + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * x * lnx + (2.0 * PZ_D - PZ_C) / 3.0 * x
    eps[m] = ex + ec
    v[m] = vx + vc
    return eps, v


def fermi_dirac(x):
    """1/(1 + e^x) written as (1 - tanh(x/2))/2 (no overflow for large |x|)."""
    return 0.5 * (1.0 - np.tanh(0.5 * np.asarray(x, dtype=np.float64)))


def occupations(lam, n_electrons: int, kT: float):
    """(occ, mu, -T S) for the Ritz values lam (ascending).

    kT = 0: occ = 2 for the n_electrons/2 lowest states, mu = the highest occupied value.
    kT > 0: occ_i = 2 f((lam_i - mu)/kT); mu by 200 bisection halvings of
    [min lam - 1 - 50 kT, max lam + 1 + 50 kT] on the electron count (monotone in mu).
    """
    lam = np.asarray(lam, dtype=np.float64)
    if kT == 0.0:
        nocc = n_electrons // 2
        occ = np.zeros(len(lam))
        occ[:nocc] = 2.0
        return occ, float(lam[nocc - 1]), 0.0
    lo = float(lam.min()) - 1.0 - 50.0 * kT
    hi = float(lam.max()) + 1.0 + 50.0 * kT
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if float(np.sum(2.0 * fermi_dirac((lam - mid) / kT))) < n_electrons:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    f = fermi_dirac((lam - mu) / kT)
    s = np.zeros(len(lam))
    inner = (f > 0.0) & (f < 1.0)
    fi = f[inner]
    s[inner] = fi * np.log(fi) + (1.0 - fi) * np.log(1.0 - fi)
    minus_ts = kT * 2.0 * float(np.sum(s))
    return 2.0 * f, mu, minus_ts


def atomic_density(points, atom_pos, atom_z, species):
    """Superposition of Gaussian valence densities (start of the SCF)."""
    table = {int(s["z_number"]): s for s in species}
    rho = np.zeros(len(points))
    for pos, z in zip(atom_pos, atom_z):
        ra = table[int(z)]["r_start"]
        zv = table[int(z)]["z_valence"]
        d = points - pos
        r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        rho += zv / (math.pi ** 1.5 * ra ** 3) * np.exp(-r2 / (ra * ra))
    return rho


def multipole_potential(rho: np.ndarray, grid, targets: np.ndarray) -> np.ndarray:
    """Potential of rho at target points from its multipoles about the grid centre:
    Q/r + p.r/r^3 + (1/2) sum_ij Q_ij r_i r_j / r^5,  Q_ij = int rho (3 x_i x_j - r^2 d_ij)."""
    h3 = grid.h ** 3
    x = grid.h * grid.ijk.astype(np.float64)
    q = h3 * rho.sum()
    p = h3 * (rho[:, None] * x).sum(0)
    r2s = (x * x).sum(1)
    Qm = h3 * (3.0 * np.einsum("n,ni,nj->ij", rho, x, x) - np.eye(3) * (rho * r2s).sum())
    t = targets - grid.center
    r2 = (t * t).sum(1)
    r = np.sqrt(r2)
    return q / r + (t @ p) / (r2 * r) + 0.5 * np.einsum("ni,ij,nj->n", t, Qm, t) / (r2 * r2 * r)


def ghost_rhs(grid, M: int = 6):
    """Ghost points (outside the domain, within M steps of a domain point along an axis)
    and the coupling matrix G with (Lap_h V)_p = (Lap_h restricted V)_p + (G V_ghost)_p."""
    import scipy.sparse as sp
    w = weights_float(M)
    h2 = grid.h * grid.h
    rows, keys = [], []
    vals = []
    for axis in range(3):
        for k in range(1, M + 1):
            for sgn in (-1, 1):
                off = np.zeros(3, dtype=np.int64)
                off[axis] = sgn * k
                q = grid.ijk + off[None, :]
                outside = grid.index_of(q) < 0
                idx = np.nonzero(outside)[0]
                rows.append(idx)
                keys.append(q[idx])
                vals.append(np.full(len(idx), w[k] / h2))
    allq = np.concatenate(keys)
    uq, inv = np.unique(allq, axis=0, return_inverse=True)
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), inv.ravel())), shape=(grid.n, len(uq)))
    return uq, G


class Poisson:
    """-Lap_h V = 4 pi rho with multipole values outside the sphere (conjugate gradients)."""

    def __init__(self, grid, M: int = 6):
        self.grid = grid
        self.A = 2.0 * kinetic_matrix(grid, M)       # -Lap_h restricted to the domain (SPD)
        self.ghost_ijk, self.G = ghost_rhs(grid, M)
        self.ghost_xyz = grid.center[None, :] + grid.h * self.ghost_ijk.astype(np.float64)

    def solve(self, rho: np.ndarray, x0=None, tol: float = 1e-12):
        vg = multipole_potential(rho, self.grid, self.ghost_xyz)
        b = 4.0 * math.pi * rho + self.G @ vg
        x, info = spla.cg(self.A, b, x0=x0, rtol=tol, atol=0.0, maxiter=20000)
        if info != 0:
            raise RuntimeError("Poisson CG did not converge")
        return x


class Kerker:
    """P f = f - q0^2 (-Lap_h + q0^2)^-1 f on the domain (zero outside): damps the slowly
    varying part of a residual, P = q^2 / (q^2 + q0^2) for a plane wave of wave number q."""

    def __init__(self, grid, q0: float, M: int = 6):
        self.q0 = q0
        self.A = 2.0 * kinetic_matrix(grid, M) + q0 * q0 * sp_identity(grid.n)

    def apply(self, f: np.ndarray, tol: float = 1e-12) -> np.ndarray:
        u, info = spla.cg(self.A, f, rtol=tol, atol=0.0, maxiter=20000)
        if info != 0:
            raise RuntimeError("Kerker CG did not converge")
        return f - self.q0 * self.q0 * u


def sp_identity(n):
    import scipy.sparse as sp
    return sp.identity(n, format="csr")


class Anderson:
    """Anderson mixing of the input potential: V_next = V_in + a P F - sum_j g_j (dV_j + a P dF_j),
    g = argmin |F - sum_j g_j dF_j|, F = V_out - V_in, history of the last m differences;
    P = identity or the Kerker preconditioner."""

    def __init__(self, alpha: float = 0.3, history: int = 8, precond=None):
        self.alpha = alpha
        self.m = history
        self.precond = precond
        self.prev = None          # (V_in, F, P F) of the previous step
        self.dV, self.dF, self.dPF = [], [], []

    def step(self, v_in: np.ndarray, f: np.ndarray) -> np.ndarray:
        pf = self.precond.apply(f) if self.precond is not None else f
        if self.prev is not None:
            self.dV.append(v_in - self.prev[0])
            self.dF.append(f - self.prev[1])
            self.dPF.append(pf - self.prev[2])
            if len(self.dV) > self.m:
                self.dV.pop(0)
                self.dF.pop(0)
                self.dPF.pop(0)
        self.prev = (v_in.copy(), f.copy(), pf.copy())
        nxt = v_in + self.alpha * pf
        if self.dF:
            DF = np.stack(self.dF, 1)
            DV = np.stack(self.dV, 1)
            DPF = np.stack(self.dPF, 1)
            g = np.linalg.solve(DF.T @ DF, DF.T @ f)
            nxt = nxt - (DV + self.alpha * DPF) @ g
        return nxt


def rayleigh_residuals(H, X):
    """(lambda_i = h^3 <x_i, H x_i>, r_i = sqrt(h^3 sum (H x_i - lambda_i x_i)^2)) for
    h^3-orthonormal columns X."""
    HX = H.apply(X)
    lam = H.h3 * (X * HX).sum(0)
    R = HX - X * lam[None, :]
    return lam, np.sqrt(H.h3 * (R * R).sum(0))


def group_degrees(lam, r, a, b, tol, m_min, m_max, group):
    """Degree of every column group (see the module docstring); tol: one value per column."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    m = np.empty(len(lam), dtype=np.int64)
    for i in range(len(lam)):
        t = (c - lam[i]) / e
        if t <= 1.0 + 1e-12:
            m[i] = m_max
        elif r[i] <= tol[i]:
            m[i] = m_min
        else:
            rho = 1.0 / (t + math.sqrt(t * t - 1.0))
            m[i] = math.ceil(math.log(tol[i] / r[i]) / math.log(rho))
    m = np.clip(m, m_min, m_max)
    return [int(m[g:g + group].max()) for g in range(0, len(lam), group)]


def total_energy(h3, e_band, rho, v_in, v_ion, vh, eps, minus_ts=0.0):
    """E = sum_i f_i lambda_i - h^3 sum rho (V_in - V_ion) + 1/2 h^3 sum rho V_H + h^3 sum rho eps_xc
    (- T S): the band energy with the double-counted Hartree and exchange-correlation
    terms removed (no ion-ion term)."""
    return (e_band - h3 * float(np.dot(rho, v_in - v_ion)) + 0.5 * h3 * float(np.dot(rho, vh))
            + h3 * float(np.dot(rho, eps)) + minus_ts)


def converged_mode(res, atom_pos, atom_z, species, degree, tol=1e-7, max_iter=400):
    """Fixed-potential CheFSI at the SCF's last input potential until the occupied states and
    the first empty one have residual norm < tol, then the energy of the converged orbitals:
    (lam, X, rho, e_total, iters).  kT = 0 occupations."""
    from .potential import kb_projectors, local_potential
    from workloads.cluster import n_electrons
    g = res["grid"]
    ne = n_electrons(atom_z)
    nocc = ne // 2
    v_ion = local_potential(g.points(), atom_pos, atom_z, species)
    P, E, _ = kb_projectors(g, atom_pos, atom_z, species)
    H = Hamiltonian(g, res["v_in"], P, E)
    conv = cf.chefsi_converged(H, res["X"], degree, nocc + 1, tol=tol, max_iter=max_iter)
    occ, _, minus_ts = occupations(conv["lam"], ne, 0.0)
    rho = cf.density(conv["X"], occ)
    vh = Poisson(g).solve(rho)
    eps, _ = lda_xc(rho)
    e = total_energy(H.h3, float(np.dot(occ, conv["lam"])), rho, res["v_in"], v_ion, vh, eps, minus_ts)
    return {"lam": conv["lam"], "X": conv["X"], "rho": rho, "e_total": e, "iters": conv["iters"], "res": conv["res"]}


def scf(atom_pos, atom_z, species, radius, h, k, degree, X0, max_steps=40, sre_tol_ry=1e-4,
        first_iters=4, alpha=0.3, history=8, center=None, kT=0.0, kerker_q0=0.0, degree_min=0,
        degree_max=0, reduction=0.1, tol_floor=1e-6, group=64):
    """Run the SCF; returns a dict with per-step reports and the final state."""
    from .grid import sphere_grid
    from .potential import kb_projectors, local_potential
    from workloads.cluster import n_electrons

    atom_pos = np.asarray(atom_pos, dtype=np.float64)
    c = atom_pos[0] if center is None else np.asarray(center)
    g = sphere_grid(c, radius, h)
    pts = g.points()
    v_ion = local_potential(pts, atom_pos, atom_z, species)
    P, E, _ = kb_projectors(g, atom_pos, atom_z, species)
    pois = Poisson(g)
    ne = n_electrons(atom_z)
    nocc = ne // 2
    rho0 = atomic_density(pts, atom_pos, atom_z, species)
    vh = pois.solve(rho0)
    _, vxc = lda_xc(rho0)
    v_in = v_ion + vh + vxc
    H = Hamiltonian(g, v_in, P, E)
    X, _ = cf.cholesky_qr(np.array(X0, dtype=np.float64), H.h3)
    lam, X, _ = cf.rayleigh_ritz(H, X, H.h3)
    mixer = Anderson(alpha, history, Kerker(g, kerker_q0) if kerker_q0 > 0 else None)
    reports = []
    vh_prev = vh
    adaptive = degree_max > 0
    for step in range(1, max_steps + 1):
        H = Hamiltonian(g, v_in, P, E)
        b = cf.spectral_upper_bound(H)
        work = 0.0
        for _ in range(first_iters if step == 1 else 1):
            if adaptive:
                rq, resid = rayleigh_residuals(H, X)
                tol = np.maximum(tol_floor, reduction * resid)
                degs = group_degrees(rq, resid, lam[-1], b, tol, degree_min, degree_max, group)
                Y = X.copy()
                for gi, m_g in enumerate(degs):
                    cols = slice(gi * group, min(k, (gi + 1) * group))
                    Y[:, cols] = cf.chebyshev_filter(H, X[:, cols], m_g, lam[-1], b, lam[0])
                    work += m_g * (cols.stop - cols.start) / k
            else:
                Y = cf.chebyshev_filter(H, X, degree, lam[-1], b, lam[0])
                work += degree
            X, _ = cf.cholesky_qr(Y, H.h3)
            lam, X, _ = cf.rayleigh_ritz(H, X, H.h3)
        occ, mu, minus_ts = occupations(lam, ne, kT)
        rho = cf.density(X, occ)
        vh = pois.solve(rho, x0=vh_prev)
        vh_prev = vh
        eps, vxc = lda_xc(rho)
        v_out = v_ion + vh + vxc
        f = v_out - v_in
        sre = 2.0 * math.sqrt(H.h3 * float(np.sum(rho * f * f)))
        e_band = float(np.dot(occ, lam))
        e_tot = total_energy(H.h3, e_band, rho, v_in, v_ion, vh, eps, minus_ts)
        reports.append({"step": step, "sre_ry": sre, "e_band": e_band, "e_total": e_tot, "mu": mu,
                        "filter_work": work,
                        "minus_ts": minus_ts,
                        "homo": float(lam[nocc - 1]), "lumo": float(lam[nocc]) if k > nocc else float("nan"),
                        "electrons": H.h3 * float(rho.sum()), "lam": lam.copy()})
        if sre < sre_tol_ry:
            break
        v_in = mixer.step(v_in, f)
    return {"reports": reports, "X": X, "lam": lam, "rho": rho, "v_in": v_in, "grid": g, "n_occ": nocc}
