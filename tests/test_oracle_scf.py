"""Pins of the oracle's SCF pieces: LDA exchange-correlation (potential = derivative of
the energy density, branch continuity of PZ81, the exchange constant), the Poisson
solver against the analytic potential of Gaussian charges, Anderson mixing on a linear
fixed-point problem, and a converged SCF of SiH4."""
import math

import numpy as np
import pytest

from oracle.grid import sphere_grid
from oracle.scf import Anderson, Poisson, lda_xc, scf


def test_vxc_is_derivative_of_energy_density():
    rho = np.logspace(-5, 1.5, 40)     # r_s from ~29 down to ~0.2: both PZ81 branches
    eps, v = lda_xc(rho)
    d = 1e-6 * rho
    ep, _ = lda_xc(rho + d)
    em, _ = lda_xc(rho - d)
    num = ((rho + d) * ep - (rho - d) * em) / (2 * d)
    assert np.max(np.abs(num - v) / np.abs(v)) < 1e-7


def test_pz81_branches_meet_and_exchange_constant():
    rs = np.array([1.0 - 1e-9, 1.0 + 1e-9])
    rho = 3.0 / (4.0 * math.pi * rs ** 3)
    eps, v = lda_xc(rho)
    ex = -0.75 * (3.0 * rho / math.pi) ** (1.0 / 3.0)
    ec = eps - ex
    # the published constants are rounded: the two branches meet to a few 1e-5 Ha
    assert abs(ec[0] - ec[1]) < 5e-5 and abs(v[0] - v[1]) < 5e-4
    assert abs(ex[0] + 0.458165) < 1e-6             # Slater exchange per electron at r_s = 1
    eps0, v0 = lda_xc(np.array([0.0, 1e-20]))
    assert np.all(eps0 == 0) and np.all(v0 == 0)


@pytest.mark.parametrize("centre,tol", [((0.0, 0.0, 0.0), 1e-5), ((0.9, -0.6, 0.4), 1e-3)])
def test_poisson_gaussian_charge(centre, tol):
    # centred: the monopole boundary values are exact; off-centre: the expansion stops at
    # the quadrupole, the octupole is ~2e-4 of max V here, while a missing dipole (~1e-2)
    # or quadrupole (~1.5e-3) term exceeds the tolerance
    from scipy.special import erf
    g = sphere_grid((0.0, 0.0, 0.0), 10.0, 0.35)
    x = g.points()
    sig, q = 1.3, 2.0
    d = x - np.array(centre)
    r = np.sqrt((d * d).sum(1))
    rho = q / (math.pi ** 1.5 * sig ** 3) * np.exp(-r * r / sig ** 2)
    V = Poisson(g).solve(rho)
    exact = q * erf(r / sig) / np.where(r > 0, r, 1.0)
    exact[r == 0] = 2 * q / (sig * math.sqrt(math.pi))
    assert np.max(np.abs(V - exact)) < tol * exact.max()


def test_anderson_solves_linear_fixed_point():
    rng = np.random.default_rng(0)
    n = 20
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    M = Q @ np.diag(np.linspace(-0.6, 0.9, n)) @ Q.T
    b = rng.standard_normal(n)
    exact = np.linalg.solve(np.eye(n) - M, b)
    mix = Anderson(alpha=0.5, history=n + 2)
    v = np.zeros(n)
    for _ in range(n + 3):
        f = (M @ v + b) - v
        v = mix.step(v, f)
    assert np.max(np.abs(v - exact)) < 1e-9


def test_scf_sih4_converges():
    from workloads import pseudo_params, random_block_lex
    dd = 1.48 / 0.529177210903 / np.sqrt(3.0)
    pos = np.array([[0.0, 0.0, 0.0], [dd, dd, dd], [dd, -dd, -dd], [-dd, dd, -dd], [-dd, -dd, dd]]) + 0.05
    z = np.array([14, 1, 1, 1, 1], dtype=np.int32)
    g = sphere_grid(pos[0], 8.0, 0.5)
    X0 = random_block_lex(1, g.n, 8)
    r = scf(pos, z, pseudo_params(), 8.0, 0.5, 8, 10, X0, max_steps=40)
    rep = r["reports"]
    assert rep[-1]["sre_ry"] < 1e-4
    assert abs(rep[-1]["electrons"] - 8.0) < 1e-9
    assert abs(rep[-1]["e_total"] - rep[-2]["e_total"]) < 1e-5
    assert rep[-1]["lumo"] > rep[-1]["homo"]
