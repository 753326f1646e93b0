"""Pins of the oracle's CheFSI steps: the filter against the Chebyshev closed form,
Cholesky-QR against orthonormality and a library QR, converged Rayleigh-Ritz against
the box-Laplacian closed-form spectrum, the harmonic oscillator, a brute-force dense
eigensolve, and the density against the electron count and the analytic ground state of
the harmonic oscillator."""
import math

import numpy as np
import pytest

from oracle.chefsi import (chebyshev_filter, cholesky_qr, chefsi, chefsi_converged, density,
                           rayleigh_ritz, residual_norms)
from oracle.grid import box_grid, sphere_grid
from oracle.hamiltonian import Hamiltonian, kinetic_matrix
from oracle.potential import kb_projectors, local_potential


class DiagOp:
    def __init__(self, d, h=1.0):
        self.d = np.asarray(d, float)
        self.h = h
        self.h3 = h ** 3

    def apply(self, Y):
        return self.d[:, None] * Y if Y.ndim == 2 else self.d * Y


def cheb(m, t):
    t = np.asarray(t, float)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1
    out[inside] = np.cos(m * np.arccos(t[inside]))
    ti = t[~inside]
    out[~inside] = np.sign(ti) ** m * np.cosh(m * np.arccosh(np.abs(ti)))
    return out


@pytest.mark.parametrize("m", [1, 2, 5, 10, 20])
def test_filter_matches_chebyshev_closed_form(m):
    lam = np.linspace(-3.0, 12.0, 301)
    a, b, a0 = 1.0, 12.5, -3.2
    X = np.eye(len(lam))[:, ::7] + 0.3
    Y = chebyshev_filter(DiagOp(lam), X, m, a, b, a0)
    e, c = (b - a) / 2, (b + a) / 2
    scale = cheb(m, (lam - c) / e) / cheb(m, np.array([(a0 - c) / e]))[0]
    assert np.allclose(Y, scale[:, None] * X, rtol=1e-12, atol=1e-12 * np.abs(scale).max())


def test_filter_bounds_validated():
    with pytest.raises(ValueError):
        chebyshev_filter(DiagOp([1.0, 2.0]), np.ones((2, 1)), 3, 5.0, 4.0, 0.0)


def test_cholesky_qr():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((500, 20)) @ np.triu(rng.standard_normal((20, 20)) + 5 * np.eye(20))
    h3 = 0.343
    Xn, R = cholesky_qr(X, h3)
    assert np.max(np.abs(h3 * Xn.T @ Xn - np.eye(20))) < 1e-12
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R) > 0)
    assert np.allclose(Xn @ R, X, rtol=0, atol=1e-11 * np.abs(X).max())
    Q, Rq = np.linalg.qr(np.sqrt(h3) * X)              # library QR, signs fixed
    sgn = np.sign(np.diag(Rq))
    assert np.allclose(Xn * math.sqrt(h3), Q * sgn, atol=1e-10)


def test_box_laplacian_chefsi_matches_closed_form():
    nx, ny, nz, h = 9, 10, 11, 0.6
    g = box_grid(nx, ny, nz, h)
    H = Hamiltonian(g, np.zeros(g.n))
    # 1D dense spectra (independent construction via the closed-form weights)
    from test_oracle_hamiltonian import closed_form_weights, toeplitz_1d
    w = closed_form_weights()
    e1 = [np.linalg.eigvalsh(toeplitz_1d(n, h, w)) for n in (nx, ny, nz)]
    allv = np.sort((e1[0][:, None, None] + e1[1][None, :, None] + e1[2][None, None, :]).ravel())
    k, nwant = 16, 10
    X0 = np.random.default_rng(5).standard_normal((g.n, k))
    r = chefsi_converged(H, X0, m=12, n_want=nwant, tol=1e-9)
    assert np.max(np.abs(r["lam"][:nwant] - allv[:nwant])) < 1e-9


@pytest.fixture(scope="module")
def oscillator():
    # V = omega^2 r^2 / 2 on a sphere large enough that the low states vanish at the wall
    omega, h, R = 1.0, 0.3, 6.5
    g = sphere_grid((0.0, 0.0, 0.0), R, h)
    x = g.points()
    V = 0.5 * omega ** 2 * (x * x).sum(1)
    H = Hamiltonian(g, V)
    X0 = np.random.default_rng(7).standard_normal((g.n, 16))
    return omega, g, chefsi_converged(H, X0, m=16, n_want=10, tol=1e-7)


def test_harmonic_oscillator(oscillator):
    # levels omega (n + 3/2) with degeneracies 1, 3, 6
    omega, _, r = oscillator
    expect = np.array([1.5] + [2.5] * 3 + [3.5] * 6) * omega
    assert np.max(np.abs(r["lam"][:10] - expect)) < 1e-6


def test_density_of_oscillator_ground_state(oscillator):
    """rho of the doubly occupied ground state = 2 |psi_0|^2 with the analytic
    psi_0(r) = (omega/pi)^(3/4) exp(-omega r^2 / 2).  Taking another column (an excited
    state), dropping the occupation factor or squaring the wrong axis of X fails."""
    omega, g, r = oscillator
    x = g.points()
    exact = 2.0 * (omega / math.pi) ** 1.5 * np.exp(-omega * (x * x).sum(1))
    rho = density(r["X"], np.array([2.0]))
    assert np.max(np.abs(rho - exact)) < 1e-5 * exact.max()
    assert abs(g.h ** 3 * rho.sum() - 2.0) < 1e-10


def _tiny_cluster(species):
    pos = np.array([[0.15, -0.1, 0.05], [2.2, 2.1, -2.3], [-1.7, 0.9, 2.6]])
    z = np.array([14, 1, 1], dtype=np.int32)
    g = sphere_grid(pos[0], 5.5, 0.7)
    V = local_potential(g.points(), pos, z, species)
    P, E, _ = kb_projectors(g, pos, z, species)
    return Hamiltonian(g, V, P, E)


def test_converged_chefsi_matches_bruteforce(species):
    H = _tiny_cluster(species)
    lam_all = np.linalg.eigvalsh(H.dense())
    k, nwant = 12, 8
    X0 = np.random.default_rng(11).standard_normal((H.n, k))
    r = chefsi_converged(H, X0, m=10, n_want=nwant, tol=1e-8)
    assert np.max(np.abs(r["lam"][:nwant] - lam_all[:nwant])) < 1e-9
    assert np.max(np.abs(H.h3 * r["X"].T @ r["X"] - np.eye(k))) < 1e-12


def test_rayleigh_ritz_on_invariant_subspace(species):
    H = _tiny_cluster(species)
    lam_all, Vec = np.linalg.eigh(H.dense())
    rot = np.linalg.qr(np.random.default_rng(2).standard_normal((6, 6)))[0]
    X = Vec[:, :6] @ rot / math.sqrt(H.h3)
    lam, Xr, HXr = rayleigh_ritz(H, X, H.h3)
    assert np.allclose(lam, lam_all[:6], atol=1e-11)
    assert np.max(residual_norms(Xr, HXr, lam, H.h3)) < 1e-9


def test_density_electron_count(species):
    H = _tiny_cluster(species)
    X0 = np.random.default_rng(4).standard_normal((H.n, 10))
    r = chefsi(H, X0, m=8, n_iter=2)
    occ = np.full(6, 2.0)
    rho = density(r["X"], occ)
    assert abs(H.h3 * rho.sum() - 12.0) < 1e-10
    assert np.all(rho >= 0)
