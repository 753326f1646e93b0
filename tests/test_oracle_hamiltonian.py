"""Pins of the oracle Hamiltonian: kinetic spectrum on a box (closed form), polynomial
exactness, Hermiticity, KB projectors against point-by-point dense assembly, the local
potential against its limits, and the spectral upper bound."""
import math
from fractions import Fraction
from math import factorial

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.grid import box_grid, sphere_grid
from oracle.hamiltonian import Hamiltonian, kinetic_matrix
from oracle.potential import kb_projectors, local_potential
from oracle.chefsi import spectral_upper_bound


def closed_form_weights(M=6):
    wk = [2 * (-1) ** (k + 1) * factorial(M) ** 2 / (k * k * factorial(M - k) * factorial(M + k))
          for k in range(1, M + 1)]
    return [-2 * sum(wk)] + wk


def toeplitz_1d(n, h, w):
    """-1/2 d^2/dx^2 on n points with zero Dirichlet outside (dense)."""
    T = np.zeros((n, n))
    for i in range(n):
        T[i, i] = -0.5 * w[0] / h ** 2
        for k in range(1, 7):
            for j in (i - k, i + k):
                if 0 <= j < n:
                    T[i, j] = -0.5 * w[k] / h ** 2
    return T


def test_box_kinetic_spectrum_is_kronecker_sum():
    nx, ny, nz, h = 5, 6, 7, 0.7
    w = closed_form_weights()
    ex, ey, ez = (np.linalg.eigvalsh(toeplitz_1d(n, h, w)) for n in (nx, ny, nz))
    expect = np.sort((ex[:, None, None] + ey[None, :, None] + ez[None, None, :]).ravel())
    g = box_grid(nx, ny, nz, h)
    T = kinetic_matrix(g).toarray()
    got = np.linalg.eigvalsh(T)
    assert np.max(np.abs(got - expect)) < 1e-11 * np.max(np.abs(expect))


def test_kinetic_exact_on_polynomials_inside():
    h, R = 0.3, 6.0
    g = sphere_grid((0.3, -0.2, 0.1), R, h)
    x, y, z = g.points().T
    f = x ** 3 * y ** 2 + z ** 5 - 2 * x * y * z + y ** 7
    lap = 6 * x * y ** 2 + 2 * x ** 3 + 20 * z ** 3 + 42 * y ** 5
    Tf = kinetic_matrix(g) @ f
    r = np.sqrt(((g.ijk.astype(float)) ** 2).sum(1)) * h
    inner = r + 6 * h <= R - 1e-9          # every axis neighbour is inside the domain
    assert inner.sum() > 100
    assert np.max(np.abs(Tf[inner] + 0.5 * lap[inner])) < 1e-8 * np.max(np.abs(lap))


def _small_system(species):
    pos = np.array([[0.1, 0.2, -0.15], [2.3, -1.1, 1.7], [-2.0, 1.9, 0.4]])
    z = np.array([14, 14, 1], dtype=np.int32)
    g = sphere_grid(pos[0], 6.0, 0.7)
    V = local_potential(g.points(), pos, z, species)
    P, E, owner = kb_projectors(g, pos, z, species)
    return g, pos, z, V, P, E, owner


def test_kb_matches_pointwise_dense_assembly(species):
    g, pos, z, V, P, E, owner = _small_system(species)
    sp = {s["z_number"]: s for s in species}
    pts = g.points()
    B = np.zeros((g.n, g.n))
    for a in range(len(pos)):
        s = sp[int(z[a])]
        if s["n_proj"] == 0:
            continue
        chis = [np.zeros(g.n) for _ in range(4)]
        for p in range(g.n):
            d = pts[p] - pos[a]
            r2 = float(d @ d)
            if r2 <= s["r_cut"] ** 2:
                gval = math.exp(-r2 / (2 * s["r_p"] ** 2))
                chis[0][p] = gval
                for m in range(3):
                    chis[m + 1][p] = d[m] / s["r_p"] * gval
        for m, e in enumerate([s["e_s"], s["e_p"], s["e_p"], s["e_p"]]):
            B += e * g.h ** 3 * np.outer(chis[m], chis[m])
    H = Hamiltonian(g, np.zeros(g.n), P, E)
    T = kinetic_matrix(g).toarray()
    assert P.shape[1] == 8 and list(owner) == [0] * 4 + [1] * 4
    got = H.dense() - T
    assert np.max(np.abs(got - B)) < 1e-13 * np.max(np.abs(B))


def test_kb_projector_symmetry(species):
    # atom on a grid point: s and p projectors are orthogonal on the grid, p_x and p_y
    # exchange under the x<->y mirror, and the support is the lattice ball of radius 3.5
    h = 0.5
    g = sphere_grid((0.0, 0.0, 0.0), 6.0, h)
    pos = np.array([[0.0, 0.0, 0.0]])
    P, E, _ = kb_projectors(g, pos, np.array([14]), species)
    P = P.toarray()
    G = P.T @ P
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-12 * G.max()
    assert abs(G[1, 1] - G[2, 2]) < 1e-12 * G[1, 1] and abs(G[2, 2] - G[3, 3]) < 1e-12 * G[1, 1]
    swapped = g.index_of(g.ijk[:, [1, 0, 2]])
    assert np.allclose(P[swapped, 1], P[:, 2], atol=1e-15)
    n_ball = sum(1 for i in range(-8, 9) for j in range(-8, 9) for k in range(-8, 9)
                 if (i * i + j * j + k * k) * h * h <= 3.5 ** 2)
    assert np.count_nonzero(P[:, 0]) == n_ball
    assert np.all(P[g.index_of(np.array([[1, 0, 0]]))[0], [1, 2, 3]] > [0, -1e-300, -1e-300])


def test_local_potential_limits(species):
    sp = {s["z_number"]: s for s in species}
    si = sp[14]
    pts = np.array([[0.0, 0.0, 0.0], [30.0, 0.0, 0.0], [0.0, 0.0, 1e-9]])
    V = local_potential(pts, np.zeros((1, 3)), np.array([14]), species)
    v0 = -2 * si["z_valence"] / (si["r_c"] * math.sqrt(math.pi)) + si["a_gauss"]
    assert abs(V[0] - v0) < 1e-14
    assert abs(V[1] + si["z_valence"] / 30.0) < 1e-14          # pure Coulomb tail far away
    assert abs(V[2] - V[0]) < 1e-9                               # continuous at r = 0
    two = local_potential(pts, np.array([[0.0, 0, 0], [1.0, 2.0, 3.0]]), np.array([14, 1]), species)
    one_h = local_potential(pts, np.array([[1.0, 2.0, 3.0]]), np.array([1]), species)
    assert np.allclose(two, V + one_h, rtol=0, atol=1e-14)       # superposition


def test_hermiticity(species):
    g, pos, z, V, P, E, _ = _small_system(species)
    H = Hamiltonian(g, V, P, E)
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal(g.n), rng.standard_normal(g.n)
    lhs, rhs = u @ H.apply(v), H.apply(u) @ v
    norm = np.linalg.norm(u) * np.linalg.norm(v) * 30.0
    assert abs(lhs - rhs) < 1e-13 * norm


def test_upper_bound_is_above_spectrum(species):
    g, pos, z, V, P, E, _ = _small_system(species)
    H = Hamiltonian(g, V, P, E)
    lam_max = np.linalg.eigvalsh(H.dense())[-1]
    b = spectral_upper_bound(H)
    assert b >= lam_max
    assert b - lam_max < 0.3 * (b - V.min())      # and not absurdly loose


def test_apply_at_rows_equals_full_apply(species):
    from oracle.hamiltonian import apply_at_rows
    g, pos, z, V, P, E, _ = _small_system(species)
    H = Hamiltonian(g, V, P, E)
    Y = np.random.default_rng(1).standard_normal((g.n, 3))
    rows = np.array([0, 5, 100, g.n - 1, 1234])
    assert np.max(np.abs(apply_at_rows(g, rows, V[rows], P, E, Y) - H.apply(Y)[rows])) < 1e-12
