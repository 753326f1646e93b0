"""Pins of the Lanczos bounds oracle (oracle/lanczos.py)."""
import numpy as np
import scipy.linalg as sla

from oracle.lanczos import lanczos, tridiag_eigs_bisect


def test_bisection_matches_lapack():
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 30):
        a = rng.standard_normal(n)
        b = rng.standard_normal(n - 1)
        ref = sla.eigvalsh_tridiagonal(a, b)
        assert np.allclose(tridiag_eigs_bisect(a, b), ref, atol=1e-12)


class Diag:
    def __init__(self, d):
        self.d = np.asarray(d, dtype=np.float64)
        self.h3 = 1.0

    def apply(self, Y):
        return self.d[:, None] * Y


def test_full_lanczos_recovers_a_diagonal_spectrum():
    d = np.array([-3.0, -1.0, 0.5, 2.0, 2.5, 7.0])
    x0 = np.ones(6)
    alpha, beta, upper, lower = lanczos(Diag(d), x0, 6)
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    assert np.allclose(np.linalg.eigvalsh(T), d, atol=1e-9)
    assert abs(lower - d[0]) < 1e-9 and upper >= d[-1] - 1e-9 and beta[-1] < 1e-6


def test_upper_bound_brackets_a_cluster_spectrum(species):
    from oracle import chefsi as orc
    from oracle.system import cluster_hamiltonian
    from workloads import random_block_lex
    pos = np.array([[0.1, 0.0, -0.1], [2.2, 2.2, 2.2], [-2.2, -2.2, 2.2]])
    z = np.array([14, 1, 1], dtype=np.int32)
    H = cluster_hamiltonian(pos, z, species, 5.0, 0.7)
    lam = np.linalg.eigvalsh(H.dense())
    x0 = random_block_lex(3, H.grid.n, 1)[:, 0]
    alpha, beta, upper, lower = lanczos(H, x0, 12)
    assert lam[-1] <= upper                    # the estimate is safe
    assert lower >= lam[0] - 1e-9              # Ritz values lie inside the spectrum
    assert lower - lam[0] < 0.6                # and approach its lower end
    alpha, beta, upper30, lower30 = lanczos(H, x0, 30)
    assert lam[-1] <= upper30 and 0 <= lower30 - lam[0] < 0.05
