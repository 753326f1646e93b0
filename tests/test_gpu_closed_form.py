"""GPU CheFSI against closed forms, with no oracle in between: the box Laplacian
spectrum (Kronecker sum of 1D Toeplitz spectra) and the harmonic oscillator."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def kscf():
    from paper_2303_00790_gb300.build import build
    build()
    from paper_2303_00790_gb300 import kscf as mod
    return mod


def run_chefsi(kscf, H, X, m, iters):
    _, b = kscf.kscf_spectral_bounds(H)
    kscf.kscf_orthonormalize(H, X)
    lam = kscf.kscf_rayleigh_ritz(H, X)
    for _ in range(iters):
        kscf.kscf_chebyshev_filter(H, X, m, lam[-1], b, lam[0])
        kscf.kscf_orthonormalize(H, X)
        lam = kscf.kscf_rayleigh_ritz(H, X)
    return lam


def test_box_laplacian_spectrum(kscf):
    from test_oracle_hamiltonian import closed_form_weights, toeplitz_1d
    nx, ny, nz, h = 9, 10, 11, 0.6
    g = kscf.kscf_build_grid_box(nx, ny, nz, h, 8)
    H = kscf.kscf_build_hamiltonian(g, np.zeros((0, 3)), np.zeros(0, np.int32), [])
    w = closed_form_weights()
    e1 = [np.linalg.eigvalsh(toeplitz_1d(n, h, w)) for n in (nx, ny, nz)]
    allv = np.sort((e1[0][:, None, None] + e1[1][None, :, None] + e1[2][None, None, :]).ravel())
    X = torch.zeros((g.info["n_slots"], 16), dtype=torch.float64, device="cuda")
    kscf.kscf_random_subspace(H, X, seed=5)
    lam = run_chefsi(kscf, H, X, 12, 40)
    assert np.max(np.abs(lam[:10] - allv[:10])) < 1e-9


def test_harmonic_oscillator(kscf):
    omega, h, R = 1.0, 0.3, 6.5
    g = kscf.kscf_build_grid((0.0, 0.0, 0.0), R, h, 8)
    H = kscf.kscf_build_hamiltonian(g, np.zeros((0, 3)), np.zeros(0, np.int32), [])
    lex, ijk = g.slots()
    r2 = ((ijk.astype(np.float64) * h) ** 2).sum(1)
    v = torch.tensor(0.5 * omega ** 2 * r2, device="cuda")
    kscf.kscf_set_potential(H, v)
    X = torch.zeros((g.info["n_slots"], 16), dtype=torch.float64, device="cuda")
    kscf.kscf_random_subspace(H, X, seed=7)
    lam = run_chefsi(kscf, H, X, 16, 60)
    expect = np.array([1.5] + [2.5] * 3 + [3.5] * 6) * omega
    assert np.max(np.abs(lam[:10] - expect)) < 1e-6
