"""DOS and gap: oracle pins (closed forms) and the library's host function against the
oracle (bin counts exact), on host values and on Ritz values computed on the GPU."""
import numpy as np
import pytest

from oracle.dos import HARTREE_EV, dos


def test_oracle_dos_closed_form():
    # three occupied levels at -0.25, -0.15 eV (twice) and the HOMO at 0, a LUMO at +1.03 eV
    lam = np.array([0.0, -0.25, -0.15, -0.15, 1.03]) / HARTREE_EV - 0.2
    h, edges, gap = dos(lam, 4, 0.1, -1.0, 30)
    assert abs(gap - 1.03) < 1e-12
    assert np.allclose(edges[:3], [-1.0, -0.9, -0.8])
    c = np.rint(h * 4 * 0.1).astype(int)
    assert c[7] == 1 and c[8] == 2 and c[10] == 1 and c[20] == 1 and c.sum() == 5
    # occupied states integrate to one
    assert abs(h[edges < 0].sum() * 0.1 + h[10] * 0.1 - 1.0) < 1e-12


def test_library_dos_matches_oracle():
    kscf = pytest.importorskip("paper_2303_00790_gb300.kscf")
    rng = np.random.default_rng(1)
    lam = np.sort(rng.uniform(-0.6, 0.1, 850))
    for n_occ in (1, 804, 850):
        h, edges, gap = kscf.kscf_dos(lam[::-1].copy(), n_occ)
        hr, er, gr = dos(lam, n_occ)
        assert np.array_equal(np.rint(h * n_occ * 0.1), np.rint(hr * n_occ * 0.1))
        assert np.allclose(h, hr, rtol=1e-14, atol=0)
        assert np.allclose(edges, er)
        assert (np.isnan(gap) and np.isnan(gr)) or abs(gap - gr) < 1e-12


@pytest.mark.gpu
def test_dos_of_gpu_ritz_values_matches_oracle(species):
    """Ritz values produced on the GPU (three CheFSI iterations on Si2H2, FP64) go through
    kscf_dos; its histogram and gap equal the oracle's on the same values (counts exact),
    and the values themselves match the oracle's CheFSI from the same X0 (1e-10)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00790_gb300.build import build
    build()
    from paper_2303_00790_gb300 import kscf
    from helpers import small_cluster, to_slots
    from oracle.chefsi import chefsi
    from oracle.system import cluster_hamiltonian
    from workloads import random_block_lex
    pos, z = small_cluster()
    g, H = kscf.build_cluster(pos, z, species, 9.0, 0.7)
    lex, _ = g.slots()
    n, k, m, n_occ = g.info["n_points"], 24, 10, 5
    X0 = random_block_lex(3, n, k)
    X = torch.tensor(to_slots(X0, lex), device="cuda")
    _, b = kscf.kscf_spectral_bounds(H)
    kscf.kscf_orthonormalize(H, X)
    lam = kscf.kscf_rayleigh_ritz(H, X)
    for _ in range(3):
        kscf.kscf_chebyshev_filter(H, X, m, lam[-1], b, lam[0])
        kscf.kscf_orthonormalize(H, X)
        lam = kscf.kscf_rayleigh_ritz(H, X)
    ref = chefsi(cluster_hamiltonian(pos, z, species, 9.0, 0.7), X0, m, 3, b=b)["lam"]
    assert np.max(np.abs(lam - ref)) < 1e-10 * np.max(np.abs(ref))
    for bin_ev, lo, nb in ((0.1, -15.0, 200), (0.25, -30.0, 160)):
        h, edges, gap = kscf.kscf_dos(lam, n_occ, bin_ev, lo, nb)
        hr, er, gr = dos(lam, n_occ, bin_ev, lo, nb)
        assert np.array_equal(np.rint(h * n_occ * bin_ev), np.rint(hr * n_occ * bin_ev))
        assert np.allclose(h, hr, rtol=1e-14, atol=0) and np.allclose(edges, er)
        assert abs(gap - gr) < 1e-12 and gap > 0
