"""DOS and gap: oracle pins (closed forms) and the library's host function against the
oracle (bin counts exact)."""
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
