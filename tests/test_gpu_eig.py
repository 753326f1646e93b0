"""GPU parity of the FP64 symmetric eigensolver of the Rayleigh-Ritz step (kscf_sym_eig,
CheFSI paragraph: Hs = Q Lambda Q^T) against numpy's LAPACK eigh and closed forms.

Bar (u = 2^-53): a backward-stable FP64 solver gives eigenvalue errors and residuals of
O(n u max|A|) and orthogonality O(n u).  At n = 850 that is ~1e-13 of max|A|; the tests
allow 1e-12 of max|lambda| (eigenvalues), 1e-12 of max|A| (residual |A Z - Z Lambda|) and
1e-12 (|Z^T Z - I|).  Eigenvectors of a repeated eigenvalue are only defined as a
subspace: those groups are compared through their projectors.
"""
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


def solve(kscf, A):
    """Eigenpairs from the library: column j of the column-major result = row j of the
    row-major torch tensor."""
    At = torch.tensor(A, dtype=torch.float64, device="cuda")
    w = kscf.kscf_sym_eig(At)
    return w.cpu().numpy(), At.cpu().numpy().T


def check(A, lam, Z, tol=1e-12):
    ref = np.linalg.eigvalsh(A)
    scale = max(np.max(np.abs(ref)), np.finfo(float).tiny)
    amax = max(np.max(np.abs(A)), np.finfo(float).tiny)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - ref)) <= tol * scale
    assert np.max(np.abs(A @ Z - Z * lam)) <= tol * amax * max(1.0, len(lam) / 100)
    assert np.max(np.abs(Z.T @ Z - np.eye(len(lam)))) <= tol


def groups(lam, gap):
    out, start = [], 0
    for i in range(1, len(lam) + 1):
        if i == len(lam) or lam[i] - lam[i - 1] > gap:
            out.append((start, i))
            start = i
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 100, 257, 850])
def test_random_symmetric_matches_eigh(kscf, n):
    rng = np.random.default_rng(100 + n)
    B = rng.standard_normal((n, n))
    A = (B + B.T) / 2
    lam, Z = solve(kscf, A)
    check(A, lam, Z)


def test_ritz_like_near_diagonal(kscf):
    """The shape Rayleigh-Ritz sees late in CheFSI: sorted Ritz values in [-0.8, 0.1] Ha
    plus a small symmetric coupling."""
    rng = np.random.default_rng(7)
    n = 850
    A = np.diag(np.sort(rng.uniform(-0.8, 0.1, n)))
    E = rng.standard_normal((n, n)) * 1e-4
    A = A + (E + E.T) / 2
    lam, Z = solve(kscf, A)
    check(A, lam, Z)


def test_degenerate_groups_span_the_same_subspaces(kscf):
    """Eigenvalues of multiplicity 4 (exactly repeated): values to 1e-12, and for every
    group the projector Z_g Z_g^T equals the one from the construction."""
    rng = np.random.default_rng(11)
    n = 256
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    vals = np.repeat(np.sort(rng.standard_normal(n // 4)), 4)
    A = (Q * vals) @ Q.T
    A = (A + A.T) / 2
    lam, Z = solve(kscf, A)
    check(A, lam, Z)
    for a, b in groups(vals, 1e-9):
        P1 = Z[:, a:b] @ Z[:, a:b].T
        P2 = Q[:, a:b] @ Q[:, a:b].T
        assert np.max(np.abs(P1 - P2)) <= 1e-10


def test_toeplitz_closed_form(kscf):
    """tridiag(-1, 2, -1): lambda_k = 2 - 2 cos(k pi / (n + 1)), eigenvector entries
    sin(i k pi / (n + 1)) up to normalisation and sign."""
    n = 300
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    lam, Z = solve(kscf, A)
    k = np.arange(1, n + 1)
    exact = 2 - 2 * np.cos(k * np.pi / (n + 1))
    assert np.max(np.abs(lam - exact)) <= 1e-13 * 4
    i = np.arange(1, n + 1)[:, None]
    S = np.sin(i * k[None, :] * np.pi / (n + 1))
    S /= np.linalg.norm(S, axis=0)
    assert np.max(np.abs(np.abs(np.sum(S * Z, axis=0)) - 1.0)) <= 1e-10


@pytest.mark.parametrize("name", ["zero", "identity", "diagonal", "rank_one", "wilkinson", "glued", "graded",
                                  "tiny_scale", "huge_scale", "two_by_two"])
def test_special_matrices(kscf, name):
    rng = np.random.default_rng(3)
    n = 200
    if name == "zero":
        A = np.zeros((n, n))
    elif name == "identity":
        A = np.eye(n)
    elif name == "diagonal":
        A = np.diag(rng.standard_normal(n))
    elif name == "rank_one":
        A = np.ones((n, n))
    elif name == "wilkinson":
        A = np.diag(np.abs(np.arange(-10, 11)).astype(float)) + np.eye(21, k=1) + np.eye(21, k=-1)
    elif name == "glued":
        W = np.diag(np.abs(np.arange(-10, 11)).astype(float)) + np.eye(21, k=1) + np.eye(21, k=-1)
        A = np.kron(np.eye(5), W)
        for q in range(1, 5):
            A[21 * q - 1, 21 * q] = A[21 * q, 21 * q - 1] = 1e-10
    elif name == "graded":
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        A = (Q * np.logspace(-12, 0, n)) @ Q.T
        A = (A + A.T) / 2
    elif name in ("tiny_scale", "huge_scale"):
        B = rng.standard_normal((n, n))
        A = (B + B.T) * (1e-200 if name == "tiny_scale" else 1e200)
    else:
        A = np.array([[2.0, 1.0], [1.0, 2.0]])
    lam, Z = solve(kscf, A)
    if name == "zero":
        assert np.all(lam == 0.0)
        assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-14
        return
    if name == "two_by_two":
        assert np.max(np.abs(lam - [1.0, 3.0])) <= 1e-14, lam - [1.0, 3.0]   # iterative secular solve
    check(A, lam, Z)


def test_nonfinite_input_is_reported(kscf):
    A = np.eye(64)
    A[3, 5] = A[5, 3] = np.nan
    with pytest.raises(kscf.KscfError) as e:
        solve(kscf, A)
    assert e.value.code == kscf.KSCF_ERR_NONFINITE
    lam, Z = solve(kscf, np.eye(64) * 2.0)   # the context stays usable
    assert np.allclose(lam, 2.0, rtol=0, atol=1e-15)


def test_column_major_leading_dimension(kscf):
    """A stored with lda > n: only the leading n x n block is read and written."""
    rng = np.random.default_rng(5)
    n, lda = 100, 128
    B = rng.standard_normal((n, n))
    A = (B + B.T) / 2
    buf = torch.full((n, lda), 7.0, dtype=torch.float64, device="cuda")   # row j = column j
    buf[:, :n] = torch.tensor(A.T, dtype=torch.float64)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    b = kscf.C.c_size_t()
    kscf._check(kscf.lib.kscf_sym_eig_work_bytes(n, kscf.C.byref(b)))
    work = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    kscf._check(kscf.lib.kscf_sym_eig(kscf.C.c_void_p(buf.data_ptr()), lda, n, kscf.C.c_void_p(w.data_ptr()),
                                      kscf.C.c_void_p(work.data_ptr()), work.numel(), None))
    out = buf.cpu().numpy()
    assert np.all(out[:, n:] == 7.0)
    check(A, w.cpu().numpy(), out[:, :n].T)


def test_large_matrix_global_rows(kscf):
    """n = 2200: the trailing matrix no longer fits in shared memory and the
    tridiagonalisation works on the rows in global memory."""
    rng = np.random.default_rng(2200)
    n = 2200
    B = rng.standard_normal((n, n))
    A = (B + B.T) / 2
    lam, Z = solve(kscf, A)
    check(A, lam, Z)


def test_bounded_barrier_times_out_and_context_survives(kscf):
    """One CTA of the tridiagonalisation leaves at its first grid barrier: the others'
    waits (limit ~1 ms) give up, the call reports KSCF_ERR_TIMEOUT and a following solve
    is exact."""
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_selftest_eig_barrier_timeout()
    assert e.value.code == kscf.KSCF_ERR_TIMEOUT
    rng = np.random.default_rng(6)
    B = rng.standard_normal((120, 120))
    A = (B + B.T) / 2
    lam, Z = solve(kscf, A)
    check(A, lam, Z)
