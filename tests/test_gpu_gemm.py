"""GPU parity of the subspace GEMM building blocks (Gram and rotation) against FP64
numpy products of the same FP32 inputs, in both GEMM modes.

Tolerance: elementwise |C - C_ref| <= tol * (|A|^T |B|)  (tol 2e-6: FP32 products and
FP32 partial sums over at most 2048 rows give ~sqrt(#adds) * 2^-24 of the magnitude;
the split-bf16 tensor mode drops terms of order 2^-24)."""
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


MODES = [0, 1]


def rand(shape, seed, scale=1.0):
    return (np.random.default_rng(seed).standard_normal(shape) * scale).astype(np.float32)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("rows,m,n", [(5000, 300, 200), (37, 5, 7), (40000, 130, 257)])
def test_gram(kscf, mode, rows, m, n):
    A = rand((rows, m), 1)
    B = rand((rows, n), 2) * np.linspace(0.1, 10, n).astype(np.float32)
    C = kscf.kscf_gram(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), scale=0.5,
                       mode=mode).cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = 0.5 * A64.T @ B64
    bound = 0.5 * np.abs(A64).T @ np.abs(B64)
    assert np.all(np.abs(C - ref) <= 2e-6 * bound)


@pytest.mark.parametrize("mode", MODES)
def test_gram_symmetric(kscf, mode):
    A = rand((30000, 290), 3)
    At = torch.tensor(A, device="cuda")
    C = kscf.kscf_gram(At, At, scale=1.0, mode=mode).cpu().numpy()
    A64 = A.astype(np.float64)
    ref = A64.T @ A64
    assert np.array_equal(C, C.T)
    assert np.all(np.abs(C - ref) <= 2e-6 * (np.abs(A64).T @ np.abs(A64)))
    # sums of squares expose any systematic truncation of long FP32 accumulation chains
    assert np.max(np.abs(np.diag(C) - np.diag(ref)) / np.diag(ref)) < 5e-7


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("rows,kin,kout", [(3000, 300, 300), (129, 40, 17), (700, 257, 260)])
def test_rotate(kscf, mode, rows, kin, kout):
    A = rand((rows, kin), 4)
    Q = np.random.default_rng(5).standard_normal((kin, kout))
    out = kscf.kscf_rotate(torch.tensor(A, device="cuda"), torch.tensor(Q, device="cuda"), mode=mode).cpu().numpy()
    A64 = A.astype(np.float64)
    ref = A64 @ Q
    assert np.all(np.abs(out - ref) <= 2e-6 * (np.abs(A64) @ np.abs(Q)) + 1e-30)


def test_rotate_near_identity(kscf):
    A = rand((5000, 200), 6)
    Q = np.eye(200) + 1e-3 * np.random.default_rng(7).standard_normal((200, 200))
    out = kscf.kscf_rotate(torch.tensor(A, device="cuda"), torch.tensor(Q, device="cuda"), mode=1,
                           minus_identity=True).cpu().numpy()
    A64 = A.astype(np.float64)
    ref = A64 @ Q
    # the error is that of the small correction A (Q - I) plus FP32 rounding of the sum
    bound = 2e-6 * (np.abs(A64) @ np.abs(Q - np.eye(200))) + 1.2e-7 * np.abs(ref)
    assert np.all(np.abs(out - ref) <= bound)
