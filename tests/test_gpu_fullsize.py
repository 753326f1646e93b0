"""Parity at the full workload sizes, in the launch configuration bench.py times.

The filter acts on each vector independently, so at the benchmark size (Si353H196 in a
2.2 nm sphere: 234,489 points, k = 850, degree 12, one 850-column block) the oracle runs
the whole degree-12 filter on a few sampled columns over all points.  At the largest
size (Si3325H876 in a 5 nm sphere: 1.84M points, k = 7700, blocks of 1024) one degree
step is checked at sampled rows with the row-wise oracle H apply."""
import numpy as np
import pytest

from helpers import from_slots

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


def device_block(kscf, H, n_slots, k, seed):
    kpad = (k + 31) // 32 * 32
    full = torch.zeros((n_slots, kpad), dtype=torch.float32, device="cuda")
    X = full[:, :k]
    kscf.kscf_random_subspace(H, X, seed=seed)
    return full, X


@pytest.mark.parametrize("brick", [8, 16])
def test_filter_fullsize_bench_config(kscf, species, brick):
    """Bricks of 8^3 (the benchmark's layout) and 16^3 (the chunk-major kernel on the
    octants of each brick): the same filter, compared with the oracle on sampled columns
    over all points."""
    from oracle.chefsi import chebyshev_filter
    from oracle.system import cluster_hamiltonian
    from workloads import random_block_lex, workload
    w = workload("si353h196")
    pos, z = w.atoms()
    g, H = kscf.build_cluster(pos, z, species, w.radius, w.h, brick=brick)
    lex, _ = g.slots()
    n, n_slots, k = g.info["n_points"], g.info["n_slots"], w.k
    full, X = device_block(kscf, H, n_slots, k, seed=3)
    lo, b = kscf.kscf_spectral_bounds(H)
    a0, a = lo, lo + 0.35 * (b - lo)
    kscf.kscf_chebyshev_filter(H, X, w.degree, a, b, a0, block=w.block)
    kscf.kscf_check_status()
    cols = [0, 1, 15, 16, 127, 128, 511, 512, 831, 832, 848, 849]
    got = from_slots(X[:, cols].double().cpu().numpy(), lex, n)
    OH = cluster_hamiltonian(pos, z, species, w.radius, w.h)
    X0 = random_block_lex(3, n, k, cols=cols).astype(np.float32).astype(np.float64)
    ref = chebyshev_filter(OH, X0, w.degree, a, b, a0)
    colmax = np.max(np.abs(ref), axis=0)
    err = np.max(np.abs(got - ref), axis=0) / colmax
    assert np.all(err <= 1e-4), err


def test_step_fullsize_largest(kscf, species):
    from oracle.grid import sphere_grid
    from oracle.hamiltonian import apply_at_rows
    from oracle.potential import kb_projectors, local_potential
    from workloads import random_block_lex, workload
    w = workload("si3325h876")
    pos, z = w.atoms()
    g, H = kscf.build_cluster(pos, z, species, w.radius, w.h)
    lex, _ = g.slots()
    n, n_slots, k = g.info["n_points"], g.info["n_slots"], w.k
    full, X = device_block(kscf, H, n_slots, k, seed=5)
    lo, b = kscf.kscf_spectral_bounds(H)
    a0, a = lo, lo + 0.35 * (b - lo)
    kscf.kscf_chebyshev_filter(H, X, 1, a, b, a0, block=w.block)     # Y_1 = (s1/e)(H X - c X)
    kscf.kscf_check_status()
    cols = [0, 1, 1023, 1024, 4095, 7680, 7698, 7699]
    og = sphere_grid(pos[0], w.radius, w.h)
    assert og.n == n
    rng = np.random.default_rng(0)
    # sampled rows: random points plus points next to atoms (KB support) and at the surface
    near = og.index_of(np.rint((pos[:200] - og.center) / w.h).astype(np.int64))
    surf = np.argsort(-(og.ijk.astype(np.float64) ** 2).sum(1))[:50]
    rows = np.unique(np.concatenate([rng.integers(0, n, 250), near[near >= 0], surf]))
    got_all = X[:, cols].double().cpu().numpy()
    slot_of_lex = np.empty(n, dtype=np.int64)
    slot_of_lex[lex[lex >= 0]] = np.nonzero(lex >= 0)[0]
    got = got_all[slot_of_lex[rows]]
    Y = random_block_lex(5, n, k, cols=cols).astype(np.float32).astype(np.float64)
    V_rows = local_potential(og.points()[rows], pos, z, species)
    P, E, _ = kb_projectors(og, pos, z, species)
    HY = apply_at_rows(og, rows, V_rows, P, E, Y)
    e, c = (b - a) / 2, (b + a) / 2
    ref = (e / (a0 - c)) / e * (HY - c * Y[rows])
    scale = np.max(np.abs(ref), axis=0)
    assert np.all(np.max(np.abs(got - ref), axis=0) <= 2e-5 * scale)


def test_tensor_orthonormalize_and_rayleigh_ritz_fullsize(kscf, species):
    """Tensor-mode CholeskyQR2 and Rayleigh-Ritz at the benchmark size (336,384 slots x 850
    FP32, rotated in place in 5 row panels of 78,848 rows).  Checks: orthonormality of the
    split-bf16 result (< 2e-6); every panel rotated by the same k x k matrix (rows at each
    panel boundary equal X_before[rows] M, M recovered in FP64 from the whole block, to
    2e-5 of the rows' maximum); Ritz values within 1e-5 of the FP64 native path started
    from the same X; and the spans of the two Ritz bases within a principal angle of 1e-4."""
    from workloads import workload
    w = workload("si353h196")
    pos, z = w.atoms()
    g, H = kscf.build_cluster(pos, z, species, w.radius, w.h)
    n_slots, k = g.info["n_slots"], w.k
    h3 = g.info["h"] ** 3
    full, X = device_block(kscf, H, n_slots, k, seed=7)
    Xb = X.double().clone()
    kscf.kscf_orthonormalize(H, X, mode=kscf.KSCF_GEMM_TENSOR)
    Xa = X.double()
    eye = torch.eye(k, dtype=torch.float64, device="cuda")
    assert (h3 * (Xa.T @ Xa) - eye).abs().max().item() < 2e-6
    prows = (256 << 20) // (k * 4) // 512 * 512
    assert prows == 78848 and n_slots > 4 * prows
    bnd = np.unique(np.concatenate([[p * prows - 2, p * prows - 1, p * prows, p * prows + 1]
                                    for p in range(1, (n_slots - 1) // prows + 1)] + [[0, n_slots - 1]]))
    rows = torch.tensor(bnd, device="cuda")

    def same_matrix(before, after):
        M = torch.linalg.solve(before.T @ before, before.T @ after)
        err = (after[rows] - before[rows] @ M).abs().amax(1)
        return bool(torch.all(err <= 2e-5 * after[rows].abs().amax(1).clamp_min(1e-30)).item())

    assert same_matrix(Xb, Xa)
    X64 = Xb.clone()
    kscf.kscf_orthonormalize(H, X64, mode=kscf.KSCF_GEMM_NATIVE)
    before = X.double().clone()
    lam32 = kscf.kscf_rayleigh_ritz(H, X, mode=kscf.KSCF_GEMM_TENSOR)
    lam64 = kscf.kscf_rayleigh_ritz(H, X64, mode=kscf.KSCF_GEMM_NATIVE)
    assert np.max(np.abs(lam32 - lam64)) <= 1e-5 * np.max(np.abs(lam64))
    after = X.double()
    assert same_matrix(before, after)
    q1, _ = torch.linalg.qr(after)
    q2, _ = torch.linalg.qr(X64)
    s = torch.linalg.svdvals(q1.T @ q2)
    assert float(torch.sqrt(torch.clamp(1.0 - s.min() ** 2, min=0.0))) < 1e-4
