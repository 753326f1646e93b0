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


def test_filter_fullsize_bench_config(kscf, species):
    from oracle.chefsi import chebyshev_filter
    from oracle.system import cluster_hamiltonian
    from workloads import random_block_lex, workload
    w = workload("si353h196")
    pos, z = w.atoms()
    g, H = kscf.build_cluster(pos, z, species, w.radius, w.h)
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
