"""GPU parity: every C-ABI call against the FP64 CPU oracle on the same seeded inputs.

Tolerances (derived from the arithmetic):
  FP64 paths: one H-apply sums ~45 terms of size <= |V| + 3*7.07/(2h^2) ~ 50 |y|, so
    rounding-order differences are <= ~1e-14 relative to max|Hy|; through the filter,
    Cholesky-QR and Rayleigh-Ritz they stay below 1e-10 relative.
  FP32 filter/apply: unit roundoff 6e-8 times the same ~45-term sums -> ~3e-6 of max|Hy|
    per step; the scaled recurrence keeps |Y_j| ~ |X| so m steps stay below 1e-4 of the
    column maximum.
"""
import numpy as np
import pytest

from helpers import from_slots, small_cluster, subspace_gap, to_slots

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


@pytest.fixture(scope="module", params=[8, 16])
def system(request, kscf, species):
    from oracle.system import cluster_hamiltonian
    pos, z = small_cluster()
    R, h = 9.0, 0.7
    g, H = kscf.build_cluster(pos, z, species, R, h, brick=request.param)
    OH = cluster_hamiltonian(pos, z, species, R, h)
    lex, ijk = g.slots()
    return {"g": g, "H": H, "OH": OH, "lex": lex, "n": g.info["n_points"], "brick": request.param}


def dev(a, dtype=torch.float64):
    return torch.tensor(a, dtype=dtype, device="cuda")


def test_potential_matches_oracle(kscf, system):
    V = kscf.kscf_get_potential(system["H"]).cpu().numpy()
    Vl = from_slots(V, system["lex"], system["n"])
    ref = system["OH"].V
    assert np.max(np.abs(Vl - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.all(V[system["lex"] < 0] == 0)


def test_spectral_bounds_match_oracle(kscf, system):
    from oracle.chefsi import spectral_upper_bound
    lo, hi = kscf.kscf_spectral_bounds(system["H"])
    ref = spectral_upper_bound(system["OH"])
    assert abs(hi - ref) <= 1e-12 * abs(ref)
    assert lo <= system["OH"].V.min() + 1e-12


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-5)])
def test_apply_matches_oracle(kscf, system, dtype, tol):
    from workloads import random_block_lex
    k = 13
    Y = random_block_lex(7, system["n"], k)
    if dtype == torch.float32:
        Y = Y.astype(np.float32).astype(np.float64)
    Yd = dev(to_slots(Y, system["lex"]), dtype)
    HYd = torch.full_like(Yd, 12345.0)
    kscf.kscf_hamiltonian_apply(system["H"], Yd, HYd)
    HY = HYd.double().cpu().numpy()
    ref = system["OH"].apply(Y)
    got = from_slots(HY, system["lex"], system["n"])
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    assert np.all(HY[system["lex"] < 0] == 0)


@pytest.mark.parametrize("dtype,tol,degree,block", [
    (torch.float64, 1e-11, 10, 0), (torch.float64, 1e-11, 7, 5), (torch.float64, 1e-11, 1, 0),
    (torch.float32, 1e-4, 10, 0), (torch.float32, 1e-4, 9, 8)])
def test_filter_matches_oracle(kscf, system, dtype, tol, degree, block):
    from oracle.chefsi import chebyshev_filter, spectral_upper_bound
    from workloads import random_block_lex
    k = 19
    X = random_block_lex(3, system["n"], k)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    b = spectral_upper_bound(system["OH"])
    a, a0 = -0.5, -9.0
    Xd = dev(to_slots(X, system["lex"]), dtype)
    kscf.kscf_chebyshev_filter(system["H"], Xd, degree, a, b, a0, block=block)
    got = from_slots(Xd.double().cpu().numpy(), system["lex"], system["n"])
    ref = chebyshev_filter(system["OH"], X, degree, a, b, a0)
    colmax = np.max(np.abs(ref), axis=0)
    assert np.all(np.max(np.abs(got - ref), axis=0) <= tol * colmax)


def test_filter_strided_columns(kscf, system):
    """X as a column slice of a wider array (ld > k): other columns untouched."""
    from oracle.chefsi import chebyshev_filter, spectral_upper_bound
    from workloads import random_block_lex
    X = random_block_lex(5, system["n"], 6)
    full = dev(to_slots(np.concatenate([X, np.ones((system["n"], 3))], 1), system["lex"]))
    view = full[:, :6]
    b = spectral_upper_bound(system["OH"])
    kscf.kscf_chebyshev_filter(system["H"], view, 4, 0.0, b, -9.0, block=4)
    got = full.cpu().numpy()
    ref = chebyshev_filter(system["OH"], X, 4, 0.0, b, -9.0)
    live = system["lex"] >= 0
    assert np.allclose(got[live, 6:], 1.0)
    g = from_slots(got[:, :6], system["lex"], system["n"])
    assert np.max(np.abs(g - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_orthonormalize_matches_oracle(kscf, system):
    from oracle.chefsi import cholesky_qr
    from workloads import random_block_lex
    k = 24
    X = random_block_lex(9, system["n"], k) + 0.5 * random_block_lex(10, system["n"], 1)
    Xd = dev(to_slots(X, system["lex"]))
    kscf.kscf_orthonormalize(system["H"], Xd)
    got = from_slots(Xd.cpu().numpy(), system["lex"], system["n"])
    ref, _ = cholesky_qr(X, system["OH"].h3)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    h3 = system["OH"].h3
    assert np.max(np.abs(h3 * got.T @ got - np.eye(k))) < 1e-12


@pytest.mark.parametrize("k", [33, 100, 200])
def test_orthonormalize_many_tiles_matches_oracle(kscf, system, k):
    # the FP64 factorisation runs on 32 x 32 tiles: blocks spanning several tiles with a
    # ragged last tile, against the oracle's Cholesky-QR (columns of very different norms)
    from oracle.chefsi import cholesky_qr
    from workloads import random_block_lex
    X = random_block_lex(11, system["n"], k) * np.logspace(0, -2, k)[None, :]
    X[:, k // 2:] += 0.3 * X[:, :k - k // 2]
    Xd = dev(to_slots(X, system["lex"]))
    kscf.kscf_orthonormalize(system["H"], Xd)
    got = from_slots(Xd.cpu().numpy(), system["lex"], system["n"])
    ref, _ = cholesky_qr(X, system["OH"].h3)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    h3 = system["OH"].h3
    assert np.max(np.abs(h3 * got.T @ got - np.eye(k))) < 1e-11
    Xf = dev(to_slots(X, system["lex"]), torch.float32)
    kscf.kscf_orthonormalize(system["H"], Xf, mode=kscf.KSCF_GEMM_TENSOR)
    gf = from_slots(Xf.double().cpu().numpy(), system["lex"], system["n"])
    assert np.max(np.abs(h3 * gf.T @ gf - np.eye(k))) < 2e-6
    assert subspace_gap(gf, X, h3) < 1e-4


def test_orthonormalize_f32_is_orthonormal(kscf, system):
    from workloads import random_block_lex
    k = 24
    X = random_block_lex(9, system["n"], k)
    Xd = dev(to_slots(X, system["lex"]), torch.float32)
    kscf.kscf_orthonormalize(system["H"], Xd)
    got = from_slots(Xd.double().cpu().numpy(), system["lex"], system["n"])
    h3 = system["OH"].h3
    assert np.max(np.abs(h3 * got.T @ got - np.eye(k))) < 2e-6
    assert subspace_gap(got, X, h3) < 1e-5


def test_rayleigh_ritz_matches_oracle(kscf, system):
    from oracle.chefsi import cholesky_qr, rayleigh_ritz
    from workloads import random_block_lex
    k = 16
    X, _ = cholesky_qr(random_block_lex(4, system["n"], k), system["OH"].h3)
    Xd = dev(to_slots(X, system["lex"]))
    lam = kscf.kscf_rayleigh_ritz(system["H"], Xd)
    ref_lam, ref_X, _ = rayleigh_ritz(system["OH"], X, system["OH"].h3)
    assert np.max(np.abs(lam - ref_lam)) <= 1e-11 * np.max(np.abs(ref_lam))
    got = from_slots(Xd.cpu().numpy(), system["lex"], system["n"])
    # eigenvectors up to sign (random subspace: simple Ritz values)
    sgn = np.sign(np.sum(got * ref_X, axis=0))
    assert np.max(np.abs(got * sgn - ref_X)) <= 1e-8 * np.max(np.abs(ref_X))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_points_slots_layout_round_trip(kscf, system, dtype):
    # a permutation with zero padding rows: bit-exact in both directions, columns >= k and
    # rows of P beyond the grid untouched
    k = 13
    rng = np.random.default_rng(21)
    P = rng.standard_normal((system["n"], k))
    Pd = torch.tensor(P, dtype=dtype, device="cuda")
    X = torch.full((system["g"].info["n_slots"], 16), 7.0, dtype=dtype, device="cuda")
    kscf.kscf_points_to_slots(system["H"], Pd, X[:, :k])
    ref = to_slots(P.astype(np.float32) if dtype == torch.float32 else P, system["lex"])
    assert np.array_equal(X[:, :k].cpu().numpy().astype(np.float64), ref.astype(np.float64))
    assert torch.all(X[:, k:] == 7.0)
    back = torch.full((system["n"] + 3, 20), -1.0, dtype=dtype, device="cuda")
    kscf.kscf_slots_to_points(system["H"], X[:, :k], back[:, :k])
    assert torch.equal(back[:system["n"], :k], Pd)
    assert torch.all(back[system["n"]:] == -1.0) and torch.all(back[:, k:] == -1.0)


def test_density_matches_oracle(kscf, system):
    from oracle.chefsi import density
    from workloads import random_block_lex
    k, nocc = 11, 7
    X = random_block_lex(12, system["n"], k)
    occ = np.linspace(2.0, 0.5, nocc)
    Xd = dev(to_slots(X, system["lex"]))
    rho = kscf.kscf_density(system["H"], Xd, nocc, occ=dev(occ)).cpu().numpy()
    ref = density(X, occ)
    assert np.max(np.abs(from_slots(rho, system["lex"], system["n"]) - ref)) <= 1e-13 * ref.max()
    rho2 = kscf.kscf_density(system["H"], Xd.float(), nocc).cpu().numpy()
    ref2 = density(X.astype(np.float32).astype(np.float64), np.full(nocc, 2.0))
    assert np.max(np.abs(from_slots(rho2, system["lex"], system["n"]) - ref2)) <= 1e-12 * ref2.max()


def test_random_subspace_matches_generator(kscf, system):
    from workloads import random_block_lex
    k = 9
    Xd = torch.full((system["g"].info["n_slots"], k + 2), 7.0, dtype=torch.float64, device="cuda")
    kscf.kscf_random_subspace(system["H"], Xd[:, :k], seed=77)
    got = Xd.cpu().numpy()
    ref = random_block_lex(77, system["n"], k)
    assert np.max(np.abs(from_slots(got[:, :k], system["lex"], system["n"]) - ref)) < 1e-13
    assert np.all(got[system["lex"] < 0, :k] == 0) and np.all(got[:, k:] == 7.0)


def test_chefsi_iterations_match_oracle(kscf, system):
    from oracle.chefsi import chefsi, spectral_upper_bound
    from workloads import random_block_lex
    k, m, iters = 12, 8, 3
    X0 = random_block_lex(1, system["n"], k)
    Xd = dev(to_slots(X0, system["lex"]))
    _, b = kscf.kscf_spectral_bounds(system["H"])
    kscf.kscf_orthonormalize(system["H"], Xd)
    lam = kscf.kscf_rayleigh_ritz(system["H"], Xd)
    for _ in range(iters):
        kscf.kscf_chebyshev_filter(system["H"], Xd, m, lam[-1], b, lam[0])
        kscf.kscf_orthonormalize(system["H"], Xd)
        lam = kscf.kscf_rayleigh_ritz(system["H"], Xd)
    ref = chefsi(system["OH"], X0, m, iters, b=spectral_upper_bound(system["OH"]))
    assert np.max(np.abs(lam - ref["lam"])) <= 1e-10 * np.max(np.abs(ref["lam"]))


def test_error_paths(kscf, system):
    H = system["H"]
    X = torch.zeros((system["g"].info["n_slots"], 4), dtype=torch.float64, device="cuda")
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_chebyshev_filter(H, X, 4, 2.0, 1.0, 0.0)           # a >= b
    assert e.value.code == kscf.KSCF_ERR_INVALID
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_chebyshev_filter(H, X, 4, 1.0, 2.0, 0.0, work=torch.empty(64, dtype=torch.uint8, device="cuda"))
    assert e.value.code == kscf.KSCF_ERR_WORKSPACE
    # duplicated columns: rank-deficient Gram -> not SPD, X unchanged
    from workloads import random_block_lex
    col = random_block_lex(2, system["n"], 1)
    Xd = dev(to_slots(np.concatenate([col, col, col * 2, col], 1), system["lex"]))
    before = Xd.clone()
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_orthonormalize(H, Xd)
    assert e.value.code == kscf.KSCF_ERR_NOT_SPD
    assert torch.equal(before, Xd)
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_orthonormalize(H, X, mode=kscf.KSCF_GEMM_TENSOR)    # tensor mode needs F32
    assert e.value.code == kscf.KSCF_ERR_UNSUPPORTED


def test_orthonormalize_tensor_mode(kscf, system):
    from workloads import random_block_lex
    k = 24
    X = random_block_lex(9, system["n"], k) + 0.5 * random_block_lex(10, system["n"], 1)
    Xd = dev(to_slots(X, system["lex"]), torch.float32)
    kscf.kscf_orthonormalize(system["H"], Xd, mode=kscf.KSCF_GEMM_TENSOR)
    got = from_slots(Xd.double().cpu().numpy(), system["lex"], system["n"])
    h3 = system["OH"].h3
    assert np.max(np.abs(h3 * got.T @ got - np.eye(k))) < 2e-6
    assert subspace_gap(got, X, h3) < 1e-5


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("log_cond", [0.5, 3.0])
def test_orthonormalize_f32_second_pass_paths(kscf, system, mode, log_cond):
    """The second FP32 pass rotates by I - E/2 when its Gram matrix I + E is within 1e-4 of I
    and by a factorised R^-1 otherwise.  Columns scaled over 10^log_cond: at 10^0.5 the first
    pass leaves |E| ~ 1e-6 (first-order path); at 10^3 it leaves |E| ~ kappa^2 u ~ 1e-2
    (factorised path).  Both must give h^3 X^T X = I to the FP32 level and the oracle's
    span."""
    from workloads import random_block_lex
    k = 40
    X = random_block_lex(21, system["n"], k) * np.logspace(0.0, -log_cond, k)[None, :]
    Xd = dev(to_slots(X, system["lex"]), torch.float32)
    kscf.kscf_orthonormalize(system["H"], Xd, mode=mode)
    got = from_slots(Xd.double().cpu().numpy(), system["lex"], system["n"])
    h3 = system["OH"].h3
    assert np.max(np.abs(h3 * got.T @ got - np.eye(k))) < 2e-6
    Xr = X.astype(np.float32).astype(np.float64)   # the span of the block as passed in
    assert subspace_gap(got, Xr, h3) < 1e-4


@pytest.mark.parametrize("mode", [0, 1])
def test_rayleigh_ritz_f32_modes(kscf, system, mode):
    from oracle.chefsi import cholesky_qr, rayleigh_ritz
    from workloads import random_block_lex
    k = 16
    X, _ = cholesky_qr(random_block_lex(4, system["n"], k), system["OH"].h3)
    X32 = X.astype(np.float32).astype(np.float64)
    Xd = dev(to_slots(X32, system["lex"]), torch.float32)
    lam = kscf.kscf_rayleigh_ritz(system["H"], Xd, mode=mode)
    ref_lam, _, _ = rayleigh_ritz(system["OH"], X32, system["OH"].h3)
    # FP32 H X and GEMM sums: ~1e-6 of the spectral scale
    assert np.max(np.abs(lam - ref_lam)) <= 2e-5 * np.max(np.abs(ref_lam))


@pytest.mark.parametrize("mode", [0, 1])
def test_chefsi_f32_tracks_oracle(kscf, system, mode):
    """Mixed path (FP32 filter, FP64 Cholesky + eigensolver) after 3 iterations from the
    same X0: Ritz values close to the FP64 oracle's, and the wanted subspace agrees."""
    from oracle.chefsi import chefsi, spectral_upper_bound
    from workloads import random_block_lex
    k, m, iters = 12, 8, 3
    X0 = random_block_lex(1, system["n"], k)
    Xd = dev(to_slots(X0, system["lex"]), torch.float32)
    _, b = kscf.kscf_spectral_bounds(system["H"])
    kscf.kscf_orthonormalize(system["H"], Xd, mode=mode)
    lam = kscf.kscf_rayleigh_ritz(system["H"], Xd, mode=mode)
    for _ in range(iters):
        kscf.kscf_chebyshev_filter(system["H"], Xd, m, lam[-1], b, lam[0])
        kscf.kscf_orthonormalize(system["H"], Xd, mode=mode)
        lam = kscf.kscf_rayleigh_ritz(system["H"], Xd, mode=mode)
    ref = chefsi(system["OH"], X0, m, iters, b=spectral_upper_bound(system["OH"]))
    assert np.max(np.abs(lam[:6] - ref["lam"][:6])) <= 1e-4 * np.max(np.abs(ref["lam"]))
    got = from_slots(Xd.double().cpu().numpy(), system["lex"], system["n"])
    assert subspace_gap(got[:, :4], ref["X"][:, :4], system["OH"].h3) < 1e-2


@pytest.mark.parametrize("k,ldpad,block", [(13, 16, 0), (19, 24, 0), (19, 24, 8), (32, 32, 16), (40, 64, 0),
                                           (70, 96, 64), (33, 64, 0), (13, 18, 0), (30, 34, 0)])
def test_f32_brick_kernel_paths(kscf, system, k, ldpad, block):
    """Padded row strides select the FP32 brick kernels (brick 8): the TMA kernel for
    strides that are multiples of 4, the cp.async kernel otherwise; compared with the
    oracle like the generic path."""
    if system["brick"] != 8:
        pytest.skip("the staged kernel is built for 8^3 bricks")
    from oracle.chefsi import chebyshev_filter, spectral_upper_bound
    from workloads import random_block_lex
    X = random_block_lex(31, system["n"], k).astype(np.float32).astype(np.float64)
    full = torch.zeros((system["g"].info["n_slots"], ldpad), dtype=torch.float32, device="cuda")
    full[:, :k] = dev(to_slots(X, system["lex"]), torch.float32)
    Y = full[:, :k]
    HYf = torch.full_like(full, 7.0)
    kscf.kscf_hamiltonian_apply(system["H"], Y, HYf[:, :k])
    got = from_slots(HYf[:, :k].double().cpu().numpy(), system["lex"], system["n"])
    ref = system["OH"].apply(X)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert torch.all(HYf[:, k:] == 7.0)
    b = spectral_upper_bound(system["OH"])
    kscf.kscf_chebyshev_filter(system["H"], Y, 10, -0.5, b, -9.0, block=block)
    got = from_slots(full[:, :k].double().cpu().numpy(), system["lex"], system["n"])
    ref = chebyshev_filter(system["OH"], X, 10, -0.5, b, -9.0)
    colmax = np.max(np.abs(ref), axis=0)
    assert np.all(np.max(np.abs(got - ref), axis=0) <= 1e-4 * colmax)


def test_bounded_barrier_times_out_and_context_survives(kscf, species):
    # one CTA of the FP64 Cholesky kernel leaves before the first grid barrier; the other's
    # wait (limit ~1 ms) must give up, report the timeout and leave the context usable
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_selftest_barrier_timeout()
    assert e.value.code == kscf.KSCF_ERR_TIMEOUT
    pos, z = small_cluster()
    g, H = kscf.build_cluster(pos, z, species, 8.0, 0.7)
    X = torch.zeros((g.info["n_slots"], 40), dtype=torch.float64, device="cuda")
    kscf.kscf_random_subspace(H, X, seed=8)
    kscf.kscf_orthonormalize(H, X)
    G = kscf.kscf_gram(X, X, scale=H.h3).cpu().numpy()
    assert np.max(np.abs(G - np.eye(40))) < 1e-12


@pytest.mark.parametrize("mode", [0, 1])
def test_orthonormalize_recovers_from_rank_deficiency(kscf, species, mode):
    # two columns equal up to a 1e-6 perturbation: in FP32 the Gram matrix is singular to
    # working precision, so plain Cholesky-QR fails; with KSCF_ORTHO_ALLOW_SHIFT the shifted
    # retry still returns an orthonormal basis of the span
    pos, z = small_cluster()
    g, H = kscf.build_cluster(pos, z, species, 8.0, 0.7)
    k = 48
    X = torch.zeros((g.info["n_slots"], 64), dtype=torch.float32, device="cuda")
    kscf.kscf_random_subspace(H, X[:, :k], seed=3)
    noise = torch.zeros_like(X[:, 0])
    kscf.kscf_random_subspace(H, noise[:, None], seed=4)
    X[:, 7] = X[:, 3] + 1e-6 * noise
    kscf.kscf_orthonormalize(H, X[:, :k], mode=mode, allow_shift=True)
    G = kscf.kscf_gram(X[:, :k], X[:, :k], scale=H.h3).cpu().numpy()
    assert np.max(np.abs(G - np.eye(k))) < 1e-4
    assert torch.all(torch.isfinite(X)).item()


def test_tensor_rayleigh_ritz_is_stable_on_ritz_vectors(kscf, species):
    # a second Rayleigh-Ritz on Ritz vectors must leave them (nearly) unchanged: the
    # eigenvector signs make Q ~ I and the rotation is applied as X + X (Q - I)
    pos, z = small_cluster()
    g, H = kscf.build_cluster(pos, z, species, 8.0, 0.7)
    k = 64
    X = torch.zeros((g.info["n_slots"], k), dtype=torch.float32, device="cuda")
    kscf.kscf_random_subspace(H, X, seed=5)
    lo, hi = kscf.kscf_spectral_bounds(H)
    kscf.kscf_orthonormalize(H, X, mode=kscf.KSCF_GEMM_TENSOR)
    lam = kscf.kscf_rayleigh_ritz(H, X, mode=kscf.KSCF_GEMM_TENSOR)
    for _ in range(6):
        kscf.kscf_chebyshev_filter(H, X, 10, lam[-1], hi, lam[0])
        kscf.kscf_orthonormalize(H, X, mode=kscf.KSCF_GEMM_TENSOR)
        lam = kscf.kscf_rayleigh_ritz(H, X, mode=kscf.KSCF_GEMM_TENSOR)
    X1 = X.clone()
    lam2 = kscf.kscf_rayleigh_ritz(H, X, mode=kscf.KSCF_GEMM_TENSOR)
    assert np.max(np.abs(lam2 - lam)) < 1e-6 * np.max(np.abs(lam))
    # columns with well separated Ritz values keep their direction and sign
    sep = np.ones(k, dtype=bool)
    gaps = np.diff(lam2)
    sep[1:] &= gaps > 1e-3
    sep[:-1] &= gaps > 1e-3
    d = torch.max(torch.abs(X - X1), dim=0).values.cpu().numpy()
    scale = torch.max(torch.abs(X1)).item()
    assert np.max(d[sep]) < 1e-4 * scale, np.max(d[sep]) / scale


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_nonfinite_inputs_are_reported(kscf, system, dtype):
    """A NaN put into X (or into the potential) on the host: the filter and the apply
    flag it on the device and kscf_check_status returns KSCF_ERR_NONFINITE, the Cholesky-QR
    returns it directly, and the context stays usable (a clean filter afterwards)."""
    from workloads import random_block_lex
    H, lex = system["H"], system["lex"]
    if dtype == torch.float64 or system["brick"] != 8:
        pytest.skip("the device-side flag covers the FP32 brick filter; the other paths are checked below")
    k = 12
    X0 = to_slots(random_block_lex(8, system["n"], k), lex)
    live = np.nonzero(lex >= 0)[0]
    _, b = kscf.kscf_spectral_bounds(H)
    assert kscf.lib.kscf_check_status() == kscf.KSCF_OK
    # NaN in X: filter
    Xn = X0.copy()
    Xn[live[len(live) // 2], 3] = np.nan
    Xd = dev(Xn, dtype)
    kscf.kscf_chebyshev_filter(H, Xd, 5, -0.5, b, -9.0)
    torch.cuda.synchronize()
    assert kscf.lib.kscf_check_status() == kscf.KSCF_ERR_NONFINITE
    assert kscf.lib.kscf_check_status() == kscf.KSCF_OK          # the flag is cleared once reported
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_orthonormalize(H, Xd)
    assert e.value.code == kscf.KSCF_ERR_NONFINITE
    # NaN in Y: apply
    Yd = dev(Xn, dtype)
    kscf.kscf_hamiltonian_apply(H, Yd, torch.empty_like(Yd))
    torch.cuda.synchronize()
    assert kscf.lib.kscf_check_status() == kscf.KSCF_ERR_NONFINITE
    # NaN in the potential: filter of a clean block
    V = kscf.kscf_get_potential(H)
    Vn = V.clone()
    Vn[int(live[7])] = float("inf")
    kscf.kscf_set_potential(H, Vn)
    try:
        Xd = dev(X0, dtype)
        kscf.kscf_chebyshev_filter(H, Xd, 5, -0.5, b, -9.0)
        torch.cuda.synchronize()
        assert kscf.lib.kscf_check_status() == kscf.KSCF_ERR_NONFINITE
    finally:
        kscf.kscf_set_potential(H, V)
    # clean again: no flag, finite result
    Xd = dev(X0, dtype)
    kscf.kscf_chebyshev_filter(H, Xd, 5, -0.5, b, -9.0)
    torch.cuda.synchronize()
    assert kscf.lib.kscf_check_status() == kscf.KSCF_OK
    assert torch.isfinite(Xd).all()


def test_nonfinite_f64_orthonormalize_and_apply(kscf, system):
    """FP64: the apply's output check and the Cholesky-QR Gram check report a NaN too."""
    from workloads import random_block_lex
    H, lex = system["H"], system["lex"]
    X = to_slots(random_block_lex(9, system["n"], 6), lex)
    X[np.nonzero(lex >= 0)[0][3], 2] = np.nan
    Xd = dev(X)
    kscf.kscf_hamiltonian_apply(H, Xd, torch.empty_like(Xd))
    torch.cuda.synchronize()
    assert kscf.lib.kscf_check_status() == kscf.KSCF_ERR_NONFINITE
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_orthonormalize(H, Xd)
    assert e.value.code == kscf.KSCF_ERR_NONFINITE
    assert kscf.lib.kscf_check_status() == kscf.KSCF_OK


def test_filter_dense_cluster_matches_oracle(kscf, species):
    """64 overlapping Si atoms in a small sphere: bricks reached by more KB atoms than the
    per-brick table holds (32), so the FP32 filter's nonlocal scatter reads its
    coefficients from global memory instead of the staged copy; against the oracle filter
    (1e-4 of the column maximum after 8 degree steps) and the FP64 filter (1e-11)."""
    from oracle.chefsi import chebyshev_filter, spectral_upper_bound
    from oracle.system import cluster_hamiltonian
    from workloads import random_block_lex
    rng = np.random.default_rng(9)
    pos = rng.uniform(-2.0, 2.0, (64, 3))
    pos[0] = 0.0
    z = np.full(64, 14, dtype=np.int32)
    R, h = 6.0, 0.7
    g, H = kscf.build_cluster(pos, z, species, R, h)
    OH = cluster_hamiltonian(pos, z, species, R, h)
    lex, _ = g.slots()
    n, k, m = g.info["n_points"], 37, 8
    X = random_block_lex(4, n, k).astype(np.float32).astype(np.float64)
    b = spectral_upper_bound(OH)
    a, a0 = b - 0.6 * (b - OH.V.min()), OH.V.min() - 5.0
    ref = chebyshev_filter(OH, X, m, a, b, a0)
    colmax = np.max(np.abs(ref), axis=0)
    for dtype, tol in ((torch.float32, 1e-4), (torch.float64, 1e-11)):
        Xd = dev(to_slots(X, lex), dtype)
        kscf.kscf_chebyshev_filter(H, Xd, m, a, b, a0)
        assert kscf.lib.kscf_check_status() == kscf.KSCF_OK
        got = from_slots(Xd.double().cpu().numpy(), lex, n)
        assert np.all(np.max(np.abs(got - ref), axis=0) <= tol * colmax), dtype
