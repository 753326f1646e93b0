"""The allocation-free H*Y entry point (kscf_hamiltonian_apply_noalloc).

It serves callers that cannot allocate device memory (a framework that owns all of
it, or a loop that must not synchronise through cudaMalloc): the projection scratch
lives in a fixed array inside the library.  Checked here through the C ABI against the
FP64 oracle's H*Y and against the work-buffer entry point, on two calls in a row (the
array keeps the previous call's contents, which must not leak into the next result);
that a call leaves the device's free memory unchanged; and the size limit.  This file
is collected last so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from helpers import from_slots, small_cluster, to_slots

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def setup(species):
    from paper_2303_00790_gb300.build import build
    build()
    from paper_2303_00790_gb300 import kscf
    from oracle.system import cluster_hamiltonian
    pos, z = small_cluster()
    g, H = kscf.build_cluster(pos, z, species, 9.0, 0.7)
    lex, _ = g.slots()
    OH = cluster_hamiltonian(pos, z, species, 9.0, 0.7)
    assert OH.n == g.info["n_points"]
    return kscf, g, H, lex, OH


# FP64: ~45-term sums of magnitude <= 50 |y| in both orders -> 1e-13 of max|Hy|;
# FP32 inputs and arithmetic -> 1e-5 of max|Hy| (the apply tolerances of the parity tests)
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-5)])
def test_noalloc_matches_oracle_twice(setup, dtype, tol):
    from workloads import random_block_lex
    kscf, g, H, lex, OH = setup
    n = g.info["n_points"]
    for call, (seed, k) in enumerate([(21, 16), (22, 9)]):
        Yl = random_block_lex(seed, n, k)
        if dtype == torch.float32:
            Yl = Yl.astype(np.float32).astype(np.float64)
        Y = torch.tensor(to_slots(Yl, lex), dtype=dtype, device="cuda")
        out = torch.full_like(Y, 3.0)
        kscf.kscf_hamiltonian_apply_noalloc(H, Y, out)
        ref = torch.empty_like(Y)
        kscf.kscf_hamiltonian_apply(H, Y, ref)
        torch.cuda.synchronize()
        exact = OH.apply(Yl)
        got = from_slots(out.cpu().double().numpy(), lex, n)
        scale = np.abs(exact).max()
        assert np.abs(got - exact).max() <= tol * scale, f"call {call} vs oracle"
        assert (out - ref).abs().max().item() <= tol * scale, f"call {call} vs kscf_hamiltonian_apply"
        assert np.all(out.cpu().numpy()[lex < 0] == 0), "padding rows of H*Y must be zero"


def test_noalloc_allocates_no_device_memory(setup):
    from workloads import random_block_lex
    kscf, g, H, lex, _ = setup
    Y = torch.tensor(to_slots(random_block_lex(5, g.info["n_points"], 32), lex), device="cuda")
    out = torch.empty_like(Y)
    kscf.kscf_hamiltonian_apply_noalloc(H, Y, out)      # first call: module loading, symbol lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        kscf.kscf_hamiltonian_apply_noalloc(H, Y, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_too_many_vectors(setup, species):
    """k one vector chunk beyond the array's limit is rejected before any launch; the
    buffers really have k columns, so a missed check could not read out of bounds."""
    kscf = setup[0]
    # 64 atoms with projectors (overlapping Si atoms in a small sphere) make the limit small
    rng = np.random.default_rng(9)
    pos = rng.uniform(-2.0, 2.0, (64, 3))
    pos[0] = 0.0
    z = np.full(64, 14, dtype=np.int32)
    g, H = kscf.build_cluster(pos, z, species, 5.0, 0.7)
    n_kb = 64
    assert all(int(s["n_proj"]) > 0 for s in species if int(s["z_number"]) == 14)
    limit = kscf.KSCF_NOALLOC_SCRATCH_BYTES // (n_kb * 4 * 8) // 32 * 32
    k = limit + 32
    Y = torch.zeros((g.info["n_slots"], k), dtype=torch.float64, device="cuda")
    HY = torch.zeros_like(Y)
    rc = kscf.lib.kscf_hamiltonian_apply_noalloc(H.handle, kscf.C.c_void_p(Y.data_ptr()), k,
                                                 kscf.C.c_void_p(HY.data_ptr()), k, k, kscf.KSCF_F64, None)
    assert rc == kscf.KSCF_ERR_INVALID
    msg = kscf.lib.kscf_last_error().decode()
    assert "fixed" in msg and str(limit) in msg, msg
    # at the limit it runs
    kscf.kscf_hamiltonian_apply_noalloc(H, Y[:, :limit], HY[:, :limit])
    torch.cuda.synchronize()
