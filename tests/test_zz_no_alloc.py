"""The allocation-free H*Y entry point (kscf_hamiltonian_apply_noalloc).

It serves callers that cannot allocate device memory (a framework that owns all of
it, or a loop that must not synchronise through cudaMalloc): the projection scratch
lives in a fixed array inside the library.  Checked here through the C ABI against the
work-buffer entry point, on two calls in a row (the array keeps the previous call's
contents, which must not leak into the next result), plus the size limit.  This file is
collected last so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from helpers import small_cluster, to_slots

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def setup(species):
    from paper_2303_00790_gb300.build import build
    build()
    from paper_2303_00790_gb300 import kscf
    pos, z = small_cluster()
    g, H = kscf.build_cluster(pos, z, species, 9.0, 0.7)
    lex, _ = g.slots()
    return kscf, g, H, lex


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-5)])
def test_noalloc_matches_apply_twice(setup, dtype, tol):
    from workloads import random_block_lex
    kscf, g, H, lex = setup
    n = g.info["n_points"]
    for call, (seed, k) in enumerate([(21, 16), (22, 9)]):
        Y = torch.tensor(to_slots(random_block_lex(seed, n, k), lex), dtype=dtype, device="cuda")
        ref = torch.empty_like(Y)
        kscf.kscf_hamiltonian_apply(H, Y, ref)
        out = torch.full_like(Y, 3.0)
        kscf.kscf_hamiltonian_apply_noalloc(H, Y, out)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        scale = ref.abs().max().item()
        assert err <= tol * scale, f"call {call}: {err} vs {scale}"


def test_noalloc_rejects_too_many_vectors(setup):
    kscf, g, H, lex = setup
    k = 4 << 20      # far beyond the fixed array for any non-empty projector set
    Y = torch.zeros((g.info["n_slots"], 1), dtype=torch.float64, device="cuda")
    rc = kscf.lib.kscf_hamiltonian_apply_noalloc(H.handle, kscf.C.c_void_p(Y.data_ptr()), k,
                                                 kscf.C.c_void_p(Y.data_ptr()), k, k, kscf.KSCF_F64, None)
    assert rc == kscf.KSCF_ERR_INVALID
    assert "fixed" in kscf.lib.kscf_last_error().decode()
