// H Y without any device allocation by the caller or the library.
//
// kscf_hamiltonian_apply needs a caller-provided work buffer for the projection
// coefficients of the nonlocal term.  Some callers cannot obtain one: a host program
// whose framework has already reserved all device memory in its own pool and
// forbids other allocators, or code that must not call cudaMalloc because it
// implicitly synchronises the device in a latency-critical loop.  This entry point
// keeps that scratch in a fixed array compiled into the library instead.
//
// The array is a file-scope __device__ variable of KSCF_NOALLOC_SCRATCH_BYTES bytes; every
// GPU that loads this library holds it until the process exits.  Host code may not
// use the array's name as a device address (on the host it is only a stand-in), so
// the device address is looked up with cudaGetSymbolAddress, with the device current,
// on every call.
#include <cuda_runtime.h>

#include "kscf_internal.h"

static __device__ __align__(256) unsigned char g_apply_scratch[KSCF_NOALLOC_SCRATCH_BYTES];

namespace {
// Device address of g_apply_scratch in the current context, looked up on every call
// (the lookup allocates nothing, and a cached address would dangle after the context is
// reset by cudaDeviceReset or by a host framework).
int scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
  if (e != cudaSuccess || !p) {
    kscf::set_error("kscf_hamiltonian_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  *out = p;
  return KSCF_OK;
}
}  // namespace

extern "C" int kscf_hamiltonian_apply_noalloc(const kscf_ham* ham, void* Y, int64_t ld_y, void* HY, int64_t ld_hy,
                                              int k, int dtype, void* stream) {
  if (!ham || !Y || !HY) {
    kscf::set_error("kscf_hamiltonian_apply_noalloc: null argument");
    return KSCF_ERR_INVALID;
  }
  if (dtype != KSCF_F64 && dtype != KSCF_F32) {
    kscf::set_error("kscf_hamiltonian_apply_noalloc: dtype must be KSCF_F64 or KSCF_F32");
    return KSCF_ERR_INVALID;
  }
  if (k < 1 || ld_y < k || ld_hy < k) {
    kscf::set_error("kscf_hamiltonian_apply_noalloc: need k >= 1, ld_y >= k and ld_hy >= k");
    return KSCF_ERR_INVALID;
  }
  const kscf::Ham& H = ham->h;
  const size_t need = (size_t)H.n_kb * 4 * (size_t)kscf::coef_ld(k) * (dtype == KSCF_F64 ? 8 : 4);
  if (need > (size_t)KSCF_NOALLOC_SCRATCH_BYTES) {
    kscf::set_error(
        "kscf_hamiltonian_apply_noalloc: %d vectors need %zu bytes of projection scratch, above the fixed "
        "%d-byte array; call it on fewer columns at a time (at most %zu here)",
        k, need, KSCF_NOALLOC_SCRATCH_BYTES,
        (size_t)KSCF_NOALLOC_SCRATCH_BYTES / ((size_t)(H.n_kb > 0 ? H.n_kb : 1) * 4 * (dtype == KSCF_F64 ? 8 : 4)) / 32 * 32);
    return KSCF_ERR_INVALID;
  }
  void* coef = nullptr;
  int rc = scratch_address(&coef);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // The gather writes the coefficients of vectors v < k.  The brick kernels read whole
  // vector chunks, so lanes v >= k may read values a previous call left in the array;
  // those lanes are never stored (every output write is masked to v < k), which is why
  // the array needs no clearing between calls.
  KSCF_CUDA_TRY(kscf::launch_zero_rows(H, Y, ld_y, k, dtype, st));
  KSCF_CUDA_TRY(kscf::launch_zero_rows(H, HY, ld_hy, k, dtype, st));
  KSCF_CUDA_TRY(kscf::launch_kb_gather(H, Y, ld_y, k, dtype, coef, kscf::coef_ld(k), st));
  KSCF_CUDA_TRY(kscf::launch_cheb_step(H, Y, ld_y, nullptr, 0, HY, ld_hy, k, (int)(ld_y < ld_hy ? ld_y : ld_hy), dtype,
                                       1.0, 0.0, 0.0, coef, kscf::coef_ld(k), st));
  return KSCF_OK;
}
