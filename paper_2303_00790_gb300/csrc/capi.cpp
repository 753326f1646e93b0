// C ABI drivers of the CheFSI hot path: Hamiltonian apply, Chebyshev filter,
// Cholesky-QR, Rayleigh-Ritz, density and the initial subspace (arXiv 2303.00790,
// CheFSI paragraph).  The FP64 Cholesky factor and its inverse come from chol.cu, the
// k x k FP64 symmetric eigensolver from eig.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kscf_internal.h"

using namespace kscf;

namespace kscf {
// rowmap (device, may be null): row r of the operands (and of out) is row rowmap[r]
cudaError_t launch_gram_tc(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t rows, int m, int n,
                           double scale, double* C, int64_t ldc, bool accumulate, void* work, size_t work_bytes,
                           cudaStream_t st, bool symmetric_result = false, const int32_t* rowmap = nullptr);
cudaError_t launch_rotate_tc(const float* A, int64_t lda, const double* Q, int64_t ldq, int64_t rows, int kin,
                             int kout, bool add_identity_input, float* out, int64_t ldo, void* work,
                             size_t work_bytes, cudaStream_t st, const int32_t* rowmap = nullptr);
size_t gram_tc_work_bytes(int64_t rows, int m, int n);
size_t rotate_tc_work_bytes(int64_t rows, int kin, int kout);
bool tc_available();
cudaError_t tc_status(bool reset, unsigned int* status);
cudaError_t filter_status(bool reset, unsigned int* status);
}  // namespace kscf

namespace {

size_t esize(int dtype) { return dtype == KSCF_F64 ? 8 : 4; }

// status words of launch_sym_eig, read back after a synchronisation
int eig_info_code(const int* info, const char* who) {
  if (info[2]) {
    set_error("%s: the matrix to diagonalise holds a NaN or Inf", who);
    return KSCF_ERR_NONFINITE;
  }
  if (info[0]) {
    set_error("%s: a bounded grid barrier of the tridiagonalisation gave up", who);
    return KSCF_ERR_TIMEOUT;
  }
  if (info[1]) {
    set_error("%s: %d secular-equation roots did not converge", who, info[1]);
    return KSCF_ERR_NO_CONVERGE;
  }
  return KSCF_OK;
}

// after a synchronisation: did a tensor-core pipeline wait time out?
int check_tc(int mode, const char* who) {
  if (mode != KSCF_GEMM_TENSOR) return KSCF_OK;
  unsigned int st = 0;
  cudaError_t e = tc_status(true, &st);
  if (e != cudaSuccess) {
    set_error("%s: reading the tensor-core status failed: %s", who, cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  if (st) {
    set_error("%s: a tensor-core pipeline wait timed out (status %u)", who, st);
    return KSCF_ERR_TIMEOUT;
  }
  return KSCF_OK;
}

int check_common(const kscf_ham* ham, const void* X, int64_t ld, int k, int dtype, const char* who) {
  if (!ham || !X) {
    set_error("%s: null argument", who);
    return KSCF_ERR_INVALID;
  }
  if (dtype != KSCF_F64 && dtype != KSCF_F32) {
    set_error("%s: dtype must be KSCF_F64 or KSCF_F32", who);
    return KSCF_ERR_INVALID;
  }
  if (k < 1 || ld < k) {
    set_error("%s: need k >= 1 and ld >= k (k=%d, ld=%lld)", who, k, (long long)ld);
    return KSCF_ERR_INVALID;
  }
  return KSCF_OK;
}

int block_width(int k, int block) { return (block <= 0 || block > k) ? k : block; }

// Carves aligned pieces out of the caller's work buffer.
struct Carver {
  char* base;
  size_t used = 0;
  explicit Carver(void* b) : base((char*)b) {}
  void* take(size_t bytes) {
    void* p = base ? base + used : nullptr;
    used += kscf_align256(bytes);
    return p;
  }
};

// rows per panel of the in-place rotation (panel buffer = rows x k)
int64_t panel_rows(int64_t n_slots, int k, int dtype) {
  const size_t target = (size_t)256 << 20;
  int64_t r = (int64_t)(target / ((size_t)k * esize(dtype)));
  r = std::max<int64_t>(r, 512);
  r = (r / 512) * 512;
  return std::min<int64_t>(r, n_slots);
}

struct OrthoPlan {
  size_t S, Rinv, info, chol, panel, tc;
  int64_t prows;
};

int ortho_plan(const Ham& H, int k, int dtype, int mode, OrthoPlan* p) {
  p->S = (size_t)k * k * 8;
  p->Rinv = (size_t)k * k * esize(dtype);
  p->info = 256;
  p->chol = chol_inv_work_bytes(k);
  p->prows = panel_rows(H.grid.n_slots, k, dtype);
  p->panel = mode == KSCF_GEMM_TENSOR ? 0 : (size_t)p->prows * k * esize(dtype);
  p->tc = 0;
  if (mode == KSCF_GEMM_TENSOR)
    p->tc = std::max(gram_tc_work_bytes(H.grid.n_slots, k, k), rotate_tc_work_bytes(p->prows, k, k));
  return KSCF_OK;
}

size_t ortho_bytes(const OrthoPlan& p) {
  return kscf_align256(p.S) + kscf_align256(p.Rinv) + kscf_align256(p.info) + kscf_align256(p.chol) +
         kscf_align256(p.panel) + kscf_align256(p.tc);
}

struct RRPlan {
  size_t hxb, coef, Hs, W, Q, info, lwork_bytes, panel, tc;
  int64_t prows;
  int w;
};

int rr_plan(const Ham& H, int k, int dtype, int mode, int block, RRPlan* p) {
  if (k > KSCF_EIG_MAX_N) {
    set_error("kscf_rayleigh_ritz: k = %d above the eigensolver's limit %d", k, KSCF_EIG_MAX_N);
    return KSCF_ERR_INVALID;
  }
  p->w = block_width(k, block);
  p->hxb = (size_t)H.grid.n_slots * coef_ld(p->w) * esize(dtype);
  p->coef = (size_t)std::max(H.n_kb, 1) * 4 * coef_ld(p->w) * esize(dtype);
  p->Hs = (size_t)k * k * 8;
  p->W = (size_t)k * 8;
  p->Q = (size_t)k * k * esize(dtype);
  p->info = 256;
  p->lwork_bytes = sym_eig_work_bytes(k);
  p->prows = panel_rows(H.grid.n_slots, k, dtype);
  p->panel = mode == KSCF_GEMM_TENSOR ? 0 : (size_t)p->prows * k * esize(dtype);
  p->tc = 0;
  if (mode == KSCF_GEMM_TENSOR)
    p->tc = std::max(gram_tc_work_bytes(H.grid.n_slots, k, p->w), rotate_tc_work_bytes(p->prows, k, k));
  return KSCF_OK;
}

size_t rr_bytes(const RRPlan& p) {
  return kscf_align256(p.hxb) + kscf_align256(p.coef) + kscf_align256(p.Hs) + kscf_align256(p.W) +
         kscf_align256(p.Q) + kscf_align256(p.info) + kscf_align256(p.lwork_bytes) + kscf_align256(p.panel) +
         kscf_align256(p.tc);
}

// FP32 on 8^3 bricks: the filter runs on two chunk-major working copies of the block
bool filter_chunk_major(const Ham& H, int dtype) { return dtype == KSCF_F32 && H.n_cells > 0; }

// The chunk-major filter runs each column block as two halves of whole 16-column chunks
// (the first with the odd chunk), one per stream: columns are filtered independently, so
// one half's projection gathers overlap the other half's degree steps.
int cm_first_half_cols(int wb) { return std::min(wb, ((wb + 15) / 16 + 1) / 2 * 16); }

size_t filter_bytes(const Ham& H, int k, int dtype, int block) {
  const int w = block_width(k, block);
  const size_t coef = kscf_align256((size_t)std::max(H.n_kb, 1) * 4 * coef_ld(w) * esize(dtype));
  if (filter_chunk_major(H, dtype)) {
    const size_t wpad = (size_t)(w + 15) / 16 * 16;   // covers chunk widths 8 and 16
    const int w0 = cm_first_half_cols(w), w1 = std::max(1, w - w0);
    const size_t coefs = kscf_align256((size_t)std::max(H.n_kb, 1) * 4 * coef_ld(w0) * 4) +
                         kscf_align256((size_t)std::max(H.n_kb, 1) * 4 * coef_ld(w1) * 4);
    return 2 * kscf_align256((size_t)H.grid.n_slots * wpad * 4) + coefs + kscf_align256(KSCF_CM_ZERO_BYTES);
  }
  return kscf_align256((size_t)H.grid.n_slots * coef_ld(w) * esize(dtype)) + coef;
}

size_t apply_bytes(const Ham& H, int k, int dtype) {
  return kscf_align256((size_t)std::max(H.n_kb, 1) * 4 * coef_ld(k) * esize(dtype));
}

int check_work(void* work, size_t have, size_t need, const char* who) {
  if (have < need || (need > 0 && !work)) {
    set_error("%s: work buffer of %zu bytes, need %zu", who, have, need);
    return KSCF_ERR_WORKSPACE;
  }
  if (((uintptr_t)work & 255) != 0) {
    set_error("%s: work buffer must be 256-byte aligned", who);
    return KSCF_ERR_INVALID;
  }
  return KSCF_OK;
}

int check_mode(int dtype, int mode, const char* who) {
  if (mode != KSCF_GEMM_NATIVE && mode != KSCF_GEMM_TENSOR) {
    set_error("%s: unknown GEMM mode %d", who, mode);
    return KSCF_ERR_INVALID;
  }
  if (mode == KSCF_GEMM_TENSOR && dtype != KSCF_F32) {
    set_error("%s: tensor-core mode needs F32 X", who);
    return KSCF_ERR_UNSUPPORTED;
  }
  return KSCF_OK;
}

// X <- X Qm (Qm column-major k x k in the dtype of X for the native path, FP64 for the
// tensor path) in row panels.  The tensor path writes each panel in place (its product
// reads the panel's bf16 pieces, made before the launch); the native path goes through
// the panel buffer.
int rotate_inplace(const Ham& H, void* X, int64_t ld, int k, int dtype, int mode, const void* Qm,
                   const double* Q64, bool near_identity, void* panel, int64_t prows, void* tcwork, size_t tcbytes,
                   cudaStream_t st) {
  const size_t es = esize(dtype);
  // the tensor path rotates the domain rows only (through the grid's list of domain slots)
  const bool live = mode == KSCF_GEMM_TENSOR && H.d_live;
  const int64_t rows = live ? H.n_live : H.grid.n_slots;
  for (int64_t r0 = 0; r0 < rows; r0 += prows) {
    const int64_t nr = std::min(prows, rows - r0);
    char* Xr = (char*)X + (size_t)r0 * ld * es;
    if (mode == KSCF_GEMM_TENSOR) {
      if (live)
        KSCF_CUDA_TRY(launch_rotate_tc((const float*)X, ld, Q64, k, nr, k, k, near_identity, (float*)X, ld, tcwork,
                                       tcbytes, st, H.d_live + r0));
      else
        KSCF_CUDA_TRY(launch_rotate_tc((const float*)Xr, ld, Q64, k, nr, k, k, near_identity, (float*)Xr, ld, tcwork,
                                       tcbytes, st));
    } else {
      KSCF_CUDA_TRY(launch_rotate_native(Xr, ld, Qm, k, nr, k, k, dtype, panel, k, st));
      KSCF_CUDA_TRY(launch_copy_cols(panel, k, Xr, ld, nr, k, dtype, st));
    }
  }
  return KSCF_OK;
}

// symmetric_result: A^T B is known to be symmetric (m == n), so the tensor path computes
// the upper-triangle tiles only and mirrors them.
int gram(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t rows, int m, int n, int dtype, int mode,
         double scale, double* C, int64_t ldc, void* tcwork, size_t tcbytes, cudaStream_t st,
         bool symmetric_result = false, const int32_t* rowmap = nullptr) {
  if (mode == KSCF_GEMM_TENSOR) {
    KSCF_CUDA_TRY(launch_gram_tc((const float*)A, lda, (const float*)B, ldb, rows, m, n, scale, C, ldc, false,
                                 tcwork, tcbytes, st, symmetric_result && m == n, rowmap));
  } else {
    KSCF_CUDA_TRY(launch_gram_native(A, lda, B, ldb, rows, m, n, dtype, scale, C, ldc, false, st));
  }
  return KSCF_OK;
}

// Second FP32 pass: when the Gram matrix S = I + E is within this of I (max norm), X is
// rotated by the first-order inverse square root W = I - E/2 instead of R^-1 from a
// Cholesky factorisation: h^3 (XW)^T (XW) = I + O(E^2), and E^2 <= 1e-8 is below the FP32
// rotation's own rounding (~3e-7), so the result is as orthonormal as after the factorised
// pass, with the same span
constexpr double kFp32PolarTol = 1e-4;

// One Cholesky-QR pass: S = h^3 X^T X, S = R^T R, X <- X R^-1 (the factor and its inverse
// from one FP64 kernel, chol.cu).  When the factorisation fails and `shifted` is non-null,
// the Gram matrix is recomputed and its diagonal shifted by 16 k u max_i S_ii (u the unit
// roundoff of X's type) before a second attempt (shifted Cholesky-QR, Fukaya, Kannan,
// Nakatsukasa, Yamamoto & Yanagisawa 2020); *shifted then reports that X is not yet
// orthonormal and needs further passes.  With `shifted` non-null the first attempt also
// fails on a pivot at the Gram matrix's own rounding level (8 u S_cc), where the plain
// factor would amplify rounding noise into the basis.
int cholqr_pass(const Ham& H, void* X, int64_t ld, int k, int dtype, int mode, const OrthoPlan& p, Carver& cv,
                bool second_pass, cudaStream_t st, bool* shifted = nullptr, double polar_tol = 0.0) {
  Carver c = cv;
  double* S = (double*)c.take(p.S);
  void* Rinv = c.take(p.Rinv);
  int* status = (int*)c.take(p.info);
  void* cwork = c.take(p.chol);
  void* panel = c.take(p.panel);
  void* tcw = c.take(p.tc);
  const double h3 = H.grid.h * H.grid.h * H.grid.h;
  // the tensor path sums over the domain rows only (the padding rows are zero)
  const int32_t* live = mode == KSCF_GEMM_TENSOR ? H.d_live : nullptr;
  const int64_t rows = live ? H.n_live : H.grid.n_slots;
  const double u = dtype == KSCF_F64 ? 0x1.0p-53 : 0x1.0p-24;
  int hst[3] = {0, 0, 0};
  auto factor = [&](double floor_rel) -> int {
    // status[2]: a NaN or Inf on the Gram diagonal (X itself is not finite)
    KSCF_CUDA_TRY(launch_diag_finite(S, k, k, status + 2, st));
    KSCF_CUDA_TRY(launch_chol_inv(S, k, k, floor_rel, S, k, cwork, status, st));
    KSCF_CUDA_TRY(cudaMemcpyAsync(hst, status, sizeof(hst), cudaMemcpyDeviceToHost, st));
    KSCF_CUDA_TRY(cudaStreamSynchronize(st));
    int r = check_tc(mode, "Cholesky-QR");
    if (r) return r;
    if (hst[1] != 0) {
      set_error("Cholesky-QR: a grid barrier of the factorisation kernel timed out");
      return KSCF_ERR_TIMEOUT;
    }
    if (hst[2] != 0) {
      set_error("Cholesky-QR: the Gram matrix has a NaN or Inf on its diagonal (X is not finite)");
      return KSCF_ERR_NONFINITE;
    }
    return KSCF_OK;
  };
  int rc = gram(X, ld, X, ld, rows, k, k, dtype, mode, h3, S, k, tcw, p.tc, st, false, live);
  if (rc) return rc;
  if (polar_tol > 0.0) {
    // S = I + E with |E| <= polar_tol: X <- X (I - E/2), no factorisation
    unsigned long long* dv = (unsigned long long*)(status + 16);   // inside the status block
    KSCF_CUDA_TRY(launch_dev_identity(S, k, k, dv, st));
    unsigned long long bits = 0;
    KSCF_CUDA_TRY(cudaMemcpyAsync(&bits, dv, sizeof(bits), cudaMemcpyDeviceToHost, st));
    KSCF_CUDA_TRY(cudaStreamSynchronize(st));
    rc = check_tc(mode, "Cholesky-QR");
    if (rc) return rc;
    double dev;
    std::memcpy(&dev, &bits, sizeof(dev));
    if (dev <= polar_tol) {
      KSCF_CUDA_TRY(launch_polar_first_order(S, k, k, st));
      if (mode != KSCF_GEMM_TENSOR) KSCF_CUDA_TRY(launch_f64_to_dtype(S, (int64_t)k * k, dtype, Rinv, st));
      rc = rotate_inplace(H, X, ld, k, dtype, mode, Rinv, S, true, panel, p.prows, tcw, p.tc, st);
      if (rc) return rc;
      KSCF_CUDA_TRY(cudaStreamSynchronize(st));
      return check_tc(mode, "Cholesky-QR");
    }
  }
  rc = factor(shifted ? 8.0 * u : 0.0);
  if (rc) return rc;
  if (hst[0] > 0 && shifted) {
    rc = gram(X, ld, X, ld, rows, k, k, dtype, mode, h3, S, k, tcw, p.tc, st, false, live);
    if (rc) return rc;
    KSCF_CUDA_TRY(launch_shift_diag(S, k, 16.0 * k * u, st));
    rc = factor(0.0);
    if (rc) return rc;
    if (hst[0] == 0) *shifted = true;
  }
  if (hst[0] != 0) {
    set_error("Cholesky-QR: Gram matrix not positive definite (pivot %d%s)", hst[0],
              second_pass ? ", second pass" : (shifted ? ", also with the diagonal shift" : ""));
    return KSCF_ERR_NOT_SPD;
  }
  // S now holds R^-1 (upper triangular, zero below); the native path takes it in X's type
  if (mode != KSCF_GEMM_TENSOR) KSCF_CUDA_TRY(launch_upper_to_dtype(S, k, dtype, Rinv, st));
  rc = rotate_inplace(H, X, ld, k, dtype, mode, Rinv, S, second_pass, panel, p.prows, tcw, p.tc, st);
  if (rc) return rc;
  KSCF_CUDA_TRY(cudaStreamSynchronize(st));
  return check_tc(mode, "Cholesky-QR");
}

}  // namespace

extern "C" int kscf_workspace_size(const kscf_ham* ham, int op, int k, int dtype, int mode, int block,
                                   size_t* bytes) {
  mode &= ~KSCF_ORTHO_ALLOW_SHIFT;
  if (!ham || !bytes || k < 1 || (dtype != KSCF_F64 && dtype != KSCF_F32)) {
    set_error("kscf_workspace_size: invalid argument");
    return KSCF_ERR_INVALID;
  }
  const Ham& H = ham->h;
  switch (op) {
    case KSCF_OP_APPLY:
      *bytes = apply_bytes(H, k, dtype);
      return KSCF_OK;
    case KSCF_OP_FILTER:
      *bytes = filter_bytes(H, k, dtype, block);
      return KSCF_OK;
    case KSCF_OP_ORTHO: {
      int rc = check_mode(dtype, mode, "kscf_workspace_size");
      if (rc) return rc;
      OrthoPlan p;
      rc = ortho_plan(H, k, dtype, mode, &p);
      if (rc) return rc;
      *bytes = ortho_bytes(p);
      return KSCF_OK;
    }
    case KSCF_OP_RR: {
      int rc = check_mode(dtype, mode, "kscf_workspace_size");
      if (rc) return rc;
      RRPlan p;
      rc = rr_plan(H, k, dtype, mode, block, &p);
      if (rc) return rc;
      *bytes = rr_bytes(p);
      return KSCF_OK;
    }
  }
  set_error("kscf_workspace_size: unknown op %d", op);
  return KSCF_ERR_INVALID;
}

extern "C" int kscf_hamiltonian_apply(const kscf_ham* ham, void* Y, int64_t ld_y, void* HY, int64_t ld_hy, int k,
                                      int dtype, void* work, size_t work_bytes, void* stream) {
  int rc = check_common(ham, Y, ld_y, k, dtype, "kscf_hamiltonian_apply");
  if (rc) return rc;
  if (!HY || ld_hy < k) {
    set_error("kscf_hamiltonian_apply: bad output");
    return KSCF_ERR_INVALID;
  }
  const Ham& H = ham->h;
  rc = check_work(work, work_bytes, apply_bytes(H, k, dtype), "kscf_hamiltonian_apply");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  KSCF_CUDA_TRY(launch_zero_rows(H, Y, ld_y, k, dtype, st));
  KSCF_CUDA_TRY(launch_zero_rows(H, HY, ld_hy, k, dtype, st));
  KSCF_CUDA_TRY(launch_kb_gather(H, Y, ld_y, k, dtype, work, coef_ld(k), st));
  KSCF_CUDA_TRY(launch_cheb_step(H, Y, ld_y, nullptr, 0, HY, ld_hy, k, (int)std::min<int64_t>(ld_y, ld_hy), dtype,
                                 1.0, 0.0, 0.0, work, coef_ld(k), st));
  // a NaN or Inf in Y or in the potential shows up in HY: flag it for kscf_check_status
  unsigned int* flag = nonfinite_flag();
  if (!flag) {
    set_error("kscf_hamiltonian_apply: status word lookup failed");
    return KSCF_ERR_CUDA;
  }
  KSCF_CUDA_TRY(launch_finite_rows(H, HY, ld_hy, k, dtype, flag, st));
  return KSCF_OK;
}

extern "C" int kscf_chebyshev_filter(const kscf_ham* ham, void* X, int64_t ld, int k, int degree, double a,
                                     double b, double a0, int dtype, int block, void* work, size_t work_bytes,
                                     void* stream) {
  int rc = check_common(ham, X, ld, k, dtype, "kscf_chebyshev_filter");
  if (rc) return rc;
  if (degree < 1 || !(a0 < a) || !(a < b) || !std::isfinite(a) || !std::isfinite(b) || !std::isfinite(a0)) {
    set_error("kscf_chebyshev_filter: need degree >= 1 and finite a0 < a < b");
    return KSCF_ERR_INVALID;
  }
  const Ham& H = ham->h;
  rc = check_work(work, work_bytes, filter_bytes(H, k, dtype, block), "kscf_chebyshev_filter");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int w = block_width(k, block);
  const size_t es = esize(dtype);
  Carver cv(work);
  const double e = (b - a) / 2.0, c = (b + a) / 2.0;
  const double sigma1 = e / (a0 - c), tau = 2.0 / sigma1;
  if (filter_chunk_major(H, dtype)) {
    // two chunk-major working copies A, B per half: A = Y_0 (converted block), B = Y_1, then
    // Y_j overwrites Y_{j-2}; the last step writes Y_m straight into the caller's block
    const int cw = cm_chunk_width();
    const size_t wpad16 = (size_t)(w + 15) / 16 * 16;
    float* A = (float*)cv.take((size_t)H.grid.n_slots * wpad16 * 4);
    float* B = (float*)cv.take((size_t)H.grid.n_slots * wpad16 * 4);
    const int w0max = cm_first_half_cols(w), w1max = std::max(1, w - w0max);
    float* coefh[2];
    coefh[0] = (float*)cv.take((size_t)std::max(H.n_kb, 1) * 4 * coef_ld(w0max) * 4);
    coefh[1] = (float*)cv.take((size_t)std::max(H.n_kb, 1) * 4 * coef_ld(w1max) * 4);
    float* zero = (float*)cv.take(KSCF_CM_ZERO_BYTES);
    KSCF_CUDA_TRY(cudaMemsetAsync(zero, 0, KSCF_CM_ZERO_BYTES, st));
    KSCF_CUDA_TRY(launch_zero_rows(H, X, ld, k, dtype, st));
    // the second half's stream and the fork/join events, released once enqueued (CUDA
    // frees them when their work is done)
    cudaStream_t st1 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    const bool split = w > cw;
    auto release = [&]() {
      if (ev_fork) cudaEventDestroy(ev_fork);
      if (ev_join) cudaEventDestroy(ev_join);
      if (st1) cudaStreamDestroy(st1);
    };
    if (split) {
      cudaError_t ce = cudaStreamCreateWithFlags(&st1, cudaStreamNonBlocking);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
      if (ce != cudaSuccess) {
        release();
        KSCF_CUDA_TRY(ce);
      }
    }
    auto run = [&](float* Xb, int wb, float* Ah, float* Bh, float* coef, cudaStream_t sh) -> cudaError_t {
      const int64_t cld = coef_ld(wb);
      cudaError_t e2 = launch_to_chunk_major(H, Xb, ld, wb, cw, Ah, Bh, sh);
      if (e2 == cudaSuccess) e2 = launch_kb_gather_cm(H, Ah, cw, wb, coef, cld, sh);
      // Y_1 = (sigma_1/e)(H X - c X)
      if (e2 == cudaSuccess)
        e2 = launch_cm_step(H, Ah, nullptr, degree == 1 ? Xb : Bh, degree == 1 ? ld : -1, wb, sigma1 / e, 0.0, c,
                            coef, cld, degree == 1, zero, sh);
      float* cur = Bh;
      float* prv = Ah;
      double sigma = sigma1;
      for (int j = 2; j <= degree && e2 == cudaSuccess; j++) {
        const double sigma_new = 1.0 / (tau - sigma);
        const bool last = j == degree;
        e2 = launch_kb_gather_cm(H, cur, cw, wb, coef, cld, sh);
        // Y_j overwrites Y_{j-2} (each element read before it is written)
        if (e2 == cudaSuccess)
          e2 = launch_cm_step(H, cur, prv, last ? Xb : prv, last ? ld : -1, wb, 2.0 * sigma_new / e, -sigma * sigma_new,
                              c, coef, cld, last, zero, sh);
        std::swap(cur, prv);
        sigma = sigma_new;
      }
      return e2;
    };
    cudaError_t err = cudaSuccess;
    for (int c0 = 0; c0 < k && err == cudaSuccess; c0 += w) {
      const int wb = std::min(w, k - c0);
      float* Xb = (float*)X + c0;
      const int wb0 = split ? cm_first_half_cols(wb) : wb, wb1 = wb - wb0;
      if (wb1 > 0) {
        err = cudaEventRecord(ev_fork, st);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(st1, ev_fork, 0);
      }
      if (err == cudaSuccess) err = run(Xb, wb0, A, B, coefh[0], st);
      if (err == cudaSuccess && wb1 > 0) {
        const size_t off = (size_t)H.grid.n_slots * wb0;   // wb0 is a multiple of 16
        err = run(Xb + wb0, wb1, A + off, B + off, coefh[1], st1);
        if (err == cudaSuccess) err = cudaEventRecord(ev_join, st1);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(st, ev_join, 0);
      }
    }
    release();
    KSCF_CUDA_TRY(err);
    return KSCF_OK;
  }
  const int64_t wpad = coef_ld(w);
  void* buf = cv.take((size_t)H.grid.n_slots * wpad * es);
  void* coef = cv.take((size_t)std::max(H.n_kb, 1) * 4 * wpad * es);
  KSCF_CUDA_TRY(launch_zero_rows(H, X, ld, k, dtype, st));
  for (int c0 = 0; c0 < k; c0 += w) {
    const int wb = std::min(w, k - c0);
    char* Xb = (char*)X + (size_t)c0 * es;
    // columns usable from the block start in every row (lets the FP32 brick kernel read
    // whole 8-vector chunks when the row has room)
    const int avail_x = (int)std::min<int64_t>(ld - c0, 1 << 30), avail_b = (int)wpad;
    KSCF_CUDA_TRY(launch_zero_rows(H, buf, wpad, wb, dtype, st));
    // Y_1 = (sigma_1/e)(H X - c X)   -> buf
    KSCF_CUDA_TRY(launch_kb_gather(H, Xb, ld, wb, dtype, coef, wpad, st));
    KSCF_CUDA_TRY(launch_cheb_step(H, Xb, ld, nullptr, 0, buf, wpad, wb, std::min(avail_x, avail_b), dtype,
                                   sigma1 / e, 0.0, c, coef, wpad, st));
    void* cur = buf;
    int64_t ld_cur = wpad;
    void* prv = Xb;
    int64_t ld_prv = ld;
    double sigma = sigma1;
    for (int j = 2; j <= degree; j++) {
      const double sigma_new = 1.0 / (tau - sigma);
      KSCF_CUDA_TRY(launch_kb_gather(H, cur, ld_cur, wb, dtype, coef, wpad, st));
      // Y_j overwrites Y_{j-2} in place (each element is read before it is written)
      KSCF_CUDA_TRY(launch_cheb_step(H, cur, ld_cur, prv, ld_prv, prv, ld_prv, wb, std::min(avail_x, avail_b), dtype,
                                     2.0 * sigma_new / e, -sigma * sigma_new, c, coef, wpad, st));
      std::swap(cur, prv);
      std::swap(ld_cur, ld_prv);
      sigma = sigma_new;
    }
    if (cur != (void*)Xb) KSCF_CUDA_TRY(launch_copy_cols(cur, ld_cur, Xb, ld, H.grid.n_slots, wb, dtype, st));
  }
  return KSCF_OK;
}

extern "C" int kscf_orthonormalize(const kscf_ham* ham, void* X, int64_t ld, int k, int dtype, int mode, void* work,
                                   size_t work_bytes, void* stream) {
  const bool allow_shift = (mode & KSCF_ORTHO_ALLOW_SHIFT) != 0;
  mode &= ~KSCF_ORTHO_ALLOW_SHIFT;
  int rc = check_common(ham, X, ld, k, dtype, "kscf_orthonormalize");
  if (rc) return rc;
  rc = check_mode(dtype, mode, "kscf_orthonormalize");
  if (rc) return rc;
  const Ham& H = ham->h;
  OrthoPlan p;
  rc = ortho_plan(H, k, dtype, mode, &p);
  if (rc) return rc;
  rc = check_work(work, work_bytes, ortho_bytes(p), "kscf_orthonormalize");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  KSCF_CUDA_TRY(launch_zero_rows(H, X, ld, k, dtype, st));
  Carver cv(work);
  bool shifted = false;
  rc = cholqr_pass(H, X, ld, k, dtype, mode, p, cv, false, st, allow_shift ? &shifted : nullptr);
  if (rc) return rc;
  if (shifted) {
    rc = cholqr_pass(H, X, ld, k, dtype, mode, p, cv, false, st);
    if (rc) return rc;
  }
  // FP32: a second pass (its rotation by the first-order inverse square root of its Gram
  // matrix when that is within kFp32PolarTol of I, else by a factorised R^-1)
  if (dtype == KSCF_F32) rc = cholqr_pass(H, X, ld, k, dtype, mode, p, cv, true, st, nullptr, kFp32PolarTol);
  return rc;
}

extern "C" int kscf_rayleigh_ritz(const kscf_ham* ham, void* X, int64_t ld, int k, int dtype, int mode,
                                  double* eigvals_host, void* work, size_t work_bytes, void* stream) {
  int rc = check_common(ham, X, ld, k, dtype, "kscf_rayleigh_ritz");
  if (rc) return rc;
  rc = check_mode(dtype, mode, "kscf_rayleigh_ritz");
  if (rc) return rc;
  if (!eigvals_host) {
    set_error("kscf_rayleigh_ritz: null eigvals_host");
    return KSCF_ERR_INVALID;
  }
  const Ham& H = ham->h;
  // block width of the H X stream: the widest (k, then halving to multiples of 32) whose
  // buffers fit the caller's work buffer, so that with the default workspace the projection
  // is one symmetric Gram over one split of X
  int block = k;
  RRPlan p;
  rc = rr_plan(H, k, dtype, mode, block, &p);
  if (rc) return rc;
  while (rr_bytes(p) > work_bytes && block > 32) {
    block = std::max(32, block / 2 / 32 * 32);
    rc = rr_plan(H, k, dtype, mode, block, &p);
    if (rc) return rc;
  }
  rc = check_work(work, work_bytes, rr_bytes(p), "kscf_rayleigh_ritz");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Carver cv(work);
  void* hxb = cv.take(p.hxb);
  void* coef = cv.take(p.coef);
  double* Hs = (double*)cv.take(p.Hs);
  double* W = (double*)cv.take(p.W);
  void* Qm = cv.take(p.Q);
  int* info = (int*)cv.take(p.info);
  void* lwork = cv.take(p.lwork_bytes);
  void* panel = cv.take(p.panel);
  void* tcw = cv.take(p.tc);
  const size_t es = esize(dtype);
  const double h3 = H.grid.h * H.grid.h * H.grid.h;
  // the tensor path sums over the domain rows only (padding rows of X and H X are zero)
  const int32_t* live = mode == KSCF_GEMM_TENSOR ? H.d_live : nullptr;
  const int64_t rows = live ? H.n_live : H.grid.n_slots;
  KSCF_CUDA_TRY(launch_zero_rows(H, X, ld, k, dtype, st));
  for (int c0 = 0; c0 < k; c0 += p.w) {
    const int wb = std::min(p.w, k - c0);
    char* Xb = (char*)X + (size_t)c0 * es;
    const int64_t wpad = coef_ld(wb);
    KSCF_CUDA_TRY(launch_zero_rows(H, hxb, wpad, wb, dtype, st));
    KSCF_CUDA_TRY(launch_kb_gather(H, Xb, ld, wb, dtype, coef, wpad, st));
    KSCF_CUDA_TRY(launch_cheb_step(H, Xb, ld, nullptr, 0, hxb, wpad, wb,
                                   (int)std::min<int64_t>(ld - c0, wpad), dtype, 1.0, 0.0, 0.0, coef, wpad, st));
    // Hs[:, c0:c0+wb] = h^3 X^T (H X_b); with a single block the product is symmetric (H is)
    rc = gram(X, ld, hxb, wpad, rows, k, wb, dtype, mode, h3, Hs + (size_t)c0 * k, k, tcw, p.tc, st, wb == k, live);
    if (rc) return rc;
  }
  KSCF_CUDA_TRY(launch_sym_eig(Hs, k, k, W, lwork, p.lwork_bytes, info, st));
  // eigenvector signs chosen so that diag(Q) >= 0: for an input block already close to
  // Ritz vectors Q is then close to the identity, and the tensor-core rotation is applied
  // as X + X (Q - I), whose rounding error scales with |Q - I| instead of |Q|
  if (mode == KSCF_GEMM_TENSOR) KSCF_CUDA_TRY(launch_sign_fix(Hs, k, st));
  if (mode != KSCF_GEMM_TENSOR) KSCF_CUDA_TRY(launch_f64_to_dtype(Hs, (int64_t)k * k, dtype, Qm, st));
  int hinfo[4] = {0, 0, 0, 0};
  KSCF_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, st));
  KSCF_CUDA_TRY(cudaMemcpyAsync(eigvals_host, W, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  KSCF_CUDA_TRY(cudaStreamSynchronize(st));
  rc = check_tc(mode, "kscf_rayleigh_ritz");
  if (rc) return rc;
  rc = eig_info_code(hinfo, "kscf_rayleigh_ritz");
  if (rc) return rc;
  for (int i = 0; i < k; i++)
    if (!std::isfinite(eigvals_host[i])) {
      set_error("kscf_rayleigh_ritz: non-finite Ritz value");
      return KSCF_ERR_NONFINITE;
    }
  return rotate_inplace(H, X, ld, k, dtype, mode, Qm, Hs, mode == KSCF_GEMM_TENSOR, panel, p.prows, tcw, p.tc, st);
}

extern "C" int kscf_sym_eig_work_bytes(int n, size_t* bytes) {
  if (n < 1 || n > KSCF_EIG_MAX_N || !bytes) {
    set_error("kscf_sym_eig_work_bytes: n = %d outside [1, %d] or null output", n, KSCF_EIG_MAX_N);
    return KSCF_ERR_INVALID;
  }
  *bytes = sym_eig_work_bytes(n) + 256;
  return KSCF_OK;
}

extern "C" int kscf_sym_eig(double* A, int64_t lda, int n, double* w, void* work, size_t work_bytes, void* stream) {
  if (!A || !w || n < 1 || n > KSCF_EIG_MAX_N || lda < n) {
    set_error("kscf_sym_eig: invalid argument (n = %d, lda = %lld)", n, (long long)lda);
    return KSCF_ERR_INVALID;
  }
  const size_t need = sym_eig_work_bytes(n) + 256;
  if (!work || work_bytes < need) {
    set_error("kscf_sym_eig: work buffer of %zu bytes, need %zu", work_bytes, need);
    return KSCF_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* info = (int*)work;   // first 256 bytes: status words
  KSCF_CUDA_TRY(launch_sym_eig(A, lda, n, w, (char*)work + 256, work_bytes - 256, info, st));
  int hinfo[4] = {0, 0, 0, 0};
  KSCF_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, st));
  KSCF_CUDA_TRY(cudaStreamSynchronize(st));
  return eig_info_code(hinfo, "kscf_sym_eig");
}

extern "C" int kscf_density(const kscf_ham* ham, const void* X, int64_t ld, int n_occ, int dtype, const double* occ,
                            double* rho, void* stream) {
  if (!ham || !X || !rho || n_occ < 0 || ld < n_occ || (dtype != KSCF_F64 && dtype != KSCF_F32)) {
    set_error("kscf_density: invalid argument");
    return KSCF_ERR_INVALID;
  }
  KSCF_CUDA_TRY(launch_density(ham->h, X, ld, n_occ, dtype, occ, rho, (cudaStream_t)stream));
  return KSCF_OK;
}

extern "C" int kscf_points_to_slots(const kscf_ham* ham, const void* P, int64_t ldp, void* X, int64_t ldx, int k,
                                    int dtype, void* stream) {
  int rc = check_common(ham, X, ldx, k, dtype, "kscf_points_to_slots");
  if (rc) return rc;
  if (!P || ldp < k) {
    set_error("kscf_points_to_slots: invalid argument");
    return KSCF_ERR_INVALID;
  }
  KSCF_CUDA_TRY(launch_points_slots(ham->h, true, P, ldp, X, ldx, k, dtype, (cudaStream_t)stream));
  return KSCF_OK;
}

extern "C" int kscf_slots_to_points(const kscf_ham* ham, const void* X, int64_t ldx, void* P, int64_t ldp, int k,
                                    int dtype, void* stream) {
  int rc = check_common(ham, X, ldx, k, dtype, "kscf_slots_to_points");
  if (rc) return rc;
  if (!P || ldp < k) {
    set_error("kscf_slots_to_points: invalid argument");
    return KSCF_ERR_INVALID;
  }
  KSCF_CUDA_TRY(launch_points_slots(ham->h, false, X, ldx, P, ldp, k, dtype, (cudaStream_t)stream));
  return KSCF_OK;
}

extern "C" int kscf_random_subspace(const kscf_ham* ham, void* X, int64_t ld, int k, int dtype, uint64_t seed,
                                    void* stream) {
  int rc = check_common(ham, X, ld, k, dtype, "kscf_random_subspace");
  if (rc) return rc;
  KSCF_CUDA_TRY(launch_random(ham->h, X, ld, k, dtype, seed, (cudaStream_t)stream));
  return KSCF_OK;
}

extern "C" int kscf_gram(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t rows, int m, int n,
                         int dtype, int mode, double scale, double* C, int64_t ldc, void* work, size_t work_bytes,
                         void* stream) {
  if (!A || !B || !C || rows < 0 || m < 1 || n < 1 || lda < m || ldb < n || ldc < m ||
      (dtype != KSCF_F64 && dtype != KSCF_F32)) {
    set_error("kscf_gram: invalid argument");
    return KSCF_ERR_INVALID;
  }
  int rc = check_mode(dtype, mode, "kscf_gram");
  if (rc) return rc;
  const size_t need = mode == KSCF_GEMM_TENSOR ? gram_tc_work_bytes(rows, m, n) : 0;
  rc = check_work(work, work_bytes, need, "kscf_gram");
  if (rc) return rc;
  return gram(A, lda, B, ldb, rows, m, n, dtype, mode, scale, C, ldc, work, work_bytes, (cudaStream_t)stream);
}

extern "C" int kscf_rotate(const void* A, int64_t lda, const double* Q, int64_t ldq, int64_t rows, int kin,
                           int kout, int dtype, int mode, int minus_identity, void* out, int64_t ldo, void* work,
                           size_t work_bytes, void* stream) {
  if (!A || !Q || !out || rows < 0 || kin < 1 || kout < 1 || lda < kin || ldq < kin || ldo < kout ||
      (dtype != KSCF_F64 && dtype != KSCF_F32) || (minus_identity && kin != kout)) {
    set_error("kscf_rotate: invalid argument");
    return KSCF_ERR_INVALID;
  }
  int rc = check_mode(dtype, mode, "kscf_rotate");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == KSCF_GEMM_TENSOR) {
    rc = check_work(work, work_bytes, rotate_tc_work_bytes(rows, kin, kout), "kscf_rotate");
    if (rc) return rc;
    KSCF_CUDA_TRY(launch_rotate_tc((const float*)A, lda, Q, ldq, rows, kin, kout, minus_identity != 0,
                                   (float*)out, ldo, work, work_bytes, st));
    return KSCF_OK;
  }
  if (minus_identity) {
    set_error("kscf_rotate: minus_identity needs the tensor mode");
    return KSCF_ERR_UNSUPPORTED;
  }
  const size_t need = (size_t)kin * kout * esize(dtype);
  rc = check_work(work, work_bytes, need, "kscf_rotate");
  if (rc) return rc;
  // native: convert Q into the work buffer (column-major, ld = kin), then rotate
  double* Qc = (double*)work;
  if (dtype == KSCF_F64 && ldq == kin) {
    KSCF_CUDA_TRY(launch_rotate_native(A, lda, Q, ldq, rows, kin, kout, dtype, out, ldo, st));
    return KSCF_OK;
  }
  (void)Qc;
  if (ldq != kin) {
    set_error("kscf_rotate: native mode needs ldq == kin");
    return KSCF_ERR_UNSUPPORTED;
  }
  KSCF_CUDA_TRY(launch_f64_to_dtype(Q, (int64_t)kin * kout, dtype, work, st));
  KSCF_CUDA_TRY(launch_rotate_native(A, lda, work, kin, rows, kin, kout, dtype, out, ldo, st));
  return KSCF_OK;
}

extern "C" int kscf_gemm_workspace_size(int op, int64_t rows, int m, int n, int dtype, int mode, size_t* bytes) {
  if (!bytes || rows < 0 || m < 1 || n < 1) {
    set_error("kscf_gemm_workspace_size: invalid argument");
    return KSCF_ERR_INVALID;
  }
  if (mode == KSCF_GEMM_TENSOR)
    *bytes = op == 0 ? gram_tc_work_bytes(rows, m, n) : rotate_tc_work_bytes(rows, m, n);
  else
    *bytes = op == 0 ? 256 : kscf_align256((size_t)m * n * esize(dtype));
  return KSCF_OK;
}

extern "C" int kscf_selftest_barrier_timeout(void* stream) {
  const int k = 64;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t sbytes = (size_t)k * k * 8, wbytes = chol_inv_work_bytes(k);
  char* buf = nullptr;
  KSCF_CUDA_TRY(cudaMalloc(&buf, kscf_align256(sbytes) + 256 + wbytes));
  double* S = (double*)buf;
  int* status = (int*)(buf + kscf_align256(sbytes));
  void* work = buf + kscf_align256(sbytes) + 256;
  std::vector<double> eye((size_t)k * k, 0.0);
  for (int i = 0; i < k; i++) eye[(size_t)i * k + i] = 1.0;
  int hst[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(S, eye.data(), sbytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_chol_inv(S, k, k, 0.0, S, k, work, status, st, 2000000LL, 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst, status, sizeof(hst), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_error("kscf_selftest_barrier_timeout: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  if (hst[1] != 0) {
    set_error("kscf_selftest_barrier_timeout: the bounded grid barrier gave up as expected");
    return KSCF_ERR_TIMEOUT;
  }
  return KSCF_OK;
}

extern "C" int kscf_selftest_eig_barrier_timeout(void* stream) {
  const int n = 64;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t abytes = kscf_align256((size_t)n * n * 8), vbytes = kscf_align256((size_t)n * 8);
  const size_t wbytes = sym_eig_work_bytes(n);
  char* buf = nullptr;
  KSCF_CUDA_TRY(cudaMalloc(&buf, abytes + vbytes + 256 + wbytes));
  double* A = (double*)buf;
  double* w = (double*)(buf + abytes);
  int* info = (int*)(buf + abytes + vbytes);
  void* work = buf + abytes + vbytes + 256;
  std::vector<double> eye((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++) eye[(size_t)i * n + i] = 1.0;
  int hi[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemsetAsync(work, 0, wbytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A, eye.data(), (size_t)n * n * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_sym_eig(A, n, n, w, work, wbytes, info, st, 2000000LL, 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hi, info, sizeof(hi), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_error("kscf_selftest_eig_barrier_timeout: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  if (hi[0] != 0) {
    set_error("kscf_selftest_eig_barrier_timeout: the bounded grid barrier gave up as expected");
    return KSCF_ERR_TIMEOUT;
  }
  return KSCF_OK;
}

extern "C" int kscf_check_status(void) {
  unsigned int st = 0, fs = 0, cs = 0, nf = 0;
  cudaError_t e = tc_status(true, &st);
  if (e == cudaSuccess) e = filter_status(true, &fs);
  if (e == cudaSuccess) e = cm_status(true, &cs, &nf);
  st |= (fs | cs) << 1;
  if (e != cudaSuccess) {
    set_error("kscf_check_status: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  if (st) {
    set_error("a bounded device wait timed out (status %u: bit 0 tensor-core GEMM, bit 1 filter)", st);
    return KSCF_ERR_TIMEOUT;
  }
  if (nf) {
    set_error("a Chebyshev filter or Hamiltonian apply stored a NaN or Inf (non-finite input X or potential)");
    return KSCF_ERR_NONFINITE;
  }
  return KSCF_OK;
}
