// Internal declarations of the SCF kernels (scf_kernels.cu) and their host driver (scf.cpp).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kscf_internal.h"

namespace kscf {

constexpr int kScfThreads = 256;    // threads per block of the reduction kernels
constexpr int kScfRedBlocks = 304;  // blocks of the reduction kernels (2 per SM); one partial each
constexpr int kAndersonMax = 8;     // longest mixing history

// Ghost points of the Poisson problem: points outside the domain that the order-12
// stencil of a domain point reaches, with the coupling of every domain slot to them.
struct PoissonPlan {
  int64_t n_ghost = 0;
  double* d_grel = nullptr;    // 3 per ghost: h (i, j, k), relative to the grid centre
  double* d_vghost = nullptr;  // multipole potential at each ghost
  int64_t* d_gptr = nullptr;   // n_slots + 1: CSR rows of the slots
  int32_t* d_gidx = nullptr;   // entry -> ghost
  double* d_gw = nullptr;      // entry -> w_k / h^2
};

// Mixing history columns in use, oldest first, and their coefficients.
struct AndersonCols {
  int m = 0;
  int idx[kAndersonMax] = {0};
  double g[kAndersonMax] = {0};
};

cudaError_t launch_finalize_partials(const double* part, int nb, int nv, double* out, cudaStream_t st);
cudaError_t launch_atomic_density(const Ham& H, const double* rel, const double* atoms, int n_atoms, double* rho,
                                  cudaStream_t st);
cudaError_t launch_lda(const Ham& H, const double* rho, double* eps, double* vxc, cudaStream_t st);
cudaError_t launch_poisson_rhs(const Ham& H, const double* rho, const PoissonPlan& P, double* b, double* part_bb,
                               cudaStream_t st);
// CG on A x = b with A = -Lap_h + shift (zero outside the domain)
cudaError_t launch_cg_init(const Ham& H, double shift, double* x, const double* b, double* r, double* p,
                           double* part_rr, cudaStream_t st);
// one CG iteration (three kernels); every kernel returns at once when r.r < rtol^2 b.b
cudaError_t launch_cg_iteration(const Ham& H, double shift, const double* part_bb, double rtol, double* x, double* r,
                                double* p, double* q, const double* part_rr, double* part_pq, double* part_rr_next,
                                int* iters, cudaStream_t st);
// b = f on the domain, partial b.b
cudaError_t launch_rhs_copy(const Ham& H, const double* f, double* b, double* part_bb, cudaStream_t st);
// out = a + c b on the domain
cudaError_t launch_lincomb(const Ham& H, const double* a, const double* b, double c, double* out, cudaStream_t st);
cudaError_t launch_ghost_values(const Ham& H, const double* rho, const double* rel, const PoissonPlan& P,
                                double* part, double* mom, cudaStream_t st);
cudaError_t launch_residual(const Ham& H, const double* rho, const double* v_in, const double* v_ion, const double* vh,
                            const double* vxc, const double* eps, double* f, double* part, double* out5,
                            cudaStream_t st);
cudaError_t launch_sum3(const Ham& H, const double* a, const double* b, const double* c, double* out,
                        cudaStream_t st);
// out[j] = sum_r X[r][j]^2 (FP64), part: kScfRedBlocks * k doubles
cudaError_t launch_col_sumsq(const void* X, int64_t ld, int64_t rows, int k, int dtype, double* part, double* out,
                             cudaStream_t st);
// out[j] = sum_r A[r][j] B[r][j] (FP64 sums)
cudaError_t launch_col_dot(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t rows, int k, int dtype,
                           double* part, double* out, cudaStream_t st);
// out[j] = sum_r (HX[r][j] - lam[j] X[r][j])^2, lam on the device
cudaError_t launch_col_resid(const double* X, const double* HX, int64_t ld, int64_t rows, int k, const double* lam,
                             double* part, double* out, cudaStream_t st);
// the same for X, HX of dtype (FP32 values, FP64 sums)
cudaError_t launch_col_resid_t(const void* X, const void* HX, int64_t ld, int64_t rows, int k, int dtype,
                               const double* lam, double* part, double* out, cudaStream_t st);
cudaError_t launch_widen(const float* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int k,
                         cudaStream_t st);
cudaError_t launch_add2(const Ham& H, const double* a, const double* b, double* out, cudaStream_t st);
cudaError_t launch_anderson_push(int64_t n, const double* v_in, const double* f, const double* pf, double* v_prev,
                                 double* f_prev, double* pf_prev, double* dv, double* df, double* dpf, bool have_prev,
                                 cudaStream_t st);
cudaError_t launch_anderson_gram(const AndersonCols& cols, const double* df, const double* f, int64_t n,
                                 double* part, double* out, cudaStream_t st);
cudaError_t launch_anderson_update(const Ham& H, const AndersonCols& cols, double alpha, const double* dv,
                                   const double* dpf, const double* pf, double* v, cudaStream_t st);

// training data of the learned start: rows in lexicographic point order
cudaError_t launch_training_rows(const Ham& H, const float* D, const double* v_in, const double* v_start, float* D_out,
                                 float* t_out, cudaStream_t st);

}  // namespace kscf
