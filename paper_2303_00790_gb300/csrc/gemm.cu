// CUDA-core GEMMs of the subspace steps (Cholesky-QR and Rayleigh-Ritz of CheFSI):
//   gram:   C += scale * A^T B      (tall-skinny reduction over grid slots)
//   rotate: out = A Q               (tall-skinny times k x k)
// These are the "native" precision path (FP64 X -> FP64 arithmetic, FP32 X -> FP32
// products with FP64 sums of partial results).  The tensor-core path is in
// gemm_tc.cu.
#include <cuda_runtime.h>

#include <algorithm>

#include "kscf_internal.h"

namespace kscf {

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// 64x64 tile of C per CTA, 256 threads with 4x4 outputs each; rows split over
// gridDim.z; partial sums in T over at most 256 rows, then FP64; FP64 atomics into C.
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const T* __restrict__ A, int64_t lda, const T* __restrict__ B,
                                                    int64_t ldb, int64_t rows, int m, int n, double scale,
                                                    double* __restrict__ C, int64_t ldc, int64_t rows_per_split) {
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64 + 1];
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t r_end = min(rows, r_begin + rows_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc64[4][4];
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      acc64[p][q] = 0.0;
      acc[p][q] = T(0);
    }
  int since_flush = 0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += 16) {
    // load 16 rows x 64 columns of A and B
    for (int q = threadIdx.x; q < 16 * 64; q += 256) {
      const int rr = q >> 6, cc = q & 63;
      const int64_t r = r0 + rr;
      As[rr][cc] = (r < r_end && i0 + cc < m) ? A[r * lda + i0 + cc] : T(0);
      Bs[rr][cc] = (r < r_end && j0 + cc < n) ? B[r * ldb + j0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 16; rr++) {
      T a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; p++) a[p] = As[rr][ty + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; q++) b[q] = Bs[rr][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] += a[p] * b[q];
    }
    __syncthreads();
    since_flush += 16;
    if (since_flush >= 256) {
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
          acc64[p][q] += (double)acc[p][q];
          acc[p][q] = T(0);
        }
      since_flush = 0;
    }
  }
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int i = i0 + ty + 16 * p, j = j0 + tx + 16 * q;
      if (i < m && j < n) atomicAdd(C + i + (int64_t)j * ldc, scale * (acc64[p][q] + (double)acc[p][q]));
    }
}

__global__ void zero_matrix_kernel(double* C, int m, int n, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * n) return;
  const int j = (int)(idx / m), i = (int)(idx - (int64_t)j * m);
  C[i + (int64_t)j * ldc] = 0.0;
}

cudaError_t launch_gram_native(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t rows, int m, int n,
                               int dtype, double scale, double* C, int64_t ldc, bool accumulate, cudaStream_t st) {
  if (!accumulate) {
    zero_matrix_kernel<<<blocks_for((int64_t)m * n, 256), 256, 0, st>>>(C, m, n, ldc), count_launch();
  }
  if (rows == 0 || m == 0 || n == 0) return cudaGetLastError();
  const int gx = (m + 63) / 64, gy = (n + 63) / 64;
  // split rows so that the grid covers the SMs a few times over
  int64_t splits = (4 * 152 + (int64_t)gx * gy - 1) / ((int64_t)gx * gy);
  splits = max((int64_t)1, min(splits, (rows + 1023) / 1024));
  int64_t per = (rows + splits - 1) / splits;
  per = (per + 15) / 16 * 16;
  splits = (rows + per - 1) / per;
  dim3 grid(gx, gy, (unsigned)splits);
  if (dtype == KSCF_F64)
    gram_kernel<double><<<grid, 256, 0, st>>>((const double*)A, lda, (const double*)B, ldb, rows, m, n, scale, C,
                                               ldc, per), count_launch();
  else
    gram_kernel<float><<<grid, 256, 0, st>>>((const float*)A, lda, (const float*)B, ldb, rows, m, n, scale, C, ldc,
                                              per), count_launch();
  return cudaGetLastError();
}

// out[r, j] = sum_i A[r, i] Q[i, j]; 64 rows x 64 columns per CTA, 4x4 per thread.
template <typename T>
__global__ void __launch_bounds__(256) rotate_kernel(const T* __restrict__ A, int64_t lda, const T* __restrict__ Q,
                                                      int64_t ldq, int64_t rows, int kin, int kout, T* __restrict__ out,
                                                      int64_t ldo) {
  __shared__ T As[64][16 + 1];
  __shared__ T Qs[16][64 + 1];
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int j0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[p][q] = T(0);
  for (int i0 = 0; i0 < kin; i0 += 16) {
    for (int q = threadIdx.x; q < 64 * 16; q += 256) {
      const int rr = q >> 4, ii = q & 15;
      const int64_t r = r0 + rr;
      As[rr][ii] = (r < rows && i0 + ii < kin) ? A[r * lda + i0 + ii] : T(0);
      const int jj = q >> 4, i2 = q & 15;
      Qs[i2][jj] = (i0 + i2 < kin && j0 + jj < kout) ? Q[(i0 + i2) + (int64_t)(j0 + jj) * ldq] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < 16; ii++) {
      T a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; p++) a[p] = As[ty + 16 * p][ii];
#pragma unroll
      for (int q = 0; q < 4; q++) b[q] = Qs[ii][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] += a[p] * b[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int64_t r = r0 + ty + 16 * p;
      const int j = j0 + tx + 16 * q;
      if (r < rows && j < kout) out[r * ldo + j] = acc[p][q];
    }
}

cudaError_t launch_rotate_native(const void* A, int64_t lda, const void* Q, int64_t ldq, int64_t rows, int kin,
                                 int kout, int dtype, void* out, int64_t ldo, cudaStream_t st) {
  if (rows == 0 || kout == 0) return cudaSuccess;
  dim3 grid((unsigned)((rows + 63) / 64), (kout + 63) / 64);
  if (dtype == KSCF_F64)
    rotate_kernel<double><<<grid, 256, 0, st>>>((const double*)A, lda, (const double*)Q, ldq, rows, kin, kout,
                                                 (double*)out, ldo), count_launch();
  else
    rotate_kernel<float><<<grid, 256, 0, st>>>((const float*)A, lda, (const float*)Q, ldq, rows, kin, kout,
                                                (float*)out, ldo), count_launch();
  return cudaGetLastError();
}

__global__ void symmetrize_kernel(double* C, int k, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * k) return;
  const int j = (int)(idx / k), i = (int)(idx - (int64_t)j * k);
  if (i < j) {
    const double a = C[i + (int64_t)j * ldc], b = C[j + (int64_t)i * ldc];
    const double m = 0.5 * (a + b);
    C[i + (int64_t)j * ldc] = m;
    C[j + (int64_t)i * ldc] = m;
  }
}

cudaError_t launch_symmetrize(double* C, int k, int64_t ldc, cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  symmetrize_kernel<<<blocks_for((int64_t)k * k, 256), 256, 0, st>>>(C, k, ldc), count_launch();
  return cudaGetLastError();
}

// Column j of the column-major k x k Q is negated when Q[j][j] < 0 (eigenvectors are
// defined up to sign; this makes Q close to the identity when the input columns are
// already close to eigenvectors).
__global__ void sign_fix_kernel(double* Q, int k) {
  const int j = blockIdx.x;
  if (j >= k) return;
  double* col = Q + (int64_t)j * k;
  if (!(col[j] < 0.0)) return;
  for (int i = threadIdx.x; i < k; i += blockDim.x) col[i] = -col[i];
}

cudaError_t launch_sign_fix(double* Q, int k, cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  sign_fix_kernel<<<k, 128, 0, st>>>(Q, k), count_launch();
  return cudaGetLastError();
}

// S[i][i] += rel * max_i S[i][i]  (one block; S column-major k x k)
__global__ void shift_diag_kernel(double* S, int k, double rel) {
  __shared__ double sm[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) m = fmax(m, S[(int64_t)i * k + i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = fmax(t, sm[w]);
    sm[0] = t;
  }
  __syncthreads();
  const double s = rel * sm[0];
  for (int i = threadIdx.x; i < k; i += blockDim.x) S[(int64_t)i * k + i] += s;
}

cudaError_t launch_shift_diag(double* S, int k, double rel, cudaStream_t st) {
  shift_diag_kernel<<<1, 256, 0, st>>>(S, k, rel), count_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void upper_kernel(const double* R, int k, T* out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * k) return;
  const int j = (int)(idx / k), i = (int)(idx - (int64_t)j * k);
  out[idx] = i <= j ? (T)R[idx] : T(0);
}

cudaError_t launch_upper_to_dtype(const double* R, int k, int dtype, void* out, cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  const int64_t n = (int64_t)k * k;
  if (dtype == KSCF_F64)
    upper_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>(R, k, (double*)out), count_launch();
  else
    upper_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>(R, k, (float*)out), count_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void convert_kernel(const double* src, int64_t n, T* out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) out[idx] = (T)src[idx];
}

cudaError_t launch_f64_to_dtype(const double* src, int64_t n, int dtype, void* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (dtype == KSCF_F64)
    convert_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>(src, n, (double*)out), count_launch();
  else
    convert_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>(src, n, (float*)out), count_launch();
  return cudaGetLastError();
}

// status = 1 when a diagonal element of the k x k matrix S (column-major) is NaN or Inf
__global__ void diag_finite_kernel(const double* S, int k, int64_t lds, int* status) {
  bool bad = false;
  for (int i = threadIdx.x; i < k; i += blockDim.x) bad |= !(fabs(S[i + i * lds]) <= 1.7976931348623157e308);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) *status = bad ? 1 : 0;
}

cudaError_t launch_diag_finite(const double* S, int k, int64_t lds, int* status, cudaStream_t st) {
  diag_finite_kernel<<<1, 256, 0, st>>>(S, k, lds, status), count_launch();
  return cudaGetLastError();
}

// *out = max_ij |S_ij - delta_ij| over the k x k matrix S (column-major, lds), as the bit
// pattern of a non-negative double (a NaN or Inf element counts as +Inf); *out is 0 before
__global__ void __launch_bounds__(256) dev_identity_kernel(const double* S, int k, int64_t lds,
                                                           unsigned long long* out) {
  double m = 0.0;
  const int64_t total = (int64_t)k * k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = q / k;
    const int r = (int)(q - c * k);
    double v = fabs(S[r + c * lds] - (r == c ? 1.0 : 0.0));
    if (!(v <= 1.7976931348623157e308)) v = __longlong_as_double(0x7ff0000000000000LL);
    m = fmax(m, v);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmax(m, wm[w]);
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
  }
}

// S <- (3 I - S) / 2 in place (k x k, column-major, lds): for S = I + E the first-order
// inverse square root I - E / 2
__global__ void polar_first_order_kernel(double* S, int k, int64_t lds) {
  const int64_t total = (int64_t)k * k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = q / k;
    const int r = (int)(q - c * k);
    double* x = S + r + c * lds;
    *x = ((r == c ? 3.0 : 0.0) - *x) * 0.5;
  }
}

cudaError_t launch_polar_first_order(double* S, int k, int64_t lds, cudaStream_t st) {
  const int64_t total = (int64_t)k * k;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(304, (total + 255) / 256));
  polar_first_order_kernel<<<grid, 256, 0, st>>>(S, k, lds), count_launch();
  return cudaGetLastError();
}

cudaError_t launch_dev_identity(const double* S, int k, int64_t lds, unsigned long long* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)k * k;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(304, (total + 255) / 256));
  dev_identity_kernel<<<grid, 256, 0, st>>>(S, k, lds, out), count_launch();
  return cudaGetLastError();
}

}  // namespace kscf
