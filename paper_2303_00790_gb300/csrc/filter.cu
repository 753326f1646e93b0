// Chebyshev filter step and Hamiltonian apply on the Hilbert-brick grid.
//
// One step computes, for every slot s and vector v of a column block,
//   out = alpha * (H in - c in) + beta * prev,
//   H in = -1/2 Lap_h in + V in + sum_i chi_i (E_i h^3 <chi_i, in>)
// which is one term of the scaled three-term Chebyshev recurrence of CheFSI
// (arXiv 2303.00790, CheFSI paragraph; recurrence of Zhou, Saad, Tiago &
// Chelikowsky 2006) with the stencil, the local potential, the nonlocal scatter and
// the recurrence update fused in one pass over the grid.  The projections
// <chi_i, in> come from kb_gather, launched just before on the same stream.
#include <cuda_runtime.h>

#include "kscf_internal.h"

namespace kscf {

template <typename T>
struct StepArgs {
  const T* in;
  int64_t ld_in;
  const T* prev;  // may alias out (read before write, same element)
  int64_t ld_prev;
  T* out;
  int64_t ld_out;
  int w;
  T alpha, beta, c;
  const T* coef;  // (n_kb*4) x w
  const T* V;
  const int32_t* nbr;
  const uint8_t* mask;
  const int64_t* kb_ptr;
  const int32_t* kb_atom;
  const T* kb_chi;
  T st[7];
  int64_t n_slots;
};

// ---------------------------------------------------------------------------
// Reference-shaped kernel: one thread per (slot, vector).
template <typename T, int B>
__global__ void __launch_bounds__(256) cheb_step_generic(StepArgs<T> a) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.n_slots * a.w) return;
  const int64_t s = idx / a.w;
  const int v = (int)(idx - s * a.w);
  constexpr int B3 = B * B * B;
  T res = T(0);
  if (a.mask[s]) {
    const int64_t brick = s / B3;
    const int li = (int)(s - brick * B3);
    const int l[3] = {li % B, (li / B) % B, li / (B * B)};
    const int stride[3] = {1, B, B * B};
    const T y = a.in[s * a.ld_in + v];
    T acc = T(3) * a.st[0] * y;
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
#pragma unroll
      for (int k = 1; k <= 6; k++) {
        T pair = T(0);
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
          const int n = l[ax] + sg * k;
          int64_t ns;
          if (n >= 0 && n < B) {
            ns = s + (int64_t)sg * k * stride[ax];
          } else {
            const int nb = a.nbr[brick * 6 + 2 * ax + (sg > 0 ? 1 : 0)];
            if (nb < 0) continue;
            ns = (int64_t)nb * B3 + li + (sg * k - sg * B) * stride[ax];
          }
          pair += a.in[ns * a.ld_in + v];
        }
        acc += a.st[k] * pair;
      }
    }
    acc += a.V[s] * y;
    for (int64_t e = a.kb_ptr[s]; e < a.kb_ptr[s + 1]; e++) {
      const T* cf = a.coef + (int64_t)a.kb_atom[e] * 4 * a.w + v;
      const T* ch = a.kb_chi + 4 * e;
      acc += ch[0] * cf[0] + ch[1] * cf[a.w] + ch[2] * cf[2 * a.w] + ch[3] * cf[3 * a.w];
    }
    res = a.alpha * (acc - a.c * y);
    if (a.prev) res += a.beta * a.prev[s * a.ld_prev + v];
  }
  a.out[s * a.ld_out + v] = res;
}

// coef[(a*4+l)*w + v] = E_l h^3 sum_{entries e of atom a} chi_l(e) Y[slot_e][v]
template <typename T>
__global__ void __launch_bounds__(256) kb_gather_kernel(const T* __restrict__ Y, int64_t ld, int w,
                                                         const int64_t* __restrict__ aptr,
                                                         const int64_t* __restrict__ aslot,
                                                         const T* __restrict__ achi,
                                                         const double* __restrict__ energy,
                                                         T* __restrict__ coef) {
  const int at = blockIdx.x;
  const int v = blockIdx.y * 32 + threadIdx.x;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  if (v < w) {
    for (int64_t e = aptr[at] + threadIdx.y; e < aptr[at + 1]; e += 8) {
      const T y = Y[aslot[e] * ld + v];
#pragma unroll
      for (int l = 0; l < 4; l++) acc[l] += achi[4 * e + l] * y;
    }
  }
  __shared__ T red[8][4][32];
#pragma unroll
  for (int l = 0; l < 4; l++) red[threadIdx.y][l][threadIdx.x] = acc[l];
  __syncthreads();
  if (threadIdx.y < 4 && v < w) {
    const int l = threadIdx.y;
    T sum = T(0);
#pragma unroll
    for (int q = 0; q < 8; q++) sum += red[q][l][threadIdx.x];
    coef[((int64_t)at * 4 + l) * w + v] = (T)energy[4 * at + l] * sum;
  }
}

template <typename T>
__global__ void zero_rows_kernel(T* X, int64_t ld, int k, const int64_t* pad, int64_t n_pad) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_pad * k) return;
  const int64_t r = idx / k;
  X[pad[r] * ld + (idx - r * k)] = T(0);
}

template <typename T>
__global__ void copy_cols_kernel(const T* src, int64_t ld_src, T* dst, int64_t ld_dst, int64_t rows, int w) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * w) return;
  const int64_t r = idx / w;
  const int j = (int)(idx - r * w);
  dst[r * ld_dst + j] = src[r * ld_src + j];
}

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_zero_rows(const Ham& H, void* X, int64_t ld, int k, int dtype, cudaStream_t st) {
  if (H.n_pad == 0 || k == 0) return cudaSuccess;
  const int64_t n = H.n_pad * k;
  if (dtype == KSCF_F64)
    zero_rows_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>((double*)X, ld, k, H.d_pad, H.n_pad), count_launch();
  else
    zero_rows_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>((float*)X, ld, k, H.d_pad, H.n_pad), count_launch();
  return cudaGetLastError();
}

cudaError_t launch_kb_gather(const Ham& H, const void* Y, int64_t ld, int w, int dtype, void* coef,
                             cudaStream_t st) {
  if (H.n_kb == 0 || w == 0) return cudaSuccess;
  dim3 grid(H.n_kb, (w + 31) / 32), block(32, 8);
  if (dtype == KSCF_F64)
    kb_gather_kernel<double><<<grid, block, 0, st>>>((const double*)Y, ld, w, H.d_kb_atom_ptr,
                                                     H.d_kb_atom_slot, H.d_kb_atom_chi64,
                                                     H.d_kb_energy, (double*)coef), count_launch();
  else
    kb_gather_kernel<float><<<grid, block, 0, st>>>((const float*)Y, ld, w, H.d_kb_atom_ptr,
                                                    H.d_kb_atom_slot, H.d_kb_atom_chi32,
                                                    H.d_kb_energy, (float*)coef), count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t step_t(const Ham& H, const void* in, int64_t ld_in, const void* prev, int64_t ld_prev,
                          void* out, int64_t ld_out, int w, double alpha, double beta, double c,
                          const void* coef, const T* V, const T* chi, cudaStream_t st) {
  StepArgs<T> a;
  a.in = (const T*)in;
  a.ld_in = ld_in;
  a.prev = (const T*)prev;
  a.ld_prev = ld_prev;
  a.out = (T*)out;
  a.ld_out = ld_out;
  a.w = w;
  a.alpha = (T)alpha;
  a.beta = (T)beta;
  a.c = (T)c;
  a.coef = (const T*)coef;
  a.V = V;
  a.nbr = H.d_nbr;
  a.mask = H.d_mask;
  a.kb_ptr = H.d_kb_slot_ptr;
  a.kb_atom = H.d_kb_slot_atom;
  a.kb_chi = chi;
  for (int k = 0; k < 7; k++) a.st[k] = (T)H.stencil[k];
  a.n_slots = H.grid.n_slots;
  const int64_t n = a.n_slots * w;
  if (H.grid.B == 8)
    cheb_step_generic<T, 8><<<blocks_for(n, 256), 256, 0, st>>>(a), count_launch();
  else
    cheb_step_generic<T, 16><<<blocks_for(n, 256), 256, 0, st>>>(a), count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cheb_step(const Ham& H, const void* in, int64_t ld_in, const void* prev, int64_t ld_prev,
                             void* out, int64_t ld_out, int w, int dtype, double alpha, double beta,
                             double c, const void* coef, cudaStream_t st) {
  if (dtype == KSCF_F64)
    return step_t<double>(H, in, ld_in, prev, ld_prev, out, ld_out, w, alpha, beta, c, coef, H.d_v64,
                          H.d_kb_slot_chi64, st);
  return step_t<float>(H, in, ld_in, prev, ld_prev, out, ld_out, w, alpha, beta, c, coef, H.d_v32,
                       H.d_kb_slot_chi32, st);
}

cudaError_t launch_copy_cols(const void* src, int64_t ld_src, void* dst, int64_t ld_dst, int64_t rows, int w,
                             int dtype, cudaStream_t st) {
  const int64_t n = rows * w;
  if (n == 0) return cudaSuccess;
  if (dtype == KSCF_F64)
    copy_cols_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>((const double*)src, ld_src, (double*)dst,
                                                                 ld_dst, rows, w), count_launch();
  else
    copy_cols_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>((const float*)src, ld_src, (float*)dst,
                                                                ld_dst, rows, w), count_launch();
  return cudaGetLastError();
}

}  // namespace kscf
