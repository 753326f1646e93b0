// Set-up and small kernels: local potential, initial subspace, density, potential
// reductions.
#include <cuda_runtime.h>

#include <algorithm>

#include <cfloat>

#include "kscf_internal.h"

namespace kscf {

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// V_loc(p) = sum_a [ -Z_a erf(r/r_c)/r + A_a exp(-r^2/r_g^2) ],  r = |p - R_a|,
// with the r -> 0 limit -2 Z_a/(r_c sqrt(pi)) of the erf term (synthetic stand-in for
// the local part of the paper's pseudopotentials, Computational details).
// atoms: 8 doubles each (x, y, z, Z, r_c, A, r_g, unused).
__global__ void vloc_kernel(const double* __restrict__ xyz, const uint8_t* __restrict__ mask,
                            const double* __restrict__ atoms, int n_atoms, int64_t n_slots,
                            double* __restrict__ V) {
  __shared__ double sat[128 * 8];
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < n_slots && mask[s];
  double px = 0, py = 0, pz = 0;
  if (live) {
    px = xyz[3 * s];
    py = xyz[3 * s + 1];
    pz = xyz[3 * s + 2];
  }
  double acc = 0.0;
  for (int a0 = 0; a0 < n_atoms; a0 += 128) {
    const int na = min(128, n_atoms - a0);
    __syncthreads();
    for (int q = threadIdx.x; q < na * 8; q += blockDim.x) sat[q] = atoms[(int64_t)a0 * 8 + q];
    __syncthreads();
    if (live) {
      for (int a = 0; a < na; a++) {
        const double* at = sat + 8 * a;
        const double dx = px - at[0], dy = py - at[1], dz = pz - at[2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double r = sqrt(r2);
        const double coul = r > 0.0 ? -at[3] * erf(r / at[4]) / r : -2.0 * at[3] / (at[4] * 1.7724538509055160273);
        acc += coul + at[5] * exp(-r2 / (at[6] * at[6]));
      }
    }
  }
  if (s < n_slots) V[s] = live ? acc : 0.0;
}

cudaError_t launch_vloc(const Ham& H, const double* d_xyz, const double* d_atoms, int n_atoms, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  vloc_kernel<<<blocks_for(n, 128), 128, 0, st>>>(d_xyz, H.d_mask, d_atoms, n_atoms, n, H.d_v64), count_launch();
  return cudaGetLastError();
}

__global__ void v_to_f32_kernel(const double* v, float* v32, int64_t n) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) v32[s] = (float)v[s];
}

cudaError_t launch_v_to_f32(const Ham& H, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  v_to_f32_kernel<<<blocks_for(n, 256), 256, 0, st>>>(H.d_v64, H.d_v32, n), count_launch();
  return cudaGetLastError();
}

__global__ void mask_v_kernel(const double* src, const uint8_t* mask, double* dst, int64_t n) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) dst[s] = mask[s] ? src[s] : 0.0;
}

cudaError_t launch_mask_v(const Ham& H, const double* src, double* dst, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  mask_v_kernel<<<blocks_for(n, 256), 256, 0, st>>>(src, H.d_mask, dst, n), count_launch();
  return cudaGetLastError();
}

__global__ void minmax_kernel(const double* v, const uint8_t* mask, int64_t n, double* out) {
  double lo = DBL_MAX, hi = -DBL_MAX;
  for (int64_t s = threadIdx.x; s < n; s += blockDim.x)
    if (mask[s]) {
      lo = fmin(lo, v[s]);
      hi = fmax(hi, v[s]);
    }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  __shared__ double slo[32], shi[32];
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); q++) {
      lo = fmin(lo, slo[q]);
      hi = fmax(hi, shi[q]);
    }
    out[0] = lo;
    out[1] = hi;
  }
}

cudaError_t launch_minmax_v(const Ham& H, double* d_out2, cudaStream_t st) {
  minmax_kernel<<<1, 1024, 0, st>>>(H.d_v64, H.d_mask, H.grid.n_slots, d_out2), count_launch();
  return cudaGetLastError();
}

// Counter-based N(0,1) generator (initial subspace of CheFSI):
//   mix64      SplitMix64 finaliser (Steele, Lea & Flood 2014)
//   key        = mix64(seed);  u64(c) = mix64(key + (c + 1) * 0x9E3779B97F4A7C15)
//   entry n:   q = n >> 1, u1 = ((u64(2q) >> 11) + 1) 2^-53, u2 = (u64(2q+1) >> 11) 2^-53,
//              x = sqrt(-2 ln u1) * (n even ? cos(2 pi u2) : sin(2 pi u2))   (Box-Muller)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

__device__ __forceinline__ double normal_entry(uint64_t key, uint64_t n) {
  const uint64_t q = n >> 1;
  const uint64_t a = mix64(key + (2 * q + 1) * 0x9E3779B97F4A7C15ull);
  const uint64_t b = mix64(key + (2 * q + 2) * 0x9E3779B97F4A7C15ull);
  const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(b >> 11) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  return (n & 1) ? r * sinpi(2.0 * u2) : r * cospi(2.0 * u2);
}

template <typename T>
__global__ void random_kernel(T* X, int64_t ld, int k, const int64_t* lex, int64_t n_slots, uint64_t key) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_slots * k) return;
  const int64_t s = idx / k;
  const int j = (int)(idx - s * k);
  const int64_t p = lex[s];
  X[s * ld + j] = p < 0 ? T(0) : (T)normal_entry(key, (uint64_t)p * (uint64_t)k + (uint64_t)j);
}

static uint64_t mix64_host(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

cudaError_t launch_random(const Ham& H, void* X, int64_t ld, int k, int dtype, uint64_t seed, cudaStream_t st) {
  const int64_t n = H.grid.n_slots * k;
  if (n == 0) return cudaSuccess;
  const uint64_t key = mix64_host(seed);
  if (dtype == KSCF_F64)
    random_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>((double*)X, ld, k, H.d_lex, H.grid.n_slots, key), count_launch();
  else
    random_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>((float*)X, ld, k, H.d_lex, H.grid.n_slots, key), count_launch();
  return cudaGetLastError();
}

// rho[s] = sum_{i < n_occ} f_i X[s][i]^2  (FP64 sums; one warp per slot)
template <typename T>
__global__ void density_kernel(const T* X, int64_t ld, int n_occ, const double* occ, int64_t n_slots,
                               double* rho) {
  const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= n_slots) return;
  double acc = 0.0;
  for (int i = lane; i < n_occ; i += 32) {
    const double x = (double)X[s * ld + i];
    acc += (occ ? occ[i] : 2.0) * x * x;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) rho[s] = acc;
}

// FP32 X: the same sum in double-float arithmetic (pairs of FP32 numbers, Dekker 1971),
// so that the FP64 pipe (about 1/70 of the FP32 rate on this part) only converts the final
// pair.  x^2 = p + e exactly (TwoProduct with an FMA); f = fh + fl (the FP64 occupation as
// an FP32 pair); each term fh p is split exactly, the small parts (fh e, fl p and the
// product error) are summed in FP32, the leading parts with Knuth's TwoSum.  Relative
// error about 2^-44 per slot, against ~2^-53 for plain FP64 sums.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__global__ void __launch_bounds__(256) density_f32_kernel(const float* __restrict__ X, int64_t ld, int n_occ,
                                                          const double* __restrict__ occ, int64_t n_slots,
                                                          double* __restrict__ rho) {
  extern __shared__ float fpair[];   // [n_occ] high parts, then [n_occ] low parts
  for (int i = threadIdx.x; i < n_occ; i += blockDim.x) {
    const double f = occ ? occ[i] : 2.0;
    const float fh = (float)f;
    fpair[i] = fh;
    fpair[n_occ + i] = (float)(f - (double)fh);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n_slots; s += nw) {
    const float* row = X + s * ld;
    float sh = 0.0f, sl = 0.0f;
    for (int i = lane; i < n_occ; i += 32) {
      const float x = row[i];
      const float p = x * x, pe = fmaf(x, x, -p);          // x^2 = p + pe
      const float fh = fpair[i], fl = fpair[n_occ + i];
      const float q = fh * p, qe = fmaf(fh, p, -q);         // fh p = q + qe
      float t, te;
      two_sum(sh, q, t, te);
      sh = t;
      sl += te + (qe + fmaf(fh, pe, fl * p));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
      float t, te;
      two_sum(sh, oh, t, te);
      sh = t;
      sl += te + ol;
    }
    if (lane == 0) rho[s] = (double)sh + (double)sl;
  }
}

// Layout conversions between a compact block (one row per grid point, lexicographic point
// order) and the slot layout; one warp per slot row.
template <typename T>
__global__ void points_to_slots_kernel(const T* __restrict__ P, int64_t ldp, T* __restrict__ X, int64_t ldx, int k,
                                       const int64_t* __restrict__ lex, int64_t n_slots) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= n_slots) return;
  const int64_t p = lex[s];
  T* x = X + s * ldx;
  if (p < 0) {
    for (int j = threadIdx.x & 31; j < k; j += 32) x[j] = T(0);
  } else {
    const T* src = P + p * ldp;
    for (int j = threadIdx.x & 31; j < k; j += 32) x[j] = src[j];
  }
}

template <typename T>
__global__ void slots_to_points_kernel(const T* __restrict__ X, int64_t ldx, T* __restrict__ P, int64_t ldp, int k,
                                       const int64_t* __restrict__ lex, int64_t n_slots) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= n_slots) return;
  const int64_t p = lex[s];
  if (p < 0) return;
  const T* x = X + s * ldx;
  T* dst = P + p * ldp;
  for (int j = threadIdx.x & 31; j < k; j += 32) dst[j] = x[j];
}

cudaError_t launch_points_slots(const Ham& H, bool to_slots, const void* src, int64_t lds, void* dst, int64_t ldd,
                                int k, int dtype, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  if (n == 0 || k == 0) return cudaSuccess;
  const unsigned grid = blocks_for(n * 32, 256);
  if (dtype == KSCF_F64) {
    if (to_slots)
      points_to_slots_kernel<double><<<grid, 256, 0, st>>>((const double*)src, lds, (double*)dst, ldd, k, H.d_lex, n),
          count_launch();
    else
      slots_to_points_kernel<double><<<grid, 256, 0, st>>>((const double*)src, lds, (double*)dst, ldd, k, H.d_lex, n),
          count_launch();
  } else {
    if (to_slots)
      points_to_slots_kernel<float><<<grid, 256, 0, st>>>((const float*)src, lds, (float*)dst, ldd, k, H.d_lex, n),
          count_launch();
    else
      slots_to_points_kernel<float><<<grid, 256, 0, st>>>((const float*)src, lds, (float*)dst, ldd, k, H.d_lex, n),
          count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_density(const Ham& H, const void* X, int64_t ld, int n_occ, int dtype, const double* occ,
                           double* rho, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  if (dtype == KSCF_F64) {
    density_kernel<double><<<blocks_for(n, 8), 256, 0, st>>>((const double*)X, ld, n_occ, occ, n, rho), count_launch();
  } else {
    // a few blocks per SM, each converting the occupations once
    const unsigned grid = (unsigned)std::min<int64_t>(blocks_for(n, 8), 152 * 8);
    const size_t smem = 2 * sizeof(float) * (size_t)std::max(n_occ, 1);
    if (smem > 48 * 1024) {
      static size_t attr = 0;
      if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(density_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
      }
    }
    density_f32_kernel<<<grid, 256, smem, st>>>((const float*)X, ld, n_occ, occ, n, rho), count_launch();
  }
  return cudaGetLastError();
}

}  // namespace kscf
