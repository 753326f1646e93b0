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
  const T* coef;  // (n_kb*4) rows of cld
  int64_t cld;
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
      const T* cf = a.coef + (int64_t)a.kb_atom[e] * 4 * a.cld + v;
      const T* ch = a.kb_chi + 4 * e;
      acc += ch[0] * cf[0] + ch[1] * cf[a.cld] + ch[2] * cf[2 * a.cld] + ch[3] * cf[3 * a.cld];
    }
    res = a.alpha * (acc - a.c * y);
    if (a.prev) res += a.beta * a.prev[s * a.ld_prev + v];
  }
  a.out[s * a.ld_out + v] = res;
}

// ---------------------------------------------------------------------------
// Brick kernel (FP32, 8^3 bricks): one CTA per (brick, 8 vectors).
//
// The brick's 512 rows (8 vectors = 32 B each) are copied into shared memory with
// asynchronous copies; the 37-point star is then evaluated as three line passes: a
// thread owns one line of 8 points along x, then y, then z, holds the 20 values of
// the line in registers (6 halo values read straight from the neighbour brick in
// global memory/L2, 8 from shared memory, 6 halo) and slides the 13-point 1D stencil
// over them.  The x and y passes leave partial sums in a shared accumulator, a
// parallel pass over the brick's nonlocal entries adds the projector scatter with
// shared-memory atomics, and the z pass adds the z terms, the local potential and
// the recurrence and writes the result.  Each lane handles two vectors with packed
// FP32x2 arithmetic.  Shared layout (32-byte point slots): core[z][y][x ^ (y & 3)]
// and acc with the same swizzle, conflict-free for all three passes.
namespace {
constexpr int SB_CORE = 0, SB_ACC = 512, SB_TOTAL = 1024;
constexpr int SB_SMEM_BYTES = SB_TOTAL * 32;

__device__ __forceinline__ int sb_core(int x, int y, int z) { return (z * 8 + y) * 8 + (x ^ (y & 3)); }

__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(*(uint64_t*)&a), "l"(*(uint64_t*)&b));
  return *(float2*)&r;
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(*(uint64_t*)&a), "l"(*(uint64_t*)&b), "l"(*(uint64_t*)&c));
  return *(float2*)&r;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(*(uint64_t*)&a), "l"(*(uint64_t*)&b));
  return *(float2*)&r;
}
__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }

// sum_k c_k (w[i+k] + w[i-k]) (+ 3 c_0 w[i]) for the line window w[0..19]
template <bool WITH_CENTRE>
__device__ __forceinline__ float2 line_terms(const float2* w, int i, const float* st) {
  float2 s = WITH_CENTRE ? f2_mul(f2(3.0f * st[0]), w[i]) : f2_mul(f2(st[1]), f2_add(w[i + 1], w[i - 1]));
  if (WITH_CENTRE) s = f2_fma(f2(st[1]), f2_add(w[i + 1], w[i - 1]), s);
#pragma unroll
  for (int k = 2; k <= 6; k++) s = f2_fma(f2(st[k]), f2_add(w[i + k], w[i - k]), s);
  return s;
}

// two vectors of row `slot` (VEC: one 8-byte load)
template <bool VEC>
__device__ __forceinline__ float2 ld2(const float* base, int64_t slot, int64_t ld, int vl) {
  const float* p = base + slot * ld + vl;
  if (VEC) return __ldg((const float2*)p);
  return make_float2(__ldg(p), __ldg(p + 1));
}
}  // namespace

// NV vectors per CTA (8 or 32): a point slot in shared memory is NV floats; the 64
// lines of a pass are spread over 64 * NV/2 threads, NV/2 lanes per line, two vectors
// per lane.  NV = 32 makes every halo load instruction cover two 128-byte row segments.
// VEC: rows are read with vector loads (ld and column offsets multiples of 4).
template <int NV, bool VEC>
__global__ void __launch_bounds__(NV * 32, NV == 8 ? 3 : 1)
    cheb_step_brick8(StepArgs<float> a, int nchunk, const uint16_t* __restrict__ entry_lslot) {
  constexpr int VPL = NV / 2;       // lanes per line
  constexpr int NT = 64 * VPL;      // threads
  constexpr int Q4 = NV / 4;        // float4 per point slot
  const int64_t cld = a.cld;
  extern __shared__ float4 sb4[];
  float* sm = (float*)sb4;
  const int brick = blockIdx.x / nchunk, chunk = blockIdx.x - (blockIdx.x / nchunk) * nchunk;
  const int v0 = chunk * NV;
  const int tid = threadIdx.x;
  const int vp = tid % VPL, line = tid / VPL;
  const int vl = v0 + 2 * vp;  // this lane's first vector
  const int64_t b0 = (int64_t)brick * 512;
  const int nbx0 = __ldg(a.nbr + (int64_t)brick * 6 + 0), nbx1 = __ldg(a.nbr + (int64_t)brick * 6 + 1);
  const int nby0 = __ldg(a.nbr + (int64_t)brick * 6 + 2), nby1 = __ldg(a.nbr + (int64_t)brick * 6 + 3);
  const int nbz0 = __ldg(a.nbr + (int64_t)brick * 6 + 4), nbz1 = __ldg(a.nbr + (int64_t)brick * 6 + 5);
  // point slot of (x, y, z): XOR swizzle for 32-byte slots, plain for 128-byte slots
  auto core = [](int x, int y, int z) { return NV == 8 ? sb_core(x, y, z) : (z * 8 + y) * 8 + x; };

  // ---- stage the brick core: 512 rows x NV floats ----
  for (int t = tid; t < 512 * Q4; t += NT) {
    const int r = t / Q4, part = t - (t / Q4) * Q4;
    const float* p = a.in + (b0 + r) * a.ld_in + v0 + part * 4;
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(&sb4[(SB_CORE + core(r & 7, (r >> 3) & 7, r >> 6)) * Q4 + part]);
    if (VEC) {
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(p) : "memory");
    } else {
#pragma unroll
      for (int q = 0; q < 4; q++) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d + 4 * q), "l"(p + q) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");

  const float2* s2 = (const float2*)sm + vp;  // point slot q -> s2[q * VPL]
  float2* a2 = (float2*)sm + vp;
  float st[7];
#pragma unroll
  for (int k = 0; k < 7; k++) st[k] = a.st[k];
  const float2 zero2 = make_float2(0.f, 0.f);

  // ---- x pass: line (y, z); halo rows lx = 2..7 of the -x brick and 0..5 of the +x brick ----
  {
    const int y = line & 7, z = line >> 3;
    float2 w[20];
#pragma unroll
    for (int xx = 0; xx < 6; xx++) {
      w[xx] = nbx0 >= 0 ? ld2<VEC>(a.in, (int64_t)nbx0 * 512 + (z * 8 + y) * 8 + 2 + xx, a.ld_in, vl) : zero2;
      w[14 + xx] = nbx1 >= 0 ? ld2<VEC>(a.in, (int64_t)nbx1 * 512 + (z * 8 + y) * 8 + xx, a.ld_in, vl) : zero2;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
#pragma unroll
    for (int x = 0; x < 8; x++) w[6 + x] = s2[(SB_CORE + core(x, y, z)) * VPL];
#pragma unroll
    for (int x = 0; x < 8; x++) a2[(SB_ACC + core(x, y, z)) * VPL] = line_terms<true>(w, 6 + x, st);
  }
  // ---- y pass: line (x, z) ----
  {
    const int x = line & 7, z = line >> 3;
    float2 w[20];
#pragma unroll
    for (int yy = 0; yy < 6; yy++) {
      w[yy] = nby0 >= 0 ? ld2<VEC>(a.in, (int64_t)nby0 * 512 + (z * 8 + 2 + yy) * 8 + x, a.ld_in, vl) : zero2;
      w[14 + yy] = nby1 >= 0 ? ld2<VEC>(a.in, (int64_t)nby1 * 512 + (z * 8 + yy) * 8 + x, a.ld_in, vl) : zero2;
    }
#pragma unroll
    for (int y = 0; y < 8; y++) w[6 + y] = s2[(SB_CORE + core(x, y, z)) * VPL];
    __syncthreads();  // x-pass accumulator writes are visible
#pragma unroll
    for (int y = 0; y < 8; y++) {
      const int q = (SB_ACC + core(x, y, z)) * VPL;
      a2[q] = f2_add(a2[q], line_terms<false>(w, 6 + y, st));
    }
  }
  __syncthreads();
  // ---- nonlocal scatter: the brick's entries are one contiguous range ----
  {
    const int64_t e0 = __ldg(a.kb_ptr + b0), e1 = __ldg(a.kb_ptr + b0 + 512);
    for (int64_t e = e0 + line; e < e1; e += 64) {
      const int ls = __ldg(entry_lslot + e);
      const float4 ch = __ldg((const float4*)(a.kb_chi + 4 * e));
      const float* cf = a.coef + (int64_t)__ldg(a.kb_atom + e) * 4 * cld + vl;
      float2 c = f2_mul(f2(ch.x), make_float2(cf[0], cf[1]));
      c = f2_fma(f2(ch.y), make_float2(cf[cld], cf[cld + 1]), c);
      c = f2_fma(f2(ch.z), make_float2(cf[2 * cld], cf[2 * cld + 1]), c);
      c = f2_fma(f2(ch.w), make_float2(cf[3 * cld], cf[3 * cld + 1]), c);
      float* acc = (float*)&a2[(SB_ACC + core(ls & 7, (ls >> 3) & 7, ls >> 6)) * VPL];
      atomicAdd(acc, c.x);
      atomicAdd(acc + 1, c.y);
    }
  }
  // ---- z pass: line (x, y); potential, recurrence, store ----
  {
    const int x = line & 7, y = line >> 3;
    float2 w[20];
#pragma unroll
    for (int zz = 0; zz < 6; zz++) {
      w[zz] = nbz0 >= 0 ? ld2<VEC>(a.in, (int64_t)nbz0 * 512 + (2 + zz) * 64 + y * 8 + x, a.ld_in, vl) : zero2;
      w[14 + zz] = nbz1 >= 0 ? ld2<VEC>(a.in, (int64_t)nbz1 * 512 + zz * 64 + y * 8 + x, a.ld_in, vl) : zero2;
    }
#pragma unroll
    for (int z = 0; z < 8; z++) w[6 + z] = s2[(SB_CORE + core(x, y, z)) * VPL];
    __syncthreads();  // scatter atomics are complete
    const bool st0 = vl < a.w, st1 = vl + 1 < a.w;
    const float2 alpha = f2(a.alpha), beta = f2(a.beta), negc = f2(-a.c);
#pragma unroll
    for (int z = 0; z < 8; z++) {
      const int64_t s = b0 + z * 64 + y * 8 + x;
      float2 res = zero2;
      if (__ldg(a.mask + s)) {
        const float2 yc = w[6 + z];
        float2 hy = f2_add(a2[(SB_ACC + core(x, y, z)) * VPL], line_terms<false>(w, 6 + z, st));
        hy = f2_fma(f2(__ldg(a.V + s)), yc, hy);
        res = f2_mul(alpha, f2_fma(negc, yc, hy));
        if (a.prev) {
          const float2 pv = VEC ? *(const float2*)(a.prev + s * a.ld_prev + vl)
                                : make_float2(a.prev[s * a.ld_prev + vl], a.prev[s * a.ld_prev + vl + 1]);
          res = f2_fma(beta, pv, res);
        }
      }
      float* o = a.out + s * a.ld_out + vl;
      if (st0 && st1 && VEC) {
        *(float2*)o = res;
      } else {
        if (st0) o[0] = res.x;
        if (st1) o[1] = res.y;
      }
    }
  }
}

// coef[(a*4+l)*w + v] = E_l h^3 sum_{entries e of atom a} chi_l(e) Y[slot_e][v]
template <typename T>
__global__ void __launch_bounds__(256) kb_gather_kernel(const T* __restrict__ Y, int64_t ld, int w, int64_t cld,
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
    coef[((int64_t)at * 4 + l) * cld + v] = (T)energy[4 * at + l] * sum;
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

cudaError_t launch_kb_gather(const Ham& H, const void* Y, int64_t ld, int w, int dtype, void* coef, int64_t cld,
                             cudaStream_t st) {
  if (H.n_kb == 0 || w == 0) return cudaSuccess;
  dim3 grid(H.n_kb, (w + 31) / 32), block(32, 8);
  if (dtype == KSCF_F64)
    kb_gather_kernel<double><<<grid, block, 0, st>>>((const double*)Y, ld, w, cld, H.d_kb_atom_ptr,
                                                     H.d_kb_atom_slot, H.d_kb_atom_chi64,
                                                     H.d_kb_energy, (double*)coef), count_launch();
  else
    kb_gather_kernel<float><<<grid, block, 0, st>>>((const float*)Y, ld, w, cld, H.d_kb_atom_ptr,
                                                    H.d_kb_atom_slot, H.d_kb_atom_chi32,
                                                    H.d_kb_energy, (float*)coef), count_launch();
  return cudaGetLastError();
}

static bool g_brick_attr[64] = {false};

template <typename T>
static cudaError_t step_t(const Ham& H, const void* in, int64_t ld_in, const void* prev, int64_t ld_prev,
                          void* out, int64_t ld_out, int w, int wavail, double alpha, double beta, double c,
                          const void* coef, int64_t cld, const T* V, const T* chi, cudaStream_t st) {
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
  a.cld = cld;
  a.V = V;
  a.nbr = H.d_nbr;
  a.mask = H.d_mask;
  a.kb_ptr = H.d_kb_slot_ptr;
  a.kb_atom = H.d_kb_slot_atom;
  a.kb_chi = chi;
  for (int k = 0; k < 7; k++) a.st[k] = (T)H.stencil[k];
  a.n_slots = H.grid.n_slots;
  const int w8 = (w + 7) / 8 * 8;
  if (sizeof(T) == 4 && H.grid.B == 8 && wavail >= w8 && cld >= w8 && cld % 2 == 0) {
    // brick kernel: every row chunk it touches lies inside the first w8 columns
    const bool wide = w >= 32 && wavail >= (w + 31) / 32 * 32 && cld >= (w + 31) / 32 * 32;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !g_brick_attr[dev]) {
      cudaError_t e = cudaFuncSetAttribute(cheb_step_brick8<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           SB_TOTAL * 128);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cheb_step_brick8<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SB_TOTAL * 128);
      if (e != cudaSuccess) return e;
      g_brick_attr[dev] = true;
    }
    const bool vec = (ld_in % 4 == 0) && (ld_out % 4 == 0) && (!prev || ld_prev % 4 == 0) && (cld % 2 == 0) &&
                     ((uintptr_t)in % 16 == 0) && ((uintptr_t)out % 16 == 0) &&
                     (!prev || (uintptr_t)prev % 16 == 0);
    StepArgs<float>& af = *reinterpret_cast<StepArgs<float>*>(&a);
    if (wide) {
      const int nchunk = (w + 31) / 32;
      const unsigned grid = (unsigned)(H.grid.n_bricks * nchunk);
      if (vec)
        cheb_step_brick8<32, true><<<grid, 1024, SB_TOTAL * 128, st>>>(af, nchunk, H.d_kb_entry_lslot), count_launch();
      else
        cheb_step_brick8<32, false><<<grid, 1024, SB_TOTAL * 128, st>>>(af, nchunk, H.d_kb_entry_lslot), count_launch();
    } else {
      const int nchunk = w8 / 8;
      const unsigned grid = (unsigned)(H.grid.n_bricks * nchunk);
      if (vec)
        cheb_step_brick8<8, true><<<grid, 256, SB_TOTAL * 32, st>>>(af, nchunk, H.d_kb_entry_lslot), count_launch();
      else
        cheb_step_brick8<8, false><<<grid, 256, SB_TOTAL * 32, st>>>(af, nchunk, H.d_kb_entry_lslot), count_launch();
    }
    return cudaGetLastError();
  }
  const int64_t n = a.n_slots * w;
  if (H.grid.B == 8)
    cheb_step_generic<T, 8><<<blocks_for(n, 256), 256, 0, st>>>(a), count_launch();
  else
    cheb_step_generic<T, 16><<<blocks_for(n, 256), 256, 0, st>>>(a), count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cheb_step(const Ham& H, const void* in, int64_t ld_in, const void* prev, int64_t ld_prev,
                             void* out, int64_t ld_out, int w, int wavail, int dtype, double alpha, double beta,
                             double c, const void* coef, int64_t cld, cudaStream_t st) {
  if (dtype == KSCF_F64)
    return step_t<double>(H, in, ld_in, prev, ld_prev, out, ld_out, w, wavail, alpha, beta, c, coef, cld,
                          H.d_v64, H.d_kb_slot_chi64, st);
  return step_t<float>(H, in, ld_in, prev, ld_prev, out, ld_out, w, wavail, alpha, beta, c, coef, cld, H.d_v32,
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
