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
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

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

// NV vectors per CTA (8 or 16): a point slot in shared memory is NV floats; the 64 lines
// of a pass are spread over 64 * NV/2 threads, NV/2 lanes per line, two vectors per lane.
// The point slots are XOR-swizzled so that the lines of one warp read distinct banks in
// every pass (x ^ (y & 3) for 32-byte slots, x ^ (y & 1) for 64-byte slots).
// VEC: rows are read with vector loads (ld and column offsets multiples of 4).
template <int NV, bool VEC>
__global__ void __launch_bounds__(NV * 32, NV == 8 ? 3 : 2)
    cheb_step_brick8(StepArgs<float> a, int nchunk, const uint16_t* __restrict__ entry_lslot) {
  static_assert(NV == 8 || NV == 16, "point slots of 32 or 64 bytes");
  constexpr int VPL = NV / 2;       // lanes per line
  constexpr int NT = 64 * VPL;      // threads
  constexpr int Q4 = NV / 4;        // float4 per point slot
  const int64_t cld = a.cld;
  extern __shared__ float4 sb4[];
  float* sm = (float*)sb4;
  // brick-major order: CTAs follow the Hilbert order of the bricks, the column chunks of
  // one brick side by side (neighbouring bricks, and so the halo rows, stay close in L2)
  const int brick = blockIdx.x / nchunk, chunk = blockIdx.x - (blockIdx.x / nchunk) * nchunk;
  const int v0 = chunk * NV;
  const int tid = threadIdx.x;
  const int vp = tid % VPL, line = tid / VPL;
  const int vl = v0 + 2 * vp;  // this lane's first vector
  const int64_t b0 = (int64_t)brick * 512;
  const int nbx0 = __ldg(a.nbr + (int64_t)brick * 6 + 0), nbx1 = __ldg(a.nbr + (int64_t)brick * 6 + 1);
  const int nby0 = __ldg(a.nbr + (int64_t)brick * 6 + 2), nby1 = __ldg(a.nbr + (int64_t)brick * 6 + 3);
  const int nbz0 = __ldg(a.nbr + (int64_t)brick * 6 + 4), nbz1 = __ldg(a.nbr + (int64_t)brick * 6 + 5);
  auto core = [](int x, int y, int z) { return NV == 8 ? sb_core(x, y, z) : (z * 8 + y) * 8 + (x ^ (y & 1)); };

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
  // ---- nonlocal scatter: the brick's entries are one contiguous range; four entries
  //      per thread and iteration, their loads issued before any is used ----
  {
    const int64_t e0 = __ldg(a.kb_ptr + b0), e1 = __ldg(a.kb_ptr + b0 + 512);
    for (int64_t eb = e0 + line; eb < e1; eb += 4 * 64) {
      int ls[4];
      float4 ch[4];
      const float* cf[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int64_t e = eb + u * 64;
        const bool ok = e < e1;
        ls[u] = ok ? __ldg(entry_lslot + e) : -1;
        ch[u] = ok ? __ldg((const float4*)(a.kb_chi + 4 * e)) : make_float4(0.f, 0.f, 0.f, 0.f);
        cf[u] = a.coef + (ok ? (int64_t)__ldg(a.kb_atom + e) * 4 * cld : 0) + vl;
      }
      float2 cv[4][4];
#pragma unroll
      for (int u = 0; u < 4; u++)
#pragma unroll
        for (int l = 0; l < 4; l++) cv[u][l] = make_float2(cf[u][l * cld], cf[u][l * cld + 1]);
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (ls[u] < 0) continue;
        float2 c = f2_mul(f2(ch[u].x), cv[u][0]);
        c = f2_fma(f2(ch[u].y), cv[u][1], c);
        c = f2_fma(f2(ch[u].z), cv[u][2], c);
        c = f2_fma(f2(ch[u].w), cv[u][3], c);
        float* acc = (float*)&a2[(SB_ACC + core(ls[u] & 7, (ls[u] >> 3) & 7, ls[u] >> 6)) * VPL];
        atomicAdd(acc, c.x);
        atomicAdd(acc + 1, c.y);
      }
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
      // padding rows are left untouched: they are zero in every buffer of the recurrence
      if (!__ldg(a.mask + s)) continue;
      const float2 yc = w[6 + z];
      float2 hy = f2_add(a2[(SB_ACC + core(x, y, z)) * VPL], line_terms<false>(w, 6 + z, st));
      hy = f2_fma(f2(__ldg(a.V + s)), yc, hy);
      float2 res = f2_mul(alpha, f2_fma(negc, yc, hy));
      if (a.prev) {
        const float2 pv = VEC ? *(const float2*)(a.prev + s * a.ld_prev + vl)
                              : make_float2(a.prev[s * a.ld_prev + vl], a.prev[s * a.ld_prev + vl + 1]);
        res = f2_fma(beta, pv, res);
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

// ---------------------------------------------------------------------------
// Wide brick kernel (FP32, 8^3 bricks): one CTA per (brick, NV = 16 or 32 vectors),
// NV/4 lanes per line and four vectors per lane (16-byte loads and stores), so that
// every address computation, load and store serves four vectors.  Same three line passes
// as the kernel above; in addition, every neighbour brick gets one 64-bit base pointer
// per CTA and rows inside a brick are addressed with 32-bit offsets; halo loads are
// branch-free (a missing neighbour is read from this brick and the value discarded);
// padding rows of the core are zero-filled instead of read.  Shared memory: core and
// accumulator, 512 point slots of 4*NV bytes each (NV = 32: a line's eight lanes cover all
// 32 banks; NV = 16: slots XOR-swizzled like the 16-vector kernel above).  NV = 16 fits two
// CTAs per SM at 128 registers, so that one CTA's loads overlap the other's arithmetic.
namespace {
__device__ __forceinline__ float4 f4_add(float4 a, float4 b) {
  const float2 lo = f2_add(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 hi = f2_add(make_float2(a.z, a.w), make_float2(b.z, b.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
// c * a + b (c broadcast)
__device__ __forceinline__ float4 f4_fma(float2 c, float4 a, float4 b) {
  const float2 lo = f2_fma(c, make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 hi = f2_fma(c, make_float2(a.z, a.w), make_float2(b.z, b.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float4 f4_mul(float2 c, float4 a) {
  const float2 lo = f2_mul(c, make_float2(a.x, a.y));
  const float2 hi = f2_mul(c, make_float2(a.z, a.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
template <bool WITH_CENTRE>
__device__ __forceinline__ float4 line_terms4(const float4* w, int i, const float2* c2) {
  float4 s = WITH_CENTRE ? f4_mul(c2[0], w[i]) : f4_mul(c2[1], f4_add(w[i + 1], w[i - 1]));
  if (WITH_CENTRE) s = f4_fma(c2[1], f4_add(w[i + 1], w[i - 1]), s);
#pragma unroll
  for (int k = 2; k <= 6; k++) s = f4_fma(c2[k], f4_add(w[i + k], w[i - k]), s);
  return s;
}
__device__ __forceinline__ float4 ld4(const float* p) { return __ldg((const float4*)p); }
}  // namespace

template <int NV>
__global__ void __launch_bounds__(NV * 16, NV == 16 ? 2 : 1)
    cheb_step_brick8w(StepArgs<float> a, int nchunk, const uint16_t* __restrict__ entry_lslot) {
  static_assert(NV == 16 || NV == 32, "16 or 32 vectors per CTA");
  constexpr int VPL = NV / 4;   // lanes per line (four vectors each)
  extern __shared__ float4 sw4[];
  float4* core4 = sw4;                // [512][VPL]
  float4* acc4 = sw4 + 512 * VPL;     // [512][VPL]
  // 64-byte point slots (NV = 16): x ^ (y & 1) keeps the lines of a warp on distinct banks
  auto sl = [](int x, int y, int z) { return (z * 8 + y) * 8 + (NV == 16 ? (x ^ (y & 1)) : x); };
  const int brick = blockIdx.x / nchunk, chunk = blockIdx.x - (blockIdx.x / nchunk) * nchunk;
  const int tid = threadIdx.x, vp = tid % VPL, line = tid / VPL;
  const int vl = chunk * NV + 4 * vp;
  const int64_t b0 = (int64_t)brick * 512;
  const int ld = (int)a.ld_in;  // 512 * ld < 2^31 (checked by the launcher)
  const float* __restrict__ in = a.in;
  const float* own = in + b0 * a.ld_in + vl;
  const float* nbp[6];
  bool nbv[6];
#pragma unroll
  for (int f = 0; f < 6; f++) {
    const int q = __ldg(a.nbr + b0 / 512 * 6 + f);
    nbv[f] = q >= 0;
    nbp[f] = q >= 0 ? in + (int64_t)q * 512 * a.ld_in + vl : own;
  }
  // ---- core: 512 rows x 128 bytes, padding rows zero-filled ----
  {
    const float* src = in + b0 * a.ld_in + chunk * NV + 4 * vp;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const int r = line + 64 * i;
      const uint32_t live = __ldg(a.mask + b0 + r);
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(&core4[sl(r & 7, (r >> 3) & 7, r >> 6) * VPL + vp]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src + r * ld), "r"(live ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  // z-pass operands of this thread's (x, y) line
  const int zx = line & 7, zy = line >> 3;
  float vv[8];
  uint32_t mk = 0;
#pragma unroll
  for (int z = 0; z < 8; z++) {
    const int64_t s = b0 + z * 64 + zy * 8 + zx;
    mk |= (uint32_t)__ldg(a.mask + s) << z;
    vv[z] = __ldg(a.V + s);
  }
  float2 c2[7];
  c2[0] = f2(3.0f * a.st[0]);
#pragma unroll
  for (int k = 1; k < 7; k++) c2[k] = f2(a.st[k]);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

  // ---- x pass: line (y, z) ----
  {
    const int y = line & 7, z = line >> 3;
    const int rb = ((z * 8 + y) * 8) * ld;
    float4 w[20];
#pragma unroll
    for (int xx = 0; xx < 6; xx++) {
      const float4 m = ld4(nbp[0] + rb + (2 + xx) * ld);
      const float4 p = ld4(nbp[1] + rb + xx * ld);
      w[xx] = nbv[0] ? m : z4;
      w[14 + xx] = nbv[1] ? p : z4;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
#pragma unroll
    for (int x = 0; x < 8; x++) w[6 + x] = core4[sl(x, y, z) * VPL + vp];
#pragma unroll
    for (int x = 0; x < 8; x++) acc4[sl(x, y, z) * VPL + vp] = line_terms4<true>(w, 6 + x, c2);
  }
  // ---- y pass: line (x, z) ----
  {
    const int x = line & 7, z = line >> 3;
    float4 w[20];
#pragma unroll
    for (int yy = 0; yy < 6; yy++) {
      const float4 m = ld4(nbp[2] + ((z * 8 + 2 + yy) * 8 + x) * ld);
      const float4 p = ld4(nbp[3] + ((z * 8 + yy) * 8 + x) * ld);
      w[yy] = nbv[2] ? m : z4;
      w[14 + yy] = nbv[3] ? p : z4;
    }
#pragma unroll
    for (int y = 0; y < 8; y++) w[6 + y] = core4[sl(x, y, z) * VPL + vp];
    __syncthreads();  // x-pass accumulator writes are visible
#pragma unroll
    for (int y = 0; y < 8; y++) {
      const int q = sl(x, y, z) * VPL + vp;
      acc4[q] = f4_add(acc4[q], line_terms4<false>(w, 6 + y, c2));
    }
  }
  __syncthreads();
  // ---- nonlocal scatter over the brick's contiguous entry range ----
  {
    const int64_t cld = a.cld;
    const int64_t e0 = __ldg(a.kb_ptr + b0), e1 = __ldg(a.kb_ptr + b0 + 512);
    for (int64_t eb = e0 + line; eb < e1; eb += 2 * 64) {
      int ls[2];
      float4 ch[2];
      const float* cf[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int64_t e = eb + u * 64;
        const bool ok = e < e1;
        ls[u] = ok ? __ldg(entry_lslot + e) : -1;
        ch[u] = ok ? __ldg((const float4*)(a.kb_chi + 4 * e)) : z4;
        cf[u] = a.coef + (ok ? (int64_t)__ldg(a.kb_atom + e) * 4 * cld : 0) + vl;
      }
      float4 cv[2][4];
#pragma unroll
      for (int u = 0; u < 2; u++)
#pragma unroll
        for (int l = 0; l < 4; l++) cv[u][l] = ld4(cf[u] + l * cld);
#pragma unroll
      for (int u = 0; u < 2; u++) {
        if (ls[u] < 0) continue;
        float4 c = f4_mul(f2(ch[u].x), cv[u][0]);
        c = f4_fma(f2(ch[u].y), cv[u][1], c);
        c = f4_fma(f2(ch[u].z), cv[u][2], c);
        c = f4_fma(f2(ch[u].w), cv[u][3], c);
        float* acc = (float*)&acc4[sl(ls[u] & 7, (ls[u] >> 3) & 7, ls[u] >> 6) * VPL + vp];
        atomicAdd(acc, c.x);
        atomicAdd(acc + 1, c.y);
        atomicAdd(acc + 2, c.z);
        atomicAdd(acc + 3, c.w);
      }
    }
  }
  // ---- z pass: line (x, y); potential, recurrence, store ----
  {
    const int x = zx, y = zy;
    float4 w[20];
#pragma unroll
    for (int zz = 0; zz < 6; zz++) {
      const float4 m = ld4(nbp[4] + ((2 + zz) * 64 + y * 8 + x) * ld);
      const float4 p = ld4(nbp[5] + (zz * 64 + y * 8 + x) * ld);
      w[zz] = nbv[4] ? m : z4;
      w[14 + zz] = nbv[5] ? p : z4;
    }
#pragma unroll
    for (int z = 0; z < 8; z++) w[6 + z] = core4[sl(x, y, z) * VPL + vp];
    __syncthreads();  // scatter atomics are complete
    const bool full = vl + 3 < a.w;
    const float2 alpha = f2(a.alpha), beta = f2(a.beta), negc = f2(-a.c);
    const float* prevp = a.prev ? a.prev + b0 * a.ld_prev + vl : nullptr;
    float* outp = a.out + b0 * a.ld_out + vl;
    const int ldp = (int)a.ld_prev, ldo = (int)a.ld_out;
#pragma unroll
    for (int z = 0; z < 8; z++) {
      const int r = z * 64 + y * 8 + x;
      // padding rows are left untouched: they are zero in every buffer of the recurrence
      if (!((mk >> z) & 1u)) continue;
      const float4 yc = w[6 + z];
      float4 hy = f4_add(acc4[sl(x, y, z) * VPL + vp], line_terms4<false>(w, 6 + z, c2));
      hy = f4_fma(f2(vv[z]), yc, hy);
      float4 res = f4_mul(alpha, f4_fma(negc, yc, hy));
      if (prevp) {
        // plain load: prev may be the output buffer (read here, then written by this thread)
        const float4 pv = *(const float4*)(prevp + r * ldp);
        res = f4_fma(beta, pv, res);
      }
      float* o = outp + r * ldo;
      if (full) {
        *(float4*)o = res;
      } else {
        if (vl < a.w) o[0] = res.x;
        if (vl + 1 < a.w) o[1] = res.y;
        if (vl + 2 < a.w) o[2] = res.z;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// TMA brick kernel (FP32, 8^3 bricks, 8 vectors per CTA): the wavefunction block is
// viewed as a 5D tensor [brick][z][y][x][column] and the Tensor Memory Accelerator
// copies the six 6-deep neighbour faces (one box each) into shared memory, densely
// (no swizzle); the x faces use a view with x and y exchanged so that they land as
// [z][x][y] and the x pass reads them without bank conflicts.  Boxes of missing
// neighbours use an out-of-range brick coordinate and arrive zero-filled.  The brick
// core is copied with cp.async into the XOR-swizzled layout of the kernel above.  All
// stencil reads then come from shared memory; the line passes, the nonlocal scatter
// and the fused recurrence are those of the kernel above.
struct BrickMaps {
  CUtensorMap fx;  // view [brick][z][x][y][col], box {8, 8 y, 6 x, 8 z, 1}
  CUtensorMap fy;  // view [brick][z][y][x][col], box {8, 8 x, 6 y, 8 z, 1}
  CUtensorMap fz;  // view [brick][z][y][x][col], box {8, 8 x, 8 y, 6 z, 1}
};

__device__ unsigned int g_filter_status;  // set when a bounded wait gave up

namespace {
constexpr int TB_CORE = 0, TB_FXM = 16384, TB_FXP = TB_FXM + 12288, TB_FYM = TB_FXP + 12288,
              TB_FYP = TB_FYM + 12288, TB_FZM = TB_FYP + 12288, TB_FZP = TB_FZM + 12288,
              TB_ACC = TB_FZP + 12288, TB_BAR = TB_ACC + 16384, TB_BYTES = TB_BAR + 64;
constexpr uint32_t TB_TX = 6 * 12288;        // bytes the TMA delivers per CTA
constexpr int TB_SMEM = TB_BYTES + 1024;      // + alignment slack

__device__ __forceinline__ void tma_load5(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}
}  // namespace

template <int dummy>
__global__ void __launch_bounds__(256, 2)
    cheb_step_tma8(StepArgs<float> a, const __grid_constant__ BrickMaps maps, int nchunk, int n_bricks,
                   int64_t wavail_prev, int core_cols, const uint16_t* __restrict__ entry_lslot) {
  extern __shared__ uint8_t tb_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)tb_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
  uint64_t* bar = (uint64_t*)(sm + TB_BAR);
  const int64_t cld = a.cld;
  const int brick = blockIdx.x / nchunk, chunk = blockIdx.x - (blockIdx.x / nchunk) * nchunk;
  const int v0 = chunk * 8;
  const int tid = threadIdx.x;
  const int vp = tid & 3, line = tid >> 2;
  const int vl = v0 + 2 * vp;
  const int64_t b0 = (int64_t)brick * 512;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(TB_TX) : "memory");
    const int32_t* nb = a.nbr + (int64_t)brick * 6;
    auto nbc = [&](int f) { const int q = __ldg(nb + f); return q >= 0 ? q : n_bricks; };  // OOB -> zeros
    tma_load5(sbase + TB_FXM, &maps.fx, v0, 0, 2, 0, nbc(0), b);
    tma_load5(sbase + TB_FXP, &maps.fx, v0, 0, 0, 0, nbc(1), b);
    tma_load5(sbase + TB_FYM, &maps.fy, v0, 0, 2, 0, nbc(2), b);
    tma_load5(sbase + TB_FYP, &maps.fy, v0, 0, 0, 0, nbc(3), b);
    tma_load5(sbase + TB_FZM, &maps.fz, v0, 0, 0, 2, nbc(4), b);
    tma_load5(sbase + TB_FZP, &maps.fz, v0, 0, 0, 0, nbc(5), b);
  }
  // brick core: 512 rows x 32 B into the XOR-swizzled layout (asynchronous copies)
  for (int t = tid; t < 1024; t += 256) {
    const int r = t >> 1, half = t & 1;
    const bool live = v0 + half * 4 < core_cols;  // columns past the block arrive as zeros
    const float* p = live ? a.in + (b0 + r) * a.ld_in + v0 + half * 4 : a.in;
    const uint32_t d = sbase + TB_CORE + (uint32_t)(sb_core(r & 7, (r >> 3) & 7, r >> 6) * 32 + half * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(p), "r"(live ? 16 : 0) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  // z-pass operands are fetched while the copies are in flight
  const int zx = line & 7, zy = line >> 3;
  float2 pv[8];
  float vv[8];
  uint32_t mk = 0;
  const bool pv_ok = vl + 1 < wavail_prev;
#pragma unroll
  for (int z = 0; z < 8; z++) {
    const int64_t s = b0 + z * 64 + zy * 8 + zx;
    mk |= (uint32_t)__ldg(a.mask + s) << z;
    vv[z] = __ldg(a.V + s);
    pv[z] = (a.prev && pv_ok && ((mk >> z) & 1u)) ? *(const float2*)(a.prev + s * a.ld_prev + vl)
                                                  : make_float2(0.f, 0.f);
  }
  {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    uint32_t done = 0;
    for (uint32_t it = 0; it < (1u << 22) && !done; it++) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(b)
          : "memory");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!done) {
      atomicOr(&g_filter_status, 1u);
      return;
    }
  }
  __syncthreads();  // core copies of all threads have landed
  auto rd = [&](int region, int point) -> float2 { return *(const float2*)(sm + region + point * 32 + 8 * vp); };
  auto rc = [&](int x, int y, int z) -> float2 { return *(const float2*)(sm + TB_CORE + sb_core(x, y, z) * 32 + 8 * vp); };
  float2* a2 = (float2*)(sm + TB_ACC) + vp;
  float st[7];
#pragma unroll
  for (int k = 0; k < 7; k++) st[k] = a.st[k];

  // ---- x pass: line (y, z) ----
  {
    const int y = line & 7, z = line >> 3;
    float2 w[20];
#pragma unroll
    for (int xx = 0; xx < 6; xx++) {
      w[xx] = rd(TB_FXM, (z * 6 + xx) * 8 + y);
      w[14 + xx] = rd(TB_FXP, (z * 6 + xx) * 8 + y);
    }
#pragma unroll
    for (int x = 0; x < 8; x++) w[6 + x] = rc(x, y, z);
#pragma unroll
    for (int x = 0; x < 8; x++) a2[sb_core(x, y, z) * 4] = line_terms<true>(w, 6 + x, st);
  }
  __syncthreads();
  // ---- y pass: line (x, z) ----
  {
    const int x = line & 7, z = line >> 3;
    float2 w[20];
#pragma unroll
    for (int yy = 0; yy < 6; yy++) {
      w[yy] = rd(TB_FYM, (z * 6 + yy) * 8 + x);
      w[14 + yy] = rd(TB_FYP, (z * 6 + yy) * 8 + x);
    }
#pragma unroll
    for (int y = 0; y < 8; y++) w[6 + y] = rc(x, y, z);
#pragma unroll
    for (int y = 0; y < 8; y++) {
      const int q = sb_core(x, y, z) * 4;
      a2[q] = f2_add(a2[q], line_terms<false>(w, 6 + y, st));
    }
  }
  __syncthreads();
  // ---- nonlocal scatter over the brick's contiguous entry range ----
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
      float* acc = (float*)&a2[sb_core(ls & 7, (ls >> 3) & 7, ls >> 6) * 4];
      atomicAdd(acc, c.x);
      atomicAdd(acc + 1, c.y);
    }
  }
  __syncthreads();
  // ---- z pass: line (x, y) ----
  {
    const int x = zx, y = zy;
    float2 w[20];
#pragma unroll
    for (int zz = 0; zz < 6; zz++) {
      w[zz] = rd(TB_FZM, (zz * 8 + y) * 8 + x);
      w[14 + zz] = rd(TB_FZP, (zz * 8 + y) * 8 + x);
    }
#pragma unroll
    for (int z = 0; z < 8; z++) w[6 + z] = rc(x, y, z);
    const bool st0 = vl < a.w, st1 = vl + 1 < a.w;
    const float2 alpha = f2(a.alpha), beta = f2(a.beta), negc = f2(-a.c);
#pragma unroll
    for (int z = 0; z < 8; z++) {
      const int64_t s = b0 + z * 64 + y * 8 + x;
      // padding rows are left untouched: they are zero in every buffer of the recurrence
      if (!((mk >> z) & 1u)) continue;
      const float2 yc = w[6 + z];
      float2 hy = f2_add(a2[sb_core(x, y, z) * 4], line_terms<false>(w, 6 + z, st));
      hy = f2_fma(f2(vv[z]), yc, hy);
      const float2 res = f2_fma(beta, pv[z], f2_mul(alpha, f2_fma(negc, yc, hy)));
      float* o = a.out + s * a.ld_out + vl;
      if (st0 && st1) {
        *(float2*)o = res;
      } else if (st0) {
        o[0] = res.x;
      }
    }
  }
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t encode_brick_maps(BrickMaps* m, const float* base, int64_t ld, int64_t cols, int64_t n_bricks) {
  std::call_once(g_encode_once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) return cudaErrorNotSupported;
  const cuuint64_t dims[5] = {(cuuint64_t)cols, 8, 8, 8, (cuuint64_t)n_bricks};
  const cuuint64_t row = (cuuint64_t)ld * 4;
  // x faces: dims (col, y, x, z, brick); y and z faces: dims (col, x, y, z, brick)
  const cuuint64_t str_xy[4] = {row * 8, row, row * 64, row * 512};
  const cuuint64_t str_n[4] = {row, row * 8, row * 64, row * 512};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const cuuint32_t box_x[5] = {8, 8, 6, 8, 1}, box_y[5] = {8, 8, 6, 8, 1}, box_z[5] = {8, 8, 8, 6, 1};
  struct Spec {
    CUtensorMap* map;
    const cuuint64_t* str;
    const cuuint32_t* box;
  } spec[3] = {{&m->fx, str_xy, box_x}, {&m->fy, str_n, box_y}, {&m->fz, str_n, box_z}};
  for (int i = 0; i < 3; i++) {
    CUresult r = g_encode(spec[i].map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, (void*)base, dims, spec[i].str,
                          spec[i].box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}
bool g_tma_attr[64] = {false};
}  // namespace

cudaError_t filter_status(bool reset, unsigned int* status) {
  cudaError_t e = cudaMemcpyFromSymbol(status, g_filter_status, sizeof(unsigned int));
  if (e == cudaSuccess && reset && *status) {
    unsigned int z = 0;
    e = cudaMemcpyToSymbol(g_filter_status, &z, sizeof(unsigned int));
  }
  return e;
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

// one warp per row: coalesced 128-byte stores, no per-element division
template <typename T>
__global__ void zero_rows_kernel(T* X, int64_t ld, int k, const int64_t* pad, int64_t n_pad) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= n_pad) return;
  T* row = X + pad[r] * ld;
  for (int j = threadIdx.x & 31; j < k; j += 32) row[j] = T(0);
}

template <typename T>
__global__ void copy_cols_kernel(const T* src, int64_t ld_src, T* dst, int64_t ld_dst, int64_t rows, int w) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  const T* s = src + r * ld_src;
  T* d = dst + r * ld_dst;
  for (int j = threadIdx.x & 31; j < w; j += 32) d[j] = s[j];
}

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// one warp per slot: sets *flag when a domain row holds a NaN or Inf in its first k values
template <typename T>
__global__ void finite_rows_kernel(const T* X, int64_t ld, int k, const uint8_t* mask, int64_t n_slots,
                                   unsigned int* flag) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  bool bad = false;
  if (r < n_slots && mask[r]) {
    const T* row = X + r * ld;
    for (int j = threadIdx.x & 31; j < k; j += 32) bad |= !(fabs((double)row[j]) <= 1.7976931348623157e308);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

cudaError_t launch_finite_rows(const Ham& H, const void* X, int64_t ld, int k, int dtype, unsigned int* flag,
                               cudaStream_t st) {
  const int64_t n = H.grid.n_slots * 32;
  if (dtype == KSCF_F64)
    finite_rows_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>((const double*)X, ld, k, H.d_mask,
                                                                    H.grid.n_slots, flag), count_launch();
  else
    finite_rows_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>((const float*)X, ld, k, H.d_mask,
                                                                   H.grid.n_slots, flag), count_launch();
  return cudaGetLastError();
}

cudaError_t launch_zero_rows(const Ham& H, void* X, int64_t ld, int k, int dtype, cudaStream_t st) {
  if (H.n_pad == 0 || k == 0) return cudaSuccess;
  const int64_t n = H.n_pad * 32;
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


static bool g_brick16_attr[64] = {false};
static bool g_brick32_attr[64] = {false};

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
  StepArgs<float>& af = *reinterpret_cast<StepArgs<float>*>(&a);
  // 0) wide brick kernel: 16-vector chunks (two CTAs per SM), 16-byte rows, 32-bit row offsets
  //    inside a brick
  {
    constexpr int WNV = 16;
    const int wn = (w + WNV - 1) / WNV * WNV;
    const bool ok = sizeof(T) == 4 && H.grid.B == 8 && w >= WNV && wavail >= wn && cld >= wn && cld % 4 == 0 &&
                    ld_in % 4 == 0 && ld_out % 4 == 0 && (!prev || ld_prev % 4 == 0) && ((uintptr_t)in % 16) == 0 &&
                    ((uintptr_t)out % 16) == 0 && (!prev || ((uintptr_t)prev % 16) == 0) &&
                    ((uintptr_t)coef % 16) == 0 && 512 * std::max(ld_in, std::max(ld_out, prev ? ld_prev : 0)) <
                                                          ((int64_t)1 << 31);
    if (ok) {
      int dev = 0;
      cudaGetDevice(&dev);
      const int smem = 2 * 512 * (WNV / 4) * 16;
      if (dev >= 0 && dev < 64 && !g_brick32_attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(cheb_step_brick8w<WNV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        g_brick32_attr[dev] = true;
      }
      const int nchunk = wn / WNV;
      cheb_step_brick8w<WNV><<<(unsigned)(H.grid.n_bricks * nchunk), WNV * 16, smem, st>>>(af, nchunk,
                                                                                           H.d_kb_entry_lslot),
          count_launch();
      return cudaGetLastError();
    }
  }
  // 1) brick kernel with register halos: rows must have room for whole 8-vector chunks
  if (sizeof(T) == 4 && H.grid.B == 8 && wavail >= w8 && cld >= w8 && cld % 2 == 0) {
    const bool vec = (ld_in % 4 == 0) && (ld_out % 4 == 0) && (!prev || ld_prev % 4 == 0) && (cld % 2 == 0) &&
                     ((uintptr_t)in % 16 == 0) && ((uintptr_t)out % 16 == 0) &&
                     (!prev || (uintptr_t)prev % 16 == 0);
    const int w16 = (w + 15) / 16 * 16;
    if (w >= 16 && wavail >= w16 && cld >= w16) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev >= 0 && dev < 64 && !g_brick16_attr[dev]) {
        // 64 KB of dynamic shared memory needs the opt-in attribute
        cudaError_t e = cudaFuncSetAttribute(cheb_step_brick8<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SB_TOTAL * 64);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(cheb_step_brick8<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   SB_TOTAL * 64);
        if (e != cudaSuccess) return e;
        g_brick16_attr[dev] = true;
      }
      const int nchunk = w16 / 16;
      const unsigned grid = (unsigned)(H.grid.n_bricks * nchunk);
      if (vec)
        cheb_step_brick8<16, true><<<grid, 512, SB_TOTAL * 64, st>>>(af, nchunk, H.d_kb_entry_lslot), count_launch();
      else
        cheb_step_brick8<16, false><<<grid, 512, SB_TOTAL * 64, st>>>(af, nchunk, H.d_kb_entry_lslot), count_launch();
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
  // 2) TMA brick kernel: rows without spare width (columns past wavail arrive as zeros);
  //    needs 16-byte row strides and a 16-byte aligned base
  if (sizeof(T) == 4 && H.grid.B == 8 && ld_in % 4 == 0 && ((uintptr_t)in % 16) == 0 && cld >= w8 && cld % 2 == 0 &&
      ld_out % 2 == 0 && (!prev || ld_prev % 2 == 0) && ((uintptr_t)out % 8) == 0 &&
      (!prev || ((uintptr_t)prev % 8) == 0)) {
    BrickMaps maps;
    cudaError_t e = encode_brick_maps(&maps, (const float*)in, ld_in, wavail, H.grid.n_bricks);
    if (e == cudaSuccess) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev >= 0 && dev < 64 && !g_tma_attr[dev]) {
        e = cudaFuncSetAttribute(cheb_step_tma8<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TB_SMEM);
        if (e != cudaSuccess) return e;
        g_tma_attr[dev] = true;
      }
      const int nchunk = w8 / 8;
      cheb_step_tma8<0><<<(unsigned)(H.grid.n_bricks * nchunk), 256, TB_SMEM, st>>>(
          af, maps, nchunk, (int)H.grid.n_bricks, (int64_t)wavail, wavail, H.d_kb_entry_lslot),
          count_launch();
      return cudaGetLastError();
    }
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
  if (rows == 0 || w == 0) return cudaSuccess;
  const int64_t n = rows * 32;
  if (dtype == KSCF_F64)
    copy_cols_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>((const double*)src, ld_src, (double*)dst,
                                                                 ld_dst, rows, w), count_launch();
  else
    copy_cols_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>((const float*)src, ld_src, (float*)dst,
                                                                ld_dst, rows, w), count_launch();
  return cudaGetLastError();
}

}  // namespace kscf
