// Chebyshev filter steps on chunk-major working buffers (FP32, bricks of 8^3 or 16^3).
//
// The filter (CheFSI paragraph of arXiv 2303.00790; three-term recurrence of Zhou,
// Saad, Tiago & Chelikowsky 2006) runs m degree steps over one column block.  Its
// working copies of the block are stored chunk-major: the block's columns are cut
// into chunks of CW vectors, and chunk c holds every slot's CW values contiguously,
//     element (c, s, v) at buf[(c * n_slots + s) * CW + v],
// so that one brick of one chunk is one contiguous range.  A CTA works on one cell of 8^3
// points: the brick itself for 8^3 bricks, one octant of a 16^3 brick (whose points stay
// x-fastest over the whole brick, so that a cell's rows are 64 runs of 8).  The
// degree-step launches walk the cells chunk by chunk (within supertiles of consecutive
// cells), so the neighbour cells whose faces a cell needs were read from DRAM moments
// before and still sit in L2, and DRAM sees long sequential runs.
//
// One step computes, for every slot s and vector v,
//   out = alpha (H in - c in) + beta prev,
//   H in = -1/2 Lap_h in + V in + sum_i chi_i (E_i h^3 <chi_i, in>),
// the nonlocal projections <chi_i, in> coming from kb_gather_cm launched just before.
// cm_step_ldg16 does it for one cell and 16 vectors per CTA: the cell core is copied
// into shared memory, the halo rows of each line come from the neighbour cells in L2
// into registers, lines that hold no domain point are skipped, and the nonlocal term of a
// point is gathered over its own KB entries (cell order) from the cell's coefficients
// and entries staged in shared memory, in the pass that writes the point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <mutex>

#include "kscf_internal.h"

namespace kscf {

__device__ unsigned int g_cm_status;     // bit 0: a bounded wait gave up
__device__ unsigned int g_nonfinite;     // set when a checked step stored a NaN or Inf

namespace {

struct CmArgs {
  const float* in;        // chunk-major, chunk width CW
  const float* prev;      // may alias out (each element read before it is written)
  int64_t cs_prev, ld_prev;  // element (c, s, v) at prev[c * cs_prev + s * ld_prev + v]
  float* out;
  int64_t cs_out, ld_out;
  int out_vec;            // out rows allow aligned vector stores
  int w;                  // valid columns of the block
  int nchunk, n_cells, super;   // CTA order: supertiles of `super` cells, chunk-major inside
  float alpha, beta, c;
  const float* coef;      // (n_kb*4) rows of cld, global column index
  int64_t cld;
  const float* V;
  const int32_t* nbr;      // face neighbour cells
  const uint8_t* mask;
  const int64_t* kb_ptr;   // KB entries in cell order: CSR over the cell-local points
  const int32_t* kb_atom;
  const float* kb_chi;
  float st[7];
  int64_t n_slots;
  int check;              // flag non-finite stored values
};

// CTA -> (chunk, cell): supertiles of `super` consecutive cells (Hilbert order of the
// bricks); inside a supertile all cells of chunk 0, then of chunk 1, ...  Returns false for
// the idle CTAs of a partial last supertile.
__device__ __forceinline__ bool cta_item(const CmArgs& a, int* chunk, int* cell) {
  const int per = a.nchunk * a.super;
  const int t = blockIdx.x / per, rem = blockIdx.x - t * per;
  const int c = rem / a.super, i = rem - c * a.super;
  const int b = t * a.super + i;
  *chunk = c;
  *cell = b;
  return b < a.n_cells;
}

// Cells of 8^3 points: a brick of 8^3, or an octant of a 16^3 brick (cell = brick * 8 +
// ox + 2 oy + 4 oz).  Slot of the cell's first point; slots of the cell-local point
// (x, y, z) are that plus z * SZ + y * SY + x with SZ = B^2, SY = B.
template <int B>
__device__ __forceinline__ int64_t cell_base(int cell) {
  if (B == 8) return (int64_t)cell * 512;
  const int o = cell & 7;
  return (int64_t)(cell >> 3) * 4096 + (o >> 2) * 2048 + ((o >> 1) & 1) * 128 + (o & 1) * 8;
}
template <int B>
__device__ __forceinline__ int cell_row(int r) {   // r = x + 8 y + 64 z
  return (r >> 6) * (B * B) + ((r >> 3) & 7) * B + (r & 7);
}

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
}  // namespace

// ---------------------------------------------------------------------------
// 16 vectors per CTA, 256 threads (64 lines x 4 lanes x float4).  Core by cp.async, the
// halo rows of each line loaded from the neighbour cells (L2) into the register window.
namespace {
__device__ __forceinline__ float4 f4_add(float4 a, float4 b) {
  const float2 lo = f2_add(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 hi = f2_add(make_float2(a.z, a.w), make_float2(b.z, b.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
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
__device__ __forceinline__ float4 line4(const float4* w, int i, const float2* c2) {
  float4 s = WITH_CENTRE ? f4_mul(c2[0], w[i]) : f4_mul(c2[1], f4_add(w[i + 1], w[i - 1]));
  if (WITH_CENTRE) s = f4_fma(c2[1], f4_add(w[i + 1], w[i - 1]), s);
#pragma unroll
  for (int k = 2; k <= 6; k++) s = f4_fma(c2[k], f4_add(w[i + k], w[i - k]), s);
  return s;
}
__device__ __forceinline__ float4 ld4(const float* p) { return __ldg((const float4*)p); }
__device__ __forceinline__ bool finite4(float4 v) {
  return fabsf(v.x) <= FLT_MAX && fabsf(v.y) <= FLT_MAX && fabsf(v.z) <= FLT_MAX && fabsf(v.w) <= FLT_MAX;
}
}  // namespace

// Shared memory of cm_step_ldg16 (bytes): core and accumulator (512 point slots x 16
// floats each), the coefficients of the cell's KB atoms (KSCF_BRICK_ATOMS x 4 x 16
// floats) and the first LDG_ENT entries of the cell (packed word + chi).
constexpr int LDG_ENT = 256;
constexpr int LDG_CORE = 0, LDG_ACC = 32768, LDG_KBC = 65536, LDG_EW = LDG_KBC + KSCF_BRICK_ATOMS * 4 * 64,
              LDG_ECHI = LDG_EW + LDG_ENT * 4, LDG_PREV = LDG_ECHI + LDG_ENT * 16, LDG_KBP = LDG_PREV + 32768,
              LDG_SMEM = LDG_KBP + 1040;   // + the cell's 513 entry offsets (uint16, from its first entry)

// Lines of a pass that hold no domain point are skipped: each pass takes its lines from
// the cell's compacted list of live lines, and the threads past the list's end idle
// (their points are padding and never stored).  The nonlocal gather of the z pass reads
// the projection coefficients of the cell's KB atoms and the cell's entries from shared
// memory, staged at the start together with the core (SMEM_KB; otherwise from global
// memory).  B: brick edge (8 or 16), which sets the slot steps inside a cell.
template <bool SMEM_KB, int B>
__global__ void __launch_bounds__(256, 2) cm_step_ldg16(CmArgs a, const uint8_t* __restrict__ lines,
                                                        const uint8_t* __restrict__ nlines,
                                                        const int32_t* __restrict__ batoms,
                                                        const int32_t* __restrict__ bnat,
                                                        const uint32_t* __restrict__ eword,
                                                        const float* __restrict__ zero) {
  constexpr int SZ = B * B, SY = B;   // slot steps of z and y inside a brick
  extern __shared__ __align__(16) uint8_t smw[];
  float4* core4 = (float4*)(smw + LDG_CORE);   // [512][4]
  float4* acc4 = (float4*)(smw + LDG_ACC);     // [512][4]
  float4* kbc = (float4*)(smw + LDG_KBC);      // [atom][l][4]
  uint32_t* ew = (uint32_t*)(smw + LDG_EW);
  float4* echi = (float4*)(smw + LDG_ECHI);
  const float4* prev4 = (const float4*)(smw + LDG_PREV);   // [512][4]: Y_{j-2} rows of this cell
  uint16_t* kbp = (uint16_t*)(smw + LDG_KBP);              // [513]: first entry of each point, from e0
  auto sl = [](int x, int y, int z) { return (z * 8 + y) * 8 + (x ^ (y & 1)); };
  int c, cell;
  if (!cta_item(a, &c, &cell)) return;
  const int tid = threadIdx.x, vp = tid & 3, L = tid >> 2;
  const int vl = 4 * vp;
  const int64_t b0 = cell_base<B>(cell);     // slot of the cell's first point
  const int64_t k0 = (int64_t)cell * 512;    // its first cell-local point (KB tables)
  const float* inc = a.in + (int64_t)c * a.n_slots * 16 + vl;   // row stride 16 floats
  const float* own = inc + b0 * 16;
  const float* nbp[6];   // a missing neighbour reads the zero brick
#pragma unroll
  for (int f = 0; f < 6; f++) {
    const int q = __ldg(a.nbr + (int64_t)cell * 6 + f);
    nbp[f] = q >= 0 ? inc + cell_base<B>(q) * 16 : zero + vl;
  }
  const uint8_t* bl = lines + (int64_t)cell * 192;
  const int nlx = __ldg(nlines + cell * 3), nly = __ldg(nlines + cell * 3 + 1), nlz = __ldg(nlines + cell * 3 + 2);
  const int lx = L < nlx ? __ldg(bl + L) : -1;
  const int ly = L < nly ? __ldg(bl + 64 + L) : -1;
  const int lz = L < nlz ? __ldg(bl + 128 + L) : -1;
  // core: 512 rows x 64 B, padding rows zero-filled without a read; with it the cell's
  // Y_{j-2} rows, so that the z pass finds them in shared memory
  const bool prev_smem = a.prev != nullptr && a.ld_prev == 16;
  const float* psrc = prev_smem ? a.prev + (int64_t)c * a.cs_prev + b0 * 16 + vl : nullptr;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const int r = L + 64 * i;
    const int ro = cell_row<B>(r);
    const uint32_t live = __ldg(a.mask + b0 + ro);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(&core4[sl(r & 7, (r >> 3) & 7, r >> 6) * 4 + vp]);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(own + ro * 16), "r"(live ? 16 : 0)
                 : "memory");
    if (prev_smem) {
      const uint32_t dp = (uint32_t)__cvta_generic_to_shared(smw + LDG_PREV + (r * 4 + vp) * 16);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dp), "l"(psrc + ro * 16), "r"(live ? 16 : 0)
                   : "memory");
    }
  }
  const int64_t e0 = __ldg(a.kb_ptr + k0), e1 = __ldg(a.kb_ptr + k0 + 512);
  const int ne = (int)(e1 - e0);
  for (int t = tid; t <= 512; t += 256) kbp[t] = (uint16_t)(__ldg(a.kb_ptr + k0 + t) - e0);
  if (SMEM_KB) {
    const int nat = __ldg(bnat + cell);
    for (int t = tid; t < nat * 16; t += 256) {
      const int at = __ldg(batoms + (int64_t)cell * KSCF_BRICK_ATOMS + (t >> 4));
      const int l = (t >> 2) & 3, q = t & 3;
      const float* src = a.coef + ((int64_t)at * 4 + l) * a.cld + c * 16 + 4 * q;
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(&kbc[((t >> 4) * 4 + l) * 4 + q]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    }
    for (int i = tid; i < min(ne, LDG_ENT); i += 256) {
      const uint32_t dw = (uint32_t)__cvta_generic_to_shared(&ew[i]);
      const uint32_t dc = (uint32_t)__cvta_generic_to_shared(&echi[i]);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dw), "l"(eword + e0 + i) : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dc), "l"(a.kb_chi + 4 * (e0 + i)) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  float vv[8];
  uint32_t mk = 0;
  const int zl = lz >= 0 ? (lz >> 3) * SY + (lz & 7) : 0;   // z line (x, y): slot offset of its z = 0 point
  if (lz >= 0) {
#pragma unroll
    for (int z = 0; z < 8; z++) {
      const int64_t s = b0 + z * SZ + zl;
      mk |= (uint32_t)__ldg(a.mask + s) << z;
      vv[z] = __ldg(a.V + s);
    }
  }
  float2 c2[7];
  c2[0] = f2(3.0f * a.st[0]);
#pragma unroll
  for (int k = 1; k < 7; k++) c2[k] = f2(a.st[k]);
  // ---- x pass: line (y, z) ----
  {
    const int y = lx & 7, z = lx >> 3;
    const int rb = (z * SZ + y * SY) * 16;
    float4 w[20];
    if (lx >= 0) {
#pragma unroll
      for (int xx = 0; xx < 6; xx++) {
        w[xx] = ld4(nbp[0] + rb + (2 + xx) * 16);
        w[14 + xx] = ld4(nbp[1] + rb + xx * 16);
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (lx >= 0) {
#pragma unroll
      for (int x = 0; x < 8; x++) w[6 + x] = core4[sl(x, y, z) * 4 + vp];
#pragma unroll
      for (int x = 0; x < 8; x++) acc4[sl(x, y, z) * 4 + vp] = line4<true>(w, 6 + x, c2);
    }
  }
  // ---- y pass: line (x, z) ----
  {
    const int x = ly & 7, z = ly >> 3;
    float4 w[20];
    if (ly >= 0) {
#pragma unroll
      for (int yy = 0; yy < 6; yy++) {
        w[yy] = ld4(nbp[2] + (z * SZ + (2 + yy) * SY + x) * 16);
        w[14 + yy] = ld4(nbp[3] + (z * SZ + yy * SY + x) * 16);
      }
#pragma unroll
      for (int y = 0; y < 8; y++) w[6 + y] = core4[sl(x, y, z) * 4 + vp];
    }
    __syncthreads();  // x-pass accumulator writes are visible
    if (ly >= 0) {
#pragma unroll
      for (int y = 0; y < 8; y++) {
        const int q = sl(x, y, z) * 4 + vp;
        acc4[q] = f4_add(acc4[q], line4<false>(w, 6 + y, c2));
      }
    }
  }
  // ---- z pass: line (x, y); potential, recurrence, store ----
  {
    const int x = lz & 7, y = lz >> 3;
    float4 w[20];
    if (lz >= 0) {
#pragma unroll
      for (int zz = 0; zz < 6; zz++) {
        w[zz] = ld4(nbp[4] + ((2 + zz) * SZ + zl) * 16);
        w[14 + zz] = ld4(nbp[5] + (zz * SZ + zl) * 16);
      }
#pragma unroll
      for (int z = 0; z < 8; z++) w[6 + z] = core4[sl(x, y, z) * 4 + vp];
    }
    __syncthreads();  // y-pass accumulator writes are visible
    if (lz >= 0) {
      const float2 alpha = f2(a.alpha), beta = f2(a.beta), negc = f2(-a.c);
      const float* prevp = a.prev ? a.prev + (int64_t)c * a.cs_prev + vl : nullptr;
      float* outp = a.out + (int64_t)c * a.cs_out + vl;
      const int col = c * 16 + vl;
      bool bad = false;
#pragma unroll
      for (int z = 0; z < 8; z++) {
        const int64_t s = b0 + z * SZ + zl;
        if (!((mk >> z) & 1u)) continue;
        const float4 yc = w[6 + z];
        float4 hy = f4_add(acc4[sl(x, y, z) * 4 + vp], line4<false>(w, 6 + z, c2));
        hy = f4_fma(f2(vv[z]), yc, hy);
        // nonlocal term of this point: sum over its KB entries (cell order) of
        // chi_l(e) * coef(atom(e), l), accumulated in registers
        const int sloc = z * 64 + lz;
        for (int i = kbp[sloc], i1 = kbp[sloc + 1]; i < i1; i++) {
          const int64_t qe = e0 + i;
          float4 ch;
          float4 cv[4];
          if (SMEM_KB) {
            uint32_t word;
            if (i < LDG_ENT) {
              word = ew[i];
              ch = echi[i];
            } else {
              word = __ldg(eword + qe);
              ch = __ldg((const float4*)(a.kb_chi + 4 * qe));
            }
            const float4* cf = kbc + (word >> 16) * 16 + vp;
#pragma unroll
            for (int l = 0; l < 4; l++) cv[l] = cf[4 * l];
          } else {
            ch = __ldg((const float4*)(a.kb_chi + 4 * qe));
            const float* g = a.coef + (int64_t)__ldg(a.kb_atom + qe) * 4 * a.cld + c * 16 + vl;
#pragma unroll
            for (int l = 0; l < 4; l++) cv[l] = ld4(g + l * a.cld);
          }
          hy = f4_fma(f2(ch.x), cv[0], hy);
          hy = f4_fma(f2(ch.y), cv[1], hy);
          hy = f4_fma(f2(ch.z), cv[2], hy);
          hy = f4_fma(f2(ch.w), cv[3], hy);
        }
        float4 r = f4_mul(alpha, f4_fma(negc, yc, hy));
        if (prevp) {
          // plain load otherwise: prev may be the output buffer
          const float4 pv = prev_smem ? prev4[(z * 64 + lz) * 4 + vp] : *(const float4*)(prevp + s * a.ld_prev);
          r = f4_fma(beta, pv, r);
        }
        if (a.check)
          bad |= !finite4(make_float4(col < a.w ? r.x : 0.f, col + 1 < a.w ? r.y : 0.f,
                                      col + 2 < a.w ? r.z : 0.f, col + 3 < a.w ? r.w : 0.f));
        float* o = outp + s * a.ld_out;
        if (a.out_vec) {
          *(float4*)o = r;
        } else {
          if (col < a.w) o[0] = r.x;
          if (col + 1 < a.w) o[1] = r.y;
          if (col + 2 < a.w) o[2] = r.z;
          if (col + 3 < a.w) o[3] = r.w;
        }
      }
      if (bad) atomicOr(&g_nonfinite, 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// coef[(a*4+l)*cld + v] = E_l h^3 sum_{entries e of atom a} chi_l(e) Y(slot_e, v) for
// v < w, and 0 for w <= v < cld (the padded columns of the last chunk then stay zero
// through the recurrence).  Y chunk-major with chunks of 16 columns.  A CTA takes one atom
// and 128 columns (8 chunks); its 8 warps stride over the atom's entries, lane (chunk
// lane / 4, quad lane % 4) reading its 4 columns of the entry's row as one float4; the
// warps' sums meet in shared memory.
__global__ void __launch_bounds__(256) kb_gather_cm(const float* __restrict__ Y, int64_t n_slots, int w, int nchunk,
                                                    int64_t cld, const int64_t* __restrict__ aptr,
                                                    const int64_t* __restrict__ aslot,
                                                    const float* __restrict__ achi,
                                                    const double* __restrict__ energy, float* __restrict__ coef) {
  const int at = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = blockIdx.y * 8 + (lane >> 2);
  float acc[16];   // [l * 4 + column of the quad]
#pragma unroll
  for (int i = 0; i < 16; i++) acc[i] = 0.f;
  if (chunk < nchunk) {
    const float* base = Y + (int64_t)chunk * n_slots * 16 + (lane & 3) * 4;
    const int64_t e1 = __ldg(aptr + at + 1);
    int64_t e = __ldg(aptr + at) + warp;
    auto add = [&](float4 c, float4 y) {
      const float cl[4] = {c.x, c.y, c.z, c.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int l = 0; l < 4; l++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[l * 4 + q] = fmaf(cl[l], yv[q], acc[l * 4 + q]);
    };
    for (; e + 8 < e1; e += 16) {
      const int64_t s0 = __ldg(aslot + e), s1 = __ldg(aslot + e + 8);
      const float4 c0 = __ldg((const float4*)(achi + 4 * e)), c1 = __ldg((const float4*)(achi + 4 * (e + 8)));
      const float4 y0 = __ldg((const float4*)(base + s0 * 16)), y1 = __ldg((const float4*)(base + s1 * 16));
      add(c0, y0);
      add(c1, y1);
    }
    if (e < e1) add(__ldg((const float4*)(achi + 4 * e)), __ldg((const float4*)(base + __ldg(aslot + e) * 16)));
  }
  __shared__ float red[8][16][33];
#pragma unroll
  for (int i = 0; i < 16; i++) red[warp][i][lane] = acc[i];
  __syncthreads();
  // output element o = l * 128 + vv (vv: column inside the CTA's 128): contiguous stores
  for (int o = threadIdx.x; o < 512; o += 256) {
    const int l = o >> 7, vv = o & 127;
    const int ln = (vv >> 4) * 4 + ((vv >> 2) & 3), i = l * 4 + (vv & 3);
    const int64_t v = (int64_t)blockIdx.y * 128 + vv;
    if (v < cld) {
      float sum = 0.f;
#pragma unroll
      for (int q = 0; q < 8; q++) sum += red[q][i][ln];
      coef[((int64_t)at * 4 + l) * cld + v] = v < w ? (float)energy[4 * at + l] * sum : 0.f;
    }
  }
}

// chunk-major copy (chunks of 16 columns) of w columns of a slot-major block (row stride
// ld), padded columns and padding rows zero (padding rows are not read); the padding rows
// of the second working buffer are zeroed too (the step kernels never write padding rows,
// and they are read as halos).  One warp per slot row, 32 consecutive columns per step.
__global__ void __launch_bounds__(256) to_chunk_major(const float* __restrict__ X, int64_t ld, int w, int wpad,
                                                      int64_t n_slots, const uint8_t* __restrict__ mask,
                                                      float* __restrict__ buf, float* __restrict__ buf2) {
  const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (s >= n_slots) return;
  const bool live = __ldg(mask + s) != 0;
  const float* xr = X + s * ld;
  float* br = buf + s * 16;
  float* b2 = buf2 + s * 16;
  const int64_t cstride = n_slots * 16;   // floats between chunks
  for (int col = threadIdx.x & 31; col < wpad; col += 32) {
    const int64_t o = (int64_t)(col >> 4) * cstride + (col & 15);
    br[o] = (live && col < w) ? __ldg(xr + col) : 0.f;
    if (!live) b2[o] = 0.f;
  }
}

namespace {

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
}  // namespace

int cm_chunk_width() { return 16; }

cudaError_t launch_to_chunk_major(const Ham& H, const float* X, int64_t ld, int w, int cw, float* buf, float* buf2,
                                  cudaStream_t st) {
  if (cw != 16) return cudaErrorInvalidValue;
  const int wpad = (w + cw - 1) / cw * cw;
  to_chunk_major<<<blocks(H.grid.n_slots, 8), 256, 0, st>>>(X, ld, w, wpad, H.grid.n_slots, H.d_mask, buf, buf2),
      count_launch();
  return cudaGetLastError();
}

cudaError_t launch_kb_gather_cm(const Ham& H, const float* Y, int cw, int w, float* coef, int64_t cld,
                                cudaStream_t st) {
  if (H.n_kb == 0 || w == 0) return cudaSuccess;
  if (cw != 16) return cudaErrorInvalidValue;
  dim3 grid(H.n_kb, (unsigned)((cld + 127) / 128));
  kb_gather_cm<<<grid, 256, 0, st>>>(Y, H.grid.n_slots, w, (w + 15) / 16, cld, H.d_kb_atom_ptr, H.d_kb_atom_slot,
                                     H.d_kb_atom_chi32, H.d_kb_energy, coef),
      count_launch();
  return cudaGetLastError();
}

// One degree step: in chunk-major (chunk width cm_chunk_width()); prev chunk-major or
// null; out chunk-major (out_ld < 0) or the caller's slot-major block (row stride out_ld).
cudaError_t launch_cm_step(const Ham& H, const float* in, const float* prev, float* out, int64_t out_ld, int w,
                           double alpha, double beta, double cshift, const float* coef, int64_t cld, bool check,
                           const float* zero, cudaStream_t st) {
  const int cw = cm_chunk_width();
  CmArgs a;
  a.in = in;
  a.prev = prev;
  a.cs_prev = H.grid.n_slots * cw;
  a.ld_prev = cw;
  a.out = out;
  if (out_ld < 0) {
    a.cs_out = H.grid.n_slots * cw;
    a.ld_out = cw;
    a.out_vec = 1;
  } else {
    a.cs_out = cw;
    a.ld_out = out_ld;
    a.out_vec = (out_ld % cw == 0 && ((uintptr_t)out % 16) == 0 && w % cw == 0) ? 1 : 0;
  }
  a.w = w;
  a.nchunk = (w + cw - 1) / cw;
  if (H.n_cells <= 0 || (H.grid.B != 8 && H.grid.B != 16)) return cudaErrorInvalidValue;
  a.n_cells = (int)H.n_cells;
  // supertiles: the cells of one chunk stay L2-resident (three buffers x 512 rows x cw x 4 B each)
  const int64_t per_cell = 3LL * 512 * cw * 4;
  a.super = (int)std::max<int64_t>(64, std::min<int64_t>(H.n_cells, (64LL << 20) / per_cell));
  a.alpha = (float)alpha;
  a.beta = (float)beta;
  a.c = (float)cshift;
  a.coef = coef;
  a.cld = cld;
  a.V = H.d_v32;
  a.nbr = H.d_cell_nbr;
  a.mask = H.d_mask;
  a.kb_ptr = H.d_cell_kb_ptr;
  a.kb_atom = H.d_cell_kb_atom;
  a.kb_chi = H.d_cell_kb_chi32;
  for (int k = 0; k < 7; k++) a.st[k] = (float)H.stencil[k];
  a.n_slots = H.grid.n_slots;
  a.check = check ? 1 : 0;
  const int n_super = (int)((H.n_cells + a.super - 1) / a.super);
  const unsigned grid = (unsigned)((int64_t)n_super * a.super * a.nchunk);
  // the shared-memory size attribute belongs to the context: set on every call
  auto run = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, LDG_SMEM);
    if (e != cudaSuccess) return e;
    kern<<<grid, 256, LDG_SMEM, st>>>(a, H.d_lines, H.d_nlines, H.d_brick_atoms, H.d_brick_natoms,
                                      H.d_kb_entry_word, zero),
        count_launch();
    return cudaGetLastError();
  };
  if (H.grid.B == 8) return H.brick_atoms_ok ? run(cm_step_ldg16<true, 8>) : run(cm_step_ldg16<false, 8>);
  return H.brick_atoms_ok ? run(cm_step_ldg16<true, 16>) : run(cm_step_ldg16<false, 16>);
}

unsigned int* nonfinite_flag() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_nonfinite) != cudaSuccess) return nullptr;
  return (unsigned int*)p;
}

cudaError_t cm_status(bool reset, unsigned int* timeout, unsigned int* nonfinite) {
  cudaError_t e = cudaMemcpyFromSymbol(timeout, g_cm_status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(nonfinite, g_nonfinite, sizeof(unsigned int));
  if (e == cudaSuccess && reset && (*timeout || *nonfinite)) {
    unsigned int z = 0;
    e = cudaMemcpyToSymbol(g_cm_status, &z, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_nonfinite, &z, sizeof(unsigned int));
  }
  return e;
}

}  // namespace kscf
