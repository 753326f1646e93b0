// Tensor-core (tcgen05) GEMMs of the subspace steps of CheFSI (Cholesky-QR and
// Rayleigh-Ritz, arXiv 2303.00790 CheFSI paragraph):
//   gram:   C (FP64) += scale * A^T B      A: rows x m, B: rows x n  (FP32)
//   rotate: out (FP32) = A Q               A: rows x kin (FP32), Q: kin x kout (FP64)
// With a row map, row r of A, B and out is row rowmap[r] of the stored matrix: the subspace
// steps pass the grid's domain slots, so that the padding slots of the brick layout (zero
// rows, 30 % of the slots of the 2.2 nm sphere) are neither split, multiplied nor written.
//
// Precision: each FP32 operand value x is split into three bf16 pieces
// x = x1 + x2 + x3 (x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)), and
// the six products x1y1, x1y2, x2y1, x1y3, x2y2, x3y1 are accumulated in FP32 in
// tensor memory; the dropped terms are O(2^-24).  Gram partial sums cover at most
// 256 rows before they are added into compensated FP32 pairs and, per CTA, into FP64.
//
// Data path: a split kernel writes the pieces in the tensor core's K-major
// "no swizzle" canonical layout, pre-tiled so that every (128 rows x 32 K) operand
// block is one contiguous 8 KB chunk; the GEMM kernel streams blocks into shared
// memory with 1D bulk TMA copies (cp.async.bulk + mbarrier transaction counts), one
// thread issues tcgen05.mma (M=128, N=256, K=16) into a TMEM accumulator, and four
// epilogue warps read TMEM with tcgen05.ld.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "kscf_internal.h"

namespace kscf {

namespace {

constexpr int TM = 128;             // M tile (TMEM lanes)
constexpr int TN = 256;             // N tile (TMEM columns)
constexpr int TK = 32;              // K per pipeline stage
constexpr int BLK_ELEMS = 128 * TK; // elements of one pre-tiled operand block (8 KB)
constexpr int STAGES = 3;
constexpr int NPIECE = 3;
constexpr int A_STAGE_BYTES = NPIECE * BLK_ELEMS * 2;       // 24 KB
constexpr int B_STAGE_BYTES = NPIECE * 2 * BLK_ELEMS * 2;   // 48 KB
constexpr int STAGE_BYTES = A_STAGE_BYTES + B_STAGE_BYTES;  // 72 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256 + 4 * 32 * 17 * 4;
constexpr int64_t GRAM_CHUNK_MIN = 16384, GRAM_CHUNK_MAX = 262144;  // rows split per launch
constexpr size_t GRAM_PIECE_BUDGET = (size_t)1 << 30;               // bytes of split pieces per launch
constexpr uint32_t WAIT_LIMIT = 1u << 20;                   // bounded spin on mbarriers

__device__ unsigned int g_tc_status;  // 0 ok, else a wait timed out

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; on timeout flags g_tc_status and returns false
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < WAIT_LIMIT; i++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 32) __nanosleep(128);
  }
  atomicOr(&g_tc_status, 1u);
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major, no-swizzle shared-memory matrix descriptor: core matrices of 8 rows x 16 B,
// LBO = byte step between K-adjacent core matrices, SBO = byte step between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, absolute LBO mode, SWIZZLE_NONE
}

// instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = n (a multiple of 16,
// 16 <= n <= 256)
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}
// N of a tile whose first `valid` columns are wanted: rounded up to 16, at most `full`
__device__ __forceinline__ int tile_n(int valid, int full) { return min(full, max(16, (valid + 15) / 16 * 16)); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
  const __nv_bfloat16* A[NPIECE];  // pre-tiled, MN blocks of 128 x K blocks of 32
  const __nv_bfloat16* B[NPIECE];
  int a_nkb, b_nkb;                // K blocks per MN block row in A and B storage
  int m_tiles, n_tiles;            // tiles of 128 (M) and 256 (N)
  int kb_total;                    // K blocks to reduce over
  int n;                           // valid output columns
  float* out;
  int64_t ldo;
  int64_t rows;                    // valid rows of out
  const float* addsrc;             // if non-null: out = A Q + addsrc (same shape as out)
  int64_t ldadd;
  const int32_t* rowmap;           // if non-null: row r of out and addsrc is row rowmap[r]
};

// products (A piece, B piece) kept: orders 2^0, 2^-8 (two), 2^-16 (three)
__constant__ int kProdA[6] = {0, 0, 1, 0, 1, 2};
__constant__ int kProdB[6] = {0, 1, 0, 2, 1, 0};

// Rotation GEMM out = A Q, persistent: CTA c handles tiles c, c + grid, ... (N tiles
// fastest, so CTAs sharing an A row panel run side by side).  The producer streams the
// K blocks of consecutive tiles through one STAGES-deep ring; the MMA thread alternates
// between two 256-column TMEM accumulators, so the four epilogue warps drain tile i
// (TMEM -> registers -> shared-memory transpose -> coalesced row stores) while tile i+1
// is being multiplied.
__global__ void __launch_bounds__(192, 1) tc_gemm_kernel(TcArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;   // 2
  uint64_t* tempty = tfull + 2;       // 2
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  float* trbuf = (float*)(tmem_slot + 4);  // 4 x 32 x 17 floats for the epilogue transpose

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = p.m_tiles * p.n_tiles;
  const int nk = p.kb_total;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: one continuous stream of K blocks over this CTA's tiles
      int g = 0;  // global stage counter
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int nt = t % p.n_tiles, mt = t / p.n_tiles;
        for (int kb = 0; kb < nk; kb++, g++) {
          const int s = g % STAGES;
          if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + s * STAGE_BYTES;
          uint8_t* sb = sa + A_STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          for (int q = 0; q < NPIECE; q++) {
            bulk_g2s(sa + q * BLK_ELEMS * 2, p.A[q] + ((int64_t)mt * p.a_nkb + kb) * BLK_ELEMS, BLK_ELEMS * 2,
                     &full[s]);
            for (int h = 0; h < 2; h++)
              bulk_g2s(sb + (q * 2 + h) * BLK_ELEMS * 2, p.B[q] + ((int64_t)(2 * nt + h) * p.b_nkb + kb) * BLK_ELEMS,
                       BLK_ELEMS * 2, &full[s]);
          }
        }
      }
      // the copies of the last stages issued have landed before the CTA can exit
      for (int q = max(0, g - STAGES); q < g; q++) mbar_wait(&full[q % STAGES], (q / STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int g = 0, it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, it++) {
        const int b = it & 1;
        if (it >= 2 && !mbar_wait(&tempty[b], ((it >> 1) - 1) & 1)) break;
        tc_fence_after();
        const uint32_t acc = tmem + b * TN;
        // the last column tile multiplies only its valid columns (rounded up to 16)
        const uint32_t idesc = idesc_n(tile_n(p.n - (t % p.n_tiles) * TN, TN));
        for (int kb = 0; kb < nk; kb++, g++) {
          const int s = g % STAGES;
          ok = mbar_wait(&full[s], (g / STAGES) & 1);
          if (!ok) break;
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
          const uint32_t sb = sa + A_STAGE_BYTES;
#pragma unroll
          for (int pr = 0; pr < 6; pr++) {
            const uint32_t a_base = sa + kProdA[pr] * BLK_ELEMS * 2;
            const uint32_t b_base = sb + kProdB[pr] * 2 * BLK_ELEMS * 2;
#pragma unroll
            for (int kk = 0; kk < TK / 16; kk++) {
              // K = 16 covers two core matrices along K (128 B apart); 8-row groups
              // are 4 core matrices (512 B) apart
              const uint64_t ad = smem_desc(a_base + kk * 256, 128, 512);
              const uint64_t bd = smem_desc(b_base + kk * 256, 128, 512);
              mma_bf16(acc, ad, bd, idesc, (kb > 0 || pr > 0 || kk > 0) ? 1u : 0u);
            }
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&tfull[b]);
      }
    }
  } else {
    // epilogue warps 2..5 -> TMEM lane quadrants 2, 3, 0, 1
    const int q = warp & 3;
    float* tr = trbuf + q * 32 * 17;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
      const int nt = t % p.n_tiles, mt = t / p.n_tiles;
      const int b = it & 1;
      // warp-uniform decision: tcgen05.ld below is executed by all lanes or none
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[b], (it >> 1) & 1));
      if (!ok) break;
      tc_fence_after();
      // the output rows of this lane's sixteen tile rows (through the row map)
      int64_t orow[16];
      {
        const int64_t ir0 = (int64_t)mt * TM + q * 32 + (lane >> 4);
#pragma unroll
        for (int r = 0; r < 16; r++) {
          const int64_t ir = ir0 + 2 * r;
          orow[r] = (p.rowmap && ir < p.rows) ? (int64_t)__ldg(p.rowmap + ir) : ir;
        }
      }
      for (int c0 = 0; c0 < TN; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + b * TN + c0, v);
        // transpose the 32 x 16 block through shared memory: each store instruction then
        // writes two contiguous 64-byte row segments
#pragma unroll
        for (int c = 0; c < 16; c++) tr[lane * 17 + c] = v[c];
        __syncwarp();
        const int jj = lane & 15, rh = lane >> 4;
        const int j = nt * TN + c0 + jj;
        if (j < p.n) {
          const int64_t ir0 = (int64_t)mt * TM + q * 32 + rh;
          float add[16];
          // the sixteen addends are loaded before any store (out may alias addsrc; each
          // element is read and written by this lane only), so their latencies overlap
#pragma unroll
          for (int r = 0; r < 16; r++) {
            const int64_t ir = ir0 + 2 * r;
            add[r] = (p.addsrc && ir < p.rows) ? p.addsrc[orow[r] * p.ldadd + j] : 0.0f;
          }
#pragma unroll
          for (int r = 0; r < 16; r++) {
            const int64_t ir = ir0 + 2 * r;
            if (ir < p.rows) {
              const float v = tr[(2 * r + rh) * 17 + jj];
              p.out[orow[r] * p.ldo + j] = p.addsrc ? v + add[r] : v;
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN));
  }
}

// ---------------------------------------------------------------------------
// Gram kernel (tile 128 x 128).  The tensor core accumulates in FP32 with a
// systematic truncation of order 2^-26 per accumulation, so long FP32 chains bias
// sums of squares.  Here the leading product x1*y1 goes to a "main" accumulator and the
// five cross products to a "side" accumulator, each chain covers one 512-row
// sub-chunk, and two TMEM buffer pairs alternate: while the MMA thread fills one pair,
// eight epilogue warps drain the other into compensated FP32 (hi, lo) register pairs
// (one row and 64 columns per thread).  The pairs are added to C in FP64 once per CTA.
constexpr int GN = 128;                                  // N tile of the Gram kernel
constexpr int G_SUB_KB = 8;                              // K blocks per FP32 chain (256 rows)
constexpr int G_STAGES = 4;
constexpr int G_A_BYTES = NPIECE * BLK_ELEMS * 2;        // 24 KB
constexpr int G_STAGE_BYTES = 2 * G_A_BYTES;             // 48 KB
constexpr int G_SMEM_BYTES = G_STAGES * G_STAGE_BYTES + 1024 + 512;
__device__ __forceinline__ void mma_bf16_n128(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

struct GramArgs {
  const __nv_bfloat16* A[NPIECE];
  const __nv_bfloat16* B[NPIECE];
  int nkb;          // K blocks of the operands (same for A and B)
  int m_tiles, n_tiles;
  int kb_per_cta;   // multiple of G_SUB_KB
  int m, n;
  int symmetric;
  double* C;
  int64_t ldc;
  double scale;
};

__global__ void __launch_bounds__(320, 1) tc_gram_kernel(GramArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + G_STAGES * G_STAGE_BYTES);
  uint64_t* empty = full + G_STAGES;
  uint64_t* tfull = empty + G_STAGES;  // 2: accumulator pair b ready
  uint64_t* tempty = tfull + 2;        // 2: accumulator pair b drained
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x % p.m_tiles, nt = blockIdx.x / p.m_tiles;
  if (p.symmetric && nt * GN + GN - 1 < mt * TM) return;
  const int kb0 = blockIdx.y * p.kb_per_cta;
  const int kb1 = min(p.nkb, kb0 + p.kb_per_cta);
  const int nk = kb1 - kb0;
  if (nk <= 0) return;
  const int nsub = (nk + G_SUB_KB - 1) / G_SUB_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < G_STAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nk; it++) {
        const int s = it % G_STAGES;
        if (it >= G_STAGES && !mbar_wait(&empty[s], ((it / G_STAGES) - 1) & 1)) break;
        uint8_t* sa = smem + s * G_STAGE_BYTES;
        uint8_t* sb = sa + G_A_BYTES;
        mbar_expect_tx(&full[s], G_STAGE_BYTES);
        const int kb = kb0 + it;
        for (int q = 0; q < NPIECE; q++) {
          bulk_g2s(sa + q * BLK_ELEMS * 2, p.A[q] + ((int64_t)mt * p.nkb + kb) * BLK_ELEMS, BLK_ELEMS * 2, &full[s]);
          bulk_g2s(sb + q * BLK_ELEMS * 2, p.B[q] + ((int64_t)nt * p.nkb + kb) * BLK_ELEMS, BLK_ELEMS * 2, &full[s]);
        }
        issued = it + 1;
      }
      for (int it = max(0, issued - G_STAGES); it < issued; it++) mbar_wait(&full[it % G_STAGES], (it / G_STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      // the last column tile multiplies only its valid columns (rounded up to 16)
      const uint32_t idesc = idesc_n(tile_n(p.n - nt * GN, GN));
      for (int c = 0; c < nsub && ok; c++) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(&tempty[b], ((c >> 1) - 1) & 1)) break;
        tc_fence_after();
        const uint32_t t_main = tmem + b * 256, t_side = t_main + 128;
        const int it0 = c * G_SUB_KB, it1 = min(nk, it0 + G_SUB_KB);
        for (int it = it0; it < it1; it++) {
          const int s = it % G_STAGES;
          ok = mbar_wait(&full[s], (it / G_STAGES) & 1);
          if (!ok) break;
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * G_STAGE_BYTES);
          const uint32_t sb = sa + G_A_BYTES;
#pragma unroll
          for (int pr = 0; pr < 6; pr++) {
            const uint32_t a_base = sa + kProdA[pr] * BLK_ELEMS * 2;
            const uint32_t b_base = sb + kProdB[pr] * BLK_ELEMS * 2;
#pragma unroll
            for (int kk = 0; kk < TK / 16; kk++) {
              const uint64_t ad = smem_desc(a_base + kk * 256, 128, 512);
              const uint64_t bd = smem_desc(b_base + kk * 256, 128, 512);
              const bool first = (it == it0) && (kk == 0) && (pr <= 1);
              mma_bf16_n128(pr == 0 ? t_main : t_side, ad, bd, idesc, first ? 0u : 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&tfull[b]);
      }
    }
  } else {
    // epilogue warps 2..9: TMEM lane quadrant warp % 4, column half (warp - 2) / 4
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    // compensated FP32 sum (hi, lo) per element: ~48 significant bits at FP32 speed
    // (GB300 runs FP64 at 1/70 of FP32, too slow for a drain every 256 rows)
    float hi[64], lo[64];
#pragma unroll
    for (int c = 0; c < 64; c++) {
      hi[c] = 0.f;
      lo[c] = 0.f;
    }
    bool ok = true;
    for (int c = 0; c < nsub; c++) {
      const int b = c & 1;
      ok = __all_sync(0xffffffffu, mbar_wait(&tfull[b], (c >> 1) & 1));
      if (!ok) break;
      tc_fence_after();
      const uint32_t lane_off = (uint32_t)(q * 32) << 16;
#pragma unroll
      for (int qt = 0; qt < 4; qt++) {
        float vm[16], vs[16];
        tmem_ld16(tmem + lane_off + b * 256 + h * 64 + qt * 16, vm);        // main accumulator
        tmem_ld16(tmem + lane_off + b * 256 + 128 + h * 64 + qt * 16, vs);  // side accumulator
#pragma unroll
        for (int e = 0; e < 16; e++) {
          // TwoSum (Knuth): hi + v = s + err exactly
          const int c = qt * 16 + e;
          const float v = vm[e] + vs[e];
          const float s2 = hi[c] + v;
          const float bp = s2 - hi[c];
          const float err = (hi[c] - (s2 - bp)) + (v - bp);
          hi[c] = s2;
          lo[c] += err;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
    }
    const int i = mt * TM + row;
    if (ok && i < p.m) {
#pragma unroll
      for (int e = 0; e < 64; e++) {
        const int j = nt * GN + h * 64 + e;
        if (j < p.n && (!p.symmetric || j >= i))
          atomicAdd(p.C + i + (int64_t)j * p.ldc, p.scale * ((double)hi[e] + (double)lo[e]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------------------
// split kernels: write three bf16 pieces in the pre-tiled layout
//   block (mb, kb) of an operand Op[MN][K] holds MN rows mb*128 .. +128 and K columns
//   kb*32 .. +32 at element offset (mb*nkb + kb)*4096; inside a block, element
//   (r, c) sits at (r/8)*256 + (c/8)*64 + (r%8)*8 + (c%8).
__device__ __forceinline__ int tiled_off(int r, int c) { return (r >> 3) * 256 + (c >> 3) * 64 + (r & 7) * 8 + (c & 7); }

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  c = __float2bfloat16_rn(r2);
}

// Eight consecutive K values of one MN index form one 16-byte row of a core matrix in the
// pre-tiled layout: split them and store the three pieces' rows directly.
__device__ __forceinline__ void split8_store(const float* x, __nv_bfloat16* P0, __nv_bfloat16* P1,
                                             __nv_bfloat16* P2, int64_t off) {
  __align__(16) __nv_bfloat16 a[8], b[8], c[8];
#pragma unroll
  for (int i = 0; i < 8; i++) split3(x[i], a[i], b[i], c[i]);
  *(uint4*)(P0 + off) = *(const uint4*)a;
  *(uint4*)(P1 + off) = *(const uint4*)b;
  *(uint4*)(P2 + off) = *(const uint4*)c;
}

// Op[i][r] = X[row(r0 + r)][c0 + i]  (gram operand: MN = columns, K = rows; row(r) = rowmap[r],
// or r without a map); one CTA per (128 x 32) block, a thread per (column, 8-row group):
// eight row loads (coalesced over the warp's columns), one 16-byte store per piece
__global__ void __launch_bounds__(256) split_T_kernel(const float* __restrict__ X, int64_t ld, int64_t r0, int nr,
                                                      int c0, int nc, int nkb, const int32_t* __restrict__ rowmap,
                                                      __nv_bfloat16* __restrict__ P0, __nv_bfloat16* __restrict__ P1,
                                                      __nv_bfloat16* __restrict__ P2) {
  const int kb = blockIdx.x, mb = blockIdx.y;
  const int64_t base = ((int64_t)mb * nkb + kb) * BLK_ELEMS;
  const int i = threadIdx.x & 127, gi = mb * 128 + i;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int ko = (threadIdx.x >> 7) + 2 * h;   // 8-row group 0..3 of the block
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int gr = kb * TK + ko * 8 + u;
      x[u] = 0.f;
      if (gi < nc && gr < nr) x[u] = X[(rowmap ? (int64_t)rowmap[r0 + gr] : r0 + gr) * ld + c0 + gi];
    }
    split8_store(x, P0, P1, P2, base + tiled_off(i, ko * 8));
  }
}

// Op[r][c] = X[row(r0 + r)][c]  (rotation A operand: MN = rows, K = columns); one CTA per
// (128 x 32) block, a thread per (row, 8-column group): two float4 loads when the row
// allows, one 16-byte store per piece
__global__ void __launch_bounds__(256) split_N_kernel(const float* __restrict__ X, int64_t ld, int64_t r0, int nr,
                                                      int nc, int nkb, const int32_t* __restrict__ rowmap,
                                                      __nv_bfloat16* __restrict__ P0, __nv_bfloat16* __restrict__ P1,
                                                      __nv_bfloat16* __restrict__ P2) {
  const int kb = blockIdx.x, mb = blockIdx.y;
  const int64_t base = ((int64_t)mb * nkb + kb) * BLK_ELEMS;
  const bool vec = (ld & 3) == 0 && (((uintptr_t)X) & 15) == 0;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int r = (threadIdx.x >> 2) + 64 * h, ko = threadIdx.x & 3;
    const int gr = mb * 128 + r, gc = kb * TK + ko * 8;
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; u++) x[u] = 0.f;
    if (gr < nr) {
      const float* row = X + (rowmap ? (int64_t)rowmap[r0 + gr] : r0 + gr) * ld;
      if (vec && gc + 8 <= nc) {
        const float4 lo = *(const float4*)(row + gc), hi = *(const float4*)(row + gc + 4);
        x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w;
        x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
      } else {
#pragma unroll
        for (int u = 0; u < 8; u++)
          if (gc + u < nc) x[u] = row[gc + u];
      }
    }
    split8_store(x, P0, P1, P2, base + tiled_off(r, ko * 8));
  }
}

// Op[j][i] = Q[i + j*ldq] - (minus_identity && i == j)  (rotation B operand from FP64 Q)
__global__ void __launch_bounds__(256) split_Q_kernel(const double* __restrict__ Q, int64_t ldq, int kin, int kout,
                                                      int minus_identity, int nkb, __nv_bfloat16* __restrict__ P0,
                                                      __nv_bfloat16* __restrict__ P1, __nv_bfloat16* __restrict__ P2) {
  __shared__ __align__(16) __nv_bfloat16 sp[3][BLK_ELEMS];
  const int kb = blockIdx.x, nb = blockIdx.y;
  for (int e = threadIdx.x; e < BLK_ELEMS; e += 256) {
    const int i = e & 31, j = e >> 5;
    const int gi = kb * TK + i, gj = nb * 128 + j;
    float x = 0.f;
    if (gi < kin && gj < kout) {
      double q = Q[gi + (int64_t)gj * ldq];
      if (minus_identity && gi == gj) q -= 1.0;
      x = (float)q;
    }
    __nv_bfloat16 a, b, c;
    split3(x, a, b, c);
    const int o = tiled_off(j, i);
    sp[0][o] = a;
    sp[1][o] = b;
    sp[2][o] = c;
  }
  __syncthreads();
  const int64_t base = ((int64_t)nb * nkb + kb) * BLK_ELEMS;
  for (int e = threadIdx.x; e < BLK_ELEMS / 8; e += 256) {
    ((uint4*)(P0 + base))[e] = ((const uint4*)sp[0])[e];
    ((uint4*)(P1 + base))[e] = ((const uint4*)sp[1])[e];
    ((uint4*)(P2 + base))[e] = ((const uint4*)sp[2])[e];
  }
}

__global__ void mirror_upper_kernel(double* C, int k, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * k) return;
  const int j = (int)(idx / k), i = (int)(idx - (int64_t)j * k);
  if (i > j) C[i + (int64_t)j * ldc] = C[j + (int64_t)i * ldc];
}

__global__ void zero_f64_kernel(double* C, int m, int n, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * n) return;
  const int j = (int)(idx / m), i = (int)(idx - (int64_t)j * m);
  C[i + (int64_t)j * ldc] = 0.0;
}

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int64_t pad_to(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

bool g_attr_set[64] = {false};

cudaError_t prepare_kernel() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && !g_attr_set[dev]) {
    e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    g_attr_set[dev] = true;
  }
  return cudaSuccess;
}

size_t piece_bytes(int64_t mn, int64_t k) { return (size_t)pad_to(mn, TN) * pad_to(k, TK) * 2; }

}  // namespace

bool tc_available() { return true; }

int64_t gram_chunk_rows(int64_t rows, int m, int n) {
  const size_t per_row = (size_t)NPIECE * 2 * (pad_to(m, TN) + pad_to(n, TN));
  int64_t c = (int64_t)(GRAM_PIECE_BUDGET / per_row) / TK * TK;
  c = std::max<int64_t>(GRAM_CHUNK_MIN, std::min<int64_t>(GRAM_CHUNK_MAX, c));
  return std::min<int64_t>(rows, c);
}

size_t gram_pieces_bytes(int m, int n, int64_t chunk) {
  return NPIECE * (kscf_align256(piece_bytes(m, chunk)) + kscf_align256(piece_bytes(n, chunk))) + 256;
}

size_t gram_tc_work_bytes(int64_t rows, int m, int n) { return gram_pieces_bytes(m, n, gram_chunk_rows(rows, m, n)); }

// largest row chunk (multiple of TK, at most GRAM_CHUNK_MAX and rows) whose pieces fit
int64_t gram_chunk_for_work(int64_t rows, int m, int n, size_t work_bytes) {
  const size_t per_row = (size_t)NPIECE * 2 * (pad_to(m, TN) + pad_to(n, TN));
  const size_t slack = 256 + 2 * NPIECE * 256;
  if (work_bytes <= slack) return 0;
  int64_t c = (int64_t)((work_bytes - slack) / per_row) / TK * TK;
  c = std::min<int64_t>(c, std::min<int64_t>(pad_to(rows, TK), GRAM_CHUNK_MAX));
  while (c > 0 && gram_pieces_bytes(m, n, c) > work_bytes) c -= TK;
  return c;
}

size_t rotate_tc_work_bytes(int64_t rows, int kin, int kout) {
  return NPIECE * (kscf_align256(piece_bytes(rows, kin)) + kscf_align256(piece_bytes(kout, kin))) + 256;
}

cudaError_t launch_gram_tc(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t rows, int m, int n,
                           double scale, double* C, int64_t ldc, bool accumulate, void* work, size_t work_bytes,
                           cudaStream_t st, bool symmetric_result, const int32_t* rowmap) {
  // same operand: one set of split pieces (no B pieces), so a chunk twice as long fits
  const bool same = (A == B && lda == ldb && m == n);
  const int64_t chunk = gram_chunk_for_work(rows, m, same ? 0 : n, work_bytes);
  if (chunk < TK && rows > 0) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel();
  if (e != cudaSuccess) return e;
  if (!accumulate) {
    zero_f64_kernel<<<cdiv((int64_t)m * n, 256), 256, 0, st>>>(C, m, n, ldc), count_launch();
  }
  if (rows == 0 || m == 0 || n == 0) return cudaGetLastError();
  // symmetric result (same operand, or a product the caller knows to be symmetric):
  // upper-triangle tiles only, mirrored at the end
  const bool sym = same || (symmetric_result && m == n && !accumulate);
  char* w = (char*)work;
  __nv_bfloat16* Ap[NPIECE];
  __nv_bfloat16* Bp[NPIECE];
  for (int q = 0; q < NPIECE; q++) {
    Ap[q] = (__nv_bfloat16*)w;
    w += kscf_align256(piece_bytes(m, chunk));
  }
  for (int q = 0; q < NPIECE; q++) {
    Bp[q] = (__nv_bfloat16*)w;
    if (!same) w += kscf_align256(piece_bytes(n, chunk));
  }
  GramArgs a = {};
  for (int q = 0; q < NPIECE; q++) {
    a.A[q] = Ap[q];
    a.B[q] = same ? Ap[q] : Bp[q];
  }
  a.m_tiles = cdiv(m, TM);
  a.n_tiles = cdiv(n, GN);
  a.m = m;
  a.n = n;
  a.symmetric = sym ? 1 : 0;
  a.C = C;
  a.ldc = ldc;
  a.scale = scale;
  const int tiles = a.m_tiles * a.n_tiles;
  for (int64_t r0 = 0; r0 < rows; r0 += chunk) {
    const int nr = (int)std::min<int64_t>(chunk, rows - r0);
    const int nkb = cdiv(nr, TK);
    // the Gram kernel reads the column blocks of its 128-wide tiles only
    split_T_kernel<<<dim3(nkb, cdiv(m, TM)), 256, 0, st>>>(A, lda, r0, nr, 0, m, nkb, rowmap, Ap[0], Ap[1], Ap[2]),
        count_launch();
    if (!same)
      split_T_kernel<<<dim3(nkb, cdiv(n, GN)), 256, 0, st>>>(B, ldb, r0, nr, 0, n, nkb, rowmap, Bp[0], Bp[1], Bp[2]),
          count_launch();
    a.nkb = nkb;
    // split the K range over CTAs: pick the split whose active CTAs fill whole waves
    // of one CTA per SM best (the lower-triangle tiles of a symmetric Gram exit at once)
    int active = 0;
    for (int t = 0; t < tiles; t++) {
      const int mt = t % a.m_tiles, nt = t / a.m_tiles;
      if (!(sym && nt * GN + GN - 1 < mt * TM)) active++;
    }
    int ks = 1;
    double best = -1.0;
    const int max_ks = std::max(1, cdiv(nkb, G_SUB_KB));
    for (int cand = 1; cand <= max_ks; cand++) {
      const int kpc = cdiv(cdiv(nkb, cand), G_SUB_KB) * G_SUB_KB;
      const int real = cdiv(nkb, kpc);
      const int64_t ctas = (int64_t)active * real;
      const double waves = (double)((ctas + 151) / 152);
      const double eff = (double)ctas / (waves * 152.0);
      // prefer filled waves, then more parallelism up to ~4 waves
      const double score = eff - 0.02 * std::max(0.0, waves - 4.0) + (ctas >= 152 ? 0.05 : 0.0);
      if (score > best + 1e-9) {
        best = score;
        ks = real;
      }
    }
    a.kb_per_cta = cdiv(cdiv(nkb, ks), G_SUB_KB) * G_SUB_KB;
    ks = cdiv(nkb, a.kb_per_cta);
    tc_gram_kernel<<<dim3(tiles, ks), 320, G_SMEM_BYTES, st>>>(a), count_launch();
  }
  if (sym) mirror_upper_kernel<<<cdiv((int64_t)m * m, 256), 256, 0, st>>>(C, m, ldc), count_launch();
  return cudaGetLastError();
}

cudaError_t launch_rotate_tc(const float* A, int64_t lda, const double* Q, int64_t ldq, int64_t rows, int kin,
                             int kout, bool add_identity_input, float* out, int64_t ldo, void* work,
                             size_t work_bytes, cudaStream_t st, const int32_t* rowmap) {
  if (work_bytes < rotate_tc_work_bytes(rows, kin, kout)) return cudaErrorInvalidValue;
  if (add_identity_input && kin != kout) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel();
  if (e != cudaSuccess) return e;
  if (rows == 0 || kout == 0) return cudaSuccess;
  char* w = (char*)work;
  __nv_bfloat16* Ap[NPIECE];
  __nv_bfloat16* Bp[NPIECE];
  for (int q = 0; q < NPIECE; q++) {
    Ap[q] = (__nv_bfloat16*)w;
    w += kscf_align256(piece_bytes(rows, kin));
  }
  for (int q = 0; q < NPIECE; q++) {
    Bp[q] = (__nv_bfloat16*)w;
    w += kscf_align256(piece_bytes(kout, kin));
  }
  const int nkb = cdiv(kin, TK);
  split_N_kernel<<<dim3(nkb, cdiv(pad_to(rows, TN), 128)), 256, 0, st>>>(A, lda, 0, (int)rows, kin, nkb, rowmap,
                                                                           Ap[0], Ap[1], Ap[2]),
      count_launch();
  split_Q_kernel<<<dim3(nkb, cdiv(pad_to(kout, TN), 128)), 256, 0, st>>>(Q, ldq, kin, kout,
                                                                           add_identity_input ? 1 : 0, nkb, Bp[0],
                                                                           Bp[1], Bp[2]),
      count_launch();
  TcArgs a = {};
  for (int q = 0; q < NPIECE; q++) {
    a.A[q] = Ap[q];
    a.B[q] = Bp[q];
  }
  a.a_nkb = nkb;
  a.b_nkb = nkb;
  a.m_tiles = cdiv(rows, TM);
  a.n_tiles = cdiv(kout, TN);
  a.kb_total = nkb;
  a.n = kout;
  a.out = out;
  a.ldo = ldo;
  a.rows = rows;
  // out = A (Q - I) + A: the epilogue adds A's own element, so out may alias A (the
  // product reads only the bf16 pieces, which are complete before the kernel starts)
  a.addsrc = add_identity_input ? A : nullptr;
  a.ldadd = lda;
  a.rowmap = rowmap;
  int sms = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int ntiles = a.m_tiles * a.n_tiles;
  tc_gemm_kernel<<<std::min(ntiles, sms), 192, SMEM_BYTES, st>>>(a), count_launch();
  return cudaGetLastError();
}

cudaError_t tc_status(bool reset, unsigned int* status) {
  cudaError_t e = cudaMemcpyFromSymbol(status, g_tc_status, sizeof(unsigned int));
  if (e != cudaSuccess) return e;
  if (reset && *status) {
    unsigned int z = 0;
    e = cudaMemcpyToSymbol(g_tc_status, &z, sizeof(unsigned int));
  }
  return e;
}

}  // namespace kscf
