// FP64 Cholesky factorisation of the Gram matrix and the inverse factor, for the
// orthonormalisation step of CheFSI (Cholesky-QR): S = R^T R, W = R^-1, both upper
// triangular, in one cooperative kernel.
//
// Blocked right-looking algorithm over 32 x 32 tiles (tile (I, J) holds rows 32I..32I+31
// and columns 32J..32J+31 of a column-major kp x kp matrix, kp = k rounded up to 32; the
// padding is the identity).  For each block row j:
//   phase B  R_jj = chol(S_jj)                    (factored ahead by CTA 0, see phase C)
//            R_jm = R_jj^-T S_jm      for m > j   (forward substitution, one warp per tile)
//            W_lj = B_lj R_jj^-1      for l <= j  (B_jj = I; B_lj accumulates below)
//   phase C  S_ml -= R_jm^T R_jl      for j < m <= l    (trailing update)
//            B_li -= W_lj R_ji        for l <= j < i    (right-looking R W = I)
// with a grid-wide barrier after each phase.  Look-ahead: in phase C of block row j, CTA 0
// takes only the update of the next diagonal tile S_{j+1,j+1} and then factors it, while
// the other CTAs apply the remaining updates, so that phase B of block row j+1 starts from
// R_{j+1,j+1} instead of a 32-step pivot chain (block row 0 and one-CTA grids factor the
// tile in phase B, in every CTA).  The two triangular recurrences are those of
// the textbook blocked Cholesky and triangular inversion (Golub & Van Loan, Matrix
// Computations, Sec. 4.2 and 3.1); every tile product is FP64 FMA.  On this part FP64
// runs at ~1 TFLOP/s, so the kernel is FP64-ALU bound: 2 k^3 / 3 flop in total.
//
// A pivot counts as failed when it is not above tau_c = S_cc * max((c + 8) u64, floor_rel)
// (or is not finite): (c + 8) u64 S_cc is the rounding level of a Cholesky pivot, so an
// exactly dependent column fails whatever the rounding order; floor_rel > 0 raises it to
// the rounding level of the Gram matrix itself.  Every CTA sees the same failed pivot (its
// own in block row 0, CTA 0's published one after that) and leaves at the same block row.  Barrier waits are bounded (about a second of clock
// cycles); a CTA that gives up sets the timeout word and the others follow.
#include <cuda_runtime.h>

#include <algorithm>

#include "kscf_internal.h"

namespace kscf {
namespace {

constexpr int TB = 32;        // tile edge
constexpr int LDT = TB + 1;   // padded shared-memory tile row
constexpr int NTHR = 256;     // threads per CTA (8 warps)

struct CholArgs {
  const double* S;
  int64_t lds;
  int k, kp, nt;
  double* A;      // kp x kp: the working matrix, R in its upper triangle at the end
  double* W;      // kp x kp: B, then W = R^-1 (upper)
  double* D;      // kp: the diagonal of S before the factorisation
  double* RC;     // kp: 1 / R_cc of the diagonal tiles factored ahead by CTA 0
  double* out;    // k x k output (may alias S): R^-1 upper, zero below
  int64_t ldo;
  unsigned* bar;  // [0] arrival count, [1] generation, [2] failed pivot of a tile factored ahead (1-based) or 0
  int* status;    // [0] first failed pivot (1-based column) or 0, [1] barrier timeout
  double floor_rel;
  long long spin_limit;
  int leave_cta;  // self-test only: this CTA returns before its first barrier (-1: none)
};

__device__ __forceinline__ double ld(const double* p) { return __ldcg(p); }

// Grid-wide barrier for a cooperative launch; false when a wait gave up (or another CTA
// reported that it did).
__device__ bool grid_sync(const CholArgs& a) {
  __shared__ int s_ok;
  if ((int)blockIdx.x == a.leave_cta) return false;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = a.bar + 1;
    volatile int* timeout = a.status + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(a.bar, 1u) == gridDim.x - 1) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (*timeout != 0 || clock64() - t0 > a.spin_limit) {
          atomicExch(a.status + 1, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ int64_t at(int kp, int row, int col) { return (int64_t)row + (int64_t)col * kp; }

// Per-CTA shared state of phase B.
struct TileSmem {
  double T[TB * LDT];   // diagonal tile: S_jj (upper), then R_jj
  double Y[TB * LDT];   // the tile being solved
  double xb[2][TB];     // broadcast row / column, double-buffered across pivots
  double dinv[TB];      // 1 / d_c of the square-root-free elimination
  double piv[TB];       // d_c
  double rc[TB];        // 1 / R_cc
  double dg[TB];        // the diagonal of S for these columns (pivot thresholds)
  int fail;
};

// 1/d for a normal d in (2^-1000, 2^1000): an FP32 seed from the leading 23 mantissa bits
// (relative error < 2^-22), then two Newton-Raphson steps r <- r + r (1 - d r) in FP64,
// each of which squares the relative error (2^-44, then below the FP64 rounding).
__device__ __forceinline__ double recip_pos(double d) {
  const long long bits = __double_as_longlong(d);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  const float mf = __int_as_float(0x3f800000 | (int)((bits >> 29) & 0x7fffff));
  const int fb = __float_as_int(__frcp_rn(mf));          // 1/mf in (0.5, 1]
  const long long fe = ((fb >> 23) & 0xff) - 127;
  double r = __longlong_as_double(((fe - e + 1023) << 52) | ((long long)(fb & 0x7fffff) << 29));
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

__device__ __forceinline__ void bar_factor() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Warps 0-3 (one per SM sub-partition, each FP64 pipe busy): factor the diagonal tile in
// sm.T.  Lane p holds row p; warp w owns columns m = w + 4i.  Square-root-free elimination
// (pivot c: T_pm -= (T_cp / d_c) T_cm for c < p <= m, d_c = T_cc), so that only a
// reciprocal lies on the pivot-to-pivot chain; then R_pm = T_pm / sqrt(d_p).  A failed
// pivot is left in sm.fail.
__device__ void factor_diag4(const CholArgs& a, int j, TileSmem& sm) {
  const int w = threadIdx.x >> 5, p = threadIdx.x & 31;
  volatile int* fail = &sm.fail;
  double t[8];
#pragma unroll
  for (int i = 0; i < 8; i++) t[i] = sm.T[p + (w + 4 * i) * LDT];
#pragma unroll
  for (int c = 0; c < TB; c++) {
    double* buf = sm.xb[c & 1];
    if (p == c) {
#pragma unroll
      for (int i = 0; i < 8; i++)
        if (w + 4 * i >= c) buf[w + 4 * i] = t[i];
      if (w == (c & 3)) {
        const double d = t[c >> 2];
        const int gc = j * TB + c;
        const double tau = fmax(sm.dg[c] * fmax((double)(gc + 8) * 0x1.0p-53, a.floor_rel), 0x1.0p-1000);
        if (!(d > tau) || !(d < 0x1.0p+1000)) {
          *fail = c;
          sm.dinv[c] = 0.0;
        } else {
          sm.dinv[c] = recip_pos(d);
        }
        sm.piv[c] = d;
      }
    }
    bar_factor();
    if (*fail >= 0) return;
    if (p > c) {
      const double g = buf[p] * sm.dinv[c];
#pragma unroll
      for (int i = 0; i < 8; i++)
        if (w + 4 * i > c && p <= w + 4 * i) t[i] = fma(-g, buf[w + 4 * i], t[i]);
    }
  }
  const double r = rsqrt(sm.piv[p]);
#pragma unroll
  for (int i = 0; i < 8; i++) sm.T[p + (w + 4 * i) * LDT] = p <= w + 4 * i ? t[i] * r : 0.0;
  if (w == 0) sm.rc[p] = r;
}

// Warps 0-3: in place on sm.Y, with R = sm.T (upper) and rc = 1 / diag(R):
//   left:  Y <- R^-T Y   (lane = column of Y, warp w owns rows w + 4i)
//   right: Y <- Y R^-1   (lane = row of Y, warp w owns columns w + 4i)
// Both are the forward recurrence x_c = y_c / R_cc, y_p -= R_cp x_c (p > c).
__device__ void tri_solve4(TileSmem& sm, bool left) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  double y[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const int q = w + 4 * i;
    y[i] = left ? sm.Y[q + l * LDT] : sm.Y[l + q * LDT];
  }
#pragma unroll
  for (int c = 0; c < TB; c++) {
    double* buf = sm.xb[c & 1];
    if (w == (c & 3)) {
      y[c >> 2] *= sm.rc[c];
      buf[l] = y[c >> 2];
    }
    bar_factor();
#pragma unroll
    for (int i = 0; i < 8; i++)
      if (w + 4 * i > c) y[i] = fma(-sm.T[c + (w + 4 * i) * LDT], buf[l], y[i]);
  }
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const int q = w + 4 * i;
    if (left)
      sm.Y[q + l * LDT] = y[i];
    else
      sm.Y[l + q * LDT] = y[i];
  }
}

// C -= P^T Q (trans_p) or C -= P Q, all 32 x 32 tiles of column-major kp x kp matrices.
// Thread t: row r = t % 32 of C, columns 4 (t / 32) .. 4 (t / 32) + 3.
__device__ void tile_update(int kp, double* C, const double* P, bool trans_p, const double* Q, double* Ps,
                            double* Qs) {
  const int t = threadIdx.x;
  // Ps[p][r] = op(P)(r, p) = P(p, r) if trans_p else P(r, p);  Qs[p][c] = Q(p, c)
  for (int q = t; q < TB * TB; q += NTHR) {
    const int lo = q & (TB - 1), hi = q >> 5;
    if (trans_p)
      Ps[lo * LDT + hi] = ld(P + at(kp, lo, hi));   // P(lo, hi): p = lo, r = hi
    else
      Ps[hi * LDT + lo] = ld(P + at(kp, lo, hi));   // P(lo, hi): r = lo, p = hi
    Qs[lo * LDT + hi] = ld(Q + at(kp, lo, hi));     // Q(lo, hi): p = lo, c = hi
  }
  __syncthreads();
  const int r = t & 31, c0 = (t >> 5) * 4;
  double acc[4];
#pragma unroll
  for (int u = 0; u < 4; u++) acc[u] = ld(C + at(kp, r, c0 + u));
#pragma unroll 8
  for (int p = 0; p < TB; p++) {
    const double pr = Ps[p * LDT + r];
#pragma unroll
    for (int u = 0; u < 4; u++) acc[u] = fma(-pr, Qs[p * LDT + c0 + u], acc[u]);
  }
#pragma unroll
  for (int u = 0; u < 4; u++) C[at(kp, r, c0 + u)] = acc[u];
  __syncthreads();
}

__global__ void __launch_bounds__(NTHR) chol_inv_kernel(CholArgs a) {
  __shared__ TileSmem sm;
  __shared__ double Ps[TB * LDT];
  __shared__ double Qs[TB * LDT];
  const int kp = a.kp, nt = a.nt;
  const int64_t n2 = (int64_t)kp * kp;
  const int64_t tid = (int64_t)blockIdx.x * NTHR + threadIdx.x, nth = (int64_t)gridDim.x * NTHR;
  // phase 0: A = upper triangle of S (identity padding), W = 0, D = diag(S)
  for (int64_t q = tid; q < n2; q += nth) {
    const int r = (int)(q % kp), c = (int)(q / kp);
    double v = 0.0;
    if (r <= c) v = c < a.k ? a.S[(int64_t)r + (int64_t)c * a.lds] : (r == c ? 1.0 : 0.0);
    a.A[q] = v;
    a.W[q] = 0.0;
  }
  for (int64_t q = tid; q < kp; q += nth) a.D[q] = q < a.k ? a.S[q + q * a.lds] : 1.0;
  if (!grid_sync(a)) return;
  for (int j = 0; j < nt; j++) {
    // phase B: the diagonal tile's factor.  Block row 0 (and a one-CTA grid): every CTA
    // factors it (the same arithmetic everywhere); later block rows: CTA 0 factored it at
    // the end of the previous phase C, as soon as its one update there was done, and every
    // CTA loads R_jj and 1 / R_cc.
    const int r0 = j * TB;
    const bool ahead_done = j > 0 && gridDim.x > 1;
    for (int q = threadIdx.x; q < TB * TB; q += NTHR) {
      const int r = q & (TB - 1), c = q >> 5;
      sm.T[r + c * LDT] = r <= c ? ld(a.A + at(kp, r0 + r, r0 + c)) : 0.0;
    }
    if (ahead_done) {
      if (threadIdx.x < TB) sm.rc[threadIdx.x] = ld(a.RC + r0 + threadIdx.x);
      __syncthreads();
      const int f = (int)__ldcg(a.bar + 2);
      if (f > 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) a.status[0] = f;
        return;
      }
    } else {
      if (threadIdx.x < TB) sm.dg[threadIdx.x] = ld(a.D + r0 + threadIdx.x);
      if (threadIdx.x == 0) sm.fail = -1;
      __syncthreads();
      if (threadIdx.x < 128) factor_diag4(a, j, sm);
      __syncthreads();
      if (sm.fail >= 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) a.status[0] = j * TB + sm.fail + 1;
        return;
      }
    }
    // items: m = j+1 .. nt-1 (panel tiles R_jm), then l = 0 .. j (inverse tiles W_lj)
    for (int it = blockIdx.x; it < nt; it += gridDim.x) {
      const bool left = it < nt - 1 - j;
      const int l = left ? 0 : it - (nt - 1 - j);
      double* tile = left ? a.A + at(kp, r0, (j + 1 + it) * TB) : a.W + at(kp, l * TB, r0);
      for (int q = threadIdx.x; q < TB * TB; q += NTHR) {
        const int r = q & (TB - 1), c = q >> 5;
        sm.Y[r + c * LDT] = (!left && l == j) ? (r == c ? 1.0 : 0.0) : ld(tile + at(kp, r, c));
      }
      __syncthreads();
      if (threadIdx.x < 128) tri_solve4(sm, left);
      __syncthreads();
      for (int q = threadIdx.x; q < TB * TB; q += NTHR) {
        const int r = q & (TB - 1), c = q >> 5;
        tile[at(kp, r, c)] = sm.Y[r + c * LDT];
      }
      __syncthreads();
    }
    if (!grid_sync(a)) return;
    // phase C.  Item 0 is the next diagonal tile (j+1, j+1), whose only update this is: with
    // more than one CTA, CTA 0 takes it alone and then factors the tile while the other CTAs
    // work through items 1, 2, ...
    const int n = nt - 1 - j;
    const int n_trail = n * (n + 1) / 2, n_inv = (j + 1) * n;
    const bool ahead = n >= 1 && gridDim.x > 1;
    const int it_step = ahead ? (blockIdx.x == 0 ? n_trail + n_inv : (int)gridDim.x - 1) : (int)gridDim.x;
    for (int it = blockIdx.x; it < n_trail + n_inv; it += it_step) {
      if (it < n_trail) {
        // it -> (m', l') with 0 <= m' <= l' < n, l'-major
        int lp = (int)((sqrt(8.0 * it + 1.0) - 1.0) * 0.5);
        while ((lp + 1) * (lp + 2) / 2 <= it) lp++;
        while (lp * (lp + 1) / 2 > it) lp--;
        const int mp = it - lp * (lp + 1) / 2;
        const int m = j + 1 + mp, l = j + 1 + lp;
        tile_update(kp, a.A + at(kp, m * TB, l * TB), a.A + at(kp, j * TB, m * TB), true,
                    a.A + at(kp, j * TB, l * TB), Ps, Qs);
      } else {
        const int q = it - n_trail;
        const int l = q % (j + 1), i = j + 1 + q / (j + 1);
        tile_update(kp, a.W + at(kp, l * TB, i * TB), a.W + at(kp, l * TB, j * TB), false,
                    a.A + at(kp, j * TB, i * TB), Ps, Qs);
      }
    }
    if (ahead && blockIdx.x == 0) {
      // factor the updated tile (j+1, j+1) now; publish R (upper), 1 / R_cc and a failure
      const int r1 = (j + 1) * TB;
      __threadfence();   // the tile's update (item 0, this CTA) is read back through L2
      __syncthreads();
      for (int q = threadIdx.x; q < TB * TB; q += NTHR) {
        const int r = q & (TB - 1), c = q >> 5;
        sm.T[r + c * LDT] = r <= c ? ld(a.A + at(kp, r1 + r, r1 + c)) : 0.0;
      }
      if (threadIdx.x < TB) sm.dg[threadIdx.x] = ld(a.D + r1 + threadIdx.x);
      if (threadIdx.x == 0) sm.fail = -1;
      __syncthreads();
      if (threadIdx.x < 128) factor_diag4(a, j + 1, sm);
      __syncthreads();
      if (sm.fail < 0) {
        for (int q = threadIdx.x; q < TB * TB; q += NTHR) {
          const int r = q & (TB - 1), c = q >> 5;
          if (r <= c) a.A[at(kp, r1 + r, r1 + c)] = sm.T[r + c * LDT];
        }
        if (threadIdx.x < TB) a.RC[r1 + threadIdx.x] = sm.rc[threadIdx.x];
      } else if (threadIdx.x == 0) {
        a.bar[2] = (unsigned)((j + 1) * TB + sm.fail + 1);
      }
    }
    if (!grid_sync(a)) return;
  }
  // output: R^-1 (upper) into out, zero below the diagonal
  const int64_t nk = (int64_t)a.k * a.k;
  for (int64_t q = tid; q < nk; q += nth) {
    const int r = (int)(q % a.k), c = (int)(q / a.k);
    a.out[(int64_t)r + (int64_t)c * a.ldo] = r <= c ? a.W[at(kp, r, c)] : 0.0;
  }
}

int grid_for(int nt) {
  static int sms = 0, per_sm = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_inv_kernel, NTHR, 0) != cudaSuccess) return 0;
  }
  int items = nt;
  for (int j = 0; j < nt; j++) {
    const int n = nt - 1 - j;
    items = std::max(items, n * (n + 1) / 2 + (j + 1) * n);
  }
  return std::max(1, std::min(items, sms * std::min(per_sm, 1)));
}

}  // namespace

size_t chol_inv_work_bytes(int k) {
  const size_t kp = (size_t)((k + TB - 1) / TB) * TB;
  return 2 * kscf_align256(kp * kp * 8) + 2 * kscf_align256(kp * 8) + 256;
}

cudaError_t launch_chol_inv(const double* S, int64_t lds, int k, double floor_rel, double* out, int64_t ldo,
                            void* work, int* status, cudaStream_t st, long long spin_limit, int leave_cta) {
  CholArgs a;
  a.S = S;
  a.lds = lds;
  a.k = k;
  a.nt = (k + TB - 1) / TB;
  a.kp = a.nt * TB;
  char* w = (char*)work;
  const size_t mat = kscf_align256((size_t)a.kp * a.kp * 8);
  a.A = (double*)w;
  a.W = (double*)(w + mat);
  a.D = (double*)(w + 2 * mat);
  a.RC = (double*)(w + 2 * mat + kscf_align256((size_t)a.kp * 8));
  a.bar = (unsigned*)(w + 2 * mat + 2 * kscf_align256((size_t)a.kp * 8));
  a.out = out;
  a.ldo = ldo;
  a.status = status;
  a.floor_rel = floor_rel;
  a.spin_limit = spin_limit;
  a.leave_cta = leave_cta;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 3 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(status, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int grid = grid_for(a.nt);
  if (grid < 1) return cudaErrorNotSupported;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)chol_inv_kernel, dim3(grid), dim3(NTHR), args, 0, st);
  count_launch();
  return e;
}

}  // namespace kscf
