// FP64 symmetric eigensolver for the k x k projected Hamiltonian of the Rayleigh-Ritz step
// of CheFSI (arXiv 2303.00790, CheFSI paragraph: Hs = Q Lambda Q^T of the filtered,
// orthonormalised subspace).  Three stages, all on the device:
//
//  1. Householder tridiagonalisation Q_H^T A Q_H = T (Golub & Van Loan, Matrix
//     Computations, Sec. 8.3.1) in one cooperative persistent kernel.  Row i of the
//     trailing matrix lives with CTA i mod P (in shared memory when it fits).  Step j:
//     every CTA updates its rows with the previous step's rank-2 correction
//     A <- A - v w^T - w v^T and forms its rows of p = tau A v in the same pass; one
//     grid-wide barrier; then every CTA forms w = p - (tau/2)(p^T v) v, row j+1 of the
//     updated matrix (published by its owner during the pass) and the next Householder
//     vector from it, redundantly, so that each step costs a single barrier.
//  2. Tridiagonal divide and conquer (Cuppen 1981) with the deflation of Dongarra &
//     Sorensen (1987) and the eigenvector formula of Gu & Eisenstat (1995).  The
//     recursion tree is balanced (node t of depth d covers [t n / 2^d, (t+1) n / 2^d))
//     with leaves of one row; every depth is a batch of independent merges.  Each
//     secular-equation root is solved by one warp with a two-pole rational model of
//     the secular function (the "middle way" of R.-C. Li, 1994) safeguarded by
//     bisection; roots are kept as an offset from their nearer pole.  The merged
//     eigenvectors are diag(Q1, Q2) M, two FP64 GEMMs per merge.
//  3. Back-transformation Z = Q_H Z_T, column-parallel: each CTA holds a few columns of
//     Z_T in shared memory and applies the reflectors from the last to the first.
//
// On this part FP64 issues one warp instruction per 64 cycles per SM sub-partition, so
// every stage is written to keep all four FP64 pipes busy and to keep the dependent
// chains (reductions, square roots, reciprocals) short: reciprocals and reciprocal square
// roots start from an FP32 seed and take two Newton-Raphson steps in FP64.  All waits
// are bounded; a wait that gives up sets a status word that the host reports.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "kscf_internal.h"

namespace kscf {
namespace {

constexpr double EPS = 2.220446049250313e-16;   // 2^-52
constexpr int NT = 256;                           // threads per CTA
constexpr int NW = NT / 32;

// ---------------------------------------------------------------- FP64 helpers ----

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 1/x.  For 2^-1000 < |x| < 2^1000: the reciprocal of the leading mantissa in FP32
// (relative error < 2^-22) scaled by the exponent, then two Newton-Raphson steps
// r <- r + r (1 - |x| r), each squaring the relative error.  Other x: IEEE division.
__device__ __forceinline__ double recip(double x) {
  const double ax = fabs(x);
  if (!(ax > 0x1p-1000 && ax < 0x1p+1000)) return 1.0 / x;
  const long long bits = __double_as_longlong(ax);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  const float m = __int_as_float(0x3f800000 | (int)((bits >> 29) & 0x7fffff));   // [1, 2)
  double r = (double)__frcp_rn(m) * __longlong_as_double((long long)(1023 - e) << 52);
  r = fma(r, fma(-ax, r, 1.0), r);
  r = fma(r, fma(-ax, r, 1.0), r);
  return copysign(r, x);
}

// 1/sqrt(x) for 2^-1000 < x < 2^1000: FP32 seed of the even-exponent mantissa in [1, 4),
// then two Newton-Raphson steps r <- r + r (1 - x r^2) / 2.  Other x: IEEE sqrt.
__device__ __forceinline__ double rsqrt_pos(double x) {
  if (!(x > 0x1p-1000 && x < 0x1p+1000)) return 1.0 / sqrt(x);
  const long long bits = __double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ff) - 1023;
  float m = __int_as_float(0x3f800000 | (int)((bits >> 29) & 0x7fffff));
  if (e & 1) {   // odd exponent: mantissa in [2, 4), even exponent
    m *= 2.0f;
    e -= 1;
  }
  double r = (double)rsqrtf(m) * __longlong_as_double((long long)(1023 - e / 2) << 52);
  double t = x * r;
  r = fma(0.5 * r, fma(-t, r, 1.0), r);
  t = x * r;
  r = fma(0.5 * r, fma(-t, r, 1.0), r);
  return r;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  v = warp_max(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = red[0];
#pragma unroll
  for (int w = 1; w < NW; w++) t = fmax(t, red[w]);
  return t;
}

// exclusive prefix sum of per-thread counts over the CTA; returns the thread's offset and
// the total in *total.  red: NW ints.
__device__ __forceinline__ int block_scan(int v, int* red, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) red[w] = x;
  __syncthreads();
  int base = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < NW; i++) {
    if (i < w) base += red[i];
    tot += red[i];
  }
  *total = tot;
  return base + x - v;
}

// ------------------------------------------------------------- scaling, checks ----

// out[0] = max |A_ij| (as the bit pattern of a non-negative double), out[1] |= 1 when an
// element is not finite
__global__ void absmax_kernel(const double* A, int64_t lda, int n, unsigned long long* out) {
  __shared__ double red[NW];
  double m = 0.0;
  int bad = 0;
  const int64_t total = (int64_t)n * n;
  for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < total; q += (int64_t)gridDim.x * NT) {
    const double v = A[(q % n) + (q / n) * lda];
    if (!isfinite(v)) bad = 1;
    else m = fmax(m, fabs(v));
  }
  m = block_max(m, red);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
    if (bad) atomicOr(out + 1, 1ull);
  }
}

// A <- sym(A) / max|A|: both triangles set to the mean of A_ij and A_ji, scaled.
__global__ void scale_sym_kernel(double* A, int64_t lda, int n, const unsigned long long* amax) {
  const double m = __longlong_as_double((long long)amax[0]);
  const double s = m > 0.0 && amax[1] == 0 ? 1.0 / m : 0.0;
  const int64_t total = (int64_t)n * n;
  for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < total; q += (int64_t)gridDim.x * NT) {
    const int i = (int)(q % n), j = (int)(q / n);
    if (i > j) continue;
    const double v = 0.5 * (A[i + (int64_t)j * lda] + A[j + (int64_t)i * lda]) * s;
    A[i + (int64_t)j * lda] = v;
    A[j + (int64_t)i * lda] = v;
  }
}

__global__ void info_nonfinite_kernel(const unsigned long long* amax, int* info) {
  if (threadIdx.x == 0 && amax[1] != 0) info[2] = 1;
}

// ---------------------------------------------------------- tridiagonalisation ----

struct TriArgs {
  double* A;          // n x n column-major, symmetric, scaled; row i = column i
  int64_t lda;
  int n, P;           // P CTAs; row i belongs to CTA i % P (local index i / P)
  double* d;          // n: diagonal of T
  double* e;          // n: off-diagonal of T (e[i] = T[i+1][i]), e[n-1] = 0
  double* tau;        // n: reflector scalars (tau[j] = 0: no reflection)
  double* V;          // n x n column-major: v_j in V[j+1 .. n-1, j], V[j+1, j] = 1
  double* pbuf;       // 2 n
  double* rowbuf;     // 2 n
  double* dotbuf;     // 2 P
  double* rwg;        // null, or P x n: the row work vectors in global memory (large n)
  unsigned* bar;      // arrival counter, zero at launch
  int* status;        // [0] = 1: a barrier wait gave up
  long long spin_limit;
  int leave_cta;      // self-test only: this CTA returns at its first barrier (-1: none)
};

// Grid-wide barrier of the tridiagonalisation: arrival by a release reduction on a
// monotonic counter, then acquire loads until all P arrivals of this step are seen (the
// bar.sync before and after orders the other threads of the CTA).  Bounded: after
// spin_limit clock cycles, or when another CTA gave up, the status word is set and
// false returned.
__device__ bool tri_barrier(const TriArgs& a, unsigned target, int* s_ok) {
  if ((int)blockIdx.x == a.leave_cta) return false;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.bar) : "memory");
    int ok = 1;
    volatile int* to = a.status;
    const long long t0 = clock64();
    for (;;) {
      unsigned c;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(a.bar) : "memory");
      if (c >= target) break;
      if (*to != 0 || clock64() - t0 > a.spin_limit) {
        atomicExch(a.status, 1);
        ok = 0;
        break;
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Scalars of the Householder reflector of x = r[s .. n-1] (Golub & Van Loan, Sec. 5.1.2,
// without the normalisation v_0 = 1): with |x|^2 = alpha^2 + sigma, beta = -sign(alpha)|x|,
// v = x - beta e_1 (so v_0 = alpha - beta = sign(alpha)(|alpha| + |x|), v_l = x_l after it)
// and tau = 2 / v^T v = 1 / (|x|^2 + |alpha| |x|), (I - tau v v^T) x = beta e_1.  A tail
// negligible against max|A| = 1 (sigma <= eps^2) gives tau = 0, beta = alpha.
// Returns tau, beta, v_0 in sc[0..2].  One thread.
__device__ __forceinline__ void reflector_scalars(double alpha, double sigma, double* sc) {
  if (sigma <= EPS * EPS) {
    sc[0] = 0.0;
    sc[1] = alpha;
    sc[2] = 1.0;
    return;
  }
  const double x2 = fma(alpha, alpha, sigma);
  const double y = rsqrt_pos(x2);
  const double nrm = x2 * y;
  const double aa = fabs(alpha);
  sc[0] = recip(fma(aa, nrm, x2));
  sc[1] = alpha >= 0.0 ? -nrm : nrm;
  sc[2] = alpha >= 0.0 ? aa + nrm : -(aa + nrm);
}

template <bool SMEM>
__global__ void __launch_bounds__(NT, 1) tridiag_kernel(TriArgs a) {
  extern __shared__ __align__(16) double smd[];
  __shared__ double red[NW];
  __shared__ double sc[4];
  __shared__ int s_ok;
  const int n = a.n, P = a.P, cta = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // three rotating vectors: v_j (current), v_{j-1} (previous), the row work vector that
  // becomes v_{j+1}; and w (w_{j-1} during the pass, then w_j)
  double* vc = smd;
  double* vp = smd + n;
  double* wp = smd + 2 * n;
  double* rw = a.rwg ? a.rwg + (int64_t)cta * n : smd + 3 * n;
  double* rows = smd + (a.rwg ? 3 : 4) * n;
  const int nown = cta < n ? (n - cta + P - 1) / P : 0;
  if (n == 1) {
    if (cta == 0 && threadIdx.x == 0) {
      a.d[0] = a.A[0];
      a.e[0] = 0.0;
      a.tau[0] = 0.0;
    }
    return;
  }
  if (SMEM) {
    for (int r = 0; r < nown; r++) {
      const double* src = a.A + (int64_t)(cta + r * P) * a.lda;
      for (int l = threadIdx.x; l < n; l += NT) rows[(int64_t)r * n + l] = src[l];
    }
  }
  // reflector 0 from row 0 of A
  double sg = 0.0;
  for (int l = threadIdx.x; l < n; l += NT) {
    const double x = a.A[l];
    vc[l] = x;
    if (l >= 2) sg = fma(x, x, sg);
  }
  sg = warp_sum(sg);
  if (lane == 0) red[warp] = sg;
  __syncthreads();
  if (warp == 0) {
    double t = lane < NW ? red[lane] : 0.0;
    t += __shfl_xor_sync(0xffffffffu, t, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    if (lane == 0) reflector_scalars(vc[1], t, sc);
  }
  __syncthreads();
  double tj = sc[0];
  const double d0 = vc[0];
  __syncthreads();
  if (threadIdx.x == 0) vc[1] = sc[2];
  __syncthreads();
  if (cta == 0) {
    for (int l = 1 + threadIdx.x; l < n; l += NT) a.V[l] = vc[l];
    if (threadIdx.x == 0) {
      a.d[0] = d0;
      a.e[0] = sc[1];
      a.tau[0] = tj;
    }
  }
  for (int j = 0; j <= n - 2; j++) {
    const int par = j & 1;
    double* pb = a.pbuf + (int64_t)par * n;
    double* rb = a.rowbuf + (int64_t)par * n;
    // pass over the owned rows i > j: A^(j) = A^(j-1) - v w^T - w v^T, p_i = tau_j A^(j)_i. v_j
    double dotp = 0.0;
    const int r0 = j + 1 > cta ? (j + 1 - cta + P - 1) / P : 0;
    const bool upd = !SMEM && j >= 1;   // shared-memory rows were updated in the last step
    for (int r = r0 + warp; r < nown; r += NW) {
      const int i = cta + r * P;
      double* row = SMEM ? rows + (int64_t)r * n : a.A + (int64_t)i * a.lda;
      const double vpi = upd ? vp[i] : 0.0, wpi = upd ? wp[i] : 0.0;
      const bool pub = i == j + 1;
      double acc0 = 0.0, acc1 = 0.0;
      for (int l = j + 1 + lane; l < n; l += 8 * 32) {
        double x[8];
#pragma unroll
        for (int q = 0; q < 8; q++) x[q] = l + 32 * q < n ? row[l + 32 * q] : 0.0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int ll = l + 32 * q;
          if (ll < n) {
            double y = x[q];
            if (upd) {
              y = fma(-vpi, wp[ll], fma(-wpi, vp[ll], y));
              row[ll] = y;
            }
            if (pub) rb[ll] = y;
            if (q & 1) acc1 = fma(y, vc[ll], acc1);
            else acc0 = fma(y, vc[ll], acc0);
          }
        }
      }
      const double pi = warp_sum(acc0 + acc1) * tj;
      if (lane == 0) {
        pb[i] = pi;
        dotp = fma(pi, vc[i], dotp);
      }
    }
    if (lane == 0) red[warp] = dotp;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < NW; w++) s += red[w];
      a.dotbuf[par * P + cta] = s;
    }
    if (!tri_barrier(a, (unsigned)P * (unsigned)(j + 1), &s_ok)) return;
    // every CTA: K = tau/2 p.v, w_j = p - K v_j, row j+1 of A^(j+1), next reflector.
    // The first 4 NT elements of p and of the published row are loaded before the
    // reduction of K so that the two L2 round trips overlap.
    const int l0 = j + 1 + threadIdx.x;
    double pv[4], rv[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int ll = l0 + q * NT;
      pv[q] = ll < n ? __ldcg(pb + ll) : 0.0;
      rv[q] = ll < n ? __ldcg(rb + ll) : 0.0;
    }
    const double p1 = __ldcg(pb + j + 1);
    if (warp == 0) {
      double s = 0.0;
      for (int c = lane; c < P; c += 32) s += __ldcg(a.dotbuf + par * P + c);
      s = warp_sum(s);
      if (lane == 0) sc[3] = 0.5 * tj * s;
    }
    __syncthreads();
    const double K = sc[3];
    const double v1 = vc[j + 1];
    const double w1 = fma(-K, v1, p1);   // w_j[j+1]
    double sig = 0.0;
    for (int l = l0; l < n; l += 4 * NT) {
      if (l > l0) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int ll = l + q * NT;
          pv[q] = ll < n ? __ldcg(pb + ll) : 0.0;
          rv[q] = ll < n ? __ldcg(rb + ll) : 0.0;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int ll = l + q * NT;
        if (ll < n) {
          const double vl = vc[ll];
          const double wl = fma(-K, vl, pv[q]);
          const double x = fma(-w1, vl, fma(-v1, wl, rv[q]));
          wp[ll] = wl;
          rw[ll] = x;
          if (ll >= j + 3) sig = fma(x, x, sig);
        }
      }
    }
    sig = warp_sum(sig);
    if (lane == 0) red[warp] = sig;
    __syncthreads();
    if (j <= n - 3) {
      if (warp == 0) {
        double t = lane < NW ? red[lane] : 0.0;
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        if (lane == 0) {
          const double dj = rw[j + 1];
          reflector_scalars(rw[j + 2], t, sc);
          rw[j + 2] = sc[2];        // v_{j+1} = rw with its first element replaced
          sc[3] = dj;
        }
      } else if (SMEM && (warp & 3) != 0) {
        // meanwhile the warps of the other three SM sub-partitions (whose FP64 pipes the
        // scalar chain does not use) update the owned rows i >= j+2 to A^(j+1) over the
        // columns l >= j+2, in items of one row x 256 columns
        const int u = (warp >> 2) * 3 + (warp & 3) - 1;
        const int rs = j + 2 > cta ? (j + 2 - cta + P - 1) / P : 0;
        const int nch = (n - (j + 2) + 255) / 256;
        const int items = (nown - rs) * nch;
        for (int it = u; it < items; it += NW - NW / 4) {
          const int r = rs + it / nch;
          const int i = cta + r * P;
          double* row = rows + (int64_t)r * n;
          const double vi = vc[i], wi = wp[i];
          const int lb = j + 2 + (it % nch) * 256 + lane;
          double x[8];
#pragma unroll
          for (int q = 0; q < 8; q++) x[q] = lb + 32 * q < n ? row[lb + 32 * q] : 0.0;
#pragma unroll
          for (int q = 0; q < 8; q++) {
            const int ll = lb + 32 * q;
            if (ll < n) row[ll] = fma(-vi, wp[ll], fma(-wi, vc[ll], x[q]));
          }
        }
      }
      __syncthreads();
      tj = sc[0];
      const int wcta = (j + 1) % P;
      if (cta == wcta) {
        for (int l = j + 2 + threadIdx.x; l < n; l += NT) a.V[l + (int64_t)(j + 1) * n] = rw[l];
        if (threadIdx.x == 0) {
          a.d[j + 1] = sc[3];
          a.e[j + 1] = sc[1];
          a.tau[j + 1] = tj;
        }
      }
      double* t = vp;   // v_{j-1} is free: it becomes the next work vector
      vp = vc;
      vc = rw;
      rw = t;
    } else if (cta == 0 && threadIdx.x == 0) {
      a.d[n - 1] = rw[n - 1];
      a.e[n - 1] = 0.0;
      a.tau[n - 1] = 0.0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- divide and conquer ----
//
// Node t of depth d covers rows [a, c) with a = floor(t n / 2^d), c = floor((t+1) n / 2^d),
// split at b = floor((2t+1) n / 2^(d+1)); a node with c - a >= 2 is a merge of its two
// children.  Per-merge arrays are indexed from a (merges of one depth are disjoint).

__device__ __forceinline__ void node_range(int n, int d, int t, int* a, int* b, int* c) {
  *a = (int)(((long long)t * n) >> d);
  *c = (int)(((long long)(t + 1) * n) >> d);
  *b = (int)(((long long)(2 * t + 1) * n) >> (d + 1));
}

struct DcArgs {
  int n;
  int64_t ldz;           // leading dimension of Z, Zt (column-major) and M, W (row-major)
  double* lam;           // n: eigenvalues of the current blocks, ascending per block
  double* es;            // n: scaled off-diagonal, negligible entries zeroed
  double* Z;             // eigenvectors of the current blocks (diagonal blocks)
  double* Zt;            // GEMM output, then rotation workspace W
  double* M;             // row-major merge matrices
  double* Ds;            // sorted pole values (rotated by deflation)
  double* zs;            // sorted z
  double* dk;            // kept poles
  double* zk;            // kept z
  double* zz;            // kept z^2
  double* tauk;          // root offset from its origin pole
  double* lamk;          // root value
  double* zh;            // Gu-Eisenstat z
  double* invn;          // 1 / |u_j|
  double* rc;            // rotation cosines
  double* rsn;           // rotation sines
  int* idx;              // sorted position -> local input index
  int* stat;             // sorted position: 0 kept, 1 deflated
  int* ntp;              // non-type-1 sorted positions, compacted
  int* kidx;             // sorted position -> kept index or -1
  int* orig;             // kept root -> origin pole (kept index)
  int* colref;           // final column -> kept root j (>= 0) or ~sorted position
  int* rp;               // rotation first position
  int* rt;               // rotation second position
  int* Kof;              // at a: kept count
  int* nrot;             // at a: rotation count
  int* cand;             // candidate flags per compacted position
  int* status;           // [1] += secular roots that did not converge
};

// leaves: scale T to max 1, zero negligible couplings, tear every coupling
// (lam_i = d_i - |e_{i-1}| - |e_i|), Z = I on the diagonal.  One CTA.
__global__ void dc_leaves_kernel(DcArgs a, const double* d, const double* e, double* tscale) {
  __shared__ double red[NW];
  const int n = a.n;
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) m = fmax(m, fmax(fabs(d[i]), i < n - 1 ? fabs(e[i]) : 0.0));
  m = block_max(m, red);
  const double s = m > 0.0 ? 1.0 / m : 0.0;
  for (int i = threadIdx.x; i < n; i += NT) {
    const double ei = i < n - 1 ? e[i] * s : 0.0;
    a.es[i] = fabs(ei) <= EPS ? 0.0 : ei;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += NT) {
    double v = d[i] * s;
    if (i > 0) v -= fabs(a.es[i - 1]);
    if (i < n - 1) v -= fabs(a.es[i]);
    a.lam[i] = v;
    a.Z[i + (int64_t)i * a.ldz] = 1.0;
  }
  if (threadIdx.x == 0) tscale[0] = m;
}

// count of x[0..len) < v (strict) or <= v
__device__ __forceinline__ int lower_count(const double* x, int len, double v, bool strict) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const bool less = strict ? x[mid] < v : x[mid] <= v;
    if (less) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One CTA per merge: z, the sorted merge of the two pole lists, deflation.
__device__ void dc_deflate_node(const DcArgs& a, int A0, int B0, int C0) {
  __shared__ double red[NW];
  __shared__ int ired[NW];
  const int N = C0 - A0, n1 = B0 - A0;
  const int64_t ld = a.ldz;
  const double beta = a.es[B0 - 1];
  const double sgn = beta >= 0.0 ? 1.0 : -1.0;
  const double rho = 2.0 * fabs(beta);
  const double r2 = 0.70710678118654752440;
  double* Ds = a.Ds + A0;
  double* zs = a.zs + A0;
  int* idx = a.idx + A0;
  int* stat = a.stat + A0;
  double dmax = 0.0;
  for (int i = threadIdx.x; i < N; i += NT) {
    const double v = a.lam[A0 + i];
    int pos;
    double z;
    if (i < n1) {
      pos = i + lower_count(a.lam + B0, C0 - B0, v, true);
      z = a.Z[(B0 - 1) + (int64_t)(A0 + i) * ld] * r2;
    } else {
      pos = (i - n1) + lower_count(a.lam + A0, n1, v, false);
      z = sgn * a.Z[B0 + (int64_t)(A0 + i) * ld] * r2;
    }
    Ds[pos] = v;
    zs[pos] = z;
    idx[pos] = i;
    dmax = fmax(dmax, fabs(v));
  }
  dmax = block_max(dmax, red);
  const double tol = 8.0 * EPS * fmax(dmax, rho);
  // type 1: rho |z| <= tol; compaction of the others (sorted order)
  const int per = (N + NT - 1) / NT;
  const int lo = threadIdx.x * per, hi = min(N, lo + per);
  int cnt = 0;
  for (int t = lo; t < hi; t++) cnt += rho * fabs(zs[t]) > tol;
  int tot;
  int off = block_scan(cnt, ired, &tot);
  int* ntp = a.ntp + A0;
  int* cand = a.cand + A0;
  for (int t = lo; t < hi; t++) {
    const bool keep = rho * fabs(zs[t]) > tol;
    stat[t] = keep ? 0 : 1;
    if (keep) ntp[off++] = t;
  }
  __syncthreads();
  const int m = tot;
  // candidate pairs (u-1, u) of the compacted list: only those closer than 2 tol can
  // deflate (|c s| <= 1/2), and a rotation only widens the next gap
  for (int u = threadIdx.x; u < m; u += NT)
    cand[u] = u > 0 && Ds[ntp[u]] - Ds[ntp[u - 1]] <= 2.0 * tol;
  __syncthreads();
  if (threadIdx.x == 0) a.nrot[A0] = 0;
  __syncthreads();
  // each chain of consecutive candidate pairs is walked by one thread, in order
  for (int u = threadIdx.x; u + 1 < m; u += NT) {
    if (!cand[u + 1] || (u > 0 && cand[u])) continue;
    for (int v = u; v + 1 < m && cand[v + 1]; v++) {
      const int p = ntp[v], t = ntp[v + 1];
      const double zp = zs[p], zt = zs[t];
      const double r = hypot(zp, zt);
      const double c = zt / r, s = zp / r;
      const double dp = Ds[p], dt = Ds[t];
      if (fabs(c * s * (dt - dp)) <= tol) {
        const int q = atomicAdd(a.nrot + A0, 1);
        a.rp[A0 + q] = p;
        a.rt[A0 + q] = t;
        a.rc[A0 + q] = c;
        a.rsn[A0 + q] = s;
        Ds[p] = c * c * dp + s * s * dt;
        Ds[t] = s * s * dp + c * c * dt;
        zs[p] = 0.0;
        zs[t] = r;
        stat[p] = 1;
      }
    }
  }
  __syncthreads();
  // kept compaction
  cnt = 0;
  for (int t = lo; t < hi; t++) cnt += stat[t] == 0;
  off = block_scan(cnt, ired, &tot);
  for (int t = lo; t < hi; t++) {
    if (stat[t] == 0) {
      a.kidx[A0 + t] = off;
      a.dk[A0 + off] = Ds[t];
      a.zk[A0 + off] = zs[t];
      a.zz[A0 + off] = zs[t] * zs[t];
      off++;
    } else {
      a.kidx[A0 + t] = -1;
    }
  }
  if (threadIdx.x == 0) a.Kof[A0] = tot;
}

__global__ void __launch_bounds__(NT) dc_deflate_kernel(DcArgs a, int depth) {
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.x, &A0, &B0, &C0);
  if (C0 - A0 >= 2) dc_deflate_node(a, A0, B0, C0);
}

// Secular equation 1 + rho sum_i z_i^2 / (d_i - lambda) = 0, one warp per root j of the K
// kept poles d_0 < ... < d_{K-1}.  Root j lies in (d_j, d_{j+1}) (j < K-1) or in
// (d_{K-1}, d_{K-1} + rho |z|^2].  The origin is the nearer pole (sign of the secular
// function at the midpoint); lambda = d_o + tau with tau bracketed in (lo, hi).  Each
// iteration evaluates psi (poles i <= j) and phi (poles i > j) with their derivatives,
// replaces each by a + b / (d_pole - tau) through the current point (pole d_j for psi,
// d_{j+1} for phi; one pole for the last root) and takes the root of that model inside
// the bracket, else bisects.  Stops when |g| is below its rounding bound or the bracket
// has collapsed.
__device__ void dc_secular_root(const DcArgs& a, int A0, int B0, int K, int j) {
  const int lane = threadIdx.x & 31;
  const double rho = 2.0 * fabs(a.es[B0 - 1]);
  const double* dk = a.dk + A0;
  const double* zz = a.zz + A0;
  int o;
  double lo, hi;
  if (j < K - 1) {
    const double mid = 0.5 * (dk[j + 1] - dk[j]);
    double f = 0.0;
    for (int i = lane; i < K; i += 32) f += zz[i] * recip((dk[i] - dk[j]) - mid);
    f = 1.0 + rho * warp_sum(f);
    if (f >= 0.0) {
      o = j;
      lo = 0.0;
      hi = mid;
    } else {
      o = j + 1;
      lo = -mid;
      hi = 0.0;
    }
  } else {
    double s = 0.0;
    for (int i = lane; i < K; i += 32) s += zz[i];
    o = K - 1;
    lo = 0.0;
    hi = rho * warp_sum(s);
  }
  const double dorg = dk[o];
  const double dl = dk[j] - dorg;
  const double dr = j < K - 1 ? dk[j + 1] - dorg : 0.0;
  double tau = 0.5 * (lo + hi);
  bool conv = false;
  for (int it = 0; it < 64; it++) {
    double ps = 0.0, dps = 0.0, ph = 0.0, dph = 0.0;
    for (int i = lane; i < K; i += 32) {
      const double r = recip((dk[i] - dorg) - tau);
      const double t1 = zz[i] * r;
      if (i <= j) {
        ps += t1;
        dps = fma(t1, r, dps);
      } else {
        ph += t1;
        dph = fma(t1, r, dph);
      }
    }
    ps = rho * warp_sum(ps);
    dps = rho * warp_sum(dps);
    ph = rho * warp_sum(ph);
    dph = rho * warp_sum(dph);
    const double g = 1.0 + ps + ph;
    if (g < 0.0) lo = tau;
    else hi = tau;
    const double bound = 8.0 * EPS * (K * (fabs(ps) + fabs(ph)) + 1.0);
    if (fabs(g) <= bound || hi - lo <= 2.0 * EPS * fmax(fabs(lo), fabs(hi))) {
      conv = true;
      break;
    }
    double nt = lo - 1.0;   // outside the bracket: bisect unless the model gives a root
    if (j < K - 1) {
      const double el = dl - tau, er = dr - tau;
      const double B1 = dps * el * el, A1 = ps - dps * el;
      const double B2 = dph * er * er, A2 = ph - dph * er;
      const double c = 1.0 + A1 + A2;
      const double bq = c * (dl + dr) + B1 + B2;
      const double cq = c * dl * dr + B1 * dr + B2 * dl;
      const double disc = bq * bq - 4.0 * c * cq;
      if (disc >= 0.0) {
        const double sq = sqrt(disc);
        if (c != 0.0) {
          const double x1 = (bq + copysign(sq, bq)) * 0.5 * recip(c);
          if (x1 > lo && x1 < hi) nt = x1;
          if (x1 != 0.0) {
            const double x2 = cq * recip(c * x1);
            if (x2 > lo && x2 < hi) nt = x2;
          }
        } else if (bq != 0.0) {
          nt = cq * recip(bq);
        }
      }
    } else {
      const double el = dl - tau;
      const double B1 = dps * el * el;
      const double c = g - B1 * recip(el);
      if (c != 0.0) nt = dl + B1 * recip(c);
    }
    tau = nt > lo && nt < hi ? nt : 0.5 * (lo + hi);
  }
  if (lane == 0) {
    a.orig[A0 + j] = o;
    a.tauk[A0 + j] = tau;
    a.lamk[A0 + j] = dorg + tau;
    if (!conv) atomicAdd(a.status + 1, 1);
  }
}

__global__ void __launch_bounds__(NT) dc_secular_kernel(DcArgs a, int depth) {
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.y, &A0, &B0, &C0);
  if (C0 - A0 < 2) return;
  const int K = a.Kof[A0];
  const int j = blockIdx.x * NW + (threadIdx.x >> 5);
  if (j < K) dc_secular_root(a, A0, B0, K, j);
}

// Gu-Eisenstat: zh_i^2 = prod_j (lambda_j - d_i) / (rho prod_{j != i} (d_j - d_i)), the
// sign of z_i; lambda_j - d_i = (d_{o_j} - d_i) + tau_j.  One warp per kept pole.
__device__ void dc_zhat_one(const DcArgs& a, int A0, int B0, int K, int i) {
  const int lane = threadIdx.x & 31;
  const double rho = 2.0 * fabs(a.es[B0 - 1]);
  const double* dk = a.dk + A0;
  const double di = dk[i];
  double p = 1.0;
  for (int jj = lane; jj < K; jj += 32) {
    const double num = (dk[min(max(a.orig[A0 + jj], 0), K - 1)] - di) + a.tauk[A0 + jj];
    p *= jj == i ? num : num * recip(dk[jj] - di);
  }
  p = warp_prod(p);
  if (lane == 0) a.zh[A0 + i] = copysign(sqrt(fabs(p) * recip(rho)), a.zk[A0 + i]);
}

__global__ void __launch_bounds__(NT) dc_zhat_kernel(DcArgs a, int depth) {
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.y, &A0, &B0, &C0);
  if (C0 - A0 < 2) return;
  const int K = a.Kof[A0];
  const int i = blockIdx.x * NW + (threadIdx.x >> 5);
  if (i < K) dc_zhat_one(a, A0, B0, K, i);
}

// 1 / |u_j|, u_j[i] = zh_i / (d_i - lambda_j).  One warp per root.
__device__ void dc_colnorm_one(const DcArgs& a, int A0, int K, int j) {
  const int lane = threadIdx.x & 31;
  const double* dk = a.dk + A0;
  const double dorg = dk[min(max(a.orig[A0 + j], 0), K - 1)], tau = a.tauk[A0 + j];
  double s = 0.0;
  for (int i = lane; i < K; i += 32) {
    const double u = a.zh[A0 + i] * recip((dk[i] - dorg) - tau);
    s = fma(u, u, s);
  }
  s = warp_sum(s);
  if (lane == 0) a.invn[A0 + j] = rsqrt_pos(s);
}

__global__ void __launch_bounds__(NT) dc_colnorm_kernel(DcArgs a, int depth) {
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.y, &A0, &B0, &C0);
  if (C0 - A0 < 2) return;
  const int K = a.Kof[A0];
  const int j = blockIdx.x * NW + (threadIdx.x >> 5);
  if (j < K) dc_colnorm_one(a, A0, K, j);
}

// order-preserving integer key of a double
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Final ascending order of the merge's N eigenvalues (kept roots and deflated poles):
// bitonic sort of (key, reference) pairs in shared memory; lam[a + col] and colref.
__device__ void dc_order_node(const DcArgs& a, int A0, int N, unsigned long long* key, int* ref) {
  const int K = a.Kof[A0];
  int p2 = 1;
  while (p2 < N) p2 <<= 1;
  // kept roots first (j), then the deflated sorted positions (~t)
  for (int q = threadIdx.x; q < p2; q += NT) {
    key[q] = ~0ull;
    ref[q] = 0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < K; j += NT) {
    key[j] = dkey(a.lamk[A0 + j]);
    ref[j] = j;
  }
  __shared__ int ired[NW];
  const int per = (N + NT - 1) / NT;
  const int lo = threadIdx.x * per, hi = min(N, lo + per);
  int cnt = 0;
  for (int t = lo; t < hi; t++) cnt += a.stat[A0 + t] != 0;
  int tot;
  int off = block_scan(cnt, ired, &tot);
  for (int t = lo; t < hi; t++) {
    if (a.stat[A0 + t] != 0) {
      key[K + off] = dkey(a.Ds[A0 + t]);
      ref[K + off] = ~t;
      off++;
    }
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int q = threadIdx.x; q < p2; q += NT) {
        const int pq = q ^ jj;
        if (pq > q) {
          const bool up = (q & k) == 0;
          const unsigned long long kq = key[q], kp = key[pq];
          if ((kq > kp) == up) {
            key[q] = kp;
            key[pq] = kq;
            const int rq = ref[q];
            ref[q] = ref[pq];
            ref[pq] = rq;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int col = threadIdx.x; col < N; col += NT) {
    const int r = ref[col];
    a.colref[A0 + col] = r;
    a.lam[A0 + col] = r >= 0 ? a.lamk[A0 + min(r, N - 1)] : a.Ds[A0 + min(~r, N - 1)];
  }
}

__global__ void __launch_bounds__(NT) dc_order_kernel(DcArgs a, int depth, int npow) {
  extern __shared__ __align__(16) unsigned char smb[];
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.x, &A0, &B0, &C0);
  if (C0 - A0 < 2) return;
  dc_order_node(a, A0, C0 - A0, (unsigned long long*)smb, (int*)((unsigned long long*)smb + npow));
}

// Merge matrix M (row-major, rows = input columns of diag(Q1, Q2) in block order, columns =
// merged eigenvectors in ascending order).  Column of kept root j: u_j[i] = zh_i /
// (d_i - lambda_j) / |u_j| at the sorted position of kept pole i; column of deflated
// position t: e_t.  With deflation rotations the columns go to W (rows = sorted
// positions) for dc_rotperm_kernel, else straight to M through the sort permutation.
// Tile: 32 columns x 64 rows per CTA.
// value of the merge matrix at sorted position t, final column with reference r (kept
// root j >= 0, or ~deflated position), with the root's origin pole, offset and 1/|u_j|
__device__ __forceinline__ double dc_m_value(const DcArgs& a, int A0, int K, int t, int r, double dorg, double tau,
                                             double inv) {
  if (r >= 0) {
    const int ki = a.kidx[A0 + t];
    return ki >= 0 && ki < K ? a.zh[A0 + ki] * recip((a.dk[A0 + ki] - dorg) - tau) * inv : 0.0;
  }
  return t == ~r ? 1.0 : 0.0;
}

// column reference of a final column, guarded (only a failed sort gives a bad one), and
// its root's origin pole, offset and 1/|u_j|
__device__ __forceinline__ int dc_col_ref(const DcArgs& a, int A0, int N, int K, int col, double* dorg, double* tau,
                                          double* inv) {
  int r = a.colref[A0 + col];
  if (r >= K || (r < 0 && ~r >= N)) r = ~0;
  *dorg = 0.0;
  *tau = 0.0;
  *inv = 0.0;
  if (r >= 0) {
    *dorg = a.dk[A0 + min(max(a.orig[A0 + r], 0), K - 1)];
    *tau = a.tauk[A0 + r];
    *inv = a.invn[A0 + r];
  }
  return r;
}

// rotations (last to first) and the sort permutation for one column of W -> M
__device__ void dc_rotperm_col(const DcArgs& a, int A0, int N, int col) {
  const int64_t ld = a.ldz;
  const int nr = a.nrot[A0];
  double* Wc = a.Zt + A0 + col;
  for (int q = min(nr, N) - 1; q >= 0; q--) {
    const int p = min(max(a.rp[A0 + q], 0), N - 1), t = min(max(a.rt[A0 + q], 0), N - 1);
    const double c = a.rc[A0 + q], s = a.rsn[A0 + q];
    const double wp = Wc[(int64_t)(A0 + p) * ld], wt = Wc[(int64_t)(A0 + t) * ld];
    Wc[(int64_t)(A0 + p) * ld] = fma(c, wp, s * wt);
    Wc[(int64_t)(A0 + t) * ld] = fma(c, wt, -s * wp);
  }
  for (int t = 0; t < N; t++)
    a.M[(int64_t)(A0 + min(max(a.idx[A0 + t], 0), N - 1)) * ld + A0 + col] = Wc[(int64_t)(A0 + t) * ld];
}

__global__ void __launch_bounds__(NT) dc_build_m_kernel(DcArgs a, int depth) {
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.z, &A0, &B0, &C0);
  const int N = C0 - A0;
  if (N < 2) return;
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int t0 = blockIdx.y * 64 + (threadIdx.x >> 5);
  if (col >= N || t0 >= N) return;
  const int64_t ld = a.ldz;
  const bool rot = a.nrot[A0] > 0;
  const int K = a.Kof[A0];
  double dorg, tau, inv;
  const int r = dc_col_ref(a, A0, N, K, col, &dorg, &tau, &inv);
  for (int t = t0; t < min(N, blockIdx.y * 64 + 64); t += NW) {
    const double v = dc_m_value(a, A0, K, t, r, dorg, tau, inv);
    if (rot) a.Zt[(int64_t)(A0 + t) * ld + A0 + col] = v;
    else a.M[(int64_t)(A0 + min(max(a.idx[A0 + t], 0), N - 1)) * ld + A0 + col] = v;
  }
}

// With deflation rotations: M = P R_1 ... R_m W, R_q acting on rows (p_q, t_q) as
// [[c, s], [-s, c]]; applied from the last to the first, then the sort permutation
// (row t of the rotated W is row idx[t] of M).  One thread per column.
__global__ void __launch_bounds__(NT) dc_rotperm_kernel(DcArgs a, int depth) {
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.y, &A0, &B0, &C0);
  const int N = C0 - A0;
  if (N < 2 || a.nrot[A0] == 0) return;
  const int col = blockIdx.x * NT + threadIdx.x;
  if (col < N) dc_rotperm_col(a, A0, N, col);
}

// Merges of at most 32 rows (the lowest depths, many small merges): one CTA per merge runs
// every phase above in one launch, the phases separated by __syncthreads (the per-merge
// arrays live in global memory and stay in L1/L2), the two block products element-wise.
constexpr int DC_SMALL = 32;
__global__ void __launch_bounds__(NT) dc_small_kernel(DcArgs a, int depth) {
  __shared__ unsigned long long key[DC_SMALL];
  __shared__ int ref[DC_SMALL];
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.x, &A0, &B0, &C0);
  const int N = C0 - A0, n1 = B0 - A0;
  if (N < 2) return;
  const int warp = threadIdx.x >> 5;
  const int64_t ld = a.ldz;
  dc_deflate_node(a, A0, B0, C0);
  __syncthreads();
  const int K = a.Kof[A0];
  for (int j = warp; j < K; j += NW) dc_secular_root(a, A0, B0, K, j);
  __syncthreads();
  for (int i = warp; i < K; i += NW) dc_zhat_one(a, A0, B0, K, i);
  __syncthreads();
  for (int j = warp; j < K; j += NW) dc_colnorm_one(a, A0, K, j);
  __syncthreads();
  dc_order_node(a, A0, N, key, ref);
  __syncthreads();
  const bool rot = a.nrot[A0] > 0;
  for (int q = threadIdx.x; q < N * N; q += NT) {
    const int t = q / N, col = q - t * N;
    double dorg, tau, inv;
    const int r = dc_col_ref(a, A0, N, K, col, &dorg, &tau, &inv);
    const double v = dc_m_value(a, A0, K, t, r, dorg, tau, inv);
    if (rot) a.Zt[(int64_t)(A0 + t) * ld + A0 + col] = v;
    else a.M[(int64_t)(A0 + min(max(a.idx[A0 + t], 0), N - 1)) * ld + A0 + col] = v;
  }
  __syncthreads();
  if (rot)
    for (int col = threadIdx.x; col < N; col += NT) dc_rotperm_col(a, A0, N, col);
  __syncthreads();
  // Zt[r, col] = sum_k Z[r, k] M[k, col] over the block of row r
  for (int q = threadIdx.x; q < N * N; q += NT) {
    const int col = q / N, r = q - col * N;
    const int k0 = r < n1 ? 0 : n1, k1 = r < n1 ? n1 : N;
    double acc = 0.0;
    for (int k = k0; k < k1; k++)
      acc = fma(a.Z[(int64_t)(A0 + r) + (int64_t)(A0 + k) * ld], a.M[(int64_t)(A0 + k) * ld + A0 + col], acc);
    a.Zt[(int64_t)(A0 + r) + (int64_t)(A0 + col) * ld] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < N * N; q += NT) {
    const int col = q / N, r = q - col * N;
    a.Z[(int64_t)(A0 + r) + (int64_t)(A0 + col) * ld] = a.Zt[(int64_t)(A0 + r) + (int64_t)(A0 + col) * ld];
  }
}

// Batched FP64 GEMM of the merge: Zt[a:b, a:c] = Z[a:b, a:b] M[a:b, a:c] and
// Zt[b:c, a:c] = Z[b:c, b:c] M[b:c, a:c] (Z, Zt column-major, M row-major).  32 x 64
// output tile per CTA (small tiles: the top merges have only a few hundred tiles for 152
// SMs), 2 x 4 per thread, k-steps of 16 through shared memory.  blockIdx.x: column tile;
// blockIdx.y: row tile (first the rt1 tiles of block 1, then those of block 2);
// blockIdx.z: node.
constexpr int GTM = 32, GTN = 64, GTK = 16;
__global__ void __launch_bounds__(NT) dc_gemm_kernel(DcArgs a, int depth, int rt1) {
  __shared__ __align__(16) double As[GTK][GTM];
  __shared__ __align__(16) double Bs[GTK][GTN];
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.z, &A0, &B0, &C0);
  const int N = C0 - A0;
  if (N < 2) return;
  int r0, kd;
  if ((int)blockIdx.y < rt1) {
    r0 = A0;
    kd = B0 - A0;
  } else {
    r0 = B0;
    kd = C0 - B0;
  }
  const int rt = (int)blockIdx.y < rt1 ? blockIdx.y : blockIdx.y - rt1;
  const int row0 = rt * GTM, col0 = blockIdx.x * GTN;
  if (row0 >= kd || col0 >= N) return;
  const int64_t ld = a.ldz;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int jj = 0; jj < 4; jj++) acc[i][jj] = 0.0;
  for (int k0 = 0; k0 < kd; k0 += GTK) {
    for (int q = threadIdx.x; q < GTK * GTM; q += NT) {
      const int kk = q / GTM, rr = q % GTM;
      const int gr = row0 + rr, gk = k0 + kk;
      As[kk][rr] = gr < kd && gk < kd ? a.Z[(int64_t)(r0 + gr) + (int64_t)(r0 + gk) * ld] : 0.0;
    }
    int nz = 0;
    for (int q = threadIdx.x; q < GTK * GTN; q += NT) {
      const int kk = q / GTN, cc = q % GTN;
      const int gk = k0 + kk, gc = col0 + cc;
      const double m = gk < kd && gc < N ? a.M[(int64_t)(r0 + gk) * ld + A0 + gc] : 0.0;
      Bs[kk][cc] = m;
      nz |= m != 0.0;
    }
    // a slice of M without a nonzero adds nothing: deflated coordinates make most rows of
    // M zero except for one unit entry, so heavily deflated merges skip most slices
    if (!__syncthreads_or(nz)) continue;
#pragma unroll
    for (int kk = 0; kk < GTK; kk++) {
      const double a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
      double bv[4];
#pragma unroll
      for (int jj = 0; jj < 4; jj++) bv[jj] = Bs[kk][tx + 16 * jj];
#pragma unroll
      for (int jj = 0; jj < 4; jj++) {
        acc[0][jj] = fma(a0, bv[jj], acc[0][jj]);
        acc[1][jj] = fma(a1, bv[jj], acc[1][jj]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const int gr = row0 + ty * 2 + i;
    if (gr >= kd) continue;
#pragma unroll
    for (int jj = 0; jj < 4; jj++) {
      const int gc = col0 + tx + 16 * jj;
      if (gc < N) a.Zt[(int64_t)(r0 + gr) + (int64_t)(A0 + gc) * ld] = acc[i][jj];
    }
  }
}

// Z[a:c, a:c] = Zt[a:c, a:c] for the merges of the depth.
__global__ void __launch_bounds__(NT) dc_copy_kernel(DcArgs a, int depth) {
  int A0, B0, C0;
  node_range(a.n, depth, blockIdx.y, &A0, &B0, &C0);
  const int N = C0 - A0;
  if (N < 2) return;
  const int64_t ld = a.ldz;
  const int64_t total = (int64_t)N * N;
  for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < total; q += (int64_t)gridDim.x * NT) {
    const int r = (int)(q % N), c = (int)(q / N);
    a.Z[(int64_t)(A0 + r) + (int64_t)(A0 + c) * ld] = a.Zt[(int64_t)(A0 + r) + (int64_t)(A0 + c) * ld];
  }
}

// w = lam * |T|max * |A|max (undoing both scalings)
__global__ void dc_unscale_kernel(const double* lam, int n, const double* tscale, const unsigned long long* amax,
                                  double* w) {
  const double s = tscale[0] * __longlong_as_double((long long)amax[0]);
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) w[i] = lam[i] * s;
}

// ------------------------------------------------------- back-transformation ----
//
// Z <- H_0 H_1 ... H_{n-2} Z: each CTA owns cw columns, g = (warps of the CTA) / cw warps
// per column, the columns held in shared memory; reflectors from the last to the first.
// With `pairs`, two consecutive reflectors are applied at once: for a = j, b = j - 1,
//   H_b H_a z = z - tau_a s_a v_a - tau_b (s_b - tau_a c s_a) v_b,
// s_a = v_a^T z, s_b = v_b^T z (one pass over z), c = v_b^T v_a (cpair[j], computed
// before); otherwise one at a time, s = tau_j v_j^T z, z <- z - s v_j.  The reflectors are
// staged in shared memory, double-buffered (the next item loaded while the current one is
// applied).  Output into O (column-major, ldo).
constexpr int BT_THREADS = 384;   // largest CTA the kernel is compiled for
__global__ void __launch_bounds__(BT_THREADS, 1) backtransform_kernel(const double* Z, int64_t ldz, const double* V,
                                                                      int64_t ldv, const double* tau,
                                                                      const double* cpair, int pairs, int n, int cw,
                                                                      double* O, int64_t ldo) {
  extern __shared__ __align__(16) double smz[];
  const int per = pairs ? 2 : 1;          // vectors per item
  double* zc = smz;                       // cw x n
  double* vbase = smz + (int64_t)cw * n;  // 2 buffers x per x n
  __shared__ double part[BT_THREADS / 32][2];
  const int nthr = blockDim.x, nwarp = nthr >> 5;
  const int g = nwarp / cw;               // warps per column
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cl = warp / g, gw = warp % g;     // column within the CTA, warp within its group
  const int col0 = blockIdx.x * cw;
  const int ncol = min(cw, n - col0);
  for (int c = 0; c < ncol; c++)
    for (int l = threadIdx.x; l < n; l += nthr) zc[(int64_t)c * n + l] = Z[l + (int64_t)(col0 + c) * ldz];
  // next item at or below j: the highest active reflector, paired with the one below it when
  // that one is active too
  auto next_item = [&](int j, int* jj, bool* pr) -> bool {
    while (j >= 0 && tau[j] == 0.0) j--;
    if (j < 0) return false;
    *jj = j;
    *pr = pairs && j >= 1 && tau[j - 1] != 0.0;
    return true;
  };
  // buffer: v_j in [0, n) for rows l >= j+1 (and a zero at row j for a pair), v_{j-1} in
  // [n, 2n) for rows l >= j
  auto stage = [&](int j, bool pr, int buf) {
    double* dst = vbase + (int64_t)buf * per * n;
    const double* src = V + (int64_t)j * ldv;
    for (int l = j + 1 + threadIdx.x; l < n; l += nthr) {
      const uint32_t da = (uint32_t)__cvta_generic_to_shared(dst + l);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(da), "l"(src + l) : "memory");
    }
    if (pr) {
      if (threadIdx.x == 0) dst[j] = 0.0;
      const double* srcb = V + (int64_t)(j - 1) * ldv;
      for (int l = j + threadIdx.x; l < n; l += nthr) {
        const uint32_t da = (uint32_t)__cvta_generic_to_shared(dst + n + l);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(da), "l"(srcb + l) : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int j;
  bool pr;
  if (next_item(n - 2, &j, &pr)) {
    stage(j, pr, 0);
    int buf = 0;
    for (;;) {
      int jn;
      bool prn;
      const bool more = next_item(pr ? j - 2 : j - 1, &jn, &prn);
      if (more) {
        __syncthreads();   // the other buffer's last readers are done
        stage(jn, prn, buf ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();
      const double* va = vbase + (int64_t)buf * per * n;
      const double* vb = va + n;
      const int lo = pr ? j : j + 1;   // first row of the item's support
      double sa = 0.0, sb = 0.0;
      if (cl < ncol) {
        const double* z = zc + (int64_t)cl * n;
        double sa1 = 0.0, sb1 = 0.0;
        int l = lo + gw * 32 + lane;
        if (pr) {
          for (; l + 32 * g < n; l += 64 * g) {
            const double z0 = z[l], z1 = z[l + 32 * g];
            sa = fma(va[l], z0, sa);
            sb = fma(vb[l], z0, sb);
            sa1 = fma(va[l + 32 * g], z1, sa1);
            sb1 = fma(vb[l + 32 * g], z1, sb1);
          }
          if (l < n) {
            sa = fma(va[l], z[l], sa);
            sb = fma(vb[l], z[l], sb);
          }
          sa = warp_sum(sa + sa1);
          sb = warp_sum(sb + sb1);
        } else {
          for (; l + 32 * g < n; l += 64 * g) {
            sa = fma(va[l], z[l], sa);
            sa1 = fma(va[l + 32 * g], z[l + 32 * g], sa1);
          }
          if (l < n) sa = fma(va[l], z[l], sa);
          sa = warp_sum(sa + sa1);
        }
      }
      if (g > 1) {
        if (lane == 0) {
          part[warp][0] = sa;
          part[warp][1] = sb;
        }
        __syncthreads();
        sa = 0.0;
        sb = 0.0;
        for (int q = 0; q < g; q++) {
          sa += part[cl * g + q][0];
          sb += part[cl * g + q][1];
        }
      }
      if (cl < ncol) {
        double* z = zc + (int64_t)cl * n;
        const double ta = tau[j];
        const double al = ta * sa;
        if (pr) {
          const double be = tau[j - 1] * fma(-ta * cpair[j], sa, sb);
          for (int l = lo + gw * 32 + lane; l < n; l += 32 * g) z[l] = fma(-be, vb[l], fma(-al, va[l], z[l]));
        } else {
          for (int l = lo + gw * 32 + lane; l < n; l += 32 * g) z[l] = fma(-al, va[l], z[l]);
        }
      }
      if (!more) break;
      buf ^= 1;
      j = jn;
      pr = prn;
    }
  }
  __syncthreads();
  for (int c = 0; c < ncol; c++)
    for (int l = threadIdx.x; l < n; l += nthr) O[l + (int64_t)(col0 + c) * ldo] = zc[(int64_t)c * n + l];
}

// cpair[j] = v_{j-1}^T v_j (rows l >= j+1, where v_j lives) for 1 <= j <= n-2: one warp per j
__global__ void __launch_bounds__(NT) bt_pair_dot_kernel(const double* V, int64_t ldv, int n, double* cpair) {
  const int j = 1 + (int)(blockIdx.x * (NT / 32) + (threadIdx.x >> 5)), lane = threadIdx.x & 31;
  if (j > n - 2) return;
  const double* va = V + (int64_t)j * ldv;
  const double* vb = V + (int64_t)(j - 1) * ldv;
  double s = 0.0;
  for (int l = j + 1 + lane; l < n; l += 32) s = fma(vb[l], va[l], s);
  s = warp_sum(s);
  if (lane == 0) cpair[j] = s;
}

}  // namespace

namespace {

struct EigLayout {
  size_t off[40];
  size_t total;
};

enum {
  L_V, L_Z, L_ZT, L_M, L_D, L_E, L_TAU, L_PBUF, L_ROWBUF, L_DOT, L_RWG, L_LAM, L_ES, L_DS, L_ZS, L_DK, L_ZK, L_ZZ,
  L_TAUK, L_LAMK, L_ZH, L_INVN, L_RC, L_RS, L_IDX, L_STAT, L_NTP, L_KIDX, L_ORIG, L_COLREF, L_RP, L_RT, L_KOF,
  L_NROT, L_CAND, L_AMAX, L_TSCALE, L_BAR, L_COUNT
};

constexpr int MAX_P = 256;

EigLayout eig_layout(int n) {
  EigLayout L;
  const size_t nn = (size_t)n * n * 8, nd = (size_t)n * 8, ni = (size_t)n * 4;
  size_t sz[L_COUNT];
  sz[L_V] = sz[L_Z] = sz[L_ZT] = sz[L_M] = nn;
  sz[L_D] = sz[L_E] = sz[L_TAU] = nd;
  sz[L_PBUF] = sz[L_ROWBUF] = 2 * nd;
  sz[L_DOT] = 2 * MAX_P * 8;
  sz[L_RWG] = (size_t)MAX_P * nd;
  for (int q = L_LAM; q <= L_RS; q++) sz[q] = nd;
  for (int q = L_IDX; q <= L_CAND; q++) sz[q] = ni;
  sz[L_AMAX] = 16;
  sz[L_TSCALE] = 8;
  sz[L_BAR] = 16;
  size_t o = 0;
  for (int q = 0; q < L_COUNT; q++) {
    L.off[q] = o;
    o += (sz[q] + 255) / 256 * 256;
  }
  L.total = o;
  return L;
}

int sm_count() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

// vectors of the tridiagonalisation in shared memory unless the row work vector must go
// to global memory (large n)
constexpr size_t SMEM_CAP = 220 * 1024;

}  // namespace

size_t sym_eig_work_bytes(int n) {
  if (n < 1) return 0;
  // the per-CTA row work vectors are only needed in global memory for large n; the
  // layout keeps them for every n (n doubles per possible CTA is small next to 4 n^2)
  return eig_layout(n).total;
}

cudaError_t launch_sym_eig(double* A, int64_t lda, int n, double* w, void* work, size_t work_bytes, int* info,
                           cudaStream_t st, long long spin_limit, int leave_cta) {
  if (n < 1 || n > KSCF_EIG_MAX_N || lda < n || !A || !w || !work || !info) return cudaErrorInvalidValue;
  const EigLayout L = eig_layout(n);
  if (work_bytes < L.total) return cudaErrorInvalidValue;
  char* base = (char*)work;
  auto P_ = [&](int q) { return (void*)(base + L.off[q]); };
  cudaError_t e;
  if ((e = cudaMemsetAsync(info, 0, 4 * sizeof(int), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(P_(L_AMAX), 0, 16, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(P_(L_BAR), 0, 16, st)) != cudaSuccess) return e;
  unsigned long long* amax = (unsigned long long*)P_(L_AMAX);
  const int nsm = sm_count();
  {
    const int64_t tot = (int64_t)n * n;
    const int blocks = (int)std::min<int64_t>(4 * nsm, (tot + NT - 1) / NT);
    absmax_kernel<<<blocks, NT, 0, st>>>(A, lda, n, amax), count_launch();
    scale_sym_kernel<<<blocks, NT, 0, st>>>(A, lda, n, amax), count_launch();
  }
  // ---- tridiagonalisation ----
  TriArgs t;
  t.A = A;
  t.lda = lda;
  t.n = n;
  t.P = std::max(1, std::min(std::min(nsm, MAX_P), (n - 1 + 3) / 4));
  t.d = (double*)P_(L_D);
  t.e = (double*)P_(L_E);
  t.tau = (double*)P_(L_TAU);
  t.V = (double*)P_(L_V);
  t.pbuf = (double*)P_(L_PBUF);
  t.rowbuf = (double*)P_(L_ROWBUF);
  t.dotbuf = (double*)P_(L_DOT);
  t.rwg = nullptr;
  t.bar = (unsigned*)P_(L_BAR);
  t.status = info;
  t.spin_limit = spin_limit;
  t.leave_cta = leave_cta;
  const int R = (n + t.P - 1) / t.P;
  size_t vec_bytes = (size_t)4 * n * 8;
  if (vec_bytes > SMEM_CAP) {
    vec_bytes = (size_t)3 * n * 8;
    t.rwg = (double*)P_(L_RWG);
  }
  const size_t rows_bytes = (size_t)R * n * 8;
  const bool smem_rows = vec_bytes + rows_bytes <= SMEM_CAP;
  const size_t tri_smem = vec_bytes + (smem_rows ? rows_bytes : 0);
  void* targs[] = {&t};
  if (smem_rows) {
    if ((e = cudaFuncSetAttribute(tridiag_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tri_smem)) !=
        cudaSuccess)
      return e;
    e = cudaLaunchCooperativeKernel((void*)tridiag_kernel<true>, dim3(t.P), dim3(NT), targs, tri_smem, st);
  } else {
    if ((e = cudaFuncSetAttribute(tridiag_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tri_smem)) != cudaSuccess)
      return e;
    e = cudaLaunchCooperativeKernel((void*)tridiag_kernel<false>, dim3(t.P), dim3(NT), targs, tri_smem, st);
  }
  count_launch();
  if (e != cudaSuccess) return e;
  // ---- divide and conquer ----
  DcArgs a;
  a.n = n;
  a.ldz = n;
  a.lam = (double*)P_(L_LAM);
  a.es = (double*)P_(L_ES);
  a.Z = (double*)P_(L_Z);
  a.Zt = (double*)P_(L_ZT);
  a.M = (double*)P_(L_M);
  a.Ds = (double*)P_(L_DS);
  a.zs = (double*)P_(L_ZS);
  a.dk = (double*)P_(L_DK);
  a.zk = (double*)P_(L_ZK);
  a.zz = (double*)P_(L_ZZ);
  a.tauk = (double*)P_(L_TAUK);
  a.lamk = (double*)P_(L_LAMK);
  a.zh = (double*)P_(L_ZH);
  a.invn = (double*)P_(L_INVN);
  a.rc = (double*)P_(L_RC);
  a.rsn = (double*)P_(L_RS);
  a.idx = (int*)P_(L_IDX);
  a.stat = (int*)P_(L_STAT);
  a.ntp = (int*)P_(L_NTP);
  a.kidx = (int*)P_(L_KIDX);
  a.orig = (int*)P_(L_ORIG);
  a.colref = (int*)P_(L_COLREF);
  a.rp = (int*)P_(L_RP);
  a.rt = (int*)P_(L_RT);
  a.Kof = (int*)P_(L_KOF);
  a.nrot = (int*)P_(L_NROT);
  a.cand = (int*)P_(L_CAND);
  a.status = info;
  double* tscale = (double*)P_(L_TSCALE);
  dc_leaves_kernel<<<1, NT, 0, st>>>(a, t.d, t.e, tscale), count_launch();
  int D = 0;
  while ((1 << D) < n) D++;
  int p2max = 1;
  while (p2max < n) p2max <<= 1;
  const size_t order_smem = (size_t)p2max * 12;
  if ((e = cudaFuncSetAttribute(dc_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)order_smem)) !=
      cudaSuccess)
    return e;
  for (int d = D - 1; d >= 0; d--) {
    const int nodes = 1 << d;
    const int Nmax = (int)(((int64_t)n + nodes - 1) / nodes);
    if (Nmax < 2) continue;
    if (Nmax <= DC_SMALL) {
      dc_small_kernel<<<nodes, NT, 0, st>>>(a, d), count_launch();
      continue;
    }
    int p2 = 1;
    while (p2 < Nmax) p2 <<= 1;
    const int rw = (Nmax + NW - 1) / NW;
    dc_deflate_kernel<<<nodes, NT, 0, st>>>(a, d), count_launch();
    dc_secular_kernel<<<dim3(rw, nodes), NT, 0, st>>>(a, d), count_launch();
    dc_zhat_kernel<<<dim3(rw, nodes), NT, 0, st>>>(a, d), count_launch();
    dc_colnorm_kernel<<<dim3(rw, nodes), NT, 0, st>>>(a, d), count_launch();
    dc_order_kernel<<<nodes, NT, (size_t)p2 * 12, st>>>(a, d, p2), count_launch();
    dc_build_m_kernel<<<dim3((Nmax + 31) / 32, (Nmax + 63) / 64, nodes), NT, 0, st>>>(a, d), count_launch();
    dc_rotperm_kernel<<<dim3((Nmax + NT - 1) / NT, nodes), NT, 0, st>>>(a, d), count_launch();
    const int rt = (Nmax / 2 + 1 + GTM - 1) / GTM;
    dc_gemm_kernel<<<dim3((Nmax + GTN - 1) / GTN, 2 * rt, nodes), NT, 0, st>>>(a, d, rt), count_launch();
    const int cb = (int)std::min<int64_t>(256, ((int64_t)Nmax * Nmax + NT - 1) / NT);
    dc_copy_kernel<<<dim3(cb, nodes), NT, 0, st>>>(a, d), count_launch();
  }
  dc_unscale_kernel<<<(n + NT - 1) / NT, NT, 0, st>>>(a.lam, n, tscale, amax, w), count_launch();
  // ---- back-transformation into A ----
  // One warp per column, ceil(n / SMs) columns per CTA (at most 8), so that every SM's FP64
  // pipes get a share; when 8 columns do not fit in shared memory, 8-warp CTAs of 4, 2, 1
  // columns of 2, 4, 8 warps (a 12-warp CTA with 6 two-warp columns was slower than one
  // warp per column: the per-reflector cross-warp sum costs a CTA-wide barrier).  Reflectors
  // in pairs when two double-buffered pairs fit beside the columns, else one at a time.
  const int sms = sm_count();
  int cw = (int)std::min<int64_t>(8, ((int64_t)n + sms - 1) / sms);
  int bt_threads = 32 * cw;
  int pairs = (size_t)(cw + 4) * n * 8 <= SMEM_CAP ? 1 : 0;
  if (!pairs && (size_t)(cw + 2) * n * 8 > SMEM_CAP) {
    cw = 8;
    while (cw > 1 && (size_t)(cw + 2) * n * 8 > SMEM_CAP) cw /= 2;
    bt_threads = NT;
  }
  const size_t bt_smem = (size_t)(cw + 2 * (pairs ? 2 : 1)) * n * 8;
  double* cpair = t.pbuf;   // free once the tridiagonalisation is done
  if (pairs && n >= 3)
    bt_pair_dot_kernel<<<(n - 2 + NT / 32 - 1) / (NT / 32), NT, 0, st>>>(t.V, n, n, cpair), count_launch();
  if ((e = cudaFuncSetAttribute(backtransform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem)) !=
      cudaSuccess)
    return e;
  backtransform_kernel<<<(n + cw - 1) / cw, bt_threads, bt_smem, st>>>(a.Z, n, t.V, n, t.tau, cpair, pairs, n, cw, A,
                                                                      lda),
      count_launch();
  // non-finite input: report through info[2]
  info_nonfinite_kernel<<<1, 32, 0, st>>>(amax, info), count_launch();
  return cudaGetLastError();
}

}  // namespace kscf
