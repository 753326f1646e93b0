// Kernels of the self-consistent field loop (arXiv 2303.00790, Computational details:
// Kohn-Sham DFT in the LDA, SCF stopped on the self-consistent residual error):
//   - Gaussian atomic valence densities (start of the SCF),
//   - LDA exchange-correlation: Slater exchange + Perdew-Zunger 1981 correlation,
//   - Hartree potential: -Lap_h V_H = 4 pi rho by conjugate gradients in FP64 on the
//     Hilbert-brick grid, with the values the order-12 stencil needs outside the sphere
//     taken from the multipole expansion (monopole, dipole, quadrupole) of rho,
//   - residual V_out - V_in, SRE and the energy integrals,
//   - Anderson mixing of the input potential.
// All arithmetic is FP64.  Reductions are deterministic: every block writes one partial
// sum per value, and consumers add the partials in a fixed order.
#include <cuda_runtime.h>

#include "kscf_internal.h"
#include "scf_internal.h"

namespace kscf {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Sum of p[0..nb) in a fixed order; every lane of the calling warp gets the same value
// (a butterfly of commutative additions).
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ p, int nb) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < nb; i += 32) s += p[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Block-wide sum of NV values per thread; thread 0 writes part[v * gridDim.x + blockIdx.x].
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* __restrict__ part) {
  __shared__ double sh[NV][kScfThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; q++) {
    double s = v[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sh[q][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) {
      double s = 0.0;
      for (int w = 0; w < kScfThreads / 32; w++) s += sh[q][w];
      part[q * gridDim.x + blockIdx.x] = s;
    }
  }
}

// out[v] = sum_b part[v * nb + b]  (one block; warp w handles values w, w + 8, ...)
__global__ void finalize_partials_kernel(const double* __restrict__ part, int nb, int nv, double* __restrict__ out) {
  const int warp = threadIdx.x >> 5;
  for (int v = warp; v < nv; v += blockDim.x >> 5) {
    const double s = warp_sum_partials(part + (int64_t)v * nb, nb);
    if ((threadIdx.x & 31) == 0) out[v] = s;
  }
}

cudaError_t launch_finalize_partials(const double* part, int nb, int nv, double* out, cudaStream_t st) {
  finalize_partials_kernel<<<1, 256, 0, st>>>(part, nb, nv, out), count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Starting density: rho(p) = sum_a Z_a / (pi^{3/2} r_a^3) exp(-|p - R_a|^2 / r_a^2).
// atoms: 5 doubles each (x, y, z, Z_valence, r_a); rel: h * (i, j, k) of every slot.
__global__ void atomic_density_kernel(const double* __restrict__ rel, double cx, double cy, double cz,
                                      const uint8_t* __restrict__ mask, const double* __restrict__ atoms,
                                      int n_atoms, int64_t n, double* __restrict__ rho) {
  __shared__ double sat[128 * 5];
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < n && mask[s];
  double px = 0, py = 0, pz = 0;
  if (live) {
    px = cx + rel[3 * s];
    py = cy + rel[3 * s + 1];
    pz = cz + rel[3 * s + 2];
  }
  double acc = 0.0;
  for (int a0 = 0; a0 < n_atoms; a0 += 128) {
    const int na = min(128, n_atoms - a0);
    __syncthreads();
    for (int q = threadIdx.x; q < na * 5; q += blockDim.x) sat[q] = atoms[(int64_t)a0 * 5 + q];
    __syncthreads();
    if (live) {
      for (int a = 0; a < na; a++) {
        const double* at = sat + 5 * a;
        const double dx = px - at[0], dy = py - at[1], dz = pz - at[2];
        const double ra = at[4];
        acc += at[3] / (5.568327996831707845 * ra * ra * ra) * exp(-(dx * dx + dy * dy + dz * dz) / (ra * ra));
      }
    }
  }
  if (s < n) rho[s] = live ? acc : 0.0;
}

cudaError_t launch_atomic_density(const Ham& H, const double* rel, const double* atoms, int n_atoms, double* rho,
                                  cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  atomic_density_kernel<<<nblk(n, 128), 128, 0, st>>>(rel, H.grid.center[0], H.grid.center[1], H.grid.center[2],
                                                     H.d_mask, atoms, n_atoms, n, rho), count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LDA (unpolarised, Hartree units).  Slater exchange eps_x = -3/4 (3 rho/pi)^{1/3},
// v_x = 4/3 eps_x.  Perdew-Zunger 1981 fit of the Ceperley-Alder correlation energy,
// rs = (3/(4 pi rho))^{1/3}:
//   rs >= 1: eps_c = gamma / (1 + beta1 sqrt(rs) + beta2 rs),
//            v_c = eps_c (1 + 7/6 beta1 sqrt(rs) + 4/3 beta2 rs) / (1 + beta1 sqrt(rs) + beta2 rs)
//   rs <  1: eps_c = A ln rs + B + C rs ln rs + D rs,
//            v_c = A ln rs + (B - A/3) + 2/3 C rs ln rs + (2D - C)/3 rs
// gamma = -0.1423, beta1 = 1.0529, beta2 = 0.3334, A = 0.0311, B = -0.048, C = 0.0020,
// D = -0.0116.  Densities at or below 1e-14 give zero.
__global__ void lda_kernel(const double* __restrict__ rho, const uint8_t* __restrict__ mask, int64_t n,
                           double* __restrict__ eps, double* __restrict__ vxc) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double e = 0.0, v = 0.0;
  const double r = rho[s];
  if (mask[s] && r > 1e-14) {
    const double pi = 3.14159265358979323846;
    const double rs = cbrt(3.0 / (4.0 * pi * r));
    const double ex = -0.75 * cbrt(3.0 * r / pi);
    const double vx = (4.0 / 3.0) * ex;
    double ec, vc;
    if (rs >= 1.0) {
      const double sq = sqrt(rs);
      const double den = 1.0 + 1.0529 * sq + 0.3334 * rs;
      ec = -0.1423 / den;
      vc = ec * (1.0 + 7.0 / 6.0 * 1.0529 * sq + 4.0 / 3.0 * 0.3334 * rs) / den;
    } else {
      const double ln = log(rs);
      ec = 0.0311 * ln + (-0.048) + 0.0020 * rs * ln + (-0.0116) * rs;
      vc = 0.0311 * ln + (-0.048 - 0.0311 / 3.0) + 2.0 / 3.0 * 0.0020 * rs * ln + (2.0 * (-0.0116) - 0.0020) / 3.0 * rs;
    }
    e = ex + ec;
    v = vx + vc;
  }
  if (eps) eps[s] = e;
  vxc[s] = v;
}

cudaError_t launch_lda(const Ham& H, const double* rho, double* eps, double* vxc, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  lda_kernel<<<nblk(n, 256), 256, 0, st>>>(rho, H.d_mask, n, eps, vxc), count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CG operator A x = -Lap_h x + shift x on the domain (zero outside: padding slots of x
// hold zero and missing bricks read as zero): shift 0 for the Poisson problem, q0^2 for
// the Kerker preconditioner.  cw[k] = -w_k / h^2 (k = 0..6); the centre term uses
// 3 cw[0].  One thread per slot.
struct LapArgs {
  const int32_t* nbr;
  const uint8_t* mask;
  double cw[7];
  double shift;
  int64_t n;
};

template <int B>
__device__ __forceinline__ double lap_at(const LapArgs& a, const double* __restrict__ x, int64_t s) {
  constexpr int B3 = B * B * B;
  const int64_t brick = s / B3;
  const int li = (int)(s - brick * B3);
  const int l[3] = {li % B, (li / B) % B, li / (B * B)};
  const int stride[3] = {1, B, B * B};
  double acc = (3.0 * a.cw[0] + a.shift) * x[s];
#pragma unroll
  for (int ax = 0; ax < 3; ax++) {
#pragma unroll
    for (int k = 1; k <= 6; k++) {
      double pair = 0.0;
#pragma unroll
      for (int sg = -1; sg <= 1; sg += 2) {
        const int nn = l[ax] + sg * k;
        if (nn >= 0 && nn < B) {
          pair += x[s + (int64_t)sg * k * stride[ax]];
        } else {
          const int nb = a.nbr[brick * 6 + 2 * ax + (sg > 0 ? 1 : 0)];
          if (nb >= 0) pair += x[(int64_t)nb * B3 + li + (sg * k - sg * B) * stride[ax]];
        }
      }
      acc += a.cw[k] * pair;
    }
  }
  return acc;
}

// Convergence state of the CG, read by every kernel from the partial sums:
// rr = r.r of the current residual, converged when rr < thr2 = rtol^2 b.b.
struct CgState {
  const double* part_bb;  // kScfRedBlocks partials of b.b
  double rtol2;
};

__device__ __forceinline__ bool cg_done(const CgState& c, double rr) {
  const double bb = warp_sum_partials(c.part_bb, kScfRedBlocks);
  return rr < c.rtol2 * bb;
}

// b = 4 pi rho + sum over the ghost points g of the slot: w_g V_ghost[g]; partial b.b
__global__ void __launch_bounds__(kScfThreads) poisson_rhs_kernel(const double* __restrict__ rho,
                                                                  const uint8_t* __restrict__ mask,
                                                                  const int64_t* __restrict__ gptr,
                                                                  const int32_t* __restrict__ gidx,
                                                                  const double* __restrict__ gw,
                                                                  const double* __restrict__ vghost, int64_t n,
                                                                  double* __restrict__ b, double* __restrict__ part) {
  double acc[1] = {0.0};
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (mask[s]) {
      v = 4.0 * 3.14159265358979323846 * rho[s];
      for (int64_t e = gptr[s]; e < gptr[s + 1]; e++) v += gw[e] * vghost[gidx[e]];
    }
    b[s] = v;
    acc[0] += v * v;
  }
  block_partials<1>(acc, part);
}

// r = b - A x, p = r, partial r.r  (x is the starting guess; padding rows set to zero)
template <int B>
__global__ void __launch_bounds__(kScfThreads) cg_init_kernel(LapArgs a, double* __restrict__ x,
                                                              const double* __restrict__ b, double* __restrict__ r,
                                                              double* __restrict__ p, double* __restrict__ part_rr) {
  double acc[1] = {0.0};
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += (int64_t)gridDim.x * blockDim.x) {
    double rv = 0.0;
    if (a.mask[s]) rv = b[s] - lap_at<B>(a, x, s);
    r[s] = rv;
    p[s] = rv;
    acc[0] += rv * rv;
  }
  block_partials<1>(acc, part_rr);
}

// q = A p, partial p.q   (no-op once converged)
template <int B>
__global__ void __launch_bounds__(kScfThreads) cg_apply_kernel(LapArgs a, CgState c, const double* __restrict__ p,
                                                               double* __restrict__ q,
                                                               const double* __restrict__ part_rr,
                                                               double* __restrict__ part_pq) {
  const double rr = warp_sum_partials(part_rr, kScfRedBlocks);
  if (cg_done(c, rr)) return;
  double acc[1] = {0.0};
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += (int64_t)gridDim.x * blockDim.x) {
    double qv = 0.0;
    if (a.mask[s]) {
      qv = lap_at<B>(a, p, s);
      acc[0] += p[s] * qv;
    }
    q[s] = qv;
  }
  block_partials<1>(acc, part_pq);
}

// alpha = rr / p.q; x += alpha p; r -= alpha q; partial of the new r.r
// (once converged: carries the partials of rr forward unchanged)
__global__ void __launch_bounds__(kScfThreads) cg_update_kernel(CgState c, int64_t n, double* __restrict__ x,
                                                                double* __restrict__ r, const double* __restrict__ p,
                                                                const double* __restrict__ q,
                                                                const double* __restrict__ part_rr,
                                                                const double* __restrict__ part_pq,
                                                                double* __restrict__ part_rr_next, int* iters) {
  const double rr = warp_sum_partials(part_rr, kScfRedBlocks);
  if (cg_done(c, rr)) {
    if (threadIdx.x == 0) part_rr_next[blockIdx.x] = part_rr[blockIdx.x];
    return;
  }
  const double pq = warp_sum_partials(part_pq, kScfRedBlocks);
  const double alpha = rr / pq;
  double acc[1] = {0.0};
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    x[s] += alpha * p[s];
    const double rv = r[s] - alpha * q[s];
    r[s] = rv;
    acc[0] += rv * rv;
  }
  block_partials<1>(acc, part_rr_next);
  if (blockIdx.x == 0 && threadIdx.x == 0) iters[0] += 1;
}

// beta = rr_new / rr; p = r + beta p
__global__ void __launch_bounds__(kScfThreads) cg_dir_kernel(CgState c, int64_t n, const double* __restrict__ r,
                                                             double* __restrict__ p,
                                                             const double* __restrict__ part_rr,
                                                             const double* __restrict__ part_rr_next) {
  const double rr = warp_sum_partials(part_rr, kScfRedBlocks);
  if (cg_done(c, rr)) return;
  const double rr_new = warp_sum_partials(part_rr_next, kScfRedBlocks);
  const double beta = rr_new / rr;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    p[s] = r[s] + beta * p[s];
}

static LapArgs lap_args(const Ham& H, double shift) {
  LapArgs a;
  a.shift = shift;
  a.nbr = H.d_nbr;
  a.mask = H.d_mask;
  // H.stencil[k] = -1/2 w_k / h^2, so -w_k / h^2 = 2 H.stencil[k]
  for (int k = 0; k <= 6; k++) a.cw[k] = 2.0 * H.stencil[k];
  a.n = H.grid.n_slots;
  return a;
}

cudaError_t launch_poisson_rhs(const Ham& H, const double* rho, const PoissonPlan& P, double* b, double* part_bb,
                               cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  poisson_rhs_kernel<<<kScfRedBlocks, kScfThreads, 0, st>>>(rho, H.d_mask, P.d_gptr, P.d_gidx, P.d_gw, P.d_vghost,
                                                            n, b, part_bb), count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const Ham& H, double shift, double* x, const double* b, double* r, double* p,
                           double* part_rr, cudaStream_t st) {
  const LapArgs a = lap_args(H, shift);
  if (H.grid.B == 8)
    cg_init_kernel<8><<<kScfRedBlocks, kScfThreads, 0, st>>>(a, x, b, r, p, part_rr), count_launch();
  else
    cg_init_kernel<16><<<kScfRedBlocks, kScfThreads, 0, st>>>(a, x, b, r, p, part_rr), count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cg_iteration(const Ham& H, double shift, const double* part_bb, double rtol, double* x, double* r,
                                double* p, double* q, const double* part_rr, double* part_pq, double* part_rr_next,
                                int* iters, cudaStream_t st) {
  const LapArgs a = lap_args(H, shift);
  CgState c;
  c.part_bb = part_bb;
  c.rtol2 = rtol * rtol;
  const int64_t n = H.grid.n_slots;
  if (H.grid.B == 8)
    cg_apply_kernel<8><<<kScfRedBlocks, kScfThreads, 0, st>>>(a, c, p, q, part_rr, part_pq), count_launch();
  else
    cg_apply_kernel<16><<<kScfRedBlocks, kScfThreads, 0, st>>>(a, c, p, q, part_rr, part_pq), count_launch();
  cg_update_kernel<<<kScfRedBlocks, kScfThreads, 0, st>>>(c, n, x, r, p, q, part_rr, part_pq, part_rr_next, iters),
      count_launch();
  cg_dir_kernel<<<kScfRedBlocks, kScfThreads, 0, st>>>(c, n, r, p, part_rr, part_rr_next), count_launch();
  return cudaGetLastError();
}

// b = f on the domain (0 outside); partial b.b
__global__ void __launch_bounds__(kScfThreads) rhs_copy_kernel(const double* __restrict__ f,
                                                               const uint8_t* __restrict__ mask, int64_t n,
                                                               double* __restrict__ b, double* __restrict__ part) {
  double acc[1] = {0.0};
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const double v = mask[s] ? f[s] : 0.0;
    b[s] = v;
    acc[0] += v * v;
  }
  block_partials<1>(acc, part);
}

cudaError_t launch_rhs_copy(const Ham& H, const double* f, double* b, double* part_bb, cudaStream_t st) {
  rhs_copy_kernel<<<kScfRedBlocks, kScfThreads, 0, st>>>(f, H.d_mask, H.grid.n_slots, b, part_bb), count_launch();
  return cudaGetLastError();
}

// out = a + c b (0 outside the domain)
__global__ void lincomb_kernel(const uint8_t* __restrict__ mask, const double* __restrict__ a,
                               const double* __restrict__ b, double c, int64_t n, double* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[s] = mask[s] ? a[s] + c * b[s] : 0.0;
}

cudaError_t launch_lincomb(const Ham& H, const double* a, const double* b, double c, double* out, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  lincomb_kernel<<<nblk(n, 256), 256, 0, st>>>(H.d_mask, a, b, c, n, out), count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Multipoles of rho about the grid centre (x = h (i, j, k)); partials of
// q = sum rho, p_i = sum rho x_i, S_ij = sum rho x_i x_j  (10 values; times h^3 later).
__global__ void __launch_bounds__(kScfThreads) multipole_kernel(const double* __restrict__ rho,
                                                                const double* __restrict__ rel, int64_t n,
                                                                double* __restrict__ part) {
  double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const double r = rho[s];
    if (r == 0.0) continue;
    const double x = rel[3 * s], y = rel[3 * s + 1], z = rel[3 * s + 2];
    v[0] += r;
    v[1] += r * x;
    v[2] += r * y;
    v[3] += r * z;
    v[4] += r * x * x;
    v[5] += r * y * y;
    v[6] += r * z * z;
    v[7] += r * x * y;
    v[8] += r * x * z;
    v[9] += r * y * z;
  }
  block_partials<10>(v, part);
}

// V at each ghost point t (relative to the centre):
//   q/|t| + p.t/|t|^3 + 1/2 t^T Q t / |t|^5,  Q_ij = 3 S_ij - delta_ij tr S  (all times h^3)
__global__ void ghost_potential_kernel(const double* __restrict__ mom, double h3, const double* __restrict__ grel,
                                       int64_t ng, double* __restrict__ vghost) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  const double q = h3 * mom[0];
  const double px = h3 * mom[1], py = h3 * mom[2], pz = h3 * mom[3];
  const double tr = mom[4] + mom[5] + mom[6];
  const double Qxx = h3 * (3.0 * mom[4] - tr), Qyy = h3 * (3.0 * mom[5] - tr), Qzz = h3 * (3.0 * mom[6] - tr);
  const double Qxy = h3 * 3.0 * mom[7], Qxz = h3 * 3.0 * mom[8], Qyz = h3 * 3.0 * mom[9];
  const double x = grel[3 * g], y = grel[3 * g + 1], z = grel[3 * g + 2];
  const double r2 = x * x + y * y + z * z;
  const double r = sqrt(r2);
  const double quad = Qxx * x * x + Qyy * y * y + Qzz * z * z + 2.0 * (Qxy * x * y + Qxz * x * z + Qyz * y * z);
  vghost[g] = q / r + (px * x + py * y + pz * z) / (r2 * r) + 0.5 * quad / (r2 * r2 * r);
}

cudaError_t launch_ghost_values(const Ham& H, const double* rho, const double* rel, const PoissonPlan& P,
                                double* part, double* mom, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  multipole_kernel<<<kScfRedBlocks, kScfThreads, 0, st>>>(rho, rel, n, part), count_launch();
  cudaError_t e = launch_finalize_partials(part, kScfRedBlocks, 10, mom, st);
  if (e != cudaSuccess) return e;
  const double h3 = H.grid.h * H.grid.h * H.grid.h;
  if (P.n_ghost > 0)
    ghost_potential_kernel<<<nblk(P.n_ghost, 256), 256, 0, st>>>(mom, h3, P.d_grel, P.n_ghost, P.d_vghost),
        count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Residual and energy integrals:
//   f = V_out - V_in with V_out = V_ion + V_H + V_xc (zero outside the domain)
//   partials of  rho f^2,  rho (V_in - V_ion),  rho V_H,  rho eps_xc,  rho
__global__ void __launch_bounds__(kScfThreads) residual_kernel(const uint8_t* __restrict__ mask,
                                                               const double* __restrict__ rho,
                                                               const double* __restrict__ v_in,
                                                               const double* __restrict__ v_ion,
                                                               const double* __restrict__ vh,
                                                               const double* __restrict__ vxc,
                                                               const double* __restrict__ eps, int64_t n,
                                                               double* __restrict__ f, double* __restrict__ part) {
  double v[5] = {0, 0, 0, 0, 0};
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    double fv = 0.0;
    if (mask[s]) {
      const double r = rho[s];
      fv = (v_ion[s] + vh[s] + vxc[s]) - v_in[s];
      v[0] += r * fv * fv;
      v[1] += r * (v_in[s] - v_ion[s]);
      v[2] += r * vh[s];
      v[3] += r * eps[s];
      v[4] += r;
    }
    f[s] = fv;
  }
  block_partials<5>(v, part);
}

cudaError_t launch_residual(const Ham& H, const double* rho, const double* v_in, const double* v_ion, const double* vh,
                            const double* vxc, const double* eps, double* f, double* part, double* out5,
                            cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  residual_kernel<<<kScfRedBlocks, kScfThreads, 0, st>>>(H.d_mask, rho, v_in, v_ion, vh, vxc, eps, n, f, part),
      count_launch();
  return launch_finalize_partials(part, kScfRedBlocks, 5, out5, st);
}

// v = a + b + c (masked)
__global__ void sum3_kernel(const uint8_t* __restrict__ mask, const double* __restrict__ a,
                            const double* __restrict__ b, const double* __restrict__ c, int64_t n,
                            double* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[s] = mask[s] ? a[s] + b[s] + c[s] : 0.0;
}

cudaError_t launch_sum3(const Ham& H, const double* a, const double* b, const double* c, double* out,
                        cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  sum3_kernel<<<nblk(n, 256), 256, 0, st>>>(H.d_mask, a, b, c, n, out), count_launch();
  return cudaGetLastError();
}

// out = a + b (masked)
__global__ void add2_kernel(const uint8_t* __restrict__ mask, const double* __restrict__ a,
                            const double* __restrict__ b, int64_t n, double* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[s] = mask[s] ? a[s] + b[s] : 0.0;
}

cudaError_t launch_add2(const Ham& H, const double* a, const double* b, double* out, cudaStream_t st) {
  const int64_t n = H.grid.n_slots;
  add2_kernel<<<nblk(n, 256), 256, 0, st>>>(H.d_mask, a, b, n, out), count_launch();
  return cudaGetLastError();
}

// Column inner products in FP64: part[j * gridDim.x + b] = this block's share of
// sum_r A[r][j] B[r][j] (B = A: column sums of squares).
template <typename T>
__global__ void __launch_bounds__(kScfThreads) col_dot_kernel(const T* __restrict__ A, int64_t lda,
                                                              const T* __restrict__ B, int64_t ldb, int64_t rows,
                                                              int k, double* __restrict__ part) {
  const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = r0 + per < rows ? r0 + per : rows;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double a0 = 0.0, a1 = 0.0;
    int64_t r = r0;
    for (; r + 1 < r1; r += 2) {
      a0 += (double)A[r * lda + j] * (double)B[r * ldb + j];
      a1 += (double)A[(r + 1) * lda + j] * (double)B[(r + 1) * ldb + j];
    }
    if (r < r1) a0 += (double)A[r * lda + j] * (double)B[r * ldb + j];
    part[(int64_t)j * gridDim.x + blockIdx.x] = a0 + a1;
  }
}

// part[j * gridDim.x + b] = this block's share of sum_r (HX[r][j] - lam[j] X[r][j])^2  (FP64)
template <typename T>
__global__ void __launch_bounds__(kScfThreads) col_resid_kernel(const T* __restrict__ X, const T* __restrict__ HX,
                                                                int64_t ld, int64_t rows, int k,
                                                                const double* __restrict__ lam,
                                                                double* __restrict__ part) {
  const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = r0 + per < rows ? r0 + per : rows;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double l = lam[j];
    double a = 0.0;
    for (int64_t r = r0; r < r1; r++) {
      const double d = (double)HX[r * ld + j] - l * (double)X[r * ld + j];
      a += d * d;
    }
    part[(int64_t)j * gridDim.x + blockIdx.x] = a;
  }
}

cudaError_t launch_col_dot(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t rows, int k, int dtype,
                           double* part, double* out, cudaStream_t st) {
  if (dtype == KSCF_F64)
    col_dot_kernel<double><<<kScfRedBlocks, kScfThreads, 0, st>>>((const double*)A, lda, (const double*)B, ldb, rows,
                                                                  k, part), count_launch();
  else
    col_dot_kernel<float><<<kScfRedBlocks, kScfThreads, 0, st>>>((const float*)A, lda, (const float*)B, ldb, rows, k,
                                                                 part), count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_finalize_partials(part, kScfRedBlocks, k, out, st);
}

cudaError_t launch_col_sumsq(const void* X, int64_t ld, int64_t rows, int k, int dtype, double* part, double* out,
                             cudaStream_t st) {
  return launch_col_dot(X, ld, X, ld, rows, k, dtype, part, out, st);
}

cudaError_t launch_col_resid(const double* X, const double* HX, int64_t ld, int64_t rows, int k, const double* lam,
                             double* part, double* out, cudaStream_t st) {
  return launch_col_resid_t(X, HX, ld, rows, k, KSCF_F64, lam, part, out, st);
}

cudaError_t launch_col_resid_t(const void* X, const void* HX, int64_t ld, int64_t rows, int k, int dtype,
                               const double* lam, double* part, double* out, cudaStream_t st) {
  if (dtype == KSCF_F64)
    col_resid_kernel<double><<<kScfRedBlocks, kScfThreads, 0, st>>>((const double*)X, (const double*)HX, ld, rows, k,
                                                                    lam, part), count_launch();
  else
    col_resid_kernel<float><<<kScfRedBlocks, kScfThreads, 0, st>>>((const float*)X, (const float*)HX, ld, rows, k,
                                                                   lam, part), count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_finalize_partials(part, kScfRedBlocks, k, out, st);
}

// dst[r][j] = (double) src[r][j]  (FP32 -> FP64), r < rows, j < k
__global__ void widen_kernel(const float* __restrict__ src, int64_t lds, double* __restrict__ dst, int64_t ldd,
                             int64_t rows, int k) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * k) return;
  const int64_t r = idx / k;
  const int j = (int)(idx - r * k);
  dst[r * ldd + j] = (double)src[r * lds + j];
}

cudaError_t launch_widen(const float* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int k,
                         cudaStream_t st) {
  widen_kernel<<<nblk(rows * k, 256), 256, 0, st>>>(src, lds, dst, ldd, rows, k), count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Anderson mixing.
// New history column: dV = V_in - V_prev, dF = F - F_prev (and dPF = PF - PF_prev when
// the residual is preconditioned); then V_prev = V_in, F_prev = F, PF_prev = PF.
__global__ void anderson_push_kernel(int64_t n, const double* __restrict__ v_in, const double* __restrict__ f,
                                     const double* __restrict__ pf, double* __restrict__ v_prev,
                                     double* __restrict__ f_prev, double* __restrict__ pf_prev,
                                     double* __restrict__ dv, double* __restrict__ df, double* __restrict__ dpf,
                                     int have_prev) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double vi = v_in[s], fi = f[s];
  if (have_prev) {
    dv[s] = vi - v_prev[s];
    df[s] = fi - f_prev[s];
  }
  v_prev[s] = vi;
  f_prev[s] = fi;
  if (pf) {
    const double pi = pf[s];
    if (have_prev) dpf[s] = pi - pf_prev[s];
    pf_prev[s] = pi;
  }
}

cudaError_t launch_anderson_push(int64_t n, const double* v_in, const double* f, const double* pf, double* v_prev,
                                 double* f_prev, double* pf_prev, double* dv, double* df, double* dpf, bool have_prev,
                                 cudaStream_t st) {
  anderson_push_kernel<<<nblk(n, 256), 256, 0, st>>>(n, v_in, f, pf, v_prev, f_prev, pf_prev, dv, df, dpf,
                                                     have_prev ? 1 : 0), count_launch();
  return cudaGetLastError();
}

// Partials of dF_i . dF_j (i <= j, packed row-major upper) and dF_i . F, i, j < m
// (the columns in the order given by cols).
__global__ void __launch_bounds__(kScfThreads) anderson_gram_kernel(AndersonCols cols, const double* __restrict__ df,
                                                                    const double* __restrict__ f, int64_t n,
                                                                    double* __restrict__ part) {
  constexpr int NV = kAndersonMax * (kAndersonMax + 1) / 2 + kAndersonMax;
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; q++) v[q] = 0.0;
  const int m = cols.m;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    double x[kAndersonMax];
#pragma unroll
    for (int i = 0; i < kAndersonMax; i++) x[i] = i < m ? df[(int64_t)cols.idx[i] * n + s] : 0.0;
    const double fv = f[s];
    int q = 0;
#pragma unroll
    for (int i = 0; i < kAndersonMax; i++) {
#pragma unroll
      for (int j = i; j < kAndersonMax; j++) v[q++] += x[i] * x[j];
    }
#pragma unroll
    for (int i = 0; i < kAndersonMax; i++) v[q++] += x[i] * fv;
  }
  block_partials<NV>(v, part);
}

cudaError_t launch_anderson_gram(const AndersonCols& cols, const double* df, const double* f, int64_t n,
                                 double* part, double* out, cudaStream_t st) {
  constexpr int NV = kAndersonMax * (kAndersonMax + 1) / 2 + kAndersonMax;
  anderson_gram_kernel<<<kScfRedBlocks, kScfThreads, 0, st>>>(cols, df, f, n, part), count_launch();
  return launch_finalize_partials(part, kScfRedBlocks, NV, out, st);
}

// V_next = V_in + alpha PF - sum_j g_j (dV_j + alpha dPF_j)   (in place on v; PF = F and
// dPF = dF without a preconditioner)
__global__ void anderson_update_kernel(AndersonCols cols, double alpha, const uint8_t* __restrict__ mask, int64_t n,
                                       const double* __restrict__ dv, const double* __restrict__ df,
                                       const double* __restrict__ f, double* __restrict__ v) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  if (!mask[s]) {
    v[s] = 0.0;
    return;
  }
  double nv = v[s] + alpha * f[s];
  for (int j = 0; j < cols.m; j++) {
    const int64_t o = (int64_t)cols.idx[j] * n + s;
    nv -= cols.g[j] * (dv[o] + alpha * df[o]);
  }
  v[s] = nv;
}

cudaError_t launch_anderson_update(const Ham& H, const AndersonCols& cols, double alpha, const double* dv,
                                   const double* dpf, const double* pf, double* v, cudaStream_t st) {
  const double* df = dpf;
  const double* f = pf;
  const int64_t n = H.grid.n_slots;
  anderson_update_kernel<<<nblk(n, 256), 256, 0, st>>>(cols, alpha, H.d_mask, n, dv, df, f, v), count_launch();
  return cudaGetLastError();
}

// row lex(s) of D_out / t_out for every domain slot s: the slot's descriptors and
// dV = V_in - V_start (training data of the learned start)
__global__ void training_rows_kernel(const float* __restrict__ D, const double* __restrict__ v_in,
                                     const double* __restrict__ v_start, const int64_t* __restrict__ lex,
                                     int64_t n_slots, float* __restrict__ D_out, float* __restrict__ t_out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = t >> 5;
  const int j = (int)(t & 31);
  if (s >= n_slots) return;
  const int64_t p = lex[s];
  if (p < 0) return;
  D_out[p * KSCF_MLP_N_IN + j] = D[s * KSCF_MLP_N_IN + j];
  if (j == 0) t_out[p] = (float)(v_in[s] - v_start[s]);
}

cudaError_t launch_training_rows(const Ham& H, const float* D, const double* v_in, const double* v_start, float* D_out,
                                 float* t_out, cudaStream_t st) {
  const int64_t n = H.grid.n_slots * 32;
  training_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(D, v_in, v_start, H.d_lex, H.grid.n_slots, D_out,
                                                                     t_out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace kscf
