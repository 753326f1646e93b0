// Host driver of the self-consistent field loop (arXiv 2303.00790, Computational
// details): start from neutral-atom densities, then per SCF step the CheFSI
// iterations (four in the first step, one afterwards), the new density, the Hartree
// and exchange-correlation potentials, the self-consistent residual error and
// Anderson mixing of the input potential.  The device work is in scf_kernels.cu and
// the CheFSI entry points of capi.cpp; this file owns buffers, the ghost-point table
// of the Poisson problem and the small host-side solves.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "kscf_internal.h"
#include "scf_internal.h"

using namespace kscf;

struct kscf_scf {
  kscf_ham* ham = nullptr;
  kscf_scf_params p{};
  void* X = nullptr;
  int64_t ld = 0;
  cudaStream_t st = nullptr;
  int n_occ = 0;
  int n_e = 0;
  int64_t n = 0;
  int n_atoms = 0;
  // device buffers (FP64, n slots each unless noted)
  double* rel = nullptr;      // 3n: h (i, j, k)
  double* atoms = nullptr;    // 5 per atom: x, y, z, Z_valence, r_a
  double *v_ion = nullptr, *v_start = nullptr, *v_in = nullptr, *rho = nullptr, *vh = nullptr, *vxc = nullptr,
         *eps = nullptr, *f = nullptr;
  double *cg_b = nullptr, *cg_r = nullptr, *cg_p = nullptr, *cg_q = nullptr;
  double *v_prev = nullptr, *f_prev = nullptr, *dv = nullptr, *df = nullptr;  // dv, df: history x n
  double *pf = nullptr, *pf_prev = nullptr, *dpf = nullptr, *ku = nullptr;  // Kerker: P F, history, solve
  void* hx = nullptr;         // adaptive degrees: H X (n_slots x ld of dtype)
  double sre_prev = 0.0;      // SRE of the previous step (Ry), 0 before the first
  double* part = nullptr;     // kScfRedBlocks x 44 partial sums
  double* part_bb = nullptr;  // kScfRedBlocks
  double* part_rr[2] = {nullptr, nullptr};
  double* part_pq = nullptr;
  double* small = nullptr;    // 128 doubles of reduction results
  int* d_iters = nullptr;
  double* part_col = nullptr; // kScfRedBlocks x k partial column sums
  double* colsq = nullptr;    // k column sums of squares
  double* d_occ = nullptr;    // k occupations divided by the vector norms
  double* host_k = nullptr;   // pinned, 2k doubles
  PoissonPlan P;
  void* work = nullptr;
  size_t work_bytes = 0;
  double* host = nullptr;     // pinned, 128 doubles
  // host state
  std::vector<double> lam;
  int step = 0;
  bool started = false;
  bool have_prev = false;
  int ring_next = 0;
  std::vector<int> order;     // history columns in use, oldest first
  double sums[5] = {0, 0, 0, 0, 0};  // last step: rho f^2, rho (V_in - V_ion), rho V_H, rho eps_xc, rho
  kscf_scf_report last{};
  bool stepped = false;
};

namespace {

// small[] layout
constexpr int kMom = 0;      // 10 multipole sums
constexpr int kRes = 16;     // 5 residual / energy sums
constexpr int kGram = 32;    // 44 Anderson sums
constexpr int kCg = 96;      // r.r, b.b

void free_scf(kscf_scf* S) {
  void* dev[] = {S->rel,    S->atoms,  S->v_ion,  S->v_start, S->v_in,       S->rho,        S->vh,
                 S->vxc,    S->eps,    S->f,      S->cg_b,    S->cg_r,       S->cg_p,       S->cg_q,
                 S->v_prev, S->f_prev, S->dv,     S->df,      S->part,       S->part_bb,    S->part_rr[0],
                 S->part_rr[1], S->part_pq, S->small, S->d_iters, S->P.d_grel, S->P.d_vghost, S->P.d_gptr,
                 S->P.d_gidx, S->P.d_gw, S->work, S->part_col, S->colsq, S->d_occ,
                 S->pf, S->pf_prev, S->dpf, S->ku, S->hx};
  for (void* q : dev)
    if (q) cudaFree(q);
  if (S->host) cudaFreeHost(S->host);
  if (S->host_k) cudaFreeHost(S->host_k);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

// Ghost points of the order-12 stencil (6 per side along each axis) and the CSR
// coupling of each domain slot to them: (Lap_h V)_s picks up w_k / h^2 V(ghost) for
// every neighbour at distance k outside the domain.
int build_poisson_plan(const Ham& H, PoissonPlan* P, cudaStream_t st) {
  const Grid& g = H.grid;
  const int64_t n = g.n_slots;
  std::vector<int64_t> ptr(n + 1, 0);
  std::vector<int32_t> gidx;
  std::vector<double> gw;
  std::vector<double> grel;
  std::unordered_map<uint64_t, int32_t> id;
  auto key = [](int i, int j, int k) {
    const uint64_t o = 1u << 20;
    return ((uint64_t)(i + o) << 42) | ((uint64_t)(j + o) << 21) | (uint64_t)(k + o);
  };
  for (int64_t s = 0; s < n; s++) {
    if (g.mask[s]) {
      int ijk[3];
      g.slot_ijk(s, ijk);
      for (int ax = 0; ax < 3; ax++)
        for (int k = 1; k <= 6; k++)
          for (int sg = -1; sg <= 1; sg += 2) {
            int q[3] = {ijk[0], ijk[1], ijk[2]};
            q[ax] += sg * k;
            const int64_t ns = g.slot_of(q[0], q[1], q[2]);
            if (ns >= 0 && g.mask[ns]) continue;
            const uint64_t kk = key(q[0], q[1], q[2]);
            auto it = id.find(kk);
            int32_t gi;
            if (it == id.end()) {
              gi = (int32_t)(grel.size() / 3);
              id.emplace(kk, gi);
              for (int d = 0; d < 3; d++) grel.push_back(g.h * (double)q[d]);
            } else {
              gi = it->second;
            }
            gidx.push_back(gi);
            gw.push_back(-2.0 * H.stencil[k]);  // H.stencil[k] = -1/2 w_k / h^2
          }
    }
    ptr[s + 1] = (int64_t)gidx.size();
  }
  P->n_ghost = (int64_t)(grel.size() / 3);
  cudaError_t e = dalloc(&P->d_grel, grel.size());
  if (e == cudaSuccess) e = dalloc(&P->d_vghost, (size_t)P->n_ghost);
  if (e == cudaSuccess) e = dalloc(&P->d_gptr, ptr.size());
  if (e == cudaSuccess) e = dalloc(&P->d_gidx, gidx.size());
  if (e == cudaSuccess) e = dalloc(&P->d_gw, gw.size());
  if (e == cudaSuccess && !grel.empty())
    e = cudaMemcpyAsync(P->d_grel, grel.data(), grel.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_gptr, ptr.data(), ptr.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !gidx.empty())
    e = cudaMemcpyAsync(P->d_gidx, gidx.data(), gidx.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !gw.empty())
    e = cudaMemcpyAsync(P->d_gw, gw.data(), gw.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
  if (e != cudaSuccess) {
    set_error("kscf_scf_create: Poisson table upload failed: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  return KSCF_OK;
}

int sync_read(kscf_scf* S, const double* src, int count, double* dst) {
  KSCF_CUDA_TRY(cudaMemcpyAsync(S->host, src, sizeof(double) * count, cudaMemcpyDeviceToHost, S->st));
  KSCF_CUDA_TRY(cudaStreamSynchronize(S->st));
  std::memcpy(dst, S->host, sizeof(double) * count);
  return KSCF_OK;
}

int read_iters(kscf_scf* S, int* it) {
  KSCF_CUDA_TRY(cudaMemcpyAsync(S->host, S->d_iters, sizeof(int), cudaMemcpyDeviceToHost, S->st));
  KSCF_CUDA_TRY(cudaStreamSynchronize(S->st));
  std::memcpy(it, S->host, sizeof(int));
  return KSCF_OK;
}

// CG on (-Lap_h + shift) x = b for the right-hand side already in S->cg_b (its partial
// squares in S->part_bb), from the guess in x.
int cg_solve(kscf_scf* S, double shift, double* x, int* iters_out, const char* what) {
  const Ham& H = S->ham->h;
  cudaStream_t st = S->st;
  KSCF_CUDA_TRY(launch_mask_v(H, x, x, st));
  KSCF_CUDA_TRY(cudaMemsetAsync(S->d_iters, 0, sizeof(int), st));
  int cur = 0;
  KSCF_CUDA_TRY(launch_cg_init(H, shift, x, S->cg_b, S->cg_r, S->cg_p, S->part_rr[cur], st));
  const double rtol = S->p.poisson_rtol;
  double cg[2];
  KSCF_CUDA_TRY(launch_finalize_partials(S->part_rr[cur], kScfRedBlocks, 1, S->small + kCg, st));
  KSCF_CUDA_TRY(launch_finalize_partials(S->part_bb, kScfRedBlocks, 1, S->small + kCg + 1, st));
  int rc = sync_read(S, S->small + kCg, 2, cg);
  if (rc) return rc;
  if (!std::isfinite(cg[0]) || !std::isfinite(cg[1])) {
    set_error("kscf_scf: non-finite %s right-hand side or guess", what);
    return KSCF_ERR_NONFINITE;
  }
  if (iters_out) *iters_out = 0;
  if (cg[1] == 0.0) {  // zero right-hand side: zero solution
    KSCF_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * S->n, st));
    return KSCF_OK;
  }
  int launched = 0;
  const int batch = 16;
  while (!(cg[0] < rtol * rtol * cg[1])) {
    if (launched >= S->p.poisson_maxiter) {
      int it = 0;
      rc = read_iters(S, &it);
      if (rc) return rc;
      if (iters_out) *iters_out = it;
      set_error("kscf_scf: %s CG not converged after %d iterations (|r|/|b| = %.3e)", what, it,
                std::sqrt(cg[0] / cg[1]));
      return KSCF_ERR_NO_CONVERGE;
    }
    for (int i = 0; i < batch; i++) {
      KSCF_CUDA_TRY(launch_cg_iteration(H, shift, S->part_bb, rtol, x, S->cg_r, S->cg_p, S->cg_q, S->part_rr[cur],
                                        S->part_pq, S->part_rr[cur ^ 1], S->d_iters, st));
      cur ^= 1;
    }
    launched += batch;
    KSCF_CUDA_TRY(launch_finalize_partials(S->part_rr[cur], kScfRedBlocks, 1, S->small + kCg, st));
    rc = sync_read(S, S->small + kCg, 1, cg);
    if (rc) return rc;
    if (!std::isfinite(cg[0])) {
      set_error("kscf_scf: %s CG produced a non-finite residual", what);
      return KSCF_ERR_NONFINITE;
    }
  }
  int it = 0;
  rc = read_iters(S, &it);
  if (rc) return rc;
  if (iters_out) *iters_out = it;
  return KSCF_OK;
}

// -Lap_h x = 4 pi rho (+ ghost terms) by CG from the guess in x.
int hartree(kscf_scf* S, const double* rho, double* x, int* iters_out) {
  const Ham& H = S->ham->h;
  cudaStream_t st = S->st;
  KSCF_CUDA_TRY(launch_ghost_values(H, rho, S->rel, S->P, S->part, S->small + kMom, st));
  KSCF_CUDA_TRY(launch_poisson_rhs(H, rho, S->P, S->cg_b, S->part_bb, st));
  return cg_solve(S, 0.0, x, iters_out, "Poisson");
}

// Kerker preconditioner: pf = f - q0^2 u with (-Lap_h + q0^2) u = f (u warm-started
// from the previous step's solution).
int kerker(kscf_scf* S, const double* f, double* pf, int* iters_out) {
  const Ham& H = S->ham->h;
  const double q2 = S->p.kerker_q0 * S->p.kerker_q0;
  KSCF_CUDA_TRY(launch_rhs_copy(H, f, S->cg_b, S->part_bb, S->st));
  int rc = cg_solve(S, q2, S->ku, iters_out, "Kerker");
  if (rc) return rc;
  KSCF_CUDA_TRY(launch_lincomb(H, f, S->ku, -q2, pf, S->st));
  return KSCF_OK;
}

// Solves the m x m system G g = r (Gaussian elimination with partial pivoting).
bool solve_small(int m, std::vector<double> G, std::vector<double> r, double* g) {
  for (int c = 0; c < m; c++) {
    int piv = c;
    for (int i = c + 1; i < m; i++)
      if (std::fabs(G[i * m + c]) > std::fabs(G[piv * m + c])) piv = i;
    if (G[piv * m + c] == 0.0) return false;
    if (piv != c) {
      for (int j = 0; j < m; j++) std::swap(G[c * m + j], G[piv * m + j]);
      std::swap(r[c], r[piv]);
    }
    for (int i = c + 1; i < m; i++) {
      const double l = G[i * m + c] / G[c * m + c];
      for (int j = c; j < m; j++) G[i * m + j] -= l * G[c * m + j];
      r[i] -= l * r[c];
    }
  }
  for (int i = m - 1; i >= 0; i--) {
    double s = r[i];
    for (int j = i + 1; j < m; j++) s -= G[i * m + j] * g[j];
    g[i] = s / G[i * m + i];
  }
  for (int i = 0; i < m; i++)
    if (!std::isfinite(g[i])) return false;
  return true;
}

// Occupations of the Ritz values lam (ascending) for n_e electrons (spin-degenerate).
// kT = 0: 2 for the n_e/2 lowest.  kT > 0: 2 f((lam - mu)/kT), f(x) = (1 - tanh(x/2))/2,
// mu by 200 bisection halvings of [min lam - 1 - 50 kT, max lam + 1 + 50 kT] on the
// electron count; minus_ts = 2 kT sum [f ln f + (1 - f) ln(1 - f)].
void occupations(const std::vector<double>& lam, int n_e, double kT, std::vector<double>& occ, double* mu,
                 double* minus_ts) {
  const int k = (int)lam.size();
  occ.assign(k, 0.0);
  *minus_ts = 0.0;
  if (kT == 0.0) {
    for (int i = 0; i < n_e / 2; i++) occ[i] = 2.0;
    *mu = lam[n_e / 2 - 1];
    return;
  }
  double lo = lam[0], hi = lam[0];
  for (double l : lam) {
    lo = std::min(lo, l);
    hi = std::max(hi, l);
  }
  lo -= 1.0 + 50.0 * kT;
  hi += 1.0 + 50.0 * kT;
  auto fd = [](double x) { return 0.5 * (1.0 - std::tanh(0.5 * x)); };
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    double cnt = 0.0;
    for (double l : lam) cnt += 2.0 * fd((l - mid) / kT);
    if (cnt < (double)n_e)
      lo = mid;
    else
      hi = mid;
  }
  *mu = 0.5 * (lo + hi);
  double s = 0.0;
  for (int i = 0; i < k; i++) {
    const double f = fd((lam[i] - *mu) / kT);
    occ[i] = 2.0 * f;
    if (f > 0.0 && f < 1.0) s += f * std::log(f) + (1.0 - f) * std::log(1.0 - f);
  }
  *minus_ts = kT * 2.0 * s;
}

// Degrees of the column groups from Rayleigh quotients and residuals with the current H
// (the per-vector degrees of ChASE): see kscf_scf_params.degree_max.
int adaptive_degrees(kscf_scf* S, double a, double b, std::vector<int>& degs) {
  const kscf_scf_params& p = S->p;
  const Ham& H = S->ham->h;
  const int k = p.k;
  const double h3 = H.grid.h * H.grid.h * H.grid.h;
  cudaStream_t st = S->st;
  int rc = kscf_hamiltonian_apply(S->ham, S->X, S->ld, S->hx, S->ld, k, p.dtype, S->work, S->work_bytes, st);
  if (rc) return rc;
  KSCF_CUDA_TRY(launch_col_dot(S->X, S->ld, S->hx, S->ld, S->n, k, p.dtype, S->part_col, S->colsq, st));
  KSCF_CUDA_TRY(cudaMemcpyAsync(S->host_k, S->colsq, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  KSCF_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<double> rq(k), r(k);
  for (int i = 0; i < k; i++) rq[i] = h3 * S->host_k[i];
  std::memcpy(S->host_k, rq.data(), sizeof(double) * k);
  KSCF_CUDA_TRY(cudaMemcpyAsync(S->d_occ, S->host_k, sizeof(double) * k, cudaMemcpyHostToDevice, st));
  KSCF_CUDA_TRY(launch_col_resid_t(S->X, S->hx, S->ld, S->n, k, p.dtype, S->d_occ, S->part_col, S->colsq, st));
  KSCF_CUDA_TRY(cudaMemcpyAsync(S->host_k, S->colsq, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  KSCF_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < k; i++) r[i] = std::sqrt(std::max(h3 * S->host_k[i], 0.0));
  const double e = (b - a) / 2.0, c = (b + a) / 2.0;
  const int G = p.degree_group;
  degs.assign((k + G - 1) / G, p.degree_min);
  for (int i = 0; i < k; i++) {
    const double t = (c - rq[i]) / e;
    const double tol = std::max(p.adapt_tol_floor, p.adapt_reduction * r[i]);
    int m;
    if (t <= 1.0 + 1e-12) {
      m = p.degree_max;
    } else if (r[i] <= tol) {
      m = p.degree_min;
    } else {
      const double rho = 1.0 / (t + std::sqrt(t * t - 1.0));
      const double mm = std::ceil(std::log(tol / r[i]) / std::log(rho));
      m = mm > (double)p.degree_max ? p.degree_max : (int)mm;
    }
    m = std::min(std::max(m, p.degree_min), p.degree_max);
    degs[i / G] = std::max(degs[i / G], m);
  }
  return KSCF_OK;
}

int eig_step(kscf_scf* S, bool filter, double b_upper, double* work_out = nullptr) {
  const kscf_scf_params& p = S->p;
  kscf_ham* ham = S->ham;
  if (filter) {
    const double a = S->lam[p.k - 1], a0 = S->lam[0];
    if (p.degree_max > 0) {
      std::vector<int> degs;
      int rc = adaptive_degrees(S, a, b_upper, degs);
      if (rc) return rc;
      const size_t es = p.dtype == KSCF_F64 ? 8 : 4;
      for (size_t g = 0; g < degs.size(); g++) {
        const int c0 = (int)g * p.degree_group;
        const int nc = std::min(p.degree_group, p.k - c0);
        rc = kscf_chebyshev_filter(ham, (char*)S->X + (size_t)c0 * es, S->ld, nc, degs[g], a, b_upper, a0, p.dtype, 0,
                                   S->work, S->work_bytes, S->st);
        if (rc) return rc;
        if (work_out) *work_out += (double)degs[g] * nc / p.k;
      }
    } else {
      int rc = kscf_chebyshev_filter(ham, S->X, S->ld, p.k, p.degree, a, b_upper, a0, p.dtype, p.block, S->work,
                                     S->work_bytes, S->st);
      if (rc) return rc;
      if (work_out) *work_out += p.degree;
    }
  }
  int rc = kscf_orthonormalize(ham, S->X, S->ld, p.k, p.dtype, p.gemm_mode | KSCF_ORTHO_ALLOW_SHIFT, S->work,
                               S->work_bytes, S->st);
  if (rc) return rc;
  return kscf_rayleigh_ritz(ham, S->X, S->ld, p.k, p.dtype, p.gemm_mode, S->lam.data(), S->work, S->work_bytes,
                            S->st);
}

}  // namespace

extern "C" int kscf_lda_xc(const kscf_ham* ham, const double* rho, double* eps, double* vxc, void* stream) {
  if (!ham || !rho || !vxc) {
    set_error("kscf_lda_xc: null argument");
    return KSCF_ERR_INVALID;
  }
  KSCF_CUDA_TRY(launch_lda(ham->h, rho, eps, vxc, (cudaStream_t)stream));
  return KSCF_OK;
}

extern "C" int kscf_scf_free(kscf_scf* scf) {
  if (!scf) return KSCF_OK;
  free_scf(scf);
  delete scf;
  return KSCF_OK;
}

extern "C" int kscf_scf_create(kscf_ham* ham, const kscf_atom* atoms, int n_atoms, const kscf_species* species,
                               int n_species, const double* start_radius, const kscf_scf_params* params, void* X,
                               int64_t ld, void* stream, kscf_scf** out) {
  if (!ham || !out || !params || !X || n_atoms < 1 || !atoms || n_species < 1 || !species || !start_radius) {
    set_error("kscf_scf_create: null or empty argument");
    return KSCF_ERR_INVALID;
  }
  const kscf_scf_params& p = *params;
  if ((p.dtype != KSCF_F64 && p.dtype != KSCF_F32) || (p.gemm_mode != KSCF_GEMM_NATIVE && p.gemm_mode != KSCF_GEMM_TENSOR) ||
      (p.gemm_mode == KSCF_GEMM_TENSOR && p.dtype != KSCF_F32) || p.degree < 1 || p.first_iters < 1 ||
      p.history < 1 || p.history > kAndersonMax || !(p.mix_alpha > 0.0 && p.mix_alpha <= 1.0) ||
      !(p.sre_tol_ry > 0.0) || !(p.poisson_rtol > 0.0) || p.poisson_maxiter < 1 || p.block < 0 || ld < p.k ||
      !(p.kT >= 0.0) || !std::isfinite(p.kT) || !(p.kerker_q0 >= 0.0) || !std::isfinite(p.kerker_q0) ||
      p.degree_max < 0 || (p.degree_max > 0 && (p.degree_min < 1 || p.degree_min > p.degree_max ||
                                                  p.degree_group < 1 || !(p.adapt_reduction > 0.0 && p.adapt_reduction < 1.0) ||
                                                  !(p.adapt_tol_floor > 0.0))) ||
      (p.upper_bound != 0 && p.upper_bound != 1)) {
    set_error("kscf_scf_create: invalid parameters");
    return KSCF_ERR_INVALID;
  }
  double n_e = 0.0;
  std::vector<double> at(5 * (size_t)n_atoms);
  for (int a = 0; a < n_atoms; a++) {
    int found = -1;
    for (int s = 0; s < n_species; s++)
      if (species[s].z_number == atoms[a].z_number) found = s;
    if (found < 0 || !(start_radius[found] > 0.0)) {
      set_error("kscf_scf_create: no species or start radius for atom %d (Z=%d)", a, atoms[a].z_number);
      return KSCF_ERR_INVALID;
    }
    n_e += species[found].z_valence;
    double* r = &at[5 * (size_t)a];
    r[0] = atoms[a].x;
    r[1] = atoms[a].y;
    r[2] = atoms[a].z;
    r[3] = species[found].z_valence;
    r[4] = start_radius[found];
  }
  const int n_e_int = (int)std::lround(n_e);
  if (std::fabs(n_e - n_e_int) > 1e-9 || n_e_int % 2 != 0 || n_e_int < 2 || p.k <= n_e_int / 2) {
    set_error("kscf_scf_create: need an even integer electron count n_e (got %.6f) and k > n_e/2", n_e);
    return KSCF_ERR_INVALID;
  }
  kscf_scf* S = new (std::nothrow) kscf_scf();
  if (!S) {
    set_error("kscf_scf_create: host allocation failed");
    return KSCF_ERR_HOST_ALLOC;
  }
  S->ham = ham;
  S->p = p;
  S->X = X;
  S->ld = ld;
  S->st = (cudaStream_t)stream;
  S->n_occ = n_e_int / 2;
  S->n_e = n_e_int;
  S->n_atoms = n_atoms;
  const Ham& H = ham->h;
  const Grid& g = H.grid;
  const int64_t n = g.n_slots;
  S->n = n;
  int rc = KSCF_OK;
  try {
    S->lam.assign(p.k, 0.0);
    cudaError_t e = cudaSuccess;
    double** vecs[] = {&S->v_ion, &S->v_start, &S->v_in, &S->rho, &S->vh, &S->vxc, &S->eps, &S->f,
                       &S->cg_b,  &S->cg_r,    &S->cg_p, &S->cg_q, &S->v_prev, &S->f_prev};
    for (double** v : vecs)
      if (e == cudaSuccess) e = dalloc(v, (size_t)n);
    if (e == cudaSuccess) e = dalloc(&S->dv, (size_t)p.history * n);
    if (e == cudaSuccess) e = dalloc(&S->df, (size_t)p.history * n);
    if (p.degree_max > 0 && e == cudaSuccess)
      e = cudaMalloc(&S->hx, (size_t)n * ld * (p.dtype == KSCF_F64 ? 8 : 4));
    if (p.kerker_q0 > 0.0) {
      double** kv[] = {&S->pf, &S->pf_prev, &S->ku};
      for (double** v : kv) {
        if (e == cudaSuccess) e = dalloc(v, (size_t)n);
        if (e == cudaSuccess) e = cudaMemsetAsync(*v, 0, sizeof(double) * n, S->st);
      }
      if (e == cudaSuccess) e = dalloc(&S->dpf, (size_t)p.history * n);
    }
    if (e == cudaSuccess) e = dalloc(&S->rel, 3 * (size_t)n);
    if (e == cudaSuccess) e = dalloc(&S->atoms, at.size());
    if (e == cudaSuccess) e = dalloc(&S->part, (size_t)kScfRedBlocks * 48);
    if (e == cudaSuccess) e = dalloc(&S->part_bb, (size_t)kScfRedBlocks);
    if (e == cudaSuccess) e = dalloc(&S->part_rr[0], (size_t)kScfRedBlocks);
    if (e == cudaSuccess) e = dalloc(&S->part_rr[1], (size_t)kScfRedBlocks);
    if (e == cudaSuccess) e = dalloc(&S->part_pq, (size_t)kScfRedBlocks);
    if (e == cudaSuccess) e = dalloc(&S->small, 128);
    if (e == cudaSuccess) e = dalloc(&S->d_iters, 1);
    if (e == cudaSuccess) e = dalloc(&S->part_col, (size_t)kScfRedBlocks * p.k);
    if (e == cudaSuccess) e = dalloc(&S->colsq, (size_t)p.k);
    if (e == cudaSuccess) e = dalloc(&S->d_occ, (size_t)p.k);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&S->host_k, 2 * (size_t)p.k * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&S->host, 128 * sizeof(double));
    if (e != cudaSuccess) {
      set_error("kscf_scf_create: device allocation failed: %s", cudaGetErrorString(e));
      rc = KSCF_ERR_CUDA;
      throw 1;
    }
    for (double** v : vecs) cudaMemsetAsync(*v, 0, sizeof(double) * n, S->st);
    std::vector<double> rel(3 * (size_t)n);
    for (int64_t s = 0; s < n; s++) {
      int ijk[3];
      g.slot_ijk(s, ijk);
      for (int d = 0; d < 3; d++) rel[3 * s + d] = g.h * (double)ijk[d];
    }
    e = cudaMemcpyAsync(S->rel, rel.data(), rel.size() * 8, cudaMemcpyHostToDevice, S->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->atoms, at.data(), at.size() * 8, cudaMemcpyHostToDevice, S->st);
    // V_ion: the Hamiltonian's local potential as built
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->v_ion, H.d_vion, sizeof(double) * n, cudaMemcpyDeviceToDevice, S->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
    if (e != cudaSuccess) {
      set_error("kscf_scf_create: upload failed: %s", cudaGetErrorString(e));
      rc = KSCF_ERR_CUDA;
      throw 1;
    }
    rc = build_poisson_plan(H, &S->P, S->st);
    if (rc) throw 1;
    size_t wf = 0, wo = 0, wr = 0;
    rc = kscf_workspace_size(ham, KSCF_OP_FILTER, p.k, p.dtype, p.gemm_mode, p.block, &wf);
    if (!rc) rc = kscf_workspace_size(ham, KSCF_OP_ORTHO, p.k, p.dtype, p.gemm_mode, 0, &wo);
    if (!rc) rc = kscf_workspace_size(ham, KSCF_OP_RR, p.k, p.dtype, p.gemm_mode, 0, &wr);
    if (rc) throw 1;
    S->work_bytes = std::max(wf, std::max(wo, wr));
    e = cudaMalloc(&S->work, S->work_bytes);
    if (e != cudaSuccess) {
      set_error("kscf_scf_create: work buffer of %zu bytes: %s", S->work_bytes, cudaGetErrorString(e));
      rc = KSCF_ERR_CUDA;
      throw 1;
    }
  } catch (const std::bad_alloc&) {
    set_error("kscf_scf_create: host allocation failed");
    rc = KSCF_ERR_HOST_ALLOC;
  } catch (int) {
  }
  if (rc != KSCF_OK) {
    free_scf(S);
    delete S;
    return rc;
  }
  *out = S;
  return KSCF_OK;
}

extern "C" int kscf_scf_hartree(kscf_scf* scf, const double* rho, double* vh, int* iters) {
  if (!scf || !rho || !vh) {
    set_error("kscf_scf_hartree: null argument");
    return KSCF_ERR_INVALID;
  }
  return hartree(scf, rho, vh, iters);
}

extern "C" int kscf_scf_start(kscf_scf* scf, const double* dv_start, int init_x, uint64_t seed, double* eigvals_host) {
  if (!scf) {
    set_error("kscf_scf_start: null handle");
    return KSCF_ERR_INVALID;
  }
  kscf_scf* S = scf;
  const Ham& H = S->ham->h;
  cudaStream_t st = S->st;
  S->step = 0;
  S->have_prev = false;
  S->ring_next = 0;
  S->order.clear();
  S->started = false;
  S->stepped = false;
  S->sre_prev = 0.0;
  if (init_x) {
    int rc = kscf_random_subspace(S->ham, S->X, S->ld, S->p.k, S->p.dtype, seed, st);
    if (rc) return rc;
  }
  KSCF_CUDA_TRY(launch_atomic_density(H, S->rel, S->atoms, S->n_atoms, S->rho, st));
  KSCF_CUDA_TRY(cudaMemsetAsync(S->vh, 0, sizeof(double) * S->n, st));
  int rc = hartree(S, S->rho, S->vh, nullptr);
  if (rc) return rc;
  KSCF_CUDA_TRY(launch_lda(H, S->rho, S->eps, S->vxc, st));
  KSCF_CUDA_TRY(launch_sum3(H, S->v_ion, S->vh, S->vxc, S->v_start, st));
  if (dv_start)
    KSCF_CUDA_TRY(launch_add2(H, S->v_start, dv_start, S->v_in, st));
  else
    KSCF_CUDA_TRY(cudaMemcpyAsync(S->v_in, S->v_start, sizeof(double) * S->n, cudaMemcpyDeviceToDevice, st));
  rc = kscf_set_potential(S->ham, S->v_in, st);
  if (rc) return rc;
  rc = eig_step(S, false, 0.0);
  if (rc) return rc;
  if (eigvals_host) std::memcpy(eigvals_host, S->lam.data(), sizeof(double) * S->p.k);
  S->started = true;
  return KSCF_OK;
}

int density_energy(kscf_scf* S, kscf_scf_report* report);
int mix(kscf_scf* S, kscf_scf_report* report);

extern "C" int kscf_scf_step(kscf_scf* scf, kscf_scf_report* report, double* eigvals_host) {
  if (!scf || !report) {
    set_error("kscf_scf_step: null argument");
    return KSCF_ERR_INVALID;
  }
  kscf_scf* S = scf;
  if (!S->started) {
    set_error("kscf_scf_step: call kscf_scf_start first");
    return KSCF_ERR_INVALID;
  }
  const Ham& H = S->ham->h;
  const kscf_scf_params& p = S->p;
  cudaStream_t st = S->st;
  const double h3 = H.grid.h * H.grid.h * H.grid.h;
  S->step++;
  std::memset(report, 0, sizeof(*report));
  report->step = S->step;

  // Hamiltonian at V_in and the CheFSI iterations
  int rc = kscf_set_potential(S->ham, S->v_in, st);
  if (rc) return rc;
  KSCF_CUDA_TRY(cudaStreamSynchronize(st));
  double lower = 0.0, upper = 0.0;
  rc = kscf_spectral_bounds(S->ham, &lower, &upper);
  if (rc) return rc;
  if (p.upper_bound == 1) {
    double lz = 0.0;
    rc = kscf_lanczos_bounds(S->ham, 12, 7, &lz, nullptr, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    upper = std::min(upper, lz);
  }
  report->upper_bound = upper;
  const int iters = S->step == 1 ? p.first_iters : 1;
  for (int it = 0; it < iters; it++) {
    rc = eig_step(S, true, upper, &report->filter_work);
    if (rc) return rc;
  }
  rc = kscf_check_status();
  if (rc) return rc;
  report->chefsi_iters = iters;

  rc = density_energy(S, report);
  if (rc) return rc;
  if (eigvals_host) std::memcpy(eigvals_host, S->lam.data(), sizeof(double) * p.k);
  report->converged = report->sre_ry < p.sre_tol_ry ? 1 : 0;
  S->sre_prev = report->sre_ry;
  S->last = *report;
  S->stepped = true;
  if (report->converged) return KSCF_OK;
  return mix(S, report);
}

// occupations of the current Ritz values, the output density of the normalised Ritz
// vectors, its Hartree and exchange-correlation potentials, the residual V_out - V_in and
// the energy integrals (S->sums); fills the density and energy figures of report
int density_energy(kscf_scf* S, kscf_scf_report* report) {
  const Ham& H = S->ham->h;
  const kscf_scf_params& p = S->p;
  cudaStream_t st = S->st;
  const double h3 = H.grid.h * H.grid.h * H.grid.h;
  int rc = KSCF_OK;
  std::vector<double> occ;
  double mu = 0.0, minus_ts = 0.0;
  occupations(S->lam, S->n_e, p.kT, occ, &mu, &minus_ts);
  const int n_used = p.kT == 0.0 ? S->n_occ : p.k;
  KSCF_CUDA_TRY(launch_col_sumsq(S->X, S->ld, S->n, n_used, p.dtype, S->part_col, S->colsq, st));
  KSCF_CUDA_TRY(cudaMemcpyAsync(S->host_k, S->colsq, sizeof(double) * n_used, cudaMemcpyDeviceToHost, st));
  KSCF_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < n_used; i++) {
    const double nrm = h3 * S->host_k[i];
    if (!(nrm > 0.0) || !std::isfinite(nrm)) {
      set_error("kscf_scf_step: Ritz vector %d has norm %g", i, nrm);
      return KSCF_ERR_NONFINITE;
    }
    S->host_k[p.k + i] = occ[i] / nrm;
  }
  KSCF_CUDA_TRY(cudaMemcpyAsync(S->d_occ, S->host_k + p.k, sizeof(double) * n_used, cudaMemcpyHostToDevice, st));
  rc = kscf_density(S->ham, S->X, S->ld, n_used, p.dtype, S->d_occ, S->rho, st);
  if (rc) return rc;
  rc = hartree(S, S->rho, S->vh, &report->poisson_iters);
  if (rc) return rc;
  KSCF_CUDA_TRY(launch_lda(H, S->rho, S->eps, S->vxc, st));
  KSCF_CUDA_TRY(launch_residual(H, S->rho, S->v_in, S->v_ion, S->vh, S->vxc, S->eps, S->f, S->part,
                                S->small + kRes, st));
  double* sums = S->sums;
  rc = sync_read(S, S->small + kRes, 5, sums);
  if (rc) return rc;
  double e_band = 0.0;
  for (int i = 0; i < p.k; i++) e_band += occ[i] * S->lam[i];
  report->sre_ry = 2.0 * std::sqrt(h3 * sums[0]);
  report->e_band = e_band;
  report->e_total = e_band - h3 * sums[1] + 0.5 * h3 * sums[2] + h3 * sums[3] + minus_ts;
  report->mu = mu;
  report->minus_ts = minus_ts;
  report->occ_last = occ[p.k - 1];
  report->electrons = h3 * sums[4];
  report->homo = S->lam[S->n_occ - 1];
  report->lumo = S->lam[S->n_occ];
  if (!std::isfinite(report->sre_ry) || !std::isfinite(report->e_total)) {
    set_error("kscf_scf_step: non-finite residual or energy");
    return KSCF_ERR_NONFINITE;
  }
  return KSCF_OK;
}

// Anderson mixing of V_in (with the Kerker-preconditioned residual when q0 > 0)
int mix(kscf_scf* S, kscf_scf_report* report) {
  const Ham& H = S->ham->h;
  const kscf_scf_params& p = S->p;
  cudaStream_t st = S->st;
  int rc = KSCF_OK;
  const int m = p.history;
  const int slot = S->ring_next;
  const bool kerk = p.kerker_q0 > 0.0;
  if (kerk) {
    rc = kerker(S, S->f, S->pf, &report->kerker_iters);
    if (rc) return rc;
  }
  KSCF_CUDA_TRY(launch_anderson_push(S->n, S->v_in, S->f, kerk ? S->pf : nullptr, S->v_prev, S->f_prev, S->pf_prev,
                                     S->dv + (size_t)slot * S->n, S->df + (size_t)slot * S->n,
                                     kerk ? S->dpf + (size_t)slot * S->n : nullptr, S->have_prev, st));
  if (S->have_prev) {
    if ((int)S->order.size() == m) S->order.erase(S->order.begin());
    S->order.push_back(slot);
    S->ring_next = (slot + 1) % m;
  }
  S->have_prev = true;
  AndersonCols cols;
  cols.m = (int)S->order.size();
  for (int j = 0; j < cols.m; j++) cols.idx[j] = S->order[j];
  if (cols.m > 0) {
    KSCF_CUDA_TRY(launch_anderson_gram(cols, S->df, S->f, S->n, S->part, S->small + kGram, st));
    double gs[kAndersonMax * (kAndersonMax + 1) / 2 + kAndersonMax];
    const int nv = kAndersonMax * (kAndersonMax + 1) / 2 + kAndersonMax;
    rc = sync_read(S, S->small + kGram, nv, gs);
    if (rc) return rc;
    const int mm = cols.m;
    std::vector<double> G((size_t)mm * mm), r(mm);
    int q = 0;
    for (int i = 0; i < kAndersonMax; i++)
      for (int j = i; j < kAndersonMax; j++, q++)
        if (i < mm && j < mm) G[i * mm + j] = G[j * mm + i] = gs[q];
    for (int i = 0; i < mm; i++) r[i] = gs[q + i];
    if (!solve_small(mm, G, r, cols.g)) {
      set_error("kscf_scf_step: singular Anderson mixing system (history %d)", mm);
      return KSCF_ERR_NONFINITE;
    }
  }
  KSCF_CUDA_TRY(launch_anderson_update(H, cols, p.mix_alpha, S->dv, kerk ? S->dpf : S->df, kerk ? S->pf : S->f,
                                       S->v_in, st));
  return KSCF_OK;
}

extern "C" int kscf_scf_evaluate(kscf_scf* scf, kscf_scf_report* report, double* eigvals_host, double* resid_host) {
  if (!scf || !report) {
    set_error("kscf_scf_evaluate: null argument");
    return KSCF_ERR_INVALID;
  }
  kscf_scf* S = scf;
  if (!S->stepped) {
    set_error("kscf_scf_evaluate: call kscf_scf_step first");
    return KSCF_ERR_INVALID;
  }
  const Ham& H = S->ham->h;
  const kscf_scf_params& p = S->p;
  const int k = p.k;
  const int64_t n = S->n;
  const double h3 = H.grid.h * H.grid.h * H.grid.h;
  cudaStream_t st = S->st;
  const int64_t ld64 = (k + 31) / 32 * 32;
  size_t wb = 0;
  int rc = kscf_workspace_size(S->ham, KSCF_OP_APPLY, k, KSCF_F64, 0, 0, &wb);
  if (rc) return rc;
  double *X64 = nullptr, *HX64 = nullptr, *lam_d = nullptr;
  void* work = nullptr;
  auto release = [&]() {
    if (p.dtype != KSCF_F64 && X64) cudaFree(X64);
    if (HX64) cudaFree(HX64);
    if (lam_d) cudaFree(lam_d);
    if (work) cudaFree(work);
  };
  int64_t ldx = ld64;
  cudaError_t e = cudaSuccess;
  if (p.dtype == KSCF_F64) {
    X64 = (double*)S->X;
    ldx = S->ld;
  } else {
    e = cudaMalloc((void**)&X64, sizeof(double) * n * ld64);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&HX64, sizeof(double) * n * ldx);
  if (e == cudaSuccess) e = cudaMalloc((void**)&lam_d, sizeof(double) * k);
  if (e == cudaSuccess) e = cudaMalloc(&work, std::max<size_t>(wb, 256));
  if (e != cudaSuccess) {
    release();
    set_error("kscf_scf_evaluate: device allocation failed: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  // the Hamiltonian of the last step (its V_in), applied in FP64 to the Ritz vectors
  rc = kscf_set_potential(S->ham, S->v_in, st);
  if (!rc && p.dtype != KSCF_F64) {
    e = launch_widen((const float*)S->X, S->ld, X64, ld64, n, k, st);
    if (e != cudaSuccess) {
      set_error("kscf_scf_evaluate: %s", cudaGetErrorString(e));
      rc = KSCF_ERR_CUDA;
    }
  }
  if (!rc) rc = kscf_hamiltonian_apply(S->ham, X64, ldx, HX64, ldx, k, KSCF_F64, work, std::max<size_t>(wb, 256), st);
  std::vector<double> num(k), den(k), res(k), lam(k);
  if (!rc) {
    e = launch_col_dot(X64, ldx, HX64, ldx, n, k, KSCF_F64, S->part_col, S->colsq, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->host_k, S->colsq, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) std::memcpy(num.data(), S->host_k, sizeof(double) * k);
    if (e == cudaSuccess) e = launch_col_dot(X64, ldx, X64, ldx, n, k, KSCF_F64, S->part_col, S->colsq, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->host_k, S->colsq, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      std::memcpy(den.data(), S->host_k, sizeof(double) * k);
      for (int i = 0; i < k; i++) lam[i] = num[i] / den[i];
      std::memcpy(S->host_k, lam.data(), sizeof(double) * k);
      e = cudaMemcpyAsync(lam_d, S->host_k, sizeof(double) * k, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = launch_col_resid(X64, HX64, ldx, n, k, lam_d, S->part_col, S->colsq, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->host_k, S->colsq, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      for (int i = 0; i < k; i++) res[i] = std::sqrt(S->host_k[i] / den[i]);
    } else {
      set_error("kscf_scf_evaluate: %s", cudaGetErrorString(e));
      rc = KSCF_ERR_CUDA;
    }
  }
  release();
  if (rc) return rc;
  for (int i = 0; i < k; i++)
    if (!std::isfinite(lam[i]) || !std::isfinite(res[i])) {
      set_error("kscf_scf_evaluate: non-finite Rayleigh quotient or residual (vector %d)", i);
      return KSCF_ERR_NONFINITE;
    }
  // energies of the last step's density with the FP64 Rayleigh quotients
  std::vector<double> occ;
  double mu = 0.0, minus_ts = 0.0;
  std::vector<double> sorted = lam;
  std::sort(sorted.begin(), sorted.end());
  occupations(sorted, S->n_e, p.kT, occ, &mu, &minus_ts);
  double e_band = 0.0;
  for (int i = 0; i < k; i++) e_band += occ[i] * sorted[i];
  *report = S->last;
  report->e_band = e_band;
  report->e_total = e_band - h3 * S->sums[1] + 0.5 * h3 * S->sums[2] + h3 * S->sums[3] + minus_ts;
  report->homo = sorted[S->n_occ - 1];
  report->lumo = sorted[S->n_occ];
  report->mu = mu;
  report->minus_ts = minus_ts;
  report->occ_last = occ[k - 1];
  if (eigvals_host) std::memcpy(eigvals_host, lam.data(), sizeof(double) * k);
  if (resid_host) std::memcpy(resid_host, res.data(), sizeof(double) * k);
  return KSCF_OK;
}

extern "C" int kscf_scf_refine(kscf_scf* scf, int max_iters, double resid_tol, kscf_scf_report* report,
                               double* eigvals_host, double* resid_host, int* iters_done) {
  if (!scf || !report || max_iters < 0 || !(resid_tol > 0.0)) {
    set_error("kscf_scf_refine: invalid argument");
    return KSCF_ERR_INVALID;
  }
  kscf_scf* S = scf;
  if (!S->stepped) {
    set_error("kscf_scf_refine: call kscf_scf_step first");
    return KSCF_ERR_INVALID;
  }
  const kscf_scf_params& p = S->p;
  const int k = p.k;
  cudaStream_t st = S->st;
  // wanted states: the occupied ones (occupation above 1e-12) and the first empty one
  std::vector<double> occ;
  double mu = 0.0, minus_ts = 0.0;
  int rc = kscf_set_potential(S->ham, S->v_in, st);
  if (rc) return rc;
  KSCF_CUDA_TRY(cudaStreamSynchronize(st));
  double lower = 0.0, upper = 0.0;
  rc = kscf_spectral_bounds(S->ham, &lower, &upper);
  if (rc) return rc;
  std::vector<double> lam(k), res(k);
  kscf_scf_report tmp;
  double best = 0.0;
  int stall = 0, it = 0;
  for (; it < max_iters; it++) {
    rc = eig_step(S, true, upper);
    if (rc) return rc;
    rc = kscf_scf_evaluate(S, &tmp, lam.data(), res.data());   // FP64 residuals of the current vectors
    if (rc) return rc;
    occupations(S->lam, S->n_e, p.kT, occ, &mu, &minus_ts);
    int n_want = 0;
    while (n_want < k && occ[n_want] > 1e-12) n_want++;
    n_want = std::min(k, n_want + 1);
    double worst = 0.0;
    for (int i = 0; i < n_want; i++) worst = std::max(worst, res[i]);
    if (worst < resid_tol) {
      it++;
      break;
    }
    // stop once the residuals no longer fall (the working precision's floor)
    if (it == 0 || worst < 0.9 * best) {
      best = worst;
      stall = 0;
    } else if (++stall >= 3) {
      it++;
      break;
    }
  }
  if (iters_done) *iters_done = it;
  rc = kscf_check_status();
  if (rc) return rc;
  // density, potentials and energy integrals of the refined vectors at the same V_in
  kscf_scf_report r;
  std::memset(&r, 0, sizeof(r));
  r.step = S->step;
  rc = density_energy(S, &r);
  if (rc) return rc;
  r.converged = S->last.converged;
  r.chefsi_iters = it;
  r.upper_bound = upper;
  S->last = r;
  return kscf_scf_evaluate(S, report, eigvals_host, resid_host);
}

extern "C" int kscf_scf_get(const kscf_scf* scf, int field, double* dst) {
  if (!scf || !dst) {
    set_error("kscf_scf_get: null argument");
    return KSCF_ERR_INVALID;
  }
  const double* src = nullptr;
  switch (field) {
    case KSCF_FIELD_RHO: src = scf->rho; break;
    case KSCF_FIELD_V_IN: src = scf->v_in; break;
    case KSCF_FIELD_V_H: src = scf->vh; break;
    case KSCF_FIELD_V_XC: src = scf->vxc; break;
    case KSCF_FIELD_V_ION: src = scf->v_ion; break;
    case KSCF_FIELD_V_START: src = scf->v_start; break;
    case KSCF_FIELD_EPS_XC: src = scf->eps; break;
    default:
      set_error("kscf_scf_get: unknown field %d", field);
      return KSCF_ERR_INVALID;
  }
  KSCF_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double) * scf->n, cudaMemcpyDeviceToDevice, scf->st));
  return KSCF_OK;
}

extern "C" int kscf_mlp_training_data(const kscf_scf* scf, const float* D_slots, float* D_out, float* t_out) {
  if (!scf || !D_slots || !D_out || !t_out) {
    set_error("kscf_mlp_training_data: null argument");
    return KSCF_ERR_INVALID;
  }
  KSCF_CUDA_TRY(launch_training_rows(scf->ham->h, D_slots, scf->v_in, scf->v_start, D_out, t_out, scf->st));
  return KSCF_OK;
}
