// Lanczos estimate of the spectral bounds of H (the filter interval of CheFSI; the
// estimate of Zhou & Li 2011 used for the Chebyshev filter by Zhou, Saad, Tiago &
// Chelikowsky 2006):  v_1 = x/|x|, w = H v_j - beta_{j-1} v_{j-1}, alpha_j = <v_j, w>,
// w -= alpha_j v_j, beta_j = |w|, v_{j+1} = w/beta_j; upper = theta_max(T_K) + beta_K,
// lower estimate = theta_min(T_K).  FP64 on the device, h^3-weighted inner products;
// the eigenvalues of the K x K tridiagonal T by Sturm-sequence bisection on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kscf_internal.h"
#include "scf_internal.h"

using namespace kscf;

namespace {

// number of eigenvalues of tridiag(b; a; b) below x
int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int count = 0;
  double d = 1.0;
  for (size_t j = 0; j < a.size(); j++) {
    d = a[j] - x - (j > 0 ? b[j - 1] * b[j - 1] / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) count++;
  }
  return count;
}

// i-th smallest eigenvalue by bisection
double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int i) {
  const size_t n = a.size();
  double lo = 0.0, hi = 0.0;
  for (size_t j = 0; j < n; j++) {
    const double r = (j > 0 ? std::fabs(b[j - 1]) : 0.0) + (j + 1 < n ? std::fabs(b[j]) : 0.0);
    lo = j ? std::min(lo, a[j] - r) : a[j] - r;
    hi = j ? std::max(hi, a[j] + r) : a[j] + r;
  }
  lo -= 1.0;
  hi += 1.0;
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(a, b, mid) > i)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

extern "C" int kscf_lanczos_bounds(const kscf_ham* ham, int steps, uint64_t seed, double* upper, double* theta_max,
                                   double* theta_min, double* alpha_out, double* beta_out, void* stream) {
  if (!ham || steps < 1 || steps > 1000 || !upper) {
    set_error("kscf_lanczos_bounds: invalid argument");
    return KSCF_ERR_INVALID;
  }
  const Ham& H = ham->h;
  const int64_t n = H.grid.n_slots;
  const double h3 = H.grid.h * H.grid.h * H.grid.h;
  cudaStream_t st = (cudaStream_t)stream;
  size_t wb = 0;
  int rc = kscf_workspace_size(ham, KSCF_OP_APPLY, 1, KSCF_F64, 0, 0, &wb);
  if (rc) return rc;
  double *v = nullptr, *vp = nullptr, *w = nullptr, *zero = nullptr, *part = nullptr, *res = nullptr, *host = nullptr;
  void* work = nullptr;
  cudaError_t e = cudaMalloc((void**)&v, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&vp, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&w, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&zero, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&part, sizeof(double) * kScfRedBlocks);
  if (e == cudaSuccess) e = cudaMalloc((void**)&res, sizeof(double) * 2);
  if (e == cudaSuccess) e = cudaMalloc(&work, std::max<size_t>(wb, 256));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&host, sizeof(double) * 2);
  std::vector<double> a(steps), b(steps);
  auto dot = [&](const double* x, const double* y, double* out) -> cudaError_t {
    cudaError_t ee = launch_col_dot(x, 1, y, 1, n, 1, KSCF_F64, part, res, st);
    if (ee == cudaSuccess) ee = cudaMemcpyAsync(host, res, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
    if (ee == cudaSuccess) *out = h3 * host[0];
    return ee;
  };
  if (e == cudaSuccess) e = cudaMemsetAsync(zero, 0, sizeof(double) * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(vp, 0, sizeof(double) * n, st);
  if (e == cudaSuccess) {
    rc = kscf_random_subspace(ham, v, 1, 1, KSCF_F64, seed, st);
    double nrm = 0.0;
    if (!rc) e = dot(v, v, &nrm);
    if (!rc && e == cudaSuccess) e = launch_lincomb(H, zero, v, 1.0 / std::sqrt(nrm), v, st);
    double beta_prev = 0.0;
    for (int j = 0; j < steps && !rc && e == cudaSuccess; j++) {
      rc = kscf_hamiltonian_apply(ham, v, 1, w, 1, 1, KSCF_F64, work, std::max<size_t>(wb, 256), st);
      if (rc) break;
      e = launch_lincomb(H, w, vp, -beta_prev, w, st);
      if (e == cudaSuccess) e = dot(v, w, &a[j]);
      if (e == cudaSuccess) e = launch_lincomb(H, w, v, -a[j], w, st);
      double bb = 0.0;
      if (e == cudaSuccess) e = dot(w, w, &bb);
      b[j] = std::sqrt(std::max(bb, 0.0));
      if (e == cudaSuccess && b[j] > 0.0) {
        std::swap(v, vp);                                      // vp <- v_j
        e = launch_lincomb(H, zero, w, 1.0 / b[j], v, st);     // v <- w / beta_j
      }
      beta_prev = b[j];
      if (b[j] == 0.0) {  // invariant subspace found: T is complete
        a.resize(j + 1);
        b.resize(j + 1);
        break;
      }
    }
  }
  cudaFree(v);
  cudaFree(vp);
  cudaFree(w);
  cudaFree(zero);
  cudaFree(part);
  cudaFree(res);
  cudaFree(work);
  if (host) cudaFreeHost(host);
  if (rc) return rc;
  if (e != cudaSuccess) {
    set_error("kscf_lanczos_bounds: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  const int K = (int)a.size();
  std::vector<double> off(b.begin(), b.begin() + (K - 1));
  const double tmax = tridiag_eig(a, off, K - 1), tmin = tridiag_eig(a, off, 0);
  *upper = tmax + b[K - 1];
  if (theta_max) *theta_max = tmax;
  if (theta_min) *theta_min = tmin;
  for (int j = 0; j < K; j++) {
    if (alpha_out) alpha_out[j] = a[j];
    if (beta_out) beta_out[j] = b[j];
  }
  return KSCF_OK;
}
