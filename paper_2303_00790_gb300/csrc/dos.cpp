// Density of states and HOMO-LUMO gap from Ritz values (arXiv 2303.00790, the DOS
// paragraph and Fig. 1: histogram of the eigenvalues in 0.1 eV bins with the highest
// occupied state at zero, every DOS scaled to the same area below the Fermi level;
// band gap = HOMO-LUMO gap, Fig. 3).  Host-only post-processing of k values.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kscf_internal.h"

// CODATA 2018 Hartree energy in eV
static const double kHartreeEv = 27.211386245988;

extern "C" int kscf_dos(const double* eigvals, int k, int n_occ, double bin_ev, double e_lo_ev, int n_bins,
                        double* hist, double* gap_ev) {
  if (!eigvals || !hist || k < 1 || n_occ < 1 || n_occ > k || !(bin_ev > 0.0) || n_bins < 1 ||
      !std::isfinite(e_lo_ev)) {
    kscf::set_error("kscf_dos: invalid argument");
    return KSCF_ERR_INVALID;
  }
  // HOMO = the n_occ-th smallest value (input need not be sorted)
  std::vector<double> v(eigvals, eigvals + k);
  for (double x : v)
    if (!std::isfinite(x)) {
      kscf::set_error("kscf_dos: non-finite eigenvalue");
      return KSCF_ERR_NONFINITE;
    }
  std::vector<double> s = v;
  std::sort(s.begin(), s.end());
  const double homo = s[n_occ - 1];
  if (gap_ev) *gap_ev = n_occ < k ? (s[n_occ] - homo) * kHartreeEv : NAN;
  for (int b = 0; b < n_bins; b++) hist[b] = 0.0;
  // area below the Fermi level = n_occ states: each state adds 1 / (n_occ * bin) so that
  // the occupied states integrate to one
  const double w = 1.0 / ((double)n_occ * bin_ev);
  for (int i = 0; i < k; i++) {
    const double e = (v[i] - homo) * kHartreeEv;
    const double t = std::floor((e - e_lo_ev) / bin_ev);
    if (t < 0.0 || t >= (double)n_bins) continue;
    hist[(int)t] += w;
  }
  return KSCF_OK;
}
