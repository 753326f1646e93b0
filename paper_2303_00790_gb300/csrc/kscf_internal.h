// Internal structures shared by the translation units of libkscf.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/kscf.h"

namespace kscf {

// thread-local error message
void set_error(const char* fmt, ...);
// counts kernel launches made by this library (all threads)
void count_launch();

struct Grid {
  double h = 0.0;
  double center[3] = {0, 0, 0};
  int B = 8;                       // brick edge
  int lo[3] = {0, 0, 0};           // smallest (i,j,k)
  int ext[3] = {0, 0, 0};          // bounding-box extent in points
  int nb[3] = {0, 0, 0};           // bricks per axis over the bounding box
  int64_t n_points = 0, n_bricks = 0, n_slots = 0;
  std::vector<int32_t> brick_xyz;     // 3 per kept brick (brick coordinates)
  std::vector<int32_t> brick_of_box;  // nb0*nb1*nb2 -> brick rank or -1
  std::vector<int32_t> nbr;           // 6 per brick: -x,+x,-y,+y,-z,+z ranks or -1
  std::vector<int64_t> lex_of_slot;   // n_slots, -1 for padding
  std::vector<uint8_t> mask;          // n_slots, 1 inside the domain

  // slot of integer point (i,j,k) or -1 when outside the bounding box / dropped brick
  int64_t slot_of(int i, int j, int k) const {
    int x = i - lo[0], y = j - lo[1], z = k - lo[2];
    if (x < 0 || y < 0 || z < 0 || x >= nb[0] * B || y >= nb[1] * B || z >= nb[2] * B) return -1;
    int bx = x / B, by = y / B, bz = z / B;
    int32_t r = brick_of_box[((int64_t)bz * nb[1] + by) * nb[0] + bx];
    if (r < 0) return -1;
    return (int64_t)r * B * B * B + ((int64_t)(z - bz * B) * B + (y - by * B)) * B + (x - bx * B);
  }
  void slot_ijk(int64_t s, int* ijk) const {
    int64_t r = s / ((int64_t)B * B * B);
    int li = (int)(s % ((int64_t)B * B * B));
    ijk[0] = lo[0] + brick_xyz[3 * r + 0] * B + li % B;
    ijk[1] = lo[1] + brick_xyz[3 * r + 1] * B + (li / B) % B;
    ijk[2] = lo[2] + brick_xyz[3 * r + 2] * B + li / (B * B);
  }
};

// Device-side tables of the Hamiltonian.
struct Ham {
  Grid grid;                       // host copy of the grid tables
  int M = 6;
  double stencil[7];               // -1/2 h^-2 w_k (k = 0..6); the centre uses 3*stencil[0]
  int device = 0;
  // device arrays
  int32_t* d_nbr = nullptr;        // n_bricks*6
  uint8_t* d_mask = nullptr;       // n_slots
  int64_t* d_lex = nullptr;        // n_slots
  int64_t* d_pad = nullptr;        // padding slots
  int64_t n_pad = 0;
  int32_t* d_live = nullptr;       // domain slots in slot order (n_live = number of grid points)
  int64_t n_live = 0;
  double* d_v64 = nullptr;         // n_slots
  double* d_vion = nullptr;        // n_slots: V_loc as built (kept when the potential is replaced)
  float* d_v32 = nullptr;          // n_slots
  // KB tables
  int n_kb = 0;                    // atoms with projectors
  int64_t n_kb_entries = 0;
  int64_t* d_kb_atom_ptr = nullptr;   // n_kb+1, entries per atom
  int64_t* d_kb_atom_slot = nullptr;  // entry -> slot
  double* d_kb_atom_chi64 = nullptr;  // entry*4
  float* d_kb_atom_chi32 = nullptr;
  int64_t* d_kb_slot_ptr = nullptr;   // n_slots+1, entries per slot
  int32_t* d_kb_slot_atom = nullptr;  // entry -> kb atom
  double* d_kb_slot_chi64 = nullptr;  // entry*4
  float* d_kb_slot_chi32 = nullptr;
  uint16_t* d_kb_entry_lslot = nullptr;  // entry -> slot index inside its brick (slot order)
  double* d_kb_energy = nullptr;      // n_kb*4: E_l * h^3
  double kb_upper = 0.0, kb_lower = 0.0;  // Gershgorin bounds of V_NL
  int max_slot_entries = 0;
  // Cells of the chunk-major FP32 filter (bricks of 8^3 or 16^3, null otherwise): cubes of
  // 8^3 points, the brick itself for 8^3 bricks, the eight octants of a 16^3 brick
  // (cell = brick * 8 + ox + 2 oy + 4 oz).  Cell-local point r = x + 8 y + 64 z.
  int64_t n_cells = 0;
  int32_t* d_cell_nbr = nullptr;       // n_cells * 6: face neighbour cells (-x, +x, -y, +y, -z, +z), -1: none
  // per cell and line pass (x, y, z) the lines holding at least one domain point,
  // compacted (line = a + 8 b for the pass's two other axes)
  uint8_t* d_lines = nullptr;          // n_cells * 3 * 64
  uint8_t* d_nlines = nullptr;         // n_cells * 3
  // the KB entries in cell order (cell, then cell-local point): CSR over the n_cells * 512
  // cell-local points, chi (4 per entry) and atom; for 8^3 bricks these are the slot-order
  // tables above (cell_tables_own false)
  int64_t* d_cell_kb_ptr = nullptr;    // n_cells * 512 + 1
  float* d_cell_kb_chi32 = nullptr;    // entry * 4
  int32_t* d_cell_kb_atom = nullptr;   // entry -> kb atom
  bool cell_tables_own = false;
  // per cell the KB atoms whose projectors reach into it (kb atom ids, at most
  // KSCF_BRICK_ATOMS; brick_atoms_ok false when a cell has more), and per entry (cell
  // order) the packed word  cell-local point | (index in its cell's atom list << 16)
  int32_t* d_brick_atoms = nullptr;    // n_cells * KSCF_BRICK_ATOMS, -1 padded
  int32_t* d_brick_natoms = nullptr;   // n_cells
  uint32_t* d_kb_entry_word = nullptr;  // n_kb_entries
  bool brick_atoms_ok = false;
};
constexpr int KSCF_BRICK_ATOMS = 32;

// ---- launchers (filter.cu) ----
cudaError_t launch_zero_rows(const Ham& H, void* X, int64_t ld, int k, int dtype, cudaStream_t st);
// coef rows have stride cld (>= w); coef_ld(w) = round_up32(w) lets the FP32 brick kernel
// read whole 32-vector chunks
cudaError_t launch_kb_gather(const Ham& H, const void* Y, int64_t ld, int w, int dtype, void* coef,
                             int64_t cld, cudaStream_t st);
// The FP32 brick kernels do not write padding rows of `out`: callers keep padding rows
// zero in every buffer they pass (launch_zero_rows once per buffer).
// wavail: columns readable and writable from in/prev/out in every row (>= w); the FP32
// brick kernel is used when wavail and cld cover round_up8(w) (32-vector CTAs when they
// cover round_up32(w))
cudaError_t launch_cheb_step(const Ham& H, const void* in, int64_t ld_in, const void* prev,
                             int64_t ld_prev, void* out, int64_t ld_out, int w, int wavail, int dtype,
                             double alpha, double beta, double c, const void* coef, int64_t cld,
                             cudaStream_t st);
inline int64_t coef_ld(int w) { return (int64_t)(w + 31) / 32 * 32; }

// ---- chunk-major filter path (filter_cm.cu, FP32, 8^3 and 16^3 bricks) ----
// Working copies of a column block are chunk-major: element (c, s, v) at
// buf[(c * n_slots + s) * cw + v], cw = cm_chunk_width().
int cm_chunk_width();
// buf = chunk-major copy of the block (padded columns zero); padding rows of buf2 zeroed
cudaError_t launch_to_chunk_major(const Ham& H, const float* X, int64_t ld, int w, int cw, float* buf, float* buf2,
                                  cudaStream_t st);
// coef rows of stride cld; columns w <= v < cld are written as zero
cudaError_t launch_kb_gather_cm(const Ham& H, const float* Y, int cw, int w, float* coef, int64_t cld,
                                cudaStream_t st);
// in: chunk-major; prev: chunk-major or null; out: chunk-major (out_ld < 0) or a slot-major
// block with row stride out_ld (padding rows untouched).  check: flag NaN/Inf outputs.
// zero: KSCF_CM_ZERO_BYTES of zeros, 256-aligned (the halo rows of missing neighbour bricks)
cudaError_t launch_cm_step(const Ham& H, const float* in, const float* prev, float* out, int64_t out_ld, int w,
                           double alpha, double beta, double c, const float* coef, int64_t cld, bool check,
                           const float* zero, cudaStream_t st);
constexpr size_t KSCF_CM_ZERO_BYTES = 4096 * 16 * 4;   // one 16^3 brick x 16 vectors
// device address of the non-finite flag that kscf_check_status reports
unsigned int* nonfinite_flag();
// sets *flag when a domain row of X holds a NaN or Inf in its first k values
cudaError_t launch_finite_rows(const Ham& H, const void* X, int64_t ld, int k, int dtype, unsigned int* flag,
                               cudaStream_t st);
// *status = 1 if a diagonal element of S is NaN or Inf, else 0
cudaError_t launch_diag_finite(const double* S, int k, int64_t lds, int* status, cudaStream_t st);
// *out = max_ij |S_ij - delta_ij| as the bits of a non-negative double (NaN or Inf: +Inf)
cudaError_t launch_dev_identity(const double* S, int k, int64_t lds, unsigned long long* out, cudaStream_t st);
// S <- (3 I - S) / 2 in place: the first-order inverse square root of S = I + E
cudaError_t launch_polar_first_order(double* S, int k, int64_t lds, cudaStream_t st);
// device status words of the chunk-major path: a timed-out wait, non-finite output
cudaError_t cm_status(bool reset, unsigned int* timeout, unsigned int* nonfinite);
cudaError_t launch_copy_cols(const void* src, int64_t ld_src, void* dst, int64_t ld_dst, int64_t rows,
                             int w, int dtype, cudaStream_t st);

// ---- launchers (setup.cu) ----
cudaError_t launch_vloc(const Ham& H, const double* d_xyz /*n_slots*3*/, const double* d_atoms /*n*8*/,
                        int n_atoms, cudaStream_t st);
cudaError_t launch_v_to_f32(const Ham& H, cudaStream_t st);
cudaError_t launch_random(const Ham& H, void* X, int64_t ld, int k, int dtype, uint64_t seed,
                          cudaStream_t st);
// to_slots: dst (slot layout) row s = src row lex(s), padding rows zero; else dst row
// lex(s) = src row s for the live slots
cudaError_t launch_points_slots(const Ham& H, bool to_slots, const void* src, int64_t lds, void* dst, int64_t ldd,
                                int k, int dtype, cudaStream_t st);
cudaError_t launch_density(const Ham& H, const void* X, int64_t ld, int n_occ, int dtype,
                           const double* occ, double* rho, cudaStream_t st);
cudaError_t launch_minmax_v(const Ham& H, double* d_out2, cudaStream_t st);
cudaError_t launch_mask_v(const Ham& H, const double* src, double* dst, cudaStream_t st);

// ---- launchers (gemm.cu) ----
// C[i + j*ldc] (+)= scale * sum_r A[r*lda + i] * B[r*ldb + j], i < m, j < n, r < rows.
cudaError_t launch_gram_native(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t rows,
                               int m, int n, int dtype, double scale, double* C, int64_t ldc,
                               bool accumulate, cudaStream_t st);
// out[r*ldo + j] = sum_i A[r*lda + i] * Q[i + j*ldq]  (Q column-major, dtype of A)
cudaError_t launch_rotate_native(const void* A, int64_t lda, const void* Q, int64_t ldq, int64_t rows,
                                 int kin, int kout, int dtype, void* out, int64_t ldo, cudaStream_t st);
cudaError_t launch_symmetrize(double* C, int k, int64_t ldc, cudaStream_t st);
// S[i][i] += rel * max_i S[i][i]
cudaError_t launch_shift_diag(double* S, int k, double rel, cudaStream_t st);
// negate the columns of Q (column-major k x k) whose diagonal element is negative
cudaError_t launch_sign_fix(double* Q, int k, cudaStream_t st);
cudaError_t launch_upper_to_dtype(const double* R, int k, int dtype, void* out, cudaStream_t st);
// S (k x k column-major, upper triangle read) = R^T R; out (may alias S) = R^-1, upper
// triangular with zeros below.  status (2 device ints, zeroed here): [0] = 1-based column
// of the first pivot not above S_cc max((c + 8) 2^-53, floor_rel) (out then unwritten),
// [1] = 1 if a bounded grid barrier gave up (each wait gives up after spin_limit clock
// cycles, ~1 s by default).  work: chol_inv_work_bytes(k), 256-aligned.  leave_cta >= 0
// (self-test only) makes that CTA return before its first barrier.
size_t chol_inv_work_bytes(int k);
cudaError_t launch_chol_inv(const double* S, int64_t lds, int k, double floor_rel, double* out, int64_t ldo,
                            void* work, int* status, cudaStream_t st, long long spin_limit = 2000000000LL,
                            int leave_cta = -1);
// FP64 symmetric eigensolver (eig.cu): A (n x n column-major, lda; the symmetric part
// (A + A^T) / 2 is diagonalised) is overwritten by the orthonormal eigenvectors, column j
// for w[j] (device, ascending).  info (4 device ints, zeroed here): [0] = 1 if a bounded
// grid barrier gave up, [1] = secular roots that did not converge, [2] = 1 if A held a
// NaN or Inf.  work: sym_eig_work_bytes(n), 256-aligned.  n <= KSCF_EIG_MAX_N.
constexpr int KSCF_EIG_MAX_N = 8192;
size_t sym_eig_work_bytes(int n);
// leave_cta >= 0 (self-test only): that CTA of the tridiagonalisation returns at its first
// grid barrier, so that the others' bounded waits run out.
cudaError_t launch_sym_eig(double* A, int64_t lda, int n, double* w, void* work, size_t work_bytes, int* info,
                           cudaStream_t st, long long spin_limit = 2000000000LL, int leave_cta = -1);
cudaError_t launch_f64_to_dtype(const double* src, int64_t n, int dtype, void* out, cudaStream_t st);

}  // namespace kscf

struct kscf_grid {
  kscf::Grid g;
};
struct kscf_ham {
  kscf::Ham h;
};

#define KSCF_CUDA_TRY(expr)                                                         \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      kscf::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),      \
                      __FILE__, __LINE__);                                          \
      return KSCF_ERR_CUDA;                                                         \
    }                                                                               \
  } while (0)

inline size_t kscf_align256(size_t x) { return (x + 255) & ~(size_t)255; }
