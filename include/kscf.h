/*
 * kscf.h -- C ABI of the GB300 (sm_103a) CheFSI hot path for real-space Kohn-Sham DFT.
 *
 * Method: Chebyshev-filtered subspace iteration (CheFSI) on a high-order
 * finite-difference Hamiltonian over a spherical Dirichlet grid whose points are
 * stored in blockwise Hilbert space-filling-curve order (arXiv 2303.00790: Abstract;
 * CheFSI paragraph before Table I; SFC paragraph after Table I; Computational details).
 *
 * Conventions for every entry point
 *   - Return value: KSCF_OK (0) or a negative KSCF_ERR_* code; kscf_last_error()
 *     returns a thread-local message describing the last failure on this thread.
 *   - Units: Hartree atomic units (bohr, Hartree).
 *   - Handles (kscf_grid, kscf_ham) are owned by the library; free them with the
 *     matching *_free call.  A kscf_ham keeps a reference to device memory only, not to
 *     the kscf_grid, so the grid may be freed after kscf_build_hamiltonian.
 *   - Device arrays (X, rho, work, ...) are owned by the caller.  `stream` is a
 *     cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *     asynchronous on `stream` unless stated otherwise.
 *   - Wavefunction blocks X are "slot-major": row s (0 <= s < n_slots) holds the k
 *     vector values of grid slot s contiguously, row stride `ld` elements (ld >= k).
 *     Slots are brick_rank * b^3 + (lz*b + ly)*b + lx with bricks in Hilbert order.
 *     Rows of slots outside the domain (padding of boundary bricks) are zero on
 *     output; the library zeroes them on input where a stencil reads them.
 *   - dtype: KSCF_F64 (double) or KSCF_F32 (float) for X and the filter arithmetic.
 *     For F32 X a row stride ld that is a multiple of 32 (16-byte aligned rows) lets
 *     every column block of the filter run on the fastest (32-vector brick) kernel; any
 *     ld >= k is accepted.
 *   - Inner products use the grid weight h^3: <u, v> = h^3 sum_s u_s v_s.
 *   - Device work buffers must be at least the size kscf_workspace_size() reports for
 *     the same (op, k, dtype, mode, block); a smaller buffer gives KSCF_ERR_WORKSPACE
 *     before any launch.  Work buffers must be 256-byte aligned.
 */
#ifndef KSCF_H
#define KSCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define KSCF_OK               0
#define KSCF_ERR_INVALID     -1   /* bad argument (null pointer, size, bounds, dtype) */
#define KSCF_ERR_CUDA        -2   /* a CUDA runtime call failed */
#define KSCF_ERR_WORKSPACE   -3   /* work buffer smaller than kscf_workspace_size */
#define KSCF_ERR_NOT_SPD     -4   /* Gram matrix not positive definite (rank-deficient X) */
#define KSCF_ERR_NONFINITE   -5   /* NaN/Inf found in an input or result */
#define KSCF_ERR_NO_CONVERGE -6   /* dense eigensolver did not converge */
#define KSCF_ERR_UNSUPPORTED -7   /* combination not built (e.g. bf16 mode with F64 X) */
#define KSCF_ERR_HOST_ALLOC  -8   /* host memory allocation failed */
#define KSCF_ERR_TIMEOUT     -9   /* a bounded device-side wait gave up (kernel returned early) */

/* ---- element types ---- */
#define KSCF_F64 0
#define KSCF_F32 1

/* ---- Gram / projection GEMM modes (orthonormalize, rayleigh_ritz) ---- */
#define KSCF_GEMM_NATIVE 0   /* CUDA-core GEMM in the dtype of X; FP32 X: FP32 products with FP64
                                sums of partial sums over at most 256 rows */
#define KSCF_GEMM_TENSOR 1   /* tensor cores (tcgen05), F32 X only: every FP32 operand is split into
                                three bf16 pieces x = x1 + x2 + x3 and the six products x1y1, x1y2,
                                x2y1, x1y3, x2y2, x3y1 are accumulated in FP32 over chunks of rows,
                                chunk sums added in FP64 */

/* ---- operations for kscf_workspace_size ---- */
#define KSCF_OP_APPLY   0
#define KSCF_OP_FILTER  1
#define KSCF_OP_ORTHO   2
#define KSCF_OP_RR      3

typedef struct kscf_grid kscf_grid;
typedef struct kscf_ham kscf_ham;

/* An atom: position (bohr) and element number (14 = Si, 1 = H, ...). */
typedef struct kscf_atom {
  double x, y, z;
  int32_t z_number;
  int32_t reserved;
} kscf_atom;

/* Synthetic pseudopotential of one element (stand-in for the paper's norm-conserving
 * Troullier-Martins potentials in Kleinman-Bylander form, Computational details):
 *   local     v(r) = -z_valence erf(r/r_c)/r + a_gauss exp(-r^2/r_gauss^2)
 *             (v(0) = -2 z_valence/(r_c sqrt(pi)) + a_gauss)
 *   projectors (n_proj = 4): s = exp(-r^2/(2 r_p^2)), p_m = (x_m/r_p) exp(-r^2/(2 r_p^2)),
 *             zero beyond r_cut; energies e_s (s) and e_p (p_x, p_y, p_z).
 *   n_proj = 0 means no nonlocal part. */
typedef struct kscf_species {
  int32_t z_number;
  int32_t n_proj;      /* 0 or 4 */
  double z_valence, r_c, a_gauss, r_gauss;
  double e_s, e_p, r_p, r_cut;
} kscf_species;

typedef struct kscf_grid_info {
  int64_t n_points;    /* grid points inside the domain */
  int64_t n_slots;     /* rows of X = n_bricks * brick^3 */
  int64_t n_bricks;
  int32_t brick;       /* brick edge b (8 or 16) */
  int32_t lo[3];       /* smallest (i, j, k) over the domain */
  int32_t extent[3];   /* bounding-box extent in points */
  int32_t reserved;
  double h;            /* grid spacing (bohr) */
  double center[3];    /* grid point (0,0,0) position (bohr) */
} kscf_grid_info;

/* Thread-local description of the last error on this thread ("" if none). */
const char* kscf_last_error(void);

/* Number of CUDA kernels this library has launched since it was loaded (all threads;
 * every kernel of the path is the library's own).  For launch accounting. */
uint64_t kscf_launch_counter(void);

/* ---------------------------------------------------------------------------------
 * Grid (host only).  Spherical domain: points center + h*(i,j,k) with
 * i^2 + j^2 + k^2 <= radius^2/h^2 + 1e-9 (zero Dirichlet outside; the paper treats
 * aperiodic clusters without a supercell, Intro).  Points are grouped into b^3
 * bricks of the bounding box; bricks holding no point are dropped; the kept bricks
 * are ordered along a 3D Hilbert curve of their brick coordinates (blockwise Hilbert
 * SFC ordering, SFC paragraph after Table I), points inside a brick in x-fastest
 * order.  brick must be 8 or 16.  *out receives a new handle. */
int kscf_build_grid(const double center[3], double radius, double h, int brick, kscf_grid** out);

/* Box domain 0 <= i < nx, 0 <= j < ny, 0 <= k < nz (closed-form tests).  Same layout. */
int kscf_build_grid_box(int nx, int ny, int nz, double h, int brick, kscf_grid** out);

int kscf_grid_get_info(const kscf_grid* grid, kscf_grid_info* info);

/* Copies the slot tables to caller host arrays (either may be NULL):
 *   lex_of_slot[n_slots]   lexicographic index (k slowest, i fastest) of the point in
 *                          each slot, -1 for padding slots;
 *   ijk_of_slot[3*n_slots] integer coordinates (i, j, k) of each slot (padding slots
 *                          hold the coordinates they would have). */
int kscf_grid_slots(const kscf_grid* grid, int64_t* lex_of_slot, int32_t* ijk_of_slot);

int kscf_grid_free(kscf_grid* grid);

/* ---------------------------------------------------------------------------------
 * Hamiltonian H = -1/2 Lap_h + V_loc + V_NL at fixed potential (Intro: high-order
 * finite differences in real space; Computational details: KB pseudopotentials).
 * Lap_h: order-12 central differences, 6 neighbours per side along each axis.
 * V_loc(p) = sum over all atoms of the species' local term (no truncation).
 * V_NL y = sum_i chi_i E_i h^3 <chi_i, y> over the atoms' projectors.
 * Builds the tables on the host, evaluates V_loc on the current CUDA device and
 * uploads everything; synchronous.  atoms/species are read only during the call. */
int kscf_build_hamiltonian(const kscf_grid* grid, const kscf_atom* atoms, int n_atoms,
                           const kscf_species* species, int n_species, kscf_ham** out);

int kscf_ham_free(kscf_ham* ham);

/* Copies the grid info of the grid the Hamiltonian was built on. */
int kscf_ham_grid_info(const kscf_ham* ham, kscf_grid_info* info);

/* Replace V_loc by v_slots (device, n_slots doubles, slot order; padding entries are
 * ignored).  Used for self-consistent updates and special potentials. */
int kscf_set_potential(kscf_ham* ham, const double* v_slots, void* stream);

/* Copy V_loc (device, n_slots doubles, zero in padding slots) to v_slots. */
int kscf_get_potential(const kscf_ham* ham, double* v_slots, void* stream);

/* Bounds of the spectrum (host doubles; synchronous):
 *   upper = 3/(2h^2) (|w_0| + 2 sum_k |w_k|) + max V_loc
 *           + max_i sum_j sqrt(E+_i E+_j) h^3 |<chi_i, chi_j>|   (Weyl + Gershgorin)
 *   lower = min V_loc - max_i sum_j sqrt(E-_i E-_j) h^3 |<chi_i, chi_j>|
 * with E+ = max(E, 0), E- = max(-E, 0).  upper is the filter's upper bound b. */
int kscf_spectral_bounds(const kscf_ham* ham, double* lower, double* upper);

/* Lanczos estimate of the spectral bounds (the filter interval; Zhou & Li 2011): `steps`
 * (K) Lanczos steps in FP64 from the unit vector of kscf_random_subspace(seed, k = 1),
 * inner products h^3-weighted; T_K = tridiag(beta; alpha; beta).  upper = theta_max(T_K)
 * + beta_K (a safe upper bound in practice), theta_max/theta_min: extreme Ritz values
 * (lower estimate of the spectrum), alpha_out/beta_out: K values each (host, may be NULL;
 * fewer when an invariant subspace ends the recurrence early).  Synchronous; allocates
 * five n_slots FP64 vectors for the call.  For the order-12 FD Hamiltonians here the
 * Weyl + Gershgorin bound of kscf_spectral_bounds is usually the tighter upper bound
 * (the kinetic term's Gershgorin radius equals the symbol maximum), so callers take the
 * minimum of the two. */
int kscf_lanczos_bounds(const kscf_ham* ham, int steps, uint64_t seed, double* upper, double* theta_max,
                        double* theta_min, double* alpha_out, double* beta_out, void* stream);

/* Bytes of device work buffer needed by `op` for k vectors of `dtype` in GEMM `mode`,
 * streaming `block` columns at a time (0 = all k). */
int kscf_workspace_size(const kscf_ham* ham, int op, int k, int dtype, int mode, int block,
                        size_t* bytes);

/* HY = H Y for k vectors (Y and HY: n_slots x k, row strides ld_y, ld_hy; must not
 * overlap).  Padding rows of Y are zeroed first. */
int kscf_hamiltonian_apply(const kscf_ham* ham, void* Y, int64_t ld_y, void* HY, int64_t ld_hy,
                           int k, int dtype, void* work, size_t work_bytes, void* stream);

/* Size in bytes of the fixed device array used by kscf_hamiltonian_apply_noalloc. */
#define KSCF_NOALLOC_SCRATCH_BYTES (4 << 20)

/* HY = H Y like kscf_hamiltonian_apply, for callers that cannot allocate device
 * memory: for example a process whose framework has reserved all device memory in
 * its own pool and forbids other allocators, or a latency-critical loop that must not
 * call cudaMalloc because it synchronises the device.  The paper has no counterpart;
 * this is a service of the library.
 *   - No work buffer: the projection coefficients live in a fixed library-owned device
 *     array of KSCF_NOALLOC_SCRATCH_BYTES bytes (held on every GPU that loads the
 *     library until the process exits).  It needs n_kb * 4 * k * sizeof(element)
 *     bytes (n_kb = atoms with projectors); larger k is rejected with
 *     KSCF_ERR_INVALID and a message giving the largest k that fits -- call it on
 *     column blocks of Y instead.
 *   - Allocates nothing and calls no allocating routine.  Every call looks up the
 *     array's device address (cudaGetSymbolAddress, with the device current), so the
 *     entry point stays usable after cudaDeviceReset or a reset of the primary context;
 *     make the first call on each device before any stream capture (the first lookup
 *     may load the library's device code).
 *   - All calls share the one array and it keeps the last call's contents; calls whose
 *     work overlaps on the GPU (different streams, or threads without ordering) race
 *     on it and give wrong results.  Serialise them (e.g. one stream).
 * Arguments and layout as kscf_hamiltonian_apply (padding rows of Y are zeroed). */
int kscf_hamiltonian_apply_noalloc(const kscf_ham* ham, void* Y, int64_t ld_y, void* HY, int64_t ld_hy,
                                   int k, int dtype, void* stream);

/* In place X <- p_m(H) X: the degree-m scaled Chebyshev filter (CheFSI paragraph;
 * Zhou, Saad, Tiago & Chelikowsky 2006).  With e = (b-a)/2, c = (b+a)/2,
 * sigma_1 = e/(a0-c), tau = 2/sigma_1:
 *   Y_1 = (sigma_1/e)(H X - c X)
 *   Y_j = (2 sigma_j/e)(H Y_{j-1} - c Y_{j-1}) - sigma_{j-1} sigma_j Y_{j-2},
 *   sigma_j = 1/(tau - sigma_{j-1}),  j = 2..m;   X <- Y_m.
 * Requires a0 < a < b, degree >= 1.  Columns are processed `block` at a time
 * (0 = all k); the result does not depend on block.  F32 on bricks of 8^3 or 16^3: each
 * block runs as two halves of whole 16-column chunks, the second on a stream the call
 * creates and releases; both halves are ordered after the work already on `stream`, and
 * the work enqueued on `stream` after the call waits for both. */
int kscf_chebyshev_filter(const kscf_ham* ham, void* X, int64_t ld, int k, int degree,
                          double a, double b, double a0, int dtype, int block,
                          void* work, size_t work_bytes, void* stream);

/* In place Cholesky-QR (orthonormalisation step of CheFSI):
 *   S = h^3 X^T X (k x k, FP64 sums), S = R^T R (FP64 Cholesky), X <- X R^-1,
 * so that h^3 X^T X = I.  For F32 X the step is repeated once (CholeskyQR2,
 * Yamamoto et al. 2015), the second rotation applied as X + X (R2^-1 - I); when the second
 * pass's Gram matrix S = I + E has max_ij |E_ij| <= 1e-4, R2^-1 is replaced by the
 * first-order inverse square root I - E/2 (no factorisation; the same span, and
 * h^3 X^T X = I + O(E^2) with E^2 below the FP32 rounding of the rotation).  Returns
 * KSCF_ERR_NOT_SPD if the Cholesky factorisation fails, i.e. a pivot c (0-based) is not
 * above (c + 8) 2^-53 S_cc (X rank-deficient to working precision); X is then left
 * unchanged.  KSCF_ERR_TIMEOUT if a bounded grid barrier of the factorisation kernel
 * gave up.
 * With mode | KSCF_ORTHO_ALLOW_SHIFT, the first factorisation also fails on a pivot not
 * above 8 u S_cc (the Gram matrix's own rounding level), and a failed first factorisation
 * is retried with the Gram diagonal raised by 16 k u max_i S_ii (u = 2^-24 for F32, 2^-53
 * for F64; shifted Cholesky-QR, Fukaya et al. 2020) and followed by one extra unshifted
 * pass: a block that
 * is rank-deficient only at its working precision then still yields an orthonormal
 * basis (its near-dependent directions filled from rounding-level components), which is
 * what subspace iteration needs; if a later pass fails, X may have been changed.
 * Synchronises on `stream` to read the factorisation status. */
#define KSCF_ORTHO_ALLOW_SHIFT 0x100
int kscf_orthonormalize(const kscf_ham* ham, void* X, int64_t ld, int k, int dtype, int mode,
                        void* work, size_t work_bytes, void* stream);

/* In place Rayleigh-Ritz (CheFSI paragraph): HX = H X, Hs = h^3 X^T (HX) symmetrised
 * (FP64 k x k; in tensor mode with HX computed in one block, only the upper-triangle
 * tiles are computed and mirrored), Hs = Q Lambda Q^T (FP64 symmetric eigensolver,
 * ascending), X <- X Q.  In tensor mode the eigenvector signs are chosen with
 * diag(Q) >= 0 and the rotation is applied as X + X (Q - I).  Requires h^3 X^T X = I on
 * entry.  HX is computed in column blocks as wide as the work buffer allows: all k columns
 * with kscf_workspace_size(..., KSCF_OP_RR, ..., block = 0), halved (multiples of 32) for a
 * smaller buffer.  eigvals_host (k doubles) receives Lambda; synchronous on `stream`. */
int kscf_rayleigh_ritz(const kscf_ham* ham, void* X, int64_t ld, int k, int dtype, int mode,
                       double* eigvals_host, void* work, size_t work_bytes, void* stream);

/* Layout conversion between a compact point-major block P (n_points rows of k values,
 * row p = the grid point with lexicographic index p, as kscf_grid_slots reports it, row
 * stride ldp >= k) and the slot layout X (n_slots rows, stride ldx >= k) that every call
 * above works on.  points_to_slots writes all n_slots rows of X (padding rows zero);
 * slots_to_points writes the n_points rows of P.  Device pointers, dtype KSCF_F64 or
 * KSCF_F32, asynchronous on `stream`.  For moving a user's block in and out of the library
 * with n_points instead of n_slots rows (the brick padding is ~30 % of the slots). */
int kscf_points_to_slots(const kscf_ham* ham, const void* P, int64_t ldp, void* X, int64_t ldx, int k, int dtype,
                         void* stream);
int kscf_slots_to_points(const kscf_ham* ham, const void* X, int64_t ldx, void* P, int64_t ldp, int k, int dtype,
                         void* stream);

/* rho[s] = sum_{i < n_occ} f_i X[s][i]^2 in FP64 (electron density of the occupied
 * states; the density evolves together with the subspace, CheFSI paragraph).  For F32 X
 * the sums run in double-float arithmetic (pairs of FP32 numbers; relative error ~1e-14)
 * and only the result is converted to FP64.
 * occ: device array of n_occ occupations, or NULL for f_i = 2 (spin-degenerate).
 * rho: device, n_slots doubles. */
int kscf_density(const kscf_ham* ham, const void* X, int64_t ld, int n_occ, int dtype,
                 const double* occ, double* rho, void* stream);

/* Initial subspace: X[s][j] = N(0,1) sample number (lex_of_slot[s] * k + j) of the
 * counter-based generator (SplitMix64 finaliser keyed by seed, Box-Muller pairs; the
 * definition is in the implementation's comments), 0 in padding rows.  The values do
 * not depend on the slot order, so any layout sees the same X0. */
int kscf_random_subspace(const kscf_ham* ham, void* X, int64_t ld, int k, int dtype,
                         uint64_t seed, void* stream);

/* ---------------------------------------------------------------------------------
 * GEMM building blocks of Cholesky-QR and Rayleigh-Ritz (exported for tests and
 * benchmarks; orthonormalize and rayleigh_ritz call the same code).
 *
 * kscf_gram: C[i + j*ldc] = scale * sum_{r < rows} A[r*lda + i] * B[r*ldb + j]
 *   (i < m, j < n; C FP64 column-major, overwritten).  A, B device arrays of dtype.
 *   mode KSCF_GEMM_TENSOR (F32 only) uses tcgen05 with split-bf16 operands (see the
 *   mode constants); KSCF_GEMM_NATIVE uses CUDA cores.  When A == B, lda == ldb and
 *   m == n, only the upper triangle is computed and mirrored.
 * kscf_rotate: out[r*ldo + j] = sum_{i < kin} A[r*lda + i] * Q'[i + j*ldq]  (r < rows,
 *   j < kout) with Q' = Q - I when minus_identity (then out += A, i.e. out = A Q
 *   evaluated as A + A (Q - I); tensor mode, kin == kout).  Q is FP64 column-major;
 *   the native mode needs ldq == kin.  In tensor mode out may be A itself (the product
 *   reads bf16 copies of A; minus_identity adds A's own element in the epilogue); in the
 *   native mode out must not overlap A.
 * Work buffers: kscf_gemm_workspace_size(op = 0 gram / 1 rotate, rows, m|kin, n|kout,
 * dtype, mode, &bytes). */
int kscf_gram(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t rows, int m, int n, int dtype,
              int mode, double scale, double* C, int64_t ldc, void* work, size_t work_bytes, void* stream);
int kscf_rotate(const void* A, int64_t lda, const double* Q, int64_t ldq, int64_t rows, int kin, int kout,
                int dtype, int mode, int minus_identity, void* out, int64_t ldo, void* work, size_t work_bytes,
                void* stream);
int kscf_gemm_workspace_size(int op, int64_t rows, int m, int n, int dtype, int mode, size_t* bytes);

/* Dense FP64 symmetric eigensolver of the Rayleigh-Ritz step (CheFSI paragraph:
 * Hs = Q Lambda Q^T, the eigenvalue problem projected onto the filtered subspace), the
 * one kscf_rayleigh_ritz calls.  A: device, n x n, column-major with leading dimension
 * lda >= n; the symmetric part (A + A^T) / 2 is diagonalised and A is overwritten by the
 * orthonormal eigenvectors (column j belongs to w[j]).  w: device, n doubles, ascending.
 * Householder tridiagonalisation, tridiagonal divide and conquer with deflation and
 * Gu-Eisenstat eigenvectors, back-transformation; everything on the device in FP64
 * (backward error O(n u max|A_ij|), u = 2^-53).  1 <= n <= 8192.
 * work: device buffer of kscf_sym_eig_work_bytes(n) bytes (about 4 n^2 doubles),
 * caller-owned, 256-byte aligned.  Synchronous on `stream`.  Errors: KSCF_ERR_NONFINITE
 * (A holds a NaN or Inf; the outputs are then those of the zero matrix),
 * KSCF_ERR_TIMEOUT (a bounded grid barrier of the tridiagonalisation gave up),
 * KSCF_ERR_NO_CONVERGE (a secular-equation root did not converge), KSCF_ERR_WORKSPACE,
 * KSCF_ERR_INVALID. */
int kscf_sym_eig_work_bytes(int n, size_t* bytes);
int kscf_sym_eig(double* A, int64_t lda, int n, double* w, void* work, size_t work_bytes, void* stream);

/* Reads and clears the device status words (synchronising):
 *   KSCF_ERR_TIMEOUT   a bounded wait of a kernel that waits on mbarriers (the tensor-core
 *                      GEMMs, the TMA filter step) gave up since the last check; the kernel
 *                      then skipped its remaining work and, for the GEMMs, freed its tensor
 *                      memory;
 *   KSCF_ERR_NONFINITE the last degree step of an FP32 filter on 8^3 bricks, or
 *                      kscf_hamiltonian_apply, stored a NaN or Inf in a domain row (a
 *                      non-finite X, Y or potential), since the last check;
 *   else KSCF_OK.  orthonormalize and rayleigh_ritz check the GEMM word themselves, and
 *   orthonormalize returns KSCF_ERR_NONFINITE when the Gram matrix of X has a non-finite
 *   diagonal; filter and apply callers check after those calls. */
int kscf_check_status(void);

/* Self-test of the bounded grid barriers of the FP64 Cholesky kernel (orthonormalize):
 * runs it on a 64 x 64 identity with a wait limit of 2e6 clock cycles (~1 ms) while one of
 * its two CTAs returns before the first barrier, so that the other CTA's wait runs out.
 * Returns KSCF_ERR_TIMEOUT when that wait gave up and the kernel returned with its timeout
 * word set (the expected outcome; the context stays usable), KSCF_OK if the kernel finished
 * without noticing, or another error code.  Allocates and frees ~70 KB of device memory;
 * synchronising. */
int kscf_selftest_barrier_timeout(void* stream);

/* The same for the grid barrier of the eigensolver's tridiagonalisation (kscf_sym_eig):
 * a 64 x 64 identity, CTA 1 of its 8 returns at the first barrier, the others' waits are
 * limited to 2e6 clock cycles.  Returns KSCF_ERR_TIMEOUT when they gave up (expected; the
 * context stays usable and the rest of the solve runs on the zeroed workspace), KSCF_OK if
 * not, or another code.  Allocates and frees ~0.3 MB of device memory; synchronising. */
int kscf_selftest_eig_barrier_timeout(void* stream);

/* ---------------------------------------------------------------------------------
 * Self-consistent field (Computational details: Kohn-Sham DFT with the LDA,
 * Ceperley-Alder correlation as parametrised by Perdew & Zunger; SCF stopped when the
 * self-consistent residual error falls below 1e-4 Ry; four CheFSI iterations in the
 * first SCF step, one in each later step).  Everything below runs on the device in
 * FP64 except the CheFSI filter/Gram arithmetic, which follows params.dtype/gemm_mode.
 *
 *   V_eff = V_ion + V_H[rho] + V_xc[rho]
 *   V_ion  the Hamiltonian's V_loc as built by kscf_build_hamiltonian
 *   V_H    -Lap_h V_H = 4 pi rho on the domain (the same order-12 Laplacian as H); the
 *          values the stencil needs outside the sphere come from the monopole, dipole
 *          and quadrupole of rho about the grid centre; conjugate gradients in FP64 until
 *          |r| < poisson_rtol |b|, warm-started from the previous V_H
 *   V_xc   Slater exchange + PZ81 correlation, unpolarised (kscf_lda_xc)
 *   rho    sum_i occ_i |x_i|^2 / (h^3 |x_i|^2_2) over the Ritz vectors (the norm is 1 up to
 *          rounding; dividing by it keeps h^3 sum rho = n_e when X is FP32), occ_i = 2 for
 *          the n_e/2 lowest states (kT = 0) or Fermi-Dirac (kT > 0; n_e = sum of z_valence)
 *   SRE    2 sqrt(h^3 sum_s rho_s (V_out - V_in)_s^2) in Ry, V_out = V_eff[rho_out]
 *   E_tot  sum_i occ_i lambda_i - h^3 sum rho (V_in - V_ion) + 1/2 h^3 sum rho V_H
 *          + h^3 sum rho eps_xc (- T S when kT > 0)   (band energy minus double counting)
 *   mixing Anderson mixing of V_in: F = V_out - V_in, history of the last `history`
 *          differences (dV_j, dF_j), g = argmin |F - sum_j g_j dF_j| by the normal
 *          equations, V_in <- V_in + alpha P F - sum_j g_j (dV_j + alpha P dF_j) with P the
 *          identity or the Kerker preconditioner (kerker_q0).
 *          (The paper names no mixing scheme; Anderson's is the Broyden-type method
 *          used here.)
 *   start  rho_0 = sum_a Z_a / (pi^{3/2} r_a^3) exp(-|r - R_a|^2 / r_a^2) (neutral-atom
 *          Gaussian valence densities, r_a per species), V_in = V_ion + V_H[rho_0] +
 *          V_xc[rho_0] (+ an optional caller correction dV, e.g. a learned one); X is
 *          orthonormalised and one Rayleigh-Ritz step gives the first filter bounds.
 *   step   kscf_set_potential(V_in); b = spectral upper bound; (4 or 1) x [filter with
 *          a = lambda_max, a0 = lambda_min of the previous Ritz values; Cholesky-QR;
 *          Rayleigh-Ritz]; rho; V_H; V_xc; SRE and energies; mixing unless converged.
 * The kscf_scf handle borrows the Hamiltonian (it rewrites its potential) and the
 * caller's X; both must outlive it.  It owns every other buffer (device memory about
 * (14 + 2 history) * n_slots doubles plus the CheFSI work buffers).  All calls are
 * synchronous (they read Ritz values and reductions on the host). */
typedef struct kscf_scf kscf_scf;

typedef struct kscf_scf_params {
  int32_t k;               /* subspace size (n_e/2 occupied + buffer), > n_e/2 */
  int32_t degree;          /* Chebyshev degree m */
  int32_t dtype;           /* KSCF_F64, or KSCF_F32 for the mixed-precision path */
  int32_t gemm_mode;       /* KSCF_GEMM_NATIVE or KSCF_GEMM_TENSOR (F32 only) */
  int32_t block;           /* filter column block, 0 = all k */
  int32_t first_iters;     /* CheFSI iterations in the first SCF step (paper: 4) */
  int32_t history;         /* Anderson history, 1..8 */
  int32_t poisson_maxiter; /* CG iteration cap per Hartree solve */
  double mix_alpha;        /* Anderson linear step (0 < alpha <= 1) */
  double sre_tol_ry;       /* converged when SRE < sre_tol_ry (paper: 1e-4 Ry) */
  double poisson_rtol;     /* CG stop |r| < rtol |b| */
  double kT;               /* electronic temperature (Ha): 0 = the n_e/2 lowest states doubly
                              occupied; > 0 = Fermi-Dirac occupations 2 f((lambda - mu)/kT),
                              mu from sum = n_e, and e_total is the free energy E - T S */
  double kerker_q0;        /* 0: plain Anderson; > 0: the residuals in the update are
                              preconditioned, P F = F - q0^2 u with (-Lap_h + q0^2) u = F on
                              the domain (Kerker's q^2/(q^2 + q0^2) damping of slowly
                              varying residuals; CG to poisson_rtol) */
  int32_t degree_max;      /* 0: every filter uses `degree`.  > 0: adaptive degrees (per-vector
                              degrees of ChASE, Winkelmann, Springer & Di Napoli 2019): before
                              each filter, lambda_i = <x_i, H x_i> and r_i = |H x_i - lambda_i x_i|
                              with the current H; with t_i = (c - lambda_i)/e and
                              rho_i = 1/(t_i + sqrt(t_i^2 - 1)), m_i = ceil(log(tol/r_i)/log rho_i)
                              (degree_min if r_i <= tol, degree_max if t_i <= 1), clamped to
                              [degree_min, degree_max]; each group of degree_group columns is
                              filtered with its largest m_i.  tol = max(adapt_tol_floor,
                              adapt_reduction * r_i): every vector is asked for the same
                              reduction of its residual per filter */
  int32_t degree_min;
  int32_t degree_group;    /* columns per group (e.g. 64) */
  int32_t upper_bound;     /* 0: b = Weyl + Gershgorin; 1: b = min(that, Lanczos estimate with
                              12 steps, kscf_lanczos_bounds) */
  double adapt_reduction;  /* 0 < reduction < 1 */
  double adapt_tol_floor;
} kscf_scf_params;

typedef struct kscf_scf_report {
  int32_t step;            /* SCF step number, 1-based (0 after kscf_scf_start) */
  int32_t converged;       /* 1 when sre_ry < sre_tol_ry (V_in then kept, no mixing) */
  int32_t poisson_iters;   /* CG iterations of this step's Hartree solve */
  int32_t chefsi_iters;    /* filter/QR/RR iterations in this step */
  double sre_ry;           /* SRE of this step (Ry) */
  double e_band;           /* sum_i f_i lambda_i (Ha) */
  double e_total;          /* Kohn-Sham total energy without ion-ion term (Ha) */
  double homo, lumo;       /* lambda_{n_occ-1}, lambda_{n_occ} (Ha) */
  double electrons;        /* h^3 sum rho */
  double mu;               /* Fermi level (kT > 0), else lambda_{n_occ-1} */
  double minus_ts;         /* -T S = 2 kT sum_i [f_i ln f_i + (1 - f_i) ln(1 - f_i)], f = occ/2 */
  double occ_last;         /* occupation of the highest Ritz state (k too small if not ~0) */
  int32_t kerker_iters;    /* CG iterations of this step's Kerker solve (0 without) */
  int32_t reserved;
  double filter_work;      /* sum over this step's filters of the column-averaged degree */
  double upper_bound;      /* the filter's b in this step */
} kscf_scf_report;

/* Creates the SCF state for the atoms the Hamiltonian was built from.  atoms/species
 * as for kscf_build_hamiltonian (read during the call); start_radius[n_species]: the
 * Gaussian width r_a (bohr) of each species' starting density.  X: caller device
 * array n_slots x ld of params->dtype (ld >= k), used as the subspace from
 * kscf_scf_start on.  Builds the ghost-point table of the Poisson problem on the host.
 * stream: where every later call of this handle runs. */
int kscf_scf_create(kscf_ham* ham, const kscf_atom* atoms, int n_atoms, const kscf_species* species,
                    int n_species, const double* start_radius, const kscf_scf_params* params, void* X,
                    int64_t ld, void* stream, kscf_scf** out);

/* Starting point.  dv_start: device, n_slots doubles added to the superposition
 * potential (NULL for none).  init_x != 0 fills X with kscf_random_subspace(seed) first;
 * 0 keeps the caller's X.  Then Cholesky-QR and Rayleigh-Ritz; eigvals_host (k doubles
 * or NULL) receives the Ritz values.  Clears the mixing history and the step count. */
int kscf_scf_start(kscf_scf* scf, const double* dv_start, int init_x, uint64_t seed, double* eigvals_host);

/* One SCF step (see above).  report receives its figures; eigvals_host (k doubles or
 * NULL) the Ritz values.  After a converged step V_in is left as it was, so a further
 * call repeats the step at the same potential. */
int kscf_scf_step(kscf_scf* scf, kscf_scf_report* report, double* eigvals_host);

/* Final evaluation in FP64 (the mixed-precision path keeps FP64 for the last residual
 * and energy evaluation): the Ritz vectors of the last step (widened to FP64 when X is
 * FP32) are applied with H at that step's V_in in FP64, giving the Rayleigh quotients
 * lambda_i = <x_i, H x_i> / <x_i, x_i> and residual norms |H x_i - lambda_i x_i| / |x_i|
 * (h^3-weighted).  report: the last step's report with e_band, e_total, homo, lumo, mu,
 * minus_ts and occ_last recomputed from the sorted Rayleigh quotients (the density terms
 * are those of the last step).  eigvals_host / resid_host: k doubles each (vector
 * order), or NULL.  Allocates about 2 n_slots k doubles of device memory for the call
 * and leaves the Hamiltonian at that V_in.  Synchronous. */
int kscf_scf_evaluate(kscf_scf* scf, kscf_scf_report* report, double* eigvals_host, double* resid_host);

/* Converged mode at the current input potential V_in (normally after the SCF has met
 * its SRE criterion, when V_in is the last step's potential): CheFSI iterations (filter,
 * Cholesky-QR, Rayleigh-Ritz, in the SCF's precision) at fixed potential until every
 * wanted state -- the occupied ones and the first empty one -- has FP64 residual norm
 * |H x - lambda x| below resid_tol (Ha), or the residuals stop falling for three
 * iterations (the working precision's floor), or max_iters iterations.  Then the density
 * of the refined vectors, its Hartree and exchange-correlation terms and the energy at
 * the same V_in are recomputed, and the result is reported as kscf_scf_evaluate does
 * (FP64 Rayleigh quotients, residuals, e_total).  iters_done (or NULL): iterations run.
 * V_in is not changed.  Synchronous; allocates like kscf_scf_evaluate. */
int kscf_scf_refine(kscf_scf* scf, int max_iters, double resid_tol, kscf_scf_report* report, double* eigvals_host,
                    double* resid_host, int* iters_done);

/* Fields for kscf_scf_get (device, n_slots doubles each, slot order, 0 in padding). */
#define KSCF_FIELD_RHO     0   /* density of the last step (start: rho_0) */
#define KSCF_FIELD_V_IN    1   /* current input potential (after mixing) */
#define KSCF_FIELD_V_H     2   /* Hartree potential of the last density */
#define KSCF_FIELD_V_XC    3   /* exchange-correlation potential of the last density */
#define KSCF_FIELD_V_ION   4   /* ionic (local pseudopotential) part */
#define KSCF_FIELD_V_START 5   /* superposition starting potential, without dv_start */
#define KSCF_FIELD_EPS_XC  6   /* exchange-correlation energy per electron */

/* Copies one field into dst (device, n_slots doubles) on the handle's stream. */
int kscf_scf_get(const kscf_scf* scf, int field, double* dst);

/* Hartree potential of an arbitrary density with the handle's Poisson solver:
 * rho (device, n_slots), vh (device, n_slots: starting guess on input, solution on
 * output), *iters (may be NULL) the CG iterations.  KSCF_ERR_NO_CONVERGE if the
 * iteration cap is reached first (vh then holds the last iterate). */
int kscf_scf_hartree(kscf_scf* scf, const double* rho, double* vh, int* iters);

int kscf_scf_free(kscf_scf* scf);

/* LDA exchange-correlation of a density (Slater exchange; Perdew-Zunger 1981 fit of the
 * Ceperley-Alder correlation, unpolarised; Hartree units):
 *   eps_x = -3/4 (3 rho/pi)^{1/3}, v_x = 4/3 eps_x, rs = (3/(4 pi rho))^{1/3},
 *   rs >= 1: eps_c = g/(1 + b1 sqrt(rs) + b2 rs),
 *            v_c = eps_c (1 + 7/6 b1 sqrt(rs) + 4/3 b2 rs)/(1 + b1 sqrt(rs) + b2 rs)
 *   rs < 1:  eps_c = A ln rs + B + C rs ln rs + D rs,
 *            v_c = A ln rs + B - A/3 + 2/3 C rs ln rs + (2D - C)/3 rs
 *   g = -0.1423, b1 = 1.0529, b2 = 0.3334, A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
 * rho <= 1e-14 gives 0.  rho, eps (may be NULL), vxc: device, n_slots doubles. */
int kscf_lda_xc(const kscf_ham* ham, const double* rho, double* eps, double* vxc, void* stream);

/* ---------------------------------------------------------------------------------
 * Learned SCF start.  The paper has no learned part: this is the library's own
 * correction dV of the superposition starting potential (passed to kscf_scf_start),
 * predicted per grid point by a small network from radial descriptors of the nearby
 * atoms, trained on converged SCF potentials by the kernels below.
 *
 * Descriptors (KSCF_MLP_N_IN = 32 per slot): for species s (0 = Si, 1 = H) and radial
 * centres c_q = q r_c / 15 (q = 0..15, r_c = 8 bohr),
 *   D[s][16 s + q] = sum over atoms of species s within r < r_c of
 *                    exp(-(r - c_q)^2 / (2 sigma^2)) (1 + cos(pi r / r_c)) / 2,  sigma = r_c/15.
 * Network: x = (D - mu) * inv_sd;  h1 = tanh(x W1 + b1) (32 -> 128);
 *   h2 = tanh(h1 W2 + b2) (128 -> 128);  y = h2 . w3 + b3.
 * Parameters: one float vector of KSCF_MLP_N_PARAMS = 20865 values in the order
 *   W1 (32 x 128 row-major), b1 (128), W2 (128 x 128 row-major), b2 (128), w3 (128), b3 (1).
 * All arrays are caller-owned device memory. */
#define KSCF_MLP_N_IN 32
#define KSCF_MLP_N_HID 128
#define KSCF_MLP_N_RADIAL 16
#define KSCF_MLP_R_CUT 8.0
#define KSCF_MLP_N_PARAMS (32 * 128 + 128 + 128 * 128 + 128 + 128 + 1)
#define KSCF_MLP_FP32 0   /* FP32 weights, activations and arithmetic */
#define KSCF_MLP_BF16 1   /* inference with weights, inputs and activations rounded to bf16,
                             products accumulated in FP32 */

/* D (device float, n_slots x 32 row-major) for the atoms (host array, Si and H only;
 * positions in bohr); padding rows are zero.  Synchronous. */
int kscf_descriptors(const kscf_ham* ham, const kscf_atom* atoms, int n_atoms, float* D, void* stream);

/* y[p] = network(D[p]) for p < n (D: n x 32 floats; mu, inv_sd: 32 floats each). */
int kscf_mlp_forward(const float* params, const float* mu, const float* inv_sd, const float* D, int64_t n,
                     int precision, float* y, void* stream);

/* Mean squared error L = (1/n) sum_p (y_p - t_p)^2 over the n rows of D and its gradient
 * grad (KSCF_MLP_N_PARAMS floats, layout of params), FP32 arithmetic with the per-block
 * partial gradients added in FP64 in block order (deterministic).  loss: device double
 * or NULL.  work: at least kscf_mlp_work_size(n) bytes. */
int kscf_mlp_work_size(int64_t n, size_t* bytes);
int kscf_mlp_loss_grad(const float* params, const float* mu, const float* inv_sd, const float* D, const float* t,
                       int64_t n, float* grad, double* loss, void* work, size_t work_bytes, void* stream);

/* Training data of one self-consistent cluster: for every domain point p (rows in
 * lexicographic point order, n_points rows), D_out[p] = the 32 descriptors of its slot
 * (D_slots from kscf_descriptors on the SCF's Hamiltonian) and t_out[p] = V_in - V_start
 * at that slot (the correction the network learns), in FP32.  Device arrays; enqueued on
 * the SCF's stream. */
int kscf_mlp_training_data(const kscf_scf* scf, const float* D_slots, float* D_out, float* t_out);

/* Standardisation of a training set (n >= 2 rows of D, targets t; device arrays):
 *   mu_j = mean_p D[p][j],  sd_j = sqrt(sum_p (D[p][j] - mu_j)^2 / (n - 1)),
 *   inv_sd_j = 1/sd_j, or 0 when sd_j <= 1e-6 (a constant feature is switched off),
 *   t_shift = mean t,  t_scale = sample standard deviation of t (1 if it is 0),
 *   t_norm = (t - t_shift) / t_scale.
 * Sums in FP64 over a fixed partition of the rows, added in a fixed order (deterministic).
 * mu, inv_sd: 32 floats; t_norm: n floats (device); t_shift_scale: 2 doubles (HOST).
 * Synchronous. */
int kscf_mlp_standardize(const float* D, const float* t, int64_t n, float* mu, float* inv_sd, float* t_norm,
                         double* t_shift_scale, void* stream);

/* The learned correction of the starting potential: dv[p] = y_p t_scale + t_shift (FP64)
 * with y = kscf_mlp_forward(params, mu, inv_sd, D, n, precision), written first into
 * y_work (n floats).  dv: n doubles (device), e.g. one per slot for kscf_scf_start. */
int kscf_mlp_correction(const float* params, const float* mu, const float* inv_sd, double t_shift, double t_scale,
                        const float* D, int64_t n, int precision, float* y_work, double* dv, void* stream);

/* One Adam step (Kingma & Ba 2015) on params with moment buffers m, v (step >= 1):
 *   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   params -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
int kscf_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                  float beta2, float eps, void* stream);

/* Density of states and HOMO-LUMO gap (host function; the DOS paragraph and Fig. 1:
 * eigenvalues histogrammed in bins of bin_ev (the paper uses 0.1 eV) with the highest
 * occupied state at zero, all DOS scaled to the same area below the Fermi level; the
 * band gap of Fig. 3 is the HOMO-LUMO gap).
 *   eigvals: k Ritz values (Ha, any order); HOMO = the n_occ-th smallest.
 *   hist[b] (b < n_bins) = (number of states with e = (lambda - HOMO) * 27.211386245988 eV
 *   in [e_lo_ev + b bin_ev, e_lo_ev + (b+1) bin_ev)) / (n_occ * bin_ev), so the occupied
 *   states integrate to one; states outside the bins are not counted.
 *   gap_ev: (LUMO - HOMO) in eV, NaN when n_occ == k (may be NULL). */
int kscf_dos(const double* eigvals, int k, int n_occ, double bin_ev, double e_lo_ev, int n_bins, double* hist,
             double* gap_ev);

/* Hilbert index of brick coordinates (x, y, z) on the 2^bits cube, as used to order the
 * bricks (Skilling 2004 transpose algorithm; bits interleaved most significant first,
 * x first).  Pure host function, exported for tests of the ordering. */
uint64_t kscf_hilbert_index3(uint32_t x, uint32_t y, uint32_t z, int bits);

#ifdef __cplusplus
}
#endif

#endif /* KSCF_H */
