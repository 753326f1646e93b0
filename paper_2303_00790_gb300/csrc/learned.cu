// Learned SCF start: radial descriptors of the atoms around every grid point and a
// 32 -> 128 -> 128 -> 1 tanh multilayer perceptron that maps them to a correction of the
// superposition starting potential (the paper has no learned part; this is the
// project's own addition to the SCF start).  Forward, backward (mean squared error) and
// Adam are hand-written kernels; the network is trained on the GPU.
//
// Descriptors: D[p, 16 s + q] = sum over atoms a of species s (s = 0: Si, 1: H) with
// r = |p - R_a| < 8 bohr of exp(-(r - c_q)^2 / (2 sigma^2)) (1 + cos(pi r / 8)) / 2,
// c_q = q * 8/15, sigma = 8/15.
// Network on standardised inputs x = (D - mu) * inv_sd:
//   h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), y = h2 . w3 + b3.
// Parameter vector (KSCF_MLP_N_PARAMS floats): W1 (32 x 128 row-major), b1, W2 (128 x 128
// row-major), b2, w3, b3.
//
// The MLP kernels tile 64 points per iteration of a persistent block of 256 threads;
// the weights stay in shared memory for the whole launch (W2 rows padded to 129 floats
// and activation rows to 129 so that both row and column walks are free of bank
// conflicts).  A thread owns 4 points x 8 hidden units of each 64 x 128 layer output
// (points t/16 + 16 r, units t%16 + 16 c).  The backward kernel keeps its share of the
// weight gradients in registers across all tiles and writes one partial gradient per
// block; a second kernel adds the partials in block order in FP64 (deterministic).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kscf_internal.h"

namespace kscf {
namespace {

constexpr int NIN = KSCF_MLP_N_IN;    // 32
constexpr int NH = KSCF_MLP_N_HID;    // 128
constexpr int NPAR = KSCF_MLP_N_PARAMS;
constexpr int TP = 64;                // points per tile
constexpr int NT = 256;               // threads per block
constexpr int HS = NH + 1;            // padded row stride of W2 and of the activations
constexpr int XS = NIN + 1;           // padded row stride of the input tile
// parameter offsets
constexpr int OW1 = 0, OB1 = NIN * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
static_assert(OB3 + 1 == NPAR, "parameter layout");

// shared-memory layout (floats)
constexpr int S_W1 = 0;
constexpr int S_W2 = S_W1 + NIN * NH;
constexpr int S_B1 = S_W2 + NH * HS;
constexpr int S_B2 = S_B1 + NH;
constexpr int S_W3 = S_B2 + NH;
constexpr int S_X = S_W3 + NH;
constexpr int S_H1 = S_X + TP * XS;
constexpr int S_H2 = S_H1 + TP * HS;
constexpr int S_Y = S_H2 + TP * HS;      // y, then dy
constexpr int S_T = S_Y + TP;
constexpr int S_ACC = S_T + TP;          // db1, db2, dw3 accumulators (backward)
constexpr int S_END = S_ACC + 3 * NH;
constexpr size_t kMlpSmem = (size_t)S_END * sizeof(float);

__device__ __forceinline__ float to_bf16_value(float x) { return __bfloat162float(__float2bfloat16(x)); }

template <bool BF16>
__device__ __forceinline__ float q(float x) {
  return BF16 ? to_bf16_value(x) : x;
}

// Loads the weights (rounded to bf16 when BF16) into shared memory.
template <bool BF16>
__device__ void load_weights(const float* __restrict__ P, float* sm) {
  for (int e = threadIdx.x; e < NIN * NH; e += NT) sm[S_W1 + e] = q<BF16>(P[OW1 + e]);
  for (int e = threadIdx.x; e < NH * NH; e += NT) sm[S_W2 + (e / NH) * HS + (e % NH)] = q<BF16>(P[OW2 + e]);
  for (int e = threadIdx.x; e < NH; e += NT) {
    sm[S_B1 + e] = P[OB1 + e];
    sm[S_B2 + e] = P[OB2 + e];
    sm[S_W3 + e] = q<BF16>(P[OW3 + e]);
  }
}

// Standardised input tile: rows p0 .. p0+63 (rows past n are zero).
template <bool BF16>
__device__ void load_tile(const float* __restrict__ D, const float* __restrict__ mu, const float* __restrict__ inv_sd,
                          int64_t n, int64_t p0, float* sm) {
  for (int e = threadIdx.x; e < TP * NIN; e += NT) {
    const int p = e / NIN, i = e % NIN;
    const int64_t row = p0 + p;
    float v = 0.0f;
    if (row < n) v = (D[row * NIN + i] - mu[i]) * inv_sd[i];
    sm[S_X + p * XS + i] = q<BF16>(v);
  }
}

// h1, h2 and y of the tile in shared memory
template <bool BF16>
__device__ void forward_tile(float* sm, float b3) {
  const int t = threadIdx.x, pr = t >> 4, hc = t & 15;
  float acc[4][8];
  // layer 1
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 8; c++) acc[r][c] = sm[S_B1 + hc + 16 * c];
  for (int i = 0; i < NIN; i++) {
    float xv[4], wv[8];
#pragma unroll
    for (int r = 0; r < 4; r++) xv[r] = sm[S_X + (pr + 16 * r) * XS + i];
#pragma unroll
    for (int c = 0; c < 8; c++) wv[c] = sm[S_W1 + i * NH + hc + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int c = 0; c < 8; c++) acc[r][c] = fmaf(xv[r], wv[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 8; c++) sm[S_H1 + (pr + 16 * r) * HS + hc + 16 * c] = q<BF16>(tanhf(acc[r][c]));
  __syncthreads();
  // layer 2
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 8; c++) acc[r][c] = sm[S_B2 + hc + 16 * c];
  for (int k = 0; k < NH; k++) {
    float hv[4], wv[8];
#pragma unroll
    for (int r = 0; r < 4; r++) hv[r] = sm[S_H1 + (pr + 16 * r) * HS + k];
#pragma unroll
    for (int c = 0; c < 8; c++) wv[c] = sm[S_W2 + k * HS + hc + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int c = 0; c < 8; c++) acc[r][c] = fmaf(hv[r], wv[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 8; c++) sm[S_H2 + (pr + 16 * r) * HS + hc + 16 * c] = q<BF16>(tanhf(acc[r][c]));
  __syncthreads();
  // output: warp w handles points 8w .. 8w+7
  const int warp = t >> 5, lane = t & 31;
  for (int pp = 0; pp < 8; pp++) {
    const int p = warp * 8 + pp;
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; c++) s = fmaf(sm[S_H2 + p * HS + lane + 32 * c], sm[S_W3 + lane + 32 * c], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sm[S_Y + p] = s + b3;
  }
  __syncthreads();
}

template <bool BF16>
__global__ void __launch_bounds__(NT, 1) mlp_forward_kernel(const float* __restrict__ P, const float* __restrict__ mu,
                                                           const float* __restrict__ inv_sd,
                                                           const float* __restrict__ D, int64_t n,
                                                           float* __restrict__ y) {
  extern __shared__ float sm[];
  load_weights<BF16>(P, sm);
  const float b3 = P[OB3];
  const int64_t tiles = (n + TP - 1) / TP;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    __syncthreads();
    load_tile<BF16>(D, mu, inv_sd, n, tile * TP, sm);
    __syncthreads();
    forward_tile<BF16>(sm, b3);
    for (int p = threadIdx.x; p < TP; p += NT) {
      const int64_t row = tile * TP + p;
      if (row < n) y[row] = sm[S_Y + p];
    }
  }
}

// Loss and gradient: every block handles tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and writes part[block * (NPAR + 1) + q] (q < NPAR: gradient, q = NPAR: sum of (y - t)^2).
__global__ void __launch_bounds__(NT, 1) mlp_grad_kernel(const float* __restrict__ P, const float* __restrict__ mu,
                                                        const float* __restrict__ inv_sd,
                                                        const float* __restrict__ D, const float* __restrict__ tgt,
                                                        int64_t n, float* __restrict__ part) {
  extern __shared__ float sm[];
  load_weights<false>(P, sm);
  const float b3 = P[OB3];
  const int t = threadIdx.x, pr = t >> 4, hc = t & 15;
  for (int e = t; e < 3 * NH; e += NT) sm[S_ACC + e] = 0.0f;
  float gW2[8][8], gW1[2][8];  // rows (t/16 + 16 a), cols (t%16 + 16 c)
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int c = 0; c < 8; c++) gW2[a][c] = 0.0f;
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int c = 0; c < 8; c++) gW1[a][c] = 0.0f;
  float loss = 0.0f, gb3 = 0.0f;
  const float scale = 2.0f / (float)n;
  const int64_t tiles = (n + TP - 1) / TP;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    __syncthreads();
    load_tile<false>(D, mu, inv_sd, n, tile * TP, sm);
    for (int p = t; p < TP; p += NT) {
      const int64_t row = tile * TP + p;
      sm[S_T + p] = row < n ? tgt[row] : 0.0f;
    }
    __syncthreads();
    forward_tile<false>(sm, b3);
    // dy = 2 (y - t) / n for the points of the tile, 0 past n
    if (t < TP) {
      const int64_t row = tile * TP + t;
      const float r = row < n ? sm[S_Y + t] - sm[S_T + t] : 0.0f;
      loss += r * r;
      sm[S_Y + t] = scale * r;
    }
    __syncthreads();
    // dw3[j] += sum_p dy_p h2[p][j]; db3 += sum_p dy_p
    if (t < NH) {
      float s = 0.0f;
      for (int p = 0; p < TP; p++) s = fmaf(sm[S_Y + p], sm[S_H2 + p * HS + t], s);
      sm[S_ACC + 2 * NH + t] += s;
    } else if (t == NH) {
      float s = 0.0f;
      for (int p = 0; p < TP; p++) s += sm[S_Y + p];
      gb3 += s;
    }
    __syncthreads();
    // g2 = dy w3 (1 - h2^2), in place over h2
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int c = 0; c < 8; c++) {
        const int p = pr + 16 * r, j = hc + 16 * c;
        const float h = sm[S_H2 + p * HS + j];
        sm[S_H2 + p * HS + j] = sm[S_Y + p] * sm[S_W3 + j] * (1.0f - h * h);
      }
    __syncthreads();
    // db2[j] += sum_p g2[p][j]; dW2[i][j] += sum_p h1[p][i] g2[p][j]
    if (t < NH) {
      float s = 0.0f;
      for (int p = 0; p < TP; p++) s += sm[S_H2 + p * HS + t];
      sm[S_ACC + NH + t] += s;
    }
    for (int p = 0; p < TP; p++) {
      float hv[8], gv[8];
#pragma unroll
      for (int a = 0; a < 8; a++) hv[a] = sm[S_H1 + p * HS + pr + 16 * a];
#pragma unroll
      for (int c = 0; c < 8; c++) gv[c] = sm[S_H2 + p * HS + hc + 16 * c];
#pragma unroll
      for (int a = 0; a < 8; a++)
#pragma unroll
        for (int c = 0; c < 8; c++) gW2[a][c] = fmaf(hv[a], gv[c], gW2[a][c]);
    }
    __syncthreads();
    // g1[p][i] = (sum_j g2[p][j] W2[i][j]) (1 - h1[p][i]^2), in place over h1
    {
      float acc[4][8];
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 8; c++) acc[r][c] = 0.0f;
      for (int j = 0; j < NH; j++) {
        float gv[4], wv[8];
#pragma unroll
        for (int r = 0; r < 4; r++) gv[r] = sm[S_H2 + (pr + 16 * r) * HS + j];
#pragma unroll
        for (int c = 0; c < 8; c++) wv[c] = sm[S_W2 + (hc + 16 * c) * HS + j];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
          for (int c = 0; c < 8; c++) acc[r][c] = fmaf(gv[r], wv[c], acc[r][c]);
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 8; c++) {
          const int p = pr + 16 * r, i = hc + 16 * c;
          const float h = sm[S_H1 + p * HS + i];
          sm[S_H1 + p * HS + i] = acc[r][c] * (1.0f - h * h);
        }
    }
    __syncthreads();
    // db1[i] += sum_p g1[p][i]; dW1[i][j] += sum_p x[p][i] g1[p][j]
    if (t < NH) {
      float s = 0.0f;
      for (int p = 0; p < TP; p++) s += sm[S_H1 + p * HS + t];
      sm[S_ACC + t] += s;
    }
    for (int p = 0; p < TP; p++) {
      float xv[2], gv[8];
#pragma unroll
      for (int a = 0; a < 2; a++) xv[a] = sm[S_X + p * XS + pr + 16 * a];
#pragma unroll
      for (int c = 0; c < 8; c++) gv[c] = sm[S_H1 + p * HS + hc + 16 * c];
#pragma unroll
      for (int a = 0; a < 2; a++)
#pragma unroll
        for (int c = 0; c < 8; c++) gW1[a][c] = fmaf(xv[a], gv[c], gW1[a][c]);
    }
  }
  __syncthreads();
  // block partials
  float* out = part + (int64_t)blockIdx.x * (NPAR + 1);
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int c = 0; c < 8; c++) out[OW1 + (pr + 16 * a) * NH + hc + 16 * c] = gW1[a][c];
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int c = 0; c < 8; c++) out[OW2 + (pr + 16 * a) * NH + hc + 16 * c] = gW2[a][c];
  if (t < NH) {
    out[OB1 + t] = sm[S_ACC + t];
    out[OB2 + t] = sm[S_ACC + NH + t];
    out[OW3 + t] = sm[S_ACC + 2 * NH + t];
  }
  if (t == NH) out[OB3] = gb3;
  // loss: threads < TP hold their points' squared residuals
  __shared__ float sl[NT / 32];
  float l = loss;
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((t & 31) == 0) sl[t >> 5] = l;
  __syncthreads();
  if (t == 0) {
    float s = 0.0f;
    for (int w = 0; w < NT / 32; w++) s += sl[w];
    out[NPAR] = s;
  }
}

// grad[q] = sum_b part[b][q] (FP64, block order); loss = sum_b part[b][NPAR] / n
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nb, int64_t n, float* __restrict__ grad,
                                  double* __restrict__ loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > NPAR) return;
  double s = 0.0;
  for (int b = 0; b < nb; b++) s += (double)part[(int64_t)b * (NPAR + 1) + q];
  if (q < NPAR)
    grad[q] = (float)s;
  else if (loss)
    loss[0] = s / (double)n;
}

// Adam (Kingma & Ba 2015), step t >= 1
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Descriptors: one thread per slot; atoms staged through shared memory.
// atoms: 4 floats each (x, y, z relative to the grid centre, species 0/1).
__global__ void descriptor_kernel(const double* __restrict__ rel, const uint8_t* __restrict__ mask,
                                  const float4* __restrict__ atoms, int n_atoms, int64_t n, float* __restrict__ D) {
  __shared__ float4 sa[256];
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < n && mask[s];
  float px = 0.f, py = 0.f, pz = 0.f;
  if (live) {
    px = (float)rel[3 * s];
    py = (float)rel[3 * s + 1];
    pz = (float)rel[3 * s + 2];
  }
  float acc[NIN];
#pragma unroll
  for (int j = 0; j < NIN; j++) acc[j] = 0.0f;
  const float rc = KSCF_MLP_R_CUT;
  const float dc = rc / (KSCF_MLP_N_RADIAL - 1);
  const float inv2s2 = 1.0f / (2.0f * dc * dc);
  for (int a0 = 0; a0 < n_atoms; a0 += 256) {
    const int na = min(256, n_atoms - a0);
    __syncthreads();
    if (threadIdx.x < na) sa[threadIdx.x] = atoms[a0 + threadIdx.x];
    __syncthreads();
    if (!live) continue;
    for (int a = 0; a < na; a++) {
      const float4 at = sa[a];
      const float dx = px - at.x, dy = py - at.y, dz = pz - at.z;
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 < rc * rc)) continue;
      const float r = sqrtf(r2);
      const float fc = 0.5f * (1.0f + cospif(r / rc));
      const float w_si = at.w == 0.0f ? fc : 0.0f;
      const float w_h = at.w == 0.0f ? 0.0f : fc;
#pragma unroll
      for (int qq = 0; qq < KSCF_MLP_N_RADIAL; qq++) {
        const float d = r - qq * dc;
        const float g = expf(-d * d * inv2s2);
        acc[qq] = fmaf(g, w_si, acc[qq]);
        acc[KSCF_MLP_N_RADIAL + qq] = fmaf(g, w_h, acc[KSCF_MLP_N_RADIAL + qq]);
      }
    }
  }
  if (s < n) {
#pragma unroll
    for (int j = 0; j < NIN; j++) D[s * NIN + j] = acc[j];
  }
}

unsigned mlp_grid(int64_t n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (n + TP - 1) / TP;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
}

cudaError_t set_smem_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kMlpSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
  if (e == cudaSuccess) done = true;
  return e;
}


// ---- standardisation statistics: deterministic FP64 sums over kStdBlocks row ranges ----
constexpr int kStdBlocks = 256, kStdCols = NIN + 1;   // 32 descriptor columns + the target

// part[b][j] = sum over the rows of block b of (x_j - centre_j)^pw (pw = 1 or 2; column NIN
// is the target t); centre null means 0.  Thread (j = tid % 32, g = tid / 32) takes rows
// g, g + 8, ... of the block's range so that one warp reads whole rows.
__global__ void __launch_bounds__(256) std_partial_kernel(const float* __restrict__ D, const float* __restrict__ t,
                                                          int64_t n, const double* __restrict__ centre, int pw,
                                                          double* __restrict__ part) {
  const int j = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t per = (n + kStdBlocks - 1) / kStdBlocks;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
  const double cj = centre ? centre[j] : 0.0, ct = centre ? centre[NIN] : 0.0;
  double sx = 0.0, st = 0.0;
  for (int64_t r = r0 + g; r < r1; r += 8) {
    const double x = (double)D[r * NIN + j] - cj;
    sx += pw == 1 ? x : x * x;
    if (j == 0) {
      const double y = (double)t[r] - ct;
      st += pw == 1 ? y : y * y;
    }
  }
  __shared__ double red[8][kStdCols];
  red[g][j] = sx;
  if (j == 0) red[g][NIN] = st;
  __syncthreads();
  if (threadIdx.x < kStdCols) {
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 8; q++) acc += red[q][threadIdx.x];
    part[(int64_t)blockIdx.x * kStdCols + threadIdx.x] = acc;
  }
}

// out[j] = (sum_b part[b][j]) / div in block order
__global__ void std_finish_kernel(const double* __restrict__ part, double div, double* __restrict__ out) {
  const int j = threadIdx.x;
  if (j >= kStdCols) return;
  double acc = 0.0;
  for (int b = 0; b < kStdBlocks; b++) acc += part[(int64_t)b * kStdCols + j];
  out[j] = acc / div;
}

// mu, inv_sd (floor 1e-6), t_shift / t_scale (1 for a constant target) from mean and variance
__global__ void std_params_kernel(const double* __restrict__ mean, const double* __restrict__ var, float* __restrict__ mu,
                                  float* __restrict__ inv_sd, double* __restrict__ shift_scale) {
  const int j = threadIdx.x;
  if (j < NIN) {
    const double sd = sqrt(var[j]);
    mu[j] = (float)mean[j];
    inv_sd[j] = sd > 1e-6 ? (float)(1.0 / sd) : 0.0f;
  } else if (j == NIN) {
    const double sc = sqrt(var[NIN]);
    shift_scale[0] = mean[NIN];
    shift_scale[1] = sc > 0.0 ? sc : 1.0;
  }
}

__global__ void std_target_kernel(const float* __restrict__ t, int64_t n, const double* __restrict__ shift_scale,
                                  float* __restrict__ t_norm) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) t_norm[r] = (float)(((double)t[r] - shift_scale[0]) / shift_scale[1]);
}

__global__ void affine_kernel(const float* __restrict__ y, int64_t n, double scale, double shift,
                              double* __restrict__ dv) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) dv[r] = (double)y[r] * scale + shift;
}
}  // namespace
}  // namespace kscf

using namespace kscf;

extern "C" int kscf_descriptors(const kscf_ham* ham, const kscf_atom* atoms, int n_atoms, float* D, void* stream) {
  if (!ham || !D || n_atoms < 0 || (n_atoms > 0 && !atoms)) {
    set_error("kscf_descriptors: invalid argument");
    return KSCF_ERR_INVALID;
  }
  const Grid& g = ham->h.grid;
  std::vector<float> at(4 * (size_t)std::max(n_atoms, 1));
  for (int a = 0; a < n_atoms; a++) {
    if (atoms[a].z_number != 14 && atoms[a].z_number != 1) {
      set_error("kscf_descriptors: atom %d has Z=%d; descriptors are defined for Si and H", a, atoms[a].z_number);
      return KSCF_ERR_INVALID;
    }
    at[4 * a + 0] = (float)(atoms[a].x - g.center[0]);
    at[4 * a + 1] = (float)(atoms[a].y - g.center[1]);
    at[4 * a + 2] = (float)(atoms[a].z - g.center[2]);
    at[4 * a + 3] = atoms[a].z_number == 14 ? 0.0f : 1.0f;
  }
  std::vector<double> rel(3 * (size_t)g.n_slots);
  for (int64_t s = 0; s < g.n_slots; s++) {
    int ijk[3];
    g.slot_ijk(s, ijk);
    for (int d = 0; d < 3; d++) rel[3 * s + d] = g.h * (double)ijk[d];
  }
  float4* d_at = nullptr;
  double* d_rel = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMalloc((void**)&d_at, at.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_rel, rel.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_at, at.data(), at.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_rel, rel.data(), rel.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    descriptor_kernel<<<(unsigned)((g.n_slots + 127) / 128), 128, 0, st>>>(d_rel, ham->h.d_mask, d_at, n_atoms,
                                                                          g.n_slots, D);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host arrays go out of scope
  if (d_at) cudaFree(d_at);
  if (d_rel) cudaFree(d_rel);
  if (e != cudaSuccess) {
    set_error("kscf_descriptors: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  return KSCF_OK;
}

extern "C" int kscf_mlp_forward(const float* params, const float* mu, const float* inv_sd, const float* D, int64_t n,
                                int precision, float* y, void* stream) {
  if (!params || !mu || !inv_sd || (n > 0 && (!D || !y)) || n < 0 ||
      (precision != KSCF_MLP_FP32 && precision != KSCF_MLP_BF16)) {
    set_error("kscf_mlp_forward: invalid argument");
    return KSCF_ERR_INVALID;
  }
  if (n == 0) return KSCF_OK;
  KSCF_CUDA_TRY(set_smem_attrs());
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == KSCF_MLP_FP32)
    mlp_forward_kernel<false><<<mlp_grid(n), NT, kMlpSmem, st>>>(params, mu, inv_sd, D, n, y);
  else
    mlp_forward_kernel<true><<<mlp_grid(n), NT, kMlpSmem, st>>>(params, mu, inv_sd, D, n, y);
  count_launch();
  KSCF_CUDA_TRY(cudaGetLastError());
  return KSCF_OK;
}

extern "C" int kscf_mlp_work_size(int64_t n, size_t* bytes) {
  if (!bytes || n < 1) {
    set_error("kscf_mlp_work_size: invalid argument");
    return KSCF_ERR_INVALID;
  }
  *bytes = (size_t)mlp_grid(n) * (NPAR + 1) * sizeof(float);
  return KSCF_OK;
}

extern "C" int kscf_mlp_loss_grad(const float* params, const float* mu, const float* inv_sd, const float* D,
                                  const float* t, int64_t n, float* grad, double* loss, void* work, size_t work_bytes,
                                  void* stream) {
  if (!params || !mu || !inv_sd || !D || !t || !grad || n < 1) {
    set_error("kscf_mlp_loss_grad: invalid argument");
    return KSCF_ERR_INVALID;
  }
  const unsigned nb = mlp_grid(n);
  const size_t need = (size_t)nb * (NPAR + 1) * sizeof(float);
  if (!work || work_bytes < need) {
    set_error("kscf_mlp_loss_grad: work buffer of %zu bytes, need %zu", work_bytes, need);
    return KSCF_ERR_WORKSPACE;
  }
  KSCF_CUDA_TRY(set_smem_attrs());
  cudaStream_t st = (cudaStream_t)stream;
  mlp_grad_kernel<<<nb, NT, kMlpSmem, st>>>(params, mu, inv_sd, D, t, n, (float*)work);
  count_launch();
  KSCF_CUDA_TRY(cudaGetLastError());
  mlp_reduce_kernel<<<(NPAR + 1 + 255) / 256, 256, 0, st>>>((const float*)work, (int)nb, n, grad, loss);
  count_launch();
  KSCF_CUDA_TRY(cudaGetLastError());
  return KSCF_OK;
}

extern "C" int kscf_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                             float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || step < 1 || !(lr > 0.0f)) {
    set_error("kscf_mlp_adam: invalid argument");
    return KSCF_ERR_INVALID;
  }
  const float c1 = (float)(1.0 - std::pow((double)beta1, step));
  const float c2 = (float)(1.0 - std::pow((double)beta2, step));
  adam_kernel<<<(NPAR + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, NPAR, lr, beta1, beta2, eps,
                                                                    c1, c2);
  count_launch();
  KSCF_CUDA_TRY(cudaGetLastError());
  return KSCF_OK;
}

extern "C" int kscf_mlp_standardize(const float* D, const float* t, int64_t n, float* mu, float* inv_sd, float* t_norm,
                                    double* t_shift_scale, void* stream) {
  if (!D || !t || !mu || !inv_sd || !t_norm || !t_shift_scale || n < 2) {
    set_error("kscf_mlp_standardize: invalid argument (n >= 2 rows needed)");
    return KSCF_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* buf = nullptr;   // partials, mean, variance, shift/scale
  const size_t nbuf = (size_t)kStdBlocks * kStdCols + 3 * kStdCols;
  KSCF_CUDA_TRY(cudaMalloc((void**)&buf, nbuf * sizeof(double)));
  double* part = buf;
  double* mean = part + (size_t)kStdBlocks * kStdCols;
  double* var = mean + kStdCols;
  double* ss = var + kStdCols;
  std_partial_kernel<<<kStdBlocks, 256, 0, st>>>(D, t, n, nullptr, 1, part), count_launch();
  std_finish_kernel<<<1, 64, 0, st>>>(part, (double)n, mean), count_launch();
  std_partial_kernel<<<kStdBlocks, 256, 0, st>>>(D, t, n, mean, 2, part), count_launch();
  std_finish_kernel<<<1, 64, 0, st>>>(part, (double)(n - 1), var), count_launch();
  std_params_kernel<<<1, 64, 0, st>>>(mean, var, mu, inv_sd, ss), count_launch();
  std_target_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, n, ss, t_norm), count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(t_shift_scale, ss, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_error("kscf_mlp_standardize: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  return KSCF_OK;
}

extern "C" int kscf_mlp_correction(const float* params, const float* mu, const float* inv_sd, double t_shift,
                                   double t_scale, const float* D, int64_t n, int precision, float* y_work, double* dv,
                                   void* stream) {
  if (!dv || (n > 0 && !y_work) || !std::isfinite(t_shift) || !std::isfinite(t_scale)) {
    set_error("kscf_mlp_correction: invalid argument");
    return KSCF_ERR_INVALID;
  }
  int rc = kscf_mlp_forward(params, mu, inv_sd, D, n, precision, y_work, stream);
  if (rc) return rc;
  if (n == 0) return KSCF_OK;
  affine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(y_work, n, t_scale, t_shift, dv);
  count_launch();
  KSCF_CUDA_TRY(cudaGetLastError());
  return KSCF_OK;
}
