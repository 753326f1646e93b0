// FP32 / packed FP32x2 / FP64 FMA throughput microbenchmark (standalone program):
// eight independent FMA chains per thread, 8 CTAs of 256 threads per SM, result written
// once per thread.  Used to state the ALU roofs that the copy/GEMM peaks do not cover.
// A second part times FP64 instruction sequences inside one CTA (1, 4 or 8 warps; 1 or 32
// active lanes) with clock64: the cost of one warp-wide FP64 instruction on one SM
// sub-partition, which sets the length of the sequential chains of small dense kernels.
#include <cstdio>
#include <cuda_runtime.h>
template <typename T> __global__ void fma_kernel(T* out, T a, T b, int iters) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; i++) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void fma2_kernel(float2* out, float a, float b, int iters) {
  float2 x[8];
  for (int q = 0; q < 8; q++) x[q] = make_float2(threadIdx.x * 1e-3f + q, q * 0.5f);
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int q = 0; q < 8; q++) {
      unsigned long long r;
      asm volatile("{.reg .b64 a2, b2; mov.b64 a2, {%1, %1}; mov.b64 b2, {%2, %2};"
                   "fma.rn.f32x2 %0, %3, a2, b2;}" : "=l"(r) : "f"(a), "f"(b), "l"(*(unsigned long long*)&x[q]));
      x[q] = *(float2*)&r;
    }
  float2 s = make_float2(0, 0);
  for (int q = 0; q < 8; q++) { s.x += x[q].x; s.y += x[q].y; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// one CTA; lanes < active run n FP64 operations: 0 = dependent FMA chain, 1 = eight
// independent FMA chains, 2 = dependent sqrt chain, 3 = dependent division chain
__global__ void fp64_chain_kernel(double* out, long long* cyc, int n, int mode, int active) {
  const int lane = threadIdx.x & 31;
  double a[8];
  for (int q = 0; q < 8; q++) a[q] = 1.0 + 1e-9 * threadIdx.x + 0.1 * q;
  const double b = 0.999999, c = 1e-7;
  __syncthreads();
  const long long t0 = clock64();
  if (lane < active) {
    if (mode == 0) {
      for (int i = 0; i < n; i++) a[0] = fma(a[0], b, c);
    } else if (mode == 1) {
      for (int i = 0; i < n; i += 8)
#pragma unroll
        for (int q = 0; q < 8; q++) a[q] = fma(a[q], b, c);
    } else if (mode == 2) {
      for (int i = 0; i < n; i++) a[0] = sqrt(a[0]) + c;
    } else {
      for (int i = 0; i < n; i++) a[0] = b / a[0] + c;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  double s = 0.0;
  for (int q = 0; q < 8; q++) s += a[q];
  out[threadIdx.x] = s;
  if (threadIdx.x == 0) *cyc = t1 - t0;
}

int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = sms * 8, threads = 256, iters = 1 << 16;
  void* out; cudaMalloc(&out, (size_t)blocks * threads * 16);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  for (int rep = 0; rep < 2; rep++) {
    fma_kernel<float><<<blocks, threads>>>((float*)out, 0.999f, 1e-4f, iters);
    cudaEventRecord(e0); fma_kernel<float><<<blocks, threads>>>((float*)out, 0.999f, 1e-4f, iters); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0 * 8 * (double)iters * blocks * threads;
    printf("fp32 fma: %.1f TFLOP/s\n", fl / ms / 1e9);
    fma2_kernel<<<blocks, threads>>>((float2*)out, 0.999f, 1e-4f, iters);
    cudaEventRecord(e0); fma2_kernel<<<blocks, threads>>>((float2*)out, 0.999f, 1e-4f, iters); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    printf("fp32x2 fma: %.1f TFLOP/s\n", 2 * fl / ms / 1e9);
    fma_kernel<double><<<blocks, threads>>>((double*)out, 0.999, 1e-4, iters / 16);
    cudaEventRecord(e0); fma_kernel<double><<<blocks, threads>>>((double*)out, 0.999, 1e-4, iters / 16); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    printf("fp64 fma: %.3f TFLOP/s\n", fl / 16 / ms / 1e9);
  }
  long long* cyc;
  cudaMalloc(&cyc, sizeof(long long));
  const char* names[] = {"dfma dependent", "dfma 8 independent", "sqrt dependent", "div dependent"};
  for (int mode = 0; mode < 4; mode++)
    for (int warps : {1, 4, 8})
      for (int active : {1, 32}) {
        const int n = mode < 2 ? 4096 : 256;
        for (int rep = 0; rep < 2; rep++) fp64_chain_kernel<<<1, 32 * warps>>>((double*)out, cyc, n, mode, active);
        long long c = 0;
        cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
        printf("%-20s warps %d lanes %2d: %7.1f cycles per operation per warp\n", names[mode], warps, active,
               (double)c / n);
      }
  printf("sms %d err %s\n", sms, cudaGetErrorString(cudaGetLastError()));
  return 0;
}
