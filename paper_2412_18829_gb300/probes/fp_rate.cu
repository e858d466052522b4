// CUDA-core FMA-rate probe (FP64 and FP32): independent FMA chains on every SM; prints TFLOP/s.
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp_rate fp_rate.cu
#include <cstdio>
#include <cuda_runtime.h>
__global__ void k(double *out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 12345.678) out[0] = s;
}
__global__ void kf(float *out, int iters, float a, float b) {
  float x[16];
  for (int j = 0; j < 16; ++j) x[j] = threadIdx.x + j;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], a, b);
  float s = 0; for (int j = 0; j < 16; ++j) s += x[j];
  if (s == 12345.678f) out[0] = s;
}
int main() {
  int sm; cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, 0);
  double *d; cudaMalloc(&d, 64);
  int iters = 1 << 16;
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  for (int blocks_per_sm : {4, 8, 16}) {
    int grid = sm * blocks_per_sm;
    k<<<grid, 256>>>(d, iters, 0.999999, 1e-7);
    cudaEventRecord(a);
    k<<<grid, 256>>>(d, iters, 0.999999, 1e-7);
    cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b);
    double flops = 2.0 * 8 * iters * (double)grid * 256;
    printf("fp64 fma: SMs %d blocks/SM %d  %.3f TFLOP/s\n", sm, blocks_per_sm, flops / ms / 1e9);
  }
  for (int blocks_per_sm : {4, 8}) {
    int grid = sm * blocks_per_sm;
    kf<<<grid, 256>>>((float*)d, iters, 0.999999f, 1e-7f);
    cudaEventRecord(a);
    kf<<<grid, 256>>>((float*)d, iters, 0.999999f, 1e-7f);
    cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b);
    double flops = 2.0 * 16 * iters * (double)grid * 256;
    printf("fp32 fma: blocks/SM %d  %.3f TFLOP/s\n", blocks_per_sm, flops / ms / 1e9);
  }
  printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
