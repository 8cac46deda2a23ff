// ALU and copy-bandwidth peaks of the GPU: FP64 / FP32 FMA and INT32 IMAD throughput from
// independent FMA chains (8 per thread, 16x unrolled), and a float4 device-to-device copy.
// Used as the denominator of the roofline fraction of ALU-bound kernels.
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_kernel(T* out, T a, T b, int iters) {
  T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)12345) out[0] = s;
}
__global__ void copy_kernel(const float4* __restrict__ a, float4* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}
template <typename T>
double run(const char* name, T a, T b, int blocks, int threads, int iters) {
  T* out; cudaMalloc(&out, sizeof(T));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  fma_kernel<T><<<blocks, threads>>>(out, a, b, 10);
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    fma_kernel<T><<<blocks, threads>>>(out, a, b, iters);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
  }
  double fmas = (double)blocks * threads * iters * 16 * 8;
  double tf = 2.0 * fmas / (best * 1e-3) / 1e12;
  printf("%s: blocks=%d threads=%d  %.3f ms  %.2f TFLOP/s (%.1f G FMA/s)\n", name, blocks, threads, best, tf, fmas / (best * 1e-3) / 1e9);
  cudaFree(out);
  return tf;
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("%s SMs=%d cc=%d.%d l2=%d MB\n", p.name, p.multiProcessorCount, p.major, p.minor, p.l2CacheSize >> 20);
  int sms = p.multiProcessorCount;
  run<double>("fp64", 1.0000001, 1e-9, sms * 8, 256, 200);
  run<double>("fp64", 1.0000001, 1e-9, sms * 16, 256, 200);
  run<float>("fp32", 1.0000001f, 1e-9f, sms * 8, 256, 4000);
  run<float>("fp32", 1.0000001f, 1e-9f, sms * 16, 256, 4000);
  run<int>("int32", 3, 7, sms * 8, 256, 4000);
  size_t n = (size_t)1 << 28;  // 4 GiB per buffer in float4 units of 16 B -> 256M*16=4GB
  float4 *a, *b; cudaMalloc(&a, n * 16); cudaMalloc(&b, n * 16);
  cudaMemset(a, 0, n * 16);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < 6; ++r) {
    cudaEventRecord(e0); copy_kernel<<<sms * 8, 512>>>(a, b, n); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); if (r > 0 && ms < best) best = ms;
  }
  printf("copy: %.1f GB/s\n", 2.0 * n * 16 / (best * 1e-3) / 1e9);
  printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
