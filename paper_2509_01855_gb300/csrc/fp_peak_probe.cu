// FP64 / FP32 FMA throughput of the GPU: eight independent FMA chains per thread, enough blocks
// to fill every SM. Not part of libbirkhoff.so; it measures the ALU peak that bounds the FP64
// transforms (the roofline denominator of the FP64 Birkhoff product).
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp_peak_probe fp_peak_probe.cu
#include <cstdio>
#include <cuda_runtime.h>
template <typename T, int ILP>
__global__ void fma_kernel(T* out, int iters, T a, T b) {
  T acc[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) acc[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < ILP; ++i) acc[i] = fma(acc[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < ILP; ++i) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <typename T>
void run(const char* name, int blocks, int threads, int iters) {
  T* d; cudaMalloc(&d, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int w = 0; w < 2; ++w) fma_kernel<T, 8><<<blocks, threads>>>(d, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e0);
  fma_kernel<T, 8><<<blocks, threads>>>(d, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double flops = 2.0 * 8 * (double)iters * blocks * threads;
  printf("%s blocks=%d threads=%d: %.3f ms, %.2f TFLOP/s (%s)\n", name, blocks, threads, ms,
         flops / ms / 1e9, cudaGetErrorString(cudaGetLastError()));
  cudaFree(d);
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("%s SMs=%d L2=%d MB smemOptin=%zu KB\n", p.name, p.multiProcessorCount,
         p.l2CacheSize >> 20, p.sharedMemPerBlockOptin >> 10);
  int sms = p.multiProcessorCount;
  run<double>("fp64", sms * 4, 256, 4096);
  run<double>("fp64", sms * 8, 256, 4096);
  run<float>("fp32", sms * 8, 256, 65536);
  run<float>("fp32", sms * 16, 256, 65536);
  return 0;
}
