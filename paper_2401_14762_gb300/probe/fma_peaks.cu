// FP32 and FP64 FMA throughput of the GPU: the denominators of the SIMT kernels'
// roofline fractions (the greedy kernels, the FP32 FISTA/ADMM paths, sparsification).
// Eight independent FMA chains per thread, 16-fold unrolled, 8 CTAs of 256 threads per
// SM; the second of two launches is timed with CUDA events.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 fma_peaks.cu -o fma_peaks && ./fma_peaks
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <typename T>
double run(int blocks, int threads, int iters) {
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  fma_loop<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  fma_loop<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  cudaFree(out);
  return flops / (ms * 1e-3) / 1e12;
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("name %s sms %d smem/blk optin %zu l2 %d cc %d.%d\n", p.name, p.multiProcessorCount, p.sharedMemPerBlockOptin, p.l2CacheSize, p.major, p.minor);
  int sms = p.multiProcessorCount;
  for (int k = 0; k < 2; ++k) {
    printf("fp32 TFLOP/s %.2f\n", run<float>(sms * 8, 256, 4000));
    printf("fp64 TFLOP/s %.3f\n", run<double>(sms * 8, 256, 200));
  }
  cudaError_t e = cudaGetLastError();
  printf("err %s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}
