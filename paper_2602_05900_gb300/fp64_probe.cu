// Device probe: latency and throughput of FP64 vs FP32 arithmetic on the GPU.
// Not part of libhotrg.  The eigensolver's design (FP32 seeds refined by FP64
// fused multiply-adds on latency-critical chains, FP64 bulk work spread over all
// SMs) rests on these numbers.  Build and run:
//   nvcc -O3 -gencode arch=compute_103a,code=sm_103a -o fp64_probe fp64_probe.cu && ./fp64_probe
// Every launch writes within its buffers and no kernel waits on anything.
#include <cstdio>
#include <cuda_runtime.h>
template <typename T, int OP>
__global__ void chain(T* out, T a, T b, int iters, long long* cycles) {
  T x = a + threadIdx.x * (T)1e-9, y = b;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      if (OP == 0) x = fma(x, y, (T)1e-30);          // dependent FMA
      else if (OP == 1) x = (T)1.0 / (x + (T)1.5);   // dependent divide
      else if (OP == 2) x = sqrt(x + (T)1.5);        // dependent sqrt
    }
  }
  long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}
template <typename T>
__global__ void thru(T* out, T a, T b, int iters) {
  T x0 = a + threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, b, (T)1e-30); x1 = fma(x1, b, (T)1e-30); x2 = fma(x2, b, (T)1e-30); x3 = fma(x3, b, (T)1e-30);
    x4 = fma(x4, b, (T)1e-30); x5 = fma(x5, b, (T)1e-30); x6 = fma(x6, b, (T)1e-30); x7 = fma(x7, b, (T)1e-30);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
int main() {
  double* dd; float* df; long long* cyc;
  cudaMalloc(&dd, 152 * 1024 * 8 * sizeof(double)); cudaMalloc(&df, 152 * 1024 * 8 * sizeof(float)); cudaMalloc(&cyc, 1024 * sizeof(long long));
  long long h[4];
  const char* names[3] = {"fma", "div", "sqrt"};
  for (int op = 0; op < 3; ++op) {
    int iters = 64;
    if (op == 0) chain<double, 0><<<1, 32>>>(dd, 1.0, 0.999999, iters, cyc);
    if (op == 1) chain<double, 1><<<1, 32>>>(dd, 1.0, 0.999999, iters, cyc);
    if (op == 2) chain<double, 2><<<1, 32>>>(dd, 1.0, 0.999999, iters, cyc);
    cudaDeviceSynchronize();
    cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
    printf("fp64 %s latency: %.1f cycles/op (1 warp)\n", names[op], (double)h[0] / (iters * 16));
    if (op == 0) chain<float, 0><<<1, 32>>>(df, 1.0f, 0.999999f, iters, cyc);
    if (op == 1) chain<float, 1><<<1, 32>>>(df, 1.0f, 0.999999f, iters, cyc);
    if (op == 2) chain<float, 2><<<1, 32>>>(df, 1.0f, 0.999999f, iters, cyc);
    cudaDeviceSynchronize();
    cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
    printf("fp32 %s latency: %.1f cycles/op (1 warp)\n", names[op], (double)h[0] / (iters * 16));
  }
  // latency with 8 warps on one SM (does the chain latency grow with warps?)
  chain<double, 0><<<1, 256>>>(dd, 1.0, 0.999999, 64, cyc);
  cudaDeviceSynchronize(); cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
  printf("fp64 fma chain with 8 warps/SM: %.1f cycles/op\n", (double)h[0] / (64 * 16));
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  for (int threads : {32, 128, 256, 1024}) {
    int iters = 4096;
    cudaEventRecord(a); thru<double><<<152, threads>>>(dd, 1.0, 0.9999999, iters); cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b);
    double flops = 2.0 * 8 * iters * 152.0 * threads;
    printf("fp64 fma throughput, 152 blocks x %d threads: %.3f TFLOP/s\n", threads, flops / ms / 1e9);
    cudaEventRecord(a); thru<float><<<152, threads>>>(df, 1.0f, 0.9999999f, iters); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    printf("fp32 fma throughput, 152 blocks x %d threads: %.3f TFLOP/s\n", threads, flops / ms / 1e9);
  }
  printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
