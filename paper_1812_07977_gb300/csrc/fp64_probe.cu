// fp64_probe.cu -- measures this GPU's arithmetic issue rates for the
// roofline of the FP64 step: DFMA, DADD, DMUL, double divide and square
// root, and FFMA for comparison.  Standalone program; prints one JSON line.
//
// Each thread runs 8 independent dependency chains so the pipes, not the
// latencies, set the rate; every chain's result is stored so nothing is
// dead code.  The grid is 8 blocks of 256 threads per SM.
#include <cstdio>

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int OP>
__global__ void __launch_bounds__(kThreads) k_rate(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + threadIdx.x * 1e-3 + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (OP == 0) x[c] = fma(x[c], a, b);
      if (OP == 1) x[c] = x[c] + a;
      if (OP == 2) x[c] = x[c] * a;
      if (OP == 3) x[c] = a / x[c] + b;
      if (OP == 4) x[c] = sqrt(x[c]) + b;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_ffma(double* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0f + threadIdx.x * 1e-3f + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <class F>
double best_ms(F&& launch) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 2; ++w) launch();
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace

int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) {
    printf("{\"error\": \"no CUDA device\"}\n");
    return 1;
  }
  const int sms = p.multiProcessorCount;
  const int blocks = sms * 8;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks * kThreads) != cudaSuccess) {
    printf("{\"error\": \"cudaMalloc failed\"}\n");
    return 1;
  }
  const double lanes = (double)blocks * kThreads * kChains;
  const int it_fast = 2000, it_slow = 200, it_sp = 20000;
  double r[6];
  r[0] = lanes * it_fast / (best_ms([&] { k_rate<0><<<blocks, kThreads>>>(d, it_fast, 0.999999, 1e-7); }) * 1e-3);
  r[1] = lanes * it_fast / (best_ms([&] { k_rate<1><<<blocks, kThreads>>>(d, it_fast, 1e-9, 0.0); }) * 1e-3);
  r[2] = lanes * it_fast / (best_ms([&] { k_rate<2><<<blocks, kThreads>>>(d, it_fast, 0.9999999, 0.0); }) * 1e-3);
  r[3] = lanes * it_slow / (best_ms([&] { k_rate<3><<<blocks, kThreads>>>(d, it_slow, 1.5, 1e-7); }) * 1e-3);
  r[4] = lanes * it_slow / (best_ms([&] { k_rate<4><<<blocks, kThreads>>>(d, it_slow, 0.0, 1e-7); }) * 1e-3);
  r[5] = lanes * it_sp / (best_ms([&] { k_ffma<<<blocks, kThreads>>>(d, it_sp, 0.999999f, 1e-7f); }) * 1e-3);
  const cudaError_t e = cudaGetLastError();
  cudaFree(d);
  if (e != cudaSuccess) {
    printf("{\"error\": \"%s\"}\n", cudaGetErrorString(e));
    return 1;
  }
  printf("{\"gpu\": \"%s\", \"sms\": %d, \"dfma_per_s\": %.6g, \"dadd_per_s\": %.6g, "
         "\"dmul_per_s\": %.6g, \"ddiv_per_s\": %.6g, \"dsqrt_per_s\": %.6g, \"ffma_per_s\": %.6g}\n",
         p.name, sms, r[0], r[1], r[2], r[3], r[4], r[5]);
  return 0;
}
