// Checks the integer-pipe conversions of fv_device32.cuh against the
// hardware conversions, and the exponent-step products x/2 and 2x of
// fv_device.cuh and fv_device32.cuh against the IEEE products, bit for bit,
// on boundary cases and 2^26 seeded random bit patterns.  Prints
// "mismatches <n>" and exits 0 when n == 0.
#include <cstdio>
#include <cuda_runtime.h>

#include "fv_device32.cuh"

__device__ unsigned long long mix(unsigned long long z) {  // SplitMix64 finaliser
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ bool same_bits(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b);
}

__global__ void k_check(unsigned long long n, unsigned long long* bad) {
  unsigned long long local = 0;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long r = mix(t * 0x9E3779B97F4A7C15ULL + 12345);
    // doubles: spread exponents over the whole range, and near the float range ends
    unsigned long long db = r;
    if (t & 1) {
      const unsigned e = 860 + (unsigned)((r >> 52) % 330);   // around [897, 1150]
      db = (r & 0x800FFFFFFFFFFFFFULL) | ((unsigned long long)e << 52);
    }
    if ((t & 7) == 2) db = (db & ~0x1FFFFFFFULL) | 0x10000000ULL;   // exact ties
    const double d = __longlong_as_double((long long)db);
    const float a = fvd32::d2f(d), b = __double2float_rn(d);
    if (__float_as_uint(a) != __float_as_uint(b) && !(a != a && b != b)) ++local;
    const float f = __uint_as_float((unsigned)(r >> 17));
    const double x = fvd32::f2d(f), y = (double)f;
    if (__double_as_longlong(x) != __double_as_longlong(y) && !(x != x && y != y)) ++local;
    // halving and doubling; every 8th operand a signed zero
    const double h = (t & 7) == 5 ? __longlong_as_double((long long)(r & 0x8000000000000000ULL)) : d;
    if (!same_bits(fvd::half(h), __dmul_rn(h, 0.5))) ++local;
    if (!same_bits(fvd32::dhalf(h), __dmul_rn(h, 0.5))) ++local;
    if (!same_bits(fvd::twice(h), __dmul_rn(h, 2.0))) ++local;
  }
  if (local) atomicAdd(bad, local);
}

__global__ void k_edges(unsigned long long* bad) {
  const double ds[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                       3.402823567797337e38, 1.1754943508222875e-38, 1.1754942106924411e-38,
                       5.877471754111438e-39, 1.401298464324817e-45, 1e-300, 1e300,
                       __longlong_as_double(0x7FF0000000000000LL),
                       __longlong_as_double((long long)0xFFF0000000000000ULL),
                       2.2250738585072014e-308, 4.450147717014403e-308, 1.7976931348623157e308,
                       -2.2250738585072014e-308, 2.225073858507201e-308,
                       __longlong_as_double(0x7FF8000000000000LL), 0.1, 2.5, 1.0 / 3.0};
  for (double d : ds) {
    const float a = fvd32::d2f(d), b = __double2float_rn(d);
    if (__float_as_uint(a) != __float_as_uint(b) && !(a != a && b != b)) atomicAdd(bad, 1ULL);
    const float f = b;
    const double x = fvd32::f2d(f), y = (double)f;
    if (__double_as_longlong(x) != __double_as_longlong(y) && !(x != x && y != y))
      atomicAdd(bad, 1ULL);
    if (!same_bits(fvd::half(d), __dmul_rn(d, 0.5)) || !same_bits(fvd32::dhalf(d), __dmul_rn(d, 0.5)) ||
        !same_bits(fvd::twice(d), __dmul_rn(d, 2.0)))
      atomicAdd(bad, 1ULL);
  }
}

int main() {
  unsigned long long* bad;
  if (cudaMalloc(&bad, sizeof *bad) != cudaSuccess) return 2;
  cudaMemset(bad, 0, sizeof *bad);
  k_edges<<<1, 1>>>(bad);
  k_check<<<152 * 8, 256>>>(1ULL << 26, bad);
  unsigned long long h = ~0ULL;
  cudaMemcpy(&h, bad, sizeof h, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  printf("mismatches %llu (%s)\n", h, cudaGetErrorString(e));
  cudaFree(bad);
  return (e == cudaSuccess && h == 0) ? 0 : 1;
}
