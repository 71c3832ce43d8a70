// Checks the Newton-Raphson reciprocal and sound speed of fv_device.cuh
// (recip_nr, sound_speed_nr; used by the FMA build) against the IEEE
// operations: the largest distance in ulps over 2^26 seeded random operands
// spread over the seed range, and bitwise equality (NaN with NaN) outside it
// and on special values.  Prints "recip_max_ulp <a> speed_max_ulp <b>
// outside_mismatches <n>".
#include <cstdio>
#include <cuda_runtime.h>

#include "fv_device.cuh"

__device__ unsigned long long mix(unsigned long long z) {  // SplitMix64 finaliser
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ unsigned long long ulps(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  if ((x ^ y) < 0) return ~0ULL;   // different signs
  return x > y ? (unsigned long long)(x - y) : (unsigned long long)(y - x);
}

__device__ bool same(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b);
}

// a double with exponent e (unbiased) and random mantissa and sign
__device__ double with_exp(unsigned long long r, int e) {
  return __longlong_as_double((long long)((r & 0x800FFFFFFFFFFFFFULL) |
                                          ((unsigned long long)(e + 1023) << 52)));
}

__global__ void k_check(unsigned long long n, unsigned long long* out) {
  unsigned long long mr = 0, ms = 0, bad = 0;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r1 = mix(t * 0x9E3779B97F4A7C15ULL + 7);
    const unsigned long long r2 = mix(r1 + 0x632BE59BD9B4E019ULL);
    // reciprocal: exponents -130 .. 129 (some outside the seed range)
    const double d = with_exp(r1, (int)(r1 >> 55) % 260 - 130);
    const double a = fvd::recip_nr(d), b = 1.0 / d;
    if (fvd::seed_range(d)) {
      const unsigned long long u = ulps(a, b);
      mr = u > mr ? u : mr;
    } else if (!same(a, b)) {
      ++bad;
    }
    // sound speed: t = gamma p and rho positive, exponents -70 .. 69
    const double tt = fabs(with_exp(r1 >> 3, (int)(r2 >> 56) % 140 - 70));
    const double rr = fabs(with_exp(r2, (int)((r2 >> 40) & 0xFF) % 140 - 70));
    const double c = fvd::sound_speed_nr(tt, rr), ci = sqrt(tt / rr);
    if (fvd::seed_range(tt * rr)) {
      const unsigned long long u = ulps(c, ci);
      ms = u > ms ? u : ms;
    } else if (!same(c, ci)) {
      ++bad;
    }
  }
  atomicMax(&out[0], mr);
  atomicMax(&out[1], ms);
  if (bad) atomicAdd(&out[2], bad);
}

__global__ void k_edges(unsigned long long* out) {
  const double inf = __longlong_as_double(0x7FF0000000000000LL);
  const double nan = __longlong_as_double(0x7FF8000000000000LL);
  const double v[] = {0.0, -0.0, 1.0, -1.0, 0.125, 1.4, 3.0, 1e-300, -1e-300, 1e300,
                      4.9e-324, inf, -inf, nan, 0x1p-120, 0x1.fffffffffffffp-121, 0x1p120,
                      0x1.fffffffffffffp119, -0x1p-120, 1.0 / 3.0};
  unsigned long long bad = 0, mr = 0, ms = 0;
  for (double x : v) {
    const double a = fvd::recip_nr(x), b = 1.0 / x;
    if (fvd::seed_range(x)) {
      const unsigned long long u = ulps(a, b);
      mr = u > mr ? u : mr;
    } else if (!same(a, b)) {
      ++bad;
    }
    for (double y : v) {
      const double c = fvd::sound_speed_nr(x, y), ci = sqrt(x / y);
      const bool fast = x > 0.0 && y > 0.0 && fvd::seed_range(x) && fvd::seed_range(y) &&
                        fvd::seed_range(x * y);
      if (fast) {
        const unsigned long long u = ulps(c, ci);
        ms = u > ms ? u : ms;
      } else if (!same(c, ci)) {
        ++bad;
      }
    }
  }
  atomicMax(&out[0], mr);
  atomicMax(&out[1], ms);
  if (bad) atomicAdd(&out[2], bad);
}

int main() {
  unsigned long long* out;
  if (cudaMalloc(&out, 3 * sizeof *out) != cudaSuccess) return 2;
  cudaMemset(out, 0, 3 * sizeof *out);
  k_edges<<<1, 1>>>(out);
  k_check<<<152 * 8, 256>>>(1ULL << 26, out);
  unsigned long long h[3] = {~0ULL, ~0ULL, ~0ULL};
  cudaMemcpy(h, out, sizeof h, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  printf("recip_max_ulp %llu speed_max_ulp %llu outside_mismatches %llu (%s)\n", h[0], h[1], h[2],
         cudaGetErrorString(e));
  cudaFree(out);
  return e == cudaSuccess ? 0 : 1;
}
