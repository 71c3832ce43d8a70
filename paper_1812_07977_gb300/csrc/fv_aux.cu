// fv_aux.cu -- ghost fill (GhostExchange), conservation sums, and the
// interior <-> ghosted copies of set/get state.  Built without FMA
// contraction.  (The FP64 time step, ComputeTimeStep, is compiled with the
// step kernels, in both of their arithmetic variants.)
#include <atomic>

#include "fv_device.cuh"
#include "fv_internal.h"

using namespace fvd;

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;   // 2048 threads: a full SM of 256-thread blocks

inline unsigned grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  const long long most = (long long)kBlocksPerSm * fv_sm_count();
  return (unsigned)(b < most ? b : most);
}

// ---------------------------------------------------------------- ghosts
__global__ void __launch_bounds__(kThreads)
k_fill_ghosts(double* __restrict__ U, Params P) {
  const long long total = ring_cells(P);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    fill_ghost_cell(U, P, t);
}

// ---------------------------------------------------------------- copies
__global__ void __launch_bounds__(kThreads)
k_scatter(const double* __restrict__ dense, double* __restrict__ U, Params P) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < NF * n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long q = t / n, m = t - q * n;
    const long long k = m / ((long long)P.nx * P.ny);
    const long long r = m - k * ((long long)P.nx * P.ny);
    const long long j = r / P.nx, i = r - j * P.nx;
    U[q * P.nfield + (k + 2) * P.sz + (j + 2) * P.sy + (i + 2)] = dense[t];
  }
}

__global__ void __launch_bounds__(kThreads)
k_gather(const double* __restrict__ U, double* __restrict__ dense, Params P) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < NF * n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long q = t / n, m = t - q * n;
    const long long k = m / ((long long)P.nx * P.ny);
    const long long r = m - k * ((long long)P.nx * P.ny);
    const long long j = r / P.nx, i = r - j * P.nx;
    dense[t] = U[q * P.nfield + (k + 2) * P.sz + (j + 2) * P.sy + (i + 2)];
  }
}

// ---------------------------------------------------------------- sums
// Fixed pairwise tree over the interior values of each field in (k, j, i)
// order, zero-padded to a power of two P2: level by level a[m] = a[2m] +
// a[2m+1].  A block reduces an aligned chunk of kChunk = 2 * kThreads
// values to one partial -- exactly the tree's level log2(kChunk) node -- and
// further passes reduce the partials the same way, so the result equals the
// whole tree's root bit for bit.
constexpr int kChunk = 2 * kThreads;

__device__ __forceinline__ void block_tree(double* s, int tid) {
  // s holds kThreads level-1 values; finish the tree in shared memory
  for (int len = kThreads; len > 1; len >>= 1) {
    __syncthreads();
    double v = 0.0;
    if (tid < len / 2) v = s[2 * tid] + s[2 * tid + 1];
    __syncthreads();
    if (tid < len / 2) s[tid] = v;
  }
  __syncthreads();
}

// First pass: values straight from the ghosted state; grid = (chunks, 5).
__global__ void __launch_bounds__(kThreads)
k_sum_state(const double* __restrict__ U, Params P, long long padded, double* __restrict__ out,
            long long out_stride) {
  __shared__ double s[kThreads];
  const int q = blockIdx.y, tid = threadIdx.x;
  const long long n = (long long)P.nx * P.ny * P.nz;
  const long long base = (long long)blockIdx.x * kChunk + 2 * tid;
  double v[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const long long m = base + e;
    v[e] = 0.0;
    if (m < n) {
      const long long k = m / ((long long)P.nx * P.ny);
      const long long r = m - k * ((long long)P.nx * P.ny);
      const long long j = r / P.nx, i = r - j * P.nx;
      v[e] = U[q * P.nfield + (k + 2) * P.sz + (j + 2) * P.sy + (i + 2)];
    }
  }
  s[tid] = v[0] + v[1];
  block_tree(s, tid);
  if (tid == 0) out[q * out_stride + blockIdx.x] = s[0];
  (void)padded;
}

// Later passes: `count` values per field (a power of two, or fewer than
// kChunk padded with zeros) -> count / kChunk partials per field.
__global__ void __launch_bounds__(kThreads)
k_sum_partials(const double* __restrict__ in, long long count, long long in_stride,
               double* __restrict__ out, long long out_stride) {
  __shared__ double s[kThreads];
  const int q = blockIdx.y, tid = threadIdx.x;
  const long long base = (long long)blockIdx.x * kChunk + 2 * tid;
  const double a = base < count ? in[q * in_stride + base] : 0.0;
  const double b = base + 1 < count ? in[q * in_stride + base + 1] : 0.0;
  s[tid] = a + b;
  block_tree(s, tid);
  if (tid == 0) out[q * out_stride + blockIdx.x] = s[0];
}

long long next_pow2(long long n) {
  long long p = 1;
  while (p < n) p <<= 1;
  return p;
}

}  // namespace

cudaError_t launch_fill_ghosts(double* U, const Params& P, cudaStream_t s) {
  k_fill_ghosts<<<grid_for(ring_cells(P)), kThreads, 0, s>>>(U, P);
  return cudaGetLastError();
}

cudaError_t launch_scatter_interior(const double* dense, double* U, const Params& P,
                                    cudaStream_t s) {
  k_scatter<<<grid_for(NF * (long long)P.nx * P.ny * P.nz), kThreads, 0, s>>>(dense, U, P);
  return cudaGetLastError();
}

cudaError_t launch_gather_interior(const double* U, double* dense, const Params& P,
                                   cudaStream_t s) {
  k_gather<<<grid_for(NF * (long long)P.nx * P.ny * P.nz), kThreads, 0, s>>>(U, dense, P);
  return cudaGetLastError();
}

size_t sums_work_doubles(const Params& P) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  const long long chunks = (next_pow2(n) + kChunk - 1) / kChunk;
  return (size_t)(2 * NF * chunks + NF);
}

cudaError_t launch_pairwise_sums(const double* U, const Params& P, double* work, double* out5,
                                 cudaStream_t s) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  const long long padded = next_pow2(n);
  long long count = (padded + kChunk - 1) / kChunk;  // partials after pass 1
  const long long stride = count;
  double* a = work;
  double* b = work + NF * stride;
  // pass 1 over the padded range: blocks beyond n read zeros only
  k_sum_state<<<dim3((unsigned)count, NF), kThreads, 0, s>>>(U, P, padded, count == 1 ? out5 : a,
                                                             count == 1 ? 1 : stride);
  while (count > 1) {
    const long long next = (count + kChunk - 1) / kChunk;
    k_sum_partials<<<dim3((unsigned)next, NF), kThreads, 0, s>>>(a, count, stride,
                                                                 next == 1 ? out5 : b,
                                                                 next == 1 ? 1 : stride);
    double* t = a;
    a = b;
    b = t;
    count = next;
  }
  return cudaGetLastError();
}

int fv_sm_count() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < kMaxDevices) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
    return 1;
  if (dev < kMaxDevices) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}
