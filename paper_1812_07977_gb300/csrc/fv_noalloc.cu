// fv_noalloc.cu -- conservation sums that allocate nothing.
//
// fv_conserved_sums needs a mesh, and creating a mesh allocates device
// memory.  Some callers cannot do that: a host code whose device memory is
// owned by its own allocator under a fixed budget, or a time loop that must
// not pay cudaMalloc's implicit device-wide synchronisation.  For them,
// fv_conserved_sums_noalloc reduces a state they already hold, keeping its
// partial sums in the file-scope device array below, which every GPU that
// loads this library holds until the process exits.
//
// The reduction is the same fixed pairwise tree as fv_conserved_sums (values
// in (k, j, i) order, zero-padded to a power of two, neighbours added level
// by level), so both entry points return identical bits.  Here a block
// reduces an aligned chunk of 2048 values (8 per thread, then a tree in
// shared memory) and later passes reduce the partials the same way.
#include <cstdio>
#include <mutex>

#include "fv.h"
#include "fv_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int kChunk = kThreads * kPerThread;  // 2048 = 2^11
constexpr long long kMaxCells = 1LL << 24;     // 256^3
constexpr int kLevel1 = (int)(kMaxCells / kChunk);  // 8192 partials per field
constexpr int kLevel2 = 8;
// layout: [5 x kLevel1] first-pass partials, [5 x kLevel2] second-pass
// partials, [5] results (padded to a multiple of 8 doubles)
constexpr int kScratchDoubles = 5 * kLevel1 + 5 * kLevel2 + 8;

static __device__ __align__(256) double g_sum_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};

thread_local char g_noalloc_error[256];  // formatted here, then handed to fv_last_error

__device__ __forceinline__ double tree8(const double v[8]) {
  return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
}

__device__ __forceinline__ void block_tree(double* s, int tid) {
  for (int len = kThreads; len > 1; len >>= 1) {
    __syncthreads();
    double v = 0.0;
    if (tid < len / 2) v = s[2 * tid] + s[2 * tid + 1];
    __syncthreads();
    if (tid < len / 2) s[tid] = v;
  }
  __syncthreads();
}

// in: `count` values per field at in[q * in_stride + i]; out: one partial
// per chunk of 2048.  Values past `count` are the tree's zero padding.
__global__ void __launch_bounds__(kThreads)
k_noalloc_pass(const double* __restrict__ in, long long count, long long in_stride,
               double* __restrict__ out, long long out_stride) {
  __shared__ double s[kThreads];
  const int q = blockIdx.y, tid = threadIdx.x;
  const long long base = (long long)blockIdx.x * kChunk + (long long)tid * kPerThread;
  double v[kPerThread];
#pragma unroll
  for (int e = 0; e < kPerThread; ++e)
    v[e] = base + e < count ? in[q * in_stride + base + e] : 0.0;
  s[tid] = tree8(v);
  block_tree(s, tid);
  if (tid == 0) out[q * out_stride + blockIdx.x] = s[0];
}

long long next_pow2(long long n) {
  long long p = 1;
  while (p < n) p <<= 1;
  return p;
}

// Device address of g_sum_scratch on the current device, looked up once.
fv_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    snprintf(g_noalloc_error, sizeof g_noalloc_error, "cudaGetDevice: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    snprintf(g_noalloc_error, sizeof g_noalloc_error, "device %d out of range", dev);
    return FV_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_sum_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(g_noalloc_error, sizeof g_noalloc_error, "cudaGetSymbolAddress: %s",
               cudaGetErrorString(e));
      return FV_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FV_OK;
}

}  // namespace

// Records the detail that fv_last_error() returns on this thread.
static fv_status fail(fv_status st) {
  fv_internal_set_error(g_noalloc_error);
  return st;
}

extern "C" fv_status fv_conserved_sums_noalloc(const double* U, int nx, int ny, int nz,
                                                double lx, double ly, double lz,
                                                void* cuda_stream, double out[5]) {
  if (!U || !out) {
    snprintf(g_noalloc_error, sizeof g_noalloc_error, "U and out must not be NULL");
    return fail(FV_ERR_INVALID_ARG);
  }
  if (nx < 1 || ny < 1 || nz < 1 || !(lx > 0.0) || !(ly > 0.0) || !(lz > 0.0)) {
    snprintf(g_noalloc_error, sizeof g_noalloc_error,
             "cell counts must be >= 1 and extents > 0 (got %d %d %d, %g %g %g)", nx, ny, nz, lx,
             ly, lz);
    return fail(FV_ERR_INVALID_ARG);
  }
  const long long n = (long long)nx * ny * nz;
  if (n > kMaxCells) {
    snprintf(g_noalloc_error, sizeof g_noalloc_error,
             "%lld cells exceed the no-allocation limit of %lld (2^24) cells", n, kMaxCells);
    return fail(FV_ERR_INVALID_ARG);
  }
  double* scratch = nullptr;
  fv_status st = scratch_address(&scratch);
  if (st != FV_OK) return fail(st);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // An error left pending by some earlier, unrelated call is reported as
  // such (and left for its owner), not as a failure of these launches.
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    snprintf(g_noalloc_error, sizeof g_noalloc_error,
             "a CUDA error was pending before the no-allocation sums started: %s",
             cudaGetErrorString(e));
    return fail(FV_ERR_CUDA);
  }
  double* level1 = scratch;
  double* level2 = scratch + 5 * kLevel1;
  double* result = scratch + 5 * kLevel1 + 5 * kLevel2;

  // pass 1 over the zero-padded power-of-two range, straight from U
  long long count = (next_pow2(n) + kChunk - 1) / kChunk;
  k_noalloc_pass<<<dim3((unsigned)count, 5), kThreads, 0, s>>>(
      U, n, n, count == 1 ? result : level1, count == 1 ? 1 : kLevel1);
  e = cudaGetLastError();   // this launch's own error
  double* a = level1;
  long long stride = kLevel1;
  while (count > 1 && e == cudaSuccess) {
    const long long next = (count + kChunk - 1) / kChunk;
    double* dst = next == 1 ? result : level2;
    k_noalloc_pass<<<dim3((unsigned)next, 5), kThreads, 0, s>>>(a, count, stride, dst,
                                                                 next == 1 ? 1 : kLevel2);
    e = cudaGetLastError();
    a = level2;
    stride = kLevel2;
    count = next;
  }
  double host[5];
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, result, sizeof host, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(g_noalloc_error, sizeof g_noalloc_error, "no-allocation sums: %s",
             cudaGetErrorString(e));
    return fail(FV_ERR_CUDA);
  }
  const double vol = ((lx / nx) * (ly / ny)) * (lz / nz);
  for (int q = 0; q < 5; ++q) out[q] = host[q] * vol;
  return FV_OK;
}
