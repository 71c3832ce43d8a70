// fv_learned.cu -- learned coarse-mesh flux correction: a 3-layer network of
// 3x3x3 convolutions (5 -> 32 -> 32 -> 5 channels, tanh) on the coarse
// mesh's primitives, whose output phi corrects every face flux by the jump
// phi(R) - phi(L); a cell's state changes by minus the divergence of those
// corrections, dU = -sum_d dt/dx_d (phi(i+e_d) - 2 phi(i) + phi(i-e_d)).
// Not in the paper: an extension that lets a coarse mesh approach fine-mesh
// solutions.  Forward and backward passes, the loss and Adam all run in the
// kernels below: BF16 weights and activations, FP32 accumulation, FP32
// gradients, FP64 loss sums.  Periodic meshes only (the shear-layer
// workload); the convolution's padding wraps like the mesh's ghost cells.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_set>
#include <vector>

#include "fv.h"
#include "fv_internal.h"

using bf16 = __nv_bfloat16;

namespace {

constexpr int CIN = 5, CH = 32, COUT = 5;
// flat parameter layout: w1 [CH][CIN][27], b1 [CH], w2 [CH][CH][27], b2 [CH],
// w3 [COUT][CH][27], b3 [COUT]
constexpr int OW1 = 0, OB1 = OW1 + CH * CIN * 27, OW2 = OB1 + CH, OB2 = OW2 + CH * CH * 27,
              OW3 = OB2 + CH, OB3 = OW3 + COUT * CH * 27, NPARAM = OB3 + COUT;
static_assert(NPARAM == 36357, "parameter layout");

constexpr int BX = 8, BY = 8, BZ = 4, BT = BX * BY * BZ;      // 256 cells per tile
constexpr int HX = BX + 2, HY = BY + 2, HZ = BZ + 2, HN = HX * HY * HZ;

struct Grid3 {
  int nx, ny, nz;
  long long n;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(bf16 v) { return __bfloat162float(v); }
template <class T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 from_f<bf16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__host__ __device__ inline int tiles(int n, int b) { return (n + b - 1) / b; }

// Loads the tile's input with a one-cell periodic halo, CI channels.
template <int CI, class TI>
__device__ __forceinline__ void load_tile(const TI* __restrict__ in, TI* s, const Grid3& g, int x0,
                                          int y0, int z0) {
  for (int t = threadIdx.x; t < CI * HN; t += blockDim.x) {
    const int c = t / HN, r = t - c * HN;
    const int lz = r / (HX * HY), ly = (r / HX) % HY, lx = r % HX;
    const int gx = wrap(x0 + lx - 1, g.nx), gy = wrap(y0 + ly - 1, g.ny),
              gz = wrap(z0 + lz - 1, g.nz);
    s[t] = in[c * g.n + ((long long)gz * g.ny + gy) * g.nx + gx];
  }
}

template <int CI, int CO, class TI>
constexpr size_t conv_smem() {
  return (size_t)CI * 27 * CO * sizeof(float) + (size_t)CI * HN * sizeof(TI);
}

// out[co][cell] = act(bias[co] + sum_{ci, o} w[co][ci][o] in[ci][cell + o - 1])
// One thread per cell of an 8x8x4 tile; weights as FP32 in shared memory,
// laid out [ci][o][co] so each thread reads 4 output channels at a time.
template <int CI, int CO, class TI, class TO, bool TANH>
__global__ void __launch_bounds__(BT)
k_conv_fwd(const TI* __restrict__ in, const bf16* __restrict__ w, const float* __restrict__ bias,
           TO* __restrict__ out, Grid3 g) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* ws = reinterpret_cast<float*>(smem);
  TI* is = reinterpret_cast<TI*>(smem + (size_t)CI * 27 * CO * sizeof(float));
  const int ntx = tiles(g.nx, BX), nty = tiles(g.ny, BY);
  const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
  const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;
  for (int t = threadIdx.x; t < CO * CI * 27; t += blockDim.x) {
    const int co = t / (CI * 27), r = t - co * CI * 27;  // r = ci * 27 + o
    ws[r * CO + co] = __bfloat162float(w[t]);
  }
  load_tile<CI, TI>(in, is, g, x0, y0, z0);
  __syncthreads();
  const int lx = threadIdx.x % BX, ly = (threadIdx.x / BX) % BY, lz = threadIdx.x / (BX * BY);
  float acc[CO];
#pragma unroll
  for (int co = 0; co < CO; ++co) acc[co] = bias ? bias[co] : 0.0f;
  for (int ci = 0; ci < CI; ++ci) {
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const int dz = o / 9, dy = (o / 3) % 3, dx = o % 3;
      const float x = to_f(is[ci * HN + ((lz + dz) * HY + (ly + dy)) * HX + (lx + dx)]);
      const float* wp = ws + (ci * 27 + o) * CO;
#pragma unroll
      for (int co = 0; co < CO; ++co) acc[co] = fmaf(wp[co], x, acc[co]);
    }
  }
  const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
  if (gx < g.nx && gy < g.ny && gz < g.nz) {
    const long long cell = ((long long)gz * g.ny + gy) * g.nx + gx;
#pragma unroll
    for (int co = 0; co < CO; ++co) out[co * g.n + cell] = from_f<TO>(TANH ? tanhf(acc[co]) : acc[co]);
  }
}

// Per-tile partial weight gradients: partial[tile][p][co] = sum over the
// tile's cells of gout[co][cell] * in[ci][cell + o - 1], p = ci * 27 + o, and
// p = CI * 27 for the bias (in = 1).  A second kernel sums the tiles in a
// fixed order, so the gradient is deterministic.
template <int CI, int CO, class TI>
__global__ void __launch_bounds__(BT)
k_conv_wgrad(const TI* __restrict__ in, const float* __restrict__ gout,
             float* __restrict__ partial, Grid3 g) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* gs = reinterpret_cast<float*>(smem);  // [CO][BT]
  TI* is = reinterpret_cast<TI*>(smem + (size_t)CO * BT * sizeof(float));
  const int ntx = tiles(g.nx, BX), nty = tiles(g.ny, BY);
  const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
  const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;
  for (int t = threadIdx.x; t < CO * BT; t += blockDim.x) {
    const int co = t / BT, c = t - co * BT;
    const int gx = x0 + c % BX, gy = y0 + (c / BX) % BY, gz = z0 + c / (BX * BY);
    gs[t] = (gx < g.nx && gy < g.ny && gz < g.nz)
                ? gout[co * g.n + ((long long)gz * g.ny + gy) * g.nx + gx]
                : 0.0f;
  }
  load_tile<CI, TI>(in, is, g, x0, y0, z0);
  __syncthreads();
  constexpr int NP = CI * 27 + 1;
  float* dst = partial + (size_t)blockIdx.x * NP * CO;
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    float acc[CO];
#pragma unroll
    for (int co = 0; co < CO; ++co) acc[co] = 0.0f;
    if (p == CI * 27) {
      for (int c = 0; c < BT; ++c)
#pragma unroll
        for (int co = 0; co < CO; ++co) acc[co] += gs[co * BT + c];
    } else {
      const int ci = p / 27, o = p % 27;
      const int dz = o / 9, dy = (o / 3) % 3, dx = o % 3;
      for (int c = 0; c < BT; ++c) {
        const int lx = c % BX, ly = (c / BX) % BY, lz = c / (BX * BY);
        const float x = to_f(is[ci * HN + ((lz + dz) * HY + (ly + dy)) * HX + (lx + dx)]);
#pragma unroll
        for (int co = 0; co < CO; ++co) acc[co] = fmaf(gs[co * BT + c], x, acc[co]);
      }
    }
#pragma unroll
    for (int co = 0; co < CO; ++co) dst[p * CO + co] = acc[co];
  }
}

// Sums the per-tile partials in tile order and scatters them into the flat
// gradient: weights at woff + (co * CI + ci) * 27 + o, biases at boff + co.
template <int CI, int CO>
__global__ void k_wgrad_reduce(const float* __restrict__ partial, int ntiles,
                               float* __restrict__ grads, int woff, int boff) {
  constexpr int NP = CI * 27 + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NP * CO) return;
  float s = 0.0f;
  for (int b = 0; b < ntiles; ++b) s += partial[(size_t)b * NP * CO + t];
  const int p = t / CO, co = t % CO;
  if (p == CI * 27) grads[boff + co] = s;
  else grads[woff + co * CI * 27 + p] = s;
}

// Weights of the adjoint convolution: wt[ci][co][26 - o] = w[co][ci][o].
__global__ void k_flip_weights(const bf16* __restrict__ w, bf16* __restrict__ wt, int CO, int CI) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= CO * CI * 27) return;
  const int co = t / (CI * 27), r = t % (CI * 27), ci = r / 27, o = r % 27;
  wt[(ci * CO + co) * 27 + (26 - o)] = w[t];
}

// Network input: normalised FP32 primitives of the interior cells, as BF16.
__global__ void k_features(const double* __restrict__ U, fvd::Params P, fvd32::Params32 Q,
                           const float* __restrict__ norm /* mean[5], scale[5] */,
                           bf16* __restrict__ x, long long n) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n;
       m += (long long)gridDim.x * blockDim.x) {
    const long long k = m / ((long long)P.nx * P.ny);
    const long long r = m - k * ((long long)P.nx * P.ny);
    const long long j = r / P.nx, i = r - j * P.nx;
    const long long g = (k + 2) * P.sz + (j + 2) * P.sy + (i + 2);
    double u[fvd::NF];
#pragma unroll
    for (int q = 0; q < fvd::NF; ++q) u[q] = U[q * P.nfield + g];
    const fvd32::Prim32 w = fvd32::prim_from_state(u, Q);
    const float v[5] = {w.r, w.vx, w.vy, w.vz, w.p};
#pragma unroll
    for (int q = 0; q < 5; ++q) x[q * n + m] = __float2bfloat16_rn((v[q] - norm[q]) / norm[5 + q]);
  }
}

// dU = -sum_d dt inv_d (phi(i+e) - 2 phi(i) + phi(i-e)), phi = out_scale * o
// (periodic neighbours).  Computes the correction of one channel-cell.
__device__ __forceinline__ float correction(const float* __restrict__ o, float scale, int q,
                                            int i, int j, int k, const Grid3& g, float dt,
                                            const float inv[3]) {
  const long long base = q * g.n;
  auto at = [&](int ii, int jj, int kk) {
    return o[base + ((long long)wrap(kk, g.nz) * g.ny + wrap(jj, g.ny)) * g.nx + wrap(ii, g.nx)];
  };
  const float c = at(i, j, k);
  const float sx = at(i + 1, j, k) - 2.0f * c + at(i - 1, j, k);
  const float sy = at(i, j + 1, k) - 2.0f * c + at(i, j - 1, k);
  const float sz = at(i, j, k + 1) - 2.0f * c + at(i, j, k - 1);
  return -dt * scale * ((inv[0] * sx + inv[1] * sy) + inv[2] * sz);
}

// Loss terms: e = (dU - r) / sigma; per-block partial sums of e^2 (FP64);
// g = dL/d(dU) = 2 e / (sigma N).
__global__ void __launch_bounds__(256)
k_loss(const float* __restrict__ o, const double* __restrict__ r, const float* __restrict__ scales,
       Grid3 g, float dt, float ix, float iy, float iz, float* __restrict__ gdu,
       double* __restrict__ partial) {
  const float inv[3] = {ix, iy, iz};
  const long long total = 5 * g.n;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / g.n);
    const long long m = t - q * g.n;
    const int i = (int)(m % g.nx), j = (int)((m / g.nx) % g.ny), k = (int)(m / ((long long)g.nx * g.ny));
    const float du = correction(o, scales[q], q, i, j, k, g, dt, inv);
    const float sig = scales[5 + q];
    const float e = (du - (float)r[t]) / sig;
    acc += (double)e * (double)e;
    gdu[t] = 2.0f * e / (sig * (float)total);
  }
  __shared__ double s[256];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int len = 128; len > 0; len >>= 1) {
    if (threadIdx.x < len) s[threadIdx.x] += s[threadIdx.x + len];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

// dL/do = out_scale * C^T(g); the periodic stencil is symmetric, C^T = C.
__global__ void __launch_bounds__(256)
k_loss_adjoint(const float* __restrict__ gdu, const float* __restrict__ scales, Grid3 g,
               float dt, float ix, float iy, float iz, float* __restrict__ go) {
  const float inv[3] = {ix, iy, iz};
  const long long total = 5 * g.n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / g.n);
    const long long m = t - q * g.n;
    const int i = (int)(m % g.nx), j = (int)((m / g.nx) % g.ny), k = (int)(m / ((long long)g.nx * g.ny));
    go[t] = correction(gdu, scales[q], q, i, j, k, g, dt, inv);
  }
}

// g *= 1 - h^2 (tanh backward), h the layer's BF16 output
__global__ void k_tanh_bwd(float* __restrict__ g, const bf16* __restrict__ h, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const float y = __bfloat162float(h[t]);
    g[t] *= 1.0f - y * y;
  }
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters; refreshes the BF16
// weight copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ pb, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.0f - b1) * gt;
  const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  const float pt = p[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  p[t] = pt;
  pb[t] = __float2bfloat16_rn(pt);
}

__global__ void k_to_bf16(const float* __restrict__ p, bf16* __restrict__ pb, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) pb[t] = __float2bfloat16_rn(p[t]);
}

// U(interior) += dU (FP32 correction added to the FP64 state)
__global__ void __launch_bounds__(256)
k_apply_correction(double* __restrict__ U, fvd::Params P, const float* __restrict__ o,
                   const float* __restrict__ scales, float dt) {
  const Grid3 g{P.nx, P.ny, P.nz, (long long)P.nx * P.ny * P.nz};
  const float inv[3] = {(float)P.inv_d[0], (float)P.inv_d[1], (float)P.inv_d[2]};
  const long long total = 5 * g.n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / g.n);
    const long long m = t - q * g.n;
    const int i = (int)(m % g.nx), j = (int)((m / g.nx) % g.ny), k = (int)(m / ((long long)g.nx * g.ny));
    const float du = correction(o, scales[q], q, i, j, k, g, dt, inv);
    U[q * P.nfield + (k + 2) * P.sz + (j + 2) * P.sy + (i + 2)] += fvd32::f2d(du);
  }
}

std::mutex g_net_mutex;
std::unordered_set<const void*> g_nets;

fv_status fail(fv_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fv_internal_set_error(buf);
  return st;
}

fv_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

struct fv_net_s {
  int device = 0;
  float* params = nullptr;   // FP32 master
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  bf16* wb = nullptr;        // BF16 copy of all parameters
  bf16* wt2 = nullptr;       // adjoint weights of layers 2 and 3
  bf16* wt3 = nullptr;
  float* scales = nullptr;   // out_scale[5], res_scale[5]
  float* norm = nullptr;     // in_mean[5], in_scale[5]
  long long adam_t = 0;
  // activations sized for `cap` cells
  long long cap = 0, cap_tiles = 0;
  bf16 *x = nullptr, *h1 = nullptr, *h2 = nullptr;
  float *o = nullptr, *gdu = nullptr, *go = nullptr, *g2 = nullptr, *g1 = nullptr;
  float* partial = nullptr;
  double* loss_partial = nullptr;
  double* host_loss = nullptr;
};

namespace {

constexpr int kLossBlocks = 512;

fv_status check(fv_net_t n) {
  if (!n) return fail(FV_ERR_BAD_HANDLE, "NULL network handle");
  std::lock_guard<std::mutex> lk(g_net_mutex);
  if (!g_nets.count(n)) return fail(FV_ERR_BAD_HANDLE, "network handle %p is not live", (void*)n);
  return FV_OK;
}

void free_act(fv_net_s* n) {
  cudaFree(n->x);
  cudaFree(n->h1);
  cudaFree(n->h2);
  cudaFree(n->o);
  cudaFree(n->gdu);
  cudaFree(n->go);
  cudaFree(n->g2);
  cudaFree(n->g1);
  cudaFree(n->partial);
  n->x = n->h1 = n->h2 = nullptr;
  n->o = n->gdu = n->go = n->g2 = n->g1 = n->partial = nullptr;
}

void free_net(fv_net_s* n) {
  free_act(n);
  cudaFree(n->params);
  cudaFree(n->grads);
  cudaFree(n->adam_m);
  cudaFree(n->adam_v);
  cudaFree(n->wb);
  cudaFree(n->wt2);
  cudaFree(n->wt3);
  cudaFree(n->scales);
  cudaFree(n->norm);
  cudaFree(n->loss_partial);
  cudaFreeHost(n->host_loss);
  delete n;
}

long long tile_count(const Grid3& g) {
  return (long long)tiles(g.nx, BX) * tiles(g.ny, BY) * tiles(g.nz, BZ);
}

// Activation and gradient buffers for a mesh of g.n cells (grown on demand).
fv_status ensure_capacity(fv_net_s* n, const Grid3& g) {
  const long long cells = g.n, nt = tile_count(g);
  if (cells <= n->cap && nt <= n->cap_tiles) return FV_OK;
  free_act(n);
  const long long cc = std::max(cells, n->cap), tt = std::max(nt, n->cap_tiles);
  cudaError_t e;
  if ((e = cudaMalloc(&n->x, CIN * cc * sizeof(bf16))) != cudaSuccess ||
      (e = cudaMalloc(&n->h1, CH * cc * sizeof(bf16))) != cudaSuccess ||
      (e = cudaMalloc(&n->h2, CH * cc * sizeof(bf16))) != cudaSuccess ||
      (e = cudaMalloc(&n->o, COUT * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->gdu, COUT * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->go, COUT * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->g2, CH * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->g1, CH * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->partial, tt * (CH * 27 + 1) * CH * sizeof(float))) != cudaSuccess) {
    cudaGetLastError();
    free_act(n);
    return fail(e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA,
                "allocating network activations for %lld cells: %s", cells, cudaGetErrorString(e));
  }
  n->cap = cc;
  n->cap_tiles = tt;
  return FV_OK;
}

template <int CI, int CO, class TI, class TO, bool TANH>
cudaError_t conv_fwd(const TI* in, const bf16* w, const float* bias, TO* out, const Grid3& g,
                     cudaStream_t s) {
  const size_t smem = conv_smem<CI, CO, TI>();
  auto k = k_conv_fwd<CI, CO, TI, TO, TANH>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nb = tiles(g.nx, BX) * tiles(g.ny, BY) * tiles(g.nz, BZ);
  k<<<nb, BT, smem, s>>>(in, w, bias, out, g);
  return cudaGetLastError();
}

template <int CI, int CO, class TI>
cudaError_t conv_wgrad(const TI* in, const float* gout, float* partial, float* grads, int woff,
                       int boff, const Grid3& g, cudaStream_t s) {
  const size_t smem = (size_t)CO * BT * sizeof(float) + (size_t)CI * HN * sizeof(TI);
  auto k = k_conv_wgrad<CI, CO, TI>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nb = tiles(g.nx, BX) * tiles(g.ny, BY) * tiles(g.nz, BZ);
  k<<<nb, BT, smem, s>>>(in, gout, partial, g);
  constexpr int NW = (CI * 27 + 1) * CO;
  k_wgrad_reduce<CI, CO><<<(NW + 255) / 256, 256, 0, s>>>(partial, nb, grads, woff, boff);
  return cudaGetLastError();
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 8 ? (b < 1 ? 1 : b) : 152 * 8);
}

// Forward pass on the mesh's current state: x, h1, h2 and o.
fv_status forward(fv_net_s* n, const MeshView& v, const Grid3& g) {
  fv_status st = ensure_capacity(n, g);
  if (st != FV_OK) return st;
  cudaStream_t s = v.stream;
  k_features<<<grid_for(g.n), 256, 0, s>>>(v.U, v.P, fv_fp32::make_params32(v.P, 0.99), n->norm,
                                           n->x, g.n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = conv_fwd<CIN, CH, bf16, bf16, true>(n->x, n->wb + OW1, n->params + OB1, n->h1, g, s);
  if (e == cudaSuccess)
    e = conv_fwd<CH, CH, bf16, bf16, true>(n->h1, n->wb + OW2, n->params + OB2, n->h2, g, s);
  if (e == cudaSuccess)
    e = conv_fwd<CH, COUT, bf16, float, false>(n->h2, n->wb + OW3, n->params + OB3, n->o, g, s);
  if (e != cudaSuccess) return cuda_fail(e, "network forward pass");
  return FV_OK;
}

fv_status view_periodic(fv_mesh_t m, MeshView* v, Grid3* g) {
  fv_status st = fv_internal_mesh(m, v);
  if (st != FV_OK) return st;
  if (v->P.bc[0] != 1 || v->P.bc[1] != 1 || v->P.bc[2] != 1)
    return fail(FV_ERR_INVALID_ARG, "the learned correction needs a periodic mesh");
  *g = Grid3{v->P.nx, v->P.ny, v->P.nz, (long long)v->P.nx * v->P.ny * v->P.nz};
  return FV_OK;
}

}  // namespace

extern "C" {

fv_status fv_net_create(fv_net_t* out) {
  if (!out) return fail(FV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  fv_net_s* n = new fv_net_s();
  cudaError_t e = cudaGetDevice(&n->device);
  if (e == cudaSuccess) e = cudaMalloc(&n->params, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->grads, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->adam_m, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->adam_v, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->wb, NPARAM * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMalloc(&n->wt2, CH * CH * 27 * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMalloc(&n->wt3, COUT * CH * 27 * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMalloc(&n->scales, 10 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->norm, 10 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->loss_partial, kLossBlocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&n->host_loss, kLossBlocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(n->params, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->grads, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->adam_m, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->adam_v, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->wb, 0, NPARAM * sizeof(bf16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_net(n);
    return cuda_fail(e, "creating the network");
  }
  const float one[10] = {0, 0, 0, 0, 0, 1, 1, 1, 1, 1};
  cudaMemcpy(n->norm, one, sizeof one, cudaMemcpyHostToDevice);
  cudaMemcpy(n->scales, one + 5, 5 * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(n->scales + 5, one + 5, 5 * sizeof(float), cudaMemcpyHostToDevice);
  {
    std::lock_guard<std::mutex> lk(g_net_mutex);
    g_nets.insert(n);
  }
  *out = n;
  return FV_OK;
}

fv_status fv_net_destroy(fv_net_t n) {
  if (!n) return FV_OK;
  {
    std::lock_guard<std::mutex> lk(g_net_mutex);
    if (!g_nets.erase(n)) return fail(FV_ERR_BAD_HANDLE, "network handle %p is not live", (void*)n);
  }
  cudaDeviceSynchronize();
  free_net(n);
  return FV_OK;
}

size_t fv_net_param_count(void) { return NPARAM; }

fv_status fv_net_set_params(fv_net_t n, const float* params) {
  fv_status st = check(n);
  if (st != FV_OK) return st;
  if (!params) return fail(FV_ERR_INVALID_ARG, "params is NULL");
  cudaError_t e = cudaMemcpy(n->params, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_to_bf16<<<(NPARAM + 255) / 256, 256>>>(n->params, n->wb, NPARAM);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemset(n->adam_m, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->adam_v, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  n->adam_t = 0;
  if (e != cudaSuccess) return cuda_fail(e, "fv_net_set_params");
  return FV_OK;
}

fv_status fv_net_get_params(fv_net_t n, float* params, float* grads) {
  fv_status st = check(n);
  if (st != FV_OK) return st;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && params)
    e = cudaMemcpy(params, n->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && grads)
    e = cudaMemcpy(grads, n->grads, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "fv_net_get_params");
  return FV_OK;
}

fv_status fv_net_set_scales(fv_net_t n, const double in_mean[5], const double in_scale[5],
                            const double out_scale[5], const double res_scale[5]) {
  fv_status st = check(n);
  if (st != FV_OK) return st;
  float nm[10], sc[10];
  for (int q = 0; q < 5; ++q) {
    if (!(in_scale[q] > 0) || !(out_scale[q] > 0) || !(res_scale[q] > 0))
      return fail(FV_ERR_INVALID_ARG, "scales must be > 0");
    nm[q] = (float)in_mean[q];
    nm[5 + q] = (float)in_scale[q];
    sc[q] = (float)out_scale[q];
    sc[5 + q] = (float)res_scale[q];
  }
  cudaError_t e = cudaMemcpy(n->norm, nm, sizeof nm, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(n->scales, sc, sizeof sc, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "fv_net_set_scales");
  return FV_OK;
}

fv_status fv_net_forward(fv_net_t n, fv_mesh_t m, float* o_out) {
  fv_status st = check(n);
  if (st != FV_OK) return st;
  MeshView v;
  Grid3 g;
  if ((st = view_periodic(m, &v, &g)) != FV_OK) return st;
  if ((st = forward(n, v, g)) != FV_OK) return st;
  if (o_out) {
    cudaError_t e = cudaMemcpyAsync(o_out, n->o, COUT * g.n * sizeof(float),
                                    cudaMemcpyDeviceToDevice, v.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
    if (e != cudaSuccess) return cuda_fail(e, "copying the network output");
  }
  return FV_OK;
}

fv_status fv_net_train_step(fv_net_t n, fv_mesh_t m, const double* residual, double dt,
                            double lr, double* loss_out) {
  fv_status st = check(n);
  if (st != FV_OK) return st;
  if (!residual || !(dt > 0.0) || !(lr >= 0.0))
    return fail(FV_ERR_INVALID_ARG, "train step needs a residual, dt > 0 and lr >= 0");
  MeshView v;
  Grid3 g;
  if ((st = view_periodic(m, &v, &g)) != FV_OK) return st;
  if ((st = forward(n, v, g)) != FV_OK) return st;
  cudaStream_t s = v.stream;
  const float fdt = (float)dt, ix = (float)v.P.inv_d[0], iy = (float)v.P.inv_d[1],
              iz = (float)v.P.inv_d[2];
  k_loss<<<kLossBlocks, 256, 0, s>>>(n->o, residual, n->scales, g, fdt, ix, iy, iz, n->gdu,
                                     n->loss_partial);
  k_loss_adjoint<<<grid_for(5 * g.n), 256, 0, s>>>(n->gdu, n->scales, g, fdt, ix, iy, iz, n->go);
  cudaError_t e = cudaGetLastError();
  // layer 3: o = conv(h2; w3, b3)
  if (e == cudaSuccess)
    e = conv_wgrad<CH, COUT, bf16>(n->h2, n->go, n->partial, n->grads, OW3, OB3, g, s);
  if (e == cudaSuccess) {
    k_flip_weights<<<(COUT * CH * 27 + 255) / 256, 256, 0, s>>>(n->wb + OW3, n->wt3, COUT, CH);
    e = conv_fwd<COUT, CH, float, float, false>(n->go, n->wt3, nullptr, n->g2, g, s);
  }
  if (e == cudaSuccess) {
    k_tanh_bwd<<<grid_for(CH * g.n), 256, 0, s>>>(n->g2, n->h2, CH * g.n);
    e = conv_wgrad<CH, CH, bf16>(n->h1, n->g2, n->partial, n->grads, OW2, OB2, g, s);
  }
  if (e == cudaSuccess) {
    k_flip_weights<<<(CH * CH * 27 + 255) / 256, 256, 0, s>>>(n->wb + OW2, n->wt2, CH, CH);
    e = conv_fwd<CH, CH, float, float, false>(n->g2, n->wt2, nullptr, n->g1, g, s);
  }
  if (e == cudaSuccess) {
    k_tanh_bwd<<<grid_for(CH * g.n), 256, 0, s>>>(n->g1, n->h1, CH * g.n);
    e = conv_wgrad<CIN, CH, bf16>(n->x, n->g1, n->partial, n->grads, OW1, OB1, g, s);
  }
  if (e == cudaSuccess && lr > 0.0) {
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)n->adam_t), c2 = 1.0f - powf(b2, (float)n->adam_t);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(n->params, n->grads, n->adam_m, n->adam_v, n->wb,
                                                NPARAM, (float)lr, b1, b2, 1e-8f, c1, c2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(n->host_loss, n->loss_partial, kLossBlocks * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "network training step");
  if (loss_out) {
    double L = 0.0;
    for (int b = 0; b < kLossBlocks; ++b) L += n->host_loss[b];
    *loss_out = L / (5.0 * (double)g.n);
  }
  return FV_OK;
}

fv_status fv_step_learned(fv_mesh_t m, fv_net_t n, double dt) {
  fv_status st = check(n);
  if (st != FV_OK) return st;
  MeshView v;
  Grid3 g;
  if ((st = view_periodic(m, &v, &g)) != FV_OK) return st;
  if ((st = forward(n, v, g)) != FV_OK) return st;      // phi from U^n
  if ((st = fv_internal_step(m, dt)) != FV_OK) return st; // RK2 step
  k_apply_correction<<<grid_for(5 * g.n), 256, 0, v.stream>>>(v.U, v.P, n->o, n->scales, (float)dt);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_fill_ghosts(v.U, v.P, v.stream);
  if (e != cudaSuccess) return cuda_fail(e, "applying the learned correction");
  return FV_OK;
}

}  // extern "C"
