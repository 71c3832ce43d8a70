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
#include <type_traits>
#include <unordered_set>
#include <vector>

#include "fv.h"
#include "fv_internal.h"
#include "fv_umma.cuh"

using bf16 = __nv_bfloat16;

namespace {

constexpr int CIN = 5, CH = 32, COUT = 5;
// flat parameter layout: w1 [CH][CIN][27], b1 [CH], w2 [CH][CH][27], b2 [CH],
// w3 [COUT][CH][27], b3 [COUT]
constexpr int OW1 = 0, OB1 = OW1 + CH * CIN * 27, OW2 = OB1 + CH, OB2 = OW2 + CH * CH * 27,
              OW3 = OB2 + CH, OB3 = OW3 + COUT * CH * 27, NPARAM = OB3 + COUT;
static_assert(NPARAM == 36357, "parameter layout");


struct Grid3 {
  int nx, ny, nz;
  long long n;
};

template <class T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 from_f<bf16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ int wrap(int v, int n) {
  // the tile halos reach at most a few cells past either end: one add or
  // subtract; the remainder (a division) only for meshes shorter than that
  if (v >= -n && v < 2 * n) return v < 0 ? v + n : (v >= n ? v - n : v);
  v %= n;
  return v < 0 ? v + n : v;
}

__host__ __device__ inline int tiles(int n, int b) { return (n + b - 1) / b; }

__device__ __forceinline__ bf16 to_bf(float v) { return __float2bfloat16_rn(v); }

// Activation layouts: channel-first [c][cell] (the network output and the
// loss-side 5-channel gradients) or channel-last [cell][P], P = C rounded up
// to 8 with zero pads (the 32-channel activations, their gradients and the
// input features), where 8 channels of a cell are one 16-byte (BF16) or
// two 16-byte (FP32) loads.
template <int C>
__host__ __device__ constexpr int pitch8() { return (C + 7) / 8 * 8; }

// Channels kc*8 .. kc*8+7 of one cell as 8 BF16 (zero beyond C).
template <int C, bool CL>
__device__ __forceinline__ uint4 gather8(const bf16* __restrict__ in, long long n, long long cell,
                                         int kc) {
  if constexpr (CL) {
    if (kc * 8 >= C) return make_uint4(0u, 0u, 0u, 0u);
    return *reinterpret_cast<const uint4*>(in + cell * pitch8<C>() + kc * 8);
  } else {
    __align__(16) bf16 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = kc * 8 + j;
      v[j] = c < C ? in[c * n + cell] : __float2bfloat16_rn(0.0f);
    }
    return *reinterpret_cast<const uint4*>(v);
  }
}
template <int C, bool CL>
__device__ __forceinline__ uint4 gather8(const float* __restrict__ in, long long n, long long cell,
                                         int kc) {
  __align__(16) bf16 v[8];
  if constexpr (CL) {
    if (kc * 8 >= C) return make_uint4(0u, 0u, 0u, 0u);
    const float4 a = *reinterpret_cast<const float4*>(in + cell * pitch8<C>() + kc * 8);
    const float4 b = *reinterpret_cast<const float4*>(in + cell * pitch8<C>() + kc * 8 + 4);
    v[0] = to_bf(a.x); v[1] = to_bf(a.y); v[2] = to_bf(a.z); v[3] = to_bf(a.w);
    v[4] = to_bf(b.x); v[5] = to_bf(b.y); v[6] = to_bf(b.z); v[7] = to_bf(b.w);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = kc * 8 + j;
      v[j] = c < C ? to_bf(in[c * n + cell]) : __float2bfloat16_rn(0.0f);
    }
  }
  return *reinterpret_cast<const uint4*>(v);
}

// ---------------------------------------------------------------- tcgen05 conv
// out[co][cell] = act(bias[co] + sum_{ci, o} w[co][ci][o] in[ci][cell + o - 1]) as an
// implicit GEMM on the tensor cores: per output plane of a CTA tile, D (128 cells x CO, FP32
// in TMEM) = sum over the 27 offsets o and over 16-channel K steps of A_o (128 x 16) B_o
// (16 x CO), BF16 operands.  The tile's input (8 x 16 x 4 cells plus a one-cell periodic
// halo) sits in shared memory channel-last in 8-channel slabs, [slab][halo cell][8 ch], so
// every A_o is the same no-swizzle K-major layout at a shifted start: 8 consecutive x cells
// form a core matrix, the next row of the tile is one halo row (160 B) further, the next 8
// channels one slab further.  The weights are [offset][slab][co][8 ch] in shared memory.
//
// Persistent CTAs (one per SM) walk the tiles with a two-deep pipeline: two input tiles in
// shared memory and two accumulators in TMEM, so that while the tensor cores run tile i+1's
// MMAs (issued by one thread, completion signalled on an mbarrier), the 12 warps write tile
// i's outputs from TMEM and then gather tile i+2's input.  The weights are copied into shared
// memory once per CTA.
constexpr int UX = 8, UY = 16, UZ = 4;                 // output tile: UZ planes of 128 cells
constexpr int UHX = UX + 2, UHY = UY + 2, UHZ = UZ + 2, UHN = UHX * UHY * UHZ;
constexpr int UThreads = 384;                          // 12 warps: gather and epilogue
constexpr int kMmaPolls = 1 << 20;                     // bounded wait for the MMAs

template <int CI, int CO>
struct UConv {
  static constexpr int CIP = (CI + 15) / 16 * 16;      // K per offset (padded with zeros)
  static constexpr int NP = (CO + 15) / 16 * 16;       // N (padded)
  static constexpr int KC = CIP / 8;                   // 8-channel slabs
  static constexpr size_t in_bytes = (size_t)KC * UHN * 16;
  static constexpr size_t w_bytes = (size_t)27 * KC * NP * 16;
  static constexpr size_t smem = 2 * in_bytes + w_bytes;   // two input tiles, the weights
  static constexpr uint32_t acc_cols = UZ * NP;             // one tile's accumulators
  static constexpr uint32_t tmem_cols = 2 * acc_cols <= 32 ? 32 : 2 * acc_cols <= 64 ? 64 :
                                        2 * acc_cols <= 128 ? 128 : 256;
  static_assert(NP <= 32 && 2 * acc_cols <= 256, "accumulator layout");
  static_assert(smem <= 227 * 1024, "shared memory");
};

// The weights in the convolution's shared-memory layout: entry (o, kc, n) =
// channels kc*8 .. kc*8+7 of w[n][.][o] (zero beyond CI and CO).  Laid out
// once per call, so every CTA copies them with 16-byte loads.
template <int CI, int CO>
__global__ void k_umma_weights(const bf16* __restrict__ w, uint4* __restrict__ wl) {
  using C = UConv<CI, CO>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 27 * C::KC * C::NP) return;
  const int n = t % C::NP, kc = (t / C::NP) % C::KC, o = t / (C::NP * C::KC);
  __align__(16) bf16 v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int ci = kc * 8 + j;
    v[j] = (n < CO && ci < CI) ? w[(n * CI + ci) * 27 + o] : __float2bfloat16_rn(0.0f);
  }
  wl[t] = *reinterpret_cast<const uint4*>(v);
}

__device__ __forceinline__ void tile_origin(int t, const Grid3& g, int& x0, int& y0, int& z0) {
  const int ntx = tiles(g.nx, UX), nty = tiles(g.ny, UY);
  x0 = (t % ntx) * UX;
  y0 = ((t / ntx) % nty) * UY;
  z0 = (t / (ntx * nty)) * UZ;
}

// Asynchronous 16-byte copy global -> shared (L2 only), and the wait for all
// of this thread's copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(umma::smem_addr(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// The input tile at (x0, y0, z0) with its periodic one-cell halo, as BF16 slabs.
// Channel-last BF16 inputs are copied asynchronously (16 bytes per cell and
// slab, already in the slab layout): the caller waits with cp_async_wait_all
// before the tile is used; other inputs are converted on the way, in place.
template <int CI, int KC, class TI, bool ICL>
__device__ __forceinline__ void gather_tile(uint4* xs, const TI* __restrict__ in, const Grid3& g,
                                            int x0, int y0, int z0) {
  constexpr bool async = ICL && std::is_same<TI, bf16>::value;
#pragma unroll 4
  for (int t = threadIdx.x; t < KC * UHN; t += UThreads) {
    const int c = t % UHN, kc = t / UHN;
    const int lz = c / (UHX * UHY), ly = (c / UHX) % UHY, lx = c % UHX;
    const long long cell = ((long long)wrap(z0 + lz - 1, g.nz) * g.ny + wrap(y0 + ly - 1, g.ny)) *
                               g.nx + wrap(x0 + lx - 1, g.nx);
    if constexpr (async) {
      if (kc * 8 < CI)
        cp_async16(&xs[t], in + cell * pitch8<CI>() + kc * 8);
      else
        xs[t] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      xs[t] = gather8<CI, ICL>(in, g.n, cell, kc);
    }
  }
}

// One tile's MMAs (one thread): plane z accumulates into columns acc + z * NP.
// The descriptors are formed once; a shifted operand is the base descriptor
// plus its byte offset / 16 (the start-address field is the low 14 bits, and
// every address here is below 256 KB), so the issuing thread spends one add
// per operand on each MMA.
// Planes are issued by UZ threads (lane 0 of warps 0 .. UZ-1, one per SM
// sub-partition), each committing to the tile's mbarrier (arrival count UZ).
template <int CI, int CO>
__device__ __forceinline__ void plane_mmas(uint32_t xa, uint32_t wa, uint32_t acc, int z) {
  using C = UConv<CI, CO>;
  constexpr uint32_t idesc = umma::idesc_bf16(128, C::NP);
  const uint64_t a0 = umma::desc(xa, UHN * 16, UHX * 16);
  const uint64_t b0 = umma::desc(wa, C::NP * 16, 128);
  const uint64_t az = a0 + (uint64_t)(z * UHY * UHX);
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int dz = o / 9, dy = (o / 3) % 3, dx = o % 3;
#pragma unroll
    for (int kk = 0; kk < C::CIP / 16; ++kk) {
      const uint64_t a = az + (uint64_t)((2 * kk) * UHN + (dz * UHY + dy) * UHX + dx);
      const uint64_t b = b0 + (uint64_t)((o * C::KC + 2 * kk) * C::NP);
      umma::mma_bf16(acc + z * C::NP, a, b, idesc, (o > 0 || kk > 0) ? 1u : 0u);
    }
  }
}

template <int CI, int CO, class TI, class TO, bool TANH, bool ICL, bool OCL>
__global__ void __launch_bounds__(UThreads, 1)
k_conv_umma(const TI* __restrict__ in, const uint4* __restrict__ wl,
            const float* __restrict__ bias, TO* __restrict__ out, Grid3 g,
            unsigned* __restrict__ status) {
  using C = UConv<CI, CO>;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint4* xs[2] = {reinterpret_cast<uint4*>(smem), reinterpret_cast<uint4*>(smem + C::in_bytes)};
  uint4* ws = reinterpret_cast<uint4*>(smem + 2 * C::in_bytes);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = tiles(g.nx, UX) * tiles(g.ny, UY) * tiles(g.nz, UZ);
  int t = blockIdx.x;
  if (t >= ntiles) return;   // (the grid has at most one CTA per tile)
#pragma unroll 4
  for (int i = tid; i < 27 * C::KC * C::NP; i += UThreads) ws[i] = wl[i];
  int x0, y0, z0;
  tile_origin(t, g, x0, y0, z0);
  gather_tile<CI, C::KC, TI, ICL>(xs[0], in, g, x0, y0, z0);
  cp_async_wait_all();
  if (tid == 0) {
    umma::mbar_init(&mbar[0], UZ);
    umma::mbar_init(&mbar[1], UZ);
  }
  if (warp == 0) umma::tmem_alloc(&tmem_slot, C::tmem_cols);
  umma::fence_smem_for_mma();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t wa = umma::smem_addr(ws);
  const uint32_t xa[2] = {umma::smem_addr(xs[0]), umma::smem_addr(xs[1])};
  const bool issuer = lane == 0 && warp < UZ;
  if (issuer) {
    plane_mmas<CI, CO>(xa[0], wa, tmem, warp);
    umma::commit(&mbar[0]);
  }
  // the epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (accumulator row m = cell
  // (m % 8, m / 8) of a plane); the three warps of a lane quarter split its 16-column chunks
  const int quarter = warp & 3, group = warp >> 2;
  const int m = quarter * 32 + lane;
  constexpr int HALVES = C::NP / 16;
  for (int i = 0;; ++i) {
    const int b = i & 1;
    const int tn = t + (int)gridDim.x;
    int nx0 = 0, ny0 = 0, nz0 = 0;
    if (tn < ntiles) {
      // the next tile's input, into the buffer its MMAs will read (free: the MMAs
      // that last read it were waited for in the previous iteration)
      tile_origin(tn, g, nx0, ny0, nz0);
      gather_tile<CI, C::KC, TI, ICL>(xs[b ^ 1], in, g, nx0, ny0, nz0);
    }
    const bool ok = umma::mbar_wait(&mbar[b], (uint32_t)((i >> 1) & 1), kMmaPolls);
    cp_async_wait_all();   // this thread's copies of the next tile have landed
    umma::fence_smem_for_mma();
    umma::fence_before_sync();
    const int all_ok = __syncthreads_and(ok);
    umma::fence_after_sync();
    if (!all_ok) {
      if (tid == 0) atomicOr(status, 1u);
      // let this tile's MMAs drain (bounded) before the accumulators are freed
      umma::mbar_wait(&mbar[b], (uint32_t)((i >> 1) & 1), kMmaPolls);
      break;
    }
    if (issuer && tn < ntiles) {
      plane_mmas<CI, CO>(xa[b ^ 1], wa, tmem + (uint32_t)(b ^ 1) * C::acc_cols, warp);
      umma::commit(&mbar[b ^ 1]);
    }
    const uint32_t acc = tmem + (uint32_t)b * C::acc_cols + ((uint32_t)(quarter * 32) << 16);
    const int gx = x0 + m % UX, gy = y0 + m / UX;
#pragma unroll 1
    for (int c = group; c < UZ * HALVES; c += 3) {
      const int z = c / HALVES, h = c % HALVES;
      float v[16];
      umma::ld16(acc + z * C::NP + h * 16, v);
      const int gz = z0 + z;
      if (gx < g.nx && gy < g.ny && gz < g.nz) {
        const long long cell = ((long long)gz * g.ny + gy) * g.nx + gx;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int co = h * 16 + j;
          if (co < CO) {
            const float a = v[j] + (bias ? bias[co] : 0.0f);
            v[j] = TANH ? tanhf(a) : a;
          }
        }
        if constexpr (OCL) {
          // the chunk's channels as 16-byte stores ([cell][pitch], zero pads)
          static_assert(sizeof(TO) == 2 || sizeof(TO) == 4, "output type");
          constexpr int P = pitch8<CO>(), PER = 16 / (int)sizeof(TO);
          const int nch = min(16, P - h * 16);
          uint4* dst = reinterpret_cast<uint4*>(out + cell * P + h * 16);
#pragma unroll
          for (int q = 0; q < 16 / PER; ++q) {
            if (q * PER < nch) {
              __align__(16) TO w[PER];
#pragma unroll
              for (int e = 0; e < PER; ++e)
                w[e] = from_f<TO>(h * 16 + q * PER + e < CO ? v[q * PER + e] : 0.0f);
              dst[q] = *reinterpret_cast<const uint4*>(w);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (h * 16 + j < CO) out[(h * 16 + j) * g.n + cell] = from_f<TO>(v[j]);
        }
      }
    }
    if (tn >= ntiles) break;
    t = tn;
    x0 = nx0;
    y0 = ny0;
    z0 = nz0;
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_free(tmem, C::tmem_cols);
}

// ---------------------------------------------------------------- tcgen05 weight gradient
// Per tile of the convolution's 8 x 16 x 4 output cells, the partial weight
// gradients partial[tile][p][co], p = ci * 27 + o,
//   sum over the tile's cells c of gout[co][c] * in[ci][c + o - 1],
// as one GEMM per offset o on the tensor cores, D_o[co][ci] += A[co][c] B_o[c][ci],
// K = the 128 cells of a plane, 16 per MMA, over the tile's four planes:
//   A = the tile's output gradient, BF16 slabs [co slab][cell][8 co] (MN-major:
//       8 output channels of a cell are one 16-byte row), M = 128 rows of which
//       the first CO are the output channels (the rest read whatever follows
//       in shared memory and land in TMEM lanes that are never read);
//   B_o = the input tile in the convolution's layout [ci slab][halo cell][8 ci]
//       (MN-major) at the start shifted by the offset: 8 x-consecutive cells
//       are 16 bytes apart and the next 8 cells of the plane are one halo row
//       (160 B) further, so every offset's operand is addressed in place, with
//       no copy.
// The 27 accumulators (N = CI padded to 16 or 32 columns each) take at most
// two passes over TMEM's 512 columns; one thread issues every MMA of a pass,
// commits them to an mbarrier, and warps 0, 4 and 8 (TMEM lanes 0..31, the
// output channels) write the pass's partials.  Bias gradients (sum of gout
// over the tile) are summed in FP32.
template <int CI, int CO>
struct UWgrad {
  static constexpr int NPC = CI <= 16 ? 16 : 32;   // N: input channels, padded
  static constexpr int KC = NPC / 8;               // input slabs
  static constexpr int PC = UX * UY;               // cells of a plane (K of a plane)
  static constexpr int TC = PC * UZ;               // cells of the tile
  static constexpr int GS = (CO + 7) / 8;          // output-gradient slabs
  static constexpr size_t g_slab = (size_t)TC * 16;
  static constexpr size_t x_off = (size_t)GS * g_slab;        // input tile after the slabs
  static constexpr size_t x_bytes = (size_t)KC * UHN * 16;
  static constexpr size_t a_span = 16 * g_slab;                // what M = 128 rows address
  static constexpr size_t smem = x_off + x_bytes > a_span ? x_off + x_bytes : a_span;
  static constexpr int OPP = 512 / NPC;            // offsets per pass
  static constexpr int NPASS = (27 + OPP - 1) / OPP;
  static_assert(CO <= 32 && CI <= 32 && smem <= 227 * 1024, "layout");
};

template <int CI, int CO, class TI, bool ICL, bool GCL>
__global__ void __launch_bounds__(UThreads)
k_wgrad_umma(const TI* __restrict__ in, const float* __restrict__ gout,
             float* __restrict__ partial, Grid3 g, unsigned* __restrict__ status) {
  using C = UWgrad<CI, CO>;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint4* gs = reinterpret_cast<uint4*>(smem);
  uint4* xs = reinterpret_cast<uint4*>(smem + C::x_off);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ float bsum[UThreads / 32][32];
  __shared__ float bthr[GCL ? UThreads : 1][8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int x0, y0, z0;
  tile_origin(blockIdx.x, g, x0, y0, z0);
  // input halo tile (periodic) as BF16 slabs [kc][halo cell][8 ch]
  gather_tile<CI, C::KC, TI, ICL>(xs, in, g, x0, y0, z0);
  // output gradients of the tile's cells (0 outside the mesh) as BF16 slabs
  // [co slab][cell][8 co]; cell = (z * UY + y) * UX + x.  Channel-last
  // gradients: item t is slab t % GS of cell t / GS, so a thread always
  // handles the same slab (UThreads is a multiple of GS) and neighbouring
  // threads read neighbouring 32-byte pieces; the thread also sums its 8
  // channels in FP32 for the bias gradients.
  static_assert(UThreads % C::GS == 0, "slab per thread");
  float bpart[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
  for (int t = tid; t < C::GS * C::TC; t += UThreads) {
    const int c = GCL ? t / C::GS : t % C::TC, cs = GCL ? t % C::GS : t / C::TC;
    const int gx = x0 + c % UX, gy = y0 + (c / UX) % UY, gz = z0 + c / C::PC;
    const bool in_mesh = gx < g.nx && gy < g.ny && gz < g.nz;
    const long long cell = ((long long)gz * g.ny + gy) * g.nx + gx;
    if constexpr (GCL) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (in_mesh) {
        const float* p = gout + cell * pitch8<CO>() + cs * 8;
        const float4 a = *reinterpret_cast<const float4*>(p);
        const float4 b = *reinterpret_cast<const float4*>(p + 4);
        const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        __align__(16) bf16 h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          bpart[j] += f[j];
          h[j] = to_bf(f[j]);
        }
        v = *reinterpret_cast<const uint4*>(h);
      }
      gs[cs * C::TC + c] = v;
    } else {
      gs[t] = in_mesh ? gather8<CO, GCL>(gout, g.n, cell, cs) : make_uint4(0u, 0u, 0u, 0u);
    }
  }
  // bias gradients in FP32, in a fixed order.  Channel-last gradients: each
  // thread's 8 channel sums go to shared memory, and the threads of a slab
  // are added in thread order below.  Channel-first: warp w sums output
  // co = w, w + 12, ... over the tile's cells (lanes along the cells, then a
  // shuffle tree).
  if constexpr (GCL) {
#pragma unroll
    for (int j = 0; j < 8; ++j) bthr[tid][j] = bpart[j];
  } else {
    for (int co = warp; co < CO; co += UThreads / 32) {
      float acc = 0.0f;
      for (int c = lane; c < C::TC; c += 32) {
        const int gx = x0 + c % UX, gy = y0 + (c / UX) % UY, gz = z0 + c / C::PC;
        if (gx < g.nx && gy < g.ny && gz < g.nz) {
          const long long cell = ((long long)gz * g.ny + gy) * g.nx + gx;
          acc += gout[co * g.n + cell];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) bsum[warp][co / (UThreads / 32)] = acc;
    }
  }
  cp_async_wait_all();
  constexpr int kIssuers = 4;   // lane 0 of warps 0 .. 3 issue the offsets o0 + w, + 4, ...
  if (tid == 0) umma::mbar_init(&mbar, kIssuers);
  if (warp == 0) umma::tmem_alloc(&tmem_slot, 512);
  umma::fence_smem_for_mma();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  constexpr uint32_t idesc = umma::idesc_bf16(128, C::NPC) | (1u << 15) | (1u << 16);  // MN-major
  float* dst = partial + (size_t)blockIdx.x * (CI * 27 + 1) * CO;
  bool ok = true;
  int issued = 0;   // passes whose MMAs were issued
  for (int pass = 0; pass < C::NPASS; ++pass) {
    const int o0 = pass * C::OPP, o1 = min(27, o0 + C::OPP);
    if (lane == 0 && warp < kIssuers) {
      // base descriptors plus byte offsets / 16 (see plane_mmas)
      const uint64_t a0 = umma::desc(umma::smem_addr(gs), 128, C::TC * 16);
      const uint64_t b0 = umma::desc(umma::smem_addr(xs), UHX * 16, UHN * 16);
#pragma unroll 1
      for (int o = o0 + warp; o < o1; o += kIssuers) {
        const int dz = o / 9, dy = (o / 3) % 3, dx = o % 3;
        const uint64_t bo = b0 + (uint64_t)((dz * UHY + dy) * UHX + dx);
        const uint32_t d = tmem + (uint32_t)((o - o0) * C::NPC);
#pragma unroll
        for (int z = 0; z < UZ; ++z) {
#pragma unroll
          for (int ks = 0; ks < C::PC / 16; ++ks) {
            // cells ks*16 .. +15 of plane z: rows y = 2 ks, 2 ks + 1 of the tile
            const uint64_t a = a0 + (uint64_t)(z * C::PC + ks * 16);
            const uint64_t b = bo + (uint64_t)((z * UHY + 2 * ks) * UHX);
            umma::mma_bf16(d, a, b, idesc, (z > 0 || ks > 0) ? 1u : 0u);
          }
        }
      }
      umma::commit(&mbar);
    }
    issued = pass + 1;
    ok = __syncthreads_and(umma::mbar_wait(&mbar, (uint32_t)(pass & 1), kMmaPolls)) != 0;
    umma::fence_after_sync();
    if (!ok) break;
    if ((warp & 3) == 0) {
      // lane = output channel; column (o - o0) * NPC + ci
      const int q = warp >> 2;   // 0, 1, 2: offsets o0 + q, o0 + q + 3, ...
#pragma unroll 1
      for (int o = o0 + q; o < o1; o += 3) {
        float v[32];
        const uint32_t ta = tmem + (uint32_t)((o - o0) * C::NPC);
        umma::ld16(ta, v);
        if (C::NPC > 16) umma::ld16(ta + 16, v + 16);
        if (lane < CO) {
#pragma unroll
          for (int ci = 0; ci < CI; ++ci) dst[(ci * 27 + o) * CO + lane] = v[ci];
        }
      }
    }
    // the pass's accumulators are read before the next pass overwrites them
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, 1u);
    // let the MMAs of the last issued pass drain (bounded) before TMEM is freed
    umma::mbar_wait(&mbar, (uint32_t)((issued - 1) & 1), kMmaPolls);
  }
  if (tid < CO) {
    float b;
    if constexpr (GCL) {
      // output co is channel co % 8 of slab co / 8: threads co / 8, + GS, ...
      b = 0.0f;
      for (int r = tid / 8; r < UThreads; r += C::GS) b += bthr[r][tid % 8];
    } else {
      b = bsum[tid % (UThreads / 32)][tid / (UThreads / 32)];
    }
    dst[(CI * 27) * CO + tid] = b;
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_free(tmem, 512);
}

// Sums the per-tile partials and scatters them into the flat gradient:
// weights at woff + (co * CI + ci) * 27 + o, biases at boff + co.  A block
// covers 32 outputs with 8 warps; warp w sums tiles w, w + 8, ... (in order,
// one coalesced row of 32 outputs per load) and the 8 warp sums are added in
// warp order: the same bits every call.
template <int CI, int CO>
__global__ void __launch_bounds__(256)
k_wgrad_reduce(const float* __restrict__ partial, int ntiles, float* __restrict__ grads,
               int woff, int boff) {
  constexpr int NP = CI * 27 + 1;
  __shared__ float ws[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  float a = 0.0f;
  if (t < NP * CO)
    for (int b = w; b < ntiles; b += 8) a += partial[(size_t)b * NP * CO + t];
  ws[w][lane] = a;
  __syncthreads();
  if (w == 0 && t < NP * CO) {
    float s = ws[0][lane];
#pragma unroll
    for (int r = 1; r < 8; ++r) s += ws[r][lane];
    const int p = t / CO, co = t % CO;
    if (p == CI * 27) grads[boff + co] = s;
    else grads[woff + co * CI * 27 + p] = s;
  }
}

// The loss from the loss kernel's N block partials, in a fixed order that
// the host (loss_from_partials) and the device (k_loss_accumulate) share: 32
// runs of N / 32 consecutive partials, each summed in order, then the 32 run
// sums in order.
constexpr int kLossRuns = 32;

// acc += loss / denom: the value a synchronous step reports, added to the
// running sum; one warp, lane l summing run l.
template <int N>
__global__ void __launch_bounds__(32)
k_loss_accumulate(const double* __restrict__ partial, double denom, double* __restrict__ acc) {
  static_assert(N % kLossRuns == 0, "runs");
  constexpr int R = N / kLossRuns;
  __shared__ double run[kLossRuns];
  double t = 0.0;
  for (int j = 0; j < R; ++j) t += partial[threadIdx.x * R + j];
  run[threadIdx.x] = t;
  __syncwarp();
  if (threadIdx.x == 0) {
    double L = 0.0;
    for (int l = 0; l < kLossRuns; ++l) L += run[l];
    *acc += L / denom;
  }
}

double loss_from_partials(const double* p, int n) {
  const int R = n / kLossRuns;
  double L = 0.0;
  for (int l = 0; l < kLossRuns; ++l) {
    double t = 0.0;
    for (int j = 0; j < R; ++j) t += p[l * R + j];
    L += t;
  }
  return L;
}

// Weights of the adjoint convolution: wt[ci][co][26 - o] = w[co][ci][o].
__global__ void k_flip_weights(const bf16* __restrict__ w, bf16* __restrict__ wt, int CO, int CI) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= CO * CI * 27) return;
  const int co = t / (CI * 27), r = t % (CI * 27), ci = r / 27, o = r % 27;
  wt[(ci * CO + co) * 27 + (26 - o)] = w[t];
}

// Network input: normalised FP32 primitives of the interior cells, as BF16,
// channel-last with three zero pads ([cell][8]).
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
    __align__(16) bf16 f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      f[q] = __float2bfloat16_rn(q < 5 ? (v[q] - norm[q]) / norm[5 + q] : 0.0f);
    reinterpret_cast<uint4*>(x)[m] = *reinterpret_cast<const uint4*>(f);
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

// (channel q, cell i, j, k) of flat index t = q n + (k ny + j) nx + i, in 32-bit
// arithmetic when every index fits (the 64-bit divisions are long sequences)
__device__ __forceinline__ void split_index(long long t, const Grid3& g, int& q, int& i, int& j,
                                            int& k) {
  if (5LL * g.n <= 0x7FFFFFFFLL) {
    const unsigned u = (unsigned)t, n = (unsigned)g.n, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
    const unsigned qq = u / n, m = u - qq * n, r = m / nx, kk = r / ny;
    q = (int)qq;
    i = (int)(m - r * nx);
    j = (int)(r - kk * ny);
    k = (int)kk;
  } else {
    q = (int)(t / g.n);
    const long long m = t - q * g.n;
    i = (int)(m % g.nx);
    j = (int)((m / g.nx) % g.ny);
    k = (int)(m / ((long long)g.nx * g.ny));
  }
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
    int q, i, j, k;
    split_index(t, g, q, i, j, k);
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
               float dt, float ix, float iy, float iz, float* __restrict__ go,
               bf16* __restrict__ gob) {
  const float inv[3] = {ix, iy, iz};
  const long long total = 5 * g.n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int q, i, j, k;
    split_index(t, g, q, i, j, k);
    const float v = correction(gdu, scales[q], q, i, j, k, g, dt, inv);
    go[t] = v;
    // the BF16 channel-last copy the adjoint convolution reads ([cell][8],
    // pads zero from allocation): the value its gather would round to
    gob[(t - (long long)q * g.n) * pitch8<5>() + q] = to_bf(v);
  }
}

// g *= 1 - h^2 (tanh backward), h the layer's BF16 output; gb (if given):
// the result rounded to BF16 in the same layout, for the next convolution
__global__ void k_tanh_bwd_bf(float* __restrict__ g, const bf16* __restrict__ h,
                              bf16* __restrict__ gb, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const float y = __bfloat162float(h[t]);
    const float v = g[t] * (1.0f - y * y);
    g[t] = v;
    gb[t] = to_bf(v);
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
    int q, i, j, k;
    split_index(t, g, q, i, j, k);
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
  bf16 *gob = nullptr, *g2b = nullptr;   // BF16 channel-last copies for the adjoint convs
  float* partial = nullptr;
  double* loss_partial = nullptr;
  double* host_loss = nullptr;
  double* loss_acc = nullptr;       // device: losses of the asynchronous steps, summed
  long long acc_steps = 0;          // steps in loss_acc
  uint4* wlay = nullptr;            // laid-out weights of the convolution being run
  unsigned* status = nullptr;       // device: set by a convolution whose MMA wait ran out
  unsigned* host_status = nullptr;  // pinned mirror
  // the last pass: its mesh's cell count and stream, and whether the
  // gradient buffers hold a training step's values
  long long last_cells = 0;
  cudaStream_t last_stream = nullptr;
  bool have_grads = false;
};

namespace {

constexpr int kLossBlocks = 512;

fv_status check(fv_net_t n) {
  if (!n) return fail(FV_ERR_BAD_HANDLE, "NULL network handle");
  std::lock_guard<std::mutex> lk(g_net_mutex);
  if (!g_nets.count(n)) return fail(FV_ERR_BAD_HANDLE, "network handle %p is not live", (void*)n);
  return FV_OK;
}

// Reports (and clears) a convolution whose tensor-core wait ran out; the
// caller has copied the device word to host_status and synchronised.
fv_status take_status(fv_net_s* n, cudaStream_t s) {
  if (*n->host_status == 0u) return FV_OK;
  *n->host_status = 0u;
  cudaMemsetAsync(n->status, 0, sizeof(unsigned), s);
  return fail(FV_ERR_TIMEOUT, "a tensor-core convolution did not complete within its wait limit");
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
  cudaFree(n->gob);
  cudaFree(n->g2b);
  cudaFree(n->partial);
  n->x = n->h1 = n->h2 = nullptr;
  n->o = n->gdu = n->go = n->g2 = n->g1 = n->partial = nullptr;
  n->gob = n->g2b = nullptr;
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
  cudaFree(n->loss_acc);
  cudaFree(n->status);
  cudaFreeHost(n->host_status);
  cudaFree(n->wlay);
  delete n;
}

// tiles of the tensor-core kernels (one partial-gradient block each)
long long tile_count(const Grid3& g) {
  return (long long)tiles(g.nx, UX) * tiles(g.ny, UY) * tiles(g.nz, UZ);
}

// Activation and gradient buffers for a mesh of g.n cells (grown on demand).
fv_status ensure_capacity(fv_net_s* n, const Grid3& g) {
  const long long cells = g.n, nt = tile_count(g);
  if (cells <= n->cap && nt <= n->cap_tiles) return FV_OK;
  free_act(n);
  const long long cc = std::max(cells, n->cap), tt = std::max(nt, n->cap_tiles);
  cudaError_t e;
  if ((e = cudaMalloc(&n->x, pitch8<CIN>() * cc * sizeof(bf16))) != cudaSuccess ||
      (e = cudaMalloc(&n->h1, CH * cc * sizeof(bf16))) != cudaSuccess ||
      (e = cudaMalloc(&n->h2, CH * cc * sizeof(bf16))) != cudaSuccess ||
      (e = cudaMalloc(&n->o, COUT * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->gdu, COUT * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->go, COUT * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->g2, CH * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->g1, CH * cc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&n->gob, pitch8<COUT>() * cc * sizeof(bf16))) != cudaSuccess ||
      (e = cudaMemset(n->gob, 0, pitch8<COUT>() * cc * sizeof(bf16))) != cudaSuccess ||
      (e = cudaMalloc(&n->g2b, CH * cc * sizeof(bf16))) != cudaSuccess ||
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

// wl: scratch for the laid-out weights (at least UConv<CI, CO>::w_bytes)
template <int CI, int CO, class TI, class TO, bool TANH, bool ICL, bool OCL>
cudaError_t conv_fwd(const TI* in, const bf16* w, const float* bias, TO* out, const Grid3& g,
                     uint4* wl, unsigned* status, cudaStream_t s) {
  using C = UConv<CI, CO>;
  const int nw = 27 * C::KC * C::NP;
  k_umma_weights<CI, CO><<<(nw + 255) / 256, 256, 0, s>>>(w, wl);
  const size_t smem = C::smem;
  auto k = k_conv_umma<CI, CO, TI, TO, TANH, ICL, OCL>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nt = tiles(g.nx, UX) * tiles(g.ny, UY) * tiles(g.nz, UZ);
  const int nb = nt < fv_sm_count() ? nt : fv_sm_count();   // persistent: one CTA per SM
  k<<<nb, UThreads, smem, s>>>(in, wl, bias, out, g, status);
  return cudaGetLastError();
}

// Weight gradients of one convolution: per-tile partials on the tensor
// cores, then the fixed-order sum over tiles.
template <int CI, int CO, class TI, bool ICL, bool GCL>
cudaError_t conv_wgrad(const TI* in, const float* gout, float* partial, float* grads, int woff,
                       int boff, const Grid3& g, unsigned* status, cudaStream_t s) {
  const size_t smem = UWgrad<CI, CO>::smem;
  auto k = k_wgrad_umma<CI, CO, TI, ICL, GCL>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nb = tiles(g.nx, UX) * tiles(g.ny, UY) * tiles(g.nz, UZ);
  k<<<nb, UThreads, smem, s>>>(in, gout, partial, g, status);
  constexpr int NW = (CI * 27 + 1) * CO;
  k_wgrad_reduce<CI, CO><<<(NW + 31) / 32, 256, 0, s>>>(partial, nb, grads, woff, boff);
  return cudaGetLastError();
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  const long long most = 8LL * fv_sm_count();
  return (unsigned)(b < most ? (b < 1 ? 1 : b) : most);
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
    e = conv_fwd<CIN, CH, bf16, bf16, true, true, true>(n->x, n->wb + OW1, n->params + OB1, n->h1, g,
                                            n->wlay, n->status, s);
  if (e == cudaSuccess)
    e = conv_fwd<CH, CH, bf16, bf16, true, true, true>(n->h1, n->wb + OW2, n->params + OB2, n->h2, g,
                                           n->wlay, n->status, s);
  if (e == cudaSuccess)
    e = conv_fwd<CH, COUT, bf16, float, false, true, false>(n->h2, n->wb + OW3, n->params + OB3, n->o, g,
                                               n->wlay, n->status, s);
  if (e != cudaSuccess) return cuda_fail(e, "network forward pass");
  n->last_cells = g.n;
  n->last_stream = s;
  n->have_grads = false;
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
  if (e == cudaSuccess) e = cudaMalloc(&n->loss_acc, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(n->loss_acc, 0, sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&n->host_loss, kLossBlocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&n->status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&n->wlay, UConv<CH, CH>::w_bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&n->host_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(n->status, 0, sizeof(unsigned));
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
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(n->host_status, n->status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                          v.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
    if (e != cudaSuccess) return cuda_fail(e, "copying the network output");
    if ((st = take_status(n, v.stream)) != FV_OK) return st;
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
  k_loss_adjoint<<<grid_for(5 * g.n), 256, 0, s>>>(n->gdu, n->scales, g, fdt, ix, iy, iz, n->go,
                                                   n->gob);
  cudaError_t e = cudaGetLastError();
  // layer 3: o = conv(h2; w3, b3)
  if (e == cudaSuccess)
    e = conv_wgrad<CH, COUT, bf16, true, false>(n->h2, n->go, n->partial, n->grads, OW3, OB3, g, n->status, s);
  if (e == cudaSuccess) {
    k_flip_weights<<<(COUT * CH * 27 + 255) / 256, 256, 0, s>>>(n->wb + OW3, n->wt3, COUT, CH);
    e = conv_fwd<COUT, CH, bf16, float, false, true, true>(n->gob, n->wt3, nullptr, n->g2, g, n->wlay,
                                                n->status, s);
  }
  if (e == cudaSuccess) {
    k_tanh_bwd_bf<<<grid_for(CH * g.n), 256, 0, s>>>(n->g2, n->h2, n->g2b, CH * g.n);
    e = conv_wgrad<CH, CH, bf16, true, true>(n->h1, n->g2, n->partial, n->grads, OW2, OB2, g, n->status, s);
  }
  if (e == cudaSuccess) {
    k_flip_weights<<<(CH * CH * 27 + 255) / 256, 256, 0, s>>>(n->wb + OW2, n->wt2, CH, CH);
    e = conv_fwd<CH, CH, bf16, float, false, true, true>(n->g2b, n->wt2, nullptr, n->g1, g, n->wlay,
                                              n->status, s);
  }
  if (e == cudaSuccess) {
    k_tanh_bwd<<<grid_for(CH * g.n), 256, 0, s>>>(n->g1, n->h1, CH * g.n);
    e = conv_wgrad<CIN, CH, bf16, true, true>(n->x, n->g1, n->partial, n->grads, OW1, OB1, g, n->status, s);
  }
  if (e == cudaSuccess && lr > 0.0) {
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)n->adam_t), c2 = 1.0f - powf(b2, (float)n->adam_t);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(n->params, n->grads, n->adam_m, n->adam_v, n->wb,
                                                NPARAM, (float)lr, b1, b2, 1e-8f, c1, c2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !loss_out) {
    // asynchronous step: the loss joins the device sum (fv_net_take_loss)
    k_loss_accumulate<kLossBlocks><<<1, kLossRuns, 0, s>>>(n->loss_partial, 5.0 * (double)g.n,
                                                           n->loss_acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "network training step");
    n->acc_steps += 1;
    n->have_grads = true;
    return FV_OK;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(n->host_loss, n->loss_partial, kLossBlocks * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(n->host_status, n->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "network training step");
  n->have_grads = true;
  if ((st = take_status(n, s)) != FV_OK) return st;
  if (loss_out) {
    *loss_out = loss_from_partials(n->host_loss, kLossBlocks) / (5.0 * (double)g.n);
  }
  return FV_OK;
}

fv_status fv_net_take_loss(fv_net_t n, double* loss_sum, long long* steps) {
  fv_status st = check(n);
  if (st != FV_OK) return st;
  cudaStream_t s = n->last_stream;
  double sum = 0.0;
  cudaError_t e = cudaMemcpyAsync(&sum, n->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(n->host_status, n->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->loss_acc, 0, sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e, "reading the training loss");
  if (loss_sum) *loss_sum = sum;
  if (steps) *steps = n->acc_steps;
  n->acc_steps = 0;
  return take_status(n, s);
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
  fv_internal_state_written(m);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_fill_ghosts(v.U, v.P, v.stream);
  if (e != cudaSuccess) return cuda_fail(e, "applying the learned correction");
  return FV_OK;
}

fv_status fv_net_get_buffer(fv_net_t n, int which, void* dst, size_t bytes) {
  fv_status st = check(n);
  if (st != FV_OK) return st;
  if (!dst) return fail(FV_ERR_INVALID_ARG, "dst is NULL");
  const long long c = n->last_cells;
  const void* src = nullptr;
  size_t size = 0;
  bool grad = false;
  switch (which) {
    case FV_NET_BUF_FEATURES: src = n->x; size = (size_t)c * pitch8<CIN>() * sizeof(bf16); break;
    case FV_NET_BUF_H1: src = n->h1; size = (size_t)c * CH * sizeof(bf16); break;
    case FV_NET_BUF_H2: src = n->h2; size = (size_t)c * CH * sizeof(bf16); break;
    case FV_NET_BUF_OUT: src = n->o; size = (size_t)c * COUT * sizeof(float); break;
    case FV_NET_BUF_GRAD_OUT: src = n->go; size = (size_t)c * COUT * sizeof(float); grad = true; break;
    case FV_NET_BUF_GRAD_A2: src = n->g2; size = (size_t)c * CH * sizeof(float); grad = true; break;
    case FV_NET_BUF_GRAD_A1: src = n->g1; size = (size_t)c * CH * sizeof(float); grad = true; break;
    default: return fail(FV_ERR_INVALID_ARG, "unknown network buffer %d", which);
  }
  if (c == 0 || (grad && !n->have_grads))
    return fail(FV_ERR_INVALID_ARG, "buffer %d has not been produced by a %s yet", which,
                grad ? "training step" : "forward pass");
  if (bytes != size)
    return fail(FV_ERR_INVALID_ARG, "buffer %d holds %zu bytes, not %zu", which, size, bytes);
  cudaError_t e = cudaMemcpyAsync(dst, src, size, cudaMemcpyDeviceToDevice, n->last_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "fv_net_get_buffer");
  return FV_OK;
}

}  // extern "C"
