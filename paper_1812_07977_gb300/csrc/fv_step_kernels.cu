// fv_step_kernels.cu -- one RK2 substep of the FP64 finite-volume method.
//
// Compiled twice: FV_NS=fv_fp64_exact with --fmad=false (every operation
// rounded on its own, in the order of the method's definition) and
// FV_NS=fv_fp64_fma with --fmad=true and the Newton-Raphson divide and
// square root.  The CFL time step (ComputeTimeStep) is here too, so each
// variant computes its own dt with its own arithmetic; its pass over the
// state also gives the first substep its primitives.
//
// Structure of one substep of Algorithm 1 (its kernel sequence):
//   k_prim            conserved -> primitive for every ghosted cell
//   k_sweep<x>        ComputeDifferences, ComputeReconstruction,
//                     RiemannSolverInput and ComputeFluxes along x, and the
//                     x part of ComputeUpdate: ACC = -(F(i+1/2)-F(i-1/2))/dx
//   k_sweep<y>        the same along y: ACC -= (G(j+1/2)-G(j-1/2))/dy
//   k_sweep<z>        the same along z, then dU = dt*ACC and the RK combine
//                     (stage 1: U1 = U + dU; stage 2: U = (U + U1 + dU)/2)
// Each thread walks one grid line along the sweep axis with a sliding
// register window (four cells of primitives, the differences and half
// slopes of two cells, the previous face flux), so every difference, slope
// and face flux is computed exactly once.  On this GPU the FP64 pipe is the
// bottleneck by a wide margin, so the design spends memory traffic (the
// primitive and accumulator arrays) to never repeat FP64 work.
#include "fv_device.cuh"
#include "fv_internal.h"

#ifndef FV_NS
#error "FV_NS must name the variant namespace"
#endif

using namespace fvd;

namespace FV_NS {
namespace {

constexpr int kPrimThreads = 256;
constexpr int kSweepThreads = 64;
constexpr int kSweepMinBlocks = 8;   // 16 warps per SM: at most 128 registers

// A cell equal bit for bit to the thread's previous cell has its primitives;
// when the whole warp has such cells (uniform regions), it reuses them.
// KEEP (substep 2): W holds the primitives of U, and keep[] marks the
// interior cells whose substep 1 copied U to U1 unchanged; such a cell, and
// every ghost cell filled from it, already has its primitives in W and is
// neither read nor written.
template <bool KEEP>
__global__ void __launch_bounds__(kPrimThreads)
k_prim(const double* __restrict__ U, double* __restrict__ W, Params P,
       const unsigned char* __restrict__ keep, DevCounters* ctr) {
  const long long nf = P.nfield;
  const int X = P.nx + 4, Y = P.ny + 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // (i, j, k) of cell c in the ghosted array, advanced by increments
  int k = (int)(c / P.sz);
  int j = (int)((c - (long long)k * P.sz) / X);
  int i = (int)(c - (long long)k * P.sz - (long long)j * X);
  const int sk = (int)(stride / P.sz);
  const int sj = (int)((stride - (long long)sk * P.sz) / X);
  const int si = (int)(stride - (long long)sk * P.sz - (long long)sj * X);
  double up[NF] = {0.0, 0.0, 0.0, 0.0, 0.0};
  Prim w = Prim{0.0, 0.0, 0.0, 0.0, 0.0};
  bool have = false;
  for (; c < nf; c += stride) {
    bool skip = false;
    if (KEEP) {
      const int ci = ghost_source(i - 2, P.nx, P.bc[0]);
      const int cj = ghost_source(j - 2, P.ny, P.bc[1]);
      const int ck = ghost_source(k - 2, P.nz, P.bc[2]);
      skip = keep[((long long)ck * P.ny + cj) * P.nx + ci] != 0;
    }
    double u[NF];
    bool eq = have;
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      u[q] = skip ? up[q] : U[q * nf + c];
      eq = eq && bits(u[q]) == bits(up[q]);
      up[q] = u[q];
    }
    eq = eq || skip;
    have = have || !skip;
    if (!__all_sync(__activemask(), eq)) w = cons_to_prim(u, P);
    if (!skip) {
      W[c] = w.r;
      W[nf + c] = w.vx;
      W[2 * nf + c] = w.vy;
      W[3 * nf + c] = w.vz;
      W[4 * nf + c] = w.p;
      if (!(is_pos(w.r) && is_pos(w.p)) && i >= 2 && i < P.nx + 2 && j >= 2 &&
          j < P.ny + 2 && k >= 2 && k < P.nz + 2)
        atomicAdd(&ctr->np_step, 1ULL);
    }
    i += si;
    j += sj;
    k += sk;
    if (i >= X) {
      i -= X;
      ++j;
    }
    if (j >= Y) {
      j -= Y;
      ++k;
    }
  }
}

__device__ __forceinline__ Prim load_prim(const double* __restrict__ W, long long off,
                                          long long nf) {
  Prim w;
  w.r = W[off];
  w.vx = W[nf + off];
  w.vy = W[2 * nf + off];
  w.vz = W[3 * nf + off];
  w.p = W[4 * nf + off];
  return w;
}

// a and b equal bit for bit (all five components)
__device__ __forceinline__ bool same(const Prim& a, const Prim& b) {
  return bits(a.r) == bits(b.r) && bits(a.vx) == bits(b.vx) && bits(a.vy) == bits(b.vy) &&
         bits(a.vz) == bits(b.vz) && bits(a.p) == bits(b.p);
}

__device__ __forceinline__ Prim sub(const Prim& a, const Prim& b) {
  return Prim{a.r - b.r, a.vx - b.vx, a.vy - b.vy, a.vz - b.vz, a.p - b.p};
}

__device__ __forceinline__ Prim add(const Prim& a, const Prim& b) {
  return Prim{a.r + b.r, a.vx + b.vx, a.vy + b.vy, a.vz + b.vz, a.p + b.p};
}

template <int TK>
__device__ __forceinline__ Prim half_slopes(double theta, const Prim& dm, const Prim& dp) {
  return Prim{half_slope<TK>(theta, dm.r, dp.r), half_slope<TK>(theta, dm.vx, dp.vx),
              half_slope<TK>(theta, dm.vy, dp.vy), half_slope<TK>(theta, dm.vz, dp.vz),
              half_slope<TK>(theta, dm.p, dp.p)};
}

// RK combine of one value: stage 1 U1 = U + du; stage 2 U = ((U + U1) + du) / 2
template <int STAGE>
__device__ __forceinline__ void rk_combine(double* __restrict__ U, double* __restrict__ U1,
                                           long long gc, double du) {
  if (STAGE == 1) U1[gc] = U[gc] + du;
  else U[gc] = half((U[gc] + U1[gc]) + du);
}

// AXIS: 0, 1, 2.  STAGE: 0 for the x and y sweeps; 1 or 2 (the RK stage)
// for the z sweep, which finishes the update.  Each grid line is cut into
// gridDim.y segments of `seg` cells (blockIdx.y picks one): a segment starts
// its window two cells before its first cell and evaluates the face on its
// left, which the segment before also evaluates (the same bits), so every
// cell gets exactly the update of an unsegmented sweep.  More, shorter work
// items keep more warps resident and let the block scheduler even out lines
// of unequal cost.
template <int AXIS, int STAGE, int TK>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinBlocks)
k_sweep(const double* __restrict__ W, double* __restrict__ ACC, double* __restrict__ U,
        double* __restrict__ U1, Params P, double dt, int seg, unsigned char* __restrict__ keep,
        DevCounters* ctr) {
  const int n_line = AXIS == 0 ? P.nx : AXIS == 1 ? P.ny : P.nz;
  const int na = AXIS == 0 ? P.ny : P.nx;
  const int nb = AXIS == 2 ? P.ny : P.nz;
  const long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (line >= (long long)na * nb) return;
  const int c0 = (int)blockIdx.y * seg;  // first cell (and face) of the segment
  if (c0 >= n_line) return;
  const int n = n_line - c0 < seg ? n_line - c0 : seg;  // cells of the segment
  const int a = (int)(line % na);
  const int b = (int)(line / na);
  const int i0 = AXIS == 0 ? c0 : a;
  const int j0 = AXIS == 0 ? a : (AXIS == 1 ? c0 : b);
  const int k0 = AXIS == 2 ? c0 : b;
  const long long nf = P.nfield;
  const long long gs = AXIS == 0 ? 1 : (AXIS == 1 ? P.sy : P.sz);
  const long long g0 = (k0 + 2) * P.sz + (j0 + 2) * P.sy + (i0 + 2);
  const long long nd = (long long)P.nx * P.ny * P.nz;
  const long long ds = AXIS == 0 ? 1 : (AXIS == 1 ? (long long)P.nx : (long long)P.nx * P.ny);
  const long long d0 = ((long long)k0 * P.ny + j0) * P.nx + i0;
  const double inv = P.inv_d[AXIS];
  const double theta = P.theta;

  // window: wl_cell = W(f-1), wc = W(f); differences D(f) = W(f) - W(f-1)
  Prim wm2 = load_prim(W, g0 - 2 * gs, nf);
  Prim wm1 = load_prim(W, g0 - gs, nf);
  Prim wc = load_prim(W, g0, nf);
  Prim dcur = sub(wc, wm1);                               // D(0)
  Prim hprev = half_slopes<TK>(theta, sub(wm1, wm2), dcur);  // cell -1
  Prim wprev = wm1;                                       // W(f-1)
  double Fprev[NF];
#pragma unroll
  for (int q = 0; q < NF; ++q) Fprev[q] = 0.0;
  // length of the run of cells equal bit for bit to the newest cell of the
  // window (counted from cell -2 of the segment, so the segment's first face
  // is always evaluated), and whether the last face fell back
  int run = same(wm1, wm2) ? 2 : 1;
  run = same(wc, wm1) ? run + 1 : 1;
  bool fell_back = false;
  unsigned evaluated = 0;

  for (int f = 0; f <= n; ++f) {
    Prim wn = load_prim(W, g0 + (long long)(f + 1) * gs, nf);  // W(f+1)
    run = same(wn, wc) ? run + 1 : 1;
    double F[NF];
    Prim dnext, hcur;
    // Face f-1/2 reads cells f-2 .. f+1.  When cells f-3 .. f+1 are equal,
    // its differences and slopes are +0 and its face states are those of
    // face f-3/2, so its flux (and fallback) is the previous face's, bit for
    // bit: reuse it.  (run >= 5 implies f >= 1.)  Decided per warp, so the
    // warp skips the flux only when every line can.
    const bool reused = __all_sync(__activemask(), run >= 5);
    if (reused) {
      dnext = Prim{0.0, 0.0, 0.0, 0.0, 0.0};
      hcur = dnext;
#pragma unroll
      for (int q = 0; q < NF; ++q) F[q] = Fprev[q];
      if (fell_back) atomicAdd(&ctr->fallback, 1ULL);
    } else {
      dnext = sub(wn, wc);                                    // D(f+1)
      hcur = half_slopes<TK>(theta, dcur, dnext);             // cell f
      // face f-1/2 between cells f-1 and f
      Prim wl = add(wprev, hprev);
      Prim wr = sub(wc, hcur);
      fell_back = !(is_pos(wl.r) && is_pos(wl.p) && is_pos(wr.r) && is_pos(wr.p));
      if (fell_back) {
        wl = wprev;
        wr = wc;
        // the first face of a later segment is the last face of the one
        // before, which counted it
        if (f > 0 || c0 == 0) atomicAdd(&ctr->fallback, 1ULL);
      }
      hll_flux<AXIS>(wl, wr, P, F);
      ++evaluated;
    }
    // With the flux reused and finite, F - Fprev is +0 for every component:
    // the x part of the divergence is -0 * inv = -0, and subtracting
    // +0 * inv leaves ACC as it is (both exactly what the arithmetic gives),
    // so the warp skips that arithmetic (and the y sweep its ACC update).
    bool finite_f = reused;
#pragma unroll
    for (int q = 0; q < NF; ++q) finite_f = finite_f && is_finite(F[q]);
    const bool zero_diff = __all_sync(__activemask(), finite_f);
    if (f > 0) {  // cell f-1 has both of its faces
      const long long dc = d0 + (long long)(f - 1) * ds;
      if (zero_diff) {
        if (AXIS == 0) {
#pragma unroll
          for (int q = 0; q < NF; ++q) ACC[q * nd + dc] = -0.0;
        }
        if (AXIS == 2) {
          // acc = ACC.  Where no axis had a flux difference every component
          // is -0 (the x sweep stored -0, the others subtracted nothing), so
          // du = dt * acc = -0 and x + du = x for every x: stage 1 is the copy
          // U1 = U and stage 2 is U = (U + U1) / 2, bit for bit.
          double acc[NF];
          bool neg_zero = true;
#pragma unroll
          for (int q = 0; q < NF; ++q) {
            acc[q] = ACC[q * nd + dc];
            neg_zero = neg_zero && is_neg_zero(acc[q]);
          }
          const long long gc0 = g0 + (long long)(f - 1) * gs;
          // (stage 1 marks the copied cells for the primitives of substep 2)
          if (__all_sync(__activemask(), neg_zero)) {
#pragma unroll
            for (int q = 0; q < NF; ++q) {
              if (STAGE == 1) U1[q * nf + gc0] = U[q * nf + gc0];
              else U[q * nf + gc0] = half(U[q * nf + gc0] + U1[q * nf + gc0]);
            }
            if (STAGE == 1) keep[dc] = 1;
          } else {
#pragma unroll
            for (int q = 0; q < NF; ++q) rk_combine<STAGE>(U, U1, q * nf + gc0, dt * acc[q]);
            if (STAGE == 1) keep[dc] = 0;
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          const double diff = F[q] - Fprev[q];
          if (AXIS == 0) {
            ACC[q * nd + dc] = -diff * inv;
          } else if (AXIS == 1) {
            ACC[q * nd + dc] = ACC[q * nd + dc] - diff * inv;
          } else {
            const double acc = ACC[q * nd + dc] - diff * inv;
            rk_combine<STAGE>(U, U1, q * nf + g0 + (long long)(f - 1) * gs, dt * acc);
          }
        }
        if (AXIS == 2 && STAGE == 1) keep[dc] = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < NF; ++q) Fprev[q] = F[q];
    wprev = wc;
    wc = wn;
    dcur = dnext;
    hprev = hcur;
  }
  warp_count(&ctr->faces, evaluated);
}

constexpr int kDtThreads = 256;

// ---------------------------------------------------------------- time step
#ifndef FV_DT_FILTER
#define FV_DT_FILTER 1
#endif

// Primitives of every ghosted cell (what k_prim gives the first substep)
// and, over the interior cells, the maximum CFL speed and the non-physical
// count, in one pass over the state.  The maximum is exact in any order:
// non-negative doubles order like their bit patterns, so the grid-wide
// maximum is an integer atomicMax, and a NaN speed never wins, as in a plain
// `if (s > smax)` loop.  A cell equal bit for bit to the thread's previous
// cell has its primitives, speed and validity; when the whole warp has such
// cells (uniform regions), it skips the arithmetic.  Non-physical interior
// cells count once, for the time step (a substep that uses these
// primitives does not count them again).  A cell whose FP32 speed bound is
// below the thread's running maximum cannot raise it: when no lane of the
// warp needs it, the FP64 speed is not computed (the maximum is unchanged,
// so the result is the same bits), and 0 stands in for it, so that a later
// equal cell changes nothing either.
__global__ void __launch_bounds__(kDtThreads)
k_prim_dt(const double* __restrict__ U, double* __restrict__ W, Params P, DevCounters* ctr) {
  const long long nf = P.nfield;
  const int X = P.nx + 4, Y = P.ny + 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // (i, j, k) of cell c in the ghosted array, advanced by the stride's own
  // (si, sj, sk) with carries
  int k = (int)(c / P.sz);
  int j = (int)((c - (long long)k * P.sz) / X);
  int i = (int)(c - (long long)k * P.sz - (long long)j * X);
  const int sk = (int)(stride / P.sz);
  const int sj = (int)((stride - (long long)sk * P.sz) / X);
  const int si = (int)(stride - (long long)sk * P.sz - (long long)sj * X);
  double smax = 0.0, s = 0.0;
  float smax_f = 0.0f;   // smax rounded toward zero
  unsigned long long bad = 0;
  double up[NF] = {0.0, 0.0, 0.0, 0.0, 0.0};
  Prim w = Prim{0.0, 0.0, 0.0, 0.0, 0.0};
  bool have = false, bad_cell = false;
  const float g32 = __double2float_ru(P.gamma);
  const float i32[3] = {__double2float_ru(P.inv_d[0]), __double2float_ru(P.inv_d[1]),
                        __double2float_ru(P.inv_d[2])};
  for (; c < nf; c += stride) {
    double u[NF];
    bool eq = have;
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      u[q] = U[q * nf + c];
      eq = eq && bits(u[q]) == bits(up[q]);
      up[q] = u[q];
    }
    have = true;
    if (!__all_sync(__activemask(), eq)) {
      w = cons_to_prim(u, P);
      bad_cell = !(is_pos(w.r) && is_pos(w.p));
      // smax_f <= smax, so bound < smax_f means the speed is below smax
      const bool need = !FV_DT_FILTER || !(speed_bound(w, g32, i32) < smax_f);
      if (__any_sync(__activemask(), need)) s = cell_speed(w, P);
      else s = 0.0;  // below smax: equal cells that follow change nothing
    }
    W[c] = w.r;
    W[nf + c] = w.vx;
    W[2 * nf + c] = w.vy;
    W[3 * nf + c] = w.vz;
    W[4 * nf + c] = w.p;
    if (i >= 2 && i < P.nx + 2 && j >= 2 && j < P.ny + 2 && k >= 2 && k < P.nz + 2) {
      bad += bad_cell;
      if (s > smax) {
        smax = s;
        smax_f = __double2float_rz(smax);
      }
    }
    i += si;
    j += sj;
    k += sk;
    if (i >= X) {
      i -= X;
      ++j;
    }
    if (j >= Y) {
      j -= Y;
      ++k;
    }
  }
  unsigned long long sb = (unsigned long long)__double_as_longlong(smax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, sb, o);
    sb = v > sb ? v : sb;
  }
  __shared__ unsigned long long warp_max[kDtThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_max[wid] = sb;
  if (bad) atomicAdd(&ctr->np_dt, bad);
  __syncthreads();
  if (wid == 0) {
    sb = lane < kDtThreads / 32 ? warp_max[lane] : 0ULL;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, sb, o);
      sb = v > sb ? v : sb;
    }
    if (lane == 0) atomicMax(&ctr->smax_bits, sb);
  }
}

}  // namespace

cudaError_t launch_prim_dt(const double* U, const StepBuffers& b, const Params& P,
                           cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&b.ctr->smax_bits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  long long blocks = (P.nfield + kDtThreads - 1) / kDtThreads;
  if (blocks > 8LL * fv_sm_count()) blocks = 8LL * fv_sm_count();
  k_prim_dt<<<(unsigned)blocks, kDtThreads, 0, s>>>(U, b.W, P, b.ctr);
  return cudaGetLastError();
}

cudaError_t launch_prim(const double* src, const StepBuffers& b, const Params& P, bool keep,
                        cudaStream_t s) {
  long long blocks = (P.nfield + kPrimThreads - 1) / kPrimThreads;
  if (blocks > 16LL * fv_sm_count()) blocks = 16LL * fv_sm_count();
  if (keep)
    k_prim<true><<<(unsigned)blocks, kPrimThreads, 0, s>>>(src, b.W, P, b.keep, b.ctr);
  else
    k_prim<false><<<(unsigned)blocks, kPrimThreads, 0, s>>>(src, b.W, P, nullptr, b.ctr);
  return cudaGetLastError();
}

// Default segments per line: enough work items for about kSweepWaves waves
// of resident warps, each segment at least kMinSegment cells long (its
// first face is evaluated twice, which costs most where the flux would
// otherwise be reused).
constexpr int kSweepWaves = 8;
constexpr int kMinSegment = 16;

template <int TK>
static cudaError_t sweep_tk(int axis, int stage, const StepBuffers& b, const Params& P,
                            double dt, int segments, int num_sms, cudaStream_t s) {
  const long long lines = axis == 0 ? (long long)P.ny * P.nz
                        : axis == 1 ? (long long)P.nx * P.nz : (long long)P.nx * P.ny;
  const int n = axis == 0 ? P.nx : axis == 1 ? P.ny : P.nz;
  if (segments < 1) {
    const long long warps = (lines + kSweepThreads - 1) / kSweepThreads * (kSweepThreads / 32);
    const long long target =
        (long long)kSweepWaves * kSweepMinBlocks * (kSweepThreads / 32) * (num_sms > 0 ? num_sms : 1);
    const long long want = (target + warps - 1) / warps;
    const int most = n / kMinSegment > 1 ? n / kMinSegment : 1;
    segments = want < most ? (int)want : most;
  }
  if (segments > n) segments = n;
  const int seg = (n + segments - 1) / segments;
  const dim3 g((unsigned)((lines + kSweepThreads - 1) / kSweepThreads),
               (unsigned)((n + seg - 1) / seg));
  if (axis == 0)
    k_sweep<0, 0, TK><<<g, kSweepThreads, 0, s>>>(b.W, b.ACC, b.U, b.U1, P, dt, seg, b.keep, b.ctr);
  else if (axis == 1)
    k_sweep<1, 0, TK><<<g, kSweepThreads, 0, s>>>(b.W, b.ACC, b.U, b.U1, P, dt, seg, b.keep, b.ctr);
  else if (stage == 1)
    k_sweep<2, 1, TK><<<g, kSweepThreads, 0, s>>>(b.W, b.ACC, b.U, b.U1, P, dt, seg, b.keep, b.ctr);
  else
    k_sweep<2, 2, TK><<<g, kSweepThreads, 0, s>>>(b.W, b.ACC, b.U, b.U1, P, dt, seg, b.keep, b.ctr);
  return cudaGetLastError();
}

cudaError_t launch_sweep(int axis, int stage, const StepBuffers& b, const Params& P, double dt,
                         int segments, int num_sms, cudaStream_t s) {
  if (P.theta == 2.0) return sweep_tk<THETA_TWO>(axis, stage, b, P, dt, segments, num_sms, s);
  return sweep_tk<THETA_GENERAL>(axis, stage, b, P, dt, segments, num_sms, s);
}

}  // namespace FV_NS
