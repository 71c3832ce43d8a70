// fv_fused64_kernels.cu -- one RK2 substep of the FP64 finite-volume method
// in one kernel: every stage of Algorithm 1's substep (the conversion to
// primitives, ComputeDifferences, ComputeReconstruction, RiemannSolverInput,
// ComputeFluxes, ComputeUpdate and the RK combine) for a tile of 32 x TY
// columns marching along z over a chunk of planes, so a substep reads its
// input state once (plus the tile's two-cell halo) and writes its output
// once: about 200 B of HBM traffic per zone-update, against the ~1 KB of
// separate per-axis passes with primitive and accumulator arrays.
//
// Compiled once per arithmetic variant (FV_NS): fv_fp64_exact with
// --fmad=false (every operation rounded on its own in the method's order:
// the same bits as a plain IEEE FP64 code) and fv_fp64_fma with --fmad=true
// and the Newton-Raphson divide and square root.
//
// Per plane k of the chunk each thread owns one column (i, j) of the tile:
//   z   a register window along its column (primitives of planes k .. k+2,
//       the z difference and half slope of plane k+1 and k, the z flux of
//       face k-1/2 carried from the previous plane) gives the z flux of face
//       k+1/2 -- every z flux computed once;
//   x,y the plane's primitives (tile plus two-cell halo) go to shared
//       memory; the half slopes of every cell (once per cell and axis), then
//       the 33 x TY x faces and 32 x (TY+1) y faces (once each) follow in
//       shared memory;
//   update  dU = dt (-(Fx(i+1/2)-Fx(i-1/2))/dx - (..)/dy - (..)/dz) and the RK
//       combine; stage 2 also folds the FP64 CFL speed of the cell it writes
//       into the next time step's maximum.
// The FP64 input of the next plane is staged into shared memory by cp.async
// while the current one is computed.  Work that repeats bit for bit is
// skipped, decided per warp: a cell whose conserved state equals the one a
// plane below keeps that cell's primitives; a slope or a face whose cells all
// equal those a plane below keeps its value (still in shared memory); a z
// face whose column has five equal cells around it takes the previous z
// flux; a cell whose six face fluxes have zero differences takes the RK
// combine's exact result without the arithmetic.  Each of these gives the
// bits that evaluating gives.
#include "fv_device.cuh"
#include "fv_device32.cuh"
#include "fv_fused_common.cuh"
#include "fv_internal.h"

#ifndef FV_NS
#error "FV_NS must name the variant namespace"
#endif

using namespace fvd;
using namespace fvfused;

namespace FV_NS {
namespace {

template <class S>
struct Smem64 {
  double col[2][NF][S::kThreads];     // staged input: the column cell of plane t+2
  double halo[2][NF][S::kHalo];       // staged input: the halo cells of plane t
  double w[NF][S::PY][S::PX];         // primitives of the plane, tile and halo
  double hx[NF][S::TY][TX + 2];       // x half slopes of cells -1 .. TX
  double hy[NF][S::TY + 2][TX];       // y half slopes of rows -1 .. TY
  double fx[NF][S::TY][TX + 1];       // x face fluxes
  double fy[NF][S::TY + 1][TX];       // y face fluxes
  unsigned char same[S::PY][S::PX];   // the cell equals (bits) the cell a plane below
};

__device__ __forceinline__ Prim load_cons_prim(const double* __restrict__ U, long long nf,
                                               long long off, const Params& P) {
  double u[NF];
#pragma unroll
  for (int q = 0; q < NF; ++q) u[q] = U[q * nf + off];
  return cons_to_prim(u, P);
}

__device__ __forceinline__ bool same_bits(const Prim& a, const Prim& b) {
  return bits(a.r) == bits(b.r) && bits(a.vx) == bits(b.vx) && bits(a.vy) == bits(b.vy) &&
         bits(a.vz) == bits(b.vz) && bits(a.p) == bits(b.p);
}

__device__ __forceinline__ Prim psub(const Prim& a, const Prim& b) {
  return Prim{a.r - b.r, a.vx - b.vx, a.vy - b.vy, a.vz - b.vz, a.p - b.p};
}
__device__ __forceinline__ Prim padd(const Prim& a, const Prim& b) {
  return Prim{a.r + b.r, a.vx + b.vx, a.vy + b.vy, a.vz + b.vz, a.p + b.p};
}

template <int TK>
__device__ __forceinline__ Prim half_slopes(double theta, const Prim& dm, const Prim& dp) {
  return Prim{half_slope<TK>(theta, dm.r, dp.r), half_slope<TK>(theta, dm.vx, dp.vx),
              half_slope<TK>(theta, dm.vy, dp.vy), half_slope<TK>(theta, dm.vz, dp.vz),
              half_slope<TK>(theta, dm.p, dp.p)};
}

__device__ __forceinline__ bool physical(const Prim& w) { return is_pos(w.r) && is_pos(w.p); }

template <class SM>
__device__ __forceinline__ Prim smem_w(const SM& s, int row, int col) {
  return Prim{s.w[0][row][col], s.w[1][row][col], s.w[2][row][col], s.w[3][row][col],
              s.w[4][row][col]};
}
template <class SM>
__device__ __forceinline__ void smem_w_store(SM& s, int row, int col, const Prim& w) {
  s.w[0][row][col] = w.r;
  s.w[1][row][col] = w.vx;
  s.w[2][row][col] = w.vy;
  s.w[3][row][col] = w.vz;
  s.w[4][row][col] = w.p;
}

// The flux through the face between cells wm (left) and wp (right) from
// their half slopes hm, hp along AXIS (first order if a face state is
// non-physical; `fb` set then).
template <int AXIS>
__device__ __forceinline__ void face_flux(const Prim& wm, const Prim& hm, const Prim& wp,
                                          const Prim& hp, const Params& P, double F[NF],
                                          bool& fb) {
  Prim wl = padd(wm, hm);
  Prim wr = psub(wp, hp);
  fb = !(physical(wl) && physical(wr));
  if (fb) {
    wl = wm;
    wr = wp;
  }
  hll_flux<AXIS>(wl, wr, P, F);
}

// Stage-1 or stage-2 substep of one tile: columns i0 .. i0+TX-1, j0 ..
// j0+TY-1, planes k0 .. k1-1.  STAGE 1: U1 = U + dU(U).  STAGE 2:
// U = ((U + U1) + dU(U1)) / 2, and the FP64 CFL speed of every cell written
// into the launch's shared maximum *gmax (smax, smax_f: the thread's
// threshold; fvd32::fold_speed) and its non-physical cells into bad_next.
// The substep's input state has its ghosts filled.
template <class S, int STAGE, int TK>
__device__ __forceinline__ void stage64_tile(Smem64<S>& s, double* __restrict__ U,
                                             double* __restrict__ U1, const Params& P,
                                             const fvd32::Params32& Q, double dt, int i0,
                                             int j0, int k0, int k1, unsigned& fallbacks_out,
                                             unsigned long long& bad_out, unsigned& evaluated,
                                             double& smax, float& smax_f,
                                             unsigned long long& bad_next,
                                             unsigned long long* gmax) {
  const double* __restrict__ src = STAGE == 1 ? U : U1;
  constexpr int kThreads = S::kThreads, kHalo = S::kHalo, kHaloPer = S::kHaloPer;
  constexpr int TY = S::TY;
  const int tid = threadIdx.x;
  const int ti = tid % TX, tj = tid / TX;
  const long long nf = P.nfield;
  const double theta = P.theta;
  // this thread's column, clamped into the ghosted array (columns past a
  // ragged edge compute values that nothing stores)
  const int gi = min(i0 + ti, P.nx + 1), gj = min(j0 + tj, P.ny + 1);
  const bool owner = (i0 + ti < P.nx) && (j0 + tj < P.ny);
  const long long col = (long long)(gj + 2) * P.sy + (gi + 2);
  int hrow[kHaloPer], hcol[kHaloPer];
  long long hcolo[kHaloPer];
#pragma unroll
  for (int e = 0; e < kHaloPer; ++e) {
    hrow[e] = hcol[e] = 0;
    if (tid + e * kThreads < kHalo) halo_cell<S>(tid + e * kThreads, hrow[e], hcol[e]);
    const int hgi = min(max(i0 + hcol[e], -2), P.nx + 1);
    const int hgj = min(max(j0 + hrow[e], -2), P.ny + 1);
    hcolo[e] = (long long)(hgj + 2) * P.sy + (hgi + 2);
  }
  // which of this thread's x / y faces (bit p: its face of pass p) this tile
  // counts: each face of the mesh is counted by one tile
  unsigned counted = 0;
#pragma unroll
  for (int p = 0; p < S::kFacePer; ++p) {
    const int f = tid + p * kThreads;
    if (f < S::kXFaces) {
      const int r = f / (TX + 1), fi = f % (TX + 1);
      if (i0 + fi <= P.nx && (fi < TX || i0 + fi == P.nx) && j0 + r < P.ny) counted |= 1u << p;
    } else if (f < S::kFaces) {
      const int g = f - S::kXFaces, fj = g / TX, c = g % TX;
      if (i0 + c < P.nx && j0 + fj <= P.ny && (fj < TY || j0 + fj == P.ny)) counted |= 1u << p;
    }
  }
  unsigned fallbacks = 0;
  unsigned xyfb = 0;           // fallback bits of this thread's x / y faces (bit p)
  unsigned long long bad = 0;
  fvd32::SpeedCache cache;
  cache.valid = false;

  // z window prologue: planes k0-2 .. k0+1 of the column
  const Prim wm2 = load_cons_prim(src, nf, col + (long long)(k0 + 0) * P.sz, P);
  Prim wm1 = load_cons_prim(src, nf, col + (long long)(k0 + 1) * P.sz, P);
  Prim w0 = load_cons_prim(src, nf, col + (long long)(k0 + 2) * P.sz, P);
  Prim w1 = load_cons_prim(src, nf, col + (long long)(k0 + 3) * P.sz, P);
  Prim d1 = psub(w1, w0);                                          // D(k0+1)
  Prim h0 = half_slopes<TK>(theta, psub(w0, wm1), d1);              // cell k0
  double fz_lo[NF];
  bool zfb;
  {
    const Prim hm1 = half_slopes<TK>(theta, psub(wm1, wm2), psub(w0, wm1));   // cell k0-1
    face_flux<2>(wm1, hm1, w0, h0, P, fz_lo, zfb);
    ++evaluated;
    if (zfb && k0 == 0 && owner) ++fallbacks;   // later chunks: the chunk below counts it
  }
  // cells of the column equal bit for bit to the newest one, from plane k0-2
  int run = same_bits(wm1, wm2) ? 2 : 1;
  run = same_bits(w0, wm1) ? run + 1 : 1;
  run = same_bits(w1, w0) ? run + 1 : 1;
  bool same0 = false;          // w0 equals the cell a plane below (not known at k0)
  bool same1 = same_bits(w1, w0);

  // FP64 input of iteration t: the column cell of plane t+2 and the halo
  // cells of plane t, into ring slot t % 2 (each thread copies and reads
  // only its own cells, so a slot is reused without a barrier)
  auto stage_in = [&](int t) {
    if (t < k1) {
      const int slot = t & 1;
      const double* c = src + col + (long long)(t + 4) * P.sz;
#pragma unroll
      for (int q = 0; q < NF; ++q) cp_async8(&s.col[slot][q][tid], c + q * nf);
#pragma unroll
      for (int e = 0; e < kHaloPer; ++e) {
        const int h = tid + e * kThreads;
        if (h < kHalo) {
          const double* hp = src + hcolo[e] + (long long)(t + 2) * P.sz;
#pragma unroll
          for (int q = 0; q < NF; ++q) cp_async8(&s.halo[slot][q][h], hp + q * nf);
        }
      }
    }
    cp_async_commit();
  };
  stage_in(k0);

  for (int k = k0; k < k1; ++k) {
    const int slot = k & 1, prev = slot ^ 1;
    const bool later = k > k0;     // the other slot and shared memory hold plane k-1
    if (owner && !physical(w0)) ++bad;   // each interior cell once per substep
    if (STAGE == 2) fvd32::refresh_max(gmax, smax, smax_f);
    // operands of this plane's RK combine, loaded before the face work
    const long long g = col + (long long)(k + 2) * P.sz;
    double rk0[NF], rk1[NF];
    if (owner) {
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        rk0[q] = U[q * nf + g];
        rk1[q] = STAGE == 2 ? U1[q * nf + g] : 0.0;
      }
    }
    cp_async_wait_all();
    // (a) the column cell of plane k+2 enters the z window: its primitives,
    // or those of plane k+1 when its state is the same bits
    double uc[NF];
    bool eqc = later;
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      uc[q] = s.col[slot][q][tid];
      eqc = eqc && bits(uc[q]) == bits(s.col[prev][q][tid]);
    }
    // (at k0 the window's plane k0+2 was not staged before: compare with w1)
    Prim w2 = w1;
    if (!__all_sync(0xffffffffu, eqc)) w2 = cons_to_prim(uc, P);
    const bool same2 = eqc || same_bits(w2, w1);
    run = same2 ? run + 1 : 1;
    // (b) the halo cells of plane k: primitives (kept where the state is the
    // same bits as a plane below) and their flags
    double uh[kHaloPer][NF];
    bool eqh[kHaloPer];
#pragma unroll
    for (int e = 0; e < kHaloPer; ++e) {
      const int h = tid + e * kThreads;
      eqh[e] = later;
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        uh[e][q] = h < kHalo ? s.halo[slot][q][h] : 0.0;
        eqh[e] = eqh[e] && (h >= kHalo || bits(uh[e][q]) == bits(s.halo[prev][q][h]));
      }
    }
    stage_in(k + 1);   // into the other slot, now compared
    // (c) z flux of face k+1/2 (planes k-1 .. k+2); with planes k-2 .. k+2 of
    // the column equal its inputs are those of face k-1/2: reuse that flux
    Prim d2, h1;
    double fz_hi[NF];
    if (__all_sync(0xffffffffu, run >= 5)) {
      d2 = Prim{0.0, 0.0, 0.0, 0.0, 0.0};
      h1 = d2;
#pragma unroll
      for (int q = 0; q < NF; ++q) fz_hi[q] = fz_lo[q];
    } else {
      d2 = psub(w2, w1);
      h1 = half_slopes<TK>(theta, d1, d2);
      face_flux<2>(w0, h0, w1, h1, P, fz_hi, zfb);
      ++evaluated;
    }
    if (zfb && owner) ++fallbacks;
    // (d) the plane's primitives into shared memory with their flags
    smem_w_store(s, tj + 2, ti + 2, w0);
    s.same[tj + 2][ti + 2] = later && same0;
#pragma unroll
    for (int e = 0; e < kHaloPer; ++e) {
      const int h = tid + e * kThreads;
      const bool all_eq = __all_sync(0xffffffffu, eqh[e] || h >= kHalo);
      if (h < kHalo) {
        if (!all_eq) smem_w_store(s, hrow[e] + 2, hcol[e] + 2, cons_to_prim(uh[e], P));
        s.same[hrow[e] + 2][hcol[e] + 2] = eqh[e];
      }
    }
    __syncthreads();
    // (e) half slopes of every cell along x and y (kept where the cell and
    // its two neighbours equal those a plane below)
#pragma unroll
    for (int p = 0; p < S::kSlopePer; ++p) {
      const int t = tid + p * kThreads;
      if (t < S::kXSlopes) {
        const int r = t / (TX + 2), c = t % (TX + 2);   // cell c-1 of row r
        const bool keep = s.same[r + 2][c] & s.same[r + 2][c + 1] & s.same[r + 2][c + 2];
        if (!__all_sync(__activemask(), keep)) {
          const Prim wa = smem_w(s, r + 2, c), wb = smem_w(s, r + 2, c + 1),
                     wc = smem_w(s, r + 2, c + 2);
          const Prim h = half_slopes<TK>(theta, psub(wb, wa), psub(wc, wb));
          s.hx[0][r][c] = h.r;
          s.hx[1][r][c] = h.vx;
          s.hx[2][r][c] = h.vy;
          s.hx[3][r][c] = h.vz;
          s.hx[4][r][c] = h.p;
        }
      } else if (t < S::kSlopes) {
        const int u = t - S::kXSlopes, r = u / TX, c = u % TX;   // row r-1, column c
        const bool keep = s.same[r][c + 2] & s.same[r + 1][c + 2] & s.same[r + 2][c + 2];
        if (!__all_sync(__activemask(), keep)) {
          const Prim wa = smem_w(s, r, c + 2), wb = smem_w(s, r + 1, c + 2),
                     wc = smem_w(s, r + 2, c + 2);
          const Prim h = half_slopes<TK>(theta, psub(wb, wa), psub(wc, wb));
          s.hy[0][r][c] = h.r;
          s.hy[1][r][c] = h.vx;
          s.hy[2][r][c] = h.vy;
          s.hy[3][r][c] = h.vz;
          s.hy[4][r][c] = h.p;
        }
      }
    }
    __syncthreads();
    // (f) x and y face fluxes (kept, with their fallbacks, where the face's
    // four cells equal those a plane below)
#pragma unroll
    for (int p = 0; p < S::kFacePer; ++p) {
      const int f = tid + p * kThreads;
      if (f < S::kXFaces) {
        const int r = f / (TX + 1), fi = f % (TX + 1);   // between cells fi-1 and fi
        const bool keep = s.same[r + 2][fi] & s.same[r + 2][fi + 1] & s.same[r + 2][fi + 2] &
                          s.same[r + 2][fi + 3];
        if (!__all_sync(__activemask(), keep)) {
          const Prim hm{s.hx[0][r][fi], s.hx[1][r][fi], s.hx[2][r][fi], s.hx[3][r][fi],
                        s.hx[4][r][fi]};
          const Prim hp{s.hx[0][r][fi + 1], s.hx[1][r][fi + 1], s.hx[2][r][fi + 1],
                        s.hx[3][r][fi + 1], s.hx[4][r][fi + 1]};
          double F[NF];
          bool fb;
          face_flux<0>(smem_w(s, r + 2, fi + 1), hm, smem_w(s, r + 2, fi + 2), hp, P, F, fb);
          xyfb = (xyfb & ~(1u << p)) | ((unsigned)fb << p);
          ++evaluated;
#pragma unroll
          for (int q = 0; q < NF; ++q) s.fx[q][r][fi] = F[q];
        }
      } else if (f < S::kFaces) {
        const int u = f - S::kXFaces, fj = u / TX, c = u % TX;   // between rows fj-1, fj
        const bool keep = s.same[fj][c + 2] & s.same[fj + 1][c + 2] & s.same[fj + 2][c + 2] &
                          s.same[fj + 3][c + 2];
        if (!__all_sync(__activemask(), keep)) {
          const Prim hm{s.hy[0][fj][c], s.hy[1][fj][c], s.hy[2][fj][c], s.hy[3][fj][c],
                        s.hy[4][fj][c]};
          const Prim hp{s.hy[0][fj + 1][c], s.hy[1][fj + 1][c], s.hy[2][fj + 1][c],
                        s.hy[3][fj + 1][c], s.hy[4][fj + 1][c]};
          double F[NF];
          bool fb;
          face_flux<1>(smem_w(s, fj + 1, c + 2), hm, smem_w(s, fj + 2, c + 2), hp, P, F, fb);
          xyfb = (xyfb & ~(1u << p)) | ((unsigned)fb << p);
          ++evaluated;
#pragma unroll
          for (int q = 0; q < NF; ++q) s.fy[q][fj][c] = F[q];
        }
      }
      fallbacks += (xyfb >> p) & (counted >> p) & 1u;
    }
    __syncthreads();
    // (g) update of cell (i, j, k): the divergence summed x, y, z, dU = dt
    // acc, the RK combine.  Where all six fluxes pair up bit for bit (and are
    // finite) every difference is +0, acc is -0 and x + dU = x exactly: the
    // combine is then a copy (stage 1) or a half sum (stage 2).
    if (owner) {
      double fxl[NF], fxr[NF], fyl[NF], fyr[NF];
      bool zero = true;
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        fxl[q] = s.fx[q][tj][ti];
        fxr[q] = s.fx[q][tj][ti + 1];
        fyl[q] = s.fy[q][tj][ti];
        fyr[q] = s.fy[q][tj + 1][ti];
        zero = zero && bits(fxl[q]) == bits(fxr[q]) && bits(fyl[q]) == bits(fyr[q]) &&
               bits(fz_lo[q]) == bits(fz_hi[q]) && is_finite(fxr[q]) && is_finite(fyr[q]) &&
               is_finite(fz_hi[q]);
      }
      double un[NF];
      if (__all_sync(__activemask(), zero)) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          if (STAGE == 1) U1[q * nf + g] = rk0[q];
          else U[q * nf + g] = un[q] = half(rk0[q] + rk1[q]);
        }
      } else {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          double acc = -(fxr[q] - fxl[q]) * P.inv_d[0];
          acc = acc - (fyr[q] - fyl[q]) * P.inv_d[1];
          acc = acc - (fz_hi[q] - fz_lo[q]) * P.inv_d[2];
          const double du = dt * acc;
          if (STAGE == 1) U1[q * nf + g] = rk0[q] + du;
          else U[q * nf + g] = un[q] = half((rk0[q] + rk1[q]) + du);
        }
      }
      if (STAGE == 2) fvd32::fold_speed(un, P, Q, smax, smax_f, bad_next, cache, gmax);
    }
    // the window moves up one plane
#pragma unroll
    for (int q = 0; q < NF; ++q) fz_lo[q] = fz_hi[q];
    w0 = w1;
    w1 = w2;
    d1 = d2;
    h0 = h1;
    same0 = same1;
    same1 = same2;
  }
  fallbacks_out += fallbacks;
  bad_out += bad;
}

// Folds a thread's CFL speed maximum (a double >= 0, ordered like its bits)
// into a grid-wide maximum.  All lanes of the warp call.
__device__ __forceinline__ void max_to(unsigned long long* dst, double smax) {
  unsigned long long b = (unsigned long long)__double_as_longlong(smax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
    b = v > b ? v : b;
  }
  if ((threadIdx.x & 31u) == 0u && b) atomicMax(dst, b);
}

constexpr int kTileY = 8;
constexpr int kMinBlocks = 1;    // 8 warps per SM: up to 255 registers

template <int STAGE, int TK>
__global__ void __launch_bounds__(TX * kTileY, kMinBlocks)
k_stage64(double* __restrict__ U, double* __restrict__ U1, Params P, fvd32::Params32 Q,
          double dt, int kchunk, DevCounters* ctr) {
  using S = Shape64<kTileY>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem64<S>& s = *reinterpret_cast<Smem64<S>*>(smem_raw);
  unsigned fallbacks = 0, evaluated = 0;
  unsigned long long bad = 0, bad_next = 0;
  double smax = 0.0;
  float smax_f = 0.0f;
  const int k0 = blockIdx.z * kchunk;
  stage64_tile<S, STAGE, TK>(s, U, U1, P, Q, dt, blockIdx.x * TX, blockIdx.y * kTileY, k0,
                             min(k0 + kchunk, P.nz), fallbacks, bad, evaluated, smax, smax_f,
                             bad_next, &ctr->smax_next);
  if (fallbacks) atomicAdd(&ctr->fallback, (unsigned long long)fallbacks);
  if (bad) atomicAdd(&ctr->np_step, bad);
  warp_count(&ctr->faces, evaluated);
  if (STAGE == 2) {
    max_to(&ctr->smax_next, smax);
    if (bad_next) atomicAdd(&ctr->np_dt, bad_next);
  }
}

// The CFL time step's maximum over the interior cells with this build's FP64
// speed (the same arithmetic as the stage-2 epilogue, so a cached maximum
// and this pass agree bit for bit); FP32 bounds skip the cells that cannot
// raise a thread's running maximum.
__global__ void __launch_bounds__(256)
k_dt64(const double* __restrict__ U, Params P, fvd32::Params32 Q, DevCounters* ctr) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  double smax = 0.0;
  float smax_f = 0.0f;
  unsigned long long bad = 0;
  fvd32::SpeedCache cache;
  cache.valid = false;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n;
       m += (long long)gridDim.x * blockDim.x) {
    const long long k = m / ((long long)P.nx * P.ny);
    const long long r = m - k * ((long long)P.nx * P.ny);
    const long long j = r / P.nx, i = r - j * P.nx;
    const long long o = (k + 2) * P.sz + (j + 2) * P.sy + (i + 2);
    double u[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) u[q] = U[q * P.nfield + o];
    fvd32::refresh_max(&ctr->smax_bits, smax, smax_f);
    fvd32::fold_speed(u, P, Q, smax, smax_f, bad, cache, &ctr->smax_bits);
  }
  if (bad) atomicAdd(&ctr->np_dt, bad);
  unsigned long long b = (unsigned long long)__double_as_longlong(smax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
    b = v > b ? v : b;
  }
  __shared__ unsigned long long wmax[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wmax[wid] = b;
  __syncthreads();
  if (wid == 0) {
    b = lane < 8 ? wmax[lane] : 0ULL;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
      b = v > b ? v : b;
    }
    if (lane == 0 && b) atomicMax(&ctr->smax_bits, b);
  }
}

template <int STAGE, int TK>
cudaError_t launch_tk(const StepBuffers& b, const Params& P, const fvd32::Params32& Q, double dt,
                      int kchunk, cudaStream_t s) {
  using S = Shape64<kTileY>;
  const dim3 grid((P.nx + TX - 1) / TX, (P.ny + kTileY - 1) / kTileY,
                  (P.nz + kchunk - 1) / kchunk);
  k_stage64<STAGE, TK><<<grid, S::kThreads, sizeof(Smem64<S>), s>>>(b.U, b.U1, P, Q, dt, kchunk,
                                                                    b.ctr);
  return cudaGetLastError();
}

template <int TK>
cudaError_t raise_smem() {
  const int bytes = (int)sizeof(Smem64<Shape64<kTileY>>);
  cudaError_t e = cudaFuncSetAttribute(k_stage64<1, TK>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_stage64<2, TK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  return e;
}

}  // namespace

cudaError_t prepare_fused() {
  cudaError_t e = raise_smem<THETA_TWO>();
  if (e == cudaSuccess) e = raise_smem<THETA_GENERAL>();
  return e;
}

cudaError_t launch_fused(int stage, const StepBuffers& b, const Params& P, double dt,
                         int kchunk, cudaStream_t s) {
  const fvd32::Params32 Q = fv_fp32::make_params32(P, 2.0);
  if (kchunk < 1) kchunk = 1;
  if (P.theta == 2.0)
    return stage == 1 ? launch_tk<1, THETA_TWO>(b, P, Q, dt, kchunk, s)
                      : launch_tk<2, THETA_TWO>(b, P, Q, dt, kchunk, s);
  return stage == 1 ? launch_tk<1, THETA_GENERAL>(b, P, Q, dt, kchunk, s)
                    : launch_tk<2, THETA_GENERAL>(b, P, Q, dt, kchunk, s);
}

cudaError_t launch_dt(const double* U, const StepBuffers& b, const Params& P, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&b.ctr->smax_bits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const long long n = (long long)P.nx * P.ny * P.nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 8LL * fv_sm_count()) blocks = 8LL * fv_sm_count();
  k_dt64<<<(unsigned)blocks, 256, 0, s>>>(U, P, fv_fp32::make_params32(P, 2.0), b.ctr);
  return cudaGetLastError();
}

}  // namespace FV_NS
