// fv_fused_ff_kernels.cu -- the fused substep with float-float face
// arithmetic (FV_PREC_FP64_FF).
//
// The same kernel structure as fv_fused64_kernels.cu (one launch per
// substep over tiles of 32 x 8 columns marching along z; primitives, half
// slopes and x / y face fluxes of each plane in shared memory, a register
// window along z, the input of the next plane staged by cp.async, flux
// reuse where cells repeat), with the work per face -- differences,
// limited slopes, face states, sound speeds, HLL fluxes -- and the flux
// divergence in float-float (fv_ff.cuh) on the FP32 pipe.  FP64 stays where
// the state is formed and read: the conversion to primitives (FP64 Newton
// forms), the RK combine on the FP64 state and the CFL maximum.  Each
// float-float operation is a few 2^-47 of its operands, so the step lands
// within a few 2^-46 of the FP64 step per substep; the library holds it to
// 1e-12 of each field's scale against the FP64 method.  Physical cells
// outside the float-float operand range (density or pressure outside
// [2^-30, 2^30), a velocity of 2^20 or more) are counted
// (DevCounters::ff_range) and reported by the next synchronising call.
//
// Built with --fmad=false: the error-free transformations need every FP32
// operation rounded on its own (they write their fused multiply-adds out).
#include "fv_device.cuh"
#include "fv_device32.cuh"
#include "fv_ff.cuh"
#include "fv_fused_common.cuh"
#include "fv_internal.h"

using namespace fvd;
using namespace fvfused;
using fvff::ff;
using fvff::PrimF;

namespace fv_fp64_ff {
namespace {

constexpr int kPrefetch = 2;   // planes ahead for the stage-2 RK operand prefetch

// STAGE 1 leaves out `last` (stage 2's CFL cache): 10 KB less shared memory
// per CTA, so that more of the multiprocessor's L1 stays free for the
// register spills.
template <class S, int STAGE>
struct SmemFF {
  double col[2][NF][S::kThreads];   // staged input: the column cell of plane t+2
  double halo[2][NF][S::kHalo];     // staged input: the halo cells of plane t
  ff w[NF][S::PY][S::PX];           // primitives of the plane, tile and halo
  ff hx[NF][S::TY][S::TX + 2];         // x half slopes of cells -1 .. TX
  ff hy[NF][S::TY + 2][S::TX];         // y half slopes of rows -1 .. TY
  ff fx[NF][S::TY][S::TX + 1];         // x face fluxes
  ff fy[NF][S::TY + 1][S::TX];         // y face fluxes
  unsigned char same[S::PY][S::PX]; // the cell equals (bits) the cell a plane below
  double last[NF][STAGE == 2 ? S::kThreads : 1];   // stage 2: the column's last cell written
};

struct ConstFF {
  fvff::ParamsF Q;
  ff inv[3];
};

__device__ __forceinline__ bool physical_ff(const PrimF& w) {
  return fvff::pos(w.r) && fvff::pos(w.p);
}

template <class SM>
__device__ __forceinline__ PrimF smem_w(const SM& s, int row, int col) {
  return PrimF{s.w[0][row][col], s.w[1][row][col], s.w[2][row][col], s.w[3][row][col],
               s.w[4][row][col]};
}
template <class SM>
__device__ __forceinline__ void smem_w_store(SM& s, int row, int col, const PrimF& w) {
  s.w[0][row][col] = w.r;
  s.w[1][row][col] = w.vx;
  s.w[2][row][col] = w.vy;
  s.w[3][row][col] = w.vz;
  s.w[4][row][col] = w.p;
}

// FP64 primitives of a conserved state as float-float; `phys`: physical in
// FP64, `ok`: physical and inside the float-float operand range, or
// non-physical (then counted as such, not as out of range).
__device__ __forceinline__ PrimF prim_ff(const double u[NF], const Params& P, bool& phys,
                                         bool& ok) {
  const Prim w = cons_to_prim(u, P);
  phys = is_pos(w.r) && is_pos(w.p);
  ok = !phys || fvff::ff_operands_ok(w);
  return fvff::to_ff(w);
}

template <int AXIS>
__device__ __forceinline__ void face_flux(const PrimF& wm, const PrimF& hm, const PrimF& wp,
                                          const PrimF& hp, const fvff::ParamsF& Q, ff F[NF],
                                          bool& fb) {
  PrimF wl = fvff::padd(wm, hm);
  PrimF wr = fvff::psub(wp, hp);
  fb = !(physical_ff(wl) && physical_ff(wr));
  if (fb) {
    wl = wm;
    wr = wp;
  }
  fvff::hll_flux<AXIS>(wl, wr, Q, F);
}

__device__ __forceinline__ bool same_ff(ff a, ff b) {
  return __float_as_uint(a.hi) == __float_as_uint(b.hi) &&
         __float_as_uint(a.lo) == __float_as_uint(b.lo);
}

__device__ __forceinline__ bool finite_ff(ff a) { return isfinite(a.hi) && isfinite(a.lo); }

// SKIP: a plane whose tile and halo cells all equal the plane below skips its
// slope and face passes (built for the default 16 x 16 tile at two CTAs per
// SM, both ways; the other shapes run every pass).
template <class S, int STAGE, bool MC, bool SKIP>
__device__ __forceinline__ void stageff_tile(SmemFF<S, STAGE>& s, double* __restrict__ U,
                                             double* __restrict__ U1, const Params& P,
                                             const fvd32::Params32& Q32, const ConstFF& C,
                                             double dt, int i0, int j0, int k0, int k1,
                                             unsigned& fallbacks_out,
                                             unsigned long long& bad_out,
                                             unsigned long long& range_out, unsigned& evaluated,
                                             double& smax, float& smax_f,
                                             unsigned long long& bad_next,
                                             unsigned long long* gmax) {
  const double* __restrict__ src = STAGE == 1 ? U : U1;
  constexpr int kThreads = S::kThreads, kHalo = S::kHalo, kHaloPer = S::kHaloPer;
  constexpr int TY = S::TY;
  constexpr int TX = S::TX;
  const int tid = threadIdx.x;
  const int ti = tid % TX, tj = tid / TX;
  const long long nf = P.nfield;
  const fvff::ParamsF& Q = C.Q;
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
  unsigned fallbacks = 0, xyfb = 0;
  unsigned long long bad = 0, range = 0;
  unsigned last_bad = 0;   // stage 2: whether the column's last cell written was non-physical
  // the x / y part of the last update's zero-divergence test (every x and y
  // flux difference of the column's cell zero and finite); a skipped plane
  // (below) has the same x and y fluxes, so the part carries over
  bool zxy_prev = false;

  // z window prologue: planes k0-2 .. k0+1 of the column; per plane whether
  // its cell is physical and inside the float-float range (counted at k)
  auto load_ff = [&](int gk, bool& phys, bool& ok) {
    double u[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) u[q] = src[q * nf + col + (long long)gk * P.sz];
    return prim_ff(u, P, phys, ok);
  };
  bool phm, okm;
  const PrimF wm2 = load_ff(k0 + 0, phm, okm);
  const PrimF wm1 = load_ff(k0 + 1, phm, okm);
  bool ph0, ok0, ph1, ok1;
  PrimF w0 = load_ff(k0 + 2, ph0, ok0);
  PrimF w1 = load_ff(k0 + 3, ph1, ok1);
  PrimF h0 = fvff::half_slopes<MC>(Q.theta, fvff::psub(w0, wm1), fvff::psub(w1, w0));
  ff fz_lo[NF];
  bool zfb;
  {
    const PrimF hm1 = fvff::half_slopes<MC>(Q.theta, fvff::psub(wm1, wm2), fvff::psub(w0, wm1));
    face_flux<2>(wm1, hm1, w0, h0, Q, fz_lo, zfb);
    ++evaluated;
    if (zfb && k0 == 0 && owner) ++fallbacks;
  }
  int run = fvff::same_bits(wm1, wm2) ? 2 : 1;
  run = fvff::same_bits(w0, wm1) ? run + 1 : 1;
  run = fvff::same_bits(w1, w0) ? run + 1 : 1;
  bool same0 = false, same1 = fvff::same_bits(w1, w0);

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
    const bool later = k > k0;
    if (owner) {
      bad += !ph0;
      range += !ok0;
    }
    // stage 2: the launch's shared CFL maximum, read now and used at the
    // plane's folds, so the read's latency overlaps the plane's work (any
    // value read is a lower bound of the final maximum)
    const unsigned long long gpeek = STAGE == 2 ? fvd32::peek_max(gmax) : 0ull;
    const long long g = col + (long long)(k + 2) * P.sz;
    cp_async_wait_all();
    // (a) the column cell of plane k+2
    double uc[NF];
    bool eqc = later;
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      uc[q] = s.col[slot][q][tid];
      eqc = eqc && bits(uc[q]) == bits(s.col[prev][q][tid]);
    }
    PrimF w2 = w1;
    bool ph2 = ph1, ok2 = ok1;
    if (!__all_sync(0xffffffffu, eqc)) w2 = prim_ff(uc, P, ph2, ok2);
    if (eqc) {
      ph2 = ph1;
      ok2 = ok1;
    }
    const bool same2 = eqc || fvff::same_bits(w2, w1);
    run = same2 ? run + 1 : 1;
    // (c) z flux of face k+1/2
    PrimF h1;
    ff fz_hi[NF];
    if (__all_sync(0xffffffffu, run >= 5)) {
      const ff z{0.0f, 0.0f};
      h1 = PrimF{z, z, z, z, z};
#pragma unroll
      for (int q = 0; q < NF; ++q) fz_hi[q] = fz_lo[q];
    } else {
      h1 = fvff::half_slopes<MC>(Q.theta, fvff::psub(w1, w0), fvff::psub(w2, w1));
      face_flux<2>(w0, h0, w1, h1, Q, fz_hi, zfb);
      ++evaluated;
    }
    if (zfb && owner) ++fallbacks;
    // (b) the halo cells of plane k
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
    // stage 2 reads U only in the update: fetch the column cell kPrefetch
    // planes ahead into L2 (inside the ghosted array: plane k + 2 + kPrefetch
    // <= nz + 1).  3.5% on the 256^3 oblique problem.
    if (STAGE == 2 && owner && k + kPrefetch < k1) {
      const double* pu = U + g + (long long)kPrefetch * P.sz;
#pragma unroll
      for (int q = 0; q < NF; ++q) prefetch_l2(pu + q * nf);
    }
    // (d) the plane's primitives into shared memory (a cell equal to the one a
    // plane below is there already, bit for bit)
    const bool col_same = later && same0;
    if (!col_same) smem_w_store(s, tj + 2, ti + 2, w0);
    s.same[tj + 2][ti + 2] = col_same;
    bool plane_same = col_same;
#pragma unroll
    for (int e = 0; e < kHaloPer; ++e) {
      const int h = tid + e * kThreads;
      const bool all_eq = __all_sync(0xffffffffu, eqh[e] || h >= kHalo);
      if (h < kHalo) {
        if (!all_eq) {
          bool ph, ok;
          smem_w_store(s, hrow[e] + 2, hcol[e] + 2, prim_ff(uh[e], P, ph, ok));
        }
        s.same[hrow[e] + 2][hcol[e] + 2] = eqh[e];
        plane_same = plane_same && eqh[e];
      }
    }
    // every cell of the tile and its halo equals the cell a plane below: each
    // slope and x / y face of this plane would keep its value (the passes
    // below would only read flags), so the CTA skips them and their barriers
    bool skip = false;
    if (SKIP) skip = __syncthreads_and(plane_same) != 0;
    else __syncthreads();
    if (skip) {
      fallbacks += __popc(xyfb & counted & ((1u << S::kFacePer) - 1u));
    } else {
    // (e) half slopes along x and y
#pragma unroll 1
    for (int p = 0; p < S::kSlopePer; ++p) {
      const int t = tid + p * kThreads;
      if (t < S::kXSlopes) {
        const int r = t / (TX + 2), c = t % (TX + 2);
        const bool keep = s.same[r + 2][c] & s.same[r + 2][c + 1] & s.same[r + 2][c + 2];
        if (!__all_sync(__activemask(), keep)) {
          const PrimF wa = smem_w(s, r + 2, c), wb = smem_w(s, r + 2, c + 1),
                      wc = smem_w(s, r + 2, c + 2);
          const PrimF h = fvff::half_slopes<MC>(Q.theta, fvff::psub(wb, wa), fvff::psub(wc, wb));
          s.hx[0][r][c] = h.r;
          s.hx[1][r][c] = h.vx;
          s.hx[2][r][c] = h.vy;
          s.hx[3][r][c] = h.vz;
          s.hx[4][r][c] = h.p;
        }
      } else if (t < S::kSlopes) {
        const int u = t - S::kXSlopes, r = u / TX, c = u % TX;
        const bool keep = s.same[r][c + 2] & s.same[r + 1][c + 2] & s.same[r + 2][c + 2];
        if (!__all_sync(__activemask(), keep)) {
          const PrimF wa = smem_w(s, r, c + 2), wb = smem_w(s, r + 1, c + 2),
                      wc = smem_w(s, r + 2, c + 2);
          const PrimF h = fvff::half_slopes<MC>(Q.theta, fvff::psub(wb, wa), fvff::psub(wc, wb));
          s.hy[0][r][c] = h.r;
          s.hy[1][r][c] = h.vx;
          s.hy[2][r][c] = h.vy;
          s.hy[3][r][c] = h.vz;
          s.hy[4][r][c] = h.p;
        }
      }
    }
    __syncthreads();
    // (f) x and y face fluxes
#pragma unroll 1
    for (int p = 0; p < S::kFacePer; ++p) {
      const int f = tid + p * kThreads;
      if (f < S::kXFaces) {
        const int r = f / (TX + 1), fi = f % (TX + 1);
        const bool keep = s.same[r + 2][fi] & s.same[r + 2][fi + 1] & s.same[r + 2][fi + 2] &
                          s.same[r + 2][fi + 3];
        if (!__all_sync(__activemask(), keep)) {
          const PrimF hm{s.hx[0][r][fi], s.hx[1][r][fi], s.hx[2][r][fi], s.hx[3][r][fi],
                         s.hx[4][r][fi]};
          const PrimF hp{s.hx[0][r][fi + 1], s.hx[1][r][fi + 1], s.hx[2][r][fi + 1],
                         s.hx[3][r][fi + 1], s.hx[4][r][fi + 1]};
          ff F[NF];
          bool fb;
          face_flux<0>(smem_w(s, r + 2, fi + 1), hm, smem_w(s, r + 2, fi + 2), hp, Q, F, fb);
          xyfb = (xyfb & ~(1u << p)) | ((unsigned)fb << p);
          ++evaluated;
#pragma unroll
          for (int q = 0; q < NF; ++q) s.fx[q][r][fi] = F[q];
        }
      } else if (f < S::kFaces) {
        const int u = f - S::kXFaces, fj = u / TX, c = u % TX;
        const bool keep = s.same[fj][c + 2] & s.same[fj + 1][c + 2] & s.same[fj + 2][c + 2] &
                          s.same[fj + 3][c + 2];
        if (!__all_sync(__activemask(), keep)) {
          const PrimF hm{s.hy[0][fj][c], s.hy[1][fj][c], s.hy[2][fj][c], s.hy[3][fj][c],
                         s.hy[4][fj][c]};
          const PrimF hp{s.hy[0][fj + 1][c], s.hy[1][fj + 1][c], s.hy[2][fj + 1][c],
                         s.hy[3][fj + 1][c], s.hy[4][fj + 1][c]};
          ff F[NF];
          bool fb;
          face_flux<1>(smem_w(s, fj + 1, c + 2), hm, smem_w(s, fj + 2, c + 2), hp, Q, F, fb);
          xyfb = (xyfb & ~(1u << p)) | ((unsigned)fb << p);
          ++evaluated;
#pragma unroll
          for (int q = 0; q < NF; ++q) s.fy[q][fj][c] = F[q];
        }
      }
      fallbacks += (xyfb >> p) & (counted >> p) & 1u;
    }
    __syncthreads();
    }
    // (g) update: float-float divergence, the RK combine in FP64 on the FP64
    // state (a copy / half sum where every flux difference is zero)
    if (owner) {
      // first the zero test over all components, then the arithmetic one
      // component at a time (few values live at once)
      bool zxy = zxy_prev, zz = true;
      if (!skip) {
        zxy = true;
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          const ff xr = s.fx[q][tj][ti + 1], yr = s.fy[q][tj + 1][ti];
          zxy = zxy && same_ff(s.fx[q][tj][ti], xr) && same_ff(s.fy[q][tj][ti], yr) &&
                finite_ff(xr) && finite_ff(yr);
        }
        zxy_prev = zxy;
      }
#pragma unroll
      for (int q = 0; q < NF; ++q) zz = zz && same_ff(fz_lo[q], fz_hi[q]) && finite_ff(fz_hi[q]);
      const bool zero = zxy && zz;
      double un[NF];
      if (__all_sync(__activemask(), zero)) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          const double r0 = U[q * nf + g];
          if (STAGE == 1) U1[q * nf + g] = r0;
          else U[q * nf + g] = un[q] = half(r0 + U1[q * nf + g]);
        }
      } else {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          ff acc = fvff::mul(fvff::sub(s.fx[q][tj][ti], s.fx[q][tj][ti + 1]), C.inv[0]);
          acc = fvff::sub(acc, fvff::mul(fvff::sub(s.fy[q][tj + 1][ti], s.fy[q][tj][ti]),
                                         C.inv[1]));
          acc = fvff::sub(acc, fvff::mul(fvff::sub(fz_hi[q], fz_lo[q]), C.inv[2]));
          const double du = dt * fvff::to_double(acc);
          const double r0 = U[q * nf + g];
          if (STAGE == 1) U1[q * nf + g] = r0 + du;
          else U[q * nf + g] = un[q] = half((r0 + U1[q * nf + g]) + du);
        }
      }
      if (STAGE == 2) {
        // the column's last cell written: a cell equal to it changes
        // nothing but the count (fvd32::fold_speed, its cache in shared memory)
        fvd32::SpeedCache cache;
        cache.valid = k > k0;
#pragma unroll
        for (int q = 0; q < NF; ++q) cache.u[q] = s.last[q][tid];
        cache.bad = last_bad;
        fvd32::raise_max(gpeek, smax, smax_f);
        fvd32::fold_speed(un, P, Q32, smax, smax_f, bad_next, cache, gmax);
#pragma unroll
        for (int q = 0; q < NF; ++q) s.last[q][tid] = un[q];
        last_bad = cache.bad;
      }
    }
#pragma unroll
    for (int q = 0; q < NF; ++q) fz_lo[q] = fz_hi[q];
    w0 = w1;
    w1 = w2;
    h0 = h1;
    same0 = same1;
    same1 = same2;
    ph0 = ph1;
    ok0 = ok1;
    ph1 = ph2;
    ok1 = ok2;
  }
  fallbacks_out += fallbacks;
  bad_out += bad;
  range_out += range;
}

__device__ __forceinline__ void max_to(unsigned long long* dst, double smax) {
  unsigned long long b = (unsigned long long)__double_as_longlong(smax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
    b = v > b ? v : b;
  }
  if ((threadIdx.x & 31u) == 0u && b) atomicMax(dst, b);
}

// TXV x TY: the tile (one thread per column); MINB: CTAs per SM the kernel
// is built for.  Built as 16 x 16 at 2 CTAs per SM (the default: 16 warps,
// 128 registers with spills; a warp covers 16 x 2 cells, so its reuse
// decisions hold more often next to the waves, and a halo cell serves 1.8
// columns) or 1 (8 warps, up to 255 registers); 32 x 8 at 2 or 1; and 32 x 16
// at 1 (16 warps, 128 registers).
template <int STAGE, bool MC, int TXV, int TY, int MINB, bool SKIP>
__global__ void __launch_bounds__(TXV * TY, MINB)
k_stageff(double* __restrict__ U, double* __restrict__ U1, Params P, fvd32::Params32 Q32,
          ConstFF C, double dt, int kchunk, DevCounters* ctr) {
  using S = Shape64<TY, TXV>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemFF<S, STAGE>& s = *reinterpret_cast<SmemFF<S, STAGE>*>(smem_raw);
  unsigned fallbacks = 0, evaluated = 0;
  unsigned long long bad = 0, range = 0, bad_next = 0;
  double smax = 0.0;
  float smax_f = 0.0f;
  const int k0 = blockIdx.z * kchunk;
  stageff_tile<S, STAGE, MC, SKIP>(s, U, U1, P, Q32, C, dt, blockIdx.x * TXV, blockIdx.y * TY, k0,
                             min(k0 + kchunk, P.nz), fallbacks, bad, range, evaluated, smax,
                             smax_f, bad_next, &ctr->smax_next);
  if (fallbacks) atomicAdd(&ctr->fallback, (unsigned long long)fallbacks);
  if (bad) atomicAdd(&ctr->np_step, bad);
  if (range) atomicAdd(&ctr->ff_range, range);
  warp_count(&ctr->faces, evaluated);
  if (STAGE == 2) {
    max_to(&ctr->smax_next, smax);
    if (bad_next) atomicAdd(&ctr->np_dt, bad_next);
  }
}

// The CFL maximum of U with the arithmetic of k_stageff's stage-2 epilogue.
__global__ void __launch_bounds__(256)
k_dtff(const double* __restrict__ U, Params P, fvd32::Params32 Q, DevCounters* ctr) {
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

// A double as float-float on the host: hi its nearest float, lo the
// remainder's.
ff host_ff(double x) {
  const float hi = (float)x;
  return ff{hi, (float)(x - (double)hi)};
}

ConstFF make_const(const Params& P) {
  ConstFF C;
  C.Q.gamma = host_ff(P.gamma);
  C.Q.igm1 = host_ff(P.igm1);
  C.Q.theta = host_ff(P.theta);
  for (int a = 0; a < 3; ++a) C.inv[a] = host_ff(P.inv_d[a]);
  return C;
}

// The shape built with the plane skip as well: 16 x 16 at two CTAs per SM
// (the default).
template <int TXV, int TY, int MINB>
constexpr bool kSkipShape = TXV == 16 && TY == 16 && MINB == 2;

template <int STAGE, bool MC, int TXV, int TY, int MINB>
cudaError_t launch_mc(const StepBuffers& b, const Params& P, double dt, int kchunk,
                      bool plane_skip, cudaStream_t s) {
  using S = Shape64<TY, TXV>;
  const dim3 grid((P.nx + TXV - 1) / TXV, (P.ny + TY - 1) / TY, (P.nz + kchunk - 1) / kchunk);
  constexpr size_t bytes = sizeof(SmemFF<S, STAGE>);
  if constexpr (kSkipShape<TXV, TY, MINB>) {
    if (plane_skip) {
      k_stageff<STAGE, MC, TXV, TY, MINB, true><<<grid, S::kThreads, bytes, s>>>(
          b.U, b.U1, P, fv_fp32::make_params32(P, 2.0), make_const(P), dt, kchunk, b.ctr);
      return cudaGetLastError();
    }
  }
  k_stageff<STAGE, MC, TXV, TY, MINB, false><<<grid, S::kThreads, bytes, s>>>(
      b.U, b.U1, P, fv_fp32::make_params32(P, 2.0), make_const(P), dt, kchunk, b.ctr);
  return cudaGetLastError();
}

template <bool MC, int TXV, int TY, int MINB, bool SKIP>
cudaError_t raise_smem_skip() {
  using S = Shape64<TY, TXV>;
  cudaError_t e = cudaFuncSetAttribute(k_stageff<1, MC, TXV, TY, MINB, SKIP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(SmemFF<S, 1>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_stageff<2, MC, TXV, TY, MINB, SKIP>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemFF<S, 2>));
  return e;
}

template <bool MC, int TXV, int TY, int MINB>
cudaError_t raise_smem() {
  if constexpr (kSkipShape<TXV, TY, MINB>) {
    const cudaError_t e = raise_smem_skip<MC, TXV, TY, MINB, true>();
    if (e != cudaSuccess) return e;
  }
  return raise_smem_skip<MC, TXV, TY, MINB, false>();
}

template <int TXV, int TY, int MINB>
cudaError_t raise_both() {
  cudaError_t e = raise_smem<true, TXV, TY, MINB>();
  return e == cudaSuccess ? raise_smem<false, TXV, TY, MINB>() : e;
}

template <int TXV, int TY, int MINB>
cudaError_t launch_shape(int stage, const StepBuffers& b, const Params& P, double dt,
                         int kchunk, bool skip, cudaStream_t s) {
  const bool mc = P.theta == 2.0;
  if (stage == 1) return mc ? launch_mc<1, true, TXV, TY, MINB>(b, P, dt, kchunk, skip, s)
                            : launch_mc<1, false, TXV, TY, MINB>(b, P, dt, kchunk, skip, s);
  return mc ? launch_mc<2, true, TXV, TY, MINB>(b, P, dt, kchunk, skip, s)
            : launch_mc<2, false, TXV, TY, MINB>(b, P, dt, kchunk, skip, s);
}

}  // namespace

bool valid_fused_config(int tile_x, int tile_y, int ctas_per_sm) {
  if (tile_x == 16) return tile_y == 16 && (ctas_per_sm == 1 || ctas_per_sm == 2);
  return tile_x == 32 && ((tile_y == 8 && (ctas_per_sm == 1 || ctas_per_sm == 2)) ||
                          (tile_y == 16 && ctas_per_sm == 1));
}

cudaError_t prepare_fused() {
  cudaError_t e = raise_both<32, 8, 1>();
  if (e == cudaSuccess) e = raise_both<32, 8, 2>();
  if (e == cudaSuccess) e = raise_both<32, 16, 1>();
  if (e == cudaSuccess) e = raise_both<16, 16, 2>();
  if (e == cudaSuccess) e = raise_both<16, 16, 1>();
  return e;
}

cudaError_t launch_fused(int stage, const StepBuffers& b, const Params& P, double dt,
                         int kchunk, int tile_x, int tile_y, int ctas_per_sm, bool plane_skip,
                         cudaStream_t s) {
  if (kchunk < 1) kchunk = 1;
  if (!valid_fused_config(tile_x, tile_y, ctas_per_sm)) return cudaErrorInvalidValue;
  const bool k = plane_skip;
  if (tile_x == 16)
    return ctas_per_sm >= 2 ? launch_shape<16, 16, 2>(stage, b, P, dt, kchunk, k, s)
                            : launch_shape<16, 16, 1>(stage, b, P, dt, kchunk, k, s);
  if (tile_y == 16) return launch_shape<32, 16, 1>(stage, b, P, dt, kchunk, k, s);
  return ctas_per_sm >= 2 ? launch_shape<32, 8, 2>(stage, b, P, dt, kchunk, k, s)
                          : launch_shape<32, 8, 1>(stage, b, P, dt, kchunk, k, s);
}

cudaError_t launch_dt(const double* U, const StepBuffers& b, const Params& P, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&b.ctr->smax_bits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const long long n = (long long)P.nx * P.ny * P.nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 8LL * fv_sm_count()) blocks = 8LL * fv_sm_count();
  k_dtff<<<(unsigned)blocks, 256, 0, s>>>(U, P, fv_fp32::make_params32(P, 2.0), b.ctr);
  return cudaGetLastError();
}

}  // namespace fv_fp64_ff
