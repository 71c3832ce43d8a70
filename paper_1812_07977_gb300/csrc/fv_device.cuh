// fv_device.cuh -- device-side building blocks of the finite-volume step.
//
// FP64 on sm_103a retires about two double-precision operations per SM per
// clock (a warp instruction occupies the DP units for ~16 clocks), while the
// integer and FP32 pipes retire ~128.  Everything here that can be done
// exactly without the DP pipe is therefore done on integers: the sign and
// magnitude tests of the limiter and of the wave-speed maxima, the positivity
// tests, and multiplication by 2 and by 1/2 (an exponent increment, exact
// except at the ends of the exponent range, where the DP multiply is used).
// Each helper returns bit for bit what the corresponding IEEE operation
// returns, so the results stay reproducible against a plain FP64 code.
#pragma once

#include <cstdint>

namespace fvd {

constexpr int NF = 5;  // rho, rho*vx, rho*vy, rho*vz, E  /  rho, vx, vy, vz, p

// Limiter parameter classes with an exact integer form of theta * x.
enum ThetaKind { THETA_GENERAL = 0, THETA_ZERO = 1, THETA_ONE = 2, THETA_TWO = 3 };

struct Params {
  int nx, ny, nz;
  long long sy, sz;       // ghosted strides of y and z (x stride is 1)
  long long nfield;       // doubles per ghosted field
  double gamma;           // ratio of specific heats
  double gm1;             // gamma - 1
  double igm1;            // 1 / (gamma - 1)
  double theta;           // limiter parameter
  double inv_d[3];        // 1 / dx, 1 / dy, 1 / dz
  int bc[3];              // 0 outflow, 1 periodic
};

// ---------------------------------------------------------------- bit tools
__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double from_bits(long long b) { return __longlong_as_double(b); }

constexpr long long kExpOne = 1LL << 52;
constexpr long long kInfBits = 0x7FF0000000000000LL;
constexpr long long kMagMask = 0x7FFFFFFFFFFFFFFFLL;

// x > 0.0 (false for NaN and for -0)
__device__ __forceinline__ bool is_pos(double x) {
  long long b = bits(x);
  return b > 0 && b <= kInfBits;
}

// x is -0 (bit pattern 0x8000000000000000; tested on the two halves)
__device__ __forceinline__ bool is_neg_zero(double x) {
  return (unsigned)__double2hiint(x) == 0x80000000u && (unsigned)__double2loint(x) == 0u;
}

// x is neither infinite nor NaN
__device__ __forceinline__ bool is_finite(double x) {
  return (((unsigned)__double2hiint(x) >> 20) & 0x7FFu) != 0x7FFu;
}

// IEEE product on the FP64 pipe for the rare operands of half() and
// twice().  A volatile asm statement cannot be executed speculatively, so
// the compiler keeps it behind its branch instead of issuing the multiply
// unconditionally and selecting the result (which it does for a plain
// `x * 0.5` and which costs an FP64 issue slot on every call).
__device__ __forceinline__ double dmul_rare(double x, double y) {
  double r;
  asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(x), "d"(y));
  return r;
}

// x * 0.5, bit-identical to the IEEE product
__device__ __forceinline__ double half(double x) {
  long long b = bits(x);
  unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  if (e > 1u && e < 0x7FFu) return from_bits(b - kExpOne);
  return dmul_rare(x, 0.5);
}

// x * 2.0, bit-identical to the IEEE product
__device__ __forceinline__ double twice(double x) {
  long long b = bits(x);
  unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  if (e >= 1u && e < 0x7FEu) return from_bits(b + kExpOne);
  return dmul_rare(x, 2.0);
}

// minmod(a, b, c): the argument of least magnitude if all three are > 0 or
// all three are < 0, else +0.  NaN counts as neither sign.
__device__ __forceinline__ double minmod3(double a, double b, double c) {
  long long ia = bits(a), ib = bits(b), ic = bits(c);
  long long ma = ia & kMagMask, mb = ib & kMagMask, mc = ic & kMagMask;
  bool nz = (ma != 0) & (mb != 0) & (mc != 0) & (ma <= kInfBits) & (mb <= kInfBits) &
            (mc <= kInfBits);
  bool same = ((ia ^ ib) >= 0) & ((ia ^ ic) >= 0);
  long long m = ma;
  long long r = ia;
  if (mb < m) { m = mb; r = ib; }
  if (mc < m) { r = ic; }
  return (nz && same) ? from_bits(r) : 0.0;
}

// max(0, a, b) evaluated as r = 0; if (a > r) r = a; if (b > r) r = b
__device__ __forceinline__ double max0(double a, double b) {
  long long r = 0;
  long long ia = bits(a), ib = bits(b);
  if (ia > 0 && ia <= kInfBits) r = ia;
  if (ib > r && ib <= kInfBits) r = ib;
  return from_bits(r);
}

template <int TK>
__device__ __forceinline__ double theta_times(double theta, double x) {
  if (TK == THETA_TWO) return twice(x);
  if (TK == THETA_ONE) return x;
  return theta * x;
}

// Half of the limited slope of one cell from its two one-sided differences:
// 0.5 * minmod(theta*dm, 0.5*(dm + dp), theta*dp).  With theta = 0 the first
// argument is +-0 (or NaN), so the minmod is +0 whatever dm and dp are.
template <int TK>
__device__ __forceinline__ double half_slope(double theta, double dm, double dp) {
  if (TK == THETA_ZERO) return 0.0;
  return half(minmod3(theta_times<TK>(theta, dm), half(dm + dp), theta_times<TK>(theta, dp)));
}

// ---------------------------------------------------------------- Newton forms
// The FMA build (held to a relative tolerance, not to the bits of IEEE
// division and square root) replaces each correctly rounded divide and
// square root -- about ten FP64 issue slots each on this GPU -- by an FP32
// seed from the SFU, refined by two Newton-Raphson steps in FP64:
//   reciprocal          y <- y + y (1 - d y)               (2 DFMA a step)
//   inverse square root y <- y + (y/2) (1 - u y^2)         (DMUL + 2 DFMA)
// Each step squares the relative error, so a seed within 2^-21 ends within
// about one ulp.  Operands outside [2^-120, 2^120) in magnitude (where the
// seed or its reciprocal would leave the normal FP32 range), zeros, infinities
// and NaNs take the IEEE operation instead.

// IEEE operations for the rare operands, kept behind their branch.
__device__ __forceinline__ double ddiv_rare(double a, double b) {
  double r;
  asm volatile("div.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ double dsqrt_rare(double a) {
  double r;
  asm volatile("sqrt.rn.f64 %0, %1;" : "=d"(r) : "d"(a));
  return r;
}

// |x| in [2^-120, 2^120) (false for zeros, subnormals, infinities and NaNs)
__device__ __forceinline__ bool seed_range(double x) {
  const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7FFu;
  return e - (1023u - 120u) < 240u;
}

// x truncated to FP32 (sign kept), for x with seed_range(x)
__device__ __forceinline__ float seed_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  return __uint_as_float((hi & 0x80000000u) | (((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) |
                         (lo >> 29));
}

// a normal FP32 value widened to FP64 (exact)
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned x = __float_as_uint(f);
  const unsigned hi = (((x & 0x7FFFFFFFu) >> 3) + (896u << 20)) | (x & 0x80000000u);
  return __hiloint2double((int)hi, (int)(x << 29));
}

// 1 / d
__device__ __forceinline__ double recip_nr(double d) {
  if (!seed_range(d)) return ddiv_rare(1.0, d);
  float s;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(seed_f32(d)));
  double y = widen_f32(s);
  double e = fma(-d, y, 1.0);
  y = fma(y, e, y);
  e = fma(-d, y, 1.0);
  return fma(y, e, y);
}

// sqrt(t / r) for the sound speed, t = gamma p: evaluated as t / sqrt(t r),
// i.e. t times the inverse square root of u = t r (no division).  Negative
// or zero operands, and t, r or t r outside the seed range, take the IEEE
// form, so non-physical states give what it gives (NaN for a negative
// quotient).
__device__ __forceinline__ double sound_speed_nr(double t, double r) {
  const double u = t * r;
  if ((__double2hiint(t) | __double2hiint(r)) < 0 || !seed_range(t) || !seed_range(r) ||
      !seed_range(u))
    return dsqrt_rare(ddiv_rare(t, r));
  float s;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(seed_f32(u)));
  double y = widen_f32(s);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double e = fma(-(u * y), y, 1.0);
    y = fma(half(y), e, y);
  }
  return t * y;
}

// ---------------------------------------------------------------- physics
struct Prim { double r, vx, vy, vz, p; };

__device__ __forceinline__ double comp(const Prim& w, int q) {
  return q == 0 ? w.r : q == 1 ? w.vx : q == 2 ? w.vy : q == 3 ? w.vz : w.p;
}

// conserved -> primitive: ir = 1/rho, v = m*ir,
// p = (gamma-1) * (E - 0.5*((mx*vx + my*vy) + mz*vz))
__device__ __forceinline__ Prim cons_to_prim(const double u[NF], const Params& P) {
  Prim w;
#ifdef FV_NEWTON_DIVSQRT
  double ir = recip_nr(u[0]);
#else
  double ir = 1.0 / u[0];
#endif
  w.r = u[0];
  w.vx = u[1] * ir;
  w.vy = u[2] * ir;
  w.vz = u[3] * ir;
  double ke = half((u[1] * w.vx + u[2] * w.vy) + u[3] * w.vz);
  w.p = P.gm1 * (u[4] - ke);
  return w;
}

// ---------------------------------------------------------------- time step
// CFL signal speed of one cell (ComputeTimeStep):
// s = ((|vx|+c)/dx + (|vy|+c)/dy) + (|vz|+c)/dz with c = sqrt((gamma p)/rho):
// IEEE operations in this order, or the Newton forms in the FMA build.
__device__ __forceinline__ double cell_speed(const Prim& w, const Params& P) {
#ifdef FV_NEWTON_DIVSQRT
  const double c = sound_speed_nr(P.gamma * w.p, w.r);
#else
  const double c = sqrt(P.gamma * w.p / w.r);
#endif
  return ((fabs(w.vx) + c) * P.inv_d[0] + (fabs(w.vy) + c) * P.inv_d[1]) +
         (fabs(w.vz) + c) * P.inv_d[2];
}

// x as a float rounded toward zero (|result| <= |x|, relative error below
// 2^-23), on the integer pipe; `ok` is cleared unless x is +-0 or
// 2^-100 <= |x| < 2^101.
__device__ __forceinline__ float trunc_f32(double x, bool& ok) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (((hi << 1) | lo) == 0u) return 0.0f;
  ok = ok && e - (1023u - 100u) <= 200u;
  const unsigned f = ((e - 896u) << 23) | ((hi & 0x000FFFFFu) << 3) | (lo >> 29);
  return __uint_as_float(f | (hi & 0x80000000u));
}

// An upper bound of cell_speed(w) from FP32 arithmetic: inputs truncated
// (relative error < 2^-23 each) and about ten FP32 operations (< 2^-23 each)
// give s32 within 2^-19 of the exact speed, and s32 (1 + 2^-14) is above
// the exact speed and above the FP64 cell_speed (within 2 ulps of it).
// +inf when rho or p is not positive or an operand is outside the range of
// trunc_f32 (the FP64 speed is then always computed).
__device__ __forceinline__ float speed_bound(const Prim& w, float g32, const float i32[3]) {
  bool ok = true;
  const float r = trunc_f32(w.r, ok), p = trunc_f32(w.p, ok);
  const float vx = trunc_f32(w.vx, ok), vy = trunc_f32(w.vy, ok), vz = trunc_f32(w.vz, ok);
  if (!(ok && r > 0.0f && p > 0.0f)) return __int_as_float(0x7F800000);
  const float c = __fsqrt_rn(__fdiv_rn(__fmul_rn(g32, p), r));
  const float sp = __fadd_rn(__fadd_rn(__fmul_rn(__fadd_rn(fabsf(vx), c), i32[0]),
                                       __fmul_rn(__fadd_rn(fabsf(vy), c), i32[1])),
                             __fmul_rn(__fadd_rn(fabsf(vz), c), i32[2]));
  return __fmul_ru(sp, 1.0f + 0x1p-14f);
}

// One side of a face: conserved state, normal flux, sound speed.
template <int AXIS>
struct Side {
  double u[NF];
  double f[NF];
  double c;
  double vn;
};

template <int AXIS>
__device__ __forceinline__ void euler_side(const Prim& w, const Params& P, Side<AXIS>& s) {
  double mx = w.r * w.vx;
  double my = w.r * w.vy;
  double mz = w.r * w.vz;
  double ke = half((mx * w.vx + my * w.vy) + mz * w.vz);
  s.u[0] = w.r;
  s.u[1] = mx;
  s.u[2] = my;
  s.u[3] = mz;
  s.u[4] = w.p * P.igm1 + ke;
  double vn = AXIS == 0 ? w.vx : AXIS == 1 ? w.vy : w.vz;
  double mn = AXIS == 0 ? mx : AXIS == 1 ? my : mz;
  s.vn = vn;
#ifdef FV_NEWTON_DIVSQRT
  s.c = sound_speed_nr(P.gamma * w.p, w.r);
#else
  s.c = sqrt(P.gamma * w.p / w.r);
#endif
  s.f[0] = mn;
  s.f[1] = mn * w.vx;
  s.f[2] = mn * w.vy;
  s.f[3] = mn * w.vz;
  s.f[1 + AXIS] = s.f[1 + AXIS] + w.p;
  s.f[4] = (s.u[4] + w.p) * vn;
}

// HLL flux (Harten, Lax & van Leer 1983) with wave bounds from both sides:
// a+ = max(0, vL + cL, vR + cR), a- = max(0, cL - vL, cR - vR),
// F = ((a+ FL + a- FR) - a+ a- (UR - UL)) * (1 / (a+ + a-)).
template <int AXIS>
__device__ __forceinline__ void hll_flux(const Prim& wl, const Prim& wr, const Params& P,
                                         double F[NF]) {
  Side<AXIS> L, R;
  euler_side<AXIS>(wl, P, L);
  euler_side<AXIS>(wr, P, R);
  double ap = max0(L.vn + L.c, R.vn + R.c);
  double am = max0(L.c - L.vn, R.c - R.vn);
#ifdef FV_NEWTON_DIVSQRT
  double r = recip_nr(ap + am);
#else
  double r = 1.0 / (ap + am);
#endif
  double apm = ap * am;
#pragma unroll
  for (int q = 0; q < NF; ++q) F[q] = ((ap * L.f[q] + am * R.f[q]) - apm * (R.u[q] - L.u[q])) * r;
}

// Source index of a ghost coordinate g along an axis of n interior cells.
__device__ __forceinline__ int ghost_source(int g, int n, int bc) {
  if (g >= 0 && g < n) return g;
  if (bc == 1) {
    int r = g % n;
    return r < 0 ? r + n : r;
  }
  return g < 0 ? 0 : n - 1;
}

// Number of ghost (ring) cells of one field.
__host__ __device__ __forceinline__ long long ring_cells(const Params& P) {
  const long long X = P.nx + 4, Y = P.ny + 4;
  return 4 * Y * X + 4 * (long long)P.nz * X + 4 * (long long)P.nz * P.ny;
}

// The (i, j, k) of ring cell t, in the integer type I (32-bit unsigned
// division is a short sequence, 64-bit a long emulated one).
template <class I>
__device__ __forceinline__ void ghost_ijk(const Params& P, I t, int& i, int& j, int& k) {
  const I X = (I)P.nx + 4, Y = (I)P.ny + 4, nz = (I)P.nz, ny = (I)P.ny;
  const I nz_slab = 4 * Y * X;
  const I ny_slab = 4 * nz * X;
  if (t < nz_slab) {
    const I s = t / (Y * X), r = t - s * (Y * X);
    k = s < 2 ? (int)s - 2 : P.nz + (int)s - 2;
    j = (int)(r / X) - 2;
    i = (int)(r % X) - 2;
  } else if (t < nz_slab + ny_slab) {
    const I u = t - nz_slab;
    const I kk = u / (4 * X), r = u - kk * (4 * X);
    const int s = (int)(r / X);
    k = (int)kk;
    j = s < 2 ? s - 2 : P.ny + s - 2;
    i = (int)(r % X) - 2;
  } else {
    const I u = t - nz_slab - ny_slab;
    const I row = u / 4;
    const int s = (int)(u - row * 4);
    k = (int)(row / ny);
    j = (int)(row % ny);
    i = s < 2 ? s - 2 : P.nx + s - 2;
  }
}

// Ghost fill of ring cell t (0 <= t < ring_cells) of all five fields.  The
// axis-by-axis fill (x, then y, then z, each over the full ghosted extent of
// the other axes) leaves every ghost cell equal to the interior cell
// (src_x(i), src_y(j), src_z(k)), so each ring cell is written once, straight
// from its source.  Ring cells are enumerated as the z slabs (4 full
// planes), the y slabs of the interior planes and the x slabs of the
// interior rows.
__device__ __forceinline__ void fill_ghost_cell(double* __restrict__ U, const Params& P,
                                                long long t) {
  int i, j, k;
  // every mesh that fits in memory has far fewer than 2^31 ring cells; the
  // 64-bit form stays for any other
  if (ring_cells(P) < (1LL << 31)) ghost_ijk<unsigned>(P, (unsigned)t, i, j, k);
  else ghost_ijk<long long>(P, t, i, j, k);
  const int si = ghost_source(i, P.nx, P.bc[0]);
  const int sj = ghost_source(j, P.ny, P.bc[1]);
  const int sk = ghost_source(k, P.nz, P.bc[2]);
  const long long dst = (k + 2) * P.sz + (j + 2) * P.sy + (i + 2);
  const long long src = (sk + 2) * P.sz + (sj + 2) * P.sy + (si + 2);
#pragma unroll
  for (int q = 0; q < NF; ++q) U[q * P.nfield + dst] = U[q * P.nfield + src];
}

}  // namespace fvd
