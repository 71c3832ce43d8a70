// fv_ff.cuh -- float-float arithmetic for the face work of the FP64 step.
//
// On sm_103a an FP64 instruction occupies the FP64 pipe for 64 times as long
// as an FP32 instruction occupies the FP32 pipe (2 against 128 lane
// operations per SM and clock), so the finite-volume step in FP64 is bound by
// the FP64 pipe.  A float-float value is an unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2: a 48-bit significand (relative
// precision 2^-48 per value, a few 2^-47 per operation) computed on the FP32
// pipe.  The operations below follow Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18 (1971), and Knuth,
// TAOCP vol. 2, Sec. 4.2.2 (TwoSum, Fast2Sum, the double-length product with
// a fused multiply-add); they are error-free transformations only under
// round-to-nearest FP32 arithmetic without reassociation, so every operation
// is written out with an explicit rounding intrinsic and the translation
// unit is built without contraction.
#pragma once

#include <cstdint>

#include "fv_device.cuh"
#include "fv_device32.cuh"

namespace fvff {

using fvd::NF;

struct ff {
  float hi, lo;
};

// ---------------------------------------------------------------- basics
// s + e == a + b exactly (TwoSum, 6 operations)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return ff{s, e};
}

// s + e == a + b exactly when |a| >= |b| or a == 0 (Fast2Sum, 3 operations)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e == a * b exactly (barring underflow)
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff neg(ff a) { return ff{-a.hi, -a.lo}; }

// a + b: the high parts summed exactly, the low parts added to the error,
// renormalised (relative error a few 2^-47 of |a| + |b|)
__device__ __forceinline__ ff add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ ff sub(ff a, ff b) { return add(a, neg(b)); }

// a * b
__device__ __forceinline__ ff mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// a * 2^k for k = -1 (half) and 1 (twice): exact unless it under- or
// overflows, which the float-float path's operand range excludes
__device__ __forceinline__ ff half(ff a) { return ff{__fmul_rn(a.hi, 0.5f), __fmul_rn(a.lo, 0.5f)}; }
__device__ __forceinline__ ff twice(ff a) { return ff{__fmul_rn(a.hi, 2.0f), __fmul_rn(a.lo, 2.0f)}; }

// 1 / a: the FP32 reciprocal refined by one Newton step in float-float,
// y1 = y0 + y0 (1 - a y0)
__device__ __forceinline__ ff recip(ff a) {
  const float y0 = __frcp_rn(a.hi);
  const ff ay = two_prod(a.hi, y0);
  // e = 1 - a y0, with a.lo's share; small, so FP32 suffices for it
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, ay.hi), ay.lo), __fmul_rn(a.lo, y0));
  return fast_two_sum(y0, __fmul_rn(y0, e));
}

// 1 / sqrt(a) for a > 0: the FP32 estimate refined by one Newton step,
// y1 = y0 + (y0 / 2)(1 - a y0^2)
__device__ __forceinline__ ff rsqrt(ff a) {
  const float y0 = rsqrtf(a.hi);
  const ff y2 = two_prod(y0, y0);
  const ff ay2 = mul(a, y2);
  const float e = __fsub_rn(__fsub_rn(1.0f, ay2.hi), ay2.lo);
  return fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e));
}

// a > 0 (false for NaN)
__device__ __forceinline__ bool pos(ff a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }

// a > b
__device__ __forceinline__ bool gt(ff a, ff b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

// max(0, a, b) in the order r = 0; if (a > r) r = a; if (b > r) r = b
__device__ __forceinline__ ff max0(ff a, ff b) {
  ff r{0.0f, 0.0f};
  if (gt(a, r)) r = a;
  if (gt(b, r)) r = b;
  return r;
}

// |a| < |b|
__device__ __forceinline__ bool abs_lt(ff a, ff b) {
  const float ah = fabsf(a.hi), bh = fabsf(b.hi);
  if (ah != bh) return ah < bh;
  const float al = a.hi < 0.0f ? -a.lo : a.lo, bl = b.hi < 0.0f ? -b.lo : b.lo;
  return al < bl;
}

// sign: +1 for a > 0, -1 for a < 0, 0 for zero (the sign of hi, which
// carries the value's sign unless hi is 0, and then lo is 0 too)
__device__ __forceinline__ int sgn(ff a) { return a.hi > 0.0f ? 1 : (a.hi < 0.0f ? -1 : 0); }

// minmod(a, b, c): the argument of least magnitude when all three have one
// strict sign, else 0
__device__ __forceinline__ ff minmod3(ff a, ff b, ff c) {
  const int s = sgn(a);
  if (s == 0 || sgn(b) != s || sgn(c) != s) return ff{0.0f, 0.0f};
  ff m = a;
  if (abs_lt(b, m)) m = b;
  if (abs_lt(c, m)) m = c;
  return m;
}

// ---------------------------------------------------------------- conversions
// A double as float-float, on the integer pipe: hi = x rounded to FP32,
// lo = (x - hi) rounded to FP32, from x's low 29 significand bits; exact to
// 48 bits for 2^-100 <= |x| < 2^100.  Below that range lo is 0 (hi alone,
// an absolute error under 2^-124); above it the result is not used (the
// range check of to_ff excludes it).
__device__ __forceinline__ ff from_double(double x) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned e = (h >> 20) & 0x7FFu;
  const float hi = fvd32::d2f(x);
  if (e - (1023u - 100u) >= 200u) return ff{hi, 0.0f};
  // x - hi in units of x's last bit (2^(e - 1075)): the low 29 bits, less
  // 2^29 when hi was rounded up (hi's bits then exceed x's top bits by one,
  // a carry into the exponent included)
  const unsigned hm = __float_as_uint(hi) & 0x7FFFFFFFu;
  const unsigned xtop = ((e - 896u) << 23) | ((h & 0x000FFFFFu) << 3) | (l >> 29);
  const int up = (int)(hm - xtop);
  const int r = (int)(l & 0x1FFFFFFFu) - (up << 29);
  // r 2^(e - 1075) = (r 2^-52) 2^(e - 1023), both factors normal floats
  float lo = __fmul_rn(__int2float_rn(r), 0x1p-52f);
  lo = __fmul_rn(lo, __uint_as_float((e - 1023u + 127u) << 23));
  if ((h >> 31) != 0u) lo = -lo;
  return ff{hi, lo};
}

// The float-float path's operand range: density and pressure of magnitude
// in [2^-30, 2^30), velocities below 2^20, so that the products of the flux
// (up to rho v^2 (a+)(a-) ~ 2^112) stay inside the FP32 normal range with
// their low parts, and the sound speed keeps its relative precision.
__device__ __forceinline__ bool in_range(double x, unsigned lo_exp, unsigned span) {
  const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7FFu;
  return e - lo_exp < span;
}
__device__ __forceinline__ bool ff_operands_ok(const fvd::Prim& w) {
  return in_range(w.r, 1023u - 30u, 60u) && in_range(w.p, 1023u - 30u, 60u) &&
         in_range(w.vx, 0u, 1023u + 20u) && in_range(w.vy, 0u, 1023u + 20u) &&
         in_range(w.vz, 0u, 1023u + 20u);
}

// hi + lo as a double (exact: 48 significant bits fit in 53)
__device__ __forceinline__ double to_double(ff a) {
  return fvd32::f2d(a.hi) + fvd32::f2d(a.lo);
}

// ---------------------------------------------------------------- physics
struct PrimF { ff r, vx, vy, vz, p; };

__device__ __forceinline__ PrimF psub(const PrimF& a, const PrimF& b) {
  return PrimF{sub(a.r, b.r), sub(a.vx, b.vx), sub(a.vy, b.vy), sub(a.vz, b.vz), sub(a.p, b.p)};
}
__device__ __forceinline__ PrimF padd(const PrimF& a, const PrimF& b) {
  return PrimF{add(a.r, b.r), add(a.vx, b.vx), add(a.vy, b.vy), add(a.vz, b.vz), add(a.p, b.p)};
}

__device__ __forceinline__ bool same_bits(const PrimF& a, const PrimF& b) {
  auto eq = [](ff x, ff y) {
    return __float_as_uint(x.hi) == __float_as_uint(y.hi) &&
           __float_as_uint(x.lo) == __float_as_uint(y.lo);
  };
  return eq(a.r, b.r) && eq(a.vx, b.vx) && eq(a.vy, b.vy) && eq(a.vz, b.vz) && eq(a.p, b.p);
}

// FP64 primitives as float-float
__device__ __forceinline__ PrimF to_ff(const fvd::Prim& w) {
  return PrimF{from_double(w.r), from_double(w.vx), from_double(w.vy), from_double(w.vz),
               from_double(w.p)};
}

// Half of the limited slope from the two one-sided differences:
// 0.5 minmod(theta dm, (dm + dp) / 2, theta dp) (theta as float-float)
template <bool MC>
__device__ __forceinline__ ff half_slope(ff theta, ff dm, ff dp) {
  const ff mid = half(add(dm, dp));
  if (MC) return half(minmod3(twice(dm), mid, twice(dp)));
  return half(minmod3(mul(theta, dm), mid, mul(theta, dp)));
}

template <bool MC>
__device__ __forceinline__ PrimF half_slopes(ff theta, const PrimF& dm, const PrimF& dp) {
  return PrimF{half_slope<MC>(theta, dm.r, dp.r), half_slope<MC>(theta, dm.vx, dp.vx),
               half_slope<MC>(theta, dm.vy, dp.vy), half_slope<MC>(theta, dm.vz, dp.vz),
               half_slope<MC>(theta, dm.p, dp.p)};
}

// The constants of the step as float-float.
struct ParamsF {
  ff gamma, igm1, theta;
};

// HLL flux normal to AXIS (the FP64 method's formulas in float-float):
// per side U = (rho, rho v, p / (gamma - 1) + ke), F = (rho vn, rho vn v +
// p e_n, (E + p) vn), c = t rsqrt(t rho) with t = gamma p; a+ = max(0,
// vL + cL, vR + cR), a- = max(0, cL - vL, cR - vR);
// F = ((a+ FL + a- FR) - a+ a- (UR - UL)) (1 / (a+ + a-)).
// Evaluated component by component (each side's U and F of a component
// formed where it is used), so few values are live at once.
template <int AXIS>
__device__ __forceinline__ void hll_flux(const PrimF& wl, const PrimF& wr, const ParamsF& Q,
                                         ff F[NF]) {
  ff vn[2], c[2], E[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const PrimF& w = s == 0 ? wl : wr;
    const ff ke = half(add(add(mul(mul(w.r, w.vx), w.vx), mul(mul(w.r, w.vy), w.vy)),
                           mul(mul(w.r, w.vz), w.vz)));
    E[s] = add(mul(w.p, Q.igm1), ke);
    vn[s] = AXIS == 0 ? w.vx : AXIS == 1 ? w.vy : w.vz;
    const ff t = mul(Q.gamma, w.p);
    c[s] = mul(t, rsqrt(mul(t, w.r)));
  }
  const ff ap = max0(add(vn[0], c[0]), add(vn[1], c[1]));
  const ff am = max0(sub(c[0], vn[0]), sub(c[1], vn[1]));
  const ff r = recip(add(ap, am));
  const ff apm = mul(ap, am);
  const ff mnl = mul(wl.r, vn[0]), mnr = mul(wr.r, vn[1]);
  auto combine = [&](ff ul, ff ur, ff fl, ff fr) {
    return mul(sub(add(mul(ap, fl), mul(am, fr)), mul(apm, sub(ur, ul))), r);
  };
  F[0] = combine(wl.r, wr.r, mnl, mnr);
#pragma unroll
  for (int q = 1; q <= 3; ++q) {
    const ff vl = q == 1 ? wl.vx : q == 2 ? wl.vy : wl.vz;
    const ff vr = q == 1 ? wr.vx : q == 2 ? wr.vy : wr.vz;
    ff fl = mul(mnl, vl), fr = mul(mnr, vr);
    if (q == 1 + AXIS) {
      fl = add(fl, wl.p);
      fr = add(fr, wr.p);
    }
    F[q] = combine(mul(wl.r, vl), mul(wr.r, vr), fl, fr);
  }
  F[4] = combine(E[0], E[1], mul(add(E[0], wl.p), vn[0]), mul(add(E[1], wr.p), vn[1]));
}

}  // namespace fvff
