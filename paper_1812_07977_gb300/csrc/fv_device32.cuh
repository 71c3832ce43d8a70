// fv_device32.cuh -- FP32 building blocks of the FP32-bulk step.
//
// The FP32 code is built without implicit contraction (--fmad=false) and
// writes its fused multiply-adds out (fmaf), so every kernel that inlines
// these helpers computes the same bits.
//
// The FP32-bulk arithmetic keeps the state in FP64 (the RK combine adds the
// FP32 update to the FP64 state; the pressure of near-vacuum cells is
// recovered in FP64) and does reconstruction and fluxes in FP32.  On sm_103a
// the double<->float conversions issue on the FP64 pipe, at the FP64 rate
// (2 per SM per clock), so they are done here on the integer pipe instead:
// d2f / f2d return exactly what the IEEE conversions return (round to
// nearest even), taking the hardware conversion only outside the float
// normal range.
#pragma once

#include <cstdint>

#include "fv_device.cuh"

namespace fvd32 {

using fvd::NF;

// Hardware conversions for the rare operands, as calls: inlined, the
// conversion would be predicated into the common path, where every
// predicated-off copy still takes an FP64 issue slot.
static __device__ __noinline__ float d2f_rare(double x) {
  float r;
  asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(r) : "d"(x));
  return r;
}
static __device__ __noinline__ double f2d_rare(float x) {
  double r;
  asm volatile("cvt.f64.f32 %0, %1;" : "=d"(r) : "f"(x));
  return r;
}

static __device__ __noinline__ double dhalf_rare(double x) {
  double r;
  asm volatile("mul.rn.f64 %0, %1, 0d3FE0000000000000;" : "=d"(r) : "d"(x));
  return r;
}

// x * 0.5 in FP64, bit-identical to the IEEE product, rare operands by call
__device__ __forceinline__ double dhalf(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e - 2u < 0x7FDu) return __hiloint2double((int)(hi - 0x00100000u), (int)lo);
  if (((hi << 1) | lo) == 0u) return x;  // +-0 (tested on the halves: as a 64-bit
                                         // test it becomes an FP64 compare)
  return dhalf_rare(x);
}

// double -> float, round to nearest even
__device__ __forceinline__ float d2f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e - 897u < 254u) {  // result exponent 1..254 (a carry may round to inf)
    unsigned field = ((e - 896u) << 23) | ((hi & 0x000FFFFFu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1FFFFFFFu;
    field += (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & (field & 1u));
    return __uint_as_float(field | (hi & 0x80000000u));
  }
  // zeros and FP64 subnormals (below half the least FP32 subnormal) -> +-0
  if (e == 0u) return __uint_as_float(hi & 0x80000000u);
  return d2f_rare(x);  // FP32 subnormal range, huge, inf or NaN
}

// float -> double (exact)
__device__ __forceinline__ double f2d(float f) {
  const unsigned x = __float_as_uint(f);
  const unsigned ex = (x >> 23) & 0xFFu;
  if (ex - 1u < 254u) {  // normal
    const unsigned hi = (((x & 0x7FFFFFFFu) >> 3) + (896u << 20)) | (x & 0x80000000u);
    return __hiloint2double((int)hi, (int)(x << 29));
  }
  if ((x << 1) == 0u) return __hiloint2double((int)(x & 0x80000000u), 0);  // +-0
  return f2d_rare(f);  // subnormal, inf or NaN
}

// Approximate reciprocal (one MUFU.RCP, within 2 ulp): the FP32-bulk
// arithmetic is held to an error bound against FP64, not bit for bit.
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }

struct Prim32 { float r, vx, vy, vz, p; };

struct Params32 {
  float gamma, gm1, igm1, theta;
  float inv_d[3];
  double gm1_d;             // gamma - 1 in FP64 (near-vacuum pressure recovery)
  float vacuum_ratio;       // recover p in FP64 when kinetic / total energy > this
  // FP32 upper bounds of the FP64 constants of the CFL speed
  float gm1_hi, gamma_hi, inv_hi[3];
};

// p = (gamma-1)(E - |m|^2 / (2 rho)) in FP64, rounded to float.
__device__ __forceinline__ float pressure_fp64(const double u[NF], double gm1) {
  const double ked = 0.5 * ((u[1] * u[1] + u[2] * u[2]) + u[3] * u[3]) / u[0];
  return d2f(gm1 * (u[4] - ked));
}

// Primitive state of one cell from its FP64 conserved state.  The pressure
// p = (gamma-1)(E - ke) cancels when the kinetic energy is nearly all of E;
// there it is recomputed in FP64 from the FP64 state.
__device__ __forceinline__ Prim32 prim_from_state(const double u[NF], const Params32& Q) {
  Prim32 w;
  const float r = d2f(u[0]), mx = d2f(u[1]), my = d2f(u[2]), mz = d2f(u[3]), E = d2f(u[4]);
  const float ir = rcp(r);
  w.r = r;
  w.vx = mx * ir;
  w.vy = my * ir;
  w.vz = mz * ir;
  const float ke = 0.5f * fmaf(mz, w.vz, fmaf(my, w.vy, mx * w.vx));
  w.p = Q.gm1 * (E - ke);
  if (ke > Q.vacuum_ratio * E) w.p = pressure_fp64(u, Q.gm1_d);
  return w;
}

// minmod(a, b, c): the argument of least magnitude when all three share a
// strict sign, else 0:  s * max(0, min(s*a, s*b, s*c)) with s = sign(a).
__device__ __forceinline__ float minmod3(float a, float b, float c) {
  const float s = copysignf(1.0f, a);
  return s * fmaxf(0.0f, fminf(fminf(s * a, s * b), s * c));
}

__device__ __forceinline__ float half_slope(float theta, float dm, float dp) {
  return 0.5f * minmod3(theta * dm, 0.5f * (dm + dp), theta * dp);
}

// The same for theta = 2 (monotonised central limiter), where
// 0.5 minmod(2 dm, (dm + dp)/2, 2 dp) = minmod(dm, (dm + dp)/4, dp) (exactly:
// the factors are powers of two).  The middle argument shares the sign of dm
// and dp whenever they agree, so the result is the least magnitude with
// dm's sign if dm and dp have one sign, else 0 (a zero operand gives 0).
__device__ __forceinline__ float half_slope_mc(float dm, float dp) {
  const float m = fminf(fminf(fabsf(dm), fabsf(dp)), fabsf(0.25f * (dm + dp)));
  const unsigned r = __float_as_uint(m) | (__float_as_uint(dm) & 0x80000000u);
  return ((__float_as_uint(dm) ^ __float_as_uint(dp)) & 0x80000000u) ? 0.0f : __uint_as_float(r);
}

__device__ __forceinline__ bool physical(const Prim32& w) { return w.r > 0.0f && w.p > 0.0f; }

__device__ __forceinline__ Prim32 operator+(const Prim32& a, const Prim32& b) {
  return Prim32{a.r + b.r, a.vx + b.vx, a.vy + b.vy, a.vz + b.vz, a.p + b.p};
}
__device__ __forceinline__ Prim32 operator-(const Prim32& a, const Prim32& b) {
  return Prim32{a.r - b.r, a.vx - b.vx, a.vy - b.vy, a.vz - b.vz, a.p - b.p};
}

// Half slopes of the five primitives; MC: theta is 2.
template <bool MC>
__device__ __forceinline__ Prim32 half_slopes(float theta, const Prim32& dm, const Prim32& dp) {
  if (MC)
    return Prim32{half_slope_mc(dm.r, dp.r), half_slope_mc(dm.vx, dp.vx),
                  half_slope_mc(dm.vy, dp.vy), half_slope_mc(dm.vz, dp.vz),
                  half_slope_mc(dm.p, dp.p)};
  return Prim32{half_slope(theta, dm.r, dp.r), half_slope(theta, dm.vx, dp.vx),
                half_slope(theta, dm.vy, dp.vy), half_slope(theta, dm.vz, dp.vz),
                half_slope(theta, dm.p, dp.p)};
}

// HLL flux normal to AXIS from face states wl, wr (the FP64 method's
// formulas in FP32, with approximate reciprocal and square root):
// F = wL FL + wR FR - wD (UR - UL), wL = a+ r, wR = a- r, wD = a+ a- r,
// r = 1 / (a+ + a-).
template <int AXIS>
__device__ __forceinline__ void hll_flux(const Prim32& wl, const Prim32& wr, const Params32& Q,
                                         float F[NF]) {
  float UL[NF], UR[NF], FL[NF], FR[NF], c[2], vn[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const Prim32& w = s == 0 ? wl : wr;
    float* U = s == 0 ? UL : UR;
    float* Fs = s == 0 ? FL : FR;
    const float mx = w.r * w.vx, my = w.r * w.vy, mz = w.r * w.vz;
    const float ke = 0.5f * fmaf(mz, w.vz, fmaf(my, w.vy, mx * w.vx));
    U[0] = w.r;
    U[1] = mx;
    U[2] = my;
    U[3] = mz;
    U[4] = fmaf(w.p, Q.igm1, ke);
    const float v = AXIS == 0 ? w.vx : AXIS == 1 ? w.vy : w.vz;
    const float mn = AXIS == 0 ? mx : AXIS == 1 ? my : mz;
    vn[s] = v;
    const float c2 = Q.gamma * w.p * rcp(w.r);
    c[s] = c2 * rsqrtf(c2);
    Fs[0] = mn;
    Fs[1] = mn * w.vx;
    Fs[2] = mn * w.vy;
    Fs[3] = mn * w.vz;
    Fs[1 + AXIS] += w.p;
    Fs[4] = (U[4] + w.p) * v;
  }
  const float ap = fmaxf(0.0f, fmaxf(vn[0] + c[0], vn[1] + c[1]));
  const float am = fmaxf(0.0f, fmaxf(c[0] - vn[0], c[1] - vn[1]));
  const float r = rcp(ap + am);
  const float wL = ap * r, wR = am * r, wD = ap * am * r;
#pragma unroll
  for (int q = 0; q < NF; ++q) F[q] = fmaf(wL, FL[q], fmaf(wR, FR[q], -(wD * (UR[q] - UL[q]))));
}

// ---------------------------------------------------------------- CFL bound
// An upper bound, in FP32, of the FP64 CFL signal speed that fvd::cell_speed
// computes (IEEE operations) for a cell of conserved state u, and whether
// the cell is certainly physical (rho > 0 and p > 0 in FP64).  The inputs
// are truncated to FP32 (relative error below 2^-23), the reciprocal and
// inverse square root are the SFU approximations (relative error below
// 2^-22, the PTX ISA's bounds for rcp.approx and rsqrt.approx), and each
// other FP32 operation rounds to nearest (2^-24): the FP32 velocity, kinetic
// energy and sound speed are within 2^-19 of the exact values of the FP64
// state, and E - ke within 2^-19 (E + ke), which an explicit margin of
// 2^-18 (E + ke) on the pressure covers (with the FP64 evaluation's own
// errors, a few 2^-53).  The final factor 1 + 2^-16 covers the relative
// errors, so the bound holds for any state inside the operand range.
// Returns +inf (sure = false) when an input is outside [2^-100, 2^101), rho
// or E is not positive, or p could be <= 0.
__device__ __forceinline__ float speed_upper(const double u[NF], const Params32& Q, bool& sure) {
  const float kInf = __int_as_float(0x7F800000);
  sure = false;
  bool ok = true;
  const float r = fvd::trunc_f32(u[0], ok), E = fvd::trunc_f32(u[4], ok);
  const float mx = fabsf(fvd::trunc_f32(u[1], ok)), my = fabsf(fvd::trunc_f32(u[2], ok)),
              mz = fabsf(fvd::trunc_f32(u[3], ok));
  if (!ok || !(r > 0.0f) || !(E > 0.0f)) return kInf;
  const float ir = rcp(r);
  const float vx = __fmul_rn(mx, ir), vy = __fmul_rn(my, ir), vz = __fmul_rn(mz, ir);
  const float ke = __fmul_rn(0.5f, __fadd_rn(__fadd_rn(__fmul_rn(mx, vx), __fmul_rn(my, vy)),
                                              __fmul_rn(mz, vz)));
  const float margin = __fmul_rn(0x1p-18f, __fadd_rn(E, ke));
  const float pm = __fsub_rn(E, ke);
  if (!(__fsub_rn(pm, margin) > 0.0f)) return kInf;
  sure = true;
  const float c2 = __fmul_rn(__fmul_rn(Q.gamma_hi, __fadd_rn(pm, margin)), __fmul_rn(Q.gm1_hi, ir));
  const float c = __fmul_rn(c2, rsqrtf(c2));
  const float sp = __fadd_rn(__fadd_rn(__fmul_rn(__fadd_rn(vx, c), Q.inv_hi[0]),
                                       __fmul_rn(__fadd_rn(vy, c), Q.inv_hi[1])),
                             __fmul_rn(__fadd_rn(vz, c), Q.inv_hi[2]));
  return __fmul_rn(sp, 1.0f + 0x1p-16f);
}

// The last cell a thread folded (fold_speed): its state and whether it was
// non-physical.  A cell equal to it bit for bit changes neither the maximum
// nor anything but the count -- the usual case in uniform regions, where
// the FP32 bound of an equal speed would not exclude it.
struct SpeedCache {
  double u[NF];
  unsigned bad;
  bool valid;
};

// Running maximum of FP64 CFL speeds shared by a whole launch: *gmax holds the
// bits of the largest speed any thread has computed so far (non-negative
// doubles order like their bits), so it is a lower bound of the final
// maximum at every moment, and any cell whose FP32 bound is below it cannot
// change the result.  refresh_max raises a thread's threshold (smax, and
// smax_f <= smax as a float) to the shared value.
__device__ __forceinline__ void set_threshold(double s, double& smax, float& smax_f) {
  smax = s;
  bool in = true;
  const float t = fvd::trunc_f32(s, in);
  smax_f = in ? t : (s > 1.0 ? 0x1p100f : 0.0f);
}

// The shared maximum's bits, read past the caches: whenever it is read, a
// lower bound of the final maximum, so a value read early stays usable.
__device__ __forceinline__ unsigned long long peek_max(const unsigned long long* gmax) {
  return *(const volatile unsigned long long*)gmax;
}

__device__ __forceinline__ void raise_max(unsigned long long g, double& smax, float& smax_f) {
  if (g > (unsigned long long)__double_as_longlong(smax))
    set_threshold(__longlong_as_double((long long)g), smax, smax_f);
}

__device__ __forceinline__ void refresh_max(const unsigned long long* gmax, double& smax,
                                            float& smax_f) {
  raise_max(peek_max(gmax), smax, smax_f);
}


// Folds one cell's FP64 CFL speed (fvd::cell_speed, IEEE operations) into the
// shared maximum *gmax, and counts the cell in `bad` if its FP64 primitives
// are non-physical.  The FP64 speed is computed only when the cell differs
// from the thread's last one and its FP32 bound could reach the threshold
// smax (a speed already computed) or it is not certainly physical: the
// maximum and the count are the bits and the number that evaluating every
// cell gives.
__device__ __forceinline__ void fold_speed(const double u[NF], const fvd::Params& P,
                                           const Params32& Q, double& smax, float& smax_f,
                                           unsigned long long& bad, SpeedCache& cache,
                                           unsigned long long* gmax) {
  bool eq = cache.valid;
#pragma unroll
  for (int q = 0; q < NF; ++q) {
    eq = eq && __double_as_longlong(u[q]) == __double_as_longlong(cache.u[q]);
    cache.u[q] = u[q];
  }
  if (eq) {
    bad += cache.bad;
    return;
  }
  cache.valid = true;
  cache.bad = 0;
  bool sure;
  const float ub = speed_upper(u, Q, sure);
  if (sure && ub < smax_f) return;
  const fvd::Prim w = fvd::cons_to_prim(u, P);
  cache.bad = !(fvd::is_pos(w.r) && fvd::is_pos(w.p));
  bad += cache.bad;
  const double s = fvd::cell_speed(w, P);
  if (s > smax) {
    set_threshold(s, smax, smax_f);
    atomicMax(gmax, (unsigned long long)__double_as_longlong(s));
  }
}

}  // namespace fvd32
