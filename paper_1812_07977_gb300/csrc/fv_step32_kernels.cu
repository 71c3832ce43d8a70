// fv_step32_kernels.cu -- one RK2 substep of the FP32-bulk method, fused.
//
// One kernel per substep does all of Algorithm 1's substep kernels
// (ComputeDifferences, ComputeReconstruction, RiemannSolverInput,
// ComputeFluxes, ComputeUpdate and the RK combine) for a tile of 32 x TY
// columns (TY = 4, 8 or 16) marching along z over a chunk of planes, so each
// substep reads its input state once (plus the tile's two-cell halo) and
// writes its output once: 120-200 B of FP64 state traffic per zone-update
// instead of the ~1 KB of the FP64 path's separate sweeps.
//
// Per plane k, each thread owns one column (i, j) of the tile; the FP64
// input of the next plane is staged into shared memory by cp.async while
// the current one is computed:
//   z  : a register window along its column (primitives of planes k..k+2,
//        the z differences and half slopes of planes k, k+1, and the z
//        flux of face k-1/2 carried from the previous plane) gives the z
//        flux of face k+1/2 -- every z flux computed once;
//   x,y: the plane's primitives (tile plus two-cell halo) go to shared
//        memory; the 33 x TY x-faces and 32 x (TY+1) y-faces are computed
//        once each (slopes of both neighbours recomputed per face) into
//        shared memory;
//   update: dU = dt * (-(Fx(i+1/2)-Fx(i-1/2))/dx - (..)/dy - (..)/dz) in FP32,
//        then the RK combine in FP64 on the FP64 state; stage 2 also takes
//        the CFL speed of the cell it writes (the next step's time step).
// Flux reuse (bit for bit what evaluating gives): a z face whose column has
// five equal cells around it takes the previous z flux; an x or y face whose
// four cells all equal those one plane below keeps that plane's flux (each
// plane's primitives are stored with a per-cell "equal to the plane below"
// flag).  Both are decided per warp.
#include <cmath>
#include <limits>

#include "fv_device32.cuh"
#include "fv_internal.h"

using namespace fvd32;

namespace fv_fp32 {
namespace {

// A tile of TX x TY columns (one thread per column: TX = 32 is one warp per
// tile row; the single-mesh kernel uses 32 x 4, 8 or 16, batches also 16 x 8,
// 64 x 4, 64 x 8 and 128 x 4) with its plane buffer (two-cell halo), halo
// cells and faces.
template <int TX_, int TY_>
struct Shape {
  static constexpr int TX = TX_;
  static constexpr int TY = TY_;
  static constexpr int kThreads = TX * TY;
  static constexpr int PX = TX + 4;
  static constexpr int PY = TY + 4;
  static constexpr int kHalo = PX * PY - TX * TY;
  static constexpr int kHaloPer = (kHalo + kThreads - 1) / kThreads;
  static constexpr int kXFaces = (TX + 1) * TY;
  static constexpr int kYFaces = TX * (TY + 1);
  static_assert(kXFaces <= 2 * kThreads && kYFaces <= 2 * kThreads, "two face passes");
};

// First y face of thread tid.  The x faces beyond the first kThreads go to
// warp 0; the y faces are assigned one warp later, so that their leftover
// row goes to warp 1 and no warp evaluates more than two x / y faces plus
// the z face per plane (the others wait for it at the plane's barrier).
template <class S>
__device__ __forceinline__ int yface0(int tid) {
  return (tid + S::kThreads - 32) % S::kThreads;
}

// Halo cell h of a tile (0 <= h < kHalo): the two rows below the tile, the
// two above, then two columns on each side of every tile row; (row, col)
// relative to the tile's first cell.
template <class S>
__device__ __forceinline__ void halo_cell(int h, int& row, int& col) {
  constexpr int PX = S::PX;
  if (h < 2 * PX) {
    row = h / PX - 2;
    col = h % PX - 2;
  } else if (h < 4 * PX) {
    row = S::TY + (h - 2 * PX) / PX;
    col = (h - 2 * PX) % PX - 2;
  } else {
    const int u = h - 4 * PX;
    row = u / 4;
    const int c = u % 4;
    col = c < 2 ? c - 2 : S::TX + c - 2;
  }
}

#ifndef FV32_STAGE_DEPTH
#define FV32_STAGE_DEPTH 1
#endif
// Iterations whose FP64 input is in flight ahead of the one being computed,
// and the ring of staging slots (one per iteration in flight plus the one in
// use).  Iteration k's slot holds the column cells of plane k+2 (the z
// window) and the halo cells of plane k, each copied by the thread that uses
// it, so a slot is reused without a barrier.
constexpr int kStageDepth = FV32_STAGE_DEPTH;
// FV32_EQ_SKIP (default 1): a cell whose FP64 input equals the previous
// plane's keeps its primitives, decided per warp; the next plane is then
// staged after this plane's input has been compared with the previous one
// (two slots).  On the 256^3 oblique problem 8% faster, on a state with no
// equal neighbours 3% slower (the compares, and the later staging).
#ifndef FV32_EQ_SKIP
#define FV32_EQ_SKIP 1
#endif
static_assert(!FV32_EQ_SKIP || FV32_STAGE_DEPTH == 1, "the equal-state skip stages one plane ahead");
constexpr int kRing = kStageDepth + 1;
constexpr bool kLateStage = FV32_EQ_SKIP != 0;

template <class S>
struct Smem {
  double col[kRing][NF][S::kThreads];
  double halo[kRing][NF][S::kHalo];
  float w[NF][S::PY][S::PX];
  float fx[NF][S::TY][S::TX + 1];
  float fy[NF][S::TY + 1][S::TX];
  unsigned char same[S::PY][S::PX];   // cell equals (bit for bit) the cell one plane below
};

// Asynchronous 8-byte copy global -> shared (completes at cp_async_wait).
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// Waits until at most N of this thread's committed copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void load_state(const double* __restrict__ U, long long nf,
                                           long long off, double u[NF]) {
#pragma unroll
  for (int q = 0; q < NF; ++q) u[q] = U[q * nf + off];
}

__device__ __forceinline__ Prim32 load_prim(const double* __restrict__ U, long long nf,
                                            long long off, const Params32& Q) {
  double u[NF];
  load_state(U, nf, off, u);
  return prim_from_state(u, Q);
}

template <class SM>
__device__ __forceinline__ Prim32 smem_prim(const SM& s, int row, int col) {
  return Prim32{s.w[0][row][col], s.w[1][row][col], s.w[2][row][col], s.w[3][row][col],
                s.w[4][row][col]};
}

__device__ __forceinline__ bool same32(const Prim32& a, const Prim32& b) {
  return __float_as_uint(a.r) == __float_as_uint(b.r) &&
         __float_as_uint(a.vx) == __float_as_uint(b.vx) &&
         __float_as_uint(a.vy) == __float_as_uint(b.vy) &&
         __float_as_uint(a.vz) == __float_as_uint(b.vz) && __float_as_uint(a.p) == __float_as_uint(b.p);
}

// Stores the plane's primitives of one cell and whether they equal the
// previous plane's in that slot (`valid`: the slot holds the previous plane).
template <class SM>
__device__ __forceinline__ void smem_store_flag(SM& s, int row, int col, const Prim32& w,
                                                bool valid) {
  s.same[row][col] = valid && same32(smem_prim(s, row, col), w);
  s.w[0][row][col] = w.r;
  s.w[1][row][col] = w.vx;
  s.w[2][row][col] = w.vy;
  s.w[3][row][col] = w.vz;
  s.w[4][row][col] = w.p;
}

// Folds a thread's CFL speed maximum (a double >= 0, ordered like its bits)
// into a grid-wide maximum held as the bits of a double.  All 32 lanes call.
__device__ __forceinline__ void max_speed_to(unsigned long long* dst, double smax) {
  unsigned long long b = (unsigned long long)__double_as_longlong(smax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
    b = v > b ? v : b;
  }
  if ((threadIdx.x & 31u) == 0u && b) atomicMax(dst, b);
}

// Face flux between cells a1 and a2 given the four cells a0..a3 along the
// face normal; falls back to first order if a face state is non-physical.
template <int AXIS, bool MC>
__device__ __forceinline__ void face_flux(const Prim32& a0, const Prim32& a1, const Prim32& a2,
                                          const Prim32& a3, const Params32& Q, float F[NF],
                                          unsigned& fallbacks) {
  const Prim32 d0 = a1 - a0, d1 = a2 - a1, d2 = a3 - a2;
  Prim32 wl = a1 + half_slopes<MC>(Q.theta, d0, d1);
  Prim32 wr = a2 - half_slopes<MC>(Q.theta, d1, d2);
  if (!(physical(wl) && physical(wr))) {
    wl = a1;
    wr = a2;
    ++fallbacks;
  }
  hll_flux<AXIS>(wl, wr, Q, F);
}

// One tile (32 x 8 columns, planes k0 .. k1-1) of a substep.
// STAGE 1: U1 = U + dU.  STAGE 2: U = ((U + U1) + dU) / 2.  The input of the
// substep (U for stage 1, U1 for stage 2) has its ghosts filled.  Counts of
// face fallbacks and non-physical cells accumulate in the caller's counters.
// MC: the limiter parameter is 2.  NEXT (stage 2): also the FP64 CFL speed
// of each output cell (the next time step's), its maximum into *gmax (a
// maximum shared by the launch, see fvd32::fold_speed; smax_next, smax_next_f
// the thread's threshold) and its non-physical cells into bad_next.
template <class S, int STAGE, bool MC, bool NEXT>
__device__ __forceinline__ void stage32_tile(Smem<S>& s, double* __restrict__ U,
                                             double* __restrict__ U1, const fvd::Params& P,
                                             const Params32& Q, float dt, int i0, int j0,
                                             int k0, int k1, unsigned& fallbacks_out,
                                             unsigned long long& bad_out, unsigned& evaluated,
                                             double& smax_next, float& smax_next_f,
                                             unsigned long long& bad_next,
                                             unsigned long long* gmax) {
  SpeedCache speed_cache;
  speed_cache.valid = false;
  const double* __restrict__ src = STAGE == 1 ? U : U1;
  constexpr int TX = S::TX;
  const int tid = threadIdx.x;
  const int ti = tid % TX, tj = tid / TX;
  const long long nf = P.nfield;
  // this thread's column, clamped into the ghosted array (columns past a
  // ragged edge compute unused values and store nothing)
  const int gi = min(i0 + ti, P.nx + 1), gj = min(j0 + tj, P.ny + 1);
  const bool owner = (i0 + ti < P.nx) && (j0 + tj < P.ny);
  const long long col = (long long)(gj + 2) * P.sy + (gi + 2);
  constexpr int kThreads = S::kThreads, kHalo = S::kHalo, kHaloPer = S::kHaloPer;
  constexpr int TY = S::TY;
  // the halo cells this thread loads each plane (h = tid + e * kThreads)
  int hrow[kHaloPer], hcol[kHaloPer];
  long long hcolo[kHaloPer];
#pragma unroll
  for (int e = 0; e < kHaloPer; ++e) {
    hrow[e] = hcol[e] = 0;
    if (tid + e * kThreads < kHalo) halo_cell<S>(tid + e * kThreads, hrow[e], hcol[e]);
    const int hgi = min(i0 + hcol[e], P.nx + 1), hgj = min(j0 + hrow[e], P.ny + 1);
    hcolo[e] = (long long)(hgj + 2) * P.sy + (hgi + 2);
  }

  unsigned fallbacks = 0;
  const float idx = Q.inv_d[0], idy = Q.inv_d[1], idz = Q.inv_d[2];

  // z window prologue: planes k0-2 .. k0+1
  Prim32 wm2 = load_prim(src, nf, col + (long long)(k0 + 0) * P.sz, Q);   // plane k0-2
  Prim32 wm1 = load_prim(src, nf, col + (long long)(k0 + 1) * P.sz, Q);   // plane k0-1
  Prim32 w0 = load_prim(src, nf, col + (long long)(k0 + 2) * P.sz, Q);    // plane k0
  Prim32 w1 = load_prim(src, nf, col + (long long)(k0 + 3) * P.sz, Q);    // plane k0+1
  Prim32 d1 = w1 - w0;                                                    // D(k0+1)
  Prim32 h0 = half_slopes<MC>(Q.theta, w0 - wm1, d1);                         // cell k0
  float fz_lo[NF];
  bool zfb;   // the last z face fell back to first order
  {
    Prim32 hm1 = half_slopes<MC>(Q.theta, wm1 - wm2, w0 - wm1);               // cell k0-1
    Prim32 wl = wm1 + hm1, wr = w0 - h0;
    zfb = !(physical(wl) && physical(wr));
    if (zfb) {
      wl = wm1;
      wr = w0;
      ++fallbacks;
    }
    hll_flux<2>(wl, wr, Q, fz_lo);
    ++evaluated;
  }
  // cells of the column equal bit for bit to the newest cell of the window,
  // counted from plane k0-2
  int run = same32(wm1, wm2) ? 2 : 1;
  run = same32(w0, wm1) ? run + 1 : 1;
  run = same32(w1, w0) ? run + 1 : 1;
  unsigned xyfb = 0;   // fallbacks of this thread's x (bits 0, 1) and y (2, 3) faces
  // which of those faces this tile counts: each face of the mesh is counted
  // by one tile (face TX of a tile is face 0 of the next)
  unsigned counted = 0;
  for (int f = tid, pass = 0; f < S::kXFaces; f += kThreads, ++pass) {
    const int r = f / (TX + 1), fi = f % (TX + 1);
    if (i0 + fi <= P.nx && (fi < TX || i0 + fi == P.nx) && j0 + r < P.ny) counted |= 1u << pass;
  }
  for (int f = yface0<S>(tid), pass = 2; f < S::kYFaces; f += kThreads, ++pass) {
    const int fj = f / TX, c = f % TX;
    if (i0 + c < P.nx && j0 + fj <= P.ny && (fj < TY || j0 + fj == P.ny)) counted |= 1u << pass;
  }
  // the first chunk's lower face is the domain boundary face; later chunks
  // recompute a face the previous chunk counted
  if (k0 != 0 || !owner) fallbacks = 0;
  unsigned long long bad = 0;

  // raw FP64 state of iteration t (column plane t+2, halo cell of plane t),
  // copied kStageDepth iterations ahead into the staging ring so that its
  // latency overlaps the face work; every iteration commits one group
  auto stage_in = [&](int t) {
    if (t < k1) {
      const int slot = t % kRing;
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
#pragma unroll
  for (int t = 0; t < kStageDepth; ++t) stage_in(k0 + t);

  for (int k = k0; k < k1; ++k) {
    if (owner && !physical(w0)) ++bad;   // each interior cell once per substep
    if (NEXT && STAGE == 2) refresh_max(gmax, smax_next, smax_next_f);
    if (kLateStage) {
      // the next plane is staged after this plane's input has been compared
      // with the previous plane's (still in the other slot)
      cp_async_wait<0>();
    } else {
      stage_in(k + kStageDepth);
      cp_async_wait<kStageDepth>();      // this iteration's group has landed
    }
    const int slot = k % kRing;
    const int pslot = (k + kRing - 1) % kRing;   // the previous plane's input
    double cur_col[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) cur_col[q] = s.col[slot][q][tid];
    // operands of this plane's RK combine, loaded before the face work
    double rk0[NF], rk1[NF];
    const long long g = col + (long long)(k + 2) * P.sz;
    if (owner) {
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        rk0[q] = U[q * nf + g];
        rk1[q] = STAGE == 2 ? U1[q * nf + g] : 0.0;
      }
    }
    // (a) z: plane k+2 enters the window; flux of face k+1/2.  Face k+1/2
    // reads planes k-1 .. k+2; when planes k-2 .. k+2 of the column are
    // equal, its slopes are +0 and its face states are those of face k-1/2:
    // its flux and fallback are the previous face's, bit for bit (reused when
    // the whole warp can).
#if FV32_EQ_SKIP
    // a column cell whose FP64 state equals the previous plane's has its
    // primitives (the same bits): skipped when the whole warp can
    bool eqc = k > k0;
#pragma unroll
    for (int q = 0; q < NF; ++q)
      eqc = eqc && fvd::bits(cur_col[q]) == fvd::bits(s.col[pslot][q][tid]);
    const Prim32 w2 = __all_sync(0xffffffffu, eqc) ? w1 : prim_from_state(cur_col, Q);
#else
    const Prim32 w2 = prim_from_state(cur_col, Q);
#endif
    run = same32(w2, w1) ? run + 1 : 1;
    Prim32 d2, h1;
    float fz_hi[NF];
    if (__all_sync(__activemask(), run >= 5)) {
      d2 = Prim32{0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      h1 = d2;
#pragma unroll
      for (int q = 0; q < NF; ++q) fz_hi[q] = fz_lo[q];
      if (zfb && owner) ++fallbacks;
    } else {
      d2 = w2 - w1;
      h1 = half_slopes<MC>(Q.theta, d1, d2);
      Prim32 wl = w0 + h0, wr = w1 - h1;
      zfb = !(physical(wl) && physical(wr));
      if (zfb) {
        wl = w0;
        wr = w1;
        if (owner) ++fallbacks;
      }
      hll_flux<2>(wl, wr, Q, fz_hi);
      ++evaluated;
    }
    // (b) the plane's primitives into shared memory, each with a flag: equal
    // to the previous plane's in its slot (never on a chunk's first plane,
    // where the slot holds another tile's data)
    smem_store_flag(s, tj + 2, ti + 2, w0, k > k0);
#pragma unroll
    for (int e = 0; e < kHaloPer; ++e) {
      const int h = tid + e * kThreads;
#if FV32_EQ_SKIP
      // a halo cell whose FP64 state equals the previous plane's keeps its
      // primitives in shared memory (the same bits), decided per warp
      double uh[NF];
      bool eqh = k > k0;
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        uh[q] = h < kHalo ? s.halo[slot][q][h] : 0.0;
        eqh = eqh && (h >= kHalo || fvd::bits(uh[q]) == fvd::bits(s.halo[pslot][q][h]));
      }
      const bool all_eq = __all_sync(0xffffffffu, eqh);
      if (h < kHalo) {
        if (all_eq)
          s.same[hrow[e] + 2][hcol[e] + 2] = 1;
        else
          smem_store_flag(s, hrow[e] + 2, hcol[e] + 2, prim_from_state(uh, Q), k > k0);
      }
#else
      if (h < kHalo) {
        double uh[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) uh[q] = s.halo[slot][q][h];
        smem_store_flag(s, hrow[e] + 2, hcol[e] + 2, prim_from_state(uh, Q), k > k0);
      }
#endif
    }
    if (kLateStage) stage_in(k + 1);   // into the other slot, now compared
    __syncthreads();
    // (c) x faces: face fi (between columns fi-1 and fi) of row r.  A face
    // whose four cells all equal the previous plane's has that plane's
    // inputs, so its flux (still in s.fx) and fallback stand.
    for (int f = tid, pass = 0; f < S::kXFaces; f += kThreads, ++pass) {
      const int r = f / (TX + 1), fi = f % (TX + 1);
      const bool keep = s.same[r + 2][fi] & s.same[r + 2][fi + 1] & s.same[r + 2][fi + 2] &
                        s.same[r + 2][fi + 3];
      unsigned fb;
      if (__all_sync(__activemask(), keep)) {
        fb = (xyfb >> pass) & 1u;
      } else {
        float F[NF];
        fb = 0;
        face_flux<0, MC>(smem_prim(s, r + 2, fi), smem_prim(s, r + 2, fi + 1),
                         smem_prim(s, r + 2, fi + 2), smem_prim(s, r + 2, fi + 3), Q, F, fb);
        xyfb = (xyfb & ~(1u << pass)) | (fb << pass);
        ++evaluated;
#pragma unroll
        for (int q = 0; q < NF; ++q) s.fx[q][r][fi] = F[q];
      }
      fallbacks += fb & (counted >> pass);
    }
    // (d) y faces: face fj (between rows fj-1 and fj) of column c
    for (int f = yface0<S>(tid), pass = 2; f < S::kYFaces; f += kThreads, ++pass) {
      const int fj = f / TX, c = f % TX;
      const bool keep = s.same[fj][c + 2] & s.same[fj + 1][c + 2] & s.same[fj + 2][c + 2] &
                        s.same[fj + 3][c + 2];
      unsigned fb;
      if (__all_sync(__activemask(), keep)) {
        fb = (xyfb >> pass) & 1u;
      } else {
        float F[NF];
        fb = 0;
        face_flux<1, MC>(smem_prim(s, fj, c + 2), smem_prim(s, fj + 1, c + 2),
                         smem_prim(s, fj + 2, c + 2), smem_prim(s, fj + 3, c + 2), Q, F, fb);
        xyfb = (xyfb & ~(1u << pass)) | (fb << pass);
        ++evaluated;
#pragma unroll
        for (int q = 0; q < NF; ++q) s.fy[q][fj][c] = F[q];
      }
      fallbacks += fb & (counted >> pass);
    }
    __syncthreads();
    // (e) update of cell (i, j, k): FP32 divergence, FP64 RK combine
    if (owner) {
      double un[NF];
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        const float acc = fmaf(fz_lo[q] - fz_hi[q], idz,
                               fmaf(s.fy[q][tj][ti] - s.fy[q][tj + 1][ti], idy,
                                    (s.fx[q][tj][ti] - s.fx[q][tj][ti + 1]) * idx));
        const double du = f2d(dt * acc);
        if (STAGE == 1) {
          U1[q * nf + g] = rk0[q] + du;
        } else {
          un[q] = dhalf((rk0[q] + rk1[q]) + du);
          U[q * nf + g] = un[q];
        }
      }
      if (NEXT && STAGE == 2)
        fold_speed(un, P, Q, smax_next, smax_next_f, bad_next, speed_cache, gmax);
    }
#pragma unroll
    for (int q = 0; q < NF; ++q) fz_lo[q] = fz_hi[q];
    w0 = w1;
    w1 = w2;
    d1 = d2;
    h0 = h1;
  }
  fallbacks_out += fallbacks;
  bad_out += bad;
}

template <int STAGE, int TX, int TY, int MINB, bool MC>
__global__ void __launch_bounds__(TX * TY, MINB)
k_stage32(double* __restrict__ U, double* __restrict__ U1, fvd::Params P, Params32 Q, float dt,
          int kchunk, DevCounters* ctr) {
  using S = Shape<TX, TY>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<S>& s = *reinterpret_cast<Smem<S>*>(smem_raw);
  unsigned fallbacks = 0, evaluated = 0;
  unsigned long long bad = 0, bad_next = 0;
  double smax_next = 0.0;
  float smax_next_f = 0.0f;
  const int k0 = blockIdx.z * kchunk;
  stage32_tile<S, STAGE, MC, STAGE == 2>(s, U, U1, P, Q, dt, blockIdx.x * TX, blockIdx.y * TY,
                                         k0, min(k0 + kchunk, P.nz), fallbacks, bad, evaluated,
                                         smax_next, smax_next_f, bad_next, &ctr->smax_next);
  if (fallbacks) atomicAdd(&ctr->fallback, (unsigned long long)fallbacks);
  if (bad) atomicAdd(&ctr->np_step, bad);
  warp_count(&ctr->faces, evaluated);
  if (STAGE == 2) {
    max_speed_to(&ctr->smax_next, smax_next);
    if (bad_next) atomicAdd(&ctr->np_dt, bad_next);
  }
}

// ---------------------------------------------------------------- batches
// Persistent kernel over the tiles of many meshes: each CTA takes work items
// (mesh, tile x, tile y, z chunk) from an atomic counter until none is left.
// Stage 2 also folds the CFL maximum of each item's output cells into its
// mesh's smax_bits (the next step's dt).
template <int STAGE, int TX, int TY, int MINB, bool MC>
__global__ void __launch_bounds__(TX * TY, MINB)
k_stage32_batch(double* __restrict__ U, double* __restrict__ U1, BatchMesh* __restrict__ meshes,
                const int4* __restrict__ items, int nitems, int kchunk,
                unsigned* __restrict__ next_item, DevCounters* ctr) {
  using S = Shape<TX, TY>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<S>& s = *reinterpret_cast<Smem<S>*>(smem_raw);
  __shared__ int s_item;
  unsigned fallbacks = 0, evaluated = 0;
  unsigned long long bad = 0, bad_next = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(next_item, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int4 w = items[it];       // mesh, tile x, tile y, chunk
    BatchMesh& m = meshes[w.x];
    const int k0 = w.w * kchunk;
    double smax_next = 0.0;
    float smax_next_f = 0.0f;
    stage32_tile<S, STAGE, MC, STAGE == 2>(s, U + m.offset, U1 + m.offset, m.P, m.Q,
                                           (float)m.dt, w.y * TX, w.z * TY, k0,
                                           min(k0 + kchunk, m.P.nz), fallbacks, bad, evaluated,
                                           smax_next, smax_next_f, bad_next, &m.smax_bits);
    if (STAGE == 2) max_speed_to(&m.smax_bits, smax_next);
  }
  if (fallbacks) atomicAdd(&ctr->fallback, (unsigned long long)fallbacks);
  if (bad) atomicAdd(&ctr->np_step, bad);
  if (bad_next) atomicAdd(&ctr->np_dt, bad_next);
  warp_count(&ctr->faces, evaluated);
}

// Folds the FP64 CFL speed of interior cell m of a mesh into a running
// maximum (fold_speed).
__device__ __forceinline__ void fold_cell(const double* __restrict__ U, const fvd::Params& P,
                                          const Params32& Q, long long m, double& smax,
                                          float& smax_f, unsigned long long& bad,
                                          SpeedCache& cache, unsigned long long* gmax) {
  const long long k = m / ((long long)P.nx * P.ny);
  const long long r = m - k * ((long long)P.nx * P.ny);
  const long long j = r / P.nx, i = r - j * P.nx;
  double u[NF];
  load_state(U, P.nfield, (k + 2) * P.sz + (j + 2) * P.sy + (i + 2), u);
  refresh_max(gmax, smax, smax_f);
  fold_speed(u, P, Q, smax, smax_f, bad, cache, gmax);
}

// Block maximum of the threads' speeds (doubles >= 0), folded into *dst;
// blocks of 256 threads.
__device__ __forceinline__ void block_max_to(unsigned long long* dst, double smax) {
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
    if (lane == 0 && b) atomicMax(dst, b);
  }
}

// The CFL time step's maximum over the interior cells with FP64 speeds (the
// FP64 method's IEEE operations); FP32 bounds skip the cells that cannot
// raise a thread's running maximum.  Exact in any order (non-negative
// doubles order like their bits); dt = cfl / max is formed in FP64 on the
// host.
__global__ void __launch_bounds__(256)
k_reduce_dt32(const double* __restrict__ U, fvd::Params P, Params32 Q, DevCounters* ctr) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  double smax = 0.0;
  float smax_f = 0.0f;
  unsigned long long bad = 0;
  SpeedCache cache;
  cache.valid = false;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n;
       m += (long long)gridDim.x * blockDim.x)
    fold_cell(U, P, Q, m, smax, smax_f, bad, cache, &ctr->smax_bits);
  if (bad) atomicAdd(&ctr->np_dt, bad);
  block_max_to(&ctr->smax_bits, smax);
}

// Batched CFL maximum: block b reduces chunk c of mesh m (dt_blocks[b]) and
// folds it into that mesh's maximum.
__global__ void __launch_bounds__(256)
k_batch_dt(const double* __restrict__ U, BatchMesh* __restrict__ meshes,
           const int2* __restrict__ blocks, DevCounters* ctr) {
  const int2 bm = blocks[blockIdx.x];
  BatchMesh& mesh = meshes[bm.x];
  const long long n = (long long)mesh.P.nx * mesh.P.ny * mesh.P.nz;
  const long long lo = (long long)bm.y * kBatchDtChunk;
  const long long hi = min(n, lo + kBatchDtChunk);
  double smax = 0.0;
  float smax_f = 0.0f;
  unsigned long long bad = 0;
  SpeedCache cache;
  cache.valid = false;
  for (long long m = lo + threadIdx.x; m < hi; m += blockDim.x)
    fold_cell(U + mesh.offset, mesh.P, mesh.Q, m, smax, smax_f, bad, cache, &mesh.smax_bits);
  if (bad) atomicAdd(&ctr->np_dt, bad);
  block_max_to(&mesh.smax_bits, smax);
}

// Clears the per-mesh maxima and the work counters before a step.
__global__ void k_batch_reset(BatchMesh* __restrict__ meshes, int nmesh, unsigned* next_item) {
  for (int m = threadIdx.x; m < nmesh; m += blockDim.x) meshes[m].smax_bits = 0ULL;
  if (threadIdx.x < 2 * kBatchClasses) next_item[threadIdx.x] = 0u;
}

// dt = cfl / max, formed in FP64 per mesh (0 if the mesh had no physical cell).
__global__ void k_batch_dt_finalize(BatchMesh* __restrict__ meshes, int nmesh, double cfl) {
  for (int m = threadIdx.x; m < nmesh; m += blockDim.x) {
    const double smax = __longlong_as_double((long long)meshes[m].smax_bits);
    meshes[m].dt = smax > 0.0 ? cfl / smax : 0.0;
  }
}

// Batched ghost fill of the state of `stage` (U after stage 2, U1 after 1).
__global__ void __launch_bounds__(256)
k_batch_ghosts(double* __restrict__ base, const BatchMesh* __restrict__ meshes,
               const int2* __restrict__ blocks) {
  const int2 bm = blocks[blockIdx.x];
  const BatchMesh& mesh = meshes[bm.x];
  const long long t = (long long)bm.y * kBatchGhostChunk + threadIdx.x;
  if (threadIdx.x < kBatchGhostChunk && t < fvd::ring_cells(mesh.P))
    fvd::fill_ghost_cell(base + mesh.offset, mesh.P, t);
}

}  // namespace

// The nearest floats below and above x (equal when x is a float).
static void bracket_f32(double x, float& lo, float& hi) {
  const float f = (float)x;
  lo = hi = f;
  if ((double)f > x) lo = std::nextafter(f, -std::numeric_limits<float>::infinity());
  if ((double)f < x) hi = std::nextafter(f, std::numeric_limits<float>::infinity());
}

Params32 make_params32(const fvd::Params& P, double vacuum_ratio) {
  Params32 Q;
  Q.gamma = (float)P.gamma;
  Q.gm1 = (float)P.gm1;
  Q.igm1 = (float)P.igm1;
  Q.theta = (float)P.theta;
  for (int a = 0; a < 3; ++a) Q.inv_d[a] = (float)P.inv_d[a];
  Q.gm1_d = P.gm1;
  Q.vacuum_ratio = (float)vacuum_ratio;
  float lo;
  bracket_f32(P.gm1, lo, Q.gm1_hi);
  bracket_f32(P.gamma, lo, Q.gamma_hi);
  for (int a = 0; a < 3; ++a) bracket_f32(P.inv_d[a], lo, Q.inv_hi[a]);
  return Q;
}

// Kernel configurations: tile (TX x TY) and CTAs per SM (MINB).  Occupancy 2
// is 16 warps per SM at up to 128 registers for every tile; occupancy 3
// (24 warps, 80 registers) exists for the 32 x 8 tile.
__host__ __device__ constexpr int minb_of(int tile_x, int tile_y, int occupancy) {
  return occupancy == 2 ? 512 / (tile_x * tile_y)
         : occupancy == 3 && tile_x == 32 && tile_y == 8 ? 3 : 0;
}

// Calls fn.template run<STAGE, TX, TY, MINB, MC>() for a configuration, or
// returns cudaErrorInvalidValue for one that is not built.  The single-mesh
// and batched kernels are built for the same shapes.
#define FV32_CASE(TXV, TYV, MB)                                                              \
  if (tile_x == TXV && tile_y == TYV && minb_of(tile_x, tile_y, occupancy) == MB) {          \
    if (mc)                                                                                  \
      return stage == 1 ? fn.template run<1, TXV, TYV, MB, true>()                           \
                        : fn.template run<2, TXV, TYV, MB, true>();                          \
    return stage == 1 ? fn.template run<1, TXV, TYV, MB, false>()                            \
                      : fn.template run<2, TXV, TYV, MB, false>();                           \
  }
template <class Fn>
static cudaError_t dispatch(int stage, int tile_x, int tile_y, int occupancy, bool mc, Fn& fn) {
  FV32_CASE(32, 4, 4)
  FV32_CASE(32, 8, 2)
  FV32_CASE(32, 8, 3)
  FV32_CASE(32, 16, 1)
  FV32_CASE(16, 8, 4)
  FV32_CASE(64, 4, 2)
  FV32_CASE(64, 8, 1)
  FV32_CASE(128, 4, 1)
  return cudaErrorInvalidValue;
}
#undef FV32_CASE

struct LaunchMesh {
  const StepBuffers& b;
  const fvd::Params& P;
  Params32 Q;
  float dt;
  int kchunk;
  cudaStream_t s;
  template <int STAGE, int TX, int TY, int MINB, bool MC>
  cudaError_t run() {
    using S = Shape<TX, TY>;
    const dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY, (P.nz + kchunk - 1) / kchunk);
    k_stage32<STAGE, TX, TY, MINB, MC><<<grid, S::kThreads, sizeof(Smem<S>), s>>>(
        b.U, b.U1, P, Q, dt, kchunk, b.ctr);
    return cudaGetLastError();
  }
};

struct LaunchBatch {
  const BatchDevice& b;
  int cls;
  int kchunk;
  int sms;
  unsigned* counter;
  cudaStream_t s;
  template <int STAGE, int TX, int TY, int MINB, bool MC>
  cudaError_t run() {
    using S = Shape<TX, TY>;
    k_stage32_batch<STAGE, TX, TY, MINB, MC><<<sms * MINB, S::kThreads, sizeof(Smem<S>), s>>>(
        b.U, b.U1, b.meshes, b.items + b.class_first[cls], b.class_count[cls], kchunk, counter,
        b.ctr);
    return cudaGetLastError();
  }
};

// Raises the dynamic shared-memory limit of a configuration's kernels (the
// plane buffers and staging ring take more than the default 48 KB).
struct RaiseSmemMesh {
  template <int STAGE, int TX, int TY, int MINB, bool MC>
  cudaError_t run() {
    return cudaFuncSetAttribute(k_stage32<STAGE, TX, TY, MINB, MC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(Smem<Shape<TX, TY>>));
  }
};
struct RaiseSmemBatch {
  template <int STAGE, int TX, int TY, int MINB, bool MC>
  cudaError_t run() {
    return cudaFuncSetAttribute(k_stage32_batch<STAGE, TX, TY, MINB, MC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(Smem<Shape<TX, TY>>));
  }
};

bool valid_config(int tile_x, int tile_y, int occupancy) {
  for (const auto& c : kShapes)
    if (c[0] == tile_x && c[1] == tile_y && c[2] == occupancy) return true;
  return false;
}

cudaError_t launch_stage(int stage, const StepBuffers& b, const fvd::Params& P, double dt,
                         int kchunk, double vacuum_ratio, int occupancy, int tile_x, int tile_y,
                         cudaStream_t s) {
  LaunchMesh fn{b, P, make_params32(P, vacuum_ratio), (float)dt, kchunk < 1 ? 1 : kchunk, s};
  return dispatch(stage, tile_x, tile_y, occupancy, fn.Q.theta == 2.0f, fn);
}

cudaError_t prepare_kernels() {
  RaiseSmemMesh fm;
  RaiseSmemBatch fb;
  cudaError_t e = cudaSuccess;
  for (int stage = 1; stage <= 2 && e == cudaSuccess; ++stage)
    for (int mc = 0; mc < 2 && e == cudaSuccess; ++mc)
      for (const auto& c : kShapes) {
        if (e == cudaSuccess) e = dispatch(stage, c[0], c[1], c[2], mc != 0, fm);
        if (e == cudaSuccess) e = dispatch(stage, c[0], c[1], c[2], mc != 0, fb);
      }
  return e;
}

cudaError_t launch_reduce_dt(const double* U, const fvd::Params& P, double vacuum_ratio,
                             DevCounters* ctr, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&ctr->smax_bits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const long long n = (long long)P.nx * P.ny * P.nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 8LL * fv_sm_count()) blocks = 8LL * fv_sm_count();
  k_reduce_dt32<<<(unsigned)blocks, 256, 0, s>>>(U, P, make_params32(P, vacuum_ratio), ctr);
  return cudaGetLastError();
}

}  // namespace fv_fp32

namespace fv_fp32 {

cudaError_t launch_batch_max(const BatchDevice& b, cudaStream_t s) {
  k_batch_reset<<<1, 128, 0, s>>>(b.meshes, b.nmesh, b.next_item);
  if (b.ndt_blocks > 0) k_batch_dt<<<b.ndt_blocks, 256, 0, s>>>(b.U, b.meshes, b.dt_blocks, b.ctr);
  return cudaGetLastError();
}

cudaError_t launch_batch_dt(const BatchDevice& b, double cfl, cudaStream_t s) {
  k_batch_dt_finalize<<<1, 128, 0, s>>>(b.meshes, b.nmesh, cfl);
  k_batch_reset<<<1, 128, 0, s>>>(b.meshes, b.nmesh, b.next_item);
  return cudaGetLastError();
}

// The MC form when every mesh of the batch has limiter parameter 2, else the
// general form for all (same results as each mesh's single-mesh kernel).
cudaError_t launch_batch_stage(int stage, const BatchDevice& b, int cls, int kchunk,
                               int occupancy, int tile_x, int tile_y, int num_sms,
                               cudaStream_t s) {
  if (b.class_count[cls] == 0) return cudaSuccess;
  LaunchBatch fn{b, cls, kchunk, num_sms, b.next_item + 2 * cls + (stage == 1 ? 0 : 1), s};
  return dispatch(stage, tile_x, tile_y, occupancy, b.all_mc, fn);
}

cudaError_t launch_batch_ghosts(int stage, const BatchDevice& b, cudaStream_t s) {
  if (b.nghost_blocks > 0)
    k_batch_ghosts<<<b.nghost_blocks, kBatchGhostChunk, 0, s>>>(stage == 1 ? b.U1 : b.U,
                                                                b.meshes, b.ghost_blocks);
  return cudaGetLastError();
}

}  // namespace fv_fp32
