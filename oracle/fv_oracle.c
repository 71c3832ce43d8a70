/*
 * fv_oracle.c -- plain, slow FP64 CPU oracle of one RK2 finite-volume step of
 * the 3D ideal-gas Euler equations (Budiardja & Cardall, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product library.  It shares
 * no source with the CUDA path.  Build with -O2 -ffp-contract=off so that
 * every + - * / sqrt below is one IEEE round-to-nearest operation.
 *
 * The step follows Algorithm 1 ("Fluid Evolution") line by line in meaning:
 *   FluidOld = FluidCurrent
 *   ComputeDifferences -> ComputeReconstruction -> ComputeFluxes
 *     (with the RiemannSolverInput stage named in the Fig. 4 caption)
 *   ComputeUpdate(TimeStep) -> FluidUpdate
 *   FluidCurrent = FluidOld + FluidUpdate;            GhostExchange
 *   ... the same kernels again ...
 *   FluidCurrent = 0.5 * (FluidOld + FluidCurrent + FluidUpdate); GhostExchange
 * Each kernel is a whole-array pass over the ghosted storage, as in the
 * paper; ComputeDifferences uses the index range of Listing 2.
 *
 * The paper does not state the limiter, the Riemann solver, the wave-speed
 * bounds, the CFL formula, the boundary condition or gamma.  This file uses
 * the readings written out at each function: primitive-variable
 * reconstruction with a generalised minmod (MC) limiter, the HLL flux with
 * Davis-type bounds that include zero, the unsplit CFL sum, outflow
 * (zero-gradient) or periodic ghosts, and a first-order fallback at faces
 * whose reconstructed density or pressure is not positive.
 *
 * Parity pins (tests/test_oracle_*.py): exact Sod Riemann solution and its
 * first->second order convergence, smooth-wave convergence rates, round-off
 * conservation, bitwise uniform-state preservation, planar 3D == 1D, mirror
 * and axis-permutation symmetry, a textbook-form HLL written independently,
 * closed-form dt, and an exact (fsum) check of the pairwise sums.
 */
#include "fv_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NF 5

size_t orc_field_size(const orc_mesh* m) {
  return (size_t)(m->nx + 4) * (size_t)(m->ny + 4) * (size_t)(m->nz + 4);
}

/* offset of cell (i,j,k), each index in [-2, n+1] */
static size_t at(const orc_mesh* m, int i, int j, int k) {
  return ((size_t)(k + 2) * (size_t)(m->ny + 4) + (size_t)(j + 2)) *
             (size_t)(m->nx + 4) + (size_t)(i + 2);
}

static int extent(const orc_mesh* m, int axis) {
  return axis == 0 ? m->nx : (axis == 1 ? m->ny : m->nz);
}

static double cell_width(const orc_mesh* m, int axis) {
  return axis == 0 ? m->lx / m->nx : (axis == 1 ? m->ly / m->ny : m->lz / m->nz);
}

/* ------------------------------------------------------------------------ */
/* GhostExchange (Algorithm 1) on a single domain: the physical boundary.    */
/* Outflow copies the nearest interior cell; periodic wraps modulo n.        */
/* ------------------------------------------------------------------------ */
static int ghost_source(int g, int n, int bc) {
  if (g >= 0 && g < n) return g;
  if (bc == ORC_BC_PERIODIC) {
    int r = g % n;
    return r < 0 ? r + n : r;
  }
  return g < 0 ? 0 : n - 1;
}

void orc_fill_ghosts(const orc_mesh* m, double* U) {
  const size_t fs = orc_field_size(m);
  const int nx = m->nx, ny = m->ny, nz = m->nz;
  const int gx[4] = {-2, -1, nx, nx + 1};
  const int gy[4] = {-2, -1, ny, ny + 1};
  const int gz[4] = {-2, -1, nz, nz + 1};
  for (int q = 0; q < NF; ++q) {
    double* V = U + (size_t)q * fs;
    /* x faces, over all j and k (ghosts included) */
    for (int k = -2; k <= nz + 1; ++k)
      for (int j = -2; j <= ny + 1; ++j)
        for (int g = 0; g < 4; ++g)
          V[at(m, gx[g], j, k)] = V[at(m, ghost_source(gx[g], nx, m->bc[0]), j, k)];
    /* y faces, over all i and k */
    for (int k = -2; k <= nz + 1; ++k)
      for (int g = 0; g < 4; ++g)
        for (int i = -2; i <= nx + 1; ++i)
          V[at(m, i, gy[g], k)] = V[at(m, i, ghost_source(gy[g], ny, m->bc[1]), k)];
    /* z faces, over all i and j */
    for (int g = 0; g < 4; ++g)
      for (int j = -2; j <= ny + 1; ++j)
        for (int i = -2; i <= nx + 1; ++i)
          V[at(m, i, j, gz[g])] = V[at(m, i, j, ghost_source(gz[g], nz, m->bc[2]))];
  }
}

/* ------------------------------------------------------------------------ */
/* Conserved <-> primitive for one state.                                    */
/* ------------------------------------------------------------------------ */
void orc_cons_to_prim(double gamma, const double u[5], double w[5]) {
  double rho = u[0];
  double ir = 1.0 / rho;
  double vx = u[1] * ir;
  double vy = u[2] * ir;
  double vz = u[3] * ir;
  double ke = 0.5 * ((u[1] * vx + u[2] * vy) + u[3] * vz);
  w[0] = rho;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = (gamma - 1.0) * (u[4] - ke);
}

void orc_prim_to_cons(double gamma, const double w[5], double u[5]) {
  double rho = w[0];
  double mx = rho * w[1];
  double my = rho * w[2];
  double mz = rho * w[3];
  double ke = 0.5 * ((mx * w[1] + my * w[2]) + mz * w[3]);
  double igm1 = 1.0 / (gamma - 1.0);
  u[0] = rho;
  u[1] = mx;
  u[2] = my;
  u[3] = mz;
  u[4] = w[4] * igm1 + ke;
}

/* ------------------------------------------------------------------------ */
/* Limiter: generalised minmod of (theta*dL, (dL+dR)/2, theta*dR).           */
/* theta = 2 is the monotonised-central limiter, 1 minmod, 0 first order.    */
/* Mixed signs or any zero give +0.                                          */
/* ------------------------------------------------------------------------ */
double orc_minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) {
    double r = a;
    if (b < r) r = b;
    if (c < r) r = c;
    return r;
  }
  if (a < 0.0 && b < 0.0 && c < 0.0) {
    double r = a;
    if (b > r) r = b;
    if (c > r) r = c;
    return r;
  }
  return 0.0;
}

double orc_limited_slope(double theta, double d_minus, double d_plus) {
  return orc_minmod3(theta * d_minus, 0.5 * (d_minus + d_plus), theta * d_plus);
}

/* ------------------------------------------------------------------------ */
/* RiemannSolverInput (Fig. 4 caption) and ComputeFluxes for one face.       */
/* ------------------------------------------------------------------------ */
typedef struct {
  double u[NF];  /* conserved face state */
  double f[NF];  /* Euler flux normal to the face */
  double c;      /* sound speed */
  double vn;     /* normal velocity */
} face_side;

static void euler_side(int axis, double gamma, const double w[5], face_side* s) {
  orc_prim_to_cons(gamma, w, s->u);
  double vn = w[1 + axis];
  double mn = s->u[1 + axis];
  s->vn = vn;
  s->c = sqrt(gamma * w[4] / w[0]);
  s->f[0] = mn;
  s->f[1] = mn * w[1];
  s->f[2] = mn * w[2];
  s->f[3] = mn * w[3];
  s->f[1 + axis] = s->f[1 + axis] + w[4];
  s->f[4] = (s->u[4] + w[4]) * vn;
}

static double max0(double a, double b) {
  double r = 0.0;
  if (a > r) r = a;
  if (b > r) r = b;
  return r;
}

/* HLL (Harten, Lax & van Leer 1983) with wave bounds from both face states:
 *   a+ = max(0, vL + cL, vR + cR),  a- = max(0, cL - vL, cR - vR)
 *   F = ((a+ FL + a- FR) - a+ a- (UR - UL)) * (1 / (a+ + a-))            */
void orc_hll_flux(int axis, double gamma, const double wl[5],
                  const double wr[5], double f[5]) {
  face_side L, R;
  euler_side(axis, gamma, wl, &L);
  euler_side(axis, gamma, wr, &R);
  double ap = max0(L.vn + L.c, R.vn + R.c);
  double am = max0(L.c - L.vn, R.c - R.vn);
  double r = 1.0 / (ap + am);
  double apm = ap * am;
  for (int q = 0; q < NF; ++q)
    f[q] = ((ap * L.f[q] + am * R.f[q]) - apm * (R.u[q] - L.u[q])) * r;
}

/* ------------------------------------------------------------------------ */
/* ComputeTimeStep: dt = cfl / max_cells sum_d (|v_d| + c) / dx_d.          */
/* ------------------------------------------------------------------------ */
static int nonphysical(const double w[5]) {
  return !(w[0] > 0.0 && w[4] > 0.0);
}

long orc_reduce_dt(const orc_mesh* m, const double* U, double cfl,
                   double* dt_out, double* smax_out) {
  const size_t fs = orc_field_size(m);
  const double idx = 1.0 / cell_width(m, 0);
  const double idy = 1.0 / cell_width(m, 1);
  const double idz = 1.0 / cell_width(m, 2);
  double smax = 0.0;
  long bad = 0;
  for (int k = 0; k < m->nz; ++k)
    for (int j = 0; j < m->ny; ++j)
      for (int i = 0; i < m->nx; ++i) {
        size_t o = at(m, i, j, k);
        double u[NF], w[NF];
        for (int q = 0; q < NF; ++q) u[q] = U[(size_t)q * fs + o];
        orc_cons_to_prim(m->gamma, u, w);
        if (nonphysical(w)) ++bad;
        double c = sqrt(m->gamma * w[4] / w[0]);
        double s = ((fabs(w[1]) + c) * idx + (fabs(w[2]) + c) * idy) +
                   (fabs(w[3]) + c) * idz;
        if (s > smax) smax = s;
      }
  if (smax_out) *smax_out = smax;
  if (dt_out) *dt_out = cfl / smax;
  return bad;
}

/* ------------------------------------------------------------------------ */
/* One substep: FluidUpdate = dt * L(FluidCurrent).                          */
/* Work arrays mirror the paper's StorageForm instances: Primitive,          */
/* Differences, Reconstruction (left/right face states) and Fluxes.          */
/* ------------------------------------------------------------------------ */
typedef struct {
  double* W[NF];      /* primitives, every ghosted cell */
  double* D[NF];      /* Differences along the current axis */
  double* S[NF];      /* limited slopes along the current axis */
  double* WL[NF];     /* Reconstruction: left state at face i-1/2, stored at i */
  double* WR[NF];     /* Reconstruction: right state at face i-1/2, stored at i */
  double* F[3][NF];   /* Fluxes per axis, face i-1/2 stored at cell i */
} work_arrays;

static void work_alloc(work_arrays* a, size_t fs) {
  for (int q = 0; q < NF; ++q) {
    a->W[q] = (double*)calloc(fs, sizeof(double));
    a->D[q] = (double*)calloc(fs, sizeof(double));
    a->S[q] = (double*)calloc(fs, sizeof(double));
    a->WL[q] = (double*)calloc(fs, sizeof(double));
    a->WR[q] = (double*)calloc(fs, sizeof(double));
    for (int d = 0; d < 3; ++d) a->F[d][q] = (double*)calloc(fs, sizeof(double));
  }
}

static void work_free(work_arrays* a) {
  for (int q = 0; q < NF; ++q) {
    free(a->W[q]); free(a->D[q]); free(a->S[q]); free(a->WL[q]); free(a->WR[q]);
    for (int d = 0; d < 3; ++d) free(a->F[d][q]);
  }
}

/* cell (i,j,k) shifted by `s` along `axis` */
static size_t at_shift(const orc_mesh* m, int i, int j, int k, int axis, int s) {
  if (axis == 0) return at(m, i + s, j, k);
  if (axis == 1) return at(m, i, j + s, k);
  return at(m, i, j, k + s);
}

/* Loop over cells whose coordinate along `axis` runs over [lo, hi] while the
 * other two coordinates run over the interior. */
#define FOR_AXIS_RANGE(m, axis, lo, hi, i, j, k)                                   \
  for (int k = ((axis) == 2 ? (lo) : 0); k <= ((axis) == 2 ? (hi) : (m)->nz - 1); ++k) \
    for (int j = ((axis) == 1 ? (lo) : 0); j <= ((axis) == 1 ? (hi) : (m)->ny - 1); ++j) \
      for (int i = ((axis) == 0 ? (lo) : 0); i <= ((axis) == 0 ? (hi) : (m)->nx - 1); ++i)

/* Primitive variables of every ghosted cell. */
static long compute_primitive(const orc_mesh* m, const double* U, work_arrays* a) {
  const size_t fs = orc_field_size(m);
  long bad = 0;
  for (int k = -2; k <= m->nz + 1; ++k)
    for (int j = -2; j <= m->ny + 1; ++j)
      for (int i = -2; i <= m->nx + 1; ++i) {
        size_t o = at(m, i, j, k);
        double u[NF], w[NF];
        for (int q = 0; q < NF; ++q) u[q] = U[(size_t)q * fs + o];
        orc_cons_to_prim(m->gamma, u, w);
        for (int q = 0; q < NF; ++q) a->W[q][o] = w[q];
        if (i >= 0 && i < m->nx && j >= 0 && j < m->ny && k >= 0 && k < m->nz &&
            nonphysical(w))
          ++bad;
      }
  return bad;
}

/* ComputeDifferences along `axis` (Listing 2): dV(i) = V(i) - V(i-1) for the
 * 1-based i = 0 .. n+2, i.e. 0-based i = -1 .. n+1. */
static void compute_differences(const orc_mesh* m, int axis, work_arrays* a) {
  const int n = extent(m, axis);
  for (int q = 0; q < NF; ++q) {
    FOR_AXIS_RANGE(m, axis, -1, n + 1, i, j, k) {
      size_t o = at(m, i, j, k);
      a->D[q][o] = a->W[q][o] - a->W[q][at_shift(m, i, j, k, axis, -1)];
    }
  }
}

/* ComputeReconstruction along `axis`: limited slope in cells -1 .. n, then
 * the two face states at faces i-1/2 for i = 0 .. n:
 *   WL = W(i-1) + 0.5 * S(i-1),   WR = W(i) - 0.5 * S(i)                */
static void compute_reconstruction(const orc_mesh* m, int axis, work_arrays* a) {
  const int n = extent(m, axis);
  for (int q = 0; q < NF; ++q) {
    FOR_AXIS_RANGE(m, axis, -1, n, i, j, k) {
      size_t o = at(m, i, j, k);
      a->S[q][o] = orc_limited_slope(m->theta, a->D[q][o],
                                     a->D[q][at_shift(m, i, j, k, axis, +1)]);
    }
    FOR_AXIS_RANGE(m, axis, 0, n, i, j, k) {
      size_t o = at(m, i, j, k);
      size_t ol = at_shift(m, i, j, k, axis, -1);
      a->WL[q][o] = a->W[q][ol] + 0.5 * a->S[q][ol];
      a->WR[q][o] = a->W[q][o] - 0.5 * a->S[q][o];
    }
  }
}

/* RiemannSolverInput + ComputeFluxes along `axis`.  A face whose
 * reconstructed density or pressure is not positive (or NaN) uses the two
 * adjacent cell averages instead (first order at that face). */
static long compute_fluxes(const orc_mesh* m, int axis, work_arrays* a) {
  const int n = extent(m, axis);
  long fallback = 0;
  FOR_AXIS_RANGE(m, axis, 0, n, i, j, k) {
    size_t o = at(m, i, j, k);
    size_t ol = at_shift(m, i, j, k, axis, -1);
    double wl[NF], wr[NF], f[NF];
    for (int q = 0; q < NF; ++q) {
      wl[q] = a->WL[q][o];
      wr[q] = a->WR[q][o];
    }
    if (nonphysical(wl) || nonphysical(wr)) {
      ++fallback;
      for (int q = 0; q < NF; ++q) {
        wl[q] = a->W[q][ol];
        wr[q] = a->W[q][o];
      }
    }
    orc_hll_flux(axis, m->gamma, wl, wr, f);
    for (int q = 0; q < NF; ++q) a->F[axis][q][o] = f[q];
  }
  return fallback;
}

/* ComputeUpdate(TimeStep): dU = dt * (-(Fx(i+1/2) - Fx(i-1/2))/dx
 *   - (Fy(j+1/2) - Fy(j-1/2))/dy - (Fz(k+1/2) - Fz(k-1/2))/dz), summed in
 * the order x, y, z with 1/dx precomputed. */
static void compute_update(const orc_mesh* m, const work_arrays* a, double dt,
                           double* dU) {
  const size_t fs = orc_field_size(m);
  const double inv[3] = {1.0 / cell_width(m, 0), 1.0 / cell_width(m, 1),
                         1.0 / cell_width(m, 2)};
  memset(dU, 0, (size_t)NF * fs * sizeof(double));
  for (int q = 0; q < NF; ++q)
    for (int k = 0; k < m->nz; ++k)
      for (int j = 0; j < m->ny; ++j)
        for (int i = 0; i < m->nx; ++i) {
          size_t o = at(m, i, j, k);
          double acc = -(a->F[0][q][at(m, i + 1, j, k)] - a->F[0][q][o]) * inv[0];
          acc = acc - (a->F[1][q][at(m, i, j + 1, k)] - a->F[1][q][o]) * inv[1];
          acc = acc - (a->F[2][q][at(m, i, j, k + 1)] - a->F[2][q][o]) * inv[2];
          dU[(size_t)q * fs + o] = dt * acc;
        }
}

static long substep_update(const orc_mesh* m, const double* U, double dt,
                           double* dU, long* n_face_fallback, work_arrays* a) {
  long bad = compute_primitive(m, U, a);
  long fb = 0;
  for (int axis = 0; axis < 3; ++axis) {
    compute_differences(m, axis, a);
    compute_reconstruction(m, axis, a);
    fb += compute_fluxes(m, axis, a);
  }
  compute_update(m, a, dt, dU);
  if (n_face_fallback) *n_face_fallback += fb;
  return bad;
}

long orc_compute_update(const orc_mesh* m, const double* U, double dt,
                        double* dU, long* n_face_fallback) {
  work_arrays a;
  work_alloc(&a, orc_field_size(m));
  if (n_face_fallback) *n_face_fallback = 0;
  long bad = substep_update(m, U, dt, dU, n_face_fallback, &a);
  work_free(&a);
  return bad;
}

/* One iteration of the Algorithm 1 loop body after ComputeTimeStep. */
long orc_step(const orc_mesh* m, double* U, double dt, long* n_face_fallback) {
  const size_t fs = orc_field_size(m);
  const size_t nv = (size_t)NF * fs;
  double* old = (double*)malloc(nv * sizeof(double));
  double* dU = (double*)malloc(nv * sizeof(double));
  work_arrays a;
  work_alloc(&a, fs);
  long bad = 0;
  if (n_face_fallback) *n_face_fallback = 0;

  memcpy(old, U, nv * sizeof(double));                    /* FluidOld = FluidCurrent */
  bad += substep_update(m, U, dt, dU, n_face_fallback, &a);
  for (int q = 0; q < NF; ++q)                            /* FluidCurrent = FluidOld + FluidUpdate */
    for (int k = 0; k < m->nz; ++k)
      for (int j = 0; j < m->ny; ++j)
        for (int i = 0; i < m->nx; ++i) {
          size_t o = (size_t)q * fs + at(m, i, j, k);
          U[o] = old[o] + dU[o];
        }
  orc_fill_ghosts(m, U);                                  /* GhostExchange */

  bad += substep_update(m, U, dt, dU, n_face_fallback, &a);
  for (int q = 0; q < NF; ++q)        /* FluidCurrent = 0.5 * (FluidOld + FluidCurrent + FluidUpdate) */
    for (int k = 0; k < m->nz; ++k)
      for (int j = 0; j < m->ny; ++j)
        for (int i = 0; i < m->nx; ++i) {
          size_t o = (size_t)q * fs + at(m, i, j, k);
          U[o] = 0.5 * ((old[o] + U[o]) + dU[o]);
        }
  orc_fill_ghosts(m, U);                                  /* GhostExchange */

  work_free(&a);
  free(dU);
  free(old);
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Conservation sums by a fixed pairwise tree.                               */
/* ------------------------------------------------------------------------ */
double orc_pairwise_sum(const double* v, size_t n) {
  if (n == 0) return 0.0;
  size_t p = 1;
  while (p < n) p <<= 1;
  double* a = (double*)calloc(p, sizeof(double));
  memcpy(a, v, n * sizeof(double));
  for (size_t len = p; len > 1; len >>= 1)
    for (size_t i = 0; i < len / 2; ++i) a[i] = a[2 * i] + a[2 * i + 1];
  double s = a[0];
  free(a);
  return s;
}

void orc_conserved_sums(const orc_mesh* m, const double* U, double out[5]) {
  const size_t fs = orc_field_size(m);
  const size_t n = (size_t)m->nx * m->ny * m->nz;
  const double vol = (cell_width(m, 0) * cell_width(m, 1)) * cell_width(m, 2);
  double* v = (double*)malloc(n * sizeof(double));
  for (int q = 0; q < NF; ++q) {
    size_t c = 0;
    for (int k = 0; k < m->nz; ++k)
      for (int j = 0; j < m->ny; ++j)
        for (int i = 0; i < m->nx; ++i) v[c++] = U[(size_t)q * fs + at(m, i, j, k)];
    out[q] = orc_pairwise_sum(v, n) * vol;
  }
  free(v);
}
