/*
 * fv_oracle.h -- plain FP64 CPU oracle of the RiemannProblem fluid step
 * (Budiardja & Cardall, "Targeting GPUs with OpenMP Directives on Summit",
 * Sec. 3, Algorithm 1 "Fluid Evolution", Listing 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may use it.  It shares no source with the CUDA path.
 *
 * Storage (Sec. 3, rank-3 remap of one StorageForm column with two ghost
 * layers, V(-1:nX+2, -1:nY+2, -1:nZ+2)): every field is a contiguous array of
 * (nx+4)*(ny+4)*(nz+4) doubles, x fastest; the 0-based cell (i,j,k) with
 * i in [-2, nx+1] lives at ((k+2)*(ny+4) + (j+2))*(nx+4) + (i+2).  A state
 * holds five such fields back to back: rho, rho*vx, rho*vy, rho*vz, E.
 */
#ifndef FV_ORACLE_H
#define FV_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_OUTFLOW = 0, ORC_BC_PERIODIC = 1 };

typedef struct {
  int nx, ny, nz;        /* interior cells per axis, >= 1 */
  double lx, ly, lz;     /* domain extents, origin at 0; dx = lx / nx */
  double gamma;          /* ratio of specific heats, > 1 */
  double theta;          /* limiter parameter: 0 first order, 1 minmod, 2 MC */
  int bc[3];             /* ORC_BC_* per axis */
} orc_mesh;

/* Number of doubles in one ghosted field. */
size_t orc_field_size(const orc_mesh* m);

/* Ghost fill ("GhostExchange", Algorithm 1): axis x, then y, then z; each
 * pass covers the full ghosted extent of the other two axes. */
void orc_fill_ghosts(const orc_mesh* m, double* U);

/* Single-state helpers (conserved u = rho, mx, my, mz, E; primitive
 * w = rho, vx, vy, vz, p). */
void orc_cons_to_prim(double gamma, const double u[5], double w[5]);
void orc_prim_to_cons(double gamma, const double w[5], double u[5]);
double orc_minmod3(double a, double b, double c);
double orc_limited_slope(double theta, double d_minus, double d_plus);
/* HLL flux through a face normal to `axis` (0,1,2) from face states wl, wr. */
void orc_hll_flux(int axis, double gamma, const double wl[5],
                  const double wr[5], double f[5]);

/* dt = cfl / max over interior cells of sum_d (|v_d| + c) / dx_d.
 * Returns the number of interior cells with rho <= 0, p <= 0 or NaN. */
long orc_reduce_dt(const orc_mesh* m, const double* U, double cfl,
                   double* dt_out, double* smax_out);

/* One substep's update FluidUpdate = dt * L(U) on interior cells (the other
 * entries of dU are set to 0).  U must have its ghosts filled.  Returns the
 * number of non-physical interior cells; *n_face_fallback (may be NULL)
 * receives the number of faces that fell back to first order. */
long orc_compute_update(const orc_mesh* m, const double* U, double dt,
                        double* dU, long* n_face_fallback);

/* One full RK2 step of Algorithm 1 on U (ghosts filled on entry and on
 * exit).  Returns the summed non-physical count of both substeps. */
long orc_step(const orc_mesh* m, double* U, double dt, long* n_face_fallback);

/* Per-field sum over interior cells times the cell volume, by a fixed
 * pairwise tree: values in (k, j, i) order, zero-padded to a power of two,
 * then a[m] = a[2m] + a[2m+1] level by level. */
void orc_conserved_sums(const orc_mesh* m, const double* U, double out[5]);

/* Pairwise tree sum of n doubles in the order given (the same tree). */
double orc_pairwise_sum(const double* v, size_t n);

#ifdef __cplusplus
}
#endif
#endif
