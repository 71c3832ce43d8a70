// fv_core.cu -- the C ABI of include/fv.h: mesh handles, validation, buffer
// ownership, stream ordering and error reporting.  All arithmetic runs in the
// kernels of fv_step_kernels.cu and fv_aux.cu.
#include "fv.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_set>
#include <vector>

#include "fv_internal.h"

namespace {

thread_local char g_last_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
  va_end(ap);
}

}  // namespace

void fv_internal_set_error(const char* msg) { set_error("%s", msg); }

namespace {
fv_status validate_desc(const fv_mesh_desc* d);
fvd::Params make_params(const fv_mesh_desc* d);
}  // namespace

fv_status fv_internal_validate_desc(const fv_mesh_desc* d) { return validate_desc(d); }
fvd::Params fv_internal_params(const fv_mesh_desc* d) { return make_params(d); }

namespace {

std::mutex g_registry_mutex;
std::unordered_set<const void*> g_registry;  // live mesh handles

}  // namespace

struct fv_mesh_s {
  fv_mesh_desc desc;
  fvd::Params P;
  cudaStream_t stream;
  int device;
  int num_sms;              // multiprocessors of the device
  size_t state_doubles;     // 5 * nfield
  size_t dense_doubles;     // 5 * nx * ny * nz
  StepBuffers buf;
  double* sums_work;        // pairwise-sum partials
  double* sums_out;         // 5 device doubles
  DevCounters* host_ctr;    // pinned mirror of the device counters
  double* host_sums;        // pinned, 5 doubles
  int stage_pending;        // 1 after fv_substep(1) until fv_substep(2)
  int kchunk;               // z planes per CTA of the fused FP32-bulk kernel
  double vacuum_ratio;      // FP32-bulk FP64 pressure-recovery threshold
  int occupancy;            // CTAs per SM the fused kernel is compiled for (2 or 3)
  int tile_x, tile_y;       // tile of the fused FP32-bulk kernel (fv_fp32::kShapes)
  int segments;             // pieces per grid line of the FP64 sweeps (0: automatic)
  bool fused64;             // FP64: one fused kernel per substep (else the per-axis sweeps)
  int ff_ctas_per_sm;       // FP64_FF: CTAs per SM its fused kernel is built for (1 or 2)
  int ff_tile_x, ff_tile_y; // FP64_FF: tile of its fused kernel (16 x 16; 32 x 8, 16)
  bool plane_skip;          // fused FP64_FF: skip the passes of unchanged planes
  bool ff_dense;            // FP64_FF: the last step evaluated >= 90% of its faces
  bool ff_sparse;           // FP64_FF: the last step evaluated < 15% of its faces
  long long faces_seen;     // evaluated / defined faces at the last fv_reduce_dt
  long long defined_seen;
  bool w_current;           // FP64 sweeps: W holds the primitives of U (from the dt pass)
  bool smax_current;        // fused paths: ctr->smax_next is the CFL maximum of U
  // profiling
  bool prof_on;
  std::vector<cudaEvent_t> event_pool;
  struct Timed { int cls; cudaEvent_t a, b; };
  std::vector<Timed> pending;
  long long launches[FV_KERNEL_NCLASS];
  long long faces_defined;  // face fluxes the method defines, since the last set_state
};

namespace {

// Makes the mesh's device current for the scope of one call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

fv_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return FV_ERR_CUDA;
}

fv_status check_handle(fv_mesh_t m) {
  if (!m) {
    set_error("NULL mesh handle");
    return FV_ERR_BAD_HANDLE;
  }
  std::lock_guard<std::mutex> lk(g_registry_mutex);
  if (!g_registry.count(m)) {
    set_error("mesh handle %p is not live (destroyed or foreign)", (void*)m);
    return FV_ERR_BAD_HANDLE;
  }
  return FV_OK;
}

fv_status validate_desc(const fv_mesh_desc* d) {
  if (!d) {
    set_error("desc is NULL");
    return FV_ERR_INVALID_ARG;
  }
  const int n[3] = {d->nx, d->ny, d->nz};
  const double l[3] = {d->lx, d->ly, d->lz};
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 1 || n[a] > (1 << 14)) {
      set_error("cell count %d on axis %d outside [1, 16384]", n[a], a);
      return FV_ERR_INVALID_ARG;
    }
    if (!(l[a] > 0.0) || !std::isfinite(l[a])) {
      set_error("extent %g on axis %d must be finite and > 0", l[a], a);
      return FV_ERR_INVALID_ARG;
    }
    if (d->bc[a] != FV_BC_OUTFLOW && d->bc[a] != FV_BC_PERIODIC) {
      set_error("boundary condition %d on axis %d unknown", d->bc[a], a);
      return FV_ERR_INVALID_ARG;
    }
  }
  const long long cells = (long long)(d->nx + 4) * (d->ny + 4) * (d->nz + 4);
  if (cells > (1LL << 31)) {
    set_error("mesh of %lld ghosted cells exceeds the 2^31 limit", cells);
    return FV_ERR_INVALID_ARG;
  }
  if (!(d->gamma > 1.0) || !std::isfinite(d->gamma)) {
    set_error("gamma %g must be finite and > 1", d->gamma);
    return FV_ERR_INVALID_ARG;
  }
  if (!(d->theta >= 0.0 && d->theta <= 2.0)) {
    set_error("theta %g outside [0, 2]", d->theta);
    return FV_ERR_INVALID_ARG;
  }
  if (d->precision != FV_PREC_FP64 && d->precision != FV_PREC_FP64_FMA &&
      d->precision != FV_PREC_FP32_BULK && d->precision != FV_PREC_FP64_FF) {
    set_error("precision %d unknown", d->precision);
    return FV_ERR_INVALID_ARG;
  }
  return FV_OK;
}

fvd::Params make_params(const fv_mesh_desc* d) {
  fvd::Params P;
  P.nx = d->nx;
  P.ny = d->ny;
  P.nz = d->nz;
  P.sy = d->nx + 4;
  P.sz = (long long)(d->nx + 4) * (d->ny + 4);
  P.nfield = P.sz * (d->nz + 4);
  P.gamma = d->gamma;
  P.gm1 = d->gamma - 1.0;
  P.igm1 = 1.0 / (d->gamma - 1.0);
  P.theta = d->theta;
  // cell widths and their inverses exactly as the method defines them
  const double dx = d->lx / d->nx, dy = d->ly / d->ny, dz = d->lz / d->nz;
  P.inv_d[0] = 1.0 / dx;
  P.inv_d[1] = 1.0 / dy;
  P.inv_d[2] = 1.0 / dz;
  for (int a = 0; a < 3; ++a) P.bc[a] = d->bc[a];
  return P;
}

void free_mesh(fv_mesh_s* m) {
  for (auto& t : m->pending) {
    m->event_pool.push_back(t.a);
    m->event_pool.push_back(t.b);
  }
  for (cudaEvent_t e : m->event_pool) cudaEventDestroy(e);
  cudaFree(m->buf.U);
  cudaFree(m->buf.U1);
  cudaFree(m->buf.W);
  cudaFree(m->buf.keep);
  cudaFree(m->buf.ACC);
  cudaFree(m->buf.ctr);
  cudaFree(m->sums_work);
  cudaFree(m->sums_out);
  cudaFreeHost(m->host_ctr);
  cudaFreeHost(m->host_sums);
  delete m;
}

// Reads the device counters (and the dt maximum) into host_ctr; syncs.
fv_status read_counters(fv_mesh_t m) {
  cudaError_t e = cudaMemcpyAsync(m->host_ctr, m->buf.ctr, sizeof(DevCounters),
                                  cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading device counters");
  return FV_OK;
}

fv_status nonphysical_status(fv_mesh_t m) {
  if (m->host_ctr->ff_range) {
    set_error("%llu cells outside the float-float operand range (density and pressure "
              "2^-30 .. 2^30, velocities below 2^20): the state since is not valid; step "
              "such states with FV_PREC_FP64 or FV_PREC_FP64_FMA", m->host_ctr->ff_range);
    return FV_ERR_INVALID_ARG;
  }
  if (m->host_ctr->np_step || m->host_ctr->np_dt) {
    set_error("non-physical state: %llu cell detections in the step, %llu in the time step",
              m->host_ctr->np_step, m->host_ctr->np_dt);
    return FV_ERR_NONPHYSICAL;
  }
  return FV_OK;
}

cudaEvent_t take_event(fv_mesh_t m) {
  if (!m->event_pool.empty()) {
    cudaEvent_t e = m->event_pool.back();
    m->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launches one kernel (or a short fixed sequence) of class `cls`, counting
// it and, while profiling is on, bracketing it with events on the stream.
template <class F>
cudaError_t timed(fv_mesh_t m, int cls, int nlaunch, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (m->prof_on) {
    a = take_event(m);
    b = take_event(m);
    if (a && b) cudaEventRecord(a, m->stream);
  }
  cudaError_t e = launch();
  m->launches[cls] += nlaunch;
  if (m->prof_on && a && b) {
    cudaEventRecord(b, m->stream);
    m->pending.push_back({cls, a, b});
  } else {
    if (a) m->event_pool.push_back(a);
    if (b) m->event_pool.push_back(b);
  }
  return e;
}

// Faces normal to `axis` (each evaluated once per substep by the method).
long long faces_normal_to(const fvd::Params& P, int axis) {
  const long long nx = P.nx, ny = P.ny, nz = P.nz;
  return axis == 0 ? (nx + 1) * ny * nz : axis == 1 ? nx * (ny + 1) * nz : nx * ny * (nz + 1);
}

// The float-float kernel's z chunk: each CTA marches over `chunk` planes after
// a 4-plane window prologue, and the launch runs in rounds of (SMs x CTAs per
// SM) resident CTAs, so its time is about rounds x (chunk + 4) plane steps.
// The chunk (16 planes at least, or the whole column) minimising that: at
// 256^3 with 16 x 16 tiles at 2 CTAs per SM, 7 chunks of 37 planes (5.9
// rounds) against 4 of 64 (3.4 rounds, the last one a third full): 5.93 ->
// 5.68 ms per step over the 200-step oblique workload (same bits; chunks do
// not change the arithmetic).
int ff_auto_kchunk(const fvd::Params& P, int tile_x, int tile_y, int ctas_per_sm) {
  const long long tiles = (long long)((P.nx + tile_x - 1) / tile_x) * ((P.ny + tile_y - 1) / tile_y);
  const long long resident = (long long)fv_sm_count() * ctas_per_sm;
  int best = P.nz;
  long long best_cost = -1;
  for (int n = 1; n <= P.nz; ++n) {
    const int chunk = (P.nz + n - 1) / n;
    if (n > 1 && chunk < 16) break;
    if (n > 1 && (P.nz + chunk - 1) / chunk != n) continue;   // the same chunk as a smaller n
    const long long rounds = (tiles * n + resident - 1) / resident;
    const long long cost = rounds * (chunk + 4);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = chunk;
    }
  }
  return best;
}

cudaError_t launch_substep(fv_mesh_t m, int stage, double dt) {
  for (int axis = 0; axis < 3; ++axis) m->faces_defined += faces_normal_to(m->P, axis);
  const bool fma = m->desc.precision == FV_PREC_FP64_FMA;
  const bool ff = m->desc.precision == FV_PREC_FP64_FF;
  if (m->desc.precision != FV_PREC_FP32_BULK && (m->fused64 || ff)) {
    // one kernel per substep; stage 2 also takes the CFL maximum of its output
    m->smax_current = false;
    m->w_current = false;
    cudaError_t e = cudaSuccess;
    if (stage == 2)
      e = cudaMemsetAsync(&m->buf.ctr->smax_next, 0, sizeof(unsigned long long), m->stream);
    if (e == cudaSuccess)
      e = timed(m, FV_KERNEL_FUSED, 1, [&] {
        if (ff)
          return fv_fp64_ff::launch_fused(stage, m->buf, m->P, dt,
                                          m->kchunk > 0 ? m->kchunk
                                          : m->ff_sparse ? m->P.nz
                                                         : ff_auto_kchunk(m->P, m->ff_tile_x,
                                                                          m->ff_tile_y,
                                                                          m->ff_ctas_per_sm),
                                          m->ff_tile_x,
                                          m->ff_tile_y, m->ff_ctas_per_sm,
                                          m->plane_skip && !m->ff_dense, m->stream);
        return fma ? fv_fp64_fma::launch_fused(stage, m->buf, m->P, dt, m->kchunk, m->stream)
                   : fv_fp64_exact::launch_fused(stage, m->buf, m->P, dt, m->kchunk,
                                                 m->stream);
      });
    if (e != cudaSuccess) return e;
    double* dst = stage == 1 ? m->buf.U1 : m->buf.U;
    e = timed(m, FV_KERNEL_GHOST, 1, [&] { return launch_fill_ghosts(dst, m->P, m->stream); });
    m->smax_current = e == cudaSuccess && stage == 2;
    return e;
  }
  if (m->desc.precision == FV_PREC_FP32_BULK) {
    // stage 2 also takes the CFL maximum of its output (the next dt's)
    m->smax_current = false;
    cudaError_t e = cudaSuccess;
    if (stage == 2)
      e = cudaMemsetAsync(&m->buf.ctr->smax_next, 0, sizeof(unsigned long long), m->stream);
    if (e == cudaSuccess)
      e = timed(m, FV_KERNEL_FUSED, 1, [&] {
        return fv_fp32::launch_stage(stage, m->buf, m->P, dt, m->kchunk, m->vacuum_ratio,
                                     m->occupancy, m->tile_x, m->tile_y, m->stream);
      });
    if (e != cudaSuccess) return e;
    double* dst = stage == 1 ? m->buf.U1 : m->buf.U;
    e = timed(m, FV_KERNEL_GHOST, 1, [&] { return launch_fill_ghosts(dst, m->P, m->stream); });
    m->smax_current = e == cudaSuccess && stage == 2;
    return e;
  }
  const double* src = stage == 1 ? m->buf.U : m->buf.U1;
  cudaError_t e = cudaSuccess;
  // the dt pass since the state last changed left U's primitives in W
  if (!(stage == 1 && m->w_current)) {
    e = timed(m, FV_KERNEL_PRIM, 1, [&] {
      // substep 2: W holds U's primitives, and the cells substep 1 copied
      // unchanged keep them
      const bool keep = stage == 2;
      return fma ? fv_fp64_fma::launch_prim(src, m->buf, m->P, keep, m->stream)
                 : fv_fp64_exact::launch_prim(src, m->buf, m->P, keep, m->stream);
    });
  }
  m->w_current = false;
  m->smax_current = false;
  for (int axis = 0; axis < 3 && e == cudaSuccess; ++axis) {
    e = timed(m, FV_KERNEL_SWEEP_X + axis, 1, [&] {
      return fma ? fv_fp64_fma::launch_sweep(axis, stage, m->buf, m->P, dt, m->segments,
                                             m->num_sms, m->stream)
                 : fv_fp64_exact::launch_sweep(axis, stage, m->buf, m->P, dt, m->segments,
                                               m->num_sms, m->stream);
    });
  }
  if (e != cudaSuccess) return e;
  double* dst = stage == 1 ? m->buf.U1 : m->buf.U;
  return timed(m, FV_KERNEL_GHOST, 1,
               [&] { return launch_fill_ghosts(dst, m->P, m->stream); });
}

}  // namespace

extern "C" {

fv_status fv_create_mesh(const fv_mesh_desc* desc, void* cuda_stream, fv_mesh_t* out) {
  if (!out) {
    set_error("out is NULL");
    return FV_ERR_INVALID_ARG;
  }
  *out = nullptr;
  fv_status st = validate_desc(desc);
  if (st != FV_OK) return st;
  fv_mesh_s* m = new fv_mesh_s();
  std::memset(&m->buf, 0, sizeof m->buf);
  m->desc = *desc;
  m->P = make_params(desc);
  m->stream = (cudaStream_t)cuda_stream;
  m->stage_pending = 0;
  m->prof_on = false;
  // z planes per CTA of the fused kernels: the FP32-bulk one measured
  // fastest with 32 at 256^3; the float-float one picks its chunk per launch
  // shape (0: ff_auto_kchunk) unless FV_TUNE_KCHUNK sets one
  m->kchunk = desc->precision == FV_PREC_FP64_FF ? 0 : desc->nz >= 64 ? 32 : desc->nz;
  m->vacuum_ratio = 0.99;
  m->occupancy = 2;
  m->tile_x = 16;   // 16 x 8: per-warp reuse decisions over 16 x 2 cells
  m->tile_y = 8;
  m->segments = 0;
  m->fused64 = false;
  m->ff_ctas_per_sm = 2;
  m->ff_tile_x = 16;   // 16 x 16 at 2 CTAs per SM (see fv_fused_ff_kernels.cu)
  m->ff_tile_y = 16;
  m->plane_skip = true;
  m->ff_dense = false;
  m->ff_sparse = false;
  m->faces_seen = m->defined_seen = 0;
  m->w_current = false;
  m->smax_current = false;
  for (int c = 0; c < FV_KERNEL_NCLASS; ++c) m->launches[c] = 0;
  m->faces_defined = 0;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  if (e == cudaSuccess && desc->precision == FV_PREC_FP32_BULK) e = fv_fp32::prepare_kernels();
  if (e == cudaSuccess && desc->precision == FV_PREC_FP64_FF) e = fv_fp64_ff::prepare_fused();
  else if (e == cudaSuccess && desc->precision != FV_PREC_FP32_BULK)
    e = desc->precision == FV_PREC_FP64_FMA ? fv_fp64_fma::prepare_fused()
                                            : fv_fp64_exact::prepare_fused();
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaGetDevice");
  }
  m->state_doubles = (size_t)fvd::NF * m->P.nfield;
  m->dense_doubles = (size_t)fvd::NF * desc->nx * desc->ny * desc->nz;
  const size_t sb = m->state_doubles * sizeof(double);
  const size_t db = m->dense_doubles * sizeof(double);
  const size_t wb = sums_work_doubles(m->P) * sizeof(double);
  // the per-axis sweeps (FP64 and FP64-FMA builds) need primitive and flag arrays
  const bool sweeps_possible =
      desc->precision == FV_PREC_FP64 || desc->precision == FV_PREC_FP64_FMA;
  if ((e = cudaMalloc(&m->buf.U, sb)) != cudaSuccess ||
      (e = cudaMalloc(&m->buf.U1, sb)) != cudaSuccess ||
      (sweeps_possible && (e = cudaMalloc(&m->buf.W, sb)) != cudaSuccess) ||
      (sweeps_possible &&
       (e = cudaMalloc(&m->buf.keep, m->dense_doubles / fvd::NF)) != cudaSuccess) ||
      (e = cudaMalloc(&m->buf.ACC, db)) != cudaSuccess ||
      (e = cudaMalloc(&m->buf.ctr, sizeof(DevCounters))) != cudaSuccess ||
      (e = cudaMalloc(&m->sums_work, wb)) != cudaSuccess ||
      (e = cudaMalloc(&m->sums_out, 5 * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&m->host_ctr, sizeof(DevCounters))) != cudaSuccess ||
      (e = cudaMallocHost(&m->host_sums, 5 * sizeof(double))) != cudaSuccess) {
    cudaGetLastError();
    set_error("allocating %.3f GB of mesh storage: %s", (3.0 * sb + db) / 1e9,
              cudaGetErrorString(e));
    free_mesh(m);
    return e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA;
  }
  if ((e = cudaMemsetAsync(m->buf.U, 0, sb, m->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(m->buf.U1, 0, sb, m->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(m->buf.ctr, 0, sizeof(DevCounters), m->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(m->stream)) != cudaSuccess) {
    free_mesh(m);
    return cuda_fail(e, "initialising mesh storage");
  }
  {
    std::lock_guard<std::mutex> lk(g_registry_mutex);
    g_registry.insert(m);
  }
  *out = m;
  return FV_OK;
}

fv_status fv_destroy_mesh(fv_mesh_t m) {
  if (!m) return FV_OK;
  {
    std::lock_guard<std::mutex> lk(g_registry_mutex);
    if (!g_registry.erase(m)) {
      set_error("mesh handle %p is not live (destroyed or foreign)", (void*)m);
      return FV_ERR_BAD_HANDLE;
    }
  }
  DeviceGuard g(m->device);
  cudaStreamSynchronize(m->stream);
  free_mesh(m);
  return FV_OK;
}

fv_status fv_set_state(fv_mesh_t m, const double* U, int on_device) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (!U) {
    set_error("U is NULL");
    return FV_ERR_INVALID_ARG;
  }
  DeviceGuard g(m->device);
  cudaError_t e;
  const double* src = U;
  if (!on_device) {  // stage through the accumulator, which is free between steps
    e = cudaMemcpyAsync(m->buf.ACC, U, m->dense_doubles * sizeof(double),
                        cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copying the state to the device");
    src = m->buf.ACC;
  }
  e = timed(m, FV_KERNEL_OTHER, 1,
            [&] { return launch_scatter_interior(src, m->buf.U, m->P, m->stream); });
  if (e != cudaSuccess) return cuda_fail(e, "scatter kernel");
  e = timed(m, FV_KERNEL_GHOST, 1, [&] { return launch_fill_ghosts(m->buf.U, m->P, m->stream); });
  if (e != cudaSuccess) return cuda_fail(e, "ghost-fill kernel");
  if ((e = cudaMemsetAsync(m->buf.ctr, 0, sizeof(DevCounters), m->stream)) != cudaSuccess)
    return cuda_fail(e, "clearing counters");
  m->faces_defined = 0;
  m->faces_seen = m->defined_seen = 0;
  m->ff_dense = false;
  m->ff_sparse = false;
  m->stage_pending = 0;
  m->w_current = false;
  m->smax_current = false;
  if (!on_device && (e = cudaStreamSynchronize(m->stream)) != cudaSuccess)
    return cuda_fail(e, "fv_set_state");
  return FV_OK;
}

static fv_status get_state_impl(fv_mesh_t m, double* U, int on_device, bool ghosted) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (!U) {
    set_error("U is NULL");
    return FV_ERR_INVALID_ARG;
  }
  DeviceGuard g(m->device);
  const double* cur = m->stage_pending ? m->buf.U1 : m->buf.U;
  cudaError_t e;
  if (ghosted) {
    e = cudaMemcpyAsync(U, cur, m->state_doubles * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copying the ghosted state");
  } else {
    double* dst = on_device ? U : m->buf.ACC;
    e = timed(m, FV_KERNEL_OTHER, 1,
              [&] { return launch_gather_interior(cur, dst, m->P, m->stream); });
    if (e != cudaSuccess) return cuda_fail(e, "gather kernel");
    if (!on_device) {
      e = cudaMemcpyAsync(U, m->buf.ACC, m->dense_doubles * sizeof(double),
                          cudaMemcpyDeviceToHost, m->stream);
      if (e != cudaSuccess) return cuda_fail(e, "copying the state to the host");
    }
  }
  if ((st = read_counters(m)) != FV_OK) return st;
  return nonphysical_status(m);
}

fv_status fv_get_state(fv_mesh_t m, double* U, int on_device) {
  return get_state_impl(m, U, on_device, false);
}

fv_status fv_get_ghosted_state(fv_mesh_t m, double* U, int on_device) {
  return get_state_impl(m, U, on_device, true);
}

fv_status fv_reduce_dt(fv_mesh_t m, double cfl, double* dt_out) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (!dt_out || !(cfl > 0.0) || !std::isfinite(cfl)) {
    set_error("fv_reduce_dt needs cfl > 0 (got %g) and a non-NULL dt_out", cfl);
    return FV_ERR_INVALID_ARG;
  }
  if (m->stage_pending) {
    set_error("fv_reduce_dt called between the two RK substeps");
    return FV_ERR_INVALID_ARG;
  }
  DeviceGuard g(m->device);
  const bool fp32 = m->desc.precision == FV_PREC_FP32_BULK;
  const bool fma = m->desc.precision == FV_PREC_FP64_FMA;
  const bool ffp = m->desc.precision == FV_PREC_FP64_FF;
  const bool fused = fp32 || ffp || m->fused64;
  // fused paths: the last stage 2 took the maximum of the current state
  const bool cached = fused && m->smax_current;
  if (!cached) {
    cudaError_t e = timed(m, FV_KERNEL_DT, 1, [&] {
      if (fp32)
        return fv_fp32::launch_reduce_dt(m->buf.U, m->P, m->vacuum_ratio, m->buf.ctr, m->stream);
      if (ffp) return fv_fp64_ff::launch_dt(m->buf.U, m->buf, m->P, m->stream);
      if (m->fused64)
        return fma ? fv_fp64_fma::launch_dt(m->buf.U, m->buf, m->P, m->stream)
                   : fv_fp64_exact::launch_dt(m->buf.U, m->buf, m->P, m->stream);
      return fma ? fv_fp64_fma::launch_prim_dt(m->buf.U, m->buf, m->P, m->stream)
                 : fv_fp64_exact::launch_prim_dt(m->buf.U, m->buf, m->P, m->stream);
    });
    if (e != cudaSuccess) return cuda_fail(e, "time-step kernel");
    m->w_current = !fused;
  }
  if ((st = read_counters(m)) != FV_OK) return st;
  if (ffp) {
    // where the steps since the last read evaluated nearly every face, no tile
    // plane repeats and the plane skip only costs its flags: the next steps
    // run the float-float kernel built without it (the same bits)
    const long long ev = (long long)m->host_ctr->faces - m->faces_seen;
    const long long de = m->faces_defined - m->defined_seen;
    if (de > 0 && ev >= 0) {
      m->ff_dense = 10 * ev >= 9 * de;
      // few faces evaluated: most tile planes repeat the plane below, and
      // one z chunk per tile column (no chunk starts past the first) beats
      // shorter chunks' balance
      m->ff_sparse = 20 * ev < 3 * de;
    }
    m->faces_seen = (long long)m->host_ctr->faces;
    m->defined_seen = m->faces_defined;
  }
  double smax;
  std::memcpy(&smax, cached ? &m->host_ctr->smax_next : &m->host_ctr->smax_bits, sizeof smax);
  *dt_out = cfl / smax;
  return nonphysical_status(m);
}

fv_status fv_substep(fv_mesh_t m, int stage, double dt) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (!(dt >= 0.0) || !std::isfinite(dt)) {
    set_error("dt %g must be finite and >= 0", dt);
    return FV_ERR_INVALID_ARG;
  }
  if (stage != 1 && stage != 2) {
    set_error("stage %d must be 1 or 2", stage);
    return FV_ERR_INVALID_ARG;
  }
  if ((stage == 1) == (m->stage_pending != 0)) {
    set_error(stage == 1 ? "substep 1 requested while substep 2 is pending"
                         : "substep 2 requested without substep 1");
    return FV_ERR_INVALID_ARG;
  }
  DeviceGuard g(m->device);
  cudaError_t e = launch_substep(m, stage, dt);
  if (e != cudaSuccess) return cuda_fail(e, "substep kernels");
  m->stage_pending = stage == 1;
  return FV_OK;
}

fv_status fv_step(fv_mesh_t m, double dt) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (m->stage_pending) {
    set_error("fv_step called between the two RK substeps");
    return FV_ERR_INVALID_ARG;
  }
  if ((st = fv_substep(m, 1, dt)) != FV_OK) return st;
  return fv_substep(m, 2, dt);
}

fv_status fv_fill_ghosts(fv_mesh_t m) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  DeviceGuard g(m->device);
  double* cur = m->stage_pending ? m->buf.U1 : m->buf.U;
  m->w_current = false;
  m->smax_current = false;
  cudaError_t e = timed(m, FV_KERNEL_GHOST, 1, [&] { return launch_fill_ghosts(cur, m->P, m->stream); });
  if (e != cudaSuccess) return cuda_fail(e, "ghost-fill kernel");
  return FV_OK;
}

fv_status fv_conserved_sums(fv_mesh_t m, double out[5]) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (!out) {
    set_error("out is NULL");
    return FV_ERR_INVALID_ARG;
  }
  DeviceGuard g(m->device);
  const double* cur = m->stage_pending ? m->buf.U1 : m->buf.U;
  cudaError_t e = timed(m, FV_KERNEL_OTHER, 1, [&] {
    return launch_pairwise_sums(cur, m->P, m->sums_work, m->sums_out, m->stream);
  });
  if (e != cudaSuccess) return cuda_fail(e, "sum kernels");
  e = cudaMemcpyAsync(m->host_sums, m->sums_out, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                      m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading sums");
  const double dx = m->desc.lx / m->desc.nx, dy = m->desc.ly / m->desc.ny,
               dz = m->desc.lz / m->desc.nz;
  const double vol = (dx * dy) * dz;
  for (int q = 0; q < 5; ++q) out[q] = m->host_sums[q] * vol;
  return FV_OK;
}

fv_status fv_get_counters(fv_mesh_t m, long long* nonphysical_cells, long long* fallback_faces) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  DeviceGuard g(m->device);
  if ((st = read_counters(m)) != FV_OK) return st;
  if (nonphysical_cells)
    *nonphysical_cells = (long long)(m->host_ctr->np_step + m->host_ctr->np_dt);
  if (fallback_faces) *fallback_faces = (long long)m->host_ctr->fallback;
  return FV_OK;
}

fv_status fv_get_face_counts(fv_mesh_t m, long long* evaluated, long long* defined) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  DeviceGuard g(m->device);
  if ((st = read_counters(m)) != FV_OK) return st;
  if (evaluated) *evaluated = (long long)m->host_ctr->faces;
  if (defined) *defined = m->faces_defined;
  return FV_OK;
}

fv_status fv_set_tuning(fv_mesh_t m, int key, double value) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (key == FV_TUNE_KCHUNK) {
    if (!(value >= 1.0 && value <= 1 << 20) || value != (double)(int)value) {
      set_error("FV_TUNE_KCHUNK must be an integer >= 1 (got %g)", value);
      return FV_ERR_INVALID_ARG;
    }
    m->kchunk = (int)value;
    return FV_OK;
  }
  if (key == FV_TUNE_VACUUM_RATIO) {
    if (!(value > 0.0) || !std::isfinite(value)) {
      set_error("FV_TUNE_VACUUM_RATIO must be finite and > 0 (got %g)", value);
      return FV_ERR_INVALID_ARG;
    }
    m->vacuum_ratio = value;
    return FV_OK;
  }
  if ((key == FV_TUNE_OCCUPANCY || key == FV_TUNE_TILE_Y || key == FV_TUNE_TILE_X) &&
      m->desc.precision == FV_PREC_FP64_FF) {
    // the float-float kernel's (tile x, tile y, CTAs per SM) must stay one of
    // its built shapes after the change
    const int v = (int)value;
    const bool integral = value == (double)v;
    const int tx = key == FV_TUNE_TILE_X ? v : m->ff_tile_x;
    const int ty = key == FV_TUNE_TILE_Y ? v : m->ff_tile_y;
    const int oc = key == FV_TUNE_OCCUPANCY ? v : m->ff_ctas_per_sm;
    if (!integral || !fv_fp64_ff::valid_fused_config(tx, ty, oc)) {
      set_error("tuning key %d = %g would make (tile_x, tile_y, CTAs per SM) = (%d, %d, %d), "
                "not a built shape of the float-float kernel: (16, 16, 1 | 2), (32, 8, 1 | 2), "
                "(32, 16, 1)",
                (int)key, value, tx, ty, oc);
      return FV_ERR_INVALID_ARG;
    }
    m->ff_tile_x = tx;
    m->ff_tile_y = ty;
    m->ff_ctas_per_sm = oc;
    return FV_OK;
  }
  if (key == FV_TUNE_OCCUPANCY || key == FV_TUNE_TILE_Y || key == FV_TUNE_TILE_X) {
    // the FP32-bulk kernel's (tile x, tile y, occupancy) must stay one of the
    // built shapes after the change
    const int v = (int)value;
    const bool integral = value == (double)v;
    const int tx = key == FV_TUNE_TILE_X ? v : m->tile_x;
    const int ty = key == FV_TUNE_TILE_Y ? v : m->tile_y;
    const int oc = key == FV_TUNE_OCCUPANCY ? v : m->occupancy;
    if (!integral || !fv_fp32::valid_config(tx, ty, oc)) {
      set_error("tuning key %d = %g would make (tile_x, tile_y, occupancy) = (%d, %d, %d), not "
                "a built shape of the FP32-bulk kernel: (32, 4|8|16, 2), (32, 8, 3), (16, 8, 2), "
                "(64, 4|8, 2), (128, 4, 2)",
                (int)key, value, tx, ty, oc);
      return FV_ERR_INVALID_ARG;
    }
    m->tile_x = tx;
    m->tile_y = ty;
    m->occupancy = oc;
    return FV_OK;
  }
  if (key == FV_TUNE_FP64_FUSED) {
    if (value != 0.0 && value != 1.0) {
      set_error("FV_TUNE_FP64_FUSED must be 0 or 1 (got %g)", value);
      return FV_ERR_INVALID_ARG;
    }
    if (m->stage_pending) {
      set_error("FV_TUNE_FP64_FUSED changed between the two RK substeps");
      return FV_ERR_INVALID_ARG;
    }
    m->fused64 = value != 0.0;
    m->w_current = false;
    m->smax_current = false;
    return FV_OK;
  }
  if (key == FV_TUNE_SWEEP_SEGMENTS) {
    if (!(value >= 0.0 && value <= 4096.0) || value != (double)(int)value) {
      set_error("FV_TUNE_SWEEP_SEGMENTS must be an integer in [0, 4096] (got %g)", value);
      return FV_ERR_INVALID_ARG;
    }
    m->segments = (int)value;
    return FV_OK;
  }
  if (key == FV_TUNE_PLANE_SKIP) {
    if (value != 0.0 && value != 1.0) {
      set_error("FV_TUNE_PLANE_SKIP must be 0 or 1 (got %g)", value);
      return FV_ERR_INVALID_ARG;
    }
    m->plane_skip = value != 0.0;
    return FV_OK;
  }
  set_error("unknown tuning key %d", key);
  return FV_ERR_INVALID_ARG;
}

fv_status fv_profile_enable(fv_mesh_t m, int on) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  m->prof_on = on != 0;
  return FV_OK;
}

fv_status fv_profile_read(fv_mesh_t m, double* ms, long long* launches) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  DeviceGuard g(m->device);
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "fv_profile_read");
  double acc[FV_KERNEL_NCLASS] = {0};
  for (auto& t : m->pending) {
    float x = 0.f;
    if (cudaEventElapsedTime(&x, t.a, t.b) == cudaSuccess) acc[t.cls] += x;
    m->event_pool.push_back(t.a);
    m->event_pool.push_back(t.b);
  }
  m->pending.clear();
  for (int c = 0; c < FV_KERNEL_NCLASS; ++c) {
    if (ms) ms[c] = acc[c];
    if (launches) launches[c] = m->launches[c];
    m->launches[c] = 0;
  }
  return FV_OK;
}

}  // extern "C"

fv_status fv_internal_mesh(fv_mesh_t m, MeshView* out) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (m->stage_pending) {
    set_error("the mesh is between the two RK substeps");
    return FV_ERR_INVALID_ARG;
  }
  m->w_current = false;  // the caller may write U
  m->smax_current = false;
  out->P = m->P;
  out->U = m->buf.U;
  out->stream = m->stream;
  out->device = m->device;
  out->precision = m->desc.precision;
  return FV_OK;
}

void fv_internal_state_written(fv_mesh_t m) {
  m->w_current = false;
  m->smax_current = false;
}

fv_status fv_internal_step(fv_mesh_t m, double dt) { return fv_step(m, dt); }

extern "C" {

fv_status fv_mesh_info(fv_mesh_t m, int dims[3], size_t* state_bytes) {
  fv_status st = check_handle(m);
  if (st != FV_OK) return st;
  if (dims) {
    dims[0] = m->desc.nx;
    dims[1] = m->desc.ny;
    dims[2] = m->desc.nz;
  }
  if (state_bytes) *state_bytes = m->state_doubles * sizeof(double);
  return FV_OK;
}

const char* fv_status_string(fv_status s) {
  switch (s) {
    case FV_OK: return "FV_OK";
    case FV_ERR_INVALID_ARG: return "FV_ERR_INVALID_ARG";
    case FV_ERR_OOM: return "FV_ERR_OOM";
    case FV_ERR_CUDA: return "FV_ERR_CUDA";
    case FV_ERR_NONPHYSICAL: return "FV_ERR_NONPHYSICAL";
    case FV_ERR_TIMEOUT: return "FV_ERR_TIMEOUT";
    case FV_ERR_BAD_HANDLE: return "FV_ERR_BAD_HANDLE";
  }
  return "FV_ERR_UNKNOWN";
}

const char* fv_last_error(void) { return g_last_error; }

}  // extern "C"
