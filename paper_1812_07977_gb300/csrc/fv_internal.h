// fv_internal.h -- host-side interfaces between the C ABI (fv_core.cu) and
// the kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include "fv.h"

#include "fv_device.cuh"
#include "fv_device32.cuh"

// Device-resident flags and results of one mesh, read back in one copy.
struct DevCounters {
  unsigned long long smax_bits;    // max CFL signal speed (bits of a double >= 0)
  unsigned long long np_step;      // non-physical interior cells seen by the step
  unsigned long long fallback;     // faces that fell back to first order
  unsigned long long np_dt;        // non-physical interior cells seen by the dt pass
  unsigned long long faces;        // face fluxes evaluated (not reused) by the flux kernels
  unsigned long long smax_next;    // fused paths: CFL maximum of the last stage 2's output
  unsigned long long ff_range;     // float-float path: cells outside its operand range
};

// Adds each lane's count to *ctr once per warp (the lanes present at the call).
__device__ __forceinline__ void warp_count(unsigned long long* ctr, unsigned n) {
  const unsigned mask = __activemask();
  const unsigned sum = __reduce_add_sync(mask, n);
  if ((threadIdx.x & 31u) == (unsigned)(__ffs(mask) - 1) && sum) atomicAdd(ctr, (unsigned long long)sum);
}

// Device buffers used by one RK2 substep.
struct StepBuffers {
  double* U;      // FluidCurrent / FluidOld, ghosted, 5 fields
  double* U1;     // first RK stage, ghosted, 5 fields
  double* W;      // primitives of the stage's input state, ghosted, 5 fields
  double* ACC;    // flux-divergence accumulator, dense interior, 5 fields
  unsigned char* keep;  // per interior cell: substep 1 copied U to U1 unchanged (dense)
  DevCounters* ctr;
};

// The step's kernels are compiled twice from one source: without (exact)
// and with (fma) fused multiply-add contraction.  A substep is launch_prim
// on its input state (U for stage 1, U1 for stage 2), then launch_sweep for
// axis 0, 1, 2; the z sweep (axis 2) applies the RK combine of `stage`.
// `segments`: pieces each grid line of a sweep is cut into (0: chosen from
// the mesh size and `num_sms`, the device's multiprocessor count).
// launch_prim with keep (substep 2): W holds U's primitives and b.keep the
// cells substep 1 left unchanged; only the other cells are converted.
// launch_prim_dt: the CFL maximum of U into ctr->smax_bits and, in the same
// pass, U's primitives into b.W, which a following substep 1 may use in
// place of its launch_prim.
// The fused form (fv_fused64_kernels.cu, the same two arithmetic variants):
// launch_fused runs a whole substep (stage 1: U1 = U + dU(U); stage 2:
// U = (U + U1 + dU(U1))/2 with the CFL maximum of the new U into
// ctr->smax_next) in one kernel over tiles of 32 x 8 columns and z chunks of
// `kchunk` planes; launch_dt takes the CFL maximum of U with the same
// arithmetic into ctr->smax_bits; prepare_fused raises the fused kernels'
// shared-memory limit on the current device (before their first launch).
#define FV_DECLARE_STEP_VARIANT(ns)                                                        \
  namespace ns {                                                                           \
  cudaError_t launch_prim(const double* src, const StepBuffers& b, const fvd::Params& P,   \
                          bool keep, cudaStream_t s);                                      \
  cudaError_t launch_sweep(int axis, int stage, const StepBuffers& b, const fvd::Params& P, \
                           double dt, int segments, int num_sms, cudaStream_t s);          \
  cudaError_t launch_prim_dt(const double* U, const StepBuffers& b, const fvd::Params& P,  \
                             cudaStream_t s);                                              \
  cudaError_t prepare_fused();                                                             \
  cudaError_t launch_fused(int stage, const StepBuffers& b, const fvd::Params& P,          \
                           double dt, int kchunk, cudaStream_t s);                         \
  cudaError_t launch_dt(const double* U, const StepBuffers& b, const fvd::Params& P,       \
                        cudaStream_t s);                                                   \
  }
FV_DECLARE_STEP_VARIANT(fv_fp64_exact)
FV_DECLARE_STEP_VARIANT(fv_fp64_fma)

// fv_fused_ff_kernels.cu: the fused substep with float-float face arithmetic
// (FV_PREC_FP64_FF), its CFL maximum, and its shared-memory set-up; the
// same contracts as the fused FP64 variants above.
namespace fv_fp64_ff {
cudaError_t prepare_fused();
// tiles of tile_x x tile_y columns at ctas_per_sm CTAs per SM: 16 x 16 or
// 32 x 8 at 2 (16 warps per SM, 128 registers) or 1 (8 warps, 255); 32 x 16
// at 1
bool valid_fused_config(int tile_x, int tile_y, int ctas_per_sm);
// plane_skip: at the default tile, a tile whose cells (with the halo) all
// equal those one plane below skips that plane's slope and face passes (the
// same bits)
cudaError_t launch_fused(int stage, const StepBuffers& b, const fvd::Params& P, double dt,
                         int kchunk, int tile_x, int tile_y, int ctas_per_sm, bool plane_skip,
                         cudaStream_t s);
cudaError_t launch_dt(const double* U, const StepBuffers& b, const fvd::Params& P,
                      cudaStream_t s);
}

// One mesh of a batch, as the batched kernels see it.
struct BatchMesh {
  fvd::Params P;
  fvd32::Params32 Q;
  long long offset;              // doubles from the batch's U (and U1) base to this mesh
  double dt;                     // this step's dt, written by the batched CFL kernels
  unsigned long long smax_bits;  // CFL maximum of this step (bits of a double >= 0)
};

// Device-side tables of a batch.  Its meshes fall into size classes by
// their x extent (fv_fp32::batch_class), each with its own launch
// configuration; the work items of class c are items[class_first[c] ..
// class_first[c] + class_count[c]).
constexpr int kBatchClasses = 3;
struct BatchDevice {
  double* U;
  double* U1;
  BatchMesh* meshes;
  int nmesh;
  int4* items;          // fused-kernel work items: mesh, tile x, tile y, z chunk
  int nitems;
  int class_first[kBatchClasses];
  int class_count[kBatchClasses];
  int2* dt_blocks;      // CFL kernel blocks: mesh, chunk of 2048 interior cells
  int ndt_blocks;
  int2* ghost_blocks;   // ghost kernel blocks: mesh, chunk of 256 ring cells
  int nghost_blocks;
  unsigned* next_item;  // two work counters (stage 1, stage 2) per class
  DevCounters* ctr;
  bool all_mc;          // every mesh has limiter parameter 2
};

// fv_step32_kernels.cu: the FP32-bulk substep (one fused kernel; z chunks
// of `kchunk` planes per CTA) and its CFL reduction.
namespace fv_fp32 {
// Raises the shared-memory limit of the fused substep kernels on the current
// device (they take more than the default 48 KB); before their first launch.
cudaError_t prepare_kernels();
// The fused substep (single-mesh and batched) is built for these (tile x,
// tile y, occupancy): occupancy 2 is 16 warps per SM at up to 128 registers,
// 3 (32 x 8 only) 24 warps at 80 registers.
constexpr int kShapes[8][3] = {{32, 4, 2}, {32, 8, 2}, {32, 8, 3}, {32, 16, 2},
                               {16, 8, 2}, {64, 4, 2}, {64, 8, 2}, {128, 4, 2}};
bool valid_config(int tile_x, int tile_y, int occupancy);
// Size class of a mesh of nx cells along x: 0 up to 24, 1 up to 64, 2 above.
inline int batch_class(int nx) { return nx <= 24 ? 0 : nx <= 64 ? 1 : 2; }
cudaError_t launch_stage(int stage, const StepBuffers& b, const fvd::Params& P, double dt,
                         int kchunk, double vacuum_ratio, int occupancy, int tile_x, int tile_y,
                         cudaStream_t s);
cudaError_t launch_reduce_dt(const double* U, const fvd::Params& P, double vacuum_ratio,
                             DevCounters* ctr, cudaStream_t s);
// Batches: per-mesh CFL maxima of the current states (launch_batch_max), dt =
// cfl / max per mesh with the maxima and work counters then cleared
// (launch_batch_dt), the fused substep over all meshes' work items (one
// persistent launch; stage 2 refills the maxima with those of its output),
// and the ghost fill.
constexpr int kBatchDtChunk = 2048;
constexpr int kBatchGhostChunk = 256;
cudaError_t launch_batch_max(const BatchDevice& b, cudaStream_t s);
cudaError_t launch_batch_dt(const BatchDevice& b, double cfl, cudaStream_t s);
// One persistent launch over the work items of size class `cls` (a no-op if
// the class has none).
cudaError_t launch_batch_stage(int stage, const BatchDevice& b, int cls, int kchunk,
                               int occupancy, int tile_x, int tile_y, int num_sms,
                               cudaStream_t s);
cudaError_t launch_batch_ghosts(int stage, const BatchDevice& b, cudaStream_t s);
fvd32::Params32 make_params32(const fvd::Params& P, double vacuum_ratio);
}

// fv_aux.cu (always built without contraction)
// Multiprocessors of the current device (queried once per device and cached;
// 1 if the query fails), for sizing grid-stride launches.
int fv_sm_count();
cudaError_t launch_fill_ghosts(double* U, const fvd::Params& P, cudaStream_t s);
cudaError_t launch_scatter_interior(const double* dense, double* U, const fvd::Params& P,
                                    cudaStream_t s);
cudaError_t launch_gather_interior(const double* U, double* dense, const fvd::Params& P,
                                   cudaStream_t s);
// Per-field pairwise sums over the interior; `work` holds at least
// sums_work_doubles(P) doubles; the 5 results land in out5 (device).
size_t sums_work_doubles(const fvd::Params& P);
cudaError_t launch_pairwise_sums(const double* U, const fvd::Params& P, double* work,
                                 double* out5, cudaStream_t s);

// fv_core.cu: sets the detail string that fv_last_error() returns on the
// calling thread (for entry points defined outside fv_core.cu).
void fv_internal_set_error(const char* msg);

// fv_core.cu: mesh description checks and derived parameters, shared with
// the batch entry points.
fv_status fv_internal_validate_desc(const fv_mesh_desc* d);
fvd::Params fv_internal_params(const fv_mesh_desc* d);

// fv_core.cu: a mesh's internals for the learned correction (fv_learned.cu).
// fv_internal_mesh returns FV_OK and fills the fields for a live mesh at a
// step boundary; U points to its current (ghosted, FP64) state.
struct MeshView {
  fvd::Params P;
  double* U;
  cudaStream_t stream;
  int device;
  int precision;
};
fv_status fv_internal_mesh(fv_mesh_t m, MeshView* out);
// The caller wrote the mesh's U through a view: drops what the mesh derived
// from the state (its primitives and CFL maximum for the next step).
void fv_internal_state_written(fv_mesh_t m);
// Run one full step of the mesh (as fv_step) / refill its ghosts.
fv_status fv_internal_step(fv_mesh_t m, double dt);
