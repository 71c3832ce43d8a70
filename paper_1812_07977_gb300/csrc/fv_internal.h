// fv_internal.h -- host-side interfaces between the C ABI (fv_core.cu) and
// the kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include "fv_device.cuh"

// Device-resident flags and results of one mesh, read back in one copy.
struct DevCounters {
  unsigned long long smax_bits;    // max CFL signal speed (bits of a double >= 0)
  unsigned long long np_step;      // non-physical interior cells seen by the step
  unsigned long long fallback;     // faces that fell back to first order
  unsigned long long np_dt;        // non-physical interior cells seen by the dt pass
};

// Device buffers used by one RK2 substep.
struct StepBuffers {
  double* U;      // FluidCurrent / FluidOld, ghosted, 5 fields
  double* U1;     // first RK stage, ghosted, 5 fields
  double* W;      // primitives of the stage's input state, ghosted, 5 fields
  double* ACC;    // flux-divergence accumulator, dense interior, 5 fields
  DevCounters* ctr;
};

// The step's kernels are compiled twice from one source: without (exact)
// and with (fma) fused multiply-add contraction.  A substep is launch_prim
// on its input state (U for stage 1, U1 for stage 2), then launch_sweep for
// axis 0, 1, 2; the z sweep (axis 2) applies the RK combine of `stage`.
#define FV_DECLARE_STEP_VARIANT(ns)                                                        \
  namespace ns {                                                                           \
  cudaError_t launch_prim(const double* src, const StepBuffers& b, const fvd::Params& P,   \
                          cudaStream_t s);                                                 \
  cudaError_t launch_sweep(int axis, int stage, const StepBuffers& b, const fvd::Params& P, \
                           double dt, cudaStream_t s);                                     \
  }
FV_DECLARE_STEP_VARIANT(fv_fp64_exact)
FV_DECLARE_STEP_VARIANT(fv_fp64_fma)

// fv_step32_kernels.cu: the FP32-bulk substep (one fused kernel; z chunks
// of `kchunk` planes per CTA) and its CFL reduction.
namespace fv_fp32 {
cudaError_t launch_stage(int stage, const StepBuffers& b, const fvd::Params& P, double dt,
                         int kchunk, double vacuum_ratio, int occupancy, cudaStream_t s);
cudaError_t launch_reduce_dt(const double* U, const fvd::Params& P, double vacuum_ratio,
                             DevCounters* ctr, cudaStream_t s);
}

// fv_aux.cu (always built without contraction)
cudaError_t launch_fill_ghosts(double* U, const fvd::Params& P, cudaStream_t s);
cudaError_t launch_reduce_dt(const double* U, const fvd::Params& P, DevCounters* ctr,
                             cudaStream_t s);
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
