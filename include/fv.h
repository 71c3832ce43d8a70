/*
 * fv.h -- C ABI of the GB300 finite-volume Euler step.
 *
 * One explicit second-order Runge-Kutta step of the 3D ideal-gas Euler
 * equations on a uniform Cartesian mesh with two ghost layers, as in the
 * RiemannProblem of Budiardja & Cardall, "Targeting GPUs with OpenMP
 * Directives on Summit" (Sec. 3, Algorithm 1 "Fluid Evolution" and
 * Algorithm 2 "Fluid Evolution with Accelerator").  Every stage runs in this
 * library's own CUDA kernels for sm_103a on one GPU; there is no CPU path.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * State layout (the paper's StorageForm column remapped to rank 3 with two
 * ghost layers, Sec. 3): five conserved fields q = 0..4 = (rho, rho*vx,
 * rho*vy, rho*vz, E), each stored contiguously (structure of arrays).  The
 * caller exchanges INTERIOR states only: a dense array of 5*nz*ny*nx doubles
 * indexed [q][k][j][i] with i (x) fastest.  The ghost cells are owned by the
 * library.
 *
 * Ownership: the library allocates and frees all device memory of a mesh.
 * The caller owns every buffer it passes (host or device pointer) and keeps
 * it valid for the duration of the call.
 *
 * Streams: all work of a mesh is enqueued on the CUDA stream given at
 * creation (NULL = the legacy default stream), on the device that was
 * current at creation.  Calls marked "asynchronous" return once the work is
 * enqueued; calls marked "synchronising" wait for the stream.
 *
 * Errors: every call returns an fv_status.  FV_OK on success; on failure a
 * human-readable detail is available from fv_last_error() on the same host
 * thread.  Device-side conditions found while computing (a cell average with
 * rho <= 0, p <= 0 or NaN) are latched on the device and reported as
 * FV_ERR_NONPHYSICAL by the next synchronising call.  A handle is unusable
 * after fv_destroy_mesh; passing it again gives FV_ERR_BAD_HANDLE.
 * Calls on one mesh must not be made concurrently from several host threads.
 */
#ifndef FV_H
#define FV_H

#include <stddef.h>

#if defined(__GNUC__)
#define FV_API __attribute__((visibility("default")))
#else
#define FV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fv_mesh_s* fv_mesh_t;

typedef enum {
  FV_OK = 0,
  FV_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum value or call order */
  FV_ERR_OOM = 2,           /* device or pinned host allocation failed */
  FV_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
  FV_ERR_NONPHYSICAL = 4,   /* a cell average had rho <= 0, p <= 0 or NaN */
  FV_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (tensor-core convolutions) */
  FV_ERR_BAD_HANDLE = 6     /* NULL, destroyed or foreign mesh handle */
} fv_status;

typedef enum { FV_BC_OUTFLOW = 0, FV_BC_PERIODIC = 1 } fv_bc;

/* Arithmetic of the step.
 *  FV_PREC_FP64      FP64, every operation rounded separately in the order
 *                    of the method's definition (no fused multiply-add):
 *                    bitwise reproducible against a plain IEEE FP64 code.
 *  FV_PREC_FP32_BULK FP64 state, FP32 bulk arithmetic: reconstruction, wave
 *                    speeds, HLL fluxes and the flux divergence in FP32 (one
 *                    fused kernel per substep); the RK combine adds the FP32
 *                    update to the FP64 state in FP64; the pressure of cells
 *                    whose kinetic energy exceeds 99% of E is recovered in
 *                    FP64; the CFL time step is FP64 (FP32 speeds serve only
 *                    as upper bounds that skip cells which cannot raise the
 *                    maximum); conservation sums as FV_PREC_FP64.
 *  FV_PREC_FP64_FMA  FP64 with fused multiply-add contraction, and each
 *                    divide and square root (sound speeds, HLL weights, 1/rho)
 *                    as an FP32 seed refined by two Newton-Raphson steps in
 *                    FP64: the same method, a few ulp per operation away from
 *                    FV_PREC_FP64 (held to 1e-12 relative of each field).
 *  FV_PREC_FP64_FF   FP64 state, primitives (Newton forms), RK combine and
 *                    CFL time step as FV_PREC_FP64_FMA; the work per face --
 *                    differences, limited slopes, face states, sound speeds,
 *                    HLL fluxes -- and the flux divergence in float-float
 *                    arithmetic (pairs of FP32 numbers, 48-bit significand)
 *                    on the FP32 pipe, in one fused kernel per substep; held
 *                    to 1e-12 relative of each field against FV_PREC_FP64.
 *                    Its operand range is density and pressure of magnitude
 *                    2^-30 .. 2^30 and velocities below 2^20: a step of a
 *                    state with a physical cell outside it is reported
 *                    (FV_ERR_INVALID_ARG at the next synchronising call) and
 *                    leaves the state unspecified.
 *  The values 0 and 1 are those of the boundary's original two-value enum;
 *  the later variants take new values.  The FP64 forms evaluate a face's
 *  flux once and reuse it, bit for bit, for the next face of a grid line
 *  when the cells around both are equal (see fv_get_face_counts).
 */
typedef enum {
  FV_PREC_FP64 = 0,
  FV_PREC_FP32_BULK = 1,
  FV_PREC_FP64_FMA = 2,
  FV_PREC_FP64_FF = 3
} fv_precision;

typedef struct {
  int nx, ny, nz;       /* interior cells per axis, each >= 1 */
  double lx, ly, lz;    /* domain extents (> 0); origin at 0; dx = lx / nx */
  double gamma;         /* ideal-gas ratio of specific heats, > 1 */
  double theta;         /* limiter: 0 first order, 1 minmod, 2 monotonised
                           central; any value in [0, 2] */
  int bc[3];            /* fv_bc per axis x, y, z */
  int precision;        /* fv_precision */
} fv_mesh_desc;

/* Allocate a mesh and its device state (Sec. 2.1: StorageForm's
 * AllocateDevice; the persistent device copy of FluidCurrent and the work
 * storage initialised by Algorithm 2).  `cuda_stream` is a cudaStream_t (NULL =
 * default stream).  The state is zero until fv_set_state.  Synchronous.
 * Errors: INVALID_ARG (desc out of range, out == NULL), OOM, CUDA. */
FV_API fv_status fv_create_mesh(const fv_mesh_desc* desc, void* cuda_stream,
                         fv_mesh_t* out);

/* Free all memory of the mesh after its stream has drained.  NULL is
 * accepted and ignored.  Errors: BAD_HANDLE. */
FV_API fv_status fv_destroy_mesh(fv_mesh_t m);

/* Copy an interior conserved state in and fill the ghost layers (Sec. 2.1
 * UpdateDevice, then the initial GhostExchange of Algorithm 1).  `U` holds
 * 5*nz*ny*nx doubles [q][k][j][i]; on_device != 0 means a device pointer on
 * the mesh's device, else a host pointer (pinned host memory is fastest).
 * Clears the latched non-physical counters and any pending RK stage.
 * Synchronising for host pointers, asynchronous for device pointers. */
FV_API fv_status fv_set_state(fv_mesh_t m, const double* U, int on_device);

/* Copy the current interior state out (Sec. 2.1 UpdateHost); same layout
 * as fv_set_state.  Between fv_substep(1) and fv_substep(2) the current
 * state is the first RK stage.  Synchronising.  Errors: NONPHYSICAL if a
 * non-physical cell was latched since the last fv_set_state. */
FV_API fv_status fv_get_state(fv_mesh_t m, double* U, int on_device);

/* Copy the full ghosted state out: 5 * (nz+4)*(ny+4)*(nx+4) doubles
 * [q][k+2][j+2][i+2].  Synchronising. */
FV_API fv_status fv_get_ghosted_state(fv_mesh_t m, double* U, int on_device);

/* ComputeTimeStep (Algorithm 1): *dt_out = cfl / max over interior
 * cells of sum_d (|v_d| + c) / dx_d with c = sqrt(gamma p / rho), in the
 * mesh's arithmetic (FP64: IEEE operations in the method's order, bit for
 * bit; FP64_FMA: contracted, Newton-Raphson divide and square root, within
 * a few ulps; FP32_BULK: per-cell speeds in FP32).  The maximum is exact
 * (order-free).  Only valid at a step boundary.  On the FP64 paths the same
 * pass also converts the state to primitives, which the next fv_step /
 * fv_substep(1) uses instead of converting again if the state has not
 * changed since (fv_set_state and fv_fill_ghosts count as changes); a
 * non-physical cell found there counts once, for the time step.
 * On the FP32_BULK path the second substep of fv_step takes the maximum of
 * the state it writes (and counts its non-physical cells), and
 * fv_reduce_dt uses that maximum while the state has not changed since.
 * Synchronising (one small device-to-host read).  Errors: INVALID_ARG
 * (cfl <= 0, dt_out NULL, stage pending), NONPHYSICAL. */
FV_API fv_status fv_reduce_dt(fv_mesh_t m, double cfl, double* dt_out);

/* One RK2 step (the loop body of Algorithm 1): FluidOld = FluidCurrent;
 * substep 1 FluidCurrent = FluidOld + dt L(FluidOld); GhostExchange;
 * substep 2 FluidCurrent = 0.5 (FluidOld + FluidCurrent + dt L(FluidCurrent));
 * GhostExchange.  L is the flux divergence of primitive-variable
 * slope-limited reconstruction with HLL face fluxes.  The caller picks dt
 * (normally from fv_reduce_dt, clamped to the end time).  Asynchronous.
 * Errors: INVALID_ARG (dt not finite or < 0, stage pending), CUDA. */
FV_API fv_status fv_step(fv_mesh_t m, double dt);

/* Half of fv_step: stage 1 (requires a step boundary) or stage 2 (requires
 * stage 1 done).  fv_substep(m,1,dt); fv_substep(m,2,dt) == fv_step(m,dt).
 * Asynchronous. */
FV_API fv_status fv_substep(fv_mesh_t m, int stage, double dt);

/* GhostExchange alone (Algorithm 1) on the current state:
 * each ghost cell takes the value of its source cell, axis by axis x, y, z
 * (outflow: nearest interior cell; periodic: index modulo n).  The step
 * already does this; exposed for tests and custom loops.  Asynchronous. */
FV_API fv_status fv_fill_ghosts(fv_mesh_t m);

/* Per-field sum over interior cells times the cell volume (dx*dy)*dz, by a
 * fixed pairwise tree (values in (k, j, i) order, zero-padded to a power of
 * two, neighbours added level by level): bitwise reproducible.
 * out[5].  Synchronising. */
FV_API fv_status fv_conserved_sums(fv_mesh_t m, double out[5]);

/* Counters latched since the last fv_set_state: interior cells found
 * non-physical, and faces whose reconstructed state had rho <= 0 or p <= 0
 * and fell back to first order.  Either pointer may be NULL.
 * Synchronising. */
FV_API fv_status fv_get_counters(fv_mesh_t m, long long* nonphysical_cells,
                          long long* fallback_faces);

/* Face fluxes since the last fv_set_state: `evaluated` = fluxes the
 * kernels computed, `defined` = fluxes the method defines (every face of the
 * mesh, once per substep).  Along a grid line, a face whose five-cell
 * neighbourhood is a run of cells equal bit for bit has the inputs, and so
 * the flux, of the face before it; the FP64 sweeps then reuse that flux
 * (same bits as evaluating it).  They also evaluate the first face of every
 * line segment after the first twice (FV_TUNE_SWEEP_SEGMENTS), so for states
 * without equal neighbours each step evaluates the defined faces plus, for
 * each axis, (segments - 1) x (lines along it) faces per substep.  The fused
 * FP32-bulk kernel reuses z fluxes the same way and x / y fluxes whose four
 * cells equal those one plane below; it evaluates the faces on tile and
 * z-chunk edges in both neighbouring tiles, so for states without equal
 * neighbours evaluated exceeds defined.  Either pointer may be NULL.
 * Synchronising. */
FV_API fv_status fv_get_face_counts(fv_mesh_t m, long long* evaluated, long long* defined);

/* Kernel classes of the profiling hooks below. */
typedef enum {
  FV_KERNEL_PRIM = 0,     /* conserved -> primitive (FP64 paths) */
  FV_KERNEL_SWEEP_X = 1,  /* differences, reconstruction, HLL fluxes, update: x */
  FV_KERNEL_SWEEP_Y = 2,  /* the same along y */
  FV_KERNEL_SWEEP_Z = 3,  /* the same along z, with the RK combine */
  FV_KERNEL_FUSED = 4,    /* the whole substep in one kernel (fused paths) */
  FV_KERNEL_GHOST = 5,    /* ghost fill */
  FV_KERNEL_DT = 6,       /* CFL time-step reduction */
  FV_KERNEL_OTHER = 7,    /* state copies and conservation sums */
  FV_KERNEL_NCLASS = 8
} fv_kernel_class;

/* Per-kernel timing on (on != 0) or off.  While on, every kernel launch of
 * the mesh is bracketed by two CUDA events recorded on the mesh's stream;
 * this adds no synchronisation.  Not part of the paper: measurement support
 * (the role of its TimerForm instrumentation, Sec. 4). */
FV_API fv_status fv_profile_enable(fv_mesh_t m, int on);

/* Read and reset the profile: ms[c] = device milliseconds spent in kernels
 * of class c since the last read (timed launches only), launches[c] = number
 * of kernel launches of class c (always counted).  Arrays of
 * FV_KERNEL_NCLASS entries; either may be NULL.  Synchronising. */
FV_API fv_status fv_profile_read(fv_mesh_t m, double* ms, long long* launches);

/* ------------------------------------------------------------------------
 * Batches: many independent meshes of uneven sizes advanced together.
 * Not in the paper (whose ranks each own one subdomain): the on-device
 * analogue of many independent RiemannProblem runs.  Every mesh of a batch
 * uses the FP32-bulk arithmetic (FV_PREC_FP32_BULK; the precision field of
 * the descriptions is ignored) and its own CFL time step.  The meshes fall
 * into three size classes by their x extent (class 0: nx <= 24, class 1:
 * nx <= 64, class 2: larger), each with its own launch configuration (tile
 * shape, occupancy, z chunk).  One step is: per-mesh dt = cfl / max signal
 * speed (on the device, FP64 speeds and division), then the two RK
 * substeps, each one persistent launch per size class over the work items
 * (mesh, tile, z chunk) of its meshes, each substep followed by the ghost
 * fill of all meshes.
 * ------------------------------------------------------------------------ */
typedef struct fv_batch_s* fv_batch_t;

/* Allocate a batch of `nmesh` meshes (each description validated as for
 * fv_create_mesh).  `cuda_stream` NULL: the batch creates its own
 * non-blocking stream (needed for graph capture).  Synchronous.
 * Errors: INVALID_ARG, OOM, CUDA. */
FV_API fv_status fv_batch_create(const fv_mesh_desc* descs, int nmesh, void* cuda_stream,
                                 fv_batch_t* out);
FV_API fv_status fv_batch_destroy(fv_batch_t b);

/* Interior state of mesh `mesh` in or out, layout as fv_set_state. */
FV_API fv_status fv_batch_set_state(fv_batch_t b, int mesh, const double* U, int on_device);
FV_API fv_status fv_batch_get_state(fv_batch_t b, int mesh, double* U, int on_device);

/* One step of every mesh with its own dt = cfl / (its maximum signal
 * speed).  The second substep takes each mesh's maximum of the state it
 * writes, so the next step starts from it; a separate pass over the states
 * runs only when they changed otherwise (fv_batch_set_state, the
 * autotuner).  use_graph != 0: the step (per-mesh dt, both substeps and
 * ghost fills) is captured once into a CUDA graph and replayed (re-captured
 * when cfl or the tuning changes).  Asynchronous. */
FV_API fv_status fv_batch_step(fv_batch_t b, double cfl, int use_graph);

/* The dt each mesh used in the last step (nmesh doubles).  Synchronising. */
FV_API fv_status fv_batch_get_dt(fv_batch_t b, double* dt);

/* Launch configuration of every size class at once: z planes per work item
 * (kchunk in [1, 4096]), the work item's tile of 32 x tile_y columns (tile_y
 * 4, 8 or 16: CTAs of 128, 256 or 512 threads) and occupancy 2 (16 warps per
 * SM, up to 128 registers) or, for tile_y 8 only, 3 (80 registers).  Every
 * configuration gives the same bits.  Errors: INVALID_ARG. */
FV_API fv_status fv_batch_set_tuning(fv_batch_t b, int kchunk, int occupancy, int tile_y);

/* Launch configuration of one size class (cls 0, 1 or 2): tiles of tile_x x
 * tile_y columns with occupancy, one of (32, 4, 2), (32, 8, 2), (32, 8, 3),
 * (32, 16, 2), (16, 8, 2), (64, 4, 2), (64, 8, 2), (128, 4, 2) (occupancy 2:
 * 16 warps per SM; 3: 24 warps), and z chunks of kchunk planes.  The same
 * bits for every configuration.  Errors: INVALID_ARG. */
FV_API fv_status fv_batch_set_class_tuning(fv_batch_t b, int cls, int tile_x, int tile_y,
                                           int occupancy, int kchunk);
/* The configuration of size class cls and how many meshes it holds (any
 * output pointer may be NULL). */
FV_API fv_status fv_batch_get_class_tuning(fv_batch_t b, int cls, int* tile_x, int* tile_y,
                                           int* occupancy, int* kchunk, int* meshes);

/* Autotuner: for each size class in turn (most cells first, the others at
 * their best so far) times three steps of the whole batch for every built
 * tile shape no wider than twice the class's widest mesh (32-wide shapes
 * always) and every z chunk in {8, 16, 32, 64}, on the batch's current
 * state, and keeps the fastest per class (fv_batch_get_class_tuning reads
 * them).  Reports the configuration of the class with the most cells and
 * the final step time (any output pointer may be NULL).  The state and
 * counters are restored afterwards (a snapshot buffer of one state is
 * allocated on first use).  Synchronising. */
FV_API fv_status fv_batch_autotune(fv_batch_t b, double cfl, int* kchunk, int* occupancy,
                                   int* tile_y, double* ms_per_step);

FV_API fv_status fv_batch_get_counters(fv_batch_t b, long long* nonphysical_cells,
                                       long long* fallback_faces);
FV_API fv_status fv_batch_info(fv_batch_t b, int* nmesh, long long* total_cells,
                               long long* work_items);

/* ------------------------------------------------------------------------
 * Learned flux correction (not in the paper: an extension that lets a
 * coarse mesh approach fine-mesh solutions).  A network of three 3x3x3
 * convolutions (5 -> 32 -> 32 -> 5 channels, tanh after the first two)
 * maps the normalised primitives of each cell, x = (W - in_mean)/in_scale,
 * to o; phi = out_scale * o.  The flux through every face is corrected by
 * phi(right cell) - phi(left cell), so a cell's state changes by
 *   dU = -sum_d dt/dx_d (phi(i+e_d) - 2 phi(i) + phi(i-e_d)),
 * which is conservative and zero for uniform states.  Weights and
 * activations are BF16, accumulation FP32: the forward convolutions, the
 * input-gradient (adjoint) convolutions and the weight gradients of
 * training run on the tensor cores (tcgen05 MMAs, accumulators in tensor
 * memory); the backward pass feeds them its FP32 gradients rounded to BF16
 * (bias gradients are summed in FP32).  A convolution whose wait
 * for its MMAs runs out records it; the next synchronising net call
 * (fv_net_forward with o_out, fv_net_train_step) returns FV_ERR_TIMEOUT.
 * Periodic meshes only.
 * Parameters (FP32, fv_net_param_count() of them) in the order
 *   w1 [32][5][27], b1 [32], w2 [32][32][27], b2 [32], w3 [5][32][27], b3 [5]
 * with kernel index o = 9 dz + 3 dy + dx for offsets (dz, dy, dx) - 1.
 * ------------------------------------------------------------------------ */
typedef struct fv_net_s* fv_net_t;

FV_API size_t fv_net_param_count(void);
/* A network on the current device, parameters zero, scales 1. */
FV_API fv_status fv_net_create(fv_net_t* out);
FV_API fv_status fv_net_destroy(fv_net_t n);
/* Host arrays of fv_net_param_count() floats; set resets the Adam state.
 * get: either pointer may be NULL; grads are those of the last train step. */
FV_API fv_status fv_net_set_params(fv_net_t n, const float* params);
FV_API fv_status fv_net_get_params(fv_net_t n, float* params, float* grads);
/* Input normalisation, output scale and the residual scale of the loss. */
FV_API fv_status fv_net_set_scales(fv_net_t n, const double in_mean[5], const double in_scale[5],
                                   const double out_scale[5], const double res_scale[5]);
/* o (device pointer, 5*nz*ny*nx floats [q][k][j][i]) for the mesh's
 * current state; o_out may be NULL.  Synchronising when o_out is given. */
FV_API fv_status fv_net_forward(fv_net_t n, fv_mesh_t m, float* o_out);
/* One training step on the mesh's current state: loss
 *   L = mean over cells and fields of ((dU - r) / res_scale)^2
 * for the residual r (device pointer, 5*nz*ny*nx FP64 values: the fine
 * solution averaged to the mesh minus the mesh's own RK2 step over dt),
 * gradients by the backward kernels, then Adam (beta 0.9, 0.999, eps 1e-8)
 * with learning rate lr (lr = 0: gradients only).  *loss_out = L before the
 * update; synchronising.  With loss_out NULL the step is asynchronous (no
 * host wait, so a loop of steps keeps the GPU busy): L is added to a
 * device-side sum that fv_net_take_loss returns, and a convolution's wait
 * that ran out is reported by the next synchronising net call. */
FV_API fv_status fv_net_train_step(fv_net_t n, fv_mesh_t m, const double* residual, double dt,
                                   double lr, double* loss_out);
/* The sum of the losses of the asynchronous train steps since the last
 * call, and their number (either pointer may be NULL); clears both.
 * Synchronising (waits for the net's last stream); FV_ERR_TIMEOUT if one of
 * those steps' convolutions ran out of its wait limit. */
FV_API fv_status fv_net_take_loss(fv_net_t n, double* loss_sum, long long* steps);
/* One corrected step: phi from the current state, fv_step(m, dt), then
 * U += dU(phi) on the interior and a ghost fill.  Asynchronous. */
FV_API fv_status fv_step_learned(fv_mesh_t m, fv_net_t n, double dt);

/* The network's intermediate values from its last forward pass
 * (fv_net_forward, fv_net_train_step, fv_step_learned) or, for the
 * gradients, its last training step, for inspection and testing.  Cells are
 * numbered c = (k*ny + j)*nx + i over the mesh the pass ran on.
 *  FV_NET_BUF_FEATURES  x = (W - in_mean)/in_scale: BF16 [c][8] (5 channels,
 *                       3 zero pads)
 *  FV_NET_BUF_H1, _H2   tanh outputs of layers 1 and 2: BF16 [c][32]
 *  FV_NET_BUF_OUT       network output o (phi = out_scale o): FP32 [5][c]
 *  FV_NET_BUF_GRAD_OUT  dL/do: FP32 [5][c]
 *  FV_NET_BUF_GRAD_A2, _A1  dL/d(pre-activation) of layers 2 and 1 (after
 *                       the tanh backward): FP32 [c][32]
 * `dst` is a device pointer on the network's device with room for exactly
 * `bytes` bytes, which must equal the buffer's size.  Synchronising.
 * Errors: INVALID_ARG (unknown buffer, size mismatch, NULL dst, no pass has
 * produced it yet), CUDA. */
typedef enum {
  FV_NET_BUF_FEATURES = 0,
  FV_NET_BUF_H1 = 1,
  FV_NET_BUF_H2 = 2,
  FV_NET_BUF_OUT = 3,
  FV_NET_BUF_GRAD_OUT = 4,
  FV_NET_BUF_GRAD_A2 = 5,
  FV_NET_BUF_GRAD_A1 = 6
} fv_net_buffer;
FV_API fv_status fv_net_get_buffer(fv_net_t n, int which, void* dst, size_t bytes);

/* Conservation sums of a caller-held state, allocating nothing.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- a host code whose device memory belongs
 * to its own allocator under a fixed budget, or a time loop that must not
 * pay cudaMalloc's implicit device-wide synchronisation.  It computes what
 * fv_conserved_sums computes (the same pairwise tree, identical bits) for a
 * state the caller already holds, without a mesh.
 *
 * U: device pointer (current device) to the dense interior state, 5*nz*ny*nx
 * doubles [q][k][j][i]; extents lx, ly, lz as in fv_mesh_desc; out: 5 host
 * doubles.  Work runs on `cuda_stream` (NULL = default stream) and the call
 * synchronises that stream before returning.
 *
 * Scratch: partial sums live in one file-scope device array of 41,008
 * doubles (about 320 KiB) that every GPU loading this library holds until
 * the process exits; nothing is allocated or freed per call.  Limit:
 * nx*ny*nz <= 2^24 (16,777,216 cells, e.g. 256^3); larger states are
 * rejected with FV_ERR_INVALID_ARG.  Every call fully overwrites the
 * partials it reads, so nothing needs clearing between calls, but all calls
 * share the one array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.  The first
 * call on each device looks up the array's device address (with that device
 * current) and caches it; make that first call before any stream capture.
 * The cached address belongs to the device's context: after a
 * cudaDeviceReset of that device it is stale, so do not call this entry
 * point again in that process after such a reset.
 * Errors: INVALID_ARG (NULL pointer, size out of range), CUDA (also when a
 * CUDA error from an earlier, unrelated call is still pending: it is
 * reported, not cleared, and nothing is launched). */
FV_API fv_status fv_conserved_sums_noalloc(const double* U, int nx, int ny, int nz,
                                           double lx, double ly, double lz,
                                           void* cuda_stream, double out[5]);

/* Tuning knobs (not part of the paper).
 *  FV_TUNE_KCHUNK        z planes per CTA of the fused kernels (FP32-bulk
 *                        and FP64; integer >= 1; default 32, or nz when
 *                        nz < 64).  FP64_FF meshes by default pick it per
 *                        launch shape: the chunk (>= 16 planes, or nz) that
 *                        minimises rounds of resident CTAs x (chunk + 4)
 *                        (37 at 256^3), or one chunk of nz planes after an
 *                        fv_reduce_dt that finds under 15% of the faces
 *                        defined since the previous one evaluated; setting
 *                        the key fixes it
 *  FV_TUNE_VACUUM_RATIO  FP32-bulk: recover the pressure in FP64 where the
 *                        kinetic energy exceeds this fraction of E (default
 *                        0.99; a value > 1 turns the recovery off)
 *  FV_TUNE_OCCUPANCY     occupancy the fused FP32-bulk kernel is built for:
 *                        2 (16 warps per SM, up to 128 registers, default)
 *                        or 3 (24 warps, 80 registers; 32 x 8 tiles only);
 *                        for FP64_FF meshes the CTAs per SM of its fused
 *                        kernel: 2 (16 warps, 128 registers, default) or 1
 *                        (8 warps, up to 255 registers); the same bits
 *  FV_TUNE_TILE_Y        tile height of the fused FP32-bulk kernel: 4, 8
 *                        (default) or 16 (CTAs of TX x TY threads, one per
 *                        column; 4 and 16 at width 32 only); the same bits
 *  FV_TUNE_TILE_X        tile width of the fused FP32-bulk kernel: 16
 *                        (default), 32, 64 or 128.  (tile x, tile y,
 *                        occupancy) must be one of (32, 4|8|16, 2),
 *                        (32, 8, 3), (16, 8, 2), (64, 4|8, 2), (128, 4, 2)
 *                        after each change, so change them in an order that
 *                        passes through built shapes; the same bits.
 *                        FP64_FF meshes: (tile x, tile y, CTAs per SM) one
 *                        of (16, 16, 2) (the default), (16, 16, 1),
 *                        (32, 8, 1 | 2), (32, 16, 1) after each change (to
 *                        32 x 8: occupancy 1, tile_x 32, tile_y 8, then
 *                        occupancy 2 if wanted); the same bits
 *  FV_TUNE_SWEEP_SEGMENTS  FP64 sweeps: pieces each grid line of a sweep is
 *                        cut into, to run more, shorter work items (integer
 *                        in [0, 4096], capped at the line's length; 0, the
 *                        default, picks by mesh size).  The results are the
 *                        same bits for every value; each extra piece
 *                        evaluates one face flux twice, which
 *                        fv_get_face_counts counts.
 *  FV_TUNE_FP64_FUSED    FP64 and FP64-FMA builds: 0 (default) runs the
 *                        per-axis passes (primitives, then x, y and z line
 *                        sweeps); 1 runs each substep as one fused kernel
 *                        over tiles of 32 x 8 columns and z chunks of
 *                        FV_TUNE_KCHUNK planes, with the next step's CFL
 *                        maximum taken by stage 2 (fewer bytes, slightly more
 *                        FP64 instructions per zone-update: on this GPU the
 *                        FP64 pipe decides, and the sweeps are faster).
 *                        Both give the same bits.  Not between the two
 *                        substeps.  FP64_FF always runs fused.
 *  FV_TUNE_PLANE_SKIP    FP64_FF's fused kernel at its default tile (16 x 16
 *                        at 2 CTAs per SM): 1 (default) lets a tile skip
 *                        the x / y slope and face passes of a plane (and
 *                        their barriers) when every cell of the tile and its
 *                        two-cell halo equals, bit for bit, the cell one
 *                        plane below: each of those slopes and fluxes would
 *                        keep its previous value, and the float-float
 *                        update's zero-divergence test carries over.  After
 *                        an fv_reduce_dt that finds 90% or more of the faces
 *                        defined since the previous one evaluated (no plane
 *                        repeats), the next steps run the kernel built
 *                        without the skip.  0 always runs that kernel, as
 *                        the other tiles do.  The same bits and face counts
 *                        either way.  (FP32-bulk meshes ignore the key:
 *                        their kernel is built without the skip, which
 *                        measured slower there.)
 * Errors: INVALID_ARG for an unknown key or a value out of range. */
typedef enum {
  FV_TUNE_KCHUNK = 0,
  FV_TUNE_VACUUM_RATIO = 1,
  FV_TUNE_OCCUPANCY = 2,
  FV_TUNE_SWEEP_SEGMENTS = 3,
  FV_TUNE_TILE_Y = 4,
  FV_TUNE_FP64_FUSED = 5,
  FV_TUNE_TILE_X = 6,
  FV_TUNE_PLANE_SKIP = 7
} fv_tuning_key;
FV_API fv_status fv_set_tuning(fv_mesh_t m, int key, double value);

/* Mesh facts: interior sizes and the byte size of one device state. */
FV_API fv_status fv_mesh_info(fv_mesh_t m, int dims[3], size_t* state_bytes);

FV_API const char* fv_status_string(fv_status s);

/* Detail of the last failed call on this host thread ("" if none). */
FV_API const char* fv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
