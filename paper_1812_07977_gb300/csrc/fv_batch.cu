// fv_batch.cu -- the C ABI of mesh batches (include/fv.h, "Batches"):
// many independent meshes of uneven sizes advanced together by the
// FP32-bulk step, one persistent launch per RK substep, the whole step
// optionally replayed from a CUDA graph, and an autotuner for the launch
// configuration.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_set>
#include <vector>

#include "fv.h"
#include "fv_internal.h"

namespace {

std::mutex g_batch_mutex;
std::unordered_set<const void*> g_batches;

fv_status fail(fv_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fv_internal_set_error(buf);
  return st;
}

fv_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

struct fv_batch_s {
  int nmesh = 0;
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<fv_mesh_desc> desc;
  std::vector<BatchMesh> host_meshes;
  long long total_cells = 0;
  size_t state_doubles = 0;          // all meshes, ghosted
  size_t max_dense = 0;              // largest mesh, dense interior doubles
  BatchDevice dev{};
  double* staging = nullptr;         // dense interior staging for host copies
  double* backup = nullptr;          // state snapshot used by the autotuner
  DevCounters* host_ctr = nullptr;
  // launch configuration per size class (fv_fp32::batch_class)
  struct Tuning {
    int tile_x = 32, tile_y = 8, occupancy = 2, kchunk = 32;
    bool operator==(const Tuning& o) const {
      return tile_x == o.tile_x && tile_y == o.tile_y && occupancy == o.occupancy &&
             kchunk == o.kchunk;
    }
  };
  Tuning tune[kBatchClasses];
  int class_meshes[kBatchClasses] = {0, 0, 0};
  long long class_cells[kBatchClasses] = {0, 0, 0};
  bool smax_current = false;         // meshes[].smax_bits hold the current states' maxima
  // CUDA graph of one whole step and the configuration it was captured with
  cudaGraphExec_t graph = nullptr;
  double graph_cfl = -1.0;
  Tuning graph_tune[kBatchClasses];
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

fv_status check(fv_batch_t b) {
  if (!b) return fail(FV_ERR_BAD_HANDLE, "NULL batch handle");
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  if (!g_batches.count(b)) return fail(FV_ERR_BAD_HANDLE, "batch handle %p is not live", (void*)b);
  return FV_OK;
}

void free_batch(fv_batch_s* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->dev.U);
  cudaFree(b->dev.U1);
  cudaFree(b->dev.meshes);
  cudaFree(b->dev.items);
  cudaFree(b->dev.dt_blocks);
  cudaFree(b->dev.ghost_blocks);
  cudaFree(b->dev.next_item);
  cudaFree(b->dev.ctr);
  cudaFree(b->staging);
  cudaFree(b->backup);
  cudaFreeHost(b->host_ctr);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Fused-kernel work items: for each size class, every (mesh, tile x, tile y,
// z chunk) of its meshes in the class's tile shape and z chunk, largest
// meshes first so the tail of each persistent launch is short.
fv_status build_items(fv_batch_t b) {
  if (b->graph) {  // the captured step refers to the item table being replaced
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  std::vector<int> order(b->nmesh);
  for (int m = 0; m < b->nmesh; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    const fvd::Params &A = b->host_meshes[a].P, &C = b->host_meshes[c].P;
    return (long long)A.nx * A.ny * A.nz > (long long)C.nx * C.ny * C.nz;
  });
  std::vector<int4> items;
  for (int cls = 0; cls < kBatchClasses; ++cls) {
    const fv_batch_s::Tuning& t = b->tune[cls];
    b->dev.class_first[cls] = (int)items.size();
    for (int m : order) {
      const fvd::Params& P = b->host_meshes[m].P;
      if (fv_fp32::batch_class(P.nx) != cls) continue;
      const int tx = (P.nx + t.tile_x - 1) / t.tile_x;
      const int ty = (P.ny + t.tile_y - 1) / t.tile_y;
      const int tz = (P.nz + t.kchunk - 1) / t.kchunk;
      for (int z = 0; z < tz; ++z)
        for (int y = 0; y < ty; ++y)
          for (int x = 0; x < tx; ++x) items.push_back(make_int4(m, x, y, z));
    }
    b->dev.class_count[cls] = (int)items.size() - b->dev.class_first[cls];
  }
  cudaFree(b->dev.items);
  b->dev.items = nullptr;
  cudaError_t e = cudaMalloc(&b->dev.items, items.size() * sizeof(int4));
  if (e != cudaSuccess) return cuda_fail(e, "allocating work items");
  e = cudaMemcpy(b->dev.items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "uploading work items");
  b->dev.nitems = (int)items.size();
  return FV_OK;
}

// One step from dt on: what the step graph holds.  The CFL maxima of the
// states it starts from are in meshes[].smax_bits (the previous step's stage
// 2, or launch_batch_max).
cudaError_t launch_step_body(fv_batch_t b, double cfl) {
  cudaError_t e = fv_fp32::launch_batch_dt(b->dev, cfl, b->stream);
  for (int stage = 1; stage <= 2 && e == cudaSuccess; ++stage) {
    for (int cls = 0; cls < kBatchClasses && e == cudaSuccess; ++cls) {
      const fv_batch_s::Tuning& t = b->tune[cls];
      e = fv_fp32::launch_batch_stage(stage, b->dev, cls, t.kchunk, t.occupancy, t.tile_x,
                                      t.tile_y, b->num_sms, b->stream);
    }
    if (e == cudaSuccess) e = fv_fp32::launch_batch_ghosts(stage, b->dev, b->stream);
  }
  return e;
}

// The maxima pass when the states changed since the last step.
cudaError_t launch_max_if_stale(fv_batch_t b) {
  if (b->smax_current) return cudaSuccess;
  return fv_fp32::launch_batch_max(b->dev, b->stream);
}

cudaError_t launch_step(fv_batch_t b, double cfl) {
  cudaError_t e = launch_max_if_stale(b);
  if (e == cudaSuccess) e = launch_step_body(b, cfl);
  b->smax_current = e == cudaSuccess;
  return e;
}

fv_status check_mesh_index(fv_batch_t b, int mesh) {
  if (mesh < 0 || mesh >= b->nmesh)
    return fail(FV_ERR_INVALID_ARG, "mesh index %d outside [0, %d)", mesh, b->nmesh);
  return FV_OK;
}

double* mesh_base(fv_batch_t b, double* base, int mesh) {
  return base + b->host_meshes[mesh].offset;
}

}  // namespace

extern "C" {

fv_status fv_batch_create(const fv_mesh_desc* descs, int nmesh, void* cuda_stream,
                          fv_batch_t* out) {
  if (!out) return fail(FV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!descs || nmesh < 1 || nmesh > (1 << 16))
    return fail(FV_ERR_INVALID_ARG, "need 1 .. 65536 mesh descriptions (got %d)", nmesh);
  for (int m = 0; m < nmesh; ++m) {
    fv_status st = fv_internal_validate_desc(&descs[m]);
    if (st != FV_OK) return st;
  }
  fv_batch_s* b = new fv_batch_s();
  b->nmesh = nmesh;
  b->desc.assign(descs, descs + nmesh);
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = fv_fp32::prepare_kernels();
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "querying the device");
  }
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {  // a stream of our own: the legacy default stream cannot be captured
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return cuda_fail(e, "creating the batch stream");
    }
    b->own_stream = true;
  }
  // per-mesh parameters and 256-byte aligned offsets into one state block
  size_t off = 0;
  std::vector<int2> dt_blocks, ghost_blocks;
  for (int m = 0; m < nmesh; ++m) {
    BatchMesh bm{};
    bm.P = fv_internal_params(&descs[m]);
    bm.Q = fv_fp32::make_params32(bm.P, 0.99);
    bm.offset = (long long)off;
    const size_t doubles = (size_t)fvd::NF * bm.P.nfield;
    off += (doubles + 31) / 32 * 32;
    const long long n = (long long)bm.P.nx * bm.P.ny * bm.P.nz;
    b->total_cells += n;
    b->class_meshes[fv_fp32::batch_class(bm.P.nx)] += 1;
    b->class_cells[fv_fp32::batch_class(bm.P.nx)] += n;
    b->max_dense = std::max(b->max_dense, (size_t)(fvd::NF * n));
    for (long long c = 0; c * fv_fp32::kBatchDtChunk < n; ++c) dt_blocks.push_back(make_int2(m, (int)c));
    const long long ring = fvd::ring_cells(bm.P);
    for (long long c = 0; c * fv_fp32::kBatchGhostChunk < ring; ++c)
      ghost_blocks.push_back(make_int2(m, (int)c));
    b->host_meshes.push_back(bm);
  }
  b->state_doubles = off;
  const size_t sb = off * sizeof(double);
  if ((e = cudaMalloc(&b->dev.U, sb)) != cudaSuccess ||
      (e = cudaMalloc(&b->dev.U1, sb)) != cudaSuccess ||
      (e = cudaMalloc(&b->dev.meshes, nmesh * sizeof(BatchMesh))) != cudaSuccess ||
      (e = cudaMalloc(&b->dev.dt_blocks, dt_blocks.size() * sizeof(int2))) != cudaSuccess ||
      (e = cudaMalloc(&b->dev.ghost_blocks, ghost_blocks.size() * sizeof(int2))) != cudaSuccess ||
      (e = cudaMalloc(&b->dev.next_item, 2 * kBatchClasses * sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMalloc(&b->dev.ctr, sizeof(DevCounters))) != cudaSuccess ||
      (e = cudaMalloc(&b->staging, b->max_dense * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&b->host_ctr, sizeof(DevCounters))) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return fail(e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA,
                "allocating %.3f GB of batch storage: %s", 2.0 * sb / 1e9, cudaGetErrorString(e));
  }
  b->dev.nmesh = nmesh;
  b->dev.all_mc = true;
  for (int m = 0; m < nmesh; ++m) b->dev.all_mc &= (b->host_meshes[m].Q.theta == 2.0f);
  b->dev.ndt_blocks = (int)dt_blocks.size();
  b->dev.nghost_blocks = (int)ghost_blocks.size();
  if ((e = cudaMemcpy(b->dev.meshes, b->host_meshes.data(), nmesh * sizeof(BatchMesh),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->dev.dt_blocks, dt_blocks.data(), dt_blocks.size() * sizeof(int2),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->dev.ghost_blocks, ghost_blocks.data(), ghost_blocks.size() * sizeof(int2),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(b->dev.U, 0, sb)) != cudaSuccess ||
      (e = cudaMemset(b->dev.U1, 0, sb)) != cudaSuccess ||
      (e = cudaMemset(b->dev.ctr, 0, sizeof(DevCounters))) != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "initialising batch storage");
  }
  fv_status st = build_items(b);
  if (st != FV_OK) {
    free_batch(b);
    return st;
  }
  {
    std::lock_guard<std::mutex> lk(g_batch_mutex);
    g_batches.insert(b);
  }
  *out = b;
  return FV_OK;
}

fv_status fv_batch_destroy(fv_batch_t b) {
  if (!b) return FV_OK;
  {
    std::lock_guard<std::mutex> lk(g_batch_mutex);
    if (!g_batches.erase(b)) return fail(FV_ERR_BAD_HANDLE, "batch handle %p is not live", (void*)b);
  }
  DeviceGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  return FV_OK;
}

fv_status fv_batch_set_state(fv_batch_t b, int mesh, const double* U, int on_device) {
  fv_status st = check(b);
  if (st == FV_OK) st = check_mesh_index(b, mesh);
  if (st != FV_OK) return st;
  if (!U) return fail(FV_ERR_INVALID_ARG, "U is NULL");
  DeviceGuard g(b->device);
  const fvd::Params& P = b->host_meshes[mesh].P;
  const size_t dense = (size_t)fvd::NF * P.nx * P.ny * P.nz;
  cudaError_t e = cudaSuccess;
  const double* src = U;
  if (!on_device) {
    e = cudaMemcpyAsync(b->staging, U, dense * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    src = b->staging;
  }
  double* dst = mesh_base(b, b->dev.U, mesh);
  if (e == cudaSuccess) e = launch_scatter_interior(src, dst, P, b->stream);
  if (e == cudaSuccess) e = launch_fill_ghosts(dst, P, b->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(b->stream);
  b->smax_current = false;
  if (e != cudaSuccess) return cuda_fail(e, "fv_batch_set_state");
  return FV_OK;
}

fv_status fv_batch_get_state(fv_batch_t b, int mesh, double* U, int on_device) {
  fv_status st = check(b);
  if (st == FV_OK) st = check_mesh_index(b, mesh);
  if (st != FV_OK) return st;
  if (!U) return fail(FV_ERR_INVALID_ARG, "U is NULL");
  DeviceGuard g(b->device);
  const fvd::Params& P = b->host_meshes[mesh].P;
  const size_t dense = (size_t)fvd::NF * P.nx * P.ny * P.nz;
  double* dst = on_device ? U : b->staging;
  cudaError_t e = launch_gather_interior(mesh_base(b, b->dev.U, mesh), dst, P, b->stream);
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(U, b->staging, dense * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "fv_batch_get_state");
  return FV_OK;
}

fv_status fv_batch_step(fv_batch_t b, double cfl, int use_graph) {
  fv_status st = check(b);
  if (st != FV_OK) return st;
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(FV_ERR_INVALID_ARG, "cfl %g must be > 0", cfl);
  DeviceGuard g(b->device);
  cudaError_t e;
  if (!use_graph) {
    e = launch_step(b, cfl);
    if (e != cudaSuccess) return cuda_fail(e, "batch step kernels");
    return FV_OK;
  }
  bool same_tuning = true;
  for (int c = 0; c < kBatchClasses; ++c) same_tuning = same_tuning && b->graph_tune[c] == b->tune[c];
  if (!b->graph || b->graph_cfl != cfl || !same_tuning) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "beginning the step capture");
    cudaError_t le = launch_step_body(b, cfl);
    e = cudaStreamEndCapture(b->stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(le != cudaSuccess ? le : e, "capturing the step");
    }
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return cuda_fail(e, "instantiating the step graph");
    }
    b->graph_cfl = cfl;
    for (int c = 0; c < kBatchClasses; ++c) b->graph_tune[c] = b->tune[c];
  }
  e = launch_max_if_stale(b);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
  b->smax_current = e == cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "launching the step graph");
  return FV_OK;
}

fv_status fv_batch_get_dt(fv_batch_t b, double* dt) {
  fv_status st = check(b);
  if (st != FV_OK) return st;
  if (!dt) return fail(FV_ERR_INVALID_ARG, "dt is NULL");
  DeviceGuard g(b->device);
  std::vector<BatchMesh> tmp(b->nmesh);
  cudaError_t e = cudaMemcpyAsync(tmp.data(), b->dev.meshes, b->nmesh * sizeof(BatchMesh),
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading dt");
  for (int m = 0; m < b->nmesh; ++m) dt[m] = tmp[m].dt;
  return FV_OK;
}

fv_status fv_batch_set_tuning(fv_batch_t b, int kchunk, int occupancy, int tile_y) {
  fv_status st = check(b);
  if (st != FV_OK) return st;
  if (kchunk < 1 || kchunk > 4096 || !fv_fp32::valid_config(32, tile_y, occupancy))
    return fail(FV_ERR_INVALID_ARG,
                "kchunk %d must be in [1, 4096], tile_y (%d) 4, 8 or 16 and occupancy (%d) 2, "
                "or 3 with tile_y 8",
                kchunk, tile_y, occupancy);
  DeviceGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  for (int c = 0; c < kBatchClasses; ++c) {
    b->tune[c].tile_x = 32;
    b->tune[c].tile_y = tile_y;
    b->tune[c].occupancy = occupancy;
    b->tune[c].kchunk = kchunk;
  }
  return build_items(b);
}

fv_status fv_batch_set_class_tuning(fv_batch_t b, int cls, int tile_x, int tile_y,
                                    int occupancy, int kchunk) {
  fv_status st = check(b);
  if (st != FV_OK) return st;
  if (cls < 0 || cls >= kBatchClasses || kchunk < 1 || kchunk > 4096 ||
      !fv_fp32::valid_config(tile_x, tile_y, occupancy))
    return fail(FV_ERR_INVALID_ARG,
                "class %d must be 0 .. 2, kchunk %d in [1, 4096] and (tile_x, tile_y, "
                "occupancy) = (%d, %d, %d) one of the built shapes",
                cls, kchunk, tile_x, tile_y, occupancy);
  DeviceGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  b->tune[cls] = fv_batch_s::Tuning{tile_x, tile_y, occupancy, kchunk};
  return build_items(b);
}

fv_status fv_batch_get_class_tuning(fv_batch_t b, int cls, int* tile_x, int* tile_y,
                                    int* occupancy, int* kchunk, int* meshes) {
  fv_status st = check(b);
  if (st != FV_OK) return st;
  if (cls < 0 || cls >= kBatchClasses) return fail(FV_ERR_INVALID_ARG, "class %d not 0 .. 2", cls);
  const fv_batch_s::Tuning& t = b->tune[cls];
  if (tile_x) *tile_x = t.tile_x;
  if (tile_y) *tile_y = t.tile_y;
  if (occupancy) *occupancy = t.occupancy;
  if (kchunk) *kchunk = t.kchunk;
  if (meshes) *meshes = b->class_meshes[cls];
  return FV_OK;
}

fv_status fv_batch_autotune(fv_batch_t b, double cfl, int* kchunk_out, int* occupancy_out,
                            int* tile_y_out, double* ms_per_step_out) {
  fv_status st = check(b);
  if (st != FV_OK) return st;
  if (!(cfl > 0.0)) return fail(FV_ERR_INVALID_ARG, "cfl must be > 0");
  DeviceGuard g(b->device);
  const size_t sb = b->state_doubles * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (!b->backup && (e = cudaMalloc(&b->backup, sb)) != cudaSuccess)
    return cuda_fail(e, "allocating the autotuner's state snapshot");
  DevCounters saved{};
  if ((e = cudaMemcpyAsync(b->backup, b->dev.U, sb, cudaMemcpyDeviceToDevice, b->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(&saved, b->dev.ctr, sizeof saved, cudaMemcpyDeviceToHost, b->stream)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
    return cuda_fail(e, "snapshotting the state");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // times three whole steps (after one to warm up) with the current tuning,
  // each candidate from the snapshot: stepping on from the previous
  // candidate's state would time later candidates on a more evolved (and
  // costlier) state and bias the search toward the shapes tried first
  auto time_step = [&](double& ms_out) -> cudaError_t {
    cudaError_t r = cudaMemcpyAsync(b->dev.U, b->backup, sb, cudaMemcpyDeviceToDevice, b->stream);
    b->smax_current = false;
    if (r == cudaSuccess) r = launch_step(b, cfl);
    cudaEventRecord(e0, b->stream);
    for (int i = 0; i < 3 && r == cudaSuccess; ++i) r = launch_step(b, cfl);
    cudaEventRecord(e1, b->stream);
    if (r == cudaSuccess) r = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (r == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    ms_out = ms / 3.0;
    return r;
  };
  // one size class at a time (largest first), the others at their best so
  // far: every built shape no wider than twice the class's widest mesh and
  // every z chunk in {8, 16, 32, 64}
  const int kcs[] = {8, 16, 32, 64};
  int cls_order[kBatchClasses] = {2, 1, 0};
  std::sort(cls_order, cls_order + kBatchClasses,
            [&](int a, int c) { return b->class_cells[a] > b->class_cells[c]; });
  double best = 1e300;
  for (int oi = 0; oi < kBatchClasses && e == cudaSuccess && st == FV_OK; ++oi) {
    const int cls = cls_order[oi];
    if (b->class_meshes[cls] == 0) continue;
    int widest = 0;
    for (const BatchMesh& m : b->host_meshes)
      if (fv_fp32::batch_class(m.P.nx) == cls) widest = std::max(widest, m.P.nx);
    fv_batch_s::Tuning keep = b->tune[cls];
    double class_best = 1e300;
    for (const auto& shape : fv_fp32::kShapes) {
      if (shape[0] > 2 * widest && shape[0] > 32) continue;
      for (int kc : kcs) {
        b->tune[cls] = fv_batch_s::Tuning{shape[0], shape[1], shape[2], kc};
        if ((st = build_items(b)) != FV_OK) break;
        double ms = 0.0;
        if ((e = time_step(ms)) != cudaSuccess) break;
        if (ms < class_best) {
          class_best = ms;
          keep = b->tune[cls];
        }
      }
      if (e != cudaSuccess || st != FV_OK) break;
    }
    b->tune[cls] = keep;
    best = class_best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == FV_OK && e == cudaSuccess) st = build_items(b);
  // restore the state (ghosts included) and the counters
  cudaError_t r = cudaMemcpyAsync(b->dev.U, b->backup, sb, cudaMemcpyDeviceToDevice, b->stream);
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(b->dev.ctr, &saved, sizeof saved, cudaMemcpyHostToDevice, b->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(b->stream);
  b->smax_current = false;
  if (e != cudaSuccess) return cuda_fail(e, "autotuning");
  if (r != cudaSuccess) return cuda_fail(r, "restoring the state after autotuning");
  if (st != FV_OK) return st;
  // report the configuration of the class with the most cells
  const fv_batch_s::Tuning& t = b->tune[cls_order[0]];
  if (kchunk_out) *kchunk_out = t.kchunk;
  if (occupancy_out) *occupancy_out = t.occupancy;
  if (tile_y_out) *tile_y_out = t.tile_y;
  if (ms_per_step_out) *ms_per_step_out = best;
  return FV_OK;
}

fv_status fv_batch_get_counters(fv_batch_t b, long long* nonphysical_cells,
                                long long* fallback_faces) {
  fv_status st = check(b);
  if (st != FV_OK) return st;
  DeviceGuard g(b->device);
  cudaError_t e = cudaMemcpyAsync(b->host_ctr, b->dev.ctr, sizeof(DevCounters),
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading batch counters");
  if (nonphysical_cells)
    *nonphysical_cells = (long long)(b->host_ctr->np_step + b->host_ctr->np_dt);
  if (fallback_faces) *fallback_faces = (long long)b->host_ctr->fallback;
  return FV_OK;
}

fv_status fv_batch_info(fv_batch_t b, int* nmesh, long long* total_cells, long long* work_items) {
  fv_status st = check(b);
  if (st != FV_OK) return st;
  if (nmesh) *nmesh = b->nmesh;
  if (total_cells) *total_cells = b->total_cells;
  if (work_items) *work_items = b->dev.nitems;
  return FV_OK;
}

}  // extern "C"
