// fv_fused_common.cuh -- tile geometry and staging helpers shared by the
// fused substep kernels of the FP64 paths (fv_fused64_kernels.cu, FP64 face
// arithmetic; fv_fused_ff_kernels.cu, float-float face arithmetic).
#pragma once

namespace fvfused {

constexpr int TX = 32;   // tile width: one warp per tile row

template <int TY_, int TX_ = TX>
struct Shape64 {
  static constexpr int TX = TX_;   // the float-float kernel also takes 16
  static constexpr int TY = TY_;
  static constexpr int kThreads = TX * TY;
  static constexpr int PX = TX + 4;
  static constexpr int PY = TY + 4;
  static constexpr int kHalo = PX * PY - TX * TY;
  static constexpr int kHaloPer = (kHalo + kThreads - 1) / kThreads;
  static constexpr int kXSlopes = (TX + 2) * TY;   // cells -1 .. TX of each tile row
  static constexpr int kYSlopes = TX * (TY + 2);   // rows -1 .. TY of each tile column
  static constexpr int kSlopes = kXSlopes + kYSlopes;
  static constexpr int kSlopePer = (kSlopes + kThreads - 1) / kThreads;
  static constexpr int kXFaces = (TX + 1) * TY;
  static constexpr int kYFaces = TX * (TY + 1);
  static constexpr int kFaces = kXFaces + kYFaces;
  static constexpr int kFacePer = (kFaces + kThreads - 1) / kThreads;
  static_assert(kFacePer <= 8, "face fallback bits");
};


// Halo cell h of a tile (0 <= h < kHalo): two rows below the tile, two
// above, then two columns on each side of every tile row; (row, col)
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

// Hint: bring the line holding p into L2 (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

}  // namespace fvfused
