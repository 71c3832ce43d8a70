// Checks the bounded mbarrier wait of fv_umma.cuh (the wait of the
// tensor-core kernels): on a barrier that nothing arrives at it gives up
// after its poll limit and reports it (the kernel then records
// FV_ERR_TIMEOUT instead of hanging); on a barrier that has completed its
// phase it reports completion.  Prints "expired <e> completed <c>" and exits
// 0 when e == 1 and c == 1.
#include <cstdio>
#include <cuda_runtime.h>

#include "fv_umma.cuh"

__global__ void k_waits(int* out) {
  __shared__ __align__(8) uint64_t never, done;
  if (threadIdx.x == 0) {
    umma::mbar_init(&never, 1);
    umma::mbar_init(&done, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // nothing arrives at `never`: the wait must give up after its 64 polls
    out[0] = umma::mbar_wait(&never, 0, 64) ? 0 : 1;
    // one arrival completes phase 0 of `done`
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(
        umma::smem_addr(&done)));
    out[1] = umma::mbar_wait(&done, 0, 64) ? 1 : 0;
  }
}

int main() {
  int* d;
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return 2;
  cudaMemset(d, 0, 2 * sizeof(int));
  k_waits<<<1, 32>>>(d);
  int h[2] = {-1, -1};
  cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  printf("expired %d completed %d (%s)\n", h[0], h[1], cudaGetErrorString(e));
  cudaFree(d);
  return (e == cudaSuccess && h[0] == 1 && h[1] == 1) ? 0 : 1;
}
