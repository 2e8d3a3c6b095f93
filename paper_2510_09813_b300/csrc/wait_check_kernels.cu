// Exercises the error path of the library's bounded device waits: one thread
// waits, through the same mbar_wait the streaming passes use, on an mbarrier
// that nothing ever completes. The wait gives up after its time limit, the
// kernel sets the error word and returns, and the host reads the word. No
// fault, trap or unbounded loop is involved.
#include "kernels.h"
#include "tma.cuh"

namespace rsv {

namespace {

__global__ void wait_check_kernel(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) atomicOr(err, 1);  // no arrival: phase 0 never completes
}

}  // namespace

cudaError_t launch_wait_check(int* err, cudaStream_t stream) {
  wait_check_kernel<<<1, 32, 0, stream>>>(err);
  return cudaGetLastError();
}

}  // namespace rsv
