// Device self-test of the bounded-wait error path.  Every tcgen05 kernel
// waits on mbarriers through tc::mbar_wait with an iteration limit; when the
// limit runs out it records BAYER_ERR_TIMEOUT in the handle's status word and
// finishes instead of hanging.  This kernel exercises exactly that path
// without a fault: one CTA initialises an mbarrier expecting one arrival and
// waits on its first phase, after arriving itself (the wait succeeds) or not
// (nothing ever arrives, the wait gives up after `limit` polls).
#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace bme {

namespace {

__global__ void wait_selftest_kernel(int* status, int arrive, unsigned limit) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) tc::mbar_arrive(&mbar);
  const bool ok = tc::mbar_wait(&mbar, 0, limit);
  if (!ok && threadIdx.x == 0) atomicExch(status, (int)BAYER_ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_selftest(int* status, bool arrive, unsigned limit, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(status, arrive ? 1 : 0, limit);
  return cudaGetLastError();
}

}  // namespace bme
