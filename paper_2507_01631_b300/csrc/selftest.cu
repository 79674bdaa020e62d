// Self-test of the bounded device waits that every mbarrier wait of the
// tensor-core field kernels uses (tc::mbar_wait): one CTA waits on an
// mbarrier.  With `arrive`, one thread arrives first and the wait completes;
// without, nothing ever arrives and the wait gives up after its time limit,
// sets the timeout bit of the state and the kernel returns -- the path a
// stalled tensor core or bulk copy would take, exercised without one.
#include "kernels.cuh"
#include "tc.cuh"

namespace snk {
namespace {

__global__ void k_wait_selftest(int arrive, snk_state *state) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) tc::mbar_arrive(&mbar);
  const bool ok = tc::mbar_wait(&mbar, 0);
  if (!ok && threadIdx.x == 0) set_status(state, kStatusTimeout);
}

}  // namespace

cudaError_t launch_wait_selftest(int arrive, snk_state *state, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(arrive, state);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace snk
