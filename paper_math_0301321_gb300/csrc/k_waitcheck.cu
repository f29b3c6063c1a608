// Self-check of the bounded-wait failure path.
//
// The staged x pass and the tensor-core y pass wait on mbarriers for their
// own asynchronous copies and commits, a bounded number of polls at most;
// a wait that runs out sets DEV_TIMEOUT in the context's status word and
// the kernel returns.  k_wait_check takes that same wait (mbar_wait_bounded)
// on a fresh mbarrier that nothing ever arrives on, so the wait runs out by
// construction, without a copy, a commit or any other work left in flight.
#include "async_copy.cuh"

namespace ibgb {

__global__ void k_wait_check(int *status, int polls)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // phase 0 of a fresh barrier completes only after one arrival; none comes
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, status, polls);
}

void launch_wait_check(int *status, int polls, cudaStream_t s)
{
    k_wait_check<<<1, 32, 0, s>>>(status, polls);
}

}  // namespace ibgb
