// Check of the bounded device waits. Every wait of the library's tensor-core kernels is an
// mbarrier wait bounded by globaltimer; when one gives up, the kernel sets the context's error
// word and the host returns SLAG_ERR_TIMEOUT. This kernel runs that path on demand, with nothing
// else in flight (no TMA copy, no MMA, no TMEM): one role waits, with the given bound, on an
// mbarrier that nothing completes, and a second role waits on another one until the first
// role's abort flag tells it to give up -- the protocol of the warp-specialised kernels.
#include "slag_internal.cuh"
#include "tc_util.cuh"

namespace slag {

namespace {

__global__ void __launch_bounds__(64) wait_check_k(uint64_t limit_ns, int complete, uint32_t *err) {
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // the role whose barrier may never complete; `complete` arrives first (the control case)
        if (complete) tc::arrive(&bar[0]);
        const bool ok = tc::wait_or_abort_for(&bar[0], 0, &abort_flag, limit_ns);
        if (!ok) atomicOr(err, 1u);
        if (ok) tc::arrive(&bar[1]);   // releases the second role on success
    } else if (threadIdx.x == 32) {
        // the second role: released by the first, or told to give up through the abort flag
        // (its own bound is the library's, far above limit_ns)
        const bool ok = tc::wait_or_abort(&bar[1], 0, &abort_flag);
        if (!ok) atomicOr(err, 2u);
    }
    __syncthreads();
}

}  // namespace

void launch_wait_check(uint64_t limit_ns, int complete, uint32_t *err, cudaStream_t st) {
    wait_check_k<<<1, 64, 0, st>>>(limit_ns, complete, err); note_launch();
}

}  // namespace slag
