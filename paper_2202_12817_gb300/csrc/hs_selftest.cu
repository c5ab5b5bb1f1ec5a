// Self-test of the bounded-wait path.  The kernels that wait on their own bulk copies (the
// shared-memory window kernel) give every mbarrier wait a time limit, after which they record
// kErrTimeout in the plan's error word and return instead of hanging.  This kernel runs that
// path on purpose: one CTA waits on a barrier phase that nothing completes (no copy is issued
// and no thread arrives), the wait gives up after limit_ns, and the CTA exits with nothing in
// flight, so the device context stays usable.
#include "hs_fwd1d_win.cuh"

namespace hs {

__global__ void k_wait_selftest(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!mbar_wait(&bar, 0, limit_ns) && threadIdx.x == 0) set_error(err, kErrTimeout);
}

const void *wait_selftest_kernel() { return reinterpret_cast<const void *>(&k_wait_selftest); }

}  // namespace hs
