// Bounded-wait self-test (jet_selftest_wait): the time-out paths of the
// tensor-core kernels and of the chained small levels exercised without
// injecting a fault.  One CTA holds tensor memory like those kernels, waits on
// an mbarrier that nothing arrives on with the same bounded-wait helper and a
// caller-set limit, records the time-out in the network's status word (bit 4),
// then waits at the chains' grid barrier for a second block that does not
// exist (bit 8), releases its tensor memory and returns; nothing asynchronous
// is in flight at any point.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace jet {

__global__ void __launch_bounds__(64, 1) wait_selftest_kernel(uint32_t *status, uint32_t *arrive, uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(32u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 32) {   // the barrier's phase 0 never completes: no thread arrives on it
        if (!mbar_wait_bounded(smem_u32(&bar), 0u, (volatile int *)&abort_flag, limit_ns)) {
            abort_flag = 1;
            atomicOr(status, 4u);
        }
        *arrive = 0u;   // one block: two arrivals never come
        if (!grid_arrive_wait(arrive, 2u, limit_ns)) atomicOr(status, 8u);
        *arrive = 0u;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_holder), "r"(32u));
}

int selftest_wait(Network &net, int64_t limit_us, void *stream)
{
    ensure_leaves_on_device(net);
    cudaStream_t s = stream ? (cudaStream_t)stream : (cudaStream_t)net.stream;
    // (the barrier counter: a word of the status buffer past the status word)
    wait_selftest_kernel<<<1, 64, 0, s>>>((uint32_t *)net.d_status, (uint32_t *)net.d_status + 4,
                                          (uint64_t)limit_us * 1000ull);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(JET_ECUDA, std::string("self-test launch: ") + cudaGetErrorString(e));
    return read_clear_status(net, stream);
}

}  // namespace jet
