// Failure-detection self-test: the bounded mbarrier wait every TMA/tcgen05
// kernel of the library uses (ptx.cuh) is run on a barrier that nothing ever
// arrives on, so it must give up after its limit, raise the abort flag and
// let the kernel report QPADL_ETIMEOUT through a status word, with the
// context still usable.  With `arrive` set, the barrier is completed first
// and the same wait must succeed at once.
#include <cstdint>
#include <cuda_runtime.h>

#include "ptx.cuh"
#include "qpadl_pir.h"

namespace qpadl {

__global__ void selftest_wait_kernel(int arrive, int *__restrict__ status, unsigned long long *__restrict__ waited_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) mbar_arrive(&bar);
        const uint64_t t0 = global_ns();
        const bool ok = mbar_wait(&bar, 0, &abort_flag);
        *waited_ns = global_ns() - t0;
        *status = ok ? 0 : kDevTimeout;
    }
}

}  // namespace qpadl

extern "C" int qpadl_selftest_bounded_wait(int arrive, int32_t *status_dev, uint64_t *waited_ns_dev,
                                           qpadl_stream_t stream) {
    if (!status_dev || !waited_ns_dev) return QPADL_EINVAL;
    qpadl::selftest_wait_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        arrive ? 1 : 0, status_dev, reinterpret_cast<unsigned long long *>(waited_ns_dev));
    return cudaGetLastError() == cudaSuccess ? QPADL_OK : QPADL_ECUDA;
}
