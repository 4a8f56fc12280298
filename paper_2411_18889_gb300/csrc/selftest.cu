// selftest.cu -- exercises the bounded-wait path every pipelined kernel uses:
// one CTA waits on an mbarrier phase that nothing completes, gives up after
// the given limit, records the timeout in the device error word and returns.
// The GPU context stays usable; the host reads the word back.
#include "nbody_internal.cuh"

namespace nbk {
namespace {

__global__ void wait_timeout_kernel(uint64_t limit_ns, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none will come
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(err, kErrTimeout);
}

}  // namespace

cudaError_t selftest_wait(uint64_t limit_ns, int* err, cudaStream_t st) {
    wait_timeout_kernel<<<1, 32, 0, st>>>(limit_ns, err);
    return cudaGetLastError();
}

}  // namespace nbk
