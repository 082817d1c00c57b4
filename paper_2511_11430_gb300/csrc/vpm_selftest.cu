// Self-test of the bounded device waits: a wait on an mbarrier phase that nothing will
// complete must give up after its time limit, latch DEV_ERR_TIMEOUT in the device error
// word and let the kernel return, leaving the context usable.
#include "vpm_internal.h"

namespace vpm {

static __device__ int g_selftest_completed;

__global__ void selftest_wait_kernel(int* dev_err, unsigned long long limit_ns, int* completed)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one expected arrival, which never comes
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) *completed = mbar_wait_bounded(&bar, 0, dev_err, limit_ns) ? 1 : 0;
}

cudaError_t run_selftest_wait(double limit_ms, int* completed, cudaStream_t st)
{
    int* d = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d), g_selftest_completed);
    if (e != cudaSuccess) return e;
    trace_launch();
    selftest_wait_kernel<<<1, 32, 0, st>>>(dev_err_ptr(), (unsigned long long)(limit_ms * 1e6), d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(completed, d, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace vpm
