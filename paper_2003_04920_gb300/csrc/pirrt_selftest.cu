// Failure detection without a fault: each self-test runs one device-side wait
// of the kind the exploitation kernels use -- the bounded grid barrier of the
// cooperative kernels, or the bounded mbarrier wait of the staged Improve --
// in a situation where nothing will ever end it, under a short limit, and
// checks that the wait gives up, raises kStatusTimeout in a status word and
// returns.  Every CTA leaves the kernel, so the context stays usable; the host
// maps the status word to PIRRT_ERR_DEVICE_TIMEOUT exactly as it does after
// an exploit.  The paper has no counterpart (its planner has no device-side
// waits that could stall).
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "improve_tma.cuh"
#include "pirrt.h"

using namespace pirrt;

namespace {

// The self-tests' own counter block: the graph handles' counters are never
// touched, so a self-test can run next to them.
__device__ DevCounters g_selftest_ctr;

__global__ void selftest_clear() {
    unsigned *w = reinterpret_cast<unsigned *>(&g_selftest_ctr);
    for (int i = threadIdx.x; i < (int)(sizeof(DevCounters) / sizeof(unsigned)); i += blockDim.x)
        w[i] = 0u;
}

// A grid of two CTAs in which CTA 1 leaves without reaching the barrier, so
// CTA 0's wait can only end by its limit (`spins` polls).
__global__ void selftest_barrier(unsigned long long spins) {
    if (blockIdx.x != 0) return;
    grid_barrier(&g_selftest_ctr, gridDim.x, spins);
}

// An mbarrier that expects one arrival nobody makes: the wait for its first
// phase can only end by its limit (`ns` nanoseconds of the global timer).
__global__ void selftest_mbarrier(unsigned long long ns) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) tma::mbar_init(&bar, 1u);
    __syncthreads();
    const bool done = tma::mbar_wait(&bar, 0u, ns);
    if (!done && threadIdx.x == 0) atomicOr(&g_selftest_ctr.status, kStatusTimeout);
}

}  // namespace

extern "C" pirrt_status pirrt_selftest_wait(int32_t which, int64_t limit, void *stream) {
    if (which != PIRRT_SELFTEST_GRID_BARRIER && which != PIRRT_SELFTEST_MBARRIER)
        return PIRRT_ERR_INVALID_ARG;
    if (limit < 1 || limit > (which == PIRRT_SELFTEST_GRID_BARRIER ? (1 << 20) : 1000000000))
        return PIRRT_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    selftest_clear<<<1, 32, 0, st>>>();
    if (cudaGetLastError() != cudaSuccess) return PIRRT_ERR_CUDA;
    if (which == PIRRT_SELFTEST_GRID_BARRIER) {
        unsigned long long spins = (unsigned long long)limit;
        void *args[] = {&spins};
        if (cudaLaunchCooperativeKernel((const void *)selftest_barrier, dim3(2), dim3(32), args, 0,
                                        st) != cudaSuccess)
            return PIRRT_ERR_CUDA;
    } else {
        selftest_mbarrier<<<1, 32, 0, st>>>((unsigned long long)limit);
        if (cudaGetLastError() != cudaSuccess) return PIRRT_ERR_CUDA;
    }
    unsigned status = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpyFromSymbol(&status, g_selftest_ctr, sizeof(unsigned),
                             offsetof(DevCounters, status)) != cudaSuccess)
        return PIRRT_ERR_CUDA;
    if (status & kStatusTimeout) return PIRRT_ERR_DEVICE_TIMEOUT;
    return status ? PIRRT_ERR_CUDA : PIRRT_OK;
}
