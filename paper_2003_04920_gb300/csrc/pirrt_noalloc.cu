// Evaluate without any allocation: g from a parent array and parent-edge
// costs, by the same pointer-jumping kernel the graph handle uses, with every
// byte of scratch memory taken from one file-scope device array.
//
// Some callers cannot call cudaMalloc at the time they need this: a real-time
// planning loop that fixes all of its memory at start-up and must not stall
// on the allocator (or fail on it) in the middle of a control cycle.  They
// pass their own inputs and outputs; the scratch (work lists, running sums,
// the counter block, the kernel's argument block) lives in kScratchBytes of
// static device memory that every GPU loading this library keeps until the
// process exits.  The call reads a status word back and synchronises its
// stream before it returns.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <functional>
#include <mutex>

#include "graph_kernels.cuh"
#include "pirrt.h"

using namespace pirrt;

namespace {

// Largest vertex count the static scratch serves.
constexpr int64_t kMaxNoAllocVertices = 1 << 18;  // 262,144

constexpr size_t round256(size_t b) { return (b + 255) & ~size_t(255); }
// Per vertex: two ancestor arrays (int32), two running-sum arrays (double),
// the finishing round (int32), two work lists (int32), the changed list
// (int32) and the FP32 copy of g; plus the counter block.  About 11.5 MB.
constexpr size_t kN = (size_t)kMaxNoAllocVertices;
constexpr size_t kScratchBytes = 2 * round256(4 * kN) + 2 * round256(8 * kN) + round256(4 * kN) +
                                 2 * round256(4 * kN) + round256(4 * kN) + round256(4 * kN) +
                                 round256(sizeof(DevCounters)) +
                                 round256(sizeof(EvaluateArgs<double>));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int blocks = 0;                    // co-resident grid for the cooperative launch
};
DeviceSetup g_setup[kMaxDevices];

// Clear the counter block and store the kernel's arguments in the scratch
// array (the evaluate kernel reads them from device memory).  One warp.
__global__ void noalloc_write_args(EvaluateArgs<double> a, EvaluateArgs<double> *dargs,
                                   DevCounters *ctr) {
    unsigned *w = reinterpret_cast<unsigned *>(ctr);
    for (int i = threadIdx.x; i < (int)(sizeof(DevCounters) / sizeof(unsigned)); i += blockDim.x)
        w[i] = 0u;
    if (threadIdx.x == 0) *dargs = a;
}

// g(root) = 0, every other vertex +inf (the evaluate kernel only writes
// vertices whose parent chain reaches the root), and a check of the caller's
// policy before any kernel follows it: every parent of a vertex other than
// the root is -1 or an id in [0, n), and every used parent-edge cost is
// finite and >= 0.  A violation raises kStatusBadInput.
__global__ void noalloc_prepare(int64_t n, int32_t root, const int32_t *__restrict__ parent,
                                const double *__restrict__ cost, double *__restrict__ g,
                                DevCounters *ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        g[v] = (v == root) ? 0.0 : CUDART_INF;
        if (v == root) continue;
        const int32_t pv = parent[v];
        if (pv == -1) continue;
        const double c = cost[v];
        if (pv < 0 || (int64_t)pv >= n || !(c >= 0.0 && c <= DBL_MAX)) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctr->status, kStatusBadInput);
}

// The evaluate kernel runs (n_switched = 1; it is launched with force = 0)
// only if the policy passed the check.
__global__ void noalloc_gate(DevCounters *ctr) {
    ctr->n_switched = __ldcg(&ctr->status) == 0u ? 1u : 0u;
}

void setup_device(DeviceSetup &s) {
    void *addr = nullptr;
    s.err = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (s.err != cudaSuccess) return;
    s.scratch = static_cast<unsigned char *>(addr);
    int dev = 0, sms = 0, occ = 0;
    if ((s.err = cudaGetDevice(&dev)) != cudaSuccess) return;
    if ((s.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return;
    if ((s.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, evaluate_kernel<double>, kThreads,
                                                               0)) != cudaSuccess)
        return;
    s.blocks = sms * (occ > 0 ? occ : 1);
}

}  // namespace

extern "C" pirrt_status pirrt_evaluate_noalloc(int64_t n, int32_t root, const int32_t *parent,
                                               const double *parent_cost, double *g_out,
                                               void *stream) {
    if (n < 0 || (n > 0 && (!parent || !parent_cost || !g_out)) || (n > 0 && (root < 0 || root >= n)))
        return PIRRT_ERR_INVALID_ARG;
    if (n > kMaxNoAllocVertices) return PIRRT_ERR_CAPACITY;
    if (n == 0) return PIRRT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIRRT_ERR_CUDA;
    DeviceSetup &s = g_setup[dev];
    std::call_once(s.once, setup_device, std::ref(s));
    if (s.err != cudaSuccess || !s.scratch || s.blocks < 1) return PIRRT_ERR_CUDA;

    // carve the static array (sized for kMaxNoAllocVertices, aligned slices)
    unsigned char *base = s.scratch;
    const size_t N = (size_t)kMaxNoAllocVertices;
    auto take = [&](size_t bytes) {
        unsigned char *q = base;
        base += round256(bytes);
        return q;
    };
    EvaluateArgs<double> a;
    a.p = parent;
    a.pc = parent_cost;
    a.g = g_out;
    a.anc[0] = reinterpret_cast<int32_t *>(take(4 * N));
    a.anc[1] = reinterpret_cast<int32_t *>(take(4 * N));
    a.acc[0] = reinterpret_cast<double *>(take(8 * N));
    a.acc[1] = reinterpret_cast<double *>(take(8 * N));
    a.done = reinterpret_cast<int32_t *>(take(4 * N));
    a.wl[0] = reinterpret_cast<int32_t *>(take(4 * N));
    a.wl[1] = reinterpret_cast<int32_t *>(take(4 * N));
    a.dg = reinterpret_cast<int32_t *>(take(4 * N));
    a.g32 = reinterpret_cast<float *>(take(4 * N));
    DevCounters *ctr = reinterpret_cast<DevCounters *>(take(sizeof(DevCounters)));
    // the kernel reads its arguments from device memory: they live in the array too
    EvaluateArgs<double> *dargs =
        reinterpret_cast<EvaluateArgs<double> *>(take(sizeof(EvaluateArgs<double>)));
    if ((size_t)(base - s.scratch) != kScratchBytes) return PIRRT_ERR_CUDA;  // layout mismatch
    a.ctr = ctr;
    a.n = n;
    a.root = root;
    a.force = 0;  // gated by noalloc_gate
    a.role = 0;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    noalloc_write_args<<<1, 32, 0, st>>>(a, dargs, ctr);
    if (cudaGetLastError() != cudaSuccess) return PIRRT_ERR_CUDA;
    const int pb = (int)((n + kThreads - 1) / kThreads);
    noalloc_prepare<<<pb < 1024 ? pb : 1024, kThreads, 0, st>>>(n, root, parent, parent_cost,
                                                                 g_out, ctr);
    if (cudaGetLastError() != cudaSuccess) return PIRRT_ERR_CUDA;
    noalloc_gate<<<1, 1, 0, st>>>(ctr);
    if (cudaGetLastError() != cudaSuccess) return PIRRT_ERR_CUDA;
    const EvaluateArgs<double> *argp = dargs;
    void *args[] = {&argp};
    if (cudaLaunchCooperativeKernel((const void *)evaluate_kernel<double>, dim3(s.blocks),
                                    dim3(kThreads), args, 0, st) != cudaSuccess)
        return PIRRT_ERR_CUDA;
    // the status word tells a cycle (or a barrier timeout) apart from success
    unsigned status = 0;
    if (cudaMemcpyAsync(&status, &ctr->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PIRRT_ERR_CUDA;
    if (status & kStatusBadInput) return PIRRT_ERR_BAD_INPUT;
    if (status & kStatusTimeout) return PIRRT_ERR_DEVICE_TIMEOUT;
    if (status & kStatusBadTree) return PIRRT_ERR_BAD_TREE;
    return PIRRT_OK;
}
