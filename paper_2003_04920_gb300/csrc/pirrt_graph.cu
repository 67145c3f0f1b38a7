// Host runtime and C ABI of the single-graph PI-RRT# exploitation path.
//
// All graph state (CSR, g, parents, work lists) stays resident on the
// device.  A Replan (Alg. 2: Improve, then Evaluate, until no parent
// switches) runs as one CUDA-graph launch whose WHILE node repeats the loop
// body on the device -- Improve, then Evaluate, which ends the iteration by
// testing convergence and setting the loop condition -- so the host waits
// once per exploit.  With profiling enabled the same kernels run from a host
// loop that reads the counter block after every iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "evaluate_async.cuh"
#include "graph_kernels.cuh"
#include "improve_push.cuh"
#include "improve_screen.cuh"
#include "improve_tma.cuh"
#include "replan_iteration.cuh"
#include "pirrt.h"

using namespace pirrt;

namespace {
// Offsets of the kernel argument structs in the device argument block.
constexpr size_t kArgImprove = 0, kArgEval = 512, kArgEvalFallback = 1024, kArgWave = 1536,
                 kArgMark = 2048, kArgMarkFallback = 2560, kArgEvalForce = 3072, kArgAsync = 3584,
                 kArgBytes = 4096;
}  // namespace

struct pirrt_graph {
    pirrt_config cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;  // private stream for recording loop bodies
    cudaStream_t copy = nullptr;     // host-to-device prefetch of the next block
    void *pre = nullptr;             // the prefetched block on the device
    size_t pre_bytes = 0;
    cudaEvent_t pre_done = nullptr;  // the prefetch copies finished (copy stream)
    cudaEvent_t pre_free = nullptr;  // the insertion that read `pre` finished (graph stream)
    const void *pre_src = nullptr, *pre_dst = nullptr, *pre_cost = nullptr;
    int64_t pre_n = -1;              // edges of the pending prefetch; -1 = none
    int num_sms = 0;
    int64_t cap_n = 0, cap_e = 0;  // vertices, directed CSR entries
    int64_t n = 0, m = 0;
    size_t entry_bytes = 0, cost_bytes = 0;
    int cur = 0;                   // live CSR pool
    RowExt *rows = nullptr;        // row extents in the live pool
    void *adj[2] = {nullptr, nullptr};  // pools; the second is allocated on the first repack
    int64_t pool_cap = 0;          // entries per pool
    int64_t pool_used = 0;         // entries taken in the live pool (rows, slack, moved-out)
    int32_t *ralloc = nullptr;     // insertion: pool space per row
    int32_t *touched = nullptr;    // insertion: old rows gaining entries
    int64_t *roff = nullptr;       // insertion / export: exclusive scan
    unsigned long long copied_seen = 0;
    int64_t *hx = nullptr;         // pinned host scalars read back by insertion
    double *g = nullptr;
    float *g32 = nullptr;  // FP32 shadow of g for candidate screening
    int32_t *p = nullptr;
    void *pc = nullptr;
    int32_t *deg = nullptr;
    long long *tile_sums = nullptr;
    unsigned *stamp = nullptr;
    int32_t *list[2] = {nullptr, nullptr};
    int32_t *switched = nullptr;
    int32_t *dg = nullptr;
    int32_t *anc[2] = {nullptr, nullptr};
    double *acc[2] = {nullptr, nullptr};
    longlong2 *wx[2] = {nullptr, nullptr};  // wave lists: row extent and depth of each entry
    int32_t *done = nullptr;
    int32_t *wl[2] = {nullptr, nullptr};  // jump work lists; also the wave's level lists
    unsigned *wstamp = nullptr;           // first-change stamps of an Evaluate
    unsigned *swstamp = nullptr;          // barrier-free Evaluate: switched-vertex stamps
    unsigned long long *cand = nullptr;   // candidate offers for the next Improve
    AsyncQueue *aq = nullptr;             // barrier-free Evaluate: walk state
    AsyncItem *aring = nullptr;           // barrier-free Evaluate: spill list
    int async_dirty = 0;                  // an exploit failed: reset the walk state first
    int32_t *pexport = nullptr;           // parents as reported (root marker -> -1)
    int deep_hint = 0;                    // AUTO: recent exploits met waves past the cap
    float *h = nullptr;                   // goal-directed Replan: heuristic h(v), cap_n entries
    int32_t goal = -1;                    // x_goal; -1 = goal-free
    int stale = 0;        // an exploit pruned subtrees: some g below them are not up to date
    int goal_dirty = 0;   // the goal or h changed since the last exploit
    int recover = 0;      // an exploit stopped on a device timeout: re-evaluate first
    int exploits = 0;
    DevCounters *ctr = nullptr;
    DevCounters *ctr_host = nullptr;  // pinned mirror
    unsigned char *dargs = nullptr;   // device copies of the kernel argument structs
    unsigned char *hargs = nullptr;   // pinned host staging of the same
    cudaEvent_t args_ev = nullptr;    // the last copy of the staging was consumed
    int args_pending = 0;
    struct ArgsKey {
        int64_t n = -1;
        int cur = -1;
        unsigned dense_limit = 0, max_levels = 0;
        int push = -1;
        unsigned tail_max = 0, local_levels = 0, local_max = 0, local_step = 0;
        const float *h = nullptr;
        bool operator==(const ArgsKey &o) const {
            return n == o.n && cur == o.cur && dense_limit == o.dense_limit &&
                   max_levels == o.max_levels && push == o.push && tail_max == o.tail_max &&
                   local_levels == o.local_levels && local_max == o.local_max &&
                   local_step == o.local_step && h == o.h;
        }
    } args_key;
    std::map<unsigned long long, cudaGraphExec_t> loops;  // captured Replan loops
    void *stage = nullptr;            // device staging for host-side inputs
    size_t stage_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int eval_blocks = 0;
    int wave_blocks = 0;                  // grid of the wave for the current exploit
    int wave_occ = 0;                     // CTAs per SM the wave can keep resident (<= 2)
    int async_blocks = 0;
    int profiling = 0;
    pirrt_profile prof{};
    std::vector<pirrt_trace_record> trace;
    cudaEvent_t it_start = nullptr;
    cudaEvent_t pev[8] = {};          // improve, evaluate, mark, insert: (start, end) pairs
    std::string last_error;
};

namespace {

pirrt_status fail(pirrt_graph *G, pirrt_status s, const char *fmt, ...) {
    if (G) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        G->last_error = buf;
    }
    return s;
}

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t err_ = (call);                                                           \
        if (err_ != cudaSuccess)                                                             \
            return fail(G, err_ == cudaErrorMemoryAllocation ? PIRRT_ERR_OOM : PIRRT_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(err_), __FILE__, __LINE__); \
    } while (0)

#define CKL()  CK(cudaGetLastError())

int grid_for(int64_t work, int threads, int max_blocks) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

pirrt_status status_from_bits(pirrt_graph *G, unsigned bits) {
    if (bits & kStatusTimeout) return fail(G, PIRRT_ERR_DEVICE_TIMEOUT, "grid barrier timed out");
    if (bits & kStatusBadTree) return fail(G, PIRRT_ERR_BAD_TREE, "parent pointers contain a cycle");
    if (bits & kStatusBadInput) return fail(G, PIRRT_ERR_BAD_INPUT, "invalid input rejected on device");
    return PIRRT_OK;
}

// Read the counter block back (synchronises the stream).
pirrt_status pull_counters(pirrt_graph *G) {
    CK(cudaMemcpyAsync(G->ctr_host, G->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

pirrt_status ensure_stage(pirrt_graph *G, size_t bytes) {
    if (bytes <= G->stage_bytes) return PIRRT_OK;
    if (G->stage) {
        CK(cudaStreamSynchronize(G->stream));
        CK(cudaFree(G->stage));
        G->stage = nullptr;
        G->stage_bytes = 0;
    }
    CK(cudaMalloc(&G->stage, bytes));
    G->stage_bytes = bytes;
    return PIRRT_OK;
}

// Write every kernel argument struct of the exploit path into the device
// argument block (stream-ordered; skipped when nothing changed).
template <typename CT>
pirrt_status write_args(pirrt_graph *G, unsigned dense_limit, unsigned max_levels, int push,
                        unsigned tail_max, unsigned local_levels = 0, unsigned local_max = 0,
                        unsigned local_step = 0) {
    pirrt_graph::ArgsKey key;
    key.n = G->n;
    key.cur = G->cur;
    key.dense_limit = dense_limit;
    key.max_levels = max_levels;
    key.push = push;
    key.tail_max = tail_max;
    key.local_levels = local_levels;
    key.local_max = local_max;
    key.local_step = local_step;
    key.h = G->goal >= 0 ? G->h : nullptr;
    if (key == G->args_key) return PIRRT_OK;
    // the pinned staging is rewritten only after its last copy has been
    // consumed (long done by now: every exploit ends with a synchronisation)
    if (G->args_pending) CK(cudaEventSynchronize(G->args_ev));
    std::memset(G->hargs, 0, kArgBytes);
    const Entry<CT> *adj = static_cast<const Entry<CT> *>(G->adj[G->cur]);
    auto *ia = reinterpret_cast<ImproveArgs<CT> *>(G->hargs + kArgImprove);
    ia->rows = G->rows;
    ia->adj = adj;
    ia->g = G->g;
    ia->g32 = G->g32;
    ia->p = G->p;
    ia->pc = static_cast<CT *>(G->pc);
    ia->list[0] = G->list[0];
    ia->list[1] = G->list[1];
    ia->switched = G->switched;
    ia->ctr = G->ctr;
    ia->n = G->n;
    ia->root = G->cfg.root;
    ia->push = push;
    ia->cand = G->cand;
    ia->h = key.h;
    for (size_t off : {kArgEval, kArgEvalFallback, kArgEvalForce}) {
        auto *ea = reinterpret_cast<EvaluateArgs<CT> *>(G->hargs + off);
        ea->p = G->p;
        ea->pc = static_cast<const CT *>(G->pc);
        ea->g = G->g;
        ea->g32 = G->g32;
        ea->anc[0] = G->anc[0];
        ea->anc[1] = G->anc[1];
        ea->acc[0] = G->acc[0];
        ea->acc[1] = G->acc[1];
        ea->done = G->done;
        ea->wl[0] = G->wl[0];
        ea->wl[1] = G->wl[1];
        ea->dg = G->dg;
        ea->ctr = G->ctr;
        ea->n = G->n;
        ea->root = G->cfg.root;
        ea->force = off == kArgEvalForce ? 1 : 0;
        ea->role = off == kArgEvalFallback ? 1 : 0;
    }
    auto *wa = reinterpret_cast<WaveArgs<CT> *>(G->hargs + kArgWave);
    wa->rows = G->rows;
    wa->adj = adj;
    wa->p = G->p;
    wa->pc = static_cast<const CT *>(G->pc);
    wa->g = G->g;
    wa->g32 = G->g32;
    wa->switched = G->switched;
    wa->lvl[0] = G->wl[0];
    wa->lvl[1] = G->wl[1];
    wa->lvg[0] = G->acc[0];
    wa->lvg[1] = G->acc[1];
    wa->lvx[0] = G->wx[0];
    wa->lvx[1] = G->wx[1];
    wa->dg = G->dg;
    wa->list_cap = G->cap_n;
    wa->tail_max = tail_max;
    wa->local_levels = local_levels;
    wa->local_max = local_max;
    wa->local_step = local_step;
    wa->wstamp = G->wstamp;
    wa->stamp = G->stamp;
    wa->list[0] = G->list[0];
    wa->list[1] = G->list[1];
    wa->ctr = G->ctr;
    wa->root = G->cfg.root;
    wa->dense_limit = dense_limit;
    wa->max_levels = max_levels;
    wa->push = push;
    wa->cand = G->cand;
    wa->h = key.h;
    wa->n = G->n;
    auto *aa = reinterpret_cast<AsyncArgs<CT> *>(G->hargs + kArgAsync);
    aa->rows = G->rows;
    aa->adj = adj;
    aa->p = G->p;
    aa->pc = static_cast<const CT *>(G->pc);
    aa->g = G->g;
    aa->g32 = G->g32;
    aa->switched = G->switched;
    aa->dg = G->dg;
    aa->wstamp = G->wstamp;
    aa->swstamp = G->swstamp;
    aa->stamp = G->stamp;
    aa->list[0] = G->list[0];
    aa->list[1] = G->list[1];
    aa->ctr = G->ctr;
    aa->q = G->aq;
    aa->ring = G->aring;
    aa->ring_cap = G->cap_n;
    aa->root = G->cfg.root;
    aa->dense_limit = dense_limit;
    aa->max_levels = max_levels;
    aa->push = push;
    aa->cand = G->cand;
    for (size_t off : {kArgMark, kArgMarkFallback}) {
        auto *ma = reinterpret_cast<MarkArgs<CT> *>(G->hargs + off);
        ma->rows = G->rows;
        ma->adj = adj;
        ma->dg = G->dg;
        ma->stamp = G->stamp;
        ma->list[0] = G->list[0];
        ma->list[1] = G->list[1];
        ma->ctr = G->ctr;
        ma->root = G->cfg.root;
        ma->dense_limit = dense_limit;
        ma->role = off == kArgMarkFallback ? 1 : 0;
        ma->push = push;
        ma->g = G->g;
        ma->cand = G->cand;
    }
    CK(cudaMemcpyAsync(G->dargs, G->hargs, kArgBytes, cudaMemcpyHostToDevice, G->stream));
    CK(cudaEventRecord(G->args_ev, G->stream));
    G->args_pending = 1;
    G->args_key = key;
    return PIRRT_OK;
}

template <typename A>
const A *dev_arg(pirrt_graph *G, size_t off) {
    return reinterpret_cast<const A *>(G->dargs + off);
}

template <typename CT>
pirrt_status reevaluate_impl(pirrt_graph *G);

// Cooperative launch (all CTAs co-resident for the grid barrier); works on a
// capturing stream as well.
template <typename A>
pirrt_status launch_coop(pirrt_graph *G, cudaStream_t st, void (*kernel)(const A *), int blocks,
                         int threads, const A *arg) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, kernel, arg));
    return PIRRT_OK;
}

template <typename CT>
pirrt_status launch_improve_tma(pirrt_graph *G, cudaStream_t st) {
    static int occ = -1;
    const size_t smem = sizeof(tma::Smem<CT>);
    if (occ < 0) {
        CK(cudaFuncSetAttribute(improve_tma_kernel<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
        int nb = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, improve_tma_kernel<CT>, tma::kThreads,
                                                         smem));
        occ = nb > 0 ? nb : 1;
    }
    improve_tma_kernel<CT><<<G->num_sms * occ, tma::kThreads, smem, st>>>(
        dev_arg<ImproveArgs<CT>>(G, kArgImprove));
    CKL();
    return PIRRT_OK;
}

template <typename CT, int GS>
pirrt_status launch_improve_g(pirrt_graph *G, cudaStream_t st) {
    static int occ = -1;
    if (occ < 0) {
        int nb = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, improve_kernel<CT, GS>, kThreads, 0));
        occ = nb > 0 ? nb : 1;
    }
    improve_kernel<CT, GS><<<G->num_sms * occ, kThreads, 0, st>>>(
        dev_arg<ImproveArgs<CT>>(G, kArgImprove));
    CKL();
    return PIRRT_OK;
}

template <int GS, int U>
pirrt_status launch_improve_screen(pirrt_graph *G, cudaStream_t st) {
    static int occ = -1;
    if (occ < 0) {
        int nb = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, improve_screen_kernel<GS, U>, 256, 0));
        occ = nb > 0 ? nb : 1;
    }
    improve_screen_kernel<GS, U><<<G->num_sms * occ, 256, 0, st>>>(
        dev_arg<ImproveArgs<float>>(G, kArgImprove));
    CKL();
    return PIRRT_OK;
}

template <typename CT>
pirrt_status launch_improve_push(pirrt_graph *G, cudaStream_t st) {
    static int occ = -1;
    if (occ < 0) {
        int nb = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, improve_push_kernel<CT, 8>, 256, 0));
        occ = nb > 0 ? nb : 1;
    }
    improve_push_kernel<CT, 8><<<G->num_sms * occ, 256, 0, st>>>(
        dev_arg<ImproveArgs<CT>>(G, kArgImprove));
    CKL();
    return PIRRT_OK;
}

// Improve kernel selection (pirrt_exploit_opts.tile / .group):
//   tile 0  list sweeps from candidate offers (improve_push_kernel), dense
//           sweeps by the tile-2 kernel (which returns at once otherwise)
//   tile 2  G lanes per vertex (group, default 4) with FP32 screening; FP64
//           costs use the exact G-lane kernel
//   tile 1  staged: producer warp bulk-copies rows into a shared-memory ring
//   tile 3  G lanes per vertex (default 8), exact FP64 for every candidate
// with_push = false: tile 0 launches only its dense-sweep kernel (the offer
// Improve then runs inside the wave's launch).
template <typename CT>
pirrt_status launch_improve(pirrt_graph *G, cudaStream_t st, int gs, int tile,
                            bool with_push = true) {
    if (tile == 0) {
        if (with_push) {
            pirrt_status rc = launch_improve_push<CT>(G, st);
            if (rc) return rc;
        }
        tile = 2;
    }
    if (tile == 2) {
        if constexpr (sizeof(CT) == 4) {
            switch (gs) {
                case 2: return launch_improve_screen<2, 8>(G, st);
                case 8: return launch_improve_screen<8, 4>(G, st);
                case 16: return launch_improve_screen<16, 4>(G, st);
                case 32: return launch_improve_screen<32, 4>(G, st);
                default: return launch_improve_screen<4, 4>(G, st);
            }
        }
        tile = 3;
    }
    if (tile == 1) return launch_improve_tma<CT>(G, st);
    switch (gs) {
        case 4: return launch_improve_g<CT, 4>(G, st);
        case 16: return launch_improve_g<CT, 16>(G, st);
        case 32: return launch_improve_g<CT, 32>(G, st);
        default: return launch_improve_g<CT, 8>(G, st);
    }
}

template <typename CT>
pirrt_status launch_evaluate(pirrt_graph *G, cudaStream_t st, size_t off) {
    return launch_coop<EvaluateArgs<CT>>(G, st, evaluate_kernel<CT>, G->eval_blocks, kThreads,
                                         dev_arg<EvaluateArgs<CT>>(G, off));
}

// The wave and the rest of the iteration (pointer-jumping finish, marking,
// advance) in one cooperative launch, with the offer Improve in front of it
// when fused_improve is set.
template <typename CT>
pirrt_status launch_wave(pirrt_graph *G, cudaStream_t st, cudaGraphConditionalHandle cond,
                         int use_cond, bool fused_improve = false, bool fuse_dense = false) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(G->wave_blocks);
    cfg.blockDim = dim3(kWaveThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const ImproveArgs<CT> *ip = fused_improve ? dev_arg<ImproveArgs<CT>>(G, kArgImprove) : nullptr;
    CK(cudaLaunchKernelEx(&cfg, wave_evaluate_kernel<CT>, dev_arg<WaveArgs<CT>>(G, kArgWave),
                          dev_arg<EvaluateArgs<CT>>(G, kArgEvalFallback),
                          dev_arg<MarkArgs<CT>>(G, kArgMarkFallback), ip, cond, use_cond,
                          fuse_dense ? 1 : 0));
    return PIRRT_OK;
}

// A captured iteration with offers whose dense sweeps run inside the wave's
// launch too (FP32 costs, the default 4 lanes): one launch per iteration.
bool fuses_dense(int cost_dtype, int tile, int gs) {
    return cost_dtype == PIRRT_COST_F32 && tile == 0 && (gs == 0 || gs == 4);
}

// Kernel launches of one Replan iteration (host loop; a captured wave
// iteration with offers runs the offer Improve inside the wave's launch, and
// with FP32 costs the dense sweep as well).
int iteration_launches(int tile, bool jump, bool async, bool graph, bool fused_dense = false) {
    const int improve = tile == 0 ? 2 : 1;
    if (jump) return improve + 3;
    if (async) return improve + 5;
    if (graph && tile == 0) return fused_dense ? 1 : 2;
    return improve + 1;
}

constexpr size_t kAsyncSmem = (size_t)kAsyncLocal * (sizeof(double) + 2 * sizeof(int32_t));

template <typename CT>
pirrt_status launch_async(pirrt_graph *G, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(G->async_blocks);
    cfg.blockDim = dim3(kAsyncThreads);
    cfg.dynamicSmemBytes = kAsyncSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, async_evaluate_kernel<CT>, dev_arg<AsyncArgs<CT>>(G, kArgAsync)));
    return PIRRT_OK;
}

template <typename CT>
pirrt_status launch_mark(pirrt_graph *G, cudaStream_t st, size_t off) {
    mark_frontier_kernel<CT><<<G->num_sms * 8, kThreads, 0, st>>>(dev_arg<MarkArgs<CT>>(G, off));
    CKL();
    return PIRRT_OK;
}

// One Replan iteration after Improve: the Evaluate strategy, then advance.
// JUMP: pointer jumping + marking + advance.  WAVE / AUTO: one launch (the
// wave ends the iteration itself, see wave_evaluate_kernel).  ASYNC: the
// walk, then a pointer-jumping finish and its marking, both no-ops unless
// the walk gave up, then advance.
template <typename CT>
pirrt_status launch_iteration(pirrt_graph *G, cudaStream_t st, int gs, int tile, bool jump,
                              bool async, cudaGraphConditionalHandle cond, int use_cond) {
    pirrt_status rc;
    if (!jump && !async && tile == 0) {
        // the dense-sweep kernel, then Improve from offers and the wave in one
        // launch; with FP32 costs that launch also runs the dense sweeps
        if (fuses_dense(G->cfg.cost_dtype, tile, gs))
            return launch_wave<CT>(G, st, cond, use_cond, true, true);
        if ((rc = launch_improve<CT>(G, st, gs, tile, false))) return rc;
        return launch_wave<CT>(G, st, cond, use_cond, true);
    }
    if ((rc = launch_improve<CT>(G, st, gs, tile))) return rc;
    if (!jump && !async) return launch_wave<CT>(G, st, cond, use_cond);
    if (jump) {
        if ((rc = launch_evaluate<CT>(G, st, kArgEval))) return rc;
        if ((rc = launch_mark<CT>(G, st, kArgMark))) return rc;
    } else {
        if ((rc = launch_async<CT>(G, st))) return rc;
        pre_jump_kernel<<<1, 1, 0, st>>>(G->ctr);
        CKL();
        if ((rc = launch_evaluate<CT>(G, st, kArgEvalFallback))) return rc;
        if ((rc = launch_mark<CT>(G, st, kArgMarkFallback))) return rc;
    }
    advance_kernel<<<1, 1, 0, st>>>(G->ctr, cond, use_cond);
    CKL();
    return PIRRT_OK;
}

// The Replan loop as a CUDA graph: a WHILE conditional node whose body is one
// iteration; advance_kernel sets the condition.  Cached per kernel choice.
template <typename CT>
pirrt_status get_loop(pirrt_graph *G, int gs, int tile, bool jump, bool async, int wave_ctas,
                      cudaGraphExec_t *out) {
    const unsigned long long key = ((unsigned long long)gs << 8) | ((unsigned long long)tile << 1) |
                                   (jump ? 1ull : 0ull) | ((unsigned long long)sizeof(CT) << 24) |
                                   (async ? 1ull << 32 : 0ull) |
                                   ((unsigned long long)wave_ctas << 40);
    auto it = G->loops.find(key);
    if (it != G->loops.end()) {
        *out = it->second;
        return PIRRT_OK;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(G->capture, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeRelaxed));
    pirrt_status rc = launch_iteration<CT>(G, G->capture, gs, tile, jump, async, cond, 1);
    cudaGraph_t captured = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(G->capture, &captured);
    if (rc) {
        cudaGraphDestroy(graph);
        return rc;
    }
    if (ec != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(G, PIRRT_ERR_CUDA, "capturing the Replan loop: %s", cudaGetErrorString(ec));
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess)
        return fail(G, PIRRT_ERR_CUDA, "instantiating the Replan loop: %s", cudaGetErrorString(ei));
    G->loops[key] = exec;
    *out = exec;
    return PIRRT_OK;
}

// Pool space of every row for an insertion (ralloc), and its exclusive scan
// (roff; roff[n_after] = the total).
pirrt_status insert_plan_scan(pirrt_graph *G, int64_t n_old, int64_t n_after, int repack) {
    const int64_t len = n_after + 1;
    insert_plan<<<grid_for(len, kThreads, G->num_sms * 32), kThreads, 0, G->stream>>>(
        n_old, n_after, G->rows, G->deg, G->ralloc, repack);
    CKL();
    const int64_t n_tiles = (len + kScanTile - 1) / kScanTile;
    scan_tile_reduce<<<(unsigned)n_tiles, kThreads, 0, G->stream>>>(G->ralloc, len, G->tile_sums);
    CKL();
    scan_tile_sums<<<1, kThreads, 0, G->stream>>>(G->tile_sums, n_tiles);
    CKL();
    scan_tile_apply<<<(unsigned)n_tiles, kThreads, 0, G->stream>>>(G->ralloc, len, G->tile_sums,
                                                                    G->roff);
    CKL();
    return PIRRT_OK;
}

template <typename CT>
pirrt_status insert_impl(pirrt_graph *G, int64_t n_new, int64_t n_edges, const int32_t *src,
                         const int32_t *dst, const CT *cost) {
    const int64_t n_old = G->n, n_after = G->n + n_new;
    const int64_t m_after = G->m + 2 * n_edges;
    const int max_blocks = G->num_sms * 32;
    const bool prof = G->profiling != 0;
    if (prof) CK(cudaEventRecord(G->pev[6], G->stream));
    // 1. validate and count new entries per row (deg is all zero between
    //    insertions: the scatter below takes every count back); the old rows
    //    gaining entries form the touched list
    insert_begin_kernel<<<1, 1, 0, G->stream>>>(G->ctr);
    CKL();
    if (n_edges > 0) {
        insert_validate_count<CT><<<grid_for(n_edges, kThreads, max_blocks), kThreads, 0, G->stream>>>(
            n_edges, src, dst, cost, n_old, n_after, G->deg, G->touched, G->ctr);
        CKL();
    }
    // 2. room at the end of the pool for the changed rows that would overflow,
    //    from a cursor (no scan over every row); one host read of the
    //    validation status and the room taken
    const int64_t changed_max = std::min<int64_t>(2 * n_edges, n_old) + n_new;
    if (changed_max > 0) {
        insert_plan_list<<<grid_for(changed_max, kThreads, max_blocks), kThreads, 0, G->stream>>>(
            n_old, n_after, G->touched, G->rows, G->deg, G->ralloc, G->roff, G->ctr);
        CKL();
    }
    CK(cudaMemcpyAsync(&G->ctr_host->status, &G->ctr->status, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, G->stream));
    CK(cudaMemcpyAsync(G->hx, &G->ctr->pool_cursor, sizeof(int64_t), cudaMemcpyDeviceToHost,
                       G->stream));
    CK(cudaStreamSynchronize(G->stream));
    if (G->ctr_host->status) {
        CK(cudaMemsetAsync(&G->ctr->status, 0, sizeof(unsigned), G->stream));
        CK(cudaMemsetAsync(G->deg, 0, sizeof(int32_t) * (size_t)(n_after + 1), G->stream));
        return fail(G, PIRRT_ERR_BAD_INPUT,
                    "insert_batch: edge with an id outside [0, %lld), a self loop, or a cost "
                    "that is not finite and > 0",
                    (long long)n_after);
    }
    const int64_t need = G->hx[0];
    // 3. move those rows to the end of the pool, or repack every row into the
    //    other pool when this one is used up; set every changed row's new length
    if (G->pool_used + need <= G->pool_cap) {
        if (changed_max > 0) {
            Entry<CT> *pool = static_cast<Entry<CT> *>(G->adj[G->cur]);
            insert_move_list<CT><<<grid_for((changed_max + 31) / 32 * 32, kThreads, max_blocks),
                                   kThreads, 0, G->stream>>>(
                n_old, n_after, G->touched, G->rows, G->deg, G->ralloc, G->roff,
                (long long)G->pool_used, pool, G->ctr);
            CKL();
        }
        G->pool_used += need;
    } else {
        const int move_blocks = grid_for((n_after + 31) / 32 * 32, kThreads, max_blocks);
        const int nxt = G->cur ^ 1;
        if (!G->adj[nxt]) {
            const cudaError_t e =
                cudaMalloc(&G->adj[nxt], G->entry_bytes * (size_t)(G->pool_cap + 16));
            if (e != cudaSuccess) {
                cudaGetLastError();
                G->adj[nxt] = nullptr;
                CK(cudaMemsetAsync(G->deg, 0, sizeof(int32_t) * (size_t)(n_after + 1), G->stream));
                return fail(G, PIRRT_ERR_OOM, "insert_batch: no memory for a second CSR pool");
            }
        }
        if (const pirrt_status rc = insert_plan_scan(G, n_old, n_after, 1)) return rc;
        CK(cudaMemcpyAsync(G->hx, &G->roff[n_after], sizeof(int64_t), cudaMemcpyDeviceToHost,
                           G->stream));
        CK(cudaStreamSynchronize(G->stream));
        const int64_t total = G->hx[0];
        if (total > G->pool_cap) {
            CK(cudaMemsetAsync(G->deg, 0, sizeof(int32_t) * (size_t)(n_after + 1), G->stream));
            return fail(G, PIRRT_ERR_CAPACITY, "insert_batch: repacked CSR needs %lld entries",
                        (long long)total);
        }
        insert_move_rows<CT><<<move_blocks, kThreads, 0, G->stream>>>(
            n_old, n_after, G->rows, G->deg, G->ralloc, G->roff, 0ll,
            static_cast<const Entry<CT> *>(G->adj[G->cur]), static_cast<Entry<CT> *>(G->adj[nxt]),
            G->ctr, 1);
        CKL();
        G->cur = nxt;
        G->pool_used = total;
        G->prof.launches += 4;
    }
    Entry<CT> *new_adj = static_cast<Entry<CT> *>(G->adj[G->cur]);
    // 4. seed the new vertices (before the scatter, whose offers may reach them)
    if (n_new > 0) {
        insert_init_vertices<CT><<<grid_for(n_new, kThreads, max_blocks), kThreads, 0, G->stream>>>(
            n_old, n_after, G->cfg.root, G->g, G->g32, G->p, static_cast<CT *>(G->pc), G->cand,
            G->stamp, G->list[0], G->list[1], G->ctr);
        CKL();
    }
    // 5. new entries at the row tails
    if (n_edges > 0) {
        insert_scatter<CT><<<grid_for(n_edges, kThreads, max_blocks), kThreads, 0, G->stream>>>(
            n_edges, src, dst, cost, G->rows, G->deg, new_adj, G->stamp, G->cfg.root,
            G->list[0], G->list[1], G->g, G->cand, G->ctr);
        CKL();
    }
    G->prof.launches += 1 + (n_edges > 0 ? 2 : 0) + (changed_max > 0 ? 2 : 0) + (n_new > 0 ? 1 : 0);
    G->prof.insert_calls += 1;
    G->prof.insert_new_entries += 2 * n_edges;
    if (prof) {
        CK(cudaEventRecord(G->pev[7], G->stream));
        CK(cudaEventSynchronize(G->pev[7]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, G->pev[6], G->pev[7]));
        G->prof.insert_ms += ms;
        unsigned long long copied = 0;
        CK(cudaMemcpy(&copied, &G->ctr->insert_copied, sizeof(copied), cudaMemcpyDeviceToHost));
        G->prof.insert_copied_entries += (int64_t)(copied - G->copied_seen);
        G->copied_seen = copied;
    }
    G->n = n_after;
    G->m = m_after;
    return PIRRT_OK;
}

template <typename CT>
pirrt_status exploit_impl(pirrt_graph *G, const pirrt_exploit_opts *opts, pirrt_exploit_stats *st) {
    pirrt_exploit_opts o{};
    if (opts) o = *opts;
    if (o.max_iters < 0 || o.eps < 0.0 || o.dense_fraction < 0.0 || o.dense_fraction > 1.0 ||
        o.wave_levels < 0 || o.evaluate < PIRRT_EVAL_AUTO || o.evaluate > PIRRT_EVAL_ASYNC ||
        !(o.tile == 0 || o.tile == 1 || o.tile == 2 || o.tile == 3) ||
        !(o.group == 0 || o.group == 2 || o.group == 4 || o.group == 8 || o.group == 16 ||
          o.group == 32) ||
        o.wave_ctas < 0 || o.wave_ctas > 2 || o.wave_local_max < 0 || o.wave_local_max > 512 ||
        o.wave_local_step < 0)
        return fail(G, PIRRT_ERR_INVALID_ARG, "exploit: invalid option");
    if (G->recover) {
        // the last exploit stopped on a device timeout part-way through an
        // iteration: clear the status word and rebuild g from the policy
        // (every vertex), so that the next Improve starts from a consistent
        // state and sweeps every vertex
        CK(cudaMemsetAsync(&G->ctr->status, 0, sizeof(unsigned), G->stream));
        const pirrt_status rr = reevaluate_impl<CT>(G);
        if (rr) return rr;
        G->recover = 0;
    }
    if (G->stale && G->goal_dirty) {
        // subtrees pruned for the previous goal or h: bring every g up to date
        const pirrt_status rr = reevaluate_impl<CT>(G);
        if (rr) return rr;
    }
    G->goal_dirty = 0;
    if (G->goal >= 0) G->stale = 1;
    const int64_t max_iters = o.max_iters > 0 ? o.max_iters : G->n + 2;
    const int gs = o.group, tile = o.tile;
    const double frac = o.dense_fraction > 0.0 ? o.dense_fraction : 0.35;
    const unsigned dense_limit = (unsigned)std::min<double>(4.0e9, frac * (double)G->n);
    const int mode = o.evaluate;
    // A wave deeper than the cap hands over to pointer jumping (AUTO); a WAVE
    // run is only capped at |V| + 2 levels, beyond which the tree has a cycle.
    // The default cap balances a wave (~levels x one grid step) against one
    // pointer-jumping Evaluate (~log2(depth) sweeps over every vertex), whose
    // cost grows with |V|.
    const unsigned cap_any = (unsigned)std::min<int64_t>(G->n + 2, 0x7fffffff);
    unsigned auto_cap = 24u;
    if (G->n > 1000000) {
        const double extra = 16.0 * std::log2((double)G->n / 1.0e6);
        auto_cap = (unsigned)std::min(128.0, 24.0 + extra);
    }
    // The barrier-free walk (ASYNC) is an explicit choice: on the 6-D
    // roadmaps its per-CTA subtree walks took about twice as long per
    // Evaluate as the level-synchronous wave, which spreads every level over
    // the whole grid.
    const bool async = mode == PIRRT_EVAL_ASYNC;
    const unsigned max_levels = (mode == PIRRT_EVAL_WAVE || mode == PIRRT_EVAL_ASYNC) ? cap_any
                                : (o.wave_levels > 0 ? (unsigned)o.wave_levels : auto_cap);
    // AUTO: after an exploit whose waves ran past the cap, use pointer
    // jumping; probe with a wave again every eighth exploit
    bool jump = mode == PIRRT_EVAL_JUMP ||
                (mode == PIRRT_EVAL_AUTO && G->deep_hint && (G->exploits % 8) != 0);
    G->exploits += 1;
    // one CTA walks levels of at most this many vertices (~34 CSR entries each
    // on the 6-D roadmaps, a few passes of the CTA's threads)
    const unsigned tail_max = o.wave_tail < 0 ? 0u : (o.wave_tail > 0 ? (unsigned)o.wave_tail : 64u);
    // tree levels a CTA walks on its own from the children it lowered, before
    // they join the next grid step
    // (while its local list is short: a wide subtree is shared by the grid)
    const unsigned local_levels =
        o.wave_local < 0 ? 0u : (o.wave_local > 0 ? (unsigned)o.wave_local : 32u);
    const unsigned local_max = o.wave_local_max > 0 ? (unsigned)o.wave_local_max : 128u;
    const unsigned local_step = o.wave_local_step > 0 ? (unsigned)o.wave_local_step : 4096u;
    pirrt_status rc = write_args<CT>(G, dense_limit, max_levels, tile == 0 ? 1 : 0, tail_max,
                                     local_levels, local_max, local_step);
    if (rc) return rc;
    const int wave_ctas = o.wave_ctas > 0 ? std::min(o.wave_ctas, G->wave_occ) : G->wave_occ;
    G->wave_blocks = G->num_sms * wave_ctas;
    const bool prof = G->profiling != 0;
    const bool use_graph = !prof && o.host_loop == 0;
    double eps = o.eps;
    unsigned long long eps_bits;
    std::memcpy(&eps_bits, &eps, sizeof(eps_bits));

    CK(cudaEventRecord(G->ev0, G->stream));
    if (G->async_dirty) {  // a failed walk may have left its state behind
        async_reset_kernel<<<1, 1, 0, G->stream>>>(G->aq);
        CKL();
        G->async_dirty = 0;
    }
    begin_exploit_kernel<<<1, 1, 0, G->stream>>>(
        G->ctr, (unsigned)std::min<int64_t>(max_iters, 0xffffffffll), eps_bits);
    CKL();
    // waves with offers leave the FP32 shadow of g out of date until a dense
    // sweep needs it; Improve kernels without offers and the barrier-free walk
    // read or keep it all the time, so they get it refreshed first
    {
        const int always = (tile != 0 || async) ? 1 : 0;
        refresh_g32_kernel<<<grid_for(G->n, kThreads, G->num_sms * 8), kThreads, 0, G->stream>>>(
            G->ctr, G->n, G->g, G->g32, always);
        CKL();
        refresh_g32_done<<<1, 1, 0, G->stream>>>(G->ctr, always);
        CKL();
    }
    pirrt_profile &P = G->prof;
    P.launches += 3;
    pirrt_exploit_stats s{};
    bool graph_ran = false;
    if (use_graph) {
        cudaGraphExec_t exec = nullptr;
        rc = get_loop<CT>(G, gs, tile, jump, async, wave_ctas, &exec);
        if (rc == PIRRT_OK) {
            CK(cudaGraphLaunch(exec, G->stream));
            graph_ran = true;
        } else {
            G->last_error.clear();  // fall back to the host loop
        }
    }
    if (!graph_ran) {
        unsigned long long prev_relax = 0, prev_improved = 0, prev_eval = 0, prev_offers = 0;
        for (int64_t it = 0; it < max_iters; ++it) {
            if (prof) CK(cudaEventRecord(G->pev[0], G->stream));
            if ((rc = launch_improve<CT>(G, G->stream, gs, tile))) return rc;
            if (prof) CK(cudaEventRecord(G->pev[1], G->stream));
            if (jump) {
                if ((rc = launch_evaluate<CT>(G, G->stream, kArgEval))) return rc;
                if (prof) CK(cudaEventRecord(G->pev[2], G->stream));
                if ((rc = launch_mark<CT>(G, G->stream, kArgMark))) return rc;
            } else if (async) {
                if ((rc = launch_async<CT>(G, G->stream))) return rc;
                if (prof) CK(cudaEventRecord(G->pev[2], G->stream));
                pre_jump_kernel<<<1, 1, 0, G->stream>>>(G->ctr);
                CKL();
                if ((rc = launch_evaluate<CT>(G, G->stream, kArgEvalFallback))) return rc;
                if ((rc = launch_mark<CT>(G, G->stream, kArgMarkFallback))) return rc;
            } else {
                if ((rc = launch_wave<CT>(G, G->stream, cudaGraphConditionalHandle{}, 0))) return rc;
                if (prof) CK(cudaEventRecord(G->pev[2], G->stream));
            }
            if (prof) CK(cudaEventRecord(G->pev[3], G->stream));
            if (jump || async) {
                advance_kernel<<<1, 1, 0, G->stream>>>(G->ctr, cudaGraphConditionalHandle{}, 0);
                CKL();
            }
            if ((rc = pull_counters(G))) return rc;
            P.launches += iteration_launches(tile, jump, async, false);
            const DevCounters *h = G->ctr_host;
            float t_imp = 0.f, t_eval = 0.f, t_mark = 0.f;
            if (prof) {
                CK(cudaEventElapsedTime(&t_imp, G->pev[0], G->pev[1]));
                CK(cudaEventElapsedTime(&t_eval, G->pev[1], G->pev[2]));
                CK(cudaEventElapsedTime(&t_mark, G->pev[2], G->pev[3]));
                if (!jump) {  // the pointer-jumping finish counts as Evaluate
                    t_eval += t_mark;
                    t_mark = 0.f;
                }
                pirrt_trace_record tr{};
                tr.iteration = (int32_t)it;
                tr.dense = h->last_dense ? 1 : 0;
                tr.improve_vertices = (int64_t)(h->improved - prev_improved);
                tr.improve_entries = (int64_t)(h->relax - prev_relax);
                tr.offers = (int64_t)(h->offers - prev_offers);
                tr.switches = (int32_t)h->last_switched;
                tr.changed = (int32_t)h->last_dg;
                tr.wave_levels = (int32_t)h->last_levels;
                tr.next_frontier = (int32_t)h->last_next;
                tr.improve_ms = t_imp;
                tr.evaluate_ms = t_eval;
                tr.mark_ms = t_mark;
                float t_it = 0.f;
                if (it > 0) CK(cudaEventElapsedTime(&t_it, G->it_start, G->pev[0]));
                tr.iteration_ms = t_it;
                if (G->trace.size() < (1u << 22)) G->trace.push_back(tr);
                CK(cudaEventRecord(G->it_start, G->stream));
            }
            P.improve_launches += 1;
            P.improve_entries += (int64_t)(h->relax - prev_relax);
            P.evaluate_offers += (int64_t)(h->offers - prev_offers);
            P.improve_vertices += (int64_t)(h->improved - prev_improved);
            if (h->last_dense) P.improve_dense_vertices += (int64_t)(h->improved - prev_improved);
            P.improve_switches += h->last_switched;
            P.improve_ms += t_imp;
            if (h->last_switched) {
                P.evaluate_launches += 1;
                P.evaluate_vertices += (int64_t)(h->evaluated - prev_eval);
                P.evaluate_ms += t_eval;
                if (jump && h->last_dg && h->last_dg <= dense_limit) {
                    P.mark_launches += 1;
                    P.mark_vertices += h->last_dg;
                    P.mark_ms += t_mark;
                }
            }
            prev_relax = h->relax;
            prev_offers = h->offers;
            prev_improved = h->improved;
            prev_eval = h->evaluated;
            if (h->status) break;
            // AUTO: a wave that ran past its cap -> pointer jumping from now on
            if (mode == PIRRT_EVAL_AUTO && !jump && h->last_jumped) jump = true;
            if (!h->cont) break;
        }
    }
    CK(cudaEventRecord(G->ev1, G->stream));
    if ((rc = pull_counters(G))) return rc;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, G->ev0, G->ev1));
    const DevCounters &h = *G->ctr_host;
    if (mode == PIRRT_EVAL_AUTO) {
        const bool saw_deep = h.cum_jump_evals > 0;
        if (saw_deep || !jump || (G->exploits % 8) == 1) G->deep_hint = saw_deep ? 1 : 0;
    }
    if (graph_ran)
        P.launches += (int64_t)h.iter * iteration_launches(tile, jump, async, true,
                                                            fuses_dense(G->cfg.cost_dtype, tile, gs));
    s.iterations = (int32_t)h.iter;
    s.converged = h.converged ? 1 : 0;
    s.relaxations = (int64_t)(h.relax + h.offers);
    s.improve_entries = (int64_t)h.relax;
    s.offers = (int64_t)h.offers;
    s.improved = (int64_t)h.improved;
    s.evaluated = (int64_t)h.evaluated;
    s.switches = (int64_t)h.switches;
    s.jump_rounds = (int32_t)h.cum_jump_rounds;
    s.dense_sweeps = (int32_t)h.cum_dense;
    s.wave_levels = (int32_t)h.cum_wave_levels;
    s.jump_evaluates = (int32_t)h.cum_jump_evals;
    s.ms_exploit = ms;
    s.graph_launch = graph_ran ? 1 : 0;
    if (st) *st = s;
    if (h.status & kStatusTimeout) G->recover = 1;
    if ((rc = status_from_bits(G, h.status))) return rc;
    if (!h.converged)
        return fail(G, PIRRT_ERR_NOT_CONVERGED, "exploit: %lld Improve rounds without convergence",
                    (long long)max_iters);
    return PIRRT_OK;
}

template <typename CT>
pirrt_status set_policy_impl(pirrt_graph *G, const int32_t *parent) {
    // look up into scratch (anc[0] for ids, acc[1] reinterpreted for costs)
    int32_t *tp = G->anc[0];
    CT *tc = reinterpret_cast<CT *>(G->acc[1]);
    const int blocks = grid_for(G->n, kThreads, G->num_sms * 32);
    CK(cudaMemsetAsync(&G->ctr->status, 0, sizeof(unsigned), G->stream));
    policy_lookup_kernel<CT><<<blocks, kThreads, 0, G->stream>>>(
        G->n, G->cfg.root, parent, G->rows, static_cast<const Entry<CT> *>(G->adj[G->cur]),
        tp, tc, G->ctr);
    CKL();
    CK(cudaMemcpyAsync(&G->ctr_host->status, &G->ctr->status, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    if (G->ctr_host->status) {
        CK(cudaMemsetAsync(&G->ctr->status, 0, sizeof(unsigned), G->stream));
        return fail(G, PIRRT_ERR_BAD_INPUT,
                    "set_policy: parent out of range, root with a parent, or a parent edge not in G");
    }
    policy_commit_kernel<CT><<<blocks, kThreads, 0, G->stream>>>(
        G->n, G->cfg.root, tp, tc, G->p, static_cast<CT *>(G->pc), G->g, G->g32);
    CKL();
    return reevaluate_impl<CT>(G);
}

// Evaluate the whole policy tree (pointer jumping, no pruning) and make the
// next Improve sweep every vertex: after set_policy, and in the goal-directed
// form after the goal or h changed, since subtrees pruned for the old goal
// may hold values that are not up to date.
template <typename CT>
pirrt_status reevaluate_impl(pirrt_graph *G) {
    pirrt_status rc = write_args<CT>(G, 0u, 1u, 0, 0u);
    if (rc) return rc;
    begin_exploit_kernel<<<1, 1, 0, G->stream>>>(G->ctr, 1u, 0ull);
    CKL();
    if ((rc = launch_evaluate<CT>(G, G->stream, kArgEvalForce))) return rc;
    if ((rc = pull_counters(G))) return rc;
    if ((rc = status_from_bits(G, G->ctr_host->status))) return rc;
    // the next Improve sweeps every vertex; the seeded list is moot
    begin_exploit_kernel<<<1, 1, 0, G->stream>>>(G->ctr, 1u, 0ull);
    CKL();
    const unsigned one = 1u;
    CK(cudaMemcpyAsync(&G->ctr->dense, &one, sizeof(unsigned), cudaMemcpyHostToDevice, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    G->stale = 0;
    return PIRRT_OK;
}

// Point the counter block at g(x_goal) (null without a goal) and give a goal
// not yet inserted g = +inf, so that the bound read at each iteration is
// defined.  Synchronous: the host sources live on the stack.
pirrt_status apply_goal(pirrt_graph *G) {
    const double *gg = G->goal >= 0 ? G->g + G->goal : nullptr;
    CK(cudaMemcpyAsync(&G->ctr->goal_g, &gg, sizeof(gg), cudaMemcpyHostToDevice, G->stream));
    if (G->goal >= 0 && G->goal >= G->n) {
        const double inf = HUGE_VAL;
        CK(cudaMemcpyAsync(G->g + G->goal, &inf, sizeof(double), cudaMemcpyHostToDevice,
                           G->stream));
    }
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

void free_all(pirrt_graph *G) {
    for (auto &kv : G->loops)
        if (kv.second) cudaGraphExecDestroy(kv.second);
    G->loops.clear();
    if (G->capture) cudaStreamDestroy(G->capture);
    if (G->copy) {
        cudaStreamSynchronize(G->copy);
        cudaStreamDestroy(G->copy);
    }
    if (G->pre) cudaFree(G->pre);
    if (G->pre_done) cudaEventDestroy(G->pre_done);
    if (G->pre_free) cudaEventDestroy(G->pre_free);
    if (G->hargs) cudaFreeHost(G->hargs);
    void *bufs[] = {G->dargs, G->pexport, G->rows, G->ralloc, G->touched, G->roff, G->adj[0], G->adj[1], G->g, G->g32, G->p, G->pc,
                    G->deg, G->tile_sums, G->stamp, G->list[0], G->list[1], G->switched,
                    G->dg, G->anc[0], G->anc[1], G->acc[0], G->acc[1], G->wx[0], G->wx[1], G->done, G->wl[0],
                    G->wl[1], G->wstamp, G->swstamp, G->cand, G->aq, G->aring, G->ctr, G->stage, G->h};
    for (void *q : bufs)
        if (q) cudaFree(q);
    if (G->ctr_host) cudaFreeHost(G->ctr_host);
    if (G->hx) cudaFreeHost(G->hx);
    if (G->ev0) cudaEventDestroy(G->ev0);
    if (G->ev1) cudaEventDestroy(G->ev1);
    for (cudaEvent_t e : G->pev)
        if (e) cudaEventDestroy(e);
    if (G->it_start) cudaEventDestroy(G->it_start);
    if (G->args_ev) cudaEventDestroy(G->args_ev);
}

// Snapshot of the mutable exploit state, for the autotuner's repeated trials.
struct StateSnapshot {
    void *buf = nullptr;
    size_t bytes = 0;
};

pirrt_status snapshot_io(pirrt_graph *G, StateSnapshot &S, bool save) {
    const size_t n = (size_t)G->n;
    const size_t parts[] = {8 * n, 4 * n, 4 * n, G->cost_bytes * n, 4 * n, 4 * n, 4 * n, 8 * n,
                            sizeof(DevCounters)};
    void *dev[] = {G->g, G->g32, G->p, G->pc, G->stamp, G->list[0], G->list[1], G->cand, G->ctr};
    size_t total = 0;
    for (size_t b : parts) total += (b + 255) & ~size_t(255);
    if (save && S.bytes < total) {
        if (S.buf) CK(cudaFree(S.buf));
        S.buf = nullptr;
        CK(cudaMalloc(&S.buf, total));
        S.bytes = total;
    }
    char *q = static_cast<char *>(S.buf);
    for (int i = 0; i < 9; ++i) {
        if (parts[i]) {
            if (save)
                CK(cudaMemcpyAsync(q, dev[i], parts[i], cudaMemcpyDeviceToDevice, G->stream));
            else
                CK(cudaMemcpyAsync(dev[i], q, parts[i], cudaMemcpyDeviceToDevice, G->stream));
        }
        q += (parts[i] + 255) & ~size_t(255);
    }
    return PIRRT_OK;
}

}  // namespace

struct pirrt_batch {
    pirrt_graph *G = nullptr;
    int32_t n_graphs = 0;
    std::vector<int64_t> base, cap_v, cap_e, staged_e;
    std::vector<int32_t> groots;  // roots in union ids
    int32_t *pend_src = nullptr, *pend_dst = nullptr;
    void *pend_cost = nullptr;
    int64_t pend_n = 0, pend_cap = 0;
};

namespace {

pirrt_status batch_flush(pirrt_batch *B) {
    pirrt_graph *G = B->G;
    if (B->pend_n == 0) return PIRRT_OK;
    pirrt_status rc;
    if (G->cfg.cost_dtype == PIRRT_COST_F32)
        rc = insert_impl<float>(G, 0, B->pend_n, B->pend_src, B->pend_dst,
                                static_cast<const float *>(B->pend_cost));
    else
        rc = insert_impl<double>(G, 0, B->pend_n, B->pend_src, B->pend_dst,
                                 static_cast<const double *>(B->pend_cost));
    if (rc == PIRRT_OK) B->pend_n = 0;
    return rc;
}

template <typename CT>
pirrt_status batch_translate(pirrt_batch *B, int32_t graph, int64_t n_edges, const int32_t *src,
                             const int32_t *dst, const CT *cost) {
    pirrt_graph *G = B->G;
    CK(cudaMemsetAsync(&G->ctr->status, 0, sizeof(unsigned), G->stream));
    batch_translate_kernel<CT><<<grid_for(n_edges, kThreads, G->num_sms * 32), kThreads, 0,
                                 G->stream>>>(
        n_edges, src, dst, cost, B->base[graph], B->cap_v[graph], B->pend_src + B->pend_n,
        B->pend_dst + B->pend_n, static_cast<CT *>(B->pend_cost) + B->pend_n, G->ctr);
    CKL();
    CK(cudaMemcpyAsync(&G->ctr_host->status, &G->ctr->status, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    if (G->ctr_host->status) {
        CK(cudaMemsetAsync(&G->ctr->status, 0, sizeof(unsigned), G->stream));
        return fail(G, PIRRT_ERR_BAD_INPUT, "batch_insert: an id outside [0, %lld) of graph %d",
                    (long long)B->cap_v[graph], graph);
    }
    B->pend_n += n_edges;
    B->staged_e[graph] += n_edges;
    return PIRRT_OK;
}

}  // namespace

extern "C" {

const char *pirrt_status_string(pirrt_status s) {
    switch (s) {
        case PIRRT_OK: return "PIRRT_OK";
        case PIRRT_ERR_INVALID_ARG: return "PIRRT_ERR_INVALID_ARG";
        case PIRRT_ERR_CAPACITY: return "PIRRT_ERR_CAPACITY";
        case PIRRT_ERR_OOM: return "PIRRT_ERR_OOM";
        case PIRRT_ERR_CUDA: return "PIRRT_ERR_CUDA";
        case PIRRT_ERR_NOT_CONVERGED: return "PIRRT_ERR_NOT_CONVERGED";
        case PIRRT_ERR_DEVICE_TIMEOUT: return "PIRRT_ERR_DEVICE_TIMEOUT";
        case PIRRT_ERR_BAD_INPUT: return "PIRRT_ERR_BAD_INPUT";
        case PIRRT_ERR_BAD_TREE: return "PIRRT_ERR_BAD_TREE";
    }
    return "PIRRT_UNKNOWN_STATUS";
}

const char *pirrt_graph_last_error(const pirrt_graph *G) { return G ? G->last_error.c_str() : ""; }

int64_t pirrt_graph_num_vertices(const pirrt_graph *G) { return G ? G->n : -1; }

int64_t pirrt_graph_num_entries(const pirrt_graph *G) { return G ? G->m : -1; }

void pirrt_graph_destroy(pirrt_graph *G) {
    if (!G) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(G->cfg.device);
    if (G->stream) cudaStreamSynchronize(G->stream);
    free_all(G);
    cudaSetDevice(prev);
    delete G;
}

pirrt_status pirrt_graph_create(const pirrt_config *cfg, pirrt_graph **out) {
    if (!out) return PIRRT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || cfg->max_vertices <= 0 || cfg->max_vertices > INT32_MAX - 1 || cfg->max_edges < 0 ||
        cfg->root < 0 || cfg->root >= cfg->max_vertices ||
        (cfg->cost_dtype != PIRRT_COST_F32 && cfg->cost_dtype != PIRRT_COST_F64))
        return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = new (std::nothrow) pirrt_graph();
    if (!G) return PIRRT_ERR_OOM;
    G->cfg = *cfg;
    G->stream = static_cast<cudaStream_t>(cfg->stream);
    G->cap_n = cfg->max_vertices;
    G->cap_e = 2 * cfg->max_edges;
    G->entry_bytes = cfg->cost_dtype == PIRRT_COST_F32 ? sizeof(Entry<float>) : sizeof(Entry<double>);
    G->cost_bytes = cfg->cost_dtype == PIRRT_COST_F32 ? sizeof(float) : sizeof(double);
    auto bail = [&](pirrt_status s) {
        free_all(G);
        delete G;
        return s;
    };
    if (cudaSetDevice(cfg->device) != cudaSuccess) return bail(PIRRT_ERR_CUDA);
    int dev = cfg->device;
    if (cudaDeviceGetAttribute(&G->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    const size_t nv = (size_t)G->cap_n;
    const size_t ne = (size_t)std::max<int64_t>(G->cap_e, 1);
    const size_t n_tiles = (nv + 1 + kScanTile - 1) / kScanTile + 1;
#define ALLOC(ptr, bytes)                                                               \
    do {                                                                                \
        cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes));                          \
        if (e_ != cudaSuccess) {                                                        \
            cudaGetLastError();                                                         \
            return bail(e_ == cudaErrorMemoryAllocation ? PIRRT_ERR_OOM : PIRRT_ERR_CUDA); \
        }                                                                               \
    } while (0)
    ALLOC(G->rows, sizeof(RowExt) * nv);
    ALLOC(G->ralloc, sizeof(int32_t) * (nv + 1));
    ALLOC(G->touched, sizeof(int32_t) * nv);
    ALLOC(G->roff, sizeof(int64_t) * (nv + 1));
    // A pool holds every row with room to grow plus the space rows moved out
    // of; a repack (1.25 x length + 2 per row) always fits.  The second pool
    // is allocated by the first repack.  +16 entries: a staged row copy is
    // rounded up to 16 bytes past the row.
    G->pool_cap = 2 * (int64_t)ne + 4 * (int64_t)nv + 64;
    ALLOC(G->adj[0], G->entry_bytes * (size_t)(G->pool_cap + 16));
    ALLOC(G->g, sizeof(double) * nv);
    ALLOC(G->g32, sizeof(float) * nv);
    ALLOC(G->p, sizeof(int32_t) * nv);
    ALLOC(G->pc, G->cost_bytes * nv);
    ALLOC(G->deg, sizeof(int32_t) * (nv + 1));
    ALLOC(G->tile_sums, sizeof(long long) * n_tiles);
    ALLOC(G->stamp, sizeof(unsigned) * nv);
    ALLOC(G->list[0], sizeof(int32_t) * nv);
    ALLOC(G->list[1], sizeof(int32_t) * nv);
    ALLOC(G->switched, sizeof(int32_t) * nv);
    ALLOC(G->dg, sizeof(int32_t) * nv);
    ALLOC(G->anc[0], sizeof(int32_t) * nv);
    ALLOC(G->anc[1], sizeof(int32_t) * nv);
    ALLOC(G->acc[0], sizeof(double) * nv);
    ALLOC(G->acc[1], sizeof(double) * nv);
    ALLOC(G->wx[0], sizeof(longlong2) * nv);
    ALLOC(G->wx[1], sizeof(longlong2) * nv);
    ALLOC(G->done, sizeof(int32_t) * nv);
    ALLOC(G->wl[0], sizeof(int32_t) * nv);
    ALLOC(G->wl[1], sizeof(int32_t) * nv);
    ALLOC(G->wstamp, sizeof(unsigned) * nv);
    ALLOC(G->swstamp, sizeof(unsigned) * nv);
    ALLOC(G->cand, sizeof(unsigned long long) * nv);
    ALLOC(G->aq, sizeof(AsyncQueue));
    ALLOC(G->aring, sizeof(AsyncItem) * nv);
    ALLOC(G->ctr, sizeof(DevCounters));
    ALLOC(G->dargs, kArgBytes);
    ALLOC(G->pexport, sizeof(int32_t) * nv);
#undef ALLOC
    if (cudaMallocHost((void **)&G->hargs, kArgBytes) != cudaSuccess) return bail(PIRRT_ERR_OOM);
    if (cudaStreamCreateWithFlags(&G->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->pre_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->pre_free, cudaEventDisableTiming) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&G->capture, cudaStreamNonBlocking) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    if (cudaMallocHost((void **)&G->hx, 2 * sizeof(int64_t)) != cudaSuccess)
        return bail(PIRRT_ERR_OOM);
    if (cudaMallocHost((void **)&G->ctr_host, sizeof(DevCounters)) != cudaSuccess)
        return bail(PIRRT_ERR_OOM);
    if (cudaEventCreate(&G->ev0) != cudaSuccess || cudaEventCreate(&G->ev1) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    for (cudaEvent_t &e : G->pev)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(PIRRT_ERR_CUDA);
    if (cudaEventCreate(&G->it_start) != cudaSuccess) return bail(PIRRT_ERR_CUDA);
    if (cudaEventCreateWithFlags(&G->args_ev, cudaEventDisableTiming) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, evaluate_kernel<float>, kThreads, 0) !=
        cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    int occ64 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, evaluate_kernel<double>, kThreads, 0) !=
        cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    occ = std::min(occ, occ64);
    if (occ < 1) return bail(PIRRT_ERR_CUDA);
    G->eval_blocks = G->num_sms * occ;
    int wocc = 0, wocc64 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wocc, wave_evaluate_kernel<float>,
                                                      kWaveThreads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wocc64, wave_evaluate_kernel<double>,
                                                      kWaveThreads, 0) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    wocc = std::min(wocc, wocc64);
    if (wocc < 1) return bail(PIRRT_ERR_CUDA);
    G->wave_occ = std::min(wocc, 2);
    G->wave_blocks = G->num_sms * G->wave_occ;
    int aocc = 0, aocc64 = 0;
    if (cudaFuncSetAttribute(async_evaluate_kernel<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAsyncSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(async_evaluate_kernel<double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAsyncSmem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&aocc, async_evaluate_kernel<float>,
                                                      kAsyncThreads, kAsyncSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&aocc64, async_evaluate_kernel<double>,
                                                      kAsyncThreads, kAsyncSmem) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    aocc = std::min(aocc, aocc64);
    if (aocc < 1) return bail(PIRRT_ERR_CUDA);
    G->async_blocks = G->num_sms * std::min(aocc, 2);
    // spill-list slots carry their index, so zeroed slots match none; the
    // walk's indices grow over the graph's lifetime and are never reset
    if (cudaMemset(G->aq, 0, sizeof(AsyncQueue)) != cudaSuccess ||
        cudaMemset(G->aring, 0, sizeof(AsyncItem) * nv) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    pirrt_status rc = pirrt_graph_reset(G);
    if (rc) return bail(rc);
    *out = G;
    return PIRRT_OK;
}

pirrt_status pirrt_graph_reset(pirrt_graph *G) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    CK(cudaSetDevice(G->cfg.device));
    CK(cudaMemsetAsync(G->stamp, 0, sizeof(unsigned) * (size_t)G->cap_n, G->stream));
    CK(cudaMemsetAsync(G->wstamp, 0, sizeof(unsigned) * (size_t)G->cap_n, G->stream));
    CK(cudaMemsetAsync(G->swstamp, 0, sizeof(unsigned) * (size_t)G->cap_n, G->stream));
    // the level trace (the tail of the counter block) survives a reset, like
    // the rest of the profile
    CK(cudaMemsetAsync(G->ctr, 0, offsetof(DevCounters, lvl_trace), G->stream));
    // insertions count into deg and leave it all zero
    CK(cudaMemsetAsync(G->deg, 0, sizeof(int32_t) * (size_t)(G->cap_n + 1), G->stream));
    // stamps start at 0, so the first list uses stamp value 1
    const unsigned one = 1u;
    CK(cudaMemcpyAsync(&G->ctr->epoch, &one, sizeof(unsigned), cudaMemcpyHostToDevice, G->stream));
    CK(cudaMemcpyAsync(&G->ctr->wave_epoch, &one, sizeof(unsigned), cudaMemcpyHostToDevice,
                       G->stream));
    CK(cudaStreamSynchronize(G->stream));
    G->pool_used = 0;
    G->copied_seen = 0;
    G->n = 0;
    G->m = 0;
    G->cur = 0;
    G->args_key = pirrt_graph::ArgsKey{};
    G->deep_hint = 0;
    G->exploits = 0;
    G->stale = 0;
    G->goal_dirty = 0;
    G->recover = 0;
    G->last_error.clear();
    return apply_goal(G);  // the goal and h stay configured
}

pirrt_status pirrt_graph_insert_batch(pirrt_graph *G, int64_t n_new, int64_t n_edges,
                                      const int32_t *src, const int32_t *dst, const void *cost,
                                      int on_device) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    if (n_new < 0 || n_edges < 0 || (n_edges > 0 && (!src || !dst || !cost)))
        return fail(G, PIRRT_ERR_INVALID_ARG, "insert_batch: negative size or NULL pointer");
    if (G->n + n_new > G->cap_n)
        return fail(G, PIRRT_ERR_CAPACITY, "insert_batch: %lld vertices exceed max_vertices %lld",
                    (long long)(G->n + n_new), (long long)G->cap_n);
    if (G->m + 2 * n_edges > G->cap_e)
        return fail(G, PIRRT_ERR_CAPACITY, "insert_batch: %lld edges exceed max_edges %lld",
                    (long long)((G->m + 2 * n_edges) / 2), (long long)(G->cap_e / 2));
    CK(cudaSetDevice(G->cfg.device));
    const int32_t *s = src, *d = dst;
    const void *c = cost;
    const bool pending = G->pre_n >= 0;
    const bool prefetched = pending && !on_device && n_edges > 0 && G->pre_n == n_edges &&
                            G->pre_src == src && G->pre_dst == dst && G->pre_cost == cost;
    G->pre_n = -1;
    if (pending && !prefetched) {
        // a prefetch this insertion does not use: its copies end before control
        // returns, so that the caller may release those host buffers
        CK(cudaStreamSynchronize(G->copy));
    }
    if (prefetched) {
        // the block was copied on the copy stream while the last exploit ran
        CK(cudaStreamWaitEvent(G->stream, G->pre_done, 0));
        const size_t a16 = (sizeof(int32_t) * (size_t)n_edges + 15) & ~size_t(15);
        char *base = static_cast<char *>(G->pre);
        s = reinterpret_cast<const int32_t *>(base);
        d = reinterpret_cast<const int32_t *>(base + a16);
        c = base + 2 * a16;
        const pirrt_status rc =
            G->cfg.cost_dtype == PIRRT_COST_F32
                ? insert_impl<float>(G, n_new, n_edges, s, d, static_cast<const float *>(c))
                : insert_impl<double>(G, n_new, n_edges, s, d, static_cast<const double *>(c));
        CK(cudaEventRecord(G->pre_free, G->stream));
        return rc;
    }
    if (!on_device && n_edges > 0) {
        const size_t ib = sizeof(int32_t) * (size_t)n_edges;
        const size_t cb = G->cost_bytes * (size_t)n_edges;
        const size_t a16 = (ib + 15) & ~size_t(15);
        pirrt_status rc = ensure_stage(G, 2 * a16 + cb);
        if (rc) return rc;
        char *base = static_cast<char *>(G->stage);
        CK(cudaMemcpyAsync(base, src, ib, cudaMemcpyHostToDevice, G->stream));
        CK(cudaMemcpyAsync(base + a16, dst, ib, cudaMemcpyHostToDevice, G->stream));
        CK(cudaMemcpyAsync(base + 2 * a16, cost, cb, cudaMemcpyHostToDevice, G->stream));
        s = reinterpret_cast<const int32_t *>(base);
        d = reinterpret_cast<const int32_t *>(base + a16);
        c = base + 2 * a16;
    }
    if (G->cfg.cost_dtype == PIRRT_COST_F32)
        return insert_impl<float>(G, n_new, n_edges, s, d, static_cast<const float *>(c));
    return insert_impl<double>(G, n_new, n_edges, s, d, static_cast<const double *>(c));
}

pirrt_status pirrt_graph_set_goal(pirrt_graph *G, int32_t goal, const float *h, int64_t n_h) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    if (goal < -1 || goal >= G->cap_n || n_h < 0 || n_h > G->cap_n || (n_h > 0 && !h))
        return fail(G, PIRRT_ERR_INVALID_ARG,
                    "set_goal: goal %d or %lld heuristic values outside the capacity %lld", goal,
                    (long long)n_h, (long long)G->cap_n);
    for (int64_t v = 0; v < n_h; ++v)
        if (!(h[v] >= 0.0f) || !std::isfinite(h[v]))
            return fail(G, PIRRT_ERR_BAD_INPUT, "set_goal: h[%lld] is negative or not finite",
                        (long long)v);
    CK(cudaSetDevice(G->cfg.device));
    if (goal >= 0) {
        if (!G->h && cudaMalloc(&G->h, sizeof(float) * (size_t)G->cap_n) != cudaSuccess) {
            G->h = nullptr;
            return fail(G, PIRRT_ERR_OOM, "set_goal: no room for h");
        }
        CK(cudaMemsetAsync(G->h, 0, sizeof(float) * (size_t)G->cap_n, G->stream));
        if (n_h > 0)
            CK(cudaMemcpyAsync(G->h, h, sizeof(float) * (size_t)n_h, cudaMemcpyHostToDevice,
                               G->stream));
    }
    G->goal = goal;
    G->goal_dirty = 1;
    G->args_key = pirrt_graph::ArgsKey{};
    return apply_goal(G);
}

pirrt_status pirrt_graph_prefetch_batch(pirrt_graph *G, int64_t n_edges, const int32_t *src,
                                        const int32_t *dst, const void *cost) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    if (n_edges < 0 || (n_edges > 0 && (!src || !dst || !cost)))
        return fail(G, PIRRT_ERR_INVALID_ARG, "prefetch_batch: negative size or NULL pointer");
    CK(cudaSetDevice(G->cfg.device));
    if (G->pre_n >= 0) {
        // an earlier prefetch that no insertion used: its copies end first, so
        // that the caller may release those host buffers
        CK(cudaStreamSynchronize(G->copy));
    }
    G->pre_n = -1;
    if (n_edges == 0) return PIRRT_OK;
    const size_t ib = sizeof(int32_t) * (size_t)n_edges;
    const size_t cb = G->cost_bytes * (size_t)n_edges;
    const size_t a16 = (ib + 15) & ~size_t(15);
    const size_t bytes = 2 * a16 + cb;
    if (bytes > G->pre_bytes) {
        CK(cudaStreamSynchronize(G->copy));
        CK(cudaEventSynchronize(G->pre_free));
        if (G->pre) CK(cudaFree(G->pre));
        G->pre = nullptr;
        G->pre_bytes = 0;
        CK(cudaMalloc(&G->pre, bytes));
        G->pre_bytes = bytes;
    }
    // the insertion that read the buffer last must be done with it
    CK(cudaStreamWaitEvent(G->copy, G->pre_free, 0));
    char *base = static_cast<char *>(G->pre);
    CK(cudaMemcpyAsync(base, src, ib, cudaMemcpyHostToDevice, G->copy));
    CK(cudaMemcpyAsync(base + a16, dst, ib, cudaMemcpyHostToDevice, G->copy));
    CK(cudaMemcpyAsync(base + 2 * a16, cost, cb, cudaMemcpyHostToDevice, G->copy));
    CK(cudaEventRecord(G->pre_done, G->copy));
    G->pre_src = src;
    G->pre_dst = dst;
    G->pre_cost = cost;
    G->pre_n = n_edges;
    return PIRRT_OK;
}

pirrt_status pirrt_graph_set_policy(pirrt_graph *G, const int32_t *parent, int64_t n, int on_device) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    if (n != G->n || (n > 0 && !parent))
        return fail(G, PIRRT_ERR_INVALID_ARG, "set_policy: n = %lld but the graph has %lld vertices",
                    (long long)n, (long long)G->n);
    if (n == 0) return PIRRT_OK;
    CK(cudaSetDevice(G->cfg.device));
    const int32_t *pp = parent;
    if (!on_device) {
        pirrt_status rc = ensure_stage(G, sizeof(int32_t) * (size_t)n);
        if (rc) return rc;
        CK(cudaMemcpyAsync(G->stage, parent, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice,
                           G->stream));
        pp = static_cast<const int32_t *>(G->stage);
    }
    if (G->cfg.cost_dtype == PIRRT_COST_F32) return set_policy_impl<float>(G, pp);
    return set_policy_impl<double>(G, pp);
}

pirrt_status pirrt_graph_exploit(pirrt_graph *G, const pirrt_exploit_opts *opts,
                                 pirrt_exploit_stats *stats) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    if (stats) *stats = pirrt_exploit_stats{};
    CK(cudaSetDevice(G->cfg.device));
    if (G->n == 0) {
        if (stats) stats->converged = 1;
        return PIRRT_OK;
    }
    const pirrt_status rc = G->cfg.cost_dtype == PIRRT_COST_F32 ? exploit_impl<float>(G, opts, stats)
                                                                : exploit_impl<double>(G, opts, stats);
    if (rc != PIRRT_OK) G->async_dirty = 1;
    return rc;
}

pirrt_status pirrt_graph_get_costs(const pirrt_graph *Gc, double *g_out, int64_t n, int on_device) {
    pirrt_graph *G = const_cast<pirrt_graph *>(Gc);
    if (!G) return PIRRT_ERR_INVALID_ARG;
    if (n != G->n || (n > 0 && !g_out))
        return fail(G, PIRRT_ERR_INVALID_ARG, "get_costs: n = %lld but the graph has %lld vertices",
                    (long long)n, (long long)G->n);
    CK(cudaSetDevice(G->cfg.device));
    if (n > 0)
        CK(cudaMemcpyAsync(g_out, G->g, sizeof(double) * (size_t)n,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_graph_get_parents(const pirrt_graph *Gc, int32_t *p_out, int64_t n, int on_device) {
    pirrt_graph *G = const_cast<pirrt_graph *>(Gc);
    if (!G) return PIRRT_ERR_INVALID_ARG;
    if (n != G->n || (n > 0 && !p_out))
        return fail(G, PIRRT_ERR_INVALID_ARG, "get_parents: n = %lld but the graph has %lld vertices",
                    (long long)n, (long long)G->n);
    CK(cudaSetDevice(G->cfg.device));
    if (n > 0) {
        int32_t *dst = on_device ? p_out : G->pexport;
        export_parents_kernel<<<grid_for(n, kThreads, G->num_sms * 8), kThreads, 0, G->stream>>>(
            n, G->p, dst);
        CKL();
        if (!on_device)
            CK(cudaMemcpyAsync(p_out, G->pexport, sizeof(int32_t) * (size_t)n,
                               cudaMemcpyDeviceToHost, G->stream));
    }
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_graph_set_profiling(pirrt_graph *G, int enable) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    CK(cudaSetDevice(G->cfg.device));
    G->profiling = enable == 1 ? 1 : 0;  // 2: the device-side trace alone
    G->prof = pirrt_profile{};
    G->trace.clear();
    CK(cudaStreamSynchronize(G->stream));
    // the device-side level trace starts afresh, on while profiling
    const size_t lvl_off = offsetof(DevCounters, lvl_trace);
    CK(cudaMemset(reinterpret_cast<char *>(G->ctr) + lvl_off, 0, sizeof(DevCounters) - lvl_off));
    const unsigned on = enable != 0 ? 1u : 0u;
    CK(cudaMemcpy(&G->ctr->lvl_trace, &on, sizeof(on), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(&G->copied_seen, &G->ctr->insert_copied, sizeof(G->copied_seen),
                  cudaMemcpyDeviceToHost));
    return PIRRT_OK;
}

int64_t pirrt_graph_get_trace(const pirrt_graph *G, pirrt_trace_record *out, int64_t cap) {
    if (!G) return -1;
    const int64_t n = (int64_t)G->trace.size();
    if (out && cap > 0) std::memcpy(out, G->trace.data(), sizeof(pirrt_trace_record) * (size_t)std::min(n, cap));
    return n;
}

pirrt_status pirrt_graph_get_profile(const pirrt_graph *Gc, pirrt_profile *out) {
    if (!Gc || !out) return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = const_cast<pirrt_graph *>(Gc);  // for the error text only
    *out = G->prof;
    CK(cudaSetDevice(G->cfg.device));
    CK(cudaStreamSynchronize(G->stream));
    DevCounters h;
    const size_t lvl_off = offsetof(DevCounters, lvl_trace);
    CK(cudaMemcpy(reinterpret_cast<char *>(&h) + lvl_off,
                  reinterpret_cast<const char *>(G->ctr) + lvl_off, sizeof(DevCounters) - lvl_off,
                  cudaMemcpyDeviceToHost));
    for (int b = 0; b < kLevelBuckets; ++b) {
        out->level_count[b] = (int64_t)h.lvl_n[b];
        out->level_vertices[b] = (int64_t)h.lvl_items[b];
        out->level_cycles[b] = (int64_t)h.lvl_cyc[b];
        out->share_tiles[b] = (int64_t)h.shr_n[b];
        out->share_vertices[b] = (int64_t)h.shr_items[b];
        out->share_cycles[b] = (int64_t)h.shr_cyc[b];
        out->local_tiles[b] = (int64_t)h.loc_n[b];
        out->local_vertices[b] = (int64_t)h.loc_items[b];
        out->local_cycles[b] = (int64_t)h.loc_cyc[b];
    }
    out->wave_pre_cycles = (int64_t)h.ph_pre_cyc;
    out->wave_post_cycles = (int64_t)h.ph_post_cyc;
    out->wave_jump_cycles = (int64_t)h.ph_jump_cyc;
    out->wave_calls = (int64_t)h.ph_calls;
    out->wave_span_ns = (int64_t)h.span_ns;
    out->wave_spans = (int64_t)h.spans;
    out->wave_gap_ns = (int64_t)h.gap_ns;
    out->wave_gaps = (int64_t)h.gaps;
    return PIRRT_OK;
}

extern "C++" {
// Packed copy of the CSR on the device: offsets in G->roff[0..n], entries in
// G->stage[0..m).
template <typename CT>
pirrt_status pack_csr(pirrt_graph *G) {
    const int64_t n = G->n, len = n + 1;
    const int max_blocks = G->num_sms * 32;
    row_lengths<<<grid_for(len, kThreads, max_blocks), kThreads, 0, G->stream>>>(n, G->rows,
                                                                               G->ralloc);
    CKL();
    const int64_t n_tiles = (len + kScanTile - 1) / kScanTile;
    scan_tile_reduce<<<(unsigned)n_tiles, kThreads, 0, G->stream>>>(G->ralloc, len, G->tile_sums);
    CKL();
    scan_tile_sums<<<1, kThreads, 0, G->stream>>>(G->tile_sums, n_tiles);
    CKL();
    scan_tile_apply<<<(unsigned)n_tiles, kThreads, 0, G->stream>>>(G->ralloc, len, G->tile_sums,
                                                                    G->roff);
    CKL();
    if (G->m > 0) {
        pirrt_status rc = ensure_stage(G, G->entry_bytes * (size_t)G->m);
        if (rc) return rc;
        export_rows<CT><<<grid_for((n + 31) / 32 * 32, kThreads, max_blocks), kThreads, 0,
                          G->stream>>>(n, G->rows, G->roff,
                                       static_cast<const Entry<CT> *>(G->adj[G->cur]),
                                       static_cast<Entry<CT> *>(G->stage));
        CKL();
    }
    return PIRRT_OK;
}

template <typename CT>
pirrt_status export_impl(pirrt_graph *G, int64_t *row_off, int32_t *col, void *cost,
                         int on_device) {
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    pirrt_status rc = pack_csr<CT>(G);
    if (rc) return rc;
    if (row_off)
        CK(cudaMemcpyAsync(row_off, G->roff, sizeof(int64_t) * (size_t)(G->n + 1), kind, G->stream));
    if (G->m > 0 && (col || cost)) {
        // entries are (col, cost) records: split with strided 2-D copies
        const char *base = static_cast<const char *>(G->stage);
        if (col)
            CK(cudaMemcpy2DAsync(col, sizeof(int32_t), base, G->entry_bytes, sizeof(int32_t),
                                 (size_t)G->m, kind, G->stream));
        if (cost) {
            const size_t off = G->cfg.cost_dtype == PIRRT_COST_F32 ? 4 : 8;
            CK(cudaMemcpy2DAsync(cost, G->cost_bytes, base + off, G->entry_bytes, G->cost_bytes,
                                 (size_t)G->m, kind, G->stream));
        }
    }
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

// Checkpoint file: a header, then the packed CSR offsets (int64, n + 1), its
// entries as stored (Entry<CT>, m), g (double, n), the parents with root
// markers (int32, n) and the parent-edge costs (CT, n).
struct CkptHeader {
    char magic[8];
    int32_t cost_dtype;
    int32_t root;
    int64_t n;
    int64_t m;
};
constexpr char kCkptMagic[8] = {'P', 'I', 'R', 'R', 'T', 'G', '0', '1'};

template <typename CT>
pirrt_status save_impl(pirrt_graph *G, FILE *f) {
    const int64_t n = G->n, m = G->m;
    pirrt_status rc = PIRRT_OK;
    // goal-directed: subtrees below pruned vertices are brought up to date,
    // so that the file holds g of the whole policy tree
    if (G->stale && (rc = reevaluate_impl<CT>(G))) return rc;
    rc = pack_csr<CT>(G);
    if (rc) return rc;
    std::vector<int64_t> off((size_t)n + 1);
    std::vector<unsigned char> ent((size_t)m * G->entry_bytes);
    std::vector<double> g((size_t)n);
    std::vector<int32_t> p((size_t)n);
    std::vector<CT> pc((size_t)n);
    CK(cudaMemcpyAsync(off.data(), G->roff, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost,
                       G->stream));
    if (m > 0)
        CK(cudaMemcpyAsync(ent.data(), G->stage, ent.size(), cudaMemcpyDeviceToHost, G->stream));
    if (n > 0) {
        CK(cudaMemcpyAsync(g.data(), G->g, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                           G->stream));
        CK(cudaMemcpyAsync(p.data(), G->p, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost,
                           G->stream));
        CK(cudaMemcpyAsync(pc.data(), G->pc, sizeof(CT) * (size_t)n, cudaMemcpyDeviceToHost,
                           G->stream));
    }
    CK(cudaStreamSynchronize(G->stream));
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.cost_dtype = G->cfg.cost_dtype;
    h.root = G->cfg.root;
    h.n = n;
    h.m = m;
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
              std::fwrite(off.data(), sizeof(int64_t), off.size(), f) == off.size() &&
              std::fwrite(ent.data(), 1, ent.size(), f) == ent.size() &&
              std::fwrite(g.data(), sizeof(double), g.size(), f) == g.size() &&
              std::fwrite(p.data(), sizeof(int32_t), p.size(), f) == p.size() &&
              std::fwrite(pc.data(), sizeof(CT), pc.size(), f) == pc.size();
    if (!ok) return fail(G, PIRRT_ERR_INVALID_ARG, "save: write failed");
    return PIRRT_OK;
}

template <typename CT>
pirrt_status load_impl(pirrt_graph *G, FILE *f, const CkptHeader &h) {
    const int64_t n = h.n, m = h.m;
    std::vector<int64_t> off((size_t)n + 1);
    std::vector<unsigned char> ent((size_t)m * G->entry_bytes);
    std::vector<double> g((size_t)n);
    std::vector<int32_t> p((size_t)n);
    std::vector<CT> pc((size_t)n);
    bool ok = std::fread(off.data(), sizeof(int64_t), off.size(), f) == off.size() &&
              std::fread(ent.data(), 1, ent.size(), f) == ent.size() &&
              std::fread(g.data(), sizeof(double), g.size(), f) == g.size() &&
              std::fread(p.data(), sizeof(int32_t), p.size(), f) == p.size() &&
              std::fread(pc.data(), sizeof(CT), pc.size(), f) == pc.size();
    if (!ok) return fail(G, PIRRT_ERR_BAD_INPUT, "load: file too short");
    // Everything a kernel will follow is checked here, before any copy: the
    // offsets are a packed CSR of m entries; every entry's column is another
    // vertex in [0, n) and its cost finite and > 0; only the root carries the
    // root marker; every other parent is -1 or a vertex in [0, n) other than
    // itself, with a finite parent-edge cost >= 0; g is not NaN and >= 0.
    ok = off[0] == 0 && off[(size_t)n] == m;
    for (int64_t v = 0; ok && v < n; ++v) ok = off[(size_t)v + 1] >= off[(size_t)v];
    if (!ok) return fail(G, PIRRT_ERR_BAD_INPUT, "load: inconsistent row offsets");
    const Entry<CT> *en = reinterpret_cast<const Entry<CT> *>(ent.data());
    for (int64_t v = 0; ok && v < n; ++v)
        for (int64_t i = off[(size_t)v]; ok && i < off[(size_t)v + 1]; ++i) {
            const double w = (double)en[i].w;
            ok = en[i].col >= 0 && en[i].col < n && en[i].col != v && w > 0.0 && w <= DBL_MAX;
        }
    if (!ok) return fail(G, PIRRT_ERR_BAD_INPUT, "load: adjacency entry out of range");
    for (int64_t v = 0; ok && v < n; ++v) {
        const int32_t q = p[(size_t)v];
        const double c = (double)pc[(size_t)v];
        const double gv = g[(size_t)v];
        if (v == h.root) ok = q == kRootMark && gv == 0.0;
        else ok = q == -1 || (q >= 0 && q < n && q != v && c >= 0.0 && c <= DBL_MAX);
        ok = ok && gv >= 0.0;  // rejects NaN; +inf marks an unreached vertex
    }
    if (!ok) return fail(G, PIRRT_ERR_BAD_INPUT, "load: inconsistent policy");
    pirrt_status rc = pirrt_graph_reset(G);
    if (rc) return rc;
    CK(cudaMemcpyAsync(G->roff, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice,
                       G->stream));
    if (m > 0)
        CK(cudaMemcpyAsync(G->adj[G->cur], ent.data(), ent.size(), cudaMemcpyHostToDevice,
                           G->stream));
    if (n > 0) {
        CK(cudaMemcpyAsync(G->g, g.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice,
                           G->stream));
        CK(cudaMemcpyAsync(G->p, p.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice,
                           G->stream));
        CK(cudaMemcpyAsync(G->pc, pc.data(), sizeof(CT) * (size_t)n, cudaMemcpyHostToDevice,
                           G->stream));
        restore_rows<<<grid_for(n, kThreads, G->num_sms * 32), kThreads, 0, G->stream>>>(
            n, G->roff, G->rows, G->g, G->g32, G->cand);
        CKL();
    }
    // the next Improve sweeps every vertex (no frontier survives a checkpoint)
    const unsigned one = 1u;
    CK(cudaMemcpyAsync(&G->ctr->dense, &one, sizeof(unsigned), cudaMemcpyHostToDevice, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    G->n = n;
    G->m = m;
    G->pool_used = m;
    return PIRRT_OK;
}
}  // extern "C++"

pirrt_status pirrt_graph_save(const pirrt_graph *Gc, const char *path) {
    pirrt_graph *G = const_cast<pirrt_graph *>(Gc);
    if (!G || !path) return PIRRT_ERR_INVALID_ARG;
    CK(cudaSetDevice(G->cfg.device));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(G, PIRRT_ERR_INVALID_ARG, "save: cannot open %s", path);
    const pirrt_status rc = G->cfg.cost_dtype == PIRRT_COST_F32 ? save_impl<float>(G, f)
                                                                : save_impl<double>(G, f);
    if (std::fclose(f) != 0 && rc == PIRRT_OK)
        return fail(G, PIRRT_ERR_INVALID_ARG, "save: cannot close %s", path);
    return rc;
}

pirrt_status pirrt_graph_load(pirrt_graph *G, const char *path) {
    if (!G || !path) return PIRRT_ERR_INVALID_ARG;
    CK(cudaSetDevice(G->cfg.device));
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(G, PIRRT_ERR_INVALID_ARG, "load: cannot open %s", path);
    CkptHeader h{};
    pirrt_status rc = PIRRT_OK;
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kCkptMagic, 8) != 0 ||
        h.n < 0 || h.m < 0)
        rc = fail(G, PIRRT_ERR_BAD_INPUT, "load: not a graph checkpoint");
    else if (h.cost_dtype != G->cfg.cost_dtype || h.root != G->cfg.root)
        rc = fail(G, PIRRT_ERR_INVALID_ARG, "load: cost type or root differ from the graph's");
    else if (h.n > G->cap_n || h.m > G->cap_e || h.m > G->pool_cap)
        rc = fail(G, PIRRT_ERR_CAPACITY, "load: %lld vertices / %lld entries exceed the graph",
                  (long long)h.n, (long long)h.m);
    else
        rc = G->cfg.cost_dtype == PIRRT_COST_F32 ? load_impl<float>(G, f, h)
                                                 : load_impl<double>(G, f, h);
    std::fclose(f);
    return rc;
}

pirrt_status pirrt_graph_get_adjacency(const pirrt_graph *Gc, int64_t *row_off, int32_t *col,
                                       void *cost, int on_device) {
    pirrt_graph *G = const_cast<pirrt_graph *>(Gc);
    if (!G) return PIRRT_ERR_INVALID_ARG;
    CK(cudaSetDevice(G->cfg.device));
    if (G->cfg.cost_dtype == PIRRT_COST_F32) return export_impl<float>(G, row_off, col, cost, on_device);
    return export_impl<double>(G, row_off, col, cost, on_device);
}


pirrt_status pirrt_batch_create(int32_t n_graphs, const int64_t *max_vertices,
                                const int64_t *max_edges, const int32_t *roots,
                                int32_t cost_dtype, int32_t device, void *stream,
                                pirrt_batch **out) {
    if (!out) return PIRRT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_graphs <= 0 || !max_vertices || !max_edges || !roots) return PIRRT_ERR_INVALID_ARG;
    int64_t tv = 0, te = 0;
    for (int32_t b = 0; b < n_graphs; ++b) {
        if (max_vertices[b] <= 0 || max_edges[b] < 0 || roots[b] < 0 || roots[b] >= max_vertices[b])
            return PIRRT_ERR_INVALID_ARG;
        tv += max_vertices[b];
        te += max_edges[b];
    }
    if (tv > INT32_MAX - 1) return PIRRT_ERR_CAPACITY;
    pirrt_batch *B = new (std::nothrow) pirrt_batch();
    if (!B) return PIRRT_ERR_OOM;
    B->n_graphs = n_graphs;
    B->base.resize(n_graphs);
    B->cap_v.assign(max_vertices, max_vertices + n_graphs);
    B->cap_e.assign(max_edges, max_edges + n_graphs);
    B->staged_e.assign(n_graphs, 0);
    int64_t acc_v = 0;
    for (int32_t b = 0; b < n_graphs; ++b) {
        B->base[b] = acc_v;
        acc_v += max_vertices[b];
    }
    pirrt_config cfg{};
    cfg.max_vertices = tv;
    cfg.max_edges = te;
    cfg.root = roots[0];
    cfg.cost_dtype = cost_dtype;
    cfg.device = device;
    cfg.stream = stream;
    pirrt_status rc = pirrt_graph_create(&cfg, &B->G);
    if (rc) {
        delete B;
        return rc;
    }
    pirrt_graph *G = B->G;
    auto bail = [&](pirrt_status r) {
        if (B->pend_src) cudaFree(B->pend_src);
        if (B->pend_dst) cudaFree(B->pend_dst);
        if (B->pend_cost) cudaFree(B->pend_cost);
        pirrt_graph_destroy(B->G);
        delete B;
        return r;
    };
    B->groots.resize(n_graphs);
    for (int32_t b = 0; b < n_graphs; ++b) B->groots[b] = (int32_t)(B->base[b] + roots[b]);
    const size_t pe = (size_t)std::max<int64_t>(te, 1);
    if (cudaMalloc((void **)&B->pend_src, 4 * pe) != cudaSuccess ||
        cudaMalloc((void **)&B->pend_dst, 4 * pe) != cudaSuccess ||
        cudaMalloc(&B->pend_cost, G->cost_bytes * pe) != cudaSuccess)
        return bail(PIRRT_ERR_OOM);
    B->pend_cap = te;
    if ((rc = pirrt_batch_reset(B))) return bail(rc);
    *out = B;
    return PIRRT_OK;
}

pirrt_status pirrt_batch_reset(pirrt_batch *B) {
    if (!B) return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = B->G;
    pirrt_status rc = pirrt_graph_reset(G);
    if (rc) return rc;
    // every member's vertices exist from the start, isolated; roots get g = 0
    int64_t tv = 0;
    for (int64_t c : B->cap_v) tv += c;
    if ((rc = pirrt_graph_insert_batch(G, tv, 0, nullptr, nullptr, nullptr, 1))) return rc;
    const size_t k = B->groots.size();
    if ((rc = ensure_stage(G, 4 * k))) return rc;
    CK(cudaMemcpyAsync(G->stage, B->groots.data(), 4 * k, cudaMemcpyHostToDevice, G->stream));
    set_roots_kernel<<<grid_for((int64_t)k, kThreads, 1024), kThreads, 0, G->stream>>>(
        (int64_t)k, static_cast<const int32_t *>(G->stage), G->g, G->g32, G->p);
    CKL();
    CK(cudaStreamSynchronize(G->stream));
    B->pend_n = 0;
    std::fill(B->staged_e.begin(), B->staged_e.end(), 0);
    return PIRRT_OK;
}

void pirrt_batch_destroy(pirrt_batch *B) {
    if (!B) return;
    if (B->G) {
        cudaSetDevice(B->G->cfg.device);
        cudaStreamSynchronize(B->G->stream);
    }
    if (B->pend_src) cudaFree(B->pend_src);
    if (B->pend_dst) cudaFree(B->pend_dst);
    if (B->pend_cost) cudaFree(B->pend_cost);
    pirrt_graph_destroy(B->G);
    delete B;
}

pirrt_graph *pirrt_batch_graph(pirrt_batch *B) { return B ? B->G : nullptr; }

pirrt_status pirrt_batch_insert(pirrt_batch *B, int32_t graph, int64_t n_edges, const int32_t *src,
                                const int32_t *dst, const void *cost, int on_device) {
    if (!B || graph < 0 || graph >= B->n_graphs || n_edges < 0 ||
        (n_edges > 0 && (!src || !dst || !cost)))
        return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = B->G;
    if (B->staged_e[graph] + n_edges > B->cap_e[graph])
        return fail(G, PIRRT_ERR_CAPACITY, "batch_insert: graph %d would exceed %lld edges", graph,
                    (long long)B->cap_e[graph]);
    if (n_edges == 0) return PIRRT_OK;
    CK(cudaSetDevice(G->cfg.device));
    const int32_t *s = src, *d = dst;
    const void *c = cost;
    if (!on_device) {
        const size_t ib = sizeof(int32_t) * (size_t)n_edges;
        const size_t cb = G->cost_bytes * (size_t)n_edges;
        const size_t a16 = (ib + 15) & ~size_t(15);
        pirrt_status rc = ensure_stage(G, 2 * a16 + cb);
        if (rc) return rc;
        char *base = static_cast<char *>(G->stage);
        CK(cudaMemcpyAsync(base, src, ib, cudaMemcpyHostToDevice, G->stream));
        CK(cudaMemcpyAsync(base + a16, dst, ib, cudaMemcpyHostToDevice, G->stream));
        CK(cudaMemcpyAsync(base + 2 * a16, cost, cb, cudaMemcpyHostToDevice, G->stream));
        s = reinterpret_cast<const int32_t *>(base);
        d = reinterpret_cast<const int32_t *>(base + a16);
        c = base + 2 * a16;
    }
    if (G->cfg.cost_dtype == PIRRT_COST_F32)
        return batch_translate<float>(B, graph, n_edges, s, d, static_cast<const float *>(c));
    return batch_translate<double>(B, graph, n_edges, s, d, static_cast<const double *>(c));
}

pirrt_status pirrt_batch_exploit(pirrt_batch *B, const pirrt_exploit_opts *opts,
                                 pirrt_exploit_stats *stats) {
    if (!B) return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = B->G;
    CK(cudaSetDevice(G->cfg.device));
    pirrt_status rc = batch_flush(B);
    if (rc) return rc;
    return pirrt_graph_exploit(G, opts, stats);
}

// Trials of the autotuners: every trial starts from the state saved when the
// tuner began and the batch is left in that state at the end.
struct TrialRunner {
    pirrt_batch *B;
    pirrt_graph *G;
    StateSnapshot snap;
    int deep0 = 0, expl0 = 0;
    unsigned wave_epoch_max = 0;
    int trials = 0;

    explicit TrialRunner(pirrt_batch *b) : B(b), G(b->G) {}

    pirrt_status begin() {
        pirrt_status rc = batch_flush(B);
        if (rc) return rc;
        if ((rc = snapshot_io(G, snap, true))) return rc;
        deep0 = G->deep_hint;
        expl0 = G->exploits;
        return PIRRT_OK;
    }

    // One exploit with `o` from the saved state; its time in *ms.
    pirrt_status run(const pirrt_exploit_opts &o, float *ms) {
        pirrt_status rc;
        if (trials > 0) {
            if ((rc = snapshot_io(G, snap, false))) return rc;
            // wave stamps written by earlier trials stay below this value
            CK(cudaMemcpyAsync(&G->ctr->wave_epoch, &wave_epoch_max, sizeof(unsigned),
                               cudaMemcpyHostToDevice, G->stream));
        }
        ++trials;
        G->deep_hint = deep0;
        G->exploits = expl0;
        pirrt_exploit_stats st{};
        rc = pirrt_graph_exploit(G, &o, &st);
        if (rc == PIRRT_OK) {
            wave_epoch_max = std::max(wave_epoch_max, G->ctr_host->wave_epoch + 1u);
            *ms = st.ms_exploit;
        }
        return rc;
    }

    // Back to the saved state.
    pirrt_status end() {
        pirrt_status rc = PIRRT_OK;
        if (trials > 0) {
            rc = snapshot_io(G, snap, false);
            if (rc == PIRRT_OK && wave_epoch_max &&
                cudaMemcpyAsync(&G->ctr->wave_epoch, &wave_epoch_max, sizeof(unsigned),
                                cudaMemcpyHostToDevice, G->stream) != cudaSuccess)
                rc = PIRRT_ERR_CUDA;
        }
        cudaStreamSynchronize(G->stream);
        G->deep_hint = deep0;
        G->exploits = expl0;
        if (snap.buf) cudaFree(snap.buf);
        snap.buf = nullptr;
        return rc;
    }
};

pirrt_status pirrt_batch_autotune(pirrt_batch *B, const pirrt_exploit_opts *cand, int32_t n,
                                  pirrt_exploit_opts *best, int32_t *best_index, float *best_ms) {
    if (!B || !cand || n <= 0 || !best) return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = B->G;
    CK(cudaSetDevice(G->cfg.device));
    TrialRunner tr(B);
    pirrt_status rc = tr.begin();
    float tbest = 0.f;
    int ibest = -1;
    for (int32_t i = 0; i < n && rc == PIRRT_OK; ++i) {
        float ms = 0.f;
        rc = tr.run(cand[i], &ms);
        if (rc == PIRRT_OK && (ibest < 0 || ms < tbest)) {
            tbest = ms;
            ibest = i;
        }
    }
    const pirrt_status rc2 = tr.end();
    if (rc) return rc;
    if (rc2) return rc2;
    *best = cand[ibest];
    if (best_index) *best_index = ibest;
    if (best_ms) *best_ms = tbest;
    return PIRRT_OK;
}

namespace {
// The option space of the searching autotuner: one list of values per
// option, searched one coordinate at a time.
struct TuneDim {
    const char *name;
    std::vector<double> values;
    void (*set)(pirrt_exploit_opts &, double);
};

std::vector<TuneDim> tune_dims(int32_t cost_dtype) {
    std::vector<TuneDim> d;
    d.push_back({"tile", {0, 2}, [](pirrt_exploit_opts &o, double v) { o.tile = (int32_t)v; }});
    d.push_back({"group",
                 cost_dtype == PIRRT_COST_F32 ? std::vector<double>{2, 4, 8}
                                              : std::vector<double>{4, 8, 16},
                 [](pirrt_exploit_opts &o, double v) { o.group = (int32_t)v; }});
    d.push_back({"dense_fraction", {0.1, 0.2, 0.35, 0.5, 0.8},
                 [](pirrt_exploit_opts &o, double v) { o.dense_fraction = v; }});
    d.push_back({"evaluate", {PIRRT_EVAL_AUTO, PIRRT_EVAL_WAVE},
                 [](pirrt_exploit_opts &o, double v) { o.evaluate = (int32_t)v; }});
    d.push_back({"wave_ctas", {1, 2}, [](pirrt_exploit_opts &o, double v) { o.wave_ctas = (int32_t)v; }});
    d.push_back({"wave_local", {-1, 4, 32},
                 [](pirrt_exploit_opts &o, double v) { o.wave_local = (int32_t)v; }});
    d.push_back({"wave_local_max", {32, 128, 512},
                 [](pirrt_exploit_opts &o, double v) { o.wave_local_max = (int32_t)v; }});
    d.push_back({"wave_local_step", {1024, 4096, 16384},
                 [](pirrt_exploit_opts &o, double v) { o.wave_local_step = (int32_t)v; }});
    d.push_back({"wave_tail", {-1, 64, 256},
                 [](pirrt_exploit_opts &o, double v) { o.wave_tail = (int32_t)v; }});
    return d;
}

bool same_opts(const pirrt_exploit_opts &a, const pirrt_exploit_opts &b) {
    return std::memcmp(&a, &b, sizeof(a)) == 0;
}
}  // namespace

pirrt_status pirrt_batch_autotune_search(pirrt_batch *B, const pirrt_exploit_opts *start,
                                         int32_t max_trials, pirrt_exploit_opts *best,
                                         float *best_ms, int32_t *trials) {
    if (!B || !best || max_trials < 1) return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = B->G;
    CK(cudaSetDevice(G->cfg.device));
    pirrt_exploit_opts cur{};
    if (start) cur = *start;
    // the defaults, written out, so that each coordinate starts from a value
    // of its list
    if (cur.group == 0) cur.group = 4;
    if (cur.dense_fraction == 0.0) cur.dense_fraction = 0.35;
    if (cur.wave_ctas == 0) cur.wave_ctas = 2;
    if (cur.wave_local == 0) cur.wave_local = 32;
    if (cur.wave_local_max == 0) cur.wave_local_max = 128;
    if (cur.wave_local_step == 0) cur.wave_local_step = 4096;
    if (cur.wave_tail == 0) cur.wave_tail = 64;
    const std::vector<TuneDim> dims = tune_dims(G->cfg.cost_dtype);
    TrialRunner tr(B);
    pirrt_status rc = tr.begin();
    float tcur = 0.f;
    if (rc == PIRRT_OK) rc = tr.run(cur, &tcur);
    // coordinate descent: a value replaces the current one only if it is
    // faster by more than 1% (trial times vary by a fraction of that), and
    // the passes stop when one changes nothing or the trials run out
    bool improved = true;
    while (rc == PIRRT_OK && improved && tr.trials < max_trials) {
        improved = false;
        for (const TuneDim &dim : dims) {
            for (double v : dim.values) {
                if (rc != PIRRT_OK || tr.trials >= max_trials) break;
                pirrt_exploit_opts o = cur;
                dim.set(o, v);
                if (same_opts(o, cur)) continue;
                float ms = 0.f;
                rc = tr.run(o, &ms);
                if (rc == PIRRT_OK && ms < 0.99f * tcur) {
                    cur = o;
                    tcur = ms;
                    improved = true;
                }
            }
        }
    }
    const int32_t n_trials = tr.trials;
    const pirrt_status rc2 = tr.end();
    if (rc) return rc;
    if (rc2) return rc2;
    *best = cur;
    if (best_ms) *best_ms = tcur;
    if (trials) *trials = n_trials;
    return PIRRT_OK;
}

pirrt_status pirrt_batch_get_costs(const pirrt_batch *B, int32_t graph, double *g_out, int64_t n,
                                   int on_device) {
    if (!B || graph < 0 || graph >= B->n_graphs || n < 0 || n > B->cap_v[graph] || (n > 0 && !g_out))
        return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = B->G;
    CK(cudaSetDevice(G->cfg.device));
    if (n > 0)
        CK(cudaMemcpyAsync(g_out, G->g + B->base[graph], sizeof(double) * (size_t)n,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_batch_get_parents(const pirrt_batch *B, int32_t graph, int32_t *p_out, int64_t n,
                                     int on_device) {
    if (!B || graph < 0 || graph >= B->n_graphs || n < 0 || n > B->cap_v[graph] || (n > 0 && !p_out))
        return PIRRT_ERR_INVALID_ARG;
    pirrt_graph *G = B->G;
    CK(cudaSetDevice(G->cfg.device));
    if (n > 0) {
        int32_t *dst = on_device ? p_out : G->pexport;
        export_parents_local_kernel<<<grid_for(n, kThreads, G->num_sms * 8), kThreads, 0,
                                      G->stream>>>(n, B->base[graph], G->p, dst);
        CKL();
        if (!on_device)
            CK(cudaMemcpyAsync(p_out, G->pexport, sizeof(int32_t) * (size_t)n,
                               cudaMemcpyDeviceToHost, G->stream));
    }
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

}  // extern "C"
