// Host runtime and C ABI of the single-graph PI-RRT# exploitation path.
//
// All graph state (CSR, g, parents, work lists) stays resident on the
// device; the host only sequences kernels on the caller's stream and reads
// one small counter block per Replan iteration to test convergence (Alg. 2:
// stop when Improve switched no parent).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "graph_kernels.cuh"
#include "improve_tma.cuh"
#include "improve_tpv.cuh"
#include "pirrt.h"

using namespace pirrt;

struct pirrt_graph {
    pirrt_config cfg{};
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int64_t cap_n = 0, cap_e = 0;  // vertices, directed CSR entries
    int64_t n = 0, m = 0;
    size_t entry_bytes = 0, cost_bytes = 0;
    int cur = 0;                   // live CSR buffer
    int64_t *row_off[2] = {nullptr, nullptr};
    void *adj[2] = {nullptr, nullptr};
    double *g = nullptr;
    float *g32 = nullptr;  // FP32 shadow of g for candidate screening
    int32_t *p = nullptr;
    void *pc = nullptr;
    int32_t *deg = nullptr;
    long long *tile_sums = nullptr;
    unsigned *stamp = nullptr;
    unsigned epoch = 1;            // stamp value of the current Improve list
    int32_t *list[2] = {nullptr, nullptr};
    int la = 0;                    // current Improve list
    int32_t *switched = nullptr;
    int32_t *dg = nullptr;
    int32_t *anc[2] = {nullptr, nullptr};
    double *acc[2] = {nullptr, nullptr};
    int32_t *done = nullptr;
    int32_t *wl[2] = {nullptr, nullptr};  // jump work lists; also the wave's level lists
    unsigned *wstamp = nullptr;           // wave child dedup
    unsigned wave_epoch = 1;
    int deep_hint = 0;                    // AUTO: recent exploits met waves past the cap
    int exploits = 0;
    DevCounters *ctr = nullptr;
    DevCounters *ctr_host = nullptr;  // pinned mirror
    void *stage = nullptr;            // device staging for host-side inputs
    size_t stage_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int eval_blocks = 0;
    int wave_blocks = 0;
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


template <typename CT, int TH, int TV, int PER>
pirrt_status launch_improve_tile_v(pirrt_graph *G, const ImproveArgs<CT> &a) {
    static int occ = -1;
    if (occ < 0) {
        int nb = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, improve_tile_kernel<CT, TH, TV, PER>,
                                                         TH, 0));
        occ = nb > 0 ? nb : 1;
    }
    improve_tile_kernel<CT, TH, TV, PER><<<G->num_sms * occ, TH, 0, G->stream>>>(a);
    CKL();
    return PIRRT_OK;
}

template <typename CT>
pirrt_status launch_improve_tma(pirrt_graph *G, const ImproveArgs<CT> &a) {
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
    improve_tma_kernel<CT><<<G->num_sms * occ, tma::kThreads, smem, G->stream>>>(a);
    CKL();
    return PIRRT_OK;
}

template <typename CT>
pirrt_status launch_improve_tpv(pirrt_graph *G, const ImproveArgs<CT> &a) {
    if constexpr (sizeof(CT) != 4) {
        return launch_improve_tile_v<CT, 64, 16, 8>(G, a);
    } else {
        static int occ = -1;
        if (occ < 0) {
            int nb = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, improve_tpv_kernel, kTpvThreads, 0));
            occ = nb > 0 ? nb : 1;
        }
        improve_tpv_kernel<<<G->num_sms * occ, kTpvThreads, 0, G->stream>>>(a);
        CKL();
        return PIRRT_OK;
    }
}

// Tiled Improve shapes (vertices per tile -> threads, entries per thread);
// 1 = the staged (bulk-copy pipelined) kernel; 2 = one thread per vertex.
template <typename CT>
pirrt_status launch_improve_tile(pirrt_graph *G, const ImproveArgs<CT> &a, int tile) {
    switch (tile) {
        case 1: return launch_improve_tma<CT>(G, a);
        case 2: return launch_improve_tpv<CT>(G, a);
        case 16: return launch_improve_tile_v<CT, 64, 16, 8>(G, a);
        case 32: return launch_improve_tile_v<CT, 128, 32, 8>(G, a);
        case 64: return launch_improve_tile_v<CT, 256, 64, 8>(G, a);
        case 128: return launch_improve_tile_v<CT, 256, 128, 8>(G, a);
        default: return launch_improve_tile_v<CT, 64, 16, 8>(G, a);
    }
}

template <typename CT, int GS>
pirrt_status launch_improve_g(pirrt_graph *G, const ImproveArgs<CT> &a) {
    static int occ = -1;
    if (occ < 0) {
        int nb = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, improve_kernel<CT, GS>, kThreads, 0));
        occ = nb > 0 ? nb : 1;
    }
    improve_kernel<CT, GS><<<G->num_sms * occ, kThreads, 0, G->stream>>>(a);
    CKL();
    return PIRRT_OK;
}

template <int GS, int U>
pirrt_status launch_improve_screen(pirrt_graph *G, const ImproveArgs<float> &a) {
    static int occ = -1;
    if (occ < 0) {
        int nb = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, improve_screen_kernel<GS, U>, 256, 0));
        occ = nb > 0 ? nb : 1;
    }
    improve_screen_kernel<GS, U><<<G->num_sms * occ, 256, 0, G->stream>>>(a);
    CKL();
    return PIRRT_OK;
}

// Improve kernel selection (pirrt_exploit_opts.tile / .group):
//   tile 0  G lanes per vertex (group, default 8) with FP32 screening; FP64
//           costs use the exact G-lane kernel
//   tile 1  staged: producer warp bulk-copies rows into a shared-memory ring
//   tile 2  one thread per vertex with FP32 screening
//   tile 3  G lanes per vertex, exact FP64 for every candidate
//   16..128 vertices per CTA tile of the unstaged tiled kernel
template <typename CT>
pirrt_status launch_improve(pirrt_graph *G, int gs, int tile) {
    ImproveArgs<CT> a;
    a.row_off = G->row_off[G->cur];
    a.adj = static_cast<const Entry<CT> *>(G->adj[G->cur]);
    a.g = G->g;
    a.g32 = G->g32;
    a.p = G->p;
    a.pc = static_cast<CT *>(G->pc);
    a.active = G->list[G->la];
    a.switched = G->switched;
    a.ctr = G->ctr;
    a.n = G->n;
    a.root = G->cfg.root;
    const int g = gs ? gs : 8;
    if (tile == 0) {
        if constexpr (sizeof(CT) == 4) {
            switch (gs) {
                case 1: return launch_improve_screen<1, 8>(G, a);
                case 2: return launch_improve_screen<2, 8>(G, a);
                case 8: return launch_improve_screen<8, 4>(G, a);
                case 16: return launch_improve_screen<16, 4>(G, a);
                case 32: return launch_improve_screen<32, 4>(G, a);
                case 5: return launch_improve_screen<4, 8>(G, a);  // 4 lanes, 8 in flight
                default: return launch_improve_screen<4, 4>(G, a);
            }
        }
        tile = 3;
    }
    if (tile == 3) {
        switch (g) {
            case 4: return launch_improve_g<CT, 4>(G, a);
            case 16: return launch_improve_g<CT, 16>(G, a);
            case 32: return launch_improve_g<CT, 32>(G, a);
            default: return launch_improve_g<CT, 8>(G, a);
        }
    }
    return launch_improve_tile<CT>(G, a, tile);
}

template <typename CT>
pirrt_status launch_evaluate(pirrt_graph *G, int force) {
    EvaluateArgs<CT> a;
    a.p = G->p;
    a.pc = static_cast<const CT *>(G->pc);
    a.g = G->g;
    a.g32 = G->g32;
    a.anc[0] = G->anc[0];
    a.anc[1] = G->anc[1];
    a.acc[0] = G->acc[0];
    a.acc[1] = G->acc[1];
    a.done = G->done;
    a.wl[0] = G->wl[0];
    a.wl[1] = G->wl[1];
    a.dg = G->dg;
    a.ctr = G->ctr;
    a.n = G->n;
    a.root = G->cfg.root;
    a.force = force;
    void *args[] = {&a};
    CK(cudaLaunchCooperativeKernel((const void *)evaluate_kernel<CT>, dim3(G->eval_blocks),
                                   dim3(kThreads), args, 0, G->stream));
    return PIRRT_OK;
}

template <typename CT>
pirrt_status launch_wave(pirrt_graph *G, unsigned dense_limit, unsigned max_levels) {
    WaveArgs<CT> a;
    a.row_off = G->row_off[G->cur];
    a.adj = static_cast<const Entry<CT> *>(G->adj[G->cur]);
    a.p = G->p;
    a.pc = static_cast<const CT *>(G->pc);
    a.g = G->g;
    a.g32 = G->g32;
    a.switched = G->switched;
    a.lvl[0] = G->wl[0];
    a.lvl[1] = G->wl[1];
    a.wstamp = G->wstamp;
    a.wave_epoch = G->wave_epoch;
    a.stamp = G->stamp;
    a.epoch = G->epoch + 1u;
    a.next = G->list[G->la ^ 1];
    a.ctr = G->ctr;
    a.root = G->cfg.root;
    a.dense_limit = dense_limit;
    a.max_levels = max_levels;
    void *args[] = {&a};
    CK(cudaLaunchCooperativeKernel((const void *)wave_evaluate_kernel<CT>, dim3(G->wave_blocks),
                                   dim3(kWaveThreads), args, 0, G->stream));
    return PIRRT_OK;
}

template <typename CT>
pirrt_status launch_mark(pirrt_graph *G, unsigned dense_limit) {
    MarkArgs<CT> a;
    a.row_off = G->row_off[G->cur];
    a.adj = static_cast<const Entry<CT> *>(G->adj[G->cur]);
    a.dg = G->dg;
    a.stamp = G->stamp;
    a.next = G->list[G->la ^ 1];
    a.ctr = G->ctr;
    a.epoch = G->epoch + 1u;
    a.root = G->cfg.root;
    a.dense_limit = dense_limit;
    mark_frontier_kernel<CT><<<G->num_sms * 8, kThreads, 0, G->stream>>>(a);
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
    // 1. validate and count new entries per row (into scratch only)
    CK(cudaMemsetAsync(G->deg, 0, sizeof(int32_t) * (size_t)(n_after + 1), G->stream));
    CK(cudaMemsetAsync(&G->ctr->status, 0, sizeof(unsigned), G->stream));
    if (n_edges > 0) {
        insert_validate_count<CT><<<grid_for(n_edges, kThreads, max_blocks), kThreads, 0, G->stream>>>(
            n_edges, src, dst, cost, n_after, G->deg, G->ctr);
        CKL();
    }
    CK(cudaMemcpyAsync(&G->ctr_host->status, &G->ctr->status, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    if (G->ctr_host->status) {
        CK(cudaMemsetAsync(&G->ctr->status, 0, sizeof(unsigned), G->stream));
        return fail(G, PIRRT_ERR_BAD_INPUT,
                    "insert_batch: edge with an id outside [0, %lld), a self loop, or a cost "
                    "that is not finite and > 0",
                    (long long)n_after);
    }
    // 2. new row offsets = old offsets + exclusive scan of the added counts
    const int nxt = G->cur ^ 1;
    const int64_t len = n_after + 1;
    const int64_t n_tiles = (len + kScanTile - 1) / kScanTile;
    scan_tile_reduce<<<(unsigned)n_tiles, kThreads, 0, G->stream>>>(G->deg, len, G->tile_sums);
    CKL();
    scan_tile_sums<<<1, kThreads, 0, G->stream>>>(G->tile_sums, n_tiles);
    CKL();
    scan_tile_apply<<<(unsigned)n_tiles, kThreads, 0, G->stream>>>(
        G->deg, len, G->tile_sums, G->row_off[G->cur], n_old, G->row_off[nxt]);
    CKL();
    // 3. old rows into the new buffer, new entries at the row tails
    const Entry<CT> *old_adj = static_cast<const Entry<CT> *>(G->adj[G->cur]);
    Entry<CT> *new_adj = static_cast<Entry<CT> *>(G->adj[nxt]);
    if (n_old > 0 && G->m > 0) {
        insert_copy_rows<CT><<<grid_for(n_old * 32, kThreads, max_blocks), kThreads, 0, G->stream>>>(
            n_old, G->row_off[G->cur], old_adj, G->row_off[nxt], new_adj);
        CKL();
    }
    if (n_edges > 0) {
        insert_scatter<CT><<<grid_for(n_edges, kThreads, max_blocks), kThreads, 0, G->stream>>>(
            n_edges, src, dst, cost, G->row_off[nxt], G->deg, new_adj, G->stamp, G->epoch,
            G->cfg.root, G->list[G->la], G->ctr);
        CKL();
    }
    // 4. seed the new vertices
    if (n_new > 0) {
        insert_init_vertices<CT><<<grid_for(n_new, kThreads, max_blocks), kThreads, 0, G->stream>>>(
            n_old, n_after, G->cfg.root, G->g, G->g32, G->p, static_cast<CT *>(G->pc), G->stamp,
            G->epoch,
            G->list[G->la], G->ctr);
        CKL();
    }
    G->prof.launches += 3 + (n_edges > 0 ? 2 : 0) + (n_old > 0 && G->m > 0 ? 1 : 0) + (n_new > 0 ? 1 : 0);
    G->prof.insert_calls += 1;
    G->prof.insert_new_entries += 2 * n_edges;
    G->prof.insert_copied_entries += G->m;
    if (prof) {
        CK(cudaEventRecord(G->pev[7], G->stream));
        CK(cudaEventSynchronize(G->pev[7]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, G->pev[6], G->pev[7]));
        G->prof.insert_ms += ms;
    }
    G->cur = nxt;
    G->n = n_after;
    G->m = m_after;
    return PIRRT_OK;
}

template <typename CT>
pirrt_status exploit_impl(pirrt_graph *G, const pirrt_exploit_opts *opts, pirrt_exploit_stats *st) {
    pirrt_exploit_opts o{};
    if (opts) o = *opts;
    if (o.max_iters < 0 || o.eps < 0.0 || o.dense_fraction < 0.0 || o.dense_fraction > 1.0 ||
        o.wave_levels < 0 || o.evaluate < PIRRT_EVAL_AUTO || o.evaluate > PIRRT_EVAL_JUMP ||
        !(o.tile == 0 || o.tile == 1 || o.tile == 2 || o.tile == 3 || o.tile == 16 ||
          o.tile == 32 || o.tile == 64 || o.tile == 128) ||
        !(o.group >= 0 && o.group <= 32))
        return fail(G, PIRRT_ERR_INVALID_ARG, "exploit: invalid option");
    const int64_t max_iters = o.max_iters > 0 ? o.max_iters : G->n + 2;
    const int gs = o.group;
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
    const unsigned max_levels = mode == PIRRT_EVAL_WAVE ? cap_any
                                : (o.wave_levels > 0 ? (unsigned)o.wave_levels : auto_cap);
    // AUTO: after an exploit whose waves ran past the cap, start with pointer
    // jumping, and probe with waves again every eighth exploit
    bool jump_first = mode == PIRRT_EVAL_AUTO && G->deep_hint && (G->exploits % 8) != 0;
    bool saw_deep = false;
    G->exploits += 1;

    CK(cudaEventRecord(G->ev0, G->stream));
    begin_exploit_kernel<<<1, 1, 0, G->stream>>>(G->ctr);
    CKL();
    G->prof.launches += 1;
    pirrt_exploit_stats s{};
    pirrt_status rc = PIRRT_OK;
    bool converged = false;
    unsigned long long prev_relax = 0, prev_improved = 0, prev_eval = 0;
    const bool prof = G->profiling != 0;
    pirrt_profile &P = G->prof;
    for (int64_t it = 0; it < max_iters; ++it) {
        // Improve, then Evaluate (+ frontier marking), then one counter read
        if (prof) CK(cudaEventRecord(G->pev[0], G->stream));
        if ((rc = launch_improve<CT>(G, gs, o.tile))) return rc;
        if (prof) CK(cudaEventRecord(G->pev[1], G->stream));
        bool jumped = false;
        if (mode == PIRRT_EVAL_JUMP || jump_first) {
            if ((rc = launch_evaluate<CT>(G, 0))) return rc;
            if (prof) CK(cudaEventRecord(G->pev[2], G->stream));
            if ((rc = launch_mark<CT>(G, dense_limit))) return rc;
            P.launches += 2;
            jumped = true;
        } else {
            if ((rc = launch_wave<CT>(G, dense_limit, max_levels))) return rc;
            if (prof) CK(cudaEventRecord(G->pev[2], G->stream));
            P.launches += 1;
        }
        if (prof) CK(cudaEventRecord(G->pev[3], G->stream));
        if ((rc = pull_counters(G))) return rc;
        P.launches += 1;
        const DevCounters *h = G->ctr_host;
        float t_imp = 0.f, t_eval = 0.f, t_mark = 0.f;
        if (prof) {
            CK(cudaEventElapsedTime(&t_imp, G->pev[0], G->pev[1]));
            CK(cudaEventElapsedTime(&t_eval, G->pev[1], G->pev[2]));
            CK(cudaEventElapsedTime(&t_mark, G->pev[2], G->pev[3]));
        }
        if (mode != PIRRT_EVAL_JUMP && !jumped) {
            G->wave_epoch += h->wave_levels + 1u;
            s.wave_levels += (int32_t)h->wave_levels;
            if (h->wave_incomplete) {
                saw_deep = true;
                if (mode == PIRRT_EVAL_AUTO) jump_first = true;
                // finish this Evaluate by pointer jumping from p and pc
                if (prof) CK(cudaEventRecord(G->pev[4], G->stream));
                pre_jump_kernel<<<1, 1, 0, G->stream>>>(G->ctr);
                CKL();
                if ((rc = launch_evaluate<CT>(G, 0))) return rc;
                if ((rc = launch_mark<CT>(G, dense_limit))) return rc;
                if (prof) CK(cudaEventRecord(G->pev[5], G->stream));
                if ((rc = pull_counters(G))) return rc;
                P.launches += 3;
                jumped = true;
                if (prof) {
                    float t = 0.f;
                    CK(cudaEventElapsedTime(&t, G->pev[4], G->pev[5]));
                    t_eval += t;
                }
            }
        }
        if (prof) {
            pirrt_trace_record tr{};
            tr.iteration = (int32_t)it;
            tr.dense = h->dense ? 1 : 0;
            tr.improve_vertices = (int64_t)(h->improved - prev_improved);
            tr.improve_entries = (int64_t)(h->relax - prev_relax);
            tr.switches = (int32_t)h->n_switched;
            tr.changed = (int32_t)h->n_dg;
            tr.wave_levels = (int32_t)h->wave_levels;
            tr.next_frontier = h->dense_next ? 0 : (int32_t)h->n_next;
            tr.improve_ms = t_imp;
            tr.evaluate_ms = t_eval;
            tr.mark_ms = jumped ? t_mark : 0.f;
            float t_it = 0.f;
            if (it > 0) CK(cudaEventElapsedTime(&t_it, G->it_start, G->pev[0]));
            tr.iteration_ms = t_it;  // previous iteration start to this one's start
            if (G->trace.size() < (1u << 22)) G->trace.push_back(tr);
            CK(cudaEventRecord(G->it_start, G->stream));
        }
        s.iterations += 1;
        s.switches += h->n_switched;
        s.jump_rounds += (int32_t)h->rounds;
        if (jumped && h->n_switched) s.jump_evaluates += 1;
        if (h->dense) s.dense_sweeps += 1;
        P.improve_launches += 1;
        P.improve_entries += (int64_t)(h->relax - prev_relax);
        P.improve_vertices += (int64_t)(h->improved - prev_improved);
        if (h->dense) P.improve_dense_vertices += (int64_t)(h->improved - prev_improved);
        P.improve_switches += h->n_switched;
        P.improve_ms += t_imp;
        prev_relax = h->relax;
        prev_improved = h->improved;
        if (h->n_switched) {
            P.evaluate_launches += 1;
            P.evaluate_vertices += (int64_t)(h->evaluated - prev_eval);
            P.evaluate_ms += t_eval;
            if (jumped) {
                for (int r = 1; r <= kMaxJumpRounds + 1; ++r) P.evaluate_visits += h->wl_count[r];
                P.evaluate_visits += G->n;  // round 0 touches every vertex
            }
            if (jumped && h->n_dg && h->n_dg <= dense_limit) {
                P.mark_launches += 1;
                P.mark_vertices += h->n_dg;
                P.mark_ms += t_mark;
            }
        }
        prev_eval = h->evaluated;
        if ((rc = status_from_bits(G, h->status))) break;
        // Alg. 2: stop once Delta g <= eps; with eps = 0 that is "no switch".
        // (The Evaluate of this iteration has already run, so g always
        // matches the returned policy.)
        double dj = 0.0;
        std::memcpy(&dj, &h->dj_bits, sizeof(dj));
        const bool stop = h->n_switched == 0u || dj <= o.eps;
        advance_kernel<<<1, 1, 0, G->stream>>>(G->ctr);
        CKL();
        P.launches += 1;
        G->la ^= 1;
        G->epoch += 1u;
        if (stop) {
            converged = true;
            break;
        }
    }
    if (mode == PIRRT_EVAL_AUTO && (saw_deep || !jump_first)) G->deep_hint = saw_deep ? 1 : 0;
    CK(cudaEventRecord(G->ev1, G->stream));
    if (rc == PIRRT_OK) {
        rc = pull_counters(G);
        if (rc) return rc;
    }
    CK(cudaEventSynchronize(G->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, G->ev0, G->ev1));
    const DevCounters &h = *G->ctr_host;
    s.converged = converged ? 1 : 0;
    s.relaxations = (int64_t)h.relax;
    s.improved = (int64_t)h.improved;
    s.evaluated = (int64_t)h.evaluated;
    s.ms_exploit = ms;
    if (st) *st = s;
    if (rc) return rc;
    if (!converged)
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
        G->n, G->cfg.root, parent, G->row_off[G->cur], static_cast<const Entry<CT> *>(G->adj[G->cur]),
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
    begin_exploit_kernel<<<1, 1, 0, G->stream>>>(G->ctr);
    CKL();
    pirrt_status rc = launch_evaluate<CT>(G, 1);
    if (rc) return rc;
    if ((rc = pull_counters(G))) return rc;
    if ((rc = status_from_bits(G, G->ctr_host->status))) return rc;
    // the next Improve sweeps every vertex; the seeded list is moot
    begin_exploit_kernel<<<1, 1, 0, G->stream>>>(G->ctr);
    CKL();
    const unsigned one = 1u;
    CK(cudaMemcpyAsync(&G->ctr->dense, &one, sizeof(unsigned), cudaMemcpyHostToDevice, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

void free_all(pirrt_graph *G) {
    void *bufs[] = {G->row_off[0], G->row_off[1], G->adj[0], G->adj[1], G->g, G->g32, G->p, G->pc,
                    G->deg, G->tile_sums, G->stamp, G->list[0], G->list[1], G->switched,
                    G->dg, G->anc[0], G->anc[1], G->acc[0], G->acc[1], G->done, G->wl[0],
                    G->wl[1], G->wstamp, G->ctr, G->stage};
    for (void *q : bufs)
        if (q) cudaFree(q);
    if (G->ctr_host) cudaFreeHost(G->ctr_host);
    if (G->ev0) cudaEventDestroy(G->ev0);
    if (G->ev1) cudaEventDestroy(G->ev1);
    for (cudaEvent_t e : G->pev)
        if (e) cudaEventDestroy(e);
    if (G->it_start) cudaEventDestroy(G->it_start);
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
    ALLOC(G->row_off[0], sizeof(int64_t) * (nv + 1));
    ALLOC(G->row_off[1], sizeof(int64_t) * (nv + 1));
    // +16 entries: a staged row copy is rounded up to 16 bytes past the row
    ALLOC(G->adj[0], G->entry_bytes * (ne + 16));
    ALLOC(G->adj[1], G->entry_bytes * (ne + 16));
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
    ALLOC(G->done, sizeof(int32_t) * nv);
    ALLOC(G->wl[0], sizeof(int32_t) * nv);
    ALLOC(G->wl[1], sizeof(int32_t) * nv);
    ALLOC(G->wstamp, sizeof(unsigned) * nv);
    ALLOC(G->ctr, sizeof(DevCounters));
#undef ALLOC
    if (cudaMallocHost((void **)&G->ctr_host, sizeof(DevCounters)) != cudaSuccess)
        return bail(PIRRT_ERR_OOM);
    if (cudaEventCreate(&G->ev0) != cudaSuccess || cudaEventCreate(&G->ev1) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    for (cudaEvent_t &e : G->pev)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(PIRRT_ERR_CUDA);
    if (cudaEventCreate(&G->it_start) != cudaSuccess) return bail(PIRRT_ERR_CUDA);
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
    G->wave_blocks = G->num_sms * std::min(wocc, 2);
    pirrt_status rc = pirrt_graph_reset(G);
    if (rc) return bail(rc);
    *out = G;
    return PIRRT_OK;
}

pirrt_status pirrt_graph_reset(pirrt_graph *G) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    CK(cudaSetDevice(G->cfg.device));
    CK(cudaMemsetAsync(G->row_off[0], 0, sizeof(int64_t), G->stream));
    CK(cudaMemsetAsync(G->row_off[1], 0, sizeof(int64_t), G->stream));
    CK(cudaMemsetAsync(G->stamp, 0, sizeof(unsigned) * (size_t)G->cap_n, G->stream));
    CK(cudaMemsetAsync(G->wstamp, 0, sizeof(unsigned) * (size_t)G->cap_n, G->stream));
    CK(cudaMemsetAsync(G->ctr, 0, sizeof(DevCounters), G->stream));
    CK(cudaStreamSynchronize(G->stream));
    G->n = 0;
    G->m = 0;
    G->cur = 0;
    G->la = 0;
    G->epoch = 1;
    G->wave_epoch = 1;
    G->deep_hint = 0;
    G->exploits = 0;
    G->last_error.clear();
    return PIRRT_OK;
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
    if (G->cfg.cost_dtype == PIRRT_COST_F32) return exploit_impl<float>(G, opts, stats);
    return exploit_impl<double>(G, opts, stats);
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
    if (n > 0)
        CK(cudaMemcpyAsync(p_out, G->p, sizeof(int32_t) * (size_t)n,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_graph_set_profiling(pirrt_graph *G, int enable) {
    if (!G) return PIRRT_ERR_INVALID_ARG;
    G->profiling = enable ? 1 : 0;
    G->prof = pirrt_profile{};
    G->trace.clear();
    return PIRRT_OK;
}

int64_t pirrt_graph_get_trace(const pirrt_graph *G, pirrt_trace_record *out, int64_t cap) {
    if (!G) return -1;
    const int64_t n = (int64_t)G->trace.size();
    if (out && cap > 0) std::memcpy(out, G->trace.data(), sizeof(pirrt_trace_record) * (size_t)std::min(n, cap));
    return n;
}

pirrt_status pirrt_graph_get_profile(const pirrt_graph *G, pirrt_profile *out) {
    if (!G || !out) return PIRRT_ERR_INVALID_ARG;
    *out = G->prof;
    return PIRRT_OK;
}

pirrt_status pirrt_graph_get_adjacency(const pirrt_graph *Gc, int64_t *row_off, int32_t *col,
                                       void *cost, int on_device) {
    pirrt_graph *G = const_cast<pirrt_graph *>(Gc);
    if (!G) return PIRRT_ERR_INVALID_ARG;
    CK(cudaSetDevice(G->cfg.device));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (row_off)
        CK(cudaMemcpyAsync(row_off, G->row_off[G->cur], sizeof(int64_t) * (size_t)(G->n + 1), kind,
                           G->stream));
    if (G->m > 0 && (col || cost)) {
        // entries are (col, cost) records: split with strided 2-D copies
        const char *base = static_cast<const char *>(G->adj[G->cur]);
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

}  // extern "C"
