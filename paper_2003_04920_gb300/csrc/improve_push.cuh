// Improve (Alg. 2; Sec. IV-B) from offered candidates.
//
// After an Improve has processed v, its parent is optimal for the g of that
// moment (it switched to the argmin, or kept a parent that attains it), and
// Evaluate only ever lowers g.  So in a later Improve the only neighbours
// that can beat v's current parent are those whose g changed since, and each
// of them offered its candidate g(u) + c(u, v) when its row was scanned after
// the change (by Evaluate, by the frontier marking after pointer jumping, or
// by an insertion for a new edge): cand[v] holds the minimum of those offers,
// kept by an atomic minimum on the FP64 bits.  A listed vertex whose cand is
// not below cur = g(p(v)) + c(p(v), v) therefore keeps its parent without
// reading its row.  The others -- a small fraction -- scan their row exactly
// for the lexicographic argmin (value, id, cost) over every neighbour: the
// same rule, hence the same parent, as a full Improve.  An offer that is
// stale or spurious can only cause a needless scan, never a wrong parent.
#pragma once

#include "graph_kernels.cuh"

namespace pirrt {

// One thread per listed vertex decides; G lanes per deciding vertex scan.
// Any grid of up to 512-thread blocks; every thread of the block calls it.
template <typename CT, int G>
__device__ void improve_push_body(const ImproveArgs<CT> &a) {
    DevCounters *c = a.ctr;
    const int64_t tid0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    if (c->dense != 0u) {
        // the full sweep runs in the pull kernel; offers start afresh
        for (int64_t v = tid0; v < a.n; v += nthreads) a.cand[v] = kCandNone;
        return;
    }
    constexpr int kStageCap = 128;
    constexpr int kUnroll = 4;
    __shared__ int32_t s_sw[512 / 32][kStageCap];
    WarpStage<kStageCap> swq{s_sw[threadIdx.x >> 5], 0u};
    const int32_t *active = (c->la & 1u) ? a.list[1] : a.list[0];
    const int64_t count = (int64_t)c->n_active;
    const unsigned long long gpol = policy_evict_last();
    const int lane = threadIdx.x & 31, grp = lane / G, gl = lane & (G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int64_t wid = tid0 >> 5, nwarps = nthreads >> 5;
    const double bound = goal_bound(c, a.h);
    unsigned long long relax = 0, improved = 0, djmax = 0;

    for (int64_t base = wid * 32; base < count; base += nwarps * 32) {
        // ---- one thread per listed vertex: take its offer, compare with cur
        const int64_t i = base + lane;
        int32_t v = -1;
        double cur = CUDART_INF;
        bool want = false;
        if (i < count) {
            v = __ldg(&active[i]);
            if (v != a.root) {
                const int32_t pv = a.p[v];
                const unsigned long long cb = a.cand[v];
                if (cb != kCandNone) a.cand[v] = kCandNone;
                if (pv != kRootMark) {
                    if (pv >= 0) cur = ld_g(&a.g[pv], gpol) + widen(a.pc[v]);
                    // goal-directed: an offer that cannot make v promising is
                    // dropped (the row's best is no larger than any offer)
                    const double cv = __longlong_as_double((long long)cb);
                    want = cb < kCandNone && cv < cur && promising(a.h, v, cv, bound);
                    improved += 1;
                }
            }
        }
        // ---- deciding vertices: G lanes each scan the row exactly
        unsigned todo = __ballot_sync(0xffffffffu, want);
        while (todo) {
            unsigned t = todo;  // this group's vertex: the grp-th deciding lane
            for (int k = 0; k < grp && t; ++k) t &= t - 1u;
            const bool mine = t != 0u;
            const int s_lane = mine ? __ffs(t) - 1 : 0;
            const int32_t sv = __shfl_sync(0xffffffffu, v, s_lane);
            const double scur = __shfl_sync(0xffffffffu, cur, s_lane);
            // drop the vertices taken in this round
            for (int k = 0; k < 32 / G && todo; ++k) todo &= todo - 1u;
            unsigned long long bv = kCandNone + 1ull;
            int32_t bid = INT_MAX;
            CT bw = CT(0);
            int64_t b = 0, e = 0;
            if (mine) {
                row_range(a.rows, sv, b, e);
                for (int64_t i0 = b + gl; i0 < e; i0 += (int64_t)G * kUnroll) {
                    Entry<CT> en[kUnroll];
#pragma unroll
                    for (int k = 0; k < kUnroll; ++k)
                        if (i0 + k * G < e) en[k] = ld_stream(&a.adj[i0 + k * G]);
                    double gv[kUnroll];
#pragma unroll
                    for (int k = 0; k < kUnroll; ++k)
                        gv[k] = (i0 + k * G < e) ? ld_g(&a.g[en[k].col], gpol) : CUDART_INF;
#pragma unroll
                    for (int k = 0; k < kUnroll; ++k) {
                        if (i0 + k * G < e) {
                            const unsigned long long vb =
                                (unsigned long long)__double_as_longlong(gv[k] + widen(en[k].w));
                            if (vb < bv || (vb == bv && (en[k].col < bid ||
                                                         (en[k].col == bid && en[k].w < bw)))) {
                                bv = vb;
                                bid = en[k].col;
                                bw = en[k].w;
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                const unsigned long long ov = __shfl_xor_sync(gmask, bv, off, G);
                const int32_t oi = __shfl_xor_sync(gmask, bid, off, G);
                const CT ow = __shfl_xor_sync(gmask, bw, off, G);
                if (ov < bv || (ov == bv && (oi < bid || (oi == bid && ow < bw)))) {
                    bv = ov;
                    bid = oi;
                    bw = ow;
                }
            }
            bool sw = false;
            if (mine && gl == 0) {
                relax += (unsigned long long)(e - b);
                if (bv < kCandNone) {
                    const double best = __longlong_as_double((long long)bv);
                    if (best < scur && promising(a.h, sv, best, bound)) {
                        a.p[sv] = bid;
                        a.pc[sv] = bw;
                        sw = true;
                        const unsigned long long dj =
                            (unsigned long long)__double_as_longlong(scur - best);
                        djmax = dj > djmax ? dj : djmax;
                    }
                }
            }
            swq.push(sw, sv, a.switched, &c->n_switched);
        }
    }
    // one atomic per block and counter (thousands of warps end together)
    __shared__ unsigned s_fl[512 / 32 + 1];
    __shared__ unsigned long long s_red[512 / 32];
    swq.flush_block(a.switched, &c->n_switched, s_fl);
    block_max(djmax, &c->dj_bits, s_red);
    block_add(relax, &c->relax, s_red);
    block_add(improved, &c->improved, s_red);
}

template <typename CT, int G>
__global__ void __launch_bounds__(256, 4)
improve_push_kernel(const ImproveArgs<CT> *__restrict__ ap) {
    const ImproveArgs<CT> a = *ap;
    improve_push_body<CT, G>(a);
}

}  // namespace pirrt
