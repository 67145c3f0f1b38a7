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

// The list is split evenly over the CTAs.  One thread per listed vertex
// decides; the deciding vertices of a chunk of up to blockDim.x listed
// vertices are compacted in shared memory, then scanned by G lanes each,
// blockDim.x / G vertices at a time, so that every CTA scans about the same
// number of rows (most listed vertices decide: the offers that list them are
// the ones that beat the vertex's g).  Any grid of up to 512-thread blocks;
// every thread of the block calls it.
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
    __shared__ int32_t s_dv[512];     // deciding vertices of the chunk
    __shared__ double s_cur[512];     // ... and their cur = g(p(v)) + c(p(v), v)
    __shared__ unsigned s_nd;
    WarpStage<kStageCap> swq{s_sw[threadIdx.x >> 5], 0u};
    const int32_t *active = (c->la & 1u) ? a.list[1] : a.list[0];
    const int64_t count = (int64_t)c->n_active;
    const unsigned long long gpol = policy_evict_last();
    const int tid = threadIdx.x, lane = tid & 31;
    const int gl = lane & (G - 1), grp = tid / G, ngrp = (int)blockDim.x / G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const double bound = goal_bound(c, a.h);
    unsigned long long relax = 0, improved = 0, djmax = 0;

    const int64_t per = (count + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per;
    const int64_t hi = lo + per < count ? lo + per : count;
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        // ---- one thread per listed vertex: take its offer, compare with cur
        if (tid == 0) s_nd = 0u;
        __syncthreads();
        const int64_t i = base + tid;
        if (i < hi) {
            const int32_t v = __ldg(&active[i]);
            if (v != a.root) {
                const int32_t pv = a.p[v];
                const unsigned long long cb = a.cand[v];
                if (cb != kCandNone) a.cand[v] = kCandNone;
                if (pv != kRootMark) {
                    double cur = CUDART_INF;
                    if (pv >= 0) cur = ld_g(&a.g[pv], gpol) + widen(a.pc[v]);
                    // goal-directed: an offer that cannot make v promising is
                    // dropped (the row's best is no larger than any offer)
                    const double cv = __longlong_as_double((long long)cb);
                    if (cb < kCandNone && cv < cur && promising(a.h, v, cv, bound)) {
                        const unsigned k = atomicAdd(&s_nd, 1u);
                        s_dv[k] = v;
                        s_cur[k] = cur;
                    }
                    improved += 1;
                }
            }
        }
        __syncthreads();
        const int nd = (int)s_nd;
        // ---- deciding vertices: G lanes each scan the row exactly
        for (int r0 = 0; r0 < nd; r0 += ngrp) {
            const int k = r0 + grp;
            const bool mine = k < nd;
            int32_t sv = 0;
            double scur = 0.0;
            unsigned long long bv = kCandNone + 1ull;
            int32_t bid = INT_MAX;
            CT bw = CT(0);
            int64_t b = 0, e = 0;
            if (mine) {
                sv = s_dv[k];
                scur = s_cur[k];
                row_range(a.rows, sv, b, e);
                for (int64_t i0 = b + gl; i0 < e; i0 += (int64_t)G * kUnroll) {
                    Entry<CT> en[kUnroll];
#pragma unroll
                    for (int q = 0; q < kUnroll; ++q)
                        if (i0 + q * G < e) en[q] = ld_stream(&a.adj[i0 + q * G]);
                    double gv[kUnroll];
#pragma unroll
                    for (int q = 0; q < kUnroll; ++q)
                        gv[q] = (i0 + q * G < e) ? ld_g(&a.g[en[q].col], gpol) : CUDART_INF;
#pragma unroll
                    for (int q = 0; q < kUnroll; ++q) {
                        if (i0 + q * G < e) {
                            const unsigned long long vb =
                                (unsigned long long)__double_as_longlong(gv[q] + widen(en[q].w));
                            if (vb < bv || (vb == bv && (en[q].col < bid ||
                                                         (en[q].col == bid && en[q].w < bw)))) {
                                bv = vb;
                                bid = en[q].col;
                                bw = en[q].w;
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
        __syncthreads();  // s_dv / s_cur / s_nd are rewritten by the next chunk
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
