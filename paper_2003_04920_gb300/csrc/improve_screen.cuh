// Improve (Alg. 2; Sec. IV-B) for FP32 edge costs with candidates screened
// in FP32 (GB300 issues FP64 at a small fraction of its FP32 rate): the
// exact FP64 sum g(u) + c(u, v) is formed only for the FP32 argmin, or for
// every candidate within the screening margin when a near tie leaves more
// than one in play, so parents and g are those of the FP64 rule.
#pragma once

#include "graph_kernels.cuh"

namespace pirrt {

__device__ __forceinline__ float ld_g32f(const float *p, unsigned long long pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}



// Improve with G lanes per vertex and FP32 screening (FP32 costs).  Each
// lane scans every G-th entry of the row, four entries and four FP32 gathers
// in flight, tracking (minimum, entry of the minimum, second minimum) of the
// FP32 screen; G-lane shuffles merge them.  The exact FP64 sum is formed for
// the FP32 argmin alone, unless another candidate lies within the screening
// margin, in which case the group rescans the row exactly.  No shared memory,
// no CTA barriers, no FP64 arithmetic per entry.
// The body, for blocks of THREADS threads (every thread of the block calls
// it): the kernel below, and the wave's launch, which runs the dense sweeps
// itself (replan_iteration.cuh).
template <int G, int kU, int THREADS>
__device__ void improve_screen_body(const ImproveArgs<float> &a) {
    const int32_t *active = a.list[a.ctr->la & 1u];
    constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;
    constexpr int kStageCap = 128;
    __shared__ int32_t s_sw[THREADS / 32][kStageCap];
    WarpStage<kStageCap> swq{s_sw[threadIdx.x >> 5], 0u};
    const unsigned long long gpol = policy_evict_last();
    const int lane = threadIdx.x & 31, gl = threadIdx.x & (G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    (void)gmask;
    const int gpb = THREADS / G;
    const int64_t gstride = (int64_t)gridDim.x * gpb;
    const bool dense = a.ctr->dense != 0u;
    if (a.push && !dense) return;  // list sweeps run from offers
    const int64_t count = dense ? a.n : (int64_t)a.ctr->n_active;
    const float kInf = __int_as_float(0x7f800000);
    const double bound = goal_bound(a.ctr, a.h);
    unsigned long long relax = 0, improved = 0, djmax = 0;
    // whole warps iterate together so the appends below are warp-collective.
    // The next iteration's vertex and row extent are loaded one iteration
    // ahead, and within a row the next batch of entries is requested before
    // the current batch's FP32 gathers are consumed.
    const int64_t first = (int64_t)blockIdx.x * gpb + (threadIdx.x >> 5) * (32 / G);
    const int64_t warp_span = 32 / G;
    auto fetch = [&](int64_t wb, int32_t &v, int64_t &b, int64_t &e) {
        const int64_t item = wb + (lane / G);
        v = -1;
        b = e = 0;
        if (item < count) {
            v = dense ? (int32_t)item : __ldg(&active[item]);
            if (v == a.root) v = -1;
            else {
                row_range(a.rows, v, b, e);
            }
        }
    };
    int32_t nv_;
    int64_t nb_, ne_;
    fetch(first, nv_, nb_, ne_);
    for (int64_t wbase = first; wbase < count; wbase += gstride) {
        const int32_t v = nv_;
        const int64_t b = nb_, e = ne_;
        if (wbase + gstride < count) fetch(wbase + gstride, nv_, nb_, ne_);
        bool sw = false;
        unsigned long long dj = 0ull;
        if (v >= 0) {  // uniform within the group
            int32_t pv = -1;
            float pcv = 0.f;
            double gp = CUDART_INF;
            if (gl == 0) {
                pv = a.p[v];
                pcv = a.pc[v];
                if (pv >= 0) gp = a.g[pv];
            }
            float m1 = kInf, m2 = kInf;
            int64_t i1 = -1;
            int exact_row = 0;
            Entry<float> en[kU];
            int64_t i0 = b + gl;
#pragma unroll
            for (int q = 0; q < kU; ++q)
                if (i0 + q * G < e) en[q] = ld_stream(&a.adj[i0 + q * G]);
            for (; i0 < e; i0 += (int64_t)G * kU) {
                float gu[kU];
#pragma unroll
                for (int q = 0; q < kU; ++q)
                    if (i0 + q * G < e) gu[q] = ld_g32f(&a.g32[en[q].col], gpol);
                Entry<float> nx[kU];
                const int64_t i1n = i0 + (int64_t)G * kU;
#pragma unroll
                for (int q = 0; q < kU; ++q)
                    if (i1n + q * G < e) nx[q] = ld_stream(&a.adj[i1n + q * G]);
#pragma unroll
                for (int q = 0; q < kU; ++q) {
                    if (i0 + q * G < e) {
                        const float av = gu[q] + en[q].w;
                        exact_row |= (gu[q] < 0.f) | (isinf(av) & !isinf(gu[q]));
                        if (av < m1) {
                            m2 = m1;
                            m1 = av;
                            i1 = i0 + q * G;
                        } else if (av < m2) {
                            m2 = av;
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kU; ++q) en[q] = nx[q];
            }
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                const float om1 = __shfl_xor_sync(gmask, m1, off, G);
                const float om2 = __shfl_xor_sync(gmask, m2, off, G);
                const int64_t oi1 = __shfl_xor_sync(gmask, i1, off, G);
                exact_row |= __shfl_xor_sync(gmask, exact_row, off, G);
                const float lo = fminf(m1, om1), hi = fmaxf(m1, om1);
                if (om1 < m1 || (om1 == m1 && oi1 >= 0 && (i1 < 0 || oi1 < i1))) i1 = oi1;
                m2 = fminf(hi, fminf(m2, om2));
                m1 = lo;
            }
            // exact FP64 lexicographic minimum over the candidates in play
            unsigned long long bv = kInfBits + 1ull;
            int32_t bid = INT_MAX;
            unsigned bw = 0xffffffffu;
            const float tau = m1 * (1.0f + 0x1p-20f) + 0x1p-125f;
            const bool rescan = exact_row || (m2 <= tau && !isinf(m1));
            if (rescan) {
                for (int64_t i = b + gl; i < e; i += G) {
                    const Entry<float> en = a.adj[i];
                    if (exact_row || ld_g32f(&a.g32[en.col], gpol) + en.w <= tau) {
                        const unsigned long long vb = (unsigned long long)__double_as_longlong(
                            ld_g(&a.g[en.col], gpol) + widen(en.w));
                        const unsigned wb = __float_as_uint(en.w);
                        if (vb < bv || (vb == bv && (en.col < bid || (en.col == bid && wb < bw)))) {
                            bv = vb;
                            bid = en.col;
                            bw = wb;
                        }
                    }
                }
#pragma unroll
                for (int off = G / 2; off > 0; off >>= 1) {
                    const unsigned long long ov = __shfl_xor_sync(gmask, bv, off, G);
                    const int32_t oi = __shfl_xor_sync(gmask, bid, off, G);
                    const unsigned ow = __shfl_xor_sync(gmask, bw, off, G);
                    if (ov < bv || (ov == bv && (oi < bid || (oi == bid && ow < bw)))) {
                        bv = ov;
                        bid = oi;
                        bw = ow;
                    }
                }
            } else if (gl == 0 && i1 >= 0 && !isinf(m1)) {
                const Entry<float> en = a.adj[i1];
                bv = (unsigned long long)__double_as_longlong(ld_g(&a.g[en.col], gpol) + widen(en.w));
                bid = en.col;
                bw = __float_as_uint(en.w);
            }
            if (gl == 0 && pv != kRootMark) {
                const double cur = pv >= 0 ? gp + widen(pcv) : CUDART_INF;
                if (bv <= kInfBits) {
                    const double best = __longlong_as_double((long long)bv);
                    if (best < cur && promising(a.h, v, best, bound)) {
                        a.p[v] = bid;
                        a.pc[v] = __uint_as_float(bw);
                        sw = true;
                        dj = (unsigned long long)__double_as_longlong(cur - best);
                    }
                }
                relax += (unsigned long long)(e - b);
                improved += 1;
            }
        }
        swq.push(sw, v, a.switched, &a.ctr->n_switched);
        djmax = dj > djmax ? dj : djmax;
        (void)warp_span;
    }
    // one atomic per block and counter (thousands of warps end together)
    __shared__ unsigned s_fl[THREADS / 32 + 1];
    __shared__ unsigned long long s_red[THREADS / 32];
    swq.flush_block(a.switched, &a.ctr->n_switched, s_fl);
    block_max(djmax, &a.ctr->dj_bits, s_red);
    block_add(relax, &a.ctr->relax, s_red);
    block_add(improved, &a.ctr->improved, s_red);
}

template <int G, int kU>
__global__ void __launch_bounds__(256)
improve_screen_kernel(const ImproveArgs<float> *__restrict__ ap) {
    const ImproveArgs<float> a = *ap;
    improve_screen_body<G, kU, 256>(a);
}

}  // namespace pirrt
