// Improve (Alg. 2; Sec. IV-B) with the CSR stream decoupled from the
// reduction: a producer warp stages each tile's rows into a ring of shared
// memory buffers with bulk asynchronous copies (cp.async.bulk, completing on
// an mbarrier), while consumer warps gather g for the staged entries and take
// the lexicographic argmin of (g(u) + c(u, v), u, c) per vertex, 8 lanes per
// vertex, in registers.  Several tiles are in flight per CTA, so HBM streams
// while the gathers and reductions of earlier tiles proceed.
#pragma once

#include "graph_kernels.cuh"

namespace pirrt {

namespace tma {

constexpr int kTV = 32;                 // vertices per tile (one producer lane each)
constexpr int kStages = 4;                 // ring depth
constexpr int kStageBytes = 16384;         // staged CSR bytes per tile
constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;  // + one producer warp
constexpr unsigned long long kWaitNs = 2000000000ull;  // give up a wait after 2 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait for the phase with the given parity; false after wait_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          unsigned long long wait_ns = kWaitNs) {
    const unsigned a = smem_addr(bar);
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > wait_ns) return false;
    }
}

// One bulk copy global -> shared, completion counted on `bar` (bytes, both
// addresses and the size multiples of 16).
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar, unsigned long long pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ float ld_g32(const float *p, unsigned long long pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
}

template <typename CT>
struct alignas(128) Stage {
    static constexpr int kCap = kStageBytes / (int)sizeof(Entry<CT>);
    Entry<CT> buf[kCap];
    int32_t v[kTV];        // vertex, -1 if none
    int32_t seg[kTV + 1];  // exclusive prefix of row lengths
    int32_t start[kTV];    // index in buf of the row's first entry
    long long gbase[kTV];  // first entry of row v (used when the tile overflows)
    int32_t overflow;         // rows did not fit: read them from global memory
};

template <typename CT>
struct alignas(128) Smem {
    Stage<CT> st[kStages];
    unsigned long long full[kStages], empty[kStages];
    int32_t abort;    // consumers: a wait ran out (written and read by consumers only)
};

}  // namespace tma

template <typename CT>
__global__ void __launch_bounds__(tma::kThreads)
improve_tma_kernel(const ImproveArgs<CT> *__restrict__ ap) {
    const ImproveArgs<CT> a = *ap;
    const int32_t *active = a.list[a.ctr->la & 1u];
    using namespace tma;
    using WB = typename CostBits<CT>::T;
    constexpr int ES = (int)sizeof(Entry<CT>);
    constexpr int kCap = Stage<CT>::kCap;
    static_assert(kCap % 2 == 0, "stage capacity");
    constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<CT> &S = *reinterpret_cast<Smem<CT> *>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool dense = a.ctr->dense != 0u;
    const int64_t count = dense ? a.n : (int64_t)a.ctr->n_active;
    const int64_t n_tiles = (count + kTV - 1) / kTV;
    const double bound = goal_bound(a.ctr, a.h);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // From here on the producer warp and the consumer warps never meet at a
    // CTA-wide barrier; consumers synchronise among themselves (named barrier
    // 1) and with the producer through the full / empty mbarriers only.

    if (warp == kConsumerWarps) {
        // ------------------------------------------------------------ producer
        const unsigned long long stream_pol = policy_evict_first();
        int it = 0;
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
            const int s = it % kStages;
            const unsigned ph = (unsigned)(it / kStages) & 1u;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&S.empty[s], ph ^ 1u);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) atomicOr(&a.ctr->status, kStatusTimeout);
                break;  // the consumers' own waits run out in turn
            }
            Stage<CT> &st = S.st[s];
            const int64_t t0 = tile * kTV;
            int32_t v = -1;
            long long b = 0;
            int deg = 0;
            if (t0 + lane < count) {
                v = dense ? (int32_t)(t0 + lane) : __ldg(&active[t0 + lane]);
                if (v == a.root) {
                    v = -1;
                } else {
                    int64_t rb, re;
                    row_range(a.rows, v, rb, re);
                    b = rb;
                    deg = (int)(re - rb);
                }
            }
            // 16-byte aligned source and destination for each row: the copy
            // starts at the row start rounded down to 16 bytes (skipping at
            // most one 8-byte entry) and is rounded up to 16 bytes, so it may
            // read one entry past the row (the CSR buffers are padded)
            const long long byte0 = b * ES;
            const int skip = deg > 0 ? (int)((byte0 & 15) / ES) : 0;
            const int alloc = deg > 0 ? ((skip + deg) * ES + 15) / 16 * (16 / ES) : 0;
            int incl = deg, ainc = alloc;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                const int z = __shfl_up_sync(0xffffffffu, ainc, off);
                if (lane >= off) {
                    incl += y;
                    ainc += z;
                }
            }
            const int aex = ainc - alloc;
            const int atotal = __shfl_sync(0xffffffffu, ainc, 31);
            const bool ovf = atotal > kCap;
            st.v[lane] = v;
            st.seg[lane + 1] = incl;
            if (lane == 0) st.seg[0] = 0;
            st.start[lane] = aex + skip;
            st.gbase[lane] = b;
            if (lane == 0) st.overflow = ovf ? 1 : 0;
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(&S.full[s], ovf ? 0u : (unsigned)(atotal * ES));
            __syncwarp();
            if (!ovf && deg > 0) {
                const char *src = reinterpret_cast<const char *>(a.adj) + (byte0 - skip * ES);
                bulk_copy(&st.buf[aex], src, (unsigned)(alloc * ES), &S.full[s], stream_pol);
            }
        }
        // before leaving, see the copies of the last stages land (also when
        // the consumers have given up), so no bulk copy outlives the CTA
        if (lane == 0) {
            const int last = it < kStages ? it : kStages;
            for (int j = 1; j <= last; ++j) {
                const int k = it - j;
                mbar_wait(&S.full[k % kStages], (unsigned)(k / kStages) & 1u);
            }
        }
        __syncwarp();
    } else {
        // ----------------------------------------------------------- consumers
        // kConsumers / kTV = 8 lanes per vertex of the tile: each lane scans
        // every 8th staged entry of its vertex's row, keeping the
        // lexicographic minimum of (value bits, id, cost bits) in registers
        // (integer compares on order-preserving bits), then three xor-shuffle
        // steps reduce the 8 lanes.  No shared-memory atomics.
        constexpr int GL = kConsumers / kTV;
        static_assert(GL == 8, "8 lanes per vertex");
        const int k = tid / GL, gl = tid % GL;
        const unsigned long long gpol = policy_evict_last();
        const unsigned gmask = 0xffu << (lane & ~(GL - 1));
        unsigned long long relax = 0, improved = 0;
        int it = 0;
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
            const int s = it % kStages;
            const unsigned ph = (unsigned)(it / kStages) & 1u;
            // every consumer thread waits (acquiring the staged bytes); a
            // timeout anywhere is agreed on before anyone leaves the loop
            if (!mbar_wait(&S.full[s], ph)) S.abort = 1;
            consumer_sync();
            if (S.abort) {
                if (tid == 0) atomicOr(&a.ctr->status, kStatusTimeout);
                break;
            }
            Stage<CT> &st = S.st[s];
            const bool ovf = st.overflow != 0;
            const int32_t v = st.v[k];
            const int deg = st.seg[k + 1] - st.seg[k];
            const int sidx = st.start[k];
            const long long gbase = st.gbase[k];
            int32_t pv = -1;
            CT pcv = CT(0);
            double gp = CUDART_INF;
            if (gl == 0 && v >= 0) {  // current parent's candidate, in flight meanwhile
                pv = a.p[v];
                pcv = a.pc[v];
                if (pv >= 0) gp = a.g[pv];
            }
            unsigned long long bv = kInfBits + 1ull;  // above +inf: "no candidate yet"
            int32_t bid = INT_MAX;
            WB bw = CostBits<CT>::kMax;
            // candidate j of this lane's share of the row
            auto entry = [&](int j) -> Entry<CT> {
                return ovf ? ld_stream(&a.adj[gbase + j]) : st.buf[sidx + j];
            };
            auto exact = [&](const Entry<CT> &e, double gu) {
                const unsigned long long vb =
                    (unsigned long long)__double_as_longlong(gu + widen(e.w));
                const WB wb = CostBits<CT>::of(e.w);
                if (vb < bv || (vb == bv && (e.col < bid || (e.col == bid && wb < bw)))) {
                    bv = vb;
                    bid = e.col;
                    bw = wb;
                }
            };
            bool screen = false;
            float tau = 0.f;
            if constexpr (sizeof(CT) == 4) {
                // Screening in FP32.  With g32 = fl32(g) and a = fl32(g32 + c),
                // |a - fl64(g + c)| <= 2^-22 a, so the exact lexicographic
                // minimum, and every candidate tying its value, satisfy
                // a <= A* (1 + 2^-22) / (1 - 2^-22) with A* = min a; tau
                // below is larger still.  Rows reading a g32 of -1 (g above
                // 2^100) or overflowing to +inf take the exact path.
                float amin = __int_as_float(0x7f800000);
                int exact_row = 0;
                for (int j0 = gl; j0 < deg; j0 += GL * 4) {
                    Entry<CT> en[4];
                    float g32u[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j0 + q * GL < deg) en[q] = entry(j0 + q * GL);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j0 + q * GL < deg) g32u[q] = ld_g32(&a.g32[en[q].col], gpol);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (j0 + q * GL < deg) {
                            const float av = g32u[q] + (float)en[q].w;
                            exact_row |= (g32u[q] < 0.f) | (isinf(av) & !isinf(g32u[q]));
                            amin = fminf(amin, av);
                        }
                    }
                }
#pragma unroll
                for (int off = GL / 2; off > 0; off >>= 1) {
                    amin = fminf(amin, __shfl_xor_sync(gmask, amin, off, GL));
                    exact_row |= __shfl_xor_sync(gmask, exact_row, off, GL);
                }
                if (!exact_row) {
                    screen = true;
                    tau = amin * (1.0f + 0x1p-20f) + 0x1p-125f;  // +inf when nothing is reachable
                }
            }
            // (a screened row whose every candidate is unreachable has tau = +inf)
            if (!(screen && isinf(tau))) {
                for (int j0 = gl; j0 < deg; j0 += GL * 4) {
                    Entry<CT> en[4];
                    bool keep[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        keep[q] = false;
                        if (j0 + q * GL < deg) {
                            en[q] = entry(j0 + q * GL);
                            keep[q] = true;
                        }
                    }
                    if constexpr (sizeof(CT) == 4) {
                        if (screen) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                if (keep[q])
                                    keep[q] = ld_g32(&a.g32[en[q].col], gpol) + (float)en[q].w <= tau;
                        }
                    }
                    double gv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (keep[q]) gv[q] = ld_g(&a.g[en[q].col], gpol);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (keep[q]) exact(en[q], gv[q]);
                }
            }
            // the staged bytes are no longer needed: release the stage
            consumer_sync();
            if (tid == 0) mbar_arrive(&S.empty[s]);
#pragma unroll
            for (int off = GL / 2; off > 0; off >>= 1) {
                const unsigned long long ov = __shfl_xor_sync(gmask, bv, off, GL);
                const int32_t oi = __shfl_xor_sync(gmask, bid, off, GL);
                const WB ow = __shfl_xor_sync(gmask, bw, off, GL);
                if (ov < bv || (ov == bv && (oi < bid || (oi == bid && ow < bw)))) {
                    bv = ov;
                    bid = oi;
                    bw = ow;
                }
            }
            // decision by each group's first lane; appends are warp-collective
            bool sw = false;
            unsigned long long dj = 0ull;
            if (gl == 0 && v >= 0 && pv != kRootMark) {
                const double cur = pv >= 0 ? gp + widen(pcv) : CUDART_INF;
                if (bv <= kInfBits) {
                    const double best = __longlong_as_double((long long)bv);
                    if (best < cur && promising(a.h, v, best, bound)) {
                        a.p[v] = bid;
                        a.pc[v] = CostBits<CT>::back(bw);
                        sw = true;
                        dj = (unsigned long long)__double_as_longlong(cur - best);
                    }
                }
                relax += (unsigned long long)deg;
                improved += 1;
            }
            warp_append(sw, v, a.switched, &a.ctr->n_switched);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, dj, off);
                dj = o > dj ? o : dj;
            }
            if (lane == 0 && dj) atomicMax(&a.ctr->dj_bits, dj);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            relax += __shfl_down_sync(0xffffffffu, relax, off);
            improved += __shfl_down_sync(0xffffffffu, improved, off);
        }
        if (lane == 0 && (relax || improved)) {
            atomicAdd(&a.ctr->relax, relax);
            atomicAdd(&a.ctr->improved, improved);
        }
    }
}

}  // namespace pirrt
