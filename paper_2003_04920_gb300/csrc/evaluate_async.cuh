// Evaluate (Alg. 2; Sec. IV-C) without level barriers.
//
// Improve only ever switches a vertex to a strictly cheaper parent, so under
// the new policy no cost-to-come rises: every value g holds at any moment of
// an Evaluate (the old value, or one computed from an ancestor's not-yet-final
// value) is at least the final one, and the final g(v) = g(p(v)) + c(p(v), v)
// is the minimum of all values ever computed for v.  Rounding is monotone, so
// this holds in FP64 as well.  g can therefore be updated with an atomic
// minimum on its bit pattern (non-negative doubles order like unsigned
// integers) in any order: a stale value can never overwrite a smaller one, and
// every vertex is recomputed once its parent holds its final value.  The
// result is the root-to-leaf sum of Alg. 2's breadth-first walk, bit for bit.
//
// Each CTA walks subtrees on its own: it takes up to kAsyncThreads vertices
// whose g was lowered, streams their concatenated rows with every thread
// (like the top-down wave), lowers each child (neighbour w with p(w) = v) to
// g(v) + c(v, w), marks every neighbour for the next Improve, and keeps the
// lowered children in a shared-memory stack for its next step.  There is no
// grid barrier per tree level: a level costs a few dependent L2 round trips
// instead of a grid-wide step.  Work moves between CTAs through an
// append-only global list: the switched vertices of Improve first, then the
// children a CTA cannot hold or hands over while other CTAs are idle.  The
// walk ends when every item is claimed and no CTA holds work.
#pragma once

#include "graph_kernels.cuh"

namespace pirrt {

constexpr int kAsyncThreads = 512;
constexpr int kAsyncUnroll = 4;
constexpr int kAsyncLocal = 4096;  // shared-memory stack entries per CTA
constexpr unsigned long long kAsyncPollLimit = 1ull << 22;  // idle polls (<= ~1 us each)

// Global state of the walk.  `tail` / `take` are monotonic over the graph's
// lifetime, so a slot of the spill list is recognised by its index (a slot
// left over from an earlier Evaluate carries an older index).
struct AsyncQueue {
    unsigned long long tail;  // spill items reserved
    unsigned long long take;  // spill items claimed
    unsigned long long base;  // tail when this Evaluate started
    unsigned start_take;      // switched vertices claimed
    int active;               // CTAs holding or claiming work
    unsigned done;            // termination detected
    unsigned abort;           // depth cap, spill-list overflow or timeout
    unsigned max_depth;       // deepest level reached
    unsigned pad[3];
};

struct AsyncItem {
    unsigned long long tag;  // index + 1 once the item is written
    double g;                // the lowered g of v
    int32_t v;
    int32_t depth;
};

template <typename CT>
struct AsyncArgs {
    const RowExt *rows;
    const Entry<CT> *adj;
    const int32_t *p;
    const CT *pc;
    double *g;
    float *g32;
    const int32_t *switched;  // vertices Improve re-parented
    int32_t *dg;              // vertices whose g changed (each once)
    unsigned *wstamp;         // first-change stamps (tag = wave_epoch)
    unsigned *swstamp;        // switched-vertex stamps (tag = wave_epoch)
    unsigned *stamp;          // Improve-list stamps
    int32_t *list[2];         // the next Improve list is list[(la & 1) ^ 1]
    DevCounters *ctr;
    AsyncQueue *q;
    AsyncItem *ring;          // spill list storage
    int64_t ring_cap;
    int32_t root;
    unsigned dense_limit;     // |changed| above this -> dense sweep next, stop marking
    unsigned max_levels;      // deeper than this: give up (wave_incomplete)
    int32_t push;             // offer g(v) + c(v, w) to every neighbour w of a lowered v
    unsigned long long *cand;
};

__device__ __forceinline__ unsigned vload(const unsigned *p) {
    return *reinterpret_cast<const volatile unsigned *>(p);
}
__device__ __forceinline__ int vload(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}
__device__ __forceinline__ unsigned long long vload(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// g(v) <- min(g(v), val); true if this call lowered it.
__device__ __forceinline__ bool lower_g(double *g, int32_t v, double val) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(val);
    const unsigned long long old = atomicMin(reinterpret_cast<unsigned long long *>(g + v), b);
    return old > b;
}

__device__ __forceinline__ void put_item(AsyncItem *ring, int64_t cap, unsigned long long idx,
                                         int32_t v, double gv, int32_t depth) {
    AsyncItem *it = &ring[idx % (unsigned long long)cap];
    __stcg(&it->g, gv);
    __stcg(&it->v, v);
    __stcg(&it->depth, depth);
    __threadfence();
    *reinterpret_cast<volatile unsigned long long *>(&it->tag) = idx + 1ull;
}

template <typename CT>
__global__ void __launch_bounds__(kAsyncThreads, 1)
async_evaluate_kernel(const AsyncArgs<CT> *__restrict__ ap) {
    const AsyncArgs<CT> a = *ap;
    DevCounters *c = a.ctr;
    AsyncQueue *q = a.q;
    const unsigned n_sw = c->n_switched;
    if (n_sw == 0u) return;

    extern __shared__ __align__(16) unsigned char async_smem[];
    double *s_lg = reinterpret_cast<double *>(async_smem);
    int32_t *s_lv = reinterpret_cast<int32_t *>(s_lg + kAsyncLocal);
    int32_t *s_ld = s_lv + kAsyncLocal;
    constexpr int NW = kAsyncThreads / 32;
    __shared__ int32_t s_u[kAsyncThreads];
    __shared__ double s_gu[kAsyncThreads];
    __shared__ int32_t s_du[kAsyncThreads];
    __shared__ long long s_base[kAsyncThreads];
    __shared__ int32_t s_seg[kAsyncThreads + 1];
    __shared__ int32_t s_wsum[NW];
    __shared__ unsigned long long s_scan[NW];
    __shared__ unsigned s_cnt;            // entries on the stack
    __shared__ int s_kind, s_nb;          // 0 stack, 1 switched list, 2 spill list, 3 stop
    __shared__ unsigned s_take0;          // first stack entry / switched index of the batch
    __shared__ unsigned long long s_spill0;
    __shared__ unsigned s_old, s_loc, s_mbase;
    __shared__ unsigned long long s_gbase;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned epoch = c->epoch + 1u;  // stamp of the list being built
    const unsigned tag = c->wave_epoch;    // first-change stamp of this Evaluate
    int32_t *next = ((c->la & 1u) ^ 1u) ? a.list[1] : a.list[0];
    const unsigned long long qbase = vload(&q->base);
    const unsigned long long gpol = policy_evict_last();
    const unsigned long long cap = (unsigned long long)a.ring_cap;
    unsigned long long recomputed = 0, offers = 0;
    int max_depth = 0;
    bool active = false;  // thread 0: this CTA is counted in q->active
    if (tid == 0) s_cnt = 0u;
    // Stamp the switched vertices.  A switched vertex whose parent also
    // switched is not a start item: the parent's walk lowers it with the
    // parent's new value, instead of a walk from a stale value that the
    // parent's walk would overtake.
    for (unsigned i = blockIdx.x * kAsyncThreads + tid; i < n_sw; i += gridDim.x * kAsyncThreads)
        a.swstamp[__ldcg(&a.switched[i])] = tag;
    if (!grid_barrier(c, gridDim.x)) return;

    for (;;) {
        // ---- acquire a batch (thread 0) --------------------------------
        if (tid == 0) {
            int kind = 3, nb = 0;
            unsigned cnt = s_cnt;
            if (cnt > 0u && vload(&q->abort) == 0u) {
                // hand half of a large stack to idle CTAs
                if (cnt > 2u * kAsyncThreads && vload(&q->active) < (int)gridDim.x) {
                    const unsigned k = cnt / 2u;
                    const unsigned long long g0 = atomicAdd(&q->tail, (unsigned long long)k);
                    if (g0 + k - qbase <= cap) {
                        s_gbase = g0;
                        s_old = cnt - k;
                        s_loc = k;
                    } else {
                        atomicExch(&q->abort, 1u);
                        s_loc = 0u;
                    }
                } else {
                    s_loc = 0u;
                }
                kind = 0;
            } else {
                if (active) {
                    __threadfence();
                    atomicSub(&q->active, 1);
                    active = false;
                }
                unsigned nap = 32;
                unsigned long long polls = 0;
                for (;;) {
                    if (++polls > kAsyncPollLimit) {
                        atomicOr(&c->status, kStatusTimeout);
                        atomicExch(&q->abort, 1u);
                        break;
                    }
                    if (vload(&q->done) != 0u || vload(&q->abort) != 0u) break;
                    if (vload(&q->start_take) < n_sw) {
                        atomicAdd(&q->active, 1);
                        const unsigned s0 = atomicAdd(&q->start_take, (unsigned)kAsyncThreads);
                        if (s0 < n_sw) {
                            kind = 1;
                            nb = (int)min(n_sw - s0, (unsigned)kAsyncThreads);
                            s_take0 = s0;
                            active = true;
                            break;
                        }
                        atomicSub(&q->active, 1);
                        continue;
                    }
                    const unsigned long long t1 = vload(&q->tail), k1 = vload(&q->take);
                    if (k1 < t1) {
                        atomicAdd(&q->active, 1);
                        const unsigned long long want =
                            min(t1 - k1, (unsigned long long)kAsyncThreads);
                        if (atomicCAS(&q->take, k1, k1 + want) == k1) {
                            kind = 2;
                            nb = (int)want;
                            s_spill0 = k1;
                            active = true;
                            break;
                        }
                        atomicSub(&q->active, 1);
                        continue;
                    }
                    // every switched vertex and spilled item is claimed; done
                    // once no CTA holds work and nothing was spilled since t1
                    __threadfence();
                    if (vload(&q->active) == 0) {
                        __threadfence();
                        if (vload(&q->tail) == t1) {
                            atomicExch(&q->done, 1u);
                            break;
                        }
                        continue;
                    }
                    __nanosleep(nap);
                    if (nap < 1024u) nap <<= 1;
                }
            }
            s_kind = kind;
            s_nb = nb;
        }
        __syncthreads();
        const int kind = s_kind;
        if (kind == 3) break;
        if (kind == 0) {
            // move the upper half of the stack to the spill list, if asked
            const unsigned k = s_loc;
            if (k) {
                const unsigned o = s_old;
                const unsigned long long g0 = s_gbase;
                for (unsigned i = tid; i < k; i += kAsyncThreads)
                    put_item(a.ring, a.ring_cap, g0 + i, s_lv[o + i], s_lg[o + i], s_ld[o + i]);
                __syncthreads();
                if (tid == 0) s_cnt = o;
                __syncthreads();
            }
            if (tid == 0) {
                const unsigned cnt = s_cnt;
                const int nb = (int)min(cnt, (unsigned)kAsyncThreads);
                s_nb = nb;
                s_take0 = cnt - (unsigned)nb;
                s_cnt = cnt - (unsigned)nb;
            }
            __syncthreads();
        }
        const int nb = s_nb;

        // ---- this thread's item: a vertex whose g was lowered -----------
        int32_t u = -1;
        double gu = 0.0;
        int du = 0;
        bool first = false;
        if (tid < nb) {
            if (kind == 0) {
                const unsigned i = s_take0 + (unsigned)tid;
                u = s_lv[i];
                gu = s_lg[i];
                du = s_ld[i];
            } else if (kind == 2) {
                const unsigned long long idx = s_spill0 + (unsigned long long)tid;
                AsyncItem *it = &a.ring[idx % cap];
                unsigned long long spins = 0;
                bool ok = true;
                while (vload(&it->tag) != idx + 1ull) {
                    if (vload(&q->abort) != 0u) {
                        ok = false;
                        break;
                    }
                    if (++spins > kAsyncPollLimit) {
                        atomicOr(&c->status, kStatusTimeout);
                        atomicExch(&q->abort, 1u);
                        ok = false;
                        break;
                    }
                    __nanosleep(32);
                }
                __threadfence();
                if (ok) {
                    u = __ldcg(&it->v);
                    gu = __ldcg(&it->g);
                    du = __ldcg(&it->depth);
                }
            } else {
                const int32_t s = __ldcg(&a.switched[s_take0 + (unsigned)tid]);
                const int32_t ps = __ldcg(&a.p[s]);
                const bool nested = __ldcg(&a.swstamp[ps]) == tag;
                const double gs = ld_g_cg(&a.g[ps], gpol) + widen(__ldcg(&a.pc[s]));
                if (!nested) ++recomputed;
                if (!nested && lower_g(a.g, s, gs)) {
                    u = s;
                    gu = gs;
                    du = 1;
                    first = atomicExch(&a.wstamp[s], tag) != tag;
                }
            }
        }
        if (kind == 1) warp_append(first, u, a.dg, &c->n_dg);
        int deg = 0;
        if (u >= 0) {
            int64_t b, e;
            row_range(a.rows, u, b, e);
            deg = (int)(e - b);
            s_base[tid] = b;
            max_depth = max(max_depth, du);
        }
        s_u[tid] = u;
        s_gu[tid] = gu;
        s_du[tid] = du;
        // block exclusive scan of the row lengths
        int incl = deg;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < NW ? s_wsum[lane] : 0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            if (lane < NW) s_wsum[lane] = w;
        }
        __syncthreads();
        s_seg[tid + 1] = incl + (warp > 0 ? s_wsum[warp - 1] : 0);
        if (tid == 0) s_seg[0] = 0;
        __syncthreads();
        const int total = s_seg[kAsyncThreads];
        const bool marking = vload(&c->dense_next) == 0u;

        // ---- stream the rows: lower children, mark neighbours ------------
        for (int p0 = 0; p0 < total; p0 += kAsyncThreads * kAsyncUnroll) {
            int32_t x[kAsyncUnroll], own[kAsyncUnroll];
            double gx[kAsyncUnroll];
#pragma unroll
            for (int j = 0; j < kAsyncUnroll; ++j) {
                const int pos = p0 + tid + j * kAsyncThreads;
                own[j] = -1;
                x[j] = 0;
                gx[j] = 0.0;
                if (pos < total) {
                    int l = 0, h = kAsyncThreads;  // last k with s_seg[k] <= pos
                    while (h - l > 1) {
                        const int mid = (l + h) >> 1;
                        if (s_seg[mid] <= pos) l = mid; else h = mid;
                    }
                    own[j] = l;
                    const Entry<CT> e = ld_stream(&a.adj[s_base[l] + (pos - s_seg[l])]);
                    x[j] = e.col;
                    // the entry's cost is c(v, w); with parallel edges the
                    // cheaper one wins the minimum, as Improve chose it
                    gx[j] = s_gu[l] + widen(e.w);
                    // the same sum is w's candidate through v in the next Improve
                    if (a.push && marking && x[j] != a.root) {
                        offer(a.cand, x[j], gx[j]);
                        ++offers;
                    }
                }
            }
            unsigned childm = 0, markm = 0, firstm = 0;
#pragma unroll
            for (int j = 0; j < kAsyncUnroll; ++j) {
                if (own[j] >= 0) {
                    if (__ldcg(&a.p[x[j]]) == s_u[own[j]] && lower_g(a.g, x[j], gx[j]))
                        childm |= 1u << j;
                    if (marking && x[j] != a.root && __ldcg(&a.stamp[x[j]]) != epoch &&
                        atomicExch(&a.stamp[x[j]], epoch) != epoch)
                        markm |= 1u << j;
                }
            }
#pragma unroll
            for (int j = 0; j < kAsyncUnroll; ++j)
                if (((childm >> j) & 1u) && atomicExch(&a.wstamp[x[j]], tag) != tag)
                    firstm |= 1u << j;
            // reserve stack slots (spilling what does not fit) and list slots
            const unsigned long long xv =
                ((unsigned long long)__popc(markm) << 32) | (unsigned)__popc(childm);
            unsigned long long inc = xv;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += y;
            }
            if (lane == 31) s_scan[warp] = inc;
            __syncthreads();
            if (tid == 0) {
                unsigned long long run = 0;
                for (int w = 0; w < NW; ++w) {
                    const unsigned long long t = s_scan[w];
                    s_scan[w] = run;
                    run += t;
                }
                const unsigned tc = (unsigned)(run & 0xffffffffull), tm = (unsigned)(run >> 32);
                const unsigned old = s_cnt;
                const unsigned room = old < (unsigned)kAsyncLocal ? (unsigned)kAsyncLocal - old : 0u;
                const unsigned loc = min(tc, room);
                s_cnt = old + loc;
                s_old = old;
                s_loc = loc;
                unsigned long long g0 = ~0ull;
                if (tc > loc) {
                    g0 = atomicAdd(&q->tail, (unsigned long long)(tc - loc));
                    if (g0 + (tc - loc) - qbase > cap) {
                        atomicExch(&q->abort, 1u);
                        g0 = ~0ull;
                    }
                }
                s_gbase = g0;
                s_mbase = tm ? atomicAdd(&c->n_next, tm) : 0u;
            }
            __syncthreads();
            const unsigned long long ex = s_scan[warp] + inc - xv;
            unsigned rc = (unsigned)(ex & 0xffffffffull);
            unsigned rm = s_mbase + (unsigned)(ex >> 32);
            const unsigned old = s_old, loc = s_loc;
            const unsigned long long g0 = s_gbase;
#pragma unroll
            for (int j = 0; j < kAsyncUnroll; ++j) {
                if ((childm >> j) & 1u) {
                    const int d = s_du[own[j]] + 1;
                    if ((unsigned)d > a.max_levels) {
                        atomicExch(&q->abort, 1u);
                    } else if (rc < loc) {
                        s_lv[old + rc] = x[j];
                        s_lg[old + rc] = gx[j];
                        s_ld[old + rc] = d;
                    } else if (g0 != ~0ull) {
                        put_item(a.ring, a.ring_cap, g0 + (rc - loc), x[j], gx[j], d);
                    }
                    ++rc;
                }
                if ((markm >> j) & 1u) next[rm++] = x[j];
            }
#pragma unroll
            for (int j = 0; j < kAsyncUnroll; ++j)
                warp_append((firstm >> j) & 1u, x[j], a.dg, &c->n_dg);
            __syncthreads();  // s_scan and the stack slots are reused
        }
        // changed-vertex count decides between a list and a dense sweep next
        if (tid == 0 && vload(&c->n_dg) > a.dense_limit)
            *reinterpret_cast<volatile unsigned *>(&c->dense_next) = 1u;
        __syncthreads();  // s_u / s_base / s_seg are rewritten by the next batch
    }

#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        recomputed += __shfl_down_sync(0xffffffffu, recomputed, off);
        offers += __shfl_down_sync(0xffffffffu, offers, off);
        max_depth = max(max_depth, __shfl_down_sync(0xffffffffu, max_depth, off));
    }
    if (lane == 0) {
        if (recomputed) atomicAdd(&c->evaluated, recomputed);
        if (offers) atomicAdd(&c->offers, offers);
        if (max_depth) atomicMax(&q->max_depth, (unsigned)max_depth);
    }
    if (!grid_barrier(c, gridDim.x)) return;
    // the FP32 shadow of every changed vertex, from its final g
    const unsigned n_dg = vload(&c->n_dg);
    for (unsigned i = blockIdx.x * kAsyncThreads + tid; i < n_dg; i += gridDim.x * kAsyncThreads) {
        const int32_t w = __ldcg(&a.dg[i]);
        a.g32[w] = g32_of(__ldcg(&a.g[w]));
    }
    if (blockIdx.x == 0 && tid == 0) {
        if (q->abort) {
            // lowered vertices whose rows were not scanned left neighbours
            // unmarked: pointer jumping finishes, the next Improve is dense
            c->wave_incomplete = 1u;
            c->dense_next = 1u;
        }
        c->wave_levels = q->max_depth;
        q->start_take = 0u;
        q->active = 0;
        q->done = 0u;
        q->abort = 0u;
        q->max_depth = 0u;
        const unsigned long long t = q->tail;
        q->take = t;
        q->base = t;
    }
}

// Reset of the walk's state before an exploit (after an error, say).
static __global__ void async_reset_kernel(AsyncQueue *q) {
    q->start_take = 0u;
    q->active = 0;
    q->done = 0u;
    q->abort = 0u;
    q->max_depth = 0u;
    const unsigned long long t = q->tail;
    q->take = t;
    q->base = t;
}

}  // namespace pirrt
