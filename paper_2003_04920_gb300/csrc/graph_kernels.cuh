// Kernels of the single-graph exploitation path of PI-RRT#:
//   Batched-Extension insertion (Alg. 3; Sec. IV-A: a coordinate list added
//   to a device CSR, here one whose rows keep room to grow), Improve (Alg. 2;
//   Sec. IV-B), Evaluate (Alg. 2; Sec. IV-C), the changed-vertex frontier and
//   the end of a Replan iteration.
#pragma once

#include <cfloat>
#include <climits>
#include <cmath>

#include <math_constants.h>

#include "device_common.cuh"

namespace pirrt {

constexpr int kThreads = 256;

// Candidate offers for the next Improve (see improve_push.cuh): cand[v] is
// the minimum, on FP64 bits, of the values g(u) + c(u, v) offered by
// neighbours u whose g changed; +inf bits when nothing was offered.
constexpr unsigned long long kCandNone = 0x7ff0000000000000ull;

// Offer g(u) + c(u, v) to v: an atomic minimum whose result is not used.
__device__ __forceinline__ void offer(unsigned long long *cand, int32_t v, double val) {
    atomicMin(cand + v, (unsigned long long)__double_as_longlong(val));
}

// ---------------------------------------------------------------------------
// Insertion
// ---------------------------------------------------------------------------

// Validate the new undirected edges and count, per endpoint, how many CSR
// entries the block adds.  Invalid input raises kStatusBadInput and is not
// counted (the host then discards the whole block).
template <typename CT>
__global__ void __launch_bounds__(kThreads)
insert_validate_count(int64_t n_edges, const int32_t *__restrict__ src,
                      const int32_t *__restrict__ dst, const CT *__restrict__ cost,
                      int64_t n_old, int64_t n_after, int32_t *__restrict__ deg,
                      int32_t *__restrict__ touched, DevCounters *ctr) {
    // an old row gaining its first new entry joins the touched list (the new
    // rows [n_old, n_after) are handled as a range)
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n_edges;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = base + threadIdx.x;
        bool ta = false, tb = false;
        int32_t a = 0, b = 0;
        if (e < n_edges) {
            a = src[e];
            b = dst[e];
            const double c = (double)cost[e];
            const bool ok = a >= 0 && b >= 0 && a < n_after && b < n_after && a != b &&
                            c > 0.0 && c <= DBL_MAX;  // rejects NaN, +inf, <= 0
            if (!ok) {
                atomicOr(&ctr->status, kStatusBadInput);
            } else {
                ta = atomicAdd(&deg[a], 1) == 0 && a < n_old;
                tb = atomicAdd(&deg[b], 1) == 0 && b < n_old;
            }
        }
        warp_append(ta, a, touched, &ctr->n_touched);
        warp_append(tb, b, touched, &ctr->n_touched);
    }
}

// Room a moving row reserves: 1.5x its new length + 4 (a few moves over a
// row's life); a repacked row gets 1.25x + 2, so a repack always fits a pool
// of 2 x (directed entries) + 4 x (vertices).
__device__ __forceinline__ int32_t row_room(int32_t need, bool repack) {
    return repack ? need + (need >> 2) + 2 : need + (need >> 1) + 4;
}

// Exclusive scan, first pass: one partial sum per tile of kScanTile entries.
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long x, long long *total) {
    __shared__ long long warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long w = (lane < kThreads / 32) ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const long long warp_base = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return warp_base + incl - x;
}

static __global__ void __launch_bounds__(kThreads)
scan_tile_reduce(const int32_t *__restrict__ deg, int64_t len, long long *__restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < len) s += deg[base + i];
    long long total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Second pass: exclusive scan of the tile sums in one block.
static __global__ void __launch_bounds__(kThreads)
scan_tile_sums(long long *__restrict__ tile_sums, int64_t n_tiles) {
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < n_tiles; b += kThreads) {
        const int64_t i = b + threadIdx.x;
        const long long x = i < n_tiles ? tile_sums[i] : 0;
        long long total;
        const long long ex = block_exclusive_scan(x, &total);
        if (i < n_tiles) tile_sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

// Third pass: new_off[v] = deg[0] + ... + deg[v - 1].  With len = n + 1 and
// deg[n] = 0, new_off[n] is the total.
static __global__ void __launch_bounds__(kThreads)
scan_tile_apply(const int32_t *__restrict__ deg, int64_t len,
                const long long *__restrict__ tile_sums, int64_t *__restrict__ new_off) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < len) ? deg[base + i] : 0;
        s += v[i];
    }
    long long total;
    long long run = block_exclusive_scan(s, &total) + tile_sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t x = base + i;
        if (x < len) new_off[x] = run;
        run += v[i];
    }
}

// Start of an insertion: empty touched list, no room taken, no error.
static __global__ void insert_begin_kernel(DevCounters *c) {
    c->n_touched = 0u;
    c->pool_cursor = 0ull;
    c->status = 0u;
}

// Item k of the rows an insertion changes: the touched old rows, then the new
// rows [n_old, n_after).
__device__ __forceinline__ int64_t changed_row(int64_t k, int64_t nt, const int32_t *touched,
                                               int64_t n_old) {
    return k < nt ? (int64_t)touched[k] : n_old + (k - nt);
}

// Plan without a scan: a changed row that would overflow (every new row with
// entries) takes room at the end of the pool from a cursor, one atomic per
// block; pool offsets (relative to the cursor's base) go to off[v].  Rows
// keep their relative order within a block only, which nothing relies on.
static __global__ void __launch_bounds__(kThreads)
insert_plan_list(int64_t n_old, int64_t n_after, const int32_t *__restrict__ touched,
                 const RowExt *__restrict__ rows, const int32_t *__restrict__ deg,
                 int32_t *__restrict__ alloc, int64_t *__restrict__ off, DevCounters *ctr) {
    const int64_t nt = (int64_t)__ldcg(&ctr->n_touched);
    const int64_t total = nt + (n_after - n_old);
    __shared__ long long s_base;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = base + threadIdx.x;
        int32_t a = 0;
        int64_t v = -1;
        if (k < total) {
            v = changed_row(k, nt, touched, n_old);
            const int32_t len = v < n_old ? rows[v].len : 0;
            const int32_t cap = v < n_old ? rows[v].cap : 0;
            const int32_t need = len + deg[v];
            if (need > cap) a = row_room(need, false);
            alloc[v] = a;
        }
        long long tot;
        const long long ex = block_exclusive_scan(a, &tot);
        if (threadIdx.x == 0)
            s_base = tot ? (long long)atomicAdd(&ctr->pool_cursor, (unsigned long long)tot) : 0;
        __syncthreads();
        if (a > 0) off[v] = s_base + ex;
        __syncthreads();
    }
}

// Move the changed rows that took new room (their old entries first) to pool
// offset base + off[v], and set every changed row's extent to its length
// after the block.  One warp per 32 changed rows.
template <typename CT>
__global__ void __launch_bounds__(kThreads)
insert_move_list(int64_t n_old, int64_t n_after, const int32_t *__restrict__ touched,
                 RowExt *__restrict__ rows, const int32_t *__restrict__ deg,
                 const int32_t *__restrict__ alloc, const int64_t *__restrict__ off,
                 long long base, Entry<CT> *__restrict__ pool, DevCounters *ctr) {
    const int lane = threadIdx.x & 31;
    const int64_t nt = (int64_t)__ldcg(&ctr->n_touched);
    const int64_t total = nt + (n_after - n_old);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long copied = 0;
    for (int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         w0 < total; w0 += warps * 32) {
        const int64_t k = w0 + lane;
        long long ob = 0, nb = 0;
        int32_t len = 0;
        bool move = false;
        if (k < total) {
            const int64_t v = changed_row(k, nt, touched, n_old);
            RowExt r{0, 0, 0};
            if (v < n_old) r = rows[v];
            const int32_t a = alloc[v];
            len = r.len;
            ob = r.beg;
            RowExt nr = r;
            nr.len = r.len + deg[v];
            if (a > 0) {
                nb = base + off[v];
                nr.beg = nb;
                nr.cap = a;
                move = len > 0;
            }
            rows[v] = nr;
        }
        unsigned todo = __ballot_sync(0xffffffffu, move);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1u;
            const long long sb = __shfl_sync(0xffffffffu, ob, l);
            const long long db = __shfl_sync(0xffffffffu, nb, l);
            const int32_t n = __shfl_sync(0xffffffffu, len, l);
            for (int32_t q = lane; q < n; q += 32) pool[db + q] = ld_stream(&pool[sb + q]);
            copied += (unsigned long long)n;
        }
    }
    if (lane == 0 && copied) atomicAdd(&ctr->insert_copied, copied);
}

// Slack CSR.  Every row owns adj[beg, beg + cap) of a pool and fills it from
// the front; a block's new entries go to the row tails.  A row that would
// overflow moves to fresh space at the end of the pool with room to grow, so
// an insertion copies only the rows that moved, not the whole graph.  When
// the pool is used up, every row is repacked into a second pool.


// Plan: the pool space each row must take (0: stays where it is).
// alloc[n_after] = 0 closes the scan.
static __global__ void __launch_bounds__(kThreads)
insert_plan(int64_t n_old, int64_t n_after, const RowExt *__restrict__ rows,
            const int32_t *__restrict__ deg, int32_t *__restrict__ alloc, int repack) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n_after;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = 0;
        if (v < n_after) {
            const int32_t len = v < n_old ? rows[v].len : 0;
            const int32_t cap = v < n_old ? rows[v].cap : 0;
            const int32_t need = len + deg[v];
            if (repack) a = need > 0 ? row_room(need, true) : 0;
            else if (need > cap) a = row_room(need, false);
        }
        alloc[v] = a;
    }
}

// Move the rows that need space (their old entries first) to pool offset
// base + off[v], and set every row's extent to its length after the block.
// One warp per 32 rows: each moving row is copied by the whole warp.
template <typename CT>
__global__ void __launch_bounds__(kThreads)
insert_move_rows(int64_t n_old, int64_t n_after, RowExt *__restrict__ rows,
                 const int32_t *__restrict__ deg, const int32_t *__restrict__ alloc,
                 const int64_t *__restrict__ off, long long base,
                 const Entry<CT> *__restrict__ src, Entry<CT> *__restrict__ dst,
                 DevCounters *ctr, int repack) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long copied = 0;
    for (int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         w0 < n_after; w0 += warps * 32) {
        const int64_t v = w0 + lane;
        long long ob = 0, nb = 0;
        int32_t len = 0;
        bool move = false;
        if (v < n_after) {
            RowExt r{0, 0, 0};
            if (v < n_old) r = rows[v];
            const int32_t add = deg[v];
            const int32_t a = alloc[v];
            len = r.len;
            ob = r.beg;
            RowExt nr = r;
            nr.len = r.len + add;
            const bool place = a > 0 || v >= n_old || repack;
            if (place) {
                nb = base + off[v];
                nr.beg = nb;
                nr.cap = a;
                move = a > 0 && len > 0;
            }
            if (place || add > 0) rows[v] = nr;
        }
        unsigned todo = __ballot_sync(0xffffffffu, move);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1u;
            const long long sb = __shfl_sync(0xffffffffu, ob, l);
            const long long db = __shfl_sync(0xffffffffu, nb, l);
            const int32_t n = __shfl_sync(0xffffffffu, len, l);
            for (int32_t k = lane; k < n; k += 32) dst[db + k] = ld_stream(&src[sb + k]);
            copied += (unsigned long long)n;
        }
    }
    if (lane == 0 && copied) atomicAdd(&ctr->insert_copied, copied);
}

// Export: row lengths (len[n] = 0 closes the scan), then each row copied to
// its compact position off[v] (one warp per 32 rows, as above).
static __global__ void __launch_bounds__(kThreads)
row_lengths(int64_t n, const RowExt *__restrict__ rows, int32_t *__restrict__ len) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x)
        len[v] = v < n ? rows[v].len : 0;
}

template <typename CT>
__global__ void __launch_bounds__(kThreads)
export_rows(int64_t n, const RowExt *__restrict__ rows, const int64_t *__restrict__ off,
            const Entry<CT> *__restrict__ adj, Entry<CT> *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; w0 < n;
         w0 += warps * 32) {
        const int64_t v = w0 + lane;
        long long sb = 0, db = 0;
        int32_t len = 0;
        if (v < n) {
            sb = rows[v].beg;
            len = rows[v].len;
            db = off[v];
        }
        unsigned todo = __ballot_sync(0xffffffffu, len > 0);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1u;
            const long long s0 = __shfl_sync(0xffffffffu, sb, l);
            const long long d0 = __shfl_sync(0xffffffffu, db, l);
            const int32_t k0 = __shfl_sync(0xffffffffu, len, l);
            for (int32_t k = lane; k < k0; k += 32) out[d0 + k] = adj[s0 + k];
        }
    }
}

// Place both directions of every new edge at the tail of its rows (filled
// from the row end, order within a row is irrelevant) and seed the next
// Improve frontier with both endpoints.
template <typename CT>
__global__ void __launch_bounds__(kThreads)
insert_scatter(int64_t n_edges, const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
               const CT *__restrict__ cost, const RowExt *__restrict__ rows,
               int32_t *__restrict__ deg, Entry<CT> *__restrict__ adj, unsigned *__restrict__ stamp,
               int32_t root, int32_t *__restrict__ list0, int32_t *__restrict__ list1,
               const double *__restrict__ g, unsigned long long *__restrict__ cand,
               DevCounters *ctr) {
    const unsigned epoch = ctr->epoch;
    int32_t *active = (ctr->la & 1u) ? list1 : list0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n_edges; base += stride) {
        const int64_t e = base + threadIdx.x;
        bool pa = false, pb = false;
        int32_t a = 0, b = 0;
        if (e < n_edges) {
            a = src[e];
            b = dst[e];
            const CT w = cost[e];
            // rows hold the lengths after the block: fill the tails from the end
            const int64_t sa = rows[a].beg + rows[a].len - atomicSub(&deg[a], 1);
            const int64_t sb = rows[b].beg + rows[b].len - atomicSub(&deg[b], 1);
            Entry<CT> ea{}, eb{};
            ea.col = b;
            ea.w = w;
            eb.col = a;
            eb.w = w;
            adj[sa] = ea;
            adj[sb] = eb;
            // the new edge offers each endpoint the other's candidate; an
            // endpoint joins the next Improve list only if that candidate beats
            // its g (g >= cur, so a candidate not below g can never win; a new
            // vertex has g = +inf and joins with its first finite neighbour)
            const double ga = g[a], gb = g[b];
            const double va = gb + widen(w), vb = ga + widen(w);
            const bool ua = a != root && gb < CUDART_INF && va < ga;
            const bool ub = b != root && ga < CUDART_INF && vb < gb;
            if (ub) offer(cand, b, vb);
            if (ua) offer(cand, a, va);
            pa = ua && atomicExch(&stamp[a], epoch) != epoch;
            pb = ub && atomicExch(&stamp[b], epoch) != epoch;
        }
        __shared__ unsigned long long s_scan[kThreads / 32 + 2];
        unsigned ba, bb;
        block_reserve2<kThreads>(pa ? 1u : 0u, pb ? 1u : 0u, &ctr->n_active, &ctr->n_active,
                                 s_scan, ba, bb);
        if (pa) active[ba] = a;
        if (pb) active[bb] = b;
    }
}

// Seed the new vertices: g = +inf (0 for the root), no parent, no offer.
// They join the next Improve frontier through the offers of their new edges
// (insert_scatter).
template <typename CT>
__global__ void __launch_bounds__(kThreads)
insert_init_vertices(int64_t n_old, int64_t n_after, int32_t root, double *__restrict__ g,
                     float *__restrict__ g32, int32_t *__restrict__ p, CT *__restrict__ pc,
                     unsigned long long *__restrict__ cand, unsigned *__restrict__ stamp,
                     int32_t *__restrict__ list0, int32_t *__restrict__ list1, DevCounters *ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = n_old + (int64_t)blockIdx.x * blockDim.x; base < n_after; base += stride) {
        const int64_t v = base + threadIdx.x;
        if (v < n_after) {
            g[v] = (v == root) ? 0.0 : CUDART_INF;
            g32[v] = (v == root) ? 0.0f : __int_as_float(0x7f800000);
            p[v] = (v == root) ? kRootMark : -1;
            pc[v] = CT(0);
            cand[v] = kCandNone;
        }
    }
}

// ---------------------------------------------------------------------------
// Improve (Alg. 2; Sec. IV-B) -- Jacobi relaxation, G threads per vertex.
// ---------------------------------------------------------------------------

// Candidate order: smaller value, then smaller id, then smaller cost (parallel
// edges).  The order is total, so the result does not depend on scan order.
template <typename CT>
__device__ __forceinline__ bool cand_less(double v1, int32_t u1, CT w1, double v2, int32_t u2,
                                          CT w2) {
    return v1 < v2 || (v1 == v2 && (u1 < u2 || (u1 == u2 && w1 < w2)));
}

template <typename CT>
struct ImproveArgs {
    const RowExt *rows;
    const Entry<CT> *adj;
    const double *g;
    const float *g32;
    int32_t *p;
    CT *pc;
    const int32_t *list[2];  // Improve reads list[la & 1] (la in the counter block)
    int32_t *switched;       // list of vertices whose parent changed
    DevCounters *ctr;
    int64_t n;
    int32_t root;
    int32_t push;            // list sweeps run from offers (improve_push_kernel); this
                             // kernel then only runs dense sweeps
    unsigned long long *cand;
    const float *h;          // goal-directed Replan: heuristic h(v); null = goal-free
};

// Goal-directed Replan (Sec. IV-C).  A vertex v is promising when
// g(v) + h(v) < g(x_goal), with h an admissible heuristic and g(x_goal) as
// the iteration began (bound_bits).  Improve takes a switch only if the new
// value makes v promising; the wave expands (offers, marks, lowers the
// children of) only promising vertices.  Without a goal h is null and every
// vertex passes.
__device__ __forceinline__ double goal_bound(const DevCounters *c, const float *h) {
    return h != nullptr ? __longlong_as_double((long long)__ldcg(&c->bound_bits)) : CUDART_INF;
}

__device__ __forceinline__ bool promising(const float *h, int32_t v, double value, double bound) {
    return h == nullptr || value + (double)__ldg(&h[v]) < bound;
}

// G lanes cooperate on one vertex: each lane scans every G-th entry of the
// row, four entries in flight at a time (loads first, then the g gathers),
// then the group reduces (value, id, cost) lexicographically with shuffles.
// Lane 0 compares the winner with the current parent's candidate, computed
// by the same expression g(p) + c, and switches only on a strict decrease.
template <typename CT, int G>
__global__ void __launch_bounds__(kThreads)
improve_kernel(const ImproveArgs<CT> *__restrict__ ap) {
    const ImproveArgs<CT> a = *ap;

    const int32_t *active = a.list[a.ctr->la & 1u];
    constexpr int kUnroll = 4;
    const int lane_g = threadIdx.x & (G - 1);
    const unsigned group_mask =
        G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int groups_per_block = kThreads / G;
    const int64_t gstride = (int64_t)gridDim.x * groups_per_block;
    const bool dense = a.ctr->dense != 0u;
    if (a.push && !dense) return;
    const int64_t count = dense ? a.n : (int64_t)a.ctr->n_active;
    const unsigned long long gpol = policy_evict_last();
    const double bound = goal_bound(a.ctr, a.h);

    unsigned long long relax = 0, improved = 0;
    for (int64_t item = (int64_t)blockIdx.x * groups_per_block + threadIdx.x / G; item < count;
         item += gstride) {
        const int32_t v = dense ? (int32_t)item : active[item];
        if (v == a.root) continue;  // uniform within the group
        int64_t b, e;
        row_range(a.rows, v, b, e);
        double best = CUDART_INF;
        int32_t bu = INT_MAX;
        CT bw = CT(0);
        for (int64_t i0 = b + lane_g; i0 < e; i0 += (int64_t)G * kUnroll) {
            Entry<CT> en[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const int64_t i = i0 + (int64_t)k * G;
                if (i < e) en[k] = ld_stream(&a.adj[i]);
            }
            double gv[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const int64_t i = i0 + (int64_t)k * G;
                gv[k] = (i < e) ? ld_g(&a.g[en[k].col], gpol) : CUDART_INF;
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const int64_t i = i0 + (int64_t)k * G;
                if (i < e) {
                    const double cand = gv[k] + (double)en[k].w;
                    if (cand_less(cand, en[k].col, en[k].w, best, bu, bw)) {
                        best = cand;
                        bu = en[k].col;
                        bw = en[k].w;
                    }
                }
            }
        }
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            const double ob = __shfl_xor_sync(group_mask, best, off, G);
            const int32_t ou = __shfl_xor_sync(group_mask, bu, off, G);
            const CT ow = __shfl_xor_sync(group_mask, bw, off, G);
            if (cand_less(ob, ou, ow, best, bu, bw)) {
                best = ob;
                bu = ou;
                bw = ow;
            }
        }
        if (lane_g == 0 && a.p[v] != kRootMark) {
            const int32_t pv = a.p[v];
            const double cur = pv >= 0 ? a.g[pv] + (double)a.pc[v] : CUDART_INF;
            if (best < cur && promising(a.h, v, best, bound)) {
                a.p[v] = bu;
                a.pc[v] = bw;
                const unsigned slot = atomicAdd(&a.ctr->n_switched, 1u);
                a.switched[slot] = v;
                // Delta g = max over switches of cur - best (> 0, or +inf for a
                // vertex reached for the first time); non-negative doubles order
                // like their bit patterns
                atomicMax(&a.ctr->dj_bits, (unsigned long long)__double_as_longlong(cur - best));
            }
            relax += (unsigned long long)(e - b);
            improved += 1;
        }
    }
    // block totals -> one atomic per block
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        relax += __shfl_down_sync(0xffffffffu, relax, off);
        improved += __shfl_down_sync(0xffffffffu, improved, off);
    }
    __shared__ unsigned long long s_relax[kThreads / 32], s_imp[kThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        s_relax[threadIdx.x >> 5] = relax;
        s_imp[threadIdx.x >> 5] = improved;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long r = 0, m = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            r += s_relax[w];
            m += s_imp[w];
        }
        if (r) atomicAdd(&a.ctr->relax, r);
        if (m) atomicAdd(&a.ctr->improved, m);
    }
}

template <typename CT>
struct CostBits;
template <>
struct CostBits<float> {
    using T = unsigned;
    static __device__ __forceinline__ unsigned of(float w) { return __float_as_uint(w); }
    static __device__ __forceinline__ float back(unsigned b) { return __uint_as_float(b); }
    static constexpr unsigned kMax = 0xffffffffu;
};
template <>
struct CostBits<double> {
    using T = unsigned long long;
    static __device__ __forceinline__ unsigned long long of(double w) {
        return (unsigned long long)__double_as_longlong(w);
    }
    static __device__ __forceinline__ double back(unsigned long long b) {
        return __longlong_as_double((long long)b);
    }
    static constexpr unsigned long long kMax = 0xffffffffffffffffull;
};

// ---------------------------------------------------------------------------
// Evaluate (Alg. 2; Sec. IV-C) -- g(v) = g(p(v)) + c(p(v), v) from the root,
// by pointer jumping over the parent tree in FP64.
// ---------------------------------------------------------------------------

template <typename CT>
struct EvaluateArgs {
    const int32_t *p;
    const CT *pc;
    double *g;
    float *g32;
    int32_t *anc[2];  // current ancestor of each unfinished vertex
    double *acc[2];   // sum of policy-edge costs from the vertex up to anc
    int32_t *done;    // round in which the vertex's g became final
    int32_t *wl[2];   // work lists of unfinished vertices
    int32_t *dg;      // vertices whose g changed
    DevCounters *ctr;
    int64_t n;
    int32_t root;
    int32_t force;    // run even if Improve switched nothing (set_policy)
    int32_t role;     // 0: the iteration's Evaluate; 1: finish a wave that hit its level cap
};

// Rounds are separated by a grid barrier.  Round 0 links every vertex to its
// parent.  In round r an unfinished vertex w with ancestor a either finishes,
// if a's g became final in an earlier round (g(w) = acc(w) + g(a)), or
// jumps: acc(w) += acc(a), anc(w) = anc(a).  Every value read in round r was
// written before round r, so the sums, hence g, do not depend on scheduling.
// The whole pointer-jumping Evaluate, for any cooperative grid; false if a
// grid barrier timed out.
template <typename CT>
__device__ bool jump_evaluate(const EvaluateArgs<CT> &a) {
    DevCounters *c = a.ctr;
    if (blockIdx.x == 0 && threadIdx.x == 0) c->jumped = 1u;
    const unsigned nblocks = gridDim.x;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid0 = (int64_t)blockIdx.x * blockDim.x;
    unsigned long long finished = 0;
    __shared__ unsigned long long s_scan[1024 / 32 + 2];

    // round 0
    for (int64_t base = tid0; base < a.n; base += wstride) {
        const int64_t v = base + threadIdx.x;
        bool keep = false;
        if (v < a.n) {
            const int32_t pv = a.p[v];
            if (v == a.root || pv < 0) {
                a.done[v] = 0;  // g(root) = 0 (parent kRootMark), unreached = +inf: already in g
            } else {
                a.anc[0][v] = pv;
                a.acc[0][v] = (double)a.pc[v];
                a.done[v] = INT_MAX;
                keep = true;
            }
        }
        unsigned bk, bd;
        block_reserve2_dyn(keep ? 1u : 0u, 0u, &c->wl_count[1], &c->n_dg, s_scan, bk, bd);
        if (keep) a.wl[0][bk] = (int32_t)v;
    }
    if (!grid_barrier(c, nblocks)) return false;

    int r = 1;
    for (;; ++r) {
        const int64_t count = (int64_t)(*(volatile unsigned *)&c->wl_count[r]);
        if (count == 0) break;
        if (r > kMaxJumpRounds) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->status, kStatusBadTree);
            break;
        }
        const int rd = (r - 1) & 1, wr = r & 1;
        const int32_t *wl_in = rd ? a.wl[1] : a.wl[0];
        int32_t *wl_out = wr ? a.wl[1] : a.wl[0];
        const int32_t *anc_r = rd ? a.anc[1] : a.anc[0];
        const double *acc_r = rd ? a.acc[1] : a.acc[0];
        int32_t *anc_w = wr ? a.anc[1] : a.anc[0];
        double *acc_w = wr ? a.acc[1] : a.acc[0];
        for (int64_t base = tid0; base < count; base += wstride) {
            const int64_t i = base + threadIdx.x;
            bool keep = false, changed = false;
            int32_t w = 0;
            if (i < count) {
                w = __ldcg(&wl_in[i]);
                const int32_t anc = __ldcg(&anc_r[w]);
                const double s = __ldcg(&acc_r[w]);
                if (__ldcg(&a.done[anc]) < r) {
                    const double gw = s + __ldcg(&a.g[anc]);
                    const double old = __ldcg(&a.g[w]);
                    changed = __double_as_longlong(gw) != __double_as_longlong(old);
                    a.g[w] = gw;
                    a.g32[w] = g32_of(gw);
                    a.done[w] = r;
                    ++finished;
                } else {
                    anc_w[w] = __ldcg(&anc_r[anc]);
                    acc_w[w] = s + __ldcg(&acc_r[anc]);
                    keep = true;
                }
            }
            unsigned bk, bd;
            block_reserve2_dyn(keep ? 1u : 0u, changed ? 1u : 0u, &c->wl_count[r + 1], &c->n_dg,
                               s_scan, bk, bd);
            if (keep) wl_out[bk] = w;
            if (changed) a.dg[bd] = w;
        }
        if (!grid_barrier(c, nblocks)) return false;
    }
    block_add(finished, &c->evaluated, s_scan);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->rounds = (unsigned)(r - 1);
        c->g32_stale = 0u;  // every vertex with a parent got its shadow above
    }
    return true;
}

template <typename CT>
__global__ void __launch_bounds__(kThreads)
evaluate_kernel(const EvaluateArgs<CT> *__restrict__ ap) {
    const EvaluateArgs<CT> a = *ap;
    DevCounters *c = a.ctr;
    if (!a.force && c->n_switched == 0u) return;
    if (a.role == 1 && c->wave_incomplete == 0u) return;
    jump_evaluate<CT>(a);
}

// ---------------------------------------------------------------------------
// Changed-vertex frontier: the next Improve examines the neighbours of every
// vertex whose g changed (only they can find a better parent), or every
// vertex when that set is large.
// ---------------------------------------------------------------------------

template <typename CT>
struct MarkArgs {
    const RowExt *rows;
    const Entry<CT> *adj;
    const int32_t *dg;
    unsigned *stamp;
    int32_t *list[2];      // the next Improve list is list[(la & 1) ^ 1]
    DevCounters *ctr;
    int32_t root;
    unsigned dense_limit;  // |dg| above this -> dense sweep next
    int32_t role;          // 0: after every Evaluate; 1: only after a pointer-jumping finish
    int32_t push;          // offer g(x) + c(x, u) to every neighbour u
    const double *g;
    unsigned long long *cand;
};

// Frontier marking (and offers) for the changed list, any grid.  The list
// and g may have been written earlier in the same kernel by other CTAs, so
// they are read through L2.  With offers only a neighbour whose g the offer
// beats is offered and listed (g is final after pointer jumping); without,
// every neighbour is listed.
template <typename CT>
__device__ void mark_changed(const MarkArgs<CT> &a) {
    DevCounters *c = a.ctr;
    const unsigned epoch = c->epoch + 1u;
    int32_t *next = ((c->la & 1u) ^ 1u) ? a.list[1] : a.list[0];
    const unsigned n_dg = *(volatile unsigned *)&c->n_dg;
    if (c->n_switched == 0u || n_dg == 0u) return;
    if (n_dg > a.dense_limit) {
        if (blockIdx.x == 0 && threadIdx.x == 0) c->dense_next = 1u;
        return;
    }
    // one warp per changed vertex; lanes stride over its row; appends are
    // staged per warp and reach the list 128 at a time
    constexpr int kCap = 128;
    __shared__ int32_t s_stage[1024 / 32][kCap];
    __shared__ unsigned s_fl[1024 / 32 + 1];
    __shared__ unsigned long long s_red[1024 / 32];
    WarpStage<kCap> stq{s_stage[threadIdx.x >> 5], 0u};
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long offers = 0;
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_dg;
         j += warps) {
        const int32_t x = __ldcg(&a.dg[j]);
        int64_t b, e;
        row_range(a.rows, x, b, e);
        const double gx = a.push ? __ldcg(&a.g[x]) : 0.0;
        for (int64_t i0 = b; i0 < e; i0 += 32) {
            const int64_t i = i0 + lane;
            bool pred = false;
            int32_t u = 0;
            if (i < e) {
                const Entry<CT> en = a.adj[i];
                u = en.col;
                if (u != a.root) {
                    if (a.push) {
                        // g is final here: an offer not below g(u) can never win
                        ++offers;
                        const double val = gx + widen(en.w);
                        if (val < __ldcg(&a.g[u])) {
                            offer(a.cand, u, val);
                            pred = atomicExch(&a.stamp[u], epoch) != epoch;
                        }
                    } else {
                        pred = atomicExch(&a.stamp[u], epoch) != epoch;
                    }
                }
            }
            stq.push(pred, u, next, &c->n_next);
        }
    }
    stq.flush_block(next, &c->n_next, s_fl);
    block_add(offers, &c->offers, s_red);
}

template <typename CT>
__global__ void __launch_bounds__(kThreads)
mark_frontier_kernel(const MarkArgs<CT> *__restrict__ ap) {
    const MarkArgs<CT> a = *ap;
    if (a.role == 1 && a.ctr->wave_incomplete == 0u) return;
    mark_changed<CT>(a);
}

// ---------------------------------------------------------------------------
// Evaluate, top-down form: recompute g only below the vertices Improve
// switched, level by level, and mark the next Improve frontier in the same
// row scan.
// ---------------------------------------------------------------------------

template <typename CT>
struct WaveArgs {
    const RowExt *rows;
    const Entry<CT> *adj;
    const int32_t *p;
    const CT *pc;
    double *g;
    float *g32;
    const int32_t *switched;  // step 0: vertices whose parent changed
    int32_t *lvl[2];          // vertices of grid step t (mod 2), their g already lowered
    double *lvg[2];           // ... the lowered g they carry
    longlong2 *lvx[2];        // ... and their row extent and depth below the switched vertex
                              // they came from: {beg, (depth << 32) | len}
    int32_t *dg;              // vertices whose g changed (each once)
    unsigned *wstamp;         // first-change stamps (tag = wave_epoch)
    unsigned *stamp;          // Improve-list stamps
    int32_t *list[2];         // the next Improve list is list[(la & 1) ^ 1]
    DevCounters *ctr;
    int32_t root;
    unsigned dense_limit;     // |changed| above this -> dense sweep next, stop marking
    unsigned max_levels;      // a vertex this deep is lowered, not expanded (wave_incomplete)
    int32_t push;             // offer g(u) + c(u, w) to every neighbour w of a changed u
    unsigned long long *cand;
    unsigned tail_max;        // steps of at most this many vertices: one CTA, no grid barrier
    unsigned local_levels;    // tree levels a CTA walks on its own within a grid step
    unsigned local_max;       // ... while its local list holds at most this many vertices,
    unsigned local_step;      // ... in grid steps of at most this many vertices
    int64_t list_cap;         // capacity of lvl[] / lvg[] / lvx[]
    const float *h;           // goal-directed Replan: heuristic h(v); null = goal-free
    int64_t n;                // vertex count (bulk refresh of the FP32 shadow)
};

// Step 0 holds the switched vertices: each takes g(s) = g(p(s)) + c(p(s), s).
// A vertex whose g was lowered is expanded: its row is scanned once, every
// neighbour joins the next Improve list (only neighbours of changed vertices
// can find a better parent) and is offered its candidate through it, and
// every child w (p(w) = u) is lowered at once to g(u) + c(u, w) -- one FP64
// addition per tree edge, root to leaf, as in Alg. 2's Evaluate -- and, if
// that lowered it, is expanded in turn carrying the value.  A vertex whose g
// does not drop prunes its subtree.
//
// Improve only switches to strictly cheaper parents, so no cost-to-come rises
// under the new policy: every value computed for a vertex (from an ancestor
// not yet final, when switched vertices lie below one another) is at least
// its final value, and g is lowered by an atomic minimum on its bit pattern
// (non-negative doubles order like unsigned integers).  A stale value can
// never overwrite a smaller one, and each vertex is reached again right after
// its parent's last drop, so the result is the root-to-leaf sum whatever the
// order in which vertices are expanded.
//
// Work is organised in grid steps separated by a grid barrier.  A step's
// global list is split evenly over the CTAs.  A CTA takes up to kWaveThreads
// vertices at a time, one per thread, then streams the concatenated rows with
// every thread (the loads of a whole tile in flight at once), locating each
// entry's row by binary search over the tile's prefix sums in shared memory.
// The children a CTA lowers go to its local list in shared memory, with their
// row extents (loaded beside the atomic minimum that lowered them), and the
// CTA walks that list on its own, one tree level per tile, for up to
// local_levels levels while the list holds at most local_max vertices: such a
// level costs a few dependent memory round trips and a CTA barrier instead of
// a grid-wide step.  Local walks run only in steps of at most local_step
// vertices: a step ends when its slowest CTA does, so in a wide step a CTA
// walking on alone would hold back every other CTA's share of the next step.
// A longer list means a subtree wide enough to be worth sharing: it goes to
// the global list of the next step, where every CTA takes a part, and so do
// children beyond the local list's room and whatever the list holds when the
// walk stops.  A step of at most tail_max vertices is walked by CTA 0 alone
// with no level limit, while the other CTAs wait at one grid barrier.
constexpr int kWaveThreads = 512;
constexpr int kWaveUnroll = 4;
constexpr int kWaveStage = 64;  // Improve-list appends staged per warp

template <typename CT>
struct WaveStepCtx;

template <typename CT>
struct WaveShared {
    // the tile being expanded
    int32_t u[kWaveThreads];
    double gu[kWaveThreads];
    long long base[kWaveThreads];
    int32_t dep[kWaveThreads];
    int32_t seg[kWaveThreads + 1];
    unsigned long long scan[kWaveThreads / 32 + 2];
    // the CTA's local list: lowered children and their row extents
    int32_t lu[kWaveThreads];
    double lg[kWaveThreads];
    long long lb[kWaveThreads];
    int32_t ll[kWaveThreads];
    int32_t ld[kWaveThreads];
    unsigned lcnt;     // local slots taken (beyond kWaveThreads: spilled to the global list)
    unsigned nfirst;   // first changes counted by this CTA in the current step
    unsigned fl[kWaveThreads / 32 + 1];
    int32_t stage[kWaveThreads / 32][kWaveStage];  // Improve-list appends
    int32_t dstage[kWaveThreads / 32][kWaveStage]; // changed-list appends (without offers)
};

// Where a tile's vertices come from.
enum WaveSource { kFromSwitched = 0, kFromGlobal = 1, kFromLocal = 2 };

// Per-step view of the lists and flags, the same for every tile of the step.
template <typename CT>
struct WaveStepCtx {
    const int32_t *in;
    const double *ing;
    const longlong2 *inx;
    int32_t *out;
    double *outg;
    longlong2 *outx;
    unsigned *out_cnt;
    int32_t *next;
    unsigned tag, epoch;
    unsigned long long gpol;
    double bound;
    bool marking, offering, stop;
};

// One tile of nv vertices (src: kFromSwitched / kFromGlobal read entries
// [s0, s0 + nv) of the switched or global list; kFromLocal takes the local
// list, which the tile empties and its children refill).  Every thread of the
// CTA calls this.
template <typename CT>
__device__ __forceinline__ void wave_tile(const WaveArgs<CT> &a, WaveShared<CT> &sh,
                                          const WaveStepCtx<CT> &x, int src, int64_t s0, int nv,
                                          WarpStage<kWaveStage> &mq, WarpStage<kWaveStage> &dq,
                                          unsigned long long &recomputed,
                                          unsigned long long &offers) {
    DevCounters *c = a.ctr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int deg = 0;
    int32_t u = -1, d = 0;
    double gu = 0.0;
    long long beg = 0;
    bool first = false;
    if (tid < nv) {
        if (src == kFromSwitched) {
            const int32_t s = __ldcg(&a.switched[s0 + tid]);
            const int32_t ps = __ldcg(&a.p[s]);
            const double gs = ld_g_cg(&a.g[ps], x.gpol) + widen(__ldcg(&a.pc[s]));
            ++recomputed;
            const unsigned long long b = (unsigned long long)__double_as_longlong(gs);
            if (atomicMin(reinterpret_cast<unsigned long long *>(&a.g[s]), b) > b) {
                u = s;
                gu = gs;
            }
        } else if (src == kFromGlobal) {
            u = __ldcg(&x.in[s0 + tid]);
            gu = __ldcg(&x.ing[s0 + tid]);
            const longlong2 e = __ldcg(&x.inx[s0 + tid]);
            beg = e.x;
            deg = (int)(unsigned)((unsigned long long)e.y & 0xffffffffull);
            d = (int)((unsigned long long)e.y >> 32);
        } else {
            u = sh.lu[tid];
            gu = sh.lg[tid];
            d = sh.ld[tid];
            beg = sh.lb[tid];
            deg = sh.ll[tid];
        }
    }
    if (src == kFromLocal) {
        __syncthreads();  // every entry of the local list is read: it refills from 0
        if (tid == 0) sh.lcnt = 0u;
    }
    if (u >= 0) {
        // each changed vertex is counted once (the result is used at the end
        // of the tile, off the critical path)
        first = atomicExch(&a.wstamp[u], x.tag) != x.tag;
        // a vertex that is not promising keeps its lowered g but is not
        // expanded: its subtree and neighbours are left as they are
        if (promising(a.h, u, gu, x.bound)) {
            if (src == kFromSwitched) {
                int64_t b, e;
                row_range(a.rows, u, b, e);
                beg = b;
                deg = (int)(e - b);
            }
        } else {
            deg = 0;
        }
        // this deep, the vertex is lowered but not expanded: pointer jumping
        // finishes the values below it
        if (x.stop || (unsigned)d >= a.max_levels) *(volatile unsigned *)&c->wave_incomplete = 1u;
    }
    sh.u[tid] = u;
    sh.gu[tid] = gu;
    sh.base[tid] = beg;
    sh.dep[tid] = (x.stop || (unsigned)d >= a.max_levels) ? -1 : d;  // -1: no children
    // one block scan of the row lengths: the tile's row offsets
    constexpr int NW = kWaveThreads / 32;
    int incl = deg;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) sh.scan[warp] = (unsigned long long)incl;
    __syncthreads();
    if (tid == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < NW; ++w) {
            const unsigned long long v = sh.scan[w];
            sh.scan[w] = run;
            run += v;
        }
        sh.seg[kWaveThreads] = (int)run;
    }
    __syncthreads();
    sh.seg[tid] = (int)sh.scan[warp] + incl - deg;
    __syncthreads();
    const int total = sh.seg[kWaveThreads];
    for (int p0 = 0; p0 < total; p0 += kWaveThreads * kWaveUnroll) {
        int32_t xv[kWaveUnroll], own[kWaveUnroll];
        double gx[kWaveUnroll];
#pragma unroll
        for (int j = 0; j < kWaveUnroll; ++j) {
            const int pos = p0 + tid + j * kWaveThreads;
            own[j] = -1;
            xv[j] = 0;
            gx[j] = 0.0;
            if (pos < total) {
                int l = 0, h = kWaveThreads;  // last k with seg[k] <= pos
                while (h - l > 1) {
                    const int mid = (l + h) >> 1;
                    if (sh.seg[mid] <= pos) l = mid; else h = mid;
                }
                own[j] = l;
                const Entry<CT> en = ld_stream(&a.adj[sh.base[l] + (pos - sh.seg[l])]);
                xv[j] = en.col;
                // c(u, w) of this entry; with parallel edges the cheaper one
                // wins the minimum, as Improve chose it
                gx[j] = sh.gu[l] + widen(en.w);
                if (x.offering && en.col != a.root) ++offers;
            }
        }
        // every load of this batch in flight at once: the parent of each
        // neighbour and, for the offers, its current g
        int32_t px[kWaveUnroll];
        double gold[kWaveUnroll];
#pragma unroll
        for (int j = 0; j < kWaveUnroll; ++j) {
            px[j] = -1;
            gold[j] = 0.0;
            if (own[j] >= 0) {
                px[j] = __ldcg(&a.p[xv[j]]);
                if (x.offering) gold[j] = ld_g_cg(&a.g[xv[j]], x.gpol);
            }
        }
        // then every atomic of the batch.  A child is lowered, and its row
        // extent is loaded beside the atomic for its own expansion.  With
        // offers, a neighbour w that is not a child is offered g(u) + c(u, w)
        // and joins the next Improve list only if that beats its g now: g only
        // falls within an Evaluate and cur(w) = g(p(w)) + c(p(w), w) <= g(w)
        // once it ends, so an offer not below g(w) can never win (and a
        // child's offer equals its own cost).  Without offers every neighbour
        // is marked.
        unsigned childm = 0, markm = 0;
        // a child's row extent is fetched with its atomic: the child is
        // expanded from the local or the global list without another load
        longlong2 ext[kWaveUnroll];
#pragma unroll
        for (int j = 0; j < kWaveUnroll; ++j) {
            ext[j] = make_longlong2(0, 0);
            if (own[j] >= 0) {
                const bool child = sh.dep[own[j]] >= 0 && px[j] == sh.u[own[j]];
                if (child) {
                    ext[j] = __ldg(reinterpret_cast<const longlong2 *>(a.rows) + xv[j]);
                    const unsigned long long b = (unsigned long long)__double_as_longlong(gx[j]);
                    if (atomicMin(reinterpret_cast<unsigned long long *>(&a.g[xv[j]]), b) > b)
                        childm |= 1u << j;
                } else if (x.offering) {
                    if (xv[j] != a.root && gx[j] < gold[j]) {
                        offer(a.cand, xv[j], gx[j]);
                        if (atomicExch(&a.stamp[xv[j]], x.epoch) != x.epoch) markm |= 1u << j;
                    }
                }
                if (x.marking && !a.push && xv[j] != a.root &&
                    __ldcg(&a.stamp[xv[j]]) != x.epoch &&
                    atomicExch(&a.stamp[xv[j]], x.epoch) != x.epoch)
                    markm |= 1u << j;
            }
        }
        recomputed += (unsigned long long)__popc(childm);
        // lowered children: one block scan; the local list takes what fits,
        // the rest goes to the next step's global list (one atomic per CTA)
        const unsigned nmine = (unsigned)__popc(childm);
        unsigned wincl = nmine;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, wincl, off);
            if (lane >= off) wincl += y;
        }
        if (lane == 31) sh.scan[warp] = wincl;
        __syncthreads();
        if (tid == 0) {
            unsigned run = 0;
            for (int w = 0; w < NW; ++w) {
                const unsigned v = (unsigned)sh.scan[w];
                sh.scan[w] = run;
                run += v;
            }
            const unsigned lbase = sh.lcnt;
            const unsigned room = lbase < (unsigned)kWaveThreads ? kWaveThreads - lbase : 0u;
            const unsigned loc = run < room ? run : room;
            sh.scan[NW] = lbase;
            sh.scan[NW + 1] = ((unsigned long long)loc << 32) |
                              (run > loc ? atomicAdd(x.out_cnt, run - loc) : 0u);
            sh.lcnt = lbase + loc;
        }
        __syncthreads();
        {
            const unsigned lbase = (unsigned)sh.scan[NW];
            const unsigned loc = (unsigned)(sh.scan[NW + 1] >> 32);
            const unsigned gbase = (unsigned)(sh.scan[NW + 1] & 0xffffffffull);
            unsigned idx = (unsigned)sh.scan[warp] + wincl - nmine;
#pragma unroll
            for (int j = 0; j < kWaveUnroll; ++j) {
                if (childm & (1u << j)) {
                    const int dd = sh.dep[own[j]] + 1;
                    if (idx < loc) {
                        const unsigned slot = lbase + idx;
                        sh.lu[slot] = xv[j];
                        sh.lg[slot] = gx[j];
                        sh.lb[slot] = ext[j].x;
                        sh.ll[slot] = (int32_t)(unsigned)((unsigned long long)ext[j].y & 0xffffffffull);
                        sh.ld[slot] = dd;
                    } else {
                        const unsigned long long k = (unsigned long long)gbase + (idx - loc);
                        if (k < (unsigned long long)a.list_cap) {  // else: see the caller
                            x.out[k] = xv[j];
                            x.outg[k] = gx[j];
                            x.outx[k] = make_longlong2(
                                ext[j].x, (long long)(((unsigned long long)(unsigned)dd << 32) |
                                                      ((unsigned long long)ext[j].y & 0xffffffffull)));
                        }
                    }
                    ++idx;
                }
            }
        }
        __syncthreads();  // sh.scan is rewritten by the next batch
#pragma unroll
        for (int j = 0; j < kWaveUnroll; ++j)
            mq.push((markm >> j) & 1u, xv[j], x.next, &c->n_next);
    }
    // the first changes of the tile: counted (offers) or listed (no offers)
    if (a.push) {
        const unsigned nf = (unsigned)__popc(__ballot_sync(0xffffffffu, first));
        if (lane == 0 && nf) atomicAdd(&sh.nfirst, nf);
    } else {
        dq.push(first, u, a.dg, &c->n_dg);
    }
    __syncthreads();  // u / gu / base / dep / seg are rewritten by the next tile
}

// One CTA's part of grid step t: the share [lo, hi) of the step's list (the
// switched vertices at step 0), then its local walk; at the end the local list
// and the step's first changes go to the global counters.  Every thread of
// the CTA calls this.
template <typename CT>
__device__ void wave_step(const WaveArgs<CT> &a, WaveShared<CT> &sh, WaveStepCtx<CT> &x,
                          bool from_switched, int64_t lo, int64_t hi, unsigned local_levels,
                          WarpStage<kWaveStage> &mq, WarpStage<kWaveStage> &dq,
                          unsigned long long &recomputed, unsigned long long &offers,
                          unsigned ndg, bool trace = false) {
    DevCounters *c = a.ctr;
    const int tid = threadIdx.x;
    // trace (thread 0 of CTA 0 while profiling): cycles of each tile, by size
    auto tile_trace = [&](unsigned long long *n, unsigned long long *items,
                          unsigned long long *cyc, int nv, long long t0) {
        int b = 32 - __clz((unsigned)nv);
        if (b >= kLevelBuckets) b = kLevelBuckets - 1;
        n[b] += 1ull;
        items[b] += (unsigned long long)nv;
        cyc[b] += (unsigned long long)(clock64() - t0);
    };
    if (tid == 0) {
        sh.lcnt = 0u;
        sh.nfirst = 0u;
    }
    __syncthreads();
    for (int64_t s0 = lo; s0 < hi; s0 += kWaveThreads) {
        const int nv = (hi - s0) < (int64_t)kWaveThreads ? (int)(hi - s0) : kWaveThreads;
        const long long t0 = trace ? clock64() : 0;
        wave_tile<CT>(a, sh, x, from_switched ? kFromSwitched : kFromGlobal, s0, nv, mq, dq,
                      recomputed, offers);
        if (trace) tile_trace(c->shr_n, c->shr_items, c->shr_cyc, nv, t0);
    }
    for (unsigned l = 0;; ++l) {
        __syncthreads();
        const unsigned taken = sh.lcnt;
        const int nl = taken < (unsigned)kWaveThreads ? (int)taken : kWaveThreads;
        if (nl == 0) break;
        if (l >= local_levels || (unsigned)nl > a.local_max) {
            // the walk stops here: the local list joins the next step's list
            __shared__ unsigned s_gb;
            if (tid == 0) s_gb = atomicAdd(x.out_cnt, (unsigned)nl);
            __syncthreads();
            const unsigned long long k = (unsigned long long)s_gb + (unsigned)tid;
            if (tid < nl && k < (unsigned long long)a.list_cap) {
                x.out[k] = sh.lu[tid];
                x.outg[k] = sh.lg[tid];
                x.outx[k] = make_longlong2(
                    sh.lb[tid], (long long)(((unsigned long long)(unsigned)sh.ld[tid] << 32) |
                                            (unsigned long long)(unsigned)sh.ll[tid]));
            }
            break;
        }
        if (tid == 0 && a.push && x.marking) {
            // past the dense limit the next sweep is dense and this CTA stops
            // offering and marking: publish this CTA's first changes so far
            // and take the count as last read (one local level behind)
            if (ndg > a.dense_limit) {
                x.marking = false;
                x.offering = false;
                *(volatile unsigned *)&c->dense_next = 1u;
            } else {
                if (sh.nfirst != 0u) {
                    atomicAdd(&c->n_dg, sh.nfirst);
                    sh.nfirst = 0u;
                }
                ndg = *(volatile unsigned *)&c->n_dg;
            }
        }
        const long long t0 = trace ? clock64() : 0;
        wave_tile<CT>(a, sh, x, kFromLocal, 0, nl, mq, dq, recomputed, offers);
        if (trace) tile_trace(c->loc_n, c->loc_items, c->loc_cyc, nl, t0);
    }
    if (a.push) {
        __syncthreads();
        if (tid == 0 && sh.nfirst != 0u) atomicAdd(&c->n_dg, sh.nfirst);
    } else {
        dq.flush_block(a.dg, &c->n_dg, sh.fl);
    }
    __syncthreads();
}

// Clear the per-iteration fields (not the current list or the dense flag).
__device__ __forceinline__ void clear_iteration(DevCounters *c) {
    c->wave_cnt[0] = 0u;
    c->wave_cnt[1] = 0u;
    c->wave_cnt[2] = 0u;
    c->wave_levels = 0u;
    c->wave_incomplete = 0u;
    c->jumped = 0u;
    c->n_next = 0u;
    c->n_switched = 0u;
    c->dj_bits = 0ull;
    c->n_dg = 0u;
    c->rounds = 0u;
    for (int r = 0; r < kMaxJumpRounds + 2; ++r) c->wl_count[r] = 0u;
}

// Before pointer jumping finishes a wave that hit its level cap: its changed
// list starts empty (the wave counted changes without listing them).  A no-op
// unless the wave stopped early.
static __global__ void pre_jump_kernel(DevCounters *c) {
    if (c->wave_incomplete == 0u) return;
    c->n_dg = 0u;
    c->rounds = 0u;
    c->bar_count = 0u;
    for (int r = 0; r < kMaxJumpRounds + 2; ++r) c->wl_count[r] = 0u;
}

// End of one Replan iteration (Alg. 2): record it, decide whether the loop
// goes on (Improve switched a parent with Delta g > eps, no error, under the
// iteration cap), and make the list built by this iteration's Evaluate the
// current one.  In a captured loop the decision drives the WHILE node.
// Called by one thread, possibly at the end of a kernel whose other CTAs
// wrote the counters: every field is read through L2 (ld.global.cg, issued
// together), then written back.
__device__ __forceinline__ void advance_iteration(DevCounters *c, cudaGraphConditionalHandle cond,
                                                  int use_cond) {
    __threadfence();
    const unsigned sw = __ldcg(&c->n_switched);
    const double dj = __longlong_as_double((long long)__ldcg(&c->dj_bits));
    const double eps = __longlong_as_double((long long)__ldcg(&c->eps_bits));
    const unsigned n_dg = __ldcg(&c->n_dg), levels = __ldcg(&c->wave_levels);
    const unsigned dense_next = __ldcg(&c->dense_next), n_next = __ldcg(&c->n_next);
    const unsigned dense = __ldcg(&c->dense), rounds = __ldcg(&c->rounds);
    const unsigned jumped = __ldcg(&c->jumped), status = __ldcg(&c->status);
    const unsigned long long switches = __ldcg(&c->switches);
    const unsigned cwl = __ldcg(&c->cum_wave_levels), cjr = __ldcg(&c->cum_jump_rounds);
    const unsigned cd = __ldcg(&c->cum_dense), cje = __ldcg(&c->cum_jump_evals);
    const unsigned wave_epoch = __ldcg(&c->wave_epoch), iter = __ldcg(&c->iter) + 1u;
    const unsigned max_iters = __ldcg(&c->max_iters), la = __ldcg(&c->la);
    const unsigned epoch = __ldcg(&c->epoch);
    const double *goal_g = c->goal_g;
    if (goal_g != nullptr)
        c->bound_bits = __ldcg(reinterpret_cast<const unsigned long long *>(goal_g));
    c->last_switched = sw;
    c->last_dg = n_dg;
    c->last_levels = levels;
    c->last_next = dense_next ? 0u : n_next;
    c->last_dense = dense;
    c->last_rounds = rounds;
    c->last_jumped = jumped;
    c->switches = switches + sw;
    c->cum_wave_levels = cwl + levels;
    c->cum_jump_rounds = cjr + rounds;
    c->cum_dense = cd + (dense ? 1u : 0u);
    c->cum_jump_evals = cje + ((jumped && sw) ? 1u : 0u);
    c->wave_epoch = wave_epoch + levels + 1u;
    c->iter = iter;
    const bool stable = sw == 0u || dj <= eps;
    const bool stop = stable || status != 0u || iter >= max_iters;
    c->converged = (stable && status == 0u) ? 1u : 0u;
    c->cont = stop ? 0u : 1u;
    c->la = la ^ 1u;
    c->epoch = epoch + 1u;
    c->n_active = dense_next ? 0u : n_next;
    c->dense = dense_next;
    c->dense_next = 0u;
    clear_iteration(c);
    __threadfence();
    if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

static __global__ void advance_kernel(DevCounters *c, cudaGraphConditionalHandle cond,
                                      int use_cond) {
    advance_iteration(c, cond, use_cond);
}



// Before an exploit or a forced Evaluate: clear the per-iteration fields and
// the whole-exploit totals.
static __global__ void begin_exploit_kernel(DevCounters *c, unsigned max_iters,
                                            unsigned long long eps_bits) {
    clear_iteration(c);
    c->bar_count = 0u;  // no kernel of the graph runs now (see grid_barrier)
    c->relax = 0ull;
    c->improved = 0ull;
    c->evaluated = 0ull;
    c->switches = 0ull;
    c->offers = 0ull;
    c->dense_next = 0u;
    c->iter = 0u;
    c->max_iters = max_iters;
    c->eps_bits = eps_bits;
    c->cont = 1u;
    c->converged = 0u;
    c->cum_wave_levels = 0u;
    c->cum_dense = 0u;
    c->cum_jump_rounds = 0u;
    c->cum_jump_evals = 0u;
    c->t_last_exit = 0ull;  // no gap is counted across exploits
    c->bound_bits = c->goal_g != nullptr
                        ? *reinterpret_cast<const unsigned long long *>(c->goal_g)
                        : 0x7ff0000000000000ull;
}

// The FP32 shadow of g for every vertex, when a wave with offers left it out
// of date (g32_stale) and the next Improve reads it: a dense sweep (dense) or
// an Improve kernel without offers (always_if_stale).  Any grid.
static __global__ void __launch_bounds__(kThreads)
refresh_g32_kernel(DevCounters *c, int64_t n, const double *__restrict__ g,
                   float *__restrict__ g32, int always_if_stale) {
    if (__ldcg(&c->g32_stale) == 0u) return;
    if (!always_if_stale && __ldcg(&c->dense) == 0u) return;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        g32[v] = g32_of(g[v]);
}

// Reset the shadow's flag once refresh_g32_kernel has run (one thread).
static __global__ void refresh_g32_done(DevCounters *c, int always_if_stale) {
    if (always_if_stale || c->dense != 0u) c->g32_stale = 0u;
}

// Parents as reported through the ABI: the root marker becomes -1.
static __global__ void export_parents_kernel(int64_t n, const int32_t *__restrict__ p,
                                             int32_t *__restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        out[v] = p[v] < 0 ? -1 : p[v];
}

// Batched form: translate one graph's local edge ids into the union graph
// (id + base), rejecting ids outside [0, limit).  Writes into the pending
// edge buffer at `out`.
template <typename CT>
__global__ void __launch_bounds__(kThreads)
batch_translate_kernel(int64_t n_edges, const int32_t *__restrict__ src,
                       const int32_t *__restrict__ dst, const CT *__restrict__ cost, int64_t base,
                       int64_t limit, int32_t *__restrict__ out_src, int32_t *__restrict__ out_dst,
                       CT *__restrict__ out_cost, DevCounters *ctr) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_edges;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || b < 0 || a >= limit || b >= limit) {
            atomicOr(&ctr->status, kStatusBadInput);
            out_src[e] = 0;
            out_dst[e] = 0;  // rejected by the union validation as a self loop
            out_cost[e] = CT(0);
            continue;
        }
        out_src[e] = (int32_t)(a + base);
        out_dst[e] = (int32_t)(b + base);
        out_cost[e] = cost[e];
    }
}

// Batched form: parents of one graph in its own ids (root marker -> -1).
static __global__ void export_parents_local_kernel(int64_t n, int64_t base,
                                                   const int32_t *__restrict__ p,
                                                   int32_t *__restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = p[base + v];
        out[v] = q < 0 ? -1 : (int32_t)(q - base);
    }
}

// Make each listed vertex a root: g = 0, parent marker kRootMark.
static __global__ void set_roots_kernel(int64_t k, const int32_t *__restrict__ roots,
                                        double *__restrict__ g, float *__restrict__ g32,
                                        int32_t *__restrict__ p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = roots[i];
        g[r] = 0.0;
        g32[r] = 0.0f;
        p[r] = kRootMark;
    }
}

// ---------------------------------------------------------------------------
// Policy replacement (set_policy): look up each parent edge's cost.
// ---------------------------------------------------------------------------

template <typename CT>
__global__ void __launch_bounds__(kThreads)
policy_lookup_kernel(int64_t n, int32_t root, const int32_t *__restrict__ parent,
                     const RowExt *__restrict__ rows, const Entry<CT> *__restrict__ adj,
                     int32_t *__restrict__ p_out, CT *__restrict__ pc_out, DevCounters *c) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = parent[v];
        if (v == root) {
            if (q != -1) atomicOr(&c->status, kStatusBadInput);
            p_out[v] = kRootMark;
            pc_out[v] = CT(0);
            continue;
        }
        if (q == -1) {
            p_out[v] = -1;
            pc_out[v] = CT(0);
            continue;
        }
        if (q < 0 || q >= n) {
            atomicOr(&c->status, kStatusBadInput);
            continue;
        }
        bool found = false;
        CT best = CT(0);
        int64_t rb, re;
        row_range(rows, v, rb, re);
        for (int64_t i = rb; i < re; ++i) {
            const Entry<CT> en = adj[i];
            if (en.col == q && (!found || en.w < best)) {
                best = en.w;
                found = true;
            }
        }
        if (!found) atomicOr(&c->status, kStatusBadInput);
        p_out[v] = q;
        pc_out[v] = best;
    }
}

// Restore (checkpoint load): packed rows from their offsets, no room to grow
// yet; the FP32 shadow from g; no pending offers.
static __global__ void __launch_bounds__(kThreads)
restore_rows(int64_t n, const int64_t *__restrict__ off, RowExt *__restrict__ rows,
             const double *__restrict__ g, float *__restrict__ g32,
             unsigned long long *__restrict__ cand) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        RowExt r;
        r.beg = off[v];
        r.len = (int32_t)(off[v + 1] - off[v]);
        r.cap = r.len;
        rows[v] = r;
        g32[v] = g32_of(g[v]);
        cand[v] = kCandNone;
    }
}

// Commit a looked-up policy and clear g (Evaluate refills it).
template <typename CT>
__global__ void __launch_bounds__(kThreads)
policy_commit_kernel(int64_t n, int32_t root, const int32_t *__restrict__ p_in,
                     const CT *__restrict__ pc_in, int32_t *__restrict__ p, CT *__restrict__ pc,
                     double *__restrict__ g, float *__restrict__ g32) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        p[v] = p_in[v];
        pc[v] = pc_in[v];
        g[v] = (v == root) ? 0.0 : CUDART_INF;
        g32[v] = (v == root) ? 0.0f : __int_as_float(0x7f800000);
    }
}

}  // namespace pirrt
