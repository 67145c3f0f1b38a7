// Device-side building blocks shared by the PI-RRT# kernels: CSR entry
// layouts, streaming loads, warp-aggregated list appends, the bounded grid
// barrier and the device counter block.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pirrt {

// Status bits a kernel may raise (never a trap).
constexpr unsigned kStatusBadInput = 1u;
constexpr unsigned kStatusTimeout = 2u;
constexpr unsigned kStatusBadTree = 4u;

// A grid barrier gives up after this many polls (each followed by a short
// sleep), i.e. well over a second: it then raises kStatusTimeout.
constexpr unsigned long long kBarrierSpinLimit = 1ull << 25;

// Evaluate stops pointer jumping after this many rounds: a parent chain of
// length L finishes in about log2(L) + 1 rounds, so anything left over after
// 40 rounds sits on a cycle.
constexpr int kMaxJumpRounds = 40;

// Size buckets of the level trace: bucket b holds the top-down Evaluate
// levels of 2^(b-1) .. 2^b - 1 vertices (the last bucket: every larger one).
constexpr int kLevelBuckets = 24;

// One adjacency entry of the device CSR.  FP32 costs pack (col, c) into 8 B
// so one 8-byte load fetches both; FP64 costs use a 16 B entry.
template <typename CT>
struct Entry;
template <>
struct __align__(8) Entry<float> {
    int32_t col;
    float w;
};
template <>
struct __align__(16) Entry<double> {
    int32_t col;
    int32_t pad;
    double w;
};

// Streaming (evict-first) load of a CSR entry: each entry is read once per
// sweep, so it should not displace g from L2.
__device__ __forceinline__ Entry<float> ld_stream(const Entry<float> *p) {
    int2 r = __ldcs(reinterpret_cast<const int2 *>(p));
    Entry<float> e;
    e.col = r.x;
    e.w = __int_as_float(r.y);
    return e;
}
__device__ __forceinline__ Entry<double> ld_stream(const Entry<double> *p) {
    int4 r = __ldcs(reinterpret_cast<const int4 *>(p));
    Entry<double> e;
    e.col = r.x;
    e.pad = 0;
    e.w = __hiloint2double(r.w, r.z);
    return e;
}

// L2 eviction priorities.  g is gathered once per CSR entry from anywhere in
// the array, so it should stay resident in L2 (evict_last) while the CSR,
// read once per sweep, passes through (evict_first).
__device__ __forceinline__ unsigned long long policy_evict_last() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Read-only load of g(u) that keeps its line in L2.
__device__ __forceinline__ double ld_g(const double *p, unsigned long long pol) {
    double v;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
// Coherent (L2) load of g(u) that keeps its line in L2 (for data written in
// the same kernel by other CTAs).
__device__ __forceinline__ double ld_g_cg(const double *p, unsigned long long pol) {
    double v;
    asm volatile("ld.global.cg.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}

// FP32 shadow of g used to screen Improve candidates (GB300 runs FP64 at a
// small fraction of its FP32 rate).  +inf stays +inf; a finite g above 2^100
// is stored as -1, which sends every row reading it down the exact FP64 path.
__device__ __forceinline__ float g32_of(double g) {
    if (g <= 1.2676506002282294e30) return __double2float_rn(g);  // g >= 0, up to 2^100
    return isinf(g) ? __int_as_float(0x7f800000) : -1.0f;
}

// Exact widening of a positive finite float to double with integer
// operations (no FP64 pipe); subnormals take the conversion instruction.
__device__ __forceinline__ double widen(float w) {
    const unsigned b = __float_as_uint(w);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)w;
    const unsigned long long d = ((unsigned long long)(b >> 31) << 63) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}
__device__ __forceinline__ double widen(double w) { return w; }

// Device counters of one graph.  The host copies the block back once per
// Replan iteration.
// Counters that every CTA of a kernel adds to sit on 128-byte lines of
// their own: atomics to one line are serialised by its L2 slice, and
// unrelated counters must not queue behind each other.
struct DevCounters {
    alignas(128) unsigned long long relax;  // adjacency entries scanned by Improve (whole exploit)
    alignas(128) unsigned long long improved;  // vertices processed by Improve (whole exploit)
    alignas(128) unsigned long long evaluated;  // vertices whose g was recomputed (whole exploit)
    alignas(128) unsigned long long offers;  // candidates offered to the next Improve (whole exploit)
    alignas(128) unsigned long long dj_bits;  // Delta g of the current Improve (bits of a double >= 0)
    alignas(128) unsigned n_switched;  // switches in the current iteration
    alignas(128) unsigned n_next;      // size of the list being built for the next Improve
    alignas(128) unsigned n_dg;        // vertices whose g changed in the current Evaluate
    alignas(128) unsigned wave_cnt[3];  // top-down Evaluate: list sizes of levels t, t+1, t+2 (mod 3)
    alignas(128) unsigned bar_count;   // grid barrier: arrivals (low bits) and phase (top bit)
    alignas(128) unsigned wave_ticket;  // CTAs done with a wave that ends without a barrier
    alignas(128) unsigned wl_count[kMaxJumpRounds + 2];  // pointer-jumping work-list sizes per round
    alignas(128) unsigned n_touched;   // insertion: old rows gaining entries (list length)
    alignas(128) unsigned long long pool_cursor;  // insertion: pool room taken by the block
    alignas(128) unsigned status;      // kStatus* bits
    unsigned long long switches;  // parent switches (whole exploit)
    unsigned long long insert_copied;  // CSR entries moved by insertions (graph lifetime)
    unsigned n_active;            // size of the current Improve list
    unsigned rounds;              // pointer-jumping rounds of the current Evaluate
    unsigned dense;               // current Improve sweeps every vertex
    unsigned dense_next;          // next Improve sweeps every vertex
    unsigned wave_levels;         // grid steps run by the last top-down Evaluate
    unsigned wave_incomplete;     // the top-down Evaluate stopped at its level cap
    // Iteration state kept on the device so that one captured loop body (and
    // the host loop alike) serves every iteration:
    unsigned la;                  // which of the two lists Improve reads
    unsigned epoch;               // stamp value of the current Improve list
    unsigned wave_epoch;          // stamp of level 1 of the next top-down Evaluate
    unsigned iter;                // Improve rounds run in this exploit
    unsigned max_iters;           // cap on Improve rounds
    unsigned cont;                // the loop continues (set by advance)
    unsigned converged;           // the last advance saw a stable policy
    unsigned jumped;              // this iteration's Evaluate ran pointer jumping
    unsigned g32_stale;           // a wave with offers changed g without its FP32 shadow
    unsigned long long eps_bits;  // Delta g threshold (bits of a double >= 0)
    // Goal-directed Replan (Sec. IV-C): &g[x_goal] (null = goal-free), and
    // g(x_goal) as the current iteration began -- the bound of the promising
    // test, the same for every CTA and every kernel of the iteration.
    const double *goal_g;
    unsigned long long bound_bits;
    // last completed iteration (read by the host after advance)
    unsigned last_switched, last_dg, last_levels, last_next, last_dense, last_rounds, last_jumped;
    // whole-exploit totals
    unsigned cum_wave_levels, cum_dense, cum_jump_rounds, cum_jump_evals;
    // Level trace, kept while profiling is on (lvl_trace = 1) and left alone
    // by a reset of the graph: the top-down Evaluate's levels by size bucket,
    // the vertices they held and CTA 0's SM cycles over them (each level's
    // grid barrier included); the cycles of a wave launch before its first
    // level (Improve from offers and its barrier), after its last, and in a
    // pointer-jumping finish; and the launches traced.  Only thread 0 of CTA 0
    // writes them.
    unsigned lvl_trace;
    unsigned long long lvl_n[kLevelBuckets], lvl_items[kLevelBuckets], lvl_cyc[kLevelBuckets];
    // CTA 0's own tiles, by tile size: its share of a grid step (shr_*) and
    // the levels it walked on its own (loc_*), with their cycles
    unsigned long long shr_n[kLevelBuckets], shr_items[kLevelBuckets], shr_cyc[kLevelBuckets];
    unsigned long long loc_n[kLevelBuckets], loc_items[kLevelBuckets], loc_cyc[kLevelBuckets];
    // Wave launches on the global timer (ns): from CTA 0's start to the end of
    // the iteration (span), and from one launch's end to the next one's start
    // within an exploit (gap: the launches in between and the launch latency)
    unsigned long long t_enter, t_last_exit, span_ns, spans, gap_ns, gaps;
    unsigned long long ph_pre_cyc, ph_post_cyc, ph_jump_cyc, ph_calls;
};

// Block-wide sum of one value per thread, added to *counter by one atomic.
// Every thread of the block must call it; s needs blockDim.x / 32 entries.
__device__ __forceinline__ void block_add(unsigned long long x, unsigned long long *counter,
                                          unsigned long long *s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    __syncthreads();
    if (lane == 0) s[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        if (t) atomicAdd(counter, t);
    }
}

// Block-wide maximum, applied to *counter by one atomic (same rules).
__device__ __forceinline__ void block_max(unsigned long long x, unsigned long long *counter,
                                          unsigned long long *s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, x, off);
        x = o > x ? o : x;
    }
    __syncthreads();
    if (lane == 0) s[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = s[w] > t ? s[w] : t;
        if (t) atomicMax(counter, t);
    }
}

// Row extent of a vertex in the slack CSR: its entries are
// adj[beg, beg + len); the row may grow in place up to beg + cap.
struct __align__(16) RowExt {
    long long beg;
    int32_t len;
    int32_t cap;
};

// [b, e) of row v, one 16-byte load.
__device__ __forceinline__ void row_range(const RowExt *rows, int64_t v, int64_t &b, int64_t &e) {
    const longlong2 r = __ldg(reinterpret_cast<const longlong2 *>(rows) + v);
    b = r.x;
    e = r.x + (long long)(int32_t)(unsigned)((unsigned long long)r.y & 0xffffffffull);
}

// Parent marker of a root vertex (g = 0, never re-parented).  Reported as -1.
constexpr int32_t kRootMark = -2;

// Append `value` to `list` for every lane with `pred`, one atomic per warp.
// Every lane of the warp must call this (warp-uniform control flow).
__device__ __forceinline__ void warp_append(bool pred, int32_t value, int32_t *list,
                                            unsigned *counter) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned ballot = __ballot_sync(0xffffffffu, pred);
    if (ballot == 0u) return;
    const int leader = __ffs(ballot) - 1;
    unsigned base = 0;
    if (lane == (unsigned)leader) base = atomicAdd(counter, (unsigned)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) list[base + __popc(ballot & ((1u << lane) - 1u))] = value;
}

// Warp-private staging of list appends in shared memory: items collect in a
// per-warp buffer (ballot offsets, no atomics) and reach the global list in
// batches, one atomicAdd per flush.  All 32 lanes must call push / flush
// together; `count` is warp-uniform.
template <int CAP>
struct WarpStage {
    int32_t *buf;    // CAP slots in shared memory, private to the warp
    unsigned count;  // items staged

    __device__ __forceinline__ void flush(int32_t *list, unsigned *counter) {
        const unsigned lane = threadIdx.x & 31u;
        if (count == 0u) return;
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(counter, count);
        base = __shfl_sync(0xffffffffu, base, 0);
        __syncwarp();
        for (unsigned i = lane; i < count; i += 32u) list[base + i] = buf[i];
        __syncwarp();
        count = 0u;
    }

    // End of a kernel: every warp of the block flushes together, one
    // atomicAdd per block.  s needs blockDim.x / 32 + 1 entries.
    __device__ __forceinline__ void flush_block(int32_t *list, unsigned *counter, unsigned *s) {
        const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) s[warp] = count;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned run = 0;
            for (unsigned w = 0; w < (blockDim.x >> 5); ++w) {
                const unsigned k = s[w];
                s[w] = run;
                run += k;
            }
            s[blockDim.x >> 5] = run ? atomicAdd(counter, run) : 0u;
        }
        __syncthreads();
        const unsigned base = s[blockDim.x >> 5] + s[warp];
        for (unsigned i = lane; i < count; i += 32u) list[base + i] = buf[i];
        count = 0u;
    }

    __device__ __forceinline__ void push(bool pred, int32_t value, int32_t *list,
                                         unsigned *counter) {
        const unsigned lane = threadIdx.x & 31u;
        const unsigned ballot = __ballot_sync(0xffffffffu, pred);
        const unsigned n = (unsigned)__popc(ballot);
        if (n == 0u) return;
        if (count + n > (unsigned)CAP) flush(list, counter);
        if (pred) buf[count + __popc(ballot & ((1u << lane) - 1u))] = value;
        count += n;
        __syncwarp();
    }
};

// Block-wide reservation in two lists at once: thread i wants na[i] slots of
// list A and nb[i] of list B.  One atomicAdd per list per block; returns this
// thread's first slot in each.  Every thread of the block must call it;
// s_scan needs THREADS / 32 + 2 entries.
template <int THREADS>
__device__ __forceinline__ void block_reserve2(unsigned na, unsigned nb, unsigned *ctr_a,
                                               unsigned *ctr_b, unsigned long long *s_scan,
                                               unsigned &base_a, unsigned &base_b) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long x = ((unsigned long long)nb << 32) | na;
    unsigned long long incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < NW; ++w) {
            const unsigned long long t = s_scan[w];
            s_scan[w] = run;
            run += t;
        }
        const unsigned ta = (unsigned)(run & 0xffffffffull), tb = (unsigned)(run >> 32);
        s_scan[NW] = ta ? atomicAdd(ctr_a, ta) : 0u;
        s_scan[NW + 1] = tb ? atomicAdd(ctr_b, tb) : 0u;
    }
    __syncthreads();
    const unsigned long long ex = s_scan[warp] + incl - x;
    base_a = (unsigned)s_scan[NW] + (unsigned)(ex & 0xffffffffull);
    base_b = (unsigned)s_scan[NW + 1] + (unsigned)(ex >> 32);
    __syncthreads();
}

// block_reserve2 for any block size (s_scan: blockDim.x / 32 + 2 entries).
__device__ __forceinline__ void block_reserve2_dyn(unsigned na, unsigned nb, unsigned *ctr_a,
                                                   unsigned *ctr_b, unsigned long long *s_scan,
                                                   unsigned &base_a, unsigned &base_b) {
    const int nw = (int)(blockDim.x >> 5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long x = ((unsigned long long)nb << 32) | na;
    unsigned long long incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < nw; ++w) {
            const unsigned long long t = s_scan[w];
            s_scan[w] = run;
            run += t;
        }
        const unsigned ta = (unsigned)(run & 0xffffffffull), tb = (unsigned)(run >> 32);
        s_scan[nw] = ta ? atomicAdd(ctr_a, ta) : 0u;
        s_scan[nw + 1] = tb ? atomicAdd(ctr_b, tb) : 0u;
    }
    __syncthreads();
    const unsigned long long ex = s_scan[warp] + incl - x;
    base_a = (unsigned)s_scan[nw] + (unsigned)(ex & 0xffffffffull);
    base_b = (unsigned)s_scan[nw + 1] + (unsigned)(ex >> 32);
    __syncthreads();
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  One
// word counts arrivals: every block adds 1 except block 0, which adds
// 2^31 - (nblocks - 1), so the last arrival flips the top bit and leaves the
// low bits as they were (0 between barriers).  A block waits for the flip of
// the top bit it saw on arrival; nobody resets the word, so a slow block can
// never miss its barrier's completion (begin_exploit_kernel clears the word
// between launches).  The wait is bounded (spin_limit polls, each followed by
// a short sleep): on timeout the block raises kStatusTimeout and the caller
// returns.  Returns false on timeout.
__device__ __forceinline__ bool grid_barrier(DevCounters *c, unsigned nblocks,
                                             unsigned long long spin_limit = kBarrierSpinLimit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1u) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(&c->bar_count, inc);
        volatile unsigned *word = &c->bar_count;
        int ok = 1;
        unsigned long long spins = 0;
        while (((old ^ *word) & 0x80000000u) == 0u) {
            if (++spins > spin_limit) {
                atomicOr(&c->status, kStatusTimeout);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The same barrier for a kernel whose CTAs know its phase: thread 0 of every
// CTA reads the phase bit once at kernel start (barrier_phase; no CTA can
// complete a barrier before every CTA has arrived, so all read the same bit)
// and passes it to each barrier, which toggles it.  The arrival is then an
// atomic whose result nobody waits for.  Use it for every grid barrier of the
// kernel up to the first grid_barrier, which does not keep the phase.
__device__ __forceinline__ unsigned barrier_phase(const DevCounters *c) {
    return *reinterpret_cast<const volatile unsigned *>(&c->bar_count) & 0x80000000u;
}

__device__ __forceinline__ bool grid_barrier_phased(DevCounters *c, unsigned nblocks,
                                                    unsigned &phase,
                                                    unsigned long long spin_limit = kBarrierSpinLimit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1u) : 1u;
        __threadfence();
        atomicAdd(&c->bar_count, inc);  // result unused: a reduction, no round trip to wait for
        phase ^= 0x80000000u;
        volatile unsigned *word = &c->bar_count;
        int ok = 1;
        unsigned long long spins = 0;
        while ((*word & 0x80000000u) != phase) {
            if (++spins > spin_limit) {
                atomicOr(&c->status, kStatusTimeout);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace pirrt
