// A Replan iteration as one cooperative launch (graph_kernels.cuh holds the
// wave's level step, pointer jumping, marking and the end of the iteration;
// improve_push.cuh the Improve from candidate offers).
#pragma once

#include <type_traits>

#include "graph_kernels.cuh"
#include "improve_push.cuh"
#include "improve_screen.cuh"

namespace pirrt {

// Level trace of one wave launch (thread 0 of CTA 0 only, while profiling):
// each level's cycles run from its start to the next level's start, so its
// grid barrier counts with it.  state: -1 off, -2 before the first level,
// -3 after the last, b >= 0 the bucket of the running level.
struct LevelClock {
    long long t;
    int state;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void lc_start(DevCounters *c, LevelClock &lc) {
    lc.state = (blockIdx.x == 0 && threadIdx.x == 0 && c->lvl_trace != 0u) ? -2 : -1;
    lc.t = clock64();
    if (lc.state != -1) {
        const unsigned long long now = global_ns();
        c->t_enter = now;
        const unsigned long long last = __ldcg(&c->t_last_exit);
        if (last != 0ull && now > last) {
            c->gap_ns += now - last;
            c->gaps += 1ull;
        }
    }
}

// The thread that ends the iteration: the launch's span (traced launches).
__device__ __forceinline__ void trace_exit(DevCounters *c) {
    if (c->lvl_trace == 0u) return;
    const unsigned long long now = global_ns();
    const unsigned long long t0 = __ldcg(&c->t_enter);
    if (t0 != 0ull && now > t0) {
        c->span_ns += now - t0;
        c->spans += 1ull;
    }
    c->t_last_exit = now;
}

// A level of `count` vertices starts now (count 0: the levels are over).
__device__ __forceinline__ void lc_level(DevCounters *c, LevelClock &lc, long long count) {
    if (lc.state == -1) return;
    const long long now = clock64();
    const unsigned long long d = (unsigned long long)(now - lc.t);
    if (lc.state == -2) c->ph_pre_cyc += d;
    else if (lc.state >= 0) c->lvl_cyc[lc.state] += d;
    else c->ph_post_cyc += d;
    lc.t = now;
    if (count > 0) {
        int b = 64 - __clzll((unsigned long long)count);
        if (b >= kLevelBuckets) b = kLevelBuckets - 1;
        c->lvl_n[b] += 1ull;
        c->lvl_items[b] += (unsigned long long)count;
        lc.state = b;
    } else {
        lc.state = -3;
    }
}

__device__ __forceinline__ void lc_end(DevCounters *c, LevelClock &lc) {
    if (lc.state == -1) return;
    lc_level(c, lc, 0);
    c->ph_calls += 1ull;
}

// One Replan iteration in one launch: Improve from offers (when `ip` is
// given; the dense-sweep kernel runs before this one), a grid barrier, the
// top-down wave in grid steps (each CTA walking the subtrees it reaches on
// its own for a few levels, see wave_step); if a vertex was too deep to
// expand, pointer jumping and the frontier marking of its changes; then the
// end of the iteration (advance_iteration), which in a captured loop sets the
// WHILE condition.
template <typename CT>
__global__ void __launch_bounds__(kWaveThreads, 2)
wave_evaluate_kernel(const WaveArgs<CT> *__restrict__ ap, const EvaluateArgs<CT> *__restrict__ ep,
                     const MarkArgs<CT> *__restrict__ mp, const ImproveArgs<CT> *__restrict__ ip,
                     cudaGraphConditionalHandle cond, int use_cond, int fuse_dense) {
    const WaveArgs<CT> a = *ap;
    __shared__ WaveShared<CT> sh;
    DevCounters *c = a.ctr;
    LevelClock lc;
    lc_start(c, lc);
    unsigned phase = 0;  // thread 0: phase bit of the grid barrier
    if (threadIdx.x == 0) phase = barrier_phase(c);
    if (ip != nullptr) {
        // fuse_dense (FP32 costs): the dense sweeps run here too, by the same
        // screened 4-lane body as the dense-sweep kernel, so that a captured
        // iteration is this one launch
        if constexpr (std::is_same<CT, float>::value) {
            if (fuse_dense && __ldcg(&c->dense) != 0u) improve_screen_body<4, 4, kWaveThreads>(*ip);
        }
        improve_push_body<CT, 8>(*ip);  // the list sweep, or the offers' reset before a dense one
        // a timeout is in the status word; the iteration still ends
        grid_barrier_phased(c, gridDim.x, phase);
    }
    const unsigned n_sw = *(volatile unsigned *)&c->n_switched;
    if (n_sw == 0u) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            lc_end(c, lc);
            trace_exit(c);
            advance_iteration(c, cond, use_cond);
        }
        return;
    }
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x;
    // the step's lists and flags, the same for every thread: kept in shared
    // memory (thread 0 writes them each step) rather than in registers
    __shared__ WaveStepCtx<CT> x;
    if (tid == 0) {
        x.epoch = c->epoch + 1u;  // stamp of the list being built
        x.tag = c->wave_epoch;    // first-change stamp of this Evaluate
        x.next = ((c->la & 1u) ^ 1u) ? a.list[1] : a.list[0];
        x.gpol = policy_evict_last();
        x.bound = goal_bound(c, a.h);
    }
    WarpStage<kWaveStage> mq{sh.stage[tid >> 5], 0u};   // Improve-list appends
    WarpStage<kWaveStage> dq{sh.dstage[tid >> 5], 0u};  // changed-list appends (no offers)
    unsigned long long recomputed = 0, offers = 0;
    // The changed vertices are counted once each (and listed without offers):
    // after every step barrier each CTA reads the count with the next step's
    // size, and past the dense limit the marking stops and the next sweep is
    // dense (whichever way this Evaluate ends).
    const bool push = a.push != 0;
    unsigned t = 0;
    for (;;) {
        int64_t count =
            t == 0 ? (int64_t)n_sw : (int64_t)(*(volatile unsigned *)&c->wave_cnt[t % 3]);
        const unsigned ndg = *(volatile unsigned *)&c->n_dg;
        lc_level(c, lc, count);
        if (count == 0) break;
        const bool over = ndg > a.dense_limit;
        const bool stop = count > a.list_cap;
        __syncthreads();  // the previous step's readers of x are done
        if (tid == 0) {
            if (over) *(volatile unsigned *)&c->dense_next = 1u;
            x.marking = !over && *(volatile unsigned *)&c->dense_next == 0u;
            x.offering = push && x.marking;
            x.in = (t & 1u) ? a.lvl[1] : a.lvl[0];
            x.ing = (t & 1u) ? a.lvg[1] : a.lvg[0];
            x.inx = (t & 1u) ? a.lvx[1] : a.lvx[0];
            x.out = (t & 1u) ? a.lvl[0] : a.lvl[1];
            x.outg = (t & 1u) ? a.lvg[0] : a.lvg[1];
            x.outx = (t & 1u) ? a.lvx[0] : a.lvx[1];
            x.out_cnt = &c->wave_cnt[(t + 1) % 3];
            x.stop = stop;
        }
        __syncthreads();
        if (stop) {
            // The step's list overflowed (children lost -- parallel edges):
            // its vertices were lowered; scan their rows for the frontier and
            // the offers only; pointer jumping finishes every value and the
            // next sweep is dense.
            if (blockIdx.x == 0 && tid == 0) c->dense_next = 1u;
            count = a.list_cap;
            const int64_t per = (count + nblocks - 1) / nblocks;
            const int64_t lo = (int64_t)blockIdx.x * per;
            const int64_t hi = lo + per < count ? lo + per : count;
            wave_step<CT>(a, sh, x, t == 0, lo, hi, 0u, mq, dq, recomputed, offers, ndg,
                          lc.state != -1);
            ++t;
            grid_barrier_phased(c, nblocks, phase);
            break;
        }
        if (blockIdx.x == 0 && tid == 0) c->wave_cnt[(t + 2) % 3] = 0u;
        if (count <= (int64_t)a.tail_max) {
            // a thin step: CTA 0 walks it on alone, with no level limit
            if (blockIdx.x == 0)
                wave_step<CT>(a, sh, x, t == 0, 0, count, 0xffffffffu, mq, dq, recomputed, offers,
                              ndg, lc.state != -1);
        } else {
            const int64_t per = (count + nblocks - 1) / nblocks;
            const int64_t lo = (int64_t)blockIdx.x * per;
            const int64_t hi = lo + per < count ? lo + per : count;
            wave_step<CT>(a, sh, x, t == 0, lo, hi,
                          count <= (int64_t)a.local_step ? a.local_levels : 0u, mq, dq, recomputed,
                          offers, ndg, lc.state != -1);
        }
        ++t;
        if (!grid_barrier_phased(c, nblocks, phase)) break;
    }
    mq.flush_block(x.next, &c->n_next, sh.fl);
    if (!push) {
        // the FP32 shadow of every changed vertex, from its final g
        const unsigned n_dg = *(volatile unsigned *)&c->n_dg;
        for (unsigned i = blockIdx.x * kWaveThreads + tid; i < n_dg; i += nblocks * kWaveThreads) {
            const int32_t w = __ldcg(&a.dg[i]);
            a.g32[w] = g32_of(__ldcg(&a.g[w]));
        }
    } else if (*(volatile unsigned *)&c->wave_incomplete == 0u) {
        // past the dense limit the next sweep is dense and reads the FP32
        // shadow, so every vertex's shadow is refreshed now; otherwise it is
        // left out of date and flagged (refresh_g32_kernel brings it up to
        // date before any Improve that reads it)
        const bool dense_next = *(volatile unsigned *)&c->n_dg > a.dense_limit;
        if (blockIdx.x == 0 && tid == 0) {
            if (dense_next) c->dense_next = 1u;
            c->g32_stale = dense_next ? 0u : 1u;
        }
        if (dense_next)
            for (int64_t v = (int64_t)blockIdx.x * kWaveThreads + tid; v < a.n;
                 v += (int64_t)nblocks * kWaveThreads)
                a.g32[v] = g32_of(__ldcg(&a.g[v]));
    }
    block_add(recomputed, &c->evaluated, sh.scan);
    block_add(offers, &c->offers, sh.scan);
    if (blockIdx.x == 0 && tid == 0) c->wave_levels = t;
    // wave_incomplete was set before the last grid barrier, so every CTA takes
    // the same branch.  A grid barrier that timed out raised kStatusTimeout:
    // the iteration still ends, which stops the loop.
    if (*(volatile unsigned *)&c->wave_incomplete != 0u) {
        // a vertex was too deep to expand: pointer jumping finishes the
        // values and its changes are marked; the wave's changed list gives way
        lc_level(c, lc, 0);
        const long long t_jump = clock64();
        bool ok = grid_barrier(c, nblocks) && *(volatile unsigned *)&c->status == 0u;
        if (ok && blockIdx.x == 0 && tid == 0) {
            c->n_dg = 0u;
            c->rounds = 0u;
            for (int r = 0; r < kMaxJumpRounds + 2; ++r) c->wl_count[r] = 0u;
        }
        if (ok) ok = grid_barrier(c, nblocks);
        if (ok) ok = jump_evaluate<CT>(*ep);
        if (ok) ok = grid_barrier(c, nblocks);
        if (ok) mark_changed<CT>(*mp);
        grid_barrier(c, nblocks);
        if (blockIdx.x == 0 && tid == 0) {
            if (lc.state != -1) c->ph_jump_cyc += (unsigned long long)(clock64() - t_jump);
            lc_end(c, lc);
            trace_exit(c);
            advance_iteration(c, cond, use_cond);
        }
        return;
    }
    // otherwise the last CTA to finish ends the iteration (no grid barrier)
    lc_end(c, lc);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&c->wave_ticket, 1u) == nblocks - 1u) {
            c->wave_ticket = 0u;
            trace_exit(c);
            advance_iteration(c, cond, use_cond);
        }
    }
}

}  // namespace pirrt
