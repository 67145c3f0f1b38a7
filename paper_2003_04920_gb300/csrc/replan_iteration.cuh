// A Replan iteration as one cooperative launch (graph_kernels.cuh holds the
// wave's level step, pointer jumping, marking and the end of the iteration;
// improve_push.cuh the Improve from candidate offers).
#pragma once

#include "graph_kernels.cuh"
#include "improve_push.cuh"

namespace pirrt {

// One Replan iteration in one launch: Improve from offers (when `ip` is
// given; the dense-sweep kernel runs before this one), a grid barrier, the
// top-down wave; if it stopped at its level cap, pointer jumping and the
// frontier marking of its changes; then the end of the iteration
// (advance_iteration), which in a captured loop sets the WHILE condition.
template <typename CT>
__global__ void __launch_bounds__(kWaveThreads, 2)
wave_evaluate_kernel(const WaveArgs<CT> *__restrict__ ap, const EvaluateArgs<CT> *__restrict__ ep,
                     const MarkArgs<CT> *__restrict__ mp, const ImproveArgs<CT> *__restrict__ ip,
                     cudaGraphConditionalHandle cond, int use_cond) {
    const WaveArgs<CT> a = *ap;
    __shared__ WaveShared<CT> sh;
    __shared__ unsigned s_t;
    DevCounters *c = a.ctr;
    if (ip != nullptr) {
        improve_push_body<CT, 8>(*ip);
        grid_barrier(c, gridDim.x);  // a timeout is in the status word; the iteration still ends
    }
    const unsigned n_sw = *(volatile unsigned *)&c->n_switched;
    if (n_sw == 0u) {
        if (blockIdx.x == 0 && threadIdx.x == 0) advance_iteration(c, cond, use_cond);
        return;
    }
    const unsigned epoch = c->epoch + 1u;  // stamp of the list being built
    const unsigned tag = c->wave_epoch;    // first-change stamp of this Evaluate
    int32_t *next = ((c->la & 1u) ^ 1u) ? a.list[1] : a.list[0];
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x;
    const unsigned long long gpol = policy_evict_last();
    unsigned long long recomputed = 0, offers = 0;
    // With offers the wave keeps no changed list, only its size n_dg (each
    // changed vertex counted once): after every level barrier each CTA reads it
    // with the next level's size, and past the dense limit the marking stops
    // and the next sweep is dense (whichever way this Evaluate ends).
    const bool push = a.push != 0;
    unsigned t = 0;
    for (;;) {
        int64_t count =
            t == 0 ? (int64_t)n_sw : (int64_t)(*(volatile unsigned *)&c->wave_cnt[t % 3]);
        const unsigned ndg = push ? *(volatile unsigned *)&c->n_dg : 0u;
        if (count == 0) break;
        const bool over = push && ndg > a.dense_limit;
        if (over && tid == 0) *(volatile unsigned *)&c->dense_next = 1u;
        if (t >= a.max_levels || count > a.list_cap) {
            // Stop: this level's vertices were lowered but not expanded.  Scan
            // their rows for the frontier and the offers only; pointer jumping
            // finishes the values below them.  (Children beyond the list's
            // capacity -- parallel edges -- were lost: the next sweep is dense.)
            if (blockIdx.x == 0 && tid == 0) {
                c->wave_incomplete = 1u;
                if (count > a.list_cap) c->dense_next = 1u;
            }
            if (count > a.list_cap) count = a.list_cap;
            const int64_t per = (count + nblocks - 1) / nblocks;
            const int64_t lo = (int64_t)blockIdx.x * per;
            const int64_t hi = lo + per < count ? lo + per : count;
            wave_level<CT>(a, sh, t, lo, hi, tag, epoch, next, gpol, recomputed, offers, false, over);
            grid_barrier(c, nblocks);
            break;
        }
        if (count <= (int64_t)a.tail_max) {
            // a thin level: CTA 0 walks on alone while the levels stay thin
            if (blockIdx.x == 0) {
                bool over_t = over;
                for (;;) {
                    if (tid == 0) c->wave_cnt[(t + 2) % 3] = 0u;
                    __syncthreads();
                    wave_level<CT>(a, sh, t, 0, count, tag, epoch, next, gpol, recomputed, offers,
                                   true, over_t);
                    ++t;
                    if (tid == 0) s_t = *(volatile unsigned *)&c->wave_cnt[t % 3];
                    __syncthreads();
                    count = (int64_t)s_t;
                    __syncthreads();
                    if (count == 0 || count > (int64_t)a.tail_max || count > a.list_cap ||
                        t >= a.max_levels)
                        break;
                    if (push) {
                        // n_dg holds this CTA's own additions (same thread)
                        if (tid == 0) s_t = *(volatile unsigned *)&c->n_dg;
                        __syncthreads();
                        over_t = s_t > a.dense_limit;
                        __syncthreads();
                        if (over_t && tid == 0) *(volatile unsigned *)&c->dense_next = 1u;
                    }
                }
                if (tid == 0) c->wave_t = t;
            }
            if (!grid_barrier(c, nblocks)) break;
            t = *(volatile unsigned *)&c->wave_t;
            continue;
        }
        if (blockIdx.x == 0 && tid == 0) c->wave_cnt[(t + 2) % 3] = 0u;
        const int64_t per = (count + nblocks - 1) / nblocks;
        const int64_t lo = (int64_t)blockIdx.x * per;
        const int64_t hi = lo + per < count ? lo + per : count;
        wave_level<CT>(a, sh, t, lo, hi, tag, epoch, next, gpol, recomputed, offers, true, over);
        ++t;
        if (!grid_barrier(c, nblocks)) break;
    }
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
        // stopped at the level cap: pointer jumping finishes the values and
        // its changes are marked; the wave's changed list gives way
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
        if (blockIdx.x == 0 && tid == 0) advance_iteration(c, cond, use_cond);
        return;
    }
    // otherwise the last CTA to finish ends the iteration (no grid barrier)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&c->wave_ticket, 1u) == nblocks - 1u) {
            c->wave_ticket = 0u;
            advance_iteration(c, cond, use_cond);
        }
    }
}

}  // namespace pirrt
