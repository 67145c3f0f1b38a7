/*
 * roadgen_gpu.h -- GPU-resident roadmap generator (input generation only).
 *
 * Builds the same kind of synthetic planning roadmap as the host generator
 * (workloads/__init__.py), entirely on one GPU, for sizes the host cannot
 * build quickly (10^7 samples and more): the sampling-based roadmap of
 * PI-RRT# (Sec. III: samples of the free space, each joined to its nearest
 * neighbours by collision-free edges with cached Euclidean costs, Sec. IV-A),
 * ordered for Batched-Extension (Alg. 3).  It holds none of the
 * policy-iteration arithmetic (Improve / Evaluate, Alg. 2).
 *
 * Definitions (each reproduced exactly by the CPU reference in the tests):
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC 2011), key = the
 *     seed's two 32-bit halves, counter = (candidate index low, high, word,
 *     0).  Candidate i's coordinate d is lo + (hi - lo) * u with u =
 *     (x >> 8) * 2^-24, x the d-th output word of counters (i, 0) and (i, 1).
 *   - A candidate is free when sum_d (p_d - c_d)^2 >= r^2 (FP64, no fused
 *     multiply-add) for every obstacle ball (c, r); the first n free
 *     candidates, in index order, are the vertices.
 *   - Nearest neighbours: the k smallest (d2, id) pairs, d2 the FP32 squared
 *     distance of the FP32-rounded coordinates (no fused multiply-add, sum
 *     over d in order), self excluded.
 *   - Edges: the union of the k-nearest relations, {u, v} once with u < v;
 *     kept when collision-free: mode 0 = the segment meets no open ball
 *     (exact closest-point test), mode 1 = none of n_check evenly spaced
 *     points t = i / (n_check - 1) lies strictly inside a ball; cost =
 *     sqrt of the FP64 squared length (FP32 or FP64 cost type); ordered by
 *     the larger endpoint v, then by u, with edge_start[v] the first edge of
 *     v (so block b of S vertices is the slice edge_start[bS] ..
 *     edge_start[(b+1)S]).
 *
 * All pointers are device pointers the caller owns.  Calls are ordered on
 * `stream` and synchronise it where they return a size to the host.
 * Return value 0 = success, 1 = invalid argument, 2 = CUDA error, 3 = a
 * capacity given by the caller is too small.
 */
#ifndef ROADGEN_GPU_H
#define ROADGEN_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* n free samples (FP64, n x dim, row-major) of the box [lo, hi]^dim outside
 * n_obs balls (centers: n_obs x dim FP64, radii: n_obs FP64).  *tried gets
 * the number of candidates drawn.  dim in [1, 8]. */
int rgg_sample(int32_t dim, double lo, double hi, int32_t n_obs, const double *centers,
               const double *radii, uint64_t seed, int64_t n, double *points, int64_t *tried,
               void *stream);

/* k nearest neighbours (ids, nearest first) of every point, by a uniform grid
 * of cells of side about `cell` (0 = chosen from n, k and the box).  knn: n x k
 * int32.  Needs k < n, k <= 128. */
int rgg_knn(int32_t dim, double lo, double hi, int64_t n, const double *points, int32_t k,
            double cell, int32_t *knn, void *stream);

/* Union-symmetrised, collision-checked edges of a k-NN table, ordered by the
 * larger endpoint: u, v (int32), cost (float if cost_f64 = 0, else double),
 * edge_start (int64, n + 1).  cap = room of u / v / cost; *m gets the edge
 * count (3 = cap too small, *m then holds the count needed). */
int rgg_edges(int32_t dim, int64_t n, const double *points, int32_t k, const int32_t *knn,
              int32_t n_obs, const double *centers, const double *radii, int32_t mode,
              int32_t n_check, int32_t cost_f64, int32_t *u, int32_t *v, void *cost,
              int64_t *edge_start, int64_t cap, int64_t *m, void *stream);

/* Incremental exploration: the Extend step of RRT# one Batched-Extension
 * block at a time (Alg. 3), for running on its own stream while the previous
 * block is exploited (the asynchronous exploration the paper leaves to future
 * work, Sec. VII).  Vertex i joins the k vertices nearest to it among the
 * vertices 0 .. i-1 (FP32 squared distance as for rgg_knn, ties by id;
 * every predecessor while i <= k) by the collision-free, positive-length
 * edges among those links, cost = sqrt of the FP64 squared length.  The
 * roadmap therefore does not depend on the block size.  The n free samples
 * are drawn at create time (rgg_sample's definition, same seed rule). */
typedef struct rgg_explorer rgg_explorer;

int rgg_explore_create(int32_t dim, double lo, double hi, int32_t n_obs, const double *centers,
                       const double *radii, uint64_t seed, int64_t n, int32_t k, int32_t mode,
                       int32_t n_check, int32_t cost_f64, int64_t max_block, void *stream,
                       rgg_explorer **out);

/* The edges of the new vertices [v0, v1) (v1 - v0 <= max_block): (u, v) with
 * u < v = the new vertex, ordered by v then by nearness, into u / v / cost
 * (room for (v1 - v0) * k edges), all ordered on `stream` with no host
 * synchronisation; *m_pinned (page-locked host memory) receives the edge
 * count when the stream gets there. */
int rgg_explore_block(rgg_explorer *x, int64_t v0, int64_t v1, int32_t *u, int32_t *v, void *cost,
                      int64_t *m_pinned, void *stream);

/* The samples (device FP64, n x dim) and their number; a copy of them into
 * out (device, n x dim), ordered on `stream`. */
const double *rgg_explore_points(const rgg_explorer *x);
int64_t rgg_explore_size(const rgg_explorer *x);
int rgg_explore_copy_points(const rgg_explorer *x, double *out, void *stream);

void rgg_explore_destroy(rgg_explorer *x);

#ifdef __cplusplus
}
#endif

#endif /* ROADGEN_GPU_H */
