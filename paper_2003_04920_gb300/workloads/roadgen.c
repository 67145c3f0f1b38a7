/*
 * Host helpers for the seeded roadmap generator (input generation only).
 *
 * These routines build the synthetic roadmaps that stand in for the paper's
 * planning queries (Sec. V: a 2-D query with obstacles; Sec. III: G = (V, E)
 * with cached edge costs c).  They hold none of the policy-iteration
 * arithmetic: they turn sample points and obstacle sets into an undirected,
 * collision-free edge list with Euclidean costs, ordered so that a
 * Batched-Extension block (Alg. 3) is a contiguous slice.
 *
 * Built with -ffp-contract=off so x86 and Arm hosts give identical roadmaps.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* Union-symmetrise a k-nearest-neighbour table.
 * knn[i*k + j] is the j-th neighbour of vertex i (self excluded, -1 = none).
 * Emits every undirected edge {u, v} once, with u < v, in a deterministic
 * order: row by row, each link owned by exactly one row.
 * Returns the number of edges, or -1 if cap is too small. */
int64_t rg_symmetrize_knn(int64_t n, int64_t k, const int64_t *knn,
                          int32_t *out_u, int32_t *out_v, int64_t cap)
{
    /* pass 1: edge (i, j) from row i is kept by row i if i < j, or if
     * i > j and i is not in row j (a one-sided link owned by the larger id). */
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t a = 0; a < k; ++a) {
            int64_t j = knn[i * k + a];
            if (j < 0 || j == i) continue;
            int dup = 0;
            for (int64_t b = 0; b < a; ++b) if (knn[i * k + b] == j) { dup = 1; break; }
            if (dup) continue;
            if (i < j) { ++c; continue; }
            int mutual = 0;
            for (int64_t b = 0; b < k; ++b) if (knn[j * k + b] == i) { mutual = 1; break; }
            if (!mutual) ++c;
        }
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int64_t m = cnt[n];
    if (m > cap) { free(cnt); return -1; }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t pos = cnt[i];
        for (int64_t a = 0; a < k; ++a) {
            int64_t j = knn[i * k + a];
            if (j < 0 || j == i) continue;
            int dup = 0;
            for (int64_t b = 0; b < a; ++b) if (knn[i * k + b] == j) { dup = 1; break; }
            if (dup) continue;
            if (i < j) { out_u[pos] = (int32_t)i; out_v[pos] = (int32_t)j; ++pos; continue; }
            int mutual = 0;
            for (int64_t b = 0; b < k; ++b) if (knn[j * k + b] == i) { mutual = 1; break; }
            if (!mutual) { out_u[pos] = (int32_t)j; out_v[pos] = (int32_t)i; ++pos; }
        }
    }
    free(cnt);
    return m;
}

/* Squared distance from point q to the segment [a, b] in d dimensions. */
static double seg_point_dist2(const double *a, const double *b, const double *q, int d)
{
    double ab2 = 0.0, t = 0.0;
    for (int x = 0; x < d; ++x) {
        double e = b[x] - a[x];
        ab2 += e * e;
        t += (q[x] - a[x]) * e;
    }
    t = ab2 > 0.0 ? t / ab2 : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double s = 0.0;
    for (int x = 0; x < d; ++x) {
        double p = a[x] + t * (b[x] - a[x]) - q[x];
        s += p * p;
    }
    return s;
}

/* Mark each edge collision-free (keep[e] = 1) or not (0).
 * mode 0: exact segment-sphere test (segment meets an open ball).
 * mode 1: n_check evenly spaced points t = i/(n_check-1), endpoints included,
 *         each tested for lying strictly inside a ball.
 * A cheap bound (midpoint distance vs radius + half length) skips most pairs. */
void rg_filter_collisions(int64_t m, int d, const double *pts,
                          const int32_t *u, const int32_t *v,
                          int64_t n_obs, const double *centers, const double *radii,
                          int mode, int n_check, uint8_t *keep)
{
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t e = 0; e < m; ++e) {
        const double *a = pts + (int64_t)u[e] * d;
        const double *b = pts + (int64_t)v[e] * d;
        double mid[16];
        double half2 = 0.0;
        for (int x = 0; x < d; ++x) {
            mid[x] = 0.5 * (a[x] + b[x]);
            double h = 0.5 * (b[x] - a[x]);
            half2 += h * h;
        }
        double half = sqrt(half2);
        uint8_t ok = 1;
        for (int64_t s = 0; s < n_obs && ok; ++s) {
            const double *c = centers + s * d;
            double r = radii[s];
            double dm2 = 0.0;
            for (int x = 0; x < d; ++x) { double w = mid[x] - c[x]; dm2 += w * w; }
            double lim = r + half;
            if (dm2 >= lim * lim) continue;
            if (mode == 0) {
                if (seg_point_dist2(a, b, c, d) < r * r) ok = 0;
            } else {
                for (int i = 0; i < n_check && ok; ++i) {
                    double t = (n_check > 1) ? (double)i / (double)(n_check - 1) : 0.0;
                    double s2 = 0.0;
                    for (int x = 0; x < d; ++x) {
                        double p = a[x] + t * (b[x] - a[x]) - c[x];
                        s2 += p * p;
                    }
                    if (s2 < r * r) ok = 0;
                }
            }
        }
        keep[e] = ok;
    }
}

/* Euclidean edge lengths in FP64. */
void rg_edge_lengths(int64_t m, int d, const double *pts, const int32_t *u,
                     const int32_t *v, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        const double *a = pts + (int64_t)u[e] * d;
        const double *b = pts + (int64_t)v[e] * d;
        double s = 0.0;
        for (int x = 0; x < d; ++x) { double w = b[x] - a[x]; s += w * w; }
        out[e] = sqrt(s);
    }
}

/* Stable counting sort of edges (u < v) by their larger endpoint v, so that a
 * Batched-Extension block of vertices [b*S, (b+1)*S) owns a contiguous slice
 * of edges.  perm receives the new order; start[x] is the first edge whose
 * larger endpoint is x (start has n + 1 entries). */
int rg_order_by_max(int64_t m, int64_t n, const int32_t *v, int64_t *perm, int64_t *start)
{
    memset(start, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < m; ++e) start[v[e] + 1]++;
    for (int64_t x = 0; x < n; ++x) start[x + 1] += start[x];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!cur) return -1;
    memcpy(cur, start, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < m; ++e) perm[cur[v[e]]++] = e;
    free(cur);
    return 0;
}
