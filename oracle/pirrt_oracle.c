/*
 * CPU oracle for the PI-RRT# exploitation path (test infrastructure).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code with the CUDA library and is deliberately
 * plain, serial and slow.  Everything is FP64; FP32 edge costs arrive
 * already widened to double.
 *
 * O1 (or_replan): serial policy iteration, Alg. 2 (Replan / Improve /
 *     Evaluate), on the adjacency-list graph of Sec. IV-A ("Adjacency List
 *     Graph", the format of the paper's CPU baseline, Sec. V).
 * O2 (or_dijkstra): Dijkstra with a binary heap keyed (distance, id).  By the
 *     correctness argument of Sec. IV ("Correctness", Batched-Extension),
 *     Replan reaches the optimal policy from any initial policy, so the O1
 *     fixpoint must equal single-source shortest paths.
 * Built a second time with OpenMP (liboracle_omp.so), the Jacobi Improve
 *     sweep is shared over the host's cores: each vertex reads only the g of
 *     the last Evaluate and writes only its own parent, so the results are
 *     those of the serial build, bit for bit (a CPU baseline on all cores).
 * Checkers: Bellman inequality on every edge, tree consistency
 *     g(v) = g(p(v)) + c(p(v), v), acyclic parent tree rooted at x_init,
 *     reachable set = component of x_init, and the "unambiguous" mask
 *     (best and second-best candidates differ by more than a relative gap).
 *
 * Goal-directed form (or_set_goal): with a goal x_goal and an admissible
 *     heuristic h (a lower bound on the cost-to-go, Sec. III), Evaluate keeps
 *     walking below a child only while it is promising, and Improve only
 *     switches a vertex that its new parent makes promising (Sec. IV-C, the
 *     promising set B of Sec. III and the vertex property b of Sec. IV-A).
 *
 * Readings of the paper taken here (the paper is silent or loose on them):
 *  - Delta g is reset once per Improve call, before the vertex loop (Alg. 2
 *    shows the reset inside the loop, which would keep only the last vertex).
 *  - The loop stops when Delta g <= eps; with eps = 0 that is "no parent
 *    switched" (a strict "< 0" would never hold).
 *  - Improve scans every vertex except x_init (goal-free form: with no goal
 *    g(x_goal) = +inf, so every vertex Evaluate reaches is promising, and a
 *    vertex not yet reached must still be scanned or it could never join).
 *  - Unreachable vertices keep g = +inf and parent -1.
 *  - Neighbours are scanned in ascending id with a strict "<", so among
 *    equal minimisers the lowest id wins and a current parent that attains
 *    the minimum is kept (its candidate equals g(v) exactly, see Evaluate).
 *  - Parallel edges between the same pair keep the smallest cost.
 *  - Improve measures a candidate against g_hat = g(pi(v)) + c(pi(v), v),
 *    the value of v's current parent edge.  After an Evaluate that reached v
 *    this is g(v) itself; the goal-directed form can leave g(v) unevaluated
 *    (below a pruned vertex), and measuring against that stale g(v) could
 *    switch v back and forth without progress.
 *  - Promising test (goal-directed form): a vertex n is promising when
 *    g(n) + h(n) < g(x_goal), strictly, with g(x_goal) taken at the start of
 *    the Evaluate (the listing tests the popped parent's g and h, which would
 *    admit every child of a promising vertex; the test on the child is the
 *    definition of B).  The value g(x_goal) at the start makes the result
 *    independent of the walk's order; it only prunes less than the running
 *    value would.
 *  - Improve in the goal-directed form examines every vertex but switches v
 *    only if its best candidate makes it promising: g_hat + h(v) < g(x_goal)
 *    (the lookahead key of RRT#).  This covers B and the neighbours of B that
 *    the paper's Improve reaches (Sec. IV-C: promising vertices and their
 *    neighbours are re-evaluated).
 *
 * Built with -ffp-contract=off: every sum below is one IEEE addition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_CAPACITY 2
#define OR_ERR_OOM 3
#define OR_ERR_BAD_INPUT 4
#define OR_ERR_NOT_CONVERGED 5

/* ------------------------------------------------------------------------ */
/* O1: adjacency-list graph with vertex properties in structure-of-arrays    */
/* form (Sec. IV-A: cost-to-come g, parent p; the promising bit b is all ones */
/* in the goal-free form and is not stored).                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t *nbr;   /* neighbour ids */
    double *c;      /* cached edge cost c(nbr, v) */
    int64_t len, cap;
    int dirty;      /* needs sort + merge of parallel edges */
} or_list;

typedef struct {
    int64_t n, cap_n;
    int32_t root;
    or_list *adj;
    double *g;      /* cost-to-come g_pi */
    int32_t *pi;    /* parent: pi(v) = (pi[v], v); -1 = none */
    double *pc;     /* cost of the policy edge, c(pi(v), v) */
    int32_t goal;   /* x_goal of the goal-directed form; -1 = goal-free */
    double *h;      /* heuristic cost-to-go h(v) >= 0 (goal-directed form) */
    uint8_t *b;     /* promising bit b(v), rebuilt by every Evaluate */
} or_graph;

or_graph *or_create(int64_t cap_n, int32_t root)
{
    if (cap_n <= 0 || root < 0 || root >= cap_n) return NULL;
    or_graph *G = (or_graph *)calloc(1, sizeof(or_graph));
    if (!G) return NULL;
    G->cap_n = cap_n;
    G->root = root;
    G->adj = (or_list *)calloc((size_t)cap_n, sizeof(or_list));
    G->g = (double *)malloc(sizeof(double) * (size_t)cap_n);
    G->pi = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap_n);
    G->pc = (double *)malloc(sizeof(double) * (size_t)cap_n);
    G->h = (double *)calloc((size_t)cap_n, sizeof(double));
    G->b = (uint8_t *)calloc((size_t)cap_n, 1);
    G->goal = -1;
    if (!G->adj || !G->g || !G->pi || !G->pc || !G->h || !G->b) {
        free(G->adj); free(G->g); free(G->pi); free(G->pc); free(G->h); free(G->b); free(G);
        return NULL;
    }
    return G;
}

void or_destroy(or_graph *G)
{
    if (!G) return;
    for (int64_t v = 0; v < G->cap_n; ++v) { free(G->adj[v].nbr); free(G->adj[v].c); }
    free(G->adj); free(G->g); free(G->pi); free(G->pc); free(G->h); free(G->b); free(G);
}

/* Goal-directed form: x_goal = goal (-1 switches it off) and h(v) = h[v] for
 * v < n_h, 0 beyond (0 is admissible).  h must be finite and >= 0. */
int or_set_goal(or_graph *G, int32_t goal, const double *h, int64_t n_h)
{
    if (goal < -1 || goal >= G->cap_n || n_h < 0 || n_h > G->cap_n || (n_h > 0 && !h))
        return OR_ERR_ARG;
    for (int64_t x = 0; x < n_h; ++x)
        if (!(h[x] >= 0.0) || !isfinite(h[x])) return OR_ERR_BAD_INPUT;
    for (int64_t x = 0; x < G->cap_n; ++x) G->h[x] = x < n_h ? h[x] : 0.0;
    G->goal = goal;
    return OR_OK;
}

/* g(x_goal), +inf while x_goal is not in the graph or unreached; +inf in the
 * goal-free form, where every reached vertex is promising. */
static double goal_cost(const or_graph *G)
{
    return (G->goal >= 0 && G->goal < G->n) ? G->g[G->goal] : INFINITY;
}

int64_t or_num_vertices(const or_graph *G) { return G->n; }

static int list_push(or_list *L, int32_t w, double c)
{
    if (L->len == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 8;
        int32_t *a = (int32_t *)realloc(L->nbr, sizeof(int32_t) * (size_t)nc);
        if (!a) return OR_ERR_OOM;
        L->nbr = a;
        double *b = (double *)realloc(L->c, sizeof(double) * (size_t)nc);
        if (!b) return OR_ERR_OOM;
        L->c = b;
        L->cap = nc;
    }
    L->nbr[L->len] = w;
    L->c[L->len] = c;
    L->len++;
    L->dirty = 1;
    return OR_OK;
}

/* Append n_new vertices (g = +inf, no parent; g(root) = 0) and m undirected
 * edges {u[e], v[e]} with cost c[e], stored in both lists. */
int or_insert(or_graph *G, int64_t n_new, int64_t m, const int32_t *u, const int32_t *v,
              const double *c)
{
    if (n_new < 0 || m < 0) return OR_ERR_ARG;
    if (G->n + n_new > G->cap_n) return OR_ERR_CAPACITY;
    int64_t n1 = G->n + n_new;
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] < 0 || u[e] >= n1 || v[e] < 0 || v[e] >= n1 || u[e] == v[e])
            return OR_ERR_BAD_INPUT;
        if (!(c[e] > 0.0) || !isfinite(c[e])) return OR_ERR_BAD_INPUT;
    }
    for (int64_t x = G->n; x < n1; ++x) {
        G->g[x] = (x == G->root) ? 0.0 : INFINITY;
        G->pi[x] = -1;
        G->pc[x] = 0.0;
    }
    G->n = n1;
    for (int64_t e = 0; e < m; ++e) {
        int rc = list_push(&G->adj[u[e]], v[e], c[e]);
        if (rc) return rc;
        rc = list_push(&G->adj[v[e]], u[e], c[e]);
        if (rc) return rc;
    }
    return OR_OK;
}

/* Sort one list by neighbour id (insertion sort keeps it obviously right;
 * lists are short) and merge parallel edges, keeping the smaller cost. */
static void list_normalise(or_list *L)
{
    if (!L->dirty) return;
    for (int64_t i = 1; i < L->len; ++i) {
        int32_t w = L->nbr[i];
        double c = L->c[i];
        int64_t j = i - 1;
        while (j >= 0 && (L->nbr[j] > w || (L->nbr[j] == w && L->c[j] > c))) {
            L->nbr[j + 1] = L->nbr[j];
            L->c[j + 1] = L->c[j];
            --j;
        }
        L->nbr[j + 1] = w;
        L->c[j + 1] = c;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < L->len; ++i) {
        if (k > 0 && L->nbr[k - 1] == L->nbr[i]) continue; /* first = cheapest */
        L->nbr[k] = L->nbr[i];
        L->c[k] = L->c[i];
        ++k;
    }
    L->len = k;
    L->dirty = 0;
}

static void normalise_all(or_graph *G)
{
    for (int64_t x = 0; x < G->n; ++x) list_normalise(&G->adj[x]);
}

/* Evaluate (Alg. 2): breadth-first walk of the policy tree from x_init,
 * g(n) <- c(v, n) + g(v) for every child n of v, and B <- the children that
 * are promising, g(n) + h(n) < g(x_goal); the walk continues below those
 * only.  With no goal (or x_goal not reached yet) every reached vertex is
 * promising and the walk covers the tree.  Returns the number of vertices
 * assigned, or -1 on allocation failure. */
static int64_t evaluate(or_graph *G)
{
    int64_t n = G->n;
    /* child lists of the policy tree, children in ascending id */
    int64_t *first = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *kids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!first || !kids || !queue) { free(first); free(kids); free(queue); return -1; }
    for (int64_t x = 0; x < n; ++x)
        if (G->pi[x] >= 0) first[G->pi[x] + 1]++;
    for (int64_t x = 0; x < n; ++x) first[x + 1] += first[x];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) { free(first); free(kids); free(queue); return -1; }
    for (int64_t x = 0; x < n; ++x) fill[x] = first[x];
    for (int64_t x = 0; x < n; ++x)
        if (G->pi[x] >= 0) kids[fill[G->pi[x]]++] = (int32_t)x;
    free(fill);

    const double bound = goal_cost(G); /* g(x_goal) before this walk */
    memset(G->b, 0, (size_t)n);
    int64_t head = 0, tail = 0, assigned = 0;
    queue[tail++] = G->root;
    G->b[G->root] = 1;
    while (head < tail) {
        int32_t x = queue[head++];
        for (int64_t i = first[x]; i < first[x + 1]; ++i) {
            int32_t y = kids[i];
            G->g[y] = G->pc[y] + G->g[x];
            ++assigned;
            if (G->g[y] + G->h[y] < bound) { /* promising: y joins B */
                queue[tail++] = y;
                G->b[y] = 1;
            }
        }
    }
    free(first); free(kids); free(queue);
    return assigned;
}

/* Improve (Alg. 2): Jacobi relaxation.  For each vertex v except x_init,
 * g_hat <- g(pi(v)) + c(pi(v), v) (+inf without a parent); for each
 * neighbour n in ascending id, if c(n, v) + g(n) < g_hat then g_hat <- that
 * value and n becomes the new parent -- taken only if it makes v promising,
 * g_hat + h(v) < g(x_goal) (always, goal-free).  Delta g is the largest
 * decrease taken.  g is read only: every candidate uses the last Evaluate. */
static double improve(or_graph *G, int64_t *relax, int64_t *switched)
{
    double dJ = 0.0;
    const double bound = goal_cost(G);
    int64_t relax_sum = 0, switched_sum = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : relax_sum, switched_sum) \
    reduction(max : dJ)
#endif
    for (int64_t x = 0; x < G->n; ++x) {
        if (x == G->root) continue;
        const or_list *L = &G->adj[x];
        const double cur = G->pi[x] >= 0 ? G->g[G->pi[x]] + G->pc[x] : INFINITY;
        double ghat = cur;
        int32_t best = -1;
        double best_c = 0.0;
        for (int64_t i = 0; i < L->len; ++i) {
            double cand = L->c[i] + G->g[L->nbr[i]];
            if (cand < ghat) {
                ghat = cand;
                best = L->nbr[i];
                best_c = L->c[i];
            }
        }
        relax_sum += L->len;
        if (best >= 0 && ghat + G->h[x] < bound) {
            G->pi[x] = best;
            G->pc[x] = best_c;
            ++switched_sum;
            double d = cur - ghat;
            if (d > dJ) dJ = d;
        }
    }
    *relax += relax_sum;
    *switched += switched_sum;
    return dJ;
}

/* Threads the Improve sweep runs on: 1 in the plain build. */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Replace the policy with parent[] (-1 = none) and evaluate it.  Every
 * parent edge must exist; its cost is the cached c of that edge. */
int or_set_policy(or_graph *G, const int32_t *parent)
{
    normalise_all(G);
    for (int64_t x = 0; x < G->n; ++x) {
        int32_t p = parent[x];
        if (x == G->root) { if (p != -1) return OR_ERR_BAD_INPUT; continue; }
        if (p == -1) { G->pi[x] = -1; G->pc[x] = 0.0; G->g[x] = INFINITY; continue; }
        if (p < 0 || p >= G->n) return OR_ERR_BAD_INPUT;
        const or_list *L = &G->adj[x];
        int64_t i = 0;
        while (i < L->len && L->nbr[i] != p) ++i;
        if (i == L->len) return OR_ERR_BAD_INPUT;
        G->pi[x] = p;
        G->pc[x] = L->c[i];
        G->g[x] = INFINITY;
    }
    G->g[G->root] = 0.0;
    return evaluate(G) < 0 ? OR_ERR_OOM : OR_OK;
}

/* Replan (Alg. 2): loop { (pi, dJ) <- Improve; if dJ <= eps break;
 * (g, B) <- Evaluate }.  stats[0..4] = iterations (Improve calls),
 * relaxations (neighbour entries scanned), vertices evaluated, parent
 * switches, converged flag. */
int or_replan(or_graph *G, double eps, int64_t max_iters, int64_t *stats)
{
    normalise_all(G);
    int64_t iters = 0, relax = 0, evaluated = 0, switched = 0;
    int converged = 0;
    if (max_iters <= 0) max_iters = G->n + 2;
    while (iters < max_iters) {
        double dJ = improve(G, &relax, &switched);
        ++iters;
        if (dJ <= eps) { converged = 1; break; }
        int64_t a = evaluate(G);
        if (a < 0) return OR_ERR_OOM;
        evaluated += a;
    }
    if (stats) {
        stats[0] = iters; stats[1] = relax; stats[2] = evaluated;
        stats[3] = switched; stats[4] = converged;
    }
    return converged ? OR_OK : OR_ERR_NOT_CONVERGED;
}

void or_get(const or_graph *G, double *g, int32_t *parent)
{
    for (int64_t x = 0; x < G->n; ++x) {
        if (g) g[x] = G->g[x];
        if (parent) parent[x] = G->pi[x];
    }
}

/* The promising set B of the last Evaluate as bits b(v) (Sec. IV-A). */
void or_get_promising(const or_graph *G, uint8_t *b)
{
    for (int64_t x = 0; x < G->n; ++x) b[x] = G->b[x];
}

/* ------------------------------------------------------------------------ */
/* Static CSR for O2 and the checkers: rows sorted by id, parallel edges      */
/* merged to their smallest cost.                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n, m;     /* m = directed entries after merging */
    int64_t *off;
    int32_t *col;
    double *c;
} or_csr;

static int cmp_entry(const void *a, const void *b)
{
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

or_csr *or_csr_build(int64_t n, int64_t m, const int32_t *u, const int32_t *v, const double *c)
{
    or_csr *A = (or_csr *)calloc(1, sizeof(or_csr));
    if (!A) return NULL;
    A->n = n;
    A->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    A->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    A->c = (double *)malloc(sizeof(double) * (size_t)(2 * m + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!A->off || !A->col || !A->c || !fill) {
        free(fill); free(A->off); free(A->col); free(A->c); free(A);
        return NULL;
    }
    for (int64_t e = 0; e < m; ++e) { A->off[u[e] + 1]++; A->off[v[e] + 1]++; }
    for (int64_t x = 0; x < n; ++x) A->off[x + 1] += A->off[x];
    for (int64_t x = 0; x <= n; ++x) fill[x] = A->off[x];
    for (int64_t e = 0; e < m; ++e) {
        A->col[fill[u[e]]] = v[e]; A->c[fill[u[e]]++] = c[e];
        A->col[fill[v[e]]] = u[e]; A->c[fill[v[e]]++] = c[e];
    }
    free(fill);
    /* sort each row by (id, cost) through a scratch array of (key, cost bits) */
    int64_t maxdeg = 0;
    for (int64_t x = 0; x < n; ++x)
        if (A->off[x + 1] - A->off[x] > maxdeg) maxdeg = A->off[x + 1] - A->off[x];
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(maxdeg + 1));
    if (!tmp) { free(A->off); free(A->col); free(A->c); free(A); return NULL; }
    int64_t w = 0;
    for (int64_t x = 0; x < n; ++x) {
        int64_t b = A->off[x], e = A->off[x + 1], d = e - b;
        for (int64_t i = 0; i < d; ++i) {
            tmp[2 * i] = A->col[b + i];
            memcpy(&tmp[2 * i + 1], &A->c[b + i], sizeof(double));
        }
        qsort(tmp, (size_t)d, 2 * sizeof(int64_t), cmp_entry);
        A->off[x] = w;
        for (int64_t i = 0; i < d; ++i) {
            int32_t y = (int32_t)tmp[2 * i];
            double cy;
            memcpy(&cy, &tmp[2 * i + 1], sizeof(double));
            if (w > A->off[x] && A->col[w - 1] == y) {
                if (cy < A->c[w - 1]) A->c[w - 1] = cy;
                continue;
            }
            A->col[w] = y;
            A->c[w] = cy;
            ++w;
        }
    }
    A->off[n] = w;
    A->m = w;
    free(tmp);
    return A;
}

void or_csr_destroy(or_csr *A)
{
    if (!A) return;
    free(A->off); free(A->col); free(A->c); free(A);
}

int64_t or_csr_entries(const or_csr *A) { return A->m; }

/* binary heap of (distance, id) pairs, smallest first */
typedef struct { double d; int32_t x; } hitem;

static int hless(hitem a, hitem b) { return a.d < b.d || (a.d == b.d && a.x < b.x); }

/* O2: Dijkstra from root.  dist = +inf and parent = -1 off the root's
 * component.  Each relaxation computes dist(x) + c, the same single FP64
 * addition O1 uses for a candidate.  Lazy deletion: stale heap items are
 * skipped when popped. */
int or_dijkstra(const or_csr *A, int32_t root, double *dist, int32_t *parent)
{
    int64_t n = A->n;
    if (root < 0 || root >= n) return OR_ERR_ARG;
    hitem *h = (hitem *)malloc(sizeof(hitem) * (size_t)(A->m + 2));
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    if (!h || !done) { free(h); free(done); return OR_ERR_OOM; }
    for (int64_t x = 0; x < n; ++x) { dist[x] = INFINITY; parent[x] = -1; }
    dist[root] = 0.0;
    int64_t hn = 0;
    h[hn++] = (hitem){0.0, root};
    while (hn > 0) {
        hitem top = h[0];
        h[0] = h[--hn];
        for (int64_t i = 0;;) { /* sift down */
            int64_t l = 2 * i + 1, r = l + 1, s = i;
            if (l < hn && hless(h[l], h[s])) s = l;
            if (r < hn && hless(h[r], h[s])) s = r;
            if (s == i) break;
            hitem t = h[i]; h[i] = h[s]; h[s] = t; i = s;
        }
        int32_t x = top.x;
        if (done[x] || top.d != dist[x]) continue;
        done[x] = 1;
        for (int64_t i = A->off[x]; i < A->off[x + 1]; ++i) {
            int32_t y = A->col[i];
            double nd = dist[x] + A->c[i];
            if (!done[y] && nd < dist[y]) {
                dist[y] = nd;
                parent[y] = x;
                int64_t j = hn++; /* sift up */
                h[j] = (hitem){nd, y};
                while (j > 0) {
                    int64_t p = (j - 1) / 2;
                    if (!hless(h[j], h[p])) break;
                    hitem t = h[j]; h[j] = h[p]; h[p] = t; j = p;
                }
            }
        }
    }
    free(h); free(done);
    return OR_OK;
}

/* Vertices of the root's connected component (plain BFS). */
int64_t or_component(const or_csr *A, int32_t root, uint8_t *reach)
{
    int64_t n = A->n, head = 0, tail = 0;
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!q) return -1;
    memset(reach, 0, (size_t)n);
    reach[root] = 1;
    q[tail++] = root;
    while (head < tail) {
        int32_t x = q[head++];
        for (int64_t i = A->off[x]; i < A->off[x + 1]; ++i) {
            int32_t y = A->col[i];
            if (!reach[y]) { reach[y] = 1; q[tail++] = y; }
        }
    }
    free(q);
    return tail;
}

/* Parent-tree check: parent[root] = -1; every other parent is -1 or an
 * adjacent vertex; following parents from any vertex with a parent reaches
 * the root without revisiting a vertex.  Returns the number of bad vertices;
 * *first_bad gets the smallest one (or -1). */
int64_t or_check_tree(const or_csr *A, int32_t root, const int32_t *parent, int64_t *first_bad)
{
    int64_t n = A->n, bad = 0;
    *first_bad = -1;
    /* state: 0 unknown, 1 on current walk, 2 reaches root, 3 broken */
    uint8_t *st = (uint8_t *)calloc((size_t)n, 1);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!st || !path) { free(st); free(path); return -1; }
    if (parent[root] != -1) { bad++; *first_bad = root; }
    st[root] = 2;
    for (int64_t s = 0; s < n; ++s) {
        if (st[s] || parent[s] == -1) continue;
        int64_t len = 0;
        int64_t x = s;
        uint8_t verdict = 3;
        for (;;) {
            if (st[x] == 2) { verdict = 2; break; }
            if (st[x] == 3 || st[x] == 1) { verdict = 3; break; }
            int32_t p = parent[x];
            if (p < 0 || p >= n) { verdict = 3; st[x] = 1; path[len++] = (int32_t)x; break; }
            int adjacent = 0;
            for (int64_t i = A->off[x]; i < A->off[x + 1]; ++i)
                if (A->col[i] == p) { adjacent = 1; break; }
            st[x] = 1;
            path[len++] = (int32_t)x;
            if (!adjacent) { verdict = 3; break; }
            x = p;
        }
        for (int64_t i = 0; i < len; ++i) {
            st[path[i]] = verdict;
            if (verdict == 3) {
                bad++;
                if (*first_bad < 0 || path[i] < *first_bad) *first_bad = path[i];
            }
        }
    }
    free(st); free(path);
    return bad;
}

/* Bellman inequality on every directed entry (y -> x): g(x) <= g(y) + c(y, x)
 * with relative slack rel.  Returns the violation count. */
int64_t or_check_bellman(const or_csr *A, const double *g, double rel, int64_t *worst)
{
    int64_t bad = 0;
    double wv = 0.0;
    *worst = -1;
    for (int64_t x = 0; x < A->n; ++x) {
        for (int64_t i = A->off[x]; i < A->off[x + 1]; ++i) {
            double bound = g[A->col[i]] + A->c[i];
            if (!(g[x] <= bound * (1.0 + rel)) && isfinite(bound)) {
                bad++;
                double gap = g[x] - bound;
                if (*worst < 0 || gap > wv) { wv = gap; *worst = x; }
            }
        }
    }
    return bad;
}

/* Tree consistency: |g(x) - (g(p(x)) + c(p(x), x))| <= rel * g(x) wherever
 * p(x) >= 0; g(root) = 0; g = +inf exactly where p = -1 (root excluded).
 * Returns the count of failing vertices. */
int64_t or_check_consistency(const or_csr *A, int32_t root, const int32_t *parent,
                             const double *g, double rel, int64_t *first_bad)
{
    int64_t bad = 0;
    *first_bad = -1;
    for (int64_t x = 0; x < A->n; ++x) {
        int ok = 1;
        if (x == root) ok = (g[x] == 0.0);
        else if (parent[x] < 0) ok = isinf(g[x]) && g[x] > 0;
        else {
            double c = NAN;
            for (int64_t i = A->off[x]; i < A->off[x + 1]; ++i)
                if (A->col[i] == parent[x]) { c = A->c[i]; break; }
            double want = g[parent[x]] + c;
            ok = isfinite(want) && fabs(g[x] - want) <= rel * fabs(want);
        }
        if (!ok) { bad++; if (*first_bad < 0) *first_bad = x; }
    }
    return bad;
}

/* For every vertex x other than the root with finite g: the best candidate
 * value min_y g(y) + c(y, x) over neighbours with the lowest minimising id
 * (argmin[x]), and whether the second-best distinct neighbour is worse by
 * more than rel * best (mask[x] = 1).  Vertices with one finite candidate are
 * unambiguous; the root and unreachable vertices get mask 0, argmin -1.
 * Returns the number of unambiguous vertices. */
int64_t or_unambiguous(const or_csr *A, int32_t root, const double *g, double rel,
                       uint8_t *mask, int32_t *argmin)
{
    int64_t count = 0;
    for (int64_t x = 0; x < A->n; ++x) {
        mask[x] = 0;
        argmin[x] = -1;
        if (x == root || !isfinite(g[x])) continue;
        double b1 = INFINITY, b2 = INFINITY;
        int32_t a1 = -1;
        for (int64_t i = A->off[x]; i < A->off[x + 1]; ++i) {
            double v = g[A->col[i]] + A->c[i];
            if (v < b1) { b2 = b1; b1 = v; a1 = A->col[i]; }
            else if (v < b2) b2 = v;
        }
        argmin[x] = a1;
        if (a1 >= 0 && (b2 - b1) > rel * b1) { mask[x] = 1; count++; }
    }
    return count;
}
