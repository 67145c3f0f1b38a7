/*
 * pirrt.h -- C ABI of the GB300 exploitation path of PI-RRT#
 * (Policy Iteration RRT#, Lawson, Wills and Tsiotras, "GPU Parallelization
 * of Policy Iteration RRT#").
 *
 * Problem (Sec. III): an undirected graph G = (V, E) with positive edge
 * costs c : E -> R+, a root x_init, a policy pi : V -> E (each vertex's
 * parent edge) and the cost-to-come g_pi : V -> R+ along the policy tree.
 * The library keeps G, pi and g resident on one GPU and runs
 *   - Batched-Extension insertion of a block of vertices and edges (Alg. 3;
 *     Sec. IV-A, the edge list is merged into a CSR on the device),
 *   - Replan (Alg. 2): Improve (every vertex re-selects its parent as the
 *     argmin over neighbours u of g(u) + c(u, v)) and Evaluate (recompute g
 *     under the new parent tree), repeated until no parent changes;
 *     optionally goal-directed (Sec. IV-C, pirrt_graph_set_goal).
 *
 * Conventions shared by every entry point:
 *   - Vertex ids are dense int32: insert_batch appends ids [n, n + n_new).
 *     The root is fixed at create time; g(root) = 0.
 *   - Edges are undirected: one (src, dst, cost) triple is stored in both
 *     directions.  Parallel edges are allowed; the cheapest one wins.
 *   - Costs are FP32 or FP64 (pirrt_config.cost_dtype); g is always FP64.
 *   - Pointers flagged "on_device" are CUDA device pointers (any allocator,
 *     e.g. PyTorch's); otherwise they are host pointers.  The caller owns
 *     every buffer it passes; the library reads inputs before the call
 *     returns and never retains caller pointers, except
 *     pirrt_graph_prefetch_batch, whose copies read the host buffers after
 *     it returns (its comment gives how long they must stay).
 *   - All device work is ordered on the stream given at create time
 *     (NULL = legacy default stream).  Calls that return results to the
 *     host (exploit, get_*) synchronise that stream before returning.
 *   - Errors are returned as pirrt_status; no exception crosses the ABI.
 *     Device kernels report errors through a status word, never by trapping.
 *     pirrt_graph_last_error() gives a human-readable detail string.
 *   - A handle is not thread-safe; the caller serialises calls on it.
 */
#ifndef PIRRT_H
#define PIRRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIRRT_OK = 0,
    PIRRT_ERR_INVALID_ARG = 1,     /* NULL handle/pointer, negative size, bad option */
    PIRRT_ERR_CAPACITY = 2,        /* max_vertices or max_edges would be exceeded */
    PIRRT_ERR_OOM = 3,             /* device or host allocation failed */
    PIRRT_ERR_CUDA = 4,            /* a CUDA runtime call failed */
    PIRRT_ERR_NOT_CONVERGED = 5,   /* max_iters Improve rounds ran with parents still switching */
    PIRRT_ERR_DEVICE_TIMEOUT = 6,  /* a device-side wait ran out (grid barrier) */
    PIRRT_ERR_BAD_INPUT = 7,       /* id out of range, self loop, cost <= 0 / NaN / Inf,
                                      or a policy edge that is not in G */
    PIRRT_ERR_BAD_TREE = 8         /* parent pointers contain a cycle */
} pirrt_status;

enum { PIRRT_COST_F32 = 0, PIRRT_COST_F64 = 1 };

/* Fixed at create time. */
typedef struct {
    int64_t max_vertices;  /* capacity of V */
    int64_t max_edges;     /* capacity of E in undirected edges (each uses two CSR entries) */
    int32_t root;          /* x_init, in [0, max_vertices) */
    int32_t cost_dtype;    /* PIRRT_COST_F32 or PIRRT_COST_F64 */
    int32_t device;        /* CUDA device ordinal */
    int32_t reserved;
    void *stream;          /* cudaStream_t for all work; NULL = legacy default stream */
} pirrt_config;

/* Per exploit call.  Zero-initialised gives the defaults. */
typedef struct {
    double eps;             /* Replan stops once Delta g <= eps (Alg. 2); 0 = until no
                               parent switches */
    int32_t max_iters;      /* cap on Improve rounds; 0 = |V| + 2 */
    int32_t group;          /* lanes per vertex of the lane-group Improve kernels: 2 (screened
                               only), 4, 8, 16 or 32; 0 = tuned (4 screened, 8 exact) */
    int32_t tile;           /* Improve kernel: 0 = list sweeps from candidate offers (every
                               vertex whose g changed offers g(u) + c(u, v) to each neighbour
                               while its row is scanned; a listed vertex reads its row only
                               when the best offer beats its parent), dense sweeps as tile 2;
                               2 = lane groups with FP32 screening (FP64 costs: exact lane
                               groups) for every sweep; 1 = staged (a producer warp bulk-
                               copies 32-row tiles into a 4-stage shared-memory ring for 8
                               consumer warps); 3 = lane groups, exact FP64 for every
                               candidate.  All give the same parents and g. */
    int32_t evaluate;       /* PIRRT_EVAL_AUTO, _WAVE, _JUMP or _ASYNC */
    int32_t wave_levels;    /* AUTO: level cap of the top-down Evaluate before it hands over
                               to pointer jumping; 0 = tuned */
    int32_t host_loop;      /* 1 = drive the Replan loop from the host, one counter read per
                               iteration; 0 = one CUDA-graph launch for the whole loop (a WHILE
                               node repeats Improve / Evaluate on the device).  Profiling
                               always uses the host loop. */
    double dense_fraction;  /* changed vertices, as a fraction of |V|, above which the next
                               Improve sweeps every vertex instead of a list; 0 = tuned */
    int32_t wave_tail;      /* top-down Evaluate: grid steps of at most this many vertices
                               are walked by one CTA, with no level limit and no grid barrier;
                               0 = tuned, < 0 = off */
    int32_t wave_ctas;      /* top-down Evaluate: CTAs per SM (1 or 2); 0 = tuned */
    int32_t wave_local;     /* top-down Evaluate: tree levels a CTA walks on its own, from the
                               children it lowered, before they join the next grid step;
                               0 = tuned, < 0 = none (one level per grid step) */
    int32_t wave_local_max; /* ... while its list of such children holds at most this many
                               vertices (a wider subtree is shared by the whole grid at the
                               next step); 1 .. 512, 0 = tuned */
    int32_t wave_local_step; /* ... in grid steps of at most this many vertices (a CTA walking on
                               alone in a wider step would hold back the others); 0 = tuned */
} pirrt_exploit_opts;

/* Evaluate strategies.  All compute g(v) = g(p(v)) + c(p(v), v) from the root
 * in FP64 (Alg. 2 Evaluate):
 *   WAVE  -- top-down over the policy tree, level by level, only below the
 *            vertices whose parent switched, pruning where g is unchanged; the
 *            next Improve frontier is marked in the same row scan.  Sums are
 *            taken root-to-leaf, one addition per edge, as in Alg. 2.  Work is
 *            shared out in grid steps separated by a grid-wide barrier; within
 *            a step each CTA walks the children it lowered for a few levels on
 *            its own (g lowered by an atomic minimum, as in ASYNC).
 *   JUMP  -- pointer jumping (parent doubling) over every vertex in about
 *            log2(depth) rounds; the sums are reassociated (within a few ulp).
 *   ASYNC -- the same walk as WAVE without level barriers: each CTA follows
 *            subtrees on its own and g is lowered by an atomic minimum, which
 *            no stale value can defeat because Improve never raises a
 *            cost-to-come (Sec. V policy improvement).  Same sums, bit for bit.
 *   AUTO  -- WAVE, handing over to JUMP when a wave exceeds its level cap. */
enum { PIRRT_EVAL_AUTO = 0, PIRRT_EVAL_WAVE = 1, PIRRT_EVAL_JUMP = 2, PIRRT_EVAL_ASYNC = 3 };

/* Filled by pirrt_graph_exploit. */
typedef struct {
    int32_t iterations;     /* Improve rounds run (the last one switched nothing if converged) */
    int32_t converged;      /* 1 if the policy is stable */
    int64_t relaxations;    /* candidates g(u) + c(u, v) formed: adjacency entries scanned by
                               Improve, plus the offers made by Evaluate (tile 0) */
    int64_t improved;       /* vertices processed by Improve, summed over rounds */
    int64_t switches;       /* parent switches, summed over rounds */
    int64_t evaluated;      /* vertices whose g Evaluate recomputed, summed over rounds */
    int32_t jump_rounds;    /* pointer-jumping rounds, summed over Evaluate calls */
    int32_t dense_sweeps;   /* Improve rounds that swept every vertex */
    int32_t wave_levels;    /* top-down Evaluate levels, summed over Evaluate calls */
    int32_t jump_evaluates; /* Evaluate calls done (or finished) by pointer jumping */
    float ms_exploit;       /* device time of the call, CUDA events on the graph's stream */
    int32_t graph_launch;   /* 1 if the loop ran as one CUDA-graph launch */
    int64_t improve_entries; /* adjacency entries scanned by Improve alone (the relaxations of
                               a pull-only Improve); the same for every run of the same input */
    int64_t offers;         /* candidates formed by Evaluate for the next Improve (tile 0):
                               relaxations = improve_entries + offers.  A vertex that Evaluate
                               lowers twice (its new parent was switched in the same round and
                               not yet lowered when it was read) forms its candidates twice,
                               so this count can differ by a fraction of a percent between
                               runs of the same input; the results do not. */
} pirrt_exploit_stats;

typedef struct pirrt_graph pirrt_graph;   /* opaque, library-owned */

/* Allocate an empty graph (no vertices) with the given capacities on
 * cfg->device.  Device memory: a CSR pool of (8 or 16 B) x (4 x max_edges +
 * 4 x max_vertices) entries -- every row keeps room to grow in place, and a
 * row that outgrows it moves to the end of the pool, so an insertion copies
 * only the rows that moved; a second pool of the same size is allocated the
 * first time the pool is used up and every row is repacked -- plus 16 B of
 * row extent and about 130 B per vertex of
 * policy and work arrays.  *out is set to NULL on failure. */
pirrt_status pirrt_graph_create(const pirrt_config *cfg, pirrt_graph **out);

/* Free every allocation of the handle (NULL is ignored). */
void pirrt_graph_destroy(pirrt_graph *g);

/* Drop every vertex and edge, keeping the allocations. */
pirrt_status pirrt_graph_reset(pirrt_graph *g);

/* Batched-Extension insertion (Alg. 3 "repeat S times: Extend"; Sec. IV-A:
 * new edges arrive as a coordinate list and are merged into the device CSR
 * once per Replan).  Appends n_new_vertices vertices (ids n .. n+n_new-1;
 * g = +inf and no parent, except g(root) = 0) and n_edges undirected edges
 * src[e] -- dst[e] with cost[e] (float or double per cost_dtype).  Endpoints
 * may be old or new vertices.  The new vertices and the endpoints of the
 * new edges seed the next exploit's Improve frontier, and each new edge
 * offers both endpoints their candidate through it.  The new entries go to
 * the tails of their rows; only rows that outgrow their room are moved.
 * Errors: PIRRT_ERR_CAPACITY, PIRRT_ERR_BAD_INPUT (ids outside
 * [0, n + n_new), src == dst, cost <= 0, NaN or Inf), PIRRT_ERR_OOM (the
 * second CSR pool could not be allocated); on error the graph is unchanged.
 * Synchronises the stream once to read the validation result and the pool
 * space the block needs (and once more when the pool is repacked). */
pirrt_status pirrt_graph_insert_batch(pirrt_graph *g, int64_t n_new_vertices, int64_t n_edges,
                                      const int32_t *src, const int32_t *dst, const void *cost,
                                      int on_device);

/* Goal-directed Replan (Sec. IV-C; the promising set B of Sec. III and the
 * vertex properties h and b of Sec. IV-A).  goal = x_goal (a vertex id below
 * the capacity, inserted already or later), or -1 to return to the
 * goal-free form.  h[v], v < n_h, is a heuristic cost-to-go from v to
 * x_goal (host memory, FP32, finite and >= 0; vertices from n_h on get 0);
 * it must be admissible -- no larger than the cost of any path from v to
 * x_goal -- for g(x_goal) to stay optimal, and consistent (h(u) <= c(u, v) +
 * h(v) on every edge) for the promising set below to be exact.
 *
 * With a goal, a vertex is promising when g(v) + h(v) < g(x_goal), g(x_goal)
 * taken as each Replan iteration begins.  Improve switches v only if the new
 * value makes v promising; the top-down Evaluate lowers g of every child it
 * reaches but expands (scans the row of, lowers the children of) only
 * promising vertices, so g below a vertex that is not promising may stay
 * above the cost of its policy path.  At a stable policy g(x_goal) is the
 * shortest-path cost, and so is g(v) of every v with d(v) + h(v) <
 * d(x_goal) (d = shortest-path cost) when h is consistent.  Pointer-jumping
 * Evaluates (deep trees, PIRRT_EVAL_JUMP) and the barrier-free walk do not
 * prune; they only do more work.
 *
 * Changing the goal or h after a goal-directed exploit makes the next exploit
 * first evaluate the whole tree and sweep every vertex (like set_policy).
 * pirrt_graph_save evaluates the whole tree first.  The goal and h are not
 * part of a checkpoint; they survive pirrt_graph_reset and _load.  h takes
 * 4 bytes per vertex of capacity, allocated on the first call with a goal.
 * Synchronises the stream.  Errors: PIRRT_ERR_INVALID_ARG (goal or n_h out of
 * range, NULL h with n_h > 0), PIRRT_ERR_BAD_INPUT (negative, NaN or infinite
 * h), PIRRT_ERR_OOM. */
pirrt_status pirrt_graph_set_goal(pirrt_graph *g, int32_t goal, const float *h, int64_t n_h);

/* Start copying the next block's host edge list to the device on a copy
 * stream of the graph, so that the copy overlaps the current exploit (the
 * paper's future work, Sec. VII, overlaps exploration with exploitation).
 * The next pirrt_graph_insert_batch called with the same host pointers and
 * edge count (on_device = 0) uses the copy instead of copying again; any
 * other call discards it (waiting for its copies to end).  The caller keeps
 * the three host buffers alive and unchanged until the next
 * pirrt_graph_insert_batch or pirrt_graph_prefetch_batch call on the graph
 * returns, or the graph is destroyed; with pageable (not page-locked) memory
 * the copy may not overlap.  Errors: PIRRT_ERR_INVALID_ARG,
 * PIRRT_ERR_OOM, PIRRT_ERR_CUDA. */
pirrt_status pirrt_graph_prefetch_batch(pirrt_graph *g, int64_t n_edges, const int32_t *src,
                                        const int32_t *dst, const void *cost);

/* Replace the policy: parent[v] for v in [0, n) (-1 = none; parent[root]
 * must be -1), n = current vertex count.  Each parent edge must exist; its
 * cost is the cheapest parallel edge.  Evaluates g under the new policy
 * (Alg. 2 Evaluate) and makes the next Improve sweep every vertex.
 * Errors: PIRRT_ERR_INVALID_ARG (n mismatch), PIRRT_ERR_BAD_INPUT,
 * PIRRT_ERR_BAD_TREE (the parents contain a cycle). */
pirrt_status pirrt_graph_set_policy(pirrt_graph *g, const int32_t *parent, int64_t n,
                                    int on_device);

/* Replan (Alg. 2): loop { Improve; stop if no parent switched (Delta g <=
 * eps); Evaluate }.  Improve is a Jacobi sweep: each vertex v != root takes
 * the lexicographic minimum over its neighbours u of (g(u) + c(u, v), u)
 * and switches to it only if that value is strictly below g(p(v)) +
 * c(p(v), v) computed the same way, so a current parent attaining the
 * minimum is kept and otherwise the lowest id wins.  Only vertices with a
 * neighbour whose g changed (or seeded by insertion) are re-examined.
 * Evaluate recomputes g(v) = g(p(v)) + c(p(v), v) in FP64 below the
 * switched vertices, by default top-down level by level (the wave of
 * PIRRT_EVAL_WAVE), handing over to pointer jumping when a wave passes its
 * level cap (PIRRT_EVAL_AUTO); see the Evaluate strategies above.  Blocks
 * until done; stats may be NULL.
 * Errors: PIRRT_ERR_NOT_CONVERGED (max_iters reached; the state stays
 * consistent and exploit may be called again), PIRRT_ERR_BAD_TREE,
 * PIRRT_ERR_DEVICE_TIMEOUT, PIRRT_ERR_CUDA. */
pirrt_status pirrt_graph_exploit(pirrt_graph *g, const pirrt_exploit_opts *opts,
                                 pirrt_exploit_stats *stats);

/* Copy g (FP64, +inf for vertices not connected to the root) into g_out[0..n),
 * n = current vertex count.  Synchronises the stream. */
pirrt_status pirrt_graph_get_costs(const pirrt_graph *g, double *g_out, int64_t n, int on_device);

/* Copy the parents (-1 for the root and for unreached vertices) into
 * p_out[0..n), n = current vertex count.  This is the tree E' = {pi(v)} that
 * Alg. 1 and Alg. 3 output.  Synchronises the stream. */
pirrt_status pirrt_graph_get_parents(const pirrt_graph *g, int32_t *p_out, int64_t n,
                                     int on_device);

/* Copy the device CSR, packed: row_off[0..n] (int64), col[0..m) (int32) and
 * cost[0..m) (float or double), m = pirrt_graph_num_entries().  Entries of
 * a row are in no particular order.  Any output pointer may be NULL. */
pirrt_status pirrt_graph_get_adjacency(const pirrt_graph *g, int64_t *row_off, int32_t *col,
                                       void *cost, int on_device);

/* Checkpoint and resume (not in the paper; it keeps an expensive roadmap and
 * its converged policy across processes).  pirrt_graph_save writes the graph
 * to `path` (a file the caller names; overwritten): the CSR packed row by row,
 * g, the parents and their edge costs, with the cost type and root in a
 * header.  pirrt_graph_load replaces the contents of `g` with a saved graph
 * of the same cost type and root that fits its capacities; the next exploit
 * then starts with a sweep of every vertex (no frontier is saved), so an
 * exploit right after a load of a converged graph converges in one Improve,
 * and later insertions and exploits give the results the saved graph would
 * have given.  Both synchronise the graph's stream.
 * Errors: PIRRT_ERR_INVALID_ARG (NULL pointer, file that cannot be opened or
 * written, other cost type or root), PIRRT_ERR_CAPACITY, PIRRT_ERR_BAD_INPUT
 * (not a checkpoint, truncated or inconsistent); on a load error before the
 * contents are replaced the graph is unchanged. */
pirrt_status pirrt_graph_save(const pirrt_graph *g, const char *path);
pirrt_status pirrt_graph_load(pirrt_graph *g, const char *path);

/* Per-kernel accounting of one handle (tracing).  Launch counts are always
 * kept; device times are measured with CUDA events on the handle's stream
 * only while profiling is enabled.  Work units let a caller turn times into
 * bandwidth: Improve scanned `improve_entries` CSR entries over
 * `improve_vertices` vertices (of which `improve_dense_vertices` in dense
 * sweeps) and switched `improve_switches` parents; Evaluate finished
 * `evaluate_vertices` vertices in `evaluate_visits` work-list visits;
 * insertion wrote `insert_new_entries` new CSR entries and moved
 * `insert_copied_entries` old ones (rows that outgrew their room, repacks). */
typedef struct {
    int64_t launches;             /* every kernel launch of this handle */
    int64_t improve_launches, evaluate_launches, mark_launches, insert_calls;
    double improve_ms, evaluate_ms, mark_ms, insert_ms;
    int64_t improve_entries, improve_vertices, improve_dense_vertices, improve_switches;
    int64_t evaluate_vertices, evaluate_visits, mark_vertices;
    int64_t insert_new_entries, insert_copied_entries;
    int64_t evaluate_offers;  /* candidates offered by Evaluate to the next Improve (tile 0) */
    /* Level trace of the top-down Evaluate (wave launches while profiling):
     * bucket b counts the levels of 2^(b-1) .. 2^b - 1 vertices (the last
     * bucket every larger one), the vertices they held, and the SM cycles of
     * one CTA from each level's start to the next level's start (so the level's
     * grid barrier is included).  wave_pre_cycles: the cycles of a wave launch
     * before its first level (Improve from offers and its barrier);
     * wave_post_cycles: after its last level; wave_jump_cycles: in the
     * pointer-jumping finish after a level cap; wave_calls: the launches
     * traced.  Cycles are of the SM clock; divide by it for time. */
    int64_t level_count[24], level_vertices[24], level_cycles[24];
    int64_t wave_pre_cycles, wave_post_cycles, wave_jump_cycles, wave_calls;
    /* The same CTA's own tiles of up to 512 vertices, by tile size (same
     * buckets): its share of a grid step, and the tree levels it walked on its
     * own from the children it lowered. */
    int64_t share_tiles[24], share_vertices[24], share_cycles[24];
    int64_t local_tiles[24], local_vertices[24], local_cycles[24];
    /* Wave launches on the global timer, in ns: from the start of CTA 0 to
     * the end of the iteration (wave_span_ns over wave_spans launches), and
     * from the end of one launch to the start of the next within an exploit
     * (wave_gap_ns over wave_gaps: the kernels in between and the launch
     * latency). */
    int64_t wave_span_ns, wave_spans, wave_gap_ns, wave_gaps;
} pirrt_profile;

/* Clear the profile and turn event timing on (enable = 1) or off (0).
 * enable = 2 keeps only the device-side wave trace (the level_*, share_*,
 * local_* and wave_* fields) and leaves every exploit a single CUDA-graph
 * launch, with no host loop and no events. */
pirrt_status pirrt_graph_set_profiling(pirrt_graph *g, int enable);

/* Copy the profile accumulated since the last pirrt_graph_set_profiling
 * (synchronises the graph's stream to read the device-side level trace). */
pirrt_status pirrt_graph_get_profile(const pirrt_graph *g, pirrt_profile *out);

/* One Replan iteration as seen while profiling is enabled (tracing). */
typedef struct {
    int32_t iteration;        /* index within its exploit call */
    int32_t dense;            /* 1 if Improve swept every vertex */
    int64_t improve_vertices; /* vertices Improve processed */
    int64_t improve_entries;  /* CSR entries Improve scanned */
    int32_t switches;         /* parents switched */
    int32_t changed;          /* vertices whose g changed in Evaluate */
    int32_t wave_levels;      /* top-down Evaluate levels (0 for pointer jumping) */
    int32_t next_frontier;    /* size of the next Improve list (0 if the next sweep is dense) */
    float improve_ms, evaluate_ms, mark_ms, iteration_ms;  /* CUDA-event times */
    int64_t offers;           /* candidates offered by this iteration's Evaluate */
} pirrt_trace_record;

/* Copy up to cap trace records (oldest first) recorded since the last
 * pirrt_graph_set_profiling; returns how many exist (may exceed cap), or -1
 * for a NULL handle. */
int64_t pirrt_graph_get_trace(const pirrt_graph *g, pirrt_trace_record *out, int64_t cap);

/* Evaluate that allocates nothing.  The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc when they need g -- a
 * real-time planning loop that fixes all of its memory at start-up and must
 * not stall on, or fail in, the allocator in the middle of a control cycle.
 * It computes g(v) = g(parent(v)) + parent_cost[v] from the root by the same
 * pointer-jumping kernel as the graph handle, FP64 throughout:
 *   n            vertex count, at most 262,144 (PIRRT_ERR_CAPACITY beyond)
 *   root         vertex with g = 0 (its parent entry is ignored)
 *   parent       device int32[n]: parent id in [0, n), or -1 for unreached
 *   parent_cost  device double[n]: cost of the edge (parent[v], v), finite
 *                and >= 0 wherever parent[v] != -1
 *   g_out        device double[n], written: +inf where the chain does not
 *                reach the root
 *   stream       cudaStream_t (NULL = legacy default stream)
 * The caller owns all four arrays.  The policy is checked on the device
 * before the evaluation follows it: a parent id outside [0, n) other than -1,
 * or a bad cost, gives PIRRT_ERR_BAD_INPUT with g_out holding only the
 * initial values (0 at the root, +inf elsewhere).  Scratch lives in one
 * file-scope device array of about 11.5 MB that every GPU loading the library
 * holds until the process exits.  The first call on a device (with that
 * device current) resolves the array's device address and the launch shape.
 * Every call shares the array and clears what it needs, so calls that
 * overlap on the GPU (other streams, other host threads) race: serialise
 * them.  The call reads its status word back and synchronises the stream
 * before it returns.  Errors: PIRRT_ERR_INVALID_ARG, PIRRT_ERR_CAPACITY,
 * PIRRT_ERR_BAD_INPUT, PIRRT_ERR_BAD_TREE (a cycle: the pointer-jumping round
 * limit ends the kernel), PIRRT_ERR_DEVICE_TIMEOUT, PIRRT_ERR_CUDA. */
pirrt_status pirrt_evaluate_noalloc(int64_t n, int32_t root, const int32_t *parent,
                                    const double *parent_cost, double *g_out, void *stream);

/* Failure detection self-test (the paper has no counterpart: its planner has
 * no device-side waits that could stall).  Every wait in the exploitation
 * kernels is bounded and ends in a status bit instead of a hang; this runs
 * one such wait where nothing will ever end it, under a short limit:
 *   which = PIRRT_SELFTEST_GRID_BARRIER: the grid barrier of the cooperative
 *           kernels, in a grid of two CTAs one of which leaves without
 *           arriving; limit = polls, 1 .. 2^20 (each about 0.1 to 1 us);
 *   which = PIRRT_SELFTEST_MBARRIER: the mbarrier wait of the staged Improve
 *           on a barrier that nothing arrives at; limit = nanoseconds of the
 *           global timer, 1 .. 10^9.
 * The kernel's status word is read back and mapped as after an exploit, so a
 * correct build returns PIRRT_ERR_DEVICE_TIMEOUT and leaves the device usable
 * (no fault, no trap).  Runs on the current device and `stream` (NULL =
 * legacy default stream) and synchronises it.  Errors: PIRRT_ERR_INVALID_ARG
 * (which or limit out of range), PIRRT_ERR_CUDA. */
enum { PIRRT_SELFTEST_GRID_BARRIER = 0, PIRRT_SELFTEST_MBARRIER = 1 };
pirrt_status pirrt_selftest_wait(int32_t which, int64_t limit, void *stream);

/* ------------------------------------------------------------------------
 * Batched form: many independent planning graphs exploited together.
 *
 * The batch is one device graph made of the disjoint union of its members:
 * member b owns the vertex ids [base_b, base_b + max_vertices[b]) and its
 * own root.  Policy iteration on the union is policy iteration on every
 * member at once (no edge joins two members), so every member reaches
 * exactly the policy of its own Replan, bit for bit; the whole batch runs in
 * one CUDA-graph launch per exploit.  Inserts are staged per member and
 * merged into the device CSR in one pass at the next exploit (Sec. IV-A:
 * one CSR rebuild per Replan).
 * ------------------------------------------------------------------------ */
typedef struct pirrt_batch pirrt_batch;   /* opaque, library-owned */

/* n_graphs members; max_vertices[b] and max_edges[b] are member b's
 * capacities, roots[b] its x_init (a member-local id).  Every member starts
 * with its full vertex capacity present and isolated (g = +inf) except its
 * root (g = 0).  Errors: PIRRT_ERR_INVALID_ARG, PIRRT_ERR_OOM, PIRRT_ERR_CUDA. */
pirrt_status pirrt_batch_create(int32_t n_graphs, const int64_t *max_vertices,
                                const int64_t *max_edges, const int32_t *roots,
                                int32_t cost_dtype, int32_t device, void *stream,
                                pirrt_batch **out);

void pirrt_batch_destroy(pirrt_batch *b);

/* Back to the state right after create (every member isolated, roots at
 * g = 0, nothing staged), keeping the allocations. */
pirrt_status pirrt_batch_reset(pirrt_batch *b);

/* Stage n_edges undirected edges of member `graph` in member-local ids (each
 * in [0, max_vertices[graph])); they join the device CSR at the next
 * exploit.  Errors: PIRRT_ERR_INVALID_ARG, PIRRT_ERR_CAPACITY,
 * PIRRT_ERR_BAD_INPUT (an id out of range; nothing is staged). */
pirrt_status pirrt_batch_insert(pirrt_batch *b, int32_t graph, int64_t n_edges,
                                const int32_t *src, const int32_t *dst, const void *cost,
                                int on_device);

/* Merge the staged edges, then Replan every member to convergence (see
 * pirrt_graph_exploit; the options and totals refer to the whole batch). */
pirrt_status pirrt_batch_exploit(pirrt_batch *b, const pirrt_exploit_opts *opts,
                                 pirrt_exploit_stats *stats);

/* Autotuner: merge the staged edges, then time pirrt_batch_exploit for each
 * of n candidate option sets from the same starting state (the device state
 * is restored after each trial) and return the fastest in *best (its index
 * in *best_index, its time in *best_ms).  The batch is left as it was
 * before the call. */
pirrt_status pirrt_batch_autotune(pirrt_batch *b, const pirrt_exploit_opts *candidates,
                                  int32_t n, pirrt_exploit_opts *best, int32_t *best_index,
                                  float *best_ms);

/* Searching autotuner: the same trials (same starting state, restored after
 * each), chosen by coordinate descent from `start` (NULL = the defaults) over
 * the Improve kernel (tile 0 or 2) and its lanes per vertex, the dense-sweep
 * fraction (0.1 .. 0.8), the Evaluate mode (AUTO or WAVE), the wave's CTAs
 * per SM, its CTA-local walk (levels, list size, step size) and its one-CTA
 * tail: each option in turn takes each of its values with the others held,
 * and keeps a value that is more than 1% faster; passes repeat until one
 * changes nothing or max_trials (>= 1) exploits have run.  Returns the
 * fastest set in *best (with every tuned field written out), its time in
 * *best_ms and the trials run in *trials (either may be NULL).  The batch is
 * left as it was before the call.  Errors: PIRRT_ERR_INVALID_ARG, and those of
 * pirrt_batch_exploit. */
pirrt_status pirrt_batch_autotune_search(pirrt_batch *b, const pirrt_exploit_opts *start,
                                         int32_t max_trials, pirrt_exploit_opts *best,
                                         float *best_ms, int32_t *trials);

/* Member `graph`'s g / parents (member-local ids, -1 for the root and for
 * unreached vertices) for its first n vertices (n <= max_vertices[graph]). */
pirrt_status pirrt_batch_get_costs(const pirrt_batch *b, int32_t graph, double *g_out, int64_t n,
                                   int on_device);
pirrt_status pirrt_batch_get_parents(const pirrt_batch *b, int32_t graph, int32_t *p_out,
                                     int64_t n, int on_device);

/* The union graph (for profiling and tracing calls). */
pirrt_graph *pirrt_batch_graph(pirrt_batch *b);

/* ------------------------------------------------------------------------
 * Learned sampling proposal (an addition on top of the method; the paper
 * samples uniformly).  A 3-layer MLP maps a scene's 64 x 64 occupancy grid
 * (4096 values in {0, 1}) and 8-D Gaussian noise to a sample position in
 * [0, 1]^2:
 *   a1 = W1g grid + W1n z + b1, h1 = relu(a1); a2 = W2 h1 + b2, h2 = relu(a2);
 *   y = sigmoid(W3 h2 + b3).
 * BF16 weights and layer inputs on the tensor cores with FP32 accumulation,
 * FP32 master weights trained by Adam.  The forward pass of forward, sample,
 * imle_select and of train_step's K draws per target runs by default as one
 * fused tcgen05 kernel (all three contractions with TMEM accumulators, the
 * activations kept on chip, 128 rows per tile); the layer-by-layer path
 * (mma.sync GEMMs, activations in HBM) computes the backward pass and can be
 * selected for the forward pass too (pirrt_proposal_set_options).  Training is implicit maximum-
 * likelihood estimation: for each target sample, K noise draws go through the
 * network and only the draw nearest the target is pulled towards it.
 * Parameters are packed FP32 in the order W1g [256 x 4096], W1n [256 x 8],
 * b1 [256], W2 [256 x 256], b2 [256], W3 [2 x 256], b3 [2].
 * All array arguments are device pointers; noise is supplied by the caller.
 * ------------------------------------------------------------------------ */
typedef struct pirrt_proposal pirrt_proposal;

/* Forward kernels for pirrt_proposal_set_options. */
enum { PIRRT_MLP_FORWARD_TCGEN05 = 0, PIRRT_MLP_FORWARD_LAYERED = 1 };

/* Number of packed parameters (1,117,186). */
int64_t pirrt_proposal_num_params(void);

/* Working space for up to max_scenes scenes and max_rows sample rows per call;
 * He-uniform initial weights from `seed`. */
pirrt_status pirrt_proposal_create(int32_t max_scenes, int32_t max_rows, uint64_t seed,
                                   int32_t device, void *stream, pirrt_proposal **out);
void pirrt_proposal_destroy(pirrt_proposal *p);

/* forward_kernel: PIRRT_MLP_FORWARD_TCGEN05 (default) or
 * PIRRT_MLP_FORWARD_LAYERED for the forward passes listed above;
 * keep_activations != 0: every later forward pass also leaves h1 and h2 (BF16)
 * of its rows for pirrt_proposal_get_activations (a diagnostic; the fused
 * kernel then writes them to HBM).  PIRRT_ERR_INVALID_ARG for an unknown
 * kernel. */
pirrt_status pirrt_proposal_set_options(pirrt_proposal *p, int32_t forward_kernel,
                                        int32_t keep_activations);

/* Device time (CUDA events on the handle's stream) of the last fused forward
 * kernel launch, in ms; PIRRT_ERR_INVALID_ARG before the first one. */
pirrt_status pirrt_proposal_kernel_ms(const pirrt_proposal *p, float *ms);

/* Copy h1 and h2 ([rows x 256] BF16 bit patterns, row-major) of the last
 * forward pass into device buffers h1_out / h2_out (either may be NULL).
 * Needs keep_activations for the fused kernel; rows must not exceed the rows
 * of that pass (PIRRT_ERR_INVALID_ARG). */
pirrt_status pirrt_proposal_get_activations(const pirrt_proposal *p, int32_t rows,
                                            uint16_t *h1_out, uint16_t *h2_out);

/* Replace / read the FP32 master weights (n = num_params); set clears the
 * Adam state and the accumulated gradient. */
pirrt_status pirrt_proposal_set_weights(pirrt_proposal *p, const float *w, int64_t n);
pirrt_status pirrt_proposal_get_weights(const pirrt_proposal *p, float *w, int64_t n);

/* Samples: out_xy[r] = network(grids[scene[r]], noise[r]) for r < rows.
 * grids: [n_scenes x 4096] FP32 0/1; scene: int32[rows], each in
 * [0, n_scenes); noise: [rows x 8], 16-byte aligned; out_xy: [rows x 2],
 * 8-byte aligned.  A scene index out of range gives PIRRT_ERR_BAD_INPUT (the
 * row is computed for scene 0); a tensor-core wait that expires gives
 * PIRRT_ERR_DEVICE_TIMEOUT.  The same rules hold for sample, imle_select and
 * train_step. */
pirrt_status pirrt_proposal_forward(pirrt_proposal *p, int32_t n_scenes, const float *grids,
                                    int32_t rows, const int32_t *scene, const float *noise,
                                    float *out_xy);

/* Sampling distribution of the planner with the proposal: row r is the
 * network's output for (grids[scene[r]], noise[r]) when coin[r] <
 * learned_fraction, else uniform_xy[r] (a 50/50 mixture at 0.5).  The caller
 * draws noise [rows x 8] ~ N(0, I), uniform_xy [rows x 2] ~ U[0,1]^2 and
 * coin [rows] ~ U[0,1); out_xy: [rows x 2].  Samples inside obstacles are
 * the caller's to reject, as for uniform sampling. */
pirrt_status pirrt_proposal_sample(pirrt_proposal *p, int32_t n_scenes, const float *grids,
                                   int32_t rows, const int32_t *scene, const float *noise,
                                   const float *uniform_xy, const float *coin,
                                   float learned_fraction, float *out_xy);

/* IMLE draw selection: rows t*K .. t*K+K-1 (scene draw_scene[row], noise
 * noise[row]) belong to target t; pick[t] = the draw whose output is nearest
 * targets[t] (lowest index on ties). */
pirrt_status pirrt_proposal_imle_select(pirrt_proposal *p, int32_t n_scenes, const float *grids,
                                        int32_t n_targets, const int32_t *draw_scene,
                                        const float *targets, int32_t K, const float *noise,
                                        int32_t *pick);

/* Accumulate the gradient of mean_r |y_r - targets_r|^2 over `rows` rows into
 * the internal gradient; *loss_out (host, may be NULL) gets the loss. */
pirrt_status pirrt_proposal_backward(pirrt_proposal *p, int32_t n_scenes, const float *grids,
                                     int32_t rows, const int32_t *scene, const float *noise,
                                     const float *targets, float *loss_out);

/* Read / clear the accumulated gradient (n = num_params). */
pirrt_status pirrt_proposal_get_grads(const pirrt_proposal *p, float *g, int64_t n);
pirrt_status pirrt_proposal_zero_grads(pirrt_proposal *p);

/* One Adam step on the accumulated gradient, which is then cleared. */
pirrt_status pirrt_proposal_adam(pirrt_proposal *p, float lr, float beta1, float beta2, float eps);

/* One IMLE training step: K draws per target (noise: [n_targets * K x 8],
 * target t owns rows t*K .. t*K+K-1, all in scene target_scene[t]), the
 * nearest draw of each target is pulled towards it (squared error, mean over
 * targets), then Adam (beta1 0.9, beta2 0.999, eps 1e-8) with rate lr.
 * *loss_out (host, may be NULL) gets the loss before the step.
 * n_targets * K must not exceed max_rows. */
pirrt_status pirrt_proposal_train_step(pirrt_proposal *p, int32_t n_scenes, const float *grids,
                                       int32_t n_targets, const int32_t *target_scene,
                                       const float *targets, int32_t K, const float *noise,
                                       float lr, float *loss_out);

/* Current vertex count, or -1 for a NULL handle. */
int64_t pirrt_graph_num_vertices(const pirrt_graph *g);

/* Current number of directed CSR entries (2 per undirected edge), or -1. */
int64_t pirrt_graph_num_entries(const pirrt_graph *g);

/* Detail of the last error on this handle ("" if none). */
const char *pirrt_graph_last_error(const pirrt_graph *g);

/* Static name of a status code. */
const char *pirrt_status_string(pirrt_status s);

#ifdef __cplusplus
}
#endif

#endif /* PIRRT_H */
