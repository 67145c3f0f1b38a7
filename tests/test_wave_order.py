"""The top-down Evaluate lowers g by an atomic minimum and expands a vertex
whenever its value drops, in whatever order the CTAs reach the work: grid
steps, a CTA's own walks of the children it lowered, or both interleaved.
The argument that this gives Alg. 2's root-to-leaf sums bit for bit -- Improve
only switches to a strictly cheaper parent, so no value ever computed for a
vertex is below its final one, and the final one arrives with its parent's
last drop -- is checked here on the CPU against the oracle's breadth-first
Evaluate, for random policies, random strict switches and random expansion
orders (a plain Python model of the schedule, no CUDA)."""
import numpy as np

import oracle as O


def _random_instance(rng, n):
    # a connected random graph with positive FP32 costs
    pts = rng.random((n, 2))
    edges = set()
    for v in range(1, n):
        edges.add((int(rng.integers(0, v)), v))
    for _ in range(3 * n):
        a, b = rng.integers(0, n, 2)
        if a != b:
            edges.add((int(min(a, b)), int(max(a, b))))
    u = np.array([e[0] for e in edges], np.int32)
    v = np.array([e[1] for e in edges], np.int32)
    cost = (np.linalg.norm(pts[u] - pts[v], axis=1) + 1e-3).astype(np.float32).astype(np.float64)
    adj = [[] for _ in range(n)]
    for a, b, c in zip(u, v, cost):
        adj[a].append((int(b), float(c)))
        adj[b].append((int(a), float(c)))
    return u, v, cost, adj


def _chain_instance(rng, n):
    """A chain 0-1-...-(n-1) of unit FP32 costs with random shortcuts that are
    cheaper than the stretch they skip, and the chain as the old policy: the
    first Improve switches many vertices, one below another, each with a
    subtree below it."""
    edges = {(i, i + 1): 1.0 for i in range(n - 1)}
    for _ in range(n // 3):
        a = int(rng.integers(0, n - 3))
        b = int(rng.integers(a + 2, min(n, a + 12)))
        edges[(a, b)] = float(np.float32(rng.uniform(0.3, 0.9) * (b - a)))
    u = np.array([e[0] for e in edges], np.int32)
    v = np.array([e[1] for e in edges], np.int32)
    cost = np.array(list(edges.values()), np.float64)
    adj = [[] for _ in range(n)]
    for a, b, c in zip(u, v, cost):
        adj[a].append((int(b), float(c)))
        adj[b].append((int(a), float(c)))
    parent = np.arange(-1, n - 1, dtype=np.int64)
    return u, v, cost, adj, parent


def _instances(rng, count):
    """(n, u, v, cost, adj, old parent) for random graphs with a perturbed
    shortest-path tree as the old policy, and for chains with shortcuts."""
    for trial in range(count):
        n = int(rng.integers(20, 120))
        if trial % 2:
            u, v, cost, adj, parent = _chain_instance(rng, n)
        else:
            u, v, cost, adj = _random_instance(rng, n)
            _, p_old = O.dijkstra(n, u, v, cost * rng.uniform(1.0, 1.6, len(cost)))
            parent = p_old.astype(np.int64).copy()
            parent[0] = -1
        yield n, u, v, cost, adj, parent


def _improve(n, adj, parent):
    """Old g from the old policy, then one Jacobi Improve: the new policy and
    the switched vertices."""
    pc = np.zeros(n)
    for w in range(1, n):
        pc[w] = min(c for x, c in adj[w] if x == parent[w])
    g_old = _bfs_evaluate(n, parent, pc)
    new_parent, new_pc, switched = parent.copy(), pc.copy(), []
    for w in range(1, n):
        best = min((g_old[x] + c, x, c) for x, c in adj[w])
        if best[0] < g_old[parent[w]] + pc[w]:
            new_parent[w], new_pc[w] = best[1], best[2]
            switched.append(w)
    return g_old, new_parent, new_pc, switched


def _bfs_evaluate(n, parent, pc):
    """g from the root by a breadth-first walk of the policy tree (Alg. 2's
    Evaluate order: one FP64 addition per tree edge, root to leaf)."""
    children = [[] for _ in range(n)]
    for w in range(1, n):
        if parent[w] >= 0:
            children[parent[w]].append(w)
    g = np.full(n, np.inf)
    g[0] = 0.0
    queue = [0]
    for x in queue:
        for w in children[x]:
            g[w] = g[x] + pc[w]
            queue.append(w)
    return g


def _wave(n, parent, pc, g_old, switched, rng, walk_prob, skip_stale):
    """Atomic-minimum Evaluate under a random schedule: items are taken from a
    shared list in random order, and with probability walk_prob a taken
    item's children are expanded at once by the same worker (a local walk)
    instead of joining the list.  The kernel expands every item with the value
    it carries (skip_stale False); skipping an item whose vertex has since
    dropped further only saves work."""
    children = [[] for _ in range(n)]
    for w in range(1, n):
        if parent[w] >= 0:
            children[parent[w]].append(w)
    g = g_old.copy()
    first = set()
    work = []
    for s in switched:  # step 0: g(s) from the parent's g as read now
        val = g[parent[s]] + pc[s]
        if val < g[s]:
            g[s] = val
            first.add(s)
            work.append((s, val))
    while work:
        k = int(rng.integers(0, len(work)))
        u, x = work.pop(k)
        stack = [(u, x)]
        while stack:
            u, x = stack.pop()
            if skip_stale and x > g[u]:
                continue  # a smaller value of u arrived since: its own item expands it
            for w in children[u]:
                val = x + pc[w]
                if val < g[w]:
                    g[w] = val
                    first.add(w)
                    (stack if rng.random() < walk_prob else work).append((w, val))
    return g, first


def test_any_expansion_order_gives_the_breadth_first_sums():
    rng = np.random.default_rng(7)
    tested = 0
    for trial, (n, u, v, cost, adj, parent) in enumerate(_instances(rng, 40)):
        A = O.CSR(n, u, v, cost)
        g_old, new_parent, new_pc, switched = _improve(n, adj, parent)
        if not switched:
            continue
        g_ref = _bfs_evaluate(n, new_parent, new_pc)
        changed = {int(w) for w in np.nonzero(g_ref != g_old)[0]}
        tested += 1
        for walk, skip in ((0.0, False), (0.5, False), (1.0, False), (0.5, True)):
            for _ in range(5):
                g, first = _wave(n, new_parent, new_pc, g_old, switched, rng, walk, skip)
                # bit for bit: the same FP64 sums as the breadth-first walk
                assert np.array_equal(g.view(np.int64), g_ref.view(np.int64)), trial
                # the set of changed vertices does not depend on the order
                assert first == changed
        assert A.check_tree(new_parent.astype(np.int32))[0] == 0
    assert tested >= 30  # most instances leave switches to make


def test_expanding_a_vertex_only_once_is_caught():
    """The same schedules with each vertex expanded only the first time its g
    drops must break the sums somewhere: when switched vertices lie below one
    another, a vertex drops again after its first expansion, and its subtree
    must follow."""
    rng = np.random.default_rng(11)
    broken = 0
    for n, u, v, cost, adj, parent in _instances(rng, 40):
        g_old, new_parent, new_pc, switched = _improve(n, adj, parent)
        if not switched:
            continue
        g_ref = _bfs_evaluate(n, new_parent, new_pc)
        children = [[] for _ in range(n)]
        for w in range(1, n):
            if new_parent[w] >= 0:
                children[new_parent[w]].append(w)
        g = g_old.copy()
        expanded = set()
        work = []
        for s in switched:
            val = g[new_parent[s]] + new_pc[s]
            if val < g[s]:
                g[s] = val
                work.append((s, val))
        while work:
            x_u, x = work.pop(int(rng.integers(0, len(work))))
            if x_u in expanded:
                continue  # planted: a vertex is expanded once only
            expanded.add(x_u)
            for w in children[x_u]:
                val = x + new_pc[w]
                if val < g[w]:
                    g[w] = val
                    work.append((w, val))
        broken += not np.array_equal(g, g_ref)
    assert broken > 0
