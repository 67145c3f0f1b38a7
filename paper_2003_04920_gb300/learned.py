"""Learned sampling proposal trained on the planner's own solutions, and the
paired comparison against uniform sampling.

This sits on top of the method (the paper samples uniformly).  The scenes are
the unit square with 200 circles (r ~ U[0.01, 0.04]), x_init = (0.05, 0.05) as
vertex 0 and x_goal = (0.95, 0.95) as vertex 1; the planner's answer for a
scene is the start-goal cost g(x_goal) of the shortest-path tree its
exploitation converges to (Alg. 2 run to a stable policy, Sec. IV).

Training data: per training scene, N free uniform samples plus x_init and
x_goal form a symmetrised k-NN roadmap (k = ceil(2e ln N)); the planner solves
it on the GPU (all roadmaps of a chunk in one pirrt_batch); every sample
within ``band`` of the start-goal path is a target.  A scene whose goal is
unreached is dropped.

Training: implicit maximum-likelihood estimation, one pirrt_proposal_train_step
per batch of targets (K noise draws per target, the nearest draw is pulled
towards it, Adam).

Evaluation: on held-out scenes and for each sample count N, the planner's
g(x_goal) with N free samples drawn 50/50 from the proposal and uniformly
(samples inside an obstacle are rejected and redrawn, as for uniform
sampling) against N uniform free samples, paired by scene and seed.

Roadmap construction (k-NN, collision checks) is host work in a process pool;
solving, the network and its training run in the library's CUDA kernels.
"""
from __future__ import annotations

import math
import os
import time

import numpy as np

from . import workloads as W

X_INIT = np.array(W.C5_X_INIT)
X_GOAL = np.array(W.C5_X_GOAL)
GOAL = 1


# ----------------------------------------------------------------------------
# host side: scenes, samples, roadmaps

def _worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"


def pool(workers: int):
    """Process pool for roadmap construction (spawned, so it holds no CUDA
    state of the parent)."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(max(1, int(workers)), initializer=_worker_init)


def uniform_points(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """x_init, x_goal and n - 2 free uniform samples of scene ``seed``."""
    sc = W.c5_scene(seed)
    rng = np.random.default_rng([int(seed), int(n), int(stream)])
    return np.vstack([X_INIT[None], X_GOAL[None], W.free_uniform(rng, sc, n - 2)])


def _roadmap_job(job):
    seed, pts = job
    if isinstance(pts, tuple):  # ("uniform", n, stream): generate in the worker
        pts = uniform_points(seed, pts[1], pts[2])
    rm = W.roadmap_from_points(f"c5-{seed}", pts, W.c5_scene(seed))
    return rm.u, rm.v, rm.cost, rm.n, rm.points


def roadmaps(jobs, workers: int = 1, pool_=None):
    """Roadmaps (u, v, cost, n, points) for jobs (seed, points or
    ("uniform", n, stream))."""
    if pool_ is not None:
        return pool_.map(_roadmap_job, jobs, chunksize=1)
    if workers > 1:
        with pool(workers) as p:
            return p.map(_roadmap_job, jobs, chunksize=1)
    return [_roadmap_job(j) for j in jobs]


def path_to_root(parent: np.ndarray, v: int) -> np.ndarray:
    """Vertices from v up to the root along the parent tree (-1 ends)."""
    out = [v]
    for _ in range(len(parent)):
        v = int(parent[v])
        if v < 0:
            break
        out.append(v)
    return np.asarray(out, dtype=np.int64)


def near_path(points: np.ndarray, path_pts: np.ndarray, band: float) -> np.ndarray:
    """Mask of points whose distance to the polyline ``path_pts`` is at most
    ``band``."""
    best = np.full(len(points), np.inf)
    for a, b in zip(path_pts[:-1], path_pts[1:]):
        ab = b - a
        L2 = float(ab @ ab)
        t = np.zeros(len(points)) if L2 == 0.0 else np.clip((points - a) @ ab / L2, 0.0, 1.0)
        d2 = np.sum((a + t[:, None] * ab - points) ** 2, axis=1)
        np.minimum(best, d2, out=best)
    return best <= band * band


# ----------------------------------------------------------------------------
# GPU side: planner and proposal

def solve(graphs, max_entries: int = 300_000_000, device: int = 0):
    """Converged g and parents for each roadmap (u, v, cost, n, ...), solved in
    chunks of one pirrt_batch each (at most ``max_entries`` undirected edges
    per chunk)."""
    from . import Batch
    out, i = [], 0
    while i < len(graphs):
        j, tot = i, 0
        while j < len(graphs) and (j == i or tot + len(graphs[j][0]) <= max_entries):
            tot += len(graphs[j][0])
            j += 1
        chunk = graphs[i:j]
        with Batch([c[3] for c in chunk], [len(c[0]) + 8 for c in chunk], device=device) as b:
            for k, c in enumerate(chunk):
                b.insert(k, c[0], c[1], c[2])
            b.exploit()
            for k, c in enumerate(chunk):
                out.append((b.get_costs(k, c[3]), b.get_parents(k, c[3])))
        i = j
    return out


def training_set(seeds, n: int, band: float = 0.02, workers: int = 1, pool_=None,
                 device: int = 0, chunk: int = 64):
    """(grids [S x 4096] float32, targets list of [T_s x 2] float32, costs,
    kept seeds) for the training scenes with a start-goal path."""
    grids, targets, costs, kept = [], [], [], []
    seeds = list(seeds)
    for c0 in range(0, len(seeds), chunk):
        part = seeds[c0:c0 + chunk]
        rms = roadmaps([(s, ("uniform", n, 0)) for s in part], workers, pool_)
        sols = solve(rms, device=device)
        for s, rm, (g, p) in zip(part, rms, sols):
            if not math.isfinite(g[GOAL]):
                continue
            pts = rm[4]
            mask = near_path(pts, pts[path_to_root(p, GOAL)], band)
            mask[:2] = False
            grids.append(W.occupancy_grid(W.c5_scene(s)))
            targets.append(pts[mask].astype(np.float32))
            costs.append(float(g[GOAL]))
            kept.append(s)
    return np.stack(grids), targets, np.asarray(costs), kept


def train(prop, grids: np.ndarray, targets, steps: int, scenes_per_step: int = 32,
          targets_per_scene: int = 64, K: int = 16, lr: float = 3e-4, seed: int = 0,
          log_every: int = 0):
    """IMLE training of ``prop`` (a Proposal with max_scenes >= scenes_per_step
    and max_rows >= scenes_per_step * targets_per_scene * K); returns the
    per-step losses and the wall time of the steps."""
    import torch
    rng = np.random.default_rng(seed)
    S = len(targets)
    counts = np.array([len(t) for t in targets], dtype=np.int64)
    offs = np.r_[0, np.cumsum(counts)[:-1]]
    gd = torch.from_numpy(np.ascontiguousarray(grids, dtype=np.float32)).cuda()
    tg_all = torch.from_numpy(np.concatenate(targets).astype(np.float32)).cuda()
    T = scenes_per_step * targets_per_scene
    local = torch.arange(scenes_per_step, dtype=torch.int32).repeat_interleave(targets_per_scene)
    local = local.cuda()
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(steps):
        pick = rng.choice(S, scenes_per_step, replace=scenes_per_step > S)
        rows = offs[pick][:, None] + (rng.random((scenes_per_step, targets_per_scene)) *
                                      counts[pick][:, None]).astype(np.int64)
        tg = tg_all[torch.from_numpy(rows.ravel()).cuda()]
        sub = gd[torch.from_numpy(pick).cuda()]
        noise = torch.from_numpy(rng.standard_normal((T * K, 8), dtype=np.float32)).cuda()
        losses.append(prop.train_step(sub, local, tg, K, noise, lr))
        if log_every and (it % log_every == 0 or it == steps - 1):
            print(f"step {it}: loss {losses[-1]:.5f}", flush=True)
    torch.cuda.synchronize()
    return np.asarray(losses), time.perf_counter() - t0


def learned_points(prop, seed: int, n: int, fraction: float = 0.5, stream: int = 0,
                   chunk: int = 65536) -> np.ndarray:
    """x_init, x_goal and n - 2 free samples of scene ``seed`` drawn from the
    mixture (``fraction`` from the proposal, the rest uniform); samples
    inside an obstacle are rejected."""
    import torch
    sc = W.c5_scene(seed)
    grid = torch.from_numpy(W.occupancy_grid(sc)[None]).cuda()
    rng = np.random.default_rng([int(seed), int(n), int(stream), 1])
    chunk = min(int(chunk), prop.max_rows)
    out, have = [], 0
    scene = torch.zeros(chunk, dtype=torch.int32, device="cuda")
    while have < n - 2:
        noise = torch.from_numpy(rng.standard_normal((chunk, 8), dtype=np.float32)).cuda()
        uni = torch.from_numpy(rng.random((chunk, 2), dtype=np.float32)).cuda()
        coin = torch.from_numpy(rng.random(chunk, dtype=np.float32)).cuda()
        xy = prop.sample(grid, scene, noise, uni, coin, fraction).cpu().numpy().astype(np.float64)
        xy = xy[~sc.inside(xy)]
        out.append(xy)
        have += len(xy)
    pts = np.concatenate(out)[:n - 2]
    return np.vstack([X_INIT[None], X_GOAL[None], pts])


def compare(prop, seeds, sizes, fraction: float = 0.5, workers: int = 1, pool_=None,
            device: int = 0, chunk: int = 16):
    """Best start-goal cost per (scene, N) for uniform and mixed sampling:
    dict N -> (uniform costs, mixed costs), +inf where the goal is unreached."""
    res = {}
    seeds = list(seeds)
    for n in sizes:
        cu, cl = [], []
        for c0 in range(0, len(seeds), chunk):
            part = seeds[c0:c0 + chunk]
            jobs = [(s, ("uniform", n, 1)) for s in part]
            jobs += [(s, learned_points(prop, s, n, fraction, 1)) for s in part]
            sols = solve(roadmaps(jobs, workers, pool_), device=device)
            cu += [float(g[GOAL]) for g, _ in sols[:len(part)]]
            cl += [float(g[GOAL]) for g, _ in sols[len(part):]]
        res[int(n)] = (np.asarray(cu), np.asarray(cl))
    return res


def summarize(res) -> dict:
    """Per N: scenes where both arms reach the goal, their mean costs, the
    mean paired difference (mixed - uniform) with its standard error, the
    fraction of scenes where mixed is cheaper, and the success counts."""
    out = {}
    for n, (cu, cl) in res.items():
        both = np.isfinite(cu) & np.isfinite(cl)
        d = cl[both] - cu[both]
        out[n] = dict(scenes=int(len(cu)), both_solved=int(both.sum()),
                      uniform_solved=int(np.isfinite(cu).sum()),
                      mixed_solved=int(np.isfinite(cl).sum()),
                      uniform_mean=float(cu[both].mean()) if both.any() else None,
                      mixed_mean=float(cl[both].mean()) if both.any() else None,
                      paired_diff=float(d.mean()) if both.any() else None,
                      paired_se=float(d.std(ddof=1) / math.sqrt(len(d))) if len(d) > 1 else None,
                      mixed_better=float((d < 0).mean()) if both.any() else None)
    return out


def main(argv=None):
    """Train on planner solutions, then compare mixed and uniform sampling on
    held-out scenes; prints one JSON document."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train-scenes", type=int, default=1000)
    ap.add_argument("--n-train", type=int, default=20_000)
    ap.add_argument("--band", type=float, default=0.02)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--scenes-per-step", type=int, default=32)
    ap.add_argument("--targets-per-scene", type=int, default=64)
    ap.add_argument("--K", type=int, default=16)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--test-scenes", type=int, default=100)
    ap.add_argument("--sizes", default="20000,100000")
    ap.add_argument("--fraction", type=float, default=0.5)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)

    from . import Proposal
    report = dict(config=vars(a))
    with pool(a.workers) as pl:
        t = time.perf_counter()
        train_seeds = range(0, a.train_scenes)
        grids, targets, costs, kept = training_set(train_seeds, a.n_train, a.band, pool_=pl)
        keep = [i for i, t_ in enumerate(targets) if len(t_) > 0]
        grids, targets = grids[keep], [targets[i] for i in keep]
        report["training_set"] = dict(scenes_solved=len(kept), scenes_used=len(keep),
                                      targets=int(sum(len(t_) for t_ in targets)),
                                      mean_cost=float(costs.mean()) if len(costs) else None,
                                      seconds=time.perf_counter() - t)
        print(json.dumps(report["training_set"]), flush=True)
        rows = a.scenes_per_step * a.targets_per_scene * a.K
        prop = Proposal(a.scenes_per_step, rows, seed=a.seed + 1)
        losses, secs = train(prop, grids, targets, a.steps, a.scenes_per_step,
                             a.targets_per_scene, a.K, a.lr, a.seed, log_every=max(1, a.steps // 10))
        report["training"] = dict(steps=a.steps, seconds=secs, ms_per_step=1e3 * secs / max(1, a.steps),
                                  loss_first=float(losses[:20].mean()),
                                  loss_last=float(losses[-20:].mean()))
        print(json.dumps(report["training"]), flush=True)
        prop_eval = Proposal(1, 65536, seed=a.seed + 1)
        w = prop.get_weights()
        prop_eval.set_weights(w)
        prop.close()
        test_seeds = range(1_000_000, 1_000_000 + a.test_scenes)
        t = time.perf_counter()
        res = compare(prop_eval, test_seeds, [int(x) for x in a.sizes.split(",")], a.fraction,
                      pool_=pl)
        report["comparison"] = {str(k): v for k, v in summarize(res).items()}
        report["comparison_seconds"] = time.perf_counter() - t
        prop_eval.close()
    text = json.dumps(report, indent=1)
    print(text)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    main()
