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
          log_every: int = 0, lr_final: float | None = None):
    """IMLE training of ``prop`` (a Proposal with max_scenes >= scenes_per_step
    and max_rows >= scenes_per_step * targets_per_scene * K); the rate falls
    linearly from lr to lr_final (default: constant).  Returns the per-step
    losses and the wall time of the steps."""
    import torch
    rng = np.random.default_rng(seed)
    S = len(targets)
    counts = np.array([len(t) for t in targets], dtype=np.int64)
    offs = np.r_[0, np.cumsum(counts)[:-1]]
    gd = torch.from_numpy(np.ascontiguousarray(grids, dtype=np.float32)).cuda()
    if all(isinstance(t, torch.Tensor) for t in targets):
        tg_all = torch.cat([t.float() for t in targets]).contiguous()
    else:
        tg_all = torch.from_numpy(np.concatenate(targets).astype(np.float32)).cuda()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(int(seed))
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
        noise = torch.randn((T * K, 8), generator=gen, dtype=torch.float32, device="cuda")
        rate = lr if lr_final is None else lr + (lr_final - lr) * it / max(1, steps - 1)
        losses.append(prop.train_step(sub, local, tg, K, noise, rate))
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


# ----------------------------------------------------------------------------
# device-resident pipeline: samples, k-NN and collision checks on the GPU
# generator (workloads.gpu), near-path bands and mixtures in torch, solving in
# the library

def _gg():
    from .workloads import gpu as GG
    GG.build()
    GG.load()
    return GG


def philox_key(*parts) -> int:
    """A 64-bit generator key from integers (seed, N, stream, ...)."""
    return int(np.random.SeedSequence([int(p) for p in parts]).generate_state(1, np.uint64)[0])


class DevScene:
    """A C5 scene with its circles on the device."""

    def __init__(self, seed: int):
        import torch
        self.seed = int(seed)
        self.scene = W.c5_scene(seed)
        self.c = torch.from_numpy(self.scene.centers).cuda()
        self.r2 = torch.from_numpy(self.scene.radii ** 2).cuda()

    def inside(self, xy):
        """Points strictly inside a circle (FP64, as Scene.inside)."""
        import torch
        out = torch.empty(xy.shape[0], dtype=torch.bool, device=xy.device)
        for i in range(0, xy.shape[0], 1 << 16):
            q = xy[i:i + (1 << 16)]
            d2 = ((q[:, None, 0] - self.c[None, :, 0]) ** 2 + (q[:, None, 1] - self.c[None, :, 1]) ** 2)
            out[i:i + (1 << 16)] = (d2 < self.r2[None]).any(dim=1)
        return out


def dev_uniform_points(seed: int, n: int, stream: int = 0):
    """x_init, x_goal and n - 2 free uniform samples of scene `seed` (FP64
    CUDA tensor n x 2), drawn by the GPU generator."""
    import torch
    GG = _gg()
    pts, _ = GG.sample(W.c5_scene(seed), n - 2, philox_key(5, seed, n, stream))
    head = torch.tensor(np.array([X_INIT, X_GOAL]), dtype=torch.float64, device="cuda")
    return torch.cat([head, pts])


def dev_roadmap(points, seed: int):
    """(u, v, cost, n, points) of the k-NN roadmap over device points (k =
    ceil(2e ln N), exact segment-circle test, FP32 costs), on the GPU."""
    GG = _gg()
    n = int(points.shape[0])
    k = min(W.knn_k(n), n - 1)
    nbr = GG.knn(points, 0.0, 1.0, k)
    u, v, c, _ = GG.edges(points, nbr, W.c5_scene(seed), True, 16, np.float32)
    del nbr
    return (u, v, c, n, points)


def dev_near_path(points, path_pts, band: float):
    """Mask of device points within `band` of the polyline path_pts (device)."""
    import torch
    best = torch.full((points.shape[0],), float("inf"), dtype=torch.float64, device=points.device)
    for a, b in zip(path_pts[:-1], path_pts[1:]):
        ab = b - a
        L2 = float(ab @ ab)
        t = torch.zeros_like(best) if L2 == 0.0 else ((points - a) @ ab / L2).clamp(0.0, 1.0)
        d2 = ((a + t[:, None] * ab - points) ** 2).sum(dim=1)
        torch.minimum(best, d2, out=best)
    return best <= band * band


def dev_training_set(seeds, n: int, band: float = 0.02, chunk: int = 32):
    """training_set on the device: (grids [S x 4096] float32 numpy, targets
    list of float32 CUDA tensors [T_s x 2], costs, kept seeds)."""
    import torch
    grids, targets, costs, kept = [], [], [], []
    seeds = list(seeds)
    for c0 in range(0, len(seeds), chunk):
        part = seeds[c0:c0 + chunk]
        rms = [dev_roadmap(dev_uniform_points(s, n, 0), s) for s in part]
        sols = solve(rms)
        for s, rm, (g, p) in zip(part, rms, sols):
            if not math.isfinite(g[GOAL]):
                continue
            pts = rm[4]
            path = torch.from_numpy(path_to_root(p, GOAL)).cuda()
            mask = dev_near_path(pts, pts[path], band)
            mask[:2] = False
            grids.append(W.occupancy_grid(W.c5_scene(s)))
            targets.append(pts[mask].float().contiguous())
            costs.append(float(g[GOAL]))
            kept.append(s)
        del rms, sols
    return (np.stack(grids) if grids else np.zeros((0, 4096), np.float32)), targets, \
        np.asarray(costs), kept


def reference_paths(seeds, n_ref: int, chunk: int = 8):
    """Per scene: (g(x_goal), path points as an FP64 CUDA tensor) of the
    uniform roadmap with n_ref samples (stream 2), or (inf, None)."""
    import torch
    out = {}
    seeds = list(seeds)
    for c0 in range(0, len(seeds), chunk):
        part = seeds[c0:c0 + chunk]
        rms = [dev_roadmap(dev_uniform_points(s, n_ref, 2), s) for s in part]
        for s, rm, (g, p) in zip(part, rms, solve(rms)):
            if math.isfinite(g[GOAL]):
                idx = torch.from_numpy(path_to_root(p, GOAL)[::-1].copy()).cuda()
                out[s] = (float(g[GOAL]), rm[4][idx].contiguous())
            else:
                out[s] = (math.inf, None)
        del rms
    return out


def _polyline_sampler(path_pts, band: float):
    """Draws near a polyline: a point uniform in arc length, then an offset
    uniform in the disc of radius `band`."""
    import torch
    seg = path_pts[1:] - path_pts[:-1]
    lens = torch.sqrt((seg ** 2).sum(dim=1))
    cum = torch.cat([torch.zeros(1, dtype=lens.dtype, device=lens.device), torch.cumsum(lens, 0)])
    total = float(cum[-1])

    def draw(m, gen):
        s = torch.rand(m, generator=gen, dtype=torch.float64, device="cuda") * total
        i = torch.clamp(torch.searchsorted(cum, s, right=True) - 1, 0, len(lens) - 1)
        t = ((s - cum[i]) / torch.clamp(lens[i], min=1e-300))[:, None]
        p = path_pts[i] + t * seg[i]
        rad = band * torch.sqrt(torch.rand(m, generator=gen, dtype=torch.float64, device="cuda"))
        th = 2 * math.pi * torch.rand(m, generator=gen, dtype=torch.float64, device="cuda")
        return p + torch.stack([rad * torch.cos(th), rad * torch.sin(th)], dim=1)
    return draw


def _corridor_sampler(half_width: float):
    """Draws uniform in the strip of half-width `half_width` around the
    straight segment x_init -> x_goal (a fixed, scene-blind prior)."""
    import torch
    a = torch.tensor(X_INIT, dtype=torch.float64, device="cuda")
    b = torch.tensor(X_GOAL, dtype=torch.float64, device="cuda")
    d = b - a
    nrm = torch.stack([-d[1], d[0]]) / torch.sqrt((d ** 2).sum())

    def draw(m, gen):
        t = torch.rand(m, generator=gen, dtype=torch.float64, device="cuda")[:, None]
        o = (2 * torch.rand(m, generator=gen, dtype=torch.float64, device="cuda") - 1)[:, None]
        return a + t * d + o * half_width * nrm
    return draw


def _learned_sampler(prop, seed: int):
    """Draws from the proposal for scene `seed` (pure network samples)."""
    import torch
    grid = torch.from_numpy(W.occupancy_grid(W.c5_scene(seed))[None]).cuda()

    def draw(m, gen):
        parts = []
        for i in range(0, m, prop.max_rows):
            k = min(prop.max_rows, m - i)
            noise = torch.randn((k, 8), generator=gen, dtype=torch.float32, device="cuda")
            scene = torch.zeros(k, dtype=torch.int32, device="cuda")
            parts.append(prop.forward(grid, scene, noise).double())
        return torch.cat(parts)
    return draw


def dev_mixture_points(seed: int, n: int, draw, fraction: float = 0.5, stream: int = 1,
                       chunk: int = 1 << 18):
    """x_init, x_goal and n - 2 free samples: each candidate comes from
    draw(m, generator) with probability `fraction`, else uniform in the unit
    square; candidates inside a circle or outside the square are rejected."""
    import torch
    sc = DevScene(seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(philox_key(7, seed, n, stream) & 0x7FFFFFFFFFFFFFFF)
    out, have = [], 0
    while have < n - 2:
        coin = torch.rand(chunk, generator=gen, device="cuda") < fraction
        uni = torch.rand((chunk, 2), generator=gen, dtype=torch.float64, device="cuda")
        k = int(coin.sum())
        cand = uni
        if k:
            drawn = draw(k, gen)
            cand = uni.clone()
            cand[coin.nonzero().squeeze(1)[:drawn.shape[0]]] = drawn
        ok = ~sc.inside(cand) & (cand >= 0).all(dim=1) & (cand <= 1).all(dim=1)
        xy = cand[ok]
        out.append(xy)
        have += xy.shape[0]
    head = torch.tensor(np.array([X_INIT, X_GOAL]), dtype=torch.float64, device="cuda")
    return torch.cat([head, torch.cat(out)[:n - 2]])


ARMS = ("uniform", "learned", "ideal", "corridor")


def dev_compare(prop, seeds, sizes, refs, fraction: float = 0.5, band: float = 0.02,
                corridor: float = 0.1, arms=ARMS, chunk: int = 8):
    """Best start-goal cost per (arm, N, scene): dict N -> {arm: costs array},
    +inf where the goal is unreached.  'uniform': N uniform free samples;
    'learned': the 50/50 mixture with the proposal; 'ideal': 50/50 with
    samples within `band` of the scene's reference path (what a perfect
    proposal would give); 'corridor': 50/50 with the fixed corridor around
    the straight start-goal segment."""
    res = {}
    seeds = list(seeds)
    for n in sizes:
        costs = {a: [] for a in arms}
        for c0 in range(0, len(seeds), chunk):
            part = seeds[c0:c0 + chunk]
            for arm in arms:
                rms = []
                for s in part:
                    if arm == "uniform":
                        pts = dev_uniform_points(s, n, 1)
                    elif arm == "learned":
                        pts = dev_mixture_points(s, n, _learned_sampler(prop, s), fraction, 11)
                    elif arm == "ideal":
                        g_ref, path = refs[s]
                        draw = _polyline_sampler(path, band) if path is not None else \
                            _corridor_sampler(corridor)
                        pts = dev_mixture_points(s, n, draw, fraction, 12)
                    else:
                        pts = dev_mixture_points(s, n, _corridor_sampler(corridor), fraction, 13)
                    rms.append(dev_roadmap(pts, s))
                costs[arm] += [float(g[GOAL]) for g, _ in solve(rms)]
                del rms
        res[int(n)] = {a: np.asarray(v) for a, v in costs.items()}
    return res


def spread(prop, seeds, refs, band: float = 0.02, m: int = 20_000):
    """How the proposal's own samples sit around each scene's reference path:
    the fraction within `band` of it, and the fraction of the path's length
    (bins of 2 * band) with at least one sample within `band` (coverage)."""
    import torch
    inb, cov, free = [], [], []
    for s in seeds:
        g_ref, path = refs[s]
        if path is None:
            continue
        gen = torch.Generator(device="cuda")
        gen.manual_seed(philox_key(9, s) & 0x7FFFFFFFFFFFFFFF)
        xy = _learned_sampler(prop, s)(m, gen)
        sc = DevScene(s)
        free.append(float((~sc.inside(xy)).double().mean()))
        near = dev_near_path(xy, path, band)
        inb.append(float(near.double().mean()))
        # arc-length position of the nearest path point, per near sample
        seg = path[1:] - path[:-1]
        lens = torch.sqrt((seg ** 2).sum(dim=1))
        cum = torch.cat([torch.zeros(1, dtype=lens.dtype, device="cuda"), torch.cumsum(lens, 0)])
        q = xy[near]
        best = torch.full((q.shape[0],), float("inf"), dtype=torch.float64, device="cuda")
        pos = torch.zeros_like(best)
        for i in range(seg.shape[0]):
            L2 = float(lens[i] ** 2)
            t = torch.zeros_like(best) if L2 == 0.0 else \
                ((q - path[i]) @ seg[i] / L2).clamp(0.0, 1.0)
            d2 = ((path[i] + t[:, None] * seg[i] - q) ** 2).sum(dim=1)
            take = d2 < best
            best = torch.where(take, d2, best)
            pos = torch.where(take, cum[i] + t * lens[i], pos)
        nb = max(1, int(math.ceil(float(cum[-1]) / (2 * band))))
        hit = torch.zeros(nb, dtype=torch.bool, device="cuda")
        if q.shape[0]:
            hit[torch.clamp((pos / (2 * band)).long(), 0, nb - 1)] = True
        cov.append(float(hit.double().mean()))
    return dict(scenes=len(inb), within_band=float(np.mean(inb)) if inb else None,
                path_coverage=float(np.mean(cov)) if cov else None,
                free_fraction=float(np.mean(free)) if free else None, samples_per_scene=m)


def paired_table(res, refs=None) -> dict:
    """Per N and arm (against uniform, paired by scene over the scenes where
    both reach the goal): mean costs, mean difference with its 95% interval
    (normal approximation), the fraction of scenes where the arm is cheaper,
    and success counts; the reference cost's mean when refs is given."""
    out = {}
    for n, by_arm in res.items():
        cu = by_arm["uniform"]
        row = {"uniform_solved": int(np.isfinite(cu).sum()), "scenes": int(len(cu))}
        for arm, ca in by_arm.items():
            if arm == "uniform":
                continue
            both = np.isfinite(cu) & np.isfinite(ca)
            d = ca[both] - cu[both]
            se = float(d.std(ddof=1) / math.sqrt(len(d))) if len(d) > 1 else None
            row[arm] = dict(solved=int(np.isfinite(ca).sum()), both_solved=int(both.sum()),
                            uniform_mean=float(cu[both].mean()) if both.any() else None,
                            arm_mean=float(ca[both].mean()) if both.any() else None,
                            paired_diff=float(d.mean()) if both.any() else None,
                            ci95=[float(d.mean() - 1.96 * se), float(d.mean() + 1.96 * se)]
                            if se is not None else None,
                            arm_better=float((d < 0).mean()) if both.any() else None,
                            sign=(None if se is None else
                                  "cheaper" if d.mean() + 1.96 * se < 0 else
                                  "costlier" if d.mean() - 1.96 * se > 0 else "no difference"))
        out[str(n)] = row
    return out


def time_mlp(prop_cls, rows: int = 1 << 20, reps: int = 20, train_targets: int = 2048,
             train_K: int = 16, train_scenes: int = 32) -> dict:
    """CUDA-event timings of the proposal's forward pass (both kernels) at
    `rows` rows -- the whole call (grid term, argument kernels, the pass, the
    host's synchronisation) and, for the fused kernel, the kernel alone --
    and of one IMLE training step, with their FLOP rates (algorithmic FLOPs:
    2 (8 * 256 + 256 * 256 + 256 * 2) per row, 2 * 4096 * 256 per scene term)."""
    import torch
    fwd_flops_row = 2 * (8 * 256 + 256 * 256 + 256 * 2)      # 136,192
    grid_flops = 2 * 4096 * 256                               # per scene and pass
    rng = np.random.default_rng(0)
    grids = torch.from_numpy((rng.random((train_scenes, 4096)) < 0.2).astype(np.float32)).cuda()
    out = {}
    P = prop_cls(train_scenes, max(rows, train_targets * train_K), seed=3)
    g1 = grids[:1].contiguous()
    scene = torch.zeros(rows, dtype=torch.int32, device="cuda")
    noise = torch.randn((rows, 8), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    for kernel in ("tcgen05", "layered"):
        P.set_options(kernel)
        for _ in range(3):
            P.forward(g1, scene, noise)
        ts, ks = [], []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            P.forward(g1, scene, noise)
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            if kernel == "tcgen05":
                ks.append(P.kernel_ms())
        ms = float(np.median(ts))
        flops = rows * fwd_flops_row + grid_flops
        rec = dict(rows=rows, call_ms=round(ms, 4), call_tflops=round(flops / (ms / 1e3) / 1e12, 1))
        if ks:
            kms = float(np.median(ks))
            rec.update(kernel_ms=round(kms, 4),
                       kernel_tflops=round(rows * fwd_flops_row / (kms / 1e3) / 1e12, 1))
        out[f"forward_{kernel}"] = rec
    P.set_options("tcgen05")
    T, K = train_targets, train_K
    tsc = torch.arange(train_scenes, dtype=torch.int32, device="cuda").repeat_interleave(
        T // train_scenes)
    tg = torch.rand((T, 2), device="cuda")
    nz = torch.randn((T * K, 8), device="cuda")
    for _ in range(3):
        P.train_step(grids, tsc, tg, K, nz, 1e-5)
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        P.train_step(grids, tsc, tg, K, nz, 1e-5)
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    bwd_row = 2 * 2 * (256 * 256) + 2 * 2 * (256 * 2) + 2 * (8 * 256)
    flops = T * K * fwd_flops_row + T * bwd_row + train_scenes * 2 * grid_flops
    out["train_step"] = dict(targets=T, K=K, scenes=train_scenes, ms=round(ms, 4),
                             tflops=round(flops / (ms / 1e3) / 1e12, 2),
                             note="device time between events around the call, including the "
                                  "host round trips between its synchronising phases")
    P.close()
    return out


def main(argv=None):
    """Train on planner solutions, then compare the mixtures with uniform
    sampling on held-out scenes, everything device-resident; prints (and with
    --out writes) one JSON document."""
    import argparse
    import json

    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train-scenes", type=int, default=5000)
    ap.add_argument("--n-train", type=int, default=200_000)
    ap.add_argument("--band", type=float, default=0.02)
    ap.add_argument("--steps", type=int, default=20_000)
    ap.add_argument("--scenes-per-step", type=int, default=32)
    ap.add_argument("--targets-per-scene", type=int, default=64)
    ap.add_argument("--K", type=int, default=16)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--lr-final", type=float, default=3e-5)
    ap.add_argument("--test-scenes", type=int, default=200)
    ap.add_argument("--sizes", default="100000,500000")
    ap.add_argument("--ref-n", type=int, default=1_000_000)
    ap.add_argument("--fraction", type=float, default=0.5)
    ap.add_argument("--corridor", type=float, default=0.1, help="corridor arm's half-width")
    ap.add_argument("--chunk", type=int, default=32, help="scenes per training-set batch")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="")
    ap.add_argument("--weights-out", default="", help="save the trained weights (.npy)")
    a = ap.parse_args(argv)

    from . import Proposal
    torch.cuda.set_device(0)
    report = dict(config=vars(a))

    def save():
        if a.out:
            with open(a.out, "w") as f:
                f.write(json.dumps(report) + "\n")
    t = time.perf_counter()
    grids, targets, costs, kept = dev_training_set(range(a.train_scenes), a.n_train, a.band,
                                                   chunk=a.chunk)
    keep = [i for i, t_ in enumerate(targets) if t_.shape[0] > 0]
    grids, targets = grids[keep], [targets[i] for i in keep]
    report["training_set"] = dict(scenes=a.train_scenes, scenes_solved=len(kept),
                                  scenes_used=len(keep),
                                  targets=int(sum(t_.shape[0] for t_ in targets)),
                                  mean_cost=float(costs.mean()) if len(costs) else None,
                                  seconds=round(time.perf_counter() - t, 1))
    print(json.dumps(report["training_set"]), flush=True)
    save()
    rows = a.scenes_per_step * a.targets_per_scene * a.K
    prop = Proposal(a.scenes_per_step, rows, seed=a.seed + 1)
    losses, secs = train(prop, grids, targets, a.steps, a.scenes_per_step, a.targets_per_scene,
                         a.K, a.lr, a.seed, log_every=max(1, a.steps // 10), lr_final=a.lr_final)
    report["training"] = dict(steps=a.steps, seconds=round(secs, 2),
                              ms_per_step=round(1e3 * secs / max(1, a.steps), 3),
                              loss_first=float(losses[:20].mean()),
                              loss_last=float(losses[-20:].mean()))
    print(json.dumps(report["training"]), flush=True)
    save()
    w = prop.get_weights()
    if a.weights_out:
        np.save(a.weights_out, w.cpu().numpy())
    prop.close()
    del targets
    torch.cuda.empty_cache()
    ev = Proposal(1, 1 << 18, seed=a.seed + 1)
    ev.set_weights(w)
    test_seeds = list(range(1_000_000, 1_000_000 + a.test_scenes))
    t = time.perf_counter()
    refs = reference_paths(test_seeds, a.ref_n)
    finite = [v[0] for v in refs.values() if math.isfinite(v[0])]
    report["reference"] = dict(n=a.ref_n, solved=len(finite),
                               mean_cost=float(np.mean(finite)) if finite else None,
                               seconds=round(time.perf_counter() - t, 1))
    print(json.dumps(report["reference"]), flush=True)
    save()
    report["spread"] = spread(ev, test_seeds, refs, a.band)
    print(json.dumps(report["spread"]), flush=True)
    save()
    t = time.perf_counter()
    res = dev_compare(ev, test_seeds, [int(x) for x in a.sizes.split(",")], refs, a.fraction,
                      a.band, a.corridor)
    report["comparison"] = paired_table(res)
    report["comparison_seconds"] = round(time.perf_counter() - t, 1)
    report["per_scene"] = {str(n): {arm: [None if not math.isfinite(x) else round(x, 6)
                                          for x in v.tolist()] for arm, v in by.items()}
                           for n, by in res.items()}
    report["reference_costs"] = [None if not math.isfinite(refs[s][0]) else round(refs[s][0], 6)
                                 for s in test_seeds]
    print(json.dumps(report["comparison"]), flush=True)
    save()
    ev.close()
    report["mlp_timing"] = time_mlp(Proposal)
    print(json.dumps(report["mlp_timing"]), flush=True)
    save()


if __name__ == "__main__":
    main()
