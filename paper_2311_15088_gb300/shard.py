"""Batched scenes across ranks, one GPU per rank.

Independent scenes are the unit that shards with no exchange between ranks:
each rank steps its own share of the scenes as one batched handle
(sph_batch_create), and the only collective is a gather of per-scene
results at the end.  The share is a greedy bin-pack by particle count (the
step's cost grows with the particles of a scene): scenes in decreasing
count, each to the rank with the least load so far.

Nothing here does arithmetic of the method; ``RankBatch`` drives the
library's kernels through the binding, and ``gather`` only moves results.
"""
from __future__ import annotations

import numpy as np


def scene_weight(sc) -> int:
    """Cost proxy of a scene: its particles (fluid and boid-attached)."""
    return int(len(sc["fluid_pos"]) + len(sc["boid_pos"]))


def assign(weights, world: int):
    """Greedy bin-pack (longest first): scene indices in decreasing weight
    (ties: lower index first) go one by one to the rank with the least load
    so far (ties: lower rank).  Returns ``world`` ascending index lists that
    partition range(len(weights))."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = np.asarray(weights, dtype=np.int64)
    order = sorted(range(len(w)), key=lambda k: (-int(w[k]), k))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += int(w[k])
    return [sorted(p) for p in parts]


def imbalance(weights, parts) -> float:
    """Largest rank load over the mean load, minus one (0: perfect)."""
    w = np.asarray(weights, dtype=np.float64)
    loads = np.array([w[p].sum() if len(p) else 0.0 for p in parts])
    mean = loads.mean()
    return float(loads.max() / mean - 1.0) if mean > 0 else 0.0


class RankBatch:
    """This rank's scenes (indices into ``scenes``) as one batched handle
    on ``device``."""

    def __init__(self, scenes, indices, device="cuda", params_of=None):
        from .sph import Scene

        self.indices = list(indices)
        self.scenes = [scenes[k] for k in self.indices]
        pick = params_of or (lambda sc: sc["params"])
        self.params = [pick(sc) for sc in self.scenes]
        self.nf = [len(sc["fluid_pos"]) for sc in self.scenes]
        self.nb = [len(sc["boid_pos"]) for sc in self.scenes]
        self.scene = None
        if self.indices:
            self.scene = Scene(self.params, self.nf, self.nb, device=device)
            cat = lambda key: np.concatenate([sc[key] for sc in self.scenes])
            self.scene.set_state(cat("fluid_pos"), cat("fluid_vel"), cat("boid_pos"), cat("boid_vel"))

    def step(self, nsteps: int = 1, graph: bool = False):
        if self.scene is not None:
            (self.scene.graph_step if graph else self.scene.step)(nsteps)

    def states(self):
        """Per scene of this rank: (fluid_pos, fluid_vel, boid_pos, boid_vel)
        float32 numpy arrays, keyed by scene index."""
        if self.scene is None:
            return {}
        fp, fv, bp, bv = (t.cpu().numpy() for t in self.scene.get_state())
        cf, cb = np.cumsum([0] + self.nf), np.cumsum([0] + self.nb)
        return {k: (fp[cf[i]:cf[i + 1]], fv[cf[i]:cf[i + 1]], bp[cb[i]:cb[i + 1]], bv[cb[i]:cb[i + 1]])
                for i, k in enumerate(self.indices)}

    def stats(self):
        """Per scene of this rank: its sph_stats row (float64), keyed by
        scene index."""
        if self.scene is None:
            return {}
        st = self.scene.stats().cpu().numpy()
        return {k: st[i] for i, k in enumerate(self.indices)}


def gather(local: dict, n_scenes: int, world: int):
    """Collect every rank's {scene index: result} on every rank (one
    all_gather of Python objects); returns the list of results in scene
    order and the rank that produced each.  Raises if a scene is missing or
    produced twice."""
    if world > 1:
        import torch.distributed as dist

        parts = [None] * world
        dist.all_gather_object(parts, local)
    else:
        parts = [local]
    out = [None] * n_scenes
    owner = [-1] * n_scenes
    for r, part in enumerate(parts):
        for k, v in part.items():
            if owner[k] != -1:
                raise RuntimeError(f"scene {k} produced by ranks {owner[k]} and {r}")
            out[k] = v
            owner[k] = r
    missing = [k for k in range(n_scenes) if owner[k] == -1]
    if missing:
        raise RuntimeError(f"scenes without a result: {missing[:8]}")
    return out, owner
