"""Autotuner of the step's launch shape.

The tuned knobs change no result bit (the per-particle arithmetic and its
order do not depend on them): the threads per block of the density and
force passes, and whether the force pass takes its pairs from the density
pass's hit segments or tests the candidates again.  For a scene (or batch) the tuner snapshots the state,
times a few steps of each candidate shape with CUDA events, restores the
state, applies the fastest shape and caches the choice in a JSON file keyed
by the workload's signature (particle, boid and cell counts).
"""
from __future__ import annotations

import json
import os

CANDIDATES = [(b, s) for b in (64, 128, 256, 512) for s in (0, 1)]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")


def signature(scene) -> str:
    """Workload signature: totals and the first scene's cell size."""
    return (f"S{len(scene.params_list)}-n{scene.n}-b{scene.n_boid}-c{scene.ncells}-"
            f"d{scene.params['cell_size']:.6g}")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(scene, steps: int = 4, warmup: int = 1, cache: str | None = DEFAULT_CACHE,
             candidates=CANDIDATES, force: bool = False) -> dict:
    """Pick the fastest bit-neutral launch shape for ``scene`` and apply it.

    Returns {"block", "use_segments", "ms_per_step": {shape: ms}, "cached"}.
    The scene's state is left exactly as it was."""
    torch = scene.torch
    key = signature(scene)
    table = _load(cache) if cache else {}
    if not force and key in table:
        best = table[key]
        scene.set_tuning(best["block"], best["use_segments"])
        return dict(best, cached=True)
    snapshot = [t.clone() for t in scene.get_state()]
    timings = {}
    for block, use_seg in candidates:
        scene.set_state(*snapshot)
        scene.set_tuning(block, use_seg)
        scene.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        scene.step(steps)
        e1.record()
        torch.cuda.synchronize(scene.device)
        timings[f"{block}/{use_seg}"] = e0.elapsed_time(e1) / steps
    best_key = min(timings, key=timings.get)
    block, use_seg = (int(x) for x in best_key.split("/"))
    scene.set_state(*snapshot)
    scene.set_tuning(block, use_seg)
    best = {"block": block, "use_segments": use_seg, "ms_per_step": timings}
    if cache:
        table = _load(cache)
        table[key] = best
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return dict(best, cached=False)
