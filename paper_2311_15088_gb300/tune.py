"""Autotuner of the step's launch shape.

The tuned knobs change no result bit (the per-particle arithmetic and its
order do not depend on them): for separate neighbour-pass launches, the
threads per block, the particles per thread and whether the force pass takes
its pairs from the density pass's hit segments or tests the candidates
again; for the fused
persistent pipeline (both passes in one cooperative launch over work items),
the sorted slots per work item (a run of cells) and the threads per CTA.
For a scene (or batch) the tuner snapshots the state, times a few steps of
each candidate shape with CUDA events, restores the state, applies the
fastest shape and caches the choice in a JSON file keyed by the workload's
signature (particle, boid and cell counts).
"""
from __future__ import annotations

import json
import os

# (block, use_segments, particles per thread, pipeline tile slots (0:
# separate launches), pipeline block)
CANDIDATES = ([(b, 0, 1, 0, 256) for b in (64, 128, 256, 512)] +
              [(b, 1, ppt, 0, 256) for b in (64, 128, 256, 512) for ppt in (1, 2, 4)] +
              [(256, 1, 1, t, pb) for t in (512, 2048, 8192) for pb in (128, 256)])
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


def apply(scene, shape: dict):
    scene.set_tuning(shape["block"], shape["use_segments"])
    scene.set_particles_per_thread(shape.get("ppt", 1))
    scene.set_pipeline(shape.get("pipe_tile", 0), shape.get("pipe_block", 256))


def autotune(scene, steps: int = 4, warmup: int = 1, cache: str | None = DEFAULT_CACHE,
             candidates=CANDIDATES, force: bool = False) -> dict:
    """Pick the fastest bit-neutral launch shape for ``scene`` and apply it.

    Returns {"block", "use_segments", "ppt", "pipe_tile", "pipe_block",
    "ms_per_step": {shape: ms}, "cached"}.  The scene's state is left
    exactly as it was."""
    torch = scene.torch
    key = signature(scene)
    table = _load(cache) if cache else {}
    if not force and key in table:
        best = table[key]
        apply(scene, best)
        return dict(best, cached=True)
    snapshot = [t.clone() for t in scene.get_state()]
    timings = {}
    for block, use_seg, ppt, tile, pblock in candidates:
        scene.set_state(*snapshot)
        apply(scene, {"block": block, "use_segments": use_seg, "ppt": ppt, "pipe_tile": tile, "pipe_block": pblock})
        scene.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        scene.step(steps)
        e1.record()
        torch.cuda.synchronize(scene.device)
        timings[f"{block}/{use_seg}/{ppt}/{tile}/{pblock}"] = e0.elapsed_time(e1) / steps
    best_key = min(timings, key=timings.get)
    block, use_seg, ppt, tile, pblock = (int(x) for x in best_key.split("/"))
    best = {"block": block, "use_segments": use_seg, "ppt": ppt, "pipe_tile": tile, "pipe_block": pblock,
            "ms_per_step": timings}
    scene.set_state(*snapshot)
    apply(scene, best)
    if cache:
        table = _load(cache)
        table[key] = best
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return dict(best, cached=False)
