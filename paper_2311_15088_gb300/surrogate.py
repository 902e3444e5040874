"""Training and evaluation driver of the boid-force surrogate.

Every arithmetic step runs in the library's kernels (features, SPH step,
MLP forward / backward / Adam); this module only schedules them:

1. ``log_pairs``: run a scene and record, at every step, the boids' stencil
   features and the exact fluid force F_b the step computes for that state.
2. ``train``: Adam on mini-batches of (features, F_b / F_scale), F_scale the
   RMS of the training forces (phase 0 of sph_mlp_train_step).
3. ``fit_error_head``: on held-out pairs, train the error head (phase 1) to
   predict log10 of each query's relative error
   |F_pred - F| / max(|F|, 0.05 F_scale).
4. ``calibrate``: the largest error-head threshold whose fallback keeps the
   aggregate error ||F_used - F||_2 / ||F||_2 of the held-out pairs at or
   below the target (5 %); queries with a feature outside the training
   range (widened by a margin, ``input_bounds``) always fall back.
5. ``evaluate``: that aggregate error, the per-query relative errors and the
   fallback fraction on fresh queries.
"""
from __future__ import annotations

import math

import numpy as np

from . import scenes
from .sph import SPH_BOID_EXACT_LOCAL, SPH_BOID_SURROGATE, SPH_BOID_SURROGATE_FALLBACK, Mlp, Scene

REL_FLOOR = 0.05  # per-query relative error is taken against max(|F|, 0.05 F_scale)
# Feature columns beyond the 256 stencil features and the boid velocity:
# the boid's offset from the stencil centre (259 .. 261) and its own
# density and kernel moments (262 .. 269); zeroing them gives the
# stencil-only network for ablations.
EXTRA_COLS = slice(259, 272)
MOMENT_COLS = slice(262, 272)


def _params(sc):
    p = dict(sc["params"])
    if p.get("mass") is None:
        from .sph import sph_lattice_mass

        p["mass"] = sph_lattice_mass(p, sc["lattice_spacing"])
    return p


def log_pairs(sc, steps: int, every: int = 1, device="cuda"):
    """Run ``steps`` steps of scene dict ``sc``; every ``every`` steps record
    (features, F_b) of all boids.  Returns (X bf16 [N][272], F float [N][3],
    the Scene) on the device."""
    import torch

    p = _params(sc)
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]), device=device)
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    xs, fs = [], []
    for t in range(steps):
        if t % every == 0:
            xs.append(s.features())
            s.step(1)
            fs.append(s.field("fb")[:, :3].clone())
        else:
            s.step(1)
    return torch.cat(xs), torch.cat(fs), s


def log_runs(make_scene, seeds, steps: int, device="cuda"):
    """Pairs from several short runs (one per seed) of make_scene(seed):
    more varied states than one long run of the same size."""
    import torch

    xs, fs = [], []
    for sd in seeds:
        X, F, _ = log_pairs(make_scene(sd), steps, device=device)
        xs.append(X)
        fs.append(F)
    return torch.cat(xs), torch.cat(fs)


def f_scale_of(F) -> float:
    """RMS force magnitude of the training targets."""
    return float(F.double().pow(2).sum(1).mean().sqrt().item())


def train(mlp: Mlp, X, F, f_scale: float, epochs: int = 8, batch: int = 8192, lr: float = 1e-3,
          seed: int = 0, lr_final: float = 1e-4):
    """Phase-0 Adam over shuffled mini-batches; returns the loss per epoch
    (mean of the batch losses).  The learning rate decays geometrically
    from lr to lr_final."""
    import torch

    n = X.shape[0] // batch * batch
    T = torch.zeros((X.shape[0], 4), dtype=torch.float32, device=X.device)
    T[:, :3] = F / f_scale
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    steps = epochs * (n // batch)
    k = 0
    for _ in range(epochs):
        perm = torch.randperm(X.shape[0], generator=g)[:n].to(X.device)
        acc = torch.zeros(1, device=X.device)
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            rate = lr * (lr_final / lr) ** (k / max(steps - 1, 1))
            acc += mlp.train_step(X[idx].contiguous(), T[idx].contiguous(), rate, phase=0)
            k += 1
        losses.append(float(acc.item()) / (n // batch))
    return losses


def rel_errors(Fp, F, f_scale: float):
    """Per-query |F_pred - F| / max(|F|, 0.05 F_scale)."""
    d = (Fp - F).double().norm(dim=1)
    return d / F.double().norm(dim=1).clamp_min(REL_FLOOR * f_scale)


def predict(mlp: Mlp, X, f_scale: float, chunk: int = 65536):
    import torch

    ys = [mlp.forward(X[i:i + chunk]) for i in range(0, X.shape[0], chunk)]
    Y = torch.cat(ys)
    return Y[:, :3] * f_scale, Y[:, 3]


def fit_error_head(mlp: Mlp, Xv, Fv, f_scale: float, epochs: int = 20, batch: int = 8192, lr: float = 1e-3):
    """Phase-1 training of the error head on held-out pairs: target
    log10(relative error + 1e-4)."""
    import torch

    Fp, _ = predict(mlp, Xv, f_scale)
    target = torch.log10(rel_errors(Fp, Fv, f_scale) + 1e-4).float()
    T = torch.zeros((Xv.shape[0], 4), dtype=torch.float32, device=Xv.device)
    T[:, 3] = target
    n = Xv.shape[0] // batch * batch
    g = torch.Generator(device="cpu").manual_seed(1)
    for _ in range(epochs):
        perm = torch.randperm(Xv.shape[0], generator=g)[:n].to(Xv.device)
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            mlp.train_step(Xv[idx].contiguous(), T[idx].contiguous(), lr, phase=1)
    return float(target.mean().item())


def aggregate_error(F_used, F) -> float:
    return float((F_used - F).double().norm() / F.double().norm().clamp_min(1e-30))


def per_query_error(F_used, F):
    """Median and 90th percentile over the queries of |F_used - F| /
    max(|F|, 0.05 RMS F) (RMS over these queries), the per-query companion
    of the aggregate error."""
    import torch

    rel = rel_errors(F_used, F, f_scale_of(F))
    return float(rel.median()), float(torch.quantile(rel, 0.9))


BOUND_MARGIN = 0.1


def input_bounds(X, margin: float = BOUND_MARGIN):
    """The gate's input range: per feature, the [min, max] of the training
    inputs X widened by ``margin`` times its width on both sides (FP32,
    SPH_MLP_IN values each)."""
    x = X.float()
    lo, hi = x.min(0).values, x.max(0).values
    w = (hi - lo) * margin
    return (lo - w).contiguous(), (hi + w).contiguous()


def out_of_range(X, bounds):
    """Queries with a feature outside ``bounds`` (None: no query)."""
    import torch

    if bounds is None:
        return torch.zeros(X.shape[0], dtype=torch.bool, device=X.device)
    lo, hi = bounds
    x = X.float()
    return ((x < lo) | (x > hi)).any(1)


def calibrate(mlp: Mlp, Xv, Fv, f_scale: float, target: float = 0.05, bounds=None):
    """Largest threshold t on the error head (queries with head > t fall
    back to the exact force; so do those out of ``bounds``) keeping the
    aggregate error <= target.  Returns (t, fallback fraction, aggregate
    error) on the held-out set."""
    import torch

    Fp, head = predict(mlp, Xv, f_scale)
    forced = out_of_range(Xv, bounds)
    nf = int(forced.sum().item())
    # out-of-range queries fall back whatever t is: order them first
    order = torch.argsort(torch.where(forced, torch.full_like(head, float("inf")), head), descending=True)
    # fall back on the k queries with the largest head, k = 0 .. N
    d2 = (Fp - Fv).double().pow(2).sum(1)[order]
    total = Fv.double().pow(2).sum()
    remaining = d2.sum() - torch.cat([torch.zeros(1, dtype=torch.float64, device=d2.device), torch.cumsum(d2, 0)])
    err = (remaining.clamp_min(0) / total).sqrt()
    ok = torch.nonzero(err <= target)
    k = max(int(ok[0].item()) if len(ok) else len(d2), nf)
    hs = head[order]
    if k >= len(hs):
        t = float(head.min().item()) - 1e-3
    elif k > nf:
        t = float(0.5 * (hs[k - 1] + hs[k]).item())
    else:
        t = float(hs[k].item()) + 1e-3  # no query in range falls back
    return t, k / len(hs), float(err[k].item())


def evaluate(mlp: Mlp, X, F, f_scale: float, threshold: float, bounds=None) -> dict:
    """Aggregate and per-query errors of the surrogate alone and with the
    fallback at ``threshold`` (and out of ``bounds``) on queries (X, F)."""
    import torch

    Fp, head = predict(mlp, X, f_scale)
    oor = out_of_range(X, bounds)
    fall = (head > threshold) | oor
    used = torch.where(fall[:, None], F, Fp)
    r = rel_errors(Fp, F, f_scale).cpu().numpy()
    return {
        "queries": int(X.shape[0]),
        "aggregate_error_surrogate": aggregate_error(Fp, F),
        "aggregate_error_with_fallback": aggregate_error(used, F),
        "aggregate_error_zero_predictor": 1.0,
        "aggregate_error_mean_predictor": aggregate_error(F.mean(0, keepdim=True).expand_as(F), F),
        "fallback_fraction": float(fall.float().mean().item()),
        "out_of_range_fraction": float(oor.float().mean().item()),
        "rel_error_median": float(np.median(r)),
        "rel_error_p90": float(np.percentile(r, 90)),
    }


def build_and_train(make_scene, train_seeds, val_seeds, steps=64, epochs=120, batch=2048, lr=1e-3,
                    device="cuda", target=0.045, seed=0, head_epochs=10, zero_cols=None, pairs=None,
                    return_pairs=False, bound_margin=BOUND_MARGIN):
    """Log training pairs (one run of ``steps`` steps per training seed of
    make_scene) and held-out pairs (validation seeds), train the network,
    fit the error head and calibrate the fallback threshold for an
    aggregate error <= target on the validation pairs (4.5 % by default: a
    margin under the 5 % goal for queries the calibration has not seen).  ``zero_cols`` (a slice) blanks feature
    columns in every pair (an ablation; such a network is for Python-side
    evaluation only, since the library's features fill them).  ``pairs``
    reuses logged (X, F, Xv, Fv).  The gate's input range is the training
    range widened by ``bound_margin`` (None: no range check); it is
    ``mlp.bounds``, for Scene.set_surrogate.  Returns (mlp, info), plus the
    pairs when ``return_pairs``."""
    import time

    import torch

    t0 = time.perf_counter()
    if pairs is None:
        X, F = log_runs(make_scene, train_seeds, steps, device=device)
        Xv, Fv = log_runs(make_scene, val_seeds, steps, device=device)
    else:
        X, F, Xv, Fv = pairs
    if zero_cols is not None:
        X, Xv = X.clone(), Xv.clone()
        X[:, zero_cols] = 0
        Xv[:, zero_cols] = 0
    torch.cuda.synchronize()
    t_log = time.perf_counter() - t0
    fs = f_scale_of(F)
    mlp = Mlp(max(batch, 65536), device=device)
    mlp.set_params(torch.from_numpy(init_params(seed)))
    t0 = time.perf_counter()
    losses = train(mlp, X, F, fs, epochs=epochs, batch=batch, lr=lr)
    fit_error_head(mlp, Xv, Fv, fs, epochs=head_epochs, batch=batch)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    mlp.bounds = input_bounds(X, bound_margin) if bound_margin is not None else None
    thr, frac, err = calibrate(mlp, Xv, Fv, fs, target, mlp.bounds)
    info = {"bound_margin": bound_margin,
            "val_out_of_range_fraction": float(out_of_range(Xv, mlp.bounds).float().mean().item()),
            "train_pairs": int(X.shape[0]), "val_pairs": int(Xv.shape[0]), "f_scale": fs,
            "epochs": epochs, "batch": batch, "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
            "threshold": thr, "val_fallback_fraction": frac, "val_aggregate_error": err,
            "train_aggregate_error": aggregate_error(predict(mlp, X[:262144], fs)[0], F[:262144]),
            "seconds_logging": t_log, "seconds_training": t_train, "status": mlp.status()}
    if return_pairs:
        return mlp, info, (X, F, Xv, Fv)
    return mlp, info


def init_params(seed: int = 0) -> np.ndarray:
    """Packed FP32 parameters: weights uniform in +-1/sqrt(fan_in), biases 0
    (layers 272 -> 256 -> 256 -> 256 -> 16)."""
    rng = np.random.default_rng(seed)
    parts = []
    for n_in, n_out in ((272, 256), (256, 256), (256, 256), (256, 16)):
        lim = 1.0 / math.sqrt(n_in)
        parts.append(rng.uniform(-lim, lim, size=n_out * n_in))
        parts.append(np.zeros(n_out))
    return np.concatenate(parts).astype(np.float32)
