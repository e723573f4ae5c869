"""Learned weight windows: an importance map trained on analog estimates.

Orchestration only; every step runs in libgbmc's kernels:

1. analog runs record their collision sites (mesh cell of the geometry x
   energy bin); after each run the sites are scored by whether their
   history left through the slab's far face (gbmc_importance_record /
   _accumulate) -- the analog estimate of the importance there;
2. the mesh's features with per-cell targets form the training set
   (gbmc_importance_training_set): a cell pools its energy bins and shrinks
   toward the overall score fraction, target ln I_c, weight N_c / (N_c + 5);
3. the 4 -> 64 -> 64 -> 1 network is trained by full-batch Adam on the GPU
   (gbmc_mlp_train: BF16 tensor-core forward and backward);
4. the windows are set from the network on the mesh
   (gbmc_weight_windows_from_net): lower bound = C / importance, the source
   cell holding survival weight 1.

The analog method stays the fallback and the reference the windows are
measured against: figure of merit FOM = 1 / (R^2 T) of the far-face leakage,
compared with the analog run's.
"""
from __future__ import annotations

import math

import numpy as np

from . import gbmc


def to_bf16(x) -> np.ndarray:
    """Round float32 values to BF16 (nearest even) bit patterns."""
    f = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f >> 16) & 1) + 0x7FFF
    return ((f + r) >> 16).astype(np.uint16)


def from_bf16(b) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases (parameter layout of the C ABI)."""
    rng = np.random.default_rng(seed)
    H = gbmc.MLP_HIDDEN
    W1 = rng.normal(0, math.sqrt(2 / 4), (H, 4))
    W2 = rng.normal(0, math.sqrt(2 / H), (H, H))
    W3 = rng.normal(0, math.sqrt(1 / H), H)
    p = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3, [0.0]])
    return to_bf16(p)


def feature_map(geom, edges):
    """Offsets and scales mapping (x, y, z, ln E) of the geometry's extent to
    about [0, 1]."""
    lo, hi = math.log(edges[0]), math.log(edges[-1])
    if geom.kind == gbmc.GEOM_SLAB:
        ext = (geom.n_layers * geom.layer_dx, 0.0, 0.0)
    elif geom.kind == gbmc.GEOM_LATTICE:
        L = geom.n * geom.pitch
        ext = (L, L, geom.height)
    else:
        ext = (0.0, 0.0, 0.0)
    scale = [1.0 / e if e > 0 else 0.0 for e in ext] + [1.0 / (hi - lo)]
    return [0.0, 0.0, 0.0, lo], scale


class LearnedWindows:
    """Importance-map weight windows for problem slot 0 of a context."""

    def __init__(self, ctx: gbmc.Context, geom, edges, seed: int = 0):
        self.ctx = ctx
        self.geom = geom
        self.offset, self.scale = feature_map(geom, edges)
        self.seed = seed
        self.rows = ctx.mesh_rows(geom)

    def collect(self, make_problem, batches, capacity, stream=None):
        """Analog runs of make_problem(b) for b in batches, recording and
        scoring collision sites."""
        self.ctx.clear_weight_windows()
        self.ctx.importance_record(self.geom, capacity)
        for b in batches:
            self.ctx.run_batch(make_problem(b), stream)
            self.ctx.importance_accumulate(stream)
        self.ctx.importance_record(None, 0)

    def train(self, steps=1500, lr=3e-3, stream=None):
        import torch
        n = self.rows
        feat = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        w = torch.empty(n, dtype=torch.float32, device="cuda")
        # the network's feature map first: the training set's features use it
        self.ctx.set_importance_net(init_params(self.seed), self.offset, self.scale)
        self.ctx.importance_training_set(self.geom, feat, y, w, stream)
        self.loss = self.ctx.mlp_train(feat, y, w, steps, lr, stream)
        self.data = (feat, y, w)
        return self.loss

    def apply(self, ratio=5.0, survival=2.5, max_split=10, stream=None):
        self.ctx.weight_windows_from_net(self.geom, ratio, survival, max_split, stream)


def figure_of_merit(ctx, make_problem, batches, n_per_batch, stream=None):
    """Far-face leakage per source particle over the batches: mean, relative
    error R of the mean, device time T (s) and FOM = 1 / (R^2 T)."""
    per_batch, t = [], 0.0
    for b in batches:
        ctx.reset_tallies(stream)
        ctx.run_batch(make_problem(b), stream)
        _, _, weights = ctx.read_tallies(0)
        t += ctx.last_run_ms() * 1e-3
        per_batch.append(weights[gbmc.S_LEAK_FAR] / n_per_batch)
    x = np.array(per_batch)
    mean = x.mean()
    rel = x.std(ddof=1) / math.sqrt(len(x)) / mean if mean > 0 else float("inf")
    fom = 1.0 / (rel * rel * t) if rel > 0 and np.isfinite(rel) else 0.0
    return dict(mean=mean, rel_err=rel, seconds=t, fom=fom, per_batch=x)
