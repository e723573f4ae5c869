"""Importance network on the GPU (BF16 tensor-core forward and backward,
Adam) against the binary64 oracle network with the same BF16 weights, and
the learned weight windows against the analog method."""
import math

import numpy as np
import pytest

import oracle
import synth
from paper_2403_12345_gb300 import gbmc
from paper_2403_12345_gb300 import importance as imp

pytestmark = pytest.mark.gpu


def _cos(a, b):
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def _ctx(params, offset=(0, 0, 0, 0), scale=(1, 1, 1, 1), prob=None):
    prob = prob or synth.make_tiny_problem(seed=61, n_nuc=2, kind=synth.GEOM_SLAB)
    ctx = gbmc.Context(0)
    ctx.load(prob)
    ctx.set_importance_net(params, offset, scale)
    return ctx, prob


def _check_grad(ctx, pd, x, y, w):
    import torch
    X, Y, W = (torch.tensor(a, device="cuda") for a in (x, y, w))
    loss, g = ctx.mlp_gradient(X, Y, W)
    lref, gref = oracle.mlp_grad(pd, x.astype(np.float64), y.astype(np.float64),
                                 w.astype(np.float64))
    assert abs(loss - lref) <= 2e-2 * lref, (loss, lref)
    assert _cos(g.astype(np.float64), gref) >= 0.999
    assert np.abs(g - gref).max() <= 2e-2 * np.abs(gref).max()


def test_forward_and_gradient_match_oracle():
    import torch
    rng = np.random.default_rng(3)
    pb = imp.to_bf16(rng.normal(0, 0.3, gbmc.MLP_NPARAM))
    pd = imp.from_bf16(pb).astype(np.float64)
    n = 3001                      # not a multiple of the 16-row tiles
    x = rng.uniform(-1, 1, (n, 4)).astype(np.float32)
    y = rng.normal(0, 1, n).astype(np.float32)
    w = rng.uniform(0.5, 2.0, n).astype(np.float32)
    ctx, _ = _ctx(pb)
    try:
        X = torch.tensor(x, device="cuda")
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.mlp_forward(X, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        ref = oracle.mlp_forward(pd, x.astype(np.float64))
        assert np.abs(o - ref).max() <= 2e-2 * np.abs(ref).max()
        assert _cos(o, ref) >= 0.999
        _check_grad(ctx, pd, x, y, w)
    finally:
        ctx.close()


def _emulate(pb, x):
    """The forward as the kernels form it: layer 1 in binary32 (no fused
    multiply-add), relu(z1) rounded to BF16 for the tensor cores, layers 2
    and 3 then exact (binary64) -- the tensor cores' binary32 accumulation
    of 64 products differs from it by a few ulp."""
    H = gbmc.MLP_HIDDEN
    p = imp.from_bf16(pb)
    W1, b1 = p[:4 * H].reshape(H, 4), p[4 * H:5 * H]
    W2, b2 = p[5 * H:5 * H + H * H].reshape(H, H), p[5 * H + H * H:6 * H + H * H]
    W3, b3 = p[6 * H + H * H:7 * H + H * H], p[7 * H + H * H]
    z1 = np.repeat(b1[None, :], len(x), 0).astype(np.float32)
    for i in range(4):
        z1 = (z1 + (W1[:, i][None, :] * x[:, i:i + 1]).astype(np.float32)).astype(np.float32)
    h1 = imp.from_bf16(imp.to_bf16(np.maximum(z1, 0))).astype(np.float64)
    z2 = h1 @ W2.astype(np.float64).T + b2
    return np.maximum(z2, 0) @ W3.astype(np.float64) + float(b3)


def test_forward_matches_bf16_emulation():
    # a tight check of the tensor-core layer (operand layouts, every row of
    # the 128-row tiles and a ragged last tile)
    import torch
    rng = np.random.default_rng(17)
    pb = imp.to_bf16(rng.normal(0, 0.3, gbmc.MLP_NPARAM))
    n = 128 * 37 + 19
    x = rng.uniform(-1, 1, (n, 4)).astype(np.float32)
    ctx, _ = _ctx(pb)
    try:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.mlp_forward(torch.tensor(x, device="cuda"), out)
        o = out.cpu().numpy().astype(np.float64)
    finally:
        ctx.close()
    ref = _emulate(pb, x)
    assert np.abs(o - ref).max() <= 1e-4 * (np.abs(ref).max() + 1.0), np.abs(o - ref).max()


def test_training_fits_and_gradients_stay_exact():
    import torch
    rng = np.random.default_rng(4)
    n = 4096
    x = rng.uniform(0, 1, (n, 4)).astype(np.float32)
    y = (np.sin(3 * x[:, 0]) + 0.5 * x[:, 3] - x[:, 1] * x[:, 2]).astype(np.float32)
    w = np.ones(n, np.float32)
    ctx, _ = _ctx(imp.init_params(1))
    try:
        X, Y, W = (torch.tensor(a, device="cuda") for a in (x, y, w))
        loss0, _ = ctx.mlp_gradient(X, Y, W)
        loss1 = ctx.mlp_train(X, Y, W, 800, 3e-3)
        assert loss1 < loss0 / 10, (loss0, loss1)
        trained = ctx.get_importance_net()
        ctx.set_importance_net(trained, (0, 0, 0, 0), (1, 1, 1, 1))
        # at the fitted point the residuals sit at the BF16 activation noise;
        # shifted targets keep the gradient a signal to compare
        _check_grad(ctx, imp.from_bf16(trained).astype(np.float64), x, y + 0.5, w)
    finally:
        ctx.close()


def test_windows_from_a_handmade_network():
    H = gbmc.MLP_HIDDEN
    p = np.zeros(gbmc.MLP_NPARAM, np.float32)
    p[0] = 1.0                       # W1[0][0]: unit 0 = feature 0 (depth)
    p[5 * H] = 1.0                   # W2[0][0]
    p[6 * H + H * H] = 2.0           # W3[0]: log-importance = 2 x / X
    prob = synth.make_config(5, n_particles=10, grid_scale=0.02)
    g = gbmc.geometry_from(prob.geom)
    off, sc = imp.feature_map(g, prob.edges)
    ctx, _ = _ctx(imp.to_bf16(p), off, sc, prob)
    try:
        ctx.weight_windows_from_net(g)
        lower = ctx.get_weight_windows(g.n_layers)
    finally:
        ctx.close()
    x = (np.arange(g.n_layers) + 0.5) * g.layer_dx
    # the feature in binary32, rounded to BF16 where it enters the tensor cores
    f0 = (x * sc[0]).astype(np.float32)
    out = 2.0 * imp.from_bf16(imp.to_bf16(f0)).astype(np.float64)
    expect = np.exp(out[0] - out) / 2.5
    assert np.allclose(lower, expect[:, None], rtol=1e-5, atol=0)


def test_learned_windows_unbiased_with_higher_figure_of_merit():
    prob = synth.make_config(5)
    g = gbmc.geometry_from(prob.geom)
    ctx = gbmc.Context(0)
    try:
        ctx.load(prob)
        n_an, n_ww = 4_000_000, 400_000

        def analog(b):
            return gbmc.problem(g, prob.seed, n_an, batch=b)

        def learned(b):
            return gbmc.problem(g, prob.seed, n_ww, batch=b)

        lw = imp.LearnedWindows(ctx, g, prob.edges, seed=5)
        lw.collect(analog, range(100, 104), capacity=16_000_000)
        loss = lw.train(steps=1500, lr=3e-3)
        assert np.isfinite(loss)
        ctx.clear_weight_windows()
        fa = imp.figure_of_merit(ctx, analog, range(8), n_an)
        lw.apply()
        fw = imp.figure_of_merit(ctx, learned, range(8), n_ww)
    finally:
        ctx.close()
    se = math.hypot(fa["mean"] * fa["rel_err"], fw["mean"] * fw["rel_err"])
    print("analog", fa, "learned", fw)
    assert fa["mean"] > 0 and fw["mean"] > 0
    assert abs(fw["mean"] - fa["mean"]) < 4.5 * se, (fa["mean"], fw["mean"], se)
    assert fw["fom"] > fa["fom"], (fw["fom"], fa["fom"])
