"""Pins of the oracle's weight-window transport and importance network.

Weight windows (split above the window, Russian roulette below) must leave
every tally unbiased; the network's back-propagated gradient must equal
central finite differences of its loss.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
import synth

Z_MAX = 4.5


# ---------------------------------------------------------------- network

def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, oracle.MLP_NPARAM)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(2)
    x = rng.uniform(-1, 1, (24, 4))
    y = rng.normal(0, 1, 24)
    w = rng.uniform(0.5, 2.0, 24)
    loss, g = oracle.mlp_grad(p, x, y, w)
    assert loss > 0
    H = oracle.MLP_HIDDEN
    offsets = [0, 4 * H, 5 * H, 5 * H + H * H, 6 * H + H * H, 7 * H + H * H]
    idx = list(rng.integers(0, oracle.MLP_NPARAM, 60)) + offsets
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = oracle.mlp_grad(p + e, x, y, w)
        lm, _ = oracle.mlp_grad(p - e, x, y, w)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_mlp_forward_closed_form():
    H = oracle.MLP_HIDDEN
    p = np.zeros(oracle.MLP_NPARAM)
    W1, b1 = 0, 4 * H
    W2, b2 = 5 * H, 5 * H + H * H
    W3, b3 = 6 * H + H * H, 7 * H + H * H
    p[W1 + 0 * 4 + 0] = 1.0        # unit 0 of layer 1 reads x0
    p[W1 + 1 * 4 + 3] = -2.0       # unit 1 reads -2 x3
    p[W2 + 0 * H + 0] = 1.0        # unit 0 of layer 2 passes unit 0
    p[W2 + 5 * H + 1] = 3.0        # unit 5 of layer 2 = 3 unit 1
    p[b2 + 5] = 0.25
    p[W3 + 0] = 2.0
    p[W3 + 5] = -1.0
    p[b3] = 0.5
    x = np.array([[0.7, 9.0, 9.0, -0.1], [-0.4, 0.0, 0.0, 0.3], [1.5, 0.0, 0.0, 0.0]])
    relu = lambda v: np.maximum(v, 0.0)
    expect = 2 * relu(relu(x[:, 0])) - relu(3 * relu(-2 * x[:, 3]) + 0.25) + 0.5
    assert np.allclose(oracle.mlp_forward(p, x), expect, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- weight windows

def _absorber_slab(tau, n_particles, seed=41):
    p = synth.make_tiny_problem(seed=seed, n_nuc=1, flat=True, f_abs=[1.0],
                                kind=synth.GEOM_SLAB, n_particles=n_particles)
    g = p.geom
    g.n_first = g.n_layers
    st = p.density[0] * p.sigma_t[0]
    g.layer_dx = tau / st / g.n_layers
    return p, st


def _importance_windows(p, st):
    """Windows from the exact uncollided importance exp(Sigma_t x) of a pure
    absorber, normalised so the survival weight in the first layer is 1."""
    g = p.geom
    xc = (np.arange(g.n_layers) + 0.5) * g.layer_dx
    imp = np.exp(st * xc)
    lower = (imp[0] / imp) / 2.5
    return np.repeat(lower[:, None], p.n_bins, axis=1)


def test_windows_that_never_trigger_leave_the_walk_unchanged():
    p = synth.make_config(5, n_particles=3000, grid_scale=0.02)
    a = oracle.run(p, seed=p.seed, n=3000)
    tiny = np.full((p.geom.n_cells(), p.n_bins), 1e-300)
    b = oracle.run(p, seed=p.seed, n=3000, ww=(tiny, 1e300, 2.5, 10))
    for k in ("n_coll", "status", "n_flights", "n_draws", "E", "x"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["flux"], b["flux"])
    off = np.zeros((p.geom.n_cells(), p.n_bins))
    c = oracle.run(p, seed=p.seed, n=3000, ww=(off, 5.0, 2.5, 10))
    assert np.array_equal(a["n_coll"], c["n_coll"]) and np.array_equal(a["flux"], c["flux"])


def test_windows_unbiased_on_pure_absorber_transmission():
    tau = 7.0
    p, st = _absorber_slab(tau, 4000)
    pt = special.expn(2, tau)               # exact transmission (uncollided)
    win = _importance_windows(p, st)
    per_batch = []
    for b in range(12):
        r = oracle.run(p, seed=11, batch=b, n=4000, ww=(win, 5.0, 2.5, 10))
        per_batch.append(r["weights"][oracle.S_LEAK_FAR] / 4000)
        assert r["counts"][oracle.S_HISTORY] == 4000
        assert r["counts"][oracle.S_SPLIT] > 0
    m = np.mean(per_batch)
    se = np.std(per_batch, ddof=1) / math.sqrt(len(per_batch))
    assert abs(m - pt) < Z_MAX * se, (m, pt, se)
    # the same number of analog histories would see ~4 transmissions per
    # batch; with windows the relative error is far smaller
    rel_ww = np.std(per_batch, ddof=1) / m
    rel_analog = math.sqrt((1 - pt) / (pt * 4000))
    assert rel_ww < rel_analog / 3, (rel_ww, rel_analog)


def test_split_copies_carry_the_weight():
    tau = 5.0
    p, st = _absorber_slab(tau, 2000, seed=43)
    win = _importance_windows(p, st)
    r = oracle.run(p, seed=3, n=2000, ww=(win, 5.0, 2.5, 10))
    # a pure absorber has one collision per surviving copy; every copy that
    # is not rouletted either is absorbed or leaks
    c, w = r["counts"], r["weights"]
    copies = c[oracle.S_HISTORY] + c[oracle.S_SPLIT]
    assert c[oracle.S_ABSORPTION] + c[oracle.S_LEAK] + c[oracle.S_ROULETTE] == copies
    assert c[oracle.S_COLLISION] == c[oracle.S_ABSORPTION]
    # primaries and copies start inside; nothing leaks back through x = 0
    assert c[oracle.S_LEAK] == c[oracle.S_LEAK_FAR]
    assert w[oracle.S_SPLIT] > 0
