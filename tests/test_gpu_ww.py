"""Weight-window transport on the GPU against the oracle: primary histories
bit for bit, tallies (split copies included) to summation order, split and
roulette counts exactly."""
import numpy as np
import pytest

import oracle
import synth
from paper_2403_12345_gb300 import gbmc

from gpu_helpers import assert_outcomes_equal, assert_tallies_close, gpu_problem, make_ctx, run_gpu

pytestmark = pytest.mark.gpu


def _absorber_slab(tau, n, seed=41):
    p = synth.make_tiny_problem(seed=seed, n_nuc=1, flat=True, f_abs=[1.0],
                                kind=synth.GEOM_SLAB, n_particles=n)
    g = p.geom
    g.n_first = g.n_layers
    st = p.density[0] * p.sigma_t[0]
    g.layer_dx = tau / st / g.n_layers
    return p, st


def _layer_windows(p, rate):
    g = p.geom
    xc = (np.arange(g.n_layers) + 0.5) * g.layer_dx
    lower = np.exp(-rate * (xc - xc[0])) / 2.5
    return np.repeat(lower[:, None], p.n_bins, axis=1)


def _compare(p, win, n, batch, **opts):
    ctx = make_ctx(p, **opts)
    try:
        ctx.set_weight_windows(win, 5.0, 2.5, 10)
        g = run_gpu(ctx, gpu_problem(p, n=n, batch=batch))
        st = ctx.read_stats()
    finally:
        ctx.close()
    ref = oracle.run(p, seed=p.seed, batch=batch, n=n, ww=(win, 5.0, 2.5, 10))
    assert_outcomes_equal(g, ref)
    assert_tallies_close(g, ref)
    return g, ref, st


def test_absorber_slab_windows_match_oracle():
    p, st = _absorber_slab(7.0, 20_000)
    win = _layer_windows(p, st)
    g, ref, _ = _compare(p, win, 20_000, batch=3, max_in_flight=8192)
    assert ref["counts"][oracle.S_SPLIT] > 1000


def test_rising_windows_roulette_matches_oracle():
    # windows that rise with depth: particles fall below them and roulette
    p = synth.make_config(5, n_particles=6000, grid_scale=0.02)
    win = _layer_windows(p, -0.05)
    g, ref, _ = _compare(p, win, 6000, batch=2)
    assert ref["counts"][oracle.S_ROULETTE] > 100


def test_scattering_slab_windows_match_oracle_with_small_bank():
    p = synth.make_config(5, n_particles=6000, grid_scale=0.02)
    win = _layer_windows(p, 0.15)
    g, ref, st = _compare(p, win, 6000, batch=1, max_in_flight=1024)
    assert ref["counts"][oracle.S_SPLIT] > 0
    assert st["histories"] == 6000


def test_zero_windows_are_analog():
    p = synth.make_config(5, n_particles=4000, grid_scale=0.02)
    win = np.zeros((p.geom.n_cells(), p.n_bins))
    ctx = make_ctx(p)
    try:
        ctx.set_weight_windows(win)
        g = run_gpu(ctx, gpu_problem(p, n=4000))
        ctx.clear_weight_windows()
        a = run_gpu(ctx, gpu_problem(p, n=4000))
    finally:
        ctx.close()
    ref = oracle.run(p, seed=p.seed, n=4000)
    assert_outcomes_equal(g, ref)
    assert_outcomes_equal(a, ref)
    assert_tallies_close(g, ref)
