"""The track-length absorption-rate tally through the C ABI against the
oracle: per bin to summation order, in both table precisions, and its
on/off/reset behaviour."""
import numpy as np
import pytest

import oracle
import synth
from paper_2403_12345_gb300 import gbmc

from gpu_helpers import gpu_problem, make_ctx

pytestmark = pytest.mark.gpu


def _close(a, b, rtol=1e-12):
    zero = b == 0
    assert np.all(a[zero] == 0)
    rel = np.abs(a[~zero] - b[~zero]) / b[~zero]
    assert rel.size == 0 or rel.max() <= rtol, rel.max()


@pytest.mark.parametrize("precision", [gbmc.FP64, gbmc.FP32])
def test_absorption_rate_matches_oracle(precision):
    p = synth.make_config(2, n_particles=20_011, grid_scale=0.02)
    ctx = make_ctx(p, (precision,), precision=precision, max_in_flight=5000)
    ctx.set_reaction_tally(True)
    gp = gpu_problem(p, batch=4)
    ctx.reset_tallies()
    ctx.run_batch(gp)
    ar = ctx.read_reaction_tally(0)
    flux, _, _ = ctx.read_tallies(0)
    ctx.close()
    ref = oracle.run(p, seed=p.seed, batch=4, n=20_011, precision=precision)
    assert ref["absrate"].sum() > 0
    _close(ar, ref["absrate"])
    _close(flux, ref["flux"])


def test_reaction_tally_switch_and_reset():
    p = synth.make_config(2, n_particles=4000, grid_scale=0.02)
    ctx = make_ctx(p)
    gp = gpu_problem(p, batch=1)
    ctx.run_batch(gp)
    with pytest.raises(gbmc.GbmcError):
        ctx.read_reaction_tally(0)           # off
    ctx.set_reaction_tally(True)             # on after a run: starts at zero
    assert np.all(ctx.read_reaction_tally(0) == 0)
    ctx.run_batch(gpu_problem(p, batch=2))
    ref = oracle.run(p, seed=p.seed, batch=2, n=4000)
    _close(ctx.read_reaction_tally(0), ref["absrate"])
    ctx.reset_tallies()
    assert np.all(ctx.read_reaction_tally(0) == 0)
    ctx.set_reaction_tally(False)
    ctx.run_batch(gp)
    with pytest.raises(gbmc.GbmcError):
        ctx.read_reaction_tally(0)
    ctx.close()
