"""Shared helpers of the GPU parity tests: run a problem through the C ABI
and compare with the CPU oracle."""
import numpy as np

import oracle
from paper_2403_12345_gb300 import gbmc

OUTCOME_FIELDS = ("n_coll", "status", "n_flights", "n_draws", "E", "x", "y", "z")
FP64_TALLY_RTOL = 1e-12   # per bin, relative: summation order only


def make_ctx(prob, precisions=(gbmc.FP64,), **options):
    ctx = gbmc.Context(0, **options)
    ctx.load(prob, precisions)
    return ctx


def gpu_problem(prob, geom_index=0, batch=0, first_id=0, n=None, problem_index=0, seed=None):
    g = gbmc.geometry_from(prob.geoms[geom_index])
    n = prob.n_particles[geom_index] if n is None else n
    return gbmc.problem(g, prob.seed if seed is None else seed, n, batch=batch,
                        problem_index=problem_index, first_id=first_id)


def run_gpu(ctx, gp, reset=True):
    if reset:
        ctx.reset_tallies()
    ctx.run_batch(gp)
    flux, counts, weights = ctx.read_tallies(0)
    out = ctx.read_outcomes(0, 0, gp.n_particles)
    return dict(out, flux=flux, counts=counts, weights=weights)


def assert_outcomes_equal(a, b, ids=None, label=""):
    """Per-particle outcomes bit for bit (floats compared as bit patterns)."""
    for k in OUTCOME_FIELDS:
        x, y = np.asarray(a[k]), np.asarray(b[k])
        if ids is not None:
            x = x[ids] if len(x) != len(ids) else x
            y = y[ids] if len(y) != len(ids) else y
        if x.dtype == np.float64:
            same = x.view(np.int64) == y.view(np.int64)
        else:
            same = x == y
        if not same.all():
            i = int(np.argmin(same))
            raise AssertionError(f"{label} outcome {k} differs at {i}: {x[i]!r} vs {y[i]!r} "
                                 f"({(~same).sum()} of {len(same)} differ)")


def assert_tallies_close(gpu, ref, rtol=FP64_TALLY_RTOL, label=""):
    f, r = np.asarray(gpu["flux"]), np.asarray(ref["flux"])
    assert f.shape == r.shape
    zero = r == 0
    assert np.all(f[zero] == 0), f"{label} flux nonzero where the oracle scored nothing"
    rel = np.abs(f[~zero] - r[~zero]) / r[~zero]
    assert rel.size == 0 or rel.max() <= rtol, f"{label} flux rel err {rel.max():.3e} > {rtol}"
    assert np.array_equal(gpu["counts"], ref["counts"]), (label, gpu["counts"], ref["counts"])
    w, rw = np.asarray(gpu["weights"]), np.asarray(ref["weights"])
    nz = rw != 0
    assert np.all(w[~nz] == 0)
    assert np.all(np.abs(w[nz] - rw[nz]) <= rtol * np.abs(rw[nz])), (label, w, rw)
