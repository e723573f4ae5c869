"""GPU path against the CPU oracle at the workloads' full sizes, in the
launch settings the benchmark uses (autotuned where it autotunes).

  - 17x17 lattice, full grids (68 + 3 nuclides x 10k-60k points), binary64:
    every one of the batch's 1e6 histories bit for bit, tallies to 1e-12;
  - the same lattice with binary32 tables: outcomes against the oracle's
    binary32 mode on the first 1e5 histories, and the binary32 tally error
    against the binary64 oracle over the whole 1e6 batch (L2 relative error
    at most 1e-4);
  - binary32, 1e7 particles per batch: id samples at the start, middle and
    end of the batch;
  - 64 lattices in one launch (binary32 tables of about 0.7 GB): the first
    histories of every problem.

Outcomes are compared bit for bit (Sec. 4.3: event-based and history-based
runs of one method agree up to summation order).
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2403_12345_gb300 import gbmc

from gpu_helpers import assert_outcomes_equal, assert_tallies_close, gpu_problem, make_ctx

pytestmark = pytest.mark.gpu

N_BATCH = 1_000_000
FP32_TALLY_L2_GATE = 1e-4   # binary32 tables against binary64, whole-batch flux


@pytest.fixture(scope="module")
def lattice():
    return synth.make_config(2)


@pytest.fixture(scope="module")
def oracle64(lattice):
    return oracle.run(lattice, seed=lattice.seed, batch=0, n=N_BATCH, precision=0)


def _run(prob, precision, n, autotune=True, **opts):
    ctx = make_ctx(prob, (precision,), precision=precision, **opts)
    try:
        gp = gpu_problem(prob, n=n, batch=0)
        if autotune:
            ctx.autotune([gpu_problem(prob, n=n, batch=40_000)], fraction=0.3)
        ctx.reset_tallies()
        ctx.run_batch(gp)
        flux, counts, weights = ctx.read_tallies(0)
        out = ctx.read_outcomes(0, 0, n)
    finally:
        ctx.close()
    return dict(out, flux=flux, counts=counts, weights=weights)


def test_lattice17_full_grids_binary64_every_history(lattice, oracle64):
    g = _run(lattice, gbmc.FP64, N_BATCH)
    assert_outcomes_equal(g, oracle64, label="17x17 binary64, 1e6")
    assert_tallies_close(g, oracle64, label="17x17 binary64, 1e6")


def test_lattice17_binary32_parity_and_tally_error(lattice, oracle64):
    g = _run(lattice, gbmc.FP32, N_BATCH)
    ref32 = oracle.run(lattice, seed=lattice.seed, batch=0, n=100_000, precision=1)
    assert_outcomes_equal({k: g[k][:100_000] for k in ("n_coll", "status", "n_flights",
                                                        "n_draws", "E", "x", "y", "z")},
                          ref32, label="17x17 binary32, first 1e5")
    f32, f64 = g["flux"], oracle64["flux"]
    l2 = np.linalg.norm(f32 - f64) / np.linalg.norm(f64)
    nz = f64 > 0
    per_bin = np.abs(f32[nz] - f64[nz]) / f64[nz]
    diverged = np.mean((g["n_coll"] != oracle64["n_coll"]) | (g["status"] != oracle64["status"]))
    msg = (f"L2 {l2:.3e}, per-bin median {np.median(per_bin):.2e} p99 "
           f"{np.percentile(per_bin, 99):.2e}, diverged walks {diverged:.4f}")
    print(msg)
    assert l2 <= FP32_TALLY_L2_GATE, msg


def test_lattice17_binary32_1e7_id_samples():
    n = 10_000_000
    p = synth.make_config(3)
    ctx = make_ctx(p, (gbmc.FP32,), precision=gbmc.FP32)
    try:
        ctx.autotune([gpu_problem(p, n=n, batch=40_000)], fraction=0.1)
        ctx.run_batch(gpu_problem(p, n=n, batch=0))
        for first in (0, n // 2 - 7_777, n - 20_000):
            out = ctx.read_outcomes(0, first, 20_000)
            ref = oracle.run(p, seed=p.seed, batch=0, first_id=first, n=20_000, precision=1)
            assert_outcomes_equal(out, ref, label=f"1e7 batch, ids {first}..")
        st = ctx.read_stats()
        assert st["histories"] == n
    finally:
        ctx.close()


def test_batched_64_lattices_first_histories_of_every_problem():
    p = synth.make_config(4)
    ctx = make_ctx(p, (gbmc.FP32,), precision=gbmc.FP32)
    try:
        probs = [gpu_problem(p, geom_index=k, problem_index=k, batch=0) for k in range(64)]
        ctx.autotune([gpu_problem(p, geom_index=k, problem_index=k, batch=40_000)
                      for k in range(64)], fraction=0.1)
        ctx.run_problems(probs)
        for k in range(64):
            m = min(2_000, p.n_particles[k])
            out = ctx.read_outcomes(k, 0, m)
            ref = oracle.run(p, seed=p.seed, batch=0, n=m, geom_index=k, problem_index=k,
                             precision=1)
            assert_outcomes_equal(out, ref, label=f"problem {k}")
    finally:
        ctx.close()
