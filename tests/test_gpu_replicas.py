"""Domain replication through the C ABI on one GPU: the id shares that
ranks of a replicated job would run, run one after another, give the one-run
per-particle outcomes exactly and, summed, its tallies to summation order."""
import numpy as np
import pytest

import synth
from paper_2403_12345_gb300 import gbmc, replicas

from gpu_helpers import assert_outcomes_equal, gpu_problem, make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
def test_id_shares_reproduce_one_run(world):
    prob = synth.make_config(2, n_particles=20_000, grid_scale=0.02)
    ctx = make_ctx(prob, max_in_flight=4096)
    full = gpu_problem(prob, batch=2)
    ctx.reset_tallies()
    ctx.run_batch(full)
    ref_flux, ref_counts, ref_weights = ctx.read_tallies(0)
    ref = ctx.read_outcomes(0, 0, full.n_particles)

    parts, flux, counts, weights = [], 0.0, 0, 0.0
    for rank in range(world):
        (q,), _ = replicas.shard_problems([full], rank, world)
        ctx.reset_tallies()
        ctx.run_batch(q)
        f, c, w = ctx.read_tallies(0)
        flux, counts, weights = flux + f, counts + c, weights + w
        parts.append(ctx.read_outcomes(0, 0, q.n_particles))
    joined = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    assert_outcomes_equal(joined, ref, label=f"world {world}")
    assert np.array_equal(counts, ref_counts)
    nz = ref_flux > 0
    assert np.all(flux[~nz] == 0)
    assert np.max(np.abs(flux[nz] - ref_flux[nz]) / ref_flux[nz]) <= 1e-12
    nzw = ref_weights != 0
    assert np.all(np.abs(weights[nzw] - ref_weights[nzw]) <= 1e-12 * np.abs(ref_weights[nzw]))
    ctx.close()


def test_problem_shares_reproduce_one_launch():
    prob = synth.make_config(4, grid_scale=0.01, n_problems=6)
    prob.n_particles = [5000, 1200, 300, 2600, 800, 4100]
    ctx = make_ctx(prob, (gbmc.FP32,), precision=gbmc.FP32)
    probs = [gpu_problem(prob, k, batch=1, problem_index=k) for k in range(6)]
    ctx.reset_tallies()
    ctx.run_problems(probs)
    ref = [ctx.read_tallies(k) for k in range(6)]
    ref_out = [ctx.read_outcomes(k, 0, p.n_particles) for k, p in enumerate(probs)]
    seen = []
    for rank in range(2):
        mine, idx = replicas.shard_problems(probs, rank, 2, by="problems")
        ctx.reset_tallies()
        ctx.run_problems(mine)
        for slot, k in enumerate(idx):
            f, c, w = ctx.read_tallies(slot)
            assert np.array_equal(c, ref[k][1]), k
            nz = ref[k][0] > 0
            assert np.all(f[~nz] == 0)
            assert np.max(np.abs(f[nz] - ref[k][0][nz]) / ref[k][0][nz]) <= 1e-12
            assert_outcomes_equal(ctx.read_outcomes(slot, 0, mine[slot].n_particles),
                                  ref_out[k], label=f"problem {k}")
            seen.append(k)
    assert sorted(seen) == list(range(6))
    ctx.close()
