"""Concurrent event loops (gbmc_run_concurrent; Sec. 2, "GPU Streams")
through the C ABI: every problem's outcomes and tallies are the oracle's, as
with one event loop, whatever the number of loops and the problems per run;
the counters add up over every run of the call."""
import numpy as np
import pytest

import oracle
import synth
from paper_2403_12345_gb300 import gbmc

from gpu_helpers import assert_outcomes_equal, assert_tallies_close, gpu_problem, make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_loops,per_run", [(2, 1), (3, 2), (4, 1), (1, 3)])
def test_concurrent_loops_match_oracle_per_problem(n_loops, per_run):
    p = synth.make_config(4, n_problems=7, grid_scale=0.02)
    for k in range(7):
        p.n_particles[k] = 1500 + 613 * k
    ctx = make_ctx(p, (gbmc.FP32,), precision=gbmc.FP32)
    try:
        probs = [gpu_problem(p, geom_index=k, problem_index=k, batch=3) for k in range(7)]
        ctx.run_concurrent(probs, n_loops=n_loops, per_run=per_run)
        st = ctx.read_stats()
        colls = flights = 0
        for k in range(7):
            ref = oracle.run(p, seed=p.seed, batch=3, geom_index=k, problem_index=k, precision=1)
            out = ctx.read_outcomes(k, 0, p.n_particles[k])
            assert_outcomes_equal(out, ref, label=f"problem {k}")
            flux, counts, weights = ctx.read_tallies(k)
            assert_tallies_close(dict(flux=flux, counts=counts, weights=weights), ref,
                                 label=f"problem {k}")
            colls += ref["counts"][oracle.S_COLLISION]
            flights += ref["counts"][oracle.S_FLIGHT]
        assert st["histories"] == sum(p.n_particles)
        assert st["collisions"] == colls and st["flights"] == flights
    finally:
        ctx.close()


def test_concurrent_batches_then_one_loop_again():
    # batches of one lattice as separate problems on three loops, each batch
    # tallied in its own slot; then an ordinary run on the same context
    p = synth.make_config(2, grid_scale=0.03)
    ctx = make_ctx(p)
    try:
        probs = [gpu_problem(p, n=9_001, batch=b) for b in range(5)]
        ctx.run_concurrent(probs, n_loops=3)
        for b in range(5):
            ref = oracle.run(p, seed=p.seed, batch=b, n=9_001)
            assert_outcomes_equal(ctx.read_outcomes(b, 0, 9_001), ref, label=f"batch {b}")
            flux, counts, weights = ctx.read_tallies(b)
            assert_tallies_close(dict(flux=flux, counts=counts, weights=weights), ref)
        ctx.reset_tallies()
        ctx.run_batch(gpu_problem(p, n=4_000, batch=9))
        ref = oracle.run(p, seed=p.seed, batch=9, n=4_000)
        assert_outcomes_equal(ctx.read_outcomes(0, 0, 4_000), ref, label="single loop after")
        assert ctx.read_stats()["histories"] == 4_000
    finally:
        ctx.close()


def test_concurrent_refuses_single_loop_features():
    p = synth.make_tiny_problem(seed=37, n_nuc=3, n_points=(10, 50), kind=synth.GEOM_SLAB,
                                n_particles=100)
    ctx = make_ctx(p)
    try:
        ctx.set_weight_windows(np.full((p.geom.n_cells(), p.n_bins), 0.1))
        with pytest.raises(gbmc.GbmcError) as ex:
            ctx.run_concurrent([gpu_problem(p, n=100)], n_loops=2)
        assert ex.value.code == gbmc.ERR_UNSUPPORTED
        ctx.clear_weight_windows()
        with pytest.raises(gbmc.GbmcError) as ex:
            ctx.run_concurrent([gpu_problem(p, n=100)], n_loops=17)
        assert ex.value.code == gbmc.ERR_INVALID_ARG
    finally:
        ctx.close()


@pytest.mark.parametrize("n_loops,pinned", [(3, True), (1, True), (2, False)])
def test_concurrent_results_copied_to_host(n_loops, pinned):
    """gbmc_run_concurrent_to_host: each run's outcomes and tallies reach the
    host arrays (pinned, or pageable) once the stream has passed the call,
    equal to the oracle and to what the synchronous readers return; a
    destination with only some arrays copies only those."""
    import torch
    p = synth.make_config(4, n_problems=5, grid_scale=0.02)
    for k in range(5):
        p.n_particles[k] = 1200 + 517 * k
    ctx = make_ctx(p, (gbmc.FP32,), precision=gbmc.FP32)

    def host(n, dtype):
        if pinned:
            tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32,
                   np.int8: torch.int8, np.uint32: torch.int32}[dtype]
            a = torch.zeros(n, dtype=tdt, pin_memory=True).numpy()
            return a.view(np.uint32) if dtype is np.uint32 else a
        return np.zeros(n, dtype)

    try:
        probs = [gpu_problem(p, geom_index=k, problem_index=k, batch=5) for k in range(5)]
        dests = []
        for k, pr in enumerate(probs):
            nc = gbmc._n_cells(pr.geom)
            n = p.n_particles[k]
            d = dict(flux=host(nc * ctx.n_bins, np.float64), counts=host(gbmc.NSCAL, np.int64),
                     weights=host(gbmc.NSCAL, np.float64))
            if k != 2:   # problem 2: tallies only
                d.update(n_coll=host(n, np.int32), status=host(n, np.int8),
                         n_flights=host(n, np.int32), n_draws=host(n, np.uint32),
                         E=host(n, np.float64), x=host(n, np.float64), y=host(n, np.float64),
                         z=host(n, np.float64))
            dests.append(d)
        stream = torch.cuda.Stream()
        ctx.run_concurrent_to_host(probs, n_loops=n_loops, dests=dests, stream=stream)
        stream.synchronize()
        for k in range(5):
            ref = oracle.run(p, seed=p.seed, batch=5, geom_index=k, problem_index=k, precision=1)
            d = dests[k]
            nc = gbmc._n_cells(probs[k].geom)
            got = dict(flux=d["flux"].reshape(nc, ctx.n_bins), counts=d["counts"],
                       weights=d["weights"])
            assert_tallies_close(got, ref, label=f"problem {k}")
            flux, counts, weights = ctx.read_tallies(k)
            assert np.array_equal(flux.ravel(), d["flux"]) and np.array_equal(counts, d["counts"])
            assert np.array_equal(weights, d["weights"])
            if k != 2:
                assert_outcomes_equal(d, ref, label=f"problem {k}")
        with pytest.raises(TypeError):   # a destination of the wrong size
            bad = [dict(dests[0]) for _ in probs]
            bad[0]["E"] = np.zeros(3)
            ctx.run_concurrent_to_host(probs, n_loops=2, dests=bad)
    finally:
        ctx.close()


def test_adjacent_host_destinations_match_the_readers():
    """Destinations that are slices of one pinned array per field (the case
    the library copies in one piece per field and run) hold what the
    synchronous readers return, with a run split by a destination outside
    the shared array (problem 4's flux and E), a run whose problems skip
    the outcomes of one of them (problem 1) and an empty problem (3)."""
    import torch
    n_prob = 6
    p = synth.make_config(4, n_problems=n_prob, grid_scale=0.02)
    for k in range(n_prob):
        p.n_particles[k] = 900 + 331 * k
    p.n_particles[3] = 0   # an empty problem opening the second run
    ctx = make_ctx(p, (gbmc.FP32,), precision=gbmc.FP32)

    def pinned(n, tdt):
        return torch.full((n,), -7, dtype=tdt, pin_memory=True).numpy()

    try:
        probs = [gpu_problem(p, geom_index=k, problem_index=k, batch=7) for k in range(n_prob)]
        ncs = [gbmc._n_cells(pr.geom) * ctx.n_bins for pr in probs]
        ns = [int(n) for n in p.n_particles[:n_prob]]
        spec = {"flux": (torch.float64, ncs), "counts": (torch.int64, [gbmc.NSCAL] * n_prob),
                "weights": (torch.float64, [gbmc.NSCAL] * n_prob),
                "n_coll": (torch.int32, ns), "status": (torch.int8, ns),
                "n_flights": (torch.int32, ns), "n_draws": (torch.int32, ns),
                "E": (torch.float64, ns), "x": (torch.float64, ns), "y": (torch.float64, ns),
                "z": (torch.float64, ns)}
        dests = [dict() for _ in range(n_prob)]
        wholes = {}
        for name, (tdt, sizes) in spec.items():
            whole = pinned(int(sum(sizes)), tdt)
            if name == "n_draws":
                whole = whole.view(np.uint32)
            wholes[name] = whole
            at = 0
            for k in range(n_prob):
                dests[k][name] = whole[at:at + sizes[k]]
                at += sizes[k]
        dests[4]["flux"] = pinned(ncs[4], torch.float64)
        dests[4]["E"] = pinned(ns[4], torch.float64)
        skipped = ("n_coll", "status", "n_flights", "n_draws", "E", "x", "y", "z")
        for name in skipped:
            del dests[1][name]
        stream = torch.cuda.Stream()
        ctx.run_concurrent_to_host(probs, n_loops=2, dests=dests, per_run=3, stream=stream)
        stream.synchronize()
        for k in range(n_prob):
            d = dests[k]
            flux, counts, weights = ctx.read_tallies(k)
            assert np.array_equal(flux.ravel(), d["flux"]), f"problem {k}: flux"
            assert np.array_equal(counts, d["counts"]) and np.array_equal(weights, d["weights"])
            if k == 1:
                continue
            out = ctx.read_outcomes(k, 0, ns[k])
            for name in skipped:
                assert np.array_equal(out[name], d[name]), f"problem {k}: {name}"
        # problem 1's outcome slices were not written: the fill value is still there
        for name in skipped:
            part = wholes[name][ns[0]:ns[0] + ns[1]]
            if name == "n_draws":
                part = part.view(np.int32)
            assert np.all(part == -7), name
        # problem 4's flux and E went to arrays of their own: its shared slices are untouched
        assert np.all(wholes["E"][sum(ns[:4]):sum(ns[:5])] == -7)
        assert np.all(wholes["flux"][sum(ncs[:4]):sum(ncs[:5])] == -7)
        assert not dests[3]["flux"].any() and not dests[3]["counts"].any()
        ref = oracle.run(p, seed=p.seed, batch=7, geom_index=4, problem_index=4, precision=1)
        assert_outcomes_equal(dests[4], ref, label="problem 4")
    finally:
        ctx.close()


def test_library_host_memory_destinations():
    """Destinations from the library's page-locked allocator (host_array,
    gbmc_host_alloc) receive what the synchronous readers return; the arrays
    are ordinary numpy arrays and are freed with their last view."""
    import gc
    import torch
    p = synth.make_config(4, n_problems=4, grid_scale=0.02)
    for k in range(4):
        p.n_particles[k] = 700 + 211 * k
    ctx = make_ctx(p, (gbmc.FP32,), precision=gbmc.FP32)
    try:
        probs = [gpu_problem(p, geom_index=k, problem_index=k, batch=9) for k in range(4)]
        ns = [int(n) for n in p.n_particles[:4]]
        ncs = [gbmc._n_cells(pr.geom) * ctx.n_bins for pr in probs]
        fields = {"flux": (np.float64, ncs), "counts": (np.int64, [gbmc.NSCAL] * 4),
                  "weights": (np.float64, [gbmc.NSCAL] * 4), "n_coll": (np.int32, ns),
                  "status": (np.int8, ns), "n_flights": (np.int32, ns),
                  "n_draws": (np.uint32, ns), "E": (np.float64, ns), "x": (np.float64, ns),
                  "y": (np.float64, ns), "z": (np.float64, ns)}
        dests = [dict() for _ in range(4)]
        for name, (dt, sizes) in fields.items():
            whole = gbmc.host_array(sum(sizes), dt)
            assert whole.dtype == np.dtype(dt) and whole.size == sum(sizes)
            whole[:] = 0
            at = 0
            for k in range(4):
                dests[k][name] = whole[at:at + sizes[k]]
                at += sizes[k]
        stream = torch.cuda.Stream()
        ctx.run_concurrent_to_host(probs, n_loops=2, dests=dests, per_run=2, stream=stream)
        stream.synchronize()
        for k in range(4):
            flux, counts, weights = ctx.read_tallies(k)
            assert np.array_equal(flux.ravel(), dests[k]["flux"])
            assert np.array_equal(counts, dests[k]["counts"])
            assert np.array_equal(weights, dests[k]["weights"])
            out = ctx.read_outcomes(k, 0, ns[k])
            for name in ("n_coll", "status", "n_flights", "n_draws", "E", "x", "y", "z"):
                assert np.array_equal(out[name], dests[k][name]), (k, name)
        del dests
        gc.collect()
    finally:
        ctx.close()
