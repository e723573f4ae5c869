"""GPU path vs the CPU oracle, through the C ABI.

Per-particle outcomes (collisions, fate, flights, draws, final energy and
position) must match bit for bit in the binary64 mode and in the binary32
table mode against the oracle run in the same precision; tallies must match
to summation order (1e-12 per bin, counts exactly).
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2403_12345_gb300 import gbmc

from gpu_helpers import (assert_outcomes_equal, assert_tallies_close, gpu_problem, make_ctx,
                         run_gpu)

pytestmark = pytest.mark.gpu


def _parity(prob, n, precision=gbmc.FP64, batch=0, **options):
    ctx = make_ctx(prob, (precision,), precision=precision, **options)
    try:
        gp = gpu_problem(prob, n=n, batch=batch)
        g = run_gpu(ctx, gp)
        stats = ctx.read_stats()
    finally:
        ctx.close()
    ref = oracle.run(prob, seed=prob.seed, batch=batch, n=n, precision=precision)
    assert_outcomes_equal(g, ref)
    assert_tallies_close(g, ref)
    return g, ref, stats


def test_infinite_medium_parity():
    p = synth.make_config(1)
    g, ref, st = _parity(p, 100_000)
    assert st["histories"] == 100_000
    assert st["collisions"] == ref["counts"][oracle.S_COLLISION]


def test_lattice_parity_with_refill_and_ragged_tail():
    p = synth.make_config(2, grid_scale=0.05)
    # in-flight cap far below the batch: many refills; 20011 is not a
    # multiple of any block or warp size
    g, ref, st = _parity(p, 20_011, max_in_flight=3_000, batch=4)
    assert st["iterations"] > 10
    assert st["flights"] == ref["counts"][oracle.S_FLIGHT]


def test_lattice_fp32_tables_parity_and_error_vs_fp64():
    p = synth.make_config(3, grid_scale=0.05)
    g, ref32, _ = _parity(p, 20_000, precision=gbmc.FP32)
    ref64 = oracle.run(p, seed=p.seed, n=20_000, precision=0)
    rel = np.linalg.norm(g["flux"] - ref64["flux"]) / np.linalg.norm(ref64["flux"])
    assert rel < 1e-2


def test_drained_warps_hand_particles_on():
    # one batch far larger than a warp's share: warps drain, and the particles
    # they hand to the next iteration end exactly as in the oracle
    p = synth.make_config(2, grid_scale=0.05)
    g, ref, st = _parity(p, 30_000)
    assert st["handoffs"] > 0
    assert st["flights"] == ref["counts"][oracle.S_FLIGHT]


def test_lattice_fp32_sparse_windows_parity():
    # the binary32 lookup's 32-byte window loads give the same results
    p = synth.make_config(3, grid_scale=0.05)
    _parity(p, 20_000, precision=gbmc.FP32, sparse_windows=1)


def test_slab_parity():
    p = synth.make_tiny_problem(seed=31, n_nuc=4, n_points=(20, 200), kind=synth.GEOM_SLAB,
                                n_particles=20_000)
    _parity(p, 20_000)


def test_all_reflective_lattice_parity():
    p = synth.make_tiny_problem(seed=32, n_nuc=4, n_points=(50, 300), kind=synth.GEOM_LATTICE,
                                lattice_n=4, n_particles=10_000)
    p.geom.bc_z = synth.BC_REFLECT
    _parity(p, 10_000)


def test_vacuum_sides_lattice_parity():
    p = synth.make_tiny_problem(seed=33, n_nuc=5, n_points=(50, 300), kind=synth.GEOM_LATTICE,
                                lattice_n=5, n_particles=10_000)
    p.geom.bc_side = synth.BC_VACUUM
    _parity(p, 10_000)


@pytest.mark.parametrize("precision", [gbmc.FP64, gbmc.FP32])
def test_thread_and_warp_lookup_modes_agree_with_oracle(precision):
    p = synth.make_config(2, grid_scale=0.05)
    ref = oracle.run(p, seed=p.seed, n=30_000, precision=precision)
    for wmax in (-1, 1 << 30):   # never / always one warp per particle
        ctx = make_ctx(p, (precision,), precision=precision, warp_lookup_max=wmax)
        try:
            g = run_gpu(ctx, gpu_problem(p, n=30_000))
        finally:
            ctx.close()
        assert_outcomes_equal(g, ref, label=f"warp_lookup_max={wmax}")
        assert_tallies_close(g, ref)


@pytest.mark.parametrize("precision,sparse", [(gbmc.FP64, 0), (gbmc.FP32, 0), (gbmc.FP32, 1)])
def test_lookup_modes_on_a_150_nuclide_material(precision, sparse):
    """More nuclides than the warp-mode lookup's four lock-step rounds of 32
    (a second pass of rounds, a ragged last round, every checkpoint), with
    the absorption-rate tally on (the Sigma_a sums): thread, warp and tail
    lookups against the oracle."""
    p = synth.make_tiny_problem(seed=41, n_nuc=150, n_points=(20, 120), n_particles=3000)
    ref = oracle.run(p, seed=p.seed, n=3000, precision=precision)
    for wmax, tmax in ((-1, -1), (1 << 30, -1), (-1, 1 << 22)):
        ctx = make_ctx(p, (precision,), precision=precision, warp_lookup_max=wmax,
                       tail_max=tmax, sparse_windows=sparse)
        try:
            ctx.set_reaction_tally(True)
            g = run_gpu(ctx, gpu_problem(p, n=3000))
            ra = ctx.read_reaction_tally(0)
        finally:
            ctx.close()
        label = f"warp_lookup_max {wmax}, tail_max {tmax}"
        assert_outcomes_equal(g, ref, label=label)
        assert_tallies_close(g, ref, label=label)
        zero = ref["absrate"] == 0
        assert ref["absrate"].sum() > 0 and np.all(ra[zero] == 0), label
        rel = np.abs(ra[~zero] - ref["absrate"][~zero]) / ref["absrate"][~zero]
        assert rel.max() <= 1e-12, (label, rel.max())


@pytest.mark.parametrize("tail_max", [-1, 4096, 1 << 22])
def test_tail_kernel_threshold_does_not_change_outcomes(tail_max):
    # -1: the event loop runs to the end; 1 << 22: once the source is
    # exhausted every particle still in flight is finished by the tail kernel
    p = synth.make_config(2, grid_scale=0.05)
    g, ref, st = _parity(p, 40_000, max_in_flight=12_000, tail_max=tail_max, batch=2)
    assert st["flights"] == ref["counts"][oracle.S_FLIGHT]
    assert st["collisions"] == ref["counts"][oracle.S_COLLISION]
    assert st["histories"] == 40_000


def test_sort_does_not_change_outcomes():
    p = synth.make_config(2, grid_scale=0.05)
    res = []
    for sort in (1, -1):
        ctx = make_ctx(p, sort=sort)
        try:
            res.append(run_gpu(ctx, gpu_problem(p, n=30_000)))
        finally:
            ctx.close()
    assert_outcomes_equal(res[0], res[1], label="sort on/off")
    assert_tallies_close(res[0], res[1])


def test_in_flight_cap_one_and_empty_batch():
    p = synth.make_tiny_problem(seed=34, n_nuc=3, n_points=(10, 50), n_particles=50)
    ctx = make_ctx(p, max_in_flight=1)
    try:
        g = run_gpu(ctx, gpu_problem(p, n=50))
        ref = oracle.run(p, seed=p.seed, n=50)
        assert_outcomes_equal(g, ref)
        assert_tallies_close(g, ref)
        g0 = run_gpu(ctx, gpu_problem(p, n=0))
        assert g0["flux"].sum() == 0 and g0["counts"].sum() == 0
    finally:
        ctx.close()


def test_id_subset_and_batches_accumulate():
    p = synth.make_config(2, grid_scale=0.02)
    ctx = make_ctx(p)
    try:
        ctx.reset_tallies()
        for b in range(3):
            ctx.run_batch(gpu_problem(p, n=4000, first_id=1000, batch=b))
            out = ctx.read_outcomes(0, 0, 4000)
            ref = oracle.run(p, seed=p.seed, batch=b, first_id=1000, n=4000)
            assert_outcomes_equal(out, ref, label=f"batch {b}")
        flux, counts, _ = ctx.read_tallies(0)
    finally:
        ctx.close()
    tot = sum(oracle.run(p, seed=p.seed, batch=b, first_id=1000, n=4000)["flux"] for b in range(3))
    nz = tot > 0
    assert np.all(np.abs(flux[nz] - tot[nz]) <= 1e-12 * tot[nz])
    assert counts[oracle.S_HISTORY] == 12_000


def test_multi_problem_run_matches_single_runs():
    p = synth.make_config(4, n_problems=5, n_particles=3000, grid_scale=0.02)
    ctx = make_ctx(p, (gbmc.FP32,), precision=gbmc.FP32, max_in_flight=5000)
    try:
        probs = [gpu_problem(p, geom_index=k, n=3000 + 7 * k, problem_index=k, batch=2)
                 for k in range(5)]
        ctx.reset_tallies()
        ctx.run_problems(probs)
        for k in range(5):
            ref = oracle.run(p, seed=p.seed, batch=2, n=3000 + 7 * k, geom_index=k,
                             problem_index=k, precision=1)
            out = ctx.read_outcomes(k, 0, 3000 + 7 * k)
            assert_outcomes_equal(out, ref, label=f"problem {k}")
            flux, counts, weights = ctx.read_tallies(k)
            assert_tallies_close(dict(flux=flux, counts=counts, weights=weights), ref)
    finally:
        ctx.close()


def test_autotuned_batched_run_matches_oracle():
    p = synth.make_config(4, n_problems=6, grid_scale=0.02)
    for k in range(6):
        p.n_particles[k] = 2000 + 997 * k
    ctx = make_ctx(p, (gbmc.FP32,), precision=gbmc.FP32)
    try:
        probs = [gpu_problem(p, geom_index=k, problem_index=k, batch=1) for k in range(6)]
        rep = ctx.autotune(probs, fraction=0.5)
        assert rep["trials"] >= 10 and rep["best_ms"] <= rep["default_ms"]
        ctx.run_problems(probs)
        for k in range(6):
            ref = oracle.run(p, seed=p.seed, batch=1, geom_index=k, problem_index=k,
                             precision=1)
            out = ctx.read_outcomes(k, 0, p.n_particles[k])
            assert_outcomes_equal(out, ref, label=f"problem {k}")
            flux, counts, weights = ctx.read_tallies(k)
            assert_tallies_close(dict(flux=flux, counts=counts, weights=weights), ref)
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", [gbmc.FP64, gbmc.FP32])
@pytest.mark.parametrize("sort", [False, True])
def test_lookup_macro_matches_oracle(precision, sort):
    import torch
    prob, E, mat = synth.make_stress_lookup(n_queries=20_011, n_nuc=40, n_in_mat=30,
                                            n_points=3000)
    mat[::3] = 1
    ctx = make_ctx(prob, (precision,))
    try:
        dE = torch.tensor(E, device="cuda")
        dm = torch.tensor(mat, device="cuda")
        st = torch.empty_like(dE)
        sa = torch.empty_like(dE)
        ctx.lookup_macro(dE, dm, st, sa, precision=precision, sort=sort)
        torch.cuda.synchronize()
        st, sa = st.cpu().numpy(), sa.cpu().numpy()
    finally:
        ctx.close()
    for m in (0, 1):
        sel = mat == m
        rt, ra = oracle.macro(prob, m, E[sel], precision=precision)
        assert np.array_equal(st[sel].view(np.int64), rt.view(np.int64))
        assert np.array_equal(sa[sel].view(np.int64), ra.view(np.int64))


def _edge_energies(prob, mat):
    """Every grid point of the material's nuclides, one ulp either side,
    interval midpoints, and energies below and above every grid."""
    pts = []
    for q in range(prob.mat_off[mat], prob.mat_off[mat + 1]):
        i = prob.nuc_id[q]
        g = prob.energy[prob.grid_off[i]:prob.grid_off[i + 1]]
        pts += [g, np.nextafter(g, 0.0), np.nextafter(g, np.inf), 0.5 * (g[1:] + g[:-1])]
    E = np.concatenate(pts + [np.array([1e-9, 1e-7, 3e7, 1e9])])
    return np.ascontiguousarray(E[E > 0.0])


def _clustered_problem():
    """Grids with tight clusters of points (30 within a relative width of
    3e-4) beside log-spaced points: coarse-index buckets that hold many
    points, so the window searches fall back to bisection there."""
    base = synth.make_tiny_problem(seed=13, n_nuc=4, n_points=(40, 80))
    en, sg, off = [], [], [0]
    rng = np.random.default_rng(5)
    for i in range(base.n_nuc):
        c = float(np.exp(rng.uniform(np.log(1.0), np.log(1e5))))
        e = np.concatenate([np.geomspace(1e-5, 2e7, 50), c * (1.0 + 1e-5 * np.arange(30))])
        e = synth.problem._grid(e)
        en.append(e)
        sg.append(rng.uniform(1.0, 50.0, len(e)))
        off.append(off[-1] + len(e))
    import dataclasses
    return dataclasses.replace(base, grid_off=np.array(off, np.int64), energy=np.concatenate(en),
                               sigma_t=np.concatenate(sg))


# short windows are a binary32 form
@pytest.mark.parametrize("precision,form", [(gbmc.FP64, "index"), (gbmc.FP64, "plain"),
                                            (gbmc.FP32, "index"), (gbmc.FP32, "plain"),
                                            (gbmc.FP32, "sparse")])
@pytest.mark.parametrize("which", ["dense", "sparse", "clustered"])
def test_lookup_macro_at_grid_points_and_edges(precision, which, form):
    """Exact hits (E - E_k = 0), neighbours, extrapolation outside the grids;
    dense grids take the integer-unit interpolation, the sparse ones (2-9
    points over 12 decades: intervals wider than 2^10) its binary64 fallback,
    the clustered ones the window searches' bisection fallback.  Forms: the
    coarse index, a plain binary search, and (binary32) the short windows."""
    import torch
    if which == "dense":
        prob, _, _ = synth.make_stress_lookup(n_queries=1, n_nuc=12, n_in_mat=8, n_points=400)
    elif which == "sparse":
        prob = synth.make_tiny_problem(seed=11, n_nuc=6, n_points=(2, 9))
    else:
        prob = _clustered_problem()
    E = _edge_energies(prob, 0)
    opts = {"index": dict(search=1), "plain": dict(search=-1),
            "sparse": dict(search=1, sparse_windows=1)}[form]
    ctx = make_ctx(prob, (precision,), **opts)
    try:
        dE = torch.tensor(E, device="cuda")
        dm = torch.zeros(len(E), dtype=torch.int32, device="cuda")
        st = torch.empty_like(dE)
        sa = torch.empty_like(dE)
        ctx.lookup_macro(dE, dm, st, sa, precision=precision)
        torch.cuda.synchronize()
        st, sa = st.cpu().numpy(), sa.cpu().numpy()
    finally:
        ctx.close()
    rt, ra = oracle.macro(prob, 0, E, precision=precision)
    assert np.array_equal(st.view(np.int64), rt.view(np.int64))
    assert np.array_equal(sa.view(np.int64), ra.view(np.int64))


def test_invalid_inputs_rejected_before_launch():
    p = synth.make_tiny_problem(seed=35, n_nuc=2, n_points=(5, 9))
    ctx = gbmc.Context(0)
    try:
        e = p.energy.copy()
        e[2] = e[1]
        with pytest.raises(gbmc.GbmcError) as ex:
            ctx.load_xs_tables(p.grid_off, e, p.sigma_t, p.f_abs, p.awr)
        assert ex.value.code == gbmc.ERR_INVALID_ARG
        s = p.sigma_t.copy()
        s[0] = -1.0
        with pytest.raises(gbmc.GbmcError):
            ctx.load_xs_tables(p.grid_off, p.energy, s, p.f_abs, p.awr)
        e = p.energy.copy()
        e[1] = np.nextafter(e[0], np.inf)   # distinct in binary64, equal in binary32
        with pytest.raises(gbmc.GbmcError):
            ctx.load_xs_tables(p.grid_off, e, p.sigma_t, p.f_abs, p.awr, gbmc.FP32)
        with pytest.raises(gbmc.GbmcError) as ex:
            ctx.run_batch(gpu_problem(p, n=10))
        assert ex.value.code == gbmc.ERR_NOT_INITIALIZED
        ctx.load(p)
        with pytest.raises(gbmc.GbmcError):
            ctx.init_materials([0, 2], [0, 7], [0.5, 0.5])
        g = gpu_problem(p, n=10)
        g.geom.E0 = 3e7   # above every grid
        with pytest.raises(gbmc.GbmcError):
            ctx.run_batch(g)
        with pytest.raises(gbmc.GbmcError) as ex:
            ctx.set_options(precision=gbmc.FP32)
            ctx.run_batch(gpu_problem(p, n=10))
        assert ex.value.code == gbmc.ERR_NOT_INITIALIZED
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", [gbmc.FP64, gbmc.FP32])
def test_lookup_macro_material_out_of_range_gives_nan(precision):
    import torch
    prob, E, mat = synth.make_stress_lookup(n_queries=4099, n_nuc=20, n_in_mat=12, n_points=500)
    mat[1::5] = 1
    bad = np.arange(2, len(mat), 7)
    mat[bad] = np.array([-1, 2, 1 << 30, -(1 << 31)], np.int32)[np.arange(len(bad)) % 4]
    ctx = make_ctx(prob, (precision,))
    try:
        for sort in (False, True):
            dE = torch.tensor(E, device="cuda")
            dm = torch.tensor(mat, device="cuda")
            st = torch.zeros_like(dE)
            sa = torch.zeros_like(dE)
            ctx.lookup_macro(dE, dm, st, sa, precision=precision, sort=sort)
            torch.cuda.synchronize()
            st, sa = st.cpu().numpy(), sa.cpu().numpy()
            assert np.isnan(st[bad]).all() and np.isnan(sa[bad]).all()
            for m in (0, 1):
                sel = mat == m
                rt, ra = oracle.macro(prob, m, E[sel], precision=precision)
                assert np.array_equal(st[sel].view(np.int64), rt.view(np.int64)), sort
                assert np.array_equal(sa[sel].view(np.int64), ra.view(np.int64)), sort
        out = torch.zeros_like(dE)
        with pytest.raises(TypeError):   # int64 material ids are refused by the binding
            ctx.lookup_macro(dE, dm.to(torch.int64), out, out)
    finally:
        ctx.close()


@pytest.mark.parametrize("sizes", [(17, 9), (5, 1), (8, 3), (2, 16), (4, 7), (40, 33)])
@pytest.mark.parametrize("reaction", [False, True])
@pytest.mark.parametrize("mode", ["thread", "group"])
def test_sorted_thread_lookups_every_group_size(sizes, reaction, mode):
    """Every lookup sorted, in thread mode (the nuclide-major tile of the
    binary64 lookup) or in group mode (four lanes per particle), on materials
    whose nuclide counts leave partial groups of every size (more than one
    32-nuclide group of the group mode too); ragged chunk tails; with and
    without Sigma_a (the absorption-rate tally); the collision's nuclide
    choice from the checkpoints the lookup stored."""
    a, b = sizes
    p = synth.make_tiny_problem(seed=36 + a, n_nuc=a + b, n_points=(200, 3000),
                                kind=synth.GEOM_LATTICE, lattice_n=6, n_particles=20_011)
    rng = np.random.default_rng(a * 100 + b)
    p.mat_off = np.array([0, a, a + b], np.int32)
    p.nuc_id = np.concatenate([rng.permutation(a), a + rng.permutation(b)]).astype(np.int32)
    p.density = rng.uniform(0.01, 1.0, a + b)
    ctx = make_ctx(p, warp_lookup_max=-1, sort_min=1, tail_max=-1, max_in_flight=7_001,
                   group_lookup_max=(1 << 30) if mode == "group" else -1)
    try:
        if reaction:
            ctx.set_reaction_tally(True)
        g = run_gpu(ctx, gpu_problem(p, n=20_011, batch=3))
        ar = ctx.read_reaction_tally(0) if reaction else None
    finally:
        ctx.close()
    ref = oracle.run(p, seed=p.seed, batch=3, n=20_011)
    assert_outcomes_equal(g, ref, label=f"materials {sizes}")
    assert_tallies_close(g, ref)
    if reaction:
        assert_tallies_close(dict(flux=ar, counts=ref["counts"], weights=ref["weights"]),
                             dict(flux=ref["absrate"], counts=ref["counts"],
                                  weights=ref["weights"]))


@pytest.mark.parametrize("precision", [gbmc.FP64, gbmc.FP32])
@pytest.mark.parametrize("wmax", [-1, 1 << 30])
def test_plain_binary_search_transport_matches_oracle(precision, wmax):
    """The plain binary search of each grid (search = -1, no coarse index
    and no bucket windows) finds the same brackets: sorted thread-mode
    lookups (the binary64 tile included) and warp-mode ones."""
    p = synth.make_config(2, grid_scale=0.05)
    ctx = make_ctx(p, (precision,), precision=precision, search=-1, warp_lookup_max=wmax)
    try:
        g = run_gpu(ctx, gpu_problem(p, n=30_011, batch=6))
    finally:
        ctx.close()
    ref = oracle.run(p, seed=p.seed, batch=6, n=30_011, precision=precision)
    assert_outcomes_equal(g, ref, label=f"plain search, warp_lookup_max {wmax}")
    assert_tallies_close(g, ref)
