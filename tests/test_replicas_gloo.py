"""Domain replication on the host with gloo ranks (world size 2 and 3).

Each rank runs only its share of the histories and the tallies are summed
with one all-reduce.  The CPU oracle stands in for each rank's GPU run, since
this test runs without a GPU.  The summed result must equal one run over
every id: per-particle outcomes exactly, and tallies to summation order.
"""
import os
import pickle
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2403_12345_gb300 import gbmc, replicas

from gpu_helpers import assert_outcomes_equal, assert_tallies_close

OUT_FIELDS = ("n_coll", "status", "n_flights", "n_draws", "E", "x", "y", "z")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _lattice():
    return synth.make_config(2, n_particles=700, grid_scale=0.02)


def _batched():
    p = synth.make_config(4, grid_scale=0.01, n_problems=4)
    p.n_particles = [260, 90, 41, 150]
    return p


def _problems(prob, batch=3):
    return [gbmc.problem(gbmc.geometry_from(g), prob.seed, prob.n_particles[k], batch=batch,
                         problem_index=k) for k, g in enumerate(prob.geoms)]


def _run(prob, q, k, threads):
    return oracle.run(prob, seed=q.seed, batch=q.batch, first_id=q.first_id, n=q.n_particles,
                      geom_index=k, problem_index=q.problem_index, threads=threads)


def _worker(rank, world, port, which, by, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _lattice() if which == "lattice" else _batched()
        probs = _problems(prob)
        mine, idx = replicas.shard_problems(probs, rank, world, by=by)
        # every rank holds every problem's tally; an unowned one stays zero
        tallies = []
        for k in range(len(probs)):
            nc = oracle.run(prob, seed=1, n=0, geom_index=k)["flux"].shape
            tallies.append([np.zeros(nc), np.zeros(oracle.NSCAL, np.int64),
                            np.zeros(oracle.NSCAL)])
        outcomes = {}
        for q, k in zip(mine, idx):
            r = _run(prob, q, k, threads=1)
            tallies[k] = [r["flux"], r["counts"], r["weights"]]
            outcomes[k] = ({f: r[f] for f in OUT_FIELDS}, q.first_id, q.n_particles)
        summed = [replicas.allreduce_tallies(*t) for t in tallies]
        gathered = None
        if by == "ids":
            gathered = [replicas.gather_outcomes(outcomes[k][0]) for k in range(len(probs))]
        shares = [None] * world if rank == 0 else None
        dist.gather_object({k: (v[1], v[2]) for k, v in outcomes.items()}, shares, dst=0)
        if rank == 0:
            with open(os.path.join(outdir, "result.pkl"), "wb") as f:
                pickle.dump(dict(summed=summed, gathered=gathered, shares=shares), f)
    finally:
        dist.destroy_process_group()


def _spawn(world, which, by, tmp_path):
    mp.spawn(_worker, args=(world, _free_port(), which, by, str(tmp_path)), nprocs=world,
             join=True)
    with open(tmp_path / "result.pkl", "rb") as f:
        return pickle.load(f)


@pytest.mark.parametrize("world", [2, 3])
def test_id_split_equals_one_run(world, tmp_path):
    res = _spawn(world, "lattice", "ids", tmp_path)
    prob = _lattice()
    q = _problems(prob)[0]
    ref = _run(prob, q, 0, threads=None)
    # the shares tile the id range in rank order
    spans = [s[0] for s in res["shares"]]
    assert spans[0][0] == 0 and sum(n for _, n in spans) == q.n_particles
    assert all(a[0] + a[1] == b[0] for a, b in zip(spans, spans[1:]))
    assert_outcomes_equal(res["gathered"][0], ref, label=f"world {world}")
    flux, counts, weights = res["summed"][0]
    assert_tallies_close(dict(flux=flux, counts=counts, weights=weights), ref,
                         label=f"world {world}")
    assert counts[oracle.S_HISTORY] == q.n_particles


def test_problem_split_equals_one_run(tmp_path):
    res = _spawn(2, "batched", "problems", tmp_path)
    prob = _batched()
    probs = _problems(prob)
    owner = replicas.balance_problems(prob.n_particles, 2)
    assert sorted(k for s in res["shares"] for k in s) == list(range(len(probs)))
    for r, s in enumerate(res["shares"]):
        assert all(owner[k] == r for k in s)
    for k, q in enumerate(probs):
        ref = _run(prob, q, k, threads=None)
        flux, counts, weights = res["summed"][k]
        # one owner: the sum adds zeros only, so it is exact
        assert np.array_equal(flux, ref["flux"]) and np.array_equal(counts, ref["counts"])
        assert np.array_equal(weights, ref["weights"])


# ---------------------------------------------------------------- host logic only

@pytest.mark.parametrize("n,world", [(0, 3), (1, 4), (10, 3), (1000, 7), (5, 5), (12, 1)])
def test_id_range_tiles(n, world):
    spans = [replicas.id_range(100, n, r, world) for r in range(world)]
    assert spans[0][0] == 100
    assert all(a[0] + a[1] == b[0] for a, b in zip(spans, spans[1:]))
    assert sum(c for _, c in spans) == n
    assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def test_id_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        replicas.id_range(0, 10, 2, 2)
    with pytest.raises(ValueError):
        replicas.id_range(0, -1, 0, 2)


def test_balance_problems_bound():
    rng = np.random.default_rng(5)
    for world in (2, 3, 4, 8):
        sizes = [int(v) for v in np.exp(rng.uniform(np.log(1e4), np.log(1e6), 64))]
        owner = replicas.balance_problems(sizes, world)
        load = np.zeros(world)
        for k, r in enumerate(owner):
            load[r] += sizes[k]
        assert load.sum() == sum(sizes)
        assert load.max() <= sum(sizes) / world + max(sizes)
        # deterministic
        assert owner == replicas.balance_problems(sizes, world)


def test_shard_problems_copies():
    prob = _batched()
    probs = _problems(prob)
    mine, idx = replicas.shard_problems(probs, 1, 3, by="ids")
    assert idx == list(range(len(probs)))
    for p, q in zip(probs, mine):
        assert (q.first_id, q.n_particles) == replicas.id_range(0, p.n_particles, 1, 3)
        assert q.batch == p.batch and q.problem_index == p.problem_index
    assert probs[0].first_id == 0 and probs[0].n_particles == 260   # inputs untouched
    with pytest.raises(ValueError):
        replicas.shard_problems(probs, 0, 2, by="cells")


# ---------------------------------------------------------------- k-eigenvalue

def _eigen_worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = synth.make_eigen_lattice(n_particles=3000, grid_scale=0.02)
        N = 3000
        first, n = replicas.id_range(0, N, rank, world)
        k, bank, ks = 1.0, None, []
        for gen in range(3):
            eig = dict(nu=p.nu, f_fis=p.f_fis, k_norm=k, max_sites=64)
            if bank is not None:
                eig["bank"] = (bank, N)
            r = oracle.run(p, seed=p.seed, batch=gen, first_id=first, n=n, eigen=eig, threads=1)
            bank = replicas.gather_bank(r["sites"])        # the source-bank exchange
            k = len(bank) / N * k
            ks.append(k)
        if rank == 0:
            with open(os.path.join(outdir, "eigen.pkl"), "wb") as f:
                pickle.dump(dict(ks=ks, bank=bank), f)
    finally:
        dist.destroy_process_group()


def test_eigen_bank_exchange_equals_one_process(tmp_path):
    mp.spawn(_eigen_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    with open(tmp_path / "eigen.pkl", "rb") as f:
        res = pickle.load(f)
    p = synth.make_eigen_lattice(n_particles=3000, grid_scale=0.02)
    k, bank, ks = 1.0, None, []
    for gen in range(3):
        eig = dict(nu=p.nu, f_fis=p.f_fis, k_norm=k, max_sites=64)
        if bank is not None:
            eig["bank"] = (bank, 3000)
        r = oracle.run(p, seed=p.seed, batch=gen, n=3000, eigen=eig)
        bank = r["sites"]
        k = len(bank) / 3000 * k
        ks.append(k)
    assert res["ks"] == ks
    assert np.array_equal(res["bank"], bank)
