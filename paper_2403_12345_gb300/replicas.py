"""Domain replication across GPUs: one process per GPU, every table on every
GPU, the particle histories of a job split between the ranks.

Histories are independent (Sec. 2: each particle's random walk is its own),
and the random stream of a history is a counter-based function of
(seed, problem, batch, particle id), so a history runs identically on any
rank.  Splitting the id range therefore reproduces the one-GPU per-particle
outcomes exactly and the tallies up to the order of summation; the only
exchange is one sum of the tally arrays at the end of a batch (Sec. 2 and
Sec. 5 run one MPI rank per GPU with replicated geometry and data).

Everything here is host logic: which ids or problems a rank owns, and the
tally sum through torch.distributed (gloo on the host, NCCL on GPUs).
"""
from __future__ import annotations

import numpy as np


def id_range(first_id: int, n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share of ids [first_id, first_id + n) for `rank` of `world`:
    (first, count).  The first n % world ranks take one id more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if n < 0:
        raise ValueError("negative history count")
    base, extra = divmod(int(n), world)
    first = int(first_id) + rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def balance_problems(sizes, world: int) -> list[int]:
    """Owner rank of each problem: largest problem first to the least loaded
    rank (ties to the lower problem index and the lower rank), so that the
    heaviest rank carries at most the mean load plus one problem."""
    sizes = [int(s) for s in sizes]
    if world < 1:
        raise ValueError("world must be positive")
    load = [0] * world
    owner = [0] * len(sizes)
    for k in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda r: (load[r], r))
        owner[k] = r
        load[r] += sizes[k]
    return owner


def _copy(p):
    return type(p).from_buffer_copy(p)


def shard_problems(probs, rank: int, world: int, by: str = "ids"):
    """The problems (gbmc.Problem structures) that `rank` runs.

    by="ids": every problem, each with its share of the id range (balanced
    for any mix of sizes; every rank holds every problem's tally).
    by="problems": whole problems, placed by `balance_problems`; a problem
    not owned by the rank is absent from its list.
    Returns (list of problems, list of their indices into `probs`)."""
    if by == "ids":
        out = []
        for p in probs:
            q = _copy(p)
            q.first_id, q.n_particles = id_range(p.first_id, p.n_particles, rank, world)
            out.append(q)
        return out, list(range(len(probs)))
    if by == "problems":
        owner = balance_problems([p.n_particles for p in probs], world)
        keep = [k for k in range(len(probs)) if owner[k] == rank]
        return [_copy(probs[k]) for k in keep], keep
    raise ValueError(f"unknown split {by!r}")


def _device_for(group):
    import torch.distributed as dist
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


def allreduce_tallies(flux, counts, weights, group=None):
    """Sum one problem's tallies (flux [cells, bins] float64, scalar counts
    int64 and weights float64) over the ranks; every rank gets the sums."""
    import torch
    import torch.distributed as dist
    dev = _device_for(group)
    f = torch.from_numpy(np.ascontiguousarray(flux, np.float64)).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(weights, np.float64)).to(dev)
    c = torch.from_numpy(np.ascontiguousarray(counts, np.int64)).to(dev)
    for t in (f, w, c):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return f.cpu().numpy(), c.cpu().numpy(), w.cpu().numpy()


def gather_outcomes(outcomes: dict, group=None, dst: int = 0):
    """Per-particle outcome arrays of the ranks' id shares, concatenated in
    rank order (that is, in id order for `id_range` shares) on rank `dst`;
    None on the other ranks."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = [None] * world if rank == dst else None
    dist.gather_object({k: np.asarray(v) for k, v in outcomes.items()}, parts, dst=dst,
                       group=group)
    if rank != dst:
        return None
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def gather_bank(xyz, group=None):
    """The fission banks of the ranks' id shares, concatenated in rank order
    (the one-run bank, when the shares are `id_range` shares): every rank
    gets the whole bank for the next generation."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, np.ascontiguousarray(xyz, np.float64).reshape(-1, 3),
                           group=group)
    return np.concatenate(parts)
