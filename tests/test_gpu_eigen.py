"""k-eigenvalue mode through the C ABI against the oracle: generations from
the box source and then from the fission bank (the device's own, or one set
from the host), bit-exact per-particle outcomes and fission banks; id shares
of replicas that share one bank; the error paths."""
import numpy as np
import pytest

import oracle
import synth
from paper_2403_12345_gb300 import gbmc

from gpu_helpers import assert_outcomes_equal, make_ctx

pytestmark = pytest.mark.gpu
N = 6007


def _setup(**opts):
    p = synth.make_eigen_lattice(n_particles=N, grid_scale=0.02)
    ctx = make_ctx(p, **opts)
    ctx.load_fission(p.nu, p.f_fis)
    return p, ctx


def _geom(p, bank_source):
    g = gbmc.geometry_from(p.geom)
    if bank_source:
        g.source = gbmc.SRC_BANK
    return g


def _same(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.int64), b.view(np.int64))


@pytest.mark.parametrize("own_bank", [True, False])
def test_generations_match_oracle(own_bank):
    p, ctx = _setup(max_in_flight=2000)
    k, bank = 1.0, None
    for gen in range(3):
        ctx.set_eigen(k, 64)
        if bank is not None:
            if own_bank:
                ctx.set_source_bank(None, N)
            else:
                ctx.set_source_bank(bank, N)
        ctx.reset_tallies()
        ctx.run_batch(gbmc.problem(_geom(p, gen > 0), p.seed, N, batch=gen))
        gbank = ctx.read_bank()
        out = ctx.read_outcomes(0, 0, N)
        eig = dict(nu=p.nu, f_fis=p.f_fis, k_norm=k, max_sites=64)
        if bank is not None:
            eig["bank"] = (bank, N)
        ref = oracle.run(p, seed=p.seed, batch=gen, n=N, eigen=eig)
        assert_outcomes_equal(out, ref, label=f"generation {gen}")
        assert _same(gbank, ref["sites"]), (gen, len(gbank), len(ref["sites"]))
        assert len(gbank) > N // 10
        k = len(gbank) / N * k
        bank = gbank
    ctx.close()


def test_replica_id_shares_share_one_bank():
    p, ctx = _setup()
    ctx.set_eigen(1.0, 64)
    ctx.run_batch(gbmc.problem(_geom(p, False), p.seed, N, batch=0))
    bank = ctx.read_bank()
    ctx.set_eigen(len(bank) / N, 64)
    ctx.set_source_bank(bank, N)
    ctx.run_batch(gbmc.problem(_geom(p, True), p.seed, N, batch=1))
    whole = ctx.read_bank()
    half = N // 2
    parts = []
    for first, n in ((0, half), (half, N - half)):
        ctx.run_batch(gbmc.problem(_geom(p, True), p.seed, n, batch=1, first_id=first))
        parts.append(ctx.read_bank())
    assert _same(np.concatenate(parts), whole)
    ctx.close()


def test_eigen_errors():
    p, ctx = _setup()
    with pytest.raises(gbmc.GbmcError):
        ctx.run_batch(gbmc.problem(_geom(p, True), p.seed, 100))      # no bank yet
    with pytest.raises(gbmc.GbmcError):
        ctx.set_eigen(1.0, 0)                                          # max_sites
    with pytest.raises(gbmc.GbmcError):
        ctx.load_fission(p.nu, p.f_abs * 1.5)                          # f_fis > f_abs
    # a history that banks more sites than allowed flags the run
    ctx.set_eigen(0.05, 1)
    ctx.run_batch(gbmc.problem(_geom(p, False), p.seed, 2000))
    with pytest.raises(gbmc.GbmcError):
        ctx.read_bank()
    ctx.close()
