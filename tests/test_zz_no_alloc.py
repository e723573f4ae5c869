"""The allocation-free sorted lookup (gbmc_lookup_macro_noalloc) against the
allocating one (gbmc_lookup_macro with sort = 1), through the C ABI.

It serves callers that cannot allocate device memory during the call: its
scratch is a fixed area in the library.  Two calls in a row, on different
queries, must each reproduce the allocating entry point's results exactly,
so the shared scratch carries nothing wrong from one call to the next; a call
at exactly the size limit uses the whole area.  This file is collected last.
"""
import numpy as np
import pytest

import synth
from paper_2403_12345_gb300 import gbmc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [gbmc.FP64, gbmc.FP32])
def test_noalloc_lookup_matches_allocating_lookup(precision):
    import torch
    prob, E, mat = synth.make_stress_lookup(n_queries=300_007, n_nuc=40, n_in_mat=30,
                                            n_points=3000)
    mat[::3] = 1
    rng = np.random.default_rng(5)
    ctx = gbmc.Context(0)
    try:
        ctx.load(prob, (precision,))
        for call in range(2):
            perm = rng.permutation(len(E))[: len(E) - 1000 * call]
            dE = torch.tensor(E[perm], device="cuda")
            dm = torch.tensor(mat[perm], device="cuda")
            ref_t, ref_a = torch.empty_like(dE), torch.empty_like(dE)
            ctx.lookup_macro(dE, dm, ref_t, ref_a, precision=precision, sort=True)
            out_t = torch.full_like(dE, float("nan"))
            out_a = torch.full_like(dE, float("nan"))
            ctx.lookup_macro_noalloc(dE, dm, out_t, out_a, precision=precision)
            torch.cuda.synchronize()
            # tolerance of the lookup tests: bit for bit
            assert torch.equal(out_t.view(torch.int64), ref_t.view(torch.int64)), call
            assert torch.equal(out_a.view(torch.int64), ref_a.view(torch.int64)), call
        # exactly the limit: every entry of the scratch in use
        nmax = gbmc.NOALLOC_MAX_QUERIES
        idx = rng.integers(0, len(E), nmax)
        dE = torch.tensor(E[idx], device="cuda")
        dm = torch.tensor(mat[idx], device="cuda")
        ref_t, ref_a = torch.empty_like(dE), torch.empty_like(dE)
        ctx.lookup_macro(dE, dm, ref_t, ref_a, precision=precision, sort=True)
        out_t, out_a = torch.full_like(dE, float("nan")), torch.full_like(dE, float("nan"))
        ctx.lookup_macro_noalloc(dE, dm, out_t, out_a, precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(out_t.view(torch.int64), ref_t.view(torch.int64))
        assert torch.equal(out_a.view(torch.int64), ref_a.view(torch.int64))
        # one more than the limit is refused before any launch
        big = torch.zeros(nmax + 1, dtype=torch.float64, device="cuda")
        bigm = torch.zeros(nmax + 1, dtype=torch.int32, device="cuda")
        with pytest.raises(gbmc.GbmcError) as ex:
            ctx.lookup_macro_noalloc(big, bigm, big, big, precision=precision)
        assert ex.value.code == gbmc.ERR_INVALID_ARG
    finally:
        ctx.close()
