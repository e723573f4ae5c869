"""Pins of the oracle's k-eigenvalue mode: fission sites banked at
collisions (expected w nu sigma_f / sigma_t / k_norm per collision) and
histories started from the bank by systematic sampling."""
import math

import numpy as np

import oracle
import synth

Z_MAX = 4.5


def _medium(f_abs=0.4, n=4000, seed=41):
    return synth.make_tiny_problem(seed=seed, n_nuc=1, flat=True, f_abs=[f_abs], awr=[1.0],
                                   n_particles=n)


def test_integer_yield_banks_exactly_that_many_sites():
    # nu f_fis / k_norm = 2 exactly: every collision banks two sites
    p = _medium()
    r = oracle.run(p, seed=5, n=4000, eigen=dict(nu=[2.0], f_fis=[0.4], k_norm=0.4,
                                                  max_sites=255))
    assert np.array_equal(r["n_sites"], 2 * r["n_coll"])
    assert len(r["sites"]) == r["n_sites"].sum()


def test_no_fission_banks_nothing_and_keeps_the_walk():
    p = _medium()
    a = oracle.run(p, seed=5, n=2000)
    b = oracle.run(p, seed=5, n=2000, eigen=dict(nu=[2.5], f_fis=[0.0], k_norm=1.0,
                                                  max_sites=8))
    assert b["n_sites"].sum() == 0
    # the banking draw shifts the stream, so only the collision counts'
    # distribution is comparable: same mean within statistics
    assert abs(a["n_coll"].mean() - b["n_coll"].mean()) < 0.1 * a["n_coll"].mean()


def test_sites_per_collision_and_k_infinity():
    # one flat nuclide in an infinite medium: a history collides 1 / f_abs
    # times on average and each collision banks nu f_fis / k_norm sites on
    # average, so sites per history estimate k_inf / k_norm = nu f_fis / f_abs / k_norm
    nu, ff, fa, kn = 2.5, 0.3, 0.4, 1.25
    p = _medium(f_abs=fa)
    per_batch, s_tot, c_tot = [], 0, 0
    for b in range(10):
        r = oracle.run(p, seed=7, batch=b, n=4000,
                       eigen=dict(nu=[nu], f_fis=[ff], k_norm=kn, max_sites=64))
        per_batch.append(r["n_sites"].mean())
        s_tot += int(r["n_sites"].sum())
        c_tot += int(r["n_coll"].sum())
    # per collision: 0 or 1 site with probability 0.6 (binomial)
    q = nu * ff / kn
    assert abs(s_tot - q * c_tot) < Z_MAX * math.sqrt(c_tot * q * (1 - q))
    x = np.array(per_batch)
    se = x.std(ddof=1) / math.sqrt(len(x))
    assert abs(x.mean() - nu * ff / fa / kn) < Z_MAX * se, (x.mean(), se)


def test_bank_source_starts_at_systematic_sites():
    p = synth.make_eigen_lattice(n_particles=10, grid_scale=0.02)
    bank = np.array([[0.3, 0.4, 10.0], [5.05, 7.2, 55.5], [20.0, 1.0, 99.0]])
    eig = dict(nu=p.nu, f_fis=p.f_fis, k_norm=1.0, max_sites=32, bank=(bank, 7))
    for i in range(7):
        st, cell = oracle.birth_state(p, p.seed, i, eigen=eig)
        s = i * 3 // 7
        assert tuple(st[:3]) == tuple(bank[s])
        assert st[6] == p.geom.E0
        pitch = p.geom.pitch
        assert cell[0] == min(int(bank[s][0] // pitch), p.geom.n - 1)
        assert cell[1] == min(int(bank[s][1] // pitch), p.geom.n - 1)
        assert abs(math.hypot(st[3], math.hypot(st[4], st[5])) - 1) < 1e-14


def test_power_iteration_renormalises_the_bank():
    # with k_norm the previous generation's estimate the bank stays near the
    # source size
    p = synth.make_eigen_lattice(n_particles=5000, grid_scale=0.02)
    k, src = 1.0, None
    sizes = []
    for g in range(5):
        eig = dict(nu=p.nu, f_fis=p.f_fis, k_norm=k, max_sites=64)
        if src is not None:
            eig["bank"] = (src, 5000)
        r = oracle.run(p, seed=p.seed, batch=g, n=5000, eigen=eig)
        sizes.append(len(r["sites"]))
        k = len(r["sites"]) / 5000 * k
        src = r["sites"]
    assert all(0.8 * 5000 < s < 1.25 * 5000 for s in sizes[2:]), sizes
