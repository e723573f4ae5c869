"""Pins of the oracle's track-length absorption-rate tally (sum of w d Sigma_a
over flight segments, per cell and energy bin)."""
import math

import numpy as np

import oracle
import synth

Z_MAX = 4.5


def test_constant_sigma_a_gives_sigma_a_times_flux():
    # one flat nuclide: Sigma_a is the same on every segment, so the tally is
    # Sigma_a times the track-length flux, bin by bin, up to rounding
    p = synth.make_tiny_problem(seed=41, n_nuc=1, flat=True, f_abs=[0.1], awr=[1.0],
                                n_particles=3000)
    r = oracle.run(p, seed=3, n=3000)
    sa = p.density[0] * p.sigma_t[0] * 0.1
    nz = r["flux"] > 0
    assert nz.sum() > 5
    assert np.all(r["absrate"][~nz] == 0)
    rel = np.abs(r["absrate"][nz] - sa * r["flux"][nz]) / (sa * r["flux"][nz])
    assert rel.max() < 1e-13, rel.max()


def test_no_absorption_scores_nothing():
    p = synth.make_tiny_problem(seed=43, n_nuc=2, flat=True, f_abs=[0.0, 0.0],
                                kind=synth.GEOM_LATTICE, n_particles=500)
    r = oracle.run(p, seed=5, n=500)
    assert r["flux"].sum() > 0
    assert np.all(r["absrate"] == 0)


def test_track_length_absorption_rate_estimates_absorptions():
    # both the absorbed weight and the track-length estimate sum w d Sigma_a
    # estimate the expected absorption per history: their per-batch difference
    # has mean zero
    p = synth.make_tiny_problem(seed=47, n_nuc=3, kind=synth.GEOM_LATTICE, n_particles=2000,
                                lattice_n=3)
    diffs = []
    for b in range(16):
        r = oracle.run(p, seed=9, batch=b, n=2000)
        diffs.append(r["absrate"].sum() - r["weights"][oracle.S_ABSORPTION])
    d = np.array(diffs)
    se = d.std(ddof=1) / math.sqrt(len(d))
    assert abs(d.mean()) < Z_MAX * se, (d.mean(), se)
    # and the estimate is not trivially zero
    assert r["absrate"].sum() > 0.05 * 2000
