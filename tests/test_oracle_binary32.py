"""Pins of the oracle's binary32-table mode (a reduced-precision variant of
the lookup; the paper's lookup itself, Sec. 2 "Sorting", is binary64).

What the mode states: each grid energy and cross section is rounded to the
nearest binary32 value; the bracket of E is the largest j <= n-2 with
(double)E_j <= E (an exact comparison: E itself is never rounded for the
search); the interpolation runs in binary32 on E rounded to nearest; the
macroscopic sums accumulate in binary32 in the listed order and are widened
to binary64; the collision compares target = xi Sigma_t (binary64) against
the widened binary32 running sums.

Each expected value below follows from IEEE-754 binary32 arithmetic by hand
(cases whose every rounding is known exactly) or from a brute-force scan, so
that each of these plausible mistakes fails a named test:
  - searching on (float)E instead of comparing (double)E_j <= E
        -> test_search_f32_brute_force_with_rounding_neighbours
  - interpolating on the binary64 E
        -> test_micro_f32_interpolates_on_rounded_energy
  - accumulating the macroscopic sums in binary64
        -> test_macro_f32_accumulates_in_binary32_in_listed_order
  - comparing the target against an unwidened binary32 sum
        -> test_pick_f32_compares_widened_sums
"""
import types
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

U32 = 2.0 ** -24   # binary32 unit roundoff


def _scan_widened(g32, E):
    """Largest j in [0, n-2] with (double)g[j] <= E, by a linear scan."""
    j = 0
    for k in range(len(g32) - 1):
        if float(g32[k]) <= E:
            j = k
    return j


def _ulp32(x):
    x = np.float32(x)
    return float(np.nextafter(x, np.float32(np.inf)) - x)


def test_search_f32_brute_force_with_rounding_neighbours():
    rng = np.random.default_rng(41)
    differs_from_rounded_search = 0
    for n in range(2, 9):
        for _ in range(60):
            g = np.unique(rng.uniform(0.5, 8.0, n).astype(np.float32))
            if len(g) < 2:
                continue
            Es = []
            for v in g:
                w = float(v)
                u = _ulp32(v)
                Es += [w, np.nextafter(w, -np.inf), np.nextafter(w, np.inf),
                       w - 0.25 * u,        # rounds UP to v in binary32, lies below it
                       w + 0.25 * u]        # rounds DOWN to v in binary32, lies above it
            Es += list(rng.uniform(0.0, 9.0, 20))
            for E in Es:
                want = _scan_widened(g, E)
                assert oracle.search_f32(g, E) == want, (g, E)
                if _scan_widened(g, float(np.float32(E))) != want:
                    differs_from_rounded_search += 1
    # the energies that round up onto a grid point are where a search on
    # (float)E would go wrong: the pin must contain such cases
    assert differs_from_rounded_search > 100


def test_micro_f32_interpolates_on_rounded_energy():
    # grid (1, 2), values (1, 3): every step is exact in binary32 for
    # Ef = RN32(E) in [1, 2): Ef - 1 (Sterbenz), / 1, * 2, and
    # 1 + 2 (Ef - 1) = 2 Ef - 1 (a multiple of 2^-23 below 2, of 2^-22 above)
    g = np.array([1.0, 2.0], np.float32)
    s = np.array([1.0, 3.0], np.float32)
    rng = np.random.default_rng(42)
    Es = [1.0 + 1.1 * 2.0 ** -25, 1.0 + 3 * 2.0 ** -25, 1.5 + 0.6 * 2.0 ** -24, 1.0, 1.75]
    Es += list(rng.uniform(1.0, 2.0, 500))
    for E in Es:
        Ef = float(np.float32(E))
        assert oracle.micro_f32(g, s, E) == 2.0 * Ef - 1.0, E
    # E = 1 + 1.1 2^-25 rounds to 1 in binary32, so the value is exactly 1;
    # interpolating on the binary64 E would give 1 + 2.2 2^-25, which rounds
    # to 1 + 2^-23
    assert oracle.micro_f32(g, s, 1.0 + 1.1 * 2.0 ** -25) == 1.0


def test_micro_f32_within_binary32_bound_of_exact_interpolant():
    # exact rational interpolant of the binary32 table at Ef = RN32(E) on the
    # exactly found bracket; six binary32 roundings bound the error
    rng = np.random.default_rng(43)
    for _ in range(40):
        n = int(rng.integers(2, 30))
        g = np.unique(np.exp(rng.uniform(-3, 5, n)).astype(np.float32))
        if len(g) < 2:
            continue
        s = np.exp(rng.uniform(-2, 6, len(g))).astype(np.float32)
        for E in np.exp(rng.uniform(np.log(float(g[0])), np.log(float(g[-1])), 60)):
            j = _scan_widened(g, E)
            Ef = Fraction(float(np.float32(E)))
            g0, g1 = Fraction(float(g[j])), Fraction(float(g[j + 1]))
            s0, s1 = Fraction(float(s[j])), Fraction(float(s[j + 1]))
            exact = s0 + (Ef - g0) / (g1 - g0) * (s1 - s0)
            got = Fraction(oracle.micro_f32(g, s, E))
            assert abs(got - exact) <= 8 * U32 * (abs(s0) + abs(s1)), (g[j], g[j + 1], E)
        # at a grid point the tabulated binary32 value is returned
        for j in range(len(g) - 1):
            assert oracle.micro_f32(g, s, float(g[j])) == float(s[j])


def _flat_problem(terms, f_abs=0.5, precision=1):
    """One material whose nuclides have flat cross sections `terms` (density
    1), listed in the given order; binary32-exact values only."""
    grid = [1e-5, 2e7]
    n = len(terms)
    off = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    energy = np.tile(np.array(grid), n)
    sigma = np.repeat(np.array(terms, dtype=np.float64), 2)
    return types.SimpleNamespace(
        grid_off=off, energy=energy, sigma_t=sigma,
        f_abs=np.full(n, f_abs), awr=np.full(n, 10.0),
        mat_off=np.array([0, n], np.int32), nuc_id=np.arange(n, dtype=np.int32),
        density=np.ones(n), edges=np.geomspace(1e-5, 2e7, 3), precision=precision,
        geoms=[synth.Geometry()], n_particles=[1])


def test_macro_f32_accumulates_in_binary32_in_listed_order():
    h = 2.0 ** -24
    E = np.array([1.0, 3e3, 1e6])
    # listed order 1, h, h: in binary32 1 + 2^-24 ties to 1 (even), twice
    st, sa = oracle.macro(_flat_problem([1.0, h, h]), 0, E, precision=1)
    assert np.all(st == 1.0)
    # Sigma_a: 0.5 + 2^-25 ties to 0.5 (even), twice
    assert np.all(sa == 0.5)
    # listed order h, h, 1: 2^-24 + 2^-24 = 2^-23 exactly, + 1 is representable
    st, sa = oracle.macro(_flat_problem([h, h, 1.0]), 0, E, precision=1)
    assert np.all(st == 1.0 + 2.0 ** -23)
    assert np.all(sa == 0.5 + 2.0 ** -24)
    # the binary64 mode keeps the small terms in either order
    st, sa = oracle.macro(_flat_problem([1.0, h, h]), 0, E, precision=0)
    assert np.all(st == 1.0 + 2.0 ** -23)
    assert np.all(sa == 0.5 + 2.0 ** -24)


def test_pick_f32_compares_widened_sums():
    h = 2.0 ** -24
    p = _flat_problem([1.0, h, h])
    E = 5e4
    # running sums in binary32: 1, 1, 1 (the small terms tie away)
    assert oracle.pick_nuclide(p, 0, E, 0.5, precision=1) == 0
    # 1 - 2^-40 < 1 exactly; rounded to binary32 the target would be 1 and
    # no sum would exceed it (the last positive term's nuclide, 2, would win)
    assert oracle.pick_nuclide(p, 0, E, 1.0 - 2.0 ** -40, precision=1) == 0
    # 1 + 2^-30 exceeds every binary32 running sum: none exceeds the target,
    # so the last nuclide with a positive term is taken; binary64 running
    # sums (1 + 2^-24 after the second) would pick nuclide 1
    assert oracle.pick_nuclide(p, 0, E, 1.0 + 2.0 ** -30, precision=1) == 2
    assert oracle.pick_nuclide(p, 0, E, 1.0 + 2.0 ** -30, precision=0) == 1
    # exactly 1: not below the first sum, and no later binary32 sum exceeds it
    assert oracle.pick_nuclide(p, 0, E, 1.0, precision=1) == 2


@pytest.mark.parametrize("seed", [44, 45])
def test_macro_f32_equals_listed_binary32_sum_of_micro(seed):
    # the macroscopic binary32 sums are the listed-order binary32 sums of the
    # pinned micro values (density and f_abs rounded to binary32)
    p = synth.make_tiny_problem(seed=seed, n_nuc=5, n_points=(3, 40))
    p.mat_off = np.array([0, 5], np.int32)
    p.nuc_id = np.array([3, 0, 4, 1, 2], np.int32)
    p.density = np.random.default_rng(seed).uniform(0.01, 1.0, 5)
    E = np.exp(np.random.default_rng(seed + 1).uniform(np.log(2e-5), np.log(1e7), 300))
    st, sa = oracle.macro(p, 0, E, precision=1)
    for k, e in enumerate(E):
        at = np.float32(0.0)
        aa = np.float32(0.0)
        for q in range(5):
            i = p.nuc_id[q]
            lo, hi = p.grid_off[i], p.grid_off[i + 1]
            sig = np.float32(oracle.micro_f32(p.energy[lo:hi].astype(np.float32),
                                              p.sigma_t[lo:hi].astype(np.float32), e))
            t = np.float32(p.density[q]) * sig
            at = np.float32(at + t)
            aa = np.float32(aa + t * np.float32(p.f_abs[i]))
        assert st[k] == float(at) and sa[k] == float(aa), (k, e)
