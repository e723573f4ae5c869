"""Seeded synthetic problem descriptions (data only, no transport arithmetic).

Recipe (paper silent on all of it; the paper's own problems need evaluated
nuclear data that is not available):

* energy grid of a nuclide: endpoints 1e-5 eV and 2e7 eV; either log-spaced
  (the infinite-medium configuration) or n-2 sorted log-uniform interior
  points, kept as binary64 values.  An interior point whose nearest binary32
  value equals the previous point's is dropped (and one equal to the last
  point's), so the binary32 copy of the tables (each value rounded to
  nearest) is strictly increasing too;
* sigma_t(E) = a / sqrt(E) + sum_k h_k (G_k/2)^2 / ((E - E_k)^2 + (G_k/2)^2)
  with a log-uniform in [1, 1e3] b eV^1/2, E_k log-uniform in [1, 1e5] eV,
  h_k log-uniform in [10, 1e4] b, G_k = E_k g_k with g_k log-uniform in
  [1e-4, 1e-2]; the analytic form only generates the table, the table
  (interpolated lin-lin) is the cross section;
* absorption fraction f (sigma_a = f sigma_t) uniform in [0.05, 0.5],
  atomic-weight ratio A uniform in [1, 240], densities uniform in [0.01, 1]
  atoms/(b cm);
* tally energy bins: log-spaced edges on [1e-5, 2e7] eV.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

BASE_SEED = 2403012345

GEOM_INFINITE = 0
GEOM_LATTICE = 1
GEOM_SLAB = 2

BC_VACUUM = 0
BC_REFLECT = 1

SRC_ORIGIN = 0      # point at the origin, isotropic (infinite medium)
SRC_BOX = 1         # uniform over the lattice box volume, isotropic
SRC_SLAB_FACE = 2   # point on the x=0 face, isotropic over the inward hemisphere

E_MIN = 1e-5
E_MAX = 2e7


@dataclass
class Geometry:
    kind: int = GEOM_INFINITE
    source: int = SRC_ORIGIN
    E0: float = 1e6
    E_cut: float = 1e-5
    # infinite medium
    mat: int = 0
    # lattice of n x n pin cells, pitch p, pin radius r, height H
    n: int = 1
    pitch: float = 1.26
    radius: float = 0.4
    height: float = 100.0
    mat_pin: int = 0
    mat_mod: int = 1
    bc_side: int = BC_REFLECT
    bc_z: int = BC_VACUUM
    # slab of n_layers layers of thickness layer_dx along x; layers < n_first
    # hold mat_a, the rest mat_b
    n_layers: int = 0
    layer_dx: float = 1.0
    n_first: int = 0
    mat_a: int = 0
    mat_b: int = 0

    def n_cells(self) -> int:
        if self.kind == GEOM_LATTICE:
            return self.n * self.n
        if self.kind == GEOM_SLAB:
            return self.n_layers
        return 1


@dataclass
class Problem:
    """Pooled nuclide tables, materials and one or more geometries."""
    name: str
    grid_off: np.ndarray          # int64 [n_nuc+1]
    energy: np.ndarray            # float64 [grid_off[-1]]
    sigma_t: np.ndarray           # float64 [grid_off[-1]]
    f_abs: np.ndarray             # float64 [n_nuc]
    awr: np.ndarray               # float64 [n_nuc]
    mat_off: np.ndarray           # int32 [n_mat+1]
    nuc_id: np.ndarray            # int32 [mat_off[-1]]
    density: np.ndarray           # float64 [mat_off[-1]]
    edges: np.ndarray             # float64 [n_bins+1]
    geoms: List[Geometry]
    n_particles: List[int]
    n_batches: int = 1
    seed: int = BASE_SEED
    precision: int = 0            # 0 = binary64 tables, 1 = binary32 tables
    extra: dict = field(default_factory=dict)
    nu: Optional[np.ndarray] = None     # float64 [n_nuc] mean neutrons per fission
    f_fis: Optional[np.ndarray] = None  # float64 [n_nuc] sigma_f / sigma_t (<= f_abs)

    @property
    def n_nuc(self) -> int:
        return len(self.grid_off) - 1

    @property
    def n_mat(self) -> int:
        return len(self.mat_off) - 1

    @property
    def n_bins(self) -> int:
        return len(self.edges) - 1

    @property
    def geom(self) -> Geometry:
        return self.geoms[0]

    def table_bytes(self, precision: Optional[int] = None) -> int:
        p = self.precision if precision is None else precision
        return int(self.grid_off[-1]) * (16 if p == 0 else 8)


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def _grid(e: np.ndarray) -> np.ndarray:
    """Strictly increasing binary64 grid from the drawn points e (first and
    last kept): an interior point is dropped when its binary32 rounding
    equals that of the point before it or that of the last point."""
    e = np.unique(np.asarray(e, dtype=np.float64))
    f = e.astype(np.float32)
    keep = np.ones(len(e), dtype=bool)
    keep[1:] = f[1:] != f[:-1]
    keep[1:-1] &= f[1:-1] != f[-1]
    keep[-1] = True
    return e[keep]


def _nuclide(rng, n_points: int, n_res: int, log_spaced: bool,
             f_range=(0.05, 0.5)):
    if log_spaced:
        e = np.geomspace(E_MIN, E_MAX, n_points)
    else:
        inner = np.sort(_loguniform(rng, E_MIN, E_MAX, n_points - 2))
        e = np.concatenate([[E_MIN], inner, [E_MAX]])
    e = _grid(e)
    a = _loguniform(rng, 1.0, 1e3)
    ek = _loguniform(rng, 1.0, 1e5, n_res)
    hk = _loguniform(rng, 10.0, 1e4, n_res)
    gk = ek * _loguniform(rng, 1e-4, 1e-2, n_res)
    sig = a / np.sqrt(e)
    for k in range(n_res):
        hw2 = (0.5 * gk[k]) ** 2
        sig += hk[k] * hw2 / ((e - ek[k]) ** 2 + hw2)
    f = rng.uniform(*f_range)
    awr = rng.uniform(1.0, 240.0)
    return e, sig, f, awr


def _pool(nucs):
    sizes = [len(n[0]) for n in nucs]
    off = np.zeros(len(nucs) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    energy = np.concatenate([n[0] for n in nucs])
    sigma = np.concatenate([n[1] for n in nucs])
    f_abs = np.array([n[2] for n in nucs], dtype=np.float64)
    awr = np.array([n[3] for n in nucs], dtype=np.float64)
    return off, energy, sigma, f_abs, awr


def _materials(mats):
    """mats: list of (nuclide ids, densities)."""
    off = np.zeros(len(mats) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(m[0]) for m in mats])
    ids = np.concatenate([np.asarray(m[0], dtype=np.int32) for m in mats])
    den = np.concatenate([np.asarray(m[1], dtype=np.float64) for m in mats])
    return off, ids, den


def _edges(nb: int) -> np.ndarray:
    return np.geomspace(E_MIN, E_MAX, nb + 1)


def _lattice_library(rng, n_pin: int, n_mod: int, nmin: int, nmax: int):
    nucs = []
    for _ in range(n_pin + n_mod):
        ng = int(rng.integers(nmin, nmax + 1))
        nr = int(rng.integers(5, 51))
        nucs.append(_nuclide(rng, ng, nr, log_spaced=False))
    dens = rng.uniform(0.01, 1.0, n_pin + n_mod)
    mats = [(np.arange(n_pin), dens[:n_pin]),
            (np.arange(n_pin, n_pin + n_mod), dens[n_pin:])]
    return nucs, mats


def make_config(k: int, n_particles: Optional[int] = None,
                n_batches: Optional[int] = None, grid_scale: float = 1.0,
                n_problems: Optional[int] = None) -> Problem:
    """Configuration k (1..5) of the workload description.

    n_particles / n_batches override the per-batch count (tests use small
    counts); grid_scale shrinks the grids of configurations 2-4 for tests.
    Configuration k draws its data from the seed BASE_SEED + k.
    """
    seed = BASE_SEED + k
    rng = np.random.default_rng(seed)
    if k == 1:
        nucs = [_nuclide(rng, 2000, 5, log_spaced=True) for _ in range(4)]
        dens = rng.uniform(0.01, 1.0, 4)
        off, en, sg, fa, aw = _pool(nucs)
        mo, ids, den = _materials([(np.arange(4), dens)])
        g = Geometry(kind=GEOM_INFINITE, source=SRC_ORIGIN, mat=0)
        return Problem("infinite-medium-4nuc", off, en, sg, fa, aw, mo, ids, den,
                       _edges(100), [g], [n_particles or 100_000],
                       n_batches or 1, seed, 0)
    if k in (2, 3):
        # configurations 2 and 3 share seeds and data (same lattice)
        rng = np.random.default_rng(BASE_SEED + 2)
        nmin, nmax = int(10_000 * grid_scale), int(60_000 * grid_scale)
        nucs, mats = _lattice_library(rng, 68, 3, max(nmin, 2), max(nmax, 2))
        off, en, sg, fa, aw = _pool(nucs)
        mo, ids, den = _materials(mats)
        g = Geometry(kind=GEOM_LATTICE, source=SRC_BOX, n=17, pitch=1.26,
                     radius=0.4, height=100.0, mat_pin=0, mat_mod=1,
                     bc_side=BC_REFLECT, bc_z=BC_VACUUM)
        npart = n_particles or (1_000_000 if k == 2 else 10_000_000)
        return Problem("lattice17-fp64" if k == 2 else "lattice17-fp32-sorted",
                       off, en, sg, fa, aw, mo, ids, den, _edges(200), [g],
                       [npart], n_batches or 10, BASE_SEED + 2, 0 if k == 2 else 1)
    if k == 4:
        nprob = n_problems or 64
        nucs, mats, geoms, nps = [], [], [], []
        for p in range(nprob):
            n = int(rng.integers(3, 18))
            n_pin = int(rng.integers(4, 69))
            npart = int(round(float(_loguniform(rng, 1e4, 1e6))))
            lib, m = _lattice_library(rng, n_pin, 3, max(int(10_000 * grid_scale), 2),
                                      max(int(60_000 * grid_scale), 2))
            base = len(nucs)
            nucs.extend(lib)
            mats.append((m[0][0] + base, m[0][1]))
            mats.append((m[1][0] + base, m[1][1]))
            geoms.append(Geometry(kind=GEOM_LATTICE, source=SRC_BOX, n=n, pitch=1.26,
                                  radius=0.4, height=100.0, mat_pin=2 * p,
                                  mat_mod=2 * p + 1, bc_side=BC_REFLECT,
                                  bc_z=BC_VACUUM))
            nps.append(npart if n_particles is None else n_particles)
        off, en, sg, fa, aw = _pool(nucs)
        mo, ids, den = _materials(mats)
        return Problem("batched-64-lattices-fp32", off, en, sg, fa, aw, mo, ids, den,
                       _edges(200), geoms, nps, n_batches or 1, seed, 1)
    if k == 5:
        nucs = [_nuclide(rng, int(rng.integers(10_000, 60_001) * grid_scale) or 2,
                         int(rng.integers(5, 51)), False) for _ in range(3)]
        nucs += [_nuclide(rng, int(rng.integers(10_000, 60_001) * grid_scale) or 2,
                          int(rng.integers(5, 51)), False, f_range=(0.3, 0.7))
                 for _ in range(20)]
        dens = rng.uniform(0.01, 1.0, 23)
        scale = SLAB_ABSORBER_SCALE
        off, en, sg, fa, aw = _pool(nucs)
        mo, ids, den = _materials([(np.arange(3), dens[:3]),
                                   (np.arange(3, 23), dens[3:] * scale)])
        g = Geometry(kind=GEOM_SLAB, source=SRC_SLAB_FACE, n_layers=110,
                     layer_dx=1.0, n_first=10, mat_a=0, mat_b=1)
        return Problem("deep-penetration-slab", off, en, sg, fa, aw, mo, ids, den,
                       _edges(100), [g], [n_particles or 10_000_000],
                       n_batches or 1, seed, 0, extra={"absorber_scale": scale})
    raise ValueError(f"unknown configuration {k}")


# Multiplier on the slab absorber densities (configuration 5), chosen by a
# pilot analog run of the CPU oracle so that the analog far-face leakage
# probability sits in [1e-6, 1e-4]: 41 of 4e6 histories (1.0e-5) at 0.1.
SLAB_ABSORBER_SCALE = 0.1


def make_eigen_lattice(n_particles: int = 1_000_000, grid_scale: float = 1.0,
                       n_fissile: int = 40) -> Problem:
    """k-eigenvalue workload: the 17x17 lattice of configuration 2 (same
    tables and seeds) with the first n_fissile pin nuclides made fissile:
    sigma_f = g f_abs sigma_t with g uniform on [0.7, 0.95] (fission is part
    of absorption) and nu uniform on [2.4, 2.9].  With 40 of the 68 pin
    nuclides k is about 1.0 at grid_scale 0.02 and about 1.47 with the full
    grids.  The source of the first
    generation is the box source; later generations start from the bank."""
    p = make_config(2, n_particles=n_particles, grid_scale=grid_scale)
    rng = np.random.default_rng(BASE_SEED + 7)
    nu = np.zeros(p.n_nuc)
    ff = np.zeros(p.n_nuc)
    nu[:n_fissile] = rng.uniform(2.4, 2.9, n_fissile)
    ff[:n_fissile] = p.f_abs[:n_fissile] * rng.uniform(0.7, 0.95, n_fissile)
    p.name = "lattice17-eigenvalue-fp64"
    p.nu, p.f_fis = nu, ff
    return p


def make_stress_lookup(n_queries: int = 10_000_000, n_nuc: int = 281,
                       n_in_mat: int = 244, n_points: int = 60_000,
                       sorted_queries: bool = False, seed_offset: int = 0):
    """Lookup-only stress set: n_nuc nuclides of n_points points, one material
    of n_in_mat nuclides (the paper's SMR fuel: 244 of 281 nuclides, Sec. 4.1)
    plus one of the rest; n_queries energies log-uniform on [1e-5, 2e7] eV.

    Returns (Problem, E[n_queries], mat[n_queries]).
    """
    seed = BASE_SEED + 100 + seed_offset
    rng = np.random.default_rng(seed)
    nucs = [_nuclide(rng, n_points, int(rng.integers(5, 51)), False)
            for _ in range(n_nuc)]
    dens = rng.uniform(0.01, 1.0, n_nuc)
    off, en, sg, fa, aw = _pool(nucs)
    mats = [(np.arange(n_in_mat), dens[:n_in_mat])]
    if n_nuc > n_in_mat:
        mats.append((np.arange(n_in_mat, n_nuc), dens[n_in_mat:]))
    mo, ids, den = _materials(mats)
    g = Geometry(kind=GEOM_INFINITE, source=SRC_ORIGIN, mat=0)
    prob = Problem("lookup-stress", off, en, sg, fa, aw, mo, ids, den, _edges(100),
                   [g], [0], 1, seed, 0)
    E = _loguniform(rng, E_MIN, E_MAX, n_queries)
    if sorted_queries:
        E = np.sort(E)
    mat = np.zeros(n_queries, dtype=np.int32)
    return prob, E, mat


def make_tiny_problem(seed: int = 7, n_nuc: int = 3, n_points=(2, 9),
                      kind: int = GEOM_INFINITE, n_particles: int = 1000,
                      flat: bool = False, f_abs=None, awr=None,
                      lattice_n: int = 3, n_bins: int = 10) -> Problem:
    """Small problems for tests: few grid points, optionally flat cross
    sections (a = const, no resonances) with a fixed absorption fraction."""
    rng = np.random.default_rng(seed)
    nucs = []
    for i in range(n_nuc):
        ng = int(rng.integers(n_points[0], n_points[1] + 1))
        if flat:
            e = _grid(np.geomspace(E_MIN, E_MAX, ng))
            sig = np.full_like(e, float(rng.uniform(1.0, 10.0)))
            f = float(rng.uniform(0.05, 0.5))
            a = float(rng.uniform(1.0, 240.0))
            nucs.append((e, sig, f, a))
        else:
            nucs.append(_nuclide(rng, ng, int(rng.integers(0, 4)), ng > 2000))
    nucs = [(e, s, (f_abs[i] if f_abs is not None else f),
             (awr[i] if awr is not None else a)) for i, (e, s, f, a) in enumerate(nucs)]
    off, en, sg, fa, aw = _pool(nucs)
    dens = rng.uniform(0.01, 1.0, n_nuc)
    half = max(1, n_nuc // 2)
    if n_nuc > 1:
        two = [(np.arange(half), dens[:half]), (np.arange(half, n_nuc), dens[half:])]
    else:
        two = [(np.arange(1), dens), (np.arange(1), dens)]
    if kind == GEOM_LATTICE:
        mats = two
        g = Geometry(kind=GEOM_LATTICE, source=SRC_BOX, n=lattice_n, mat_pin=0,
                     mat_mod=1 if n_nuc > 1 else 0, height=20.0)
    elif kind == GEOM_SLAB:
        mats = two
        g = Geometry(kind=GEOM_SLAB, source=SRC_SLAB_FACE, n_layers=8, layer_dx=1.0,
                     n_first=2, mat_a=0, mat_b=1 if n_nuc > 1 else 0)
    else:
        mats = [(np.arange(n_nuc), dens)]
        g = Geometry(kind=GEOM_INFINITE, source=SRC_ORIGIN, mat=0)
    mo, ids, den = _materials(mats)
    return Problem("tiny", off, en, sg, fa, aw, mo, ids, den, _edges(n_bins), [g],
                   [n_particles], 1, seed, 0)
