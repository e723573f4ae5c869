"""ctypes front end of the CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg.  The product package never imports it.

The problem argument is any object with the attributes of a pooled problem
description (grid_off, energy, sigma_t, f_abs, awr, mat_off, nuc_id, density,
edges, precision, geoms[]); no module of the product is imported here.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

STATUS_ALIVE, STATUS_ABSORBED, STATUS_LEAKED, STATUS_CUTOFF, STATUS_LIMIT, STATUS_LEAKED_FAR, \
    STATUS_ROULETTE = range(7)
S_COLLISION, S_ABSORPTION, S_LEAK, S_CUTOFF, S_LIMIT, S_LEAK_FAR, S_FLIGHT, S_HISTORY, S_SPLIT, \
    S_ROULETTE = range(10)
NSCAL = 10
MLP_HIDDEN = 64
MLP_NPARAM = 64 * 4 + 64 + 64 * 64 + 64 + 64 + 1
MAX_FLIGHTS = 100000

_P = C.POINTER


class _Problem(C.Structure):
    _fields_ = [
        ("n_nuc", C.c_int32), ("grid_off", _P(C.c_int64)), ("energy", _P(C.c_double)),
        ("sigma_t", _P(C.c_double)), ("f_abs", _P(C.c_double)), ("awr", _P(C.c_double)),
        ("n_mat", C.c_int32), ("mat_off", _P(C.c_int32)), ("nuc_id", _P(C.c_int32)),
        ("density", _P(C.c_double)), ("n_bins", C.c_int32), ("edges", _P(C.c_double)),
        ("precision", C.c_int32),
        ("kind", C.c_int32), ("source", C.c_int32), ("E0", C.c_double), ("E_cut", C.c_double),
        ("mat", C.c_int32), ("n", C.c_int32), ("pitch", C.c_double), ("radius", C.c_double),
        ("height", C.c_double), ("mat_pin", C.c_int32), ("mat_mod", C.c_int32),
        ("bc_side", C.c_int32), ("bc_z", C.c_int32), ("n_layers", C.c_int32),
        ("layer_dx", C.c_double), ("n_first", C.c_int32), ("mat_a", C.c_int32),
        ("mat_b", C.c_int32), ("ww_lower", _P(C.c_double)), ("ww_ratio", C.c_double),
        ("ww_survival", C.c_double), ("ww_max_split", C.c_int32),
        ("nu", _P(C.c_double)), ("f_fis", _P(C.c_double)), ("k_norm", C.c_double),
        ("max_sites", C.c_int32), ("bank", _P(C.c_double)), ("bank_n", C.c_int64),
        ("bank_total", C.c_int64),
    ]


class _Result(C.Structure):
    _fields_ = [
        ("n_coll", _P(C.c_int32)), ("status", _P(C.c_int8)), ("n_flights", _P(C.c_int32)),
        ("n_draws", _P(C.c_uint32)), ("E", _P(C.c_double)), ("x", _P(C.c_double)),
        ("y", _P(C.c_double)), ("z", _P(C.c_double)), ("flux", _P(C.c_double)),
        ("absrate", _P(C.c_double)), ("counts", _P(C.c_int64)), ("weights", _P(C.c_double)),
        ("sites", _P(C.c_double)), ("n_sites", _P(C.c_int32)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        L.or_philox4x64_10.argtypes = [_P(C.c_uint64), _P(C.c_uint64), _P(C.c_uint64)]
        L.or_u01.argtypes = [C.c_uint64]
        L.or_u01.restype = C.c_double
        L.or_log.argtypes = [C.c_double]
        L.or_log.restype = C.c_double
        L.or_search.argtypes = [_P(C.c_double), C.c_int64, C.c_double]
        L.or_search.restype = C.c_int64
        L.or_micro.argtypes = [_P(_Problem), C.c_int32, C.c_double]
        L.or_micro.restype = C.c_double
        L.or_search_f32.argtypes = [_P(C.c_float), C.c_int64, C.c_double]
        L.or_search_f32.restype = C.c_int64
        L.or_micro_f32.argtypes = [_P(C.c_float), _P(C.c_float), C.c_int64, C.c_double]
        L.or_micro_f32.restype = C.c_float
        L.or_pick_nuclide.argtypes = [_P(_Problem), C.c_int32, C.c_double, C.c_double]
        L.or_pick_nuclide.restype = C.c_int32
        L.or_macro.argtypes = [_P(_Problem), C.c_int32, _P(C.c_double), C.c_int64,
                               _P(C.c_double), _P(C.c_double)]
        L.or_macro.restype = C.c_int
        L.or_dist_cylinder.argtypes = [C.c_double] * 5 + [C.c_int]
        L.or_dist_cylinder.restype = C.c_double
        L.or_elastic.argtypes = [C.c_double, C.c_double, C.c_double, _P(C.c_double), _P(C.c_double)]
        L.or_rotate.argtypes = [_P(C.c_double)] * 3 + [C.c_double] * 3
        L.or_run.argtypes = [_P(_Problem), C.c_uint64, C.c_uint64, C.c_int64, C.c_int64,
                             C.c_int, _P(_Result)]
        L.or_run.restype = C.c_int
        L.or_mlp_nparam.restype = C.c_int
        L.or_mlp_forward.argtypes = [_P(C.c_double), _P(C.c_double), C.c_int64, _P(C.c_double)]
        L.or_mlp_grad.argtypes = [_P(C.c_double), _P(C.c_double), _P(C.c_double),
                                  _P(C.c_double), C.c_int64, _P(C.c_double)]
        L.or_mlp_grad.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(_P(ctype))


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(_ptr(c, C.c_uint64), _ptr(k, C.c_uint64), _ptr(out, C.c_uint64))
    return out


def u01(x: int) -> float:
    return lib().or_u01(int(x))


def log(x: float) -> float:
    return lib().or_log(float(x))


def search(g, E: float) -> int:
    g = np.ascontiguousarray(g, dtype=np.float64)
    return int(lib().or_search(_ptr(g, C.c_double), len(g), float(E)))


def search_f32(g, E: float) -> int:
    """Bracket of E on a binary32 grid g (compared exactly, in binary64)."""
    g = np.ascontiguousarray(g, dtype=np.float32)
    return int(lib().or_search_f32(_ptr(g, C.c_float), len(g), float(E)))


def micro_f32(g, s, E: float) -> float:
    """Binary32 lin-lin micro cross section of one nuclide's binary32 grid g
    and values s at E."""
    g = np.ascontiguousarray(g, dtype=np.float32)
    s = np.ascontiguousarray(s, dtype=np.float32)
    if len(g) != len(s):
        raise ValueError("grid and values differ in length")
    return float(np.float32(lib().or_micro_f32(_ptr(g, C.c_float), _ptr(s, C.c_float), len(g),
                                               float(E))))


def pick_nuclide(prob, mat: int, E: float, target: float, precision=None) -> int:
    """Collision nuclide of material mat at E for target = xi Sigma_t."""
    b = _Bound(prob, precision=precision)
    i = lib().or_pick_nuclide(C.byref(b.p), int(mat), float(E), float(target))
    if i < 0:
        raise MemoryError("oracle tables could not be built")
    return int(i)


def dist_cylinder(dx, dy, u, v, r, inside) -> float:
    return lib().or_dist_cylinder(dx, dy, u, v, r, int(inside))


def elastic(E, A, mu):
    e = C.c_double()
    m = C.c_double()
    lib().or_elastic(E, A, mu, C.byref(e), C.byref(m))
    return e.value, m.value


def rotate(u, v, w, mu, cphi, sphi):
    a, b, c = C.c_double(u), C.c_double(v), C.c_double(w)
    lib().or_rotate(C.byref(a), C.byref(b), C.byref(c), mu, cphi, sphi)
    return a.value, b.value, c.value


class _Bound:
    """Keeps the numpy arrays alive while the C structure points at them."""

    def __init__(self, prob, geom_index: int = 0, precision=None, ww=None, eigen=None):
        g = prob.geoms[geom_index]
        self.arrs = dict(
            grid_off=np.ascontiguousarray(prob.grid_off, dtype=np.int64),
            energy=np.ascontiguousarray(prob.energy, dtype=np.float64),
            sigma_t=np.ascontiguousarray(prob.sigma_t, dtype=np.float64),
            f_abs=np.ascontiguousarray(prob.f_abs, dtype=np.float64),
            awr=np.ascontiguousarray(prob.awr, dtype=np.float64),
            mat_off=np.ascontiguousarray(prob.mat_off, dtype=np.int32),
            nuc_id=np.ascontiguousarray(prob.nuc_id, dtype=np.int32),
            density=np.ascontiguousarray(prob.density, dtype=np.float64),
            edges=np.ascontiguousarray(prob.edges, dtype=np.float64),
        )
        a = self.arrs
        p = _Problem()
        p.n_nuc = len(a["grid_off"]) - 1
        p.grid_off = _ptr(a["grid_off"], C.c_int64)
        p.energy = _ptr(a["energy"], C.c_double)
        p.sigma_t = _ptr(a["sigma_t"], C.c_double)
        p.f_abs = _ptr(a["f_abs"], C.c_double)
        p.awr = _ptr(a["awr"], C.c_double)
        p.n_mat = len(a["mat_off"]) - 1
        p.mat_off = _ptr(a["mat_off"], C.c_int32)
        p.nuc_id = _ptr(a["nuc_id"], C.c_int32)
        p.density = _ptr(a["density"], C.c_double)
        p.n_bins = len(a["edges"]) - 1
        p.edges = _ptr(a["edges"], C.c_double)
        p.precision = int(prob.precision if precision is None else precision)
        for name in ("kind", "source", "mat", "n", "mat_pin", "mat_mod", "bc_side", "bc_z",
                     "n_layers", "n_first", "mat_a", "mat_b"):
            setattr(p, name, int(getattr(g, name)))
        for name in ("E0", "E_cut", "pitch", "radius", "height", "layer_dx"):
            setattr(p, name, float(getattr(g, name)))
        if ww is not None:
            lower, ratio, survival, max_split = ww
            self.ww = np.ascontiguousarray(lower, dtype=np.float64).reshape(-1)
            if self.ww.size != g.n_cells() * p.n_bins:
                raise ValueError("weight-window table must be [n_cells, n_bins]")
            p.ww_lower = _ptr(self.ww, C.c_double)
            p.ww_ratio, p.ww_survival, p.ww_max_split = float(ratio), float(survival), int(max_split)
        if eigen is not None:
            self.nu = np.ascontiguousarray(eigen["nu"], dtype=np.float64)
            self.ffis = np.ascontiguousarray(eigen["f_fis"], dtype=np.float64)
            p.nu = _ptr(self.nu, C.c_double)
            p.f_fis = _ptr(self.ffis, C.c_double)
            p.k_norm = float(eigen.get("k_norm", 1.0))
            p.max_sites = int(eigen.get("max_sites", 32))
            bank = eigen.get("bank")
            if bank is not None:
                xyz, total = bank
                self.bank = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
                if len(self.bank) < 1 or int(total) < 1:
                    raise ValueError("empty source bank")
                p.bank = _ptr(self.bank, C.c_double)
                p.bank_n, p.bank_total = len(self.bank), int(total)
                p.source = 3
        self.p = p
        self.n_cells = g.n_cells()
        self.n_bins = p.n_bins


def micro(prob, nuc: int, E: float) -> float:
    b = _Bound(prob, precision=0)
    return lib().or_micro(C.byref(b.p), int(nuc), float(E))


def macro(prob, mat: int, E, precision=None):
    b = _Bound(prob, precision=precision)
    E = np.ascontiguousarray(E, dtype=np.float64)
    st = np.zeros_like(E)
    sa = np.zeros_like(E)
    rc = lib().or_macro(C.byref(b.p), int(mat), _ptr(E, C.c_double), len(E),
                        _ptr(st, C.c_double), _ptr(sa, C.c_double))
    if rc != 0:
        raise MemoryError("oracle lookup failed")
    return st, sa


def key_hi(problem_index: int, batch: int) -> int:
    """Second Philox key word: problem index in the high 32 bits, batch low."""
    return ((int(problem_index) & 0xFFFFFFFF) << 32) | (int(batch) & 0xFFFFFFFF)


def run(prob, seed: int, batch: int = 0, first_id: int = 0, n=None, geom_index: int = 0,
        problem_index: int = 0, threads=None, precision=None, ww=None, eigen=None):
    """Histories [first_id, first_id + n) of one batch; returns a dict with
    per-particle outcomes, the flux tally [n_cells, n_bins], the track-length
    absorption-rate tally sum w d Sigma_a [n_cells, n_bins] and the scalars.
    ww = (lower [n_cells, n_bins], ratio, survival, max_split) turns on
    weight windows; split copies are transported depth first and scored in
    the tallies (the outcomes are the primary histories').
    eigen = dict(nu, f_fis, k_norm, max_sites[, bank=(xyz [m, 3], n_total)])
    banks fission sites (k-eigenvalue mode; with `bank` the histories start
    from it); the result then holds n_sites per history and `sites`, the
    bank in history order."""
    b = _Bound(prob, geom_index, precision, ww, eigen)
    if n is None:
        n = prob.n_particles[geom_index]
    n = int(n)
    if threads is None:
        threads = len(os.sched_getaffinity(0))
    out = dict(
        n_coll=np.zeros(n, np.int32), status=np.zeros(n, np.int8),
        n_flights=np.zeros(n, np.int32), n_draws=np.zeros(n, np.uint32),
        E=np.zeros(n), x=np.zeros(n), y=np.zeros(n), z=np.zeros(n),
        flux=np.zeros((b.n_cells, b.n_bins)), absrate=np.zeros((b.n_cells, b.n_bins)),
        counts=np.zeros(NSCAL, np.int64),
        weights=np.zeros(NSCAL),
    )
    r = _Result()
    r.n_coll = _ptr(out["n_coll"], C.c_int32)
    r.status = _ptr(out["status"], C.c_int8)
    r.n_flights = _ptr(out["n_flights"], C.c_int32)
    r.n_draws = _ptr(out["n_draws"], C.c_uint32)
    for k in ("E", "x", "y", "z", "flux", "absrate", "weights"):
        setattr(r, k, _ptr(out[k], C.c_double))
    r.counts = _ptr(out["counts"], C.c_int64)
    if eigen is not None:
        ms = int(b.p.max_sites)
        raw = np.zeros((n, ms, 3))
        out["n_sites"] = np.zeros(n, np.int32)
        r.sites = _ptr(raw, C.c_double)
        r.n_sites = _ptr(out["n_sites"], C.c_int32)
    rc = lib().or_run(C.byref(b.p), int(seed) & 0xFFFFFFFFFFFFFFFF,
                      key_hi(problem_index, batch), int(first_id), n, int(threads), C.byref(r))
    if rc == -2:
        raise RuntimeError("oracle split stack overflow (more than 2^24 pending copies)")
    if rc == -3:
        raise RuntimeError("a history banked more than max_sites fission sites")
    if eigen is not None:
        ns = out["n_sites"]
        out["sites"] = np.concatenate([raw[k, :ns[k]] for k in range(n)]) if n else np.zeros((0, 3))
    if rc != 0:
        raise MemoryError("oracle run failed")
    return out


def birth_state(prob, seed: int, id_: int, batch: int = 0, problem_index: int = 0,
                geom_index: int = 0, eigen=None):
    """(x, y, z, u, v, w, E), (i, j, inside, material) of a particle at birth."""
    b = _Bound(prob, geom_index, eigen=eigen)
    st = np.zeros(7)
    cell = np.zeros(4, np.int32)
    L = lib()
    L.or_birth_state.argtypes = [_P(_Problem), C.c_uint64, C.c_uint64, C.c_int64,
                                 _P(C.c_double), _P(C.c_int32)]
    L.or_birth_state(C.byref(b.p), int(seed), key_hi(problem_index, batch), int(id_),
                     _ptr(st, C.c_double), _ptr(cell, C.c_int32))
    return st, cell


def mlp_forward(params, x):
    """Binary64 forward pass of the importance network on features x [n, 4]."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 4)
    out = np.zeros(len(x))
    lib().or_mlp_forward(_ptr(p, C.c_double), _ptr(x, C.c_double), len(x), _ptr(out, C.c_double))
    return out


def mlp_grad(params, x, y, w):
    """Weighted MSE loss and its gradient with respect to the parameters."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 4)
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.zeros(MLP_NPARAM)
    loss = lib().or_mlp_grad(_ptr(p, C.c_double), _ptr(x, C.c_double), _ptr(y, C.c_double),
                             _ptr(w, C.c_double), len(x), _ptr(g, C.c_double))
    return loss, g
