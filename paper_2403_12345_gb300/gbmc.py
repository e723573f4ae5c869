"""Python binding of the gbmc C ABI (include/gbmc.h): argument marshalling only.

Every step of the transport hot path runs in the CUDA kernels of
libgbmc.so; this module converts arrays and structures and checks return
codes.  PyTorch supplies device memory and streams where an entry point takes
device pointers.  There is no CPU fallback: if the library cannot be loaded,
importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbmc.so")

OK = 0
ERR_INVALID_ARG, ERR_NOT_INITIALIZED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_DEVICE_FLAG, \
    ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
FP64, FP32 = 0, 1
GEOM_INFINITE, GEOM_LATTICE, GEOM_SLAB = 0, 1, 2
BC_VACUUM, BC_REFLECT = 0, 1
SRC_ORIGIN, SRC_BOX, SRC_SLAB_FACE, SRC_BANK = 0, 1, 2, 3
STATUS_ABSORBED, STATUS_LEAKED, STATUS_CUTOFF, STATUS_LIMIT, STATUS_LEAKED_FAR, \
    STATUS_ROULETTE = 1, 2, 3, 4, 5, 6
S_COLLISION, S_ABSORPTION, S_LEAK, S_CUTOFF, S_LIMIT, S_LEAK_FAR, S_FLIGHT, S_HISTORY, S_SPLIT, \
    S_ROULETTE = range(10)
NSCAL = 10
MAX_FLIGHTS = 100000

EXPORTS = ["gbmc_default_options", "gbmc_create", "gbmc_destroy", "gbmc_last_error",
           "gbmc_set_options", "gbmc_load_xs_tables", "gbmc_init_materials", "gbmc_set_tally",
           "gbmc_reset_tallies", "gbmc_run_batch", "gbmc_run_problems", "gbmc_read_tallies",
           "gbmc_read_outcomes", "gbmc_read_stats", "gbmc_lookup_macro", "gbmc_last_run_ms",
           "gbmc_profile_problems", "gbmc_lookup_macro_noalloc", "gbmc_autotune",
           "gbmc_set_weight_windows", "gbmc_clear_weight_windows", "gbmc_set_importance_net",
           "gbmc_get_importance_net", "gbmc_mlp_forward", "gbmc_mlp_gradient", "gbmc_mlp_train",
           "gbmc_mesh_features", "gbmc_weight_windows_from_net", "gbmc_importance_record",
           "gbmc_importance_accumulate", "gbmc_importance_training_set",
           "gbmc_get_weight_windows", "gbmc_set_reaction_tally", "gbmc_read_reaction_tally",
           "gbmc_load_fission", "gbmc_set_eigen", "gbmc_read_bank", "gbmc_set_source_bank",
           "gbmc_check_division", "gbmc_run_concurrent", "gbmc_measure_fp64_rate",
           "gbmc_run_concurrent_to_host", "gbmc_host_alloc", "gbmc_host_free"]
MLP_HIDDEN = 64
MLP_NPARAM = 4545
NOALLOC_MAX_QUERIES = 1 << 20
KERNEL_NAMES = ["plan", "source", "sort_scan", "sort_scatter", "lookup", "raytrace",
                "collision", "tail"]


class GbmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gbmc error {code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_in_flight", C.c_int64), ("sort", C.c_int32),
                ("block_lookup", C.c_int32), ("block_event", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("max_iterations", C.c_int32),
                ("sort_min", C.c_int32), ("warp_lookup_max", C.c_int32),
                ("tail_max", C.c_int32), ("sparse_windows", C.c_int32),
                ("group_lookup_max", C.c_int32), ("search", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class Geometry(C.Structure):
    _fields_ = [("kind", C.c_int32), ("source", C.c_int32), ("E0", C.c_double),
                ("E_cut", C.c_double), ("mat", C.c_int32), ("n", C.c_int32),
                ("pitch", C.c_double), ("radius", C.c_double), ("height", C.c_double),
                ("mat_pin", C.c_int32), ("mat_mod", C.c_int32), ("bc_side", C.c_int32),
                ("bc_z", C.c_int32), ("n_layers", C.c_int32), ("layer_dx", C.c_double),
                ("n_first", C.c_int32), ("mat_a", C.c_int32), ("mat_b", C.c_int32)]


class HostResults(C.Structure):
    """gbmc_host_results: host destinations of one problem's results."""
    _fields_ = [("flux", C.c_void_p), ("counts", C.c_void_p), ("weights", C.c_void_p),
                ("n_coll", C.c_void_p), ("status", C.c_void_p), ("n_flights", C.c_void_p),
                ("n_draws", C.c_void_p), ("E", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p),
                ("z", C.c_void_p)]


# dtype of each HostResults field and whether it has one entry per particle
# (else: flux [cells * bins], counts / weights [NSCAL])
_RESULT_FIELDS = {"flux": (np.float64, None), "counts": (np.int64, None),
                  "weights": (np.float64, None), "n_coll": (np.int32, True),
                  "status": (np.int8, True), "n_flights": (np.int32, True),
                  "n_draws": (np.uint32, True), "E": (np.float64, True),
                  "x": (np.float64, True), "y": (np.float64, True), "z": (np.float64, True)}


class Problem(C.Structure):
    _fields_ = [("geom", Geometry), ("seed", C.c_uint64), ("problem_index", C.c_uint32),
                ("batch", C.c_uint32), ("first_id", C.c_int64), ("n_particles", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("lookups", C.c_int64), ("micro_lookups", C.c_int64),
                ("flights", C.c_int64), ("crossings", C.c_int64), ("collisions", C.c_int64),
                ("histories", C.c_int64), ("device_error", C.c_int32), ("reserved", C.c_int32),
                ("handoffs", C.c_int64)]


class AutotuneReport(C.Structure):
    _fields_ = [("trials", C.c_int32), ("reserved", C.c_int32), ("default_ms", C.c_double),
                ("best_ms", C.c_double), ("in_flight_fraction", C.c_double)]


class KernelTimes(C.Structure):
    _fields_ = [("ms", C.c_double * len(KERNEL_NAMES)), ("launches", C.c_int64 * len(KERNEL_NAMES))]


_P = C.POINTER
_lib = None


def lib():
    """The loaded libgbmc.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "paper_2403_12345_gb300/build.py (there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.gbmc_default_options.argtypes = [_P(Options)]
        L.gbmc_create.argtypes = [_P(vp), C.c_int, _P(Options)]
        L.gbmc_destroy.argtypes = [vp]
        L.gbmc_last_error.argtypes = [vp]
        L.gbmc_last_error.restype = C.c_char_p
        L.gbmc_set_options.argtypes = [vp, _P(Options)]
        L.gbmc_load_xs_tables.argtypes = [vp, C.c_int32, _P(C.c_int64), _P(C.c_double),
                                          _P(C.c_double), _P(C.c_double), _P(C.c_double),
                                          C.c_int32]
        L.gbmc_init_materials.argtypes = [vp, C.c_int32, _P(C.c_int32), _P(C.c_int32),
                                          _P(C.c_double)]
        L.gbmc_set_tally.argtypes = [vp, C.c_int32, _P(C.c_double)]
        L.gbmc_reset_tallies.argtypes = [vp, vp]
        L.gbmc_run_batch.argtypes = [vp, _P(Problem), vp]
        L.gbmc_run_problems.argtypes = [vp, C.c_int32, _P(Problem), vp]
        L.gbmc_run_concurrent.argtypes = [vp, C.c_int32, _P(Problem), C.c_int32, C.c_int32, vp]
        L.gbmc_run_concurrent_to_host.argtypes = [vp, C.c_int32, _P(Problem), C.c_int32, C.c_int32,
                                                  _P(HostResults), vp]
        L.gbmc_measure_fp64_rate.argtypes = [vp, _P(C.c_double)]
        L.gbmc_read_tallies.argtypes = [vp, C.c_int32, _P(C.c_double), C.c_int64,
                                        _P(C.c_int64), _P(C.c_double)]
        L.gbmc_set_reaction_tally.argtypes = [vp, C.c_int32]
        L.gbmc_load_fission.argtypes = [vp, C.c_int32, _P(C.c_double), _P(C.c_double)]
        L.gbmc_check_division.argtypes = [vp, C.c_int32, C.c_int64, C.c_uint64, _P(C.c_int64),
                                          _P(C.c_double)]
        L.gbmc_set_eigen.argtypes = [vp, C.c_double, C.c_int32]
        L.gbmc_read_bank.argtypes = [vp, _P(C.c_double), C.c_int64, _P(C.c_int64)]
        L.gbmc_set_source_bank.argtypes = [vp, _P(C.c_double), C.c_int64, C.c_int64]
        L.gbmc_read_reaction_tally.argtypes = [vp, C.c_int32, _P(C.c_double), C.c_int64]
        L.gbmc_read_outcomes.argtypes = [vp, C.c_int32, C.c_int64, C.c_int64, _P(C.c_int32),
                                         _P(C.c_int8), _P(C.c_int32), _P(C.c_uint32),
                                         _P(C.c_double), _P(C.c_double), _P(C.c_double),
                                         _P(C.c_double)]
        L.gbmc_read_stats.argtypes = [vp, _P(Stats)]
        L.gbmc_lookup_macro.argtypes = [vp, C.c_int32, vp, vp, C.c_int64, vp, vp, C.c_int32, vp]
        L.gbmc_last_run_ms.argtypes = [vp, _P(C.c_double)]
        L.gbmc_autotune.argtypes = [vp, C.c_int32, _P(Problem), C.c_double, vp, _P(Options),
                                    _P(AutotuneReport)]
        L.gbmc_set_weight_windows.argtypes = [vp, C.c_int32, C.c_int32, _P(C.c_double),
                                              C.c_double, C.c_double, C.c_int32]
        L.gbmc_clear_weight_windows.argtypes = [vp]
        L.gbmc_get_weight_windows.argtypes = [vp, _P(C.c_double), C.c_int64]
        L.gbmc_set_importance_net.argtypes = [vp, _P(C.c_uint16), C.c_int32, _P(C.c_double),
                                              _P(C.c_double)]
        L.gbmc_get_importance_net.argtypes = [vp, _P(C.c_uint16), C.c_int32]
        L.gbmc_mlp_forward.argtypes = [vp, vp, C.c_int64, vp, vp]
        L.gbmc_mlp_gradient.argtypes = [vp, vp, vp, vp, C.c_int64, _P(C.c_float), _P(C.c_float), vp]
        L.gbmc_mlp_train.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int32, C.c_float,
                                     _P(C.c_float), vp]
        L.gbmc_mesh_features.argtypes = [vp, _P(Geometry), vp, C.c_int64, _P(C.c_int64), vp]
        L.gbmc_weight_windows_from_net.argtypes = [vp, _P(Geometry), C.c_double, C.c_double,
                                                   C.c_int32, vp]
        L.gbmc_importance_record.argtypes = [vp, _P(Geometry), C.c_int64]
        L.gbmc_importance_accumulate.argtypes = [vp, vp]
        L.gbmc_importance_training_set.argtypes = [vp, _P(Geometry), vp, vp, vp, C.c_int64,
                                                   _P(C.c_int64), vp]
        L.gbmc_lookup_macro_noalloc.argtypes = [vp, C.c_int32, vp, vp, C.c_int64, vp, vp, vp]
        L.gbmc_profile_problems.argtypes = [vp, C.c_int32, _P(Problem), vp, _P(KernelTimes),
                                            C.c_int32, _P(C.c_double), _P(C.c_int32),
                                            _P(C.c_int32)]
        L.gbmc_host_alloc.argtypes = [C.c_size_t, _P(vp)]
        L.gbmc_host_free.argtypes = [vp]
        for name in EXPORTS:
            if name != "gbmc_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class _HostBlock:
    """One gbmc_host_alloc allocation seen as a 1-D array (numpy's array
    interface); numpy arrays made from it keep it alive, and it is freed
    with the last of them."""

    def __init__(self, n: int, dt: np.dtype):
        ptr = C.c_void_p()
        nbytes = max(n * dt.itemsize, 1)
        rc = lib().gbmc_host_alloc(C.c_size_t(nbytes), C.byref(ptr))
        if rc:
            raise GbmcError(rc, f"gbmc_host_alloc of {nbytes} bytes failed")
        self.ptr = ptr.value
        self.__array_interface__ = {"data": (self.ptr, False), "shape": (n,),
                                    "typestr": dt.str, "version": 3}

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().gbmc_host_free(C.c_void_p(self.ptr))
            except Exception:   # interpreter shutdown: the process releases it
                pass
            self.ptr = None


def host_array(n: int, dtype) -> np.ndarray:
    """A numpy array of n elements in page-locked host memory from the
    library's allocator (gbmc_host_alloc), e.g. for the destinations of
    run_concurrent_to_host; the memory is freed with the last view of it."""
    return np.asarray(_HostBlock(int(n), np.dtype(dtype)))


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a, ct):
    return a.ctypes.data_as(_P(ct))


def _stream(stream):
    """cudaStream_t from None / int / torch.cuda.Stream."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def geometry(**kw) -> Geometry:
    g = Geometry()
    g.E0, g.E_cut = 1e6, 1e-5
    g.pitch, g.radius, g.height, g.layer_dx = 1.26, 0.4, 100.0, 1.0
    g.n = 1
    for k, v in kw.items():
        setattr(g, k, v)
    return g


def geometry_from(obj) -> Geometry:
    """Geometry from any object carrying the same field names."""
    return geometry(**{name: getattr(obj, name) for name, _ in Geometry._fields_})


def problem(geom: Geometry, seed: int, n_particles: int, batch: int = 0,
            problem_index: int = 0, first_id: int = 0) -> Problem:
    p = Problem()
    p.geom = geom
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.problem_index = int(problem_index)
    p.batch = int(batch)
    p.first_id = int(first_id)
    p.n_particles = int(n_particles)
    return p


class Context:
    """One gbmc context (gbmc_create ... gbmc_destroy) on one CUDA device."""

    def __init__(self, device: int = 0, **options):
        L = lib()
        opt = Options()
        L.gbmc_default_options(C.byref(opt))
        for k, v in options.items():
            setattr(opt, k, v)
        h = C.c_void_p()
        rc = L.gbmc_create(C.byref(h), int(device), C.byref(opt))
        if rc != OK:
            raise GbmcError(rc, L.gbmc_last_error(None).decode())
        self._h = h
        self.options = opt
        self.n_bins = 0
        self._cells = []

    def _ck(self, rc):
        if rc != OK:
            raise GbmcError(rc, lib().gbmc_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().gbmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- set-up ---------------------------------------------------------------
    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        self._ck(lib().gbmc_set_options(self._h, C.byref(self.options)))

    def load_xs_tables(self, grid_off, energy, sigma_t, f_abs, awr, precision=FP64):
        go = _arr(grid_off, np.int64)
        e, s = _arr(energy, np.float64), _arr(sigma_t, np.float64)
        fa, aw = _arr(f_abs, np.float64), _arr(awr, np.float64)
        self._ck(lib().gbmc_load_xs_tables(self._h, len(go) - 1, _p(go, C.c_int64),
                                           _p(e, C.c_double), _p(s, C.c_double),
                                           _p(fa, C.c_double), _p(aw, C.c_double),
                                           int(precision)))

    def init_materials(self, mat_off, nuc_id, density):
        mo, ni, de = _arr(mat_off, np.int32), _arr(nuc_id, np.int32), _arr(density, np.float64)
        self._ck(lib().gbmc_init_materials(self._h, len(mo) - 1, _p(mo, C.c_int32),
                                           _p(ni, C.c_int32), _p(de, C.c_double)))

    def set_tally(self, edges):
        ed = _arr(edges, np.float64)
        self._ck(lib().gbmc_set_tally(self._h, len(ed) - 1, _p(ed, C.c_double)))
        self.n_bins = len(ed) - 1

    def load(self, prob, precisions=(FP64,)):
        """Tables, materials and tally edges of a pooled problem description
        (any object with grid_off, energy, sigma_t, f_abs, awr, mat_off,
        nuc_id, density and edges)."""
        for prec in precisions:
            self.load_xs_tables(prob.grid_off, prob.energy, prob.sigma_t, prob.f_abs,
                                prob.awr, prec)
        self.init_materials(prob.mat_off, prob.nuc_id, prob.density)
        self.set_tally(prob.edges)

    def set_weight_windows(self, lower, ratio=5.0, survival=2.5, max_split=10):
        """Windows for problem slot 0: lower [n_cells, n_bins] (0: none)."""
        lo = np.ascontiguousarray(lower, dtype=np.float64)
        if lo.ndim != 2:
            raise ValueError("lower must be [n_cells, n_bins]")
        self._ck(lib().gbmc_set_weight_windows(self._h, lo.shape[0], lo.shape[1],
                                               _p(lo, C.c_double), float(ratio), float(survival),
                                               int(max_split)))

    def get_weight_windows(self, n_cells):
        lo = np.zeros((n_cells, self.n_bins))
        self._ck(lib().gbmc_get_weight_windows(self._h, _p(lo, C.c_double), lo.size))
        return lo

    def clear_weight_windows(self):
        self._ck(lib().gbmc_clear_weight_windows(self._h))

    # -- importance network ----------------------------------------------------
    def set_importance_net(self, bf16_params, feat_offset, feat_scale):
        """bf16_params: uint16 BF16 bit patterns [MLP_NPARAM]."""
        p = np.ascontiguousarray(bf16_params, dtype=np.uint16)
        off = np.ascontiguousarray(feat_offset, dtype=np.float64)
        sc = np.ascontiguousarray(feat_scale, dtype=np.float64)
        self._ck(lib().gbmc_set_importance_net(self._h, _p(p, C.c_uint16), len(p),
                                               _p(off, C.c_double), _p(sc, C.c_double)))

    def get_importance_net(self):
        p = np.zeros(MLP_NPARAM, np.uint16)
        self._ck(lib().gbmc_get_importance_net(self._h, _p(p, C.c_uint16), MLP_NPARAM))
        return p

    @staticmethod
    def _dptr(t):
        return C.c_void_p(t if isinstance(t, int) else t.data_ptr())

    def mlp_forward(self, feat, out, stream=None):
        n = feat.shape[0]
        self._ck(lib().gbmc_mlp_forward(self._h, self._dptr(feat), int(n), self._dptr(out),
                                        _stream(stream)))

    def mlp_gradient(self, feat, target, weight, stream=None):
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = C.c_float()
        self._ck(lib().gbmc_mlp_gradient(self._h, self._dptr(feat), self._dptr(target),
                                         self._dptr(weight), int(feat.shape[0]),
                                         _p(g, C.c_float), C.byref(loss), _stream(stream)))
        return loss.value, g

    def mlp_train(self, feat, target, weight, steps, lr, stream=None):
        loss = C.c_float()
        self._ck(lib().gbmc_mlp_train(self._h, self._dptr(feat), self._dptr(target),
                                      self._dptr(weight), int(feat.shape[0]), int(steps),
                                      float(lr), C.byref(loss), _stream(stream)))
        return loss.value

    def mesh_rows(self, geom) -> int:
        n = C.c_int64()
        self._ck(lib().gbmc_mesh_features(self._h, C.byref(geom), None, 0, C.byref(n), None))
        return n.value

    def mesh_features(self, geom, feat, stream=None):
        n = C.c_int64()
        self._ck(lib().gbmc_mesh_features(self._h, C.byref(geom), self._dptr(feat),
                                          int(feat.shape[0]), C.byref(n), _stream(stream)))
        return n.value

    def weight_windows_from_net(self, geom, ratio=5.0, survival=2.5, max_split=10, stream=None):
        self._ck(lib().gbmc_weight_windows_from_net(self._h, C.byref(geom), float(ratio),
                                                    float(survival), int(max_split),
                                                    _stream(stream)))

    def importance_record(self, geom=None, capacity=0):
        self._ck(lib().gbmc_importance_record(self._h, C.byref(geom) if geom is not None else None,
                                              int(capacity)))

    def importance_accumulate(self, stream=None):
        self._ck(lib().gbmc_importance_accumulate(self._h, _stream(stream)))

    def importance_training_set(self, geom, feat, target, weight, stream=None):
        n = C.c_int64()
        self._ck(lib().gbmc_importance_training_set(self._h, C.byref(geom), self._dptr(feat),
                                                    self._dptr(target), self._dptr(weight),
                                                    int(feat.shape[0]), C.byref(n),
                                                    _stream(stream)))
        return n.value

    def reset_tallies(self, stream=None):
        self._ck(lib().gbmc_reset_tallies(self._h, _stream(stream)))

    # -- runs -----------------------------------------------------------------
    def run_batch(self, prob: Problem, stream=None):
        self._ck(lib().gbmc_run_batch(self._h, C.byref(prob), _stream(stream)))
        self._cells = [_n_cells(prob.geom)]

    def run_problems(self, probs, stream=None):
        arr = (Problem * len(probs))(*probs)
        self._ck(lib().gbmc_run_problems(self._h, len(probs), arr, _stream(stream)))
        self._cells = [_n_cells(p.geom) for p in probs]

    def run_concurrent(self, probs, n_loops: int, per_run: int = 1, stream=None):
        """gbmc_run_concurrent: the results of run_problems(probs), computed by
        n_loops concurrent event loops, each taking runs of per_run
        consecutive problems in turn."""
        arr = (Problem * len(probs))(*probs)
        self._ck(lib().gbmc_run_concurrent(self._h, len(probs), arr, int(n_loops), int(per_run),
                                           _stream(stream)))
        self._cells = [_n_cells(p.geom) for p in probs]

    def run_concurrent_to_host(self, probs, n_loops: int, dests, per_run: int = 1, stream=None):
        """gbmc_run_concurrent_to_host: run_concurrent, each run's results
        copied to the host as soon as it ends.  dests[p] is a dict with any of
        the keys flux, counts, weights, n_coll, status, n_flights, n_draws, E,
        x, y, z, each a C-contiguous numpy array (pinned memory for the copies
        to overlap the work) of the dtype and size read_tallies / read_outcomes
        give for problem p; the arrays hold the results once `stream` has
        passed the call.  The arrays must stay alive until then."""
        if len(dests) != len(probs):
            raise ValueError("one destination per problem")
        arr = (Problem * len(probs))(*probs)
        dst = (HostResults * len(probs))()
        for p, (pr, d) in enumerate(zip(probs, dests)):
            cells = _n_cells(pr.geom)
            for name, a in d.items():
                if name not in _RESULT_FIELDS:
                    raise KeyError(name)
                dt, per_particle = _RESULT_FIELDS[name]
                want = (pr.n_particles if per_particle else
                        cells * self.n_bins if name == "flux" else NSCAL)
                if (not isinstance(a, np.ndarray) or a.dtype != dt or a.size != want
                        or not a.flags["C_CONTIGUOUS"]):
                    raise TypeError(f"problem {p}: {name} must be a C-contiguous {np.dtype(dt)} "
                                    f"array of {want}")
                setattr(dst[p], name, a.ctypes.data)
        self._ck(lib().gbmc_run_concurrent_to_host(self._h, len(probs), arr, int(n_loops),
                                                   int(per_run), dst, _stream(stream)))
        self._cells = [_n_cells(p.geom) for p in probs]

    def profile_problems(self, probs, stream=None, trace_cap: int = 0):
        """Run with every kernel launched eagerly between CUDA events; returns
        {kernel: (total ms, launches)}, and with trace_cap > 0 also a
        per-iteration trace (ms [iters, len(KERNEL_NAMES)]; lookups, ray-traced particles,
        collisions and particles in flight [iters, 4])."""
        arr = (Problem * len(probs))(*probs)
        kt = KernelTimes()
        tms = np.zeros((max(trace_cap, 1), len(KERNEL_NAMES)))
        tq = np.zeros((max(trace_cap, 1), 4), np.int32)
        tl = C.c_int32(0)
        self._ck(lib().gbmc_profile_problems(self._h, len(probs), arr, _stream(stream),
                                             C.byref(kt), int(trace_cap), _p(tms, C.c_double),
                                             _p(tq, C.c_int32), C.byref(tl)))
        self._cells = [_n_cells(p.geom) for p in probs]
        totals = {name: (kt.ms[k], kt.launches[k]) for k, name in enumerate(KERNEL_NAMES)}
        if trace_cap > 0:
            return totals, tms[:tl.value], tq[:tl.value]
        return totals

    def autotune(self, probs, fraction: float = 0.1, stream=None) -> dict:
        """gbmc_autotune: pick launch/queue settings by timing probe runs of
        these problems scaled by `fraction`; the context keeps the choice."""
        arr = (Problem * len(probs))(*probs)
        best = Options()
        rep = AutotuneReport()
        self._ck(lib().gbmc_autotune(self._h, len(probs), arr, float(fraction), _stream(stream),
                                     C.byref(best), C.byref(rep)))
        self.options = best
        out = {name: getattr(rep, name) for name, _ in AutotuneReport._fields_ if name != "reserved"}
        out["options"] = {name: getattr(best, name) for name, _ in Options._fields_
                          if name != "reserved"}
        return out

    # -- read-back ------------------------------------------------------------
    def read_tallies(self, slot: int = 0, out=None):
        """(flux [cells, bins], counts, weights) of a problem slot; `out` may
        hold preallocated arrays of those shapes (for example in pinned host
        memory) to fill instead."""
        nc = self._cells[slot]
        if out is not None:
            flux, counts, weights = out
        else:
            flux = np.zeros((nc, self.n_bins))
            counts = np.zeros(NSCAL, np.int64)
            weights = np.zeros(NSCAL)
        self._ck(lib().gbmc_read_tallies(self._h, int(slot), _p(flux, C.c_double), flux.size,
                                         _p(counts, C.c_int64), _p(weights, C.c_double)))
        return flux, counts, weights

    # -- k-eigenvalue -------------------------------------------------------------
    def load_fission(self, nu, f_fis):
        a, b = _arr(nu, np.float64), _arr(f_fis, np.float64)
        self._ck(lib().gbmc_load_fission(self._h, len(a), _p(a, C.c_double), _p(b, C.c_double)))

    def set_eigen(self, k_norm: float, max_sites: int = 32):
        self._ck(lib().gbmc_set_eigen(self._h, float(k_norm), int(max_sites)))

    def read_bank(self, sites: bool = True):
        """The last run's fission bank [n, 3] in history order (or its size)."""
        n = C.c_int64()
        self._ck(lib().gbmc_read_bank(self._h, None, 0, C.byref(n)))
        if not sites:
            return n.value
        out = np.zeros((n.value, 3))
        self._ck(lib().gbmc_read_bank(self._h, _p(out, C.c_double), n.value, C.byref(n)))
        return out

    def set_source_bank(self, xyz=None, n_total: int = 0):
        """Source bank for GBMC_SRC_BANK runs: host sites [n, 3], or None for
        the last run's own bank."""
        if xyz is None:
            self._ck(lib().gbmc_set_source_bank(self._h, None, 0, int(n_total)))
        else:
            a = _arr(xyz, np.float64).reshape(-1, 3)
            self._ck(lib().gbmc_set_source_bank(self._h, _p(a, C.c_double), len(a), int(n_total)))

    def check_division(self, n: int, seed: int = 1, kind: int = 0):
        """gbmc_check_division: kind 0 checks the integer-unit division, kind 1
        the lookup's interpolation factor from interval records; returns
        (results that differ from the hardware binary64 ones, first such
        operand pair)."""
        bad = C.c_int64()
        first = np.zeros(2)
        self._ck(lib().gbmc_check_division(self._h, int(kind), int(n),
                                           int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(bad),
                                           _p(first, C.c_double)))
        return bad.value, first

    def measure_fp64_rate(self) -> float:
        """gbmc_measure_fp64_rate: binary64 instructions per second (per thread)."""
        r = C.c_double()
        self._ck(lib().gbmc_measure_fp64_rate(self._h, C.byref(r)))
        return r.value

    def set_reaction_tally(self, on: bool = True):
        self._ck(lib().gbmc_set_reaction_tally(self._h, 1 if on else 0))

    def read_reaction_tally(self, slot: int = 0):
        """Track-length absorption rate sum w d Sigma_a [cells, bins] of a slot."""
        out = np.zeros((self._cells[slot], self.n_bins))
        self._ck(lib().gbmc_read_reaction_tally(self._h, int(slot), _p(out, C.c_double), out.size))
        return out

    def read_outcomes(self, slot: int = 0, first: int = 0, n: int = 0, out=None):
        """Per-particle outcomes of ids [first, first + n) of a slot; `out` may
        be a dict of preallocated arrays (n_coll int32, status int8, n_flights
        int32, n_draws uint32, E, x, y, z float64) to fill instead."""
        o = out if out is not None else dict(
            n_coll=np.zeros(n, np.int32), status=np.zeros(n, np.int8),
            n_flights=np.zeros(n, np.int32), n_draws=np.zeros(n, np.uint32),
            E=np.zeros(n), x=np.zeros(n), y=np.zeros(n), z=np.zeros(n))
        self._ck(lib().gbmc_read_outcomes(
            self._h, int(slot), int(first), int(n), _p(o["n_coll"], C.c_int32),
            _p(o["status"], C.c_int8), _p(o["n_flights"], C.c_int32),
            _p(o["n_draws"], C.c_uint32), _p(o["E"], C.c_double), _p(o["x"], C.c_double),
            _p(o["y"], C.c_double), _p(o["z"], C.c_double)))
        return o

    def read_stats(self) -> dict:
        s = Stats()
        self._ck(lib().gbmc_read_stats(self._h, C.byref(s)))
        return {name: getattr(s, name) for name, _ in Stats._fields_ if name != "reserved"}

    def last_run_ms(self) -> float:
        ms = C.c_double()
        self._ck(lib().gbmc_last_run_ms(self._h, C.byref(ms)))
        return ms.value

    def lookup_macro(self, E, mat, sigma_t, sigma_a, precision=FP64, sort=False, stream=None):
        """E (float64), mat (int32), sigma_t, sigma_a (float64): contiguous
        CUDA tensors of equal length on this context's device, written in
        query order."""
        n = _lookup_args(E, mat, sigma_t, sigma_a)
        self._ck(lib().gbmc_lookup_macro(self._h, int(precision), C.c_void_p(E.data_ptr()),
                                         C.c_void_p(mat.data_ptr()), n,
                                         C.c_void_p(sigma_t.data_ptr()),
                                         C.c_void_p(sigma_a.data_ptr()), 1 if sort else 0,
                                         _stream(stream)))

    def lookup_macro_noalloc(self, E, mat, sigma_t, sigma_a, precision=FP64, stream=None):
        """The sorted lookup of lookup_macro(sort=True) with no device
        allocation, for callers that cannot allocate device memory while they
        call the library.  At most NOALLOC_MAX_QUERIES queries per call;
        calls that overlap on the GPU must not be issued (they share one
        scratch area).  Make the first call on a device before any stream
        capture.  Arguments as in lookup_macro."""
        n = _lookup_args(E, mat, sigma_t, sigma_a)
        self._ck(lib().gbmc_lookup_macro_noalloc(self._h, int(precision),
                                                 C.c_void_p(E.data_ptr()),
                                                 C.c_void_p(mat.data_ptr()), n,
                                                 C.c_void_p(sigma_t.data_ptr()),
                                                 C.c_void_p(sigma_a.data_ptr()),
                                                 _stream(stream)))


def _lookup_args(E, mat, sigma_t, sigma_a) -> int:
    """Checks the standalone lookup's tensors (the library cannot check device
    buffers): float64 energies and outputs, int32 materials, all contiguous
    CUDA tensors of one length on one device.  Returns the length."""
    want = (("E", E, "torch.float64"), ("mat", mat, "torch.int32"),
            ("sigma_t", sigma_t, "torch.float64"), ("sigma_a", sigma_a, "torch.float64"))
    dev = None
    for name, t, dt in want:
        if not (hasattr(t, "data_ptr") and hasattr(t, "is_cuda")):
            raise TypeError(f"{name} must be a torch tensor")
        if str(t.dtype) != dt:
            raise TypeError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError(f"{name} is on {t.device}, E on {dev}")
    n = E.numel()
    if any(t.numel() != n for _, t, _ in want):
        raise ValueError("E, mat, sigma_t and sigma_a must have the same length")
    return int(n)


def _n_cells(g: Geometry) -> int:
    if g.kind == GEOM_LATTICE:
        return g.n * g.n
    if g.kind == GEOM_SLAB:
        return g.n_layers
    return 1
