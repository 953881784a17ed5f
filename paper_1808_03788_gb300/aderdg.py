"""ctypes binding of libaderdg.so with the names of include/aderdg.h.

Argument marshalling only: every step of the ADER-DG path runs in the CUDA
kernels of the library.  PyTorch provides device memory (through the
library's allocator hook, so buffers come from torch's caching allocator)
and streams.  There is no CPU fallback: if the library cannot be built or
loaded, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

ADERDG_OK = 0
ADERDG_PENDING = 1
ADERDG_E_INVAL = -1
ADERDG_E_NOMEM = -2
ADERDG_E_CUDA = -3
ADERDG_E_NONFINITE = -4
ADERDG_E_TIMEOUT = -5
ADERDG_E_BUSY = -6
ADERDG_E_UNSUPPORTED = -7
ADERDG_E_CANCELLED = -8

ADERDG_PDE_ADVECTION, ADERDG_PDE_EULER, ADERDG_PDE_ELASTICITY, ADERDG_PDE_DIFFUSE_ELASTICITY = 1, 2, 3, 4
ADERDG_FP64, ADERDG_MIXED_FP32 = 0, 1
ADERDG_HOST, ADERDG_DEVICE = 0, 1
ADERDG_NUM_PRED_SHAPES, ADERDG_NUM_CORR_SHAPES = 9, 6
ADERDG_SHAPE_DEFAULT, ADERDG_SHAPE_AUTOTUNE = 0, -1
ADERDG_TUNE_FORCE = 1
ADERDG_GUESS_TRIVIAL, ADERDG_GUESS_ORDER2, ADERDG_GUESS_ORDER3, ADERDG_GUESS_EXTRAP, ADERDG_GUESS_CERK = 0, 1, 2, 3, 4


class AderdgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("aderdg error %d: %s" % (code, msg))
        self.code = code


class aderdg_mesh_t(C.Structure):
    _fields_ = [("dim", C.c_int), ("cells", C.c_int64 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class aderdg_pde_t(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 8)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class aderdg_alloc_t(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class aderdg_config_t(C.Structure):
    _fields_ = [("precision", C.c_int), ("picard_iters", C.c_int), ("cfl_alpha", C.c_double),
                ("cuda_stream", C.c_void_p), ("alloc", C.POINTER(aderdg_alloc_t)),
                ("pred_shape", C.c_int), ("corr_shape", C.c_int), ("tune_cache", C.c_char_p),
                ("initial_guess", C.c_int), ("limiter", C.c_int)]


class aderdg_info_t(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("nvar", C.c_int), ("precision", C.c_int),
                ("picard_iters", C.c_int), ("elements", C.c_int64), ("dofs", C.c_int64),
                ("cfl_alpha", C.c_double), ("flops_predictor", C.c_double),
                ("flops_corrector", C.c_double), ("bytes_predictor", C.c_double),
                ("bytes_corrector", C.c_double), ("device_bytes", C.c_size_t),
                ("pred_shape", C.c_int), ("pred_threads", C.c_int), ("pred_epb", C.c_int),
                ("corr_shape", C.c_int), ("corr_threads", C.c_int), ("corr_epb", C.c_int),
                ("initial_guess", C.c_int)]


class aderdg_dd_block_t(C.Structure):
    _fields_ = [("rank", C.c_int), ("coords", C.c_int * 3), ("offset", C.c_int64 * 3), ("cells", C.c_int64 * 3),
                ("neighbour", (C.c_int * 2) * 3), ("elements", C.c_int64), ("boundary_elements", C.c_int64),
                ("face_chunks", (C.c_int64 * 2) * 3)]


class aderdg_solve_spec_t(C.Structure):
    _fields_ = [("mesh", aderdg_mesh_t), ("N", C.c_int), ("pde", aderdg_pde_t)]


class aderdg_server_config_t(C.Structure):
    _fields_ = [("device_budget_bytes", C.c_size_t), ("max_queue", C.c_int), ("steps_per_round", C.c_int),
                ("precision", C.c_int), ("cuda_stream", C.c_void_p), ("pred_shape", C.c_int),
                ("corr_shape", C.c_int), ("tune_cache", C.c_char_p), ("initial_guess", C.c_int)]


class aderdg_request_t(C.Structure):
    _fields_ = [("spec", aderdg_solve_spec_t), ("u0", C.POINTER(C.c_double)), ("t_end", C.c_double),
                ("precision", C.c_int), ("initial_guess", C.c_int)]


class aderdg_result_t(C.Structure):
    _fields_ = [("status", C.c_int), ("latency_s", C.c_double), ("queue_s", C.c_double), ("t", C.c_double),
                ("steps", C.c_int64), ("u", C.POINTER(C.c_double)), ("n_values", C.c_size_t)]


_lib = None
_lock = threading.Lock()

_DP = C.POINTER(C.c_double)
_H = C.c_void_p

# name -> (restype, argtypes); mirrors include/aderdg.h
_SIGS = {
    "aderdg_last_error": (C.c_char_p, []),
    "aderdg_version": (C.c_int, []),
    "aderdg_gl_nodes": (C.c_int, [C.c_int, _DP, _DP]),
    "aderdg_default_alpha": (C.c_double, [C.c_int]),
    "aderdg_create": (C.c_int, [C.POINTER(aderdg_mesh_t), C.c_int, C.c_int, C.POINTER(aderdg_pde_t),
                                C.POINTER(aderdg_config_t), C.POINTER(_H)]),
    "aderdg_destroy": (C.c_int, [_H]),
    "aderdg_get_info": (C.c_int, [_H, C.POINTER(aderdg_info_t)]),
    "aderdg_set_state": (C.c_int, [_H, C.c_void_p, C.c_int, C.c_double]),
    "aderdg_get_state": (C.c_int, [_H, C.c_void_p, C.c_int, _DP, C.POINTER(C.c_int64)]),
    "aderdg_predictor": (C.c_int, [_H, C.c_double]),
    "aderdg_corrector": (C.c_int, [_H, C.c_double]),
    "aderdg_get_predictor_outputs": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "aderdg_troubled": (C.c_int, [_H, C.c_void_p, C.POINTER(C.c_int64)]),
    "aderdg_set_subcell_state": (C.c_int, [_H, C.c_void_p, C.c_int, C.c_double]),
    "aderdg_get_subcell_state": (C.c_int, [_H, C.c_void_p, C.c_int]),
    "aderdg_step": (C.c_int, [_H, C.c_double, _DP]),
    "aderdg_advance": (C.c_int, [_H, C.c_double, C.c_int64]),
    "aderdg_cfl_dt": (C.c_int, [_H, _DP]),
    "aderdg_mass": (C.c_int, [_H, _DP]),
    "aderdg_sync": (C.c_int, [_H]),
    "aderdg_profile": (C.c_int, [_H, C.c_int]),
    "aderdg_profile_read": (C.c_int, [_H, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "aderdg_peak_tflops": (C.c_int, [C.c_int, _DP]),
    "aderdg_device_recip": (C.c_int, [_DP, _DP, C.c_longlong, C.c_int]),
    "aderdg_autotune": (C.c_int, [C.POINTER(aderdg_solve_spec_t), C.c_int, C.c_char_p, C.c_int,
                                  C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "aderdg_batch_create": (C.c_int, [C.POINTER(aderdg_solve_spec_t), C.c_int, C.POINTER(aderdg_config_t),
                                      C.POINTER(_H)]),
    "aderdg_batch_destroy": (C.c_int, [_H]),
    "aderdg_batch_set_state": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_int, C.c_double]),
    "aderdg_batch_get_state": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_int, _DP, C.POINTER(C.c_int64)]),
    "aderdg_batch_step": (C.c_int, [_H, _DP]),
    "aderdg_batch_advance": (C.c_int, [_H, _DP, C.c_int64]),
    "aderdg_batch_info": (C.c_int, [_H, C.POINTER(C.c_int64), C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "aderdg_batch_status": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "aderdg_batch_troubled": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "aderdg_server_create": (C.c_int, [C.POINTER(aderdg_server_config_t), C.POINTER(_H)]),
    "aderdg_server_destroy": (C.c_int, [_H]),
    "aderdg_submit": (C.c_int, [_H, C.POINTER(aderdg_request_t), C.POINTER(C.c_uint64)]),
    "aderdg_poll": (C.c_int, [_H, C.c_uint64, C.POINTER(aderdg_result_t)]),
    "aderdg_release": (C.c_int, [_H, C.c_uint64]),
    "aderdg_cancel": (C.c_int, [_H, C.c_uint64]),
    "aderdg_server_stats": (C.c_int, [_H, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_size_t)]),
    "aderdg_step_noalloc": (C.c_int, [C.POINTER(aderdg_mesh_t), C.c_int, C.c_int, C.POINTER(aderdg_pde_t),
                                      C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "aderdg_dd_plan": (C.c_int, [C.POINTER(aderdg_mesh_t), C.POINTER(C.c_int), C.c_int,
                                 C.POINTER(aderdg_dd_block_t)]),
    "aderdg_dd_face_elements": (C.c_int, [C.POINTER(aderdg_mesh_t), C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int,
                                          C.c_void_p]),
    "aderdg_dd_element_lists": (C.c_int, [C.POINTER(aderdg_mesh_t), C.POINTER(C.c_int), C.c_int, C.c_void_p,
                                          C.c_void_p]),
    "aderdg_dd_create": (C.c_int, [C.POINTER(aderdg_mesh_t), C.c_int, C.c_int, C.POINTER(aderdg_pde_t),
                                   C.POINTER(aderdg_config_t), C.POINTER(C.c_int), C.POINTER(_H)]),
    "aderdg_dd_destroy": (C.c_int, [_H]),
    "aderdg_dd_set_state": (C.c_int, [_H, C.c_void_p, C.c_int, C.c_double]),
    "aderdg_dd_get_state": (C.c_int, [_H, C.c_void_p, C.c_int, _DP, C.POINTER(C.c_int64)]),
    "aderdg_dd_step": (C.c_int, [_H, C.c_double, _DP]),
    "aderdg_dd_advance": (C.c_int, [_H, C.c_double, C.c_int64]),
    "aderdg_dd_info": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_size_t),
                                 C.POINTER(C.c_size_t)]),
}


def library_path() -> str:
    return _build.LIB


def load():
    """Build (if stale) and load libaderdg.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc < 0:
        raise AderdgError(rc, load().aderdg_last_error().decode())
    return rc


# ---- thin functions with the C names ------------------------------------------

def aderdg_version() -> int:
    return load().aderdg_version()


def aderdg_gl_nodes(N: int):
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    _check(load().aderdg_gl_nodes(N, x.ctypes.data_as(_DP), w.ctypes.data_as(_DP)))
    return x, w


def aderdg_default_alpha(N: int) -> float:
    return load().aderdg_default_alpha(N)


def nvar(pde: int, dim: int) -> int:
    return {1: 1, 2: dim + 2, 3: 9, 4: 13 if dim == 3 else 9}[pde]


def _torch_ready():
    """Device tensors handed to the library are read on the library's stream:
    wait until torch's current stream has finished writing them."""
    import torch
    torch.cuda.current_stream().synchronize()


class _TorchAllocator:
    """aderdg_alloc_t backed by torch's CUDA caching allocator."""

    def __init__(self):
        import torch
        self._torch = torch
        self._blocks = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = aderdg_alloc_t(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device="cuda")
        except Exception:
            return None
        p = t.data_ptr()
        self._blocks[p] = t
        return p

    def _do_free(self, ptr, ctx):
        self._blocks.pop(ptr, None)


def _set_shapes(cfg, shapes, tune_cache):
    """Tile-shape request: (predictor, corrector) indices, ADERDG_SHAPE_AUTOTUNE,
    or the string "auto" for both."""
    if shapes == "auto":
        shapes = (ADERDG_SHAPE_AUTOTUNE, ADERDG_SHAPE_AUTOTUNE)
    cfg.pred_shape, cfg.corr_shape = int(shapes[0]), int(shapes[1])
    cfg.tune_cache = None if tune_cache is None else os.fsencode(tune_cache)


class Solver:
    """One ADER-DG solve on a periodic Cartesian mesh (a handle of the C ABI).

    u layout: [E, n^d, m] float64, variable fastest, x-fastest nodes,
    x-fastest elements (include/aderdg.h)."""

    def __init__(self, pde: int, dim: int, cells, lo, hi, N: int, params=(),
                 precision: int = ADERDG_FP64, picard: int = 0, alpha: float = 0.0,
                 stream=None, torch_alloc: bool = True, shapes=(0, 0), tune_cache=None,
                 guess: int = ADERDG_GUESS_TRIVIAL, limiter: int = 0):
        """limiter: 0 / False none, 1 / True the subcell limiter, 2 the
        limiter keeping the limited elements' subcell data between steps."""
        L = load()
        self.dim, self.N, self.pde = dim, N, pde
        self.m = nvar(pde, dim)
        self.n = N + 1
        self.ns = self.n ** dim
        self.cells = tuple(int(c) for c in cells[:dim])
        self.E = int(np.prod(self.cells))
        mesh = aderdg_mesh_t()
        mesh.dim = dim
        for d in range(3):
            mesh.cells[d] = self.cells[d] if d < dim else 1
            mesh.lo[d] = float(lo[d]) if d < dim else 0.0
            mesh.hi[d] = float(hi[d]) if d < dim else 1.0
        p = aderdg_pde_t()
        p.kind = pde
        for i, v in enumerate(params):
            p.p[i] = float(v)
        cfg = aderdg_config_t()
        cfg.precision = precision
        cfg.picard_iters = picard
        cfg.cfl_alpha = alpha
        cfg.initial_guess = guess
        cfg.limiter = int(limiter)
        self.nsub = (2 * N + 1) ** dim
        _set_shapes(cfg, shapes, tune_cache)
        self._alloc = None
        if stream is not None:
            cfg.cuda_stream = C.c_void_p(int(stream))
        if torch_alloc:
            self._alloc = _TorchAllocator()
            cfg.alloc = C.pointer(self._alloc.struct)
        self._h = _H()
        _check(L.aderdg_create(C.byref(mesh), N, self.m, C.byref(p), C.byref(cfg), C.byref(self._h)))
        self._L = L

    # lifetime
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.aderdg_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # state
    def set_state(self, u, t: float = 0.0):
        if hasattr(u, "data_ptr"):  # torch tensor on the device
            assert u.dtype.itemsize == 8 and u.is_contiguous() and u.numel() == self.E * self.ns * self.m
            _torch_ready()
            _check(self._L.aderdg_set_state(self._h, C.c_void_p(u.data_ptr()), ADERDG_DEVICE, float(t)))
            return
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == self.E * self.ns * self.m, (u.shape, self.E, self.ns, self.m)
        _check(self._L.aderdg_set_state(self._h, u.ctypes.data, ADERDG_HOST, float(t)))

    def get_state(self, out=None, check=True):
        """Returns (u [E, n^d, m], t, step).  out may be a device tensor."""
        t = C.c_double(0)
        k = C.c_int64(0)
        if out is not None and hasattr(out, "data_ptr"):
            assert out.is_cuda and out.is_contiguous() and out.numel() * out.element_size() == self.E * self.ns * self.m * 8
            rc = self._L.aderdg_get_state(self._h, C.c_void_p(out.data_ptr()), ADERDG_DEVICE, C.byref(t), C.byref(k))
            u = out
        elif out is not None:  # host numpy array (e.g. a view of pinned memory)
            assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.E * self.ns * self.m
            rc = self._L.aderdg_get_state(self._h, out.ctypes.data, ADERDG_HOST, C.byref(t), C.byref(k))
            u = out
        else:
            u = np.empty((self.E, self.ns, self.m))
            rc = self._L.aderdg_get_state(self._h, u.ctypes.data, ADERDG_HOST, C.byref(t), C.byref(k))
        if check:
            _check(rc)
        return u, t.value, k.value

    # the hot path
    def predictor(self, dt: float):
        _check(self._L.aderdg_predictor(self._h, float(dt)))

    def corrector(self, dt: float):
        _check(self._L.aderdg_corrector(self._h, float(dt)))

    def troubled(self):
        """(flags[E], count) of the last limited step."""
        flags = np.zeros(self.E, dtype=np.int32)
        cnt = C.c_int64(0)
        _check(self._L.aderdg_troubled(self._h, flags.ctypes.data, C.byref(cnt)))
        return flags, cnt.value

    def set_subcell_state(self, avg, t: float = 0.0):
        """The state from the subcell averages avg [E, (2N+1)^d, m] of every
        element (limiter 2)."""
        avg = np.ascontiguousarray(avg, dtype=np.float64)
        assert avg.size == self.E * self.nsub * self.m, (avg.shape, self.E, self.nsub, self.m)
        _check(self._L.aderdg_set_subcell_state(self._h, avg.ctypes.data, ADERDG_HOST, float(t)))

    def get_subcell_state(self):
        """The kept subcell averages [E, (2N+1)^d, m] (rows of the elements
        troubled() marks; the others unspecified)."""
        avg = np.empty((self.E, self.nsub, self.m))
        _check(self._L.aderdg_get_subcell_state(self._h, avg.ctypes.data, ADERDG_HOST))
        return avg

    def predictor_outputs(self):
        nf = self.n ** (self.dim - 1)
        V = np.empty((self.E, self.ns, self.m))
        qf = np.empty((self.E, self.dim, 2, nf, self.m))
        ff = np.empty((self.E, self.dim, 2, nf, self.m))
        _check(self._L.aderdg_get_predictor_outputs(self._h, V.ctypes.data, qf.ctypes.data, ff.ctypes.data,
                                                    ADERDG_HOST))
        return V, qf, ff

    def step(self, t_end: float, sync_dt: bool = False):
        if sync_dt:
            dt = C.c_double(0)
            _check(self._L.aderdg_step(self._h, float(t_end), C.byref(dt)))
            return dt.value
        _check(self._L.aderdg_step(self._h, float(t_end), None))
        return None

    def advance(self, t_end: float, max_steps: int = 2 ** 62):
        _check(self._L.aderdg_advance(self._h, float(t_end), int(max_steps)))

    def cfl_dt(self) -> float:
        dt = C.c_double(0)
        _check(self._L.aderdg_cfl_dt(self._h, C.byref(dt)))
        return dt.value

    def mass(self) -> np.ndarray:
        M = np.zeros(self.m)
        _check(self._L.aderdg_mass(self._h, M.ctypes.data_as(_DP)))
        return M

    def sync(self):
        _check(self._L.aderdg_sync(self._h))

    def profile(self, enable: bool = True):
        _check(self._L.aderdg_profile(self._h, int(enable)))

    def profile_read(self):
        a, b = C.c_float(0), C.c_float(0)
        _check(self._L.aderdg_profile_read(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def info(self) -> dict:
        i = aderdg_info_t()
        _check(self._L.aderdg_get_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in aderdg_info_t._fields_}

    def node_coords(self, lo, hi) -> np.ndarray:
        """Physical coordinates of every node from the library's GL nodes."""
        x, _ = aderdg_gl_nodes(self.N)
        n, dim = self.n, self.dim
        X = np.empty((self.E, self.ns, dim))
        idx = np.indices(self.cells[::-1]).reshape(dim, -1)[::-1]  # x fastest
        sd = np.indices((n,) * dim).reshape(dim, -1)[::-1]
        for d in range(dim):
            h = (hi[d] - lo[d]) / self.cells[d]
            X[:, :, d] = lo[d] + (idx[d][:, None] + x[sd[d]][None, :]) * h
        return X


# functions with the C names, on Solver handles
def aderdg_create(pde, dim, cells, lo, hi, N, params=(), **kw) -> Solver:
    return Solver(pde, dim, cells, lo, hi, N, params, **kw)


def aderdg_destroy(s: Solver):
    s.close()


def aderdg_set_state(s: Solver, u, t=0.0):
    s.set_state(u, t)


def aderdg_get_state(s: Solver):
    return s.get_state()


def aderdg_predictor(s: Solver, dt):
    s.predictor(dt)


def aderdg_corrector(s: Solver, dt):
    s.corrector(dt)


def aderdg_get_predictor_outputs(s: Solver):
    return s.predictor_outputs()


def aderdg_step(s: Solver, t_end, sync_dt=False):
    return s.step(t_end, sync_dt)


def aderdg_advance(s: Solver, t_end, max_steps=2 ** 62):
    s.advance(t_end, max_steps)


def aderdg_cfl_dt(s: Solver):
    return s.cfl_dt()


def aderdg_mass(s: Solver):
    return s.mass()


def aderdg_sync(s: Solver):
    s.sync()


def aderdg_get_info(s: Solver):
    return s.info()


def aderdg_profile(s: Solver, enable=True):
    s.profile(enable)


def aderdg_profile_read(s: Solver):
    return s.profile_read()


def aderdg_peak_tflops(kind: int) -> float:
    """Measured FMA throughput (TFLOP/s): kind 0 FP64, kind 1 FP32."""
    v = C.c_double(0)
    _check(load().aderdg_peak_tflops(int(kind), C.byref(v)))
    return v.value


def aderdg_device_recip(x, precision: int = ADERDG_FP64):
    """1/x as the kernels compute it on the device (check utility)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    _check(load().aderdg_device_recip(x.ctypes.data_as(_DP), y.ctypes.data_as(_DP), x.size, int(precision)))
    return y


def aderdg_autotune(spec: aderdg_solve_spec_t, precision: int = ADERDG_MIXED_FP32, tune_cache=None,
                    force: bool = False):
    """Fastest (predictor, corrector) tile shapes for spec's (PDE, d, N) and
    the measured ms per launch of every shape (-1: not timed, found cached)."""
    shapes = (C.c_int * 2)()
    ms = (C.c_float * (ADERDG_NUM_PRED_SHAPES + ADERDG_NUM_CORR_SHAPES))()
    _check(load().aderdg_autotune(C.byref(spec), int(precision),
                                  None if tune_cache is None else os.fsencode(tune_cache),
                                  ADERDG_TUNE_FORCE if force else 0, shapes, ms))
    return (shapes[0], shapes[1]), list(ms)


ADERDG_NOALLOC_SCRATCH_BYTES = 32 << 20


def aderdg_step_noalloc(pde: int, dim: int, cells, lo, hi, N: int, params, u_in, u_out, dt: float,
                        precision: int = ADERDG_FP64, picard: int = 0, stream=None):
    """One step u_in -> u_out (device tensors, float64, state layout) that
    allocates nothing; see include/aderdg.h."""
    mesh = aderdg_mesh_t()
    mesh.dim = dim
    for d in range(3):
        mesh.cells[d] = int(cells[d]) if d < dim else 1
        mesh.lo[d] = float(lo[d]) if d < dim else 0.0
        mesh.hi[d] = float(hi[d]) if d < dim else 1.0
    p = aderdg_pde_t()
    p.kind = pde
    for i, v in enumerate(params):
        p.p[i] = float(v)
    _check(load().aderdg_step_noalloc(C.byref(mesh), N, nvar(pde, dim), C.byref(p), precision, picard,
                                      C.c_void_p(u_in.data_ptr()), C.c_void_p(u_out.data_ptr()),
                                      float(dt), C.c_void_p(int(stream) if stream else 0)))


# ---- domain decomposition --------------------------------------------------------

def _mesh(dim, cells, lo, hi) -> aderdg_mesh_t:
    mesh = aderdg_mesh_t()
    mesh.dim = dim
    for d in range(3):
        mesh.cells[d] = int(cells[d]) if d < dim else 1
        mesh.lo[d] = float(lo[d]) if d < dim else 0.0
        mesh.hi[d] = float(hi[d]) if d < dim else 1.0
    return mesh


def _parts(parts):
    a = (C.c_int * 3)()
    for d in range(3):
        a[d] = int(parts[d]) if d < len(parts) else 1
    return a


def aderdg_dd_plan(dim: int, cells, parts, rank: int) -> dict:
    """Block `rank` of the partition (host logic; no device needed)."""
    b = aderdg_dd_block_t()
    _check(load().aderdg_dd_plan(C.byref(_mesh(dim, cells, (0,) * 3, (1,) * 3)), _parts(parts), rank, C.byref(b)))
    return {"rank": b.rank, "coords": list(b.coords), "offset": list(b.offset), "cells": list(b.cells),
            "neighbour": [list(b.neighbour[d]) for d in range(3)], "elements": b.elements,
            "boundary_elements": b.boundary_elements, "face_chunks": [list(b.face_chunks[d]) for d in range(3)]}


def aderdg_dd_face_elements(dim: int, cells, parts, rank: int, d: int, side: int) -> np.ndarray:
    """Block-local elements on face (d, side), in the order of the chunks sent across it."""
    n = aderdg_dd_plan(dim, cells, parts, rank)["face_chunks"][d][side]
    out = np.zeros(max(1, n), dtype=np.int64)
    _check(load().aderdg_dd_face_elements(C.byref(_mesh(dim, cells, (0,) * 3, (1,) * 3)), _parts(parts), rank, d,
                                          side, out.ctypes.data))
    return out[:n]


def aderdg_dd_element_lists(dim: int, cells, parts, rank: int):
    """(boundary, interior) block-local element lists of block `rank`."""
    b = aderdg_dd_plan(dim, cells, parts, rank)
    bl = np.zeros(max(1, b["boundary_elements"]), dtype=np.int64)
    il = np.zeros(max(1, b["elements"] - b["boundary_elements"]), dtype=np.int64)
    _check(load().aderdg_dd_element_lists(C.byref(_mesh(dim, cells, (0,) * 3, (1,) * 3)), _parts(parts), rank,
                                          bl.ctypes.data, il.ctypes.data))
    return bl[:b["boundary_elements"]], il[:b["elements"] - b["boundary_elements"]]


class Partitioned(Solver):
    """One solve on a mesh split into parts[0] x parts[1] (x parts[2]) blocks
    (aderdg_dd_* of the C ABI): boundary-first predictor, face-trace
    exchange overlapping the interior predictor, global wave-speed
    reduction.  States are in the global layout, as for Solver."""

    def __init__(self, pde: int, dim: int, cells, lo, hi, N: int, params=(), parts=(2, 2, 1),
                 precision: int = ADERDG_FP64, picard: int = 0, alpha: float = 0.0, stream=None,
                 torch_alloc: bool = True, shapes=(0, 0), tune_cache=None, guess: int = ADERDG_GUESS_TRIVIAL):
        L = load()
        self.dim, self.N, self.pde = dim, N, pde
        self.m = nvar(pde, dim)
        self.n = N + 1
        self.ns = self.n ** dim
        self.cells = tuple(int(c) for c in cells[:dim])
        self.E = int(np.prod(self.cells))
        self.parts = tuple(int(p) for p in parts[:dim])
        mesh = _mesh(dim, cells, lo, hi)
        p = aderdg_pde_t()
        p.kind = pde
        for i, v in enumerate(params):
            p.p[i] = float(v)
        cfg = aderdg_config_t()
        cfg.precision = precision
        cfg.picard_iters = picard
        cfg.cfl_alpha = alpha
        cfg.initial_guess = guess
        _set_shapes(cfg, shapes, tune_cache)
        self._alloc = None
        if stream is not None:
            cfg.cuda_stream = C.c_void_p(int(stream))
        if torch_alloc:
            self._alloc = _TorchAllocator()
            cfg.alloc = C.pointer(self._alloc.struct)
        self._h = _H()
        _check(L.aderdg_dd_create(C.byref(mesh), N, self.m, C.byref(p), C.byref(cfg), _parts(parts),
                                  C.byref(self._h)))
        self._L = L

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.aderdg_dd_destroy(self._h)
            self._h = _H()

    def set_state(self, u, t: float = 0.0):
        if hasattr(u, "data_ptr"):
            assert u.dtype.itemsize == 8 and u.is_contiguous() and u.numel() == self.E * self.ns * self.m
            _torch_ready()
            _check(self._L.aderdg_dd_set_state(self._h, C.c_void_p(u.data_ptr()), ADERDG_DEVICE, float(t)))
            return
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == self.E * self.ns * self.m
        _check(self._L.aderdg_dd_set_state(self._h, u.ctypes.data, ADERDG_HOST, float(t)))

    def get_state(self, out=None, check=True):
        t = C.c_double(0)
        k = C.c_int64(0)
        u = np.empty((self.E, self.ns, self.m)) if out is None else out
        if hasattr(u, "data_ptr"):
            rc = self._L.aderdg_dd_get_state(self._h, C.c_void_p(u.data_ptr()), ADERDG_DEVICE, C.byref(t), C.byref(k))
        else:
            rc = self._L.aderdg_dd_get_state(self._h, u.ctypes.data, ADERDG_HOST, C.byref(t), C.byref(k))
        if check:
            _check(rc)
        return u, t.value, k.value

    def step(self, t_end: float, sync_dt: bool = False):
        if sync_dt:
            dt = C.c_double(0)
            _check(self._L.aderdg_dd_step(self._h, float(t_end), C.byref(dt)))
            return dt.value
        _check(self._L.aderdg_dd_step(self._h, float(t_end), None))
        return None

    def advance(self, t_end: float, max_steps: int = 2 ** 62):
        _check(self._L.aderdg_dd_advance(self._h, float(t_end), int(max_steps)))

    def dd_info(self) -> dict:
        k, nb, hb, db = C.c_int(0), C.c_int64(0), C.c_size_t(0), C.c_size_t(0)
        _check(self._L.aderdg_dd_info(self._h, C.byref(k), C.byref(nb), C.byref(hb), C.byref(db)))
        return {"blocks": k.value, "boundary_elements": nb.value, "halo_bytes_per_step": hb.value,
                "device_bytes": db.value}

    def _unsupported(self, *a, **k):
        raise AderdgError(ADERDG_E_UNSUPPORTED, "not available on a partitioned solver")

    predictor = corrector = troubled = predictor_outputs = cfl_dt = mass = sync = _unsupported
    profile = profile_read = info = _unsupported


# ---- batched solves -------------------------------------------------------------

def make_spec(pde: int, dim: int, cells, lo, hi, N: int, params=()) -> aderdg_solve_spec_t:
    sp = aderdg_solve_spec_t()
    sp.mesh.dim = dim
    for d in range(3):
        sp.mesh.cells[d] = int(cells[d]) if d < dim else 1
        sp.mesh.lo[d] = float(lo[d]) if d < dim else 0.0
        sp.mesh.hi[d] = float(hi[d]) if d < dim else 1.0
    sp.N = N
    sp.pde.kind = pde
    for i, v in enumerate(params):
        sp.pde.p[i] = float(v)
    return sp


def spec_size(sp: aderdg_solve_spec_t) -> int:
    dim = sp.mesh.dim
    E = 1
    for d in range(dim):
        E *= sp.mesh.cells[d]
    return E * (sp.N + 1) ** dim * nvar(sp.pde.kind, dim)


class Batch:
    """Many independent solves advanced together (aderdg_batch_*)."""

    def __init__(self, specs, precision: int = ADERDG_FP64, picard: int = 0, alpha: float = 0.0,
                 stream=None, torch_alloc: bool = True, shapes=(0, 0), tune_cache=None,
                 guess: int = ADERDG_GUESS_TRIVIAL, limiter: bool = False):
        L = load()
        self._L = L
        self.specs = list(specs)
        arr = (aderdg_solve_spec_t * len(self.specs))(*self.specs)
        cfg = aderdg_config_t()
        cfg.precision = precision
        cfg.picard_iters = picard
        cfg.cfl_alpha = alpha
        cfg.initial_guess = guess
        cfg.limiter = int(limiter)
        _set_shapes(cfg, shapes, tune_cache)
        if stream is not None:
            cfg.cuda_stream = C.c_void_p(int(stream))
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator()
            cfg.alloc = C.pointer(self._alloc.struct)
        self._h = _H()
        _check(L.aderdg_batch_create(arr, len(self.specs), C.byref(cfg), C.byref(self._h)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.aderdg_batch_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.specs)

    def set_state(self, i: int, u, t: float = 0.0):
        if hasattr(u, "data_ptr"):  # device tensor
            assert u.is_cuda and u.is_contiguous() and u.numel() == spec_size(self.specs[i])
            _torch_ready()
            _check(self._L.aderdg_batch_set_state(self._h, i, C.c_void_p(u.data_ptr()), ADERDG_DEVICE, float(t)))
            return
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == spec_size(self.specs[i])
        _check(self._L.aderdg_batch_set_state(self._h, i, u.ctypes.data, ADERDG_HOST, float(t)))

    def get_state(self, i: int, check: bool = True):
        u = np.empty(spec_size(self.specs[i]))
        t = C.c_double(0)
        k = C.c_int64(0)
        rc = self._L.aderdg_batch_get_state(self._h, i, u.ctypes.data, ADERDG_HOST, C.byref(t), C.byref(k))
        if check:
            _check(rc)
        return u, t.value, k.value

    def step(self, t_end=None):
        te = None if t_end is None else np.ascontiguousarray(np.broadcast_to(t_end, (len(self),)), dtype=np.float64)
        _check(self._L.aderdg_batch_step(self._h, None if te is None else te.ctypes.data_as(_DP)))

    def advance(self, t_end=None, max_steps: int = 2 ** 62, check: bool = True):
        te = None if t_end is None else np.ascontiguousarray(np.broadcast_to(t_end, (len(self),)), dtype=np.float64)
        rc = self._L.aderdg_batch_advance(self._h, None if te is None else te.ctypes.data_as(_DP), int(max_steps))
        if check:
            _check(rc)
        return rc

    def status(self):
        st = (C.c_int * len(self))()
        _check(self._L.aderdg_batch_status(self._h, st))
        return list(st)

    def troubled(self, i: int):
        """(flags[E], count) of solve i's last limited step."""
        E = 1
        m = self.specs[i].mesh
        for d in range(m.dim):
            E *= m.cells[d]
        flags = np.zeros(E, dtype=np.int32)
        cnt = C.c_int64(0)
        _check(self._L.aderdg_batch_troubled(self._h, i, flags.ctypes.data_as(C.POINTER(C.c_int)), C.byref(cnt)))
        return flags, cnt.value

    def info(self):
        d, b, g = C.c_int64(0), C.c_size_t(0), C.c_int(0)
        _check(self._L.aderdg_batch_info(self._h, C.byref(d), C.byref(b), C.byref(g)))
        return {"dofs": d.value, "device_bytes": b.value, "groups": g.value}


# ---- serving ------------------------------------------------------------------------

class Server:
    """Continuous-batching request server (aderdg_server_*)."""

    def __init__(self, precision: int = ADERDG_FP64, budget_bytes: int = 0, max_queue: int = 0,
                 steps_per_round: int = 0, shapes=(0, 0), tune_cache=None,
                 guess: int = ADERDG_GUESS_TRIVIAL):
        L = load()
        self._L = L
        cfg = aderdg_server_config_t()
        cfg.device_budget_bytes = budget_bytes
        cfg.max_queue = max_queue
        cfg.steps_per_round = steps_per_round
        cfg.precision = precision
        cfg.initial_guess = guess
        _set_shapes(cfg, shapes, tune_cache)
        self._cache = cfg.tune_cache  # keeps the bytes alive while the server runs
        self._h = _H()
        _check(L.aderdg_server_create(C.byref(cfg), C.byref(self._h)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.aderdg_server_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, spec: aderdg_solve_spec_t, u0, t_end: float, precision: int = -1, guess: int = -1) -> int:
        """Queue a solve; precision / guess -1 take the server's."""
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        assert u0.size == spec_size(spec)
        req = aderdg_request_t()
        req.spec = spec
        req.u0 = u0.ctypes.data_as(_DP)
        req.t_end = float(t_end)
        req.precision = int(precision)
        req.initial_guess = int(guess)
        tk = C.c_uint64(0)
        _check(self._L.aderdg_submit(self._h, C.byref(req), C.byref(tk)))
        return tk.value

    def poll(self, ticket: int):
        """None while pending, else a dict (state copied out as numpy)."""
        r = aderdg_result_t()
        rc = self._L.aderdg_poll(self._h, C.c_uint64(ticket), C.byref(r))
        if rc == ADERDG_PENDING:
            return None
        out = {"status": r.status, "latency_s": r.latency_s, "queue_s": r.queue_s, "t": r.t, "steps": r.steps,
               "u": None}
        if r.status == ADERDG_OK and r.u:
            out["u"] = np.ctypeslib.as_array(r.u, shape=(r.n_values,)).copy()
        if rc < 0 and r.status == ADERDG_PENDING:
            _check(rc)
        return out

    def release(self, ticket: int):
        _check(self._L.aderdg_release(self._h, C.c_uint64(ticket)))

    def cancel(self, ticket: int):
        _check(self._L.aderdg_cancel(self._h, C.c_uint64(ticket)))

    def stats(self):
        q, a, f, b = C.c_int64(0), C.c_int64(0), C.c_int64(0), C.c_size_t(0)
        _check(self._L.aderdg_server_stats(self._h, C.byref(q), C.byref(a), C.byref(f), C.byref(b)))
        return {"queued": q.value, "active": a.value, "finished": f.value, "bytes": b.value}
