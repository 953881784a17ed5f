"""Plain FP64 CPU oracle of the unlimited ADER-DG scheme (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

The arithmetic lives in ``aderdg_oracle.c`` (plain loops, strict IEEE FP64,
compiled with ``-ffp-contract=off``); this module compiles it with gcc on
first use and wraps it with ctypes + numpy.  Section / equation references
are to Dumbser et al. (2018):

* ``operators``      1D basis: GL nodes and weights, nodal derivative,
                     stiffness and time matrices (Sec. 2.1, eq. D_kl)
* ``predictor``      element-local space-time predictor, Picard iteration
                     (Sec. 2.2, eq. pde.st2)
* ``volume``/``traces``/``rusanov``  pieces of the corrector
                     (Sec. 2.1, eq. pde.nc.gw2, pc.scheme, rusanov)
* ``step``/``run``   whole ADER-DG steps on a periodic Cartesian mesh,
                     CFL step of Sec. 3
* ``mass``           conserved totals (diagnostic)

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, exact solutions and brute-force solves.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aderdg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

PDE_ADVECTION, PDE_EULER, PDE_ELASTICITY, PDE_DIFFUSE_ELASTICITY = 1, 2, 3, 4


class Cfg(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("cells", C.c_int * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("N", C.c_int),
        ("m", C.c_int),
        ("pde", C.c_int),
        ("prm", C.c_double * 8),
        ("picard", C.c_int),
        ("alpha", C.c_double),
        ("guess", C.c_int),
        ("limiter", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (strict FP64, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
               "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            cp = C.POINTER(Cfg)
            L.orc_gauss_legendre.argtypes = [C.c_int, dp, dp]
            L.orc_lagrange_eval.argtypes = [C.c_int, dp, C.c_double, dp]
            L.orc_lagrange_deriv.argtypes = [C.c_int, dp, C.c_double, dp]
            L.orc_operators.argtypes = [C.c_int, dp, dp, dp, dp, dp, dp, dp]
            L.orc_nvar.argtypes = [C.c_int, C.c_int]
            L.orc_flux.argtypes = [cp, dp, C.c_int, dp]
            L.orc_flux.restype = None
            L.orc_max_eig.argtypes = [cp, dp, C.c_int]
            L.orc_max_eig.restype = C.c_double
            L.orc_max_eigs.argtypes = [cp, dp, dp]
            L.orc_max_eigs.restype = None
            L.orc_predictor.argtypes = [cp, dp, C.c_double, dp, dp, dp, C.POINTER(C.c_int)]
            L.orc_initial_guess.argtypes = [cp, dp, C.c_double, dp]
            L.orc_initial_guess_extrap.argtypes = [cp, dp, C.c_double, dp, C.c_double, dp]
            L.orc_volume.argtypes = [cp, dp, dp]
            L.orc_traces.argtypes = [cp, dp, dp, dp, dp]
            L.orc_rusanov.argtypes = [cp, C.c_int, dp, dp, dp, dp, dp]
            L.orc_rusanov.restype = None
            L.orc_ncp.argtypes = [cp, dp, C.c_int, dp, dp]
            L.orc_ncp.restype = None
            L.orc_detect.argtypes = [cp, dp, dp, C.POINTER(C.c_int)]
            L.orc_detect.restype = C.c_long
            L.orc_source.argtypes = [cp, dp, dp]
            L.orc_source.restype = None
            L.orc_path_jump.argtypes = [cp, C.c_int, dp, dp, dp]
            L.orc_path_jump.restype = None
            L.orc_face_flux.argtypes = [cp, C.c_int, dp, dp, dp, dp, dp, dp]
            L.orc_face_flux.restype = None
            L.orc_nevolved.argtypes = [cp]
            L.orc_cerk_weights.argtypes = [C.c_int, C.c_double, dp]
            L.orc_cerk_weights.restype = None
            L.orc_cerk_scheme.argtypes = [C.c_int, dp, dp, C.POINTER(C.c_int)]
            L.orc_cerk_scheme.restype = C.c_int
            L.orc_step_limited.argtypes = [cp, dp, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_long)]
            L.orc_subcell_ops.argtypes = [C.c_int, dp, dp]
            ip = C.POINTER(C.c_int)
            L.orc_step_limited_kept.argtypes = [cp, dp, dp, ip, C.c_double, ip, C.POINTER(C.c_long)]
            L.orc_cfl_dt_kept.argtypes = [cp, dp, dp, ip]
            L.orc_cfl_dt_kept.restype = C.c_double
            L.orc_subcell_init.argtypes = [cp, dp, dp]
            L.orc_run_kept.argtypes = [cp, dp, dp, ip, C.c_double, C.c_double, C.c_long, dp,
                                       C.POINTER(C.c_long), dp]
            L.orc_cfl_dt.argtypes = [cp, dp]
            L.orc_cfl_dt.restype = C.c_double
            L.orc_step_ex.argtypes = [cp, dp, C.c_double, dp, dp, dp]
            L.orc_step.argtypes = [cp, dp, C.c_double]
            L.orc_run.argtypes = [cp, dp, C.c_double, C.c_double, C.c_long, dp,
                                  C.POINTER(C.c_long), dp]
            L.orc_step_sampled.argtypes = [cp, dp, C.c_double, C.c_long, C.POINTER(C.c_long), dp]
            L.orc_mass.argtypes = [cp, dp, dp]
            L.orc_node_coords.argtypes = [cp, dp]
            L.orc_picard_count.argtypes = [cp]
            L.orc_alpha.argtypes = [cp]
            L.orc_alpha.restype = C.c_double
            L.orc_threads.argtypes = []
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = None
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def nvar(pde: int, dim: int) -> int:
    return lib().orc_nvar(pde, dim)


GUESS_TRIVIAL, GUESS_ORDER2, GUESS_ORDER3, GUESS_EXTRAP, GUESS_CERK = 0, 1, 2, 3, 4


def make_cfg(dim, cells, lo, hi, N, pde, prm=(), picard=0, alpha=0.0, guess=GUESS_TRIVIAL, limiter=0) -> Cfg:
    c = Cfg()
    c.dim = dim
    for d in range(3):
        c.cells[d] = int(cells[d]) if d < dim else 1
        c.lo[d] = float(lo[d]) if d < dim else 0.0
        c.hi[d] = float(hi[d]) if d < dim else 1.0
    c.N = N
    c.pde = pde
    c.m = nvar(pde, dim)
    for i, v in enumerate(prm):
        c.prm[i] = float(v)
    c.picard = picard
    c.alpha = alpha
    c.guess = guess
    c.limiter = limiter
    return c


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss_legendre(n, _p(x), _p(w)):
        raise ValueError("n out of range")
    return x, w


def lagrange_eval(nodes: np.ndarray, xi: float) -> np.ndarray:
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    out = np.zeros(len(nodes))
    lib().orc_lagrange_eval(len(nodes), _p(nodes), float(xi), _p(out))
    return out


def lagrange_deriv(nodes: np.ndarray, xi: float) -> np.ndarray:
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    out = np.zeros(len(nodes))
    lib().orc_lagrange_deriv(len(nodes), _p(nodes), float(xi), _p(out))
    return out


def operators(n: int) -> dict:
    """1D operators for n = N+1 nodes: x, w, Dhat[j,k] = phi_k'(x_j),
    Kxi[k,l] = int phi_k' phi_l, K1 = F1 F1^T - Kxi, F0, F1."""
    x, w, F0, F1 = (np.zeros(n) for _ in range(4))
    Dhat, Kxi, K1 = (np.zeros((n, n)) for _ in range(3))
    if lib().orc_operators(n, _p(x), _p(w), _p(Dhat), _p(Kxi), _p(K1), _p(F0), _p(F1)):
        raise ValueError("n out of range")
    return dict(x=x, w=w, Dhat=Dhat, Kxi=Kxi, K1=K1, F0=F0, F1=F1)


def flux(cfg: Cfg, q: np.ndarray, d: int) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    f = np.zeros(cfg.m)
    lib().orc_flux(C.byref(cfg), _p(q), d, _p(f))
    return f


def max_eig(cfg: Cfg, q: np.ndarray, d: int) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().orc_max_eig(C.byref(cfg), _p(q), d)


def max_eigs(cfg: Cfg, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_max_eigs(C.byref(cfg), _p(U), _p(out))
    return out[: cfg.dim]


def predictor(cfg: Cfg, u: np.ndarray, dt: float):
    """One element: returns (qhat[n, n^d, m], qbar[n^d, m], Fbar[d, n^d, m], iters)."""
    n = cfg.N + 1
    ns = n ** cfg.dim
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.size == ns * cfg.m
    qhat = np.zeros((n, ns, cfg.m))
    qbar = np.zeros((ns, cfg.m))
    Fbar = np.zeros((cfg.dim, ns, cfg.m))
    it = C.c_int(0)
    rc = lib().orc_predictor(C.byref(cfg), _p(u), float(dt), _p(qhat), _p(qbar), _p(Fbar), C.byref(it))
    if rc:
        raise RuntimeError("orc_predictor failed: %d" % rc)
    return qhat, qbar, Fbar, it.value


def initial_guess(cfg: Cfg, u: np.ndarray, dt: float) -> np.ndarray:
    """One element: the initial guess q0[n, n^d, m] of cfg.guess (Sec. 2.2)."""
    n = cfg.N + 1
    ns = n ** cfg.dim
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.size == ns * cfg.m
    q0 = np.zeros((n, ns, cfg.m))
    if lib().orc_initial_guess(C.byref(cfg), _p(u), float(dt), _p(q0)):
        raise RuntimeError("orc_initial_guess failed")
    return q0


def cerk_scheme(N: int):
    """The continuous Runge-Kutta scheme of the CERK guess for degree N:
    (A [s, s] strictly lower triangular, beta [s, p]) with the dense-output
    weights b_i(theta) = sum_k beta[i, k] theta^(k+1); p is its order."""
    a = np.zeros(256)  # s <= 16 stages, order <= 16
    beta = np.zeros(256)
    p = C.c_int()
    s = lib().orc_cerk_scheme(int(N), _p(a), _p(beta), C.byref(p))
    return a[:s * s].reshape(s, s).copy(), beta[:s * p.value].reshape(s, p.value).copy()


def cerk_weights(theta: float, N: int = 4) -> np.ndarray:
    """The dense-output weights b_i(theta) of the CERK guess for degree N."""
    out = np.zeros(16)
    lib().orc_cerk_weights(int(N), float(theta), _p(out))
    return out[:cerk_scheme(N)[0].shape[0]].copy()


def initial_guess_extrap(cfg: Cfg, u: np.ndarray, dt: float, qprev: np.ndarray, ratio: float) -> np.ndarray:
    """One element: the extrapolation guess (cfg.guess == GUESS_EXTRAP) from the
    previous predictor qprev[n, n^d, m] over an interval dt / ratio."""
    n = cfg.N + 1
    ns = n ** cfg.dim
    u = np.ascontiguousarray(u, dtype=np.float64)
    qprev = np.ascontiguousarray(qprev, dtype=np.float64)
    assert u.size == ns * cfg.m and qprev.size == n * ns * cfg.m
    q0 = np.zeros((n, ns, cfg.m))
    if lib().orc_initial_guess_extrap(C.byref(cfg), _p(u), float(dt), _p(qprev), float(ratio), _p(q0)):
        raise RuntimeError("orc_initial_guess_extrap failed")
    return q0


def volume(cfg: Cfg, Fbar: np.ndarray) -> np.ndarray:
    ns = (cfg.N + 1) ** cfg.dim
    Fbar = np.ascontiguousarray(Fbar, dtype=np.float64)
    V = np.zeros((ns, cfg.m))
    lib().orc_volume(C.byref(cfg), _p(Fbar), _p(V))
    return V


def traces(cfg: Cfg, qbar: np.ndarray, Fbar: np.ndarray):
    """Returns (qface, fface), each [d, 2, n^{d-1}, m] (side 0: xi_d = 0)."""
    nf = (cfg.N + 1) ** (cfg.dim - 1)
    qf = np.zeros((cfg.dim, 2, nf, cfg.m))
    ff = np.zeros((cfg.dim, 2, nf, cfg.m))
    lib().orc_traces(C.byref(cfg), _p(np.ascontiguousarray(qbar, dtype=np.float64)),
                     _p(np.ascontiguousarray(Fbar, dtype=np.float64)), _p(qf), _p(ff))
    return qf, ff


def rusanov(cfg: Cfg, d: int, qL, fL, qR, fR) -> np.ndarray:
    out = np.zeros(cfg.m)
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (qL, fL, qR, fR)]
    lib().orc_rusanov(C.byref(cfg), d, *[_p(x) for x in a], _p(out))
    return out


def ncp(cfg: Cfg, q: np.ndarray, d: int, g: np.ndarray) -> np.ndarray:
    """Non-conservative product B_d(q) g."""
    out = np.zeros(cfg.m)
    lib().orc_ncp(C.byref(cfg), _p(np.ascontiguousarray(q, dtype=np.float64)), d,
                  _p(np.ascontiguousarray(g, dtype=np.float64)), _p(out))
    return out


def source(cfg: Cfg, q: np.ndarray) -> np.ndarray:
    out = np.zeros(cfg.m)
    lib().orc_source(C.byref(cfg), _p(np.ascontiguousarray(q, dtype=np.float64)), _p(out))
    return out


def path_jump(cfg: Cfg, d: int, qL, qR) -> np.ndarray:
    """int_0^1 B_d(qL + s (qR - qL)) ds (qR - qL), three-point Gauss-Legendre."""
    out = np.zeros(cfg.m)
    lib().orc_path_jump(C.byref(cfg), d, _p(np.ascontiguousarray(qL, dtype=np.float64)),
                        _p(np.ascontiguousarray(qR, dtype=np.float64)), _p(out))
    return out


def face_flux(cfg: Cfg, d: int, qL, fL, qR, fR):
    """(f_lower, f_upper): the face fluctuations of the lower and upper element."""
    lo, up = np.zeros(cfg.m), np.zeros(cfg.m)
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (qL, fL, qR, fR)]
    lib().orc_face_flux(C.byref(cfg), d, *[_p(x) for x in a], _p(lo), _p(up))
    return lo, up


def nevolved(cfg: Cfg) -> int:
    return lib().orc_nevolved(C.byref(cfg))


def n_elems(cfg: Cfg) -> int:
    E = 1
    for d in range(cfg.dim):
        E *= cfg.cells[d]
    return E


def cfl_dt(cfg: Cfg, U: np.ndarray) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_cfl_dt(C.byref(cfg), _p(U))


def step(cfg: Cfg, U: np.ndarray, dt: float, with_parts: bool = False):
    """One step with a given dt; returns u^{n+1} (and V, qface, fface if asked)."""
    n = cfg.N + 1
    ns, nf = n ** cfg.dim, n ** (cfg.dim - 1)
    E = n_elems(cfg)
    out = np.array(U, dtype=np.float64, copy=True, order="C")
    assert out.size == E * ns * cfg.m
    if with_parts:
        V = np.zeros((E, ns, cfg.m))
        qf = np.zeros((E, cfg.dim, 2, nf, cfg.m))
        ff = np.zeros((E, cfg.dim, 2, nf, cfg.m))
        rc = lib().orc_step_ex(C.byref(cfg), _p(out), float(dt), _p(V), _p(qf), _p(ff))
    else:
        rc = lib().orc_step(C.byref(cfg), _p(out), float(dt))
    if rc:
        raise RuntimeError("orc_step failed: %d" % rc)
    return (out, V, qf, ff) if with_parts else out


def step_limited(cfg: Cfg, U: np.ndarray, dt: float):
    """One step with the subcell limiter: (u^{n+1}, troubled[E] flags, count)."""
    out = np.array(U, dtype=np.float64, copy=True, order="C")
    E = n_elems(cfg)
    flags = np.zeros(E, dtype=np.int32)
    cnt = C.c_long(0)
    rc = lib().orc_step_limited(C.byref(cfg), _p(out), float(dt), flags.ctypes.data_as(C.POINTER(C.c_int)),
                                C.byref(cnt))
    if rc:
        raise RuntimeError("orc_step_limited failed: %d" % rc)
    return out, flags, cnt.value


class Kept:
    """The limiter's kept subcell data (R35, limiter mode 2): sub[E, (2N+1)^d,
    m], the subcell averages of the elements the last step limited, and
    kept[E], set for those elements."""

    def __init__(self, cfg: Cfg, sub=None, kept=None):
        E, nsub = n_elems(cfg), (2 * cfg.N + 1) ** cfg.dim
        self.sub = np.zeros((E, nsub, cfg.m)) if sub is None else np.array(sub, dtype=np.float64, order="C")
        self.kept = np.zeros(E, dtype=np.int32) if kept is None else np.array(kept, dtype=np.int32, order="C")
        assert self.sub.size == E * nsub * cfg.m and self.kept.size == E

    def _k(self):
        return self.kept.ctypes.data_as(C.POINTER(C.c_int))


def subcell_init(cfg: Cfg, avg: np.ndarray):
    """R35: a state given as the subcell averages avg[E, (2N+1)^d, m] of every
    element: (U, Kept) with U their least-squares reconstruction (R28) and
    every element carrying avg."""
    avg = np.ascontiguousarray(avg, dtype=np.float64)
    E, ns = n_elems(cfg), (cfg.N + 1) ** cfg.dim
    U = np.zeros((E, ns, cfg.m))
    if lib().orc_subcell_init(C.byref(cfg), _p(avg), _p(U)):
        raise RuntimeError("orc_subcell_init failed")
    return U, Kept(cfg, avg, np.ones(E, dtype=np.int32))


def step_limited_kept(cfg: Cfg, U: np.ndarray, kept: Kept, dt: float):
    """One step with the subcell limiter keeping the limited elements'
    subcell data (R35): (u^{n+1}, troubled flags, count); kept is updated in
    place."""
    out = np.array(U, dtype=np.float64, copy=True, order="C")
    flags = np.zeros(n_elems(cfg), dtype=np.int32)
    cnt = C.c_long(0)
    rc = lib().orc_step_limited_kept(C.byref(cfg), _p(out), _p(kept.sub), kept._k(), float(dt),
                                     flags.ctypes.data_as(C.POINTER(C.c_int)), C.byref(cnt))
    if rc:
        raise RuntimeError("orc_step_limited_kept failed: %d" % rc)
    return out, flags, cnt.value


def cfl_dt_kept(cfg: Cfg, U: np.ndarray, kept: Kept) -> float:
    """The CFL step with the kept elements' wave speeds from their subcell
    averages (R35)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_cfl_dt_kept(C.byref(cfg), _p(U), _p(kept.sub), kept._k())


def run_kept(cfg: Cfg, U: np.ndarray, kept: Kept, t_end: float, t0: float = 0.0, max_steps: int = 10**9):
    """CFL time loop to t_end with the kept subcell data of R35 (updated in
    place).  Returns (U, t, steps, dt_history)."""
    out = np.array(U, dtype=np.float64, copy=True, order="C")
    hist_len = int(min(max_steps, 10**6))
    hist = np.zeros(hist_len)
    t = C.c_double(0.0)
    k = C.c_long(0)
    rc = lib().orc_run_kept(C.byref(cfg), _p(out), _p(kept.sub), kept._k(), float(t0), float(t_end),
                            int(hist_len), C.byref(t), C.byref(k), _p(hist))
    if rc:
        raise RuntimeError("orc_run_kept failed: %d" % rc)
    return out, t.value, k.value, hist[: k.value].copy()


def detect(cfg: Cfg, U0: np.ndarray, U: np.ndarray):
    """The limiter's detection alone (Sec. 2.3, R25): (troubled[E] flags,
    count) of the candidate U against the state U0 at t^n."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    flags = np.zeros(n_elems(cfg), dtype=np.int32)
    cnt = lib().orc_detect(C.byref(cfg), _p(U0), _p(U), flags.ctypes.data_as(C.POINTER(C.c_int)))
    if cnt < 0:
        raise RuntimeError("orc_detect failed: %d" % cnt)
    return flags, int(cnt)


def subcell_ops(N: int):
    """1D subcell operators: Pr[(2N+1), N+1] (subcell averages of the nodal
    basis) and Rc[N+1, 2N+1] (least-squares reconstruction)."""
    n, S = N + 1, 2 * N + 1
    Pr = np.zeros((S, n))
    Rc = np.zeros((n, S))
    if lib().orc_subcell_ops(N, _p(Pr), _p(Rc)):
        raise RuntimeError("orc_subcell_ops failed")
    return Pr, Rc


def run(cfg: Cfg, U: np.ndarray, t_end: float, t0: float = 0.0, max_steps: int = 10**9):
    """CFL time loop to t_end.  Returns (U, t, steps, dt_history)."""
    out = np.array(U, dtype=np.float64, copy=True, order="C")
    hist_len = int(min(max_steps, 10**6))
    hist = np.zeros(hist_len)
    t = C.c_double(0.0)
    k = C.c_long(0)
    rc = lib().orc_run(C.byref(cfg), _p(out), float(t0), float(t_end), int(hist_len),
                       C.byref(t), C.byref(k), _p(hist))
    if rc:
        raise RuntimeError("orc_run failed: %d" % rc)
    return out, t.value, k.value, hist[: k.value].copy()


def step_sampled(cfg: Cfg, U: np.ndarray, dt: float, elems) -> np.ndarray:
    """u^{n+1} of the listed elements only: [len(elems), n^d, m]."""
    ns = (cfg.N + 1) ** cfg.dim
    U = np.ascontiguousarray(U, dtype=np.float64)
    el = np.ascontiguousarray(np.asarray(elems, dtype=np.int64))
    out = np.zeros((len(el), ns, cfg.m))
    rc = lib().orc_step_sampled(C.byref(cfg), _p(U), float(dt), len(el),
                                el.ctypes.data_as(C.POINTER(C.c_long)), _p(out))
    if rc:
        raise RuntimeError("orc_step_sampled failed: %d" % rc)
    return out


def mass(cfg: Cfg, U: np.ndarray) -> np.ndarray:
    M = np.zeros(cfg.m)
    lib().orc_mass(C.byref(cfg), _p(np.ascontiguousarray(U, dtype=np.float64)), _p(M))
    return M


def node_coords(cfg: Cfg) -> np.ndarray:
    """Physical coordinates of every node, [E, n^d, dim]."""
    ns = (cfg.N + 1) ** cfg.dim
    X = np.zeros((n_elems(cfg), ns, cfg.dim))
    lib().orc_node_coords(C.byref(cfg), _p(X))
    return X


def picard_count(cfg: Cfg) -> int:
    return lib().orc_picard_count(C.byref(cfg))


def alpha(cfg: Cfg) -> float:
    return lib().orc_alpha(C.byref(cfg))


def threads() -> int:
    return lib().orc_threads()


def set_threads(n: int) -> None:
    """OpenMP threads of later oracle calls (n <= 0: the default)."""
    lib().orc_set_threads(int(n))
