"""The partitioned solver (aderdg_dd_*) on one GPU: the mesh split into
blocks, the boundary-first predictor, the face-trace exchange overlapping
the interior predictor, the corrector on the received traces and the
global wave-speed reduction (the distributed-memory structure of Sec. 2.2).
Every block does the undivided mesh's arithmetic on the same data, so the
states must equal the single-domain solver's bit for bit, and the oracle's
within the FP64 tolerance."""
import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import aderdg as A
from paper_1808_03788_gb300 import inputs
from helpers import l2_rel

pytestmark = pytest.mark.gpu

EL = (1.0, 2.0, 1.0)


def _ic(pde, dim, X, L):
    if pde == A.ADERDG_PDE_DIFFUSE_ELASTICITY:
        return inputs.diffuse_terrain(X, width=0.1) if dim == 3 else None
    return inputs.smooth_random_state(pde, X, [L] * dim, seed=5)


def _pair_run(pde, dim, cells, L, N, params, parts, steps, **kw):
    lo, hi = (0.0,) * dim, (L,) * dim
    cfg = oracle.make_cfg(dim, cells, lo, hi, N, pde, params)
    X = oracle.node_coords(cfg)
    U0 = _ic(pde, dim, X, L)
    out = []
    for cls, extra in ((A.Solver, {}), (A.Partitioned, {"parts": parts})):
        with cls(pde, dim, cells, lo, hi, N, params, **kw, **extra) as s:
            s.set_state(U0)
            s.advance(1e30, max_steps=steps)
            out.append(s.get_state())
    return cfg, U0, out


CASES = [
    (A.ADERDG_PDE_EULER, 2, (24, 20), 2.0, 3, (1.4,), (2, 2)),
    (A.ADERDG_PDE_EULER, 2, (24, 20), 2.0, 4, (1.4,), (3, 1)),
    (A.ADERDG_PDE_EULER, 2, (17, 9), 2.0, 2, (1.4,), (1, 4)),
    (A.ADERDG_PDE_ADVECTION, 2, (8, 4), 1.0, 3, (1.0, -0.5), (4, 4)),  # no interior elements
    (A.ADERDG_PDE_ELASTICITY, 3, (6, 5, 4), 1.0, 2, EL, (2, 1, 2)),
    (A.ADERDG_PDE_EULER, 3, (5, 4, 6), 1.0, 2, (1.4,), (2, 2, 3)),
]


def _ids(c):
    return "%s-%dd-N%d-parts%s" % ({1: "adv", 2: "euler", 3: "elastic", 4: "diffuse"}[c[0]], c[1], c[4],
                                    "x".join(map(str, c[6])))


@pytest.mark.parametrize("precision", [A.ADERDG_FP64, A.ADERDG_MIXED_FP32], ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_partitioned_equals_single_domain_bitwise(case, precision):
    pde, dim, cells, L, N, params, parts = case
    _, _, ((U1, t1, k1), (U2, t2, k2)) = _pair_run(pde, dim, cells, L, N, params, parts, 12, precision=precision)
    assert (t1, k1) == (t2, k2) and k1 == 12
    np.testing.assert_array_equal(U2, U1)


@pytest.mark.parametrize("precision", [A.ADERDG_FP64, A.ADERDG_MIXED_FP32], ids=["fp64", "mixed"])
@pytest.mark.parametrize("shapes", [(1, 5), (0, 4), (0, 3)])
def test_partitioned_corrector_shapes_read_the_halos(shapes, precision):
    """Every corrector shape reads the neighbouring blocks' traces and (FP32
    path) reference states from the halos: the pipelined shape 5 stages them
    with the next group of elements.  Bitwise the undivided mesh's result."""
    for case in (CASES[0], CASES[4]):
        pde, dim, cells, L, N, params, parts = case
        lo, hi = (0.0,) * dim, (L,) * dim
        cfg = oracle.make_cfg(dim, cells, lo, hi, N, pde, params)
        U0 = _ic(pde, dim, oracle.node_coords(cfg), L)
        out = []
        for cls, extra in ((A.Solver, {}), (A.Partitioned, {"parts": parts, "shapes": shapes})):
            with cls(pde, dim, cells, lo, hi, N, params, precision=precision, **extra) as s:
                s.set_state(U0)
                s.advance(1e30, max_steps=6)
                out.append(s.get_state())
        (U1, t1, k1), (U2, t2, k2) = out
        assert (t1, k1) == (t2, k2)
        np.testing.assert_array_equal(U2, U1)


def test_partitioned_matches_the_oracle():
    pde, dim, cells, L, N, params, parts = CASES[0]
    cfg, U0, (_, (Ug, t, k)) = _pair_run(pde, dim, cells, L, N, params, parts, 8)
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=1e30, max_steps=8)
    assert ko == k == 8 and abs(to - t) <= 1e-14 * t
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


@pytest.mark.parametrize("guess", [A.ADERDG_GUESS_ORDER3, A.ADERDG_GUESS_EXTRAP, A.ADERDG_GUESS_CERK],
                         ids=["order3", "extrap", "cerk"])
def test_partitioned_initial_guesses_bitwise(guess):
    pde, dim, cells, L, N, params, parts = CASES[1]
    _, _, ((U1, t1, k1), (U2, t2, k2)) = _pair_run(pde, dim, cells, L, N, params, parts, 10, guess=guess)
    assert (t1, k1) == (t2, k2)
    np.testing.assert_array_equal(U2, U1)


def test_partitioned_non_conservative_system_bitwise():
    """The diffuse-interface system (path-conservative faces read the halo
    states of the neighbouring block)."""
    for precision in (A.ADERDG_FP64, A.ADERDG_MIXED_FP32):
        _, _, ((U1, t1, k1), (U2, t2, k2)) = _pair_run(A.ADERDG_PDE_DIFFUSE_ELASTICITY, 3, (6, 4, 5), 1.0, 2, (),
                                                       (2, 2, 1), 6, precision=precision)
        assert (t1, k1) == (t2, k2)
        np.testing.assert_array_equal(U2, U1)


def test_partitioned_step_clips_and_reports_dt():
    pde, dim, cells, L, N, params, parts = CASES[0]
    cfg = oracle.make_cfg(dim, cells, (0,) * dim, (L,) * dim, N, pde, params)
    U0 = _ic(pde, dim, oracle.node_coords(cfg), L)
    dt0 = oracle.cfl_dt(cfg, U0)
    with A.Partitioned(pde, dim, cells, (0,) * dim, (L,) * dim, N, params, parts=parts) as s:
        s.set_state(U0)
        assert abs(s.step(1.0, sync_dt=True) - dt0) <= 1e-14 * dt0
        t_end = 1.5 * dt0
        dt1 = s.step(t_end, sync_dt=True)
        _, t, k = s.get_state()
        assert t == t_end and k == 2 and 0 < dt1 <= dt0 * 1.01
        info = s.dd_info()
        assert info["blocks"] == 4 and info["boundary_elements"] > 0 and info["halo_bytes_per_step"] > 0


def test_partitioned_rejects_the_limiter_and_bad_parts():
    import ctypes as C
    L = A.load()
    mesh = A._mesh(2, (8, 8), (0, 0), (1, 1))
    p = A.aderdg_pde_t()
    p.kind = A.ADERDG_PDE_EULER
    p.p[0] = 1.4
    cfg = A.aderdg_config_t()
    cfg.limiter = 1
    h = A._H()
    assert L.aderdg_dd_create(C.byref(mesh), 3, 4, C.byref(p), C.byref(cfg), A._parts((2, 2)),
                              C.byref(h)) == A.ADERDG_E_UNSUPPORTED
    cfg.limiter = 0
    assert L.aderdg_dd_create(C.byref(mesh), 3, 4, C.byref(p), C.byref(cfg), A._parts((9, 1)),
                              C.byref(h)) == A.ADERDG_E_INVAL
