"""Parity of the CUDA path (through the C ABI) with the FP64 oracle for the
purely non-conservative diffuse-interface elasticity system of Sec. 3.2
(B(q) grad q in the predictor and the volume term, path-conservative
Rusanov faces with the three-point path integral) and for the algebraic
source (advection with reaction).

Tolerances as for the conservative systems: one predictor/corrector call
within 1e-12 of the data scale, full runs within 1e-11 relative L2 in FP64
and 1e-6 in the mixed mode.  The material fields (alpha, lambda, mu, rho)
stay bitwise constant on both paths."""
import math

import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import aderdg as A
from paper_1808_03788_gb300 import inputs
from helpers import l2_rel

pytestmark = pytest.mark.gpu

DI = A.ADERDG_PDE_DIFFUSE_ELASTICITY
CASES = [(2, N, (5, 3)) for N in (2, 3, 4)] + [(3, N, (3, 2, 3)) for N in (2, 3)]


def _ids(c):
    return "%dd-N%d" % (c[0], c[1])


def _di_state(cfg, seed, alpha_vac=0.05):
    """Smooth random stresses and velocities with element-wise noise; a
    diffuse free surface across the last coordinate (alpha from 1 to
    alpha_vac) and smoothly varying lambda, mu, rho."""
    dim = cfg.dim
    X = oracle.node_coords(cfg)
    L = [cfg.hi[d] - cfg.lo[d] for d in range(dim)]
    nsig = 6 if dim == 3 else 3
    ev = inputs.smooth_random_state(1, X, L, seed=seed, amp=0.3, modes=3)[..., 0]
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    fields = [ev * rng.uniform(-1, 1) + 0.05 * rng.uniform(-1, 1, ev.shape) for _ in range(nsig + dim)]
    z = X[..., dim - 1]
    alpha = inputs.smooth_step(z, 0.5 * L[-1], 0.12 * L[-1], 1.0, alpha_vac)
    lam = 2.0 + 0.5 * np.sin(2 * math.pi * X[..., 0] / L[0])
    mu = 1.0 + 0.3 * np.cos(2 * math.pi * X[..., 1] / L[1])
    rho = 1.2 + 0.2 * np.sin(2 * math.pi * (X[..., 0] + X[..., 1]) / L[0])
    w = [alpha * f for f in fields[nsig:]]
    return inputs.diffuse_pack(dim, fields[:nsig], w, alpha, lam, mu, rho)


def _pair(dim, N, cells, precision=A.ADERDG_FP64, **kw):
    cfg = oracle.make_cfg(dim, cells, [0.0] * dim, [1.0] * dim, N, oracle.PDE_DIFFUSE_ELASTICITY, [],
                          picard=kw.get("picard", 0), guess=kw.get("guess", 0))
    s = A.Solver(DI, dim, cells, [0.0] * dim, [1.0] * dim, N, (), precision=precision, **kw)
    return cfg, s


def _scale(a):
    return max(1.0, float(np.abs(a).max()))


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_predictor_outputs_match_oracle(case):
    """The volume term (the oracle averages B(q_t) grad q_t over the time
    nodes; the kernel evaluates it once at qbar -- equal for this system)
    and the face traces."""
    dim, N, cells = case
    cfg, s = _pair(dim, N, cells)
    U = _di_state(cfg, seed=300 + N)
    dt = oracle.cfl_dt(cfg, U)
    _, Vo, qfo, ffo = oracle.step(cfg, U, dt, with_parts=True)
    s.set_state(U)
    s.predictor(dt)
    V, qf, ff = s.predictor_outputs()
    s.close()
    assert np.abs(V - Vo).max() <= 1e-12 * _scale(Vo)
    assert np.abs(qf - qfo).max() <= 1e-12 * _scale(qfo)
    assert np.all(ff == 0.0) and np.all(ffo == 0.0)
    nev = oracle.nevolved(cfg)
    assert np.all(V[..., nev:] == 0.0)


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("precision", [A.ADERDG_FP64, A.ADERDG_MIXED_FP32])
def test_corrector_matches_oracle(case, precision):
    dim, N, cells = case
    cfg, s = _pair(dim, N, cells, precision=precision)
    U = _di_state(cfg, seed=400 + N)
    dt = oracle.cfl_dt(cfg, U)
    Uo = oracle.step(cfg, U, dt)
    s.set_state(U)
    s.predictor(dt)
    s.corrector(dt)
    Ug, _, _ = s.get_state()
    s.close()
    nev = oracle.nevolved(cfg)
    assert np.array_equal(Ug[..., nev:], U[..., nev:])
    if precision == A.ADERDG_FP64:
        assert np.abs(Ug - Uo).max() <= 1e-12 * _scale(Uo)
    else:
        # one step changes u by O(dt); its FP32 part is the increment
        assert np.abs(Ug - Uo).max() <= 1e-6 * _scale(Uo - U) + 1e-12 * _scale(Uo)


@pytest.mark.parametrize("case", [(2, 3, (8, 6)), (3, 2, (4, 3, 4))], ids=_ids)
@pytest.mark.parametrize("precision", [A.ADERDG_FP64, A.ADERDG_MIXED_FP32])
def test_full_run_matches_oracle(case, precision):
    """Full CFL runs through a diffuse surface (alpha from 1 to 0.3, where
    multi-dimensional runs of the scheme stay bounded; with alpha <= 0.1
    they grow, and both paths amplify their rounding differences)."""
    dim, N, cells = case
    cfg, s = _pair(dim, N, cells, precision=precision)
    U0 = _di_state(cfg, seed=500 + N, alpha_vac=0.3)
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.08)
    s.set_state(U0)
    s.advance(0.08)
    Ug, t, k = s.get_state()
    s.close()
    assert (t, k) == (to, ko) and k >= 10
    nev = oracle.nevolved(cfg)
    assert np.array_equal(Ug[..., nev:], U0[..., nev:])
    tol = 1e-11 if precision == A.ADERDG_FP64 else 1e-6
    err = l2_rel(cfg, Ug[..., :nev], Uo[..., :nev])
    assert err <= tol, err


def test_free_surface_slab_matches_oracle():
    """The quasi-1D free-surface reflection of the oracle's pins (alpha
    from 1 to 0.01 over two elements), run to the reflection on the GPU."""
    c = oracle.make_cfg(2, (80, 1), [0, 0], [2.0, 2.0 / 80], 3, oracle.PDE_DIFFUSE_ELASTICITY, [])
    X = oracle.node_coords(c)
    x = X[..., 0]
    alpha = inputs.smooth_step(x, 1.25, 0.025, 1.0, 1e-2) + inputs.smooth_step(-x, -0.25, 0.025, 1.0, 1e-2) - 1.0
    f = np.exp(-((x - 0.6) / 0.08) ** 2)
    U0 = inputs.diffuse_pack(2, [-2.0 * f, -1.0 * f, 0 * f], [alpha * f, 0 * f], alpha, 2.0, 1.0, 1.0)
    Uo, to, ko, _ = oracle.run(c, U0, 0.55)
    with A.Solver(DI, 2, (80, 1), (0, 0), (2.0, 2.0 / 80), 3, ()) as s:
        s.set_state(U0)
        s.advance(0.55)
        Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    live = [0, 1, 3]  # sxx, syy, w_x; sxy and w_y stay at rounding level (~1e-16) on both sides
    assert l2_rel(c, Ug[..., live], Uo[..., live]) <= 1e-11
    assert np.abs(Ug[..., [2, 4]]).max() < 1e-12 and np.abs(Uo[..., [2, 4]]).max() < 1e-12
    assert Ug[..., 0][(x > 0.3) & (x < 1.1)].max() > 1.7  # the reflected, sign-flipped stress


def test_alpha_one_equals_the_conservative_elastic_path():
    """alpha = 1 with constant material: the non-conservative kernels and
    the conservative elasticity kernels give the same run (rounding)."""
    cells, N = (4, 3, 3), 3
    cfg = oracle.make_cfg(3, cells, [0] * 3, [1] * 3, N, oracle.PDE_ELASTICITY, [1.0, 2.0, 1.0])
    U9 = inputs.smooth_random_state(3, oracle.node_coords(cfg), (1, 1, 1), seed=11)
    U13 = inputs.diffuse_pack(3, [U9[..., i] for i in range(6)], [U9[..., 6 + i] for i in range(3)], 1.0, 2.0,
                              1.0, 1.0)
    with A.Solver(3, 3, cells, (0, 0, 0), (1, 1, 1), N, (1.0, 2.0, 1.0)) as s:
        s.set_state(U9)
        s.advance(0.04)
        Ue, te, ke = s.get_state()
    with A.Solver(DI, 3, cells, (0, 0, 0), (1, 1, 1), N, ()) as s:
        s.set_state(U13)
        s.advance(0.04)
        Ud, td, kd = s.get_state()
    assert (te, ke) == (td, kd)
    assert l2_rel(cfg, Ud[..., :9], Ue) <= 1e-12


@pytest.mark.parametrize("guess,picard", [(A.ADERDG_GUESS_ORDER3, 1), (A.ADERDG_GUESS_EXTRAP, 1)])
def test_initial_guesses_match_oracle(guess, picard):
    """The L operator of the initial guesses (Sec. 2.2) with the
    non-conservative product; the extrapolation guess across steps."""
    dim, N, cells = 2, 3, (6, 5)
    cfg, s = _pair(dim, N, cells, guess=guess, picard=picard)
    U0 = _di_state(cfg, seed=600, alpha_vac=0.3)  # bounded regime: rounding differences do not grow
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.05)
    s.set_state(U0)
    s.advance(0.05)
    Ug, t, k = s.get_state()
    s.close()
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug[..., :5], Uo[..., :5]) <= 1e-11


def test_batch_mixes_non_conservative_and_conservative_solves():
    """A batch holding a diffuse-interface solve, an Euler solve and an
    advection-reaction solve: each bitwise equal to the same solve alone."""
    specs = [A.make_spec(DI, 2, (6, 4), (0, 0), (1, 1), 3, ()),
             A.make_spec(2, 2, (5, 5), (0, 0), (10, 10), 3, (1.4,)),
             A.make_spec(1, 2, (7, 3), (0, 0), (1, 1), 2, (1.0, 0.5, 0.0, 0.7))]
    cfg0 = oracle.make_cfg(2, (6, 4), [0, 0], [1, 1], 3, oracle.PDE_DIFFUSE_ELASTICITY, [])
    cfg1 = oracle.make_cfg(2, (5, 5), [0, 0], [10, 10], 3, oracle.PDE_EULER, [1.4])
    cfg2 = oracle.make_cfg(2, (7, 3), [0, 0], [1, 1], 2, oracle.PDE_ADVECTION, [1.0, 0.5, 0.0, 0.7])
    states = [_di_state(cfg0, seed=700), inputs.euler_vortex(oracle.node_coords(cfg1)),
              inputs.advection_sine(oracle.node_coords(cfg2), a=(1.0, 0.5))]
    t_end = [0.05, 0.2, 0.1]
    b = A.Batch(specs)
    for i, U in enumerate(states):
        b.set_state(i, U)
    b.advance(t_end)
    for i, (sp, U) in enumerate(zip(specs, states)):
        a = [(1, 1), (10, 10), (1, 1)][i]
        with A.Solver(sp.pde.kind, 2, (sp.mesh.cells[0], sp.mesh.cells[1]), (0, 0), a, sp.N,
                      tuple(sp.pde.p[:4])) as s:
            s.set_state(U)
            s.advance(t_end[i])
            alone = s.get_state()[0].reshape(-1)
        np.testing.assert_array_equal(b.get_state(i)[0], alone)
    b.close()


# ---- algebraic source: advection with reaction ----------------------------

RCASES = [(2, 3, (6, 5), (1.0, -0.6, 0.0, 0.9)), (2, 6, (4, 3), (0.4, 1.0, 0.0, 2.0)),
          (3, 2, (3, 3, 2), (0.5, -0.3, 0.9, 1.5))]


@pytest.mark.parametrize("case", RCASES, ids=lambda c: "%dd-N%d" % (c[0], c[1]))
@pytest.mark.parametrize("precision", [A.ADERDG_FP64, A.ADERDG_MIXED_FP32])
def test_reaction_full_run_matches_oracle(case, precision):
    dim, N, cells, prm = case
    cfg = oracle.make_cfg(dim, cells, [0.0] * dim, [1.0] * dim, N, oracle.PDE_ADVECTION, prm)
    U0 = inputs.advection_sine(oracle.node_coords(cfg), a=prm[:dim]) + 0.3
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.3)
    with A.Solver(1, dim, cells, [0.0] * dim, [1.0] * dim, N, prm, precision=precision) as s:
        s.set_state(U0)
        s.advance(0.3)
        Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    tol = 1e-11 if precision == A.ADERDG_FP64 else 1e-6
    assert l2_rel(cfg, Ug, Uo) <= tol
    assert abs(np.mean(Ug) / np.mean(U0) - math.exp(-prm[3] * 0.3)) < 0.02  # decays like exp(-kappa t)


@pytest.mark.parametrize("shapes", [(3, 0), (4, 1)])
def test_reaction_plane_kernel_matches_oracle(shapes):
    """The plane-owning 2D FP32 predictor carries the source too."""
    prm = (1.0, -0.6, 0.0, 0.9)
    cfg = oracle.make_cfg(2, (6, 5), [0, 0], [1, 1], 3, oracle.PDE_ADVECTION, prm)
    U0 = inputs.advection_sine(oracle.node_coords(cfg), a=prm[:2]) + 0.3
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.3)
    with A.Solver(1, 2, (6, 5), (0, 0), (1, 1), 3, prm, precision=A.ADERDG_MIXED_FP32, shapes=shapes) as s:
        s.set_state(U0)
        s.advance(0.3)
        Ug, t, k = s.get_state()
        assert s.info()["pred_shape"] == shapes[0]
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-6


def test_server_serves_the_non_conservative_system_and_cerk_requests():
    """Requests of the diffuse-interface system (FP64 and mixed) and an Euler
    request with the CERK guess, served together: each result bitwise equal
    to the same solve alone."""
    import time
    cfg = oracle.make_cfg(2, (6, 4), [0, 0], [1, 1], 3, oracle.PDE_DIFFUSE_ELASTICITY, [])
    ud = _di_state(cfg, seed=900, alpha_vac=0.3)
    ue = inputs.euler_vortex(oracle.node_coords(oracle.make_cfg(2, (8, 8), [0, 0], [10, 10], 4, 2, [1.4])))
    reqs = [(A.make_spec(DI, 2, (6, 4), (0, 0), (1, 1), 3, ()), ud, 0.05, A.ADERDG_FP64, 0),
            (A.make_spec(DI, 2, (6, 4), (0, 0), (1, 1), 3, ()), ud, 0.05, A.ADERDG_MIXED_FP32, 0),
            (A.make_spec(2, 2, (8, 8), (0, 0), (10, 10), 4, (1.4,)), ue, 0.2, A.ADERDG_MIXED_FP32,
             A.ADERDG_GUESS_CERK)]
    srv = A.Server(precision=A.ADERDG_FP64, steps_per_round=4)
    tickets = [srv.submit(sp, u0, te, precision=prec, guess=g) for sp, u0, te, prec, g in reqs]
    res = {}
    t0 = time.time()
    while len(res) < len(tickets) and time.time() - t0 < 120:
        for tk in tickets:
            if tk not in res:
                r = srv.poll(tk)
                if r is not None:
                    res[tk] = r
        time.sleep(0.002)
    assert len(res) == len(tickets)
    for tk, (sp, u0, te, prec, g) in zip(tickets, reqs):
        assert res[tk]["status"] == A.ADERDG_OK
        dim = sp.mesh.dim
        with A.Solver(sp.pde.kind, dim, [sp.mesh.cells[d] for d in range(dim)], [sp.mesh.lo[d] for d in range(dim)],
                      [sp.mesh.hi[d] for d in range(dim)], sp.N, tuple(sp.pde.p[:1]) if sp.pde.kind == 2 else (),
                      precision=prec, guess=g) as s:
            s.set_state(u0)
            s.advance(te)
            alone, t, k = s.get_state()
        assert res[tk]["steps"] == k and res[tk]["t"] == t
        np.testing.assert_array_equal(res[tk]["u"], alone.reshape(-1))
        srv.release(tk)
    srv.close()
