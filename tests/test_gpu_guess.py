"""Parity of the CUDA path with the oracle for the initial guesses of the
Picard iteration (Sec. 2.2: second and third order, extrapolation of the
previous predictor, CERK), through the C ABI.
Same tolerances as the trivial guess: one predictor call within 1e-12 of
the data scale, full runs within 1e-11 relative L2 in FP64 and 1e-6 in the
mixed path; batched solves equal the same solves alone bitwise."""
import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import aderdg as A
from paper_1808_03788_gb300 import inputs
from helpers import l2_abs, l2_rel

pytestmark = pytest.mark.gpu

GAMMA = 1.4
EL = (1.0, 2.0, 1.0)
GUESSES = [A.ADERDG_GUESS_ORDER2, A.ADERDG_GUESS_ORDER3, A.ADERDG_GUESS_EXTRAP, A.ADERDG_GUESS_CERK]

# (pde, dim, N, cells, L, params)
CASES = (
    [(1, 2, N, (5, 3), 1.0, (0.7, -1.1)) for N in (1, 3, 6)]
    + [(2, 2, N, (5, 3), 2.0, (GAMMA,)) for N in (1, 2, 3, 4, 5, 7)]
    + [(2, 3, N, (3, 2, 2), 2.0, (GAMMA,)) for N in (2, 4)]
    + [(3, 3, N, (3, 2, 2), 1.0, EL) for N in (1, 3)]
)


def _ids(c):
    return "pde%d-%dd-N%d" % (c[0], c[1], c[2])


def _pair(pde, dim, N, cells, L, params, guess, precision=A.ADERDG_FP64, picard=0):
    cfg = oracle.make_cfg(dim, cells, [0.0] * dim, [L] * dim, N, pde, params, picard=picard, guess=guess)
    s = A.Solver(pde, dim, cells, [0.0] * dim, [L] * dim, N, params, precision=precision, picard=picard,
                 guess=guess)
    return cfg, s


def _state(cfg, pde, seed):
    X = oracle.node_coords(cfg)
    L = [cfg.hi[d] - cfg.lo[d] for d in range(cfg.dim)]
    U = inputs.smooth_random_state(pde, X, L, seed=seed, amp=0.2)
    if pde == 2:
        return 0.5 * (U + inputs.random_state(pde, cfg.dim, *U.shape[:2], seed=seed + 1, amp=0.05))
    return U + 0.1 * inputs.random_state(pde, cfg.dim, *U.shape[:2], seed=seed + 1)


def _scale(a):
    return max(1.0, float(np.abs(a).max()))


@pytest.mark.parametrize("guess", GUESSES)
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_predictor_outputs_match_oracle(case, guess):
    pde = case[0]
    cfg, s = _pair(*case, guess=guess)
    assert s.info()["picard_iters"] == oracle.lib().orc_picard_count(cfg)
    assert s.info()["initial_guess"] == guess
    U = _state(cfg, pde, seed=500 + case[2])
    dt = oracle.cfl_dt(cfg, U)
    _, Vo, qfo, ffo = oracle.step(cfg, U, dt, with_parts=True)
    s.set_state(U)
    s.predictor(dt)
    V, qf, ff = s.predictor_outputs()
    assert np.abs(V - Vo).max() <= 1e-12 * _scale(Vo)
    assert np.abs(qf - qfo).max() <= 1e-12 * _scale(qfo)
    assert np.abs(ff - ffo).max() <= 1e-12 * _scale(ffo)


@pytest.mark.parametrize("picard", [0, 2])
def test_full_run_euler_vortex_third_order_guess(picard):
    """FP64 full run, default count (N-1) and the paper's minimum (N-2)."""
    case = (2, 2, 4, (24, 20), 10.0, (GAMMA,))
    cfg, s = _pair(*case, guess=A.ADERDG_GUESS_ORDER3, picard=picard)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.4)
    s.set_state(U0)
    s.advance(0.4)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


def test_full_run_elasticity_third_order_guess():
    case = (3, 3, 3, (5, 4, 4), 1.0, EL)
    cfg, s = _pair(*case, guess=A.ADERDG_GUESS_ORDER3, picard=1)
    U0 = inputs.elastic_pulse(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.05)
    s.set_state(U0)
    s.advance(0.05)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


def test_mixed_full_run_third_order_guess():
    case = (2, 2, 4, (24, 20), 10.0, (GAMMA,))
    cfg, s = _pair(*case, guess=A.ADERDG_GUESS_ORDER3, picard=2, precision=A.ADERDG_MIXED_FP32)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.4)
    s.set_state(U0)
    s.advance(0.4)
    Ug, t, k = s.get_state()
    assert t == to and abs(k - ko) <= 1
    assert l2_rel(cfg, Ug, Uo) <= 1e-6


def test_third_order_guess_same_error_as_trivial_guess():
    """At the vortex's resolution the third-order guess with N-2 iterations
    has the L2 error of the trivial guess with N+1 against the exact
    solution (both FP64, GPU)."""
    N, cells = 4, (40, 40)
    errs = []
    for guess, picard in ((A.ADERDG_GUESS_TRIVIAL, 0), (A.ADERDG_GUESS_ORDER3, N - 2)):
        cfg, s = _pair(2, 2, N, cells, 10.0, (GAMMA,), guess=guess, picard=picard)
        X = oracle.node_coords(cfg)
        s.set_state(inputs.euler_vortex(X))
        s.advance(0.5)
        Ug, t, _ = s.get_state()
        errs.append(l2_abs(cfg, Ug, inputs.euler_vortex(X, t=t)))
    np.testing.assert_allclose(errs[1], errs[0], rtol=1e-6)


@pytest.mark.parametrize("picard", [0, 1])
def test_full_run_euler_vortex_extrapolation_guess(picard):
    """FP64 full run with the extrapolation of the previous predictor (the
    first step takes the third-order guess): default count (2) and one
    Picard iteration, against the oracle's run."""
    case = (2, 2, 4, (24, 20), 10.0, (GAMMA,))
    cfg, s = _pair(*case, guess=A.ADERDG_GUESS_EXTRAP, picard=picard)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.4)
    s.set_state(U0)
    s.advance(0.4)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko) and k > 2
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


def test_extrapolation_guess_elasticity_and_mixed():
    case = (3, 3, 3, (5, 4, 4), 1.0, EL)
    cfg, s = _pair(*case, guess=A.ADERDG_GUESS_EXTRAP, picard=1)
    U0 = inputs.elastic_pulse(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.05)
    s.set_state(U0)
    s.advance(0.05)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-11
    for case in [(2, 2, 4, (24, 20), 10.0, (GAMMA,)), (2, 2, 2, (24, 20), 10.0, (GAMMA,))]:
        cfg, s = _pair(*case, guess=A.ADERDG_GUESS_EXTRAP, picard=1, precision=A.ADERDG_MIXED_FP32)
        U0 = inputs.euler_vortex(oracle.node_coords(cfg))
        Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.4)
        s.set_state(U0)
        s.advance(0.4)
        Ug, t, k = s.get_state()
        assert t == to and abs(k - ko) <= 1
        assert l2_rel(cfg, Ug, Uo) <= 1e-6


def test_extrapolation_restarts_after_set_state():
    """A state upload drops the previous predictor: the next step takes the
    third-order guess again (same result as a fresh handle)."""
    case = (2, 2, 3, (8, 8), 2.0, (GAMMA,))
    cfg, s = _pair(*case, guess=A.ADERDG_GUESS_EXTRAP)
    U0 = _state(cfg, 2, seed=77)
    s.set_state(U0)
    s.advance(1e30, max_steps=3)
    s.set_state(U0)
    s.advance(1e30, max_steps=2)
    a = s.get_state()[0]
    _, s2 = _pair(*case, guess=A.ADERDG_GUESS_EXTRAP)
    s2.set_state(U0)
    s2.advance(1e30, max_steps=2)
    np.testing.assert_array_equal(a, s2.get_state()[0])


@pytest.mark.parametrize("picard", [0, 1])
def test_full_run_euler_vortex_cerk_guess(picard):
    """FP64 and mixed full runs with the CERK guess (the classical
    method's cubic dense output at N = 4): default count (N-2) and one
    Picard iteration (a degree N-1 guess for N = 4)."""
    case = (2, 2, 4, (24, 20), 10.0, (GAMMA,))
    for prec, tol in ((A.ADERDG_FP64, 1e-11), (A.ADERDG_MIXED_FP32, 1e-6)):
        cfg, s = _pair(*case, guess=A.ADERDG_GUESS_CERK, picard=picard, precision=prec)
        U0 = inputs.euler_vortex(oracle.node_coords(cfg))
        Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.4)
        s.set_state(U0)
        s.advance(0.4)
        Ug, t, k = s.get_state()
        assert (t, k) == (to, ko) and k > 2
        assert l2_rel(cfg, Ug, Uo) <= tol


CERK_ORDER = {5: 4, 6: 5, 7: 5}


@pytest.mark.parametrize("N", [5, 6, 7])
def test_full_run_euler_vortex_high_order_cerk_guess(N):
    """The six-stage scheme with quartic weights (N = 5) and the
    eleven-stage scheme with quintic weights (N >= 6): a degree N-1 guess at
    N = 5 and 6, so one Picard iteration; FP64 and mixed full runs against
    the oracle, and the default count N + 1 - p."""
    case = (2, 2, N, (14, 12), 10.0, (GAMMA,))
    for picard in (0, 1):
        for prec, tol in ((A.ADERDG_FP64, 1e-11), (A.ADERDG_MIXED_FP32, 1e-6)):
            cfg, s = _pair(*case, guess=A.ADERDG_GUESS_CERK, picard=picard, precision=prec)
            assert s.info()["picard_iters"] == (picard or N + 1 - CERK_ORDER[N])
            U0 = inputs.euler_vortex(oracle.node_coords(cfg))
            Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.3)
            s.set_state(U0)
            s.advance(0.3)
            Ug, t, k = s.get_state()
            s.close()
            assert (t, k) == (to, ko) and k > 2
            assert l2_rel(cfg, Ug, Uo) <= tol


@pytest.mark.parametrize("N", [5, 6])
@pytest.mark.parametrize("shapes", [(0, 0), (1, 1), (2, 2), (7, 3), (8, 0)])
def test_high_order_cerk_guess_every_predictor_shape(shapes, N):
    """Each predictor shape of the FP32 path holds the earlier stages in its
    exchange field's free time slices (its own layout per shape; five of
    them for the six-stage scheme, ten for the eleven-stage one): within the
    mixed tolerance of the oracle."""
    cfg = oracle.make_cfg(2, (9, 7), [0, 0], [10, 10], N, 2, (GAMMA,), picard=1, guess=oracle.GUESS_CERK)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.2)
    with A.Solver(2, 2, (9, 7), (0, 0), (10, 10), N, (GAMMA,), precision=A.ADERDG_MIXED_FP32, picard=1,
                  guess=A.ADERDG_GUESS_CERK, shapes=shapes) as s:
        s.set_state(U0)
        s.advance(0.2)
        Ug, t, k = s.get_state()
        assert s.info()["pred_shape"] == shapes[0]
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-6


@pytest.mark.parametrize("N,shapes", [(5, (3, 0)), (6, (4, 1)), (5, (0, 0)), (7, (3, 0)), (6, (0, 0))])
def test_high_order_cerk_guess_advection_plane_kernel(N, shapes):
    """2D advection with the order-4 (N = 5) and order-5 (N >= 6) schemes on
    the plane-owning FP32 kernel (the stages' k in registers) and on
    k_predictor: one Picard iteration, against the oracle."""
    a = (0.7, -1.1)
    cfg = oracle.make_cfg(2, (6, 5), [0, 0], [1, 1], N, 1, a, picard=1, guess=oracle.GUESS_CERK)
    X = oracle.node_coords(cfg)
    U0 = inputs.smooth_random_state(1, X, [1.0, 1.0], seed=9)
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.05)
    with A.Solver(1, 2, (6, 5), (0, 0), (1, 1), N, a, precision=A.ADERDG_MIXED_FP32, picard=1,
                  guess=A.ADERDG_GUESS_CERK, shapes=shapes) as s:
        s.set_state(U0)
        s.advance(0.05)
        Ug, t, k = s.get_state()
        assert s.info()["pred_shape"] == shapes[0]
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-6


@pytest.mark.parametrize("shapes", [(3, 0), (4, 1)])
def test_cerk_guess_plane_kernel(shapes):
    """The plane-owning 2D FP32 predictor with the CERK guess."""
    case = (2, 2, 2, (12, 10), 10.0, (GAMMA,))
    cfg = oracle.make_cfg(2, case[3], [0, 0], [10, 10], 2, 2, case[5], picard=1, guess=oracle.GUESS_CERK)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.3)
    with A.Solver(2, 2, case[3], (0, 0), (10, 10), 2, case[5], precision=A.ADERDG_MIXED_FP32, picard=1,
                  guess=A.ADERDG_GUESS_CERK, shapes=shapes) as s:
        s.set_state(U0)
        s.advance(0.3)
        Ug, t, k = s.get_state()
        assert s.info()["pred_shape"] == shapes[0]
    assert t == to and abs(k - ko) <= 1
    assert l2_rel(cfg, Ug, Uo) <= 1e-6


@pytest.mark.parametrize("guess", [A.ADERDG_GUESS_ORDER3, A.ADERDG_GUESS_EXTRAP, A.ADERDG_GUESS_CERK])
def test_batch_with_guess_equals_alone(guess):
    mix = [(2, 2, (6, 5), (0, 0), (10, 10), 2, (GAMMA,)), (2, 2, (8, 8), (0, 0), (10, 10), 4, (GAMMA,)),
           (3, 3, (3, 3, 2), (0, 0, 0), (1, 1, 1), 3, EL),
           (2, 2, (5, 4), (0, 0), (10, 10), 5, (GAMMA,)),  # N = 5: the six-stage CERK scheme
           (2, 2, (4, 5), (0, 0), (10, 10), 6, (GAMMA,))]  # N = 6: the eleven-stage one
    t_end = [0.3, 0.2, 0.02, 0.15, 0.1]
    ics = []
    for c in mix:
        X = oracle.node_coords(oracle.make_cfg(c[1], c[2], c[3], c[4], c[5], c[0], c[6]))
        ics.append(inputs.euler_vortex(X) if c[0] == 2 else inputs.elastic_pulse(X, width=0.05))
    for prec in (A.ADERDG_FP64, A.ADERDG_MIXED_FP32):
        b = A.Batch([A.make_spec(*c) for c in mix], precision=prec, guess=guess)
        for i, u in enumerate(ics):
            b.set_state(i, u)
        b.advance(t_end)
        for i, c in enumerate(mix):
            with A.Solver(*c, precision=prec, guess=guess) as s:
                s.set_state(ics[i])
                s.advance(t_end[i])
                alone = s.get_state()[0]
            np.testing.assert_array_equal(b.get_state(i)[0], alone.reshape(-1))
        b.close()


def test_server_with_guess_equals_solves_alone():
    """A server configured with the third-order guess serves results bitwise
    equal to the same solves alone with that guess (mixed path)."""
    import time
    mix = [(2, 2, (6, 5), (0, 0), (10, 10), 2, (GAMMA,), 0.3), (2, 2, (8, 8), (0, 0), (10, 10), 4, (GAMMA,), 0.2),
           (3, 3, (3, 3, 2), (0, 0, 0), (1, 1, 1), 3, EL, 0.02)]
    srv = A.Server(precision=A.ADERDG_MIXED_FP32, steps_per_round=4, guess=A.ADERDG_GUESS_ORDER3)
    ics, tickets = [], []
    for c in mix:
        X = oracle.node_coords(oracle.make_cfg(c[1], c[2], c[3], c[4], c[5], c[0], c[6]))
        u0 = inputs.euler_vortex(X) if c[0] == 2 else inputs.elastic_pulse(X, width=0.05)
        ics.append(u0)
        tickets.append(srv.submit(A.make_spec(*c[:7]), u0, c[7]))
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
    for tk, c, u0 in zip(tickets, mix, ics):
        assert res[tk]["status"] == A.ADERDG_OK
        with A.Solver(*c[:7], precision=A.ADERDG_MIXED_FP32, guess=A.ADERDG_GUESS_ORDER3) as s:
            s.set_state(u0)
            s.advance(c[7])
            alone, t, k = s.get_state()
        assert res[tk]["steps"] == k and res[tk]["t"] == t
        np.testing.assert_array_equal(res[tk]["u"], alone.reshape(-1))
        srv.release(tk)
    srv.close()
