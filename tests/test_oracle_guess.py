"""Pins of the oracle's initial guesses of the Picard iteration (Sec. 2.2:
the second-order guess u + tau L(u), the third-order guess
u + tau k1 + tau^2 (k2 - k1) / (2 dt), k1 = L(u), k2 = L(u + dt k1), and
the extrapolation of the previous step's predictor).

For linear advection u_t + a.grad u = 0 the exact solution is
u0(x - a t), and L(u) = -a.grad u is exact on polynomial data, so each
guess reproduces the exact space-time solution when it is a polynomial in
t of the guess's degree, and misses it by exactly the next Taylor term
otherwise.  A guess only moves the starting point: iterated to
convergence, every guess reaches the same space-time solution."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import inputs
from helpers import euler_cfg, l2_abs, order


def _poly(dim, degree, seed):
    """Random polynomial of total degree <= degree: {exponents: coefficient}."""
    rng = np.random.default_rng(seed)
    return {k: rng.uniform(-1, 1) for k in itertools.product(range(degree + 1), repeat=dim) if sum(k) <= degree}


def _eval(coef, X):
    out = np.zeros(X.shape[0])
    for k, c in coef.items():
        term = np.full(X.shape[0], c)
        for d, p in enumerate(k):
            term = term * X[:, d] ** p
        out += term
    return out


def _space_time(cfg, coef, a, dt):
    """Exact q(x_s, t^n + tau_t) = u0(x_s - a tau_t) at the element-0 nodes."""
    n = cfg.N + 1
    X = oracle.node_coords(cfg)[0]
    tau, _ = oracle.gauss_legendre(n)
    return np.stack([_eval(coef, X - np.asarray(a)[None, :] * (t * dt)) for t in tau])[:, :, None], X, tau


@pytest.mark.parametrize("dim,N", [(1, 3), (2, 2), (2, 4)])
def test_second_order_guess_is_exact_for_linear_data(dim, N):
    a = [1.7, -0.6][:dim]
    cfg = oracle.make_cfg(dim, [4] * dim, [0.0] * dim, [1.0] * dim, N, oracle.PDE_ADVECTION, a,
                          guess=oracle.GUESS_ORDER2)
    coef = _poly(dim, 1, seed=dim + N)
    dt = 0.03
    ex, X, _ = _space_time(cfg, coef, a, dt)
    q0 = oracle.initial_guess(cfg, _eval(coef, X)[:, None], dt)
    np.testing.assert_allclose(q0, ex, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim,N", [(1, 3), (2, 2), (2, 4), (3, 2)])
def test_third_order_guess_is_exact_for_quadratic_data(dim, N):
    a = [1.7, -0.6, 0.9][:dim]
    cfg = oracle.make_cfg(dim, [4] * dim, [0.0] * dim, [1.0] * dim, N, oracle.PDE_ADVECTION, a,
                          guess=oracle.GUESS_ORDER3)
    coef = _poly(dim, 2, seed=10 * dim + N)
    dt = 0.05
    ex, X, _ = _space_time(cfg, coef, a, dt)
    q0 = oracle.initial_guess(cfg, _eval(coef, X)[:, None], dt)
    np.testing.assert_allclose(q0, ex, rtol=0, atol=1e-12)
    # and the second-order guess is not (the data is quadratic)
    cfg.guess = oracle.GUESS_ORDER2
    assert np.abs(oracle.initial_guess(cfg, _eval(coef, X)[:, None], dt) - ex).max() > 1e-5


def test_third_order_guess_misses_exactly_the_cubic_term():
    """u0 = x^3: the exact solution (x - a tau)^3 minus the guess is
    -a^3 tau^3; every lower Taylor term (coefficients 1, -3a x^2, 3 a^2 x)
    is reproduced."""
    a, N, dt = 1.3, 3, 0.07
    cfg = oracle.make_cfg(1, [3], [0.0], [1.0], N, oracle.PDE_ADVECTION, [a], guess=oracle.GUESS_ORDER3)
    coef = {(3,): 1.0}
    ex, X, tau = _space_time(cfg, coef, [a], dt)
    q0 = oracle.initial_guess(cfg, _eval(coef, X)[:, None], dt)
    want = (a * tau * dt) ** 3
    np.testing.assert_allclose((q0 - ex)[:, :, 0], np.broadcast_to(want[:, None], (N + 1, N + 1)),
                               rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("guess", [oracle.GUESS_TRIVIAL, oracle.GUESS_ORDER2, oracle.GUESS_ORDER3])
def test_constant_state_guess_is_the_state(guess):
    cfg = euler_cfg((3, 3), N=3)
    cfg.guess = guess
    q = inputs.random_state(oracle.PDE_EULER, 2, 1, 1, seed=4)[0, 0]
    u = np.tile(q, (16, 1))
    np.testing.assert_allclose(oracle.initial_guess(cfg, u, 0.02), np.broadcast_to(u, (4, 16, 4)), atol=1e-13)


@pytest.mark.parametrize("guess", [oracle.GUESS_ORDER2, oracle.GUESS_ORDER3])
def test_guess_only_moves_the_starting_point(guess):
    """Iterated to convergence (nonlinear Euler), every guess reaches the
    same space-time solution as the trivial guess."""
    cfg = euler_cfg((5, 5), N=3, L=2.0, picard=-1)
    X = oracle.node_coords(cfg)
    U = inputs.smooth_random_state(oracle.PDE_EULER, X, [2.0, 2.0], seed=5)
    dt = 0.5 * oracle.cfl_dt(cfg, U)
    ref = oracle.predictor(cfg, U[7], dt)
    cfg.guess = guess
    got = oracle.predictor(cfg, U[7], dt)
    np.testing.assert_allclose(got[0], ref[0], rtol=0, atol=1e-12)
    # and it gets there in fewer iterations
    assert got[3] < ref[3], (got[3], ref[3])


def test_default_picard_counts():
    for N in range(1, 8):
        for guess, want in ((0, N + 1), (1, N), (2, max(1, N - 1))):
            cfg = euler_cfg((2, 2), N=N)
            cfg.guess = guess
            assert oracle.lib().orc_picard_count(cfg) == want


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_third_order_guess_converged_for_linear_advection(N):
    """For 1D linear advection the third-order guess followed by
    max(1, N-2) Picard iterations is the converged predictor (the trivial
    guess needs N), so whole steps agree to round-off."""
    K = 5
    rng = np.random.default_rng(N)
    U = rng.standard_normal((K, N + 1, 1))
    mk = lambda g, P: oracle.make_cfg(1, [K], [0.0], [1.0], N, oracle.PDE_ADVECTION, [1.0], picard=P, guess=g)
    ref = oracle.step(mk(0, N + 1), U, 0.02)
    got = oracle.step(mk(2, max(1, N - 2)), U, 0.02)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N", [3, 4])
def test_third_order_guess_design_order(N):
    """Euler density wave with the third-order guess and the paper's minimum
    of N-2 Picard iterations keeps the design order N+1."""
    errs = []
    for c in (8, 16):
        cfg = euler_cfg((c, c), N=N, L=1.0, picard=max(1, N - 2))
        cfg.guess = oracle.GUESS_ORDER3
        X = oracle.node_coords(cfg)
        U1, t, _, _ = oracle.run(cfg, inputs.euler_density_wave(X, L=1.0), t_end=0.2)
        errs.append(l2_abs(cfg, U1, inputs.euler_density_wave(X, L=1.0, t=t))[0])
    assert order(*errs) > N + 1 - 0.5, errs


# ---- extrapolation of the previous step's predictor (Sec. 2.2) ----------------

def _prev_interval(cfg, coef, a, dt_prev):
    """Exact q at the time nodes of the previous interval [-dt_prev, 0]."""
    n = cfg.N + 1
    X = oracle.node_coords(cfg)[0]
    tau, _ = oracle.gauss_legendre(n)
    return np.stack([_eval(coef, X - np.asarray(a)[None, :] * ((-1.0 + t) * dt_prev)) for t in tau])[:, :, None]


@pytest.mark.parametrize("dim,N,ratio", [(1, 3, 1.0), (1, 4, 0.7), (2, 3, 1.3)])
def test_extrapolation_guess_is_exact_for_polynomials_in_time(dim, N, ratio):
    """Linear advection of a polynomial of degree <= N: the solution is a
    polynomial of degree <= N in time, so extrapolating its interpolant on
    the previous interval reproduces it on the next one."""
    a = [1.7, -0.6][:dim]
    cfg = oracle.make_cfg(dim, [4] * dim, [0.0] * dim, [1.0] * dim, N, oracle.PDE_ADVECTION, a,
                          guess=oracle.GUESS_EXTRAP)
    coef = _poly(dim, N, seed=30 + N)
    dt = 0.04
    ex, X, _ = _space_time(cfg, coef, a, dt)
    qprev = _prev_interval(cfg, coef, a, dt / ratio)
    q0 = oracle.initial_guess_extrap(cfg, _eval(coef, X)[:, None], dt, qprev, ratio)
    np.testing.assert_allclose(q0, ex, rtol=0, atol=1e-11)


def test_extrapolation_guess_misses_the_nodal_polynomial():
    """u0 = x^{N+1}: in time the solution (x - a t)^{N+1} has leading
    coefficient c = (-a)^{N+1}; interpolation on the previous interval's
    nodes tau_k misses c w(tau), w(tau) = prod_k (tau - tau_k), and the
    shift to u at tau = 0 removes w(0): q0 - exact = -c (w(tau) - w(0))."""
    N, a, dt, ratio = 3, 1.3, 0.05, 0.8
    cfg = oracle.make_cfg(1, [3], [0.0], [1.0], N, oracle.PDE_ADVECTION, [a], guess=oracle.GUESS_EXTRAP)
    coef = {(N + 1,): 1.0}
    ex, X, tau = _space_time(cfg, coef, [a], dt)
    dtp = dt / ratio
    qprev = _prev_interval(cfg, coef, [a], dtp)
    q0 = oracle.initial_guess_extrap(cfg, _eval(coef, X)[:, None], dt, qprev, ratio)
    nodes = -dtp + tau * dtp
    w = lambda s: np.prod(s - nodes)
    c = (-a) ** (N + 1)
    want = np.array([-c * (w(t * dt) - w(0.0)) for t in tau])
    np.testing.assert_allclose((q0 - ex)[:, :, 0], np.broadcast_to(want[:, None], (N + 1, N + 1)),
                               rtol=1e-9, atol=1e-14)


def test_extrapolation_first_step_is_the_third_order_guess():
    """A single step has no previous predictor: guess 3 falls back to the
    third-order guess with its default count (bitwise)."""
    cfg = euler_cfg((5, 4), N=4, L=2.0)
    X = oracle.node_coords(cfg)
    U = inputs.smooth_random_state(oracle.PDE_EULER, X, [2.0, 2.0], seed=8)
    dt = oracle.cfl_dt(cfg, U)
    cfg.guess = oracle.GUESS_EXTRAP
    a = oracle.step(cfg, U, dt)
    cfg.guess = oracle.GUESS_ORDER3
    b = oracle.step(cfg, U, dt)
    np.testing.assert_array_equal(a, b)
    cfg.guess = oracle.GUESS_EXTRAP
    assert oracle.lib().orc_picard_count(cfg) == 2


@pytest.mark.parametrize("N", [3, 4])
def test_extrapolation_guess_design_order(N):
    """Euler density wave, extrapolation guess and one Picard iteration per
    step: design order N+1."""
    errs = []
    for c in (8, 16):
        cfg = euler_cfg((c, c), N=N, L=1.0, picard=1)
        cfg.guess = oracle.GUESS_EXTRAP
        X = oracle.node_coords(cfg)
        U1, t, _, _ = oracle.run(cfg, inputs.euler_density_wave(X, L=1.0), t_end=0.2)
        errs.append(l2_abs(cfg, U1, inputs.euler_density_wave(X, L=1.0, t=t))[0])
    assert order(*errs) > N + 1 - 0.5, errs


def test_extrapolation_guess_vortex_error_matches_trivial():
    """Isentropic vortex, N = 4: one Picard iteration after the extrapolation
    guess gives the trivial guess's L2 error within 0.1 %."""
    errs = []
    for guess, picard in ((oracle.GUESS_TRIVIAL, 0), (oracle.GUESS_EXTRAP, 1)):
        cfg = euler_cfg((20, 20), N=4, L=10.0, picard=picard)
        cfg.guess = guess
        X = oracle.node_coords(cfg)
        U1, t, _, _ = oracle.run(cfg, inputs.euler_vortex(X), t_end=0.5)
        errs.append(l2_abs(cfg, U1, inputs.euler_vortex(X, t=t))[0])
    assert abs(errs[1] - errs[0]) <= 1e-3 * errs[0], errs


# ---- continuous Runge-Kutta (CERK) guess (Sec. 2.2) -------------------------
#
# The guess for degree N uses a continuous explicit Runge-Kutta scheme of
# order p = max(3, N - 1), capped at the highest order built: the classical
# fourth-order method with its cubic dense output (p = 3) up to N = 4, a
# six-stage scheme with quartic weights (p = 4) at N = 5, an eleven-stage
# scheme with quintic weights (p = 5) from N = 6.

RK_C = np.array([0.0, 0.5, 0.5, 1.0])
RK_A = np.array([[0, 0, 0, 0], [0.5, 0, 0, 0], [0, 0.5, 0, 0], [0, 0, 1.0, 0]])
CERK_ORDER = {1: 3, 2: 3, 3: 3, 4: 3, 5: 4, 6: 5, 7: 5}


def _trees(A, p):
    """(order, gamma, elementary weight vector) of every rooted tree of order
    <= p for the stage matrix A (Butcher's trees; c = A 1)."""
    one = np.ones(A.shape[0])
    c = A @ one
    Ac = A @ c
    T = [(1, 1, one), (2, 2, c), (3, 3, c ** 2), (3, 6, Ac),
         (4, 4, c ** 3), (4, 8, c * Ac), (4, 12, A @ c ** 2), (4, 24, A @ Ac)]
    if p >= 5:
        T += [(5, 5, c ** 4), (5, 10, c ** 2 * Ac), (5, 15, c * (A @ c ** 2)), (5, 30, c * (A @ Ac)),
              (5, 20, Ac * Ac), (5, 20, A @ c ** 3), (5, 40, A @ (c * Ac)), (5, 60, A @ (A @ c ** 2)),
              (5, 120, A @ (A @ Ac))]
    return [t for t in T if t[0] <= p]


def test_cerk_schemes_have_the_orders_the_guess_needs():
    for N, p in CERK_ORDER.items():
        A, beta = oracle.cerk_scheme(N)
        assert beta.shape[1] == p and A.shape == (beta.shape[0],) * 2
        assert np.all(np.triu(A) == 0)  # explicit
    np.testing.assert_array_equal(oracle.cerk_scheme(4)[0], RK_A)  # the classical method


@pytest.mark.parametrize("N", [4, 5, 6])
@pytest.mark.parametrize("theta", [0.0, 0.1, 0.3, 0.5, 0.77, 1.0])
def test_cerk_weights_satisfy_the_continuous_order_conditions(theta, N):
    """The dense-output weights b_i(theta) meet every order condition of a
    continuous Runge-Kutta scheme up to its order p at each theta,
    sum_i b_i(theta) Phi_i(t) = theta^|t| / gamma(t); the weights of the
    classical method end in 1/6, 1/3, 1/3, 1/6."""
    A, beta = oracle.cerk_scheme(N)
    p = CERK_ORDER[N]
    b = oracle.cerk_weights(theta, N)
    # rounding of the weight polynomials: a few ulps of sum_k |beta_ik theta^(k+1)|
    # (up to 19 in the eleven-stage scheme's coefficients)
    mag = np.abs(beta) @ theta ** np.arange(1, p + 1)
    np.testing.assert_allclose(b, beta @ theta ** np.arange(1, p + 1), rtol=0, atol=1e-15 + 4e-16 * mag.max())
    for order_, gamma, phi in _trees(A, p):
        assert abs(b @ phi - theta ** order_ / gamma) < 2e-15 + 4e-16 * (mag @ np.abs(phi)), (order_, gamma)
    if N <= 4:
        for order_, gamma, phi in _trees(RK_A, 3):
            assert abs(b @ phi - theta ** order_ / gamma) < 1e-15
        if theta == 1.0:
            np.testing.assert_allclose(b, [1 / 6, 1 / 3, 1 / 3, 1 / 6], rtol=0, atol=1e-15)


def test_cerk_order4_scheme_misses_an_order5_condition():
    """The order-4 scheme is not of order 5 (so the quintic test below
    measures a real miss)."""
    A, _ = oracle.cerk_scheme(5)
    b = oracle.cerk_weights(1.0, 5)
    misses = [abs(b @ phi - 1 / g) for o, g, phi in _trees(A, 5) if o == 5]
    assert max(misses) > 1e-4


def test_cerk_order5_scheme_is_explicit_bounded_and_consistent():
    """The eleven-stage scheme: nodes c = A 1 inside [0, 1], weights summing
    to theta (the first-order condition) with the b_i(theta) small on a fine
    grid (the scheme does not cancel large terms), and b(1) . A^5 1 away
    from 1/6!, so it is not of order 6 on the tall tree."""
    A, beta = oracle.cerk_scheme(6)
    assert A.shape == (11, 11) and beta.shape == (11, 5)
    c = A.sum(axis=1)
    assert c.min() >= 0.0 and c.max() <= 1.0
    th = np.linspace(0, 1, 201)
    B = np.array([oracle.cerk_weights(t, 6) for t in th])
    np.testing.assert_allclose(B.sum(axis=1), th, rtol=0, atol=2e-14)  # coefficients up to 19: a few ulps
    assert np.abs(B).max() < 0.35
    chain = np.linalg.matrix_power(A, 5) @ np.ones(11)
    assert abs(oracle.cerk_weights(1.0, 6) @ chain - 1 / 720) > 1e-5


@pytest.mark.parametrize("dim,N", [(1, 3), (2, 3), (2, 4), (3, 3), (1, 5), (2, 5), (2, 6)])
def test_cerk_guess_is_exact_for_data_of_its_order(dim, N):
    """Linear advection of a polynomial of total degree <= p: L^(p+1) u = 0
    and the CERK guess reproduces the exact space-time solution."""
    p = CERK_ORDER[N]
    a = [1.7, -0.6, 0.9][:dim]
    cfg = oracle.make_cfg(dim, [4] * dim, [0.0] * dim, [1.0] * dim, N, oracle.PDE_ADVECTION, a,
                          guess=oracle.GUESS_CERK)
    coef = _poly(dim, p, seed=50 + 10 * dim + N)
    dt = 0.05
    ex, X, _ = _space_time(cfg, coef, a, dt)
    q0 = oracle.initial_guess(cfg, _eval(coef, X)[:, None], dt)
    np.testing.assert_allclose(q0, ex, rtol=0, atol=1e-11)
    cfg.guess = oracle.GUESS_ORDER3  # the third-order guess is not exact here
    assert np.abs(oracle.initial_guess(cfg, _eval(coef, X)[:, None], dt) - ex).max() > 1e-6


@pytest.mark.parametrize("N", [4, 5, 6])
def test_cerk_guess_misses_exactly_the_next_taylor_term(N):
    """u0 = x^(p+1), L = -a d/dx: the stages give k = sum_j dt^j A^j 1
    L^(j+1) u, so the dense output carries dt^(p+1) (b(theta) . A^p 1)
    L^(p+1) u where the exact solution has (theta dt)^(p+1) L^(p+1) u /
    (p+1)!; with L^(p+1) u = (-a)^(p+1) (p+1)! the miss is
    (-a)^(p+1) dt^(p+1) ((p+1)! b(theta) . A^p 1 - theta^(p+1))."""
    p = CERK_ORDER[N]
    a, dt = 1.3, 0.07
    A, _ = oracle.cerk_scheme(N)
    chain = np.linalg.matrix_power(A, p) @ np.ones(A.shape[0])
    cfg = oracle.make_cfg(1, [3], [0.0], [1.0], N, oracle.PDE_ADVECTION, [a], guess=oracle.GUESS_CERK)
    coef = {(p + 1,): 1.0}
    ex, X, tau = _space_time(cfg, coef, [a], dt)
    q0 = oracle.initial_guess(cfg, _eval(coef, X)[:, None], dt)
    fact = float(np.prod(np.arange(1, p + 2)))
    want = np.array([(-a) ** (p + 1) * dt ** (p + 1) * (fact * (oracle.cerk_weights(t, N) @ chain) - t ** (p + 1))
                     for t in tau])
    if N == 4:  # the classical method: A^3 1 = (0, 0, 0, 1/4), the miss a^4 dt^4 (6 b_4 - theta^4)
        np.testing.assert_allclose(want, [a ** 4 * dt ** 4 * (6 * oracle.cerk_weights(t, 4)[3] - t ** 4)
                                          for t in tau], rtol=1e-12)
    assert np.abs(want).max() > 1e-9
    np.testing.assert_allclose((q0 - ex)[:, :, 0], np.broadcast_to(want[:, None], (N + 1, N + 1)),
                               rtol=1e-8, atol=1e-15)


def test_cerk_guess_constant_state_and_picard_count():
    cfg = euler_cfg((3, 3), N=3)
    cfg.guess = oracle.GUESS_CERK
    q = inputs.random_state(oracle.PDE_EULER, 2, 1, 1, seed=4)[0, 0]
    u = np.tile(q, (16, 1))
    np.testing.assert_allclose(oracle.initial_guess(cfg, u, 0.02), np.broadcast_to(u, (4, 16, 4)), atol=1e-13)
    for N in range(1, 8):
        cfg = euler_cfg((2, 2), N=N)
        cfg.guess = oracle.GUESS_CERK
        assert oracle.lib().orc_picard_count(cfg) == max(1, N + 1 - CERK_ORDER[N])


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_cerk_guess_converged_for_linear_advection(N):
    """1D linear advection: the guess is exact to order p in time, and each
    Picard iteration adds one order, so max(1, N - p) iterations reach the
    converged predictor (the space-time solution of degree N)."""
    K = 5
    p = CERK_ORDER[N]
    rng = np.random.default_rng(40 + N)
    U = rng.standard_normal((K, N + 1, 1))
    mk = lambda g, P: oracle.make_cfg(1, [K], [0.0], [1.0], N, oracle.PDE_ADVECTION, [1.0], picard=P, guess=g)
    ref = oracle.step(mk(0, N + 1), U, 0.02)
    got = oracle.step(mk(oracle.GUESS_CERK, max(1, N - p)), U, 0.02)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    if N - p >= 1:  # one iteration fewer does not converge
        short = oracle.step(mk(oracle.GUESS_CERK, N - p - 1), U, 0.02) if N - p >= 2 else None
        if short is not None:
            assert np.abs(short - ref).max() > 1e-12


@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_cerk_guess_design_order_with_one_iteration(N):
    """A guess of degree N-1 (or more) in time needs one Picard iteration
    (Sec. 2.2): Euler density wave, CERK guess, one iteration per step,
    design order N+1."""
    errs = []
    for c in (8, 16):
        cfg = euler_cfg((c, c), N=N, L=1.0, picard=1)
        cfg.guess = oracle.GUESS_CERK
        X = oracle.node_coords(cfg)
        U1, t, _, _ = oracle.run(cfg, inputs.euler_density_wave(X, L=1.0), t_end=0.2)
        errs.append(l2_abs(cfg, U1, inputs.euler_density_wave(X, L=1.0, t=t))[0])
    assert order(*errs) > N + 1 - 0.5, errs
