"""Pins of the oracle's space-time predictor (Sec. 2.2, eq. pde.st2, Picard
iteration) against exact solutions, a brute-force linear solve assembled
from numpy's own basis, and the termination property of the Picard
iteration for linear systems."""
import numpy as np
import numpy.polynomial.polynomial as P
import pytest

import oracle
from paper_1808_03788_gb300 import inputs
from helpers import advection_cfg, elastic_cfg, euler_cfg


def _element_nodes(cfg, n):
    """Node coordinates of element 0 and the time nodes."""
    X = oracle.node_coords(cfg)[0]
    tau, _ = oracle.gauss_legendre(n)
    return X, tau


@pytest.mark.parametrize("pde,mk", [(oracle.PDE_EULER, lambda: euler_cfg((3, 3), N=3)),
                                    (oracle.PDE_ELASTICITY, lambda: elastic_cfg((2, 2, 2), N=2)),
                                    (oracle.PDE_ADVECTION, lambda: advection_cfg((3, 3), N=4))])
def test_constant_state_is_fixed_point(pde, mk):
    cfg = mk()
    n = cfg.N + 1
    ns = n ** cfg.dim
    q0 = inputs.random_state(pde, cfg.dim, 1, 1, seed=2)[0, 0]
    u = np.tile(q0, (ns, 1))
    qhat, qbar, Fbar, _ = oracle.predictor(cfg, u, 0.01)
    np.testing.assert_allclose(qhat, np.broadcast_to(u, qhat.shape), rtol=0, atol=1e-13)
    np.testing.assert_allclose(qbar, u, rtol=0, atol=1e-13)
    for d in range(cfg.dim):
        np.testing.assert_allclose(Fbar[d], np.tile(oracle.flux(cfg, q0, d), (ns, 1)), atol=1e-13)


def _poly_coefs(dim, N, seed):
    """Random polynomial of total degree <= N."""
    rng = np.random.default_rng(seed)
    coef = {}
    import itertools
    for k in itertools.product(range(N + 1), repeat=dim):
        if sum(k) <= N:
            coef[k + (0,) * (3 - dim)] = rng.uniform(-1, 1)
    return coef


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_1d_advection_exact_within_n_plus_1_iterations(N):
    """The paper states the Picard iteration terminates after at most N+1
    steps for linear homogeneous systems.  In 1D, with data of degree <= N,
    the fixed point is the space-time interpolant of u(x - a t): P = N+1
    iterations reproduce it to round-off.  Started from q = u(t^n) the
    initial error already lies in the range of the iteration operator, so
    N iterations are exact too, and N-1 are not."""
    a = 1.7
    n = N + 1
    mk = lambda P: oracle.make_cfg(1, [5], [0.0], [1.0], N, oracle.PDE_ADVECTION, [a], picard=P)
    X, tau = _element_nodes(mk(1), n)
    coef = _poly_coefs(1, N, seed=N)
    u = inputs.advection_poly(X, coef, [a, 0, 0])
    dt = 0.05
    exact = np.stack([inputs.advection_poly(X, coef, [a, 0, 0], t=tau[t] * dt) for t in range(n)])
    for P in (N + 1, N):
        qhat, _, _, it = oracle.predictor(mk(P), u, dt)
        assert it == P
        np.testing.assert_allclose(qhat, exact, atol=1e-13)
    if N >= 2:
        qhat, _, _, _ = oracle.predictor(mk(N - 1), u, dt)
        assert np.abs(qhat - exact).max() > 1e-10


@pytest.mark.parametrize("dim,N", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_multid_advection_termination_index(dim, N):
    """In d dimensions the Picard error operator (dt iK1 W) x L_s with
    L_s = sum_d a_d Dhat_d / dx_d has nilpotency index d N + 1 (mixed
    derivatives survive, so N+1 is not enough in general).  From the
    trivial guess the iteration is exact after d N steps and not before
    (reading 4).  Data of total degree <= N is reproduced exactly."""
    a = [1.0, -0.6, 0.8][:dim]
    mk = lambda P: oracle.make_cfg(dim, [3] * dim, [0.0] * dim, [1.0] * dim, N,
                                   oracle.PDE_ADVECTION, a, picard=P)
    n = N + 1
    X, tau = _element_nodes(mk(-1), n)
    rng = np.random.default_rng(dim * 10 + N)
    u = rng.uniform(-1, 1, size=(n ** dim, 1))
    dt = 0.04
    q_conv, _, _, _ = oracle.predictor(mk(-1), u, dt)
    k = dim * N
    q_k, _, _, it = oracle.predictor(mk(k), u, dt)
    assert it == k
    np.testing.assert_allclose(q_k, q_conv, atol=1e-13)
    q_km1, _, _, _ = oracle.predictor(mk(k - 1), u, dt)
    assert np.abs(q_km1 - q_conv).max() > 1e-8
    if dim > 1 and N > 1:
        q_n1, _, _, _ = oracle.predictor(mk(N + 1), u, dt)
        assert np.abs(q_n1 - q_conv).max() > 1e-8
    # exact reproduction of a total-degree <= N polynomial
    coef = _poly_coefs(dim, N, seed=3)
    up = inputs.advection_poly(X, coef, a + [0] * (3 - dim))
    qp, _, _, _ = oracle.predictor(mk(-1), up, dt)
    for t in range(n):
        exact = inputs.advection_poly(X, coef, a + [0] * (3 - dim), t=tau[t] * dt)
        np.testing.assert_allclose(qp[t], exact, atol=1e-12)


def _numpy_basis(n):
    """Independent 1D basis from numpy: GL rule, Lagrange polynomials by
    polyfit, their derivatives by polyder."""
    xr, wr = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (xr + 1), 0.5 * wr
    coeffs = [P.polyfit(x, np.eye(n)[k], n - 1) for k in range(n)]
    D = np.array([[P.polyval(x[j], P.polyder(coeffs[k])) for k in range(n)] for j in range(n)])
    F0 = np.array([P.polyval(0.0, c) for c in coeffs])
    F1 = np.array([P.polyval(1.0, c) for c in coeffs])
    # int_0^1 phi_k' phi_l by exact polynomial integration
    Kxi = np.zeros((n, n))
    for k in range(n):
        for l in range(n):
            prod = P.polyint(P.polymul(P.polyder(coeffs[k]), coeffs[l]))
            Kxi[k, l] = P.polyval(1.0, prod) - P.polyval(0.0, prod)
    return x, w, D, F0, F1, Kxi


@pytest.mark.parametrize("N", [1, 2, 3])
def test_2d_advection_matches_bruteforce_spacetime_solve(N):
    """Assemble the whole space-time system of eq. pde.st2 for linear
    advection with Kronecker products of numpy's basis and solve it
    directly; the oracle's converged Picard iterate must match."""
    n = N + 1
    a = (0.9, -1.4)
    cfg = oracle.make_cfg(2, [4, 5], [0.0, 0.0], [1.0, 1.0], N, oracle.PDE_ADVECTION, a, picard=-1)
    dx, dy = 0.25, 0.2
    x, w, D, F0, F1, Kxi = _numpy_basis(n)
    I = np.eye(n)
    K1 = np.outer(F1, F1) - Kxi
    Ls = a[0] / dx * np.kron(I, D) + a[1] / dy * np.kron(D, I)  # acts on [sy, sx]
    A = np.kron(K1, np.eye(n * n)) + 0.03 * np.kron(np.diag(w), Ls)
    rng = np.random.default_rng(N)
    u = rng.uniform(-1, 1, size=n * n)
    rhs = np.kron(F0, u)
    q_ref = np.linalg.solve(A, rhs).reshape(n, n * n)
    qhat, _, _, _ = oracle.predictor(cfg, u.reshape(-1, 1), 0.03)
    np.testing.assert_allclose(qhat[..., 0], q_ref, atol=1e-12)


def test_3d_elasticity_matches_bruteforce_spacetime_solve():
    """Same brute-force check for the 9-variable linear elasticity system,
    with numerically extracted flux matrices A_d (F_d(q) = A_d q)."""
    N, n = 1, 2
    cfg = elastic_cfg((2, 2, 2), N=N, picard=-1)
    h = 0.5
    m = 9
    A_d = []
    for d in range(3):
        A_d.append(np.stack([oracle.flux(cfg, np.eye(m)[k], d) for k in range(m)], axis=1))
    x, w, D, F0, F1, Kxi = _numpy_basis(n)
    I = np.eye(n)
    K1 = np.outer(F1, F1) - Kxi
    Dx = np.kron(np.kron(I, I), D)  # acts on [sz, sy, sx]
    Dy = np.kron(np.kron(I, D), I)
    Dz = np.kron(np.kron(D, I), I)
    Ls = (np.kron(Dx, A_d[0]) + np.kron(Dy, A_d[1]) + np.kron(Dz, A_d[2])) / h  # [s, v] ordering
    dt = 0.02
    A = np.kron(K1, np.eye(n ** 3 * m)) + dt * np.kron(np.diag(w), Ls)
    rng = np.random.default_rng(9)
    u = rng.uniform(-1, 1, size=(n ** 3, m))
    q_ref = np.linalg.solve(A, np.kron(F0, u.reshape(-1))).reshape(n, n ** 3, m)
    qhat, _, _, _ = oracle.predictor(cfg, u, dt)
    np.testing.assert_allclose(qhat, q_ref, atol=1e-12)


@pytest.mark.parametrize("N", [2, 3])
def test_euler_predictor_local_accuracy(N):
    """For the exact Euler density wave, the converged predictor on one
    element approximates the exact space-time solution with error
    O(h^{N+1}) (dt proportional to h)."""
    errs = []
    for h in (0.5, 0.25):
        cfg = euler_cfg((1, 1), N=N, L=h, picard=-1)
        n = N + 1
        X = oracle.node_coords(cfg)[0] + 1.1  # element [1.1, 1.1 + h]^2
        tau, _ = oracle.gauss_legendre(n)
        u = inputs.euler_density_wave(X, amp=0.2, L=3.0)
        dt = 0.2 * h
        qhat, _, _, _ = oracle.predictor(cfg, u, dt)
        e = 0.0
        for t in range(n):
            ex = inputs.euler_density_wave(X, amp=0.2, L=3.0, t=tau[t] * dt)
            e = max(e, np.abs(qhat[t] - ex).max())
        errs.append(e)
    order = np.log(errs[0] / errs[1]) / np.log(2)
    assert order > N + 0.6, (errs, order)
