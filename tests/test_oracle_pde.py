"""Pins of the oracle's PDE functions and Riemann solver.

Fluxes are pinned through their Jacobians: the eigenvalues of dF_d/dQ
(finite differences, numpy.linalg.eigvals) must match the oracle's wave
speed, and known invariances must hold.  The Rusanov flux (eq. rusanov) is
pinned by consistency, the sum rule of swapped states, and its reduction
to upwinding for linear advection."""
import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import inputs

GAMMA = 1.4


def _cfg(pde, dim, prm):
    return oracle.make_cfg(dim, [4] * dim, [0.0] * dim, [1.0] * dim, 2, pde, prm)


def _jacobian(cfg, q, d, h=1e-6):
    m = cfg.m
    J = np.zeros((m, m))
    for k in range(m):
        dq = np.zeros(m)
        dq[k] = h * max(1.0, abs(q[k]))
        J[:, k] = (oracle.flux(cfg, q + dq, d) - oracle.flux(cfg, q - dq, d)) / (2 * dq[k])
    return J


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_flux_jacobian_eigenvalues(dim):
    cfg = _cfg(oracle.PDE_EULER, dim, [GAMMA])
    U = inputs.random_state(inputs.PDE_EULER, dim, 6, 1, seed=11 + dim, amp=0.4)[:, 0, :]
    for q in U:
        rho = q[0]
        v = q[1:1 + dim] / rho
        p = (GAMMA - 1) * (q[dim + 1] - 0.5 * rho * np.dot(v, v))
        c = np.sqrt(GAMMA * p / rho)
        for d in range(dim):
            ev = np.sort(np.linalg.eigvals(_jacobian(cfg, q, d)).real)
            expect = np.sort([v[d] - c] + [v[d]] * dim + [v[d] + c])
            np.testing.assert_allclose(ev, expect, atol=1e-6)
            assert abs(oracle.max_eig(cfg, q, d) - np.max(np.abs(ev))) < 1e-6


def test_euler_flux_rotation_and_mass_row():
    cfg = _cfg(oracle.PDE_EULER, 2, [GAMMA])
    q = inputs.random_state(inputs.PDE_EULER, 2, 1, 1, seed=5)[0, 0]
    # F_y(q) = P F_x(P q) with P swapping the two momenta
    Pm = np.eye(4)[[0, 2, 1, 3]]
    np.testing.assert_allclose(oracle.flux(cfg, q, 1), Pm @ oracle.flux(cfg, Pm @ q, 0), rtol=1e-15)
    # mass flux is the momentum; a state at rest has flux (0, p, 0, 0)
    assert oracle.flux(cfg, q, 0)[0] == q[1]
    rest = np.array([1.3, 0.0, 0.0, 2.5])
    p = (GAMMA - 1) * 2.5
    np.testing.assert_allclose(oracle.flux(cfg, rest, 0), [0, p, 0, 0], atol=1e-15)


def test_elasticity_flux_jacobian_spectrum():
    rho, lam, mu = 1.0, 2.0, 1.0
    cfg = _cfg(oracle.PDE_ELASTICITY, 3, [rho, lam, mu])
    q = inputs.random_state(inputs.PDE_ELASTICITY, 3, 1, 1, seed=3)[0, 0]
    cp, cs = np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho)
    for d in range(3):
        J = _jacobian(cfg, q, d)
        # linear system: the flux is exactly J q
        np.testing.assert_allclose(J @ q, oracle.flux(cfg, q, d), atol=1e-9)
        ev = np.sort(np.linalg.eigvals(J).real)
        np.testing.assert_allclose(ev, np.sort([-cp, -cs, -cs, 0, 0, 0, cs, cs, cp]), atol=1e-7)
        assert abs(oracle.max_eig(cfg, q, d) - cp) < 1e-15


def test_elasticity_plane_wave_is_exact_solution():
    """Q(x,t) = plane wave: Q_t + dF_x/dx = 0 checked by finite differences
    of the oracle's flux along x."""
    cfg = _cfg(oracle.PDE_ELASTICITY, 3, [1.0, 2.0, 1.0])
    for kind in ("p", "s"):
        x = np.array([[0.3, 0.1, 0.7]])
        h = 1e-5
        qt = (inputs.elastic_plane_wave(x, kind, t=h) - inputs.elastic_plane_wave(x, kind, t=-h))[0] / (2 * h)
        fx = [oracle.flux(cfg, inputs.elastic_plane_wave(x + s * np.array([h, 0, 0]), kind)[0], 0)
              for s in (1, -1)]
        np.testing.assert_allclose(qt + (fx[0] - fx[1]) / (2 * h), 0.0, atol=1e-6)


def test_euler_density_wave_is_exact_solution():
    cfg = _cfg(oracle.PDE_EULER, 2, [GAMMA])
    x = np.array([[1.3, 4.4]])
    h = 1e-5
    qt = (inputs.euler_density_wave(x, t=h) - inputs.euler_density_wave(x, t=-h))[0] / (2 * h)
    div = np.zeros(4)
    for d in range(2):
        e = np.zeros(2)
        e[d] = h
        div += (oracle.flux(cfg, inputs.euler_density_wave(x + e)[0], d)
                - oracle.flux(cfg, inputs.euler_density_wave(x - e)[0], d)) / (2 * h)
    np.testing.assert_allclose(qt + div, 0.0, atol=1e-8)


@pytest.mark.parametrize("pde,dim,prm", [(oracle.PDE_EULER, 2, [GAMMA]),
                                         (oracle.PDE_ELASTICITY, 3, [1.0, 2.0, 1.0]),
                                         (oracle.PDE_ADVECTION, 2, [0.7, -1.3])])
def test_rusanov_consistency_and_sum_rule(pde, dim, prm):
    cfg = _cfg(pde, dim, prm)
    U = inputs.random_state(pde, dim, 2, 1, seed=7)[:, 0, :]
    qL, qR = U[0], U[1]
    for d in range(dim):
        fL, fR = oracle.flux(cfg, qL, d), oracle.flux(cfg, qR, d)
        np.testing.assert_allclose(oracle.rusanov(cfg, d, qL, fL, qL, fL), fL, rtol=1e-15, atol=1e-15)
        s1 = oracle.rusanov(cfg, d, qL, fL, qR, fR)
        s2 = oracle.rusanov(cfg, d, qR, fR, qL, fL)
        np.testing.assert_allclose(s1 + s2, fL + fR, atol=1e-14)
        # dissipation has the sign that damps the jump
        smax = max(oracle.max_eig(cfg, qL, d), oracle.max_eig(cfg, qR, d))
        np.testing.assert_allclose(s1 - s2, -smax * (qR - qL), atol=1e-14)


def test_rusanov_is_upwind_for_advection():
    cfg = _cfg(oracle.PDE_ADVECTION, 2, [0.8, -1.5])
    qL, qR = np.array([0.3]), np.array([-1.1])
    f = lambda q, d: oracle.flux(cfg, q, d)
    np.testing.assert_allclose(oracle.rusanov(cfg, 0, qL, f(qL, 0), qR, f(qR, 0)), 0.8 * qL, rtol=1e-15)
    np.testing.assert_allclose(oracle.rusanov(cfg, 1, qL, f(qL, 1), qR, f(qR, 1)), -1.5 * qR, rtol=1e-15)
