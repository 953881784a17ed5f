"""Pins of the oracle's a posteriori subcell finite-volume limiter (Sec. 2.3).

- The subcell operators: averages of the nodal basis over the 2N+1 equal
  subcells are exact for polynomials of degree <= N, rows sum to one, the
  least-squares reconstruction inverts them on the DG space and keeps the
  element's mass.
- Smooth data stays unlimited (the density wave: nothing flagged, the step
  equals the unlimited one bitwise).
- Sod's shock tube (quasi-1D): the unlimited scheme breaks down, the
  limited one stays admissible, conserves mass to rounding and follows the
  exact Riemann solution (shock position, plateau densities; the exact
  solution from the Rankine-Hugoniot and rarefaction relations, solved here).
- A 2D explosion: mass conserved to rounding through limited / unlimited
  couplings, and the x <-> y mirror symmetry of the data kept to rounding
  (a wrong index or orientation in the subcell sweeps or the face coupling
  breaks it).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import inputs
from helpers import node_weights


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_subcell_operators(N):
    n, S = N + 1, 2 * N + 1
    Pr, Rc = oracle.subcell_ops(N)
    x, w = oracle.gauss_legendre(n)
    np.testing.assert_allclose(Pr.sum(axis=1), 1.0, atol=1e-14)
    for p in range(N + 1):
        exact = np.array([((j + 1) ** (p + 1) - j ** (p + 1)) / ((p + 1) * S ** p) for j in range(S)])
        np.testing.assert_allclose(Pr @ x ** p, exact, atol=1e-13)
    np.testing.assert_allclose(Rc @ Pr, np.eye(n), atol=1e-12)
    # the reconstruction keeps the element's mass: int u' = mean of the averages
    np.testing.assert_allclose(w @ Rc, np.full(S, 1.0 / S), atol=1e-14)


def test_smooth_data_is_not_limited():
    c = oracle.make_cfg(2, (10, 10), [0, 0], [10, 10], 3, oracle.PDE_EULER, [1.4], limiter=1)
    U = inputs.euler_density_wave(oracle.node_coords(c), L=10.0)
    dt = oracle.cfl_dt(c, U)
    Ul, flags, cnt = oracle.step_limited(c, U, dt)
    assert cnt == 0 and not flags.any()
    c.limiter = 0
    np.testing.assert_array_equal(Ul, oracle.step(c, U, dt))


def _sod_exact(x, t, x0, g=1.4, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Density of the exact Riemann solution (left rarefaction, right shock
    for Sod's data): the star pressure solves f_L(p) + f_R(p) + du = 0 with
    the shock (Rankine-Hugoniot) and rarefaction (Riemann invariant)
    branches of f."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)

    def f(p, r, pk, ck):
        if p > pk:
            A, B = 2 / ((g + 1) * r), (g - 1) / (g + 1) * pk
            return (p - pk) * math.sqrt(A / (p + B))
        return 2 * ck / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)

    lo, hi = 1e-10, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid, rL, pL, cL) + f(mid, rR, pR, cR) + (uR - uL) > 0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (uL + uR) + 0.5 * (f(ps, rR, pR, cR) - f(ps, rL, pL, cL))
    rsR = rR * (ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1)
    SR = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
    rsL = rL * (ps / pL) ** (1 / g)
    csL = cL * (ps / pL) ** ((g - 1) / (2 * g))
    xi = (np.asarray(x) - x0) / t
    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - xi))
    fan = rL * (np.maximum(c, 1e-300) / cL) ** (2 / (g - 1))
    rho = np.where(xi < uL - cL, rL, np.where(xi < us - csL, fan, np.where(xi < us, rsL, np.where(xi < SR, rsR, rR))))
    return rho, dict(p=ps, u=us, rho_star_left=rsL, rho_star_right=rsR, shock=SR)


def _sod_state(c):
    """Periodic double shock tube on [0, 1]: high state on (0.25, 0.75)."""
    x = oracle.node_coords(c)[..., 0]
    high = (x > 0.25) & (x < 0.75)
    rho = np.where(high, 1.0, 0.125)
    p = np.where(high, 1.0, 0.1)
    return x, np.stack([rho, 0 * rho, 0 * rho, p / 0.4], axis=-1)


def test_unlimited_scheme_breaks_down_on_sod():
    c = oracle.make_cfg(2, (64, 1), [0, 0], [1.0, 1.0 / 64], 3, oracle.PDE_EULER, [1.4])
    _, U = _sod_state(c)
    for _ in range(30):
        U = oracle.step(c, U, oracle.cfl_dt(c, U))
        if not np.isfinite(U).all():
            break
    assert not np.isfinite(U).all()


def test_limited_sod_follows_the_exact_solution():
    nx = 64
    c = oracle.make_cfg(2, (nx, 1), [0, 0], [1.0, 1.0 / nx], 3, oracle.PDE_EULER, [1.4], limiter=1)
    x, U0 = _sod_state(c)
    M0 = oracle.mass(c, U0)
    U, t, k, _ = oracle.run(c, U0, 0.1)
    assert t == 0.1 and np.isfinite(U).all()
    rho = U[..., 0]
    kin = 0.5 * (U[..., 1] ** 2 + U[..., 2] ** 2) / rho
    assert rho.min() > 0 and (0.4 * (U[..., 3] - kin)).min() > 0
    np.testing.assert_allclose(oracle.mass(c, U), M0, rtol=0, atol=1e-14)
    ex_r, star = _sod_exact(x, t, 0.75)
    ex_l, _ = _sod_exact(1.0 - x, t, 0.75)
    ex = np.where(x >= 0.5, ex_r, ex_l)
    assert abs(star["shock"] - 1.75216) < 1e-4 and abs(star["p"] - 0.30313) < 1e-4  # Sod's star state
    l1 = nx * np.sum(node_weights(c) * np.abs(rho - ex))  # per unit length
    assert l1 < 0.02, l1
    # shock position: last node right of the contact above the mid density
    xs = 0.75 + star["shock"] * t
    right = x > 0.75 + star["u"] * t + 0.02
    mid = 0.5 * (star["rho_star_right"] + 0.125)
    pos = x[right & (rho > mid)].max()
    assert abs(pos - xs) < 1.5 / nx, (pos, xs)
    # plateau between contact and shock
    plateau = rho[(x > 0.75 + star["u"] * t + 0.02) & (x < xs - 0.02)]
    assert np.abs(plateau - star["rho_star_right"]).max() < 0.05 * star["rho_star_right"]


def _explosion(cells=(16, 16), N=3):
    """Blast with a tanh edge of width 0.03 (admissible subcell averages)."""
    c = oracle.make_cfg(2, cells, [0, 0], [1, 1], N, oracle.PDE_EULER, [1.4], limiter=1)
    X = oracle.node_coords(c)
    r = np.sqrt((X[..., 0] - 0.5) ** 2 + (X[..., 1] - 0.5) ** 2)
    rho = inputs.smooth_step(r, 0.2, 0.03, 1.0, 0.125)
    p = inputs.smooth_step(r, 0.2, 0.03, 1.0, 0.1)
    return c, np.stack([rho, 0 * rho, 0 * rho, p / 0.4], axis=-1)


def test_limited_explosion_conserves_and_keeps_symmetry():
    c, U = _explosion()
    M0 = oracle.mass(c, U)
    seen = 0
    for _ in range(20):
        U, flags, cnt = oracle.step_limited(c, U, oracle.cfl_dt(c, U))
        seen = max(seen, cnt)
    assert 0 < seen < 256  # limited and unlimited elements side by side
    np.testing.assert_allclose(oracle.mass(c, U), M0, rtol=0, atol=5e-14)
    assert U[..., 0].min() > 0
    E = U.reshape(16, 16, 4, 4, 4)  # [ey, ex, sy, sx, v]
    mirror = E.transpose(1, 0, 3, 2, 4)[..., [0, 2, 1, 3]]
    assert np.abs(E - mirror).max() < 1e-13


def test_limiter_rejects_what_it_does_not_cover():
    c = oracle.make_cfg(2, (4, 4), [0, 0], [1, 1], 2, oracle.PDE_DIFFUSE_ELASTICITY, [], limiter=1)
    with pytest.raises(RuntimeError):
        oracle.step_limited(c, np.ones((16, 9, 9)), 1e-3)
    c = oracle.make_cfg(2, (4, 4), [0, 0], [1, 1], 2, oracle.PDE_EULER, [1.4], limiter=1,
                        guess=oracle.GUESS_EXTRAP)
    with pytest.raises(RuntimeError):
        oracle.step_limited(c, np.ones((16, 9, 4)), 1e-3)
