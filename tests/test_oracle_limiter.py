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
- Detection (R25) against closed-form flip points: the floor delta = 1e-4
  on uniform data, delta = 1e-3 (hi - lo) over the face neighbours (not the
  diagonal ones), non-finite values, negative pressure within the bounds.
- Non-conservative products and sources (eq. pde.nc.fv): with alpha = 1 the
  diffuse-interface subcell scheme is the conservative elasticity one; a
  soft inclusion keeps the mirror symmetry; the reaction source on uniform
  data gives the second-order Taylor step in closed form.
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
    c = oracle.make_cfg(2, (4, 4), [0, 0], [1, 1], 2, oracle.PDE_EULER, [1.4], limiter=1,
                        guess=oracle.GUESS_EXTRAP)
    with pytest.raises(RuntimeError):
        oracle.step_limited(c, np.ones((16, 9, 4)), 1e-3)


def test_limited_diffuse_interface_with_alpha_one_equals_limited_elasticity():
    """alpha = 1 and constant material: the path-conservative subcell scheme
    (fluctuations +-J/2 at subcell faces, B(w~) s inside the subcells,
    B_d(w) s in the half-step) is the conservative MUSCL-Hancock scheme of
    the elasticity flux, since B_d is then that flux's constant Jacobian;
    and the unlimited neighbours' coupled fluctuations are the conservative
    fluxes (R30: the path integral between the two states of the unlimited
    element's side is then their flux difference).  Limited runs agree to
    rounding with equal troubled sets; the material fields stay bitwise
    constant."""
    cells, N = (12, 2, 2), 2
    ce = oracle.make_cfg(3, cells, [0] * 3, [1] * 3, N, oracle.PDE_ELASTICITY, [1.0, 2.0, 1.0], limiter=1)
    cd = oracle.make_cfg(3, cells, [0] * 3, [1] * 3, N, oracle.PDE_DIFFUSE_ELASTICITY, [], limiter=1)
    X = oracle.node_coords(ce)
    v = np.where((X[..., 0] > 1 / 3) & (X[..., 0] < 2 / 3), 1.0, 0.0)
    z = 0 * v
    U9 = np.stack([z] * 6 + [v, 0.5 * v, z], axis=-1)
    U13 = inputs.diffuse_pack(3, [U9[..., i] for i in range(6)], [U9[..., 6 + i] for i in range(3)], 1.0, 2.0, 1.0,
                              1.0)
    seen = 0
    for _ in range(6):
        dt = oracle.cfl_dt(ce, U9)
        assert dt == oracle.cfl_dt(cd, U13)
        U9, fe, ne = oracle.step_limited(ce, U9, dt)
        Ud, fd, nd = oracle.step_limited(cd, U13, dt)
        np.testing.assert_array_equal(fe, fd)
        assert np.array_equal(Ud[..., 9:], U13[..., 9:])
        U13 = Ud
        seen = max(seen, ne)
        assert np.abs(U13[..., :9] - U9).max() <= 1e-13 * np.abs(U9).max()
    assert 0 < seen < 48  # limited and unlimited elements side by side


def _mirror2d(U, cells, n):
    """x <-> y mirror of a 2D diffuse-interface state [e][s][v]: the element
    and node grids transposed, sigma_xx <-> sigma_yy, w_x <-> w_y."""
    E = U.reshape(cells[1], cells[0], n, n, -1)
    return E.transpose(1, 0, 3, 2, 4)[..., [1, 0, 2, 4, 3, 5, 6, 7, 8]].reshape(U.shape)


def test_limited_diffuse_interface_keeps_mirror_symmetry():
    """A soft inclusion (alpha from 1 to 0.3 across r = 0.25) hit by two
    mirrored velocity boxes: the limited run keeps the x <-> y mirror
    symmetry of the data to rounding (a wrong index, orientation or sign of
    the alpha-gradient terms in the subcell sweeps or the coupling breaks
    it) and the material fields bitwise."""
    cells, N = (12, 12), 3
    c = oracle.make_cfg(2, cells, [0, 0], [1, 1], N, oracle.PDE_DIFFUSE_ELASTICITY, [], limiter=1)
    X = oracle.node_coords(c)
    x, y = X[..., 0], X[..., 1]
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2)
    alpha = inputs.smooth_step(r, 0.25, 0.04, 0.3, 1.0)
    box = lambda a, b: np.where((a > 0.1) & (a < 0.3) & (b > 0.3) & (b < 0.6), 1.0, 0.0)
    z = 0 * x
    U = inputs.diffuse_pack(2, [z, z, z], [alpha * box(x, y), alpha * box(y, x)], alpha, 2.0, 1.0, 1.0)
    assert np.abs(U - _mirror2d(U, cells, N + 1)).max() == 0
    U0 = U.copy()
    seen = 0
    for _ in range(15):
        U, flags, cnt = oracle.step_limited(c, U, oracle.cfl_dt(c, U))
        seen = max(seen, cnt)
    assert 0 < seen < 144
    assert np.isfinite(U).all()
    assert np.abs(U - _mirror2d(U, cells, N + 1)).max() < 1e-13 * np.abs(U).max()
    assert np.array_equal(U[..., 5:], U0[..., 5:])


def test_limited_reaction_on_uniform_data_is_the_second_order_taylor_step():
    """Advection with the reaction S = -kappa q on uniform data: the decay
    leaves the relaxed maximum principle, so every element is troubled; with
    no gradients the subcell scheme reduces to the source at the half-step
    centre, u (1 - z + z^2 / 2), z = kappa dt, at every node (the DG step
    alone gives the subdiagonal Pade value instead)."""
    kappa = 2.0
    c = oracle.make_cfg(2, (4, 4), [0, 0], [1, 1], 3, oracle.PDE_ADVECTION, [1.0, 0.5, 0.0, kappa], limiter=1)
    U = np.full((16, 16, 1), 0.8)
    dt = oracle.cfl_dt(c, U)
    Ul, flags, cnt = oracle.step_limited(c, U, dt)
    assert cnt == 16 and flags.all()
    zt = kappa * dt
    np.testing.assert_allclose(Ul, 0.8 * (1 - zt + zt * zt / 2), rtol=1e-14)
    c.limiter = 0
    assert np.abs(oracle.step(c, U, dt) - 0.8 * (1 - zt + zt * zt / 2)).max() > 1e-6


def _grid_index(cells, i, j):
    return j * cells[0] + i


@pytest.mark.parametrize("eps, flagged", [(0.9e-4, False), (1.1e-4, True), (-1.1e-4, True)])
def test_detection_floor_of_the_relaxed_maximum_principle(eps, flagged):
    """Uniform u^n (range 0): the relaxed bounds are [c - 1e-4, c + 1e-4]
    (delta = max(1e-4, 1e-3 * 0)).  A candidate element shifted by eps has
    every subcell average at c + eps (the averages of a constant are that
    constant), so it is troubled exactly when |eps| > 1e-4, and no other
    element is."""
    cells = (6, 6)
    c = oracle.make_cfg(2, cells, [0, 0], [1, 1], 3, oracle.PDE_ADVECTION, [1.0, 0.5], limiter=1)
    U0 = np.full((36, 16, 1), 0.7)
    U = U0.copy()
    k = _grid_index(cells, 2, 3)
    U[k] += eps
    flags, cnt = oracle.detect(c, U0, U)
    assert cnt == int(flagged) and bool(flags[k]) == flagged


@pytest.mark.parametrize("eps, flagged", [(0.9e-3, False), (1.1e-3, True)])
def test_detection_bounds_span_the_face_neighbours(eps, flagged):
    """u^n = c except one element j at c + 1: every face neighbour k of j
    has bounds [c - delta, c + 1 + delta] with delta = 1e-3 * 1, so a
    candidate k at c + 1 + eps is troubled exactly when eps > 1e-3.  A
    diagonal neighbour of j does not see j (face neighbours only): shifted
    by 5e-4 it is troubled (its delta is 1e-4)."""
    cells = (6, 6)
    c = oracle.make_cfg(2, cells, [0, 0], [1, 1], 3, oracle.PDE_ADVECTION, [1.0, 0.5], limiter=1)
    U0 = np.full((36, 16, 1), 0.7)
    j = _grid_index(cells, 2, 2)
    U0[j] += 1.0
    for k in (_grid_index(cells, 3, 2), _grid_index(cells, 2, 1), _grid_index(cells, 1, 2), _grid_index(cells, 2, 3)):
        U = U0.copy()
        U[k] = 0.7 + 1.0 + eps
        flags, cnt = oracle.detect(c, U0, U)
        assert cnt == int(flagged) and bool(flags[k]) == flagged
    U = U0.copy()
    d = _grid_index(cells, 3, 3)
    U[d] += 5e-4
    flags, cnt = oracle.detect(c, U0, U)
    assert cnt == 1 and flags[d] == 1


def test_detection_flags_non_finite_and_negative_pressure():
    """Non-finite values flag an element; so does negative pressure where
    the maximum principle alone would not: u^n holds a moving element (rho
    1, momentum 3, rho E 10) next to resting ones (rho E 2.5), and a
    candidate element with momentum 3 and rho E 2.5 stays within every
    variable's bounds but has p = 0.4 (2.5 - 4.5) < 0."""
    cells = (4, 4)
    c = oracle.make_cfg(2, cells, [0, 0], [1, 1], 2, oracle.PDE_EULER, [1.4], limiter=1)
    U0 = np.zeros((16, 9, 4))
    U0[..., 0] = 1.0
    U0[..., 3] = 2.5
    j, k = _grid_index(cells, 1, 1), _grid_index(cells, 2, 1)
    U0[j, :, 1] = 3.0
    U0[j, :, 3] = 10.0
    assert oracle.detect(c, U0, U0.copy())[1] == 0
    U = U0.copy()
    U[5, 4, 0] = np.nan
    flags, cnt = oracle.detect(c, U0, U)
    assert cnt == 1 and flags[5] == 1
    U = U0.copy()
    U[k, :, 1] = 3.0  # rho E stays 2.5
    flags, cnt = oracle.detect(c, U0, U)
    assert cnt == 1 and flags[k] == 1
    U[k, :, 3] = 10.0  # the same momentum with enough energy: admissible, within bounds
    assert oracle.detect(c, U0, U)[1] == 0


# ---------------------------------------------------------------------------
# Kept subcell data (limiter mode 2, R35): a limited element keeps the subcell
# averages its subcell scheme produced as its subcell data at t^n, and an
# initial state can be given as subcell averages.


def _mono_avg(a, b, p):
    """Mean of x^p over [a, b]."""
    return (b ** (p + 1) - a ** (p + 1)) / ((p + 1) * (b - a))


@pytest.mark.parametrize("dim,N,cells", [(2, 3, (3, 2)), (3, 2, (2, 2, 3))])
def test_subcell_init_reconstructs_polynomials(dim, N, cells):
    """Subcell averages of a polynomial of degree <= N per direction, in
    closed form (monomial means over each subcell), give back that
    polynomial at the nodes: the least-squares reconstruction is exact on
    the DG space, in every direction and variable."""
    hi = [1.0, 1.5, 0.7][:dim]
    c = oracle.make_cfg(dim, cells, [0.0] * dim, hi, N, oracle.PDE_EULER, [1.4], limiter=2)
    m, S = c.m, 2 * N + 1
    rng = np.random.default_rng(35)
    expo = rng.integers(0, N + 1, size=(m, 4, dim))  # four monomials per variable
    coef = rng.normal(size=(m, 4))
    X = oracle.node_coords(c)
    want = np.zeros(X.shape[:-1] + (m,))
    for v in range(m):
        for t in range(4):
            want[..., v] += coef[v, t] * np.prod([X[..., d] ** expo[v, t, d] for d in range(dim)], axis=0)
    E = int(np.prod(cells))
    avg = np.zeros((E, S ** dim, m))
    for e in range(E):
        ie, r = [], e
        for d in range(dim):
            ie.append(r % cells[d]); r //= cells[d]
        for a in range(S ** dim):
            ia, r = [], a
            for d in range(dim):
                ia.append(r % S); r //= S
            lo_ = [(ie[d] * S + ia[d]) * hi[d] / (cells[d] * S) for d in range(dim)]
            hi_ = [(ie[d] * S + ia[d] + 1) * hi[d] / (cells[d] * S) for d in range(dim)]
            for v in range(m):
                avg[e, a, v] = sum(coef[v, t] * np.prod([_mono_avg(lo_[d], hi_[d], expo[v, t, d]) for d in range(dim)])
                                   for t in range(4))
    U, kept = oracle.subcell_init(c, avg)
    assert kept.kept.all() and np.array_equal(kept.sub, avg)
    np.testing.assert_allclose(U, want, rtol=0, atol=1e-12)


def test_kept_cfl_takes_the_subcell_averages():
    """Wave speeds of kept elements come from their subcell averages: a
    uniform state given as averages gives alpha / sum_d (|v_d| + c) / dx_d
    in closed form, whatever the kept elements' nodes hold (NaN here); the
    same nodes without kept data give no finite step."""
    cells, hi, g = (6, 4), (1.0, 2.0), 1.4
    c = oracle.make_cfg(2, cells, [0, 0], list(hi), 2, oracle.PDE_EULER, [g], limiter=2)
    rho, vx, vy, p = 1.3, 0.4, -0.2, 0.9
    q = np.array([rho, rho * vx, rho * vy, p / (g - 1) + 0.5 * rho * (vx * vx + vy * vy)])
    E, S = 24, 5
    avg = np.broadcast_to(q, (E, S * S, 4)).copy()
    U, kept = oracle.subcell_init(c, avg)
    cs = math.sqrt(g * p / rho)
    want = oracle.alpha(c) / ((abs(vx) + cs) / (hi[0] / cells[0]) + (abs(vy) + cs) / (hi[1] / cells[1]))
    assert abs(oracle.cfl_dt_kept(c, U, kept) - want) <= 1e-14 * want
    Unan = np.full_like(U, np.nan)
    assert abs(oracle.cfl_dt_kept(c, Unan, kept) - want) <= 1e-14 * want
    kept.kept[:12] = 0  # half the elements from their nodes again
    Uhalf = Unan.copy()
    Uhalf[:12] = q
    assert abs(oracle.cfl_dt_kept(c, Uhalf, kept) - want) <= 1e-14 * want
    kept.kept[:] = 0
    assert not np.isfinite(oracle.cfl_dt_kept(c, Unan, kept))


def test_kept_mode_without_kept_data_is_the_plain_limiter():
    """From a nodal state (nothing kept) a kept-mode step is the plain
    limited step bit for bit; it keeps the troubled elements' new subcell
    averages, whose reconstruction is exactly their new nodal state."""
    c, U = _explosion()
    dt = oracle.cfl_dt(c, U)
    U1, f1, n1 = oracle.step_limited(c, U, dt)
    c.limiter = 2
    kept = oracle.Kept(c)
    U2, f2, n2 = oracle.step_limited_kept(c, U, kept, dt)
    assert n1 == n2 > 0
    np.testing.assert_array_equal(U1, U2)
    np.testing.assert_array_equal(f1, f2)
    np.testing.assert_array_equal(kept.kept, f2)
    R, _ = oracle.subcell_init(c, kept.sub)
    np.testing.assert_array_equal(R[f2 == 1], U2[f2 == 1])


def test_sharp_sod_with_kept_subcell_data():
    """Sod's tubes with the discontinuities inside elements, given as
    subcell averages: the nodal interpolant of such data is not admissible,
    but with kept subcell data the run stays positive, conserves mass to
    rounding and follows the exact Riemann solution (shock position, star
    plateau)."""
    nx, N, s = 64, 3, 0.4 / 64
    c = oracle.make_cfg(2, (nx, 1), [0, 0], [1.0, 1.0 / nx], N, oracle.PDE_EULER, [1.4], limiter=2)

    def tubes(X):
        x = X[..., 0]
        high = (x > 0.25 + s) & (x < 0.75 + s)
        rho = np.where(high, 1.0, 0.125)
        p = np.where(high, 1.0, 0.1)
        z = 0 * rho
        return np.stack([rho, z, z, p / 0.4], axis=-1)

    avg = inputs.subcell_means(tubes, (nx, 1), (0.0, 0.0), (1.0, 1.0 / nx), N, k=5)
    U0, kept = oracle.subcell_init(c, avg)
    M0 = oracle.mass(c, U0)
    np.testing.assert_allclose(M0[0], (0.5 * 1.0 + 0.5 * 0.125) / nx, rtol=1e-13)  # the averages' mass
    c.limiter = 1  # the plain limiter re-projects the reconstruction, whose subcells are not admissible
    assert not np.isfinite(oracle.run(c, U0, 0.1)[0]).all()
    c.limiter = 2
    U, t, k, _ = oracle.run_kept(c, U0, kept, 0.1)
    assert t == 0.1 and np.isfinite(U).all()
    np.testing.assert_allclose(oracle.mass(c, U), M0, rtol=0, atol=1e-14)
    ks = kept.sub[kept.kept == 1]
    assert ks.size and ks[..., 0].min() > 0
    assert (0.4 * (ks[..., 3] - 0.5 * (ks[..., 1] ** 2 + ks[..., 2] ** 2) / ks[..., 0])).min() > 0
    x = oracle.node_coords(c)[..., 0]
    rho = U[..., 0]
    ok = kept.kept == 0  # unlimited elements: their nodes are the solution
    x0 = 0.75 + s
    ex_r, star = _sod_exact(x, t, x0)
    ex_l, _ = _sod_exact(2 * (0.5 + s) - x, t, x0)
    ex = np.where(x >= 0.5 + s, ex_r, ex_l)
    l1 = nx * np.sum(node_weights(c) * np.abs(rho - ex))
    assert l1 < 0.02, l1
    xs = x0 + star["shock"] * t
    right = (x > x0 + star["u"] * t + 0.02) & ok[:, None]
    mid = 0.5 * (star["rho_star_right"] + 0.125)
    pos = x[right & (rho > mid)].max()
    assert abs(pos - xs) < 1.5 / nx, (pos, xs)
    plateau = rho[(x > x0 + star["u"] * t + 0.02) & (x < xs - 0.02) & ok[:, None]]
    assert np.abs(plateau - star["rho_star_right"]).max() < 0.05 * star["rho_star_right"]


def test_sharp_blast_with_kept_subcell_data_keeps_symmetry_and_mass():
    """A blast with a sharp circular edge (rho 1 / 0.125, p 1 / 0.1) given as
    subcell averages: 20 limited steps with kept subcell data stay finite,
    keep the kept averages admissible, conserve mass to rounding and keep
    the x <-> y mirror symmetry of the data (states and troubled sets)."""
    C, N = 16, 4
    c = oracle.make_cfg(2, (C, C), [0, 0], [1, 1], N, oracle.PDE_EULER, [1.4], limiter=2)
    avg = inputs.subcell_means(inputs.euler_sharp_blast((0.5, 0.5), 0.2), (C, C), (0.0, 0.0), (1.0, 1.0), N)
    U, kept = oracle.subcell_init(c, avg)
    M0 = oracle.mass(c, U)
    seen = 0
    for _ in range(20):
        U, flags, cnt = oracle.step_limited_kept(c, U, kept, oracle.cfl_dt_kept(c, U, kept))
        seen = max(seen, cnt)
        F = flags.reshape(C, C)
        assert np.array_equal(F, F.T)
    assert 0 < seen < C * C
    assert np.isfinite(U).all()
    ks = kept.sub[kept.kept == 1]
    assert ks[..., 0].min() > 0 and (0.4 * (ks[..., 3] - 0.5 * (ks[..., 1] ** 2 + ks[..., 2] ** 2) / ks[..., 0])).min() > 0
    np.testing.assert_allclose(oracle.mass(c, U), M0, rtol=0, atol=5e-14)
    n = N + 1
    Eu = U.reshape(C, C, n, n, 4)  # [ey, ex, sy, sx, v]
    mirror = Eu.transpose(1, 0, 3, 2, 4)[..., [0, 2, 1, 3]]
    assert np.abs(Eu - mirror).max() < 1e-12


def test_subcell_means_layout_and_linear_fields():
    """The subcell-average input generator: for a linear field the midpoint
    samples average to the field at the subcell centre, in the layout
    [element (x fastest)][subcell (x fastest)][variable]; a constant field
    gives the constant."""
    cells, lo, hi, N = (3, 2), (0.5, -1.0), (2.0, 1.0), 2
    S = 2 * N + 1
    field = lambda X: np.stack([1.0 + 2.0 * X[..., 0] + 3.0 * X[..., 1], 0 * X[..., 0] + 7.0], axis=-1)
    avg = inputs.subcell_means(field, cells, lo, hi, N, k=3)
    assert avg.shape == (6, S * S, 2)
    h = [(hi[d] - lo[d]) / (cells[d] * S) for d in range(2)]
    for e in range(6):
        ex, ey = e % cells[0], e // cells[0]
        for a in range(S * S):
            ax, ay = a % S, a // S
            x = lo[0] + (ex * S + ax + 0.5) * h[0]
            y = lo[1] + (ey * S + ay + 0.5) * h[1]
            assert abs(avg[e, a, 0] - (1.0 + 2.0 * x + 3.0 * y)) < 1e-13
            assert avg[e, a, 1] == 7.0


def test_kept_run_equals_kept_steps():
    """The oracle's CFL time loop with kept subcell data is its kept-data
    step repeated with the kept-data CFL step (the reference the GPU runs
    are compared with step by step)."""
    C, N = 8, 3
    c = oracle.make_cfg(2, (C, C), [0, 0], [1, 1], N, oracle.PDE_EULER, [1.4], limiter=2)
    avg = inputs.subcell_means(inputs.euler_sharp_blast((0.5, 0.5), 0.25), (C, C), (0.0, 0.0), (1.0, 1.0), N, k=4)
    U0, k0 = oracle.subcell_init(c, avg)
    Ur, t, steps, hist = oracle.run_kept(c, U0, oracle.Kept(c, k0.sub, k0.kept), 0.02)
    U, kept = U0.copy(), oracle.Kept(c, k0.sub, k0.kept)
    tt = 0.0
    for k in range(steps):
        dt = min(oracle.cfl_dt_kept(c, U, kept), 0.02 - tt)
        assert dt == hist[k]
        U, _, _ = oracle.step_limited_kept(c, U, kept, dt)
        tt += dt
    assert steps > 2 and t == 0.02
    np.testing.assert_array_equal(U, Ur)


def test_sedov_blast_with_kept_subcell_data():
    """The Sedov blast of Sec. 3.1's limiter example: unit density at rest,
    pressure 1e-14, and the energy E0 = 0.979264 deposited in a disk 2.5
    subcells wide at the centre, given as subcell averages; 2D, 20^2, N = 3,
    limiter with kept subcell data.  The run stays finite with positive
    density and kept pressures, conserves mass to rounding, keeps the
    x <-> y mirror symmetry, and its shock (the densest node) moves
    self-similarly, r ~ t^(1/2) (dimensional analysis of the point blast in
    2D: r = xi (E t^2 / rho)^(1/4)), reaching r = 1 at t = 1 for this E0 and
    gamma = 1.4."""
    C, N, L = 20, 3, 1.2
    c = oracle.make_cfg(2, (C, C), [-L, -L], [L, L], N, oracle.PDE_EULER, [1.4], limiter=2)
    h = 2 * L / (C * (2 * N + 1))
    r0, E0 = 2.5 * h, 0.979264

    def field(X):
        r = np.sqrt(X[..., 0] ** 2 + X[..., 1] ** 2)
        return np.stack([np.ones_like(r), 0 * r, 0 * r, np.where(r < r0, E0 / (math.pi * r0 ** 2), 1e-14 / 0.4)],
                        axis=-1)

    avg = inputs.subcell_means(field, (C, C), (-L, -L), (L, L), N, k=8)
    U, kept = oracle.subcell_init(c, avg)
    M0 = oracle.mass(c, U)
    X = oracle.node_coords(c)
    r = np.sqrt(X[..., 0] ** 2 + X[..., 1] ** 2)
    radii = {}
    t = 0.0
    for t_end in (0.25, 1.0):
        U, t, _, _ = oracle.run_kept(c, U, kept, t_end, t0=t)
        assert t == t_end and np.isfinite(U).all() and U[..., 0].min() > 0
        radii[t_end] = r.reshape(-1)[np.argmax(U[..., 0])]
        ks = kept.sub[kept.kept == 1]
        assert ks[..., 0].min() > 0
        assert (0.4 * (ks[..., 3] - 0.5 * (ks[..., 1] ** 2 + ks[..., 2] ** 2) / ks[..., 0])).min() > 0
    np.testing.assert_allclose(oracle.mass(c, U), M0, rtol=0, atol=1e-12)
    n = N + 1
    Eu = U.reshape(C, C, n, n, 4)
    assert np.abs(Eu - Eu.transpose(1, 0, 3, 2, 4)[..., [0, 2, 1, 3]]).max() < 1e-12
    assert abs(radii[1.0] / radii[0.25] - 2.0) < 0.15, radii
    assert abs(radii[1.0] - 1.0) < 0.05, radii
