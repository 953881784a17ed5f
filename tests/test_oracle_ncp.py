"""Pins of the oracle's non-conservative products, path-conservative faces
and algebraic sources (eq. pde, eq. pde.nc.gw2, eq. pc.scheme; the
diffuse-interface elasticity system of Sec. 3.2; a linear reaction source
on advection).

Each pin is fixed outside the oracle's own formulas:
- with alpha = 1 the diffuse-interface products equal the Jacobian of the
  conservative elasticity flux (a separate routine), and whole runs equal
  the conservative scheme;
- the alpha terms are the product rules they stand for: the stress rows
  see the velocity gradient dv = d(w / alpha), the momentum rows the
  divergence of alpha sigma;
- the eigenvalues of B_d do not depend on alpha;
- path integrals against closed forms, exact where the integrand is a
  polynomial of degree <= 5 and within the three-point Gauss-Legendre error
  bound where it is rational;
- a free surface (alpha -> 0) reflects a P-wave with the stress sign
  flipped and a material interface transmits the impedance ratio;
- the reaction term reproduces the subdiagonal Pade approximant of the
  time-DG method and the design order of accuracy.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import inputs

DI = oracle.PDE_DIFFUSE_ELASTICITY
RNG = np.random.default_rng(1808)

# 3-point Gauss-Legendre rule on [0, 1]: error = f^(6)(eta) (3!)^4 / (7 (6!)^3)
GL3_ERR = math.factorial(3) ** 4 / (7 * math.factorial(6) ** 3)


def _cfg(dim, N=2, cells=None):
    cells = cells or (2,) * dim
    return oracle.make_cfg(dim, cells, [0] * dim, [1] * dim, N, DI, [])


def _state(dim, sigma, w, alpha, lam, mu, rho):
    return inputs.diffuse_pack(dim, sigma, w, alpha, lam, mu, rho)


def _nsig(dim):
    return 6 if dim == 3 else 3


def _sym(dim, i, j):
    i, j = min(i, j), max(i, j)
    if dim == 2:
        return i if i == j else 2
    return i if i == j else {(0, 1): 3, (1, 2): 4, (0, 2): 5}[(i, j)]


def _hooke(dim, lam, mu, G):
    """E : G for a velocity-gradient matrix G, in the state's stress order."""
    out = np.zeros(_nsig(dim))
    tr = np.trace(G)
    for i in range(dim):
        for j in range(i, dim):
            out[_sym(dim, i, j)] = lam * tr * (i == j) + mu * (G[i, j] + G[j, i])
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_ncp_with_alpha_one_is_the_elastic_flux_jacobian(dim):
    """alpha = 1, no alpha gradient: B_d(q) g = dF_d/dq g of the
    conservative velocity-stress system (the flux routine of PDE 3), on the
    plane-strain rows in 2D; the material rows are zero."""
    lam, mu, rho = 2.3, 0.7, 1.6
    ce = oracle.make_cfg(3, (2, 2, 2), [0] * 3, [1] * 3, 2, oracle.PDE_ELASTICITY, [rho, lam, mu])
    cd = _cfg(dim)
    ev = [0, 1, 2, 3, 4, 5, 6, 7, 8] if dim == 3 else [0, 1, 3, 6, 7]  # elastic indices of the evolved rows
    for _ in range(3):
        q9 = RNG.uniform(-1, 1, 9)
        q = np.concatenate([q9[ev], [1.0, lam, mu, rho]])
        for d in range(dim):
            J = np.zeros((9, 9))
            for k in range(9):
                e = np.zeros(9)
                e[k] = 1.0
                J[:, k] = (oracle.flux(ce, q9 + e, d) - oracle.flux(ce, q9 - e, d)) / 2.0
            g9 = np.zeros(9)
            g9[ev] = RNG.uniform(-1, 1, len(ev))
            g = np.concatenate([g9[ev], [0.0] + list(RNG.uniform(-1, 1, 3))])  # material gradients do not enter
            out = oracle.ncp(cd, q, d, g)
            np.testing.assert_allclose(out[: len(ev)], (J @ g9)[ev], rtol=1e-14, atol=1e-14)
            assert np.all(out[len(ev):] == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_alpha_terms_are_the_product_rules(dim):
    """Along a line x(s) = x0 + s e_d with smooth v(s), alpha(s), sigma(s):
    the stress rows of B_d(q) dq/ds are -E : (dv/ds (x) e_d) and the
    momentum rows -(1/rho) d(alpha sigma_{i d})/ds, whatever alpha does."""
    lam, mu, rho = 1.7, 0.9, 2.2
    nsig = _nsig(dim)
    cv, ca, cs = RNG.uniform(-1, 1, (dim, 3)), RNG.uniform(0.2, 0.6, 3), RNG.uniform(-1, 1, (nsig, 3))

    def fields(s):
        v = cv[:, 0] + cv[:, 1] * s + cv[:, 2] * s * s
        a = 0.3 + ca[0] * s * s + ca[1] * math.sin(s) ** 2 + 0.1 * ca[2]
        sig = cs[:, 0] + cs[:, 1] * math.cos(s) + cs[:, 2] * s ** 3
        return v, a, sig

    def q_of(s):
        v, a, sig = fields(s)
        return _state(dim, list(sig), list(a * v), a, lam, mu, rho)

    cd = _cfg(dim)
    for d in range(dim):
        for s in (0.1, 0.7):
            h = 1e-5
            g = (q_of(s + h) - q_of(s - h)) / (2 * h)  # central difference, O(h^2)
            out = oracle.ncp(cd, q_of(s), d, g)
            v, a, sig = fields(s)
            dv = (fields(s + h)[0] - fields(s - h)[0]) / (2 * h)
            G = np.zeros((dim, dim))
            G[:, d] = dv
            np.testing.assert_allclose(out[:nsig], -_hooke(dim, lam, mu, G), atol=1e-8)
            dasig = (fields(s + h)[1] * fields(s + h)[2] - fields(s - h)[1] * fields(s - h)[2]) / (2 * h)
            for i in range(dim):
                assert abs(out[nsig + i] + dasig[_sym(dim, i, d)] / rho) < 1e-8


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("alpha", [1.0, 0.3, 0.01])
def test_eigenvalues_do_not_depend_on_alpha(dim, alpha):
    """The quasi-linear matrix of the system (F = 0, A_d = B_d) has real
    eigenvalues with largest modulus c_p = sqrt((lambda + 2 mu) / rho) for any
    alpha > 0 (Sec. 3.2), and max_eig reports it."""
    lam, mu, rho = 2.0, 1.1, 1.3
    cd = _cfg(dim)
    nsig = _nsig(dim)
    q = _state(dim, list(RNG.uniform(-1, 1, nsig)), list(alpha * RNG.uniform(-1, 1, dim)), alpha, lam, mu, rho)
    cp = math.sqrt((lam + 2 * mu) / rho)
    for d in range(dim):
        A = np.stack([oracle.ncp(cd, q, d, e) for e in np.eye(cd.m)], axis=1)
        ev = np.linalg.eigvals(A)
        assert np.max(np.abs(ev.imag)) < 1e-7
        assert abs(np.max(np.abs(ev.real)) - cp) < 1e-9
        assert abs(oracle.max_eig(cd, q, d) - cp) < 1e-15


def _side(dim, sig, w, a, lam, mu, rho):
    return _state(dim, list(sig), list(w), a, lam, mu, rho)


@pytest.mark.parametrize("dim", [2, 3])
def test_path_integral_alpha_jump(dim):
    """Equal material, alpha jumping: the momentum rows integrate the
    derivative of a quadratic, exact with three Gauss points,
    -(alpha_R sigma_R - alpha_L sigma_L)_{id} / rho; the stress rows
    integrate -E : d(w/alpha)/ds, a rational function, whose exact value
    -E : (dv (x) e_d) the rule meets within its error bound."""
    lam, mu, rho = 2.0, 1.0, 1.5
    nsig = _nsig(dim)
    cd = _cfg(dim)
    for aL, aR in ((1.0, 0.5), (0.4, 1.0), (1.0, 0.98)):
        sL, sR = RNG.uniform(-1, 1, nsig), RNG.uniform(-1, 1, nsig)
        wL, wR = RNG.uniform(-1, 1, dim), RNG.uniform(-1, 1, dim)
        qL, qR = _side(dim, sL, wL, aL, lam, mu, rho), _side(dim, sR, wR, aR, lam, mu, rho)
        for d in range(dim):
            J = oracle.path_jump(cd, d, qL, qR)
            for i in range(dim):
                k = _sym(dim, i, d)
                assert abs(J[nsig + i] + (aR * sR[k] - aL * sL[k]) / rho) < 1e-14
            G = np.zeros((dim, dim))
            G[:, d] = wR / aR - wL / aL
            exact = -_hooke(dim, lam, mu, G)
            # integrand K / alpha(s)^2 with K = -E : ((dw aL - wL da) (x) e_d)
            Gk = np.zeros((dim, dim))
            Gk[:, d] = (wR - wL) * aL - wL * (aR - aL)
            K = np.abs(_hooke(dim, lam, mu, Gk))
            da = abs(aR - aL)
            bound = GL3_ERR * K * math.factorial(7) * da ** 6 / min(aL, aR) ** 8 + 1e-14
            assert np.all(np.abs(J[:nsig] - exact) <= bound), (J[:nsig] - exact, bound)
            assert np.all(J[nsig + dim:] == 0.0)


def test_path_integral_density_and_lame_jumps():
    """rho jumping: momentum rows -alpha dsigma int ds / rho(s) against the
    closed form ln(rho_R/rho_L)/(rho_R - rho_L) within the rule's bound;
    lambda, mu jumping: the stress rows integrate a linear E(s), exact:
    -E((lam_L+lam_R)/2, (mu_L+mu_R)/2) : (dv (x) e_d)."""
    dim, nsig = 3, 6
    cd = _cfg(dim)
    sL, sR = RNG.uniform(-1, 1, nsig), RNG.uniform(-1, 1, nsig)
    w = RNG.uniform(-1, 1, dim)
    for rL, rR in ((1.0, 2.0), (2.7, 1.1)):
        qL, qR = _side(dim, sL, w, 1.0, 2.0, 1.0, rL), _side(dim, sR, w, 1.0, 2.0, 1.0, rR)
        for d in range(dim):
            J = oracle.path_jump(cd, d, qL, qR)
            integ = math.log(rR / rL) / (rR - rL)
            bound_unit = GL3_ERR * 720 * abs(rR - rL) ** 6 / min(rL, rR) ** 7
            for i in range(dim):
                k = _sym(dim, i, d)
                ds = sR[k] - sL[k]
                assert abs(J[nsig + i] + ds * integ) <= abs(ds) * bound_unit + 1e-15
    wL, wR = RNG.uniform(-1, 1, dim), RNG.uniform(-1, 1, dim)
    s = RNG.uniform(-1, 1, nsig)
    qL, qR = _side(dim, s, wL, 1.0, 1.0, 0.5, 1.3), _side(dim, s, wR, 1.0, 3.0, 1.5, 1.3)
    for d in range(dim):
        J = oracle.path_jump(cd, d, qL, qR)
        G = np.zeros((dim, dim))
        G[:, d] = wR - wL
        np.testing.assert_allclose(J[:nsig], -_hooke(dim, 2.0, 1.0, G), atol=1e-14)
        np.testing.assert_allclose(J[nsig:nsig + dim], 0.0, atol=1e-15)


def test_face_flux_splits_the_fluctuation():
    """Conservative systems: both sides receive the Rusanov flux (bitwise).
    Diffuse interface: f_lower - f_upper = J, f_lower + f_upper = -Theta dq
    on the evolved rows, and the material rows receive nothing (R20)."""
    ceu = oracle.make_cfg(2, (2, 2), [0, 0], [1, 1], 2, oracle.PDE_EULER, [1.4])
    qL, qR = np.array([1.0, 0.2, -0.1, 2.6]), np.array([1.2, 0.1, 0.3, 2.9])
    fL, fR = oracle.flux(ceu, qL, 0), oracle.flux(ceu, qR, 0)
    lo, up = oracle.face_flux(ceu, 0, qL, fL, qR, fR)
    rus = oracle.rusanov(ceu, 0, qL, fL, qR, fR)
    assert np.array_equal(lo, rus) and np.array_equal(up, rus)
    cd = _cfg(2)
    qL = _side(2, RNG.uniform(-1, 1, 3), RNG.uniform(-1, 1, 2), 1.0, 2.0, 1.0, 1.0)
    qR = _side(2, RNG.uniform(-1, 1, 3), RNG.uniform(-1, 1, 2), 0.2, 2.5, 0.8, 1.4)
    z = np.zeros(9)
    for d in range(2):
        lo, up = oracle.face_flux(cd, d, qL, z, qR, z)
        J = oracle.path_jump(cd, d, qL, qR)
        smax = max(oracle.max_eig(cd, qL, d), oracle.max_eig(cd, qR, d))
        np.testing.assert_allclose(lo - up, J, atol=1e-15)
        np.testing.assert_allclose((lo + up)[:5], -smax * (qR - qL)[:5], atol=1e-15)
        assert np.all(lo[5:] == 0.0) and np.all(up[5:] == 0.0)
        assert oracle.nevolved(cd) == 5


def test_alpha_one_runs_equal_the_conservative_scheme():
    """alpha = 1 and constant material: the non-conservative scheme (strong
    form volume term, path-conservative faces) and the conservative one
    (weak form, Rusanov) are the same discrete operator -- summation by
    parts holds exactly on Gauss-Legendre nodes -- so whole runs agree to
    rounding; the material fields stay bitwise constant."""
    cells, N = (3, 3, 3), 2
    ce = oracle.make_cfg(3, cells, [0] * 3, [1] * 3, N, oracle.PDE_ELASTICITY, [1.0, 2.0, 1.0])
    cd = oracle.make_cfg(3, cells, [0] * 3, [1] * 3, N, DI, [])
    X = oracle.node_coords(ce)
    U9 = inputs.smooth_random_state(3, X, (1, 1, 1), seed=3)
    U13 = inputs.diffuse_pack(3, [U9[..., i] for i in range(6)], [U9[..., 6 + i] for i in range(3)], 1.0, 2.0, 1.0,
                              1.0)
    Ue, te, ke, _ = oracle.run(ce, U9, 0.05)
    Ud, td, kd, _ = oracle.run(cd, U13, 0.05)
    assert (te, ke) == (td, kd) and ke >= 5
    assert np.abs(Ud[..., :9] - Ue).max() <= 1e-13 * np.abs(Ue).max()
    assert np.array_equal(Ud[..., 9:], U13[..., 9:])


def _slab_run(alpha_vac, width, nx, t_end, surface=True, interface=None):
    """Quasi-1D run (nx x 1 periodic cells on [0, 2]): a right-going P-wave
    pulse centred at x = 0.6 in a solid slab; optionally free surfaces at
    x = 0.25 and 1.25 (alpha from 1 to alpha_vac) or a material change at
    x = 1 (alpha = 1)."""
    lam, mu, rho = 2.0, 1.0, 1.0
    cp = math.sqrt((lam + 2 * mu) / rho)
    c = oracle.make_cfg(2, (nx, 1), [0, 0], [2.0, 2.0 / nx], 3, DI, [])
    X = oracle.node_coords(c)
    x = X[..., 0]
    alpha = np.ones_like(x)
    if surface:
        alpha = (inputs.smooth_step(x, 1.25, width, 1.0, alpha_vac)
                 + inputs.smooth_step(-x, -0.25, width, 1.0, alpha_vac) - 1.0)
    L, M, R = (np.full_like(x, v) for v in (lam, mu, rho))
    if interface is not None:
        L, M, R = (inputs.smooth_step(x, 1.0, width, a, b) for a, b in zip((lam, mu, rho), interface))
    f = np.exp(-((x - 0.6) / 0.08) ** 2)
    U = inputs.diffuse_pack(2, [-(lam + 2 * mu) / cp * f, -lam / cp * f, 0 * f], [alpha * f, 0 * f], alpha, L, M, R)
    Uo, t, k, _ = oracle.run(c, U, t_end)
    assert np.isfinite(Uo).all()
    return x, Uo, (lam + 2 * mu) / cp


def test_free_surface_reflects_with_flipped_stress():
    """Sec. 3.2: alpha from 1 to ~0 acts as a free surface (sigma . n = 0).
    The incident pulse (sigma_xx = -2) returns with sigma_xx = +2 and the
    velocity's sign kept (the velocity doubles at the surface); without the
    surface nothing comes back."""
    x, U, amp = _slab_run(1e-2, 0.025, 80, 0.55)
    win = (x > 0.3) & (x < 1.1)
    sxx, v = U[..., 0][win], (U[..., 3] / U[..., 5])[win]
    assert 0.85 * amp <= sxx.max() <= 1.1 * amp
    assert sxx.min() > -0.1 * amp
    assert v.max() > 0.85 * amp / 2.0 and v.min() > -0.1
    x, U, _ = _slab_run(1e-2, 0.025, 80, 0.55, surface=False)
    assert np.abs(U[..., 0][(x > 0.3) & (x < 1.1)]).max() < 1e-6


def test_material_interface_transmits_the_impedance_ratio():
    """alpha = 1, material (2, 1, 1) -> (8, 4, 2) at x = 1: the stress of
    the transmitted and reflected P-waves are 2 Z2/(Z1+Z2) and
    (Z2-Z1)/(Z1+Z2) times the incident one (Z = rho c_p), here within the
    smearing of a two-element-wide interface."""
    x, U, amp = _slab_run(1e-2, 0.02, 120, 0.45, surface=False, interface=(8.0, 4.0, 2.0))
    Z1, Z2 = 2.0, 2.0 * math.sqrt(8.0)
    s = U[..., 0]
    trans = s[(x > 1.3) & (x < 1.95)].min()
    refl = s[(x > 0.2) & (x < 0.8)].min()
    assert abs(trans / (-amp * 2 * Z2 / (Z1 + Z2)) - 1) < 0.05
    assert abs(refl / (-amp * (Z2 - Z1) / (Z1 + Z2)) - 1) < 0.15


def test_multidimensional_run_with_a_soft_surface_stays_bounded():
    """2D run through a diffuse surface (alpha 1 -> 0.3, tanh of width 0.12)
    with varying material: bounded energy-like amplitudes to t = 1 (with
    alpha <= 0.1 this discretization grows without bound in 2D and 3D)."""
    c = oracle.make_cfg(2, (8, 6), [0, 0], [1, 1], 3, DI, [])
    X = oracle.node_coords(c)
    z = X[..., 1]
    alpha = inputs.smooth_step(z, 0.5, 0.12, 1.0, 0.3)
    f = np.sin(2 * math.pi * X[..., 0]) * np.cos(2 * math.pi * z)
    U0 = inputs.diffuse_pack(2, [0.3 * f, 0.2 * f, 0.1 * f], [alpha * f, -alpha * f], alpha,
                             2.0 + 0.5 * np.sin(2 * math.pi * X[..., 0]), 1.0, 1.2)
    U, t, k, _ = oracle.run(c, U0, 1.0)
    assert t == 1.0 and np.isfinite(U).all()
    assert np.abs(U[..., :5]).max() < 3.0 * np.abs(U0[..., :5]).max()


def _pade_sub(N, z):
    """[N / N+1] Pade approximant of exp(z) (closed-form coefficients)."""
    L, M = N, N + 1
    num = sum(math.factorial(L + M - j) * math.factorial(L) / (math.factorial(L + M) * math.factorial(j)
                                                                * math.factorial(L - j)) * z ** j
              for j in range(L + 1))
    den = sum(math.factorial(L + M - j) * math.factorial(M) / (math.factorial(L + M) * math.factorial(j)
                                                                * math.factorial(M - j)) * (-z) ** j
              for j in range(M + 1))
    return num / den


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_reaction_step_is_the_subdiagonal_pade(N):
    """A spatially constant state under q_t = -kappa q: with the Picard
    iteration converged the predictor is the time-DG solution, whose end
    value the corrector reproduces, so one step multiplies u by the
    [N/N+1] Pade approximant of exp(-kappa dt)."""
    kappa, dt = 1.3, 0.4
    c = oracle.make_cfg(2, (2, 2), [0, 0], [1, 1], N, oracle.PDE_ADVECTION, [0.0, 0.0, 0.0, kappa], picard=-1)
    U = np.full((4, (N + 1) ** 2, 1), 0.7)
    U1 = oracle.step(c, U, dt)
    np.testing.assert_allclose(U1 / U, _pade_sub(N, -kappa * dt), rtol=1e-13)
    if N <= 3:  # distinguishable from the exponential itself
        assert abs(_pade_sub(N, -kappa * dt) - math.exp(-kappa * dt)) > 1e-10


def test_reaction_keeps_the_design_order():
    """u = exp(-kappa t) sin(2 pi (x - a t)) sin(2 pi (y - a t)): the error
    at t = 0.25 falls at the design order N+1 = 3 under refinement."""
    kappa, N, a = 0.8, 2, (1.0, 1.0)
    errs = []
    for k in (8, 16):
        c = oracle.make_cfg(2, (k, k), [0, 0], [1, 1], N, oracle.PDE_ADVECTION, [a[0], a[1], 0.0, kappa])
        X = oracle.node_coords(c)
        U0 = inputs.advection_sine(X, a=a)
        U, t, _, _ = oracle.run(c, U0, 0.25)
        ex = math.exp(-kappa * t) * inputs.advection_sine(X, a=a, t=t)
        errs.append(np.sqrt(np.mean((U - ex) ** 2)))
    order = math.log2(errs[0] / errs[1])
    assert order > 2.6, (errs, order)
