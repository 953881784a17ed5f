"""Pins of the oracle's conserved totals M_v = sum_e |Omega_e| sum_s w_s u[e][s][v]
(the diagonal mass of Sec. 2.1 applied to the state and summed) against
totals worked out by hand: a constant on an anisotropic box, monomials
that the (N+1)-point Gauss-Legendre rule integrates exactly, the periodic
sine plus a constant, and the Euler density wave.  A wrong cell volume, a
weight taken along the wrong direction or a dropped factor fails one of
them; conservation alone (the other mass tests) would not see those."""
import math

import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import inputs


def _cfg(dim, cells, lo, hi, N, pde=oracle.PDE_ADVECTION, prm=(1.0, 1.0, 1.0)):
    return oracle.make_cfg(dim, cells, lo, hi, N, pde, list(prm))


@pytest.mark.parametrize("dim,cells,lo,hi", [
    (2, (5, 3), (0.0, -1.0), (3.0, 1.0)),           # area 6, dx = 0.6, dy = 2/3
    (3, (2, 3, 4), (-0.5, 0.0, 1.0), (0.5, 2.0, 4.0)),  # volume 6
])
def test_constant_state_gives_value_times_volume(dim, cells, lo, hi):
    N = 3
    c = 1.75
    cfg = _cfg(dim, cells, lo, hi, N)
    E = oracle.n_elems(cfg)
    U = np.full((E, (N + 1) ** dim, 1), c)
    vol = float(np.prod([hi[d] - lo[d] for d in range(dim)]))
    assert abs(oracle.mass(cfg, U)[0] - c * vol) < 1e-13 * c * vol


@pytest.mark.parametrize("N", [1, 2, 4])
def test_monomials_integrate_exactly(N):
    """x^a y^b z^c with a, b, c <= 2N+1 (the Gauss-Legendre rule's exactness)
    on an anisotropic box: the total is prod_d (hi^(k+1) - lo^(k+1))/(k+1).
    Different powers per direction catch a weight taken along the wrong
    direction; different box sides catch a wrong cell volume."""
    lo, hi = (0.0, -1.0, 0.5), (2.0, 0.5, 1.5)
    cells = (3, 2, 4)
    cfg = _cfg(3, cells, lo, hi, N)
    X = oracle.node_coords(cfg)
    kmax = 2 * N + 1
    for a, b, c in ((kmax, 0, 1), (1, kmax, 0), (0, 2, kmax), (kmax, kmax - 1, 1)):
        U = (X[..., 0] ** a * X[..., 1] ** b * X[..., 2] ** c)[..., None]
        want = 1.0
        for k, d in ((a, 0), (b, 1), (c, 2)):
            want *= (hi[d] ** (k + 1) - lo[d] ** (k + 1)) / (k + 1)
        got = oracle.mass(cfg, U)[0]
        assert abs(got - want) < 1e-12 * max(1.0, abs(want)), (a, b, c, got, want)
    # one degree past the rule's exactness is not integrated exactly
    U = (X[..., 0] ** (kmax + 1))[..., None]
    want = (hi[0] ** (kmax + 2) - lo[0] ** (kmax + 2)) / (kmax + 2) * (hi[1] - lo[1]) * (hi[2] - lo[2])
    assert abs(oracle.mass(cfg, U)[0] - want) > 1e-11 * abs(want)


def test_periodic_sine_plus_constant_gives_the_constant():
    """On [0,1]^2 with K x K cells the nodal sine sums to zero over the
    periodic grid (sums of roots of unity), so the total is the constant."""
    cfg = _cfg(2, (16, 16), (0.0, 0.0), (1.0, 1.0), 3)
    X = oracle.node_coords(cfg)
    c = 0.3
    U = inputs.advection_sine(X) + c
    assert abs(oracle.mass(cfg, U)[0] - c) < 1e-14


def test_euler_density_wave_totals():
    """rho = 1 + 0.2 sin(2 pi (x + y) / 10), v = (1, 1), p = 1 on [0, 10]^2:
    mass 100, each momentum 100, energy int p/(gamma-1) + rho |v|^2 / 2 =
    100 / 0.4 + 100 = 350."""
    cfg = oracle.make_cfg(2, (20, 16), [0.0, 0.0], [10.0, 10.0], 4, oracle.PDE_EULER, [1.4])
    U = inputs.euler_density_wave(oracle.node_coords(cfg))
    M = oracle.mass(cfg, U)
    np.testing.assert_allclose(M, [100.0, 100.0, 100.0, 350.0], rtol=1e-13, atol=0)


def test_elastic_pulse_total_velocity():
    """u = v = w = exp(-|x - x0|^2 / 0.01) on the unit cube (centred, so the
    tail beyond the box is ~e^-25): each velocity total is (pi 0.01)^(3/2)
    within the quadrature error of the resolved Gaussian; the stresses are 0."""
    cfg = oracle.make_cfg(3, (16, 16, 16), [0.0] * 3, [1.0] * 3, 3, oracle.PDE_ELASTICITY, [1.0, 2.0, 1.0])
    U = inputs.elastic_pulse(oracle.node_coords(cfg))
    M = oracle.mass(cfg, U)
    want = (math.pi * 0.01) ** 1.5
    np.testing.assert_allclose(M[6:], want, rtol=1e-6)
    np.testing.assert_array_equal(M[:6], 0.0)
