"""Pins of the oracle's 1D basis (Sec. 2.1 nodal basis, eq. D_kl) against
numpy's Gauss-Legendre rule, numpy polynomial algebra and closed-form
identities.  None of these re-types the oracle's formulas."""
import numpy as np
import numpy.polynomial.polynomial as P
import pytest

import oracle

NS = list(range(1, 11))


@pytest.mark.parametrize("n", NS)
def test_gl_matches_numpy_leggauss(n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (xr + 1.0), rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, 0.5 * wr, rtol=0, atol=2e-15)


@pytest.mark.parametrize("n", NS)
def test_gl_exactness_degree(n):
    x, w = oracle.gauss_legendre(n)
    assert abs(w.sum() - 1.0) < 1e-14
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14
    # degree 2n is not integrated exactly: the rule is Gauss, not better
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-13


def _numpy_lagrange_coeffs(nodes):
    """Monomial coefficients of each Lagrange polynomial via numpy.polyfit."""
    n = len(nodes)
    return [P.polyfit(nodes, np.eye(n)[k], n - 1) for k in range(n)]


@pytest.mark.parametrize("n", range(1, 9))
def test_dhat_matches_numpy_polyder(n):
    op = oracle.operators(n)
    coeffs = _numpy_lagrange_coeffs(op["x"])
    ref = np.array([[P.polyval(op["x"][j], P.polyder(coeffs[k])) for k in range(n)]
                    for j in range(n)])
    np.testing.assert_allclose(op["Dhat"], ref, atol=1e-8 * max(1.0, abs(ref).max()))


@pytest.mark.parametrize("n", range(1, 11))
def test_dhat_differentiates_polynomials_and_is_nilpotent(n):
    op = oracle.operators(n)
    D, x = op["Dhat"], op["x"]
    scale = max(1.0, abs(D).max())
    np.testing.assert_allclose(D @ np.ones(n), 0.0, atol=1e-13 * scale)
    for k in range(1, n):
        np.testing.assert_allclose(D @ x ** k, k * x ** (k - 1), atol=1e-12 * scale ** 1)
    # D^n annihilates every polynomial of degree < n (the nodal space)
    Dn = np.linalg.matrix_power(D, n)
    assert abs(Dn).max() < 1e-9 * scale ** n


@pytest.mark.parametrize("n", range(1, 11))
def test_lagrange_interpolation_property(n):
    x, _ = oracle.gauss_legendre(n)
    for j in range(n):
        np.testing.assert_allclose(oracle.lagrange_eval(x, x[j]), np.eye(n)[j], atol=1e-14)
    for xi in (0.0, 0.123, 0.77, 1.0):
        assert abs(oracle.lagrange_eval(x, xi).sum() - 1.0) < 1e-13
        assert abs(oracle.lagrange_deriv(x, xi).sum()) < 1e-10


@pytest.mark.parametrize("n", range(1, 11))
def test_stiffness_summation_by_parts(n):
    """Kxi[k,l] = int phi_k' phi_l: Kxi + Kxi^T = F1 F1^T - F0 F0^T
    (integration by parts), column sums vanish (sum_k phi_k = 1), and the
    GL nodal form w_l Dhat[l,k] agrees (quadrature exact at degree 2N-1)."""
    op = oracle.operators(n)
    K, F0, F1 = op["Kxi"], op["F0"], op["F1"]
    scale = max(1.0, abs(K).max())
    np.testing.assert_allclose(K + K.T, np.outer(F1, F1) - np.outer(F0, F0), atol=1e-12 * scale)
    np.testing.assert_allclose(np.ones(n) @ K, 0.0, atol=1e-12 * scale)
    np.testing.assert_allclose(K @ np.ones(n), F1 - F0, atol=1e-12 * scale)
    np.testing.assert_allclose(K, (op["w"][:, None] * op["Dhat"]).T, atol=1e-12 * scale)


@pytest.mark.parametrize("n", range(1, 11))
def test_time_matrix_identities(n):
    """K1 = F1 F1^T - Kxi: K1 1 = F0 (so the predictor's constant guess is
    consistent), K1 invertible, and solving K1 q = W 1 integrates a constant
    in time exactly: q = tau at the nodes (degree 1 <= N)."""
    op = oracle.operators(n)
    K1, F0, w, x = op["K1"], op["F0"], op["w"], op["x"]
    np.testing.assert_allclose(K1 @ np.ones(n), F0, atol=1e-12 * max(1, abs(K1).max()))
    assert np.linalg.cond(K1) < 1e8
    if n >= 2:
        q = np.linalg.solve(K1, w)
        np.testing.assert_allclose(q, x, atol=1e-12)
    np.testing.assert_allclose(F0.sum(), 1.0, atol=1e-13)
    if n >= 2:
        np.testing.assert_allclose(op["F1"] @ x, 1.0, atol=1e-13)
        np.testing.assert_allclose(F0 @ x, 0.0, atol=1e-13)


def test_time_dg_matches_numpy_exponential():
    """The time part of eq. pde.st2 for the scalar ODE q' = z q is a DG-in-
    time scheme whose value at tau = 1 matches exp(z) with local error
    O(z^{2n}) (superconvergence of DG in time with exact quadrature):
    solve (K1 - z W) q = F0, extrapolate with F1, compare with exp(z)."""
    zpair = {1: 0.1, 2: 0.1, 3: 0.1, 4: 0.4, 5: 0.8, 6: 1.6}
    for n, z0 in zpair.items():
        op = oracle.operators(n)
        errs = []
        for z in (z0, z0 / 2):
            q = np.linalg.solve(op["K1"] - z * np.diag(op["w"]), op["F0"])
            errs.append(abs(op["F1"] @ q - np.exp(z)))
        order = np.log(errs[0] / errs[1]) / np.log(2.0)
        assert order > 2 * n - 0.5, (n, errs, order)
