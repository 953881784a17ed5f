"""Von Neumann stability of the oracle's scheme (Sec. 3: the CFL coefficient
alpha < 1/(2N+1) 'can be obtained via a numerical von Neumann stability
analysis').  The step operator for 1D linear advection is linear and
translation invariant; its Bloch symbol G(theta) = sum_k C_k e^{-i theta k}
is assembled from the oracle's own step applied to unit vectors, and the
largest stable alpha is found by bisection.  This pins the default alpha
table (0.9 x the limit) and shows 0.9/(2N+1) is unstable for N >= 3."""
import numpy as np
import pytest

import oracle


def _gmax(N, alpha, ntheta=361):
    K = 5
    cfg = oracle.make_cfg(1, [K], [0.0], [1.0], N, oracle.PDE_ADVECTION, [1.0], alpha=alpha)
    n = N + 1
    dt = alpha / K
    C = {k: np.zeros((n, n)) for k in (-1, 0, 1)}
    for i in range(n):
        e = np.zeros((K, n, 1))
        e[0, i, 0] = 1.0
        r = oracle.step(cfg, e, dt)[:, :, 0]
        for k in C:
            C[k][:, i] = r[k % K]
    th = np.linspace(0.0, 2 * np.pi, ntheta)
    return max(np.abs(np.linalg.eigvals(sum(C[k] * np.exp(-1j * t * k) for k in C))).max() for t in th)


def _limit(N, tol=1e-3):
    lo, hi = 0.0, 1.2 / (2 * N + 1)
    for _ in range(18):
        mid = 0.5 * (lo + hi)
        if _gmax(N, mid, 181) <= 1 + tol:
            lo = mid
        else:
            hi = mid
    return lo


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_default_alpha_is_nine_tenths_of_von_neumann_limit(N):
    lim = _limit(N)
    cfg = oracle.make_cfg(1, [4], [0.0], [1.0], N, oracle.PDE_ADVECTION, [1.0])
    a = oracle.alpha(cfg)
    assert 0.88 * lim <= a <= 0.92 * lim, (N, a, lim)
    assert lim <= 1.0 / (2 * N + 1) + 1e-3  # the paper's necessary bound holds
    assert _gmax(N, a) <= 1 + 2e-4          # stable (up to a weak mode for N >= 4)
    assert _gmax(N, 1.1 * lim) > 1.05       # and the limit is sharp


@pytest.mark.parametrize("N", [3, 4])
def test_paper_bound_times_0_9_is_unstable(N):
    assert _gmax(N, 0.9 / (2 * N + 1)) > 1.05
