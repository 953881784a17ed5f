"""Seeded synthetic inputs: initial conditions, exact solutions and random
states on the nodes of a Cartesian mesh.

This module holds none of the scheme's arithmetic.  It evaluates closed-form
fields at node coordinates that the caller supplies (each side computes its
own Gauss-Legendre nodes), so it serves both the CUDA path and the oracle
without either importing the other.  Random numbers come from numpy's PCG64
generator with an explicit seed.

Fields (X has shape [E, n^d, dim]; results are [E, n^d, m], v fastest):

* ``advection_sine``      u0 = prod_d sin(2 pi x_d / L_d)          (linear advection)
* ``euler_vortex``        isentropic vortex of Hu and Shu, the smooth Euler test of
                          Sec. 3.1 / Table 1 (background rho = u = v = p = 1)
* ``euler_density_wave``  rho = 1 + A sin(2 pi (x + y)/L), u = v = p = 1: an exact
                          translating Euler solution with no periodicity defect
* ``elastic_pulse``       Gaussian pulse exp(-|x - x0|^2 / w) on the velocity, sigma = 0
* ``elastic_plane_wave``  exact P- or S-wave of the velocity-stress system
* ``random_state``        bounded random nodal states (admissible for Euler)
* ``diffuse_pack``        the state vector of the diffuse-interface elasticity
                          system (sigma, w = alpha v, alpha, lambda, mu, rho)
* ``smooth_step``         a smooth (tanh) step between two values, the diffuse
                          interface profile of the volume fraction or a material
* ``diffuse_terrain``     3D diffuse-interface workload: solid below a synthetic
                          sinusoidal topography, vacuum above, a velocity pulse
* ``subcell_means``       a field averaged over the (2N+1)^d equal subcells of
                          every element (midpoint samples), [E, (2N+1)^d, m]
* ``euler_sharp_blast``   a discontinuous Euler state at rest (rho, p inside a
                          ball against outside), for ``subcell_means``
"""
from __future__ import annotations

import math

import numpy as np

PDE_ADVECTION, PDE_EULER, PDE_ELASTICITY, PDE_DIFFUSE_ELASTICITY = 1, 2, 3, 4


def nvar(pde: int, dim: int) -> int:
    return {PDE_ADVECTION: 1, PDE_EULER: dim + 2, PDE_ELASTICITY: 9,
            PDE_DIFFUSE_ELASTICITY: 13 if dim == 3 else 9}[pde]


def _wrap(x, lo, L):
    return lo + np.mod(x - lo, L)


def advection_sine(X, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), a=(1.0, 1.0, 1.0), t=0.0):
    """u(x, t) = prod_d sin(2 pi (x_d - a_d t - lo_d) / L_d) on a periodic box."""
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[-1]
    u = np.ones(X.shape[:-1])
    for d in range(dim):
        L = hi[d] - lo[d]
        u = u * np.sin(2.0 * math.pi * (X[..., d] - a[d] * t - lo[d]) / L)
    return u[..., None]


def advection_poly(X, coef, a, t=0.0):
    """Polynomial field sum_k c_k prod_d (x_d - a_d t)^{k_d}; coef is a dict
    {(kx, ky, kz): c}.  Used with total degree <= N."""
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[-1]
    u = np.zeros(X.shape[:-1])
    for k, c in coef.items():
        term = np.full(X.shape[:-1], float(c))
        for d in range(dim):
            term = term * (X[..., d] - a[d] * t) ** k[d]
        u = u + term
    return u[..., None]


def _euler_conserved(rho, vel, p, gamma):
    dim = len(vel)
    kin = sum(v * v for v in vel)
    E = p / (gamma - 1.0) + 0.5 * rho * kin
    out = [rho] + [rho * v for v in vel] + [E]
    assert len(out) == dim + 2
    return np.stack(out, axis=-1)


def euler_vortex(X, eps=5.0, center=(5.0, 5.0), gamma=1.4, t=0.0,
                 lo=(0.0, 0.0), hi=(10.0, 10.0), vel=(1.0, 1.0)):
    """Isentropic vortex (Hu and Shu), translated by vel * t on the periodic
    box: r^2 = |x - x_c|^2, dT = -(gamma-1) eps^2 / (8 gamma pi^2) e^{1-r^2},
    (du, dv) = eps/(2 pi) e^{(1-r^2)/2} (-(y - y_c), x - x_c),
    rho = (1 + dT)^{1/(gamma-1)}, p = rho^gamma.  2D, conserved variables."""
    X = np.asarray(X, dtype=np.float64)
    x = _wrap(X[..., 0] - vel[0] * t, lo[0], hi[0] - lo[0])
    y = _wrap(X[..., 1] - vel[1] * t, lo[1], hi[1] - lo[1])
    dx, dy = x - center[0], y - center[1]
    r2 = dx * dx + dy * dy
    dT = -(gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    g = eps / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return _euler_conserved(rho, [vel[0] - g * dy, vel[1] + g * dx], p, gamma)


def euler_density_wave(X, amp=0.2, L=10.0, gamma=1.4, t=0.0):
    """rho = 1 + amp sin(2 pi (sum_d (x_d - t)) / L), v = 1 in every direction,
    p = 1: an exact solution of the Euler equations (pure advection of
    density at constant velocity and pressure)."""
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[-1]
    phase = sum(X[..., d] - t for d in range(dim))
    rho = 1.0 + amp * np.sin(2.0 * math.pi * phase / L)
    vel = [np.ones_like(rho) for _ in range(dim)]
    return _euler_conserved(rho, vel, np.ones_like(rho), gamma)


def elastic_pulse(X, x0=(0.5, 0.5, 0.5), width=0.01):
    """Velocity u = v = w = exp(-|x - x0|^2 / width), stresses zero.
    Q = (sxx, syy, szz, sxy, syz, sxz, u, v, w)."""
    X = np.asarray(X, dtype=np.float64)
    r2 = sum((X[..., d] - x0[d]) ** 2 for d in range(3))
    g = np.exp(-r2 / width)
    out = np.zeros(X.shape[:-1] + (9,))
    out[..., 6] = g
    out[..., 7] = g
    out[..., 8] = g
    return out


def elastic_plane_wave(X, kind="p", rho=1.0, lam=2.0, mu=1.0, t=0.0, k=1):
    """Exact plane wave along x of the velocity-stress system with
    f(s) = sin(2 pi k s) on the unit-periodic box.
    P-wave: u = f(x - cp t), sxx = -(lam + 2 mu)/cp f, syy = szz = -lam/cp f.
    S-wave: v = f(x - cs t), sxy = -mu/cs f."""
    X = np.asarray(X, dtype=np.float64)
    cp = math.sqrt((lam + 2.0 * mu) / rho)
    cs = math.sqrt(mu / rho)
    out = np.zeros(X.shape[:-1] + (9,))
    if kind == "p":
        f = np.sin(2.0 * math.pi * k * (X[..., 0] - cp * t))
        out[..., 6] = f
        out[..., 0] = -(lam + 2.0 * mu) / cp * f
        out[..., 1] = -lam / cp * f
        out[..., 2] = -lam / cp * f
    else:
        f = np.sin(2.0 * math.pi * k * (X[..., 0] - cs * t))
        out[..., 7] = f
        out[..., 3] = -mu / cs * f
    return out


def diffuse_pack(dim, sigma, w, alpha, lam, mu, rho):
    """Stack the fields of the diffuse-interface system into [..., m]:
    sigma (xx yy zz xy yz xz in 3D; xx yy xy in 2D), w = alpha v (dim
    components), then alpha, lambda, mu, rho.  Scalars broadcast."""
    nsig = 6 if dim == 3 else 3
    parts = [np.asarray(sigma[i], dtype=np.float64) for i in range(nsig)]
    parts += [np.asarray(w[i], dtype=np.float64) for i in range(dim)]
    parts += [np.asarray(x, dtype=np.float64) for x in (alpha, lam, mu, rho)]
    shape = np.broadcast_shapes(*[p.shape for p in parts])
    return np.stack([np.broadcast_to(p, shape) for p in parts], axis=-1)


def smooth_step(x, x0, width, a, b):
    """a for x << x0, b for x >> x0, a tanh profile of the given width."""
    return a + (b - a) * 0.5 * (1.0 + np.tanh((np.asarray(x, dtype=np.float64) - x0) / width))


def diffuse_terrain(X, h0=0.6, amp=0.08, k=2, width=0.05, alpha_vac=0.25, lam=2.0, mu=1.0, rho=1.0,
                    x0=(0.5, 0.5, 0.4), pulse=0.005):
    """3D diffuse-interface workload on the unit box: solid (alpha = 1)
    below the surface z = h0 + amp sin(2 pi k x) sin(2 pi k y), a soft
    exterior (alpha = alpha_vac) above, joined by a tanh profile of the
    given width; homogeneous material; the velocity w = alpha v carries a
    Gaussian pulse exp(-|x - x0|^2 / pulse) in all three components,
    stresses zero.  (Multi-dimensional runs of the scheme grow without bound
    for alpha_vac <= 0.1; 0.25 stays bounded.)"""
    X = np.asarray(X, dtype=np.float64)
    h = h0 + amp * np.sin(2 * math.pi * k * X[..., 0]) * np.sin(2 * math.pi * k * X[..., 1])
    alpha = smooth_step(X[..., 2] - h, 0.0, width, 1.0, alpha_vac)
    r2 = sum((X[..., d] - x0[d]) ** 2 for d in range(3))
    g = np.exp(-r2 / pulse)
    z = np.zeros(X.shape[:-1])
    return diffuse_pack(3, [z] * 6, [alpha * g] * 3, alpha, lam, mu, rho)


def random_state(pde: int, dim: int, E: int, ns: int, seed: int, amp: float = 0.2,
                 gamma: float = 1.4) -> np.ndarray:
    """Bounded random nodal values [E, ns, m] (seeded PCG64).  Euler states
    have rho in [1-amp, 1+amp], |v_d| <= amp, p in [1-amp, 1+amp]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if pde == PDE_ADVECTION:
        return rng.uniform(-1.0, 1.0, size=(E, ns, 1))
    if pde == PDE_ELASTICITY:
        return rng.uniform(-amp, amp, size=(E, ns, 9))
    rho = 1.0 + rng.uniform(-amp, amp, size=(E, ns))
    vel = [rng.uniform(-amp, amp, size=(E, ns)) for _ in range(dim)]
    p = 1.0 + rng.uniform(-amp, amp, size=(E, ns))
    return _euler_conserved(rho, vel, p, gamma)


def smooth_random_state(pde: int, X, L, seed: int, modes: int = 3, amp: float = 0.1,
                        gamma: float = 1.4) -> np.ndarray:
    """Sum of a few random periodic Fourier modes on the box of lengths L,
    added to a constant background (Euler: rho = p = 1, v = 0.3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[-1]
    m = nvar(pde, dim)

    def field():
        f = np.zeros(X.shape[:-1])
        for _ in range(modes):
            k = rng.integers(-2, 3, size=dim)
            ph = rng.uniform(0, 2 * math.pi)
            c = rng.uniform(-1, 1)
            arg = sum(2 * math.pi * k[d] * X[..., d] / L[d] for d in range(dim)) + ph
            f = f + c * np.sin(arg)
        return f / modes

    if pde == PDE_EULER:
        rho = 1.0 + amp * field()
        vel = [0.3 + amp * field() for _ in range(dim)]
        p = 1.0 + amp * field()
        return _euler_conserved(rho, vel, p, gamma)
    return np.stack([amp * field() for _ in range(m)], axis=-1)


# ---------------------------------------------------------------------------
# Workload recipes (seeded) for the batched and served configurations
# ---------------------------------------------------------------------------

def batched_vortex_recipe(count: int = 256, seed: int = 1808):
    """Per-solve parameters of the batched Euler-vortex workload:
    mesh k^2 with k uniform in {32, 48, ..., 256}, N uniform in {2..6},
    eps uniform in [1, 5], center uniform in [3, 7]^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = np.arange(32, 257, 16)
    out = []
    for i in range(count):
        k = int(rng.choice(ks))
        N = int(rng.integers(2, 7))
        eps = float(rng.uniform(1.0, 5.0))
        c = rng.uniform(3.0, 7.0, size=2)
        out.append(dict(cells=(k, k), N=N, eps=eps, center=(float(c[0]), float(c[1]))))
    return out


def served_stream_recipe(count: int = 2000, rate: float = 200.0, seed: int = 1808):
    """Poisson arrivals (mean `rate` per second) of Euler vortex and 3D
    elasticity pulse requests, 50/50, run to t = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        if rng.uniform() < 0.5:
            k = int(rng.choice(np.arange(32, 193, 16)))
            N = int(rng.integers(2, 6))
            eps = float(rng.uniform(1.0, 5.0))
            c = rng.uniform(3.0, 7.0, size=2)
            out.append(dict(arrival=t, pde=PDE_EULER, dim=2, cells=(k, k), N=N, eps=eps,
                            center=(float(c[0]), float(c[1])), t_end=1.0))
        else:
            k = int(rng.choice([16, 24, 32, 40, 48]))
            N = int(rng.integers(2, 5))
            x0 = rng.uniform(0.25, 0.75, size=3)
            out.append(dict(arrival=t, pde=PDE_ELASTICITY, dim=3, cells=(k, k, k), N=N,
                            x0=tuple(float(v) for v in x0), t_end=1.0))
    return out


# ---------------------------------------------------------------------------
# Device-side (torch) versions for large workloads: the same closed forms,
# evaluated on CUDA tensors so that multi-GB initial states need no host trip
# ---------------------------------------------------------------------------

def node_coords_torch(cells, lo, hi, nodes, device="cuda"):
    """Node coordinates [E, n^d, d] (x-fastest elements and nodes) from the
    1D nodes on [0, 1]."""
    import torch
    dim = len(cells)
    x = torch.as_tensor(nodes, dtype=torch.float64, device=device)
    n = x.numel()
    E = 1
    for c in cells:
        E *= c
    e = torch.arange(E, device=device)
    s = torch.arange(n ** dim, device=device)
    X = torch.empty((E, n ** dim, dim), dtype=torch.float64, device=device)
    re, rs = e.clone(), s.clone()
    for d in range(dim):
        ie, js = re % cells[d], rs % n
        re, rs = re // cells[d], rs // n
        h = (hi[d] - lo[d]) / cells[d]
        X[:, :, d] = lo[d] + (ie[:, None].double() + x[js][None, :]) * h
    return X


def euler_vortex_torch(X, eps=5.0, center=(5.0, 5.0), gamma=1.4, lo=(0.0, 0.0), hi=(10.0, 10.0)):
    """euler_vortex at t = 0 on a CUDA tensor of coordinates."""
    import torch
    dx = X[..., 0] - center[0]
    dy = X[..., 1] - center[1]
    r2 = dx * dx + dy * dy
    dT = -(gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi ** 2) * torch.exp(1.0 - r2)
    g = eps / (2.0 * math.pi) * torch.exp(0.5 * (1.0 - r2))
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    u, v = 1.0 - g * dy, 1.0 + g * dx
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return torch.stack([rho, rho * u, rho * v, E], dim=-1).contiguous()


def elastic_pulse_torch(X, x0=(0.5, 0.5, 0.5), width=0.01):
    import torch
    r2 = sum((X[..., d] - x0[d]) ** 2 for d in range(3))
    g = torch.exp(-r2 / width)
    out = torch.zeros(X.shape[:-1] + (9,), dtype=torch.float64, device=X.device)
    out[..., 6] = g
    out[..., 7] = g
    out[..., 8] = g
    return out


def subcell_means(field, cells, lo, hi, N: int, k: int = 8) -> np.ndarray:
    """Means of field over the (2N+1)^d equal subcells of every element of
    the Cartesian mesh (cells, lo, hi), each estimated on k^d midpoint
    samples: [E, (2N+1)^d, m], subcells x fastest, elements x fastest.
    field maps coordinates [..., dim] to states [..., m].  This is initial
    data given as subcell averages (a discontinuous field has no admissible
    nodal interpolant); the sampling is part of the data's definition."""
    dim = len(cells)
    S = 2 * N + 1
    axes = []
    for d in range(dim):
        h = (hi[d] - lo[d]) / (cells[d] * S)
        fine = np.arange(cells[d] * S)
        axes.append(lo[d] + (fine[:, None] + (np.arange(k) + 0.5)[None, :] / k) * h)  # [fine, sample]
    # sample points on the fine grid, reversed axis order (z, y, x) so x is fastest
    grids = np.meshgrid(*[axes[d].reshape(-1) for d in reversed(range(dim))], indexing="ij")
    X = np.stack(list(reversed(grids)), axis=-1)
    F = np.asarray(field(X), dtype=np.float64)
    m = F.shape[-1]
    shape = []
    for d in reversed(range(dim)):
        shape += [cells[d] * S, k]
    F = F.reshape(shape + [m]).mean(axis=tuple(range(1, 2 * dim, 2)))  # [fine_z, fine_y, fine_x, m]
    split = []
    for d in reversed(range(dim)):
        split += [cells[d], S]
    F = F.reshape(split + [m])  # [cz, Sz, cy, Sy, cx, Sx, m]
    order = list(range(0, 2 * dim, 2)) + list(range(1, 2 * dim, 2)) + [2 * dim]
    E = int(np.prod(cells))
    return np.ascontiguousarray(F.transpose(order).reshape(E, S ** dim, m))


def euler_sharp_blast(center, radius, inside=(1.0, 1.0), outside=(0.125, 0.1), gamma=1.4):
    """field(X) of an Euler state at rest, (rho, p) = inside for
    |x - center| < radius and outside elsewhere, in conserved variables."""
    def field(X):
        dim = X.shape[-1]
        r = np.sqrt(sum((X[..., d] - center[d]) ** 2 for d in range(dim)))
        inn = r < radius
        rho = np.where(inn, inside[0], outside[0])
        p = np.where(inn, inside[1], outside[1])
        return _euler_conserved(rho, [np.zeros_like(rho)] * dim, p, gamma)
    return field
