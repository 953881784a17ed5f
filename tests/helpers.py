"""Shared test helpers: mesh configs, node coordinates and norms (reading 13
of the paper's unstated choices: GL-weighted L2 norms on the solution nodes)."""
import numpy as np

import oracle
from paper_1808_03788_gb300 import inputs


def node_weights(cfg):
    """|Omega_e| w_s for every node of every element, [E, n^d]."""
    n = cfg.N + 1
    _, w = oracle.gauss_legendre(n)
    ws = np.ones(1)
    for d in range(cfg.dim):
        ws = np.kron(w, ws)  # x fastest: last kron factor is x
    vol = 1.0
    for d in range(cfg.dim):
        vol *= (cfg.hi[d] - cfg.lo[d]) / cfg.cells[d]
    return np.broadcast_to(vol * ws, (oracle.n_elems(cfg), n ** cfg.dim))


def l2_abs(cfg, a, b, var=None):
    """Unnormalised L2 norm of a - b (per variable, or the one asked)."""
    W = node_weights(cfg)[..., None]
    e = np.sqrt(np.sum(W * (a - b) ** 2, axis=(0, 1)))
    return e if var is None else e[var]


def l2_rel(cfg, a, b):
    """max over variables of ||a - b|| / ||b|| (weighted L2); variables with
    ||b|| == 0 are measured absolutely."""
    W = node_weights(cfg)[..., None]
    num = np.sqrt(np.sum(W * (a - b) ** 2, axis=(0, 1)))
    den = np.sqrt(np.sum(W * b ** 2, axis=(0, 1)))
    den = np.where(den > 0, den, 1.0)
    return float(np.max(num / den))


def advection_cfg(cells=(16, 16), N=3, a=(1.0, 1.0), picard=0):
    dim = len(cells)
    return oracle.make_cfg(dim, cells, [0.0] * dim, [1.0] * dim, N, oracle.PDE_ADVECTION,
                           list(a), picard=picard)


def euler_cfg(cells=(8, 8), N=3, L=10.0, gamma=1.4, picard=0):
    dim = len(cells)
    return oracle.make_cfg(dim, cells, [0.0] * dim, [L] * dim, N, oracle.PDE_EULER, [gamma],
                           picard=picard)


def elastic_cfg(cells=(4, 4, 4), N=2, prm=(1.0, 2.0, 1.0), picard=0):
    return oracle.make_cfg(3, cells, [0.0] * 3, [1.0] * 3, N, oracle.PDE_ELASTICITY, list(prm),
                           picard=picard)


def order(e_coarse, e_fine, ratio=2.0):
    return float(np.log(e_coarse / e_fine) / np.log(ratio))
