"""Host logic of the domain decomposition (no GPU): the partition plan of
the C ABI (aderdg_dd_plan, aderdg_dd_face_elements, aderdg_dd_element_lists)
and, with two gloo processes standing in for two GPUs, the per-step
exchange of the time-averaged face traces (the paper's boundary-first
predictor and trace messages, Sec. 2.2) and the global wave-speed
reduction that makes every block take the undivided mesh's dt.  The traces
and wave speeds come from the oracle, so the test checks the plan against
the scheme's own neighbour relation."""
import itertools
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import aderdg as A
from paper_1808_03788_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PLANS = [(2, (9, 6), (2, 1)), (2, (7, 5), (3, 2)), (2, (4, 4), (4, 4)), (3, (5, 4, 3), (2, 2, 3)),
         (3, (6, 2, 2), (3, 1, 2))]


def _global_index(plan, e_local):
    c = plan["cells"]
    ix, r = e_local % c[0], e_local // c[0]
    iy, iz = r % c[1], r // c[1]
    return ix + plan["offset"][0], iy + plan["offset"][1], iz + plan["offset"][2]


@pytest.mark.parametrize("dim,cells,parts", PLANS)
def test_plan_covers_the_mesh_once_and_neighbours_are_mutual(dim, cells, parts):
    K = int(np.prod(parts))
    owner = {}
    plans = [A.aderdg_dd_plan(dim, cells, parts, k) for k in range(K)]
    for k, p in enumerate(plans):
        for e in range(p["elements"]):
            g = _global_index(p, e)
            assert g not in owner
            owner[g] = k
        for d in range(dim):
            for s in (0, 1):
                nb = p["neighbour"][d][s]
                if parts[d] == 1:
                    assert nb == -1 and p["face_chunks"][d][s] == 0
                    continue
                q = plans[nb]
                assert q["neighbour"][d][1 - s] == k            # mutual
                assert q["face_chunks"][d][1 - s] == p["face_chunks"][d][s]
                for dd in range(dim):                          # aligned in the other directions
                    if dd != d:
                        assert q["offset"][dd] == p["offset"][dd] and q["cells"][dd] == p["cells"][dd]
    full = set(itertools.product(*(range(cells[d]) if d < dim else [0] for d in range(3))))
    assert set(owner) == full
    # block sizes differ by at most one cell per direction
    for d in range(dim):
        sizes = {p["cells"][d] for p in plans}
        assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("dim,cells,parts", PLANS)
def test_element_lists_split_boundary_and_interior(dim, cells, parts):
    K = int(np.prod(parts))
    for k in range(K):
        p = A.aderdg_dd_plan(dim, cells, parts, k)
        bl, il = A.aderdg_dd_element_lists(dim, cells, parts, k)
        assert len(bl) == p["boundary_elements"]
        assert sorted(np.concatenate([bl, il]).tolist()) == list(range(p["elements"]))
        faces = set()
        for d in range(dim):
            for s in (0, 1):
                if p["face_chunks"][d][s]:
                    fe = A.aderdg_dd_face_elements(dim, cells, parts, k, d, s)
                    assert len(fe) == p["face_chunks"][d][s]
                    faces |= set(fe.tolist())
        assert faces == set(bl.tolist())  # boundary elements are exactly those on a split face


def test_plan_rejects_bad_partitions():
    with pytest.raises(A.AderdgError):
        A.aderdg_dd_plan(2, (4, 4), (5, 1), 0)   # more blocks than cells
    with pytest.raises(A.AderdgError):
        A.aderdg_dd_plan(2, (4, 4), (2, 2), 4)   # rank out of range
    with pytest.raises(A.AderdgError):
        A.aderdg_dd_plan(2, (4, 4), (0, 1), 0)


def _neighbour(g, cells, d, off):
    g = list(g)
    g[d] = (g[d] + off) % cells[d]
    return tuple(g)


def _rank_exchange(rank, world, port, dim, cells, parts, q):
    """One block per rank: send the face chunks of the boundary elements
    across every split face, receive the neighbours' into the halo, check
    each received chunk against the oracle's trace of the true neighbour
    element, and reduce the wave-speed maxima."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = 2.0
        cfg = oracle.make_cfg(dim, cells, [0.0] * dim, [L] * dim, 2, oracle.PDE_EULER, [1.4])
        X = oracle.node_coords(cfg)
        U = inputs.smooth_random_state(oracle.PDE_EULER, X, [L] * dim, seed=77)
        dt = oracle.cfl_dt(cfg, U)
        _, _, qf, ff = oracle.step(cfg, U, dt, with_parts=True)  # [E, dim, 2, nf, m]
        gidx = lambda g: g[0] + cells[0] * (g[1] + (cells[1] if dim > 1 else 1) * g[2])
        chunk = lambda ge, d, s: np.concatenate([qf[ge, d, s].ravel(), ff[ge, d, s].ravel()])
        p = A.aderdg_dd_plan(dim, cells, parts, rank)
        ok = True
        for d in range(dim):
            if parts[d] == 1:
                continue
            for s in (0, 1):  # send side s, receive into the halo of side 1 - s
                fe = A.aderdg_dd_face_elements(dim, cells, parts, rank, d, s)
                send = torch.from_numpy(np.stack([chunk(gidx(_global_index(p, e)), d, s) for e in fe]))
                recv = torch.empty_like(send)
                # the block across face s receives it on its face 1 - s; ours
                # across face 1 - s sends us its side-s chunks
                reqs = [dist.isend(send, p["neighbour"][d][s]), dist.irecv(recv, p["neighbour"][d][1 - s])]
                for r in reqs:
                    r.wait()
                # halo chunk j of face 1 - s: the neighbour element across it
                mine = A.aderdg_dd_face_elements(dim, cells, parts, rank, d, 1 - s)
                for j, e in enumerate(mine):
                    g = _neighbour(_global_index(p, e), (cells + (1,) * 3)[:3], d, 1 if (1 - s) == 1 else -1)
                    ok &= bool(np.array_equal(recv[j].numpy(), chunk(gidx(g), d, s)))
        # the global time step: max-reduce the per-direction wave speeds of the blocks
        rows = [gidx(_global_index(p, e)) for e in range(p["elements"])]
        cfg_b = oracle.make_cfg(dim, p["cells"][:dim], [0.0] * dim, [L] * dim, 2, oracle.PDE_EULER, [1.4])
        lam = torch.from_numpy(oracle.max_eigs(cfg_b, U[rows]).copy())
        dist.all_reduce(lam, op=dist.ReduceOp.MAX)
        S = 0.0
        for d in range(dim):  # the oracle's CFL formula with the reduced maxima
            S += float(lam[d]) / (L / cells[d])
        dt_blocks = oracle.alpha(cfg) / S
        q.put((rank, ok, dt_blocks == dt))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dim,cells,parts", [(2, (9, 6), (2, 1)), (2, (5, 7), (1, 2)), (3, (4, 3, 5), (1, 1, 2))])
def test_two_gloo_ranks_exchange_traces_and_reduce_dt(dim, cells, parts):
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_exchange, args=(r, 2, port, dim, cells, parts, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(180)
        assert p.exitcode == 0
    got = {r: (ok, same) for r, ok, same in (q.get(timeout=5) for _ in range(2))}
    assert got == {0: (True, True), 1: (True, True)}, got
