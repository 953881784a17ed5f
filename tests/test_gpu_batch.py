"""Batched solves (aderdg_batch_*) and the continuous-batching server
(aderdg_server_*): each solve's result must be bitwise the one it gets
alone through the single-solve handle (its arithmetic does not depend on
the mix), match the oracle within the stated tolerance, and a failing or
cancelled solve must not disturb the others."""
import time

import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import aderdg as A
from paper_1808_03788_gb300 import inputs
from helpers import l2_rel

pytestmark = pytest.mark.gpu

EL = (1.0, 2.0, 1.0)

# (pde, dim, cells, lo, hi, N, params, t_end)
MIX = [
    (2, 2, (6, 5), (0, 0), (10, 10), 2, (1.4,), 0.30),
    (2, 2, (8, 8), (0, 0), (10, 10), 4, (1.4,), 0.20),
    (2, 2, (4, 7), (0, 0), (10, 10), 3, (1.4,), 0.25),
    (2, 2, (9, 9), (0, 0), (10, 10), 4, (1.4,), 0.10),
    (3, 3, (3, 3, 2), (0, 0, 0), (1, 1, 1), 2, EL, 0.02),
    (1, 2, (5, 4), (0, 0), (1, 1), 3, (1.0, 1.0), 0.05),
]


def _ic(case, X):
    pde = case[0]
    if pde == 2:
        return inputs.euler_vortex(X)
    if pde == 3:
        return inputs.elastic_pulse(X, width=0.05)
    return inputs.advection_sine(X)


def _cfg(case):
    pde, dim, cells, lo, hi, N, params, _ = case
    return oracle.make_cfg(dim, cells, lo, hi, N, pde, params)


def _single(case, U0, precision=A.ADERDG_FP64):
    pde, dim, cells, lo, hi, N, params, t_end = case
    with A.Solver(pde, dim, cells, lo, hi, N, params, precision=precision) as s:
        s.set_state(U0)
        s.advance(t_end)
        U, t, k = s.get_state()
    return U.reshape(-1), t, k


@pytest.mark.parametrize("precision", [A.ADERDG_FP64, A.ADERDG_MIXED_FP32])
def test_batch_equals_solves_alone_and_oracle(precision):
    U0s = [_ic(c, oracle.node_coords(_cfg(c))) for c in MIX]
    b = A.Batch([A.make_spec(*c[:7]) for c in MIX], precision=precision)
    for i, U0 in enumerate(U0s):
        b.set_state(i, U0)
    b.advance([c[7] for c in MIX])
    assert b.status() == [1] * len(MIX)
    tol = 1e-11 if precision == A.ADERDG_FP64 else 1e-6
    for i, c in enumerate(MIX):
        Ub, tb, kb = b.get_state(i)
        Us, ts, ks = _single(c, U0s[i], precision)
        assert (tb, kb) == (ts, ks) and tb == c[7]
        np.testing.assert_array_equal(Ub, Us)  # bitwise: alone == in the mix
        Uo, to, ko, _ = oracle.run(_cfg(c), U0s[i], t_end=c[7])
        assert abs(kb - ko) <= (0 if precision == A.ADERDG_FP64 else 1)
        assert l2_rel(_cfg(c), Ub.reshape(Uo.shape), Uo) <= tol
    b.close()


def test_batch_permutation_invariance():
    perm = [3, 0, 5, 2, 4, 1]
    U0s = [_ic(c, oracle.node_coords(_cfg(c))) for c in MIX]
    b1 = A.Batch([A.make_spec(*c[:7]) for c in MIX])
    b2 = A.Batch([A.make_spec(*MIX[p][:7]) for p in perm])
    for i in range(len(MIX)):
        b1.set_state(i, U0s[i])
        b2.set_state(i, U0s[perm[i]])
    b1.advance([c[7] for c in MIX])
    b2.advance([MIX[p][7] for p in perm])
    for j, p in enumerate(perm):
        np.testing.assert_array_equal(b2.get_state(j)[0], b1.get_state(p)[0])


def test_batch_nonfinite_solve_is_isolated():
    U0s = [_ic(c, oracle.node_coords(_cfg(c))) for c in MIX]
    bad = U0s[1].copy()
    bad[3, 2, 0] = np.nan
    b = A.Batch([A.make_spec(*c[:7]) for c in MIX])
    for i, U0 in enumerate(U0s):
        b.set_state(i, bad if i == 1 else U0)
    rc = b.advance([c[7] for c in MIX], check=False)
    assert rc == A.ADERDG_E_NONFINITE
    st = b.status()
    assert st[1] == A.ADERDG_E_NONFINITE
    assert all(s == 1 for i, s in enumerate(st) if i != 1)
    Us, _, _ = _single(MIX[0], U0s[0])
    np.testing.assert_array_equal(b.get_state(0)[0], Us)


def _wait(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for tk in tickets:
            if tk not in out:
                r = srv.poll(tk)
                if r is not None:
                    out[tk] = r
        if time.time() - t0 > timeout:
            raise TimeoutError("server did not finish")
        time.sleep(0.002)
    return out


def test_server_results_equal_solves_alone():
    """Requests arrive while others run (continuous batching); every result
    is bitwise the single-solve result, and latencies are reported."""
    srv = A.Server(steps_per_round=4)
    cases = MIX * 2
    U0s = [_ic(c, oracle.node_coords(_cfg(c))) for c in cases]
    tickets = []
    for i, c in enumerate(cases):
        tickets.append(srv.submit(A.make_spec(*c[:7]), U0s[i], c[7]))
        if i % 3 == 2:
            time.sleep(0.01)  # later arrivals join a running mix
    res = _wait(srv, tickets)
    for tk, c, U0 in zip(tickets, cases, U0s):
        r = res[tk]
        assert r["status"] == A.ADERDG_OK and r["t"] == c[7]
        Us, ts, ks = _single(c, U0)
        assert r["steps"] == ks
        np.testing.assert_array_equal(r["u"], Us)
        assert r["latency_s"] >= r["queue_s"] >= 0.0
        srv.release(tk)
    st = srv.stats()
    assert st["queued"] == 0 and st["active"] == 0 and st["finished"] == len(cases)
    srv.close()


def test_server_failure_and_cancel_are_isolated():
    srv = A.Server(steps_per_round=2)
    c_ok, c_long = MIX[0], (2, 2, (8, 8), (0, 0), (10, 10), 3, (1.4,), 50.0)
    U0 = _ic(c_ok, oracle.node_coords(_cfg(c_ok)))
    bad = U0.copy()
    bad[0, 0, 3] = np.inf
    t_bad = srv.submit(A.make_spec(*c_ok[:7]), bad, c_ok[7])
    t_long = srv.submit(A.make_spec(*c_long[:7]), _ic(c_long, oracle.node_coords(_cfg(c_long))), c_long[7])
    t_ok = srv.submit(A.make_spec(*c_ok[:7]), U0, c_ok[7])
    time.sleep(0.05)
    srv.cancel(t_long)
    res = _wait(srv, [t_bad, t_long, t_ok])
    assert res[t_bad]["status"] == A.ADERDG_E_NONFINITE
    assert res[t_long]["status"] == A.ADERDG_E_CANCELLED
    assert res[t_ok]["status"] == A.ADERDG_OK
    np.testing.assert_array_equal(res[t_ok]["u"], _single(c_ok, U0)[0])
    with pytest.raises(A.AderdgError):
        srv.release(12345)
    srv.close()


def test_server_admission_limits():
    c = MIX[1]
    U0 = _ic(c, oracle.node_coords(_cfg(c)))
    # a budget below one request: refused at submit
    tiny = A.Server(budget_bytes=100_000)
    with pytest.raises(A.AderdgError) as ei:
        tiny.submit(A.make_spec(*c[:7]), U0, c[7])
    assert ei.value.code == A.ADERDG_E_NOMEM
    tiny.close()
    # a full queue: ADERDG_E_BUSY, and the accepted requests still finish
    srv = A.Server(max_queue=2, budget_bytes=300_000)  # one request in flight
    tks, busy = [], 0
    for _ in range(12):
        try:
            tks.append(srv.submit(A.make_spec(*c[:7]), U0, c[7]))
        except A.AderdgError as e:
            assert e.code == A.ADERDG_E_BUSY
            busy += 1
    assert busy > 0 and tks
    res = _wait(srv, tks)
    assert all(r["status"] == A.ADERDG_OK for r in res.values())
    srv.close()


@pytest.mark.parametrize("precision,tol", [(A.ADERDG_FP64, 1e-12), (A.ADERDG_MIXED_FP32, 1e-6)])
def test_batched_recipe_sampled_step_vs_oracle(precision, tol):
    """The batched workload's first 16 solves at their real sizes (meshes up
    to 256^2, N in 2..6, seeded eps and centres) in one batch: one device-CFL
    step; each solve's dt, and sampled elements of u^{n+1} against the
    oracle's step of the same elements (FP64 1e-12 of the data scale, mixed
    1e-6)."""
    rec = inputs.batched_vortex_recipe(16)
    b = A.Batch([A.make_spec(2, 2, r["cells"], (0, 0), (10, 10), r["N"], (1.4,)) for r in rec],
                precision=precision)
    cases = []
    for i, r in enumerate(rec):
        cfg = oracle.make_cfg(2, r["cells"], (0, 0), (10, 10), r["N"], 2, (1.4,))
        U0 = inputs.euler_vortex(oracle.node_coords(cfg), eps=r["eps"], center=r["center"])
        b.set_state(i, U0)
        cases.append((cfg, U0))
    b.step([1e30] * len(rec))
    rng = np.random.default_rng(11)
    for i, (cfg, U0) in enumerate(cases):
        Ug, t, k = b.get_state(i)
        assert k == 1
        dto = oracle.cfl_dt(cfg, U0)
        if precision == A.ADERDG_FP64:
            assert abs(t - dto) <= 1e-14 * dto
        else:  # wave speeds in FP32
            assert abs(t - dto) <= 1e-6 * dto
        E = oracle.n_elems(cfg)
        cx = cfg.cells[0]
        sel = np.unique(np.concatenate([[0, E - 1, cx - 1, E - cx], rng.integers(0, E, 24)]))
        Uo = oracle.step_sampled(cfg, U0, t, sel)
        Ug = Ug.reshape(U0.shape)[sel]
        scale = max(1.0, float(np.abs(Uo).max()))
        if precision == A.ADERDG_FP64:
            assert np.abs(Ug - Uo).max() <= tol * scale
        else:
            assert np.linalg.norm(Ug - Uo) <= tol * np.linalg.norm(Uo)
    b.close()


def test_server_mixes_precisions_and_guesses_per_request():
    """Requests of both precisions and different initial guesses run in one
    server at once (separate kernel groups of one engine); each result is
    bitwise the same solve alone with its precision and guess."""
    srv = A.Server(precision=A.ADERDG_FP64, steps_per_round=3)
    cases = [(MIX[0], A.ADERDG_FP64, -1), (MIX[0], A.ADERDG_MIXED_FP32, -1), (MIX[1], A.ADERDG_MIXED_FP32, 2),
             (MIX[4], -1, 2), (MIX[4], A.ADERDG_MIXED_FP32, 0), (MIX[5], A.ADERDG_MIXED_FP32, -1),
             (MIX[1], A.ADERDG_MIXED_FP32, 3), (MIX[2], A.ADERDG_FP64, 3)]
    U0s = [_ic(c, oracle.node_coords(_cfg(c))) for c, _, _ in cases]
    tickets = [srv.submit(A.make_spec(*c[:7]), U0s[i], c[7], precision=p, guess=g)
               for i, (c, p, g) in enumerate(cases)]
    res = _wait(srv, tickets)
    for tk, (c, p, g), U0 in zip(tickets, cases, U0s):
        r = res[tk]
        assert r["status"] == A.ADERDG_OK
        pde, dim, cells, lo, hi, N, params, t_end = c
        prec = A.ADERDG_FP64 if p < 0 else p
        with A.Solver(pde, dim, cells, lo, hi, N, params, precision=prec, guess=max(g, 0)) as s:
            s.set_state(U0)
            s.advance(t_end)
            Us, ts, ks = s.get_state()
        assert r["steps"] == ks and r["t"] == ts
        np.testing.assert_array_equal(r["u"], Us.reshape(-1))
        srv.release(tk)
    srv.close()


def test_server_rejects_bad_request_precision():
    srv = A.Server()
    c = MIX[0]
    with pytest.raises(A.AderdgError):
        srv.submit(A.make_spec(*c[:7]), _ic(c, oracle.node_coords(_cfg(c))), c[7], precision=7)
    srv.close()
