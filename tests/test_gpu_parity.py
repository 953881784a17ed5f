"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle
on the same seeded inputs.

Tolerances: FP64 path -- one predictor/corrector call max-abs error within
1e-12 of the data scale, full runs within 1e-11 relative L2 (the stated
FP64 target; the two sides differ only by rounding order and FMA
contraction).  Mixed path (FP32 predictor / FP64 update) -- 1e-6 relative
L2 (the stated mixed target), after one step on rough data and after full
runs."""
import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import aderdg as A
from paper_1808_03788_gb300 import inputs
from helpers import l2_rel

pytestmark = pytest.mark.gpu

GAMMA = 1.4
EL = (1.0, 2.0, 1.0)

# (pde, dim, N, cells, L, params)
CASES = (
    [(1, 2, N, (5, 3), 1.0, (0.7, -1.1)) for N in range(1, 8)]
    + [(2, 2, N, (5, 3), 2.0, (GAMMA,)) for N in range(1, 8)]
    + [(1, 3, N, (3, 2, 2), 1.0, (0.5, -0.3, 0.9)) for N in (1, 2, 3, 4)]
    + [(2, 3, N, (3, 2, 2), 2.0, (GAMMA,)) for N in (1, 2, 3, 4)]
    + [(3, 3, N, (3, 2, 2), 1.0, EL) for N in (1, 2, 3, 4)]
)


def _ids(c):
    return "pde%d-%dd-N%d" % (c[0], c[1], c[2])


def _pair(pde, dim, N, cells, L, params, precision=A.ADERDG_FP64, picard=0, alpha=0.0):
    cfg = oracle.make_cfg(dim, cells, [0.0] * dim, [L] * dim, N, pde, params, picard=picard, alpha=alpha)
    s = A.Solver(pde, dim, cells, [0.0] * dim, [L] * dim, N, params, precision=precision, picard=picard,
                 alpha=alpha)
    return cfg, s


def _state(cfg, pde, seed):
    X = oracle.node_coords(cfg)
    L = [cfg.hi[d] - cfg.lo[d] for d in range(cfg.dim)]
    U = inputs.smooth_random_state(pde, X, L, seed=seed, amp=0.2)
    # add element-wise noise so every mode of the element operators is exercised
    if pde == 2:
        noise = inputs.random_state(pde, cfg.dim, *U.shape[:2], seed=seed + 1, amp=0.05)
        return 0.5 * (U + noise)
    return U + 0.1 * inputs.random_state(pde, cfg.dim, *U.shape[:2], seed=seed + 1)


def _scale(a):
    return max(1.0, float(np.abs(a).max()))


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_predictor_outputs_match_oracle(case):
    pde, dim, N, cells, L, params = case
    cfg, s = _pair(*case)
    U = _state(cfg, pde, seed=100 + N)
    dt = oracle.cfl_dt(cfg, U)
    _, Vo, qfo, ffo = oracle.step(cfg, U, dt, with_parts=True)
    s.set_state(U)
    s.predictor(dt)
    V, qf, ff = s.predictor_outputs()
    assert np.abs(V - Vo).max() <= 1e-12 * _scale(Vo)
    assert np.abs(qf - qfo).max() <= 1e-12 * _scale(qfo)
    assert np.abs(ff - ffo).max() <= 1e-12 * _scale(ffo)


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_corrector_matches_oracle(case):
    pde, dim, N, cells, L, params = case
    cfg, s = _pair(*case)
    U = _state(cfg, pde, seed=200 + N)
    dt = oracle.cfl_dt(cfg, U)
    Uo = oracle.step(cfg, U, dt)
    s.set_state(U)
    s.predictor(dt)
    s.corrector(dt)
    Ug, t, _ = s.get_state()
    assert t == 0.0  # explicit predictor/corrector calls do not advance time
    assert np.abs(Ug - Uo).max() <= 1e-12 * _scale(Uo)
    # the device CFL step of the new state matches the oracle's
    assert abs(s.cfl_dt() - oracle.cfl_dt(cfg, Uo)) <= 1e-14 * oracle.cfl_dt(cfg, Uo)


def test_full_run_advection_config():
    """2D advection a = (1,1), 16x16, N = 3, to t = 1 (342 CFL steps)."""
    case = (1, 2, 3, (16, 16), 1.0, (1.0, 1.0))
    cfg, s = _pair(*case)
    U0 = inputs.advection_sine(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=1.0)
    s.set_state(U0)
    s.advance(1.0)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko) == (1.0, 342)
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


def test_full_run_euler_vortex():
    case = (2, 2, 4, (24, 20), 10.0, (GAMMA,))
    cfg, s = _pair(*case)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.4)
    s.set_state(U0)
    s.advance(0.4)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


def test_full_run_elasticity_pulse():
    case = (3, 3, 3, (5, 4, 4), 1.0, EL)
    cfg, s = _pair(*case)
    U0 = inputs.elastic_pulse(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.05)
    s.set_state(U0)
    s.advance(0.05)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


def test_step_by_step_equals_advance_and_clips():
    case = (2, 2, 3, (8, 8), 2.0, (GAMMA,))
    cfg, s1 = _pair(*case)
    _, s2 = _pair(*case)
    U0 = _state(cfg, 2, seed=5)
    s1.set_state(U0)
    s2.set_state(U0)
    dts = []
    while True:
        dt = s1.step(0.05, sync_dt=True)
        if dt == 0.0:
            break
        dts.append(dt)
    s2.advance(0.05)
    U1, t1, k1 = s1.get_state()
    U2, t2, k2 = s2.get_state()
    assert t1 == t2 == 0.05 and k1 == k2 == len(dts)
    np.testing.assert_array_equal(U1, U2)
    Uo, to, ko, hist = oracle.run(cfg, U0, t_end=0.05)
    np.testing.assert_allclose(dts, hist, rtol=1e-13)
    assert s1.step(0.05, sync_dt=True) == 0.0  # at t_end: no further step


def test_mass_conserved_on_gpu():
    case = (2, 2, 4, (32, 32), 10.0, (GAMMA,))
    cfg, s = _pair(*case)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    s.set_state(U0)
    M0 = s.mass()
    # different summation order than the oracle: round-off of ~sqrt(#nodes) ulp
    np.testing.assert_allclose(M0, oracle.mass(cfg, U0), rtol=1e-13)
    s.advance(10.0, max_steps=32)
    M1 = s.mass()
    np.testing.assert_allclose(M1, M0, rtol=2e-14, atol=1e-13)


def test_mass_is_deterministic():
    case = (3, 3, 2, (6, 5, 4), 1.0, EL)
    cfg, s = _pair(*case)
    s.set_state(inputs.elastic_pulse(oracle.node_coords(cfg)))
    a = s.mass()
    b = s.mass()
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("cells,N", [((200, 200), 4)])
def test_bench_workload_sampled_step(cells, N):
    """The 200 x 200, N = 4 Euler vortex as bench.py runs it (device CFL,
    aderdg_step): dt and sampled elements of u^{n+1} against the oracle."""
    case = (2, 2, N, cells, 10.0, (GAMMA,))
    cfg, s = _pair(*case)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    s.set_state(U0)
    dt = s.step(10.0, sync_dt=True)
    dto = oracle.cfl_dt(cfg, U0)
    assert abs(dt - dto) <= 1e-14 * dto
    Ug, t, k = s.get_state()
    rng = np.random.default_rng(7)
    E = oracle.n_elems(cfg)
    sel = np.unique(np.concatenate([[0, E - 1, cells[0] - 1, E - cells[0]], rng.integers(0, E, 200)]))
    Uo = oracle.step_sampled(cfg, U0, dto, sel)
    assert np.abs(Ug[sel] - Uo).max() <= 1e-12 * _scale(Uo)


def test_elasticity_bench_size_sampled_step():
    """64^3 elasticity, N = 3 (the 3D workload) in FP64: sampled elements."""
    case = (3, 3, 3, (64, 64, 64), 1.0, EL)
    cfg, s = _pair(*case)
    U0 = inputs.elastic_pulse(oracle.node_coords(cfg))
    s.set_state(U0)
    dt = s.step(1.0, sync_dt=True)
    dto = oracle.cfl_dt(cfg, U0)
    assert abs(dt - dto) <= 1e-14 * dto
    Ug, _, _ = s.get_state()
    E = oracle.n_elems(cfg)
    c = 64 // 2
    centre = c + 64 * (c + 64 * c)
    sel = np.unique(np.concatenate([[0, E - 1, centre, centre - 1, centre + 64],
                                    np.random.default_rng(3).integers(0, E, 100)]))
    Uo = oracle.step_sampled(cfg, U0, dto, sel)
    assert np.abs(Ug[sel] - Uo).max() <= 1e-12 * _scale(Uo)


def test_single_element_periodic_mesh():
    """A 1 x 1 mesh: every face is periodic with the element itself."""
    case = (2, 2, 3, (1, 1), 1.0, (GAMMA,))
    cfg, s = _pair(*case)
    U0 = _state(cfg, 2, seed=9)
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.01)
    s.set_state(U0)
    s.advance(0.01)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


def test_anisotropic_mesh_and_picard_count():
    cfg = oracle.make_cfg(2, (7, 4), [0, 0], [1.0, 3.0], 3, 2, (GAMMA,), picard=6)
    s = A.Solver(2, 2, (7, 4), [0, 0], [1.0, 3.0], 3, (GAMMA,), picard=6)
    U0 = inputs.smooth_random_state(2, oracle.node_coords(cfg), [1.0, 3.0], seed=4)
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.02)
    s.set_state(U0)
    s.advance(0.02)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko)
    assert l2_rel(cfg, Ug, Uo) <= 1e-11


def test_nonfinite_state_is_reported_and_isolated():
    case = (2, 2, 2, (4, 4), 1.0, (GAMMA,))
    cfg, bad = _pair(*case)
    _, good = _pair(*case)
    U0 = _state(cfg, 2, seed=1)
    Ub = U0.copy()
    Ub[5, 3, 0] = np.nan
    good.set_state(U0)
    bad.set_state(Ub)
    with pytest.raises(A.AderdgError) as ei:
        bad.step(1.0, sync_dt=True)
    assert ei.value.code == A.ADERDG_E_NONFINITE
    good.advance(0.01)
    Ug, t, _ = good.get_state()
    assert t == 0.01 and np.isfinite(Ug).all()


def test_constant_state_preserved_on_gpu():
    case = (3, 3, 2, (4, 3, 2), 1.0, EL)
    cfg, s = _pair(*case)
    q0 = inputs.random_state(3, 3, 1, 1, seed=3)[0, 0]
    U = np.tile(q0, (24, 27, 1))
    s.set_state(U)
    s.advance(1.0, max_steps=10)
    Ug, _, k = s.get_state()
    assert k == 10
    np.testing.assert_allclose(Ug, U, atol=1e-13)


# ---- mixed precision (FP32 predictor, FP64 update) -------------------------------

@pytest.mark.parametrize("case", [c for c in CASES if c[2] in (2, 3, 4)], ids=_ids)
def test_mixed_one_step_close_to_oracle(case):
    pde, dim, N, cells, L, params = case
    cfg, s = _pair(*case, precision=A.ADERDG_MIXED_FP32)
    U = _state(cfg, pde, seed=300 + N)
    dt = oracle.cfl_dt(cfg, U)
    Uo = oracle.step(cfg, U, dt)
    s.set_state(U)
    s.predictor(dt)
    s.corrector(dt)
    Ug, _, _ = s.get_state()
    assert l2_rel(cfg, Ug, Uo) <= 1e-6


def test_mixed_full_run_euler_vortex():
    case = (2, 2, 4, (24, 20), 10.0, (GAMMA,))
    cfg, s = _pair(*case, precision=A.ADERDG_MIXED_FP32)
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=0.4)
    s.set_state(U0)
    s.advance(0.4)
    Ug, t, k = s.get_state()
    assert t == to and abs(k - ko) <= 1
    assert l2_rel(cfg, Ug, Uo) <= 1e-6


def test_mixed_full_run_advection_config():
    """The advection configuration (16x16, N = 3, a = (1, 1)) to t = 1 on
    the FP32 path: the same 342 steps as the oracle and within the mixed
    tolerance of its FP64 result."""
    case = (1, 2, 3, (16, 16), 1.0, (1.0, 1.0))
    cfg, s = _pair(*case, precision=A.ADERDG_MIXED_FP32)
    U0 = inputs.advection_sine(oracle.node_coords(cfg))
    Uo, to, ko, _ = oracle.run(cfg, U0, t_end=1.0)
    s.set_state(U0)
    s.advance(1.0)
    Ug, t, k = s.get_state()
    assert (t, k) == (to, ko) == (1.0, 342)
    assert l2_rel(cfg, Ug, Uo) <= 1e-6


def test_mixed_and_fp64_vortex_to_the_end_time():
    """The vortex to t = 10 (a full period: the exact solution is the
    initial state again) on 40^2 elements, N = 4: the FP32 path stays within
    1e-6 relative L2 of the FP64 path over the whole run (about 3.6k steps),
    and the two L2 errors of rho against the exact solution differ by less
    than that tolerance times the norm of the exact rho (at this resolution
    the error is ~9e-7 and the FP32 rounding of 3.6k steps adds ~3e-7)."""
    from helpers import l2_abs
    cells, N = (40, 40), 4
    res = {}
    for prec in (A.ADERDG_FP64, A.ADERDG_MIXED_FP32):
        cfg, s = _pair(2, 2, N, cells, 10.0, (GAMMA,), precision=prec)
        X = oracle.node_coords(cfg)
        s.set_state(inputs.euler_vortex(X))
        s.advance(10.0)
        res[prec] = s.get_state()
    (U64, t64, k64), (Umx, tmx, kmx) = res[A.ADERDG_FP64], res[A.ADERDG_MIXED_FP32]
    assert t64 == tmx == 10.0 and k64 > 3000 and abs(k64 - kmx) <= 1
    assert l2_rel(cfg, Umx, U64) <= 1e-6
    e64 = l2_abs(cfg, U64, inputs.euler_vortex(X, t=t64))[0]
    emx = l2_abs(cfg, Umx, inputs.euler_vortex(X, t=tmx))[0]
    rho_norm = l2_abs(cfg, inputs.euler_vortex(X, t=t64), 0 * U64)[0]
    assert abs(emx - e64) <= 1e-6 * rho_norm, (e64, emx, rho_norm)
    assert e64 < 1e-5 and emx < 1e-5, (e64, emx)


def test_mixed_tracks_fp64_over_a_long_run():
    """The FP32 predictor works on perturbations about a per-element FP64
    reference, so its rounding stays far below the discretisation error:
    after 600 steps of the vortex the mixed state is within 1e-6 relative L2
    of the FP64 one, and both have the same L2 error against the exact
    solution."""
    cells, N = (48, 48), 4
    res = {}
    for prec in (A.ADERDG_FP64, A.ADERDG_MIXED_FP32):
        cfg, s = _pair(2, 2, N, cells, 10.0, (GAMMA,), precision=prec)
        X = oracle.node_coords(cfg)
        s.set_state(inputs.euler_vortex(X))
        s.advance(1e30, max_steps=600)
        res[prec] = s.get_state()
    (U64, t64, _), (Umx, tmx, _) = res[A.ADERDG_FP64], res[A.ADERDG_MIXED_FP32]
    assert l2_rel(cfg, Umx, U64) <= 1e-6
    from helpers import l2_abs
    e64 = l2_abs(cfg, U64, inputs.euler_vortex(X, t=t64))[0]
    emx = l2_abs(cfg, Umx, inputs.euler_vortex(X, t=tmx))[0]
    assert abs(emx - e64) <= 0.05 * e64, (e64, emx)


def test_mixed_mass_conservation():
    case = (2, 2, 4, (32, 32), 10.0, (GAMMA,))
    cfg, s = _pair(*case, precision=A.ADERDG_MIXED_FP32)
    s.set_state(inputs.euler_vortex(oracle.node_coords(cfg)))
    M0 = s.mass()
    s.advance(1e30, max_steps=64)
    # FP32 rounding of the reference differences across faces: ~1e-11 per 64 steps
    np.testing.assert_allclose(s.mass(), M0, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("precision,limiter", [(A.ADERDG_FP64, False), (A.ADERDG_MIXED_FP32, False),
                                               (A.ADERDG_FP64, True)])
def test_checkpoint_and_resume_is_bitwise(precision, limiter):
    """Checkpoint = (state, time) read back to the host; a fresh handle that
    resumes from it continues bitwise like the uninterrupted run (every step
    depends only on u^n and t; the step counter restarts)."""
    case = (2, 2, 3, (12, 10), 10.0, (GAMMA,))
    cfg = oracle.make_cfg(2, case[3], [0, 0], [10, 10], 3, 2, case[5])
    U0 = inputs.euler_vortex(oracle.node_coords(cfg))
    kw = dict(precision=precision, limiter=limiter)
    with A.Solver(2, 2, case[3], (0, 0), (10, 10), 3, case[5], **kw) as s:
        s.set_state(U0)
        s.advance(0.5)
        ref, t_ref, k_ref = s.get_state()
    with A.Solver(2, 2, case[3], (0, 0), (10, 10), 3, case[5], **kw) as s:
        s.set_state(U0)
        s.advance(0.5, max_steps=20)  # stop after 20 steps (a stop at a time would clip one step)
        ck, t_ck, k_ck = s.get_state()  # the checkpoint
    with A.Solver(2, 2, case[3], (0, 0), (10, 10), 3, case[5], **kw) as s:
        s.set_state(ck, t=t_ck)
        s.advance(0.5)
        got, t, k = s.get_state()
    assert k_ck == 20 and t == t_ref and k_ck + k == k_ref
    np.testing.assert_array_equal(got, ref)
