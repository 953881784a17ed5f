"""Tile shapes and the autotuner: every CTA-size shape of the predictor and
the corrector gives a result bitwise equal to the default shape's (the
per-element arithmetic does not depend on how elements are grouped into
CTAs); the plane-owning predictor variant and the tensor-core one agree
within the mixed tolerance (each bitwise across its own shapes); the autotuner returns valid shapes, keeps them in its cache file
and reads them back; autotuned batches equal the same solves alone."""
import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import aderdg as A
from paper_1808_03788_gb300 import inputs

pytestmark = pytest.mark.gpu

EL = (1.0, 2.0, 1.0)

# (pde, dim, cells, lo, hi, N, params, t_end): ragged element counts so
# that every shape has a partial last tile
CASES = [
    (2, 2, (7, 5), (0, 0), (10, 10), 4, (1.4,), 0.2),
    (2, 2, (5, 3), (0, 0), (10, 10), 2, (1.4,), 0.3),
    (3, 3, (3, 2, 3), (0, 0, 0), (1, 1, 1), 3, EL, 0.02),
    (1, 2, (6, 5), (0, 0), (1, 1), 6, (1.0, 1.0), 0.03),
]


def _ic(case):
    pde, dim, cells, lo, hi, N, params, _ = case
    X = oracle.node_coords(oracle.make_cfg(dim, cells, lo, hi, N, pde, params))
    if pde == 2:
        return inputs.euler_vortex(X)
    if pde == 3:
        return inputs.elastic_pulse(X, width=0.05)
    return inputs.advection_sine(X)


def _run(case, shapes, precision):
    pde, dim, cells, lo, hi, N, params, t_end = case
    with A.Solver(pde, dim, cells, lo, hi, N, params, precision=precision, shapes=shapes) as s:
        s.set_state(_ic(case))
        s.advance(t_end)
        U, t, k = s.get_state()
        info = s.info()
    return U, k, info


def _tc_applies(case, precision):
    """Predictor shapes 5-6 take the derivative contractions on the tensor
    cores on the FP32 path (they round differently from shapes 0-2); in
    FP64 they repeat shapes 0 and 1."""
    return precision == A.ADERDG_MIXED_FP32 and case[5] + 1 <= 8


def _xt_applies(case, precision):
    """Predictor shapes 3-4 are the plane-owning kernel for 2D FP32 solves
    with n^2 m <= 100 (they round differently from shapes 0-2)."""
    pde, dim, N = case[0], case[1], case[5]
    m = {1: 1, 2: dim + 2, 3: 9}[pde]
    return precision == A.ADERDG_MIXED_FP32 and dim == 2 and (N + 1) ** 2 * m <= 100


@pytest.mark.parametrize("precision", [A.ADERDG_FP64, A.ADERDG_MIXED_FP32])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "pde%d_d%d_N%d" % (c[0], c[1], c[5]))
def test_every_shape_is_bitwise_the_default(case, precision):
    """Every corrector shape, and every predictor shape of the same kernel
    layout, gives bitwise the default's result; the plane-owning predictor
    (shapes 3-4 where it applies) gives bitwise its own shape 3's result and
    stays within the mixed tolerance of the default."""
    U0, k0, info0 = _run(case, (0, 0), precision)
    assert k0 > 0
    assert info0["pred_shape"] == 0 and info0["corr_shape"] == 0
    xt = _xt_applies(case, precision)
    tc = _tc_applies(case, precision)
    U3 = _run(case, (3, 0), precision)[0] if xt else U0
    U5 = _run(case, (5, 0), precision)[0] if tc else U0
    seen = set()
    for ps in range(A.ADERDG_NUM_PRED_SHAPES):
        for cs in range(A.ADERDG_NUM_CORR_SHAPES):
            if (ps, cs) == (0, 0):
                continue
            U, k, info = _run(case, (ps, cs), precision)
            assert (info["pred_shape"], info["corr_shape"]) == (ps, cs)
            seen.add((info["pred_threads"], info["pred_epb"], info["corr_threads"], info["corr_epb"]))
            assert k == k0
            ref = U5 if (tc and ps in (5, 6)) else (U3 if (xt and ps in (3, 4)) else U0)
            np.testing.assert_array_equal(U, ref, err_msg="shapes %d/%d" % (ps, cs))
    for other, applies in ((U3, xt), (U5, tc)):
        if applies:
            num = np.sqrt(np.sum((other - U0) ** 2, axis=(0, 1)))
            den = np.maximum(np.sqrt(np.sum(U0 ** 2, axis=(0, 1))), 1e-300)
            assert float(np.max(num / den)) <= 1e-6
    if tc:
        assert not np.array_equal(U5, U0)  # the tensor-core kernel really ran
    assert len(seen) >= 2  # the shapes really differ


def test_autotune_cache_roundtrip(tmp_path):
    cache = tmp_path / "shapes.txt"
    sp = A.make_spec(2, 2, (40, 40), (0, 0), (10, 10), 4, (1.4,))
    shapes, ms = A.aderdg_autotune(sp, A.ADERDG_MIXED_FP32, tune_cache=str(cache), force=True)
    assert 0 <= shapes[0] < A.ADERDG_NUM_PRED_SHAPES and 0 <= shapes[1] < A.ADERDG_NUM_CORR_SHAPES
    assert all(t > 0 for t in ms), ms
    # the chosen shapes are the fastest up to the 2 % hysteresis
    P, Cr = ms[:A.ADERDG_NUM_PRED_SHAPES], ms[A.ADERDG_NUM_PRED_SHAPES:]
    assert P[shapes[0]] <= min(P) / 0.98 + 1e-9 and Cr[shapes[1]] <= min(Cr) / 0.98 + 1e-9
    line = cache.read_text().strip().splitlines()[-1].split()
    assert line[0].startswith("pde2_d2_N4_p1_") and (int(line[1]), int(line[2])) == tuple(shapes)
    # a second call finds the choice without timing
    again, ms2 = A.aderdg_autotune(sp, A.ADERDG_MIXED_FP32, tune_cache=str(cache))
    assert tuple(again) == tuple(shapes) and all(t == -1 for t in ms2)
    # handles created with the autotune request use it
    with A.Solver(2, 2, (12, 12), (0, 0), (10, 10), 4, (1.4,), precision=A.ADERDG_MIXED_FP32,
                  shapes="auto", tune_cache=str(cache)) as s:
        info = s.info()
    assert (info["pred_shape"], info["corr_shape"]) == tuple(shapes)


def test_autotuned_batch_equals_autotuned_solves_alone():
    """With the autotune request a batch and the same solves alone use the
    same shapes (one process-wide choice per key), so their results are
    bitwise equal; and the autotuned batch is within the mixed tolerance of
    the default-shape batch."""
    cases = CASES[:3]
    b = A.Batch([A.make_spec(*c[:7]) for c in cases], precision=A.ADERDG_MIXED_FP32, shapes="auto")
    d = A.Batch([A.make_spec(*c[:7]) for c in cases], precision=A.ADERDG_MIXED_FP32, shapes=(0, 0))
    for bb in (b, d):
        for i, c in enumerate(cases):
            bb.set_state(i, _ic(c))
        bb.advance([c[7] for c in cases])
    for i, c in enumerate(cases):
        pde, dim, cells, lo, hi, N, params, t_end = c
        with A.Solver(pde, dim, cells, lo, hi, N, params, precision=A.ADERDG_MIXED_FP32, shapes="auto") as s:
            s.set_state(_ic(c))
            s.advance(t_end)
            alone = s.get_state()[0].reshape(-1)
        got = b.get_state(i)[0]
        np.testing.assert_array_equal(got, alone)
        dflt = d.get_state(i)[0]
        assert np.linalg.norm(got - dflt) <= 1e-6 * np.linalg.norm(dflt)
    b.close()
    d.close()
