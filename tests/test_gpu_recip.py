"""The device reciprocal of the flux kernels (the density in the Euler flux
and wave speeds, the volume fractions of the diffuse-interface system): a
hardware approximation refined by Newton-Raphson steps.  It must stay
within one ulp of the correctly rounded 1/x, which numpy computes on the
host, over the magnitudes the solvers meet and far beyond."""
import numpy as np
import pytest

from paper_1808_03788_gb300 import aderdg as A

pytestmark = pytest.mark.gpu


def _samples(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    mag = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    x = mag * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    # powers of two and their neighbours, where the seed's table is coarsest
    p2 = 2.0 ** np.arange(int(np.log2(lo)), int(np.log2(hi)))
    edges = np.concatenate([p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), 1.5 * p2, -p2])
    return np.concatenate([x, edges])


def test_fp64_reciprocal_within_one_ulp():
    x = _samples(1e-30, 1e30, 1 << 20, 3)
    y = A.aderdg_device_recip(x, A.ADERDG_FP64)
    ref = 1.0 / x
    ulp = np.spacing(np.abs(ref))
    err = np.abs(y - ref) / ulp
    assert err.max() <= 1.0, (x[np.argmax(err)], err.max())
    assert np.mean(y == ref) > 0.9  # mostly correctly rounded


def test_fp32_reciprocal_within_one_ulp():
    x = _samples(1e-18, 1e18, 1 << 20, 4)
    xf = x.astype(np.float32)
    y = A.aderdg_device_recip(xf.astype(np.float64), A.ADERDG_MIXED_FP32)
    assert np.all(y.astype(np.float32) == y)  # a float widened
    ref = np.float32(1) / xf
    err = np.abs(y - ref.astype(np.float64)) / np.spacing(np.abs(ref)).astype(np.float64)
    assert err.max() <= 1.0, (xf[np.argmax(err)], err.max())


def test_recip_rejects_bad_arguments():
    with pytest.raises(A.AderdgError):
        A.aderdg_device_recip(np.ones(4), 7)
