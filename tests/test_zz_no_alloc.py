"""The step entry point that allocates nothing (aderdg_step_noalloc), for
callers that cannot call cudaMalloc: frameworks whose device memory must
all come from their own allocator, code that cannot take cudaMalloc's
implicit device synchronisation, and hosts that forbid allocation after
start-up.  Called through the C ABI on caller-owned device buffers, it must
give the same state as the handle path (aderdg_predictor + aderdg_corrector
with the same dt; the same kernels and shapes, so bit for bit), on two
calls in a row -- the second reusing the fixed scratch the first one left
behind -- and must refuse meshes whose scratch exceeds its fixed size and
meshes or parameters that aderdg_create refuses.

This file is collected last so that a stop at its first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
from paper_1808_03788_gb300 import aderdg as A
from paper_1808_03788_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    (A.ADERDG_PDE_EULER, 2, (20, 16), 4, (0.0, 0.0), (10.0, 10.0), (1.4,), A.ADERDG_FP64),
    (A.ADERDG_PDE_ELASTICITY, 3, (6, 5, 4), 3, (0.0,) * 3, (1.0,) * 3, (1.0, 2.0, 1.0), A.ADERDG_FP64),
    (A.ADERDG_PDE_EULER, 2, (20, 16), 4, (0.0, 0.0), (10.0, 10.0), (1.4,), A.ADERDG_MIXED_FP32),
    (A.ADERDG_PDE_DIFFUSE_ELASTICITY, 3, (5, 4, 4), 3, (0.0,) * 3, (1.0,) * 3, (), A.ADERDG_MIXED_FP32),
]


def _ic(pde, X):
    if pde == A.ADERDG_PDE_DIFFUSE_ELASTICITY:
        return inputs.diffuse_terrain(X, width=0.1)
    return inputs.euler_vortex(X) if pde == A.ADERDG_PDE_EULER else inputs.elastic_pulse(X)


@pytest.mark.parametrize("case", CASES, ids=["euler2d-fp64", "elastic3d-fp64", "euler2d-mixed", "diffuse3d-mixed"])
def test_noalloc_step_matches_handle_path_twice(case):
    import torch

    pde, dim, cells, N, lo, hi, params, prec = case
    cfg = oracle.make_cfg(dim, cells, lo, hi, N, pde, params)
    U0 = _ic(pde, oracle.node_coords(cfg))
    dt1 = oracle.cfl_dt(cfg, U0)
    dt2 = 0.7 * dt1

    # existing entry points on a handle: two steps with explicit dt
    s = A.Solver(pde, dim, cells, lo, hi, N, params, precision=prec)
    s.set_state(U0)
    s.predictor(dt1)
    s.corrector(dt1)
    U1, _, _ = s.get_state()
    s.predictor(dt2)
    s.corrector(dt2)
    U2, _, _ = s.get_state()
    s.close()

    # the allocation-free entry point on caller-owned device buffers
    u_in = torch.tensor(U0, dtype=torch.float64, device="cuda")
    u_mid = torch.empty_like(u_in)
    u_out = torch.empty_like(u_in)
    stream = torch.cuda.current_stream().cuda_stream
    A.aderdg_step_noalloc(pde, dim, cells, lo, hi, N, params, u_in, u_mid, dt1, precision=prec, stream=stream)
    A.aderdg_step_noalloc(pde, dim, cells, lo, hi, N, params, u_mid, u_out, dt2, precision=prec, stream=stream)
    torch.cuda.synchronize()
    V1 = u_mid.cpu().numpy()
    V2 = u_out.cpu().numpy()
    # the same kernels, shapes and operands as the handle path: bit for bit
    np.testing.assert_array_equal(V1, U1)
    np.testing.assert_array_equal(V2, U2)
    # the input buffer is left untouched
    np.testing.assert_array_equal(u_in.cpu().numpy(), U0)


def test_noalloc_rejects_meshes_beyond_the_scratch():
    import torch

    cells, N = (400, 400), 4  # ~390 MB of scratch needed
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(A.AderdgError) as ei:
        A.aderdg_step_noalloc(A.ADERDG_PDE_EULER, 2, cells, (0, 0), (1, 1), N, (1.4,), u, u, 1e-3)
    assert ei.value.code == A.ADERDG_E_INVAL
    assert "too large for the static scratch" in str(ei.value)
    assert str(A.ADERDG_NOALLOC_SCRATCH_BYTES) in str(ei.value)


@pytest.mark.parametrize("cells", [
    (7, 0x6DB6DB6DB6DB6DB7),   # the int64 product wraps to 1
    (1 << 31, 1),              # one direction beyond 2^30
    (1 << 16, 1 << 16),        # E = 2^32 > 2^31
    (0, 4),
])
def test_noalloc_rejects_the_mesh_limits_of_create(cells):
    import torch

    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(A.AderdgError) as ei:
        A.aderdg_step_noalloc(A.ADERDG_PDE_EULER, 2, cells, (0, 0), (1, 1), 2, (1.4,), u, u, 1e-3)
    assert ei.value.code == A.ADERDG_E_INVAL
    assert "scratch" not in str(ei.value)  # refused before any scratch size is formed


@pytest.mark.parametrize("pde,dim,params", [
    (A.ADERDG_PDE_EULER, 2, (1.0,)),               # gamma must exceed 1
    (A.ADERDG_PDE_ELASTICITY, 3, (1.0, 2.0, 0.0)),  # mu must be positive
    (A.ADERDG_PDE_ADVECTION, 2, (1.0, 1.0, 0.0, -0.5)),  # kappa must be >= 0
])
def test_noalloc_rejects_the_parameters_create_rejects(pde, dim, params):
    import torch

    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    cells = (4,) * dim
    with pytest.raises(A.AderdgError) as ei:
        A.aderdg_step_noalloc(pde, dim, cells, (0,) * dim, (1,) * dim, 2, params, u, u, 1e-3)
    assert ei.value.code == A.ADERDG_E_INVAL
    with pytest.raises(A.AderdgError) as ec:
        A.Solver(pde, dim, cells, (0,) * dim, (1,) * dim, 2, params)
    assert ec.value.code == A.ADERDG_E_INVAL
