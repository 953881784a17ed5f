"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every function include/aderdg.h declares, its host
basis agrees with numpy's Gauss-Legendre rule, and argument validation
rejects bad input before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1808_03788_gb300 import aderdg as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "aderdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aderdg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    L = A.load()
    names = _declared()
    assert "aderdg_create" in names and "aderdg_step" in names and len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding marshals all of them
    assert set(names) <= set(A._SIGS), set(names) - set(A._SIGS)


def test_library_is_built_for_sm_103a():
    from paper_1808_03788_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


@pytest.mark.parametrize("N", range(1, 10))
def test_host_gl_nodes_match_numpy(N):
    x, w = A.aderdg_gl_nodes(N)
    xr, wr = np.polynomial.legendre.leggauss(N + 1)
    np.testing.assert_allclose(x, 0.5 * (xr + 1), atol=2e-15)
    np.testing.assert_allclose(w, 0.5 * wr, atol=2e-15)


def test_default_alpha_table():
    import oracle
    for N in range(1, 10):
        cfg = oracle.make_cfg(2, [2, 2], [0, 0], [1, 1], N, oracle.PDE_ADVECTION, [1, 1])
        assert A.aderdg_default_alpha(N) == oracle.alpha(cfg)
        assert A.aderdg_default_alpha(N) < 1.0 / (2 * N + 1)


def _create(**kw):
    L = A.load()
    mesh = A.aderdg_mesh_t()
    mesh.dim = kw.get("dim", 2)
    for d in range(3):
        mesh.cells[d] = kw.get("cells", (4, 4, 4))[d]
        mesh.lo[d] = 0.0
        mesh.hi[d] = kw.get("hi", 1.0)
    p = A.aderdg_pde_t()
    p.kind = kw.get("kind", A.ADERDG_PDE_EULER)
    p.p[0] = kw.get("gamma", 1.4)
    p.p[3] = kw.get("kappa", 0.0)
    cfg = A.aderdg_config_t()
    cfg.precision = kw.get("precision", 0)
    h = A._H()
    rc = L.aderdg_create(C.byref(mesh), kw.get("N", 3), kw.get("nvar", 4), C.byref(p), C.byref(cfg), C.byref(h))
    return rc, h, L.aderdg_last_error().decode()


@pytest.mark.parametrize("kw,code", [
    (dict(dim=4), A.ADERDG_E_INVAL),
    (dict(nvar=5), A.ADERDG_E_INVAL),
    (dict(kind=7), A.ADERDG_E_INVAL),
    (dict(N=0), A.ADERDG_E_INVAL),
    (dict(N=8), A.ADERDG_E_UNSUPPORTED),
    (dict(cells=(0, 4, 4)), A.ADERDG_E_INVAL),
    (dict(hi=-1.0), A.ADERDG_E_INVAL),
    (dict(gamma=1.0), A.ADERDG_E_INVAL),
    (dict(precision=9), A.ADERDG_E_INVAL),
    (dict(kind=A.ADERDG_PDE_ELASTICITY, dim=2, nvar=9), A.ADERDG_E_UNSUPPORTED),
    (dict(kind=A.ADERDG_PDE_DIFFUSE_ELASTICITY, dim=2, nvar=13), A.ADERDG_E_INVAL),
    (dict(kind=A.ADERDG_PDE_DIFFUSE_ELASTICITY, dim=3, nvar=9), A.ADERDG_E_INVAL),
    (dict(kind=A.ADERDG_PDE_DIFFUSE_ELASTICITY, dim=2, nvar=9, N=1), A.ADERDG_E_UNSUPPORTED),
    (dict(kind=A.ADERDG_PDE_ADVECTION, nvar=1, gamma=1.0, kappa=-0.5), A.ADERDG_E_INVAL),
])
def test_create_rejects_bad_arguments(kw, code):
    rc, h, msg = _create(**kw)
    assert rc == code, (rc, msg)
    assert not h.value
    assert msg


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks the no-GPU refusal")
def test_no_cpu_fallback_without_gpu():
    rc, h, msg = _create()
    assert rc == A.ADERDG_E_CUDA
    assert "no CUDA device" in msg
    with pytest.raises(A.AderdgError):
        A.Solver(A.ADERDG_PDE_EULER, 2, (4, 4), (0, 0), (1, 1), 3, [1.4], torch_alloc=False)


_STRUCTS = ["aderdg_mesh_t", "aderdg_pde_t", "aderdg_alloc_t", "aderdg_config_t", "aderdg_info_t",
            "aderdg_solve_spec_t", "aderdg_server_config_t", "aderdg_request_t", "aderdg_result_t"]


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Size and field offsets of every ABI struct as the C compiler lays it
    out from include/aderdg.h == the ctypes mirror of the binding."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "aderdg.h"', 'int main(void) {']
    for name in _STRUCTS:
        st = getattr(A, name)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in st._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name in _STRUCTS:
        st = getattr(A, name)
        assert got[(name, "size")] == C.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)


def test_tile_shape_requests_are_validated():
    """A shape index outside 0..ADERDG_NUM_PRED_SHAPES-1 (other than the
    autotune request) is rejected before any device work."""
    cfg = A.aderdg_config_t()
    cfg.precision = A.ADERDG_FP64
    cfg.pred_shape = A.ADERDG_NUM_PRED_SHAPES
    sp = A.make_spec(A.ADERDG_PDE_EULER, 2, (4, 4), (0, 0), (1, 1), 2, (1.4,))
    h = A._H()
    rc = A.load().aderdg_batch_create(C.byref(sp), 1, C.byref(cfg), C.byref(h))
    assert rc == A.ADERDG_E_INVAL
    assert b"tile shape" in A.load().aderdg_last_error()


def test_instance_list_covers_the_documented_orders():
    """The build compiles 2D advection/Euler for N = 1..7, 3D advection,
    Euler and elasticity for N = 1..4 and the diffuse-interface system for
    N = 2..4 (2D) and 2, 3 (3D), each in double and float."""
    from paper_1808_03788_gb300 import build
    inst = build.instances()
    keys = {(name.split("_")[1], d, n, t) for name, _, d, n, t in inst}
    want = {(tag + "%dd" % d, d, n, t) for tag, d, ns in [("advection", 2, range(1, 8)), ("euler", 2, range(1, 8)),
                                                           ("advection", 3, range(1, 5)), ("euler", 3, range(1, 5)),
                                                           ("elastic", 3, range(1, 5)), ("diffuse", 2, range(2, 5)),
                                                           ("diffuse", 3, range(2, 4))]
            for n in ns for t in ("double", "float")}
    assert keys == want
