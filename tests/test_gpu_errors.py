"""Error paths of the C ABI (every failure is made on the host: bad meshes, bad
arguments, non-finite inputs, iteration caps); nothing here faults the GPU.

* Mesh checks of sie_mesh_create (Sec. II-A: RWG functions need a closed,
  consistently oriented 2-manifold with non-degenerate triangles).
* SIE_ERR_NOT_CONVERGED with the last iterate when maxit stops GMRES, and when
  the nested interior solve of Eq. (nest2) stops above tol_inner (the graph
  path and the stream path then give the same inexact product).
* Non-finite right-hand sides are refused instead of iterated.
"""
import ctypes
import os

import numpy as np
import pytest

from synth import cn_vector, icosphere

pytestmark = pytest.mark.gpu

SIE_ERR_ARG, SIE_ERR_MESH, SIE_ERR_NOT_CONVERGED = 1, 2, 5


def _mesh_code(lib, ctx, V, T):
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    h = ctypes.c_void_p()
    code = lib.lib().sie_mesh_create(ctx.h, V.ctypes.data, len(V), T.ctypes.data, len(T), ctypes.byref(h))
    if code == 0:
        lib.lib().sie_mesh_destroy(h)
    return code, lib.lib().sie_last_error().decode()


def test_mesh_errors(lib, ctx):
    V, T = icosphere(1, 0.01)
    assert _mesh_code(lib, ctx, V, T)[0] == 0
    # open: one triangle removed
    code, msg = _mesh_code(lib, ctx, V, T[1:])
    assert code == SIE_ERR_MESH, msg
    # non-manifold: a triangle repeated (its edges are shared by three or more triangles)
    code, msg = _mesh_code(lib, ctx, V, np.vstack([T, T[:1]]))
    assert code == SIE_ERR_MESH, msg
    # inconsistent orientation: one triangle flipped
    Tf = T.copy()
    Tf[0] = Tf[0, ::-1]
    code, msg = _mesh_code(lib, ctx, V, Tf)
    assert code == SIE_ERR_MESH and "orientation" in msg, msg
    # degenerate: the three vertices of one triangle made collinear
    Vd = V.copy()
    a, b, c = T[0]
    Vd[c] = 0.5 * (Vd[a] + Vd[b])
    code, msg = _mesh_code(lib, ctx, Vd, T)
    assert code == SIE_ERR_MESH and "degenerate" in msg, msg
    # index out of range
    Ti = T.copy()
    Ti[3, 1] = len(V)
    assert _mesh_code(lib, ctx, V, Ti)[0] == SIE_ERR_MESH
    # non-finite coordinate
    Vn = V.copy()
    Vn[5, 2] = np.nan
    code, msg = _mesh_code(lib, ctx, Vn, T)
    assert code == SIE_ERR_ARG and "finite" in msg, msg


@pytest.fixture(scope="module")
def small(lib, ctx):
    """Dielectric sphere, 80 triangles (eps_r 4, r 1 cm, 3 GHz)."""
    V, T = icosphere(1, 0.01, equal_volume=True)
    mesh = lib.Mesh(ctx, V, T)
    op = lib.Operator(mesh, 3e9, 4.0, 1.0, 0.0)
    yield mesh, op
    op.close()
    mesh.close()


def test_bad_arguments(lib, small):
    mesh, op = small
    L = lib.lib()
    n = mesh.ne + mesh.nt
    x = np.zeros(n, complex)
    y = np.zeros(n, complex)
    assert L.sie_matvec(op.h, lib.SIE_OP_SYS, x.ctypes.data, y.ctypes.data, 0, 0) == SIE_ERR_ARG
    assert L.sie_matvec(op.h, 99, x.ctypes.data, y.ctypes.data, 1, 0) == SIE_ERR_ARG
    d = np.array([0.0, 0.0, 1.0])
    r = np.zeros(1)
    assert L.sie_rcs(op.h, x.ctypes.data, d.ctypes.data, 0, r.ctypes.data, 0) == SIE_ERR_ARG
    assert L.sie_solve(op.h, None, x.ctypes.data, 1, None, None, 0) == SIE_ERR_ARG


def test_maxit_returns_last_iterate(lib, small):
    """maxit = 3: SIE_ERR_NOT_CONVERGED, 3 iterations, and x is the iterate whose
    residual GMRES reported (checked with an independent product)."""
    mesh, op = small
    b = op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    op.set_solver(maxit=3)
    try:
        L = lib.lib()
        x = np.zeros_like(b)
        it = np.zeros(1, np.int32)
        rr = np.zeros(1)
        code = L.sie_solve(op.h, b.ctypes.data, x.ctypes.data, 1, it.ctypes.data, rr.ctypes.data, 0)
        assert code == SIE_ERR_NOT_CONVERGED
        assert "maxit" in L.sie_last_error().decode()
        assert it[0] == 3 and rr[0] > 1e-4
        res = np.linalg.norm(b - op.matvec(lib.SIE_OP_SYS, x)) / np.linalg.norm(b)
        # the product holds a nested solve to tol_inner = 1e-6: agreement to that level
        assert abs(res - rr[0]) <= 1e-3 * rr[0] + 1e-5, (res, rr[0])
    finally:
        op.set_solver()


def test_nan_rhs_is_refused(lib, small):
    mesh, op = small
    b = op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    b[7] = np.nan
    x = np.zeros_like(b)
    code = lib.lib().sie_solve(op.h, b.ctypes.data, x.ctypes.data, 1, None, None, 0)
    assert code == SIE_ERR_ARG
    assert "finite" in lib.lib().sie_last_error().decode()


def test_inexact_nested_solve_is_reported(lib, ctx):
    """Conductive sphere (1e4 S/m, 10 GHz, near-region-only interior) with the
    nested solve capped at one iteration and tol_inner = 1e-14: the product
    is inexact on purpose.  The graph replay (device pointers) and the stream
    path (SIE_GRAPH=0) run the same single iteration, so they agree to
    rounding; host-pointer products, solves and RCS report
    SIE_ERR_NOT_CONVERGED instead of passing the inexact Z_i on."""
    import torch
    V, T = icosphere(1, 1e-3, equal_volume=True)
    mesh = lib.Mesh(ctx, V, T)
    op = lib.Operator(mesh, 10e9, 1.0, 1.0, 1e4, lib.params(inner_maxit=1, tol_inner=1e-14, maxit=30))
    try:
        n = mesh.ne + mesh.nt
        x = np.concatenate([cn_vector(mesh.ne, 5), cn_vector(mesh.nt, 6)])
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros_like(xd)
        op.matvec(lib.SIE_OP_SYS, xd, yd)  # graph path, no synchronisation, no status
        st = op.stats()
        assert st["inner_iters_max"] == 1 and st["inner_relres_max"] > 1e-14
        assert int(op.info()[16]) & 1
        y_graph = yd.cpu().numpy()
        os.environ["SIE_GRAPH"] = "0"
        try:
            y = np.zeros(n, complex)
            code = lib.lib().sie_matvec(op.h, lib.SIE_OP_SYS, x.ctypes.data, y.ctypes.data, 1, 0)
        finally:
            del os.environ["SIE_GRAPH"]
        assert code == SIE_ERR_NOT_CONVERGED
        assert "tol_inner" in lib.lib().sie_last_error().decode()
        assert np.linalg.norm(y - y_graph) <= 1e-12 * np.linalg.norm(y)
        b = op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
        xs = np.zeros_like(b)
        code = lib.lib().sie_solve(op.h, b.ctypes.data, xs.ctypes.data, 1, None, None, 0)
        assert code == SIE_ERR_NOT_CONVERGED
        d = np.array([0.0, 0.0, 1.0])
        r = np.zeros(1)
        assert lib.lib().sie_rcs(op.h, xs.ctypes.data, d.ctypes.data, 1, r.ctypes.data, 0) == SIE_ERR_NOT_CONVERGED
        assert r[0] > 0
    finally:
        op.close()
        mesh.close()
