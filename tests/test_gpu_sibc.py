"""Surface impedance boundary condition (interior_model = SIE_SIBC), the
high-conductivity comparator of the paper's GIBC: Z' = (eta_i / eta0) G^-1 I_x
with the RWG Gram matrix, solved on the GPU by the nested FGMRES (inside the
system-product graph).  Against the oracle's SIBC (dense Gram solve) and its
AIM form of Eq. (sys); the solve's RCS against the Mie series and against the
GIBC solve of the same copper sphere.

Tolerances: Z' and the system product share their definitions with the
oracle; the Gram solve runs to tol_inner 1e-13, so 1e-10.  RCS within 1% of
Mie (the paper's check) and within 0.5% of the GIBC solution (the SIBC is
the GIBC's limit for skin depths far below the radius).
"""
import numpy as np
import pytest

from oracle import aim, mie, system
from oracle.rwg import Mesh
from synth import cn_vector, icosphere

pytestmark = pytest.mark.gpu

F, SIGMA, R = 10e9, 5.8e7, 1e-3


@pytest.fixture(scope="module")
def sibc(lib, ctx):
    V, T = icosphere(2, R, equal_volume=True)
    m = Mesh(V, T)
    gm = lib.Mesh(ctx, V, T)
    op = lib.Operator(gm, F, 1.0, 1.0, SIGMA, lib.params(interior_model=lib.SIE_SIBC, tol_inner=1e-13))
    S = system.AimGIBC(m, F, 1.0, SIGMA, aim.grid_params(m, M=2), interior="sibc")
    yield m, gm, op, S
    op.close()
    gm.close()


def test_sibc_impedance(lib, sibc):
    m, gm, op, S = sibc
    x = cn_vector(m.ne, 201)
    y = op.matvec(lib.SIE_OP_ZI, x)
    ref = S.Z(x)
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)


def test_sibc_system_product(lib, sibc):
    m, gm, op, S = sibc
    H, rho = cn_vector(m.ne, 202), cn_vector(m.nt, 203)
    y = op.matvec(lib.SIE_OP_SYS, np.concatenate([H, rho]))
    r1, r2 = S.apply(H, rho)
    assert np.linalg.norm(y[:m.ne] - r1) <= 1e-10 * np.linalg.norm(r1)
    assert np.linalg.norm(y[m.ne:] - r2) <= 1e-13 * np.linalg.norm(r2)


def test_sibc_solve_rcs(lib, ctx, sibc):
    m, gm, op, S = sibc
    b = op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    x, it, rr = op.solve(b)
    th = np.linspace(0.3, np.pi, 7)
    dirs = np.stack([np.sin(th), 0 * th, -np.cos(th)], 1)
    rcs = op.rcs(x, dirs)
    ref = mie.bistatic_rcs(th, 0.0, R, F, 1.0, SIGMA)
    assert np.abs(rcs / ref - 1).max() < 0.01
    gibc = lib.Operator(gm, F, 1.0, 1.0, SIGMA)
    try:
        xg, _, _ = gibc.solve(b)
        rg = gibc.rcs(xg, dirs)
    finally:
        gibc.close()
    print("SIBC vs GIBC rcs", np.abs(rcs / rg - 1).max(), "vs Mie", np.abs(rcs / ref - 1).max())
    assert np.abs(rcs / rg - 1).max() < 0.005


def test_sibc_has_no_interior_operators(lib, sibc):
    m, gm, op, S = sibc
    with pytest.raises(lib.SieError) as e:
        op.matvec(lib.SIE_OP_LI, cn_vector(m.ne, 1))
    assert e.value.code == 7
