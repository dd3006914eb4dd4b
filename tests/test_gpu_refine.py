"""Mixed-precision iterative refinement (sie_solve with SIE_SOLVE_REFINE): the
corrections run on the complex64 product, the residuals on the FP64 one, so
the result meets the FP64 criterion (true relative residual below tol_outer)
and its RCS equals the plain FP64 solve's up to that tolerance amplified by
the conditioning (1e-3 relative is asked), and stays within 1% of Mie.  The
system product holds the nested interior solve, so its own accuracy is
tol_inner: tol_inner = 1e-9 keeps it well below tol_outer = 1e-5.
"""
import numpy as np
import pytest

from oracle import mie
from synth import icosphere

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("radius,f,eps_r,sigma", [(0.01, 3e9, 4.0, 0.0), (1e-3, 10e9, 1.0, 1e4)],
                         ids=["dielectric", "conductor"])
def test_refinement_meets_the_fp64_tolerance(lib, ctx, radius, f, eps_r, sigma):
    V, T = icosphere(2, radius, equal_volume=True)
    mesh = lib.Mesh(ctx, V, T)
    op = lib.Operator(mesh, f, eps_r, 1.0, sigma, lib.params(tol_outer=1e-5, tol_inner=1e-9))
    try:
        b = op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
        x64, it64, rr64 = op.solve(b, check=False)
        st64 = op.stats()
        xr, itr, rrr = op.solve(b, refine=True, check=False)
        str_ = op.stats()
        print("fp64", it64[0], rr64[0], st64, "refined", itr[0], rrr[0], str_)
        assert rrr[0] < 1e-5 and rr64[0] < 1e-5
        th = np.linspace(0.3, np.pi, 9)
        dirs = np.stack([np.sin(th), 0 * th, -np.cos(th)], 1)
        r64, rr = op.rcs(x64, dirs), op.rcs(xr, dirs)
        print("iters fp64", it64[0], "refined", itr[0], "rcs diff", np.abs(rr / r64 - 1).max())
        assert np.abs(rr - r64).max() <= 1e-3 * np.abs(r64).max()
        ref = mie.bistatic_rcs(th, 0.0, radius, f, eps_r, sigma)
        assert np.abs(rr / ref - 1).max() < 0.01
    finally:
        op.close()
        mesh.close()
