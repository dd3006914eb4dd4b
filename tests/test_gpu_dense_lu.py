"""The GPU dense LU behind the constraint preconditioners (complex64 blocked LU
with partial pivoting, triangular solves by dependency-ordered blocks), through
sie_dense_solve, against numpy's LAPACK solve.

Tolerance: A and b are rounded to complex64 and the factorisation runs in
FP32, so the relative error is a few units of 6e-8 times the condition number
(the matrices here have condition numbers below 1e3): 2e-4.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), \
        rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("inverse", [False, True], ids=["triangular", "inverse"])
@pytest.mark.parametrize("n", [1, 63, 64, 65, 300, 1031])
def test_dense_solve_matches_lapack(lib, n, inverse):
    A, b = _rand(n, n)
    A = A + 4.0 * np.sqrt(n) * np.eye(n)  # well conditioned
    x = lib.dense_solve(A, b, inverse=inverse)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 2e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("inverse", [False, True], ids=["triangular", "inverse"])
def test_dense_solve_needs_pivoting(lib, inverse):
    """Zero diagonal (a cyclic shift plus a small perturbation): without row
    exchanges the first pivot would be tiny."""
    n = 200
    rng = np.random.default_rng(5)
    A = np.roll(np.eye(n), 1, axis=1) * (2.0 + rng.random(n))[:, None] + 1e-3 * rng.standard_normal((n, n))
    np.fill_diagonal(A, 0.0)
    A = A.astype(complex)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = lib.dense_solve(A, b, inverse=inverse)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 2e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("inverse", [False, True], ids=["triangular", "inverse"])
def test_dense_solve_large(lib, inverse):
    """Several panels and trailing-update tiles (n = 3000)."""
    n = 3000
    A, b = _rand(n, 11)
    A = A + 3.0 * np.sqrt(n) * np.eye(n)
    x = lib.dense_solve(A, b, inverse=inverse)
    r = A @ x - b
    assert np.linalg.norm(r) <= 2e-5 * np.linalg.norm(A, 2) * np.linalg.norm(x)


@pytest.mark.parametrize("inverse", [False, True], ids=["triangular", "inverse"])
@pytest.mark.parametrize("n", [257, 1000])
def test_dense_solve_several_rhs(lib, n, inverse):
    """11 right-hand sides (a block of 8 through one pass over the inverse,
    then 3; odd n falls back to one product per right-hand side): each equals
    LAPACK's solve."""
    A, _ = _rand(n, 21)
    A = A + 4.0 * np.sqrt(n) * np.eye(n)
    rng = np.random.default_rng(22)
    B = rng.standard_normal((11, n)) + 1j * rng.standard_normal((11, n))
    X = lib.dense_solve(A, B, inverse=inverse)
    ref = np.linalg.solve(A, B.T).T
    for q in range(11):
        assert np.linalg.norm(X[q] - ref[q]) <= 2e-4 * np.linalg.norm(ref[q])


def test_singular_matrix_is_an_error(lib):
    A, b = _rand(100, 2)
    A[:, 17] = 0.0
    with pytest.raises(lib.SieError) as e:
        lib.dense_solve(A, b)
    assert e.value.code == 1 and "pivot" in str(e.value)


def test_constraint_lu_solves_like_the_iterative_path(lib, ctx):
    """Dielectric sphere (320 triangles, AIM interior): with the dense LUs as
    their preconditioners the constraint preconditioners' triangle systems take
    a few GMRES iterations, and the solve gives the same solution as with the
    plain iterative constraint solve (dense_pc_max = 0), to the solver
    tolerances."""
    from synth import icosphere
    V, T = icosphere(2, 0.01, equal_volume=True)
    mesh = lib.Mesh(ctx, V, T)
    ops = [lib.Operator(mesh, 3e9, 4.0, 1.0, 0.0, lib.params(tol_outer=1e-8, tol_inner=1e-10, dense_pc_max=m))
           for m in (32768, 0)]
    try:
        assert ops[0].info()[19] > 0 and ops[1].info()[19] == 0
        b = ops[0].rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
        xs, st = [], []
        for op in ops:
            x, it, rr = op.solve(b)
            xs.append(x)
            st.append(op.stats())
        print("with LU", st[0], "iterative", st[1])
        assert st[0]["constraint_iters_max"] <= 5 < st[1]["constraint_iters_max"]
        assert np.linalg.norm(xs[0] - xs[1]) <= 1e-5 * np.linalg.norm(xs[1])
    finally:
        for op in ops:
            op.close()
        mesh.close()
