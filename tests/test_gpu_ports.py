"""Ports on the GPU (the delta-gap port model of oracle/ports.py and
sie_port_*), through the C ABI, against the oracle.

Workload: a copper bar (40 x 4 x 4 um, sigma = 5.8e7 S/m, 100 GHz; structured
mesh of 336 triangles / 504 RWG) with two ports across its cross-section at
x = -10 um and x = +10 um, interior near-region only (the library's choice:
5 skin depths, 1.0 um, fit inside the near region) or the surface impedance
condition.  (At 20 GHz, k0 l = 8e-4, the outer solve stagnates: see the
design notes on low-frequency convergence.)

* Port edges and signs: identical to the oracle's selection (integers).
* Right-hand sides and port currents: the same closed forms, 1e-14.
* Admittance matrix from the GPU solves (tol_outer 1e-9, nested 1e-13)
  against the oracle's AIM form of Eq. (sys) (O2, same grid, GMRES to 1e-13
  preconditioned by the dense O1 system):
  within the bound that the solve's weighted residual implies, and against
  the dense method of moments (O1):
  the AIM approximation error (1.3e-5 between the two oracles; 1e-4).
* Lockstep (one block of both ports) equals one solve after another.
* S parameters: the library's host routine against the oracle's formula.
"""
import numpy as np
import pytest

from oracle import aim, ports, system
from oracle.rwg import Mesh
from synth import box, cn_vector

pytestmark = pytest.mark.gpu

F, SIGMA = 100e9, 5.8e7
PORTS = [((-10e-6, 0.0, 0.0), (1.0, 0.0, 0.0), 8e-6), ((10e-6, 0.0, 0.0), (1.0, 0.0, 0.0), 8e-6)]


def _cutoff():
    return 5.0 / abs(system.k_medium(F, 1.0, SIGMA).imag)


def _o1_augmented(m, D, Z):
    """Dense Eq. (sys) of O1 (dense exterior matrices of D, interior Z') in the
    augmented unknowns [H; c0 rho]: B = -diag(A), F = diag(1/A)."""
    Dm = m.incidence()
    top = np.hstack([1j * D.k0 * D.LA0 - (D.K0 + 0.5 * D.Ix) @ Z, -(Dm.T @ D.Lp0) * m.area[None, :]])
    bot = np.hstack([Dm / m.area[:, None], 1j * D.k0 * np.eye(m.nt)])
    return np.vstack([top, bot])


def oracle_admittances(m):
    """For the near-region-only interior and for SIBC (both share the
    exterior operators):
    * Y of O2, the AIM system the GPU solves, with c0 rho eliminated (the
      charge rows of Eq. sys with zero right-hand side give c0 rho =
      -F D H / (j k0)), by GMRES to 1e-12 preconditioned by the dense O1
      matrix of the same form;
    * Y of O1;
    * G[i] = W^-1 A1^-T [p_i; 0] with W = diag(1, q_w) (q_w = mean |L_A,mm|,
      the weight of the library's residual norm): the error of port current
      i after a solve with weighted residual r is |G[i] . (W r)|."""
    import scipy.linalg as sla
    import scipy.sparse.linalg as spl
    from oracle import mom
    g = aim.grid_params(m, M=2)
    s_near = system.AimGIBC(m, F, 1.0, SIGMA, g, interior="near", cutoff=_cutoff())
    s_sibc = s_near.with_sibc()
    d = system.DenseGIBC(m, F, 1.0, SIGMA, interior="near", cutoff=_cutoff())
    z_sibc = system.z_sibc(m, F, 1.0, SIGMA, mom.gram(m), d.Ix)
    Dm = system.incidence_sparse(m)
    qw = np.mean(np.abs(np.diag(d.LA0)))
    w = np.concatenate([np.ones(m.ne), np.full(m.nt, qw)])
    P = np.array([ports.port_vector(m, pt) for pt in PORTS])
    out = {}
    for name, S, Z in (("near", s_near, d.Z), ("sibc", s_sibc, z_sibc)):
        A1 = 1j * d.k0 * d.L0 - (d.K0 + 0.5 * d.Ix) @ Z
        lu1 = sla.lu_factor(A1)

        def o2(H, S=S):
            E = S.Z(H)
            return (1j * S.k0 * S.LA(H) + Dm.T @ S.Lphi(Dm @ H) / (1j * S.k0)
                    - S.ext.K(E) - 0.5 * (S.Ix @ E))

        n = m.ne
        A2 = spl.LinearOperator((n, n), matvec=o2, dtype=complex)
        M = spl.LinearOperator((n, n), matvec=lambda v, lu=lu1: sla.lu_solve(lu, v), dtype=complex)

        def solve2(b):
            x, info = spl.gmres(A2, b, rtol=1e-12, atol=0.0, restart=40, maxiter=3, M=M)
            assert info == 0
            return x

        luA = sla.lu_factor(_o1_augmented(m, d, Z))
        G = np.array([sla.lu_solve(luA, np.concatenate([p, np.zeros(m.nt)]), trans=1) / w for p in P])
        out[name] = (ports.admittance(m, PORTS, solve2), ports.admittance(m, PORTS, lambda b: sla.lu_solve(lu1, b)),
                     S, G, w)
    return out


@pytest.fixture(scope="module")
def oracle_y():
    return oracle_admittances(Mesh(*box((40e-6, 4e-6, 4e-6), (20, 2, 2))))


@pytest.fixture(scope="module", params=["near", "sibc"])
def bar(request, lib, ctx, oracle_y):
    interior = request.param
    V, T = box((40e-6, 4e-6, 4e-6), (20, 2, 2))
    m = Mesh(V, T)
    gm = lib.Mesh(ctx, V, T)
    # restart 400: unrestarted in effect (restarted GMRES(100) slows down on
    # this elongated, electrically small bar; see the design notes)
    prm = lib.params(tol_outer=1e-9, tol_inner=1e-13, restart=400,
                     interior_model=lib.SIE_SIBC if interior == "sibc" else lib.SIE_GIBC)
    op = lib.Operator(gm, F, 1.0, 1.0, SIGMA, prm)
    y_o2, y_o1, S, G, w = oracle_y[interior]
    yield interior, m, gm, op, S, y_o2, y_o1, G, w
    op.close()
    gm.close()


def test_grid_and_interior(bar):
    interior, m, gm, op, S, *_ = bar
    assert np.array_equal(op.grid()[2], S.ext.g.N)
    if interior == "near":
        assert op.info()[9] == 1.0   # near-region-only interior


def test_port_edges_match_oracle(bar):
    _, m, gm, op, *_ = bar
    for pt in PORTS:
        e, s = gm.port_edges(pt)
        e_ref, s_ref = ports.port_edges(m, *pt)
        assert np.array_equal(e, e_ref) and np.array_equal(s, s_ref)


def test_rhs_and_currents_match_oracle(bar):
    _, m, gm, op, *_ = bar
    b = op.rhs_ports(PORTS, volts=[1.0, -2.5])
    ref = ports.port_rhs(m, PORTS, volts=[1.0, -2.5])
    assert np.abs(b[:, :m.ne] - ref).max() <= 1e-14 * np.abs(ref).max()
    assert not np.any(b[:, m.ne:])
    x = np.stack([cn_vector(m.ne + m.nt, 31), cn_vector(m.ne + m.nt, 32), cn_vector(m.ne + m.nt, 33)])
    got = op.port_currents(PORTS, x, nrhs=3)
    want = ports.port_currents(m, PORTS, x[:, :m.ne])
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_admittance_matches_oracle_aim_system(lib, bar):
    """GPU Y against O2.  Bound: the port current error of a solve with
    weighted relative residual rr is at most |G_i| rr |W b| (G and W from
    the oracle's dense O1 system, which differs from O2 by the AIM error:
    factor 2), plus O2's own GMRES error (1e-12)."""
    interior, m, gm, op, S, y_o2, y_o1, G, w = bar
    Y, it, rr = op.port_admittance(PORTS, check=False)
    B = op.rhs_ports(PORTS)
    bound = np.array([[2 * np.linalg.norm(G[i]) * rr[j] * np.linalg.norm(w * B[j]) for j in range(2)]
                      for i in range(2)]) + 1e-12 * np.abs(y_o2).max()
    err = np.abs(Y - y_o2)
    print(interior, "Y", Y, "iters", it, "relres", rr, "err / |Y|", err.max() / np.abs(y_o2).max(),
          "bound / |Y|", bound.max() / np.abs(y_o2).max())
    assert np.all(rr <= 1e-8)
    assert np.all(err <= bound)
    # the lockstep block (both ports together) equals one solve after another
    Ys, _, rs = op.port_admittance(PORTS, sequential=True, check=False)
    assert np.all(rs <= 1e-8)
    assert np.all(np.abs(Ys - y_o2) <= bound * np.maximum(1.0, rs / rr)[None, :])


def test_admittance_vs_dense_method_of_moments(bar):
    """Against O1 (dense MoM, no grid): the AIM approximation error of Y."""
    interior, m, gm, op, S, y_o2, y_o1, *_ = bar
    Y, _, rr = op.port_admittance(PORTS, check=False)
    assert np.all(rr <= 1e-8)
    err = np.abs(Y - y_o1).max() / np.abs(y_o1).max()
    print(interior, "vs O1", err, "O2 vs O1", np.abs(y_o2 - y_o1).max() / np.abs(y_o1).max())
    assert err <= 1e-4   # 1.3e-5 measured between the two oracles


def test_sparams(lib, bar):
    _, m, gm, op, S, y_o2, *_ = bar
    assert np.abs(lib.port_sparams(y_o2, 50.0) - ports.sparams(y_o2, 50.0)).max() <= 1e-13


def test_port_errors(lib, bar):
    _, m, gm, op, *_ = bar
    with pytest.raises(lib.SieError) as e:
        op.rhs_ports([((-11e-6, 0.0, 0.0), (1.0, 0.0, 0.0), 8e-6)])    # between mesh planes
    assert e.value.code == 1
    with pytest.raises(lib.SieError) as e:
        gm.port_edges(((20e-6, 0.0, 0.0), (1.0, 0.0, 0.0), 8e-6))      # the end cap
    assert e.value.code == 1
    with pytest.raises(lib.SieError) as e:
        op.port_admittance([((0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 8e-6)])  # zero normal
    assert e.value.code == 1
