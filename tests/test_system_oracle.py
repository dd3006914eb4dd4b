"""Pins of the oracle's GIBC system, excitation and RCS (CPU)."""
import numpy as np
import pytest

from oracle import mie, mom, system
from oracle.rwg import Mesh
from synth import cn_vector, icosphere


@pytest.fixture(scope="module")
def diel1():
    V, T = icosphere(1, 0.01, equal_volume=True)
    m = Mesh(V, T)
    return m, system.DenseGIBC(m, 3e9, 4.0, 0.0)


def test_aefie_schur_complement_is_gibc(diel1):
    """Eliminating c0 rho from Eq. (sys) gives Eq. (GIBCsys)/eta0: with
    c0 rho = -(F D H)/(j k0) the charge rows vanish and the current rows equal
    [j k0 L_0 - (K_0 + Ix/2) Z'] H (pins D, B, F of the augmented form)."""
    m, S = diel1
    H = cn_vector(m.ne, 3)
    c0rho = -(m.incidence() @ H) / m.area / (1j * S.k0)
    r1, r2 = S.sys_apply(H, c0rho)
    assert np.abs(r2).max() <= 1e-12 * np.abs(H).max() * np.abs(m.incidence()).max() / m.area.min()
    ref = S.A @ H
    assert np.linalg.norm(r1 - ref) <= 1e-12 * np.linalg.norm(ref)


def test_ix_orientation_antisymmetric():
    V, T = icosphere(1, 1.0)
    m = Mesh(V, T)
    X = mom.Ix(m)
    assert np.abs(X + X.T).max() == 0.0 and np.abs(X).max() > 0


@pytest.fixture(scope="module")
def diel2():
    V, T = icosphere(2, 0.01, equal_volume=True)
    m = Mesh(V, T)
    return m, system.DenseGIBC(m, 3e9, 4.0, 0.0)


def test_gibc_rcs_matches_mie(diel2):
    """Sec. V-A check: the dense GIBC solution's RCS matches the Mie series
    (dielectric sphere, eps_r = 4, k0 a = 0.63, 320 equal-volume triangles):
    monostatic and an E-plane bistatic cut within 1%."""
    m, S = diel2
    b = system.rhs_planewave(m, S.k0, [0, 0, -1], [1, 0, 0])
    H, E = S.solve(b)
    th = np.linspace(0.3, np.pi, 9)
    dirs = np.stack([np.sin(th), 0 * th, -np.cos(th)], 1)  # theta from the propagation direction (-z)
    got = system.rcs(m, S.k0, H, E, dirs)
    ref = mie.bistatic_rcs(th, 0.0, 0.01, 3e9, 4.0)
    assert np.abs(got / ref - 1).max() < 0.01


def test_pec_limit_rcs(diel2):
    """Z -> 0 (perfect conductor): the EFIE part alone matches PEC Mie."""
    m, S = diel2
    b = system.rhs_planewave(m, S.k0, [0, 0, -1], [1, 0, 0])
    H = np.linalg.solve(1j * S.k0 * S.L0, b)
    got = system.rcs(m, S.k0, H, np.zeros(m.ne, complex), [[0, 0, 1]])[0]
    assert abs(got / mie.backscatter_rcs(0.01, 3e9, pec=True) - 1) < 0.01


@pytest.fixture(scope="module")
def lossy2():
    """Conductive sphere (sigma = 1e4 S/m, 10 GHz, r = 1 mm, skin depth 50 um,
    320 triangles), interior operators restricted to the 5-skin-depth cutoff
    (Sec. V), solved for the x-polarised plane wave along -z."""
    V, T = icosphere(2, 1e-3, equal_volume=True)
    m = Mesh(V, T)
    ki = system.k_medium(10e9, 1.0, 1e4)
    S = system.DenseGIBC(m, 10e9, 1.0, 1e4, interior="near", cutoff=5.0 / abs(ki.imag))
    H, E = S.solve(system.rhs_planewave(m, S.k0, [0, 0, -1], [1, 0, 0]))
    return m, S, H, E


def test_lossy_near_only_interior_rcs(lossy2):
    """Near-only Z_i as a sparse solve: RCS within 1% of Mie."""
    m, S, H, E = lossy2
    got = system.rcs(m, S.k0, H, E, [[0, 0, 1]])[0]
    ref = mie.backscatter_rcs(1e-3, 10e9, 1.0, 1e4)
    assert abs(got / ref - 1) < 0.01


def test_powers_match_mie_cross_sections(lossy2):
    """The radiated and absorbed powers of oracle/ports.py (the pins of the
    port model): plane wave of 1 V/m on the lossy sphere, scattered power =
    C_sca / (2 eta0), power into the object through its surface =
    (C_ext - C_sca) / (2 eta0), the cross sections from the Mie
    coefficients."""
    from oracle import ports
    m, S, H, E = lossy2
    a, b = mie.coefficients(S.k0 * 1e-3, mie.rel_index(1.0, 1e4, 10e9))
    n = np.arange(1, len(a) + 1)
    c_ext = 2 * np.pi / S.k0 ** 2 * np.sum((2 * n + 1) * (a + b).real)
    c_sca = 2 * np.pi / S.k0 ** 2 * np.sum((2 * n + 1) * (abs(a) ** 2 + abs(b) ** 2))
    i0 = 1.0 / (2 * system.ETA0)
    p_sca = ports.radiated_power(m, S.k0, H, E)
    p_abs = ports.object_power(S.Ix, H, E)
    print("P_sca", p_sca, c_sca * i0, "P_abs", p_abs, (c_ext - c_sca) * i0)
    assert abs(p_sca / (c_sca * i0) - 1) <= 1e-3
    assert abs(p_abs / ((c_ext - c_sca) * i0) - 1) <= 2e-3


@pytest.fixture(scope="module")
def aimsys():
    """Conductive sphere (1e4 S/m, 10 GHz, r = 1 mm, 80 triangles): the AIM form
    of Eq. (sys) (oracle O2) beside the dense form, both with the near-region-only
    interior of the 5-skin-depth rule."""
    from oracle import aim
    V, T = icosphere(1, 1e-3, equal_volume=True)
    m = Mesh(V, T)
    ki = system.k_medium(10e9, 1.0, 1e4)
    cut = 5.0 / abs(ki.imag)
    g = aim.grid_params(m, M=2)
    return m, system.AimGIBC(m, 10e9, 1.0, 1e4, g, interior="near", cutoff=cut), \
        system.DenseGIBC(m, 10e9, 1.0, 1e4, interior="near", cutoff=cut)


def test_aim_system_scalar_split_is_aim_L(aimsys):
    """L_A,AIM - k0^-2 D^T L_phi,AIM D equals the oracle's one-pass AIM product
    L_AIM (Eq. AIM_Lin): pins the separate vector and scalar grid paths and the
    triangle near correction of L_phi against the combined path."""
    m, S, _ = aimsys
    H = cn_vector(m.ne, 31)
    split = S.LA(H) - (S.D.T @ S.Lphi(S.D @ H)) / S.k0 ** 2
    ref = S.ext.L(H)
    assert np.linalg.norm(split - ref) <= 1e-12 * np.linalg.norm(ref)


def test_aim_system_interior_and_rows(aimsys):
    """Z' by the sparse LU equals the dense solve; the charge rows are exact; the
    current rows match the dense system to the AIM approximation error."""
    m, S, Dn = aimsys
    H, rho = cn_vector(m.ne, 32), cn_vector(m.nt, 33)
    assert np.linalg.norm(S.Z(H) - Dn.Z @ H) <= 1e-12 * np.linalg.norm(Dn.Z @ H)
    r1, r2 = S.apply(H, rho)
    d1, d2 = Dn.sys_apply(H, rho)
    assert np.linalg.norm(r2 - d2) <= 1e-13 * np.linalg.norm(d2)
    assert np.linalg.norm(r1 - d1) <= 2e-3 * np.linalg.norm(d1)


def test_stored_mie_backscatter_is_the_oracle():
    """tests/golden/mie_backscatter.txt (read by bench.py to check its solves)
    holds what oracle/mie.py gives."""
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_mie_backscatter as g
    stored = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden", "mie_backscatter.txt"))
              if not l.startswith("#")]
    for row, s in zip(g.rows(), stored):
        assert row[0] == s[0] and abs(row[5] - float(s[5])) <= 1e-15 * row[5]


def test_gram_matrix_closed_form_vs_quadrature():
    """The oracle's RWG Gram matrix (closed form per triangle) against a product
    Gauss rule exact for its quadratic integrand."""
    from oracle import aim
    V, T = icosphere(1, 1.0)
    m = Mesh(V, T)
    G = mom.gram(m)
    pts, wts = aim.tri_rule_pts(m, 3)
    cf = m.coef()
    ref = np.zeros_like(G)
    for t in range(m.nt):
        f = [cf[t, i] * (pts[t] - m.V[m.tri_free[t, i]]) for i in range(3)]
        for i in range(3):
            for j in range(3):
                ref[m.tri_edge[t, i], m.tri_edge[t, j]] += np.sum(wts[t] * np.einsum("qa,qa->q", f[i], f[j]))
    assert np.abs(G - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("sigma", [1e6, 5.8e7])
def test_sibc_rcs_matches_mie(sigma):
    """The surface impedance condition (the paper's high-conductivity
    comparator): its RCS matches the Mie series (r = 1 mm, 10 GHz)."""
    V, T = icosphere(2, 1e-3, equal_volume=True)
    m = Mesh(V, T)
    S = system.DenseGIBC(m, 10e9, 1.0, sigma, interior="sibc")
    b = system.rhs_planewave(m, S.k0, [0, 0, -1], [1, 0, 0])
    H, E = S.solve(b)
    got = system.rcs(m, S.k0, H, E, [[0, 0, 1]])[0]
    assert abs(got / mie.backscatter_rcs(1e-3, 10e9, 1.0, sigma) - 1) < 1e-3


def test_sibc_is_the_gibc_limit():
    """At copper conductivity Z'_SIBC is within 3e-3 of the near-only GIBC Z'
    (curvature corrections of order delta / r; 1.7e-3 measured)."""
    V, T = icosphere(2, 1e-3, equal_volume=True)
    m = Mesh(V, T)
    S = system.DenseGIBC(m, 10e9, 1.0, 5.8e7, interior="sibc")
    ki = system.k_medium(10e9, 1.0, 5.8e7)
    Sg = system.DenseGIBC(m, 10e9, 1.0, 5.8e7, interior="near", cutoff=5.0 / abs(ki.imag))
    x = cn_vector(m.ne, 3)
    d = np.linalg.norm(S.Z @ x - Sg.Z @ x) / np.linalg.norm(Sg.Z @ x)
    assert d < 3e-3, d


def test_aim_system_with_sibc_interior(aimsys):
    """AimGIBC.with_sibc(): the same exterior, Z' = (eta_i / eta0) G^-1 Ix as
    in the dense SIBC form (the near-only system it was made from is left
    unchanged)."""
    m, S, D = aimsys
    H = cn_vector(m.ne, 51)
    z_near = S.Z(H)
    sb = S.with_sibc()
    ref = system.z_sibc(m, 10e9, 1.0, 1e4, mom.gram(m), mom.Ix(m)) @ H
    assert sb.ext is S.ext
    assert np.linalg.norm(sb.Z(H) - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.array_equal(S.Z(H), z_near)


def test_objects_oracle_one_object_is_aim_system():
    """The several-object oracle with one object reduces to the one-object AIM
    system (its per-object restriction and block assembly pinned)."""
    from oracle import aim
    V, T = icosphere(1, 1e-3, equal_volume=True)
    m = Mesh(V, T)
    g = aim.grid_params(m, M=2)
    ki = system.k_medium(10e9, 1.0, 1e4)
    one = system.AimGIBC(m, 10e9, 1.0, 1e4, g, interior="near", cutoff=5.0 / abs(ki.imag))
    multi = system.ObjectsGIBC(m, np.zeros(m.nt, int), [(1.0, 1e4)], 10e9, g)
    H, rho = cn_vector(m.ne, 41), cn_vector(m.nt, 42)
    assert np.linalg.norm(multi.Z(H) - one.Z(H)) <= 1e-12 * np.linalg.norm(one.Z(H))
    a1, a2 = multi.apply(H, rho)
    b1, b2 = one.apply(H, rho)
    assert np.linalg.norm(a1 - b1) <= 1e-12 * np.linalg.norm(b1) and np.linalg.norm(a2 - b2) <= 1e-14 * np.linalg.norm(b2)
