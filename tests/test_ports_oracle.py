"""Pins of the oracle's port model (oracle/ports.py) and of the library's host
routine for S parameters (CPU).

* Port selection and signs: the flux functional p . J of two ports differs by
  the divergence of J integrated between them (the discrete divergence
  theorem, with the oracle's incidence matrix D), exactly, for any J.
* Perfect-conductor limit (Z' = 0, system j k0 L0 H = b): the power a port
  delivers, (1/2) Re(V I*), equals the power radiated to infinity computed
  from the far field (Poynting), and Y = Y^T (reciprocity; L0 is complex
  symmetric), both to quadrature accuracy.  (A sign slip in the port vector,
  the excitation or the current extraction breaks the first pin.)
* The radiated and absorbed powers themselves are pinned against the Mie
  cross sections of a lossy sphere in tests/test_system_oracle.py.
* S from Y: the textbook series-impedance two-port and one-port loads; S
  measured directly with Thevenin sources and loads inside the field solve;
  the library's sie_port_sparams (host code) against it.
"""
import numpy as np
import pytest

from oracle import mom, ports, system
from oracle.rwg import Mesh
from synth import box, cn_vector

BAR = ((0.1, 0.01, 0.01), (10, 2, 2))   # 10 cm bar, 1 cm x 1 cm section, 176 triangles
P2 = [((-0.02, 0.0, 0.0), (1.0, 0.0, 0.0), 0.02), ((0.02, 0.0, 0.0), (1.0, 0.0, 0.0), 0.02)]


@pytest.fixture(scope="module")
def bar():
    return Mesh(*box(*BAR))


def test_port_edges_of_a_box_cross_section(bar):
    """A cross-section of a structured box is a loop of 2 (ny + nz) edges."""
    for pt in P2 + [((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), 0.05)]:
        e, s = ports.port_edges(bar, *pt)
        assert len(e) == 2 * (2 + 2)
        assert set(np.abs(s)) == {1}
    # reversing the normal flips every sign
    e1, s1 = ports.port_edges(bar, *P2[0])
    e2, s2 = ports.port_edges(bar, P2[0][0], (-1.0, 0.0, 0.0), P2[0][2])
    assert np.array_equal(e1, e2) and np.array_equal(s1, -s2)


def test_port_flux_obeys_the_divergence_theorem(bar):
    """For any coefficient vector J: p_2 . J - p_1 . J = sum over the triangles
    between the two ports of (D J)_t (net flux out of that strip)."""
    D = bar.incidence()
    J = cn_vector(bar.ne, 5)
    p1, p2 = (ports.port_vector(bar, pt) for pt in P2)
    x = bar.centroid[:, 0]
    strip = (x > P2[0][0][0]) & (x < P2[1][0][0])
    lhs = p2 @ J - p1 @ J
    rhs = np.sum((D @ J)[strip])
    assert abs(lhs - rhs) <= 1e-13 * np.abs(D @ J).sum()
    # the whole surface beyond port 2 (to the +x end) carries -p_2 . J out
    beyond = x > P2[1][0][0]
    assert abs(-(p2 @ J) - np.sum((D @ J)[beyond])) <= 1e-13 * np.abs(D @ J).sum()


def test_port_selection_errors(bar):
    with pytest.raises(ValueError, match="no edge"):
        ports.port_edges(bar, (-0.025, 0, 0), (1, 0, 0), 0.02)   # between mesh planes
    with pytest.raises(ValueError, match="no edge"):
        ports.port_edges(bar, (0.0, 0, 0), (1, 0, 0), 1e-4)      # radius excludes every edge
    with pytest.raises(ValueError, match="separate"):
        ports.port_edges(bar, (0.05, 0, 0), (1, 0, 0), 0.05)     # the end cap itself


@pytest.fixture(scope="module")
def pec(bar):
    """Perfect-conductor limit at two frequencies: L/lambda = 0.1 and 0.5."""
    out = {}
    for f in (0.3e9, 1.5e9):
        k0 = 2 * np.pi * f / system.C0
        LA, Lp, _ = mom.dense(bar, k0, want=("LA", "Lphi"))
        A = 1j * k0 * mom.L_full(bar, LA, Lp, k0)
        out[f] = (k0, A)
    return out


@pytest.mark.parametrize("f", [0.3e9, 1.5e9])
def test_pec_port_power_equals_radiated_power(bar, pec, f):
    k0, A = pec[f]
    Y = ports.admittance(bar, P2, lambda b: np.linalg.solve(A, b))
    B = ports.port_rhs(bar, P2)
    for j in range(2):
        H = np.linalg.solve(A, B[j])
        p_in = 0.5 * Y[j, j].real            # V = 1 V
        p_rad = ports.radiated_power(bar, k0, H, np.zeros_like(H))
        print(f, j, "P_in", p_in, "P_rad", p_rad)
        assert p_in > 0
        assert abs(p_in / p_rad - 1) <= 1e-6


@pytest.mark.parametrize("f", [0.3e9, 1.5e9])
def test_pec_reciprocity(bar, pec, f):
    k0, A = pec[f]
    Y = ports.admittance(bar, P2, lambda b: np.linalg.solve(A, b))
    # exact for the continuous operator; the oracle's near-pair quadrature
    # is not symmetric in (t, s) to the last bit (about 1e-9 of an entry),
    # and the low-frequency solve amplifies that (2.6e-8 at L/lambda = 0.1)
    print(f, "reciprocity", abs(Y[0, 1] - Y[1, 0]) / abs(Y[0, 1]))
    assert abs(Y[0, 1] - Y[1, 0]) <= 1e-6 * abs(Y[0, 1])
    # the two ports sit symmetrically on the bar
    assert abs(Y[0, 0] - Y[1, 1]) <= 1e-6 * abs(Y[0, 0])


@pytest.mark.parametrize("f", [0.3e9, 1.5e9])
def test_sparams_equal_thevenin_excitation(bar, pec, f):
    """S from Y (ports shorted, one driven) equals S measured directly with a
    Thevenin source and load of z_ref on every port (the loads inside the
    field solve), the excitation the paper uses (Sec. V)."""
    k0, A = pec[f]
    Y = ports.admittance(bar, P2, lambda b: np.linalg.solve(A, b))
    S_th = ports.thevenin_sparams(bar, P2, A, 50.0)
    S_y = ports.sparams(Y, 50.0)
    print(f, "S", S_y, "thevenin vs Y", np.abs(S_th - S_y).max())
    assert np.abs(S_th - S_y).max() <= 1e-9


def test_sparams_closed_forms():
    z0 = 50.0
    Z = 30.0 + 40.0j
    # series impedance between the two ports: Y = (1/Z) [[1, -1], [-1, 1]]
    S = ports.sparams(np.array([[1, -1], [-1, 1]]) / Z, z0)
    assert np.allclose(S, [[Z / (Z + 2 * z0), 2 * z0 / (Z + 2 * z0)], [2 * z0 / (Z + 2 * z0), Z / (Z + 2 * z0)]],
                       rtol=1e-14, atol=1e-15)
    # one-port loads: matched, open, and an impedance Z
    assert np.allclose(ports.sparams([[1 / z0]], z0), [[0.0]], atol=1e-15)       # matched load
    assert np.allclose(ports.sparams([[0.0]], z0), [[1.0]], atol=1e-15)          # open
    assert np.allclose(ports.sparams([[1 / Z]], z0), [[(Z - z0) / (Z + z0)]], rtol=1e-14)


def test_library_sparams_host_routine():
    """sie_port_sparams (host code of the library, no device work) against the
    oracle's formula on random admittance matrices."""
    import ctypes
    import os
    so = os.path.join(os.path.dirname(__file__), "..", "paper_2003_11679_gb300", "_libsie.so")
    if not os.path.exists(so):
        pytest.skip("library not built")
    L = ctypes.CDLL(so)
    L.sie_port_sparams.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    rng = np.random.Generator(np.random.PCG64(3))
    for n in (1, 2, 5):
        Y = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / 40.0
        S = np.zeros((n, n), complex)
        assert L.sie_port_sparams(n, Y.ctypes.data, 50.0, S.ctypes.data) == 0
        ref = ports.sparams(Y, 50.0)
        assert np.abs(S - ref).max() <= 1e-13 * np.abs(ref).max()
    Y = np.array([[-1 / 50.0]], complex)                 # 1 + z Y singular
    assert L.sie_port_sparams(1, Y.ctypes.data, 50.0, S.ctypes.data) == 1
    assert L.sie_port_sparams(1, Y.ctypes.data, -50.0, S.ctypes.data) == 1
