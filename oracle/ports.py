"""Port excitation and network parameters (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper excites its IC-package and interconnect examples through ports
(Sec. II, which allows a port excitation in place of the plane wave, and
Sec. V, where Thevenin-equivalent ports give the S parameters), but it
only cites the port model.  The model used here is the delta gap, in its
plainest reading:

* A port is a closed loop of mesh edges that cuts a conductor's surface.
  It is given by a plane (a point o and a unit normal n) and a radius rho.
  Its edges are those whose two end points lie in the plane (within 1e-6 of
  the mean edge length) and within rho of o.  Each of them must have its two
  triangles on opposite sides of the plane.
* The port's impressed field is E_gap = V delta(xi) n on the surface, with
  xi = n . (r - o).  It enters Eq. (EFIE01dis) exactly as the incident field
  does: b_m = -(1/eta0) I f_m . E_gap dS = -(V/eta0) s_m l_m.  Here s_m = +1
  when T+ of edge m lies on the -n side, since f_m flows from T+ to T- and
  its normal component on the edge is 1.
* The port current is the current that crosses the loop along +n,
  I = sum_m s_m l_m J_m.  Here J_m is the coefficient of the surface current
  of RWG m.  The system's first block of unknowns is the RWG expansion of
  -n x H (Eq. EFIE01dis tested with rotated RWG and -E_inc on the right), so
  J_m = -H_m and I = -p . H with p_m = s_m l_m.  The power balance pins that
  sign: (1/2) Re(V I*) equals the radiated power (tests/test_ports_oracle.py).
* Y_ij = I_i / V_j with every other port shorted (no impressed field there).
  S = (I - z Y)(I + z Y)^-1 for one real reference impedance z on every port.

Power quantities (the pins of this model):
* radiated: P_rad = (1 / 2 eta0) |r E_s|^2 integrated over the sphere of
  directions, with r E_s = (k0 eta0 / 4 pi) |N_perp(H) + rhat x N(E')| as in
  system.rcs;
* into the object: P_obj = -(1/2) Re I (E x H*) . n dS.  With the RWG
  expansions e = n x E (coefficients eta0 E') and j = n x H this is
  -(eta0/2) Re(H^H I_x E'), with (I_x)_mn = I f_m . (n x f_n).  The overall
  sign of H and E' cancels in both powers.
"""
import numpy as np

from .system import ETA0


def _edge_vertices(mesh):
    """(ne, 2) vertex ids of each edge: slot i of triangle t is the edge
    (T[t, i+1], T[t, i+2]) opposite T[t, i] (Sec. II-A RWG table)."""
    ev = np.zeros((mesh.ne, 2), np.int64)
    for i in range(3):
        a = mesh.T[:, (i + 1) % 3]
        b = mesh.T[:, (i + 2) % 3]
        ev[mesh.tri_edge[:, i], 0] = np.minimum(a, b)
        ev[mesh.tri_edge[:, i], 1] = np.maximum(a, b)
    return ev


def port_edges(mesh, origin, normal, radius):
    """Edges of one port and their signs s_m (see the module docstring).
    Raises ValueError when the port selects no edge or an edge whose
    triangles do not straddle the plane."""
    o = np.asarray(origin, float)
    n = np.asarray(normal, float)
    n = n / np.linalg.norm(n)
    tol = 1e-6 * mesh.mean_edge()
    ev = _edge_vertices(mesh)
    d = (mesh.V - o) @ n
    r = np.linalg.norm(mesh.V - o, axis=1)
    on = (np.abs(d[ev]) <= tol).all(axis=1) & (r[ev] <= radius).all(axis=1)
    edges = np.nonzero(on)[0]
    if len(edges) == 0:
        raise ValueError("port selects no edge")
    side_p = (mesh.centroid[mesh.edge_tri[edges, 0]] - o) @ n
    side_m = (mesh.centroid[mesh.edge_tri[edges, 1]] - o) @ n
    if np.any(side_p * side_m >= 0):
        raise ValueError("a port edge does not separate its two triangles")
    return edges, np.where(side_p < 0, 1, -1)


def port_vector(mesh, port):
    """p with p_m = s_m l_m on the port's edges (0 elsewhere)."""
    edges, s = port_edges(mesh, *port)
    p = np.zeros(mesh.ne)
    p[edges] = s * mesh.edge_len[edges]
    return p


def port_rhs(mesh, ports, volts=None):
    """First-block right-hand sides (nport, ne), one per port driven with
    volts[j] (1 V by default): b = -(V / eta0) p."""
    P = np.array([port_vector(mesh, pt) for pt in ports])
    v = np.ones(len(ports)) if volts is None else np.asarray(volts)
    return -(v[:, None] / ETA0) * P


def port_currents(mesh, ports, H):
    """I[r, i] = current through port i of solution r: -p_i . H_r."""
    P = np.array([port_vector(mesh, pt) for pt in ports])
    H = np.atleast_2d(H)
    return -(H @ P.T)


def admittance(mesh, ports, solve):
    """Y (nport x nport): Y[i, j] = current through port i when port j is
    driven with 1 V and the others are shorted.  solve(b) -> H."""
    B = port_rhs(mesh, ports)
    H = np.array([solve(b) for b in B])
    return port_currents(mesh, ports, H).T


def sparams(Y, z_ref=50.0):
    """S = (I - z Y)(I + z Y)^-1 for one real reference impedance z."""
    Y = np.atleast_2d(np.asarray(Y, complex))
    E = np.eye(len(Y))
    return (E - z_ref * Y) @ np.linalg.inv(E + z_ref * Y)


def thevenin_sparams(mesh, ports_, A, z_ref=50.0):
    """S of the ports from Thevenin sources: every port loaded by z_ref, port
    j driven by a 1 V source in series with it.  The port voltage V = e -
    z_ref I enters the right-hand side, and with I = -p . H the load moves
    to the matrix: (A + (z_ref/eta0) P^T P) H = -(e_j/eta0) p_j (first
    block of Eq. sys, A: the ne x ne system with the charge unknowns
    eliminated).  Incident and reflected waves a = (V + z I) / (2 sqrt z),
    b = (V - z I) / (2 sqrt z) give S_ij = delta_ij - 2 z I_i."""
    P = np.array([port_vector(mesh, pt) for pt in ports_])
    Az = A + (z_ref / ETA0) * (P.T @ P)
    n = len(ports_)
    S = np.zeros((n, n), complex)
    for j in range(n):
        H = np.linalg.solve(Az, -P[j] / ETA0)
        I = -(P @ H)
        S[:, j] = np.eye(n)[:, j] - 2 * z_ref * I
    return S


def sphere_rule(nth, nph):
    """Directions and weights integrating over the unit sphere: Gauss-Legendre
    in cos(theta), the trapezoidal rule in phi (exact on spherical harmonics
    of degree < min(2 nth, nph))."""
    x, w = np.polynomial.legendre.leggauss(nth)
    ph = 2 * np.pi * np.arange(nph) / nph
    st = np.sqrt(1 - x ** 2)
    d = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(x, np.ones(nph))], -1)
    wt = np.outer(w, np.full(nph, 2 * np.pi / nph))
    return d.reshape(-1, 3), wt.ravel()


def radiated_power(mesh, k0, H, Ep, nth=24, nph=48):
    """P_rad of the surface currents (coefficients H, E' as in system.rcs)."""
    from .system import far_vectors
    rh, wt = sphere_rule(nth, nph)
    F = far_vectors(mesh, k0, rh)
    NH = np.einsum("n,nda->da", H, F)
    NE = np.einsum("n,nda->da", Ep, F)
    v = NH - np.einsum("da,da->d", NH, rh)[:, None] * rh + np.cross(rh, NE)
    return k0 ** 2 * ETA0 / (32 * np.pi ** 2) * np.sum(wt * np.sum(np.abs(v) ** 2, axis=1))


def object_power(Ix, H, Ep):
    """Power entering the object through its surface: -(eta0/2) Re(H^H I_x E')."""
    return -0.5 * ETA0 * np.real(np.conj(H) @ (Ix @ Ep))
