"""Independent singular quadrature for touching triangle pairs (test-only).

Computes the 14 moments that the oracle's near-field rule produces for an
ordered triangle pair (t test, s source), origin c at the centroid of t:

    Q0 = II G,  Q1 = II (r - c) G,  Q2 = II (r' - c) G,  Q3 = II (r - c).(r' - c) G,
    U  = II g (r - c) x (r' - c),   V = II g (r - r'),

with G = exp(-j k R) / (4 pi R) and grad G = g (r - r'),
g = -(1 + j k R) exp(-j k R) / (4 pi R^3)  (Eq. Grrpki and its gradient).

The method shares nothing with the oracle's polar inner integration: it
follows the relative-coordinate (Sauter-Schwab type) idea, derived here for
flat triangles.  In coordinates in which the singular set is a single point,
a Duffy (cone) map from that point turns the integrand into an analytic
function of the radial variable times a smooth angular factor, so tensor
Gauss-Legendre rules converge exponentially (the radial variable gets
geometrically graded panels when |k| times the triangle size is large).

* identical triangles: difference z = u - v of the two reference
  coordinates; the overlap of the triangle with its translate by z is a
  scaled copy of the reference triangle (size s(z) piecewise linear), so the
  4D integral is a 2D integral over the difference hexagon, split into six
  sectors (triangles with a vertex at z = 0);
* edge-adjacent triangles: the shared edge is the first coordinate of both
  parametrisations; with w = s - s' the singular set is (w, t, t') = 0 and the
  remaining coordinate s runs over an interval whose ends are linear in
  (w, t, t') on four sub-regions (split by w = 0 and w = t' - t); each
  sub-region is a convex polyhedron with the origin on its boundary, taken as
  the union of cones over its facets;
* vertex-adjacent triangles: the product of the two reference triangles is the
  union of the cones from the shared vertex over its two facets
  {s + t = 1} x T and T x {s' + t' = 1}.
"""
import numpy as np


def gl(n, a=0.0, b=1.0):
    x, w = np.polynomial.legendre.leggauss(n)
    return a + (b - a) * 0.5 * (x + 1.0), (b - a) * 0.5 * w


def radial_rule(kL, n):
    """Composite Gauss-Legendre on [0, 1], panels [2^-m, 2^-m+1] graded toward
    0 (down to a panel of about 1 / (8 |k| L)), n points per panel."""
    m = int(max(3, np.ceil(np.log2(max(kL, 1.0))) + 4))
    edges = np.concatenate([[0.0], 2.0 ** -np.arange(m, -1, -1)])
    xs, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        x, w = gl(n, a, b)
        xs.append(x)
        ws.append(w)
    return np.concatenate(xs), np.concatenate(ws)


def unit_triangle_rule(n):
    """Collapsed Gauss rule on {a, b >= 0, a + b <= 1}: points (q, 2), weights (sum 1/2)."""
    x, w = gl(n)
    A, B = np.meshgrid(x, x, indexing="ij")
    WA, WB = np.meshgrid(w, w, indexing="ij")
    a = A.ravel()
    b = (B * (1.0 - A)).ravel()
    return np.stack([a, b], 1), (WA * WB * (1.0 - A)).ravel()


def _moments(X, Y, D, W, c, k):
    """The 14 moments from points X (test), Y (source), D = X - Y (computed
    without cancellation where possible) and weights W (all flattened)."""
    R = np.linalg.norm(D, axis=-1)
    e = np.exp(-1j * k * R)
    G = e / (4 * np.pi * R)
    g = -(1 + 1j * k * R) * e / (4 * np.pi * R ** 3)
    rt, rs = X - c, Y - c
    WG, Wg = W * G, W * g
    out = np.zeros(14, complex)
    out[0] = WG.sum()
    out[1:4] = WG @ rt
    out[4:7] = WG @ rs
    out[7] = WG @ np.einsum("na,na->n", rt, rs)
    out[8:11] = Wg @ np.cross(rt, rs)
    out[11:14] = Wg @ D
    return out


def self_moments(A, B, C, k, n=10):
    """Identical triangles (A, B, C): x(u) = A + u1 (B - A) + u2 (C - B) on
    {0 <= u2 <= u1 <= 1}.  U = V = 0 by the antisymmetry of their integrands
    under r <-> r' (returned as computed from the symmetric sector pairs)."""
    A, B, C = (np.asarray(v, float) for v in (A, B, C))
    J1, J2 = B - A, C - B
    area2 = np.linalg.norm(np.cross(J1, J2))
    c = (A + B + C) / 3.0
    L = max(np.linalg.norm(J1), np.linalg.norm(J2), np.linalg.norm(C - A))
    rho, wr = radial_rule(abs(k) * L, n)
    lam, wl = gl(n)
    # inner rule on the reference triangle {0 <= w2 <= w1 <= 1}: w1 = xi, w2 = xi eta
    xi, wx = gl(6)
    XI, ET = np.meshgrid(xi, xi, indexing="ij")
    WX, WE = np.meshgrid(wx, wx, indexing="ij")
    wref = np.stack([XI.ravel(), (XI * ET).ravel()], 1)
    wwref = (WX * WE * XI).ravel()
    sectors = [((0, 1), (1, 1)), ((1, 0), (1, 1)), ((0, 1), (-1, 0)), ((1, 0), (0, -1)),
               ((-1, -1), (-1, 0)), ((-1, -1), (0, -1))]
    total = np.zeros(14, complex)
    for P1, P2 in sectors:
        P1, P2 = np.array(P1, float), np.array(P2, float)
        det = abs(P1[0] * P2[1] - P1[1] * P2[0])
        dirs = (1 - lam)[:, None] * P1 + lam[:, None] * P2  # (nl, 2)
        z = rho[:, None, None] * dirs[None, :, :]  # (nr, nl, 2)
        wz = (rho[:, None] * det * wr[:, None] * wl[None, :])  # (nr, nl)
        z = z.reshape(-1, 2)
        wz = wz.ravel()
        a = np.maximum(0.0, z[:, 1])
        b = np.minimum(1.0, 1.0 + z[:, 0])
        cc = np.minimum(0.0, z[:, 1] - z[:, 0])
        s = b - a + cc
        o = np.stack([a - cc, a], 1)
        u = o[:, None, :] + s[:, None, None] * wref[None, :, :]  # (nz, q, 2)
        v = u - z[:, None, :]
        X = A + u[..., 0:1] * J1 + u[..., 1:2] * J2
        Y = A + v[..., 0:1] * J1 + v[..., 1:2] * J2
        D = np.broadcast_to((z[:, 0:1] * J1 + z[:, 1:2] * J2)[:, None, :], X.shape)
        W = (area2 ** 2) * (wz * s * s)[:, None] * wwref[None, :]
        total += _moments(X.reshape(-1, 3), Y.reshape(-1, 3), D.reshape(-1, 3), W.ravel(), c, k)
    return total


def _cones_of_region(halfspaces, interior):
    """Facet triangles (V1, V2, V3) not containing the origin of the convex
    polyhedron {x : H[:, :3] x + H[:, 3] <= 0}."""
    from scipy.spatial import ConvexHull, HalfspaceIntersection
    hs = HalfspaceIntersection(np.asarray(halfspaces, float), np.asarray(interior, float))
    pts = hs.intersections
    hull = ConvexHull(pts)
    tris = []
    for simplex, eq in zip(hull.simplices, hull.equations):
        if abs(eq[3]) < 1e-12:  # the facet's plane passes through the origin
            continue
        tris.append(pts[simplex])
    return tris


# sub-regions of (w, t, t') for edge-adjacent pairs: half-spaces a.x + b <= 0 and
# the s-interval [lo, hi] (coefficients of (w, t, t', 1)) on each
_EA_REGIONS = [
    # w >= 0, w >= t' - t, w <= 1 - t:  s in [w, 1 - t]
    ([[-1, 0, 0, 0], [-1, -1, 1, 0], [1, 1, 0, -1], [0, -1, 0, 0], [0, 0, -1, 0]], [0.3, 0.1, 0.1],
     [1, 0, 0, 0], [0, -1, 0, 1]),
    # w >= 0, w <= t' - t, t' <= 1:  s in [w, 1 - t' + w]
    ([[-1, 0, 0, 0], [1, 1, -1, 0], [0, 0, 1, -1], [0, -1, 0, 0], [0, 0, -1, 0]], [0.1, 0.1, 0.5],
     [1, 0, 0, 0], [1, 0, -1, 1]),
    # w <= 0, w >= t' - t, t <= 1:  s in [0, 1 - t]
    ([[1, 0, 0, 0], [-1, -1, 1, 0], [0, 1, 0, -1], [0, -1, 0, 0], [0, 0, -1, 0]], [-0.1, 0.5, 0.1],
     [0, 0, 0, 0], [0, -1, 0, 1]),
    # w <= 0, w <= t' - t, w >= t' - 1:  s in [0, 1 - t' + w]
    ([[1, 0, 0, 0], [1, 1, -1, 0], [-1, 0, 1, -1], [0, -1, 0, 0], [0, 0, -1, 0]], [-0.3, 0.1, 0.2],
     [0, 0, 0, 0], [1, 0, -1, 1]),
]


def edge_moments(P, P2, Q, Qs, k, n=10, c=None):
    """Test triangle (P, P2, Q) and source triangle (P, P2, Qs) sharing the edge
    P-P2: x = P + s e + t a, y = P + s' e + t' b (e = P2 - P, a = Q - P,
    b = Qs - P), s, t, s', t' >= 0, s + t <= 1, s' + t' <= 1."""
    P, P2, Q, Qs = (np.asarray(v, float) for v in (P, P2, Q, Qs))
    e, a, b = P2 - P, Q - P, Qs - P
    if c is None:
        c = (P + P2 + Q) / 3.0
    jac = np.linalg.norm(np.cross(e, a)) * np.linalg.norm(np.cross(e, b))
    L = max(np.linalg.norm(e), np.linalg.norm(a), np.linalg.norm(b))
    rho, wr = radial_rule(abs(k) * L, n)
    ab, wab = unit_triangle_rule(n)
    sq, wsq = gl(4)
    total = np.zeros(14, complex)
    for H, inter, lo_c, hi_c in _EA_REGIONS:
        for V1, V2, V3 in _cones_of_region(H, inter):
            E1, E2 = V2 - V1, V3 - V1
            det = abs(np.linalg.det(np.stack([V1, E1, E2])))
            dirs = V1 + ab[:, 0:1] * E1 + ab[:, 1:2] * E2  # (q, 3)
            p = rho[:, None, None] * dirs[None]  # (nr, q, 3): (w, t, t')
            wp = (rho ** 2 * wr)[:, None] * (det * wab)[None, :]
            p = p.reshape(-1, 3)
            wp = wp.ravel()
            lo = p @ np.array(lo_c[:3], float) + lo_c[3]
            hi = p @ np.array(hi_c[:3], float) + hi_c[3]
            s = lo[:, None] + (hi - lo)[:, None] * sq[None, :]  # (np, 4)
            w, t, tp = p[:, 0:1], p[:, 1:2], p[:, 2:3]
            X = P + s[..., None] * e + (t * np.ones_like(s))[..., None] * a
            Y = P + (s - w)[..., None] * e + (tp * np.ones_like(s))[..., None] * b
            D = (w * e + t * a - tp * b)[:, None, :] * np.ones_like(s)[..., None]
            W = jac * (wp * (hi - lo))[:, None] * wsq[None, :]
            total += _moments(X.reshape(-1, 3), Y.reshape(-1, 3), D.reshape(-1, 3), W.ravel(), c, k)
    return total


def vertex_moments(P, a1, a2, b1, b2, k, n=10, c=None):
    """Test triangle (P, P + a1, P + a2) and source (P, P + b1, P + b2) sharing
    the vertex P: x = P + s a1 + t a2, y = P + s' b1 + t' b2."""
    P, a1, a2, b1, b2 = (np.asarray(v, float) for v in (P, a1, a2, b1, b2))
    if c is None:
        c = P + (a1 + a2) / 3.0
    jac = np.linalg.norm(np.cross(a1, a2)) * np.linalg.norm(np.cross(b1, b2))
    L = max(np.linalg.norm(v) for v in (a1, a2, b1, b2, a2 - a1, b2 - b1))
    rho, wr = radial_rule(abs(k) * L, n)
    mu, wmu = gl(n)
    st, wst = unit_triangle_rule(n)
    total = np.zeros(14, complex)
    for facet in (0, 1):
        # facet 0: (s, t) = (mu, 1 - mu), (s', t') over the triangle; facet 1: the reverse
        M = np.repeat(mu, len(st))
        S = np.tile(st, (len(mu), 1))
        wf = np.repeat(wmu, len(st)) * np.tile(wst, len(mu))
        if facet == 0:
            q = np.stack([M, 1 - M, S[:, 0], S[:, 1]], 1)
        else:
            q = np.stack([S[:, 0], S[:, 1], M, 1 - M], 1)
        vX = q[:, 0:1] * a1 + q[:, 1:2] * a2
        vY = q[:, 2:3] * b1 + q[:, 3:4] * b2
        X = P + rho[:, None, None] * vX[None]
        Y = P + rho[:, None, None] * vY[None]
        D = rho[:, None, None] * (vX - vY)[None]
        W = jac * (rho ** 3 * wr)[:, None] * wf[None, :]
        total += _moments(X.reshape(-1, 3), Y.reshape(-1, 3), D.reshape(-1, 3), W.ravel(), c, k)
    return total


def touching_moments(V, T, t, s, k, n=10):
    """The 14 moments of the touching ordered pair (t, s) of mesh (V, T)."""
    tt, ss = [int(v) for v in T[t]], [int(v) for v in T[s]]
    c = V[tt].mean(0)
    shared = [v for v in tt if v in ss]
    if t == s:
        return self_moments(V[tt[0]], V[tt[1]], V[tt[2]], k, n)
    if len(shared) == 2:
        p, q = shared
        ft = [v for v in tt if v not in shared][0]
        fs = [v for v in ss if v not in shared][0]
        return edge_moments(V[p], V[q], V[ft], V[fs], k, n, c=c)
    if len(shared) == 1:
        p = shared[0]
        ta = [v for v in tt if v != p]
        sa = [v for v in ss if v != p]
        return vertex_moments(V[p], V[ta[0]] - V[p], V[ta[1]] - V[p], V[sa[0]] - V[p], V[sa[1]] - V[p], k, n, c=c)
    raise ValueError("pair does not touch")
