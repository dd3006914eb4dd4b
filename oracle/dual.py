"""Dual (Buffa-Christiansen) basis functions on the barycentric refinement
(oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's discussion of its results (Sec. V) expects dual basis functions
to improve the convergence of Eqs. (sys) and (nest2) further.  Their point is
the identity-like terms: Eqs. (MFIE1dis) and (EFIE01dis) pair RWG functions
with rotated RWG functions (the matrix I_x), a pairing that is not stable,
whereas RWG functions paired with dual functions give a well-conditioned
Gram matrix.  Construction (the standard one, written here from its
definition):

* Barycentric refinement: each triangle (v0, v1, v2) is split into the six
  triangles (v_i, m_i, c), (m_i, v_{i+1}, c) through its centroid c and the
  midpoints m_i of its edges (v_i, v_{i+1}), with the coarse orientation.
  Fine vertex ids: the coarse vertices, then nv + (coarse edge), then
  nv + ne + (coarse triangle).
* The dual function of coarse edge e (vertices lo < hi) is a combination of
  fine RWG functions.  It carries half a unit of coefficient across each of
  the two fine edges (m_e, c_{T+}) and (m_e, c_{T-}) that make up the dual
  edge, from the dual cell of lo to the dual cell of hi: the direction of
  n x f_e, which runs along e from lo to hi.  Around lo, with its 2 N fine
  triangles numbered tau_1..tau_2N from one side of e to the other, the fine
  edge between tau_i and tau_{i+1} carries (N - i) / (2 N) from tau_{i+1} to
  tau_i: each fine triangle around lo is then a source of the same strength
  1 / (2 N) in coefficient units, and the flow runs around lo to the dual
  edge.  Around hi the mirror image (sinks 1 / (2 N_hi)).
* Coarse RWG functions are exactly fine Raviart-Thomas functions: the fine
  coefficient of f_m on fine edge k is f_m . nu_k at the edge (constant
  along it), nu_k the unit normal from T+_k to T-_k.
"""
import numpy as np

from .rwg import Mesh


def edge_vertices(mesh):
    """(ne, 2): (lo, hi) vertex ids of each edge (slot i of a triangle is the
    edge (T[t, i+1], T[t, i+2]))."""
    ev = np.zeros((mesh.ne, 2), np.int64)
    for i in range(3):
        a = mesh.T[:, (i + 1) % 3]
        b = mesh.T[:, (i + 2) % 3]
        ev[mesh.tri_edge[:, i], 0] = np.minimum(a, b)
        ev[mesh.tri_edge[:, i], 1] = np.maximum(a, b)
    return ev


def barycentric_refine(mesh):
    """(fine Mesh, parent): parent[f] = coarse triangle of fine triangle f."""
    nv, ne, nt = len(mesh.V), mesh.ne, mesh.nt
    ev = edge_vertices(mesh)
    V = np.vstack([mesh.V, 0.5 * (mesh.V[ev[:, 0]] + mesh.V[ev[:, 1]]), mesh.centroid])
    T, parent = [], []
    for t in range(nt):
        c = nv + ne + t
        for i in range(3):
            a, b = mesh.T[t, i], mesh.T[t, (i + 1) % 3]
            m = nv + mesh.tri_edge[t, (i + 2) % 3]    # the edge (v_i, v_{i+1}) is opposite v_{i+2}
            T += [(a, m, c), (m, b, c)]
            parent += [t, t]
    return Mesh(V, np.array(T, np.int32)), np.array(parent)


def _fine_edge_of(fine, t, u, w):
    """Fine edge of fine triangle t joining fine vertices u and w."""
    for i in range(3):
        if fine.T[t, i] != u and fine.T[t, i] != w:
            return fine.tri_edge[t, i]
    raise ValueError("vertices not in triangle")


def _other(fine, k, t):
    a, b = fine.edge_tri[k]
    return b if a == t else a


def _ring(fine, v, start_edge):
    """Fine triangles around fine vertex v in cyclic order, starting with the
    T+ triangle of the fine edge start_edge (which contains v), and the fine
    edges between consecutive ones: tris[i], edges[i] between tris[i] and
    tris[i+1] (the last closes the ring through start_edge)."""
    tris, edges = [fine.edge_tri[start_edge, 0]], []
    prev = start_edge
    while True:
        t = tris[-1]
        nxt = [fine.tri_edge[t, i] for i in range(3) if fine.T[t, i] != v and fine.tri_edge[t, i] != prev]
        assert len(nxt) == 1
        k = nxt[0]
        edges.append(k)
        if k == start_edge:
            return tris, edges
        tris.append(_other(fine, k, t))
        prev = k


def _add_flux(C, row, fine, k, src, dst, value):
    """Coefficient on fine RWG k for a flow of `value` from fine triangle src
    to dst (their shared edge k)."""
    assert {src, dst} == set(fine.edge_tri[k])
    C[row, k] += value if fine.edge_tri[k, 0] == src else -value


def bc_matrix(mesh, fine):
    """C (ne_coarse x ne_fine): dual function e = sum_k C[e, k] f_k (fine RWG)."""
    nv, ne = len(mesh.V), mesh.ne
    ev = edge_vertices(mesh)
    C = np.zeros((ne, fine.ne))
    for e in range(ne):
        lo, hi = ev[e]
        m = nv + e
        for t in mesh.edge_tri[e]:                      # the two halves of the dual edge
            c = nv + ne + t
            # fine triangles of coarse t on the lo side and the hi side of the fine edge (m, c)
            k = None
            for f in np.nonzero((fine.T == m).any(1) & (fine.T == c).any(1))[0]:
                k = _fine_edge_of(fine, f, m, c)
            a, b = fine.edge_tri[k]
            src = a if lo in fine.T[a] else b
            dst = b if src == a else a
            assert lo in fine.T[src] and hi in fine.T[dst]
            _add_flux(C, e, fine, k, src, dst, 0.5)
        for v, sign in ((lo, 1.0), (hi, -1.0)):
            # fine edge (v, m) along e, then the ring around v from one side of e to the other
            f0 = np.nonzero((fine.T == v).any(1) & (fine.T == m).any(1))[0][0]
            start = _fine_edge_of(fine, f0, v, m)
            tris, edges = _ring(fine, v, start)
            n2 = len(tris)                              # 2 N
            N = n2 // 2
            for i in range(1, n2):                      # edges[i-1] lies between tau_i and tau_{i+1}
                val = (N - i) / n2
                if sign > 0:   # source around lo: flow (N - i) / 2N from tau_{i+1} to tau_i
                    _add_flux(C, e, fine, edges[i - 1], tris[i], tris[i - 1], val)
                else:          # sink around hi: flow (N - i) / 2N from tau_i to tau_{i+1}
                    _add_flux(C, e, fine, edges[i - 1], tris[i - 1], tris[i], val)
    return C


def rwg_in_fine(mesh, fine, parent):
    """D (ne_coarse x ne_fine): coarse f_m = sum_k D[m, k] f_k exactly."""
    D = np.zeros((mesh.ne, fine.ne))
    cf = mesh.coef()
    fv = edge_vertices(fine)
    for k in range(fine.ne):
        p, q = fine.V[fv[k, 0]], fine.V[fv[k, 1]]
        mid = 0.5 * (p + q)
        tp = fine.edge_tri[k, 0]
        # unit normal of edge k in the plane of T+_k, pointing away from T+_k
        nrm = fine.normal[tp]
        d = q - p
        nu = np.cross(d, nrm)
        nu /= np.linalg.norm(nu)
        if np.dot(nu, mid - fine.centroid[tp]) < 0:
            nu = -nu
        ct = parent[tp]
        for i in range(3):
            m = mesh.tri_edge[ct, i]
            fm = cf[ct, i] * (mid - mesh.V[mesh.tri_free[ct, i]])
            D[m, k] += fm @ nu
    return D
