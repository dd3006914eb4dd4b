"""RWG basis on a closed triangle mesh (Sec. II-A: n x E and n x H expanded with
RWG functions, tested with rotated RWG functions).

Edge n joins triangles T+ and T-.  Its undirected vertex pair is (lo, hi),
lo < hi; T+ is the triangle in which the edge runs lo -> hi in counter-clockwise
order, T- the one where it runs hi -> lo.  Edges are numbered in increasing
(lo, hi) order.  On triangle t the function is f_n = s l_n / (2 A_t) (r - p),
s = +1 on T+, -1 on T-, p the vertex of t opposite the edge, so that
div f_n = s l_n / A_t.
"""
import numpy as np


class Mesh:
    """Triangle mesh with its RWG table.

    Attributes: V (nv,3), T (nt,3), area (nt,), normal (nt,3), centroid (nt,3),
    tri_edge/tri_sign (nt,3) (slot i = edge opposite local vertex i),
    tri_free (nt,3) (= T, the free vertex of slot i), edge_len (ne,),
    edge_tri (ne,2) = (T+, T-), edge_free (ne,2).
    """

    def __init__(self, V, T):
        self.V = np.ascontiguousarray(V, dtype=np.float64)
        self.T = np.ascontiguousarray(T, dtype=np.int32)
        V, T = self.V, self.T
        nt, nv = len(T), len(V)
        a = np.stack([T[:, (i + 1) % 3] for i in range(3)], 1).astype(np.int64)
        b = np.stack([T[:, (i + 2) % 3] for i in range(3)], 1).astype(np.int64)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo * nv + hi
        uniq, inv, cnt = np.unique(key.ravel(), return_inverse=True, return_counts=True)
        if np.any(cnt != 2):
            raise ValueError("mesh is not a closed 2-manifold (edge not shared by exactly 2 triangles)")
        self.tri_edge = inv.reshape(nt, 3).astype(np.int32)
        self.tri_sign = np.where(a < b, 1, -1).astype(np.int32)
        self.tri_free = T.copy()
        ne = len(uniq)
        self.ne, self.nt = ne, nt
        elo, ehi = uniq // nv, uniq % nv
        self.edge_len = np.linalg.norm(V[ehi] - V[elo], axis=1)
        self.edge_tri = np.zeros((ne, 2), np.int32)
        self.edge_free = np.zeros((ne, 2), np.int32)
        for s, col in ((1, 0), (-1, 1)):
            m = self.tri_sign == s
            tt, ii = np.nonzero(m)
            if np.bincount(self.tri_edge[tt, ii], minlength=ne).max() != 1:
                raise ValueError("edge orientation inconsistent (mesh not oriented)")
            self.edge_tri[self.tri_edge[tt, ii], col] = tt
            self.edge_free[self.tri_edge[tt, ii], col] = T[tt, ii]
        e1 = V[T[:, 1]] - V[T[:, 0]]
        e2 = V[T[:, 2]] - V[T[:, 0]]
        nn = np.cross(e1, e2)
        self.area = 0.5 * np.linalg.norm(nn, axis=1)
        self.normal = nn / (2.0 * self.area[:, None])
        self.centroid = (V[T[:, 0]] + V[T[:, 1]] + V[T[:, 2]]) / 3.0

    def coef(self):
        """c_{t,i} = s l / (2 A_t) for each triangle slot."""
        return self.tri_sign * self.edge_len[self.tri_edge] / (2.0 * self.area[:, None])

    def incidence(self):
        """D (nt x ne): D[p, n] = +l_n on T+, -l_n on T- (div f_n = D[p,n] / A_p)."""
        D = np.zeros((self.nt, self.ne))
        for i in range(3):
            D[np.arange(self.nt), self.tri_edge[:, i]] += self.tri_sign[:, i] * self.edge_len[self.tri_edge[:, i]]
        return D

    def mean_edge(self):
        return float(self.edge_len.mean())
