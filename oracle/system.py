"""Dense GIBC system, plane-wave excitation and RCS (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Interior impedance (Eq. GIBCdef): E_i = Z_i H_i,
  Z_i = -(j w eps~_i)^-1 L_i^-1 (K_i - Ix/2), eps~_i = eps0 eps_r - j sigma / w.
  Divided by eta0 (the scaling of Eq. sys): Z' = Z_i / eta0 =
  -(j k0 eps_r + sigma eta0)^-1 L_i^-1 (K_i - Ix/2).
* System (Eq. GIBCsys / eta0): [j k0 L_0 - (K_0 + Ix/2) Z'] H = -E_inc / eta0.
* Augmented form (Eq. sys): unknowns [H; c0 rho]
    row 1: j k0 LA H - (K_0 + Ix/2) Z' H + D^T Lphi B c0 rho = -E_inc/eta0
    row 2: F D H + j k0 c0 rho = 0
  with D the signed edge-length incidence, B = -diag(A), F = diag(1/A):
  eliminating c0 rho gives back Eq. (GIBCsys) because L_0 = LA - k0^-2 D^T Lphi D.
* Excitation (Sec. II): E_inc = e_pol exp(-j k0 khat . r); b_m = -(1/eta0) I f_m . E_inc.
* RCS (Sec. V-A): with J = n x H (coefficients H) and M = -n x E (E = eta0 Z' H),
  E_s ~ (-j k0 e^{-j k0 r} / 4 pi r) eta0 [N_perp(H) + rhat x N(E')],
  N(X) = sum_n X_n I f_n exp(j k0 rhat . r') dS', so
  sigma = k0^2 eta0^2 / (4 pi) |N_perp(H) + rhat x N(E')|^2.
"""
import numpy as np

from . import aim, mom

C0 = 299792458.0
MU0 = 4e-7 * np.pi
EPS0 = 1.0 / (MU0 * C0 ** 2)
ETA0 = MU0 * C0


def k_medium(f, eps_r, sigma, mu_r=1.0):
    """Eq. (kin): k = sqrt(w mu (w eps - j sigma)), branch Im k <= 0."""
    w = 2 * np.pi * f
    k = np.sqrt(w * MU0 * mu_r * (w * EPS0 * eps_r - 1j * sigma) + 0j)
    return -k if k.imag > 0 else k


def zscale(f, eps_r, sigma):
    """j k0 eps_r + sigma eta0 = j w eps~ eta0."""
    k0 = 2 * np.pi * f / C0
    return 1j * k0 * eps_r + sigma * ETA0


def rhs_planewave(mesh, k0, khat, epol, p=6):
    pts, wts = aim.tri_rule_pts(mesh, p)
    khat = np.asarray(khat, float)
    epol = np.asarray(epol, float)
    ph = np.exp(-1j * k0 * np.einsum("tqa,a->tq", pts, khat))
    cf = mesh.coef()
    b = np.zeros(mesh.ne, complex)
    for i in range(3):
        fm = cf[:, i, None, None] * (pts - mesh.V[mesh.tri_free[:, i]][:, None, :])  # (t, q, 3)
        val = np.einsum("tq,tqa,a,tq->t", wts, fm, epol, ph)
        np.add.at(b, mesh.tri_edge[:, i], -val / ETA0)
    return b


def z_dense(mesh, f, eps_r, sigma, Li, Ki, Ix):
    return -np.linalg.solve(Li, Ki - 0.5 * Ix) / zscale(f, eps_r, sigma)


def eta_medium(f, eps_r, sigma, mu_r=1.0):
    """Wave impedance of the object's medium, eta_i = sqrt(j w mu / (sigma + j w eps)),
    branch Re eta_i > 0."""
    w = 2 * np.pi * f
    eta = np.sqrt(1j * w * MU0 * mu_r / (sigma + 1j * w * EPS0 * eps_r) + 0j)
    return -eta if eta.real < 0 else eta


def z_sibc(mesh, f, eps_r, sigma, G, Ix):
    """Surface impedance boundary condition (the high-conductivity limit the
    paper compares against): n x E = eta_i n x (n x H) on the surface, i.e.
    the coefficients of n x E and n x H satisfy G E = eta_i Ix H with the RWG
    Gram matrix G; divided by eta0: Z'_SIBC = (eta_i / eta0) G^-1 Ix."""
    return eta_medium(f, eps_r, sigma) / ETA0 * np.linalg.solve(G, Ix)


def far_vectors(mesh, k0, rhat, p=6):
    """F[n, d, a] = I f_n . e_a exp(j k0 rhat_d . r) dS (ne, ndir, 3)."""
    pts, wts = aim.tri_rule_pts(mesh, p)
    rhat = np.atleast_2d(rhat)
    ph = np.exp(1j * k0 * np.einsum("tqa,da->tqd", pts, rhat))
    cf = mesh.coef()
    F = np.zeros((mesh.ne, len(rhat), 3), complex)
    for i in range(3):
        fm = cf[:, i, None, None] * (pts - mesh.V[mesh.tri_free[:, i]][:, None, :])
        val = np.einsum("tq,tqa,tqd->tda", wts, fm, ph)
        np.add.at(F, mesh.tri_edge[:, i], val)
    return F


def rcs(mesh, k0, H, Ep, rhat):
    """sigma(rhat) in m^2 for unit incident amplitude."""
    rhat = np.atleast_2d(np.asarray(rhat, float))
    F = far_vectors(mesh, k0, rhat)
    NH = np.einsum("n,nda->da", H, F)
    NE = np.einsum("n,nda->da", Ep, F)
    Nperp = NH - np.einsum("da,da->d", NH, rhat)[:, None] * rhat
    v = Nperp + np.cross(rhat, NE)
    return k0 ** 2 * ETA0 ** 2 / (4 * np.pi) * np.sum(np.abs(v) ** 2, axis=1)


class DenseGIBC:
    """Dense direct solution of Eq. (GIBCsys) for one homogeneous object."""

    def __init__(self, mesh, f, eps_r, sigma, quad=None, interior="dense", cutoff=None):
        self.mesh, self.f, self.eps_r, self.sigma = mesh, f, eps_r, sigma
        self.k0 = 2 * np.pi * f / C0
        self.ki = k_medium(f, eps_r, sigma)
        LA0, Lp0, K0 = mom.dense(mesh, self.k0, quad)
        self.LA0, self.Lp0, self.K0 = LA0, Lp0, K0
        self.L0 = mom.L_full(mesh, LA0, Lp0, self.k0)
        self.Ix = mom.Ix(mesh)
        if interior == "sibc":
            self.Li = self.Ki = None
            self.Z = z_sibc(mesh, f, eps_r, sigma, mom.gram(mesh), self.Ix)
        else:
            if interior == "dense":
                LAi, Lpi, Ki = mom.dense(mesh, self.ki, quad)
                Li = mom.L_full(mesh, LAi, Lpi, self.ki)
            else:  # near-region-only interior with the skin-depth cutoff (Sec. V)
                no = aim.NearOnly(mesh, self.ki, cutoff, quad)
                Li, Ki = no.NL.toarray(), no.NK.toarray()
            self.Li, self.Ki = Li, Ki
            self.Z = z_dense(mesh, f, eps_r, sigma, Li, Ki, self.Ix)
        self.A = 1j * self.k0 * self.L0 - (K0 + 0.5 * self.Ix) @ self.Z

    def solve(self, b):
        H = np.linalg.solve(self.A, b)
        return H, self.Z @ H

    def sys_apply(self, H, c0rho):
        """Eq. (sys) rows for the augmented unknowns."""
        m = self.mesh
        D = m.incidence()
        r1 = 1j * self.k0 * (self.LA0 @ H) - (self.K0 + 0.5 * self.Ix) @ (self.Z @ H) \
            + D.T @ (self.Lp0 @ (-m.area * c0rho))
        r2 = (D @ H) / m.area + 1j * self.k0 * c0rho
        return r1, r2


# ---------------------------------------------------------------- AIM form of Eq. (sys) (oracle O2)
def incidence_sparse(mesh):
    """D (nt x ne) as a sparse matrix: D[p, n] = +l_n on T+, -l_n on T-."""
    import scipy.sparse as sp
    rows = np.repeat(np.arange(mesh.nt), 3)
    cols = mesh.tri_edge.ravel()
    vals = (mesh.tri_sign * mesh.edge_len[mesh.tri_edge]).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(mesh.nt, mesh.ne)).tocsr()


def Ix_sparse(mesh):
    """I_x of mom.Ix (same closed form per triangle) as a sparse matrix."""
    import scipy.sparse as sp
    cf = mesh.coef()
    rows, cols, vals = [], [], []
    for i in range(3):
        for j in range(3):
            c = mesh.centroid
            pi = mesh.V[mesh.tri_free[:, i]] - c
            pj = mesh.V[mesh.tri_free[:, j]] - c
            v = cf[:, i] * cf[:, j] * mesh.area * np.einsum("ta,ta->t", mesh.normal, np.cross(pj, pi))
            rows.append(mesh.tri_edge[:, i])
            cols.append(mesh.tri_edge[:, j])
            vals.append(v)
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(mesh.ne, mesh.ne)).tocsr()


def grid_LA(A, H):
    """W G P H: the grid part of the vector-potential operator L_A (Eq. AIM_Lin
    without its scalar term)."""
    J, _ = A.project(H)
    return A.interpolate(A._conv(J, A.kG), None, 0.0)


def grid_Lphi(A, sig):
    """Grid part of L_phi applied to triangle charges sig:
    (1/A_p) sum_u w0[p,u] sum_v G(u - v) sum_q w0[q,v] sig_q / A_q."""
    m = A.mesh
    rho = np.zeros(A.Ng, complex)
    np.add.at(rho, A.nodes.ravel(), (A.w0 * (sig / m.area)[:, None]).ravel())
    Phi = A._conv(rho, A.kG)
    return np.einsum("tu,tu->t", A.w0, Phi[A.nodes]) / m.area


class AimGIBC:
    """Eq. (sys) with every exterior operator in its AIM form (Eqs. AIM_Lin,
    AIM_Kin and the near corrections of Eqs. LinNRP, KinNRP), the operators
    of the GPU's system product:

      row 1: j k0 L_A,AIM H - (K_0,AIM + Ix/2) Z' H + D^T L_phi,AIM B c0 rho
      row 2: F D H + j k0 c0 rho,

    and Z' = -(j k0 eps_r + sigma eta0)^-1 L_i^-1 (K_i - Ix/2) (Eq. GIBCdef / eta0)
    with the interior operators near-region only (the 5-skin-depth rule of
    Sec. V; L_i,NR factorised by a sparse LU, Eq. nest2pc solved exactly), in
    their AIM form on the same grid (formed column by column, dense LU), or the
    surface impedance condition Z' = (eta_i / eta0) G^-1 Ix (interior="sibc")."""

    def __init__(self, mesh, f, eps_r, sigma, g, interior="near", cutoff=None, quad=None):
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        self.mesh, self.f, self.eps_r, self.sigma = mesh, f, eps_r, sigma
        self.k0 = 2 * np.pi * f / C0
        self.ki = k_medium(f, eps_r, sigma)
        self.ext = aim.AIM(mesh, self.k0, g, quad)
        self.Ix = Ix_sparse(mesh)
        self.D = incidence_sparse(mesh)
        self.zs = zscale(f, eps_r, sigma)
        if interior == "sibc":
            self._sibc = eta_medium(f, eps_r, sigma) / ETA0
            self._lu_gram = spl.splu(sp.csc_matrix(mom.gram(mesh).astype(complex)))
        elif interior == "near":
            self.inn = aim.NearOnly(mesh, self.ki, cutoff, quad)
            self._lu = spl.splu(self.inn.NL.tocsc())
            self._Ki = self.inn.NK
        else:
            self.inn = aim.AIM(mesh, self.ki, g, quad)
            n = mesh.ne
            Li = np.zeros((n, n), complex)
            Ki = np.zeros((n, n), complex)
            for c in range(n):
                e = np.zeros(n)
                e[c] = 1.0
                Li[:, c] = self.inn.L(e)
                Ki[:, c] = self.inn.K(e)
            import scipy.linalg as sla
            self._lu_dense = sla.lu_factor(Li)
            self._Ki = Ki

    def with_sibc(self):
        """The same system with the surface impedance condition as its
        interior (the exterior operators shared, not rebuilt)."""
        import copy
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        other = copy.copy(self)
        for name in ("_lu", "_lu_dense", "_Ki", "inn"):
            other.__dict__.pop(name, None)
        other._sibc = eta_medium(self.f, self.eps_r, self.sigma) / ETA0
        other._lu_gram = spl.splu(sp.csc_matrix(mom.gram(self.mesh).astype(complex)))
        return other

    def Z(self, H):
        if hasattr(self, "_sibc"):
            return self._sibc * self._lu_gram.solve(self.Ix @ H)
        rhs = self._Ki @ H - 0.5 * (self.Ix @ H)
        if hasattr(self, "_lu"):
            y = self._lu.solve(rhs)
        else:
            import scipy.linalg as sla
            y = sla.lu_solve(self._lu_dense, rhs)
        return -y / self.zs

    def LA(self, H):
        return self.ext.NLA @ H + grid_LA(self.ext, H)

    def Lphi(self, sig):
        return self.ext.NLphi @ sig + grid_Lphi(self.ext, sig)

    def apply(self, H, c0rho):
        m = self.mesh
        E = self.Z(H)
        r1 = 1j * self.k0 * self.LA(H) - self.ext.K(E) - 0.5 * (self.Ix @ E) \
            + self.D.T @ self.Lphi(-m.area * c0rho)
        r2 = (self.D @ H) / m.area + 1j * self.k0 * c0rho
        return r1, r2


# ---------------------------------------------------------------- several objects
class ObjectsGIBC:
    """Eq. (sys) for several homogeneous objects (Sec. II: N_obj objects, each
    with its own eps_i, sigma_i), exterior operators in their AIM form on one
    grid around all of them; the interior problem of each object couples only
    that object's triangles (Eq. GIBCdef per object), so Z' is block diagonal.
    Interiors: near-region only with each object's 5-skin-depth cutoff, Z'
    by a sparse LU per object, or SIBC.  obj: object index per triangle;
    mats: (eps_r, sigma) per object."""

    def __init__(self, mesh, obj, mats, f, g, interior="near", quad=None):
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        self.mesh, self.f = mesh, f
        self.k0 = 2 * np.pi * f / C0
        self.ext = aim.AIM(mesh, self.k0, g, quad)
        self.Ix = Ix_sparse(mesh)
        self.D = incidence_sparse(mesh)
        obj = np.asarray(obj)
        eobj = obj[mesh.edge_tri[:, 0]]
        self.blocks = []
        for o, (er, sg) in enumerate(mats):
            edges = np.nonzero(eobj == o)[0]
            if interior == "sibc":
                G = sp.csc_matrix(mom.gram(mesh)[np.ix_(edges, edges)].astype(complex))
                self.blocks.append((edges, "sibc", spl.splu(G), eta_medium(f, er, sg) / ETA0, None))
                continue
            ki = k_medium(f, er, sg)
            cut = 5.0 / abs(ki.imag)
            no = near_only_object(mesh, obj, o, ki, cut, quad)
            L = no[0][np.ix_(edges, edges)].tocsc()
            K = no[1][np.ix_(edges, edges)].tocsr()
            self.blocks.append((edges, "near", spl.splu(L), zscale(f, er, sg), K))

    def Z(self, H):
        E = np.zeros_like(H)
        for edges, kind, lu, fac, K in self.blocks:
            Ix = self.Ix[edges][:, edges]
            if kind == "sibc":
                E[edges] = fac * lu.solve(Ix @ H[edges])
            else:
                E[edges] = -lu.solve(K @ H[edges] - 0.5 * (Ix @ H[edges])) / fac
        return E

    def apply(self, H, c0rho):
        m = self.mesh
        E = self.Z(H)
        r1 = 1j * self.k0 * (self.ext.NLA @ H + grid_LA(self.ext, H)) - self.ext.K(E) - 0.5 * (self.Ix @ E) \
            + self.D.T @ (self.ext.NLphi @ (-m.area * c0rho) + grid_Lphi(self.ext, -m.area * c0rho))
        r2 = (self.D @ H) / m.area + 1j * self.k0 * c0rho
        return r1, r2


def near_only_object(mesh, obj, o, k, cutoff, quad=None):
    """Near-region-only interior matrices (L_NR, K_NR, whole-mesh numbering) of
    object o: pairs (t, s) of its triangles that touch or lie within the
    cutoff (the rule of aim.near_pairs_cutoff restricted to the object)."""
    import scipy.sparse as sp
    obj = np.asarray(obj)
    tris = np.nonzero(obj == o)[0]
    pairs = aim.near_pairs_cutoff_of(mesh, cutoff, tris)
    pairs = pairs[obj[pairs[:, 1]] == o]
    L, K, _, _ = aim.exact_local(mesh, complex(k), pairs[:, 0], pairs[:, 1], quad)
    t, s = pairs[:, 0], pairs[:, 1]
    rows = np.repeat(mesh.tri_edge[t], 3, axis=1).ravel()
    cols = np.tile(mesh.tri_edge[s], (1, 3)).ravel()
    sh = (mesh.ne, mesh.ne)
    return (sp.coo_matrix((L.ravel(), (rows, cols)), shape=sh).tocsr(),
            sp.coo_matrix((K.ravel(), (rows, cols)), shape=sh).tocsr())
