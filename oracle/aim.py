"""CPU FP64 AIM product (oracle O2): Eqs. (AIM_Lin), (AIM_Kin), (LinNRP), (KinNRP).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  L ~ L_NR + W G P + k^-2 W_phi G_phi P_phi - L_P          Eq. (AIM_Lin)
  K ~ K_NR + W G_grad P - K_P                                Eq. (AIM_Kin)

Readings of the parts the paper defers to the pFFT/AIM literature:

* Grid (Sec. III-A, Sec. IV): uniform spacing h, origin
  o = lo - (margin + s) h with s = (1/sqrt2, 1/sqrt3, 1/sqrt5)/2 so that no
  centroid falls on a rounding tie, margin = ceil(M/2) + 1 nodes,
  N_d = floor((hi_d - o_d)/h) + 2 + margin.
* Projection P / interpolation W = P^T by moment matching with tensor
  Lagrange polynomials of order M on the (M+1)^3 stencil nodes of each
  triangle: w0[t,u] = I_t l_u dS, w1[t,u,a] = I_t (r - c_t)_a l_u dS.  The
  stencil centre is round((c_t - o)/h) for even M (floor for odd M).
* Convolution with G sampled at lattice lags, G(0) := 0 and grad G(0) := 0;
  every pair that meets lag 0 is a near pair, so the value cancels.
* Near region: triangle pair (t, s) is near iff the Chebyshev distance of the
  stencil centres is <= R_near (diameter 2 R_near + 1 = 11 grid points for
  R_near = 5, Sec. IV).  The near correction adds, per near triangle pair, the
  direct-integration entries minus the grid's own entries for that pair.
"""
import numpy as np
import scipy.sparse as sp

from . import mom


class Grid:
    def __init__(self, origin, h, N, M, Rnear):
        self.origin = np.asarray(origin, dtype=np.float64)
        self.h = float(h)
        self.N = np.asarray(N, dtype=np.int64)
        self.M = int(M)
        self.Rnear = int(Rnear)

    @property
    def S(self):
        return (self.M + 1) ** 3


def margin_of(M):
    return (M + 1) // 2 + 1


def grid_params(mesh, M=2, Rnear=5, h=None, h_over_edge=0.5, grid_n=None, lam_r=None):
    """Grid of Sec. III-A around the mesh: spacing h (given, or h_over_edge x mean
    edge capped by lambda_r/20 (Sec. IV), or fitted so that the largest
    dimension has grid_n nodes)."""
    V = mesh.V
    lo, hi = V.min(axis=0), V.max(axis=0)
    mg = margin_of(M)
    if h is None:
        if grid_n is not None:
            h = float((hi - lo).max()) / (grid_n - 2 * mg - 3)
        else:
            h = h_over_edge * float(np.sum(mesh.edge_len)) / mesh.ne
            if lam_r is not None:
                h = min(h, lam_r / 20.0)
    s = 0.5 * np.array([1.0 / np.sqrt(2.0), 1.0 / np.sqrt(3.0), 1.0 / np.sqrt(5.0)])
    origin = lo - (mg + s) * h
    N = np.floor((hi - origin) / h).astype(np.int64) + 2 + mg
    return Grid(origin, h, N, M, Rnear)


def stencil_base(mesh, g):
    """Lowest stencil node per triangle (nt, 3) int."""
    x = (mesh.centroid - g.origin) / g.h
    if g.M % 2 == 0:
        c = np.floor(x + 0.5).astype(np.int64)
        base = c - g.M // 2
    else:
        base = np.floor(x).astype(np.int64) - (g.M - 1) // 2
    if base.min() < 0 or np.any(base + g.M > g.N - 1):
        raise ValueError("stencil outside grid")
    return base


def stencil_center(base, g):
    return base + g.M // 2


def lagrange_1d(xi, M):
    """l_j(xi) for nodes 0..M; xi array -> (len, M+1)."""
    xi = np.asarray(xi, dtype=np.float64)
    out = np.ones(xi.shape + (M + 1,))
    for j in range(M + 1):
        for i in range(M + 1):
            if i != j:
                out[..., j] *= (xi - i) / (j - i)
    return out


def tri_rule_pts(mesh, p):
    """Collapsed Gauss-Legendre rule on every triangle: points (nt, q, 3), weights (nt, q)."""
    x, w = mom.gl01(p)
    U, Vv = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    U, Vv, WU, WV = U.ravel(), Vv.ravel(), WU.ravel(), WV.ravel()
    a = mesh.V[mesh.T[:, 0]]
    e1 = mesh.V[mesh.T[:, 1]] - a
    e2 = mesh.V[mesh.T[:, 2]] - a
    pts = a[:, None, :] + U[None, :, None] * e1[:, None, :] + (Vv * (1 - U))[None, :, None] * e2[:, None, :]
    wts = (2.0 * mesh.area)[:, None] * ((1 - U) * WU * WV)[None, :]
    return pts, wts


def weights(mesh, g, base):
    """Moment-matching weights w0 (nt, S), w1 (nt, S, 3); local node index
    u = ux + (M+1) uy + (M+1)^2 uz.  The rule is exact for total degree
    3M + 1 (collapsed Gauss with ceil((3M+3)/2) points per direction)."""
    M = g.M
    p = int(np.ceil((3 * M + 3) / 2.0))
    pts, wts = tri_rule_pts(mesh, p)
    xi = (pts - g.origin) / g.h - base[:, None, :]
    lx = lagrange_1d(xi[..., 0], M)
    ly = lagrange_1d(xi[..., 1], M)
    lz = lagrange_1d(xi[..., 2], M)
    # l_u = lx[ux] ly[uy] lz[uz], u = ux + (M+1)(uy + (M+1) uz)
    lu = np.einsum("tqi,tqj,tqk->tqkji", lx, ly, lz).reshape(mesh.nt, -1, (M + 1) ** 3)
    w0 = np.einsum("tq,tqu->tu", wts, lu)
    rel = pts - mesh.centroid[:, None, :]
    w1 = np.einsum("tq,tqa,tqu->tua", wts, rel, lu)
    return w0, w1


def stencil_nodes(g, base):
    """Global grid index (nt, S) of each stencil node (x fastest)."""
    M = g.M
    o = np.arange(M + 1)
    uz, uy, ux = np.meshgrid(o, o, o, indexing="ij")
    off = np.stack([ux.ravel(), uy.ravel(), uz.ravel()], 1)  # (S, 3), u = ux + (M+1)(uy + (M+1) uz)
    node = base[:, None, :] + off[None]
    Nx, Ny = g.N[0], g.N[1]
    return node[..., 0] + Nx * (node[..., 1] + Ny * node[..., 2]), off


# ---------------------------------------------------------------- kernels
def green_lag(k, h, lag):
    """G and grad G at integer lag vectors (.., 3) times h; both 0 at lag 0."""
    d = h * np.asarray(lag, dtype=np.float64)
    R = np.linalg.norm(d, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.exp(-1j * k * R)
        G = e / (4 * np.pi * R)
        g = -(1 + 1j * k * R) * e / (4 * np.pi * R ** 3)
    z = R == 0
    G = np.where(z, 0.0, G)
    with np.errstate(invalid="ignore"):  # lag 0: g is inf there and is replaced by 0
        gv = np.where(z[..., None], 0.0, g[..., None] * d)
    return G, gv


def conv_direct(src, N, kern):
    """A[u] = sum_v kern(u - v) src[v] by the plain double sum (tiny grids only).
    src (..., Nz, Ny, Nx) flattened x-fastest as (..., Ng); kern(lag) -> value."""
    Nx, Ny, Nz = N
    idx = np.stack(np.meshgrid(np.arange(Nx), np.arange(Ny), np.arange(Nz), indexing="ij"), -1)
    idx = idx.transpose(2, 1, 0, 3).reshape(-1, 3)  # x fastest
    lag = idx[:, None, :] - idx[None, :, :]
    Kmat = kern(lag)
    return np.einsum("uv,...v->...u", Kmat, src)


def conv_fft(src, N, kern):
    """Same linear convolution by circulant embedding on a (2N)^3 lattice and numpy FFTs."""
    Nx, Ny, Nz = (int(v) for v in N)
    n = (2 * Nz, 2 * Ny, 2 * Nx)

    def lag_axis(nn, NN):
        i = np.arange(nn)
        lag = np.where(i < NN, i, i - nn)
        ok = (i < NN) | (i > nn - NN)
        return lag, ok

    lz, oz = lag_axis(n[0], Nz)
    ly, oy = lag_axis(n[1], Ny)
    lx, ox = lag_axis(n[2], Nx)
    LZ, LY, LX = np.meshgrid(lz, ly, lx, indexing="ij")
    lag = np.stack([LX, LY, LZ], -1)
    kv = kern(lag)
    ok = oz[:, None, None] & oy[None, :, None] & ox[None, None, :]
    kv = np.where(ok, kv, 0.0)
    KF = np.fft.fftn(kv)
    shp = src.shape[:-1]
    s = src.reshape(shp + (Nz, Ny, Nx))
    pad = np.zeros(shp + n, complex)
    pad[..., :Nz, :Ny, :Nx] = s
    out = np.fft.ifftn(np.fft.fftn(pad, axes=(-3, -2, -1)) * KF, axes=(-3, -2, -1))
    return out[..., :Nz, :Ny, :Nx].reshape(shp + (Nx * Ny * Nz,))


# ---------------------------------------------------------------- grid product
class AIM:
    """AIM operator of one medium (wavenumber k) on one grid."""

    def __init__(self, mesh, k, g, quad=None, conv="fft", kernel=None, near=True):
        self.mesh, self.k, self.g = mesh, complex(k), g
        self.base = stencil_base(mesh, g)
        self.w0, self.w1 = weights(mesh, g, self.base)
        self.nodes, self.off = stencil_nodes(g, self.base)
        self.coef = mesh.coef()
        self.q = mesh.centroid[:, None, :] - mesh.V[mesh.tri_free]  # (nt, 3 slots, 3): c_t - p
        self.conv = conv
        kk, h = self.k, g.h
        # kern(lag) -> (G, gradG[..., 3]) at integer lags; tests may substitute a
        # polynomial kernel to pin the projection / convolution / interpolation chain
        self.kern = kernel if kernel is not None else (lambda lag: green_lag(kk, h, lag))
        self.kG = lambda lag: self.kern(lag)[0]
        self.kD = [lambda lag, b=b: self.kern(lag)[1][..., b] for b in range(3)]
        self.Ng = int(np.prod(g.N))
        self.near = None
        if near:
            self.pairs = near_pairs(self, g)
            self.build_near(quad)

    # -- projection / interpolation (Eq. AIM_Lin/AIM_Kin: P, P_phi, W, W_phi)
    def _alpha_beta(self, x):
        m = self.mesh
        xe = x[m.tri_edge] * self.coef  # (nt, 3)
        alpha = xe.sum(1)
        beta = np.einsum("ti,tia->ta", xe, self.q)
        return alpha, beta

    def project(self, x):
        """J_a (3, Ng) and rho (Ng,) grid sources of edge coefficients x."""
        alpha, beta = self._alpha_beta(x)
        J = np.zeros((3, self.Ng), complex)
        for a in range(3):
            vals = alpha[:, None] * self.w1[:, :, a] + beta[:, a, None] * self.w0
            np.add.at(J[a], self.nodes.ravel(), vals.ravel())
        rho = np.zeros(self.Ng, complex)
        np.add.at(rho, self.nodes.ravel(), (2.0 * alpha[:, None] * self.w0).ravel())
        return J, rho

    def interpolate(self, A, Phi, scal):
        """y_m = sum_t c_{t,m} [S1_t + (c_t - p_m).T0_t + scal * 2 P0_t]."""
        m = self.mesh
        Ag = A[:, self.nodes]  # (3, nt, S)
        S1 = np.einsum("tua,atu->t", self.w1, Ag)
        T0 = np.einsum("tu,atu->ta", self.w0, Ag)
        val = S1[:, None] + np.einsum("tia,ta->ti", self.q, T0)
        if Phi is not None:
            P0 = np.einsum("tu,tu->t", self.w0, Phi[self.nodes])
            val = val + scal * 2.0 * P0[:, None]
        val = val * self.coef
        y = np.zeros(m.ne, complex)
        np.add.at(y, m.tri_edge.ravel(), val.ravel())
        return y

    def _conv(self, src, kern):
        f = conv_fft if self.conv == "fft" else conv_direct
        return f(src, self.g.N, kern)

    def grid_L(self, x):
        """W G P x + k^-2 W_phi G_phi P_phi x (Eq. AIM_Lin without near terms)."""
        J, rho = self.project(x)
        A = self._conv(J, self.kG)
        Phi = self._conv(rho, self.kG)
        return self.interpolate(A, Phi, -1.0 / self.k ** 2)

    def grid_K(self, x):
        """W G_grad P x (Eq. AIM_Kin without near terms): A_a = eps_abc dG_b * J_c."""
        J, _ = self.project(x)
        D = [[self._conv(J[c], self.kD[b]) for c in range(3)] for b in range(3)]
        A = np.zeros_like(J)
        for a, b, c, s in ((0, 1, 2, 1), (0, 2, 1, -1), (1, 2, 0, 1), (1, 0, 2, -1), (2, 0, 1, 1), (2, 1, 0, -1)):
            A[a] += s * D[b][c]
        return self.interpolate(A, None, 0.0)

    # -- near region (Eqs. LinNRP, KinNRP)
    def grid_local(self, t, s):
        """The grid's own 3x3 L and K entries for pairs (t[i], s[i]) (precorrection L_P, K_P)."""
        off = self.off
        lag = (self.base[t][:, None, None, :] + off[None, :, None, :]) - (self.base[s][:, None, None, :] + off[None, None, :, :])
        # near pairs only meet lags with |lag_d| <= R_near + M: tabulate once
        if getattr(self, "_lagtab", None) is None:
            Lm = self.g.Rnear + self.g.M
            ax = np.arange(-Lm, Lm + 1)
            LZ, LY, LX = np.meshgrid(ax, ax, ax, indexing="ij")
            self._lagtab = (Lm,) + tuple(self.kern(np.stack([LX, LY, LZ], -1)))
        Lm, Gt, Dt = self._lagtab
        ix, iy, iz = lag[..., 0] + Lm, lag[..., 1] + Lm, lag[..., 2] + Lm
        G = Gt[iz, iy, ix]  # (np, S, S)
        Dg = [Dt[..., b][iz, iy, ix] for b in range(3)]  # 3 x (np, S, S), contiguous for matmul
        n = len(t)
        S = off.shape[0]
        # P^a_{t,i}[u] = c_{t,i} (w1[t,u,a] + q_{t,i,a} w0[t,u]);  P^phi_{t,i}[u] = 2 c_{t,i} w0[t,u]
        def Pmat(x):
            P = self.coef[x][:, :, None, None] * (self.w1[x][:, None, :, :] + self.q[x][:, :, None, :] * self.w0[x][:, None, :, None])
            P = P.transpose(0, 2, 1, 3).reshape(n, S, 9)  # column = 3 slot + comp
            Ph = 2.0 * self.coef[x][:, None, :] * self.w0[x][:, :, None]  # (n, S, 3)
            return np.concatenate([P, Ph], axis=2)  # (n, S, 12)
        Xt, Xs = Pmat(t), Pmat(s)
        XtT = np.ascontiguousarray(Xt.transpose(0, 2, 1))
        Xs = np.ascontiguousarray(Xs)
        Y = XtT @ (G @ Xs)  # (n, 12, 12)
        Yv = Y[:, :9, :9].reshape(n, 3, 3, 3, 3)  # (i, a, j, c)
        LA = np.einsum("piaja->pij", Yv)
        Lph = Y[:, 9:, 9:]
        L = LA - Lph / self.k ** 2
        K = np.zeros_like(L)
        Xs9 = np.ascontiguousarray(Xs[:, :, :9])
        XtT9 = np.ascontiguousarray(XtT[:, :9, :])
        Z = [(XtT9 @ (Dg[b] @ Xs9)).reshape(n, 3, 3, 3, 3) for b in range(3)]
        for a, b, c, sg in ((0, 1, 2, 1), (0, 2, 1, -1), (1, 2, 0, 1), (1, 0, 2, -1), (2, 0, 1, 1), (2, 1, 0, -1)):
            K += sg * Z[b][:, :, a, :, c]
        Lphi = np.einsum("pu,puv,pv->p", self.w0[t], G, self.w0[s], optimize=True) / (self.mesh.area[t] * self.mesh.area[s])
        return L, K, LA, Lphi

    def exact_local(self, t, s, quad=None):
        return exact_local(self.mesh, self.k, t, s, quad)

    def build_near(self, quad=None, chunk=256):
        m = self.mesh
        t, s = self.pairs[:, 0], self.pairs[:, 1]
        rows, cols, vL, vK, vLA, vLp = [], [], [], [], [], []
        for i0 in range(0, len(t), chunk):
            tt, ss = t[i0:i0 + chunk], s[i0:i0 + chunk]
            Le, Ke, LAe, Lpe = self.exact_local(tt, ss, quad)
            Lg, Kg, LAg, Lpg = self.grid_local(tt, ss)
            vL.append((Le - Lg).ravel())
            vK.append((Ke - Kg).ravel())
            vLA.append((LAe - LAg).ravel())
            vLp.append(Lpe - Lpg)
            rows.append(np.repeat(m.tri_edge[tt], 3, axis=1).ravel())
            cols.append(np.tile(m.tri_edge[ss], (1, 3)).ravel())
        r, c = np.concatenate(rows), np.concatenate(cols)
        sh = (m.ne, m.ne)
        self.NL = sp.coo_matrix((np.concatenate(vL), (r, c)), shape=sh).tocsr()
        self.NK = sp.coo_matrix((np.concatenate(vK), (r, c)), shape=sh).tocsr()
        self.NLA = sp.coo_matrix((np.concatenate(vLA), (r, c)), shape=sh).tocsr()
        self.NLphi = sp.coo_matrix((np.concatenate(vLp), (t, s)), shape=(m.nt, m.nt)).tocsr()

    # -- full AIM products
    def L(self, x):
        return self.NL @ x + self.grid_L(x)

    def K(self, x):
        return self.NK @ x + self.grid_K(x)


def exact_local(m, k, t, s, quad=None):
    """Direct-integration 3x3 entries of pairs (t[i], s[i]) from the oracle moments:
    returns L, K, LA (np, 3, 3) and Lphi (np,)."""
    k = complex(k)
    Mo = mom.pair_moments(m, np.stack([t, s], 1), k, quad)
    coef = m.coef()
    ct = m.centroid[t]
    cm, cn = coef[t], coef[s]
    pm = m.V[m.tri_free[t]] - ct[:, None, :]
    pn = m.V[m.tri_free[s]] - ct[:, None, :]
    Q0, Q1, Q2, Q3, U, Vv = Mo[:, 0], Mo[:, 1:4], Mo[:, 4:7], Mo[:, 7], Mo[:, 8:11], Mo[:, 11:14]
    LA = Q3[:, None, None] - np.einsum("pja,pa->pj", pn, Q1)[:, None, :] - np.einsum("pia,pa->pi", pm, Q2)[:, :, None] \
        + np.einsum("pia,pja->pij", pm, pn) * Q0[:, None, None]
    cc = cm[:, :, None] * cn[:, None, :]
    LA = cc * LA
    L = LA - 4.0 * cc * Q0[:, None, None] / k ** 2
    dl = pn[:, None, :, :] - pm[:, :, None, :]
    cx = np.cross(pn[:, None, :, :], pm[:, :, None, :])
    K = cc * (np.einsum("pija,pa->pij", dl, U) + np.einsum("pija,pa->pij", cx, Vv))
    Lphi = Q0 / (m.area[t] * m.area[s])
    return L, K, LA, Lphi


def near_pairs_cutoff(m, cutoff):
    """Interior skin-depth rule (Sec. V): keep the ordered pair (t, s) iff the
    triangles touch or the gap |c_t - c_s| - R_t - R_s is <= cutoff (R = farthest
    vertex from the centroid).  Sorted by (t, s).  Brute force (small meshes)."""
    c = m.centroid
    R = np.linalg.norm(m.V[m.T] - c[:, None, :], axis=2).max(1)
    out = []
    Tset = [set(tt) for tt in m.T.tolist()]
    for t in range(m.nt):
        gap = np.sqrt(((c - c[t]) ** 2).sum(1)) - R - R[t]
        cand = np.nonzero(gap <= cutoff)[0].tolist()
        touch = [s for s in range(m.nt) if Tset[t] & Tset[s]]
        for s in sorted(set(cand) | set(touch)):
            out.append((t, s))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


class NearOnly:
    """Interior operator when every pair kept by the skin-depth cutoff is a
    near pair (Sec. III-C): L = L_NR, K = K_NR, no grid."""

    def __init__(self, mesh, k, cutoff, quad=None, chunk=256):
        self.mesh, self.k = mesh, complex(k)
        self.pairs = near_pairs_cutoff(mesh, cutoff)
        t, s = self.pairs[:, 0], self.pairs[:, 1]
        rows, cols, vL, vK = [], [], [], []
        for i0 in range(0, len(t), chunk):
            tt, ss = t[i0:i0 + chunk], s[i0:i0 + chunk]
            L, K, _, _ = exact_local(mesh, self.k, tt, ss, quad)
            vL.append(L.ravel())
            vK.append(K.ravel())
            rows.append(np.repeat(mesh.tri_edge[tt], 3, axis=1).ravel())
            cols.append(np.tile(mesh.tri_edge[ss], (1, 3)).ravel())
        r, c = np.concatenate(rows), np.concatenate(cols)
        sh = (mesh.ne, mesh.ne)
        self.NL = sp.coo_matrix((np.concatenate(vL), (r, c)), shape=sh).tocsr()
        self.NK = sp.coo_matrix((np.concatenate(vK), (r, c)), shape=sh).tocsr()

    def L(self, x):
        return self.NL @ x

    def K(self, x):
        return self.NK @ x


def near_pairs(aim, g):
    """All ordered (t, s) with Chebyshev distance of stencil centres <= R_near,
    sorted by t then s (integer rule; bit-exact)."""
    c = stencil_center(aim.base, g)
    R = g.Rnear
    # bucket by centre cell
    from collections import defaultdict
    buckets = defaultdict(list)
    for i, cc in enumerate(map(tuple, c)):
        buckets[cc].append(i)
    out = []
    rng = range(-R, R + 1)
    for t in range(len(c)):
        ct = c[t]
        lst = []
        for dz in rng:
            for dy in rng:
                for dx in rng:
                    b = buckets.get((ct[0] + dx, ct[1] + dy, ct[2] + dz))
                    if b:
                        lst.extend(b)
        lst.sort()
        out.extend((t, s) for s in lst)
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def kappa(A, B):
    """Matrix error metric of Sec. IV: max|A - B| / max|A|."""
    return np.abs(A - B).max() / np.abs(A).max()


# ---------------------------------------------------------------- sampled rows (large meshes)
def near_pairs_of(aim, g, tris):
    """The near pairs (t, s) of the AIM rule (Chebyshev distance of stencil
    centres <= R_near) for the test triangles t in `tris` only, sorted."""
    c = stencil_center(aim.base, g)
    out = []
    for t in sorted(set(int(v) for v in tris)):
        d = np.abs(c - c[t]).max(axis=1)
        out.extend((t, int(s)) for s in np.nonzero(d <= g.Rnear)[0])
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def near_pairs_cutoff_of(m, cutoff, tris):
    """near_pairs_cutoff restricted to the test triangles in `tris`."""
    c = m.centroid
    R = np.linalg.norm(m.V[m.T] - c[:, None, :], axis=2).max(1)
    out = []
    for t in sorted(set(int(v) for v in tris)):
        gap = np.sqrt(((c - c[t]) ** 2).sum(1)) - R - R[t]
        touch = np.isin(m.T, m.T[t]).any(axis=1)
        out.extend((t, int(s)) for s in np.nonzero((gap <= cutoff) | touch)[0])
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def _assemble_rows(m, rows, pairs, local):
    """Dense rows (len(rows), ne) of an edge matrix from 3x3 local blocks of
    triangle pairs: entry (m, n) sums block[i, j] over pairs (t, s) with edge m
    in slot i of t and edge n in slot j of s."""
    out = np.zeros((len(rows), m.ne), complex)
    pos = {int(r): i for i, r in enumerate(rows)}
    for p, (t, s) in enumerate(pairs):
        for i in range(3):
            r = pos.get(int(m.tri_edge[t, i]))
            if r is None:
                continue
            for j in range(3):
                out[r, m.tri_edge[s, j]] += local[p, i, j]
    return out


def near_rows(A, rows, quad=None):
    """Rows of the precorrected exterior near matrices (NL, NK) of AIM operator
    A for the edges in `rows` (exact local entries minus the grid's own)."""
    m = A.mesh
    tris = m.edge_tri[np.asarray(rows)].ravel()
    pairs = near_pairs_of(A, A.g, tris)
    t, s = pairs[:, 0], pairs[:, 1]
    Le, Ke, _, _ = exact_local(m, A.k, t, s, quad)
    Lg, Kg, _, _ = A.grid_local(t, s)
    return _assemble_rows(m, rows, pairs, Le - Lg), _assemble_rows(m, rows, pairs, Ke - Kg)


def near_only_rows(m, k, cutoff, rows, quad=None):
    """Rows of the near-region-only interior matrices (L_NR, K_NR) for `rows`."""
    tris = m.edge_tri[np.asarray(rows)].ravel()
    pairs = near_pairs_cutoff_of(m, cutoff, tris)
    L, K, _, _ = exact_local(m, complex(k), pairs[:, 0], pairs[:, 1], quad)
    return _assemble_rows(m, rows, pairs, L), _assemble_rows(m, rows, pairs, K)
