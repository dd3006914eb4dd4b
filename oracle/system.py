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
