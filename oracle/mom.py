"""Dense FP64 Galerkin matrices of the L and K operators (oracle O1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definitions (Sec. II, Eqs. (opL), (opK), (Grrpki); rotated-RWG testing of
n x L[.] and n x K[.] equals RWG testing of the tangential fields):

  L_mn  = II [f_m . f_n - k^-2 (div f_m)(div' f_n)] G dS' dS   (mixed-potential
          Galerkin form of Eq. (opL); the k^-2 grad div term changes sign on
          integration by parts over the closed surface)
  LA_mn = II f_m . f_n G,     Lphi_pq = II_{T_p x T_q} G / (A_p A_q)
  so that L = LA - k^-2 D^T Lphi D  with D the signed edge-length incidence.
  K_mn  = I f_m . PV I grad G x f_n dS' dS                     (Eq. (opK))
  Ix_mn = I f_m . (n x f_n) dS                                  (Sec. II-A)

The near-field integration rule (the paper only says "direct integration")
is fixed by QUAD below and implemented in mom.c.
"""
import ctypes
import os
import subprocess

import numpy as np

from .rwg import Mesh

_here = os.path.dirname(os.path.abspath(__file__))
_so = os.path.join(_here, "_libmom.so")
_lib = None

# near-field quadrature of the method (both triangle-pair classes):
#  pf: far pairs, pf x pf collapsed Gauss points per triangle
#  po: close pairs, outer po x po points; na: angular points per sub-triangle;
#  nr: radial points per panel; npan panels graded by ratio; cf, kres: close test;
#  alen: longest panel of the angular (asinh) variable;
#  touching pairs: outer rule graded toward the shared edge / vertex with opan
#  panels (ratio oratio) of olam points, times omu points across (vertex shared) or
#  2 x emupan graded panels of emu points along a shared edge; the self pair
#  splits the triangle at its centroid and grades toward the three edges
QUAD = dict(pf=5, po=5, na=8, nr=8, npan=5, ratio=0.25, cf=2.0, kres=1.0, alen=1.5,
            opan=7, oratio=0.25, olam=5, omu=6, emupan=2, emu=4)


def build(force=False):
    """Compile mom.c (plain C, OpenMP) into oracle/_libmom.so."""
    src = os.path.join(_here, "mom.c")
    if not force and os.path.exists(_so) and os.path.getmtime(_so) >= os.path.getmtime(src):
        return _so
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", _so, src, "-lm"]
    subprocess.check_call(cmd)
    return _so


def lib():
    global _lib
    if _lib is None:
        build()
        # idle OpenMP workers must not spin: they would starve numpy's BLAS threads
        os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
        L = ctypes.CDLL(_so)
        P = ctypes.c_void_p
        L.om_pair_moments.argtypes = [P, P, P, ctypes.c_long, ctypes.c_double, ctypes.c_double, P, P, P, P]
        L.om_is_close.argtypes = [P, P, P, ctypes.c_long, ctypes.c_double, ctypes.c_double, P, P]
        L.om_inner.argtypes = [P, P, ctypes.c_long, ctypes.c_double, ctypes.c_double, P, P, P, ctypes.c_int, P]
        L.om_dense.argtypes = [P, P, ctypes.c_int, P, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               P, P, P, P, P, P]
        _lib = L
    return _lib


def gl01(n):
    """Gauss-Legendre nodes/weights on [0, 1] (numpy's leggauss, mapped)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _rules(q):
    parts, ns = [], []
    for n in (q["pf"], q["po"], q["na"], q["nr"], q["olam"], q["omu"], q["emu"]):
        x, w = gl01(n)
        parts += [x, w]
        ns.append(n)
    rules = np.ascontiguousarray(np.concatenate(parts))
    rn = np.array(ns, dtype=np.int32)
    par = np.array([q["npan"], q["ratio"], q["cf"], q["kres"], q["alen"], q["opan"], q["oratio"], q["olam"],
                    q["omu"], q["emupan"]], dtype=np.float64)
    return rules, rn, par


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def pair_moments(mesh, pairs, k, quad=None):
    """14 complex moments per ordered triangle pair (t, t'):
    Q0, Q1[3], Q2[3], Q3, U[3], V[3] as defined in mom.c (origin = centroid of t)."""
    q = dict(QUAD, **(quad or {}))
    rules, rn, par = _rules(q)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.zeros((len(pairs), 14), np.complex128)
    k = complex(k)
    lib().om_pair_moments(_p(mesh.V), _p(mesh.T), _p(pairs), len(pairs), k.real, k.imag, _p(rules), _p(rn),
                          _p(par), _p(out))
    return out


def is_close(mesh, pairs, k, quad=None):
    q = dict(QUAD, **(quad or {}))
    _, _, par = _rules(q)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(len(pairs), np.int32)
    k = complex(k)
    lib().om_is_close(_p(mesh.V), _p(mesh.T), _p(pairs), len(pairs), k.real, k.imag, _p(par), _p(out))
    return out.astype(bool)


def inner(tri, pts, k, mode="polar", quad=None):
    """Inner integrals at points over one triangle: (Is, Iv[3], Ig[3]) with
    Is = I G, Iv = I (r'-r) G, Ig = I grad G (principal value at d = 0)."""
    q = dict(QUAD, **(quad or {}))
    rules, rn, par = _rules(q)
    tri = np.ascontiguousarray(tri, dtype=np.float64).reshape(9)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(pts), 7), np.complex128)
    k = complex(k)
    lib().om_inner(_p(tri), _p(pts), len(pts), k.real, k.imag, _p(rules), _p(rn), _p(par),
                   0 if mode == "polar" else 1, _p(out))
    return out


def dense(mesh, k, quad=None, want=("LA", "Lphi", "K")):
    """Dense LA (ne x ne), Lphi (nt x nt), K (ne x ne) over all triangle pairs."""
    q = dict(QUAD, **(quad or {}))
    rules, rn, par = _rules(q)
    ne, nt = mesh.ne, mesh.nt
    LA = np.zeros((ne, ne), np.complex128) if "LA" in want else None
    Lp = np.zeros((nt, nt), np.complex128) if "Lphi" in want else None
    K = np.zeros((ne, ne), np.complex128) if "K" in want else None
    k = complex(k)
    nul = ctypes.c_void_p(0)
    lib().om_dense(_p(mesh.V), _p(mesh.T), nt, _p(mesh.tri_edge), _p(mesh.tri_sign), _p(mesh.tri_free),
                   _p(mesh.edge_len), ne, k.real, k.imag, _p(rules), _p(rn), _p(par),
                   _p(LA) if LA is not None else nul, _p(Lp) if Lp is not None else nul,
                   _p(K) if K is not None else nul)
    return LA, Lp, K


def L_full(mesh, LA, Lphi, k):
    """L = LA - k^-2 D^T Lphi D (mixed-potential form of Eq. (opL))."""
    D = mesh.incidence()
    return LA - (D.T @ Lphi @ D) / (complex(k) ** 2)


def local_entries(mesh, t, s, M, k):
    """3x3 local L and K entries of pair (t, s) from its 14 moments M.
    Rows: slots of t, columns: slots of s.  Returns (L3, K3, LA3)."""
    ct = mesh.centroid[t]
    cm = mesh.coef()[t]
    cn = mesh.coef()[s]
    pm = mesh.V[mesh.tri_free[t]] - ct
    pn = mesh.V[mesh.tri_free[s]] - ct
    Q0, Q1, Q2, Q3, U, Vv = M[0], M[1:4], M[4:7], M[7], M[8:11], M[11:14]
    LA3 = np.zeros((3, 3), complex)
    K3 = np.zeros((3, 3), complex)
    for i in range(3):
        for j in range(3):
            LA3[i, j] = cm[i] * cn[j] * (Q3 - pn[j] @ Q1 - pm[i] @ Q2 + (pm[i] @ pn[j]) * Q0)
            K3[i, j] = cm[i] * cn[j] * ((pn[j] - pm[i]) @ U + np.cross(pn[j], pm[i]) @ Vv)
    L3 = LA3 - 4.0 * np.outer(cm, cn) * Q0 / complex(k) ** 2
    return L3, K3, LA3


def Ix(mesh):
    """Dense I_x of Eqs. (MFIE1dis), (EFIE01dis): (Ix)_mn = I_T f_m . (n x f_n) dS,
    nonzero only when m, n share a triangle.  This orientation is the one for
    which the paper's signs (K_i - Ix/2 inside, K_0 + Ix/2 outside, -E_inc on
    the right) reproduce the Mie series (tests/test_system_oracle.py); the
    opposite orientation gives a 7x wrong RCS.  With origin at the centroid
    (where I (r - c) dS = 0) the integral is closed form:
    c_m c_n A n . ((p_n - c) x (p_m - c))."""
    ne = mesh.ne
    X = np.zeros((ne, ne))
    cf = mesh.coef()
    for t in range(mesh.nt):
        c = mesh.centroid[t]
        p = mesh.V[mesh.tri_free[t]] - c
        for i in range(3):
            for j in range(3):
                val = cf[t, i] * cf[t, j] * mesh.area[t] * (mesh.normal[t] @ np.cross(p[j], p[i]))
                X[mesh.tri_edge[t, i], mesh.tri_edge[t, j]] += val
    return X


def gram(mesh):
    """RWG Gram matrix G_mn = I f_m . f_n dS (dense).  On triangle t with centroid
    c, f_i = c_i (r - p_i) = c_i ((r - c) + (c - p_i)), and I (r - c) dS = 0,
    I |r - c|^2 dS = A (l_1^2 + l_2^2 + l_3^2) / 36, so the 3 x 3 block is
    c_i c_j A [(l_1^2 + l_2^2 + l_3^2) / 36 + (c - p_i).(c - p_j)]."""
    ne = mesh.ne
    G = np.zeros((ne, ne))
    cf = mesh.coef()
    for t in range(mesh.nt):
        c = mesh.centroid[t]
        v = mesh.V[mesh.T[t]]
        l2 = sum(np.sum((v[(i + 1) % 3] - v[i]) ** 2) for i in range(3))
        q = c - mesh.V[mesh.tri_free[t]]
        for i in range(3):
            for j in range(3):
                G[mesh.tri_edge[t, i], mesh.tri_edge[t, j]] += cf[t, i] * cf[t, j] * mesh.area[t] * (l2 / 36.0 + q[i] @ q[j])
    return G
