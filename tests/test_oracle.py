"""Pins of the oracle against things other than itself (closed forms, brute force,
invariants, the paper's worked example).  CPU only."""
import os
from math import factorial

import numpy as np
import pytest

from oracle import aim, bounds, mie, mom
from oracle.rwg import Mesh
from synth import cn_vector, icosphere

C0 = 299792458.0
K0_3GHZ = 2 * np.pi * 3e9 / C0
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _equilateral(a=1.0):
    return np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * np.sqrt(3) / 2, 0]], dtype=np.float64)


def _brute(tri, r, k, levels=5, n=8):
    """Brute-force inner integrals: 4^levels sub-triangles x n^2 collapsed Gauss."""
    x, w = mom.gl01(n)
    tris = [tri]
    for _ in range(levels):
        nt = []
        for t in tris:
            A, B, C = t
            ab, bc, ca = (A + B) / 2, (B + C) / 2, (C + A) / 2
            nt += [np.array([A, ab, ca]), np.array([ab, B, bc]), np.array([ca, bc, C]), np.array([ab, bc, ca])]
        tris = nt
    T = np.array(tris)
    U, Vv = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    U, Vv, W0 = U.ravel(), Vv.ravel(), ((1 - U) * WU * WV).ravel()
    e1, e2 = T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]
    twoA = np.linalg.norm(np.cross(e1, e2), axis=1)
    P = T[:, None, 0] + U[None, :, None] * e1[:, None] + (Vv * (1 - U))[None, :, None] * e2[:, None]
    W = twoA[:, None] * W0[None]
    d = P - r
    R = np.linalg.norm(d, axis=-1)
    e = np.exp(-1j * k * R)
    G = e / (4 * np.pi * R)
    g = -(1 + 1j * k * R) * e / (4 * np.pi * R ** 3)
    Is = (W * G).sum()
    Iv = np.einsum("tq,tqa->a", W * G, d)
    Ig = np.einsum("tq,tqa->a", W * g, -d)
    return np.concatenate([[Is], Iv, Ig])


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("p", [3, 5, 6])
def test_collapsed_rule_exact_monomials(p):
    """Collapsed Gauss p x p on the unit right triangle integrates x^a y^b exactly
    (a! b! / (a+b+2)!) for a + b <= 2p - 2."""
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    m = Mesh(np.vstack([tri, [[0, 0, -1]]]), np.array([[0, 1, 2], [0, 3, 1], [1, 3, 2], [2, 3, 0]]))
    pts, wts = aim.tri_rule_pts(m, p)
    for a in range(2 * p - 1):
        for b in range(2 * p - 1 - a):
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            got = np.sum(wts[0] * pts[0, :, 0] ** a * pts[0, :, 1] ** b)
            assert abs(got - exact) < 1e-14, (a, b)


# ------------------------------------------------------------------ inner integrals
def test_static_potential_closed_form():
    ref = float(open(os.path.join(GOLD, "equilateral_static_potential.txt")).read().split("\n")[-2])
    tri = _equilateral()
    o = mom.inner(tri, [tri.mean(0)], 1e-12)
    assert abs(4 * np.pi * o[0, 0].real - ref) < 1e-13


@pytest.mark.parametrize("r,k", [((0.3, 0.2, 0.25), 2.0), ((0.3, 0.2, 0.6), 0.3), ((0.5, 0.3, 0.05), 5.0 - 1.0j),
                                 ((1.3, 0.4, 0.1), 3.0), ((0.5, -0.1, 0.0), 1.0), ((0.45, 0.25, -0.02), 0.5),
                                 ((1.1, 0.3, 0.05), 1.5)])
def test_inner_polar_vs_brute_force(r, k):
    """Polar inner integration (mom.c) vs brute-force subdivision at points off
    the source triangle (both the series and the panel radial branches)."""
    tri = _equilateral()
    r = np.array(r)
    b = _brute(tri, r, k, levels=6)
    p = mom.inner(tri, [r], k)[0]
    assert np.abs(p - b).max() / np.abs(b).max() < 1e-8


@pytest.mark.parametrize("d", [0.0, 1e-3, -3e-3])
def test_inner_lossy_half_space_limit(d):
    """|k| size >> 1 (skin depth << triangle): over a point well inside, the
    triangle acts as the whole plane, where I G dS' = exp(-jk|d|)/(2jk),
    I dG/dn dS' = -sign(d) exp(-jk|d|)/2 and I (r'-r).n G dS' = -d exp(-jk|d|)/(2jk)."""
    tri = _equilateral()
    k = (1 - 1j) * 200.0
    p = mom.inner(tri, [[0.5, 0.3, d]], k)[0]
    e = np.exp(-1j * k * abs(d))
    assert abs(p[0] - e / (2j * k)) < 1e-8 * abs(e / (2j * k))
    assert abs(p[3] - (-d * e / (2j * k))) < 1e-8 * abs(e / (2j * k)) + 1e-20
    assert abs(p[6] - (-0.5 * np.sign(d) * e)) < 1e-10
    assert max(abs(p[1]), abs(p[2]), abs(p[4]), abs(p[5])) < 1e-7


def test_polar_matches_gauss_far():
    """Far from the triangle the smooth product rule is accurate: both agree."""
    tri = _equilateral()
    for r in ([2.5, 1.0, 0.7], [-1.5, 2.0, -1.0]):
        a = mom.inner(tri, [r], 1.2, mode="polar")[0]
        b = mom.inner(tri, [r], 1.2, mode="gauss")[0]
        assert np.abs(a - b).max() / np.abs(b).max() < 1e-9


# ------------------------------------------------------------------ RWG + dense operators
@pytest.fixture(scope="module")
def sphere2():
    V, T = icosphere(2, 0.01)
    m = Mesh(V, T)
    LA, Lp, K = mom.dense(m, K0_3GHZ)
    return m, LA, Lp, K


def test_rwg_table():
    V, T = icosphere(2, 1.0)
    m = Mesh(V, T)
    assert m.ne == 3 * m.nt // 2
    D = m.incidence()
    # total divergence of every RWG function vanishes: l_n - l_n = 0
    assert np.abs(D.sum(axis=0)).max() < 1e-14
    # every edge is + on one triangle, - on the other
    assert np.all(np.bincount(m.tri_edge[m.tri_sign > 0], minlength=m.ne) == 1)
    assert np.all(np.bincount(m.tri_edge[m.tri_sign < 0], minlength=m.ne) == 1)


def test_dense_reciprocity(sphere2):
    """Reciprocity of G (Eq. Grecip) makes L and K complex symmetric; Ix is
    antisymmetric.  The residual asymmetry is the quadrature error."""
    m, LA, Lp, K = sphere2
    L = mom.L_full(m, LA, Lp, K0_3GHZ)
    asym = lambda A: np.abs(A - A.T).max() / np.abs(A).max()
    assert asym(L) < 2e-6
    assert asym(Lp) < 2e-6
    assert asym(K) < 2e-4
    X = mom.Ix(m)
    assert np.abs(X + X.T).max() == 0.0


def test_quadrature_refinement(sphere2):
    """Near-field moments converge under refinement of every quadrature knob."""
    m, _, _, _ = sphere2
    pairs = np.array([[0, s] for s in range(m.nt)])
    close = mom.is_close(m, pairs, K0_3GHZ)
    pairs = pairs[close]
    a = mom.pair_moments(m, pairs, K0_3GHZ)
    b = mom.pair_moments(m, pairs, K0_3GHZ, dict(po=7, na=12, nr=10, opan=9, olam=6, omu=8, pf=7, emu=5, emupan=3))
    rel = np.abs(a - b).max(axis=0) / np.abs(b).max(axis=0)
    assert rel[:8].max() < 1e-5  # L moments
    assert rel[8:].max() < 1e-4  # K moments (edge-adjacent pairs limit)


# ------------------------------------------------------------------ AIM machinery
def test_weights_moment_matching():
    """Sum_u w0[t,u] p(r_u) = I_t p dS for every monomial of degree <= M per axis."""
    V, T = icosphere(2, 0.01)
    m = Mesh(V, T)
    for M in (1, 2, 3):
        g = aim.grid_params(m, M=M)
        base = aim.stencil_base(m, g)
        w0, w1 = aim.weights(m, g, base)
        _, off = aim.stencil_nodes(g, base)
        node = (base[:, None, :] + off[None]) * g.h + g.origin
        pts, wts = aim.tri_rule_pts(m, 8)
        x0 = m.centroid[:, None, :]
        for e in [(0, 0, 0), (1, 0, 0), (M, M, M), (M, 0, M), (1, M, 0)]:
            # monomials in (r - c_t)/h keep every term O(1) (no cancellation)
            mono = lambda p: (((p - x0) / g.h) ** np.array(e)).prod(-1)
            lhs = (w0 * mono(node)).sum(1)
            rhs = (wts * mono(pts)).sum(1)
            # exact values can vanish (I (r - c) dS = 0): scale by area and area*h
            assert np.abs(lhs - rhs).max() <= 1e-12 * m.area.max()
            lhs1 = np.einsum("tu,tua->ta", mono(node), w1)
            rhs1 = np.einsum("tq,tqa->ta", wts * mono(pts), pts - m.centroid[:, None, :])
            assert np.abs(lhs1 - rhs1).max() <= 1e-12 * m.area.max() * g.h


def test_fft_convolution_equals_direct():
    rng = np.random.default_rng(3)
    N = np.array([5, 4, 6])
    src = rng.standard_normal((2, N.prod())) + 1j * rng.standard_normal((2, N.prod()))
    for kern in (lambda lag: aim.green_lag(3.0 - 0.5j, 0.1, lag)[0], lambda lag: aim.green_lag(2.0, 0.1, lag)[1][..., 1]):
        a = aim.conv_direct(src, N, kern)
        b = aim.conv_fft(src, N, kern)
        assert np.abs(a - b).max() / np.abs(a).max() < 1e-13


def _poly_kernel(h):
    """A kernel polynomial of degree <= 2 per axis in (r - r')/h, and its gradient."""
    def p(u):
        x, y, z = u[..., 0], u[..., 1], u[..., 2]
        val = 1.0 + 0.3 * x - 0.2 * y * z + 0.1 * x * x * y + 0.05 * x * y * z * z - 0.07 * z * z
        gx = 0.3 + 0.2 * x * y + 0.05 * y * z * z
        gy = -0.2 * z + 0.1 * x * x + 0.05 * x * z * z
        gz = -0.2 * y + 0.1 * x * y * z - 0.14 * z
        return val, np.stack([gx, gy, gz], -1) / h
    return p


def test_polynomial_kernel_grid_product_is_exact():
    """With a kernel polynomial of degree <= M per axis, moment matching makes
    W G P exact: the grid product equals the direct double integral (no near
    correction).  Pins projection, FFT convolution, interpolation, the vector
    (P) and scalar (P_phi) paths and the curl assembly of G_grad."""
    V, T = icosphere(1, 1.0)
    m = Mesh(V, T)
    g = aim.grid_params(m, M=2)
    p = _poly_kernel(g.h)
    kern = lambda lag: p(np.asarray(lag, dtype=float))
    k = 1.7 - 0.2j
    A = aim.AIM(m, k, g, kernel=kern, near=False)
    x = cn_vector(m.ne, 5)
    # direct double integral with an exact product rule
    pts, wts = aim.tri_rule_pts(m, 6)
    cf = m.coef()
    Lx = np.zeros(m.ne, complex)
    Kx = np.zeros(m.ne, complex)
    for t in range(m.nt):
        d = (pts[t][:, None, None, :] - pts[:, None, :, :].transpose(1, 0, 2, 3)) / g.h  # (q, s, q', 3)
        val, grad = p(d)
        fm = cf[t][:, None, None] * (pts[t][None] - m.V[m.tri_free[t]][:, None, :])  # (3 slots, q, 3)
        fn = cf[:, :, None, None] * (pts[:, None, :, :] - m.V[m.tri_free][:, :, None, :])  # (s, 3, q', 3)
        xn = x[m.tri_edge]  # (s, 3)
        Jn = np.einsum("sj,sjqa->sqa", xn, fn)  # source current at source points
        divn = 2.0 * (xn * cf).sum(1)  # (s,)
        w = wts[t][:, None, None] * wts[None, :, :]  # (q, s, q')
        pot = np.einsum("qsr,qsr,sra->qa", w, val, Jn)
        phi = np.einsum("qsr,qsr,s->q", w, val, divn)
        for i in range(3):
            Lx[m.tri_edge[t, i]] += np.sum(fm[i] * pot) - (2.0 * cf[t, i]) * phi.sum() / k ** 2
        curl = np.einsum("qsr,qsrb,src->qbc", w, grad, Jn)  # I grad_b P J_c
        e = np.zeros((3, 3, 3))
        e[0, 1, 2] = e[1, 2, 0] = e[2, 0, 1] = 1
        e[0, 2, 1] = e[2, 1, 0] = e[1, 0, 2] = -1
        cr = np.einsum("abc,qbc->qa", e, curl)
        for i in range(3):
            Kx[m.tri_edge[t, i]] += np.sum(fm[i] * cr)
    gL = A.grid_L(x)
    gK = A.grid_K(x)
    assert np.linalg.norm(gL - Lx) / np.linalg.norm(Lx) < 1e-12
    assert np.linalg.norm(gK - Kx) / np.linalg.norm(Kx) < 1e-12


@pytest.mark.parametrize("kfac", [1.0, 2.0])
def test_aim_matvec_vs_dense(sphere2, kfac):
    """AIM product (Eqs. AIM_Lin, AIM_Kin with near correction) vs the dense
    direct-integration matrices: relative 2-norm error <= 1e-3, and the matrix
    error kappa of Sec. IV on a random column block."""
    m, LA, Lp, K = sphere2
    k = K0_3GHZ * kfac
    if kfac != 1.0:
        LA, Lp, K = mom.dense(m, k)
    L = mom.L_full(m, LA, Lp, k)
    g = aim.grid_params(m, M=2)
    A = aim.AIM(m, k, g)
    x = cn_vector(m.ne, 11)
    eL = np.linalg.norm(A.L(x) - L @ x) / np.linalg.norm(L @ x)
    eK = np.linalg.norm(A.K(x) - K @ x) / np.linalg.norm(K @ x)
    assert eL < 1e-3 and eK < 1e-3, (eL, eK)
    cols = np.arange(0, m.ne, 37)
    AL = np.stack([A.L(np.eye(m.ne)[c]) for c in cols], 1)
    assert aim.kappa(L[:, cols], AL) < 1e-3


def test_near_pairs_rule():
    V, T = icosphere(2, 0.01)
    m = Mesh(V, T)
    g = aim.grid_params(m, M=2)
    A = aim.AIM(m, K0_3GHZ, g, near=False)
    P = aim.near_pairs(A, g)
    c = aim.stencil_center(A.base, g)
    cheb = np.abs(c[:, None, :] - c[None, :, :]).max(-1)
    ref = np.argwhere(cheb <= g.Rnear)
    assert np.array_equal(P, ref)


# ------------------------------------------------------------------ paper's worked example
def test_interpolation_bound_worked_example():
    line = [l for l in open(os.path.join(GOLD, "interp_bound_n2.txt")) if not l.startswith("#")][0].split()
    n, rmax, th0, s0 = int(line[0]), float(line[1]), float(line[2]), float(line[3])
    got, th, s = bounds.max_lossy_ratio(n)
    assert abs(got - rmax) < 1e-3
    assert abs(th - th0) < 2e-3
    assert abs(bounds.lossy_ratio(n, th0, s0) - rmax) < 1e-3
    # the flat maximum in s: the paper's s = 2.894 is within 2% of ours
    assert abs(s - s0) / s0 < 0.02


def test_interpolation_bound_is_derivative():
    """D_n is the (n+1)-th theta-derivative of exp(-j theta sqrt(1 - j s))/theta (Eq. Ddef)."""
    sp = pytest.importorskip("sympy")
    th = sp.symbols("theta", positive=True)
    for n in (1, 2, 3):
        for s in (0.0, 2.894, 50.0):
            f = sp.exp(-sp.I * th * sp.sqrt(1 - sp.I * s)) / th
            ref = complex(sp.diff(f, th, n + 1).subs(th, 1.3).evalf(30))
            assert abs(bounds.D(n, 1.3, s) - ref) < 1e-13 * abs(ref)


# ------------------------------------------------------------------ Mie
def test_mie_rayleigh_limit():
    a, f = 1e-3, 1e9
    k = 2 * np.pi * f / C0
    for er, s in ((4.0, 0.0), (2.5, 0.1)):
        m2 = er - 1j * s / (2 * np.pi * f * mie.EPS0)
        ray = 4 * np.pi * k ** 4 * a ** 6 * abs((m2 - 1) / (m2 + 2)) ** 2
        assert abs(mie.backscatter_rcs(a, f, er, s) / ray - 1) < 2e-4


def test_mie_identities():
    x = 3.0
    A, B = mie.coefficients(x, 1.7)
    n = np.arange(1, len(A) + 1)
    qext = 2 / x ** 2 * np.sum((2 * n + 1) * (A + B).real)
    qsca = 2 / x ** 2 * np.sum((2 * n + 1) * (abs(A) ** 2 + abs(B) ** 2))
    assert abs(qext - qsca) < 1e-12 * qext  # lossless: no absorption
    assert abs(mie.backscatter_rcs(0.01, 3e9, 4.0) - mie.bistatic_rcs(np.pi, 0.0, 0.01, 3e9, 4.0)[0]) < 1e-12
    # a good conductor approaches the PEC limit
    pec = mie.backscatter_rcs(1e-3, 10e9, pec=True)
    cu = mie.backscatter_rcs(1e-3, 10e9, 1.0, 5.8e7)
    assert abs(cu / pec - 1) < 2e-3


# ------------------------------------------------------------------ touching pairs: independent rule
# tests/touching_quadrature.py integrates the same 14 moments by relative
# coordinates and Duffy cone maps (no polar inner integration, no graded outer
# rule), so it shares no step with the oracle's near-field rule (mom.c).
import sys  # noqa: E402

sys.path.insert(0, os.path.dirname(__file__))
import touching_quadrature as tq  # noqa: E402

# the oracle's rule with every knob refined well past the defaults
REFINED = dict(po=9, na=16, nr=16, opan=14, olam=10, omu=10, emu=8, emupan=4, npan=12, alen=0.75)


def test_touching_rule_static_self_similarity():
    """For the kernel 1/R (homogeneous of degree -1) the self term of a triangle
    equals twice the sum of the touching child pairs of its midpoint subdivision
    (the four self terms are each 1/8 of the parent's): ties the identical,
    edge-adjacent and vertex-adjacent branches together; plus convergence in n."""
    A, B, C = np.array([0, 0, 0.0]), np.array([1, 0, 0.0]), np.array([0.4, 0.8, 0.0])
    V = np.array([A, B, C, (A + B) / 2, (B + C) / 2, (C + A) / 2])
    T = np.array([(0, 3, 5), (3, 1, 4), (5, 4, 2), (4, 5, 3)])
    k = 1e-14
    parent = tq.self_moments(A, B, C, k, n=16)[0]
    kids = sum(tq.touching_moments(V, T, i, j, k, n=16)[0] for i in range(4) for j in range(4) if i != j)
    assert abs(2 * kids - parent) <= 1e-12 * abs(parent)
    for s in range(1, 4):
        a = tq.touching_moments(V, T, 0 if s != 3 else 3, s if s != 3 else 0, 5.0 - 5.0j, n=12)
        b = tq.touching_moments(V, T, 0 if s != 3 else 3, s if s != 3 else 0, 5.0 - 5.0j, n=18)
        assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()


def _touching_case(kl):
    V, T = icosphere(2, 1.0)
    m = Mesh(V, T)
    t = 5
    nb = [s for s in range(m.nt) if len(set(T[t]) & set(T[s])) > 0]
    lbar = m.edge_len.mean()
    k = (kl / np.sqrt(2)) * (1 - 1j) / lbar if kl > 1 else kl / lbar
    ref = np.array([tq.touching_moments(V, T, t, s, k, n=14) for s in nb])
    return m, t, nb, k, ref


def _touching_errors(m, t, nb, k, ref, quad):
    got = mom.pair_moments(m, np.array([[t, s] for s in nb]), k, quad)
    eQ = max(np.abs(got[i, :8] - ref[i, :8]).max() / np.abs(ref[i, :8]).max() for i in range(len(nb)))
    # self pair: U = V = 0 (antisymmetric integrands), compared on the other pairs
    eK = max(np.abs(got[i, 8:] - ref[i, 8:]).max() / np.abs(ref[i, 8:]).max() for i, s in enumerate(nb) if s != t)
    return eQ, eK


# lighter refinement for the copper regime (more outer points per graded panel
# and along the shared edge, more radial points): the dominant knobs there
REFINED_LOSSY = dict(olam=10, emu=8, nr=12)


@pytest.mark.parametrize("kl,quad,tol_ref,tol_def", [(0.2, REFINED, (1e-10, 5e-8), (2e-6, 3e-5)),
                                                     (80.0, REFINED_LOSSY, (5e-6, 1e-4), (5e-3, 6e-3))],
                         ids=["lossless", "copper"])
def test_oracle_touching_moments_vs_independent_rule(kl, quad, tol_ref, tol_def):
    """All 14 moments of the self, 3 edge-adjacent and 9 vertex-adjacent pairs of
    one triangle: (a) the oracle's rule with refined knobs converges to the
    independent relative-coordinate rule (a wrong sign, index or term in either
    would not); (b) the error of the default knobs, |k| l = 0.2 (lossless) and
    |k| l = 80 with Im k = -Re k (copper at 10 GHz on 38 um edges): Q moments
    (L operators) and U, V (K operator)."""
    m, t, nb, k, ref = _touching_case(kl)
    eQ, eK = _touching_errors(m, t, nb, k, ref, quad)
    assert eQ <= tol_ref[0] and eK <= tol_ref[1], (eQ, eK)
    eQ, eK = _touching_errors(m, t, nb, k, ref, None)
    print(f"default rule |k|l={kl}: Q {eQ:.2e} K {eK:.2e}")
    assert eQ <= tol_def[0] and eK <= tol_def[1], (eQ, eK)


# ------------------------------------------------------------------ Mie: plain definition at high precision
def _mie_plain(x, m, nmax, dps=60):
    """a_n, b_n from their definition with Riccati-Bessel functions
    psi_n(z) = z j_n(z), xi_n(z) = z h_n^(1)(z) evaluated in mpmath (no
    logarithmic-derivative recurrence)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    x = mp.mpf(x)
    m = mp.mpc(m.real, m.imag)
    z = m * x

    def jn(n, u):
        return mp.sqrt(mp.pi / (2 * u)) * mp.besselj(n + mp.mpf(1) / 2, u)

    def yn(n, u):
        return mp.sqrt(mp.pi / (2 * u)) * mp.bessely(n + mp.mpf(1) / 2, u)

    def psi(n, u):
        return u * jn(n, u)

    def dpsi(n, u):  # d/du [u j_n(u)] = u j_{n-1}(u) - n j_n(u)
        return u * jn(n - 1, u) - n * jn(n, u)

    def xi(n, u):
        return u * (jn(n, u) + 1j * yn(n, u))

    def dxi(n, u):
        return u * (jn(n - 1, u) + 1j * yn(n - 1, u)) - n * (jn(n, u) + 1j * yn(n, u))

    a, b = [], []
    for n in range(1, nmax + 1):
        pz, dpz, px, dpx, xx, dxx = psi(n, z), dpsi(n, z), psi(n, x), dpsi(n, x), xi(n, x), dxi(n, x)
        a.append(complex((m * pz * dpx - px * dpz) / (m * pz * dxx - xx * dpz)))
        b.append(complex((pz * dpx - m * px * dpz) / (pz * dxx - m * xx * dpz)))
    return np.array(a), np.array(b)


@pytest.mark.parametrize("x,eps_r,sigma_over_weps0", [(0.6283, 4.0, 0.0), (3.0, 2.25, 0.3), (0.2096, 1.0, 1.043e8)],
                         ids=["dielectric", "lossy", "copper"])
def test_mie_coefficients_vs_plain_definition(x, eps_r, sigma_over_weps0):
    """The oracle's a_n, b_n (downward log-derivative recurrence, scipy Bessel
    functions) equal the Bohren-Huffman definition evaluated at 60 digits,
    including the copper case where |m x| is about 2e3."""
    m = np.sqrt(eps_r + 1j * sigma_over_weps0 + 0j)
    a, b = mie.coefficients(x, m)
    pa, pb = _mie_plain(x, m, len(a))
    assert np.abs(a - pa).max() <= 1e-11 * np.abs(pa).max()
    assert np.abs(b - pb).max() <= 1e-11 * np.abs(pb).max()


def test_mie_angular_functions_low_orders():
    """S1, S2 with only a_1 or b_1 or a_2 or b_2 set: (3/2) pi_1 = 3/2,
    (3/2) tau_1 = (3/2) cos t, (5/6) pi_2 = (5/2) cos t, (5/6) tau_2 = (5/2) cos 2t."""
    th = np.linspace(0.0, np.pi, 7)
    c = np.cos(th)
    cases = [((1, 0), (0, 0), 1.5 * np.ones_like(th), 1.5 * c), ((0, 0), (1, 0), 1.5 * c, 1.5 * np.ones_like(th)),
             ((0, 1), (0, 0), 2.5 * c, 2.5 * np.cos(2 * th)), ((0, 0), (0, 1), 2.5 * np.cos(2 * th), 2.5 * c)]
    for a, b, s1, s2 in cases:
        S1, S2 = mie.amplitudes(th, 1.0, np.array(a, complex), np.array(b, complex))
        assert np.abs(S1 - s1).max() < 1e-14 and np.abs(S2 - s2).max() < 1e-14
