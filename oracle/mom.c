/*
 * oracle/mom.c -- plain FP64 CPU reference for the Galerkin RWG operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this code.  It shares no source with
 * the CUDA library.
 *
 * What it computes (Sharma & Triverio, Sec. II, Eqs. (opL), (opK), (Grrpki)):
 *   G(R)   = exp(-j k R) / (4 pi R)                                 Eq. (Grrpki)
 *   grad G = g(R) (r - r'),  g(R) = -(1 + j k R) exp(-j k R) / (4 pi R^3)
 * and, for every ordered triangle pair (t test, t' source), the moments
 *   Q0 = II G,  Q1 = II rt G,  Q2 = II rt' G,  Q3 = II rt.rt' G,
 *   U  = II g (rt x rt'),  V = II g (r - r'),
 * with rt = r - c_t, rt' = r' - c_t (c_t = centroid of the test triangle) and
 * II = double surface integral over t (outer, r) and t' (inner, r').
 * The Galerkin entries of Eq. (opL) in mixed-potential form and of Eq. (opK)
 * tested with RWG functions (equivalently rotated-RWG testing of n x L, n x K)
 * follow from these moments; see oracle/mom.py for the assembly formulas.
 *
 * Quadrature (the method's near-field integration rule; the paper leaves it
 * open):
 *   - "far" pairs: collapsed Gauss-Legendre product rule, pf x pf points on
 *     each triangle;
 *   - "close" pairs (shared vertex, centroid distance < cf (R_t + R_t'), or
 *     |k| (R_t + R_t') > kres): outer collapsed rule po x po on t, inner
 *     integral by polar integration about the projection of r onto the plane
 *     of t', split into three signed sub-triangles; the angular variable of
 *     each sub-triangle is integrated in s = asinh(tangential / height); the
 *     radial integrals of the 1/R and static gradient parts are closed forms,
 *     the bounded remainders use Gauss-Legendre on geometrically graded
 *     panels.  The principal value of Eq. (opK) drops the solid-angle term at
 *     d = 0, and the self pair (t == t') contributes U = V = 0 (flat
 *     triangle: (r - r') and rt x rt' are orthogonal to the test function).
 * Gauss-Legendre nodes are supplied by the caller (numpy's leggauss).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define PI 3.14159265358979323846
#define RCUT 36.0 /* exp(-36) < 1e-15 */

typedef struct {
    const double *x, *w;
    int n;
} rule1d;

typedef struct {
    rule1d far, out, ang, rad, olaml, omul, emul;
    int npan;
    double pan_ratio, cf, kres, ang_len;
    int opan, olam, omu, emupan;
    double oratio;
} qparams;

static void sub3(const double *a, const double *b, double *c) { c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* (exp(z) - 1) / z */
static cplx phi1(cplx z)
{
    if (cabs(z) < 0.5) {
        cplx term = 1.0, s = 1.0;
        for (int n = 1; n < 20; n++) {
            term *= z / (double)(n + 1);
            s += term;
        }
        return s;
    }
    return (cexp(z) - 1.0) / z;
}

/* (1 + z) exp(-z) - 1, z = j k R; series near 0 avoids cancellation */
static cplx hfun(cplx z)
{
    if (cabs(z) < 0.2) {
        cplx s = 0.0, zn = z; /* zn = z^n */
        double fact = 1.0;
        for (int n = 2; n < 16; n++) {
            zn *= z;
            fact *= n;
            double sgn = (n % 2 == 0) ? -1.0 : 1.0; /* (-1)^(n+1) */
            s += sgn * (double)(n - 1) * zn / fact;
        }
        return s;
    }
    return (1.0 + z) * cexp(-z) - 1.0;
}

/* Collapsed Gauss rule on triangle (a,b,c): point a + u (b-a) + v (1-u)(c-a),
 * weight 2A (1-u) wu wv.  Returns the number of points. */
static int tri_rule(const double *a, const double *b, const double *c, const rule1d *r,
                    double *pts, double *wts)
{
    double e1[3], e2[3], nn[3];
    sub3(b, a, e1);
    sub3(c, a, e2);
    cross3(e1, e2, nn);
    double twoA = norm3(nn);
    int k = 0;
    for (int i = 0; i < r->n; i++) {
        double u = r->x[i];
        for (int j = 0; j < r->n; j++) {
            double v = r->x[j] * (1.0 - u);
            for (int d = 0; d < 3; d++) pts[3 * k + d] = a[d] + u * e1[d] + v * e2[d];
            wts[k] = twoA * (1.0 - u) * r->w[i] * r->w[j];
            k++;
        }
    }
    return k;
}


/* Outer rule for touching pairs, graded toward the shared feature.
 * r = apex + lam ((b - apex) + mu (c - b)), dS = 2A lam dlam dmu.
 * toward_edge = 1: the edge b-c is shared, panels in lam graded toward 1;
 * toward_edge = 0: the apex is shared, panels graded toward 0.
 * lam uses opan geometric panels (ratio oratio) of olam Gauss points; mu uses
 * omu Gauss points when the apex is shared, and when the edge is shared
 * emupan panels per half graded toward both shared vertices (emu points each). */
static int mu_rule(const qparams *qp, int graded, double *mx, double *mw)
{
    /* plain omu-point rule, or panels graded geometrically toward both ends */
    int n = 0;
    if (!graded) {
        for (int j = 0; j < qp->omul.n; j++) {
            mx[n] = qp->omul.x[j];
            mw[n++] = qp->omul.w[j];
        }
        return n;
    }
    for (int side = 0; side < 2; side++) {
        double hi = 0.5;
        for (int p = 0; p < qp->emupan; p++) {
            double lo = (p == qp->emupan - 1) ? 0.0 : hi * qp->oratio;
            for (int j = 0; j < qp->emul.n; j++) {
                double s = lo + (hi - lo) * qp->emul.x[j];
                mx[n] = side ? 1.0 - s : s;
                mw[n++] = (hi - lo) * qp->emul.w[j];
            }
            hi = lo;
        }
    }
    return n;
}

static int tri_rule_graded(const double *apex, const double *b, const double *c, int toward_edge,
                           int graded_mu, const qparams *qp, const rule1d *rl, const rule1d *rm,
                           double *pts, double *wts)
{
    double mx[256], mw[256];
    int nmu = mu_rule(qp, graded_mu, mx, mw);
    (void)rm;
    double e1[3], e2[3], nn[3];
    sub3(b, apex, e1);
    sub3(c, b, e2);
    cross3(e1, e2, nn);
    double twoA = norm3(nn);
    int k = 0;
    double hi = 1.0;
    for (int p = 0; p < qp->opan; p++) {
        double lo = (p == qp->opan - 1) ? 0.0 : hi * qp->oratio;
        for (int i = 0; i < rl->n; i++) {
            double sg = lo + (hi - lo) * rl->x[i]; /* distance-like variable from the feature */
            double wsg = (hi - lo) * rl->w[i];
            double lam = toward_edge ? 1.0 - sg : sg;
            for (int j = 0; j < nmu; j++) {
                double mu = mx[j];
                for (int d = 0; d < 3; d++) pts[3 * k + d] = apex[d] + lam * (e1[d] + mu * e2[d]);
                wts[k] = twoA * lam * wsg * mw[j];
                k++;
            }
        }
        hi = lo;
    }
    return k;
}

/* Inner integrals at observation point r over a source triangle:
 *   Is = I G dS',  Iv = I (r' - r) G dS',  Ig = I g (r - r') dS' (= I grad G). */
typedef struct {
    cplx Is, Iv[3], Ig[3];
} inner_t;

static void inner_gauss(const double *r, const double *ipts, const double *iw, int ni, cplx k,
                        inner_t *o)
{
    memset(o, 0, sizeof(*o));
    for (int q = 0; q < ni; q++) {
        double dv[3];
        sub3(ipts + 3 * q, r, dv); /* r' - r */
        double R = norm3(dv);
        cplx e = cexp(-I * k * R);
        cplx G = e / (4.0 * PI * R);
        cplx g = -(1.0 + I * k * R) * e / (4.0 * PI * R * R * R);
        o->Is += iw[q] * G;
        for (int d = 0; d < 3; d++) {
            o->Iv[d] += iw[q] * dv[d] * G;
            o->Ig[d] += iw[q] * g * (-dv[d]);
        }
    }
}


/* Ein(z) = I_0^z (1 - exp(-t))/t dt, Re z >= 0: power series for |z| < 2,
 * otherwise E1(z) + log z + Euler's gamma with E1 from its continued
 * fraction e^-z / (z + 1/(1 + 1/(z + 2/(1 + 2/(z + ...))))) (modified Lentz). */
static cplx ein(cplx z)
{
    if (cabs(z) < 2.0) {
        cplx s = 0.0, t = 1.0;
        for (int n = 1; n < 60; n++) {
            t *= z / (double)n; /* z^n / n! */
            cplx term = ((n % 2) ? 1.0 : -1.0) * t / (double)n;
            s += term;
            if (cabs(term) < 1e-17 * cabs(s)) break;
        }
        return s;
    }
    /* Lentz on b0 + a1/(b1 + a2/(b2 + ...)) with b = z, 1, z, 1, ... and
     * a = 1, 1, 1, 2, 2, 3, 3, ... */
    const double tiny = 1e-300;
    cplx f = z, C = z, D = 0.0;
    for (int i = 1; i < 500; i++) {
        double a = (double)((i + 1) / 2);
        cplx b = (i % 2) ? 1.0 : z;
        D = b + a * D;
        if (cabs(D) < tiny) D = tiny;
        C = b + a / C;
        if (cabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        cplx delta = C * D;
        f *= delta;
        if (cabs(delta - 1.0) < 1e-16) break;
    }
    const double euler = 0.57721566490153286061;
    return cexp(-z) / f + clog(z) + euler;
}

/* Bounded radial remainders of the polar scheme at one angle:
 *   f1 = I_0^rhom rho^2 exp(-jkR)/R drho,
 *   f2 = I_0^rhom rho^2 [(1 + jkR) exp(-jkR) - 1]/R^3 drho,   R^2 = rho^2 + d^2.
 * If |k| Rmax <= 1 both are summed from the Taylor series of exp(-jkR), whose
 * terms need A_m = I rho^2 R^m drho = B_{m+2} - d^2 B_m with
 * B_m = I R^m drho = (rhom Rm^m + m d^2 B_{m-2}) / (m + 1), B_0 = rhom,
 * B_-1 = asinh(rhom/|d|) (only ever needed times d^2, which is 0 at d = 0).
 * Lengths are scaled by Rmax.  Otherwise Gauss-Legendre on npan panels graded
 * geometrically toward rho = 0, over rho <= RCUT/|Im k| (closed-form tail). */
static void radial(cplx k, double rhom, double d, double Rmax, const qparams *qp, cplx *f1, cplx *f2)
{
    if (cabs(k) * Rmax <= 1.0) {
        double rs = rhom / Rmax, ds = d / Rmax, Rs = sqrt(rs * rs + ds * ds), d2 = ds * ds;
        cplx ks = k * Rmax;
        enum { NT = 26 };
        double B[NT + 4]; /* B[m + 1], m = -1 .. NT + 2 */
        B[0] = (d2 > 0.0) ? d2 * asinh(rs / fabs(ds)) : 0.0; /* d^2 B_-1 */
        B[1] = rs;                                          /* B_0 */
        double Rp = 1.0;                                    /* Rs^m */
        double Bodd_prev = 0.0; /* d^2 B_{m-2} for odd m */
        double Beven_prev = rs; /* B_{m-2} for even m */
        for (int m = 1; m <= NT + 2; m++) {
            Rp *= Rs;
            double bm;
            if (m % 2 == 1) {
                double d2Bm2 = (m == 1) ? B[0] : d2 * Bodd_prev;
                bm = (rs * Rp + m * d2Bm2) / (m + 1);
                Bodd_prev = bm;
            } else {
                bm = (rs * Rp + m * d2 * Beven_prev) / (m + 1);
                Beven_prev = bm;
            }
            B[m + 1] = bm;
        }
        /* A_m for m = -1 .. NT: A_-1 = B_1 - d^2 B_-1 */
        double A[NT + 2];
        A[0] = B[2] - B[0];
        for (int m = 0; m <= NT; m++) A[m + 1] = B[m + 3] - d2 * B[m + 1];
        cplx s1 = 0.0, s2 = 0.0, t1 = 1.0; /* t1 = (-j ks)^n / n! */
        for (int n = 0; n <= NT; n++) {
            if (n > 0) t1 *= -I * ks / (double)n;
            s1 += t1 * A[n]; /* A_{n-1} */
            if (n >= 2) {
                /* (-1)^(n+1) (n-1) (j ks)^n / n! = -(n-1) (-j ks)^n / n! */
                s2 += -(double)(n - 1) * t1 * A[n - 2]; /* A_{n-3} */
            }
        }
        *f1 = s1 * Rmax * Rmax;
        *f2 = s2;
        return;
    }
    if (d == 0.0) {
        /* coplanar point: closed forms, z = j k rhom:
         * f1 = I rho exp(-jk rho) drho, f2 = 1 - exp(-z) - Ein(z) */
        cplx z = I * k * rhom, e = cexp(-z);
        *f1 = (1.0 - e * (1.0 + z)) / ((I * k) * (I * k));
        *f2 = 1.0 - e - ein(z);
        return;
    }
    /* beyond R = RCUT/|Im k| the exponential is below 1e-15: there f1 has no
     * contribution and (1 + jkR) exp(-jkR) - 1 = -1, whose integral is the
     * static closed form S = log(rho + R) - rho/R */
    double rc = rhom, tail = 0.0;
    double kim = fabs(cimag(k));
    if (kim > 0.0) {
        double Rc = RCUT / kim, Rm = sqrt(rhom * rhom + d * d);
        if (Rc < Rm) {
            rc = Rc > fabs(d) ? sqrt(Rc * Rc - d * d) : 0.0;
            double Rcc = sqrt(rc * rc + d * d);
            tail = (log(rhom + Rm) - rhom / Rm) - (log(rc + Rcc) - rc / Rcc);
        }
    }
    cplx a1 = 0, a2 = 0;
    double hi = rc;
    for (int p = 0; p < qp->npan && rc > 0.0; p++) {
        double lo = (p == qp->npan - 1) ? 0.0 : hi * qp->pan_ratio;
        for (int q = 0; q < qp->rad.n; q++) {
            double rho = lo + (hi - lo) * qp->rad.x[q];
            double wr = (hi - lo) * qp->rad.w[q];
            double R = sqrt(rho * rho + d * d);
            cplx z = I * k * R;
            cplx e = cexp(-z);
            cplx hz = cabs(z) < 0.2 ? hfun(z) : (1.0 + z) * e - 1.0;
            a1 += wr * rho * rho * e / R;
            a2 += wr * rho * rho * hz / (R * R * R);
        }
        hi = lo;
    }
    a2 -= tail;
    *f1 = a1;
    *f2 = a2;
}

static void inner_polar(const double *r, const double *v0, const double *v1, const double *v2,
                        cplx k, const qparams *qp, inner_t *o)
{
    const double *vv[3] = {v0, v1, v2};
    double e1[3], e2[3], nrm[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, nrm);
    double nn = norm3(nrm);
    for (int d = 0; d < 3; d++) nrm[d] /= nn;
    double rv0[3];
    sub3(r, v0, rv0);
    double dd = dot3(rv0, nrm);
    double rho0[3];
    for (int d = 0; d < 3; d++) rho0[d] = r[d] - dd * nrm[d];

    double Rmax = 0.0, Rmin = 1e300; /* farthest / nearest vertex */
    for (int i = 0; i < 3; i++) {
        double dv[3];
        sub3(vv[i], r, dv);
        double rr = norm3(dv);
        if (rr > Rmax) Rmax = rr;
        if (rr < Rmin) Rmin = rr;
    }
    if (fabs(dd) < 1e-12 * Rmax) dd = 0.0; /* on the plane up to rounding */
    double ad = fabs(dd);
    memset(o, 0, sizeof(*o));
    /* whole triangle beyond RCUT/|Im k|: every term below exp(-RCUT) */
    double kim = fabs(cimag(k));
    if (kim > 0.0) {
        double c[3] = {(v0[0] + v1[0] + v2[0]) / 3.0, (v0[1] + v1[1] + v2[1]) / 3.0, (v0[2] + v1[2] + v2[2]) / 3.0};
        double rc = 0.0, dc[3];
        for (int i = 0; i < 3; i++) {
            double dv[3];
            sub3(vv[i], c, dv);
            double q = norm3(dv);
            if (q > rc) rc = q;
        }
        sub3(r, c, dc);
        if (norm3(dc) - rc > RCUT / kim) return;
    }
    cplx Is = 0, Iv[3] = {0, 0, 0}, Ign = 0, Igt[3] = {0, 0, 0};
    double Omega = 0.0;
    for (int i = 0; i < 3; i++) {
        const double *A = vv[i], *B = vv[(i + 1) % 3];
        double e[3], et[3], m[3], Ar[3], Br[3];
        sub3(B, A, e);
        double L = norm3(e);
        for (int d = 0; d < 3; d++) et[d] = e[d] / L;
        cross3(et, nrm, m); /* outward in-plane normal of edge i */
        sub3(A, rho0, Ar);
        sub3(B, rho0, Br);
        double h = dot3(Ar, m);
        if (fabs(h) < 1e-12 * L) continue;
        double sh = h > 0 ? 1.0 : -1.0, ah = fabs(h);
        double u[3];
        for (int d = 0; d < 3; d++) u[d] = sh * m[d];
        double ta = dot3(Ar, et), tb = dot3(Br, et);
        Omega += sh * (atan2(tb, ah) - atan2(ta, ah));
        double sa = asinh(ta / ah), sb = asinh(tb / ah);
        /* composite rule in s: panels no longer than ang_len */
        int npa = (int)ceil((sb - sa) / qp->ang_len);
        if (npa < 1) npa = 1;
        double ds = (sb - sa) / npa;
        for (int j = 0; j < qp->ang.n * npa; j++) {
            int jp = j / qp->ang.n, jq = j % qp->ang.n;
            double s = sa + ds * (jp + qp->ang.x[jq]);
            double ch = cosh(s);
            double wa = sh * ds * qp->ang.w[jq] / ch; /* d alpha = ds / cosh s */
            double ca = 1.0 / ch, sn = tanh(s);
            double eh[3];
            for (int d = 0; d < 3; d++) eh[d] = u[d] * ca + et[d] * sn;
            double rhom = ah * ch;
            double Rm = sqrt(rhom * rhom + dd * dd);
            /* closed form: I_0^rhom exp(-jkR)/R rho drho = I_|d|^Rm exp(-jkR) dR */
            cplx is = cexp(-I * k * ad) * (Rm - ad) * phi1(-I * k * (Rm - ad));
            cplx f1, f2;
            radial(k, rhom, dd, Rmax, qp, &f1, &f2);
            /* I_0^rhom rho^2/R^3 drho = asinh(rhom/|d|) - rhom/Rm; the
             * alpha-independent -log|d| cancels over the signed sub-triangles */
            cplx igt = log(rhom + Rm) - rhom / Rm + f2;
            cplx ign = -dd * cexp(-I * k * Rm) / Rm;
            Is += wa * is;
            Ign += wa * ign;
            for (int d = 0; d < 3; d++) {
                Iv[d] += wa * (eh[d] * f1 - dd * nrm[d] * is);
                Igt[d] += wa * eh[d] * igt;
            }
        }
    }
    cplx jump = 0.0;
    if (dd != 0.0) jump = Omega * (dd > 0 ? 1.0 : -1.0) * cexp(-I * k * ad);
    o->Is = Is / (4.0 * PI);
    for (int d = 0; d < 3; d++) {
        o->Iv[d] = Iv[d] / (4.0 * PI);
        o->Ig[d] = -(nrm[d] * (jump + Ign) - Igt[d]) / (4.0 * PI);
    }
}

static void centroid(const double *V, const int *t, double *c)
{
    for (int d = 0; d < 3; d++) c[d] = (V[3 * t[0] + d] + V[3 * t[1] + d] + V[3 * t[2] + d]) / 3.0;
}

static double radius(const double *V, const int *t, const double *c)
{
    double R = 0;
    for (int i = 0; i < 3; i++) {
        double dv[3];
        sub3(V + 3 * t[i], c, dv);
        double r = norm3(dv);
        if (r > R) R = r;
    }
    return R;
}

static int is_close(const double *V, const int *t, const int *s, cplx k, const qparams *qp)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (t[i] == s[j]) return 1;
    double ct[3], cs[3], dv[3];
    centroid(V, t, ct);
    centroid(V, s, cs);
    double Rt = radius(V, t, ct), Rs = radius(V, s, cs);
    sub3(ct, cs, dv);
    double D = norm3(dv);
    if (D < qp->cf * (Rt + Rs)) return 1;
    if (cabs(k) * (Rt + Rs) > qp->kres) return 1;
    return 0;
}

/* moments of one ordered pair; out = 14 complex: Q0, Q1[3], Q2[3], Q3, U[3], V[3] */
static void pair_moments(const double *V, const int *T, int t, int s, cplx k, const qparams *qp,
                         cplx *out)
{
    const int *tt = T + 3 * t, *ss = T + 3 * s;
    const double *a = V + 3 * tt[0], *b = V + 3 * tt[1], *c = V + 3 * tt[2];
    const double *a2 = V + 3 * ss[0], *b2 = V + 3 * ss[1], *c2 = V + 3 * ss[2];
    double ct[3];
    centroid(V, tt, ct);
    int close = is_close(V, tt, ss, k, qp);
    const rule1d *ro = close ? &qp->out : &qp->far;
    /* shared vertices decide the outer rule of touching pairs */
    int shared[3], nsh = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (tt[i] == ss[j]) shared[nsh++] = i;
    int no = ro->n * ro->n;
    int nmu = qp->omul.n > 2 * qp->emupan * qp->emul.n ? qp->omul.n : 2 * qp->emupan * qp->emul.n;
    int ng = 3 * qp->opan * qp->olaml.n * nmu;
    if (ng > no) no = ng;
    double *op = malloc(sizeof(double) * 3 * no), *ow = malloc(sizeof(double) * no);
    if (t != s && nsh == 2) {
        int ia = 3 - shared[0] - shared[1]; /* the vertex of t not on the shared edge */
        no = tri_rule_graded(V + 3 * tt[ia], V + 3 * tt[(ia + 1) % 3], V + 3 * tt[(ia + 2) % 3], 1, 1, qp,
                             &qp->olaml, &qp->omul, op, ow);
    } else if (t != s && nsh == 1) {
        int ia = shared[0];
        no = tri_rule_graded(V + 3 * tt[ia], V + 3 * tt[(ia + 1) % 3], V + 3 * tt[(ia + 2) % 3], 0, 0, qp,
                             &qp->olaml, &qp->omul, op, ow);
    } else if (t == s) {
        /* self pair: three sub-triangles from the centroid, graded toward the edges */
        no = 0;
        for (int i = 0; i < 3; i++)
            no += tri_rule_graded(ct, V + 3 * tt[i], V + 3 * tt[(i + 1) % 3], 1, 1, qp, &qp->olaml,
                                  &qp->omul, op + 3 * no, ow + no);
    } else {
        no = tri_rule(a, b, c, ro, op, ow);
    }
    int ni = qp->far.n * qp->far.n;
    double *ip = malloc(sizeof(double) * 3 * ni), *iw = malloc(sizeof(double) * ni);
    tri_rule(a2, b2, c2, &qp->far, ip, iw);
    memset(out, 0, 14 * sizeof(cplx));
    for (int q = 0; q < no; q++) {
        const double *r = op + 3 * q;
        inner_t in;
        if (close)
            inner_polar(r, a2, b2, c2, k, qp, &in);
        else
            inner_gauss(r, ip, iw, ni, k, &in);
        double rt[3];
        sub3(r, ct, rt);
        double w = ow[q];
        cplx I2[3];
        for (int d = 0; d < 3; d++) I2[d] = in.Iv[d] + rt[d] * in.Is;
        out[0] += w * in.Is;
        for (int d = 0; d < 3; d++) {
            out[1 + d] += w * rt[d] * in.Is;
            out[4 + d] += w * I2[d];
        }
        out[7] += w * (rt[0] * I2[0] + rt[1] * I2[1] + rt[2] * I2[2]);
        if (t != s) {
            /* U += -w rt x Ig ; V += w Ig */
            out[8] += -w * (rt[1] * in.Ig[2] - rt[2] * in.Ig[1]);
            out[9] += -w * (rt[2] * in.Ig[0] - rt[0] * in.Ig[2]);
            out[10] += -w * (rt[0] * in.Ig[1] - rt[1] * in.Ig[0]);
            for (int d = 0; d < 3; d++) out[11 + d] += w * in.Ig[d];
        }
    }
    free(op);
    free(ow);
    free(ip);
    free(iw);
}

static void load_params(const double *rules, const int *rn, const double *par, qparams *qp)
{
    const double *p = rules;
    rule1d *rr[7] = {&qp->far, &qp->out, &qp->ang, &qp->rad, &qp->olaml, &qp->omul, &qp->emul};
    for (int i = 0; i < 7; i++) {
        rr[i]->n = rn[i];
        rr[i]->x = p;
        rr[i]->w = p + rn[i];
        p += 2 * rn[i];
    }
    qp->npan = (int)par[0];
    qp->pan_ratio = par[1];
    qp->cf = par[2];
    qp->kres = par[3];
    qp->ang_len = par[4];
    qp->opan = (int)par[5];
    qp->oratio = par[6];
    qp->olam = (int)par[7];
    qp->omu = (int)par[8];
    qp->emupan = (int)par[9];
}

/* rules = [x_far, w_far, x_out, w_out, x_ang, w_ang, x_rad, w_rad] (GL on [0,1]);
 * rn = their sizes; par = [npan, pan_ratio, cf, kres]. */
int om_pair_moments(const double *V, const int *T, const int *pairs, long npairs, double kr,
                    double ki, const double *rules, const int *rn, const double *par, double *out)
{
    qparams qp;
    load_params(rules, rn, par, &qp);
    cplx k = kr + I * ki;
#pragma omp parallel for schedule(dynamic, 16)
    for (long p = 0; p < npairs; p++)
        pair_moments(V, T, pairs[2 * p], pairs[2 * p + 1], k, &qp, (cplx *)(out + 28 * p));
    return 0;
}

int om_is_close(const double *V, const int *T, const int *pairs, long npairs, double kr, double ki,
                const double *par, int *out)
{
    qparams qp;
    memset(&qp, 0, sizeof(qp));
    qp.cf = par[2];
    qp.kres = par[3];
    cplx k = kr + I * ki;
    for (long p = 0; p < npairs; p++)
        out[p] = is_close(V, T + 3 * pairs[2 * p], T + 3 * pairs[2 * p + 1], k, &qp);
    return 0;
}

/* Inner integrals alone (for pinning against closed forms / brute force):
 * out = 7 complex per point: Is, Iv[3], Ig[3]. mode 0 = polar, 1 = Gauss. */
int om_inner(const double *tri9, const double *pts, long npts, double kr, double ki,
             const double *rules, const int *rn, const double *par, int mode, double *out)
{
    qparams qp;
    load_params(rules, rn, par, &qp);
    cplx k = kr + I * ki;
    int ni = qp.far.n * qp.far.n;
    double *ip = malloc(sizeof(double) * 3 * ni), *iw = malloc(sizeof(double) * ni);
    tri_rule(tri9, tri9 + 3, tri9 + 6, &qp.far, ip, iw);
    for (long q = 0; q < npts; q++) {
        inner_t in;
        if (mode == 0)
            inner_polar(pts + 3 * q, tri9, tri9 + 3, tri9 + 6, k, &qp, &in);
        else
            inner_gauss(pts + 3 * q, ip, iw, ni, k, &in);
        cplx *o = (cplx *)(out + 14 * q);
        o[0] = in.Is;
        for (int d = 0; d < 3; d++) {
            o[1 + d] = in.Iv[d];
            o[4 + d] = in.Ig[d];
        }
    }
    free(ip);
    free(iw);
    return 0;
}

/* Dense Galerkin matrices over all triangle pairs.
 * tri_edge/tri_sign/tri_free: per triangle, per local slot i (edge opposite
 * local vertex i): RWG edge index, +1/-1 (T+ / T-), free vertex index.
 * edge_len: RWG edge lengths.  Outputs (row-major, complex as re/im pairs):
 *   LA   ne x ne : II f_m . f_n G
 *   Lphi nt x nt : II G / (A_p A_q)
 *   K    ne x ne : I f_m . PV I grad G x f_n
 * Any output pointer may be NULL. */
int om_dense(const double *V, const int *T, int nt, const int *tri_edge, const int *tri_sign,
             const int *tri_free, const double *edge_len, int ne, double kr, double ki,
             const double *rules, const int *rn, const double *par, double *LA, double *Lphi,
             double *K)
{
    qparams qp;
    load_params(rules, rn, par, &qp);
    cplx k = kr + I * ki;
    cplx *la = (cplx *)LA, *lp = (cplx *)Lphi, *kk = (cplx *)K;
    double *area = malloc(sizeof(double) * nt);
    for (int t = 0; t < nt; t++) {
        double e1[3], e2[3], c[3];
        sub3(V + 3 * T[3 * t + 1], V + 3 * T[3 * t], e1);
        sub3(V + 3 * T[3 * t + 2], V + 3 * T[3 * t], e2);
        cross3(e1, e2, c);
        area[t] = 0.5 * norm3(c);
    }
    /* parallel over test triangles; rows of an edge receive contributions from
     * both of its triangles, so accumulate per test triangle into private
     * buffers and add them in a fixed order afterwards */
    cplx *mom = malloc(sizeof(cplx) * 14 * (size_t)nt * nt);
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nt; t++)
        for (int s = 0; s < nt; s++) pair_moments(V, T, t, s, k, &qp, mom + 14 * ((size_t)t * nt + s));
    for (int t = 0; t < nt; t++) {
        double ct[3];
        centroid(V, T + 3 * t, ct);
        for (int s = 0; s < nt; s++) {
            const cplx *M = mom + 14 * ((size_t)t * nt + s);
            if (lp) lp[(size_t)t * nt + s] = M[0] / (area[t] * area[s]);
            for (int i = 0; i < 3; i++) {
                int m = tri_edge[3 * t + i];
                double cm = tri_sign[3 * t + i] * edge_len[m] / (2.0 * area[t]);
                double pm[3];
                sub3(V + 3 * tri_free[3 * t + i], ct, pm);
                for (int j = 0; j < 3; j++) {
                    int n = tri_edge[3 * s + j];
                    double cn = tri_sign[3 * s + j] * edge_len[n] / (2.0 * area[s]);
                    double pn[3];
                    sub3(V + 3 * tri_free[3 * s + j], ct, pn);
                    cplx lav = M[7] - (pn[0] * M[1] + pn[1] * M[2] + pn[2] * M[3]) -
                               (pm[0] * M[4] + pm[1] * M[5] + pm[2] * M[6]) + dot3(pm, pn) * M[0];
                    if (la) la[(size_t)m * ne + n] += cm * cn * lav;
                    if (kk) {
                        double dl[3], cx[3];
                        sub3(pn, pm, dl);
                        cross3(pn, pm, cx);
                        cplx kv = dl[0] * M[8] + dl[1] * M[9] + dl[2] * M[10] + cx[0] * M[11] +
                                  cx[1] * M[12] + cx[2] * M[13];
                        kk[(size_t)m * ne + n] += cm * cn * kv;
                    }
                }
            }
        }
    }
    free(mom);
    free(area);
    return 0;
}
