// Near-region matrices of the AIM (Eqs. LinNRP, KinNRP): direct FP64
// integration of every near triangle pair minus the grid's own contribution
// for that pair (the precorrection L_P, K_P of Eqs. AIM_Lin, AIM_Kin), then
// assembly into edge CSR rows.
//
// Direct integration rule (the paper only says "direct integration"; this is
// the library's reading, documented with the parameters in sie.h):
//   far-near pairs  : collapsed Gauss product rule on both triangles;
//   close pairs     : outer collapsed Gauss on the test triangle, inner polar
//                     integration about the projection of the observation
//                     point (three signed sub-triangles, angular variable
//                     asinh(t/h), closed-form radial parts for 1/R and the
//                     static gradient, series or graded Gauss for the rest);
//   touching pairs  : outer rule graded toward the shared edge / vertex
//                     (self pair: three centroid sub-triangles graded toward
//                     the edges).
#include <cmath>
#include <complex>
#include <cstdio>

#include "internal.h"

namespace sie {

__constant__ QuadDev cq;
// per near pair: [0..8] LA exact-grid, [9..17] K exact-grid, [18] Lphi exact-grid,
// [19..27] LA exact, [28] Lphi exact
#define NLOC 29
#define RCUT 36.0  // exp(-36) < 1e-15

// ------------------------------------------------------------------ complex helpers
struct cd {
    double re, im;
};
__device__ __forceinline__ cd mk(double a, double b) { return {a, b}; }
__device__ __forceinline__ cd operator+(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd operator-(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd operator*(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd operator*(double s, cd a) { return {s * a.re, s * a.im}; }
__device__ __forceinline__ cd operator*(cd a, double s) { return {s * a.re, s * a.im}; }
__device__ __forceinline__ cd cdivc(cd a, cd b)
{
    double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ cd cexpc(cd z)
{
    double e = exp(z.re), s, c;
    sincos(z.im, &s, &c);
    return {e * c, e * s};
}
__device__ __forceinline__ double cabsc(cd z) { return hypot(z.re, z.im); }

// (exp(z) - 1)/z
__device__ cd phi1(cd z)
{
    if (cabsc(z) < 0.5) {
        cd term = mk(1, 0), s = mk(1, 0);
        for (int n = 1; n < 20; n++) {
            term = term * z * (1.0 / (double)(n + 1));
            s = s + term;
        }
        return s;
    }
    return cdivc(cexpc(z) - mk(1, 0), z);
}

// (1 + z) exp(-z) - 1 with a series near 0
__device__ cd hfun(cd z)
{
    if (cabsc(z) < 0.2) {
        cd s = mk(0, 0), zn = z;
        double fact = 1.0;
        for (int n = 2; n < 16; n++) {
            zn = zn * z;
            fact *= n;
            double sg = (n % 2 == 0) ? -1.0 : 1.0;
            s = s + (sg * (double)(n - 1) / fact) * zn;
        }
        return s;
    }
    return (mk(1, 0) + z) * cexpc(mk(-z.re, -z.im)) - mk(1, 0);
}

struct v3 {
    double x, y, z;
};
__device__ __forceinline__ v3 ld3(const double* p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ v3 operator-(v3 a, v3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ v3 operator+(v3 a, v3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ v3 operator*(double s, v3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ v3 cross(v3 a, v3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ double nrm(v3 a) { return sqrt(dot(a, a)); }

struct Inner {
    cd Is;
    cd Iv[3];
    cd Ig[3];
};

__device__ __forceinline__ cd clogc(cd z) { return mk(log(hypot(z.re, z.im)), atan2(z.im, z.re)); }

// Ein(z) = I_0^z (1 - exp(-t))/t dt for Re z >= 0: series for |z| < 2, else
// E1(z) + log z + gamma, E1 by its continued fraction (modified Lentz)
__device__ cd ein(cd z)
{
    if (cabsc(z) < 2.0) {
        cd s = mk(0, 0), t = mk(1, 0);
        for (int n = 1; n < 60; n++) {
            t = t * z * (1.0 / (double)n);
            cd term = ((n & 1) ? 1.0 : -1.0) / (double)n * t;
            s = s + term;
            if (cabsc(term) < 1e-17 * cabsc(s)) break;
        }
        return s;
    }
    const double tiny = 1e-300;
    cd f = z, C = z, D = mk(0, 0);
    for (int i = 1; i < 500; i++) {
        double a = (double)((i + 1) / 2);
        cd b = (i & 1) ? mk(1, 0) : z;
        D = b + a * D;
        if (cabsc(D) < tiny) D = mk(tiny, 0);
        C = b + cdivc(mk(a, 0), C);
        if (cabsc(C) < tiny) C = mk(tiny, 0);
        D = cdivc(mk(1, 0), D);
        cd delta = C * D;
        f = f * delta;
        if (cabsc(delta - mk(1, 0)) < 1e-16) break;
    }
    const double euler = 0.57721566490153286061;
    return cdivc(cexpc(mk(-z.re, -z.im)), f) + clogc(z) + mk(euler, 0);
}

// Numeric radial integrals over [0, rc] at height d.  Beyond R = RCUT/|Im k|
// every direction whose edge lies farther away integrates the same truncated
// range [0, rc(d)], so one evaluation serves all those directions of an
// observation point (same sums, computed once).
struct RadCache {
    bool valid;
    double rc;
    cd a1, a2;
};

__device__ void radial_numeric(cd k, double rc, double d, cd* a1o, cd* a2o)
{
    cd a1 = mk(0, 0), a2 = mk(0, 0);
    double hi = rc;
    for (int p = 0; p < cq.npan && rc > 0.0; p++) {
        double lo = (p == cq.npan - 1) ? 0.0 : hi * cq.ratio;
        for (int qq = 0; qq < cq.n[QR_RAD]; qq++) {
            double rho = lo + (hi - lo) * cq.x[QR_RAD][qq];
            double wr = (hi - lo) * cq.w[QR_RAD][qq];
            double R = sqrt(rho * rho + d * d);
            cd z = mk(-k.im * R, k.re * R);  // j k R
            cd e = cexpc(mk(-z.re, -z.im));
            cd hz = cabsc(z) < 0.2 ? hfun(z) : (mk(1, 0) + z) * e - mk(1, 0);
            a1 = a1 + (wr * rho * rho / R) * e;
            a2 = a2 + (wr * rho * rho / (R * R * R)) * hz;
        }
        hi = lo;
    }
    *a1o = a1;
    *a2o = a2;
}

// bounded radial remainders (series when |k| Rmax <= 1, else graded Gauss)
__device__ void radial(cd k, double rhom, double d, double Rmax, cd* f1, cd* f2, RadCache* cache)
{
    if (cabsc(k) * Rmax <= 1.0) {
        double rs = rhom / Rmax, ds = d / Rmax, Rs = sqrt(rs * rs + ds * ds), d2 = ds * ds;
        cd ks = k * Rmax;
        const int NT = 26;
        double B[NT + 4];
        B[0] = (d2 > 0.0) ? d2 * asinh(rs / fabs(ds)) : 0.0;  // d^2 B_-1
        B[1] = rs;                                           // B_0
        double Rp = 1.0, bodd = 0.0, beven = rs;
        for (int m = 1; m <= NT + 2; m++) {
            Rp *= Rs;
            double bm;
            if (m & 1) {
                double d2b = (m == 1) ? B[0] : d2 * bodd;
                bm = (rs * Rp + m * d2b) / (m + 1);
                bodd = bm;
            } else {
                bm = (rs * Rp + m * d2 * beven) / (m + 1);
                beven = bm;
            }
            B[m + 1] = bm;
        }
        double A[NT + 2];
        A[0] = B[2] - B[0];
        for (int m = 0; m <= NT; m++) A[m + 1] = B[m + 3] - d2 * B[m + 1];
        cd s1 = mk(0, 0), s2 = mk(0, 0), t1 = mk(1, 0);
        cd mjk = mk(ks.im, -ks.re);  // -j ks
        for (int n = 0; n <= NT; n++) {
            if (n > 0) t1 = t1 * mjk * (1.0 / (double)n);
            s1 = s1 + A[n] * t1;
            if (n >= 2) s2 = s2 + (-(double)(n - 1) * A[n - 2]) * t1;
        }
        *f1 = s1 * (Rmax * Rmax);
        *f2 = s2;
        return;
    }
    if (d == 0.0) {
        // coplanar point: closed forms with z = j k rhom
        cd z = mk(-k.im * rhom, k.re * rhom), e = cexpc(mk(-z.re, -z.im));
        cd jk = mk(-k.im, k.re);
        *f1 = cdivc(mk(1, 0) - e * (mk(1, 0) + z), jk * jk);
        *f2 = mk(1, 0) - e - ein(z);
        return;
    }
    // beyond R = RCUT/|Im k| the exponential is below 1e-15: f1 has no
    // contribution there and (1 + jkR) exp(-jkR) - 1 = -1 integrates in closed form
    double rc = rhom, tail = 0.0;
    bool trunc = false;
    double kim = fabs(k.im);
    if (kim > 0.0) {
        double Rc = RCUT / kim, Rm = sqrt(rhom * rhom + d * d);
        if (Rc < Rm) {
            trunc = true;
            rc = Rc > fabs(d) ? sqrt(Rc * Rc - d * d) : 0.0;
            double Rcc = sqrt(rc * rc + d * d);
            tail = (log(rhom + Rm) - rhom / Rm) - (log(rc + Rcc) - rc / Rcc);
        }
    }
    cd a1, a2;
    if (trunc) {
        // truncated: the range [0, rc] depends on d only
        if (!cache->valid || cache->rc != rc) {
            radial_numeric(k, rc, d, &cache->a1, &cache->a2);
            cache->rc = rc;
            cache->valid = true;
        }
        a1 = cache->a1;
        a2 = cache->a2;
    } else {
        radial_numeric(k, rc, d, &a1, &a2);
    }
    a2 = a2 - mk(tail, 0);
    *f1 = a1;
    *f2 = a2;
}

__device__ void inner_polar(v3 r, v3 v0, v3 v1, v3 v2, cd k, Inner& o)
{
    v3 vv[3] = {v0, v1, v2};
    v3 nm = cross(v1 - v0, v2 - v0);
    nm = (1.0 / nrm(nm)) * nm;
    double dd = dot(r - v0, nm);
    v3 rho0 = r - dd * nm;
    double Rmax = fmax(nrm(v0 - r), fmax(nrm(v1 - r), nrm(v2 - r)));
    if (fabs(dd) < 1e-12 * Rmax) dd = 0.0;  // on the plane up to rounding
    double ad = fabs(dd);
    o.Is = mk(0, 0);
    for (int d = 0; d < 3; d++) o.Iv[d] = o.Ig[d] = mk(0, 0);
    if (k.im != 0.0) {  // whole triangle beyond RCUT/|Im k|: every term below exp(-RCUT)
        v3 c = (1.0 / 3.0) * (v0 + v1 + v2);
        double rc = fmax(nrm(v0 - c), fmax(nrm(v1 - c), nrm(v2 - c)));
        if (nrm(r - c) - rc > RCUT / fabs(k.im)) return;
    }
    cd Is = mk(0, 0), Ign = mk(0, 0), Iv[3] = {mk(0, 0), mk(0, 0), mk(0, 0)}, Igt[3] = {mk(0, 0), mk(0, 0), mk(0, 0)};
    RadCache rcache;
    rcache.valid = false;
    double Omega = 0.0;
    cd mjk = mk(k.im, -k.re);  // -j k
    for (int i = 0; i < 3; i++) {
        v3 A = vv[i], B = vv[(i + 1) % 3];
        v3 e = B - A;
        double L = nrm(e);
        v3 et = (1.0 / L) * e;
        v3 m = cross(et, nm);
        v3 Ar = A - rho0, Br = B - rho0;
        double h = dot(Ar, m);
        if (fabs(h) < 1e-12 * L) continue;
        double sh = h > 0 ? 1.0 : -1.0, ah = fabs(h);
        v3 u = sh * m;
        double ta = dot(Ar, et), tb = dot(Br, et);
        Omega += sh * (atan2(tb, ah) - atan2(ta, ah));
        double sa = asinh(ta / ah), sb = asinh(tb / ah);
        int npa = (int)ceil((sb - sa) / cq.alen);
        if (npa < 1) npa = 1;
        double ds = (sb - sa) / npa;
        const int na = cq.n[QR_ANG];
        for (int j = 0; j < na * npa; j++) {
            int jp = j / na, jq = j % na;
            double s = sa + ds * (jp + cq.x[QR_ANG][jq]);
            double ch = cosh(s);
            double wa = sh * ds * cq.w[QR_ANG][jq] / ch;
            double ca = 1.0 / ch, sn = tanh(s);
            v3 eh = ca * u + sn * et;
            double rhom = ah * ch;
            double Rm = sqrt(rhom * rhom + dd * dd);
            cd is = cexpc(mjk * ad) * (Rm - ad) * phi1(mjk * (Rm - ad));
            cd f1, f2;
            radial(k, rhom, dd, Rmax, &f1, &f2, &rcache);
            cd igt = mk(log(rhom + Rm) - rhom / Rm, 0) + f2;
            cd ign = (-dd / Rm) * cexpc(mjk * Rm);
            Is = Is + wa * is;
            Ign = Ign + wa * ign;
            double ehv[3] = {eh.x, eh.y, eh.z}, nmv[3] = {nm.x, nm.y, nm.z};
            for (int d = 0; d < 3; d++) {
                Iv[d] = Iv[d] + wa * (ehv[d] * f1 - (dd * nmv[d]) * is);
                Igt[d] = Igt[d] + (wa * ehv[d]) * igt;
            }
        }
    }
    cd jump = mk(0, 0);
    if (dd != 0.0) jump = (Omega * (dd > 0 ? 1.0 : -1.0)) * cexpc(mjk * ad);
    const double f = 1.0 / (4.0 * M_PI);
    double nmv[3] = {nm.x, nm.y, nm.z};
    o.Is = f * Is;
    for (int d = 0; d < 3; d++) {
        o.Iv[d] = f * Iv[d];
        o.Ig[d] = (-f) * (nmv[d] * (jump + Ign) - Igt[d]);
    }
}

__device__ void inner_gauss(v3 r, v3 a, v3 b, v3 c, cd k, Inner& o)
{
    v3 e1 = b - a, e2 = c - a;
    double twoA = nrm(cross(e1, e2));
    o.Is = mk(0, 0);
    for (int d = 0; d < 3; d++) o.Iv[d] = o.Ig[d] = mk(0, 0);
    const int n = cq.n[QR_FAR];
    for (int i = 0; i < n; i++) {
        double u = cq.x[QR_FAR][i];
        for (int j = 0; j < n; j++) {
            double v = cq.x[QR_FAR][j] * (1.0 - u);
            double w = twoA * (1.0 - u) * cq.w[QR_FAR][i] * cq.w[QR_FAR][j];
            v3 p = a + u * e1 + v * e2;
            v3 dv = p - r;
            double R = nrm(dv);
            cd e = cexpc(mk(k.im * R, -k.re * R));
            cd G = (1.0 / (4.0 * M_PI * R)) * e;
            cd g = (-1.0 / (4.0 * M_PI * R * R * R)) * (mk(1.0 - k.im * R, k.re * R) * e);
            o.Is = o.Is + w * G;
            double dvv[3] = {dv.x, dv.y, dv.z};
            for (int d = 0; d < 3; d++) {
                o.Iv[d] = o.Iv[d] + (w * dvv[d]) * G;
                o.Ig[d] = o.Ig[d] + (-w * dvv[d]) * g;
            }
        }
    }
}

// ------------------------------------------------------------------ outer rules
// point and weight of outer node q of a graded rule (apex shared: toward 0;
// edge b-c shared: toward 1 in lam and graded toward both ends in mu)
__device__ void graded_point(v3 apex, v3 b, v3 c, int toward_edge, int q, v3& p, double& w)
{
    const int olam = cq.n[QR_OLAM];
    const int nmu = toward_edge ? 2 * cq.emupan * cq.n[QR_EMU] : cq.n[QR_OMU];
    int pan = q / (olam * nmu), rr = q % (olam * nmu), i = rr / nmu, j = rr % nmu;
    double hi = 1.0;
    for (int t = 0; t < pan; t++) hi *= cq.oratio;
    double lo = (pan == cq.opan - 1) ? 0.0 : hi * cq.oratio;
    double sg = lo + (hi - lo) * cq.x[QR_OLAM][i];
    double wsg = (hi - lo) * cq.w[QR_OLAM][i];
    double lam = toward_edge ? 1.0 - sg : sg;
    double mu, wmu;
    if (!toward_edge) {
        mu = cq.x[QR_OMU][j];
        wmu = cq.w[QR_OMU][j];
    } else {
        const int ne = cq.n[QR_EMU];
        int side = j / (cq.emupan * ne), r2 = j % (cq.emupan * ne), pp = r2 / ne, jj = r2 % ne;
        double h2 = 0.5;
        for (int t = 0; t < pp; t++) h2 *= cq.oratio;
        double l2 = (pp == cq.emupan - 1) ? 0.0 : h2 * cq.oratio;
        double s = l2 + (h2 - l2) * cq.x[QR_EMU][jj];
        mu = side ? 1.0 - s : s;
        wmu = (h2 - l2) * cq.w[QR_EMU][jj];
    }
    v3 e1 = b - apex, e2 = c - b;
    double twoA = nrm(cross(e1, e2));
    p = apex + lam * (e1 + mu * e2);
    w = twoA * lam * wsg * wmu;
}

__device__ int graded_count(int toward_edge)
{
    const int nmu = toward_edge ? 2 * cq.emupan * cq.n[QR_EMU] : cq.n[QR_OMU];
    return cq.opan * cq.n[QR_OLAM] * nmu;
}

// 14 moments per pair: Q0, Q1[3], Q2[3], Q3, U[3], V[3] (origin: centroid of t).
// One warp per pair; lanes split the outer points.
// obj_k: per-object wavenumbers of a several-object interior (null: kr + j ki)
__global__ void __launch_bounds__(128) k_near_moments(const int32_t* __restrict__ pairs, int64_t np, DevMesh M,
                                                      double kr, double ki, const double2* __restrict__ obj_k,
                                                      double2* __restrict__ mom)
{
    int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (p >= np) return;
    int t = pairs[2 * p], s = pairs[2 * p + 1];
    if (obj_k) {
        const double2 ko = obj_k[M.obj[t]];
        kr = ko.x;
        ki = ko.y;
    }
    cd k = mk(kr, ki);
    int tt[3] = {M.T[3 * t], M.T[3 * t + 1], M.T[3 * t + 2]};
    int ss[3] = {M.T[3 * s], M.T[3 * s + 1], M.T[3 * s + 2]};
    v3 a = ld3(M.V + 3 * tt[0]), b = ld3(M.V + 3 * tt[1]), c = ld3(M.V + 3 * tt[2]);
    v3 a2 = ld3(M.V + 3 * ss[0]), b2 = ld3(M.V + 3 * ss[1]), c2 = ld3(M.V + 3 * ss[2]);
    v3 ct = ld3(M.cen + 3 * t);
    int shared[3], nsh = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (tt[i] == ss[j]) shared[nsh++] = i;
    bool close = nsh > 0;
    if (!close) {
        v3 cs = ld3(M.cen + 3 * s);
        double D = nrm(ct - cs), Rt = M.rad[t], Rs = M.rad[s];
        if (D < cq.cf * (Rt + Rs) || hypot(kr, ki) * (Rt + Rs) > cq.kres) close = true;
    }
    // outer rule
    int kind;  // 0 plain collapsed, 1 edge shared, 2 vertex shared, 3 self
    int nout;
    v3 ap, bp, cp;
    if (t == s) {
        kind = 3;
        nout = 3 * graded_count(1);
    } else if (nsh == 2) {
        kind = 1;
        int ia = 3 - shared[0] - shared[1];
        v3 vt[3] = {a, b, c};
        ap = vt[ia];
        bp = vt[(ia + 1) % 3];
        cp = vt[(ia + 2) % 3];
        nout = graded_count(1);
    } else if (nsh == 1) {
        kind = 2;
        int ia = shared[0];
        v3 vt[3] = {a, b, c};
        ap = vt[ia];
        bp = vt[(ia + 1) % 3];
        cp = vt[(ia + 2) % 3];
        nout = graded_count(0);
    } else {
        kind = 0;
        int n = close ? cq.n[QR_OUT] : cq.n[QR_FAR];
        nout = n * n;
    }
    cd acc[14];
    for (int i = 0; i < 14; i++) acc[i] = mk(0, 0);
    double twoA = nrm(cross(b - a, c - a));
    for (int qo = lane; qo < nout; qo += 32) {
        v3 r;
        double w;
        if (kind == 0) {
            int ridx = close ? QR_OUT : QR_FAR;
            int n = cq.n[ridx];
            int i = qo / n, j = qo % n;
            double u = cq.x[ridx][i], v = cq.x[ridx][j] * (1.0 - u);
            r = a + u * (b - a) + v * (c - a);
            w = twoA * (1.0 - u) * cq.w[ridx][i] * cq.w[ridx][j];
        } else if (kind == 3) {
            int per = graded_count(1), sub = qo / per;
            v3 vt[3] = {a, b, c};
            graded_point(ct, vt[sub], vt[(sub + 1) % 3], 1, qo % per, r, w);
        } else {
            graded_point(ap, bp, cp, kind == 1, qo, r, w);
        }
        Inner in;
        if (close)
            inner_polar(r, a2, b2, c2, k, in);
        else
            inner_gauss(r, a2, b2, c2, k, in);
        v3 rt = r - ct;
        double rtv[3] = {rt.x, rt.y, rt.z};
        cd I2[3];
        for (int d = 0; d < 3; d++) I2[d] = in.Iv[d] + rtv[d] * in.Is;
        acc[0] = acc[0] + w * in.Is;
        for (int d = 0; d < 3; d++) {
            acc[1 + d] = acc[1 + d] + (w * rtv[d]) * in.Is;
            acc[4 + d] = acc[4 + d] + w * I2[d];
        }
        acc[7] = acc[7] + w * (rtv[0] * I2[0] + rtv[1] * I2[1] + rtv[2] * I2[2]);
        if (t != s) {
            acc[8] = acc[8] + (-w) * (rtv[1] * in.Ig[2] - rtv[2] * in.Ig[1]);
            acc[9] = acc[9] + (-w) * (rtv[2] * in.Ig[0] - rtv[0] * in.Ig[2]);
            acc[10] = acc[10] + (-w) * (rtv[0] * in.Ig[1] - rtv[1] * in.Ig[0]);
            for (int d = 0; d < 3; d++) acc[11 + d] = acc[11 + d] + w * in.Ig[d];
        }
    }
    for (int i = 0; i < 14; i++)
        for (int off = 16; off > 0; off >>= 1) {
            acc[i].re += __shfl_down_sync(0xffffffffu, acc[i].re, off);
            acc[i].im += __shfl_down_sync(0xffffffffu, acc[i].im, off);
        }
    if (lane == 0)
        for (int i = 0; i < 14; i++) mom[14 * p + i] = make_double2(acc[i].re, acc[i].im);
}

// kernel values at integer lags |l_d| <= Lm: (G, dG/dx, dG/dy, dG/dz), zero at lag 0
__global__ void k_lagtab(int Lm, double h, double kr, double ki, double2* __restrict__ tab)
{
    int W = 2 * Lm + 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= W * W * W) return;
    int lx = idx % W - Lm, ly = (idx / W) % W - Lm, lz = idx / (W * W) - Lm;
    double dx = h * lx, dy = h * ly, dz = h * lz;
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    cd G = mk(0, 0), gx = mk(0, 0), gy = mk(0, 0), gz = mk(0, 0);
    if (R > 0) {
        cd e = cexpc(mk(ki * R, -kr * R));
        G = (1.0 / (4.0 * M_PI * R)) * e;
        cd g = (-1.0 / (4.0 * M_PI * R * R * R)) * (mk(1.0 - ki * R, kr * R) * e);
        gx = dx * g;
        gy = dy * g;
        gz = dz * g;
    }
    tab[4 * idx + 0] = make_double2(G.re, G.im);
    tab[4 * idx + 1] = make_double2(gx.re, gx.im);
    tab[4 * idx + 2] = make_double2(gy.re, gy.im);
    tab[4 * idx + 3] = make_double2(gz.re, gz.im);
}

// Per pair: exact local entries (LA 3x3, K 3x3, Lphi) minus the grid's own
// entries for the pair when the operator has a grid, plus the exact LA and
// Lphi.  One warp per pair; lanes own the test-stencil nodes u.  out: NLOC
// complex per pair.
__global__ void __launch_bounds__(128) k_near_local(const int32_t* __restrict__ pairs, int64_t np, DevMesh M,
                                                    const double2* __restrict__ mom, int has_grid, int S, int Mord,
                                                    const int32_t* __restrict__ base, const double* __restrict__ Wt,
                                                    const double2* __restrict__ tab, int Lm, double2* __restrict__ out)
{
    int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (p >= np) return;
    int t = pairs[2 * p], s = pairs[2 * p + 1];
    // grid part: partial sums over the test nodes owned by this lane
    cd gLA[9], gK[9], g0 = mk(0, 0);
    for (int i = 0; i < 9; i++) gLA[i] = gK[i] = mk(0, 0);
    if (has_grid) {
        const int Mp = Mord + 1;
        int bt[3] = {base[3 * t], base[3 * t + 1], base[3 * t + 2]};
        int bs[3] = {base[3 * s], base[3 * s + 1], base[3 * s + 2]};
        const double* ct = M.coef + 3 * t;
        const double* cs = M.coef + 3 * s;
        const double* qt = M.q + 9 * t;
        const double* qs = M.q + 9 * s;
        const int Wd = 2 * Lm + 1;
        for (int u = lane; u < S; u += 32) {
            int ux = u % Mp, uy = (u / Mp) % Mp, uz = u / (Mp * Mp);
            const double* wu = Wt + ((size_t)t * S + u) * 4;
            double xt[3][3];  // test projection weights of slot i, component a
            for (int i = 0; i < 3; i++)
                for (int aa = 0; aa < 3; aa++) xt[i][aa] = ct[i] * (wu[1 + aa] + qt[3 * i + aa] * wu[0]);
            for (int v = 0; v < S; v++) {
                int vx = v % Mp, vy = (v / Mp) % Mp, vz = v / (Mp * Mp);
                int lx = bt[0] + ux - bs[0] - vx, ly = bt[1] + uy - bs[1] - vy, lz = bt[2] + uz - bs[2] - vz;
                const double2* kv = tab + 4 * (((lz + Lm) * Wd + (ly + Lm)) * Wd + (lx + Lm));
                cd G = mk(kv[0].x, kv[0].y), Dx = mk(kv[1].x, kv[1].y), Dy = mk(kv[2].x, kv[2].y),
                   Dz = mk(kv[3].x, kv[3].y);
                const double* wv = Wt + ((size_t)s * S + v) * 4;
                g0 = g0 + (wu[0] * wv[0]) * G;
                for (int j = 0; j < 3; j++) {
                    double xs[3];
                    for (int cc = 0; cc < 3; cc++) xs[cc] = cs[j] * (wv[1 + cc] + qs[3 * j + cc] * wv[0]);
                    for (int i = 0; i < 3; i++) {
                        double la = xt[i][0] * xs[0] + xt[i][1] * xs[1] + xt[i][2] * xs[2];
                        // sum_abc eps_abc xt_a D_b xs_c = D . (xs x xt)
                        double wx = xs[1] * xt[i][2] - xs[2] * xt[i][1];
                        double wy = xs[2] * xt[i][0] - xs[0] * xt[i][2];
                        double wz = xs[0] * xt[i][1] - xs[1] * xt[i][0];
                        gLA[3 * i + j] = gLA[3 * i + j] + la * G;
                        gK[3 * i + j] = gK[3 * i + j] + wx * Dx + wy * Dy + wz * Dz;
                    }
                }
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            for (int i = 0; i < 9; i++) {
                gLA[i].re += __shfl_down_sync(0xffffffffu, gLA[i].re, off);
                gLA[i].im += __shfl_down_sync(0xffffffffu, gLA[i].im, off);
                gK[i].re += __shfl_down_sync(0xffffffffu, gK[i].re, off);
                gK[i].im += __shfl_down_sync(0xffffffffu, gK[i].im, off);
            }
            g0.re += __shfl_down_sync(0xffffffffu, g0.re, off);
            g0.im += __shfl_down_sync(0xffffffffu, g0.im, off);
        }
    }
    if (lane != 0) return;
    // exact entries from the moments
    const double2* mm = mom + 14 * p;
    cd Q0 = mk(mm[0].x, mm[0].y);
    cd Q1[3], Q2[3], U[3], Vv[3];
    for (int d = 0; d < 3; d++) {
        Q1[d] = mk(mm[1 + d].x, mm[1 + d].y);
        Q2[d] = mk(mm[4 + d].x, mm[4 + d].y);
        U[d] = mk(mm[8 + d].x, mm[8 + d].y);
        Vv[d] = mk(mm[11 + d].x, mm[11 + d].y);
    }
    cd Q3 = mk(mm[7].x, mm[7].y);
    v3 ctc = ld3(M.cen + 3 * t);
    double At = M.area[t], As = M.area[s];
    double2* o = out + NLOC * p;
    for (int i = 0; i < 3; i++) {
        double cm = M.coef[3 * t + i];
        v3 pm = ld3(M.V + 3 * M.T[3 * t + i]) - ctc;
        for (int j = 0; j < 3; j++) {
            double cn = M.coef[3 * s + j];
            v3 pn = ld3(M.V + 3 * M.T[3 * s + j]) - ctc;
            cd la = Q3 - (pn.x * Q1[0] + pn.y * Q1[1] + pn.z * Q1[2]) - (pm.x * Q2[0] + pm.y * Q2[1] + pm.z * Q2[2]) +
                    dot(pm, pn) * Q0;
            v3 dl = pn - pm, cx = cross(pn, pm);
            cd kk = dl.x * U[0] + dl.y * U[1] + dl.z * U[2] + cx.x * Vv[0] + cx.y * Vv[1] + cx.z * Vv[2];
            la = (cm * cn) * la;
            o[19 + 3 * i + j] = make_double2(la.re, la.im);  // exact
            la = la - gLA[3 * i + j];
            kk = (cm * cn) * kk - gK[3 * i + j];
            o[3 * i + j] = make_double2(la.re, la.im);
            o[9 + 3 * i + j] = make_double2(kk.re, kk.im);
        }
    }
    cd lp = (1.0 / (At * As)) * (Q0 - g0);
    o[18] = make_double2(lp.re, lp.im);
    cd lpe = (1.0 / (At * As)) * Q0;
    o[28] = make_double2(lpe.re, lpe.im);  // exact
}

// CSR values: entry (m, n) sums the local entries of the near pairs (t, s)
// with t in supp(f_m), s in supp(f_n), in a fixed order (deterministic).
// vL = L (exact - grid), vK = K (exact - grid), vLA = LA (exact - grid);
// diagonal entries also give the exact LA and L diagonals (dLA, dL).
__global__ void k_csr_fill(int ne, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const int64_t* __restrict__ pstart, const int32_t* __restrict__ pairs,
                           const double2* __restrict__ loc, DevMesh M, double2 invk2,
                           const double2* __restrict__ obj_invk2, double2* __restrict__ vL,
                           double2* __restrict__ vK, double2* __restrict__ vLA, double2* __restrict__ dLA,
                           double2* __restrict__ dL)
{
    int m = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (m >= ne) return;
    if (obj_invk2) invk2 = obj_invk2[M.obj[M.edge_tri[2 * m]]];  // row m's object
    cd ik2 = mk(invk2.x, invk2.y);
    for (int64_t e = row_ptr[m] + lane; e < row_ptr[m + 1]; e += 32) {
        int n = col[e];
        cd L = mk(0, 0), K = mk(0, 0), LA = mk(0, 0), LAx = mk(0, 0), Lx = mk(0, 0);
        for (int a = 0; a < 2; a++) {
            int t = M.edge_tri[2 * m + a], i = M.edge_slot[2 * m + a];
            int64_t lo = pstart[t], hi = pstart[t + 1];
            for (int b = 0; b < 2; b++) {
                int s = M.edge_tri[2 * n + b], j = M.edge_slot[2 * n + b];
                // binary search s in pairs[lo..hi)
                int64_t l = lo, r = hi;
                while (l < r) {
                    int64_t mid = (l + r) >> 1;
                    if (pairs[2 * mid + 1] < s)
                        l = mid + 1;
                    else
                        r = mid;
                }
                if (l < hi && pairs[2 * l + 1] == s) {
                    const double2* o = loc + NLOC * l;
                    double c4 = 4.0 * M.coef[3 * t + i] * M.coef[3 * s + j] * M.area[t] * M.area[s];
                    cd lp = mk(o[18].x, o[18].y), lpe = mk(o[28].x, o[28].y);
                    cd la = mk(o[3 * i + j].x, o[3 * i + j].y), lae = mk(o[19 + 3 * i + j].x, o[19 + 3 * i + j].y);
                    LA = LA + la;
                    L = L + la - c4 * (ik2 * lp);
                    K = K + mk(o[9 + 3 * i + j].x, o[9 + 3 * i + j].y);
                    LAx = LAx + lae;
                    Lx = Lx + lae - c4 * (ik2 * lpe);
                }
            }
        }
        vL[e] = make_double2(L.re, L.im);
        vK[e] = make_double2(K.re, K.im);
        vLA[e] = make_double2(LA.re, LA.im);
        if (n == m) {
            dLA[m] = make_double2(LAx.re, LAx.im);
            dL[m] = make_double2(Lx.re, Lx.im);
        }
    }
}

__global__ void k_lphi_vals(int64_t np, const double2* __restrict__ loc, double2* __restrict__ v,
                            double2* __restrict__ vnr)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) {
        v[p] = loc[NLOC * p + 18];    // exact - grid
        vnr[p] = loc[NLOC * p + 28];  // exact (near-region matrix, preconditioner)
    }
}

sie_status near_build(sie_op* op, AimOp& a, const QuadDev& q)
{
    cudaStream_t st = op->mesh->ctx->stream;
    const DevMesh& M = op->mesh->d;
    const HostMesh& H = op->mesh->h;
    SIE_CUDA_TRY(cudaMemcpyToSymbolAsync(cq, &q, sizeof(QuadDev), 0, cudaMemcpyHostToDevice, st));
    a.npairs = (int64_t)a.hpairs.size() / 2;
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.pairs, sizeof(int32_t) * 2 * std::max<int64_t>(a.npairs, 1), st));
    SIE_CUDA_TRY(cudaMemcpyAsync(a.pairs, a.hpairs.data(), sizeof(int32_t) * 2 * a.npairs, cudaMemcpyHostToDevice, st));
    double2 *mom = nullptr, *loc = nullptr, *tab = nullptr;
    SIE_CUDA_TRY(cudaMallocAsync((void**)&mom, sizeof(double2) * 14 * std::max<int64_t>(a.npairs, 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&loc, sizeof(double2) * NLOC * std::max<int64_t>(a.npairs, 1), st));
    const int wpb = 4;
    if (a.npairs > 0) {
        k_near_moments<<<(unsigned)((a.npairs + wpb - 1) / wpb), 32 * wpb, 0, st>>>(a.pairs, a.npairs, M, a.kr, a.ki,
                                                                                    a.obj_k, mom);
        SIE_CUDA_TRY(cudaGetLastError());
    }
    int Lm = a.g.Rnear + a.g.M;
    int S = (a.g.M + 1) * (a.g.M + 1) * (a.g.M + 1);
    if (a.has_grid) {
        int W = 2 * Lm + 1;
        SIE_CUDA_TRY(cudaMallocAsync((void**)&tab, sizeof(double2) * 4 * W * W * W, st));
        k_lagtab<<<(W * W * W + 127) / 128, 128, 0, st>>>(Lm, a.g.h, a.kr, a.ki, tab);
        SIE_CUDA_TRY(cudaGetLastError());
    }
    if (a.npairs > 0) {
        k_near_local<<<(unsigned)((a.npairs + wpb - 1) / wpb), 32 * wpb, 0, st>>>(
            a.pairs, a.npairs, M, mom, a.has_grid ? 1 : 0, S, a.g.M, op->base, op->W, tab, Lm, loc);
        SIE_CUDA_TRY(cudaGetLastError());
    }
    // CSR over edges
    edge_csr_pattern(H, a.hpairs, a.csr);
    a.nnz = (int64_t)a.csr.col.size();
    std::vector<int64_t> pstart(H.nt + 1, 0);
    for (int64_t p = 0; p < a.npairs; p++) pstart[a.hpairs[2 * p] + 1]++;
    for (int64_t t = 0; t < H.nt; t++) pstart[t + 1] += pstart[t];
    int64_t* dps = nullptr;
    SIE_CUDA_TRY(cudaMallocAsync((void**)&dps, sizeof(int64_t) * (H.nt + 1), st));
    SIE_CUDA_TRY(cudaMemcpyAsync(dps, pstart.data(), sizeof(int64_t) * (H.nt + 1), cudaMemcpyHostToDevice, st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.row_ptr, sizeof(int64_t) * (H.ne + 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.col, sizeof(int32_t) * std::max<int64_t>(a.nnz, 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.valL, sizeof(double2) * std::max<int64_t>(a.nnz, 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.valK, sizeof(double2) * std::max<int64_t>(a.nnz, 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.valLA, sizeof(double2) * std::max<int64_t>(a.nnz, 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.dLA, sizeof(double2) * H.ne, st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.dL, sizeof(double2) * H.ne, st));
    SIE_CUDA_TRY(cudaMemsetAsync(a.dLA, 0, sizeof(double2) * H.ne, st));
    SIE_CUDA_TRY(cudaMemsetAsync(a.dL, 0, sizeof(double2) * H.ne, st));
    SIE_CUDA_TRY(cudaMemcpyAsync(a.row_ptr, a.csr.row_ptr.data(), sizeof(int64_t) * (H.ne + 1), cudaMemcpyHostToDevice, st));
    SIE_CUDA_TRY(cudaMemcpyAsync(a.col, a.csr.col.data(), sizeof(int32_t) * a.nnz, cudaMemcpyHostToDevice, st));
    std::complex<double> kk(a.kr, a.ki);
    std::complex<double> ik2 = 1.0 / (kk * kk);
    k_csr_fill<<<(unsigned)((H.ne + 3) / 4), 128, 0, st>>>((int)H.ne, a.row_ptr, a.col, dps, a.pairs, loc, M,
                                                           make_double2(ik2.real(), ik2.imag()), a.obj_ik2, a.valL,
                                                           a.valK,
                                                           a.valLA, a.dLA, a.dL);
    SIE_CUDA_TRY(cudaGetLastError());
    // triangle CSR of Lphi (exact - grid): rows = pair blocks, columns = s
    a.tri_row_ptr_h = pstart;
    a.tri_col_h.resize(a.npairs);
    for (int64_t p = 0; p < a.npairs; p++) a.tri_col_h[p] = a.hpairs[2 * p + 1];
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.tri_row_ptr, sizeof(int64_t) * (H.nt + 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.tri_col, sizeof(int32_t) * std::max<int64_t>(a.npairs, 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.valLphi, sizeof(double2) * std::max<int64_t>(a.npairs, 1), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.valLphiNR, sizeof(double2) * std::max<int64_t>(a.npairs, 1), st));
    SIE_CUDA_TRY(cudaMemcpyAsync(a.tri_row_ptr, a.tri_row_ptr_h.data(), sizeof(int64_t) * (H.nt + 1),
                                 cudaMemcpyHostToDevice, st));
    SIE_CUDA_TRY(cudaMemcpyAsync(a.tri_col, a.tri_col_h.data(), sizeof(int32_t) * a.npairs, cudaMemcpyHostToDevice, st));
    if (a.npairs > 0) {
        k_lphi_vals<<<(unsigned)((a.npairs + 255) / 256), 256, 0, st>>>(a.npairs, loc, a.valLphi, a.valLphiNR);
        SIE_CUDA_TRY(cudaGetLastError());
    }
    SIE_CUDA_TRY(cudaFreeAsync(dps, st));
    SIE_CUDA_TRY(cudaFreeAsync(mom, st));
    SIE_CUDA_TRY(cudaFreeAsync(loc, st));
    if (tab) SIE_CUDA_TRY(cudaFreeAsync(tab, st));
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    return SIE_OK;
}

}  // namespace sie
