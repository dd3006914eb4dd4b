// Host side of the library: RWG table, AIM grid, near-pair lists, CSR
// patterns, Gauss rules and the C ABI entry points.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <numeric>

#include "internal.h"

namespace sie {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// ------------------------------------------------------------------ RWG (Sec. II-A)
sie_status build_mesh(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, HostMesh& m)
{
    if (!xyz || !tri || nv < 3 || nt < 4) {
        set_error("sie_mesh_create: need at least 3 vertices and 4 triangles");
        return SIE_ERR_ARG;
    }
    for (int64_t i = 0; i < 3 * nv; i++)
        if (!std::isfinite(xyz[i])) {
            set_error("sie_mesh_create: vertex coordinate " + std::to_string(i) + " is not finite");
            return SIE_ERR_ARG;
        }
    m.nv = nv;
    m.nt = nt;
    m.V.assign(xyz, xyz + 3 * nv);
    m.T.assign(tri, tri + 3 * nt);
    for (int64_t i = 0; i < 3 * nt; i++)
        if (tri[i] < 0 || tri[i] >= nv) {
            set_error("sie_mesh_create: vertex index out of range");
            return SIE_ERR_MESH;
        }
    // directed edge of slot i: (v[i+1], v[i+2]); undirected key lo*nv+hi
    std::vector<std::pair<int64_t, int64_t>> keys(3 * nt);
    for (int64_t t = 0; t < nt; t++)
        for (int i = 0; i < 3; i++) {
            int64_t a = tri[3 * t + (i + 1) % 3], b = tri[3 * t + (i + 2) % 3];
            int64_t lo = std::min(a, b), hi = std::max(a, b);
            keys[3 * t + i] = {lo * nv + hi, 3 * t + i};
        }
    std::sort(keys.begin(), keys.end());
    if (keys.size() % 2) {
        set_error("sie_mesh_create: mesh is not closed");
        return SIE_ERR_MESH;
    }
    m.ne = (int64_t)keys.size() / 2;
    m.tri_edge.assign(3 * nt, -1);
    m.tri_sign.assign(3 * nt, 0);
    m.edge_len.assign(m.ne, 0.0);
    m.edge_tri.assign(2 * m.ne, -1);
    m.edge_slot.assign(2 * m.ne, -1);
    for (int64_t e = 0; e < m.ne; e++) {
        auto k0 = keys[2 * e], k1 = keys[2 * e + 1];
        if (k0.first != k1.first || (2 * e + 2 < (int64_t)keys.size() && keys[2 * e + 2].first == k0.first) ||
            (e > 0 && keys[2 * e - 1].first == k0.first)) {
            set_error("sie_mesh_create: an edge is not shared by exactly two triangles");
            return SIE_ERR_MESH;
        }
        for (auto kk : {k0, k1}) {
            int64_t t = kk.second / 3;
            int i = (int)(kk.second % 3);
            int64_t a = tri[3 * t + (i + 1) % 3], b = tri[3 * t + (i + 2) % 3];
            int s = a < b ? 1 : -1;
            int col = s > 0 ? 0 : 1;
            if (m.edge_tri[2 * e + col] >= 0) {
                set_error("sie_mesh_create: inconsistent triangle orientation");
                return SIE_ERR_MESH;
            }
            m.edge_tri[2 * e + col] = (int32_t)t;
            m.edge_slot[2 * e + col] = (int8_t)i;
            m.tri_edge[3 * t + i] = (int32_t)e;
            m.tri_sign[3 * t + i] = (int8_t)s;
        }
        int64_t lo = k0.first / nv, hi = k0.first % nv;
        double d0 = xyz[3 * hi] - xyz[3 * lo], d1 = xyz[3 * hi + 1] - xyz[3 * lo + 1],
               d2 = xyz[3 * hi + 2] - xyz[3 * lo + 2];
        m.edge_len[e] = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    m.area.resize(nt);
    m.cen.resize(3 * nt);
    m.nrm.resize(3 * nt);
    m.coef.resize(3 * nt);
    m.q.resize(9 * nt);
    m.rad.resize(nt);
    for (int64_t t = 0; t < nt; t++) {
        const double *a = &m.V[3 * tri[3 * t]], *b = &m.V[3 * tri[3 * t + 1]], *c = &m.V[3 * tri[3 * t + 2]];
        double e1[3], e2[3], n[3];
        for (int d = 0; d < 3; d++) {
            e1[d] = b[d] - a[d];
            e2[d] = c[d] - a[d];
        }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double twoA = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        double e3[3] = {c[0] - b[0], c[1] - b[1], c[2] - b[2]};
        double lmax2 = std::max({e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2],
                                 e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2],
                                 e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]});
        // collinear up to rounding: area below 1e-10 of the longest edge squared
        if (!(twoA > 1e-10 * lmax2)) {
            set_error("sie_mesh_create: degenerate triangle");
            return SIE_ERR_MESH;
        }
        m.area[t] = 0.5 * twoA;
        for (int d = 0; d < 3; d++) {
            m.nrm[3 * t + d] = n[d] / twoA;
            m.cen[3 * t + d] = (a[d] + b[d] + c[d]) / 3.0;
        }
        double R = 0;
        for (int i = 0; i < 3; i++) {
            const double* v = &m.V[3 * tri[3 * t + i]];
            double dx = v[0] - m.cen[3 * t], dy = v[1] - m.cen[3 * t + 1], dz = v[2] - m.cen[3 * t + 2];
            R = std::max(R, std::sqrt(dx * dx + dy * dy + dz * dz));
            int e = m.tri_edge[3 * t + i];
            m.coef[3 * t + i] = m.tri_sign[3 * t + i] * m.edge_len[e] / (2.0 * m.area[t]);
            for (int d = 0; d < 3; d++) m.q[9 * t + 3 * i + d] = m.cen[3 * t + d] - v[d];
        }
        m.rad[t] = R;
    }
    double s = 0;
    for (double l : m.edge_len) s += l;
    m.mean_edge = s / (double)m.ne;
    m.obj.assign(nt, 0);
    m.nobj = 1;
    return SIE_OK;
}

// objects of a mesh: each a closed surface of its own (no edge between objects)
static sie_status set_objects(HostMesh& m, const int32_t* obj)
{
    int nobj = 0;
    for (int64_t t = 0; t < m.nt; t++) {
        if (obj[t] < 0) {
            set_error("sie_mesh_create_objects: negative object index");
            return SIE_ERR_MESH;
        }
        nobj = std::max(nobj, obj[t] + 1);
    }
    for (int64_t e = 0; e < m.ne; e++)
        if (obj[m.edge_tri[2 * e]] != obj[m.edge_tri[2 * e + 1]]) {
            set_error("sie_mesh_create_objects: edge " + std::to_string(e) +
                      " joins two objects; every object must be a closed surface of its own");
            return SIE_ERR_MESH;
        }
    m.obj.assign(obj, obj + m.nt);
    m.nobj = nobj;
    return SIE_OK;
}

// ------------------------------------------------------------------ grid (Sec. III-A, Sec. IV)
static int next_pow2(int v)
{
    int n = 1;
    while (n < v) n <<= 1;
    return n;
}

sie_status make_grid(const HostMesh& m, const sie_params& p, GridDesc& g)
{
    if (p.stencil_order < 1 || p.stencil_order > 3 || p.near_radius < p.stencil_order) {
        set_error("stencil_order must be 1..3 and near_radius >= stencil_order");
        return SIE_ERR_ARG;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t v = 0; v < m.nv; v++)
        for (int d = 0; d < 3; d++) {
            lo[d] = std::min(lo[d], m.V[3 * v + d]);
            hi[d] = std::max(hi[d], m.V[3 * v + d]);
        }
    int M = p.stencil_order, mg = (M + 1) / 2 + 1;
    double h = p.h;
    if (!(h > 0)) {
        if (p.grid_n > 0) {
            double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
            if (p.grid_n - 2 * mg - 3 < 1) {
                set_error("grid_n too small for the stencil margin");
                return SIE_ERR_ARG;
            }
            h = ext / (double)(p.grid_n - 2 * mg - 3);
        } else {
            h = p.h_over_edge * m.mean_edge;
        }
    }
    const double s[3] = {0.5 * (1.0 / std::sqrt(2.0)), 0.5 * (1.0 / std::sqrt(3.0)), 0.5 * (1.0 / std::sqrt(5.0))};
    g.h = h;
    g.M = M;
    g.Rnear = p.near_radius;
    for (int d = 0; d < 3; d++) {
        g.o[d] = lo[d] - ((double)mg + s[d]) * h;
        g.N[d] = (int)std::floor((hi[d] - g.o[d]) / h) + 2 + mg;
        g.n[d] = next_pow2(2 * g.N[d] - 1);
        if (g.n[d] > 1024) {
            set_error("grid too large for this build (FFT length > 1024 per axis)");
            return SIE_ERR_UNSUPPORTED;
        }
        if (g.n[d] < 16) g.n[d] = 16;
    }
    return SIE_OK;
}

void stencil_base(const HostMesh& m, const GridDesc& g, std::vector<int32_t>& base)
{
    base.resize(3 * m.nt);
    for (int64_t t = 0; t < m.nt; t++)
        for (int d = 0; d < 3; d++) {
            double x = (m.cen[3 * t + d] - g.o[d]) / g.h;
            base[3 * t + d] = (g.M % 2 == 0) ? (int32_t)std::floor(x + 0.5) - g.M / 2
                                             : (int32_t)std::floor(x) - (g.M - 1) / 2;
        }
}

void near_pairs_grid(const HostMesh& m, const GridDesc& g, const std::vector<int32_t>& base,
                     std::vector<int32_t>& pairs)
{
    // triangles sorted by stencil-centre cell (z, y, x); x-runs are contiguous
    const int64_t nt = m.nt, half = g.M / 2;
    auto key = [&](int64_t cx, int64_t cy, int64_t cz) { return (cz * (int64_t)g.N[1] + cy) * (int64_t)g.N[0] + cx; };
    std::vector<std::pair<int64_t, int32_t>> cells(nt);
    for (int64_t t = 0; t < nt; t++)
        cells[t] = {key(base[3 * t] + half, base[3 * t + 1] + half, base[3 * t + 2] + half), (int32_t)t};
    std::sort(cells.begin(), cells.end());
    const int R = g.Rnear;
    pairs.clear();
    std::vector<int32_t> lst;
    for (int64_t t = 0; t < nt; t++) {
        int64_t cx = base[3 * t] + half, cy = base[3 * t + 1] + half, cz = base[3 * t + 2] + half;
        lst.clear();
        for (int64_t dz = -R; dz <= R; dz++)
            for (int64_t dy = -R; dy <= R; dy++) {
                int64_t yy = cy + dy, zz = cz + dz;
                if (yy < 0 || zz < 0 || yy >= g.N[1] || zz >= g.N[2]) continue;
                int64_t k0 = key(std::max<int64_t>(cx - R, 0), yy, zz), k1 = key(std::min<int64_t>(cx + R, g.N[0] - 1), yy, zz);
                auto it = std::lower_bound(cells.begin(), cells.end(), std::make_pair(k0, (int32_t)-1));
                for (; it != cells.end() && it->first <= k1; ++it) lst.push_back(it->second);
            }
        std::sort(lst.begin(), lst.end());
        for (int32_t s : lst) {
            pairs.push_back((int32_t)t);
            pairs.push_back(s);
        }
    }
}

static bool touching(const HostMesh& m, int64_t t, int64_t s)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (m.T[3 * t + i] == m.T[3 * s + j]) return true;
    return false;
}

void near_pairs_cutoff(const HostMesh& m, double cutoff, std::vector<int32_t>& pairs)
{
    // uniform cells of size >= 2 max radius + cutoff: candidates lie in the 27 neighbours
    double rmax = 0, lo[3] = {1e300, 1e300, 1e300};
    for (int64_t t = 0; t < m.nt; t++) {
        rmax = std::max(rmax, m.rad[t]);
        for (int d = 0; d < 3; d++) lo[d] = std::min(lo[d], m.cen[3 * t + d]);
    }
    double cs = 2 * rmax + cutoff;
    auto cell = [&](int64_t t, int d) { return (int64_t)std::floor((m.cen[3 * t + d] - lo[d]) / cs); };
    std::vector<std::pair<std::tuple<int64_t, int64_t, int64_t>, int32_t>> cells(m.nt);
    for (int64_t t = 0; t < m.nt; t++) cells[t] = {{cell(t, 2), cell(t, 1), cell(t, 0)}, (int32_t)t};
    std::sort(cells.begin(), cells.end());
    pairs.clear();
    std::vector<int32_t> lst;
    for (int64_t t = 0; t < m.nt; t++) {
        lst.clear();
        int64_t cx = cell(t, 0), cy = cell(t, 1), cz = cell(t, 2);
        for (int64_t dz = -1; dz <= 1; dz++)
            for (int64_t dy = -1; dy <= 1; dy++) {
                auto k0 = std::make_pair(std::make_tuple(cz + dz, cy + dy, cx - 1), (int32_t)-1);
                auto it = std::lower_bound(cells.begin(), cells.end(), k0);
                for (; it != cells.end() && it->first <= std::make_tuple(cz + dz, cy + dy, cx + 1); ++it) {
                    int64_t s = it->second;
                    double dx = m.cen[3 * t] - m.cen[3 * s], dy2 = m.cen[3 * t + 1] - m.cen[3 * s + 1],
                           dz2 = m.cen[3 * t + 2] - m.cen[3 * s + 2];
                    double gap = std::sqrt(dx * dx + dy2 * dy2 + dz2 * dz2) - m.rad[t] - m.rad[s];
                    if (gap <= cutoff || touching(m, t, s)) lst.push_back((int32_t)s);
                }
            }
        std::sort(lst.begin(), lst.end());
        for (int32_t s : lst) {
            pairs.push_back((int32_t)t);
            pairs.push_back(s);
        }
    }
}

void near_pairs_cutoff_objects(const HostMesh& m, const std::vector<double>& cutoff, std::vector<int32_t>& pairs)
{
    double cmax = 0;
    for (double c : cutoff) cmax = std::max(cmax, c);
    std::vector<int32_t> all;
    near_pairs_cutoff(m, cmax, all);
    pairs.clear();
    for (size_t p = 0; p < all.size() / 2; p++) {
        const int32_t t = all[2 * p], s = all[2 * p + 1];
        const int ob = m.obj[t];
        if (m.obj[s] != ob) continue;
        const double dx = m.cen[3 * t] - m.cen[3 * s], dy = m.cen[3 * t + 1] - m.cen[3 * s + 1],
                     dz = m.cen[3 * t + 2] - m.cen[3 * s + 2];
        const double gap = std::sqrt(dx * dx + dy * dy + dz * dz) - m.rad[t] - m.rad[s];
        if (gap <= cutoff[ob] || touching(m, t, s)) {
            pairs.push_back(t);
            pairs.push_back(s);
        }
    }
}

void edge_csr_pattern(const HostMesh& m, const std::vector<int32_t>& pairs, CsrPattern& csr)
{
    std::vector<int64_t> start(m.nt + 1, 0);
    for (size_t p = 0; p < pairs.size() / 2; p++) start[pairs[2 * p] + 1]++;
    for (int64_t t = 0; t < m.nt; t++) start[t + 1] += start[t];
    csr.row_ptr.assign(m.ne + 1, 0);
    csr.col.clear();
    std::vector<int32_t> cols;
    for (int64_t e = 0; e < m.ne; e++) {
        cols.clear();
        for (int side = 0; side < 2; side++) {
            int64_t t = m.edge_tri[2 * e + side];
            for (int64_t p = start[t]; p < start[t + 1]; p++) {
                int64_t s = pairs[2 * p + 1];
                for (int j = 0; j < 3; j++) cols.push_back(m.tri_edge[3 * s + j]);
            }
        }
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        csr.col.insert(csr.col.end(), cols.begin(), cols.end());
        csr.row_ptr[e + 1] = (int64_t)csr.col.size();
    }
}

void gauss_legendre01(int n, double* x, double* w)
{
    for (int i = 0; i < n; i++) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) {
                p1 = z;
                p0 = 1;
            }
            pp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) p0 = 1;
            pp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        // node z in (-1,1) descending -> map to [0,1] ascending
        x[n - 1 - i] = 0.5 * (z + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * pp * pp);
    }
}

void make_quad(const sie_params& p, QuadDev& q)
{
    std::memset(&q, 0, sizeof(q));
    int ns[7] = {p.q_far, p.q_out, p.q_ang, p.q_rad, p.q_olam, p.q_omu, p.q_emu};
    for (int r = 0; r < 7; r++) {
        q.n[r] = ns[r];
        gauss_legendre01(ns[r], q.x[r], q.w[r]);
    }
    q.npan = p.q_npan;
    q.opan = p.q_opan;
    q.emupan = p.q_emupan;
    q.ratio = p.q_ratio;
    q.cf = p.q_cf;
    q.kres = p.q_kres;
    q.alen = p.q_alen;
    q.oratio = p.q_oratio;
}

static cudaEvent_t prof_event(Prof& p)
{
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

Stage::Stage(sie_ctx* ctx, const char* name) : c(ctx)
{
    if (!c || !c->prof.on) return;
    Prof& p = c->prof;
    for (size_t i = 0; i < p.names.size(); i++)
        if (p.names[i] == name) id = (int)i;
    if (id < 0) {
        id = (int)p.names.size();
        p.names.push_back(name);
        p.ms.push_back(0.0);
        p.count.push_back(0);
    }
    b = prof_event(p);
    cudaEventRecord(b, c->stream);
}

Stage::~Stage()
{
    if (id < 0) return;
    Prof& p = c->prof;
    cudaEvent_t e = prof_event(p);
    cudaEventRecord(e, c->stream);
    p.pending.push_back({id, b, e});  // (start, end)
}

static void prof_drain(Prof& p)
{
    for (auto& r : p.pending) {
        cudaEventSynchronize(r.b);
        float t = 0;
        cudaEventElapsedTime(&t, r.a, r.b);
        p.ms[r.stage] += t;
        p.count[r.stage] += 1;
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.pending.clear();
}

}  // namespace sie

using namespace sie;

// ------------------------------------------------------------------ C ABI
extern "C" {

void sie_params_default(sie_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->h = 0;
    p->h_over_edge = 0.5;
    p->grid_n = 0;
    p->stencil_order = 2;
    p->near_radius = 5;
    p->skin_cutoff = 5.0;
    p->precision = SIE_FP64;
    p->tol_outer = 1e-4;
    p->tol_inner = 1e-6;
    p->maxit = 800;
    p->restart = 100;
    p->inner_maxit = 200;
    p->tol_constraint = 1e-6;
    p->constraint_maxit = 1000;
    p->constraint_restart = 100;
    p->tol_constraint_inner = 1e-3;
    p->q_far = 5;
    p->q_out = 5;
    p->q_ang = 8;
    p->q_rad = 8;
    p->q_npan = 5;
    p->q_opan = 7;
    p->q_olam = 5;
    p->q_omu = 6;
    p->q_emupan = 2;
    p->q_emu = 4;
    p->q_ratio = 0.25;
    p->q_cf = 2.0;
    p->q_kres = 1.0;
    p->q_alen = 1.5;
    p->q_oratio = 0.25;
    p->dense_pc_max = 32768;
    p->interior_model = SIE_GIBC;
}

const char* sie_last_error(void) { return g_err.c_str(); }

sie_status sie_ctx_create(int device, void* stream, sie_ctx** out)
{
    if (!out) {
        set_error("sie_ctx_create: out is NULL");
        return SIE_ERR_ARG;
    }
    int nd = 0;
    SIE_CUDA_TRY(cudaGetDeviceCount(&nd));
    if (device < 0 || device >= nd) {
        set_error("sie_ctx_create: no such device");
        return SIE_ERR_ARG;
    }
    SIE_CUDA_TRY(cudaSetDevice(device));
    auto* c = new sie_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;  // NULL: the legacy default stream
    c->own_stream = false;
    *out = c;
    return SIE_OK;
}

sie_status sie_ctx_destroy(sie_ctx* ctx)
{
    if (!ctx) return SIE_ERR_ARG;
    cudaSetDevice(ctx->device);
    prof_drain(ctx->prof);
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return SIE_OK;
}

sie_status sie_profile_enable(sie_ctx* ctx, int enable)
{
    if (!ctx) return SIE_ERR_ARG;
    SIE_CUDA_TRY(cudaSetDevice(ctx->device));
    prof_drain(ctx->prof);
    if (enable) {
        std::fill(ctx->prof.ms.begin(), ctx->prof.ms.end(), 0.0);
        std::fill(ctx->prof.count.begin(), ctx->prof.count.end(), 0);
    }
    ctx->prof.on = enable != 0;
    return SIE_OK;
}

sie_status sie_profile_read(sie_ctx* ctx, int cap, char* names, double* ms, int64_t* count, int* n)
{
    if (!ctx || !n) return SIE_ERR_ARG;
    SIE_CUDA_TRY(cudaSetDevice(ctx->device));
    prof_drain(ctx->prof);
    const Prof& p = ctx->prof;
    *n = (int)p.names.size();
    for (int i = 0; i < *n && i < cap; i++) {
        if (names) {
            std::strncpy(names + 32 * i, p.names[i].c_str(), 31);
            names[32 * i + 31] = 0;
        }
        if (ms) ms[i] = p.ms[i];
        if (count) count[i] = p.count[i];
    }
    return SIE_OK;
}

sie_status sie_mesh_create(sie_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                           sie_mesh** out)
{
    if (!ctx || !out) {
        set_error("sie_mesh_create: null argument");
        return SIE_ERR_ARG;
    }
    auto* m = new sie_mesh();
    m->ctx = ctx;
    sie_status s = build_mesh(xyz, nv, tri, nt, m->h);
    if (s == SIE_OK) s = dev_upload_mesh(m);
    if (s != SIE_OK) {
        dev_free_mesh(m);
        delete m;
        return s;
    }
    m->mat.assign(1, sie_mesh::Material());
    *out = m;
    return SIE_OK;
}

sie_status sie_mesh_create_objects(sie_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                                   const int32_t* obj_id, sie_mesh** out, int* nobj)
{
    if (!ctx || !out) {
        set_error("sie_mesh_create_objects: null argument");
        return SIE_ERR_ARG;
    }
    auto* m = new sie_mesh();
    m->ctx = ctx;
    sie_status s = build_mesh(xyz, nv, tri, nt, m->h);
    if (s == SIE_OK && obj_id) s = set_objects(m->h, obj_id);
    if (s == SIE_OK) s = dev_upload_mesh(m);
    if (s != SIE_OK) {
        dev_free_mesh(m);
        delete m;
        return s;
    }
    m->mat.assign(m->h.nobj, sie_mesh::Material());
    if (nobj) *nobj = m->h.nobj;
    *out = m;
    return SIE_OK;
}

sie_status sie_set_material(sie_mesh* m, int obj, double eps_r, double mu_r, double sigma)
{
    if (!m || obj < 0 || obj >= m->h.nobj || !(eps_r > 0) || !(mu_r > 0) || !(sigma >= 0)) {
        set_error("sie_set_material: invalid object index or material");
        return SIE_ERR_ARG;
    }
    if ((int)m->mat.size() < m->h.nobj) m->mat.resize(m->h.nobj);
    m->mat[obj].set = true;
    m->mat[obj].eps_r = eps_r;
    m->mat[obj].mu_r = mu_r;
    m->mat[obj].sigma = sigma;
    return SIE_OK;
}

sie_status sie_mesh_destroy(sie_mesh* m)
{
    if (!m) return SIE_ERR_ARG;
    dev_free_mesh(m);
    delete m;
    return SIE_OK;
}

sie_status sie_mesh_counts(const sie_mesh* m, int64_t out[3])
{
    if (!m || !out) return SIE_ERR_ARG;
    out[0] = m->h.ne;
    out[1] = m->h.nt;
    out[2] = m->h.nv;
    return SIE_OK;
}

sie_status sie_op_info(const sie_op* op, double info[20])
{
    if (!op || !info) return SIE_ERR_ARG;
    const GridDesc& g = op->ext.g;
    for (int d = 0; d < 3; d++) {
        info[d] = g.N[d];
        info[3 + d] = g.n[d];
    }
    info[6] = g.h;
    info[7] = (double)op->ext.npairs;
    info[8] = (double)op->ext.nnz;
    info[9] = op->inn.has_grid ? 0.0 : 1.0;
    info[10] = (double)op->inn.npairs;
    info[11] = g.o[0];
    for (int i = 0; i < 4; i++) info[12 + i] = op->build_ms[i];
    info[16] = (op->gexec[0] ? 1.0 : 0.0) + (op->gexec[1] ? 2.0 : 0.0) + (op->gfailed ? 4.0 : 0.0);
    info[17] = (double)op->gnodes[0];
    info[18] = (double)op->gnodes[1];
    info[19] = op->lu_ms;
    return SIE_OK;
}

sie_status sie_op_set_solver(sie_op* op, const sie_params* p)
{
    if (!op || !p || !(p->tol_outer > 0) || !(p->tol_inner > 0) || p->maxit < 1 || p->restart < 1 ||
        p->inner_maxit < 1 || !(p->tol_constraint > 0) || p->constraint_maxit < 1 || p->constraint_restart < 1) {
        set_error("sie_op_set_solver: invalid argument");
        return SIE_ERR_ARG;
    }
    // the captured system-product graph bakes in the nested-solve settings
    if (p->tol_inner != op->p.tol_inner || p->inner_maxit != op->p.inner_maxit)
        sie::sys_graph_reset(op);
    op->p.tol_outer = p->tol_outer;
    op->p.tol_inner = p->tol_inner;
    op->p.maxit = p->maxit;
    op->p.restart = p->restart;
    op->p.inner_maxit = p->inner_maxit;
    op->p.tol_constraint = p->tol_constraint;
    op->p.constraint_maxit = p->constraint_maxit;
    op->p.constraint_restart = p->constraint_restart;
    if (p->tol_constraint_inner > 0) op->p.tol_constraint_inner = p->tol_constraint_inner;
    if (p->precision == SIE_FP64 || p->precision == SIE_MIXED) op->p.precision = p->precision;
    return SIE_OK;
}

sie_status sie_op_stats(const sie_op* op, double out[6])
{
    if (!op || !out) return SIE_ERR_ARG;
    sie::sys_stats_fold(const_cast<sie_op*>(op));  // nested-solve counts of graph runs
    for (int i = 0; i < 6; i++) out[i] = op->stats[i];
    return SIE_OK;
}

sie_status sie_op_grid(const sie_op* op, double origin[3], double* h, int64_t N[3])
{
    if (!op) return SIE_ERR_ARG;
    for (int d = 0; d < 3; d++) {
        if (origin) origin[d] = op->ext.g.o[d];
        if (N) N[d] = op->ext.g.N[d];
    }
    if (h) *h = op->ext.g.h;
    return SIE_OK;
}

}  // extern "C"
