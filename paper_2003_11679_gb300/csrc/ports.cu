// Delta-gap ports and network parameters.
//
// The paper drives its package and interconnect examples through ports
// (Sec. II admits a port excitation in place of the plane wave; Sec. V
// extracts S parameters) but only cites the port model.  The model here is
// the delta gap:
//   * a port is a closed loop of mesh edges cutting a conductor's surface,
//     selected by a plane (point o, unit normal n) and a radius: the edges
//     with both end points in the plane (within 1e-6 mean edge lengths) and
//     within the radius of o; each must separate its two triangles;
//   * s_m = +1 when T+ of edge m lies on the -n side (f_m then crosses the
//     loop along +n), and p_m = s_m l_m;
//   * the impressed field V delta(n . (r - o)) n enters Eq. (EFIE01dis) like
//     the incident field: b_m = -(V / eta0) p_m;
//   * the first block of the solution holds the RWG coefficients of -n x H
//     (the sign of Eq. EFIE01dis), so the current through the port along +n
//     is I = -p . H;
//   * Y_ij = I_i / V_j with the other ports shorted, S = (1 - z Y)(1 + z Y)^-1.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

using namespace sie;

namespace {

const double ETA0_P = 4e-7 * M_PI * 299792458.0;

// edges of one port (sorted by edge index) and their signed lengths s_m l_m
sie_status select_port(const HostMesh& m, const sie_port& pt, std::vector<int32_t>& edges,
                       std::vector<int32_t>& sign, std::vector<double>& w)
{
    double nn = std::sqrt(pt.normal[0] * pt.normal[0] + pt.normal[1] * pt.normal[1] + pt.normal[2] * pt.normal[2]);
    bool fin = std::isfinite(nn) && std::isfinite(pt.radius);
    for (int d = 0; d < 3; d++) fin = fin && std::isfinite(pt.origin[d]);
    if (!fin || !(nn > 0) || !(pt.radius > 0)) {
        set_error("port: origin, normal and radius must be finite, normal nonzero, radius positive");
        return SIE_ERR_ARG;
    }
    const double n[3] = {pt.normal[0] / nn, pt.normal[1] / nn, pt.normal[2] / nn};
    const double tol = 1e-6 * m.mean_edge;
    std::vector<double> dist(m.nv), rad(m.nv);
    for (int64_t v = 0; v < m.nv; v++) {
        double r[3] = {m.V[3 * v] - pt.origin[0], m.V[3 * v + 1] - pt.origin[1], m.V[3 * v + 2] - pt.origin[2]};
        dist[v] = r[0] * n[0] + r[1] * n[1] + r[2] * n[2];
        rad[v] = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    }
    auto in_port = [&](int64_t v) { return std::fabs(dist[v]) <= tol && rad[v] <= pt.radius; };
    auto side = [&](int32_t t) {
        double s = 0;
        for (int d = 0; d < 3; d++) s += (m.cen[3 * t + d] - pt.origin[d]) * n[d];
        return s;
    };
    std::vector<char> seen(m.ne, 0);
    edges.clear();
    for (int64_t t = 0; t < m.nt; t++)
        for (int i = 0; i < 3; i++) {
            int32_t e = m.tri_edge[3 * t + i];
            if (seen[e]) continue;
            seen[e] = 1;
            if (in_port(m.T[3 * t + (i + 1) % 3]) && in_port(m.T[3 * t + (i + 2) % 3])) edges.push_back(e);
        }
    if (edges.empty()) {
        set_error("port: no mesh edge lies in the port plane within the radius");
        return SIE_ERR_ARG;
    }
    std::sort(edges.begin(), edges.end());
    sign.resize(edges.size());
    w.resize(edges.size());
    for (size_t k = 0; k < edges.size(); k++) {
        int32_t e = edges[k];
        double sp = side(m.edge_tri[2 * e]), sm = side(m.edge_tri[2 * e + 1]);
        if (!(sp * sm < 0)) {
            set_error("port: edge " + std::to_string(e) + " lies in the port plane but does not separate its "
                      "two triangles");
            return SIE_ERR_ARG;
        }
        sign[k] = sp < 0 ? 1 : -1;
        w[k] = sign[k] * m.edge_len[e];
    }
    return SIE_OK;
}

// all ports: concatenated edge lists with offsets (host)
struct PortSet {
    std::vector<int32_t> edge, ptr{0};
    std::vector<double> w;
};

sie_status select_ports(const HostMesh& m, const sie_port* ports, int nport, PortSet& ps)
{
    std::vector<int32_t> e, s;
    std::vector<double> w;
    for (int i = 0; i < nport; i++) {
        sie_status st = select_port(m, ports[i], e, s, w);
        if (st != SIE_OK) {
            set_error("port " + std::to_string(i) + ": " + sie_last_error());
            return st;
        }
        ps.edge.insert(ps.edge.end(), e.begin(), e.end());
        ps.w.insert(ps.w.end(), w.begin(), w.end());
        ps.ptr.push_back((int32_t)ps.edge.size());
    }
    return SIE_OK;
}

// b_r = -(V_r / eta0) p_r on the first block of right-hand side r (the rest
// of b already zero): one thread per port edge
__global__ void k_port_rhs(int nport, const int32_t* __restrict__ ptr, const int32_t* __restrict__ edge,
                           const double* __restrict__ w, const double* __restrict__ volts, int64_t len,
                           double2* __restrict__ b)
{
    const int r = blockIdx.y;
    const double v = -volts[r] / ETA0_P;
    for (int k = ptr[r] + blockIdx.x * blockDim.x + threadIdx.x; k < ptr[r + 1]; k += gridDim.x * blockDim.x)
        b[r * len + edge[k]] = make_double2(v * w[k], 0.0);
}

// I[r * nport + i] = -sum_k w_k x_r[edge_k] over port i: one warp per (r, i)
__global__ void k_port_currents(int nport, int nrhs, const int32_t* __restrict__ ptr,
                                const int32_t* __restrict__ edge, const double* __restrict__ w, int64_t len,
                                const double2* __restrict__ x, double2* __restrict__ I)
{
    const int pair = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (pair >= nport * nrhs) return;
    const int r = pair / nport, i = pair % nport;
    double re = 0, im = 0;
    for (int k = ptr[i] + lane; k < ptr[i + 1]; k += 32) {
        double2 v = x[r * len + edge[k]];
        re += w[k] * v.x;
        im += w[k] * v.y;
    }
    for (int o = 16; o; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) I[pair] = make_double2(-re, -im);
}

// device copies of a port set (stream-ordered; freed with dev_ports_free)
struct DevPorts {
    int32_t *ptr = nullptr, *edge = nullptr;
    double* w = nullptr;
};

sie_status dev_ports(cudaStream_t st, const PortSet& ps, DevPorts& d)
{
    SIE_CUDA_TRY(cudaMallocAsync((void**)&d.ptr, sizeof(int32_t) * ps.ptr.size(), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&d.edge, sizeof(int32_t) * ps.edge.size(), st));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&d.w, sizeof(double) * ps.w.size(), st));
    SIE_CUDA_TRY(cudaMemcpyAsync(d.ptr, ps.ptr.data(), sizeof(int32_t) * ps.ptr.size(), cudaMemcpyHostToDevice, st));
    SIE_CUDA_TRY(cudaMemcpyAsync(d.edge, ps.edge.data(), sizeof(int32_t) * ps.edge.size(), cudaMemcpyHostToDevice, st));
    SIE_CUDA_TRY(cudaMemcpyAsync(d.w, ps.w.data(), sizeof(double) * ps.w.size(), cudaMemcpyHostToDevice, st));
    return SIE_OK;
}

void dev_ports_free(cudaStream_t st, DevPorts& d)
{
    if (d.ptr) cudaFreeAsync(d.ptr, st);
    if (d.edge) cudaFreeAsync(d.edge, st);
    if (d.w) cudaFreeAsync(d.w, st);
    d = DevPorts{};
}

// b (device): nport right-hand sides, port r driven with volts_h[r]
sie_status port_rhs_dev(sie_op* op, const PortSet& ps, const DevPorts& d, int nport, const double* volts_h,
                        double2* b)
{
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    double* vd = nullptr;
    SIE_CUDA_TRY(cudaMallocAsync((void**)&vd, sizeof(double) * nport, st));
    std::vector<double> v(nport, 1.0);
    if (volts_h) v.assign(volts_h, volts_h + nport);
    cudaError_t e = cudaMemcpyAsync(vd, v.data(), sizeof(double) * nport, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b, 0, sizeof(double2) * len * nport, st);
    if (e == cudaSuccess) {
        int most = 0;
        for (int i = 0; i < nport; i++) most = std::max(most, ps.ptr[i + 1] - ps.ptr[i]);
        dim3 grid((unsigned)std::max(1, (most + 255) / 256), (unsigned)nport);
        k_port_rhs<<<grid, 256, 0, st>>>(nport, d.ptr, d.edge, d.w, vd, len, b);
        e = cudaGetLastError();
    }
    // the host vector v must outlive the copy
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFreeAsync(vd, st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        set_error(std::string("port right-hand sides: ") + cudaGetErrorString(e));
        return SIE_ERR_CUDA;
    }
    return SIE_OK;
}

// I (host, nrhs x nport) from device solutions x
sie_status port_currents_dev(sie_op* op, const DevPorts& d, int nport, const double2* x, int nrhs, double2* I_h)
{
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    double2* Id = nullptr;
    SIE_CUDA_TRY(cudaMallocAsync((void**)&Id, sizeof(double2) * nport * nrhs, st));
    const int pairs = nport * nrhs;
    k_port_currents<<<(pairs + 7) / 8, 256, 0, st>>>(nport, nrhs, d.ptr, d.edge, d.w, len, x, Id);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(I_h, Id, sizeof(double2) * pairs, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(Id, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        set_error(std::string("port currents: ") + cudaGetErrorString(e));
        return SIE_ERR_CUDA;
    }
    return SIE_OK;
}

}  // namespace

extern "C" {

sie_status sie_port_edges(const sie_mesh* mesh, const sie_port* port, int32_t* edge, int32_t* sign, int64_t* n)
{
    if (!mesh || !port || !n) {
        set_error("sie_port_edges: invalid argument");
        return SIE_ERR_ARG;
    }
    std::vector<int32_t> e, s;
    std::vector<double> w;
    SIE_TRY(select_port(mesh->h, *port, e, s, w));
    if (edge && sign) {
        if (*n < (int64_t)e.size()) {
            set_error("sie_port_edges: buffers hold fewer entries than the port has edges");
            return SIE_ERR_ARG;
        }
        std::memcpy(edge, e.data(), sizeof(int32_t) * e.size());
        std::memcpy(sign, s.data(), sizeof(int32_t) * s.size());
    }
    *n = (int64_t)e.size();
    return SIE_OK;
}

sie_status sie_rhs_ports(sie_op* op, const sie_port* ports, int nport, const double* volts, double* b, int flags)
{
    if (!op || !ports || !b || nport < 1) {
        set_error("sie_rhs_ports: invalid argument");
        return SIE_ERR_ARG;
    }
    PortSet ps;
    SIE_TRY(select_ports(op->mesh->h, ports, nport, ps));
    SIE_CUDA_TRY(cudaSetDevice(op->mesh->ctx->device));
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    const bool dev = flags & SIE_DEVICE_PTRS;
    DevPorts d;
    double2* bd = dev ? (double2*)b : nullptr;
    sie_status s = dev_ports(st, ps, d);
    if (s == SIE_OK && !dev) {
        cudaError_t e = cudaMallocAsync((void**)&bd, sizeof(double2) * len * nport, st);
        if (e != cudaSuccess) {
            set_error(std::string("sie_rhs_ports: ") + cudaGetErrorString(e));
            s = e == cudaErrorMemoryAllocation ? SIE_ERR_OOM : SIE_ERR_CUDA;
        }
    }
    if (s == SIE_OK) s = port_rhs_dev(op, ps, d, nport, volts, bd);
    if (s == SIE_OK && !dev) {
        cudaError_t e = cudaMemcpyAsync(b, bd, sizeof(double2) * len * nport, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("sie_rhs_ports: ") + cudaGetErrorString(e));
            s = SIE_ERR_CUDA;
        }
    }
    if (!dev && bd) cudaFreeAsync(bd, st);
    dev_ports_free(st, d);
    return s;
}

sie_status sie_port_currents(sie_op* op, const sie_port* ports, int nport, const double* x, int nrhs, double* I,
                             int flags)
{
    if (!op || !ports || !x || !I || nport < 1 || nrhs < 1) {
        set_error("sie_port_currents: invalid argument");
        return SIE_ERR_ARG;
    }
    PortSet ps;
    SIE_TRY(select_ports(op->mesh->h, ports, nport, ps));
    SIE_CUDA_TRY(cudaSetDevice(op->mesh->ctx->device));
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    const bool dev = flags & SIE_DEVICE_PTRS;
    DevPorts d;
    double2* xd = dev ? (double2*)x : nullptr;
    sie_status s = dev_ports(st, ps, d);
    if (s == SIE_OK && !dev) {
        cudaError_t e = cudaMallocAsync((void**)&xd, sizeof(double2) * len * nrhs, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(xd, x, sizeof(double2) * len * nrhs, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            set_error(std::string("sie_port_currents: ") + cudaGetErrorString(e));
            s = e == cudaErrorMemoryAllocation ? SIE_ERR_OOM : SIE_ERR_CUDA;
        }
    }
    if (s == SIE_OK) s = port_currents_dev(op, d, nport, xd, nrhs, (double2*)I);
    if (!dev && xd) cudaFreeAsync(xd, st);
    dev_ports_free(st, d);
    cudaStreamSynchronize(st);
    return s;
}

sie_status sie_port_admittance(sie_op* op, const sie_port* ports, int nport, double* Y, int* iters, double* relres,
                               int flags)
{
    if (!op || !ports || !Y || nport < 1 || (flags & SIE_DEVICE_PTRS)) {
        set_error("sie_port_admittance: invalid argument");
        return SIE_ERR_ARG;
    }
    PortSet ps;
    SIE_TRY(select_ports(op->mesh->h, ports, nport, ps));
    SIE_CUDA_TRY(cudaSetDevice(op->mesh->ctx->device));
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    DevPorts d;
    double2* bx = nullptr;  // b then x, nport vectors each
    sie_status s = dev_ports(st, ps, d);
    if (s == SIE_OK) {
        cudaError_t e = cudaMallocAsync((void**)&bx, sizeof(double2) * 2 * len * nport, st);
        if (e != cudaSuccess) {
            set_error(std::string("sie_port_admittance: ") + cudaGetErrorString(e));
            s = e == cudaErrorMemoryAllocation ? SIE_ERR_OOM : SIE_ERR_CUDA;
        }
    }
    sie_status solved = SIE_OK;
    std::vector<double2> Ih((size_t)nport * nport);
    if (s == SIE_OK) s = port_rhs_dev(op, ps, d, nport, nullptr, bx);
    if (s == SIE_OK) {
        // one right-hand side per port, in lockstep blocks (or one after another)
        solved = sie_solve(op, (const double*)bx, (double*)(bx + len * nport), nport, iters, relres,
                           SIE_DEVICE_PTRS | (flags & (SIE_SOLVE_REFINE | SIE_SOLVE_SEQUENTIAL)));
        if (solved != SIE_OK && solved != SIE_ERR_NOT_CONVERGED) s = solved;
    }
    if (s == SIE_OK) s = port_currents_dev(op, d, nport, bx + len * nport, nport, Ih.data());
    if (bx) cudaFreeAsync(bx, st);
    dev_ports_free(st, d);
    cudaStreamSynchronize(st);
    if (s != SIE_OK) return s;
    // Ih[j * nport + i] = current through port i for right-hand side j (1 V on port j)
    for (int i = 0; i < nport; i++)
        for (int j = 0; j < nport; j++) {
            Y[2 * (i * nport + j)] = Ih[j * nport + i].x;
            Y[2 * (i * nport + j) + 1] = Ih[j * nport + i].y;
        }
    if (solved == SIE_ERR_NOT_CONVERGED) set_error("sie_port_admittance: a port's solve reached maxit");
    return solved;
}

sie_status sie_port_sparams(int nport, const double* Y, double z_ref, double* S)
{
    if (nport < 1 || !Y || !S || !(z_ref > 0) || !std::isfinite(z_ref)) {
        set_error("sie_port_sparams: invalid argument");
        return SIE_ERR_ARG;
    }
    // S = (1 - z Y)(1 + z Y)^-1, i.e. S^T = (1 + z Y)^-T (1 - z Y)^T: solve
    // (1 + z Y)^T S^T = (1 - z Y)^T by Gaussian elimination with partial pivoting
    const int n = nport;
    std::vector<double2> A((size_t)n * n), B((size_t)n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double yr = Y[2 * (j * n + i)], yi = Y[2 * (j * n + i) + 1];  // (Y^T)_ij
            double d = i == j ? 1.0 : 0.0;
            A[i * n + j] = make_double2(d + z_ref * yr, z_ref * yi);
            B[i * n + j] = make_double2(d - z_ref * yr, -z_ref * yi);
        }
    auto mul = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int i = k + 1; i < n; i++)
            if (std::hypot(A[i * n + k].x, A[i * n + k].y) > std::hypot(A[p * n + k].x, A[p * n + k].y)) p = i;
        double piv = std::hypot(A[p * n + k].x, A[p * n + k].y);
        if (!(piv > 0)) {
            set_error("sie_port_sparams: 1 + z_ref Y is singular");
            return SIE_ERR_ARG;
        }
        if (p != k)
            for (int j = 0; j < n; j++) {
                std::swap(A[k * n + j], A[p * n + j]);
                std::swap(B[k * n + j], B[p * n + j]);
            }
        double2 a = A[k * n + k];
        double den = a.x * a.x + a.y * a.y;
        double2 inv = make_double2(a.x / den, -a.y / den);
        for (int i = k + 1; i < n; i++) {
            double2 f = mul(A[i * n + k], inv);
            for (int j = k; j < n; j++) {
                double2 t = mul(f, A[k * n + j]);
                A[i * n + j].x -= t.x;
                A[i * n + j].y -= t.y;
            }
            for (int j = 0; j < n; j++) {
                double2 t = mul(f, B[k * n + j]);
                B[i * n + j].x -= t.x;
                B[i * n + j].y -= t.y;
            }
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        double2 a = A[k * n + k];
        double den = a.x * a.x + a.y * a.y;
        double2 inv = make_double2(a.x / den, -a.y / den);
        for (int j = 0; j < n; j++) {
            double2 acc = B[k * n + j];
            for (int c = k + 1; c < n; c++) {
                double2 t = mul(A[k * n + c], B[c * n + j]);
                acc.x -= t.x;
                acc.y -= t.y;
            }
            B[k * n + j] = mul(acc, inv);
        }
    }
    // B = S^T
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            S[2 * (i * n + j)] = B[j * n + i].x;
            S[2 * (i * n + j) + 1] = B[j * n + i].y;
        }
    return SIE_OK;
}

}  // extern "C"
