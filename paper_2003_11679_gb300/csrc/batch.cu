// Multi-right-hand-side AIM products (Eqs. AIM_Lin, AIM_Kin) for a block of up
// to RB vectors: the kernel spectra, the stencil weights and the near-region
// values are read once per block instead of once per vector.
//   * projection: one grid of CTAs per right-hand side (weights from L2);
//   * FFTs: one launch per pass over all grids of the block;
//   * spectral multiply: G (or grad G) loaded once per node, applied to every
//     vector of the block;
//   * interpolation: one grid of CTAs per right-hand side;
//   * near region: CSR x panel product, each (column, value) pair loaded once
//     and multiplied into RB accumulators.
// Vectors are rhs-major (vector r at r * len), as everywhere in the ABI.
#include <algorithm>
#include <complex>

#include "internal.h"

namespace sie {

constexpr int RB = 8;  // right-hand sides per block

// projection of vector r = blockIdx.y into grids src + (r * ngrid + a) * Ng
__global__ void k_project_b(int nt, int S, int Mord, DevMesh M, const int32_t* __restrict__ base,
                            const double* __restrict__ W, const double2* __restrict__ x, int64_t ldx, GridDesc g,
                            int ngrid, double2* __restrict__ src, int64_t Ng)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nt * S) return;
    const int r = blockIdx.y;
    x += (int64_t)r * ldx;
    src += (int64_t)r * ngrid * Ng;
    int t = idx / S, u = idx % S;
    const int Mp = Mord + 1;
    double2 al = make_double2(0, 0);
    double2 be[3] = {al, al, al};
    for (int i = 0; i < 3; i++) {
        double2 xv = x[M.tri_edge[3 * t + i]];
        double c = M.coef[3 * t + i];
        al.x += c * xv.x;
        al.y += c * xv.y;
        for (int a = 0; a < 3; a++) {
            double qq = c * M.q[9 * t + 3 * i + a];
            be[a].x += qq * xv.x;
            be[a].y += qq * xv.y;
        }
    }
    int nx = base[3 * t] + u % Mp, ny = base[3 * t + 1] + (u / Mp) % Mp, nz = base[3 * t + 2] + u / (Mp * Mp);
    int64_t node = ((int64_t)nz * g.N[1] + ny) * g.N[0] + nx;
    const double* w = W + (size_t)idx * 4;
    for (int a = 0; a < 3; a++) {
        double2* d = src + a * Ng + node;
        atomicAdd(&d->x, al.x * w[1 + a] + be[a].x * w[0]);
        atomicAdd(&d->y, al.y * w[1 + a] + be[a].y * w[0]);
    }
    if (ngrid == 4) {
        double2* d = src + 3 * Ng + node;
        atomicAdd(&d->x, 2.0 * al.x * w[0]);
        atomicAdd(&d->y, 2.0 * al.y * w[0]);
    }
}

// spectral multiply of nr vectors, the spectra read once per node: mode 0
// (L): every grid times G; mode 1 (K): J <- grad G x J
__global__ void k_specmul_b(int mode, int nr, const double2* __restrict__ spec, double2* __restrict__ buf, int64_t nn)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    auto mul = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
    if (mode == 0) {
        const double2 G = spec[i];
        for (int c = 0; c < 4 * nr; c++) buf[c * nn + i] = mul(G, buf[c * nn + i]);
    } else {
        const double2 gx = spec[nn + i], gy = spec[2 * nn + i], gz = spec[3 * nn + i];
        for (int r = 0; r < nr; r++) {
            double2* b = buf + (int64_t)3 * r * nn;
            double2 jx = b[i], jy = b[nn + i], jz = b[2 * nn + i];
            double2 p = mul(gy, jz), q = mul(gz, jy);
            b[i] = make_double2(p.x - q.x, p.y - q.y);
            p = mul(gz, jx);
            q = mul(gx, jz);
            b[nn + i] = make_double2(p.x - q.x, p.y - q.y);
            p = mul(gx, jy);
            q = mul(gy, jx);
            b[2 * nn + i] = make_double2(p.x - q.x, p.y - q.y);
        }
    }
}

// interpolation of vector r = blockIdx.y: one warp per triangle, y[e] +=
// c_{t,i} [S1 + (c_t - p_i).T0 + scal 2 P0]
__global__ void k_interp_b(int nt, int S, int Mord, DevMesh M, const int32_t* __restrict__ base,
                           const double* __restrict__ W, const double2* __restrict__ out, GridDesc g, int ngrid,
                           double2 scal, int64_t Ng, double2* __restrict__ y, int64_t ldy)
{
    int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (t >= nt) return;
    const int r = blockIdx.y;
    out += (int64_t)r * ngrid * Ng;
    y += (int64_t)r * ldy;
    const int Mp = Mord + 1;
    double s1r = 0, s1i = 0, t0r[3] = {0, 0, 0}, t0i[3] = {0, 0, 0}, p0r = 0, p0i = 0;
    for (int u = lane; u < S; u += 32) {
        int nx = base[3 * t] + u % Mp, ny = base[3 * t + 1] + (u / Mp) % Mp, nz = base[3 * t + 2] + u / (Mp * Mp);
        int64_t node = ((int64_t)nz * g.N[1] + ny) * g.N[0] + nx;
        const double* w = W + ((size_t)t * S + u) * 4;
        for (int a = 0; a < 3; a++) {
            double2 A = out[a * Ng + node];
            s1r += w[1 + a] * A.x;
            s1i += w[1 + a] * A.y;
            t0r[a] += w[0] * A.x;
            t0i[a] += w[0] * A.y;
        }
        if (ngrid == 4) {
            double2 P = out[3 * Ng + node];
            p0r += w[0] * P.x;
            p0i += w[0] * P.y;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        s1r += __shfl_down_sync(0xffffffffu, s1r, off);
        s1i += __shfl_down_sync(0xffffffffu, s1i, off);
        p0r += __shfl_down_sync(0xffffffffu, p0r, off);
        p0i += __shfl_down_sync(0xffffffffu, p0i, off);
        for (int a = 0; a < 3; a++) {
            t0r[a] += __shfl_down_sync(0xffffffffu, t0r[a], off);
            t0i[a] += __shfl_down_sync(0xffffffffu, t0i[a], off);
        }
    }
    if (lane < 3) {
        const int i = lane;
        double S1r = __shfl_sync(0x7u, s1r, 0), S1i = __shfl_sync(0x7u, s1i, 0);
        double P0r = __shfl_sync(0x7u, p0r, 0), P0i = __shfl_sync(0x7u, p0i, 0);
        double T0r[3], T0i[3];
        for (int a = 0; a < 3; a++) {
            T0r[a] = __shfl_sync(0x7u, t0r[a], 0);
            T0i[a] = __shfl_sync(0x7u, t0i[a], 0);
        }
        double vr = S1r, vi = S1i;
        for (int a = 0; a < 3; a++) {
            double qq = M.q[9 * t + 3 * i + a];
            vr += qq * T0r[a];
            vi += qq * T0i[a];
        }
        vr += 2.0 * (scal.x * P0r - scal.y * P0i);
        vi += 2.0 * (scal.x * P0i + scal.y * P0r);
        double c = M.coef[3 * t + i];
        double2* d = y + M.tri_edge[3 * t + i];
        atomicAdd(&d->x, c * vr);
        atomicAdd(&d->y, c * vi);
    }
}

// Y[r] (+)= A X[r] for r < NR: a warp per row; each (column, value) pair
// loaded once, its product accumulated into NR sums per lane
template <int NR>
__global__ void __launch_bounds__(128) k_csr_panel(int nrow, const int64_t* __restrict__ rp,
                                                   const int32_t* __restrict__ col, const double2* __restrict__ val,
                                                   const double2* __restrict__ X, int64_t ldx, int acc,
                                                   double2* __restrict__ Y, int64_t ldy)
{
    const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= nrow) return;
    double sr[NR], si[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) sr[k] = si[k] = 0.0;
    for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
        const int c = __ldg(col + e);
        const double2 v = __ldg(val + e);
#pragma unroll
        for (int k = 0; k < NR; k++) {
            const double2 xv = __ldg(X + k * ldx + c);
            sr[k] += v.x * xv.x - v.y * xv.y;
            si[k] += v.x * xv.y + v.y * xv.x;
        }
    }
#pragma unroll
    for (int k = 0; k < NR; k++) {
        for (int off = 16; off > 0; off >>= 1) {
            sr[k] += __shfl_xor_sync(0xffffffffu, sr[k], off);
            si[k] += __shfl_xor_sync(0xffffffffu, si[k], off);
        }
    }
    if (lane < NR) {
        double yr = 0, yi = 0;
#pragma unroll
        for (int k = 0; k < NR; k++)
            if (k == lane) {
                yr = sr[k];
                yi = si[k];
            }
        double2* o = Y + lane * ldy + r;
        if (acc) {
            yr += o->x;
            yi += o->y;
        }
        *o = make_double2(yr, yi);
    }
}

sie_status csr_panel(cudaStream_t st, int nrow, const int64_t* rp, const int32_t* col, const double2* val,
                            const double2* X, int64_t ldx, int nr, bool acc, double2* Y, int64_t ldy)
{
    const unsigned blocks = (unsigned)((nrow + 3) / 4);
    switch (nr) {
        case 1: k_csr_panel<1><<<blocks, 128, 0, st>>>(nrow, rp, col, val, X, ldx, acc, Y, ldy); break;
        case 2: k_csr_panel<2><<<blocks, 128, 0, st>>>(nrow, rp, col, val, X, ldx, acc, Y, ldy); break;
        case 3: k_csr_panel<3><<<blocks, 128, 0, st>>>(nrow, rp, col, val, X, ldx, acc, Y, ldy); break;
        case 4: k_csr_panel<4><<<blocks, 128, 0, st>>>(nrow, rp, col, val, X, ldx, acc, Y, ldy); break;
        case 5: k_csr_panel<5><<<blocks, 128, 0, st>>>(nrow, rp, col, val, X, ldx, acc, Y, ldy); break;
        case 6: k_csr_panel<6><<<blocks, 128, 0, st>>>(nrow, rp, col, val, X, ldx, acc, Y, ldy); break;
        case 7: k_csr_panel<7><<<blocks, 128, 0, st>>>(nrow, rp, col, val, X, ldx, acc, Y, ldy); break;
        default: k_csr_panel<8><<<blocks, 128, 0, st>>>(nrow, rp, col, val, X, ldx, acc, Y, ldy); break;
    }
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// the block workspace: padded and compact grids for RB vectors of 4 grids
static sie_status batch_workspace(sie_op* op, double2** bufs, double2** src)
{
    const GridDesc& g = op->ext.g;
    const int64_t nn = (int64_t)g.n[0] * g.n[1] * g.n[2], Ng = (int64_t)g.N[0] * g.N[1] * g.N[2];
    cudaStream_t st = op->mesh->ctx->stream;
    if (!op->bws_bufs) {
        SIE_CUDA_TRY(cudaMallocAsync((void**)&op->bws_bufs, sizeof(double2) * 4 * RB * nn, st));
        SIE_CUDA_TRY(cudaMallocAsync((void**)&op->bws_src, sizeof(double2) * 4 * RB * Ng, st));
    }
    *bufs = op->bws_bufs;
    *src = op->bws_src;
    return SIE_OK;
}

// Y = A X for nr vectors (nr <= RB, rhs-major, length N_e), A = L (which_LK 0)
// or K (1) of operator a
sie_status aim_apply_block(sie_op* op, AimOp& a, int which_LK, const double2* X, double2* Y, int nr)
{
    sie_ctx* pc = op->mesh->ctx;
    cudaStream_t st = pc->stream;
    const DevMesh& M = op->mesh->d;
    const int64_t ne = M.ne;
    if (nr < 1 || nr > RB) {
        set_error("aim_apply_block: block size out of range");
        return SIE_ERR_ARG;
    }
    if (a.has_grid) {
        SIE_CUDA_TRY(cudaMemsetAsync(Y, 0, sizeof(double2) * ne * nr, st));
        const GridDesc& g = a.g;
        const int S = (g.M + 1) * (g.M + 1) * (g.M + 1);
        const int64_t Ng = (int64_t)g.N[0] * g.N[1] * g.N[2];
        const int64_t nn = (int64_t)g.n[0] * g.n[1] * g.n[2];
        const int ngrid = which_LK == 0 ? 4 : 3;
        double2 *buf, *src;
        SIE_TRY(batch_workspace(op, &buf, &src));
        {
            Stage s_(pc, "project_block");
            SIE_CUDA_TRY(cudaMemsetAsync(src, 0, sizeof(double2) * ngrid * nr * Ng, st));
            k_project_b<<<dim3((M.nt * S + 255) / 256, nr), 256, 0, st>>>(M.nt, S, g.M, M, op->base, op->W, X, ne, g,
                                                                           ngrid, src, Ng);
            SIE_CUDA_TRY(cudaGetLastError());
        }
        SIE_TRY(fft3d(st, buf, src, g, -1, 1, pc, ngrid * nr));
        {
            Stage s_(pc, "specmul_block");
            k_specmul_b<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(which_LK, nr, a.spec, buf, nn);
            SIE_CUDA_TRY(cudaGetLastError());
        }
        SIE_TRY(fft3d(st, buf, src, g, +1, 1, pc, ngrid * nr));
        std::complex<double> kk(a.kr, a.ki);
        std::complex<double> sc = which_LK == 0 ? -1.0 / (kk * kk) : std::complex<double>(0.0);
        {
            Stage s_(pc, "interp_block");
            k_interp_b<<<dim3((M.nt + 3) / 4, nr), 128, 0, st>>>(M.nt, S, g.M, M, op->base, op->W, src, g, ngrid,
                                                                 make_double2(sc.real(), sc.imag()), Ng, Y, ne);
            SIE_CUDA_TRY(cudaGetLastError());
        }
    }
    {
        Stage s_(pc, a.has_grid ? "spmv_block" : "spmv_near_only_block");
        const double2* v = which_LK == 0 ? a.valL : a.valK;
        SIE_TRY(csr_panel(st, (int)ne, a.row_ptr, a.col, v, X, ne, nr, a.has_grid, Y, ne));
    }
    return SIE_OK;
}

}  // namespace sie
