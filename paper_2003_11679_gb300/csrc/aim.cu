// AIM grid path of Eqs. (AIM_Lin), (AIM_Kin) on sm_103a:
//   projection P / P_phi (moment-matching stencils, scatter),
//   zero-padded 3D FFT (shared-memory radix-2 pencils, pruned passes),
//   spectral multiply with the sampled Green's function and its gradient,
//   pruned inverse FFT, interpolation W = P^T (gather), and the
//   precorrected near-region CSR product (Eqs. LinNRP, KinNRP).
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "spmv.cuh"
#include "sysmul.cuh"

namespace sie {

// ------------------------------------------------------------------ device mesh
template <class T>
static sie_status up(cudaStream_t st, T** d, const T* h, size_t n)
{
    SIE_CUDA_TRY(cudaMallocAsync((void**)d, sizeof(T) * std::max<size_t>(n, 1), st));
    SIE_CUDA_TRY(cudaMemcpyAsync(*d, h, sizeof(T) * n, cudaMemcpyHostToDevice, st));
    return SIE_OK;
}

sie_status dev_upload_mesh(sie_mesh* m)
{
    cudaStream_t st = m->ctx->stream;
    const HostMesh& h = m->h;
    DevMesh& d = m->d;
    d.nt = (int)h.nt;
    d.ne = (int)h.ne;
    d.nv = (int)h.nv;
    SIE_TRY(up(st, &d.V, h.V.data(), h.V.size()));
    SIE_TRY(up(st, &d.T, h.T.data(), h.T.size()));
    SIE_TRY(up(st, &d.tri_edge, h.tri_edge.data(), h.tri_edge.size()));
    SIE_TRY(up(st, &d.coef, h.coef.data(), h.coef.size()));
    SIE_TRY(up(st, &d.q, h.q.data(), h.q.size()));
    SIE_TRY(up(st, &d.cen, h.cen.data(), h.cen.size()));
    SIE_TRY(up(st, &d.area, h.area.data(), h.area.size()));
    SIE_TRY(up(st, &d.rad, h.rad.data(), h.rad.size()));
    SIE_TRY(up(st, &d.edge_tri, h.edge_tri.data(), h.edge_tri.size()));
    SIE_TRY(up(st, &d.edge_slot, h.edge_slot.data(), h.edge_slot.size()));
    SIE_TRY(up(st, &d.obj, h.obj.data(), h.obj.size()));
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    return SIE_OK;
}

sie_status dev_free_mesh(sie_mesh* m)
{
    DevMesh& d = m->d;
    void* ptrs[] = {d.V, d.T, d.tri_edge, d.coef, d.q, d.cen, d.area, d.rad, d.edge_tri, d.edge_slot, d.obj};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    d = DevMesh();
    return SIE_OK;
}

// ------------------------------------------------------------------ weights (moment matching)
__constant__ double c_glx[16], c_glw[16];

// w[t][u] = (I_t l_u, I_t (r - c_t) l_u): tensor Lagrange basis of order M on the
// stencil nodes base + {0..M}^3, collapsed Gauss rule with p points per direction.
__global__ void k_weights(int nt, int Mord, int p, DevMesh M, const int32_t* __restrict__ base, double ox, double oy,
                          double oz, double h, double* __restrict__ W)
{
    const int Mp = Mord + 1, S = Mp * Mp * Mp;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nt * S) return;
    int t = idx / S, u = idx % S;
    int ux = u % Mp, uy = (u / Mp) % Mp, uz = u / (Mp * Mp);
    const double* a = M.V + 3 * M.T[3 * t];
    const double* b = M.V + 3 * M.T[3 * t + 1];
    const double* c = M.V + 3 * M.T[3 * t + 2];
    double e1[3], e2[3];
    for (int d = 0; d < 3; d++) {
        e1[d] = b[d] - a[d];
        e2[d] = c[d] - a[d];
    }
    double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2], nz = e1[0] * e2[1] - e1[1] * e2[0];
    double twoA = sqrt(nx * nx + ny * ny + nz * nz);
    const double o[3] = {ox, oy, oz};
    const int uu[3] = {ux, uy, uz};
    double w0 = 0, w1[3] = {0, 0, 0};
    for (int i = 0; i < p; i++) {
        double uq = c_glx[i];
        for (int j = 0; j < p; j++) {
            double vq = c_glx[j] * (1.0 - uq);
            double wq = twoA * (1.0 - uq) * c_glw[i] * c_glw[j];
            double r[3], l = 1.0;
            for (int d = 0; d < 3; d++) {
                r[d] = a[d] + uq * e1[d] + vq * e2[d];
                double xi = (r[d] - o[d]) / h - base[3 * t + d];
                for (int m = 0; m < Mp; m++)
                    if (m != uu[d]) l *= (xi - m) / (double)(uu[d] - m);
            }
            w0 += wq * l;
            for (int d = 0; d < 3; d++) w1[d] += wq * (r[d] - M.cen[3 * t + d]) * l;
        }
    }
    double* o4 = W + (size_t)idx * 4;
    o4[0] = w0;
    o4[1] = w1[0];
    o4[2] = w1[1];
    o4[3] = w1[2];
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// complex64 copy of a complex128 array (allocated here)
static sie_status to_c64(cudaStream_t st, const double2* a, int64_t n, float2** out)
{
    SIE_CUDA_TRY(cudaMallocAsync((void**)out, sizeof(float2) * std::max<int64_t>(n, 1), st));
    if (n > 0) k_to_f32<<<(unsigned)((2 * n + 255) / 256), 256, 0, st>>>((const double*)a, (float*)*out, 2 * n);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// out[e] = (a[e], b[e]) in complex64: two matrices of one pattern interleaved
__global__ void k_to_c64_pair(const double2* __restrict__ a, const double2* __restrict__ b, float4* __restrict__ out,
                              int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float4((float)a[i].x, (float)a[i].y, (float)b[i].x, (float)b[i].y);
}

static sie_status to_c64_pair(cudaStream_t st, const double2* a, const double2* b, int64_t n, float4** out)
{
    SIE_CUDA_TRY(cudaMallocAsync((void**)out, sizeof(float4) * std::max<int64_t>(n, 1), st));
    if (n > 0) k_to_c64_pair<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, *out, n);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

sie_status aim_weights(sie_op* op)
{
    cudaStream_t st = op->mesh->ctx->stream;
    const GridDesc& g = op->ext.g;
    int p = (3 * g.M + 4) / 2;  // ceil((3M+3)/2): exact to degree 3M+1
    double x[16], w[16];
    gauss_legendre01(p, x, w);
    SIE_CUDA_TRY(cudaMemcpyToSymbolAsync(c_glx, x, sizeof(double) * p, 0, cudaMemcpyHostToDevice, st));
    SIE_CUDA_TRY(cudaMemcpyToSymbolAsync(c_glw, w, sizeof(double) * p, 0, cudaMemcpyHostToDevice, st));
    int S = (g.M + 1) * (g.M + 1) * (g.M + 1);
    int nt = op->mesh->d.nt;
    SIE_CUDA_TRY(cudaMallocAsync((void**)&op->W, sizeof(double) * 4 * (size_t)nt * S, st));
    k_weights<<<(nt * S + 127) / 128, 128, 0, st>>>(nt, g.M, p, op->mesh->d, op->base, g.o[0], g.o[1], g.o[2], g.h,
                                                    op->W);
    SIE_CUDA_TRY(cudaGetLastError());
    SIE_CUDA_TRY(cudaMallocAsync((void**)&op->W32, sizeof(float) * 4 * (size_t)nt * S, st));
    k_to_f32<<<(unsigned)((4 * (size_t)nt * S + 255) / 256), 256, 0, st>>>(op->W, op->W32, 4 * (int64_t)nt * S);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// ------------------------------------------------------------------ FFT
// Twiddles exp(-2 pi i k / n), k < n, for n = 2^l (l <= 10): one table per
// device and length, made on first use (guarded: contexts may run in threads).
constexpr int TW_MAXDEV = 64;
static double2* g_tw[TW_MAXDEV][11] = {};
static float2* g_tw32[TW_MAXDEV][11] = {};
static std::mutex g_tw_mu;

static sie_status twiddles_dev(int logn, int dev, double2** out, float2** out32)
{
    std::lock_guard<std::mutex> lk(g_tw_mu);
    if (!g_tw[dev][logn]) {
        int n = 1 << logn;
        std::vector<double2> h(std::max(n, 1));
        for (int k = 0; k < n; k++) {
            long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)n;
            h[k] = make_double2((double)cosl(a), (double)sinl(a));
        }
        double2* d = nullptr;
        SIE_CUDA_TRY(cudaMalloc((void**)&d, sizeof(double2) * h.size()));
        SIE_CUDA_TRY(cudaMemcpy(d, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice));
        std::vector<float2> hf(h.size());
        for (size_t k = 0; k < h.size(); k++) hf[k] = make_float2((float)h[k].x, (float)h[k].y);
        float2* f = nullptr;
        SIE_CUDA_TRY(cudaMalloc((void**)&f, sizeof(float2) * hf.size()));
        SIE_CUDA_TRY(cudaMemcpy(f, hf.data(), sizeof(float2) * hf.size(), cudaMemcpyHostToDevice));
        g_tw[dev][logn] = d;
        g_tw32[dev][logn] = f;
    }
    if (out) *out = g_tw[dev][logn];
    if (out32) *out32 = g_tw32[dev][logn];
    return SIE_OK;
}

static sie_status twiddles(int logn, cudaStream_t, double2** out)
{
    int dev = 0;
    SIE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= TW_MAXDEV) {
        set_error("twiddles: device ordinal out of range");
        return SIE_ERR_ARG;
    }
    return twiddles_dev(logn, dev, out, nullptr);
}

static sie_status twiddles(int logn, cudaStream_t, float2** out)
{
    int dev = 0;
    SIE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= TW_MAXDEV) {
        set_error("twiddles: device ordinal out of range");
        return SIE_ERR_ARG;
    }
    return twiddles_dev(logn, dev, nullptr, out);
}

struct PassGeom {
    int n_in, n_out;       // elements read / written per pencil (zero padding / truncation)
    int64_t npencil;       // pencils
    int L;                 // pencil p -> lo = p % L, hi = p / L
    int64_t slo_in, shi_in, st_in;
    int64_t slo_out, shi_out, st_out;
    int contig;            // 1: elements of a pencil are contiguous (x pass)
    int64_t bs_in = 0, bs_out = 0;  // offsets between the grids of a batch (blockIdx.y)
};

// One CTA transforms PB pencils of length n = 2^LOGN held in shared memory.
// Load at bit-reversed positions, log2(n) radix-2 DIT stages (the first two
// fused into one radix-4 pass without multiplications), store.
template <class C>
__device__ __forceinline__ C cmake(double a, double b);
template <>
__device__ __forceinline__ double2 cmake<double2>(double a, double b) { return make_double2(a, b); }
template <>
__device__ __forceinline__ float2 cmake<float2>(double a, double b) { return make_float2((float)a, (float)b); }

// C = double2 (FP64 path) or float2 (complex64 grid path)
template <int LOGN, int PB, class C>
__global__ void __launch_bounds__(256) k_fft_pass(const C* in, C* out,  // may alias (in place)
                                                  const C* __restrict__ tw, int inv, PassGeom G)
{
    constexpr int n = 1 << LOGN;
    constexpr int pitch = n + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int64_t p0 = (int64_t)blockIdx.x * PB;
    // load (zero padded)
    for (int idx = threadIdx.x; idx < PB * n; idx += blockDim.x) {
        int pl, j;
        if (G.contig) {
            pl = idx / n;
            j = idx % n;
        } else {
            pl = idx % PB;
            j = idx / PB;
        }
        int64_t p = p0 + pl;
        C v = cmake<C>(0.0, 0.0);
        if (p < G.npencil && j < G.n_in) {
            int64_t b = (p % G.L) * G.slo_in + (p / G.L) * G.shi_in + blockIdx.y * G.bs_in;
            v = in[b + (int64_t)j * G.st_in];
        }
        sm[pl * pitch + (__brev(j) >> (32 - LOGN))] = v;
    }
    __syncthreads();
    // stages 1 and 2 have trivial twiddles (1 and -+j): adds and swaps only
    for (int q = threadIdx.x; q < PB * (n / 4); q += blockDim.x) {
        int pl = q / (n / 4), base = 4 * (q % (n / 4));
        C* p = sm + pl * pitch + base;
        C x0 = p[0], x1 = p[1], x2 = p[2], x3 = p[3];
        C a0, a1, b0, b1;
        a0.x = x0.x + x1.x;
        a0.y = x0.y + x1.y;
        a1.x = x0.x - x1.x;
        a1.y = x0.y - x1.y;
        b0.x = x2.x + x3.x;
        b0.y = x2.y + x3.y;
        b1.x = x2.x - x3.x;
        b1.y = x2.y - x3.y;
        // stage 2: w = 1 for (a0, b0); w = -j (forward) or +j (inverse) for (a1, b1)
        C t;
        if (inv) {
            t.x = -b1.y;
            t.y = b1.x;
        } else {
            t.x = b1.y;
            t.y = -b1.x;
        }
        C y0, y1, y2, y3;
        y0.x = a0.x + b0.x;
        y0.y = a0.y + b0.y;
        y2.x = a0.x - b0.x;
        y2.y = a0.y - b0.y;
        y1.x = a1.x + t.x;
        y1.y = a1.y + t.y;
        y3.x = a1.x - t.x;
        y3.y = a1.y - t.y;
        p[0] = y0;
        p[1] = y1;
        p[2] = y2;
        p[3] = y3;
    }
    __syncthreads();
#pragma unroll 1
    for (int s = 3; s <= LOGN; s++) {
        const int half = 1 << (s - 1);
        for (int bfly = threadIdx.x; bfly < PB * (n / 2); bfly += blockDim.x) {
            int pl = bfly / (n / 2), bb = bfly % (n / 2);
            int grp = bb >> (s - 1), pos = bb & (half - 1);
            int i0 = grp * 2 * half + pos, i1 = i0 + half;
            C w = tw[pos << (LOGN - s)];
            if (inv) w.y = -w.y;
            C u = sm[pl * pitch + i0], v = sm[pl * pitch + i1];
            C vw;
            vw.x = v.x * w.x - v.y * w.y;
            vw.y = v.x * w.y + v.y * w.x;
            C a0, a1;
            a0.x = u.x + vw.x;
            a0.y = u.y + vw.y;
            a1.x = u.x - vw.x;
            a1.y = u.y - vw.y;
            sm[pl * pitch + i0] = a0;
            sm[pl * pitch + i1] = a1;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < PB * n; idx += blockDim.x) {
        int pl, j;
        if (G.contig) {
            pl = idx / n;
            j = idx % n;
        } else {
            pl = idx % PB;
            j = idx / PB;
        }
        int64_t p = p0 + pl;
        if (p < G.npencil && j < G.n_out) {
            int64_t b = (p % G.L) * G.slo_out + (p / G.L) * G.shi_out + blockIdx.y * G.bs_out;
            out[b + (int64_t)j * G.st_out] = sm[pl * pitch + j];
        }
    }
}


// ------------------------------------------------------------------ Stockham FFT (register radix-8)
// Self-sorting Stockham formulation (Govindaraju et al., SC'08): pass p with
// current span Ns and radix R: thread j loads a[r] = x[j + r n/R], multiplies
// by exp(-+2 pi i (j mod Ns) r / (Ns R)), does an R-point DFT in registers and
// stores y[(j / Ns) Ns R + (j mod Ns) + r Ns].  n/8 threads per pencil; the
// first pass reads the (zero padded) pencil straight from global memory, the
// last writes the (truncated) output straight to global memory, the passes in
// between exchange through shared memory.
template <class C, int INV>
__device__ __forceinline__ void cmulw(C& a, C w)
{
    C t;
    if (INV) w.y = -w.y;
    t.x = a.x * w.x - a.y * w.y;
    t.y = a.x * w.y + a.y * w.x;
    a = t;
}

template <class C, int INV>
__device__ __forceinline__ void bfly2(C& a, C& b)
{
    C t = a;
    a.x = t.x + b.x;
    a.y = t.y + b.y;
    b.x = t.x - b.x;
    b.y = t.y - b.y;
}

// multiply by -j (forward) or +j (inverse)
template <class C, int INV>
__device__ __forceinline__ C mulmj(C a)
{
    C t;
    if (INV) {
        t.x = -a.y;
        t.y = a.x;
    } else {
        t.x = a.y;
        t.y = -a.x;
    }
    return t;
}

template <class C, int INV>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3)
{
    // X0 = (a0+a2)+(a1+a3), X2 = (a0+a2)-(a1+a3), X1 = (a0-a2) -+j (a1-a3), X3 = (a0-a2) +-j (a1-a3)
    bfly2<C, INV>(a0, a2);
    bfly2<C, INV>(a1, a3);
    a3 = mulmj<C, INV>(a3);
    bfly2<C, INV>(a0, a1);
    bfly2<C, INV>(a2, a3);
    // now a0 = X0, a1 = X2, a2 = X1, a3 = X3 -> reorder
    C t = a1;
    a1 = a2;
    a2 = t;
}

template <class C, int INV>
__device__ __forceinline__ void dft8(C* a)
{
    // even/odd split: E = DFT4(a0,a2,a4,a6), O = DFT4(a1,a3,a5,a7)
    dft4<C, INV>(a[0], a[2], a[4], a[6]);
    dft4<C, INV>(a[1], a[3], a[5], a[7]);
    const double r = 0.70710678118654752440;
    // O[k] *= W8^k : W8 = (1 -+ j)/sqrt2, W8^2 = -+j, W8^3 = (-1 -+ j)/sqrt2
    C o1 = a[3], o2 = a[5], o3 = a[7];
    C t;
    if (!INV) {
        t.x = (o1.x + o1.y) * r;
        t.y = (o1.y - o1.x) * r;
    } else {
        t.x = (o1.x - o1.y) * r;
        t.y = (o1.y + o1.x) * r;
    }
    o1 = t;
    o2 = mulmj<C, INV>(o2);
    if (!INV) {
        t.x = (o3.y - o3.x) * r;
        t.y = -(o3.x + o3.y) * r;
    } else {
        t.x = -(o3.x + o3.y) * r;
        t.y = (o3.x - o3.y) * r;
    }
    o3 = t;
    // E[k] in a[0], a[2], a[4], a[6]; O[k] (twiddled) in a[1], o1, o2, o3
    C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], q0 = a[1];
    a[0].x = e0.x + q0.x; a[0].y = e0.y + q0.y;
    a[4].x = e0.x - q0.x; a[4].y = e0.y - q0.y;
    a[1].x = e1.x + o1.x; a[1].y = e1.y + o1.y;
    a[5].x = e1.x - o1.x; a[5].y = e1.y - o1.y;
    a[2].x = e2.x + o2.x; a[2].y = e2.y + o2.y;
    a[6].x = e2.x - o2.x; a[6].y = e2.y - o2.y;
    a[3].x = e3.x + o3.x; a[3].y = e3.y + o3.y;
    a[7].x = e3.x - o3.x; a[7].y = e3.y - o3.y;
}

template <class C, int INV, int R>
__device__ __forceinline__ void dftR(C* a)
{
    if constexpr (R == 8)
        dft8<C, INV>(a);
    else if constexpr (R == 4)
        dft4<C, INV>(a[0], a[1], a[2], a[3]);
    else
        bfly2<C, INV>(a[0], a[1]);
}

// one Stockham pass of radix R over the pencil held by (tp = thread in pencil);
// SRC / DST: 0 = global, 1 = shared memory
template <int LOGN, int R, int SRC, int DST, class C, int INV>
__device__ __forceinline__ void stockham_pass(int Ns, int tp, const C* gin, int64_t gbase_in, int64_t gst_in,
                                              int n_in, C* gout, int64_t gbase_out, int64_t gst_out, int n_out,
                                              bool valid, const C* sin, C* sout, const C* __restrict__ tw)
{
    constexpr int n = 1 << LOGN;
    constexpr int TPP = n / 8;  // threads per pencil
    constexpr int NB = n / R;   // butterflies per pencil
    constexpr int LR = R == 8 ? 3 : (R == 4 ? 2 : 1);
    const int lns = __ffs(Ns) - 1;  // log2(Ns)
    for (int jj = tp; jj < NB; jj += TPP) {
        C a[R];
        for (int r = 0; r < R; r++) {
            int idx = jj + r * NB;
            if (SRC == 0) {
                C v;
                v.x = 0;
                v.y = 0;
                if (valid && idx < n_in) v = gin[gbase_in + (int64_t)idx * gst_in];
                a[r] = v;
            } else {
                a[r] = sin[idx];
            }
        }
        // Ns and R are powers of two: masks and shifts instead of divisions
        const int k = jj & (Ns - 1);
        if (Ns > 1)
            for (int r = 1; r < R; r++) cmulw<C, INV>(a[r], tw[(k * r) << (LOGN - lns - LR)]);
        dftR<C, INV, R>(a);
        const int o = ((jj >> lns) << (lns + LR)) + k;
        for (int r = 0; r < R; r++) {
            int idx = o + r * Ns;
            if (DST == 0) {
                if (valid && idx < n_out) gout[gbase_out + (int64_t)idx * gst_out] = a[r];
            } else {
                sout[idx] = a[r];
            }
        }
    }
}

template <int LOGN, int PB, class C, int INV>
__global__ void __launch_bounds__(PB*(1 << LOGN) / 8) k_fft_stockham(const C* in, C* out, const C* __restrict__ tw,
                                                                     PassGeom G)
{
    constexpr int n = 1 << LOGN;
    constexpr int TPP = n / 8;
    constexpr int pitch = n + 1;
    extern __shared__ __align__(16) unsigned char smraw2[];
    C* sm0 = reinterpret_cast<C*>(smraw2);
    C* sm1 = sm0 + PB * pitch;
    // pencil-fastest thread order on strided passes keeps rows coalesced
    int pl, tp;
    if (G.contig) {
        pl = threadIdx.x / TPP;
        tp = threadIdx.x % TPP;
    } else {
        pl = threadIdx.x % PB;
        tp = threadIdx.x / PB;
    }
    int64_t p = (int64_t)blockIdx.x * PB + pl;
    bool valid = p < G.npencil;
    int64_t bin = valid ? (p % G.L) * G.slo_in + (p / G.L) * G.shi_in + blockIdx.y * G.bs_in : 0;
    int64_t bout = valid ? (p % G.L) * G.slo_out + (p / G.L) * G.shi_out + blockIdx.y * G.bs_out : 0;
    C* s0 = sm0 + pl * pitch;
    C* s1 = sm1 + pl * pitch;
    // radix plan: 8^a x (1, 2 or 4)
    constexpr int NP8 = LOGN / 3, REM = LOGN % 3;
    constexpr int NPASS = NP8 + (REM ? 1 : 0);
    int Ns = 1;
    // pass 0 (global -> smem or global)
    if constexpr (NPASS == 1) {
        stockham_pass<LOGN, 8, 0, 0, C, INV>(Ns, tp, in, bin, G.st_in, G.n_in, out, bout, G.st_out, G.n_out, valid,
                                             nullptr, nullptr, tw);
        return;
    } else {
        stockham_pass<LOGN, 8, 0, 1, C, INV>(Ns, tp, in, bin, G.st_in, G.n_in, nullptr, 0, 0, 0, valid, nullptr, s0,
                                             tw);
    }
    Ns *= 8;
    __syncthreads();
    C* cur = s0;
    C* nxt = s1;
    for (int ps = 1; ps < NP8; ps++) {
        bool last = (ps == NPASS - 1);
        if (last) {
            stockham_pass<LOGN, 8, 1, 0, C, INV>(Ns, tp, nullptr, 0, 0, 0, out, bout, G.st_out, G.n_out, valid, cur,
                                                 nullptr, tw);
            return;
        }
        stockham_pass<LOGN, 8, 1, 1, C, INV>(Ns, tp, nullptr, 0, 0, 0, nullptr, 0, 0, 0, valid, cur, nxt, tw);
        Ns *= 8;
        __syncthreads();
        C* t = cur;
        cur = nxt;
        nxt = t;
    }
    if constexpr (REM == 1)
        stockham_pass<LOGN, 2, 1, 0, C, INV>(Ns, tp, nullptr, 0, 0, 0, out, bout, G.st_out, G.n_out, valid, cur,
                                             nullptr, tw);
    else if constexpr (REM == 2)
        stockham_pass<LOGN, 4, 1, 0, C, INV>(Ns, tp, nullptr, 0, 0, 0, out, bout, G.st_out, G.n_out, valid, cur,
                                             nullptr, tw);
}

template <int LOGN, int PB, class C>
static sie_status launch_pass_pb(cudaStream_t st, const C* in, C* out, int inv, const PassGeom& G, const C* tw,
                                 int nbatch)
{
    constexpr int n = 1 << LOGN;
    size_t smem = sizeof(C) * PB * (n + 1);
    // once per instantiation (thread-safe static initialisation)
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_fft_pass<LOGN, PB, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    SIE_CUDA_TRY(attr);
    unsigned blocks = (unsigned)((G.npencil + PB - 1) / PB);
    k_fft_pass<LOGN, PB, C><<<dim3(blocks, nbatch), 256, smem, st>>>(in, out, tw, inv, G);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// Pencils per CTA: as many as keep at least ~4 CTAs per SM in flight (more
// pencils per CTA give longer coalesced rows on the strided passes, fewer
// leave SMs idle on the small passes); SIE_FFT_PB overrides for tuning.
static int pick_pb(int n, int64_t npencil)
{
    static int forced = -1;
    if (forced < 0) {
        const char* e = getenv("SIE_FFT_PB");
        forced = e ? atoi(e) : 0;
    }
    if (forced == 4 || forced == 8 || forced == 16) return (n >= 512 && forced == 16) ? 8 : forced;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (!sms) sms = 152;
    }
    for (int pb : {16, 8, 4}) {
        if (n >= 512 && pb == 16) continue;
        if (npencil / pb >= 4LL * sms) return pb;
    }
    return 4;
}

template <int LOGN, int PB, class C>
static sie_status launch_stockham(cudaStream_t st, const C* in, C* out, int inv, const PassGeom& G, const C* tw,
                                  int nbatch)
{
    constexpr int n = 1 << LOGN;
    size_t smem = sizeof(C) * 2 * PB * (n + 1);
    // once per instantiation (thread-safe static initialisation)
    static const cudaError_t attr = [smem] {
        cudaError_t e = cudaFuncSetAttribute(k_fft_stockham<LOGN, PB, C, 0>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_fft_stockham<LOGN, PB, C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    }();
    SIE_CUDA_TRY(attr);
    unsigned blocks = (unsigned)((G.npencil + PB - 1) / PB);
    constexpr int threads = PB * n / 8;
    if (inv)
        k_fft_stockham<LOGN, PB, C, 1><<<dim3(blocks, nbatch), threads, smem, st>>>(in, out, tw, G);
    else
        k_fft_stockham<LOGN, PB, C, 0><<<dim3(blocks, nbatch), threads, smem, st>>>(in, out, tw, G);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// ------------------------------------------------------------------ fused z stage of the system product
// Forward z-transforms of the seven source grids, the spectral products of
// Eq. (sys) (sys_specmul) and the inverse z-transforms of the four result
// grids, PB (x, y) columns per CTA: the full-length z spectra of a column
// stay in shared memory, so the 7 + 4 grids of n^3 are neither written out by
// the forward z pass nor read back by the spectral multiply and the inverse z
// pass.  Reads z < nz_phys of the seven grids, writes z < nz_phys of grids
// 0..3 (the inverse y pass reads nothing else).  Thread layout: grid g (7),
// then pencil-fastest within the grid (coalesced rows along x).  Shared
// memory: two pitch-(n + 1) arrays per (grid, pencil), the spectrum A and one
// Stockham ping-pong buffer T; the passes alternate so that the forward chain
// ends in A and the inverse chain starts from it.
template <int LOGN, int PB, class C, class R>
__global__ void __launch_bounds__(7 * PB * (1 << LOGN) / 8)
    k_fft_z_sys(C* __restrict__ buf, const C* __restrict__ spec, const C* __restrict__ tw, int nz_phys,
                int64_t ncol, int64_t plane, int64_t bnn, R k0)
{
    constexpr int n = 1 << LOGN;
    constexpr int TPP = n / 8;
    constexpr int pitch = n + 1;
    constexpr int NP8 = LOGN / 3, REM = LOGN % 3;
    constexpr int NPASS = NP8 + (REM ? 1 : 0);
    extern __shared__ __align__(16) unsigned char smz[];
    C* sm = reinterpret_cast<C*>(smz);
    const int gi = threadIdx.x / (PB * TPP);
    const int rr = threadIdx.x % (PB * TPP);
    const int pl = rr % PB, tp = rr / PB;
    const int64_t col = (int64_t)blockIdx.x * PB + pl;
    const bool valid = col < ncol;
    C* A = sm + (int64_t)(gi * PB + pl) * 2 * pitch;
    C* T = A + pitch;
    // pass ps writes A when (NPASS - 1 - ps) is even, so the last lands in A
    auto dst_of = [&](int ps) { return ((NPASS - 1 - ps) & 1) ? T : A; };
    // kernel spectra of this thread's spectral-product points
    constexpr int NT = 7 * PB * TPP;
    constexpr int NPT = (PB * n + NT - 1) / NT;
    C sp[NPT][4];
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        const int idx = threadIdx.x + k * NT;
        const int p2 = idx % PB, kz = idx / PB;
        const int64_t c2 = (int64_t)blockIdx.x * PB + p2;
        if (idx < PB * n && c2 < ncol) {
            const int64_t i = (int64_t)kz * plane + c2;
#pragma unroll
            for (int q = 0; q < 4; q++) sp[k][q] = spec[q * bnn + i];
        }
    }
    // ---- forward: global (z < nz_phys, zero padded) -> ... -> A
    int Ns = 1;
    const int64_t gbase = gi * bnn + (valid ? col : 0);
    stockham_pass<LOGN, 8, 0, 1, C, 0>(Ns, tp, buf, gbase, plane, nz_phys, nullptr, 0, 0, 0, valid, nullptr,
                                       dst_of(0), tw);
    Ns *= 8;
    __syncthreads();
    for (int ps = 1; ps < NP8; ps++) {
        stockham_pass<LOGN, 8, 1, 1, C, 0>(Ns, tp, nullptr, 0, 0, 0, nullptr, 0, 0, 0, valid, dst_of(ps - 1),
                                           dst_of(ps), tw);
        Ns *= 8;
        __syncthreads();
    }
    if constexpr (REM == 1)
        stockham_pass<LOGN, 2, 1, 1, C, 0>(Ns, tp, nullptr, 0, 0, 0, nullptr, 0, 0, 0, valid, T, A, tw);
    else if constexpr (REM == 2)
        stockham_pass<LOGN, 4, 1, 1, C, 0>(Ns, tp, nullptr, 0, 0, 0, nullptr, 0, 0, 0, valid, T, A, tw);
    if constexpr (REM != 0) __syncthreads();
    // ---- spectral products, in place into A of grids 0..3 (kernel spectra
    // loaded before the forward passes, so their latency overlaps them)
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        const int idx = threadIdx.x + k * NT;
        if (idx >= PB * n) break;
        const int p2 = idx % PB, kz = idx / PB;
        const int64_t c2 = (int64_t)blockIdx.x * PB + p2;
        if (c2 >= ncol) continue;
        C in[7], out[4];
#pragma unroll
        for (int g = 0; g < 7; g++) in[g] = sm[(int64_t)(g * PB + p2) * 2 * pitch + kz];
        sys_specmul(sp[k][0], sp[k][1], sp[k][2], sp[k][3], k0, in, out);
#pragma unroll
        for (int g = 0; g < 4; g++) sm[(int64_t)(g * PB + p2) * 2 * pitch + kz] = out[g];
    }
    __syncthreads();
    // ---- inverse of grids 0..3: A -> T -> A ... -> global (z < nz_phys)
    const bool act = gi < 4;
    Ns = 1;
    C* cur = A;
    C* nxt = T;
    if constexpr (NPASS == 1) {
        if (act)
            stockham_pass<LOGN, 8, 1, 0, C, 1>(Ns, tp, nullptr, 0, 0, 0, buf, gbase, plane, nz_phys, valid, A,
                                               nullptr, tw);
        return;
    } else {
        if (act)
            stockham_pass<LOGN, 8, 1, 1, C, 1>(Ns, tp, nullptr, 0, 0, 0, nullptr, 0, 0, 0, valid, cur, nxt, tw);
    }
    Ns *= 8;
    __syncthreads();
    {
        C* t = cur;
        cur = nxt;
        nxt = t;
    }
    for (int ps = 1; ps < NP8; ps++) {
        if (ps == NPASS - 1) {
            if (act)
                stockham_pass<LOGN, 8, 1, 0, C, 1>(Ns, tp, nullptr, 0, 0, 0, buf, gbase, plane, nz_phys, valid, cur,
                                                   nullptr, tw);
            return;
        }
        if (act)
            stockham_pass<LOGN, 8, 1, 1, C, 1>(Ns, tp, nullptr, 0, 0, 0, nullptr, 0, 0, 0, valid, cur, nxt, tw);
        Ns *= 8;
        __syncthreads();
        C* t = cur;
        cur = nxt;
        nxt = t;
    }
    if constexpr (REM == 1) {
        if (act)
            stockham_pass<LOGN, 2, 1, 0, C, 1>(Ns, tp, nullptr, 0, 0, 0, buf, gbase, plane, nz_phys, valid, cur,
                                               nullptr, tw);
    } else if constexpr (REM == 2) {
        if (act)
            stockham_pass<LOGN, 4, 1, 0, C, 1>(Ns, tp, nullptr, 0, 0, 0, buf, gbase, plane, nz_phys, valid, cur,
                                               nullptr, tw);
    }
}

template <int LOGN, int PB, class C, class R>
static sie_status launch_z_sys_pb(cudaStream_t st, C* buf, const C* spec, const C* tw, int nz_phys, int64_t ncol,
                                  int64_t plane, int64_t bnn, R k0)
{
    constexpr int n = 1 << LOGN;
    const size_t smem = sizeof(C) * 7 * PB * 2 * (n + 1);
    static const cudaError_t attr = cudaFuncSetAttribute(k_fft_z_sys<LOGN, PB, C, R>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    SIE_CUDA_TRY(attr);
    const unsigned blocks = (unsigned)((ncol + PB - 1) / PB);
    k_fft_z_sys<LOGN, PB, C, R><<<blocks, 7 * PB * n / 8, smem, st>>>(buf, spec, tw, nz_phys, ncol, plane, bnn, k0);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// columns per CTA of k_fft_z_sys: 4 (complex64) or 2 (complex128) by default,
// 57.8 KB of shared memory at n = 128; SIE_ZSYS_PB = 2, 4 or 8 overrides
// (complex64; complex128 takes half of it, at least 1), for tuning
static int zsys_pb(bool c64)
{
    static int forced = -1;
    if (forced < 0) {
        const char* e = getenv("SIE_ZSYS_PB");
        forced = e ? atoi(e) : 0;
    }
    int pb = (forced == 2 || forced == 4 || forced == 8) ? forced : 4;
    return c64 ? pb : std::max(1, pb / 2);
}

template <int LOGN, class C, class R>
static sie_status launch_z_sys(cudaStream_t st, C* buf, const C* spec, int nz_phys, int64_t ncol, int64_t plane,
                               int64_t bnn, R k0)
{
    C* tw = nullptr;
    SIE_TRY(twiddles(LOGN, st, &tw));
    const int pb = zsys_pb(sizeof(C) == 8);
    if constexpr (sizeof(C) == 8) {
        if (pb == 2) return launch_z_sys_pb<LOGN, 2, C, R>(st, buf, spec, tw, nz_phys, ncol, plane, bnn, k0);
        if (pb == 8 && LOGN <= 7) return launch_z_sys_pb<LOGN, 8, C, R>(st, buf, spec, tw, nz_phys, ncol, plane, bnn, k0);
        return launch_z_sys_pb<LOGN, 4, C, R>(st, buf, spec, tw, nz_phys, ncol, plane, bnn, k0);
    } else {
        if (pb == 1) return launch_z_sys_pb<LOGN, 1, C, R>(st, buf, spec, tw, nz_phys, ncol, plane, bnn, k0);
        if (pb == 4 && LOGN <= 7) return launch_z_sys_pb<LOGN, 4, C, R>(st, buf, spec, tw, nz_phys, ncol, plane, bnn, k0);
        return launch_z_sys_pb<LOGN, 2, C, R>(st, buf, spec, tw, nz_phys, ncol, plane, bnn, k0);
    }
}

static int fft_kernel_choice()
{
    static int k = -1;
    if (k < 0) {
        const char* e = getenv("SIE_FFT_KERNEL");
        k = (e && e[0] == 'r') ? 1 : 0;  // 0: Stockham radix-8 (default), 1: shared-memory radix-2
    }
    return k;
}

template <int LOGN, class C>
static sie_status launch_pass_n(cudaStream_t st, const C* in, C* out, int inv, const PassGeom& G, int nbatch)
{
    C* tw = nullptr;
    SIE_TRY(twiddles(LOGN, st, &tw));
    if (fft_kernel_choice() == 0) {
        // 256 threads per CTA (n/8 per pencil); halve the pencils per CTA when
        // that leaves fewer than ~4 CTAs per SM
        constexpr int PB = 2048 >> LOGN;
        constexpr int PBh = PB >= 2 ? PB / 2 : 1;
        int pb = pick_pb(1 << LOGN, G.npencil * nbatch);
        if (pb >= 16 || G.npencil * nbatch / PB >= 4LL * 152)
            return launch_stockham<LOGN, PB, C>(st, in, out, inv, G, tw, nbatch);
        return launch_stockham<LOGN, PBh, C>(st, in, out, inv, G, tw, nbatch);
    }
    switch (pick_pb(1 << LOGN, G.npencil * nbatch)) {
        case 16:
            if constexpr (LOGN < 9) return launch_pass_pb<LOGN, 16, C>(st, in, out, inv, G, tw, nbatch);
            [[fallthrough]];
        case 8: return launch_pass_pb<LOGN, 8, C>(st, in, out, inv, G, tw, nbatch);
        default: return launch_pass_pb<LOGN, 4, C>(st, in, out, inv, G, tw, nbatch);
    }
}

template <class C>
static sie_status launch_pass(cudaStream_t st, int n, const C* in, C* out, int inv, const PassGeom& G, int nb = 1)
{
    switch (n) {
        case 16: return launch_pass_n<4>(st, in, out, inv, G, nb);
        case 32: return launch_pass_n<5>(st, in, out, inv, G, nb);
        case 64: return launch_pass_n<6>(st, in, out, inv, G, nb);
        case 128: return launch_pass_n<7>(st, in, out, inv, G, nb);
        case 256: return launch_pass_n<8>(st, in, out, inv, G, nb);
        case 512: return launch_pass_n<9>(st, in, out, inv, G, nb);
        case 1024: return launch_pass_n<10>(st, in, out, inv, G, nb);
    }
    set_error("unsupported FFT length");
    return SIE_ERR_UNSUPPORTED;
}

// dir = -1: forward transform of the compact N grid `src` (or, prune = 0, of the
// full n grid already in buf) into the full spectrum in buf.
// dir = +1: inverse of the spectrum in buf; prune = 1 writes only the physical
// N box into the compact array `src` (used as output), prune = 0 keeps n^3 in buf.
// nbatch grids at once: grid k at buf + k n^3 and (compact) src + k N^3
template <class C>
static sie_status fft3d_t(cudaStream_t st, C* buf, const C* src, const GridDesc& g, int dir, int prune, sie_ctx* pc,
                          int nbatch)
{
    const int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int64_t Nx = prune ? g.N[0] : nx, Ny = prune ? g.N[1] : ny, Nz = prune ? g.N[2] : nz;
    const int64_t pyz = nx * ny;  // padded plane
    const int64_t bnn = nx * ny * nz, bNg = (int64_t)g.N[0] * g.N[1] * g.N[2];
    if (dir < 0) {
        // x pass: pencils (y < Ny, z < Nz)
        PassGeom X{(int)Nx, (int)nx, Ny * Nz, (int)Ny, prune ? Nx : nx, prune ? Nx * Ny : pyz, 1, nx, pyz, 1, 1,
                   prune ? bNg : bnn, bnn};
        {
            Stage s_(pc, "fft_fwd_x");
            SIE_TRY(launch_pass(st, (int)nx, prune ? src : buf, buf, 0, X, nbatch));
        }
        // y pass: pencils (x < nx, z < Nz)
        PassGeom Y{(int)Ny, (int)ny, nx * Nz, (int)nx, 1, pyz, nx, 1, pyz, nx, 0, bnn, bnn};
        {
            Stage s_(pc, "fft_fwd_y");
            SIE_TRY(launch_pass(st, (int)ny, buf, buf, 0, Y, nbatch));
        }
        // z pass: pencils (x < nx, y < ny)
        PassGeom Z{(int)Nz, (int)nz, nx * ny, (int)nx, 1, nx, pyz, 1, nx, pyz, 0, bnn, bnn};
        {
            Stage s_(pc, "fft_fwd_z");
            SIE_TRY(launch_pass(st, (int)nz, buf, buf, 0, Z, nbatch));
        }
    } else {
        PassGeom Z{(int)nz, (int)Nz, nx * ny, (int)nx, 1, nx, pyz, 1, nx, pyz, 0, bnn, bnn};
        {
            Stage s_(pc, "fft_inv_z");
            SIE_TRY(launch_pass(st, (int)nz, buf, buf, 1, Z, nbatch));
        }
        PassGeom Y{(int)ny, (int)Ny, nx * Nz, (int)nx, 1, pyz, nx, 1, pyz, nx, 0, bnn, bnn};
        {
            Stage s_(pc, "fft_inv_y");
            SIE_TRY(launch_pass(st, (int)ny, buf, buf, 1, Y, nbatch));
        }
        C* dst = prune ? const_cast<C*>(src) : buf;
        PassGeom X{(int)nx, (int)Nx, Ny * Nz, (int)Ny, nx, pyz, 1, prune ? Nx : nx, prune ? Nx * Ny : pyz, 1, 1,
                   bnn, prune ? bNg : bnn};
        {
            Stage s_(pc, "fft_inv_x");
            SIE_TRY(launch_pass(st, (int)nx, buf, dst, 1, X, nbatch));
        }
    }
    return SIE_OK;
}

sie_status fft3d(cudaStream_t st, double2* buf, const double2* src, const GridDesc& g, int dir, int prune, sie_ctx* pc,
                 int nbatch)
{
    return fft3d_t(st, buf, src, g, dir, prune, pc, nbatch);
}

sie_status fft3d(cudaStream_t st, float2* buf, const float2* src, const GridDesc& g, int dir, int prune, sie_ctx* pc,
                 int nbatch)
{
    return fft3d_t(st, buf, src, g, dir, prune, pc, nbatch);
}

// Grid part of the system product (Eq. sys) with the fused z stage: forward x
// and y passes of the seven compact source grids in src (into buf), the fused
// forward-z / spectral-product / inverse-z kernel, then the inverse y and x
// passes of the four result grids back into the compact src.  Same arithmetic
// as fft3d(-1) + k_specmul_sys + fft3d(+1), in another order of memory passes.
template <class C, class R>
static sie_status fft_sys_t(cudaStream_t st, C* buf, C* src, const GridDesc& g, const C* spec, R k0, sie_ctx* pc)
{
    const int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int64_t Nx = g.N[0], Ny = g.N[1], Nz = g.N[2];
    const int64_t pyz = nx * ny, bnn = nx * ny * nz, bNg = Nx * Ny * Nz;
    PassGeom X{(int)Nx, (int)nx, Ny * Nz, (int)Ny, Nx, Nx * Ny, 1, nx, pyz, 1, 1, bNg, bnn};
    {
        Stage s_(pc, "fft_fwd_x");
        SIE_TRY(launch_pass(st, (int)nx, src, buf, 0, X, 7));
    }
    PassGeom Y{(int)Ny, (int)ny, nx * Nz, (int)nx, 1, pyz, nx, 1, pyz, nx, 0, bnn, bnn};
    {
        Stage s_(pc, "fft_fwd_y");
        SIE_TRY(launch_pass(st, (int)ny, buf, buf, 0, Y, 7));
    }
    {
        Stage s_(pc, "fft_z_specmul");
        sie_status s;
        switch (nz) {
            case 16: s = launch_z_sys<4>(st, buf, spec, (int)Nz, pyz, pyz, bnn, k0); break;
            case 32: s = launch_z_sys<5>(st, buf, spec, (int)Nz, pyz, pyz, bnn, k0); break;
            case 64: s = launch_z_sys<6>(st, buf, spec, (int)Nz, pyz, pyz, bnn, k0); break;
            case 128: s = launch_z_sys<7>(st, buf, spec, (int)Nz, pyz, pyz, bnn, k0); break;
            case 256: s = launch_z_sys<8>(st, buf, spec, (int)Nz, pyz, pyz, bnn, k0); break;
            default:
                set_error("fused z stage: unsupported FFT length");
                return SIE_ERR_UNSUPPORTED;
        }
        SIE_TRY(s);
    }
    PassGeom Yi{(int)ny, (int)Ny, nx * Nz, (int)nx, 1, pyz, nx, 1, pyz, nx, 0, bnn, bnn};
    {
        Stage s_(pc, "fft_inv_y");
        SIE_TRY(launch_pass(st, (int)ny, buf, buf, 1, Yi, 4));
    }
    PassGeom Xi{(int)nx, (int)Nx, Ny * Nz, (int)Ny, nx, pyz, 1, Nx, Nx * Ny, 1, 1, bnn, bNg};
    {
        Stage s_(pc, "fft_inv_x");
        SIE_TRY(launch_pass(st, (int)nx, buf, src, 1, Xi, 4));
    }
    return SIE_OK;
}

bool fft_sys_supported(const GridDesc& g) { return g.n[2] >= 16 && g.n[2] <= 256; }

sie_status fft_sys(cudaStream_t st, double2* buf, double2* src, const GridDesc& g, const double2* spec, double k0,
                   sie_ctx* pc)
{
    return fft_sys_t(st, buf, src, g, spec, k0, pc);
}

sie_status fft_sys(cudaStream_t st, float2* buf, float2* src, const GridDesc& g, const float2* spec, float k0,
                   sie_ctx* pc)
{
    return fft_sys_t(st, buf, src, g, spec, k0, pc);
}

// ------------------------------------------------------------------ kernel spectra
// circulant samples of G, dG/dx, dG/dy, dG/dz at lattice lags (c9 reading:
// index i -> lag i if i < N, i - n if i > n - N, else unused); G(0) = 0.
// Scaled by 1/(nx ny nz) so the unnormalised inverse FFT gives the convolution.
__global__ void k_sample(GridDesc g, double kr, double ki, double2* __restrict__ spec, int64_t nn)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nn) return;
    int ix = (int)(idx % g.n[0]), iy = (int)((idx / g.n[0]) % g.n[1]), iz = (int)(idx / ((int64_t)g.n[0] * g.n[1]));
    int ii[3] = {ix, iy, iz};
    double d[3];
    bool ok = true;
    for (int a = 0; a < 3; a++) {
        int lag;
        if (ii[a] < g.N[a])
            lag = ii[a];
        else if (ii[a] > g.n[a] - g.N[a])
            lag = ii[a] - g.n[a];
        else {
            lag = 0;
            ok = false;
        }
        d[a] = g.h * lag;
    }
    double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double2 G = make_double2(0, 0), gx = G, gy = G, gz = G;
    if (ok && R > 0) {
        double sc = 1.0 / ((double)g.n[0] * g.n[1] * g.n[2]);
        double e = exp(ki * R), s, c;
        sincos(-kr * R, &s, &c);
        double er = e * c, ei = e * s;  // exp(-j k R)
        G = make_double2(sc * er / (4 * M_PI * R), sc * ei / (4 * M_PI * R));
        // g = -(1 + j k R) e / (4 pi R^3)
        double ar = 1.0 - ki * R, ai = kr * R;
        double fr = -(ar * er - ai * ei) / (4 * M_PI * R * R * R) * sc;
        double fi = -(ar * ei + ai * er) / (4 * M_PI * R * R * R) * sc;
        gx = make_double2(fr * d[0], fi * d[0]);
        gy = make_double2(fr * d[1], fi * d[1]);
        gz = make_double2(fr * d[2], fi * d[2]);
    }
    spec[idx] = G;
    spec[nn + idx] = gx;
    spec[2 * nn + idx] = gy;
    spec[3 * nn + idx] = gz;
}

__global__ void k_to_c64(const double2* __restrict__ a, float2* __restrict__ b, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

sie_status aim_spectra(sie_op* op, AimOp& a)
{
    cudaStream_t st = op->mesh->ctx->stream;
    const GridDesc& g = a.g;
    int64_t nn = (int64_t)g.n[0] * g.n[1] * g.n[2];
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.spec, sizeof(double2) * 4 * nn, st));
    k_sample<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(g, a.kr, a.ki, a.spec, nn);
    SIE_CUDA_TRY(cudaGetLastError());
    SIE_TRY(fft3d(st, a.spec, (const double2*)nullptr, g, -1, 0, nullptr, 4));
    SIE_CUDA_TRY(cudaMallocAsync((void**)&a.spec32, sizeof(float2) * 4 * nn, st));
    k_to_c64<<<(unsigned)((4 * nn + 255) / 256), 256, 0, st>>>(a.spec, a.spec32, 4 * nn);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// ------------------------------------------------------------------ projection (P, P_phi)
// one thread per (triangle, stencil node): J_t(r) = alpha (r - c_t) + beta,
// alpha = sum_i c_i x_i, beta = sum_i c_i x_i (c_t - p_i), div J_t = 2 alpha.
// mode 0: grids Jx, Jy, Jz, rho; mode 1: Jx, Jy, Jz only.
__global__ void k_project(int nt, int S, int Mord, DevMesh M, const int32_t* __restrict__ base,
                          const double* __restrict__ W, const double2* __restrict__ x, GridDesc g, int ngrid,
                          double2* __restrict__ src, int64_t Ng)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nt * S) return;
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

// ------------------------------------------------------------------ spectral multiply
// mode 0 (L): J_a *= G, rho *= G.  mode 1 (K): J <- Ghat_grad x J.
__global__ void k_specmul(int mode, const double2* __restrict__ spec, double2* __restrict__ buf, int64_t nn)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    auto mul = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
    if (mode == 0) {
        double2 G = spec[i];
        for (int c = 0; c < 4; c++) buf[c * nn + i] = mul(G, buf[c * nn + i]);
    } else {
        double2 gx = spec[nn + i], gy = spec[2 * nn + i], gz = spec[3 * nn + i];
        double2 jx = buf[i], jy = buf[nn + i], jz = buf[2 * nn + i];
        double2 a = mul(gy, jz), b = mul(gz, jy);
        buf[i] = make_double2(a.x - b.x, a.y - b.y);
        a = mul(gz, jx);
        b = mul(gx, jz);
        buf[nn + i] = make_double2(a.x - b.x, a.y - b.y);
        a = mul(gx, jy);
        b = mul(gy, jx);
        buf[2 * nn + i] = make_double2(a.x - b.x, a.y - b.y);
    }
}

// ------------------------------------------------------------------ interpolation (W = P^T)
// one warp per triangle; lanes gather stencil nodes; y[e] += c_{t,i}
// [S1 + (c_t - p_i) . T0 + scal 2 P0]  (scal = -1/k^2 for L, 0 for K)
__global__ void k_interp(int nt, int S, int Mord, DevMesh M, const int32_t* __restrict__ base,
                         const double* __restrict__ W, const double2* __restrict__ out, GridDesc g, int has_phi,
                         double2 scal, int64_t Ng, double2* __restrict__ y)
{
    int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (t >= nt) return;
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
        if (has_phi) {
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
        int i = lane;
        // broadcast from lane 0
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
        if (has_phi) {
            vr += 2.0 * (scal.x * P0r - scal.y * P0i);
            vi += 2.0 * (scal.x * P0i + scal.y * P0r);
        }
        double c = M.coef[3 * t + i];
        double2* d = y + M.tri_edge[3 * t + i];
        atomicAdd(&d->x, c * vr);
        atomicAdd(&d->y, c * vi);
    }
}

// ------------------------------------------------------------------ near CSR product
// y[m] += sum_e val[e] x[col[e]]; one warp per row

sie_status csr_mv(cudaStream_t st, int nrow, int64_t nnz, const int64_t* rp, const int32_t* col,
                  const double2* val, const double2* x, double2* y)
{
    SIE_CUDA_TRY(csr_launch(st, nrow, nnz, rp, col, val, x, make_double2(1.0, 0.0), false, y));
    return SIE_OK;
}

// y += W applied to the inverse-transformed grids (3 vector grids, + scalar grid)
sie_status aim_interp(sie_op* op, const double2* grids, int has_phi, double2 scal, double2* y)
{
    const DevMesh& M = op->mesh->d;
    const GridDesc& g = op->ext.g;
    int S = (g.M + 1) * (g.M + 1) * (g.M + 1);
    int64_t Ng = (int64_t)g.N[0] * g.N[1] * g.N[2];
    k_interp<<<(M.nt + 3) / 4, 128, 0, op->mesh->ctx->stream>>>(M.nt, S, g.M, M, op->base, op->W, grids, g, has_phi,
                                                                scal, Ng, y);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// y = A x for one right-hand side, A = L (which_LK = 0) or K (1) of operator a
sie_status aim_apply(sie_op* op, AimOp& a, int which_LK, const double2* x, double2* y)
{
    sie_ctx* pc = op->mesh->ctx;
    cudaStream_t st = pc->stream;
    const DevMesh& M = op->mesh->d;
    if (a.has_grid) {
        SIE_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double2) * M.ne, st));
        const GridDesc& g = a.g;
        int S = (g.M + 1) * (g.M + 1) * (g.M + 1);
        int64_t Ng = (int64_t)g.N[0] * g.N[1] * g.N[2];
        int64_t nn = (int64_t)g.n[0] * g.n[1] * g.n[2];
        int ngrid = which_LK == 0 ? 4 : 3;
        double2* src = op->ws.src;
        double2* buf = op->ws.bufs;
        {
            Stage s_(pc, "project");
            SIE_CUDA_TRY(cudaMemsetAsync(src, 0, sizeof(double2) * ngrid * Ng, st));
            k_project<<<(M.nt * S + 255) / 256, 256, 0, st>>>(M.nt, S, g.M, M, op->base, op->W, x, g, ngrid, src, Ng);
            SIE_CUDA_TRY(cudaGetLastError());
        }
        SIE_TRY(fft3d(st, buf, src, g, -1, 1, pc, ngrid));
        {
            Stage s_(pc, "specmul");
            k_specmul<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(which_LK, a.spec, buf, nn);
            SIE_CUDA_TRY(cudaGetLastError());
        }
        SIE_TRY(fft3d(st, buf, src, g, +1, 1, pc, ngrid));
        std::complex<double> kk(a.kr, a.ki);
        std::complex<double> sc = -1.0 / (kk * kk);
        {
            Stage s_(pc, "interp");
            SIE_TRY(aim_interp(op, src, which_LK == 0, make_double2(sc.real(), sc.imag()), y));
        }
    }
    {
        Stage s_(pc, a.has_grid ? "spmv_aim" : "spmv_near_only");
        // near-only operators have no grid term: the product overwrites y
        const double2* v = which_LK == 0 ? a.valL : a.valK;
        SIE_CUDA_TRY(csr_launch(st, M.ne, a.nnz, a.row_ptr, a.col, v, x, make_double2(1.0, 0.0), a.has_grid, y));
        SIE_CUDA_TRY(cudaGetLastError());
    }
    return SIE_OK;
}

static void free_aim(AimOp& a)
{
    void* ptrs[] = {a.spec, a.spec32, a.pairs, a.row_ptr, a.col, a.valL, a.valK, a.valLA, a.dLA, a.dL,
                    a.tri_row_ptr, a.tri_col, a.valLphi, a.valLphiNR, a.valM, a.valLK32, a.valLphi32,
                    a.obj_k, a.obj_ik2};
    a.obj_k = a.obj_ik2 = nullptr;
    for (void* p : ptrs)
        if (p) cudaFree(p);
    a.valLA = a.dLA = a.dL = a.valLphi = a.valLphiNR = a.valM = nullptr;
    a.valLK32 = nullptr;
    a.valLphi32 = nullptr;
    a.tri_row_ptr = nullptr;
    a.tri_col = nullptr;
    a.spec = nullptr;
    a.spec32 = nullptr;
    a.pairs = nullptr;
    a.row_ptr = nullptr;
    a.col = nullptr;
    a.valL = a.valK = nullptr;
}

}  // namespace sie

using namespace sie;

extern "C" {

sie_status sie_op_destroy(sie_op* op)
{
    if (!op) return SIE_ERR_ARG;
    cudaSetDevice(op->mesh->ctx->device);
    cudaStreamSynchronize(op->mesh->ctx->stream);
    sys_release(op);
    free_aim(op->ext);
    free_aim(op->inn);
    void* ptrs[] = {op->base, op->W, op->W32, op->ws.bufs, op->ws.src, op->xtmp, op->bws_bufs, op->bws_src, op->bws_vec,
                    op->edge_zf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete op;
    return SIE_OK;
}

sie_status sie_op_build(sie_mesh* mesh, double freq_hz, double eps_r, double mu_r, double sigma,
                        const sie_params* params, sie_op** out)
{
    if (!mesh || !out || !(freq_hz > 0) || !(eps_r > 0) || !(mu_r > 0) || sigma < 0) {
        set_error("sie_op_build: invalid argument");
        return SIE_ERR_ARG;
    }
    SIE_CUDA_TRY(cudaSetDevice(mesh->ctx->device));
    cudaStream_t st = mesh->ctx->stream;
    auto* op = new sie_op();
    op->mesh = mesh;
    if (params)
        op->p = *params;
    else
        sie_params_default(&op->p);
    if (op->p.interior_model != SIE_GIBC && op->p.interior_model != SIE_SIBC) {
        delete op;
        set_error("sie_op_build: interior_model must be SIE_GIBC or SIE_SIBC");
        return SIE_ERR_ARG;
    }
    const double c0 = 299792458.0, mu0 = 4e-7 * M_PI, eps0 = 1.0 / (mu0 * c0 * c0), eta0 = mu0 * c0;
    const double w = 2 * M_PI * freq_hz;
    // per-object materials (Sec. II): sie_set_material, else the arguments
    const int nobj = mesh->h.nobj;
    struct ObjMat {
        double eps_r, mu_r, sigma;
        std::complex<double> k, zs, eta;  // Eq. kin; j k0 eps_r + sigma eta0; eta_i / eta0
        double cut;                        // skin-depth cutoff of the interior near region
    };
    std::vector<ObjMat> om(nobj);
    for (int o = 0; o < nobj; o++) {
        const bool set = o < (int)mesh->mat.size() && mesh->mat[o].set;
        ObjMat& m = om[o];
        m.eps_r = set ? mesh->mat[o].eps_r : eps_r;
        m.mu_r = set ? mesh->mat[o].mu_r : mu_r;
        m.sigma = set ? mesh->mat[o].sigma : sigma;
        // Eq. (kin): k_i = sqrt(w mu (w eps - j sigma)), branch Im k <= 0
        m.k = std::sqrt(std::complex<double>(w * mu0 * m.mu_r) * std::complex<double>(w * eps0 * m.eps_r, -m.sigma));
        if (m.k.imag() > 0) m.k = -m.k;
        m.zs = std::complex<double>(m.sigma * eta0, w / c0 * m.eps_r);
        // eta_i / eta0 = sqrt(mu_r / eps~_r), eps~_r = eps_r - j sigma / (w eps0), branch Re > 0
        m.eta = std::sqrt(std::complex<double>(m.mu_r) / std::complex<double>(m.eps_r, -m.sigma / (w * eps0)));
        if (m.eta.real() < 0) m.eta = -m.eta;
        const double delta = m.k.imag() < 0 ? -1.0 / m.k.imag() : 1e300;
        m.cut = op->p.skin_cutoff * delta;
    }
    op->freq = freq_hz;
    op->eps_r = om[0].eps_r;
    op->mu_r = om[0].mu_r;
    op->sigma = om[0].sigma;
    op->k0 = w / c0;
    const std::complex<double> ki = om[0].k;
    auto fail = [&](sie_status s) {
        sie_op_destroy(op);
        return s;
    };
    sie_status s;
    // exterior grid (Sec. III-D: one global grid around the structure)
    GridDesc g;
    if ((s = make_grid(mesh->h, op->p, g)) != SIE_OK) return fail(s);
    std::vector<int32_t> hb;
    stencil_base(mesh->h, g, hb);
    for (int64_t t = 0; t < mesh->h.nt; t++)
        for (int d = 0; d < 3; d++)
            if (hb[3 * t + d] < 0 || hb[3 * t + d] + g.M > g.N[d] - 1) {
                set_error("stencil outside the grid");
                return fail(SIE_ERR_MESH);
            }
    if ((s = up(st, &op->base, hb.data(), hb.size())) != SIE_OK) return fail(s);
    op->ext.g = g;
    op->ext.kr = op->k0;
    op->ext.ki = 0.0;
    op->ext.has_grid = true;
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
        return std::chrono::duration<double, std::milli>(b - a).count();
    };
    auto t0 = now();
    if ((s = aim_weights(op)) != SIE_OK) return fail(s);
    QuadDev q;
    make_quad(op->p, q);
    if ((s = aim_spectra(op, op->ext)) != SIE_OK) return fail(s);
    cudaStreamSynchronize(st);
    auto t1 = now();
    op->build_ms[0] = ms(t0, t1);
    near_pairs_grid(mesh->h, g, hb, op->ext.hpairs);
    auto t2 = now();
    op->build_ms[3] = ms(t1, t2);
    if ((s = near_build(op, op->ext, q)) != SIE_OK) return fail(s);
    {
        AimOp& X = op->ext;
        const int64_t ntri = X.tri_row_ptr_h.empty() ? 0 : X.tri_row_ptr_h.back();
        if ((s = to_c64_pair(st, X.valLA, X.valK, X.nnz, &X.valLK32)) != SIE_OK ||
            (s = to_c64(st, X.valLphi, ntri, &X.valLphi32)) != SIE_OK)
            return fail(s);
    }
    auto t3 = now();
    op->build_ms[1] = ms(t2, t3);
    // interior operator (Sec. III-C): near-only when every pair inside the
    // skin-depth cutoff is a near pair, else AIM on the object grid (shared
    // with the exterior grid for a single object)
    op->inn.kr = ki.real();
    op->inn.ki = ki.imag();
    op->inn.g = g;
    const double cut = om[0].cut;
    op->eta_re = om[0].eta.real();
    op->eta_im = om[0].eta.imag();
    if (nobj > 1) {
        // block-diagonal Z': a per-edge factor from the edge's object
        const HostMesh& H = mesh->h;
        std::vector<double2> zf(H.ne);
        for (int64_t e = 0; e < H.ne; e++) {
            const ObjMat& m = om[H.obj[H.edge_tri[2 * e]]];
            const std::complex<double> f = op->p.interior_model == SIE_SIBC ? m.eta : -1.0 / m.zs;
            zf[e] = make_double2(f.real(), f.imag());
        }
        if ((s = up(st, &op->edge_zf, zf.data(), zf.size())) != SIE_OK) return fail(s);
    }
    if (op->p.interior_model == SIE_SIBC) {
        op->inn.has_grid = false;  // no interior operators: Z' comes from the Gram system
    } else if (nobj > 1) {
        for (int o = 0; o < nobj; o++)
            if (om[o].cut > (g.Rnear - g.M) * g.h) {
                set_error("sie_op_build: object " + std::to_string(o) +
                          " needs an interior AIM grid; several objects need near-region-only interiors "
                          "(5 skin depths inside the near region) or interior_model = SIE_SIBC");
                return fail(SIE_ERR_UNSUPPORTED);
            }
        op->inn.has_grid = false;
        std::vector<double> cuts(nobj);
        std::vector<double2> kk(nobj), ik2(nobj);
        for (int o = 0; o < nobj; o++) {
            cuts[o] = om[o].cut;
            kk[o] = make_double2(om[o].k.real(), om[o].k.imag());
            const std::complex<double> v = 1.0 / (om[o].k * om[o].k);
            ik2[o] = make_double2(v.real(), v.imag());
        }
        near_pairs_cutoff_objects(mesh->h, cuts, op->inn.hpairs);
        if ((s = up(st, &op->inn.obj_k, kk.data(), kk.size())) != SIE_OK) return fail(s);
        if ((s = up(st, &op->inn.obj_ik2, ik2.data(), ik2.size())) != SIE_OK) return fail(s);
    } else if (cut <= (g.Rnear - g.M) * g.h) {
        op->inn.has_grid = false;
        near_pairs_cutoff(mesh->h, cut, op->inn.hpairs);
    } else {
        op->inn.has_grid = true;
        if ((s = aim_spectra(op, op->inn)) != SIE_OK) return fail(s);
        op->inn.hpairs = op->ext.hpairs;
    }
    auto t4 = now();
    if (op->p.interior_model != SIE_SIBC) {
        if ((s = near_build(op, op->inn, q)) != SIE_OK) return fail(s);
        // near-only interior: approximate inverse of L_i,NR for the nested solve
        if (!op->inn.has_grid && (s = spai_build(st, op->inn.csr, op->inn.valL, &op->inn.valM)) != SIE_OK)
            return fail(s);
    }
    op->build_ms[2] = ms(t4, now());
    // workspace
    int64_t nn = (int64_t)g.n[0] * g.n[1] * g.n[2], Ng = (int64_t)g.N[0] * g.N[1] * g.N[2];
    op->ws.grid_elems = nn;
    cudaError_t e1 = cudaMallocAsync((void**)&op->ws.bufs, sizeof(double2) * 7 * nn, st);
    cudaError_t e2 = cudaMallocAsync((void**)&op->ws.src, sizeof(double2) * 7 * Ng, st);
    cudaError_t e3 = cudaMallocAsync((void**)&op->xtmp, sizeof(double2) * 4 * mesh->h.ne, st);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        set_error("sie_op_build: workspace allocation failed");
        return fail(SIE_ERR_OOM);
    }
    if ((s = sys_prepare(op)) != SIE_OK) return fail(s);
    if ((s = constraint_lu_build(op)) != SIE_OK) return fail(s);
    if ((s = csr_tune_op(op)) != SIE_OK) return fail(s);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error(std::string("sie_op_build: ") + cudaGetErrorString(e));
        return fail(SIE_ERR_CUDA);
    }
    *out = op;
    return SIE_OK;
}

sie_status sie_matvec(sie_op* op, int which, const double* x, double* y, int nrhs, int flags)
{
    if (!op || !x || !y || nrhs < 1 || which < SIE_OP_L0 || which > SIE_OP_ZI) {
        set_error("sie_matvec: invalid argument");
        return SIE_ERR_ARG;
    }
    if (op->p.interior_model == SIE_SIBC && (which == SIE_OP_LI || which == SIE_OP_KI)) {
        set_error("sie_matvec: an operator built with SIE_SIBC has no interior operators");
        return SIE_ERR_STATE;
    }
    SIE_CUDA_TRY(cudaSetDevice(op->mesh->ctx->device));
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t ne = op->mesh->h.ne, nt = op->mesh->h.nt;
    const int64_t len = which == SIE_OP_SYS ? ne + nt : ne;
    bool dev = flags & SIE_DEVICE_PTRS;
    if (which >= SIE_OP_SYS) SIE_TRY(nested_clear(op));
    if (which < SIE_OP_SYS && nrhs > 1) {
        // blocks of up to 8 right-hand sides: spectra, weights and near values read once per block
        AimOp& a = (which == SIE_OP_L0 || which == SIE_OP_K0) ? op->ext : op->inn;
        const int lk = (which == SIE_OP_L0 || which == SIE_OP_LI) ? 0 : 1;
        const int RBLK = 8;
        if (!dev && !op->bws_vec)
            SIE_CUDA_TRY(cudaMallocAsync((void**)&op->bws_vec, sizeof(double2) * 2 * RBLK * ne, st));
        for (int r0 = 0; r0 < nrhs; r0 += RBLK) {
            const int nr = std::min(RBLK, nrhs - r0);
            const double2* X = (const double2*)x + (int64_t)r0 * ne;
            double2* Y = (double2*)y + (int64_t)r0 * ne;
            if (!dev) {
                SIE_CUDA_TRY(cudaMemcpyAsync(op->bws_vec, X, sizeof(double2) * nr * ne, cudaMemcpyHostToDevice, st));
                X = op->bws_vec;
            }
            double2* Yd = dev ? Y : op->bws_vec + RBLK * ne;
            SIE_TRY(aim_apply_block(op, a, lk, X, Yd, nr));
            if (!dev) SIE_CUDA_TRY(cudaMemcpyAsync(Y, Yd, sizeof(double2) * nr * ne, cudaMemcpyDeviceToHost, st));
        }
        if (!dev) SIE_CUDA_TRY(cudaStreamSynchronize(st));
        return SIE_OK;
    }
    for (int r = 0; r < nrhs; r++) {
        const double2* xr;
        double2* yr;
        if (dev) {
            xr = (const double2*)x + r * len;
            yr = (double2*)y + r * len;
        } else {
            SIE_CUDA_TRY(cudaMemcpyAsync(op->sys_vec, (const double2*)x + r * len, sizeof(double2) * len,
                                         cudaMemcpyHostToDevice, st));
            xr = op->sys_vec;
            yr = op->sys_vec + len;
        }
        if (which >= SIE_OP_SYS) {
            SIE_TRY(sys_matvec(op, which, xr, yr));
        } else {
            AimOp& a = (which == SIE_OP_L0 || which == SIE_OP_K0) ? op->ext : op->inn;
            int lk = (which == SIE_OP_L0 || which == SIE_OP_LI) ? 0 : 1;
            SIE_TRY(aim_apply(op, a, lk, xr, yr));
        }
        if (!dev)
            SIE_CUDA_TRY(cudaMemcpyAsync((double2*)y + r * len, yr, sizeof(double2) * len, cudaMemcpyDeviceToHost, st));
    }
    if (!dev) {
        SIE_CUDA_TRY(cudaStreamSynchronize(st));
        // host buffers: the call synchronises anyway, so an inexact nested solve is reported here
        if (which >= SIE_OP_SYS) return nested_check(op, "sie_matvec");
    }
    return SIE_OK;
}

sie_status sie_op_near_csr(const sie_op* op, int which, int64_t* row_ptr, int32_t* col, double* val, int64_t* nnz)
{
    if (!op || !row_ptr || !nnz || which < SIE_OP_L0 || which > SIE_OP_KI) {
        set_error("sie_op_near_csr: invalid argument");
        return SIE_ERR_ARG;
    }
    if (op->p.interior_model == SIE_SIBC && (which == SIE_OP_LI || which == SIE_OP_KI)) {
        set_error("sie_op_near_csr: an operator built with SIE_SIBC has no interior operators");
        return SIE_ERR_STATE;
    }
    const AimOp& a = (which == SIE_OP_L0 || which == SIE_OP_K0) ? op->ext : op->inn;
    int lk = (which == SIE_OP_L0 || which == SIE_OP_LI) ? 0 : 1;
    *nnz = a.nnz;
    std::memcpy(row_ptr, a.csr.row_ptr.data(), sizeof(int64_t) * a.csr.row_ptr.size());
    if (col) std::memcpy(col, a.csr.col.data(), sizeof(int32_t) * a.nnz);
    if (val) {
        SIE_CUDA_TRY(cudaSetDevice(op->mesh->ctx->device));
        SIE_CUDA_TRY(cudaMemcpy(val, lk == 0 ? a.valL : a.valK, sizeof(double2) * a.nnz, cudaMemcpyDeviceToHost));
    }
    return SIE_OK;
}

sie_status sie_rhs_planewave(sie_op* op, const double* khat, const double* epol, int nrhs, double* b, int flags)
{
    if (!op || !khat || !epol || !b || nrhs < 1) {
        set_error("sie_rhs_planewave: invalid argument");
        return SIE_ERR_ARG;
    }
    SIE_CUDA_TRY(cudaSetDevice(op->mesh->ctx->device));
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    for (int r = 0; r < nrhs; r++) {
        double2* br = (flags & SIE_DEVICE_PTRS) ? (double2*)b + r * len : op->sys_vec;
        SIE_TRY(sys_rhs(op, khat + 3 * r, epol + 3 * r, br));
        if (!(flags & SIE_DEVICE_PTRS))
            SIE_CUDA_TRY(cudaMemcpyAsync((double2*)b + r * len, br, sizeof(double2) * len, cudaMemcpyDeviceToHost, st));
    }
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    return SIE_OK;
}

sie_status sie_solve(sie_op* op, const double* b, double* x, int nrhs, int* iters, double* relres, int flags)
{
    if (!op || !b || !x || nrhs < 1) {
        set_error("sie_solve: invalid argument");
        return SIE_ERR_ARG;
    }
    SIE_CUDA_TRY(cudaSetDevice(op->mesh->ctx->device));
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    sie_status worst = SIE_OK;
    if (nrhs > 1 && !(flags & SIE_SOLVE_SEQUENTIAL)) {
        // blocks of up to 8 right-hand sides solved in lockstep
        const bool dev = flags & SIE_DEVICE_PTRS;
        if (!dev && !op->mvec)
            SIE_CUDA_TRY(cudaMallocAsync((void**)&op->mvec, sizeof(double2) * 2 * 8 * len, st));
        for (int r0 = 0; r0 < nrhs; r0 += 8) {
            const int R = std::min(8, nrhs - r0);
            const double2* bq[8];
            double2* xq[8];
            for (int q = 0; q < R; q++) {
                if (dev) {
                    bq[q] = (const double2*)b + (r0 + q) * len;
                    xq[q] = (double2*)x + (r0 + q) * len;
                } else {
                    double2* bd = op->mvec + (int64_t)q * len;
                    SIE_CUDA_TRY(cudaMemcpyAsync(bd, (const double2*)b + (r0 + q) * len, sizeof(double2) * len,
                                                 cudaMemcpyHostToDevice, st));
                    bq[q] = bd;
                    xq[q] = op->mvec + (int64_t)(8 + q) * len;
                }
            }
            sie_status s = sys_solve_multi(op, R, bq, xq, iters ? iters + r0 : nullptr,
                                           relres ? relres + r0 : nullptr, (flags & SIE_SOLVE_REFINE) != 0);
            if (s != SIE_OK && s != SIE_ERR_NOT_CONVERGED) return s;
            if (s == SIE_ERR_NOT_CONVERGED) worst = s;
            if (!dev)
                for (int q = 0; q < R; q++)
                    SIE_CUDA_TRY(cudaMemcpyAsync((double2*)x + (r0 + q) * len, xq[q], sizeof(double2) * len,
                                                 cudaMemcpyDeviceToHost, st));
        }
        SIE_CUDA_TRY(cudaStreamSynchronize(st));
        if (worst != SIE_OK) set_error("sie_solve: GMRES reached maxit before the tolerance");
        return worst;
    }
    for (int r = 0; r < nrhs; r++) {
        const double2* br;
        double2* xr;
        if (flags & SIE_DEVICE_PTRS) {
            br = (const double2*)b + r * len;
            xr = (double2*)x + r * len;
        } else {
            SIE_CUDA_TRY(cudaMemcpyAsync(op->sys_vec + 2 * len, (const double2*)b + r * len, sizeof(double2) * len,
                                         cudaMemcpyHostToDevice, st));
            br = op->sys_vec + 2 * len;
            xr = op->sys_vec + 3 * len;
        }
        int it = 0;
        double rr = 0;
        sie_status s = (flags & SIE_SOLVE_REFINE) ? sys_solve_refined(op, br, xr, &it, &rr)
                                                  : sys_solve(op, br, xr, &it, &rr);
        if (s != SIE_OK && s != SIE_ERR_NOT_CONVERGED) return s;
        if (s == SIE_ERR_NOT_CONVERGED) worst = s;
        if (iters) iters[r] = it;
        if (relres) relres[r] = rr;
        if (!(flags & SIE_DEVICE_PTRS))
            SIE_CUDA_TRY(cudaMemcpyAsync((double2*)x + r * len, xr, sizeof(double2) * len, cudaMemcpyDeviceToHost, st));
    }
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    if (worst != SIE_OK) set_error("sie_solve: GMRES reached maxit before the tolerance");
    return worst;
}

sie_status sie_rcs(sie_op* op, const double* x, const double* rhat, int ndir, double* rcs, int flags)
{
    if (!op || !x || !rhat || !rcs || ndir < 1) {
        set_error("sie_rcs: invalid argument");
        return SIE_ERR_ARG;
    }
    SIE_CUDA_TRY(cudaSetDevice(op->mesh->ctx->device));
    cudaStream_t st = op->mesh->ctx->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    const double2* xr = (const double2*)x;
    if (!(flags & SIE_DEVICE_PTRS)) {
        SIE_CUDA_TRY(cudaMemcpyAsync(op->sys_vec, x, sizeof(double2) * len, cudaMemcpyHostToDevice, st));
        xr = op->sys_vec;
    }
    return sys_rcs(op, xr, rhat, ndir, rcs);
}

}  // extern "C"
