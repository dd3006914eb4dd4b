// CSR sparse products (complex128) for the near-region matrices.
//
// A group of G lanes (G = 4, 8 or 32) works on one row; each lane keeps four
// (column, value) loads and then four gathers of x in flight before using
// them, so that short rows (the near-only interior operators hold ~30 entries
// per row) are not one long dependent load chain per warp.  The group sums by
// a fixed xor-shuffle tree: the result is the same on every run.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

namespace sie {

// VT = double2: FP64 throughout.  VT = float2 (complex64 values of the mixed
// precision path): FP32 products and per-lane sums, the group sum in FP64.
// XT: type of x (float2 with float2 values: no conversion in the inner loop)
template <int G, class VT, class XT>
__device__ __forceinline__ double2 csr_row_dot(int64_t e0, int64_t e1, const int32_t* __restrict__ col,
                                               const VT* __restrict__ val, const XT* __restrict__ x, int l)
{
    using R = decltype(VT{}.x);
    R ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};  // one set per unrolled slot (independent chains)
    int64_t e = e0 + l;
    for (; e + 3 * G < e1; e += 4 * G) {
        int c[4];
        VT v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            c[u] = __ldg(col + e + u * G);
            v[u] = __ldg(val + e + u * G);
        }
        XT xv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) xv[u] = __ldg(x + c[u]);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const R xr = (R)xv[u].x, xi = (R)xv[u].y;
            ar[u] += v[u].x * xr - v[u].y * xi;
            ai[u] += v[u].x * xi + v[u].y * xr;
        }
    }
    {  // at most 3 more entries per lane: their loads issued together
        int c[3];
        VT v[3];
        XT xv[3];
#pragma unroll
        for (int u = 0; u < 3; u++) {
            const bool ok = e + u * G < e1;
            c[u] = ok ? __ldg(col + e + u * G) : -1;
            if (ok) v[u] = __ldg(val + e + u * G);
        }
#pragma unroll
        for (int u = 0; u < 3; u++)
            if (c[u] >= 0) xv[u] = __ldg(x + c[u]);
#pragma unroll
        for (int u = 0; u < 3; u++)
            if (c[u] >= 0) {
                const R xr = (R)xv[u].x, xi = (R)xv[u].y;
                ar[u] += v[u].x * xr - v[u].y * xi;
                ai[u] += v[u].x * xi + v[u].y * xr;
            }
    }
    double sr = ((double)ar[0] + (double)ar[1]) + ((double)ar[2] + (double)ar[3]);
    double si = ((double)ai[0] + (double)ai[1]) + ((double)ai[2] + (double)ai[3]);
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    return make_double2(sr, si);
}

// y = alpha A x (ACC = false) or y += alpha A x (ACC = true); blockDim 256
template <int G, bool ACC, class VT, class XT>
__global__ void __launch_bounds__(256) k_csr(int nrow, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                             const VT* __restrict__ val, const XT* __restrict__ x,
                                             double2 alpha, double2* __restrict__ y)
{
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G);
    const int l = threadIdx.x % G;
    const bool ok = r < nrow;
    // rows past the end still take part in the shuffles, with an empty range
    const int64_t e0 = ok ? __ldg(rp + r) : 0, e1 = ok ? __ldg(rp + r + 1) : 0;
    const double2 s = csr_row_dot<G, VT, XT>(e0, e1, col, val, x, l);
    if (ok && l == 0) {
        double2 t = make_double2(alpha.x * s.x - alpha.y * s.y, alpha.x * s.y + alpha.y * s.x);
        if (ACC) {
            double2 o = y[r];
            t.x += o.x;
            t.y += o.y;
        }
        y[r] = t;
    }
}

// lanes per row from the mean row length (the default before tuning)
inline int csr_group(int64_t nrow, int64_t nnz)
{
    const int64_t avg = nrow > 0 ? nnz / nrow : 0;
    return avg <= 12 ? 4 : (avg <= 48 ? 8 : 32);
}

// Lanes per row chosen by measurement (csr_autotune), per matrix pattern
// (row pointer, rows, entries) and value width; csr_launch falls back to
// csr_group for patterns never tuned.
struct CsrTuneTable {
    std::mutex mu;
    std::map<std::tuple<const void*, int, int64_t, int>, int> g;
};
inline CsrTuneTable& csr_tune_table()
{
    static CsrTuneTable t;
    return t;
}
inline int csr_group_for(const int64_t* rp, int nrow, int64_t nnz, int vbytes)
{
    CsrTuneTable& t = csr_tune_table();
    std::lock_guard<std::mutex> lk(t.mu);
    auto it = t.g.find(std::make_tuple((const void*)rp, nrow, nnz, vbytes));
    return it != t.g.end() ? it->second : csr_group(nrow, nnz);
}

template <class VT, class XT>
inline cudaError_t csr_launch_g(cudaStream_t st, int G, int nrow, const int64_t* rp, const int32_t* col,
                                const VT* val, const XT* x, double2 alpha, bool acc, double2* y);

template <class VT, class XT>
inline cudaError_t csr_launch(cudaStream_t st, int nrow, int64_t nnz, const int64_t* rp, const int32_t* col,
                              const VT* val, const XT* x, double2 alpha, bool acc, double2* y)
{
    if (nrow <= 0) return cudaSuccess;
    return csr_launch_g(st, csr_group_for(rp, nrow, nnz, (int)sizeof(VT)), nrow, rp, col, val, x, alpha, acc, y);
}

// the product with G lanes per row (4, 8, 16 or 32)
template <class VT, class XT>
inline cudaError_t csr_launch_g(cudaStream_t st, int G, int nrow, const int64_t* rp, const int32_t* col,
                                const VT* val, const XT* x, double2 alpha, bool acc, double2* y)
{
    const unsigned blocks = (unsigned)(((int64_t)nrow * G + 255) / 256);
    if (G == 4) {
        if (acc) k_csr<4, true, VT, XT><<<blocks, 256, 0, st>>>(nrow, rp, col, val, x, alpha, y);
        else k_csr<4, false, VT, XT><<<blocks, 256, 0, st>>>(nrow, rp, col, val, x, alpha, y);
    } else if (G == 8) {
        if (acc) k_csr<8, true, VT, XT><<<blocks, 256, 0, st>>>(nrow, rp, col, val, x, alpha, y);
        else k_csr<8, false, VT, XT><<<blocks, 256, 0, st>>>(nrow, rp, col, val, x, alpha, y);
    } else if (G == 16) {
        if (acc) k_csr<16, true, VT, XT><<<blocks, 256, 0, st>>>(nrow, rp, col, val, x, alpha, y);
        else k_csr<16, false, VT, XT><<<blocks, 256, 0, st>>>(nrow, rp, col, val, x, alpha, y);
    } else {
        if (acc) k_csr<32, true, VT, XT><<<blocks, 256, 0, st>>>(nrow, rp, col, val, x, alpha, y);
        else k_csr<32, false, VT, XT><<<blocks, 256, 0, st>>>(nrow, rp, col, val, x, alpha, y);
    }
    return cudaGetLastError();
}

// Autotuner of the CSR products: on a matrix's first tuning call (never
// while the stream is being captured) time each group size on it -- one
// warm-up and three timed launches into the scratch y_tmp (nrow values), on
// the stream st, CUDA events -- and keep the fastest for csr_launch.
template <class VT, class XT>
inline cudaError_t csr_autotune(cudaStream_t st, int nrow, int64_t nnz, const int64_t* rp, const int32_t* col,
                                const VT* val, const XT* x, double2* y_tmp)
{
    if (nrow <= 0 || nnz <= 0) return cudaSuccess;
    const auto key = std::make_tuple((const void*)rp, nrow, nnz, (int)sizeof(VT));
    {
        CsrTuneTable& t = csr_tune_table();
        std::lock_guard<std::mutex> lk(t.mu);
        if (t.g.count(key)) return cudaSuccess;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    int best = csr_group(nrow, nnz);
    float best_ms = 1e30f;
    for (int G : {4, 8, 16, 32}) {
        if ((e = csr_launch_g(st, G, nrow, rp, col, val, x, make_double2(1.0, 0.0), false, y_tmp)) != cudaSuccess) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; r++)
            if ((e = csr_launch_g(st, G, nrow, rp, col, val, x, make_double2(1.0, 0.0), false, y_tmp)) != cudaSuccess)
                break;
        cudaEventRecord(e1, st);
        if (e != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = G;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) {
        CsrTuneTable& t = csr_tune_table();
        std::lock_guard<std::mutex> lk(t.mu);
        t.g[key] = best;
    }
    return e;
}

}  // namespace sie
