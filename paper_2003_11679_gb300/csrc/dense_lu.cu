// Dense complex LU on the GPU for the triangle (charge) system of the AEFIE
// constraint preconditioner (Sec. III-D) and of the nested preconditioner's
// constraint form (Eq. nest2pc).  The paper factorises its sparse
// preconditioner by a sparse LU; here the N_t x N_t triangle system that
// block elimination leaves is assembled densely and factorised once per
// operator in complex64:
//   * right-looking blocked LU with partial pivoting, NB = 64 columns per
//     panel, row-major storage (row swaps are contiguous copies);
//   * panel: one pivot-search/swap launch and one update launch per column;
//   * the block row U12 = L11^-1 A12 and the trailing update A22 -= L21 U12 are
//     complex GEMMs on the FP32 pipes (128 x 128 output tiles, the whole
//     K = NB slice in shared memory);
//   * the inverses of the diagonal blocks are kept, so each block step of a
//     triangular solve is a 64 x 64 matrix-vector product;
//   * triangular solves: one CTA per 64-row block, blocks taken in dispatch
//     order from a ticket counter; a block waits (bounded) for the flags of the
//     blocks it depends on, accumulates their products as they complete and
//     publishes its own result with a flag.  A wait that runs out sets an error
//     flag the host reads (SIE_ERR_TIMEOUT); nothing spins forever.
// The factorisation serves as the preconditioner of an FP64 GMRES on the exact
// sparse triangle system, so its FP32 rounding costs iterations, not accuracy.
#include <cmath>
#include <vector>

#include <algorithm>

#include "internal.h"

namespace sie {

constexpr int LU_NB = 64;
constexpr int GEMM_BM = 128, GEMM_BN = 128, GEMM_PAD = 4;
constexpr long long SPIN_LIMIT = 1LL << 22;  // polls of a flag before a wait gives up

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c)  // c + a b
{
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cdivf(float2 a, float2 b)
{
    // scaled division: (a conj b) / |b|^2 with |b| scaled to ~1
    float s = fmaxf(fabsf(b.x), fabsf(b.y));
    float2 bs = make_float2(b.x / s, b.y / s);
    float d = bs.x * bs.x + bs.y * bs.y;
    return make_float2((a.x * bs.x + a.y * bs.y) / (d * s), (a.y * bs.x - a.x * bs.y) / (d * s));
}

// ------------------------------------------------------------------ assembly
// T = I - kappa Dop diag(1/dLA) DTop Lphi_NR, row-major complex64, where
// (Dop y)_t = sum_i 2 c_{t,i} A_t y_{e(t,i)}, (DTop phi)_m = l_m (phi_T+ - phi_T-)
// and Lphi_NR is the triangle CSR (row p: pairs (p, s)).  One CTA per row;
// the six (edge, triangle) contributions of a row are added one after another.
__global__ void __launch_bounds__(256) k_assemble_T(int nt, DevMesh M, const double* __restrict__ elen,
                                                    const double2* __restrict__ dLA, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ col, const double2* __restrict__ val,
                                                    double2 kappa, float2* __restrict__ T, int64_t ldt)
{
    const int t = blockIdx.x;
    float2* row = T + (int64_t)t * ldt;
    for (int s = threadIdx.x; s < nt; s += blockDim.x) row[s] = make_float2(s == t ? 1.f : 0.f, 0.f);
    __syncthreads();
    for (int i = 0; i < 3; i++) {
        const int e = M.tri_edge[3 * t + i];
        const double cw = 2.0 * M.coef[3 * t + i] * M.area[t];
        const double2 d = dLA[e];
        const double den = d.x * d.x + d.y * d.y;
        // w = -kappa cw / d
        const double2 q = make_double2(cw * d.x / den, -cw * d.y / den);
        const double2 w = make_double2(-(kappa.x * q.x - kappa.y * q.y), -(kappa.x * q.y + kappa.y * q.x));
        for (int b = 0; b < 2; b++) {
            const int p = M.edge_tri[2 * e + b];
            const double sg = b == 0 ? elen[e] : -elen[e];
            const double2 cf = make_double2(sg * w.x, sg * w.y);
            for (int64_t k = rp[p] + threadIdx.x; k < rp[p + 1]; k += blockDim.x) {
                const double2 v = val[k];
                float2& o = row[col[k]];
                o.x += (float)(cf.x * v.x - cf.y * v.y);
                o.y += (float)(cf.x * v.y + cf.y * v.x);
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ panel
// pivot of column c = k + j among rows c..n-1 (largest |a|, lowest index on
// ties), recorded in ipiv[c]; rows c and p swapped inside the panel columns
// [k, k + kb); the pivot row's panel part copied to prow.  One CTA.
__global__ void __launch_bounds__(1024) k_panel_pivot(int n, int k, int kb, int j, float2* __restrict__ A, int64_t lda,
                                                      int* __restrict__ ipiv, float2* __restrict__ prow,
                                                      int* __restrict__ err)
{
    const int c = k + j;
    __shared__ float sv[32];
    __shared__ int si[32];
    float best = -1.f;
    int bi = c;
    for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
        float2 a = A[(int64_t)r * lda + c];
        float v = fabsf(a.x) + fabsf(a.y);
        if (v > best) {  // rows visited in increasing order per thread: keeps the lowest index on ties
            best = v;
            bi = r;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        float ov = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sv[warp] = best;
        si[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) / 32;
        best = lane < nw ? sv[lane] : -1.f;
        bi = lane < nw ? si[lane] : n;
        for (int off = 16; off > 0; off >>= 1) {
            float ov = __shfl_down_sync(0xffffffffu, best, off);
            int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            si[0] = bi;
            ipiv[c] = bi;
            if (!(best > 0.f)) atomicExch(err, 2);  // singular (or non-finite) pivot column
        }
    }
    __syncthreads();
    const int p = si[0];
    for (int q = threadIdx.x; q < kb; q += blockDim.x) {
        float2* rc = A + (int64_t)c * lda + k + q;
        float2* rpv = A + (int64_t)p * lda + k + q;
        float2 vc = *rc, vp = *rpv;
        *rc = vp;
        *rpv = vc;
        prow[q] = vp;
    }
}

// rows r > c: l = a[r, c] / a[c, c]; a[r, c] = l; a[r, c+1 .. k+kb) -= l prow
__global__ void __launch_bounds__(256) k_panel_update(int n, int k, int kb, int j, float2* __restrict__ A,
                                                      int64_t lda, const float2* __restrict__ prow)
{
    const int c = k + j;
    const int r = c + 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float2* a = A + (int64_t)r * lda + k;
    const float2 piv = prow[j];
    if (piv.x == 0.f && piv.y == 0.f) return;
    const float2 l = cdivf(a[j], piv);
    a[j] = l;
    for (int q = j + 1; q < kb; q++) {
        float2 u = prow[q];
        a[q] = make_float2(a[q].x - (l.x * u.x - l.y * u.y), a[q].y - (l.x * u.y + l.y * u.x));
    }
}

// the panel's row swaps applied to the columns outside [k, k + kb)
__global__ void k_laswp(int n, int k, int kb, float2* __restrict__ A, int64_t lda, const int* __restrict__ ipiv)
{
    int cc = blockIdx.x * blockDim.x + threadIdx.x;
    const int width = n - kb;
    if (cc >= width) return;
    const int col = cc < k ? cc : cc + kb;
    for (int j = 0; j < kb; j++) {
        const int r = k + j, p = ipiv[r];
        if (p != r) {
            float2 t = A[(int64_t)r * lda + col];
            A[(int64_t)r * lda + col] = A[(int64_t)p * lda + col];
            A[(int64_t)p * lda + col] = t;
        }
    }
}

// inverses of the unit-lower and the upper triangle of diagonal block b
// (kb x kb, padded to 64 with the identity); one CTA of 64 threads, thread c
// computes column c of each inverse (written to, and read back from, its own
// column of the output)
__global__ void __launch_bounds__(64) k_tri_inv(int n, int b, const float2* __restrict__ A, int64_t lda,
                                                float2* __restrict__ invL, float2* __restrict__ invU)
{
    __shared__ float2 D[LU_NB][LU_NB + 1];
    const int k = b * LU_NB, kb = min(LU_NB, n - k), c = threadIdx.x;
    for (int r = 0; r < LU_NB; r++)
        D[r][c] = (r < kb && c < kb) ? A[(int64_t)(k + r) * lda + k + c] : make_float2(r == c ? 1.f : 0.f, 0.f);
    __syncthreads();
    float2* XL = invL + (int64_t)b * LU_NB * LU_NB;
    float2* XU = invU + (int64_t)b * LU_NB * LU_NB;
    // L X = e_c, unit diagonal
    for (int r = 0; r < LU_NB; r++) {
        float2 s = make_float2(r == c ? 1.f : 0.f, 0.f);
        for (int q = c; q < r; q++) {
            float2 t = cmulf(D[r][q], XL[q * LU_NB + c]);
            s.x -= t.x;
            s.y -= t.y;
        }
        XL[r * LU_NB + c] = r < c ? make_float2(0.f, 0.f) : s;
    }
    // U X = e_c
    for (int r = LU_NB - 1; r >= 0; r--) {
        if (r > c) {
            XU[r * LU_NB + c] = make_float2(0.f, 0.f);
            continue;
        }
        float2 s = make_float2(r == c ? 1.f : 0.f, 0.f);
        for (int q = r + 1; q <= c; q++) {
            float2 t = cmulf(D[r][q], XU[q * LU_NB + c]);
            s.x -= t.x;
            s.y -= t.y;
        }
        XU[r * LU_NB + c] = cdivf(s, D[r][r]);
    }
}

// ------------------------------------------------------------------ complex GEMM (FP32 pipes)
// C (M x N) = A (M x K) B (K x N)  (sub = 0)   or   C -= A B  (sub = 1);
// row-major, K <= 64.  Tile 128 x 128 per CTA of 256 threads, thread (ty, tx)
// owns rows ty + 16 i and columns tx + 16 j (i, j < 8).  A CTA loads its whole
// B slice before it writes C, so C may alias B when M <= 128 (one row tile).
__global__ void __launch_bounds__(256) k_cgemm(int M, int N, int K, const float2* __restrict__ A, int64_t lda,
                                               const float2* B, int64_t ldb, float2* C, int64_t ldc, int sub)
{
    extern __shared__ __align__(16) unsigned char smraw_lu[];
    float2* As = reinterpret_cast<float2*>(smraw_lu);          // [64][BM + PAD]: As[k][m]
    float2* Bs = As + LU_NB * (GEMM_BM + GEMM_PAD);              // [64][BN + PAD]: Bs[k][n]
    const int m0 = blockIdx.y * GEMM_BM, n0 = blockIdx.x * GEMM_BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int idx = tid; idx < GEMM_BM * LU_NB; idx += 256) {
        const int m = idx / LU_NB, kk = idx % LU_NB;
        float2 v = make_float2(0.f, 0.f);
        if (m0 + m < M && kk < K) v = A[(int64_t)(m0 + m) * lda + kk];
        As[kk * (GEMM_BM + GEMM_PAD) + m] = v;
    }
    for (int idx = tid; idx < LU_NB * GEMM_BN; idx += 256) {
        const int kk = idx / GEMM_BN, nn = idx % GEMM_BN;
        float2 v = make_float2(0.f, 0.f);
        if (kk < K && n0 + nn < N) v = B[(int64_t)kk * ldb + n0 + nn];
        Bs[kk * (GEMM_BN + GEMM_PAD) + nn] = v;
    }
    __syncthreads();
    float2 acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = make_float2(0.f, 0.f);
    for (int kk = 0; kk < K; kk++) {
        float2 a[8], b[8];
#pragma unroll
        for (int i = 0; i < 8; i++) a[i] = As[kk * (GEMM_BM + GEMM_PAD) + ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 8; j++) b[j] = Bs[kk * (GEMM_BN + GEMM_PAD) + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 8; i++)
#pragma unroll
            for (int j = 0; j < 8; j++) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int nn = n0 + tx + 16 * j;
            if (nn >= N) continue;
            float2* c = C + (int64_t)m * ldc + nn;
            if (sub)
                *c = make_float2(c->x - acc[i][j].x, c->y - acc[i][j].y);
            else
                *c = acc[i][j];
        }
    }
}

static size_t gemm_smem() { return sizeof(float2) * LU_NB * (GEMM_BM + GEMM_PAD + GEMM_BN + GEMM_PAD); }

static sie_status cgemm(cudaStream_t st, int M, int N, int K, const float2* A, int64_t lda, const float2* B,
                        int64_t ldb, float2* C, int64_t ldc, int sub)
{
    if (M <= 0 || N <= 0) return SIE_OK;
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_cgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem());
    SIE_CUDA_TRY(attr);
    dim3 grid((N + GEMM_BN - 1) / GEMM_BN, (M + GEMM_BM - 1) / GEMM_BM);
    k_cgemm<<<grid, 256, gemm_smem(), st>>>(M, N, K, A, lda, B, ldb, C, ldc, sub);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// ------------------------------------------------------------------ triangular solves
// Block b's flag equals the solve's epoch once its 64 results are in memory.
// Thread 0 waits; a wait that exceeds SPIN_LIMIT polls sets *err = 1 and the
// CTA publishes its flag anyway (its result is then garbage, and the host
// reports SIE_ERR_TIMEOUT), so no CTA waits on one that gave up.
__device__ __forceinline__ bool wait_flag(const int* flags, int j, int epoch, int* err)
{
    int ok = 1;
    if (threadIdx.x == 0) {
        long long it = 0;
        const volatile int* f = flags + j;
        while (*f != epoch && ++it < SPIN_LIMIT) {
        }
        ok = (it < SPIN_LIMIT);
        if (!ok) atomicExch(err, 1);
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;  // barrier: block j's results are visible after it
}

__device__ __forceinline__ void publish(int* flags, int b, int epoch)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(flags + b, epoch);
}

// dir = 0: forward, L y = z (unit lower, blocks in increasing order);
// dir = 1: backward, U x = y (blocks in decreasing order).  256 threads:
// row r = tid / 4 of the block, quarter q = tid % 4 of each 64-column slice.
__global__ void __launch_bounds__(256) k_trsv(int n, int nblk, int dir, const float2* __restrict__ A, int64_t lda,
                                              const float2* __restrict__ invD, const float2* __restrict__ rhs,
                                              float2* out, int* flags, int epoch, int* counter, int* err)
{
    __shared__ int sticket;
    __shared__ float2 z[LU_NB];
    if (threadIdx.x == 0) sticket = atomicAdd(counter, 1);
    __syncthreads();
    const int t = sticket;
    const int b = dir == 0 ? t : nblk - 1 - t;
    const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
    const int row = b * LU_NB + r;
    float2 acc = make_float2(0.f, 0.f);
    bool good = true;
    for (int s = 0; s < t; s++) {
        const int jb = dir == 0 ? s : nblk - 1 - s;
        good = wait_flag(flags, jb, epoch, err) && good;
        if (row < n) {
            const int c0 = jb * LU_NB + q * 16;
            const float2* a = A + (int64_t)row * lda + c0;
#pragma unroll 4
            for (int c = 0; c < 16; c++) {
                if (c0 + c < n) {
                    float2 v = __ldcg(out + c0 + c);
                    acc = cfma(a[c], v, acc);
                }
            }
        }
    }
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
    if (q == 0) {
        float2 v = row < n ? rhs[row] : make_float2(0.f, 0.f);
        z[r] = make_float2(v.x - acc.x, v.y - acc.y);
    }
    __syncthreads();
    // out_b = invD_b z
    const float2* D = invD + ((int64_t)b * LU_NB + r) * LU_NB + q * 16;
    float2 s2 = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int c = 0; c < 16; c++) s2 = cfma(D[c], z[q * 16 + c], s2);
    s2.x += __shfl_xor_sync(0xffffffffu, s2.x, 1);
    s2.y += __shfl_xor_sync(0xffffffffu, s2.y, 1);
    s2.x += __shfl_xor_sync(0xffffffffu, s2.x, 2);
    s2.y += __shfl_xor_sync(0xffffffffu, s2.y, 2);
    if (q == 0 && row < n) __stcg(out + row, good ? s2 : make_float2(0.f, 0.f));
    publish(flags, b, epoch);
}

// Y = P: row i has its one in column perm[i] (row i of P A is row perm[i] of A)
__global__ void k_perm_matrix(int n, const int* __restrict__ perm, float2* __restrict__ Y)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    Y[idx] = make_float2(j == perm[i] ? 1.f : 0.f, 0.f);
}

// y = X b for the explicit inverse X (row-major): a warp per row, FP32
// products, the row sum in FP64; b complex128, converted on the fly
// x = X b for the explicit inverse X (complex64, n x n row-major); b first
// converted to complex64 once (k_c128_to_c64), so the inner loop holds no
// FP64 -> FP32 conversions (those run on the FP64 pipe).  One warp per GR
// consecutive rows: each complex64 pair of b (one 16-byte load) serves GR
// rows, so b is read n / GR times from L1/L2 instead of n times.  Lanes take
// 16-byte (two-entry) slices of the rows; FP32 products and per-lane sums,
// the warp sum in FP64.  Needs n even (16-byte aligned rows).
constexpr int GEMV_GR = 4;
__global__ void __launch_bounds__(256) k_cgemv_inv(int n, const float4* __restrict__ X, const float4* __restrict__ b,
                                                   double2* __restrict__ y)
{
    const int r0 = (blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * GEMV_GR;
    const int lane = threadIdx.x & 31;
    if (r0 >= n) return;
    const int h = n / 2;  // float4 per row
    float ar[GEMV_GR], ai[GEMV_GR];
#pragma unroll
    for (int g = 0; g < GEMV_GR; g++) ar[g] = ai[g] = 0.f;
    const float4* rows[GEMV_GR];
#pragma unroll
    for (int g = 0; g < GEMV_GR; g++) rows[g] = X + (int64_t)min(r0 + g, n - 1) * h;
    int c = lane;
    for (; c + 32 < h; c += 64) {
        float4 bv[2], a[2][GEMV_GR];
#pragma unroll
        for (int u = 0; u < 2; u++) bv[u] = __ldg(b + c + 32 * u);
#pragma unroll
        for (int u = 0; u < 2; u++)
#pragma unroll
            for (int g = 0; g < GEMV_GR; g++) a[u][g] = __ldg(rows[g] + c + 32 * u);
#pragma unroll
        for (int u = 0; u < 2; u++)
#pragma unroll
            for (int g = 0; g < GEMV_GR; g++) {
                const float4 m = a[u][g], v = bv[u];
                ar[g] = fmaf(m.x, v.x, fmaf(-m.y, v.y, fmaf(m.z, v.z, fmaf(-m.w, v.w, ar[g]))));
                ai[g] = fmaf(m.x, v.y, fmaf(m.y, v.x, fmaf(m.z, v.w, fmaf(m.w, v.z, ai[g]))));
            }
    }
    for (; c < h; c += 32) {
        const float4 v = __ldg(b + c);
#pragma unroll
        for (int g = 0; g < GEMV_GR; g++) {
            const float4 m = __ldg(rows[g] + c);
            ar[g] = fmaf(m.x, v.x, fmaf(-m.y, v.y, fmaf(m.z, v.z, fmaf(-m.w, v.w, ar[g]))));
            ai[g] = fmaf(m.x, v.y, fmaf(m.y, v.x, fmaf(m.z, v.w, fmaf(m.w, v.z, ai[g]))));
        }
    }
#pragma unroll
    for (int g = 0; g < GEMV_GR; g++) {
        double sr = ar[g], si = ai[g];
        for (int off = 16; off > 0; off >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, off);
            si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == 0 && r0 + g < n) y[r0 + g] = make_double2(sr, si);
    }
}

// odd n: one warp per row, complex64 b
__global__ void __launch_bounds__(256) k_cgemv_inv1(int n, const float2* __restrict__ X, const float2* __restrict__ b,
                                                    double2* __restrict__ y)
{
    const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float2* row = X + (int64_t)r * n;
    float ar = 0, ai = 0;
    for (int c = lane; c < n; c += 32) {
        const float2 a = __ldg(row + c), v = __ldg(b + c);
        ar = fmaf(a.x, v.x, fmaf(-a.y, v.y, ar));
        ai = fmaf(a.x, v.y, fmaf(a.y, v.x, ai));
    }
    double sr = ar, si = ai;
    for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    if (lane == 0) y[r] = make_double2(sr, si);
}

// X B for up to MULTI_R right-hand sides at once (the explicit inverse read
// once for all of them): B packed as R complex64 vectors of n (n even).  A CTA
// takes MR_ROWS rows (2 per warp) and walks the columns in chunks of
// MR_CHUNK entry pairs; each chunk of B (R x MR_CHUNK float4) is staged in
// shared memory and read by every warp, the matrix streams from HBM once.
// Within a chunk a lane takes 4 column steps at a time (8 loads of 16 bytes
// for its 2 rows), and the next 4 steps' loads are issued before the current
// ones are used, so about 16 loads per lane stay in flight.  FP32 products
// and per-lane sums, warp sums in FP64; out: pointers to the R complex128
// results.
constexpr int MULTI_R = 8;
constexpr int MR_WROWS = 2;
constexpr int MR_ROWS = 8 * MR_WROWS;
constexpr int MR_CHUNK = 512;
struct OutPtrs {
    double2* p[MULTI_R];
};
__global__ void __launch_bounds__(256, 2) k_cgemm_inv_multi(int n, int R, const float4* __restrict__ X,
                                                            const float4* __restrict__ B, OutPtrs out)
{
    extern __shared__ float4 Bs[];  // [MULTI_R][MR_CHUNK]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * MR_ROWS + warp * MR_WROWS;
    const int h = n / 2;
    float ar[MR_WROWS][MULTI_R], ai[MR_WROWS][MULTI_R];
#pragma unroll
    for (int g = 0; g < MR_WROWS; g++)
#pragma unroll
        for (int q = 0; q < MULTI_R; q++) ar[g][q] = ai[g][q] = 0.f;
    const float4* rows[MR_WROWS];
#pragma unroll
    for (int g = 0; g < MR_WROWS; g++) rows[g] = X + (int64_t)min(r0 + g, n - 1) * h;
    auto load = [&](float4 (&m)[4][MR_WROWS], int base, int cl, int c0) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int c = base + lane + 32 * u;
#pragma unroll
            for (int g = 0; g < MR_WROWS; g++)
                m[u][g] = c < cl ? __ldg(rows[g] + c0 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    for (int c0 = 0; c0 < h; c0 += MR_CHUNK) {
        const int cl = min(MR_CHUNK, h - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < MULTI_R * MR_CHUNK; i += blockDim.x) {
            const int q = i / MR_CHUNK, c = i % MR_CHUNK;
            Bs[q * MR_CHUNK + c] = (q < R && c < cl) ? B[(int64_t)q * h + c0 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float4 cur[4][MR_WROWS], nxt[4][MR_WROWS];
        load(cur, 0, cl, c0);
        __syncthreads();
        for (int base = 0; base < MR_CHUNK; base += 128) {
            if (base + 128 < MR_CHUNK) load(nxt, base + 128, cl, c0);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int c = base + lane + 32 * u;
#pragma unroll
                for (int q = 0; q < MULTI_R; q++) {
                    const float4 v = Bs[q * MR_CHUNK + c];
#pragma unroll
                    for (int g = 0; g < MR_WROWS; g++) {
                        const float4 mm = cur[u][g];
                        ar[g][q] = fmaf(mm.x, v.x, fmaf(-mm.y, v.y, fmaf(mm.z, v.z, fmaf(-mm.w, v.w, ar[g][q]))));
                        ai[g][q] = fmaf(mm.x, v.y, fmaf(mm.y, v.x, fmaf(mm.z, v.w, fmaf(mm.w, v.z, ai[g][q]))));
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int g = 0; g < MR_WROWS; g++) cur[u][g] = nxt[u][g];
        }
    }
#pragma unroll
    for (int g = 0; g < MR_WROWS; g++)
#pragma unroll
        for (int q = 0; q < MULTI_R; q++) {
            double sr = ar[g][q], si = ai[g][q];
            for (int off = 16; off > 0; off >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, off);
                si += __shfl_xor_sync(0xffffffffu, si, off);
            }
            if (lane == 0 && q < R && r0 + g < n) out.p[q][r0 + g] = make_double2(sr, si);
        }
}

__global__ void k_c128_to_c64(int n, const double2* __restrict__ b, float2* __restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = make_float2((float)b[i].x, (float)b[i].y);
}

__global__ void k_perm_to_f32(int n, const int* __restrict__ perm, const double2* __restrict__ b,
                              float2* __restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double2 v = b[perm[i]];
        y[i] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void k_f32_to_f64(int n, const float2* __restrict__ a, double2* __restrict__ b)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_double2(a[i].x, a[i].y);
}

// ------------------------------------------------------------------ host side
void DenseLU::release()
{
    for (void* p : {(void*)A, (void*)Xinv, (void*)invL, (void*)invU, (void*)ipiv, (void*)perm, (void*)flags,
                    (void*)counter, (void*)err, (void*)y0, (void*)y1, (void*)prow, (void*)bpack})
        if (p) cudaFree(p);
    A = Xinv = invL = invU = y0 = y1 = prow = bpack = nullptr;
    ipiv = perm = flags = counter = err = nullptr;
    n = nblk = 0;
}

sie_status DenseLU::alloc(int n_)
{
    release();
    n = n_;
    nblk = (n + LU_NB - 1) / LU_NB;
    SIE_CUDA_TRY(cudaMalloc((void**)&A, sizeof(float2) * (size_t)n * n));
    SIE_CUDA_TRY(cudaMalloc((void**)&invL, sizeof(float2) * (size_t)nblk * LU_NB * LU_NB));
    SIE_CUDA_TRY(cudaMalloc((void**)&invU, sizeof(float2) * (size_t)nblk * LU_NB * LU_NB));
    SIE_CUDA_TRY(cudaMalloc((void**)&ipiv, sizeof(int) * n));
    SIE_CUDA_TRY(cudaMalloc((void**)&perm, sizeof(int) * n));
    SIE_CUDA_TRY(cudaMalloc((void**)&flags, sizeof(int) * 2 * nblk));
    SIE_CUDA_TRY(cudaMalloc((void**)&counter, sizeof(int) * 2));
    SIE_CUDA_TRY(cudaMalloc((void**)&err, sizeof(int)));
    SIE_CUDA_TRY(cudaMalloc((void**)&y0, sizeof(float2) * n));
    SIE_CUDA_TRY(cudaMalloc((void**)&y1, sizeof(float2) * n));
    SIE_CUDA_TRY(cudaMalloc((void**)&prow, sizeof(float2) * LU_NB));
    SIE_CUDA_TRY(cudaMemset(flags, 0, sizeof(int) * 2 * nblk));
    SIE_CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
    epoch = 0;
    return SIE_OK;
}

// Factorise the matrix in A (n x n, row-major, complex64) in place.
sie_status DenseLU::factor(cudaStream_t st)
{
    for (int k = 0; k < n; k += LU_NB) {
        const int kb = std::min(LU_NB, n - k);
        for (int j = 0; j < kb; j++) {
            k_panel_pivot<<<1, 1024, 0, st>>>(n, k, kb, j, A, n, ipiv, prow, err);
            const int rows = n - (k + j) - 1;
            if (rows > 0) k_panel_update<<<(rows + 255) / 256, 256, 0, st>>>(n, k, kb, j, A, n, prow);
        }
        if (n > kb) k_laswp<<<(n - kb + 255) / 256, 256, 0, st>>>(n, k, kb, A, n, ipiv);
        k_tri_inv<<<1, LU_NB, 0, st>>>(n, k / LU_NB, A, n, invL, invU);
        SIE_CUDA_TRY(cudaGetLastError());
        const int rest = n - k - kb;
        if (rest > 0) {
            // U12 = L11^-1 A12 (in place: one row tile), A22 -= L21 U12
            float2* A12 = A + (int64_t)k * n + k + kb;
            SIE_TRY(cgemm(st, kb, rest, kb, invL + (int64_t)(k / LU_NB) * LU_NB * LU_NB, LU_NB, A12, n, A12, n, 0));
            SIE_TRY(cgemm(st, rest, rest, kb, A + (int64_t)(k + kb) * n + k, n, A12, n, A + (int64_t)(k + kb) * n + k + kb,
                          n, 1));
        }
    }
    // the row permutation as a gather: row i of P A is row perm[i] of A
    std::vector<int> piv(n), pm(n);
    SIE_CUDA_TRY(cudaMemcpyAsync(piv.data(), ipiv, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    int herr = 0;
    SIE_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) {
        set_error("dense LU of the constraint triangle system: zero pivot (singular matrix)");
        return SIE_ERR_ARG;
    }
    for (int i = 0; i < n; i++) pm[i] = i;
    for (int i = 0; i < n; i++) std::swap(pm[i], pm[piv[i]]);
    SIE_CUDA_TRY(cudaMemcpyAsync(perm, pm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    return SIE_OK;
}

// Replace the factors by the explicit inverse A^-1 = U^-1 L^-1 P (complex64):
// Y = P, then L Y = P and U X = Y by blocked right-looking substitution, each
// block step an in-place product with the inverted diagonal block and a GEMM
// update of the remaining block rows.  Afterwards every solve is one
// matrix-vector product (no dependency chain between blocks).
sie_status DenseLU::invert(cudaStream_t st)
{
    float2* X = nullptr;
    SIE_CUDA_TRY(cudaMalloc((void**)&X, sizeof(float2) * (size_t)n * n));
    const int64_t nn = (int64_t)n * n;
    k_perm_matrix<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, perm, X);
    SIE_CUDA_TRY(cudaGetLastError());
    for (int b = 0; b < nblk; b++) {  // L Y = P
        const int k = b * LU_NB, kb = std::min(LU_NB, n - k);
        float2* Yb = X + (int64_t)k * n;
        SIE_TRY(cgemm(st, kb, n, kb, invL + (int64_t)b * LU_NB * LU_NB, LU_NB, Yb, n, Yb, n, 0));
        const int below = n - k - kb;
        if (below > 0) SIE_TRY(cgemm(st, below, n, kb, A + (int64_t)(k + kb) * n + k, n, Yb, n, Yb + (int64_t)kb * n, n, 1));
    }
    for (int b = nblk - 1; b >= 0; b--) {  // U X = Y
        const int k = b * LU_NB, kb = std::min(LU_NB, n - k);
        float2* Xb = X + (int64_t)k * n;
        SIE_TRY(cgemm(st, kb, n, kb, invU + (int64_t)b * LU_NB * LU_NB, LU_NB, Xb, n, Xb, n, 0));
        if (k > 0) SIE_TRY(cgemm(st, k, n, kb, A + k, n, Xb, n, X, n, 1));
    }
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(A);
    A = nullptr;
    Xinv = X;
    return SIE_OK;
}

// x = A^-1 b (FP64 in and out, complex64 inside)
sie_status DenseLU::solve(cudaStream_t st, const double2* b, double2* x)
{
    if (Xinv) {
        k_c128_to_c64<<<(n + 255) / 256, 256, 0, st>>>(n, b, y0);
        if (n % 2 == 0) {
            const int warps = (n + GEMV_GR - 1) / GEMV_GR;
            k_cgemv_inv<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(n, reinterpret_cast<const float4*>(Xinv),
                                                                    reinterpret_cast<const float4*>(y0), x);
        } else {
            k_cgemv_inv1<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, Xinv, y0, x);
        }
        SIE_CUDA_TRY(cudaGetLastError());
        return SIE_OK;
    }
    epoch++;
    SIE_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int) * 2, st));
    k_perm_to_f32<<<(n + 255) / 256, 256, 0, st>>>(n, perm, b, y0);
    k_trsv<<<nblk, 256, 0, st>>>(n, nblk, 0, A, n, invL, y0, y1, flags, epoch, counter, err);
    k_trsv<<<nblk, 256, 0, st>>>(n, nblk, 1, A, n, invU, y1, y0, flags + nblk, epoch, counter + 1, err);
    k_f32_to_f64<<<(n + 255) / 256, 256, 0, st>>>(n, y0, x);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// x_q = A^-1 b_q for R right-hand sides (R <= MULTI_R); with the explicit
// inverse and n even one pass over it for all of them, else one solve each
sie_status DenseLU::solve_multi(cudaStream_t st, int R, const double2* const* b, double2* const* x)
{
    if (R < 1 || R > MULTI_R) {
        set_error("DenseLU::solve_multi: 1 to 8 right-hand sides");
        return SIE_ERR_ARG;
    }
    if (!Xinv || n % 2 != 0 || R == 1) {
        for (int q = 0; q < R; q++) SIE_TRY(solve(st, b[q], x[q]));
        return SIE_OK;
    }
    if (!bpack) SIE_CUDA_TRY(cudaMalloc((void**)&bpack, sizeof(float2) * (size_t)MULTI_R * n));
    OutPtrs o{};
    for (int q = 0; q < R; q++) {
        k_c128_to_c64<<<(n + 255) / 256, 256, 0, st>>>(n, b[q], bpack + (size_t)q * n);
        o.p[q] = x[q];
    }
    const size_t smem = sizeof(float4) * MULTI_R * MR_CHUNK;  // 64 KB
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_cgemm_inv_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    SIE_CUDA_TRY(attr);
    k_cgemm_inv_multi<<<(unsigned)((n + MR_ROWS - 1) / MR_ROWS), 256, smem, st>>>(
        n, R, reinterpret_cast<const float4*>(Xinv), reinterpret_cast<const float4*>(bpack), o);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

// 0, or SIE_ERR_TIMEOUT when a triangular-solve wait ran out (synchronises)
sie_status DenseLU::check(cudaStream_t st)
{
    if (!err) return SIE_OK;
    int h = 0;
    SIE_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    if (h == 1) {
        set_error("dense LU triangular solve: a wait for a preceding block ran out");
        return SIE_ERR_TIMEOUT;
    }
    return SIE_OK;
}

sie_status dense_lu_assemble(cudaStream_t st, DenseLU& f, const sie_op* op, const AimOp& a, double2 kappa)
{
    const DevMesh& M = op->mesh->d;
    k_assemble_T<<<M.nt, 256, 0, st>>>(M.nt, M, op->elen, a.dLA, a.tri_row_ptr, a.tri_col, a.valLphiNR, kappa, f.A,
                                       f.n);
    SIE_CUDA_TRY(cudaGetLastError());
    return SIE_OK;
}

}  // namespace sie

__global__ void k_f64_to_f32(int64_t n, const double2* __restrict__ a, float2* __restrict__ b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

extern "C" sie_status sie_dense_solve(int device, int n, int nrhs, const double* A, const double* b, double* x,
                                      int flags)
{
    using namespace sie;
    if (n < 1 || nrhs < 1 || !A || !b || !x) {
        set_error("sie_dense_solve: invalid argument");
        return SIE_ERR_ARG;
    }
    SIE_CUDA_TRY(cudaSetDevice(device));
    cudaStream_t st = nullptr;
    DenseLU f;
    double2 *dA = nullptr, *db = nullptr, *dx = nullptr;
    sie_status s = SIE_OK;
    auto done = [&](sie_status r) {
        cudaStreamSynchronize(st);
        f.release();
        for (void* p : {(void*)dA, (void*)db, (void*)dx})
            if (p) cudaFree(p);
        return r;
    };
    if ((s = f.alloc(n)) != SIE_OK) return done(s);
    const size_t nn = (size_t)n * n, nb = (size_t)n * nrhs;
    if (cudaMalloc((void**)&dA, sizeof(double2) * nn) != cudaSuccess ||
        cudaMalloc((void**)&db, sizeof(double2) * nb) != cudaSuccess ||
        cudaMalloc((void**)&dx, sizeof(double2) * nb) != cudaSuccess) {
        set_error("sie_dense_solve: device allocation failed");
        return done(SIE_ERR_OOM);
    }
    if (cudaMemcpy(dA, A, sizeof(double2) * nn, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(db, b, sizeof(double2) * nb, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("sie_dense_solve: copy failed");
        return done(SIE_ERR_CUDA);
    }
    k_f64_to_f32<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>((int64_t)nn, dA, f.A);
    if ((s = f.factor(st)) != SIE_OK) return done(s);
    if ((flags & 1) && (s = f.invert(st)) != SIE_OK) return done(s);
    for (int r0 = 0; r0 < nrhs; r0 += MULTI_R) {
        const int R = std::min(MULTI_R, nrhs - r0);
        const double2* bq[MULTI_R];
        double2* xq[MULTI_R];
        for (int q = 0; q < R; q++) {
            bq[q] = db + (size_t)(r0 + q) * n;
            xq[q] = dx + (size_t)(r0 + q) * n;
        }
        if ((s = f.solve_multi(st, R, bq, xq)) != SIE_OK) return done(s);
    }
    if ((s = f.check(st)) != SIE_OK) return done(s);
    if (cudaMemcpy(x, dx, sizeof(double2) * nb, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("sie_dense_solve: copy failed");
        return done(SIE_ERR_CUDA);
    }
    return done(SIE_OK);
}
