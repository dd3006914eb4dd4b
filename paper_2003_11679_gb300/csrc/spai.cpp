// Sparse approximate inverse of a near-region matrix, used as the right
// preconditioner of the nested interior solve when the interior operator is
// near-region only.  The paper's preconditioner (Eq. nest2pc) is the near-region
// matrix L_i,NR itself, applied through a sparse LU factorisation; when the
// skin depth is below the near-region size L_i,NR = L_i and that makes the
// nested solve direct.  Triangular solves serialise on a GPU, so here the
// inverse is approximated instead: M has the sparsity pattern of A and column j
// minimises ||A m_j - e_j||_2, i.e. M minimises ||A M - I||_F column by column.
// For the strongly diagonally dominant L_i of a good conductor (a scaled
// Gram-like matrix) this brings the nested solve down to a few iterations, each
// one CSR product more.
//
// Host FP64: the normal equations (A_J^H A_J) m = A_J^H e_j of each column are
// solved by Cholesky; columns are independent and split over threads.  The
// near-region pattern is structurally symmetric (pair lists hold both orders).
#include <cuda_runtime.h>

#include <algorithm>
#include <complex>
#include <thread>
#include <vector>

#include "internal.h"

namespace sie {

using cd = std::complex<double>;

// Hermitian positive definite solve G m = b (n x n, column-major, overwritten
// by its Cholesky factor); false if a pivot is not positive.
static bool chol_solve(int n, std::vector<cd>& G, std::vector<cd>& b)
{
    for (int j = 0; j < n; j++) {
        double d = G[j + (size_t)j * n].real();
        for (int k = 0; k < j; k++) d -= std::norm(G[j + (size_t)k * n]);
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        G[j + (size_t)j * n] = d;
        for (int i = j + 1; i < n; i++) {
            cd s = G[i + (size_t)j * n];
            for (int k = 0; k < j; k++) s -= G[i + (size_t)k * n] * std::conj(G[j + (size_t)k * n]);
            G[i + (size_t)j * n] = s / d;
        }
    }
    // forward: R y = b with R lower (R R^H = G)
    for (int i = 0; i < n; i++) {
        cd s = b[i];
        for (int k = 0; k < i; k++) s -= G[i + (size_t)k * n] * b[k];
        b[i] = s / G[i + (size_t)i * n].real();
    }
    // backward: R^H m = y
    for (int i = n - 1; i >= 0; i--) {
        cd s = b[i];
        for (int k = i + 1; k < n; k++) s -= std::conj(G[k + (size_t)i * n]) * b[k];
        b[i] = s / G[i + (size_t)i * n].real();
    }
    return true;
}

// M (values on the pattern of P) from the CSR values val; returns the number
// of columns that fell back to the inverse diagonal, or -1 if the pattern is
// not structurally symmetric
int64_t spai_host(const CsrPattern& P, const std::complex<double>* val, std::complex<double>* M)
{
    const int64_t n = (int64_t)P.row_ptr.size() - 1;
    const int64_t nnz = (int64_t)P.col.size();
    const std::vector<int64_t>& rp = P.row_ptr;
    const std::vector<int32_t>& col = P.col;
    // tpos[e] for e = (i, k): position of (k, i)
    std::vector<int64_t> tpos(nnz);
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
            const int32_t k = col[e];
            auto b = col.begin() + rp[k], f = col.begin() + rp[k + 1];
            auto it = std::lower_bound(b, f, (int32_t)i);
            if (it == f || *it != (int32_t)i) return -1;
            tpos[e] = it - col.begin();
        }
    unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<int> bad(nth, 0);
    auto work = [&](unsigned t) {
        std::vector<int32_t> loc(n, -1), I;
        std::vector<cd> A, G, b;
        for (int64_t j = t; j < n; j += nth) {
            const int64_t j0 = rp[j];
            const int nJ = (int)(rp[j + 1] - j0);
            I.clear();
            // rows reached by the columns k in J = pattern of row j
            for (int c = 0; c < nJ; c++) {
                const int32_t k = col[j0 + c];
                for (int64_t e = rp[k]; e < rp[k + 1]; e++)
                    if (loc[col[e]] < 0) {
                        loc[col[e]] = (int32_t)I.size();
                        I.push_back(col[e]);
                    }
            }
            const int nI = (int)I.size();
            A.assign((size_t)nI * nJ, cd(0.0, 0.0));
            for (int c = 0; c < nJ; c++) {
                const int32_t k = col[j0 + c];
                // column k of the matrix: entries (i, k) for i in row k's pattern
                for (int64_t e = rp[k]; e < rp[k + 1]; e++) A[loc[col[e]] + (size_t)c * nI] = val[tpos[e]];
            }
            G.assign((size_t)nJ * nJ, cd(0.0, 0.0));
            for (int c2 = 0; c2 < nJ; c2++)
                for (int c1 = c2; c1 < nJ; c1++) {
                    cd s(0.0, 0.0);
                    for (int r = 0; r < nI; r++) s += std::conj(A[r + (size_t)c1 * nI]) * A[r + (size_t)c2 * nI];
                    G[c1 + (size_t)c2 * nJ] = s;  // lower triangle: G[c1, c2] = a_c1^H a_c2
                    G[c2 + (size_t)c1 * nJ] = std::conj(s);
                }
            b.assign(nJ, cd(0.0, 0.0));
            const int lj = loc[j];
            for (int c = 0; c < nJ; c++) b[c] = std::conj(A[lj + (size_t)c * nI]);
            if (!chol_solve(nJ, G, b)) {
                // fall back to the diagonal for this column
                bad[t]++;
                for (int c = 0; c < nJ; c++) b[c] = col[j0 + c] == j ? 1.0 / val[j0 + c] : cd(0.0, 0.0);
            }
            // M[k, j] = m_j[c] for k = J[c], stored at (k, j) = tpos of (j, k)
            for (int c = 0; c < nJ; c++) M[tpos[j0 + c]] = b[c];
            for (int32_t i : I) loc[i] = -1;
        }
    };
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nth; t++) th.emplace_back(work, t);
    for (auto& x : th) x.join();
    int64_t nbad = 0;
    for (int v : bad) nbad += v;
    return nbad;
}

sie_status spai_build(cudaStream_t st, const CsrPattern& P, const double2* dval, double2** dM)
{
    const int64_t nnz = (int64_t)P.col.size();
    std::vector<cd> val(nnz), M(nnz);
    SIE_CUDA_TRY(cudaMemcpyAsync(val.data(), dval, sizeof(double2) * nnz, cudaMemcpyDeviceToHost, st));
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    if (spai_host(P, val.data(), M.data()) < 0) {
        set_error("spai_build: near-region pattern is not structurally symmetric");
        return SIE_ERR_STATE;
    }
    double2* d = nullptr;
    SIE_CUDA_TRY(cudaMallocAsync((void**)&d, sizeof(double2) * std::max<int64_t>(nnz, 1), st));
    SIE_CUDA_TRY(cudaMemcpyAsync(d, M.data(), sizeof(double2) * nnz, cudaMemcpyHostToDevice, st));
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    *dM = d;
    return SIE_OK;
}

}  // namespace sie
