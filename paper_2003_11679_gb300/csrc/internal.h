// Internal declarations of the sm_103a AIM/SIE library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sie.h"

namespace sie {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
struct Status {
    sie_status code = SIE_OK;
};
#define SIE_CUDA_TRY(call)                                                                       \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            ::sie::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                 \
            return e_ == cudaErrorMemoryAllocation ? SIE_ERR_OOM : SIE_ERR_CUDA;                  \
        }                                                                                         \
    } while (0)
#define SIE_TRY(call)                      \
    do {                                   \
        sie_status s_ = (call);            \
        if (s_ != SIE_OK) return s_;       \
    } while (0)

// ------------------------------------------------------------------ geometry
// Host-side mesh with its RWG table.  Slot i of triangle t is the edge
// opposite local vertex i; sign +1 on T+, -1 on T-; the free vertex of slot i
// is vertex i of the triangle.
struct HostMesh {
    int64_t nv = 0, nt = 0, ne = 0;
    std::vector<double> V;           // nv*3
    std::vector<int32_t> T;          // nt*3
    std::vector<int32_t> tri_edge;   // nt*3
    std::vector<int8_t> tri_sign;    // nt*3
    std::vector<double> edge_len;    // ne
    std::vector<int32_t> edge_tri;   // ne*2 (T+, T-)
    std::vector<int8_t> edge_slot;   // ne*2 slot of the edge in T+, T-
    std::vector<double> area;        // nt
    std::vector<double> cen;         // nt*3
    std::vector<double> nrm;         // nt*3 unit normal
    std::vector<double> coef;        // nt*3 = s l / (2A)
    std::vector<double> q;           // nt*9 = c_t - p (slot-major, then xyz)
    std::vector<double> rad;         // nt farthest vertex from the centroid
    std::vector<int32_t> obj;        // nt object index (0 for a one-object mesh)
    int nobj = 1;
    double mean_edge = 0;
};
sie_status build_mesh(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, HostMesh& m);

struct GridDesc {
    double o[3];
    double h;
    int N[3];     // physical nodes per axis
    int n[3];     // FFT lengths (powers of two >= 2N-1)
    int M;        // Lagrange order
    int Rnear;    // near radius (nodes)
};
sie_status make_grid(const HostMesh& m, const sie_params& p, GridDesc& g);
void stencil_base(const HostMesh& m, const GridDesc& g, std::vector<int32_t>& base);

// near triangle pairs, sorted by (t, s): AIM rule (Chebyshev distance of the
// stencil centres <= Rnear) or interior cutoff rule (touching, or gap <= cutoff)
void near_pairs_grid(const HostMesh& m, const GridDesc& g, const std::vector<int32_t>& base,
                     std::vector<int32_t>& pairs);
void near_pairs_cutoff(const HostMesh& m, double cutoff, std::vector<int32_t>& pairs);
// the same with one cutoff per object; pairs are kept only inside an object
void near_pairs_cutoff_objects(const HostMesh& m, const std::vector<double>& cutoff, std::vector<int32_t>& pairs);

// CSR pattern over edges from a sorted triangle-pair list
struct CsrPattern {
    std::vector<int64_t> row_ptr;  // ne+1
    std::vector<int32_t> col;      // nnz
};
void edge_csr_pattern(const HostMesh& m, const std::vector<int32_t>& pairs, CsrPattern& csr);

// Gauss-Legendre on [0, 1] by Newton iteration on the Legendre recurrence
void gauss_legendre01(int n, double* x, double* w);

// sparse approximate inverse (pattern of P) of the device CSR values dval;
// result allocated on the device in *dM
sie_status spai_build(cudaStream_t st, const CsrPattern& P, const double2* dval, double2** dM);

// ------------------------------------------------------------------ device data
struct DevMesh {
    int nt = 0, ne = 0, nv = 0;
    double* V = nullptr;        // nv*3
    int32_t* T = nullptr;       // nt*3
    int32_t* tri_edge = nullptr;
    double* coef = nullptr;     // nt*3
    double* q = nullptr;        // nt*9
    double* cen = nullptr;      // nt*3
    double* area = nullptr;     // nt
    double* rad = nullptr;      // nt
    int32_t* edge_tri = nullptr;   // ne*2
    int8_t* edge_slot = nullptr;   // ne*2
    int32_t* obj = nullptr;        // nt object index
};

// quadrature description handed to the near-field kernel
struct QuadDev {
    double x[7][32], w[7][32];  // far, out, ang, rad, olam, omu, emu
    int n[7];
    int npan, opan, emupan;
    double ratio, cf, kres, alen, oratio;
};
enum { QR_FAR = 0, QR_OUT, QR_ANG, QR_RAD, QR_OLAM, QR_OMU, QR_EMU };
void make_quad(const sie_params& p, QuadDev& q);

// Dense complex64 LU (partial pivoting) of a triangle system, on the device
struct DenseLU {
    int n = 0, nblk = 0, epoch = 0;
    float2* A = nullptr;      // n x n row-major: the matrix, then its L and U factors
    float2* Xinv = nullptr;   // explicit inverse (after invert(); A is freed then)
    float2* invL = nullptr;   // inverses of the unit-lower diagonal blocks (nblk x 64 x 64)
    float2* invU = nullptr;   // inverses of the upper diagonal blocks
    int* ipiv = nullptr;      // row swaps of the factorisation
    int* perm = nullptr;      // the resulting row permutation as a gather
    int* flags = nullptr;     // 2 nblk: per-block completion flags of the two triangular solves
    int* counter = nullptr;   // 2: ticket counters of the two triangular solves
    int* err = nullptr;       // 1: a triangular-solve wait ran out; 2: zero pivot
    float2 *y0 = nullptr, *y1 = nullptr, *prow = nullptr;
    float2* bpack = nullptr;  // up to 8 right-hand sides in complex64 (solve_multi)
    sie_status alloc(int n_);
    void release();
    sie_status factor(cudaStream_t st);
    sie_status invert(cudaStream_t st);
    sie_status solve(cudaStream_t st, const double2* b, double2* x);
    sie_status solve_multi(cudaStream_t st, int R, const double2* const* b, double2* const* x);
    sie_status check(cudaStream_t st);
};

// One operator (one medium, one grid or near only)
struct AimOp {
    double kr = 0, ki = 0;          // wavenumber k = kr + j ki
    bool has_grid = true;
    GridDesc g{};
    double2* spec = nullptr;        // 4 spectra (G, dG/dx, dG/dy, dG/dz), each n^3, scaled 1/n^3
    float2* spec32 = nullptr;       // complex64 copy for the mixed path
    int64_t npairs = 0;
    int32_t* pairs = nullptr;       // device (t,s)
    std::vector<int32_t> hpairs;
    CsrPattern csr;
    int64_t nnz = 0;
    int64_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    double2* valL = nullptr;        // near-corrected L
    double2* valK = nullptr;        // near-corrected K
    double2* valLA = nullptr;       // near-corrected LA (vector potential part)
    double2* dLA = nullptr;         // exact diagonal of LA
    double2* dL = nullptr;          // exact diagonal of L
    // triangle CSR of the near-corrected Lphi (pairs in (t, s) order)
    std::vector<int64_t> tri_row_ptr_h;
    std::vector<int32_t> tri_col_h;
    int64_t* tri_row_ptr = nullptr;
    int32_t* tri_col = nullptr;
    double2* valLphi = nullptr;
    double2* valLphiNR = nullptr;   // exact near Lphi (constraint preconditioner)
    double2* valM = nullptr;        // sparse approximate inverse of valL (near-only interiors)
    // complex64 copies of the exterior near values for the mixed-precision product
    float4* valLK32 = nullptr;      // (LA, K) of each stored entry, interleaved
    float2* valLphi32 = nullptr;
    // dense LU of the constraint triangle system (null: iterative constraint solve)
    DenseLU* lu = nullptr;
    // several-object near-region-only interior: per-object k and 1/k^2 (device)
    double2* obj_k = nullptr;
    double2* obj_ik2 = nullptr;
};

struct Workspace {
    size_t grid_elems = 0;          // n^3
    double2* bufs = nullptr;        // 4 padded grids (n^3 each)
    double2* src = nullptr;         // 4 compact grids (N^3 each)
};

}  // namespace sie

namespace sie {
// CUDA-event stage timers on the context's stream (sie_profile_enable)
struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};
struct Prof {
    bool on = false;
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int64_t> count;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> pool;
};
}  // namespace sie

struct sie_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    sie::Prof prof;
};

namespace sie {
// scoped stage timer: records events only while profiling is enabled
struct Stage {
    sie_ctx* c;
    int id = -1;
    cudaEvent_t b{};
    Stage(sie_ctx* ctx, const char* name);
    ~Stage();
};
}  // namespace sie

struct sie_mesh {
    sie_ctx* ctx = nullptr;
    sie::HostMesh h;
    sie::DevMesh d;
    struct Material {
        bool set = false;
        double eps_r = 1, mu_r = 1, sigma = 0;
    };
    std::vector<Material> mat;       // per object
};

namespace sie {
// Krylov workspace of one restarted FGMRES (basis V, preconditioned basis Z)
struct KrylovWork {
    int64_t n = 0;
    int m = 0;
    double2 *V = nullptr, *Z = nullptr, *w = nullptr, *h = nullptr, *r = nullptr, *part = nullptr;
    double2* cgsp = nullptr;        // per-chunk partial sums of the fused Gram-Schmidt passes
    double2* dv = nullptr;          // device-controlled cycle: v_j and z_j (2 n)
    int* dj = nullptr;              // device-controlled cycle: iteration index, iterations done
    double2* Hd = nullptr;          // Hessenberg, rotations, g, y (device)
    double* sc = nullptr;           // |b|, beta, per-iteration relative residuals (device)
    double* resid_h = nullptr;      // pinned copies of the residuals
    std::vector<cudaEvent_t> ev;    // one per iteration: residual copy done
    sie_status alloc(cudaStream_t st, int64_t n_, int m_);
    void release(cudaStream_t st);
};
// Krylov workspace of a panel solve: R right-hand sides whose vectors sit side
// by side (basis V[j][q][n], Z[j][q][n]); one launch per Gram-Schmidt step
// serves all of them (gridDim.y = R)
struct PanelWork {
    int64_t n = 0;
    int m = 0, R = 0;
    double2 *V = nullptr, *Z = nullptr, *W = nullptr, *Rv = nullptr;  // bases, A z panel, residual panel
    double2 *P = nullptr, *h = nullptr, *Hd = nullptr, *part = nullptr, *wd = nullptr;
    double* sc = nullptr;     // per right-hand side: |b|, beta, residuals
    double* res = nullptr;    // residual of iteration j, right-hand side q at [j R + q]
    double* res_h = nullptr;  // pinned copy of res
    std::vector<cudaEvent_t> ev;
    sie_status alloc(cudaStream_t st, int64_t n_, int m_, int R_);
    void release(cudaStream_t st);
};
}  // namespace sie

struct sie_op {
    sie_mesh* mesh = nullptr;
    sie_params p{};
    double freq = 0, eps_r = 1, mu_r = 1, sigma = 0;
    double k0 = 0;
    sie::AimOp ext, inn;
    int32_t* base = nullptr;        // stencil base (nt*3), shared by ext and inner grids
    double* W = nullptr;            // weights nt * S * 4
    float* W32 = nullptr;           // complex64 grid path copy of W
    sie::Workspace ws;
    double2* xtmp = nullptr;        // scratch vectors (ne * 4)
    double build_ms[4] = {0, 0, 0, 0};  // weights+spectra, exterior near, interior near, host lists
    // system operator (Eq. sys)
    int64_t* ix_row_ptr = nullptr;  // Ix as edge CSR (real values stored as double2)
    int64_t ix_nnz = 0;
    int32_t* ix_col = nullptr;
    double2* ix_val = nullptr;
    double* elen = nullptr;         // edge lengths
    double2* sys_E = nullptr;       // E' = Z' H (ne)
    double2* sys_tmp = nullptr;     // ne + 2 nt scratch
    double2* sys_vec = nullptr;     // 4 (ne + nt) scratch for host-pointer calls
    float4* pk_he = nullptr;        // mixed near product: complex64 (H, E) side by side (ne)
    float2* pk_sig = nullptr;       // mixed near product: complex64 triangle charges (nt)
    sie::KrylovWork kin, kout, kcs_in, kcs_out;
    sie::KrylovWork kmulti[8];      // lockstep solves: one Krylov basis per right-hand side
    sie::KrylovWork kcs_multi[8];   // ... and per triangle system of their constraint preconditioner
    sie::PanelWork kzp;             // lockstep block products: the nested interior solves of the block
    double2* zp = nullptr;          // block products: H, E, rhs and scratch panels (4 x 8 ne)
    double2* mscr = nullptr;        // lockstep solves: per right-hand side scratch (8 blocks)
    double2* ir_multi = nullptr;    // lockstep refinement: residuals, corrections, products (3 x 8 (ne + nt))
    double2* mvec = nullptr;        // lockstep solves from host buffers: 2 x 8 (ne + nt)
    double2 *cs_e = nullptr, *cs_t = nullptr, *pc_e = nullptr, *pc_t = nullptr;  // preconditioner scratch
    // last solve: outer iters, relres; max nested iters, relres; max constraint iters, relres
    double stats[6] = {0, 0, 0, 0, 0, 0};
    // CUDA graph of the system product (near-only interior, profiling off): the
    // nested solve is a device-controlled while loop inside the graph
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // one per precision (SIE_FP64, SIE_MIXED)
    bool gfailed = false;           // capture or instantiation failed: stream path only
    bool capturing = false;         // apply_Z emits the device-controlled nested solve
    cudaStream_t gs[2] = {nullptr, nullptr};  // capture streams: graph, while-loop body
    double2* g_io = nullptr;        // graph input x and output y, 2 (ne + nt)
    double* gstat = nullptr;        // device: max nested iterations and residual of graph runs
    size_t gnodes[2] = {0, 0};      // nodes of the last captured graph: outside the loop, loop body
    double2* ir_buf = nullptr;      // iterative refinement: residual, correction, product (3 (ne + nt))
    double q_w = 0.0;               // charge-row weight of the GMRES residual norm (0: not yet computed)
    double2* bal = nullptr;         // weighted right-hand side and preconditioner input (2 (ne + nt))
    double lu_ms = 0;               // wall time of the dense constraint-preconditioner factorisations
    // surface impedance boundary condition (interior_model = SIE_SIBC): RWG Gram
    // matrix as edge CSR, its diagonal, and eta_i / eta0
    int64_t* gr_row_ptr = nullptr;
    int64_t gr_nnz = 0;
    int32_t* gr_col = nullptr;
    double2* gr_val = nullptr;
    double2* gr_diag = nullptr;
    double eta_re = 0, eta_im = 0;
    // projection of the system product as a gather: touched grid nodes, CSR
    // of their stencil entries (t * S + u), per-triangle coefficients
    int64_t pm_nnode = 0;
    int64_t *pm_node = nullptr, *pm_ptr = nullptr;
    int32_t* pm_ent = nullptr;
    double2* pm_tc = nullptr;       // 9 per triangle (FP64; the complex64 path uses its first half)
    // multi-right-hand-side block workspace (allocated on first use)
    double2 *bws_bufs = nullptr, *bws_src = nullptr, *bws_vec = nullptr;
    // several objects: per-edge factor of the interior impedance, -1/(j k0 eps_r + sigma eta0)
    // of the edge's object (GIBC) or eta_i/eta0 (SIBC); null for one object
    double2* edge_zf = nullptr;
};

// ------------------------------------------------------------------ launchers (aim.cu, near.cu)
namespace sie {
sie_status dev_upload_mesh(sie_mesh* m);
sie_status dev_free_mesh(sie_mesh* m);
sie_status aim_weights(sie_op* op);
sie_status aim_spectra(sie_op* op, AimOp& a);
sie_status near_build(sie_op* op, AimOp& a, const QuadDev& q);
sie_status aim_apply(sie_op* op, AimOp& a, int which_LK, const double2* x, double2* y);
// Y = A X for nr <= 8 vectors at once (spectra, weights and near values read once)
sie_status aim_apply_block(sie_op* op, AimOp& a, int which_LK, const double2* X, double2* Y, int nr);
sie_status aim_interp(sie_op* op, const double2* grids, int has_phi, double2 scal, double2* y);
sie_status sys_prepare(sie_op* op);
sie_status csr_tune_op(sie_op* op);
// Y = A X (acc: Y += A X) for nr <= 8 vectors of a CSR matrix: X, Y rhs-major
// with leading dimensions ldx, ldy; the values read once for all nr
sie_status csr_panel(cudaStream_t st, int nrow, const int64_t* rp, const int32_t* col, const double2* val,
                     const double2* X, int64_t ldx, int nr, bool acc, double2* Y, int64_t ldy);  // group sizes of the operator's CSR products, by measurement
void sys_release(sie_op* op);
sie_status sys_matvec(sie_op* op, int which, const double2* x, double2* y);
sie_status sys_solve(sie_op* op, const double2* b, double2* x, int* iters, double* relres);
sie_status sys_solve_refined(sie_op* op, const double2* b, double2* x, int* iters, double* relres);
sie_status sys_solve_multi(sie_op* op, int R, const double2* const* b, double2* const* x, int* iters, double* relres,
                           bool refine);
sie_status sys_rhs(sie_op* op, const double* khat, const double* epol, double2* b);
// y = A x for an edge CSR matrix (overwrites y)
sie_status csr_mv(cudaStream_t st, int nrow, int64_t nnz, const int64_t* rp, const int32_t* col,
                  const double2* val, const double2* x, double2* y);
sie_status sys_rcs(sie_op* op, const double2* x, const double* rhat, int ndir, double* rcs);
bool sys_z_workspace_ready(const sie_op* op);
// drop the captured system-product graph (solver settings changed)
void sys_graph_reset(sie_op* op);
// fold the nested-solve statistics of graph runs into op->stats (synchronises)
void sys_stats_fold(sie_op* op);
sie_status sys_far_sums(sie_op* op, const double2* x, const double* rhat_d, int ndir, double2* sums,
                        double* nested_res);
// nested-solve statistics: clear them, or fold the graph's copy and return
// SIE_ERR_NOT_CONVERGED when a nested solve ended above tol_inner
sie_status nested_clear(sie_op* op);
sie_status proj_map_ready(sie_op* op);
sie_status nested_check(sie_op* op, const char* who);
double sys_rcs_scale(const sie_op* op);
// nbatch consecutive grids (buf + k n^3, src + k N^3) in one launch per pass
// T = I - kappa D diag(LA)^-1 D^T Lphi_NR into f.A (f allocated for N_t)
sie_status dense_lu_assemble(cudaStream_t st, DenseLU& f, const sie_op* op, const AimOp& a, double2 kappa);
// build (assemble + factorise) the dense constraint LUs of op (ext, and inn when it has a grid)
sie_status constraint_lu_build(sie_op* op);
void constraint_lu_release(sie_op* op);
// SIE_ERR_TIMEOUT when a triangular-solve wait of a constraint LU ran out (synchronises)
sie_status constraint_lu_check(sie_op* op);
// grid part of the system product: forward x, y; fused forward z + spectral
// products + inverse z; inverse y, x (seven source grids in the compact src,
// four result grids back into it)
bool fft_sys_supported(const GridDesc& g);  // z length 16 .. 256
sie_status fft_sys(cudaStream_t st, double2* buf, double2* src, const GridDesc& g, const double2* spec, double k0,
                   sie_ctx* pc);
sie_status fft_sys(cudaStream_t st, float2* buf, float2* src, const GridDesc& g, const float2* spec, float k0,
                   sie_ctx* pc);
sie_status fft3d(cudaStream_t st, double2* buf, const double2* src, const GridDesc& g, int dir, int prune,
                 sie_ctx* prof_ctx, int nbatch = 1);
sie_status fft3d(cudaStream_t st, float2* buf, const float2* src, const GridDesc& g, int dir, int prune,
                 sie_ctx* prof_ctx, int nbatch = 1);
}  // namespace sie
