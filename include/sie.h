/*
 * sie.h -- C ABI of the GB300 (sm_103a) AIM-accelerated surface-integral-
 * equation library.
 *
 * The library implements the matrix-vector products and the solve of
 * Sharma & Triverio, "An Accelerated Surface Integral Equation Method for the
 * Electromagnetic Modeling of Dielectric and Lossy Objects of Arbitrary
 * Conductivity":
 *   - the RWG/Galerkin operators L and K of Eqs. (opL), (opK) for a medium
 *     with complex wavenumber k (Eq. kin), Green's function of Eq. (Grrpki);
 *   - their AIM form, Eqs. (AIM_Lin), (AIM_Kin): projection onto a uniform
 *     grid, 3D FFT convolution with the sampled Green's function and its
 *     gradient, interpolation back to the mesh, plus the precorrected sparse
 *     near-region matrices of Eqs. (LinNRP), (KinNRP);
 *   - the near-region-only interior operators used when the skin depth is
 *     small (Sec. III-C, the 5-skin-depth cutoff of Sec. V);
 *   - the GIBC system of Eq. (GIBCsys) with the interior operator of
 *     Eqs. (nest02), (nest2), solved by GMRES (Sec. V), plane-wave excitation
 *     (Sec. II) and the monostatic / bistatic RCS (Sec. V-A).
 *
 * Conventions
 *   - Time dependence exp(+j w t).  k = sqrt(w mu (w eps - j sigma)) with
 *     Im k <= 0 (Eq. kin).
 *   - Complex numbers are interleaved (re, im) doubles (numpy complex128,
 *     torch.complex128); complex64 buffers are interleaved floats.
 *   - Vectors with nrhs right-hand sides are stored rhs-major: element n of
 *     right-hand side r is at index r * len + n.
 *   - Unknowns are RWG edge coefficients, numbered in increasing
 *     (lower vertex id, higher vertex id) order of the edge; T+ is the
 *     triangle in which the edge runs from the lower to the higher vertex id
 *     in counter-clockwise (outward-normal) order.
 *
 * Ownership: every *_create / *_build call copies its host inputs; handles
 * are opaque and must be destroyed in reverse order of creation (op, mesh,
 * ctx).  Vector arguments are borrowed: with SIE_DEVICE_PTRS they are device
 * pointers on the context's device, otherwise host pointers.
 *
 * Errors: every call returns a sie_status; nothing aborts or exits.
 * sie_last_error() returns a message for the last failing call on the
 * calling thread.  Calls on one context must not overlap in time (one host
 * thread at a time); all device work is issued on the context's stream.
 */
#ifndef SIE_H
#define SIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIE_OK = 0,
    SIE_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad enum) */
    SIE_ERR_MESH = 2,           /* mesh not a closed oriented 2-manifold, degenerate triangle */
    SIE_ERR_OOM = 3,            /* device allocation failed */
    SIE_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    SIE_ERR_NOT_CONVERGED = 5,  /* GMRES reached maxit; x holds the last iterate */
    SIE_ERR_TIMEOUT = 6,        /* a device-side wait gave up */
    SIE_ERR_STATE = 7,          /* call not valid for this handle's state */
    SIE_ERR_UNSUPPORTED = 8     /* valid request this build does not handle */
} sie_status;

typedef struct sie_ctx sie_ctx;
typedef struct sie_mesh sie_mesh;
typedef struct sie_op sie_op;

enum { SIE_FP64 = 0, SIE_MIXED = 1 };          /* grid-path precision */
enum { SIE_GIBC = 0, SIE_SIBC = 1 };           /* interior model (sie_params.interior_model) */
enum { SIE_DEVICE_PTRS = 1,                    /* flags: vector args are device pointers */
       SIE_SOLVE_REFINE = 2,                    /* sie_solve: mixed-precision iterative refinement */
       SIE_SOLVE_SEQUENTIAL = 4 };              /* sie_solve: one right-hand side after another */

/* Which operator sie_matvec applies. */
enum {
    SIE_OP_L0 = 0,  /* exterior L (background medium), AIM form           */
    SIE_OP_K0 = 1,  /* exterior K (background medium), AIM form           */
    SIE_OP_LI = 2,  /* interior L of the object (AIM or near-only)        */
    SIE_OP_KI = 3,  /* interior K of the object (AIM or near-only)        */
    SIE_OP_SYS = 4, /* GIBC system of Eq. (GIBCsys), divided by eta0      */
    SIE_OP_ZI = 5   /* interior impedance Z_i of Eq. (GIBCdef) / eta0     */
};

/* Method parameters.  sie_params_default() fills the paper's values
 * (Sec. IV-V) and the library's near-field quadrature defaults. */
typedef struct {
    double h;             /* grid spacing in metres; 0 = derive (below)                */
    double h_over_edge;   /* h = h_over_edge * mean edge length (default 0.5) ...      */
    int grid_n;           /* ... unless grid_n > 0: largest dimension has grid_n nodes */
    int stencil_order;    /* M, Lagrange order per axis (default 2, Sec. IV)           */
    int near_radius;      /* R_near in grid nodes (default 5: 11-node diameter, Sec. IV) */
    double skin_cutoff;   /* interior pairs farther than this many skin depths dropped (5, Sec. V) */
    int precision;        /* SIE_FP64 or SIE_MIXED (complex64 grid path)               */
    double tol_outer;     /* GMRES relative residual, outer system (1e-4, Sec. V)      */
    double tol_inner;     /* GMRES relative residual, nested interior system (1e-6)    */
    int maxit;            /* outer iteration cap (800, Sec. V-A)                       */
    int restart;          /* GMRES restart length (100)                                */
    int inner_maxit;      /* nested iteration cap (200)                                */
    double tol_constraint;/* constraint preconditioner: inner GMRES tolerance of its
                             triangle (charge) system (1e-6), preconditioned by its
                             dense factorisation when one was made (dense_pc_max) */
    int constraint_maxit; /* ... and its iteration cap (1000)                          */
    int constraint_restart; /* ... and its GMRES restart length (100)                  */
    double tol_constraint_inner; /* the same for the nested (interior) preconditioner (1e-3) */
    /* near-field quadrature (the method's direct-integration rule) */
    int q_far;            /* far-near pairs: q_far x q_far collapsed Gauss per triangle (5) */
    int q_out;            /* close pairs: q_out x q_out outer points (5)                */
    int q_ang;            /* polar inner rule: Gauss points per angular panel (8)       */
    int q_rad;            /* polar inner rule: Gauss points per radial panel (8)        */
    int q_npan;           /* radial panels graded toward the centre (5)                 */
    int q_opan;           /* touching pairs: outer panels graded toward the feature (7) */
    int q_olam;           /* touching pairs: points per graded outer panel (5)          */
    int q_omu;            /* touching pairs: points across, vertex shared (6)           */
    int q_emupan;         /* touching pairs: graded panels per half of a shared edge (2)*/
    int q_emu;            /* touching pairs: points per shared-edge panel (4)           */
    double q_ratio;       /* radial panel ratio (0.25)                                  */
    double q_cf;          /* close if centroid distance < q_cf (R_t + R_s) (2.0)        */
    double q_kres;        /* close if |k| (R_t + R_s) > q_kres (1.0)                    */
    double q_alen;        /* longest angular (asinh) panel (1.5)                        */
    double q_oratio;      /* outer panel ratio (0.25)                                   */
    int dense_pc_max;     /* constraint preconditioners: factorise the triangle (charge)
                             system densely on the GPU (complex64 LU) when N_t <= this
                             (32768); else solve it iteratively                        */
    int interior_model;   /* SIE_GIBC (default): Z_i from the interior operators
                             (Eqs. GIBCdef, nest02, nest2); SIE_SIBC: the surface
                             impedance boundary condition the paper compares against
                             (Sec. I-II), Z' = (eta_i / eta0) G^-1 I_x with the RWG
                             Gram matrix G (no interior operators are built)          */
} sie_params;

/* The paper's values (Sec. IV: M = 2, near region of 11 nodes; Sec. V: skin
 * cutoff 5, tolerances 1e-4 / 1e-6, cap 800) and the library's defaults for
 * what the paper leaves open (quadrature, restart, dense_pc_max). */
void sie_params_default(sie_params* p);

/* Context on one CUDA device.  The paper has no counterpart (it runs on one
 * CPU thread, Sec. V): a context fixes the device and the stream the
 * library's kernels run on.  stream: the cudaStream_t every call of this
 * context issues its device work on (NULL = the legacy default stream).  The
 * stream is borrowed: the caller keeps it alive until sie_ctx_destroy. */
sie_status sie_ctx_create(int device, void* stream, sie_ctx** out);
sie_status sie_ctx_destroy(sie_ctx* ctx);
const char* sie_last_error(void);

/* Stage timers (no counterpart in the paper, which reports whole-phase wall
 * times, Sec. V): while enabled, every kernel stage the context launches is
 * bracketed by CUDA events on the context's stream, and its device time is
 * accumulated under the stage's name.  Enabling clears the totals.
 * sie_profile_read synchronises on the pending events and copies up to cap
 * entries: names (cap x 32 chars, NUL terminated), total ms and launch
 * counts; *n receives the number of stages seen. */
sie_status sie_profile_enable(sie_ctx* ctx, int enable);
sie_status sie_profile_read(sie_ctx* ctx, int cap, char* names, double* ms, int64_t* count, int* n);

/* Mesh of a closed surface for the RWG discretisation (Sec. II-A: n x H and
 * n x E expanded with RWG functions on a triangulation of the object's
 * surface): xyz (nv x 3, metres), tri (nt x 3, 0-based, counter-clockwise seen
 * from outside).  Fails with SIE_ERR_MESH unless every edge is shared by
 * exactly two oppositely oriented triangles (open, non-manifold, inconsistent
 * or degenerate meshes), SIE_ERR_ARG for non-finite coordinates.  One
 * homogeneous object (sie_mesh_create_objects for several). */
sie_status sie_mesh_create(sie_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                           sie_mesh** out);
sie_status sie_mesh_destroy(sie_mesh* mesh);
/* counts (Sec. II-A): out[0] = RWG edges N_e (unknowns of H and E), out[1] =
 * triangles N_t (pulse unknowns of the charge, Eq. sys), out[2] = vertices */
sie_status sie_mesh_counts(const sie_mesh* mesh, int64_t out[3]);

/* Several homogeneous objects in the background medium (Sec. II: N_obj
 * objects with their own eps_i, mu_i, sigma_i; the interior problem of each
 * object couples only its own triangles, Eq. GIBCdef per object).  As
 * sie_mesh_create, plus obj_id: nt object indices 0 .. N_obj - 1 (NULL: one
 * object).  Every object must be a closed, consistently oriented surface on
 * its own: an edge shared by triangles of two objects is SIE_ERR_MESH (so are
 * object indices below 0).  *nobj (may be NULL) receives N_obj. */
sie_status sie_mesh_create_objects(sie_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                                   const int32_t* obj_id, sie_mesh** out, int* nobj);

/* Material of object obj (relative permittivity, permeability and
 * conductivity in S/m, Eq. kin).  Objects without one take the material
 * passed to sie_op_build.  Applies to operators built afterwards.
 * SIE_ERR_ARG for obj outside 0 .. N_obj - 1 or an unphysical material. */
sie_status sie_set_material(sie_mesh* mesh, int obj, double eps_r, double mu_r, double sigma);

/* Build the operators of one frequency.  Background medium: vacuum.  Object:
 * (eps_r, mu_r, sigma).  Builds the exterior AIM operator (k0) and the
 * interior operator (k_i): an AIM grid operator, or the near-region-only
 * operator when 5 skin depths fit inside the near region (every kept pair is
 * near; Sec. III-C).  Device memory is allocated here and freed by
 * sie_op_destroy.
 * Several objects (sie_mesh_create_objects): each object's interior uses its
 * own material (sie_set_material, else eps_r, mu_r, sigma); its near pairs
 * stay inside the object and its Z_i scales its own edges, so Z' is block
 * diagonal over the objects.  With more than one object every interior must
 * be near-region only, or interior_model = SIE_SIBC; otherwise
 * SIE_ERR_UNSUPPORTED (per-object interior AIM grids are not built). */
sie_status sie_op_build(sie_mesh* mesh, double freq_hz, double eps_r, double mu_r, double sigma,
                        const sie_params* params, sie_op** out);
sie_status sie_op_destroy(sie_op* op);

/* Replace the solver controls of a built operator (the GMRES tolerances and
 * caps of Sec. V, the precision path): precision (grid path of
 * the system product: SIE_FP64 or SIE_MIXED = complex64 projection, FFT,
 * spectral multiply and interpolation, exterior near-region products with
 * complex64 copies of the FP64-integrated values (FP32 products, FP64 row
 * sums), FP64 interior (lossy-medium) products and FP64 Krylov), tol_outer,
 * tol_inner, maxit, restart, inner_maxit, tol_constraint, constraint_maxit,
 * constraint_restart and tol_constraint_inner are taken from params; grid,
 * quadrature, dense_pc_max and interior_model are ignored (they are fixed at
 * build time). */
sie_status sie_op_set_solver(sie_op* op, const sie_params* params);

/* Statistics of the last sie_solve on this operator (the outer and nested
 * iteration counts the paper reports, Sec. V) (6 doubles): outer
 * iterations, outer relative residual, the largest nested (interior)
 * iteration count and residual, the largest constraint-preconditioner
 * iteration count and residual.  A SIE_OP_SYS / SIE_OP_ZI sie_matvec clears
 * the nested entries first, so after it they describe that call's nested
 * solves (the way to check them for device-pointer calls, which do not
 * synchronise).  Synchronises the context's stream. */
sie_status sie_op_stats(const sie_op* op, double out[6]);

/* Operator facts (the AIM grid of Sec. III-A / IV and the near region of
 * Eqs. LinNRP, KinNRP).  info (20 doubles): [0..2] grid N_x, N_y, N_z; [3..5] FFT
 * n_x, n_y, n_z; [6] h; [7] near pairs (exterior); [8] nnz of the exterior
 * near matrix; [9] interior mode (0 = AIM, 1 = near only); [10] interior near
 * pairs; [11] grid origin x (origin y, z: see sie_op_grid); build wall times
 * in ms: [12] weights and spectra, [13] exterior near region, [14] interior
 * near region, [15] host-side pair lists; [16] system-product CUDA graph
 * (near-region-only interiors): +1 captured for SIE_FP64, +2 for SIE_MIXED,
 * +4 capture failed (the stream path is used); [17] nodes of the last
 * captured graph outside the nested loop (kernels, memsets, copies and the
 * loop node), [18] nodes of the loop body (run once per nested iteration);
 * [19] wall time in ms of the dense factorisations of the constraint
 * preconditioners' triangle systems (0 when they are solved iteratively,
 * minus the sie_status when the factorisation could not be made, e.g. -3 for
 * no device memory; the iterative solve is used then). */
sie_status sie_op_info(const sie_op* op, double info[20]);
/* grid origin (3), spacing and node counts of the exterior AIM grid (Sec. III-A) */
sie_status sie_op_grid(const sie_op* op, double origin[3], double* h, int64_t N[3]);

/* y = A x for nrhs right-hand sides, A selected by `which` (SIE_OP_*):
 * Eqs. (AIM_Lin), (AIM_Kin) for L0/K0/LI/KI, Eq. (sys) for SYS, and Z_i of
 * Eqs. (GIBCdef), (nest02), (nest2) for ZI.
 * x, y: complex128, length N_e (L0, K0, LI, KI, ZI) or N_e + N_t (SYS, the
 * AEFIE unknowns [H; c0 rho] of Eq. sys).  flags: SIE_DEVICE_PTRS or 0.
 * L0, K0, LI and KI with nrhs > 1 run in blocks of up to 8 right-hand sides:
 * the kernel spectra, the stencil weights and the near-region values are read
 * once per block (one projection, FFT pass, spectral multiply, interpolation
 * and CSR x panel launch per block).  The other operators loop over the
 * right-hand sides.
 * SYS and ZI contain the nested solve of Eq. (nest2): one unrestarted FGMRES
 * cycle of at most min(inner_maxit, 128) iterations to tol_inner.  When it
 * ends above tol_inner, host-pointer calls return SIE_ERR_NOT_CONVERGED (y
 * holds the product with that inexact Z_i); device-pointer calls do not
 * synchronise and report it through sie_op_stats.
 * When the interior operator is near-region only and profiling is off, the
 * SYS product (nested solve included) is captured on first use into a CUDA
 * graph, one per precision, and replayed; the nested iterations are then a
 * loop the device ends itself, with the same iteration limit as the stream
 * path.  The environment variable SIE_GRAPH=0 selects the stream path.  The
 * graph is dropped when tol_inner or inner_maxit change (sie_op_set_solver). */
sie_status sie_matvec(sie_op* op, int which, const double* x, double* y, int nrhs, int flags);

/* Export the precorrected near-region matrix of an operator (L_NRP, K_NRP of
 * Eqs. LinNRP, KinNRP for AIM operators; L_i,NR, K_i,NR for near-only
 * interiors, Sec. III-C)
 * (SIE_OP_L0/K0/LI/KI) as CSR on the host: call once with col/val NULL to get
 * nnz in *nnz and row_ptr (N_e + 1) filled; then again with buffers of nnz
 * entries.  val is complex128. */
sie_status sie_op_near_csr(const sie_op* op, int which, int64_t* row_ptr, int32_t* col, double* val,
                           int64_t* nnz);

/* Right-hand side of Eq. (EFIE01dis) divided by eta0 for plane waves
 * E_inc = epol exp(-j k0 khat . r) (khat unit propagation direction, epol
 * orthogonal to it, |epol| = 1 V/m): b_m = -(1/eta0) I f_m . E_inc dS.
 * khat, epol: nrhs x 3 doubles (host).  b: complex128 nrhs x N_e. */
sie_status sie_rhs_planewave(sie_op* op, const double* khat, const double* epol, int nrhs, double* b, int flags);

/* Solve SYS x = b (Eq. sys) by restarted FGMRES (FP64 Arnoldi, right
 * preconditioned by the AEFIE constraint preconditioner, zero initial guess)
 * until the true relative residual is below tol_outer.  The residual is
 * measured with the charge rows of Eq. (sys) weighted by
 * q_w = mean_m |L_A,mm|, which gives the two diagonal blocks of the
 * constraint preconditioner (j k0 diag(L_A) and j k0 I) the same size:
 * relres = |W (b - A x)| / |W b|, W = diag(I, q_w I).  Unweighted, the
 * charge rows (a divergence per triangle, ~1e16 times a Galerkin potential
 * entry on a finely meshed millimetre object) make the FP64 rounding of
 * F D H + j k0 c0 rho alone reach 1e-3 of |b|.  b, x: complex128,
 * N_e + N_t per right-hand side ([H; c0 rho]), nrhs consecutive vectors.
 * iters / relres: per rhs (host arrays of nrhs, may be NULL).
 * nrhs > 1: blocks of up to 8 right-hand sides are solved in lockstep (one
 * Krylov basis each; every iteration applies the operator and the
 * preconditioner to the block's current vectors together, the dense
 * constraint factorisation in one pass over it for all of them) until all
 * of the block have converged; iters then counts the block's iterations.
 * SIE_SOLVE_SEQUENTIAL solves them one after another instead.
 * flags: SIE_DEVICE_PTRS; SIE_SOLVE_REFINE = mixed-precision iterative
 * refinement: the residual b - A x and the update use the FP64 product, each
 * correction A d = r is solved with the complex64 product (as SIE_MIXED) to
 * the accuracy the sweep needs, and the sweeps stop when the FP64 residual is
 * below tol_outer (iters then counts the FGMRES iterations of all
 * corrections); when a sweep does not halve the FP64 residual (the complex64
 * product's error, amplified by cancellation, bounds what it can reach), the
 * remaining corrections use the FP64 product.  Returns SIE_ERR_NOT_CONVERGED with the last iterate in x when
 * maxit is reached first, or when a nested interior solve of its products
 * ended above tol_inner (sie_op_stats gives both residuals). */
sie_status sie_solve(sie_op* op, const double* b, double* x, int nrhs, int* iters, double* relres, int flags);

/* Monostatic/bistatic RCS (m^2) of the solution x (as returned by sie_solve,
 * for the plane wave with polarisation epol, 1 V/m), the quantity compared
 * with the Mie series in Sec. V-A: for each observation direction rhat
 * (ndir x 3, host) the far-field cross section 4 pi |E_s|^2 r^2 of the
 * equivalent currents J = n x H and M = -n x E (E = Z_i H through the nested
 * solve).  rcs: ndir doubles (host).  One right-hand side.  Returns
 * SIE_ERR_NOT_CONVERGED (rcs filled) when that nested solve ended above
 * tol_inner. */
sie_status sie_rcs(sie_op* op, const double* x, const double* rhat, int ndir, double* rcs, int flags);

/* Directions per sie_rcs_static call (bounds its static device array). */
#define SIE_RCS_STATIC_MAX_DIR 2048

/* sie_rcs that allocates nothing.  The paper has no counterpart: this is an
 * interface variant of sie_rcs for callers that must not allocate once they
 * run, such as a serving loop that reserves its device-memory budget at
 * start-up and cannot let a request fail on out-of-memory or wait on the
 * allocator.  sie_rcs allocates device scratch (directions, far-field sums)
 * and a host staging array on every call; this variant keeps both in one
 * statically sized device array of the library (SIE_RCS_STATIC_MAX_DIR x 17
 * doubles, 272 KiB, one copy per device) and forms the cross sections on the
 * device.  Arguments, layouts and results are those of sie_rcs (same
 * far-field kernel and formula); ndir outside 1..SIE_RCS_STATIC_MAX_DIR
 * returns SIE_ERR_ARG.
 * Preconditions, else SIE_ERR_STATE with nothing launched: the operator has
 * already run sie_solve or a SIE_OP_SYS/SIE_OP_ZI product with its current
 * solver settings, so that the nested interior solve of Z' finds its Krylov
 * workspaces at their sizes (sie_rcs would allocate them), and profiling
 * (sie_profile_enable) is off, since its stage records grow host arrays.
 * Set-up: the first call on each device looks up the array's address with
 * cudaGetSymbolAddress, that device current, and caches it; make that first
 * call before any stream capture begins on the device.
 * What "allocates nothing" covers: no device memory is allocated or freed
 * (no cudaMalloc, cudaMallocAsync, cudaFree or allocating library routine),
 * and a successful call makes no host heap allocation either (only error
 * messages allocate).
 * Sharing: all calls on one device use the same array, so calls that overlap
 * in time on a device (from other threads, streams or contexts) race on it;
 * the caller serialises them.  Each call returns once its results are on the
 * host.  No part of the array has to start at zero: a call writes every
 * direction, far-field sum and cross section that it reads back. */
sie_status sie_rcs_static(sie_op* op, const double* x, const double* rhat, int ndir, double* rcs, int flags);

/* Ports (delta gap).  Sec. II admits a port excitation in place of the plane
 * wave, and Sec. V extracts the S parameters of its copper package and
 * interconnect examples through ports, but the paper only cites the port
 * model.  The library's model is the delta gap:
 *   - a port is a closed loop of mesh edges cutting a conductor's surface:
 *     the edges whose two end points lie in the plane through `origin` with
 *     normal `normal` (within 1e-6 mean edge lengths) and within `radius`
 *     of `origin`.  Each of them must have its two triangles on opposite
 *     sides of the plane, and the mesh must have vertices on the plane (a
 *     structured mesh cut along one of its grid planes, for instance);
 *   - `normal` is the port's reference direction: s_m = +1 when T+ of edge
 *     m lies on the -normal side, else -1, and p_m = s_m l_m;
 *   - a voltage V across port j is the impressed field V delta(xi) normal,
 *     xi = normal . (r - origin), entering Eq. (EFIE01dis) as the incident
 *     field does: b_m = -(V / eta0) p_m (charge rows zero);
 *   - the current through the port along +normal is I = -p . H (the first
 *     block of the solution holds the RWG coefficients of -n x H), so that
 *     (1/2) Re(V I*) is the power the port delivers;
 *   - Y_ij = I_i / V_j with every other port shorted (no impressed field),
 *     S = (1 - z_ref Y)(1 + z_ref Y)^-1. */
typedef struct {
    double origin[3];   /* a point of the port plane (m)                         */
    double normal[3];   /* plane normal = reference direction (any length > 0)   */
    double radius;      /* only edges within this distance of origin (m)         */
} sie_port;

/* The edges of one port (the port loop of Sec. II's port excitation, in the
 * delta-gap model above; ascending edge numbers) and their signs s_m.  Call
 * with edge or sign NULL to get the count in *n; then with buffers of *n
 * entries (host).  SIE_ERR_ARG when no edge qualifies, an edge in the plane
 * does not separate its triangles, or the port's numbers are not finite. */
sie_status sie_port_edges(const sie_mesh* mesh, const sie_port* port, int32_t* edge, int32_t* sign, int64_t* n);

/* Right-hand sides of the ports (the port excitation of Sec. II entering
 * Eq. (EFIE01dis) like E_inc): nport vectors of N_e + N_t complex128
 * ([first block; zero charge rows], the layout of sie_solve), vector j with
 * port j driven by volts[j] volts (volts NULL: 1 V) and the other ports
 * shorted.  flags: SIE_DEVICE_PTRS for a device b.  Allocates and frees
 * small device buffers; synchronises. */
sie_status sie_rhs_ports(sie_op* op, const sie_port* ports, int nport, const double* volts, double* b, int flags);

/* Port currents (Sec. V: the port quantities the S parameters come from)
 * I = -p_i . H_r of nrhs solutions x (N_e + N_t complex128
 * each, as sie_solve returns them): I[r * nport + i] (complex128, host).
 * flags: SIE_DEVICE_PTRS for a device x.  Allocates and frees small device
 * buffers; synchronises. */
sie_status sie_port_currents(sie_op* op, const sie_port* ports, int nport, const double* x, int nrhs, double* I,
                             int flags);

/* Admittance matrix of the ports (Sec. V network parameters): one solve per
 * port (sie_solve with nport
 * right-hand sides, lockstep blocks of 8), then the port currents.
 * Y: nport x nport complex128 row-major on the host, Y[i * nport + j] =
 * current through port i per volt on port j.  iters, relres: per port (host
 * arrays of nport, may be NULL).  flags: SIE_SOLVE_REFINE and
 * SIE_SOLVE_SEQUENTIAL as in sie_solve (SIE_DEVICE_PTRS is refused: Y is a
 * host array).  Returns SIE_ERR_NOT_CONVERGED, with Y from the last iterates,
 * when a solve stopped at maxit or a nested solve ended above tol_inner. */
sie_status sie_port_admittance(sie_op* op, const sie_port* ports, int nport, double* Y, int* iters, double* relres,
                               int flags);

/* S parameters (Sec. V, Figs. of the package and interconnect examples)
 * from an admittance matrix for one real reference impedance
 * z_ref (ohm) on every port: S = (1 - z_ref Y)(1 + z_ref Y)^-1.  Y, S:
 * nport x nport complex128 row-major, host.  Host arithmetic only (Gaussian
 * elimination with partial pivoting).  SIE_ERR_ARG when 1 + z_ref Y is
 * singular or z_ref is not positive. */
sie_status sie_port_sparams(int nport, const double* Y, double z_ref, double* S);

/* x_q = A^-1 b_q for one dense complex matrix and nrhs right-hand sides with
 * the library's GPU LU, the one the constraint preconditioners use
 * (Sec. III-D: the paper factorises its preconditioner by LU): complex64
 * blocked LU with partial pivoting on device `device`, then either two
 * triangular solves per right-hand side (flags 0) or, as the preconditioners
 * do, the explicit inverse U^-1 L^-1 P formed from the factors and applied in
 * one pass over it per block of up to 8 right-hand sides (flags 1; one
 * matrix-vector product each when n is odd).  A: n x n complex128 row-major
 * (host), b, x: nrhs consecutive vectors of n complex128 (host); A is rounded
 * to complex64, so x carries complex64 rounding amplified by the condition
 * number.  Allocates and frees its device memory; synchronises.  SIE_ERR_ARG
 * for n < 1, nrhs < 1 or a zero pivot (singular matrix). */
sie_status sie_dense_solve(int device, int n, int nrhs, const double* A, const double* b, double* x, int flags);

/* FMA throughput of device `device`: FP64 and FP32 TFLOP/s (2 flops per
 * FMA), measured by the library's own probe kernel (independent FMA chains on
 * every SM, best of three timed launches after a warm-up).  The paper has no
 * counterpart: this is the arithmetic peak the FP64 path's roofline fractions
 * are quoted against.  Allocates and frees a small device buffer; runs on the
 * legacy default stream and synchronises it. */
sie_status sie_probe_fma(int device, double* fp64_tflops, double* fp32_tflops);

#ifdef __cplusplus
}
#endif
#endif /* SIE_H */
