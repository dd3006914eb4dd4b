// sie_rcs_static: the far-field RCS of sie_rcs without any allocation.  No
// counterpart in the paper; it serves callers that must not allocate after
// start-up (a serving loop holding a fixed device-memory budget, where an
// allocation per request could fail or stall).  Its scratch is one file-scope
// device array of fixed size, one copy per device.
#include <math.h>

#include <mutex>

#include "internal.h"

namespace {
constexpr int MAXDIR = SIE_RCS_STATIC_MAX_DIR;
constexpr int MAXDEV = 64;
// layout (doubles): directions 3 per direction (4 reserved), far-field sums
// N(H), N(E') 6 complex per direction, cross sections 1 per direction
constexpr size_t OFF_RHAT = 0;
constexpr size_t OFF_SUMS = 4 * (size_t)MAXDIR;  // 16-byte aligned (double2)
constexpr size_t OFF_RCS = OFF_SUMS + 12 * (size_t)MAXDIR;
constexpr size_t NSCRATCH = OFF_RCS + (size_t)MAXDIR;  // 17 x MAXDIR doubles
}  // namespace

static __device__ __align__(256) double rcs_scratch[NSCRATCH];

namespace sie {

static std::mutex g_scratch_mu;
static double* g_scratch[MAXDEV];

// Device address of rcs_scratch on device dev (current), looked up once.
static sie_status scratch_of(int dev, double** out)
{
    if (dev < 0 || dev >= MAXDEV) {
        set_error("sie_rcs_static: device ordinal out of range");
        return SIE_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, rcs_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("sie_rcs_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SIE_ERR_CUDA;
        }
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return SIE_OK;
}

// sigma_d = scale |N_perp(H) + rhat x N(E')|^2, one thread per direction
__global__ void k_rcs_sigma(int ndir, double scale, const double* __restrict__ rhat,
                            const double2* __restrict__ sums, double* __restrict__ rcs)
{
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndir) return;
    const double2* NH = sums + 6 * d;
    const double2* NE = NH + 3;
    const double r0 = rhat[3 * d], r1 = rhat[3 * d + 1], r2 = rhat[3 * d + 2];
    const double rnx = r0 * NH[0].x + r1 * NH[1].x + r2 * NH[2].x;
    const double rny = r0 * NH[0].y + r1 * NH[1].y + r2 * NH[2].y;
    double2 v[3];
    v[0] = make_double2(NH[0].x - rnx * r0 + (r1 * NE[2].x - r2 * NE[1].x),
                        NH[0].y - rny * r0 + (r1 * NE[2].y - r2 * NE[1].y));
    v[1] = make_double2(NH[1].x - rnx * r1 + (r2 * NE[0].x - r0 * NE[2].x),
                        NH[1].y - rny * r1 + (r2 * NE[0].y - r0 * NE[2].y));
    v[2] = make_double2(NH[2].x - rnx * r2 + (r0 * NE[1].x - r1 * NE[0].x),
                        NH[2].y - rny * r2 + (r0 * NE[1].y - r1 * NE[0].y));
    double s = 0.0;
    for (int k = 0; k < 3; k++) s += v[k].x * v[k].x + v[k].y * v[k].y;
    rcs[d] = scale * s;
}

}  // namespace sie

using namespace sie;

extern "C" {

sie_status sie_rcs_static(sie_op* op, const double* x, const double* rhat, int ndir, double* rcs, int flags)
{
    if (!op || !x || !rhat || !rcs || ndir < 1) {
        set_error("sie_rcs_static: invalid argument");
        return SIE_ERR_ARG;
    }
    if (ndir > MAXDIR) {
        set_error("sie_rcs_static: ndir " + std::to_string(ndir) + " exceeds SIE_RCS_STATIC_MAX_DIR (" +
                  std::to_string(MAXDIR) + "); split the directions over several calls");
        return SIE_ERR_ARG;
    }
    sie_ctx* c = op->mesh->ctx;
    if (c->prof.on) {
        set_error("sie_rcs_static: profiling is on (its stage records allocate); disable it first");
        return SIE_ERR_STATE;
    }
    if (!sys_z_workspace_ready(op)) {
        set_error("sie_rcs_static: the interior solver's workspace is not allocated for the current settings; "
                  "run sie_solve or a SIE_OP_SYS product on this operator first");
        return SIE_ERR_STATE;
    }
    SIE_CUDA_TRY(cudaSetDevice(c->device));
    double* s = nullptr;
    SIE_TRY(scratch_of(c->device, &s));
    cudaStream_t st = c->stream;
    const int64_t len = op->mesh->h.ne + op->mesh->h.nt;
    const double2* xr = (const double2*)x;
    if (!(flags & SIE_DEVICE_PTRS)) {
        SIE_CUDA_TRY(cudaMemcpyAsync(op->sys_vec, x, sizeof(double2) * len, cudaMemcpyHostToDevice, st));
        xr = op->sys_vec;
    }
    SIE_CUDA_TRY(cudaMemcpyAsync(s + OFF_RHAT, rhat, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, st));
    double2* sums = reinterpret_cast<double2*>(s + OFF_SUMS);
    double nres = 0.0;
    SIE_TRY(sys_far_sums(op, xr, s + OFF_RHAT, ndir, sums, &nres));
    k_rcs_sigma<<<(ndir + 127) / 128, 128, 0, st>>>(ndir, sys_rcs_scale(op), s + OFF_RHAT, sums, s + OFF_RCS);
    SIE_CUDA_TRY(cudaGetLastError());
    SIE_CUDA_TRY(cudaMemcpyAsync(rcs, s + OFF_RCS, sizeof(double) * ndir, cudaMemcpyDeviceToHost, st));
    SIE_CUDA_TRY(cudaStreamSynchronize(st));
    if (nres >= op->p.tol_inner) {
        set_error("sie_rcs_static: the nested interior solve of Z_i H ended above tol_inner");
        return SIE_ERR_NOT_CONVERGED;
    }
    return SIE_OK;
}

}  // extern "C"
