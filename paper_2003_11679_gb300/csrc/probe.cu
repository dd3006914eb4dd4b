// FMA throughput probe: the FP64 and FP32 arithmetic peaks that the FP64
// path's roofline fractions are quoted against (the measured peaks
// cover HBM copy bandwidth and bf16 tensor throughput only).  No counterpart
// in the paper.
#include <algorithm>

#include "internal.h"

namespace sie {

// CH independent FMA chains per thread, ITER iterations, each unrolled 16 ways;
// the chains' sum is stored so that no chain is dead code
template <class T, int CH>
__global__ void __launch_bounds__(256) k_fma(int iter, T b, T c, T* __restrict__ out)
{
    T a[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iter; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++) {
#pragma unroll
            for (int i = 0; i < CH; i++) a[i] = a[i] * b + c;
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < CH; i++) s += a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
static sie_status run_probe(int sms, int iter, double* tflops)
{
    const int blocks = sms * 8, threads = 256;
    constexpr int CH = 8;
    T* out = nullptr;
    SIE_CUDA_TRY(cudaMalloc((void**)&out, sizeof(T) * blocks * threads));
    cudaEvent_t e0, e1;
    SIE_CUDA_TRY(cudaEventCreate(&e0));
    SIE_CUDA_TRY(cudaEventCreate(&e1));
    // b, c keep the chains bounded: a -> a b + c converges to c / (1 - b)
    const T b = (T)0.999, c = (T)1e-3;
    double best = 0;
    sie_status s = SIE_OK;
    for (int rep = 0; rep < 4 && s == SIE_OK; rep++) {
        cudaEventRecord(e0, 0);
        k_fma<T, CH><<<blocks, threads>>>(iter, b, c, out);
        cudaEventRecord(e1, 0);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error(std::string("sie_probe_fma: ") + cudaGetErrorString(e));
            s = SIE_ERR_CUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        double flops = 2.0 * CH * 16.0 * (double)iter * blocks * threads;
        if (rep > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);  // first launch: warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *tflops = best;
    return s;
}

}  // namespace sie

extern "C" sie_status sie_probe_fma(int device, double* fp64_tflops, double* fp32_tflops)
{
    using namespace sie;
    if (!fp64_tflops || !fp32_tflops) {
        set_error("sie_probe_fma: null output");
        return SIE_ERR_ARG;
    }
    SIE_CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    SIE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    SIE_TRY(run_probe<double>(sms, 2048, fp64_tflops));
    SIE_TRY(run_probe<float>(sms, 131072, fp32_tflops));
    return SIE_OK;
}
