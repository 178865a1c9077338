// Arithmetic-peak probes: the FP64 and FP32 fused multiply-add throughput of the device, measured
// with long chains of independent FMAs per thread.  They give the denominators of the roofline
// fractions of the FP64-bound evaluation kernels and the FP32 parts of the mixed modes.
#include <cuda_runtime.h>

#include <algorithm>

#include "qbx_internal.cuh"
#include "qbx_peaks.h"

namespace qbx {

constexpr int PEAK_CHAINS = 8;  // independent accumulators per thread: hide the FMA latency

template <class T>
__global__ void __launch_bounds__(256) k_fma_chain(int iters, T a, T b, T *out)
{
    T acc[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = acc[k] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += acc[k];
    if (s == (T)1234567.0) out[0] = s;  // keeps the chains live; practically never taken
}

template <class T>
static double run_peak(int blocks_per_sm, int iters, int reps, cudaStream_t st)
{
    int dev = 0, nsm = 0;
    QBX_CUDA_TRY(cudaGetDevice(&dev));
    QBX_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    T *out = dalloc<T>(1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    try {
        QBX_CUDA_TRY(cudaEventCreate(&e0));
        QBX_CUDA_TRY(cudaEventCreate(&e1));
        const unsigned grid = (unsigned)(nsm * blocks_per_sm);
        // a = 1 - 2^-20, b = 2^-30: the chains stay finite and non-denormal
        const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1073741824.0);
        k_fma_chain<T><<<grid, 256, 0, st>>>(iters / 8, a, b, out);  // warm-up
        QBX_LAUNCH_CHECK();
        for (int r = 0; r < reps; ++r) {
            QBX_CUDA_TRY(cudaEventRecord(e0, st));
            k_fma_chain<T><<<grid, 256, 0, st>>>(iters, a, b, out);
            QBX_LAUNCH_CHECK();
            QBX_CUDA_TRY(cudaEventRecord(e1, st));
            QBX_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            QBX_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            const double flops = 2.0 * PEAK_CHAINS * (double)iters * grid * 256.0;
            if (ms > 0.f) best = std::max(best, flops / (ms * 1e-3));
        }
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        dfree(out);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(out);
    return best;
}

}  // namespace qbx

using namespace qbx;

extern "C" int qbx_peak_flops(int kind, int reps, double *flops_host, void *stream)
{
    try {
        set_error("");
        if (!flops_host || reps < 1 || (kind != QBX_PEAK_FP64 && kind != QBX_PEAK_FP32))
            throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        cudaStream_t st = (cudaStream_t)stream;
        // the best over several occupancies (blocks of 256 threads per SM), so that neither too few warps
        // in flight nor register or issue limits of one shape understate the peak
        double best = 0.0;
        for (int bps : {2, 4, 8})
            best = std::max(best, kind == QBX_PEAK_FP64 ? run_peak<double>(bps, 1 << 14, reps, st)
                                                        : run_peak<float>(bps, 1 << 16, reps, st));
        *flops_host = best;
        return QBX_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected exception");
        return QBX_ERR_CUDA;
    }
}
