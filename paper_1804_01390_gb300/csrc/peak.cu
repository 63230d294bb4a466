// Arithmetic peak of the GPU, measured by the library's own kernel: every thread runs
// eight independent fused multiply-add chains for a fixed number of iterations, and the
// elapsed time of the launch (CUDA events on the caller's stream) gives the FMA rate.
// FP64 is the denominator of the FP64 step's roofline (that path is bound by the FP64
// pipe, which is narrow on this part); FP32 is reported beside it for context.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "pml.h"

namespace pml {
void set_global_error(const char *msg);   // runtime.cu: text for pml_last_error(NULL)

namespace {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 512;

// Never equal to any reachable chain value: the store only keeps the chains alive.
static __device__ double g_peak_sink;

template <typename T> __global__ void __launch_bounds__(kPeakThreads, 4) k_fma_peak(int64_t iters, T b, T c)
{
    T a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int64_t i = 0; i < iters; i += 16) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += a[k];
    if (s == T(-7.0e30)) g_peak_sink = double(s);   // the chains converge to c / (1 - b) > 0
}

template <typename T>
cudaError_t run_peak(cudaStream_t st, int64_t iters, int blocks, float *ms_out)
{
    // a = a * b + c with b slightly below 1 and c > 0 converges to c / (1 - b): the
    // chains stay finite and normal for any number of iterations
    const T b = T(0.999), c = T(1e-3);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    k_fma_peak<T><<<blocks, kPeakThreads, 0, st>>>(iters / 8 + 16, b, c);   // warm-up (clocks, code)
    cudaEventRecord(e0, st);
    k_fma_peak<T><<<blocks, kPeakThreads, 0, st>>>(iters, b, c);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms_out, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace pml

extern "C" pml_status pml_fma_peak(int precision, void *cuda_stream, int64_t iters, double *tflops, double *ms)
{
    using namespace pml;
    if ((precision != 32 && precision != 64) || iters < 16 || iters % 16 != 0 || !tflops) {
        set_global_error("pml_fma_peak: precision must be 32 or 64, iters a positive multiple of 16, "
                         "tflops not NULL");
        return PML_EINVAL;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_global_error("pml_fma_peak: no CUDA device");
        return PML_ECUDA;
    }
    const int blocks = 4 * sms;   // 2048 threads per SM: every scheduler has 16 warps of 8 chains
    float t = 0.f;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const cudaError_t e = precision == 64 ? run_peak<double>(st, iters, blocks, &t) : run_peak<float>(st, iters, blocks, &t);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return PML_ECUDA;
    }
    const double fmas = double(blocks) * kPeakThreads * kPeakChains * double(iters);
    *tflops = 2.0 * fmas / (double(t) * 1e-3) / 1e12;
    if (ms) *ms = t;
    return PML_OK;
}
