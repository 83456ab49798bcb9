// k_peak.cu -- arithmetic-peak probes for the roofline denominators (measurement support,
// not part of the paper's method).  HBM bandwidth and the bf16 tensor rate are measured by
// the pool; the FP64 and FP32 FMA rates that bound this library's FP64 kernels and its FP32 /
// double-float kernels are measured here: eight independent FMA chains per thread (enough to
// cover the pipe latency), every SM filled, CUDA events around one launch.
#include "internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int64_t iters, T x, T y) {
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], x, y);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (T)12345.678) out[0] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" expm_status expm_peak_fma(int kind, int64_t iters, double* tflops, void* stream) {
    if ((kind != 0 && kind != 1) || iters < 1 || !tflops) return EXPM_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return EXPM_CUDA_ERROR;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return EXPM_CUDA_ERROR;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return EXPM_CUDA_ERROR;
    }
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {   // the first launch warms up
        ok = cudaEventRecord(e0, s) == cudaSuccess;
        if (kind == 0) k_fma_chains<double><<<blocks, threads, 0, s>>>(nullptr, iters, 0.9999999, 1e-9);
        else k_fma_chains<float><<<blocks, threads, 0, s>>>(nullptr, iters, 0.9999999f, 1e-9f);
        ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess &&
             cudaEventSynchronize(e1) == cudaSuccess;
    }
    float ms = 0.f;
    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return EXPM_CUDA_ERROR;
    const double flops = 2.0 * 8.0 * (double)iters * threads * (double)blocks;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return EXPM_OK;
}
