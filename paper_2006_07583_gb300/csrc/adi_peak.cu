// adi_peak.cu -- adi_fma_peak: the device's measured fused multiply-add throughput in FP64 or
// FP32, the denominator of the ALU roofline of the line solvers in that precision.  Every
// thread runs 16 independent FMA chains (enough to cover the FMA latency at full occupancy);
// the grid fills every SM several times over.  Nothing about the GPU's settings is changed.
#include <cuda_runtime.h>

#include "../../include/adi.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int iters, T b, T c, T *out) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * kThreads + threadIdx.x] = s;  // keeps the chains live
}

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return ADI_OK;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return ADI_ENOTSUP;
    return ADI_ECUDA;
}

template <typename T>
int run(double *flops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return status_of(e); }
    const int blocks = sms * 8;
    const int iters = sizeof(T) == 8 ? 4096 : 16384;
    T *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(T));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            fma_chains_kernel<T><<<blocks, kThreads, 0, s>>>(iters, (T)0.9999999, (T)1e-7, out);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e == cudaSuccess && best > 0.0f)
        *flops = 2.0 * (double)blocks * kThreads * kChains * iters / (best * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return status_of(e); }
    return ADI_OK;
}

}  // namespace

extern "C" int adi_fma_peak(int precision, double *flops_per_s) {
    if (!flops_per_s || (precision != ADI_FP32 && precision != ADI_FP64)) return ADI_EINVAL;
    *flops_per_s = 0.0;
    return precision == ADI_FP64 ? run<double>(flops_per_s) : run<float>(flops_per_s);
}
