// Arithmetic peaks of the current GPU, measured (declared in include/rt3d.h
// as rt_probe_peaks): the denominators of the formal-solution rooflines,
// which are bound by FP64 or FP32 arithmetic rather than by memory.
//
// Each thread runs kChains independent fused multiply-add chains of
// kSteps steps in registers (no memory traffic inside the timed kernel),
// enough blocks to fill every SM several times over; the result is stored
// only under a condition the data never meets, so the chains cannot be
// removed.  Time: CUDA events around the second of two identical launches.
#include "../../include/rt3d.h"

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kSteps = 4096;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(T a, T b, T* sink)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int s = 0; s < kSteps; ++s) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
    }
    T acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += x[c];
    if (acc == (T)-1.2345) sink[blockIdx.x] = acc;   // never true for a, b below
}

template <typename T>
cudaError_t time_chain(int blocks, T* sink, double* tflops)
{
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return err;
    err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return err;
    }
    // x <- 0.999 x + 1e-4 stays bounded and positive
    const T a = (T)0.999, b = (T)1e-4;
    k_fma_chain<T><<<blocks, kThreads>>>(a, b, sink);
    cudaEventRecord(e0);
    k_fma_chain<T><<<blocks, kThreads>>>(a, b, sink);
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    const double flops = 2.0 * (double)blocks * kThreads * kChains * kSteps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace

extern "C" int rt_probe_peaks(int device, double* fp64_tflops, double* fp32_tflops)
{
    if (!fp64_tflops || !fp32_tflops) return RT_EINVAL;
    int sms = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return RT_ECUDA;
    double* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(double) * 64 * sms) != cudaSuccess) return RT_ENOMEM;
    cudaError_t err = time_chain<double>(8 * sms, sink, fp64_tflops);
    if (err == cudaSuccess) err = time_chain<float>(64 * sms, reinterpret_cast<float*>(sink), fp32_tflops);
    cudaFree(sink);
    return err == cudaSuccess ? RT_OK : RT_ECUDA;
}
