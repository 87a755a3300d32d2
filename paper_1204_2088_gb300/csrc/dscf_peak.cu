// Measured CUDA-core FMA throughput (FP32 and FP64), the denominator of the arithmetic roofline of
// the stencil kernels: independent fused multiply-add chains on every SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "../../include/dscf.h"

namespace dscf {
void set_thread_error(const char* msg);
}

namespace {

__device__ double g_peak_sink;   // keeps the chains alive; written only if a chain reaches 0.5

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-7;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = a[i] * b + c;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == (T)0.5) g_peak_sink = (double)s;
}

}  // namespace

extern "C" int dscf_fma_peak(int32_t precision, void* stream, double* tflops) {
    if (!tflops || (precision != DSCF_FP64 && precision != DSCF_FP32)) {
        dscf::set_thread_error("dscf_fma_peak: bad argument");
        return DSCF_ERR_ARG;
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        dscf::set_thread_error("dscf_fma_peak: device query failed");
        return DSCF_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = nsm * 8, threads = 256;
    // about 20 ms per FP32 run and 40 ms per FP64 run on a GB300-class part
    const int iters = precision == DSCF_FP32 ? 4096 : 128;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return DSCF_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DSCF_ERR_CUDA;
    }
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {   // the first run warms up
        cudaEventRecord(e0, s);
        if (precision == DSCF_FP32)
            k_fma_chains<float><<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-7f);
        else
            k_fma_chains<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || best >= 1e29f) {
        dscf::set_thread_error(err != cudaSuccess ? cudaGetErrorString(err) : "dscf_fma_peak: timing failed");
        return DSCF_ERR_CUDA;
    }
    const double flop = 2.0 * blocks * threads * (double)iters * 16.0 * kChains;
    *tflops = flop / (best * 1e-3) / 1e12;
    return DSCF_OK;
}
