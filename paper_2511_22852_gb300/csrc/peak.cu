// peak.cu -- measurement support: the FP64 and FP32 fused multiply-add rates of the device,
// the denominators of the arithmetic rooflines of the step's kernels (no kernel of the step
// is a dense contraction; the neighbour sums and the EoS inversion are bound by the FP32 and
// FP64 pipes).
//
// Each thread runs kChains independent multiply-add chains (enough independent work per warp
// to cover the pipe latency), over a grid of kBlocksPerSM resident blocks on every SM; the
// launch is timed with CUDA events, best of `reps`.  flops = 2 per multiply-add.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "sph_gb300.h"
#include "sph_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T m, T c, int iters, T *sink)
{
    T acc[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int j = 0; j < kChains; ++j) acc[j] = fma(acc[j], m, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += acc[j];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" sph_status sph_measure_fma_peak(int32_t fp64, int32_t reps, double *gflops, double *best_ms)
{
    if (!gflops || reps < 1) {
        sphg::set_last_error("null gflops or reps < 1");
        return SPH_ERR_ARG;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        sphg::set_last_error("no CUDA device");
        return SPH_ERR_CUDA;
    }
    const int blocks = std::max(sms, 1) * kBlocksPerSM;
    // about 20 ms per launch at the nominal rates (FP64 1.25, FP32 80 TFLOP/s)
    const int iters = fp64 ? 640 : 40000;
    void *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        if (sink) cudaFree(sink);
    };
    if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        sphg::set_last_error("allocation of the measurement buffers failed");
        return SPH_ERR_OOM;
    }
    float best = 1e30f;
    for (int r = 0; r <= reps; ++r) {  // r = 0: warm-up
        cudaEventRecord(e0, st);
        if (fp64) k_fma_chains<double><<<blocks, kThreads, 0, st>>>(1.0000001, 1e-9, iters, (double *)sink);
        else k_fma_chains<float><<<blocks, kThreads, 0, st>>>(1.0000001f, 1e-9f, iters, (float *)sink);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            sphg::set_last_error(cudaGetErrorString(e));
            return SPH_ERR_CUDA;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, ms);
    }
    cleanup();
    const double flops = 2.0 * kChains * 16.0 * (double)iters * (double)blocks * kThreads;
    *gflops = flops / (1e-3 * best) / 1e9;
    if (best_ms) *best_ms = best;
    return SPH_OK;
}
