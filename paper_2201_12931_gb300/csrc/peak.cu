// Arithmetic-peak microbenchmark of the CUDA cores (instrumentation; the
// paper has no counterpart).  The roofline of an ALU-bound kernel needs the
// rate the device actually sustains: every thread of a full-occupancy grid
// (blocks = 8 per SM of 256 threads) runs kChains independent fused
// multiply-add chains for `iters` steps, so the pipe is never idle for a
// dependency; the chains' results are written out so that nothing is
// removed by the compiler.  Flops = 2 per FMA (4 per paired FP32 FMA).
#include <cuda_runtime.h>

#include "common.cuh"

namespace topo {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_f64(int iters, double a, double b, double* out) {
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f32(int iters, float a, float b, float* out) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = __fmaf_rn(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f32x2(int iters, float a, float b, float* out) {
    float2 v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = make_float2(threadIdx.x * 1e-3f + c, c - threadIdx.x * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c].x + v[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace topo

extern "C" topo_status topo_measure_peak(int kind, void* stream, double* tflops_out, double* ms_out) {
    using namespace topo;
    if (kind < 0 || kind > 2 || !tflops_out || !ms_out) {
        set_global_error("topo_measure_peak: kind must be 0, 1 or 2 and the outputs non-NULL");
        return TOPO_BADARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_global_error(cudaGetErrorString(cudaGetLastError()));
        return TOPO_CUDA;
    }
    const int blocks = 8 * nsm, threads = 256;
    // FP64 runs at a small fraction of the FP32 rate: fewer steps, similar time
    const int iters = kind == 0 ? 4096 : 65536;
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    topo_status st = TOPO_OK;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) {
        set_global_error("topo_measure_peak: out of device memory");
        cudaGetLastError();
        return TOPO_OOM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = -1.f;
    for (int rep = 0; rep < 4; ++rep) {   // first launch is a warm-up; best of the other three
        cudaEventRecord(e0, s);
        if (kind == 0) k_peak_f64<<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, (double*)out);
        else if (kind == 1) k_peak_f32<<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)out);
        else k_peak_f32x2<<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)out);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            set_global_error(cudaGetErrorString(cudaGetLastError()));
            st = TOPO_CUDA;
            break;
        }
        if (rep > 0 && (best < 0.f || ms < best)) best = ms;
    }
    if (st == TOPO_OK) {
        const double flops = 2.0 * (kind == 2 ? 2 : 1) * kChains * (double)iters * blocks * threads;
        *ms_out = best;
        *tflops_out = flops / (best * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
