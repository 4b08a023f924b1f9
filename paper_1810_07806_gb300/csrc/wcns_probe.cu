// wcns_probe.cu -- arithmetic-throughput probe (a measurement utility; the
// paper has no counterpart).  Every thread runs independent fused
// multiply-add chains; the rate it reaches is the ALU ceiling the sweep
// kernels are compared with beside the peak derived from unit counts.
#include <cuda_runtime.h>
#include <stdio.h>

#include "../../include/wcns.h"
#include "wcns_internal.h"

namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kIters = 4096;   // multiply-adds per chain

// x <- x * a + b on kChains chains; the results are stored only when they hit
// an impossible value, which keeps the work without writing memory.
__global__ void __launch_bounds__(256) fma_f32(float a, float b, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_f32x2(float a, float b, float* sink)
{
    float2 x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = make_float2((float)(threadIdx.x + k), (float)k);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_f64(double a, double b, float* sink)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < kIters / 16; ++i) {   // the FP64 unit is much slower: fewer iterations
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.2345) sink[blockIdx.x] = (float)s;
}

}  // namespace

extern "C" wcns_status wcns_alu_probe(int kind, double* tflops, void* stream)
{
    using namespace wcns;
    set_last_error(nullptr);
    if (!tflops || kind < 0 || kind > 2) {
        set_last_error("wcns_alu_probe: kind must be 0 (FP32), 1 (packed FP32) or 2 (FP64)");
        return WCNS_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    float* sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void**)&sink, sizeof(float) * blocks);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {   // the first run warms up
        e = cudaEventRecord(e0, s);
        if (kind == 0) fma_f32<<<blocks, threads, 0, s>>>(1.0000001f, 1e-7f, sink);
        else if (kind == 1) fma_f32x2<<<blocks, threads, 0, s>>>(1.0000001f, 1e-7f, sink);
        else fma_f64<<<blocks, threads, 0, s>>>(1.0000000001, 1e-10, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof buf, "wcns_alu_probe: %s", cudaGetErrorString(e));
        set_last_error(buf);
        return WCNS_ERR_CUDA;
    }
    const double iters = kind == 2 ? kIters / 16 : kIters;
    const double lanes = kind == 1 ? 2.0 : 1.0;
    const double flops = 2.0 * lanes * kChains * iters * (double)blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return WCNS_OK;
}
