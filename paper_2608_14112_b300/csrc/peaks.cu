// peaks.cu -- throughput microbenchmarks of the pipes the evaluator runs on:
// scalar float32 FMA (FFMA), packed float32x2 FMA (fma.rn.f32x2, two lanes
// of arithmetic per instruction) and the SFU exponential (ex2.approx).  They
// give the measured denominators of the roofline fractions: the path is not a
// dense contraction, so its ceiling is the FP32 / SFU issue rate, not a
// tensor-core or HBM figure.
//
// Each thread runs kChains independent dependency chains (enough independent
// work per warp to hide the pipe latency with 16 warps per SM) for `iters`
// rounds; the grid is 8 CTAs of 256 threads per SM, resident at once.  The
// chains' results feed one conditional store that never happens for finite
// inputs, so nothing is dead code.  Operations are counted per lane: one FMA
// = 1, one packed FMA = 2, one ex2 = 1.
#include "gve_int.cuh"

namespace gve {

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_peak_ffma(long long iters, float a, float b, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_ffma2(long long iters, float a, float b, float* sink)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_ex2(long long iters, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -(float)(threadIdx.x + c) * 1e-3f;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = ex2_approx(-x[c]);   // stays in (1/2, 1]
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

}  // namespace

}  // namespace gve

using namespace gve;

extern "C" gve_status gve_peak_bench(int32_t kind, int64_t iters, double* ops_per_s, float* ms_out, void* stream)
{
    if (kind < 0 || kind > 2 || iters < 1 || iters > (int64_t)1 << 40 || !ops_per_s) return GVE_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = 8 * num_sms();
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gve_status st = GVE_OK;
    if (cudaMalloc(&sink, 256 * sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        st = GVE_E_CUDA;
    } else {
        cudaEventRecord(e0, s);
        if (kind == 0) k_peak_ffma<<<blocks, 256, 0, s>>>(iters, 0.999f, 1e-3f, sink);
        else if (kind == 1) k_peak_ffma2<<<blocks, 256, 0, s>>>(iters, 0.999f, 1e-3f, sink);
        else k_peak_ex2<<<blocks, 256, 0, s>>>(iters, sink);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
            st = GVE_E_CUDA;
        } else {
            const double lanes = (double)blocks * 256.0 * (double)iters * kUnroll * kChains;
            *ops_per_s = lanes * (kind == 1 ? 2.0 : 1.0) / (ms * 1e-3);
            if (ms_out) *ms_out = ms;
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return st;
}
