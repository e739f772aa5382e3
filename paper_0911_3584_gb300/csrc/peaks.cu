// Measured ALU rates of this GPU, for the rooflines of the SIMT products.
//
// The FP32 and FP64 products are bound by the fused multiply-add pipes, whose
// nominal rates follow from the SM count and clock (FP32: 128 lanes x 2 flop
// per clock per SM; FP64: 4 flop per clock per SM on GB300).  This probe
// measures what a kernel can actually issue: every thread runs eight
// independent FMA chains, enough warps per SM to hide the pipe latency, and
// the best of a few CUDA-event timed launches is reported.
#include <algorithm>

#include "lnv_impl.cuh"

namespace lnv {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T *out, int iters, T mul, T add)
{
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], mul, add);
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    // one store per thread keeps the chains live
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
lnv_status fma_rate(lnv_ctx *ctx, int iters, double *tflops)
{
    const int blocks = ctx->sm_count * 8, threads = 256;
    T *out = nullptr;
    LNV_CUDA(cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, ctx->stream);
        if (e == cudaSuccess) {
            k_fma_chains<T><<<blocks, threads, 0, ctx->stream>>>(out, iters, (T)0.999, (T)1e-4);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;  // rep 0 warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) {
        set_error("FMA probe: %s", cudaGetErrorString(e));
        return LNV_ERR_CUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return LNV_OK;
}

}  // namespace
}  // namespace lnv

extern "C" lnv_status lnv_probe_fma_rate(lnv_ctx *ctx, lnv_prec prec, double *tflops)
{
    LNV_ARG(ctx && tflops, "null pointer");
    LNV_ARG(prec == LNV_FP64 || prec == LNV_FP32, "unknown precision");
    LNV_CUDA(cudaSetDevice(ctx->device));
    return prec == LNV_FP64 ? lnv::fma_rate<double>(ctx, 256, tflops) : lnv::fma_rate<float>(ctx, 4096, tflops);
}
