// lnv_trace_product_noalloc: Tr[A B] without any device allocation.
//
// lnv_trace_product needs n doubles of caller-provided scratch for its
// per-row partial sums.  Some callers cannot provide it: code that runs under
// a fixed device-memory budget managed by its own pool (where a stray
// cudaMalloc fails or breaks the budget), or a host program whose interface
// has no place to pass a scratch buffer through.  This variant keeps the
// partial sums in a file-scope device array instead.
//
// The array holds kNoAllocMaxRows doubles (2 MiB).  Every GPU that loads this
// library holds it until the process exits.  All calls on one device share
// it, so calls whose kernels overlap on the GPU (different streams, or
// different host threads) race and give wrong sums; serialise them.  The
// trace kernel writes the partial sum of every row before the reduction
// reads it, so nothing left from an earlier call is ever read and no
// clearing is needed.
#include <mutex>

#include "lnv_impl.cuh"

namespace {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 18;  // 262144 rows
constexpr int kMaxDevices = 128;

static __device__ __align__(256) double g_trace_scratch[kNoAllocMaxRows];

std::mutex g_scratch_mu;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of g_trace_scratch on the current device (ctx->device).  In
// host code the array's name is only a host-side stand-in and must never be
// passed to a kernel.  The address is looked up again on every call made
// outside a stream capture (so it stays right after cudaDeviceReset, which
// gives the array a new address in the new context) and cached for calls
// made during a capture, where the lookup is not allowed.
lnv_status scratch_address(int device, bool refresh, double **out)
{
    if (device < 0 || device >= kMaxDevices) {
        lnv::set_error("device index %d is beyond the %d devices this entry point supports",
                       device, kMaxDevices);
        return LNV_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (refresh || !g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_trace_scratch);
        if (e != cudaSuccess || !p) {
            lnv::set_error("cudaGetSymbolAddress of the trace scratch array failed: %s",
                           cudaGetErrorString(e));
            return LNV_ERR_CUDA;
        }
        g_scratch_addr[device] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[device];
    return LNV_OK;
}

}  // namespace

extern "C" lnv_status lnv_trace_product_noalloc(lnv_ctx *ctx, const lnv_pattern *P, int nsf,
                                                lnv_prec prec, const void *A_dev,
                                                const void *B_dev, double *out_dev)
{
    LNV_ARG(ctx && P && A_dev && B_dev && out_dev, "null pointer");
    LNV_ARG((((uintptr_t)A_dev | (uintptr_t)B_dev) & 15u) == 0, "value arrays must be 16-byte aligned");
    if (P->n > kNoAllocMaxRows) {
        lnv::set_error("lnv_trace_product_noalloc: pattern has %lld rows, the built-in scratch "
                       "holds at most %lld; use lnv_trace_product with caller scratch",
                       (long long)P->n, (long long)kNoAllocMaxRows);
        return LNV_ERR_UNSUPPORTED;
    }
    LNV_CUDA(cudaSetDevice(ctx->device));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LNV_CUDA(cudaStreamIsCapturing(ctx->stream, &cs));
    double *scratch = nullptr;
    LNV_TRY(scratch_address(ctx->device, cs == cudaStreamCaptureStatusNone, &scratch));
    const void *A[1] = {A_dev}, *B[1] = {B_dev};
    LNV_TRY(lnv::trace_rows(ctx, P, nsf, prec, 1, A, B, scratch));
    return lnv::reduce_rows(ctx, scratch, P->n, 1, 1, nullptr, out_dev, 1, 0);
}
