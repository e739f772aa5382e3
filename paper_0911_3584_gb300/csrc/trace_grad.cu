// a4: FP64 traces of block products; a7: gradient assembly on L's pattern.
//
// Traces (N_e = 2 Tr[KS], Sec. 2 condition 2; E = 2 Tr[KH]): for A and B on
// one symmetric pattern, Tr[AB] = sum_p sum_{x,z} A[p][x][z] B[tr p][z][x],
// tr p the block (j, i) of block p = (i, j).  One warp per row sums its blocks
// in FP64 (lanes over blocks, then a fixed butterfly), rows are reduced per
// system by one CTA in a fixed order: the result is run-to-run deterministic.
// FP32 operands are widened to FP64 before they are multiplied (exactly).
//
// Gradient: dE/dL = 6(SLH + HLS) - 4(SLSLH + SLHLS + HLSLS) on L's range.
// With U = SLH (on the R_T pattern), W = SLHLS and Q = HLSLS (on L's
// pattern), SLH^T = HLS and HLSLS^T = SLSLH (S, H, L symmetric), so
//   G_ij = 6 (U_ij + (U_ji)^T) - 4 ((Q_ji)^T + W_ij + Q_ij)
// is formed in FP64 and stored in the value precision.
#include "lnv_impl.cuh"

namespace lnv {
namespace {

template <typename T, int NSF, int NT>
__global__ void __launch_bounds__(256)
k_trace_rows(int64_t n, const int64_t *__restrict__ rp, const int64_t *__restrict__ tr,
             const T *__restrict__ A0, const T *__restrict__ B0, const T *__restrict__ A1,
             const T *__restrict__ B1, const T *__restrict__ A2, const T *__restrict__ B2,
             const T *__restrict__ A3, const T *__restrict__ B3, double *__restrict__ row_part)
{
    constexpr int BS = NSF * NSF;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const T *As[4] = {A0, A1, A2, A3};
    const T *Bs[4] = {B0, B1, B2, B3};
    double s[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) s[t] = 0.0;
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
        const int64_t q = tr[p];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const T *a = As[t] + p * BS;
            const T *b = Bs[t] + q * BS;
#pragma unroll
            for (int x = 0; x < NSF; ++x)
#pragma unroll
                for (int z = 0; z < NSF; ++z)
                    s[t] = fma((double)__ldg(a + x * NSF + z), (double)__ldg(b + z * NSF + x), s[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        double v = s[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) row_part[t * n + i] = v;
    }
}

// out[stride s + offset + t] = sum over the rows of system s of row_part[t][row]
// (seg_off == nullptr: one system holding every row)
__global__ void __launch_bounds__(256)
k_reduce_rows(const double *__restrict__ row_part, int64_t n, int nterms,
              const int64_t *__restrict__ seg_off, double *out, int stride, int offset)
{
    __shared__ double red[256];
    const int s = blockIdx.x, t = blockIdx.y;
    const int64_t b = seg_off ? seg_off[s] : 0, e = seg_off ? seg_off[s + 1] : n;
    double v = 0.0;
    for (int64_t r = b + threadIdx.x; r < e; r += blockDim.x) v += row_part[t * n + r];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(int64_t)stride * s + offset + t] = red[0];
}

// E = 2 Tr[KH] = 2 (3 Tr[LSLH] - 2 Tr[LSLSLH]); N_e = 2 (3 Tr[LSLS] - 2 Tr[LSLSLS]).
__global__ void k_combine(int n_seg, double *out)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_seg) return;
    double t1 = out[6 * s + 2], t2 = out[6 * s + 3], n1 = out[6 * s + 4], n2 = out[6 * s + 5];
    out[6 * s + 0] = 2.0 * (3.0 * t1 - 2.0 * t2);
    out[6 * s + 1] = 2.0 * (3.0 * n1 - 2.0 * n2);
}

template <typename T, int NSF>
__global__ void __launch_bounds__(256)
k_grad(int64_t nnzb, const int64_t *__restrict__ tr, const int64_t *__restrict__ sub,
       const T *__restrict__ U, const T *__restrict__ W, const T *__restrict__ Q, T *__restrict__ G)
{
    constexpr int BS = NSF * NSF;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnzb * BS) return;
    const int64_t p = e / BS;
    const int r = (int)(e - p * BS), x = r / NSF, y = r % NSF;
    const int64_t pt = tr[p];
    const int64_t u1 = sub[p], u2 = sub[pt];
    // L's pattern lies inside U's (R_L < R_T), so both positions exist; a
    // missing block would stand for a zero block.
    double u = (u1 >= 0 ? (double)U[u1 * BS + x * NSF + y] : 0.0) +
               (u2 >= 0 ? (double)U[u2 * BS + y * NSF + x] : 0.0);
    double q = (double)Q[pt * BS + y * NSF + x] + (double)W[p * BS + r] + (double)Q[p * BS + r];
    G[p * BS + r] = (T)(6.0 * u - 4.0 * q);
}

template <typename T, int NSF>
lnv_status trace_launch(lnv_ctx *ctx, const lnv_pattern *P, int nterms, const void *const *A,
                        const void *const *B, double *row_part)
{
    const T *a[4] = {nullptr, nullptr, nullptr, nullptr}, *b[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int t = 0; t < nterms; ++t) {
        a[t] = (const T *)A[t];
        b[t] = (const T *)B[t];
    }
    unsigned grid = (unsigned)((P->n * 32 + 255) / 256);
    if (P->n == 0) return LNV_OK;
    switch (nterms) {
    case 1: k_trace_rows<T, NSF, 1><<<grid, 256, 0, ctx->stream>>>(P->n, P->row_ptr, P->tr, a[0], b[0], a[1], b[1], a[2], b[2], a[3], b[3], row_part); break;
    case 2: k_trace_rows<T, NSF, 2><<<grid, 256, 0, ctx->stream>>>(P->n, P->row_ptr, P->tr, a[0], b[0], a[1], b[1], a[2], b[2], a[3], b[3], row_part); break;
    case 4: k_trace_rows<T, NSF, 4><<<grid, 256, 0, ctx->stream>>>(P->n, P->row_ptr, P->tr, a[0], b[0], a[1], b[1], a[2], b[2], a[3], b[3], row_part); break;
    default: set_error("trace: %d terms not supported", nterms); return LNV_ERR_ARG;
    }
    LNV_LAUNCHED();
    return LNV_OK;
}

template <typename T>
lnv_status trace_nsf(lnv_ctx *ctx, const lnv_pattern *P, int nsf, int nterms, const void *const *A,
                     const void *const *B, double *row_part)
{
    switch (nsf) {
    case 1: return trace_launch<T, 1>(ctx, P, nterms, A, B, row_part);
    case 2: return trace_launch<T, 2>(ctx, P, nterms, A, B, row_part);
    case 4: return trace_launch<T, 4>(ctx, P, nterms, A, B, row_part);
    case 9: return trace_launch<T, 9>(ctx, P, nterms, A, B, row_part);
    default: set_error("NSF=%d is not built (1, 2, 4, 9 are)", nsf); return LNV_ERR_UNSUPPORTED;
    }
}

template <typename T>
lnv_status grad_nsf(lnv_ctx *ctx, const lnv_pattern *PL, const int64_t *sub, int nsf, const void *U,
                    const void *W, const void *Q, void *G)
{
    int64_t total = PL->nnzb * (int64_t)nsf * nsf;
    if (total == 0) return LNV_OK;
    unsigned grid = (unsigned)((total + 255) / 256);
#define GL(N) k_grad<T, N><<<grid, 256, 0, ctx->stream>>>(PL->nnzb, PL->tr, sub, (const T *)U, (const T *)W, (const T *)Q, (T *)G)
    switch (nsf) {
    case 1: GL(1); break;
    case 2: GL(2); break;
    case 4: GL(4); break;
    case 9: GL(9); break;
    default: set_error("NSF=%d is not built (1, 2, 4, 9 are)", nsf); return LNV_ERR_UNSUPPORTED;
    }
#undef GL
    LNV_LAUNCHED();
    return LNV_OK;
}

}  // namespace

lnv_status trace_rows(lnv_ctx *ctx, const lnv_pattern *P, int nsf, lnv_prec prec, int nterms,
                      const void *const *A, const void *const *B, double *row_part)
{
    if (!P->symmetric) {
        set_error("trace needs a symmetric pattern");
        return LNV_ERR_PATTERN;
    }
    if (prec == LNV_FP64) return trace_nsf<double>(ctx, P, nsf, nterms, A, B, row_part);
    if (prec == LNV_FP32) return trace_nsf<float>(ctx, P, nsf, nterms, A, B, row_part);
    set_error("unknown precision %d", (int)prec);
    return LNV_ERR_ARG;
}

lnv_status reduce_rows(lnv_ctx *ctx, const double *row_part, int64_t n, int nterms, int n_seg,
                       const int64_t *seg_off_dev, double *out, int stride, int offset)
{
    dim3 grid((unsigned)n_seg, (unsigned)nterms);
    k_reduce_rows<<<grid, 256, 0, ctx->stream>>>(row_part, n, nterms, seg_off_dev, out, stride, offset);
    LNV_LAUNCHED();
    return LNV_OK;
}

lnv_status lnv_combine(lnv_ctx *ctx, int n_seg, double *out)
{
    k_combine<<<(n_seg + 127) / 128, 128, 0, ctx->stream>>>(n_seg, out);
    LNV_LAUNCHED();
    return LNV_OK;
}

lnv_status grad_assemble(lnv_ctx *ctx, const lnv_pattern *PL, const int64_t *sub_LT, int nsf,
                         lnv_prec prec, const void *U, const void *W, const void *Q, void *G)
{
    if (prec == LNV_FP64) return grad_nsf<double>(ctx, PL, sub_LT, nsf, U, W, Q, G);
    if (prec == LNV_FP32) return grad_nsf<float>(ctx, PL, sub_LT, nsf, U, W, Q, G);
    set_error("unknown precision %d", (int)prec);
    return LNV_ERR_ARG;
}

}  // namespace lnv
