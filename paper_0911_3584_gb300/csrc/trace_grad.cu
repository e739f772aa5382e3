// a4: FP64 traces of block products; a7: gradient assembly on L's pattern.
//
// Traces (N_e = 2 Tr[KS], Sec. 2 condition 2; E = 2 Tr[KH]): for A and B on
// one symmetric pattern, Tr[AB] = sum_p sum_{x,z} A[p][x][z] B[tr p][z][x],
// tr p the block (j, i) of block p = (i, j).  One warp per row sums its blocks
// in FP64 (lanes over blocks, then a fixed butterfly), rows are reduced per
// system by one CTA in a fixed order: the result is run-to-run deterministic.
// The generic kernel widens FP32 operands to FP64 before multiplying
// (exactly); the fused four-trace kernels (NSF = 4 and 9) form each block's
// dot products in the value precision and sum the blocks in FP64.
//
// Gradient: dE/dL = 6(SLH + HLS) - 4(SLSLH + SLHLS + HLSLS) on L's range.
// With U = SLH (on the R_T pattern), W = SLHLS (symmetric, kept on the upper
// triangle of L's pattern) and Q = HLSLS (on L's pattern), SLH^T = HLS and
// HLSLS^T = SLSLH (S, H, L symmetric), so
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

// The four traces of one evaluation in one pass (NSF = 4): for block p = (i, j)
// of the R_X pattern and q = (j, i), t1 += <X_p, Y_q^T>, t2 += <Z_p, Y_q^T>,
// n1 += <X_p, X_q^T>, n2 += <Z_p, X_q^T>; each of X_p, Z_p, X_q, Y_q is loaded
// once, 16 bytes at a time.  One warp per row, FP64 sums over blocks, fixed
// butterfly.
template <typename T>
__device__ __forceinline__ void ld_blk4(const T *__restrict__ p, T (&b)[16])
{
    if constexpr (sizeof(T) == 4) {
        const float4 *v = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float4 q = __ldg(v + r);
            b[4 * r] = q.x; b[4 * r + 1] = q.y; b[4 * r + 2] = q.z; b[4 * r + 3] = q.w;
        }
    } else {
        const double2 *v = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const double2 q = __ldg(v + r);
            b[2 * r] = q.x; b[2 * r + 1] = q.y;
        }
    }
}

// Each block pair's 16-term dot products are formed in the value precision
// (T), then accumulated across blocks in FP64: for FP32 values this keeps the
// trace reduction in FP64 with one conversion per block pair and term.
template <typename T>
__global__ void __launch_bounds__(256)
k_trace_lnv4(int64_t n, const int64_t *__restrict__ rp, const int64_t *__restrict__ tr,
             const T *__restrict__ X, const T *__restrict__ Y, const T *__restrict__ Z,
             double *__restrict__ row_part)
{
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double t1 = 0.0, t2 = 0.0, n1 = 0.0, n2 = 0.0;
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
        const int64_t q = __ldg(tr + p);
        T xp[16], zp[16], xq[16], yq[16];
        ld_blk4<T>(X + p * 16, xp);
        ld_blk4<T>(Z + p * 16, zp);
        ld_blk4<T>(X + q * 16, xq);
        ld_blk4<T>(Y + q * 16, yq);
        T a1 = T(0), a2 = T(0), a3 = T(0), a4 = T(0);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int z = 0; z < 4; ++z) {
                const T a = xp[x * 4 + z], c = zp[x * 4 + z];
                const T by = yq[z * 4 + x], bx = xq[z * 4 + x];
                a1 = fma(a, by, a1);
                a2 = fma(c, by, a2);
                a3 = fma(a, bx, a3);
                a4 = fma(c, bx, a4);
            }
        t1 += (double)a1;
        t2 += (double)a2;
        n1 += (double)a3;
        n2 += (double)a4;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        t2 += __shfl_xor_sync(0xffffffffu, t2, o);
        n1 += __shfl_xor_sync(0xffffffffu, n1, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if (lane == 0) {
        row_part[i] = t1;
        row_part[n + i] = t2;
        row_part[2 * n + i] = n1;
        row_part[3 * n + i] = n2;
    }
}

// The same four traces with 9 x 9 blocks.  One warp per row takes the row's
// blocks one after another, the 81 elements of a block over its lanes
// (lane e holds e, e + 32, e + 64): X_p and Z_p are read in order, the
// partner blocks X_q and Y_q (q = tr p) at the transposed index 9 z + x,
// so every load of the warp covers one block.  Four blocks are loaded
// before any is used; each lane's share of their four dot products (12
// products per trace) is formed in the value precision and added to FP64
// sums; a fixed butterfly ends the row.
template <typename T>
__global__ void __launch_bounds__(256)
k_trace_lnv9(int64_t n, const int64_t *__restrict__ rp, const int64_t *__restrict__ tr,
             const T *__restrict__ X, const T *__restrict__ Y, const T *__restrict__ Z,
             double *__restrict__ row_part)
{
    constexpr int BS = 81, U = 4;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    int e[3], et[3];
    bool ev[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e[c] = lane + 32 * c;
        ev[c] = e[c] < BS;
        const int x = e[c] / 9, z = e[c] - 9 * x;
        e[c] = ev[c] ? e[c] : 0;
        et[c] = ev[c] ? 9 * z + x : 0;
    }
    double t1 = 0.0, t2 = 0.0, n1 = 0.0, n2 = 0.0;
    const int64_t p0 = rp[i], p1 = rp[i + 1];
    for (int64_t pb = p0; pb < p1; pb += U) {
        T xp[U][3], zp[U][3], xq[U][3], yq[U][3];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t p = pb + u;
            const bool pv = p < p1;
            const int64_t q = pv ? __ldg(tr + p) : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool v = pv && ev[c];
                xp[u][c] = v ? __ldg(X + p * BS + e[c]) : T(0);
                zp[u][c] = v ? __ldg(Z + p * BS + e[c]) : T(0);
                xq[u][c] = v ? __ldg(X + q * BS + et[c]) : T(0);
                yq[u][c] = v ? __ldg(Y + q * BS + et[c]) : T(0);
            }
        }
        // a lane's 12 products of the four blocks per trace in the value
        // precision, then one FP64 addition
        T a1 = T(0), a2 = T(0), a3 = T(0), a4 = T(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a1 = fma(xp[u][c], yq[u][c], a1);
                a2 = fma(zp[u][c], yq[u][c], a2);
                a3 = fma(xp[u][c], xq[u][c], a3);
                a4 = fma(zp[u][c], xq[u][c], a4);
            }
        t1 += (double)a1;
        t2 += (double)a2;
        n1 += (double)a3;
        n2 += (double)a4;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        t2 += __shfl_xor_sync(0xffffffffu, t2, o);
        n1 += __shfl_xor_sync(0xffffffffu, n1, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if (lane == 0) {
        row_part[i] = t1;
        row_part[n + i] = t2;
        row_part[2 * n + i] = n1;
        row_part[3 * n + i] = n2;
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
k_grad(int64_t nnzb, const int64_t *__restrict__ tr, const int32_t *__restrict__ row,
       const int32_t *__restrict__ col, const int64_t *__restrict__ sub, const int64_t *__restrict__ wmap,
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
    // W = SLHLS is symmetric and stored on the upper triangle: W_ij = (W_ji)^T
    const int64_t wp = wmap[p];
    const double w = col[p] >= row[p] ? (double)W[wp * BS + r] : (double)W[wp * BS + y * NSF + x];
    double q = (double)Q[pt * BS + y * NSF + x] + w + (double)Q[p * BS + r];
    G[p * BS + r] = (T)(6.0 * u - 4.0 * q);
}

// dN_e/dL = 12 (SLS - SLSLS) on L's pattern (N_e = 2 Tr[KS] with Eq. 3, every
// stored entry of L independent, S and L symmetric): T = SLS read through the
// submap of L's pattern in T's, V = S Z = SLSLS formed on L's pattern.
template <typename T, int NSF>
__global__ void __launch_bounds__(256)
k_grad_ne(int64_t nnzb, const int64_t *__restrict__ sub, const T *__restrict__ Tm, const T *__restrict__ V,
          T *__restrict__ GN)
{
    constexpr int BS = NSF * NSF;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnzb * BS) return;
    const int64_t p = e / BS;
    const int r = (int)(e - p * BS);
    const int64_t pt = sub[p];
    const double t = pt >= 0 ? (double)Tm[pt * BS + r] : 0.0;
    GN[p * BS + r] = (T)(12.0 * (t - (double)V[p * BS + r]));
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
lnv_status grad_nsf(lnv_ctx *ctx, const lnv_pattern *PL, const int64_t *sub, const int64_t *wmap, int nsf,
                    const void *U, const void *W, const void *Q, void *G)
{
    int64_t total = PL->nnzb * (int64_t)nsf * nsf;
    if (total == 0) return LNV_OK;
    unsigned grid = (unsigned)((total + 255) / 256);
#define GL(N) k_grad<T, N><<<grid, 256, 0, ctx->stream>>>(PL->nnzb, PL->tr, PL->row, PL->col, sub, wmap, (const T *)U, (const T *)W, (const T *)Q, (T *)G)
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
    // the LNV four-trace pass {X, Z, X, Z} x {Y, Y, X, X} with 4x4 or 9x9 blocks
    if (nterms == 4 && (nsf == 4 || nsf == 9) && A[0] == A[2] && A[1] == A[3] && B[0] == B[1] && B[2] == B[3] &&
        B[2] == A[0] && P->n > 0) {
        const unsigned grid = (unsigned)((P->n * 32 + 255) / 256);
        if (nsf == 4 && prec == LNV_FP64)
            k_trace_lnv4<double><<<grid, 256, 0, ctx->stream>>>(P->n, P->row_ptr, P->tr, (const double *)A[0],
                                                                (const double *)B[0], (const double *)A[1], row_part);
        else if (nsf == 4)
            k_trace_lnv4<float><<<grid, 256, 0, ctx->stream>>>(P->n, P->row_ptr, P->tr, (const float *)A[0],
                                                               (const float *)B[0], (const float *)A[1], row_part);
        else if (prec == LNV_FP64)
            k_trace_lnv9<double><<<grid, 256, 0, ctx->stream>>>(P->n, P->row_ptr, P->tr, (const double *)A[0],
                                                                (const double *)B[0], (const double *)A[1], row_part);
        else
            k_trace_lnv9<float><<<grid, 256, 0, ctx->stream>>>(P->n, P->row_ptr, P->tr, (const float *)A[0],
                                                               (const float *)B[0], (const float *)A[1], row_part);
        LNV_LAUNCHED();
        return LNV_OK;
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

lnv_status grad_ne_assemble(lnv_ctx *ctx, const lnv_pattern *PL, const int64_t *sub_LT, int nsf,
                            lnv_prec prec, const void *T, const void *V, void *GN)
{
    const int64_t total = PL->nnzb * (int64_t)nsf * nsf;
    if (total == 0) return LNV_OK;
    const unsigned grid = (unsigned)((total + 255) / 256);
#define GN_L(TY, N)                                                                                   \
    k_grad_ne<TY, N><<<grid, 256, 0, ctx->stream>>>(PL->nnzb, sub_LT, (const TY *)T, (const TY *)V, \
                                                    (TY *)GN)
    if (prec != LNV_FP64 && prec != LNV_FP32) {
        set_error("unknown precision %d", (int)prec);
        return LNV_ERR_ARG;
    }
    const bool f64 = prec == LNV_FP64;
    switch (nsf) {
    case 1: if (f64) GN_L(double, 1); else GN_L(float, 1); break;
    case 2: if (f64) GN_L(double, 2); else GN_L(float, 2); break;
    case 4: if (f64) GN_L(double, 4); else GN_L(float, 4); break;
    case 9: if (f64) GN_L(double, 9); else GN_L(float, 9); break;
    default: set_error("NSF=%d is not built (1, 2, 4, 9 are)", nsf); return LNV_ERR_UNSUPPORTED;
    }
#undef GN_L
    LNV_LAUNCHED();
    return LNV_OK;
}

lnv_status grad_assemble(lnv_ctx *ctx, const lnv_pattern *PL, const int64_t *sub_LT,
                         const int64_t *w_map, int nsf, lnv_prec prec, const void *U, const void *W,
                         const void *Q, void *G)
{
    if (prec == LNV_FP64) return grad_nsf<double>(ctx, PL, sub_LT, w_map, nsf, U, W, Q, G);
    if (prec == LNV_FP32) return grad_nsf<float>(ctx, PL, sub_LT, w_map, nsf, U, W, Q, G);
    set_error("unknown precision %d", (int)prec);
    return LNV_ERR_ARG;
}

}  // namespace lnv
