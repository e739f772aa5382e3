// Kernels of the masked block products; instantiated per (precision, NSF) in
// mult_inst_*.cu so that the library compiles in parallel.
#pragma once
#include <algorithm>

#include "lnv_impl.cuh"

namespace lnv {
namespace prod {

__device__ __forceinline__ int64_t lower_bound_g(const int32_t *__restrict__ col, int64_t lo,
                                                 int64_t hi, int32_t j)
{
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(col + mid) < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// First position >= p whose column is >= j (galloping from p).
__device__ __forceinline__ int64_t gallop_g(const int32_t *__restrict__ col, int64_t p, int64_t hi,
                                            int32_t j)
{
    if (p >= hi || __ldg(col + p) >= j) return p;
    int64_t step = 1, lo = p;
    while (lo + step < hi && __ldg(col + lo + step) < j) {
        lo += step;
        step <<= 1;
    }
    return lower_bound_g(col, lo + 1, min(lo + step + 1, hi), j);
}

__device__ __forceinline__ int lower_bound_s(const int32_t *col, int n, int32_t j)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Element (z, y) of block p of op(B): B[p][z][y], or B[tr][y][z] when transposed.
template <typename T, int NSF, bool TR>
__device__ __forceinline__ void load_row(const T *__restrict__ blk, int z, T (&r)[NSF])
{
#pragma unroll
    for (int y = 0; y < NSF; ++y) r[y] = TR ? __ldg(blk + y * NSF + z) : __ldg(blk + z * NSF + y);
}

// ------------------------------------------------------------------ push

template <typename T, int NSF, int NOUT, bool TA, bool TB>
__global__ void __launch_bounds__(128)
k_push(const int64_t *__restrict__ a_rp, const int32_t *__restrict__ a_col,
       const int64_t *__restrict__ a_tr, const T *__restrict__ a_val,
       const int64_t *__restrict__ b_rp, const int32_t *__restrict__ b_col,
       const int64_t *__restrict__ b_tr, const T *__restrict__ b_val1,
       const T *__restrict__ b_val2, const int64_t *__restrict__ c_rp,
       const int32_t *__restrict__ c_col, T *__restrict__ c_val1, T *__restrict__ c_val2,
       int chunk)
{
    constexpr int BS = NSF * NSF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *acc = reinterpret_cast<T *>(smem_raw);                  // [NOUT][chunk][BS]
    T *a_s = acc + (size_t)NOUT * chunk * BS;                  // [BS]
    int32_t *ccol = reinterpret_cast<int32_t *>(a_s + BS);     // [chunk]

    const int64_t i = blockIdx.x;
    const int64_t cb = c_rp[i], ce = c_rp[i + 1];
    const int64_t ab = a_rp[i], ae = a_rp[i + 1];
    for (int64_t c0 = cb; c0 < ce; c0 += chunk) {
        const int cn = (int)min((int64_t)chunk, ce - c0);
        for (int t = threadIdx.x; t < cn; t += blockDim.x) ccol[t] = c_col[c0 + t];
        for (int t = threadIdx.x; t < NOUT * cn * BS; t += blockDim.x) {
            int o = t / (cn * BS), r = t - o * cn * BS;
            acc[(size_t)o * chunk * BS + r] = T(0);
        }
        __syncthreads();
        const int32_t jlo = ccol[0], jhi = ccol[cn - 1];
        for (int64_t q = ab; q < ae; ++q) {
            const int32_t k = a_col[q];
            if (threadIdx.x < BS) {
                int x = threadIdx.x / NSF, z = threadIdx.x % NSF;
                a_s[threadIdx.x] = TA ? a_val[a_tr[q] * BS + z * NSF + x] : a_val[q * BS + threadIdx.x];
            }
            const int64_t bb = b_rp[k], be = b_rp[k + 1];
            const int64_t lo = lower_bound_g(b_col, bb, be, jlo);
            const int64_t hi = lower_bound_g(b_col, lo, be, jhi + 1);
            __syncthreads();
            for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                const int32_t j = b_col[p];
                const int s = lower_bound_s(ccol, cn, j);
                if (s >= cn || ccol[s] != j) continue;
                const int64_t pb = TB ? b_tr[p] : p;
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    const T *bblk = (o == 0 ? b_val1 : b_val2) + pb * BS;
                    T *ac = acc + ((size_t)o * chunk + s) * BS;
#pragma unroll
                    for (int z = 0; z < NSF; ++z) {
                        T br[NSF];
                        load_row<T, NSF, TB>(bblk, z, br);
#pragma unroll
                        for (int x = 0; x < NSF; ++x) {
                            const T ax = a_s[x * NSF + z];
#pragma unroll
                            for (int y = 0; y < NSF; ++y) ac[x * NSF + y] = fma(ax, br[y], ac[x * NSF + y]);
                        }
                    }
                }
            }
            __syncthreads();
        }
        for (int t = threadIdx.x; t < NOUT * cn * BS; t += blockDim.x) {
            int o = t / (cn * BS), r = t - o * cn * BS;
            T *dst = o == 0 ? c_val1 : c_val2;
            dst[c0 * BS + r] = acc[(size_t)o * chunk * BS + r];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ pull

template <typename T, int NSF, int OPT, bool TA, bool TB>
__global__ void __launch_bounds__(128)
k_pull(const int64_t *__restrict__ a_rp, const int32_t *__restrict__ a_col,
       const int64_t *__restrict__ a_tr, const T *__restrict__ a_val,
       const int64_t *__restrict__ b_rp, const int32_t *__restrict__ b_col,
       const int64_t *__restrict__ b_tr, const T *__restrict__ b_val,
       const int64_t *__restrict__ c_rp, const int32_t *__restrict__ c_col, T *__restrict__ c_val,
       int kchunk)
{
    constexpr int BS = NSF * NSF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *a_s = reinterpret_cast<T *>(smem_raw);                    // [kchunk][BS]
    int32_t *a_k = reinterpret_cast<int32_t *>(a_s + (size_t)kchunk * BS);  // [kchunk]

    const int64_t i = blockIdx.x;
    const int64_t cb = c_rp[i], ce = c_rp[i + 1];
    const int64_t ab = a_rp[i], ae = a_rp[i + 1];
    const int nc = (int)(ce - cb);
    const int per_pass = blockDim.x * OPT;
    for (int g0 = 0; g0 < nc; g0 += per_pass) {
        const int s0 = g0 + threadIdx.x * OPT;
        int nmine = min(OPT, nc - s0);
        if (nmine < 0) nmine = 0;
        int32_t jj[OPT];
#pragma unroll
        for (int o = 0; o < OPT; ++o) jj[o] = o < nmine ? c_col[cb + s0 + o] : 0;
        T acc[OPT][BS];
#pragma unroll
        for (int o = 0; o < OPT; ++o)
#pragma unroll
            for (int e = 0; e < BS; ++e) acc[o][e] = T(0);

        for (int64_t k0 = ab; k0 < ae; k0 += kchunk) {
            const int kn = (int)min((int64_t)kchunk, ae - k0);
            __syncthreads();
            for (int t = threadIdx.x; t < kn * BS; t += blockDim.x) {
                int qq = t / BS, e = t - qq * BS;
                int64_t q = k0 + qq;
                if (TA) {
                    int x = e / NSF, z = e % NSF;
                    a_s[t] = a_val[a_tr[q] * BS + z * NSF + x];
                } else {
                    a_s[t] = a_val[q * BS + e];
                }
            }
            for (int t = threadIdx.x; t < kn; t += blockDim.x) a_k[t] = a_col[k0 + t];
            __syncthreads();
            if (nmine == 0) continue;
            for (int qq = 0; qq < kn; ++qq) {
                const int32_t k = a_k[qq];
                const int64_t be = b_rp[k + 1];
                int64_t p = lower_bound_g(b_col, b_rp[k], be, jj[0]);
                const T *as = a_s + (size_t)qq * BS;
#pragma unroll
                for (int o = 0; o < OPT; ++o) {
                    if (o >= nmine) break;
                    if (o > 0) p = gallop_g(b_col, p, be, jj[o]);
                    if (p >= be) break;
                    if (__ldg(b_col + p) != jj[o]) continue;
                    const T *bblk = b_val + (TB ? b_tr[p] : p) * BS;
#pragma unroll
                    for (int z = 0; z < NSF; ++z) {
                        T br[NSF];
                        load_row<T, NSF, TB>(bblk, z, br);
#pragma unroll
                        for (int x = 0; x < NSF; ++x) {
                            const T ax = as[x * NSF + z];
#pragma unroll
                            for (int y = 0; y < NSF; ++y)
                                acc[o][x * NSF + y] = fma(ax, br[y], acc[o][x * NSF + y]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int o = 0; o < OPT; ++o) {
            if (o >= nmine) break;
            T *dst = c_val + (cb + s0 + o) * BS;
#pragma unroll
            for (int e = 0; e < BS; ++e) dst[e] = acc[o][e];
        }
    }
}

// ------------------------------------------------------------------ launch

constexpr int kThreads = 128;

template <typename T, int NSF>
constexpr int pull_opt()
{
    return NSF >= 9 ? 1 : (sizeof(T) == 8 ? 2 : (NSF <= 2 ? 4 : 4));
}

template <typename T, int NSF, int NOUT, bool TA, bool TB>
lnv_status launch_push(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1,
                       const void *B2, void *C1, void *C2)
{
    constexpr int BS = NSF * NSF;
    const lnv_pattern *PA = pl->A, *PB = pl->B, *PC = pl->C;
    if (PC->n == 0) return LNV_OK;
    size_t budget = std::min<size_t>(ctx->smem_optin, 96 * 1024);
    size_t per_slot = (size_t)NOUT * BS * sizeof(T) + sizeof(int32_t);
    size_t fixed = BS * sizeof(T) + 64;
    int chunk = (int)std::min<size_t>((budget - fixed) / per_slot, (size_t)std::max(pl->max_c_row, 1));
    if (chunk < 1) {
        set_error("push product: shared memory too small for one block");
        return LNV_ERR_UNSUPPORTED;
    }
    size_t smem = (size_t)NOUT * chunk * BS * sizeof(T) + BS * sizeof(T) + sizeof(int32_t) * chunk + 16;
    auto kern = k_push<T, NSF, NOUT, TA, TB>;
    LNV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)PC->n, kThreads, smem, ctx->stream>>>(
        PA->row_ptr, PA->col, PA->tr, (const T *)A, PB->row_ptr, PB->col, PB->tr, (const T *)B1,
        (const T *)B2, PC->row_ptr, PC->col, (T *)C1, (T *)C2, chunk);
    LNV_LAUNCHED();
    return LNV_OK;
}

template <typename T, int NSF, bool TA, bool TB>
lnv_status launch_pull(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B, void *C)
{
    constexpr int BS = NSF * NSF;
    constexpr int OPT = pull_opt<T, NSF>();
    const lnv_pattern *PA = pl->A, *PB = pl->B, *PC = pl->C;
    if (PC->n == 0) return LNV_OK;
    size_t budget = std::min<size_t>(ctx->smem_optin, 64 * 1024);
    size_t per_k = BS * sizeof(T) + sizeof(int32_t);
    int kchunk = (int)std::min<size_t>(budget / per_k, (size_t)std::max(pl->max_a_row, 1));
    size_t smem = (size_t)kchunk * per_k + 16;
    auto kern = k_pull<T, NSF, OPT, TA, TB>;
    LNV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)PC->n, kThreads, smem, ctx->stream>>>(
        PA->row_ptr, PA->col, PA->tr, (const T *)A, PB->row_ptr, PB->col, PB->tr, (const T *)B,
        PC->row_ptr, PC->col, (T *)C, kchunk);
    LNV_LAUNCHED();
    return LNV_OK;
}

template <typename T, int NSF, bool TA, bool TB>
lnv_status dispatch_mode(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1,
                         const void *B2, void *C1, void *C2)
{
    if (pl->mode == 0) {
        if (B2) return launch_push<T, NSF, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2);
        return launch_push<T, NSF, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr);
    }
    LNV_TRY((launch_pull<T, NSF, TA, TB>(ctx, pl, A, B1, C1)));
    if (B2) LNV_TRY((launch_pull<T, NSF, TA, TB>(ctx, pl, A, B2, C2)));
    return LNV_OK;
}

template <typename T, int NSF>
lnv_status dispatch_trans(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1,
                          const void *B2, void *C1, void *C2)
{
    if (pl->trans_a && pl->trans_b) return dispatch_mode<T, NSF, true, true>(ctx, pl, A, B1, B2, C1, C2);
    if (pl->trans_a) return dispatch_mode<T, NSF, true, false>(ctx, pl, A, B1, B2, C1, C2);
    if (pl->trans_b) return dispatch_mode<T, NSF, false, true>(ctx, pl, A, B1, B2, C1, C2);
    return dispatch_mode<T, NSF, false, false>(ctx, pl, A, B1, B2, C1, C2);
}

}  // namespace prod
}  // namespace lnv

#define LNV_PROD_EXTERN(T, N)                                                                     \
    extern template lnv_status lnv::prod::dispatch_trans<T, N>(lnv_ctx *, const lnv_plan *,       \
                                                               const void *, const void *,      \
                                                               const void *, void *, void *);
LNV_PROD_EXTERN(double, 1)
LNV_PROD_EXTERN(double, 2)
LNV_PROD_EXTERN(double, 4)
LNV_PROD_EXTERN(double, 9)
LNV_PROD_EXTERN(float, 1)
LNV_PROD_EXTERN(float, 2)
LNV_PROD_EXTERN(float, 4)
LNV_PROD_EXTERN(float, 9)
#undef LNV_PROD_EXTERN
