// a1-a3, a5, a6: range-truncated block-sparse products C = mask_C(op(A) op(B)).
//
// The paper names sparse matrix multiplication as the main computational load
// (Sec. 3) and K = 3LSL - 2LSLSL (Eq. 3) as the quantity built from it.  Each
// product keeps only the blocks of C's range pattern.  This file holds the
// symbolic pass, the plans and the dispatch; the kernels are in
// mult_kernels.cuh:
//
//  0  push: one CTA per (output row, column chunk), the chunk accumulated in
//     shared memory; warps own column slices, so no two lanes touch one slot
//     within a k.  Best for full-range products (X = LS, T = SX) in FP64.
//  1  pull with a binary search per k; 2 pull with a merge-join walk of B's
//     row j (symmetric B): output owners, for narrow C rows.
//  3, 4  row groups of 4 rows (position table or hit lists): one fetch of
//     op(B)_kj serves every row of the group holding A_ik.
//  5, 8  row groups with independent warps, per-warp k lists and a cp.async
//     ring (FP32, NSF = 4); kernel 8 with warp slices of half the width.
//  6  row groups on TF32 tensor cores (mma.sync, hi/lo split).
//  7  listed triples: per output block its (A, B) pairs, listed once per plan.
//  9  row groups of 8 rows as dense tiles on the tcgen05 tensor cores (umma.cu):
//     FP32 values, NSF = 4, op(B) = B^T, split-TF32 operands.
//  10 the same for NSF = 9 (umma9.cu): row groups of 7 rows, tiles of 14
//     output columns, either op(B).
//
// A product declared symmetric (LNV_SYM_C, T = SLS) may be formed on its
// upper triangle and mirrored (mirror_lower).  Sums are formed in k order in
// every kernel (deterministic).  Operand transposes (op = ^T) read block
// (k, i) through the pattern's transpose map.
#include <algorithm>
#include <type_traits>
#include <cstring>
#include <vector>

#include "mult_kernels.cuh"

namespace lnv {
namespace {

using prod::lower_bound_g;
using prod::dispatch_trans;

// ------------------------------------------------------------------ symbolic

// Per row i: contributing triples, push scan length, pull candidates.
template <bool TA, bool TB>
__global__ void k_symbolic(int64_t n, const int64_t *__restrict__ a_rp,
                           const int32_t *__restrict__ a_col, const int64_t *__restrict__ b_rp,
                           const int32_t *__restrict__ b_col, const int64_t *__restrict__ c_rp,
                           const int32_t *__restrict__ c_col, unsigned long long *counts)
{
    // one CTA per row; threads over C's row
    const int64_t i = blockIdx.x;
    if (i >= n) return;
    const int64_t cb = c_rp[i], ce = c_rp[i + 1], ab = a_rp[i], ae = a_rp[i + 1];
    unsigned long long trip = 0, trip_up = 0, scan = 0;
    for (int64_t s = cb + threadIdx.x; s < ce; s += blockDim.x) {
        int32_t j = c_col[s];
        unsigned long long t = 0;
        for (int64_t q = ab; q < ae; ++q) {
            int32_t k = a_col[q];
            int64_t bb = b_rp[k], be = b_rp[k + 1];
            int64_t p = lower_bound_g(b_col, bb, be, j);
            if (p < be && b_col[p] == j) ++t;
        }
        trip += t;
        if (j >= i) trip_up += t;
    }
    if (threadIdx.x == 0)
        for (int64_t q = ab; q < ae; ++q) scan += (unsigned long long)(b_rp[a_col[q] + 1] - b_rp[a_col[q]]);
    atomicAdd(&counts[0], trip);
    atomicAdd(&counts[3], trip_up);
    if (threadIdx.x == 0) {
        atomicAdd(&counts[1], scan);
        atomicAdd(&counts[2], (unsigned long long)((ae - ab) * (ce - cb)));
    }
}

// Strict lower triangle of a symmetric-valued matrix from its upper triangle,
// one thread per block: block p = (i, j) with j < i becomes the transpose of
// block tr[p] = (j, i), and a diagonal block's elements (a, b), a > b, become
// its elements (b, a).  Every element read lies on or above the diagonal, and
// none of those is written.
template <typename T, int NSF>
__global__ void k_mirror_lower(int64_t nnzb, const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                               const int64_t *__restrict__ tr, T *vals)
{
    constexpr int BS = NSF * NSF;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnzb; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = __ldg(row + p), j = __ldg(col + p);
        if (j > i) continue;
        T *dst = vals + p * BS;
        if (j == i) {
#pragma unroll
            for (int a = 1; a < NSF; ++a)
#pragma unroll
                for (int b = 0; b < a; ++b) dst[a * NSF + b] = dst[b * NSF + a];
            continue;
        }
        const T *src = vals + __ldg(tr + p) * BS;
        T blk[BS];
        if constexpr (NSF == 4) {
            // 16-byte loads and stores (blocks start on 64- or 128-byte boundaries)
            constexpr int V = 16 / sizeof(T);
            using Vec = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
#pragma unroll
            for (int e = 0; e < BS; e += V) *reinterpret_cast<Vec *>(blk + e) = *reinterpret_cast<const Vec *>(src + e);
            T out[BS];
#pragma unroll
            for (int a = 0; a < NSF; ++a)
#pragma unroll
                for (int b = 0; b < NSF; ++b) out[a * NSF + b] = blk[b * NSF + a];
#pragma unroll
            for (int e = 0; e < BS; e += V) *reinterpret_cast<Vec *>(dst + e) = *reinterpret_cast<const Vec *>(out + e);
        } else {
#pragma unroll
            for (int e = 0; e < BS; ++e) blk[e] = src[e];
#pragma unroll
            for (int a = 0; a < NSF; ++a)
#pragma unroll
                for (int b = 0; b < NSF; ++b) dst[a * NSF + b] = blk[b * NSF + a];
        }
    }
}

template <typename T>
lnv_status mirror_launch(lnv_ctx *ctx, const lnv_pattern *P, int nsf, T *vals)
{
    // one block per thread: as many loads in flight as the pattern has blocks
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(1 << 30, (P->nnzb + 255) / 256));
    switch (nsf) {
    case 1: k_mirror_lower<T, 1><<<grid, 256, 0, ctx->stream>>>(P->nnzb, P->row, P->col, P->tr, vals); break;
    case 2: k_mirror_lower<T, 2><<<grid, 256, 0, ctx->stream>>>(P->nnzb, P->row, P->col, P->tr, vals); break;
    case 4: k_mirror_lower<T, 4><<<grid, 256, 0, ctx->stream>>>(P->nnzb, P->row, P->col, P->tr, vals); break;
    case 9: k_mirror_lower<T, 9><<<grid, 256, 0, ctx->stream>>>(P->nnzb, P->row, P->col, P->tr, vals); break;
    default:
        set_error("NSF=%d is not built (1, 2, 4, 9 are)", nsf);
        return LNV_ERR_UNSUPPORTED;
    }
    LNV_LAUNCHED();
    return LNV_OK;
}

template <typename T>
lnv_status dispatch_nsf(lnv_ctx *ctx, const lnv_plan *pl, int nsf, const void *A, const void *B1,
                        const void *B2, void *C1, void *C2)
{
    switch (nsf) {
    case 1: return dispatch_trans<T, 1>(ctx, pl, A, B1, B2, C1, C2);
    case 2: return dispatch_trans<T, 2>(ctx, pl, A, B1, B2, C1, C2);
    case 4: return dispatch_trans<T, 4>(ctx, pl, A, B1, B2, C1, C2);
    case 9: return dispatch_trans<T, 9>(ctx, pl, A, B1, B2, C1, C2);
    default:
        set_error("NSF=%d is not built (1, 2, 4, 9 are)", nsf);
        return LNV_ERR_UNSUPPORTED;
    }
}

}  // namespace

lnv_status plan_pull_items(lnv_plan *pl);

lnv_status plan_create(lnv_ctx *ctx, const lnv_pattern *A, const lnv_pattern *B,
                       const lnv_pattern *C, int flags, lnv_plan **out)
{
    LNV_ARG(ctx && A && B && C && out, "null pointer");
    LNV_ARG((flags & ~(LNV_TRANS_A | LNV_TRANS_B | LNV_SYM_C)) == 0, "unknown flags");
    const int sym1 = (flags & LNV_SYM_C) != 0;
    if (sym1 && (!C->symmetric || !C->tr)) {
        set_error("a symmetric output needs a symmetric pattern");
        return LNV_ERR_PATTERN;
    }
    if (A->n != B->n || A->n != C->n) {
        set_error("patterns of a product must have the same number of atoms (%lld, %lld, %lld)",
                  (long long)A->n, (long long)B->n, (long long)C->n);
        return LNV_ERR_PATTERN;
    }
    const int ta = (flags & LNV_TRANS_A) != 0, tb = (flags & LNV_TRANS_B) != 0;
    if ((ta && !A->symmetric) || (tb && !B->symmetric)) {
        set_error("a transposed operand needs a symmetric pattern");
        return LNV_ERR_PATTERN;
    }
    lnv_plan *pl = new lnv_plan();
    pl->A = A; pl->B = B; pl->C = C;
    pl->trans_a = ta; pl->trans_b = tb;
    pl->sym1 = pl->split = sym1 ? 1 : 0;
    pl->max_a_row = A->max_row;
    pl->max_c_row = C->max_row;
    unsigned long long *d_counts = nullptr;
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMalloc(&d_counts, sizeof(h));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counts, 0, sizeof(h), ctx->stream);
    if (e == cudaSuccess && C->n > 0) {
        // Symmetric patterns: op(A)'s row pattern equals A's, op(B)'s equals B's.
        k_symbolic<false, false><<<(unsigned)C->n, 128, 0, ctx->stream>>>(
            C->n, A->row_ptr, A->col, B->row_ptr, B->col, C->row_ptr, C->col, d_counts);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_counts, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d_counts);
    if (e != cudaSuccess) {
        delete pl;
        set_error("symbolic product pass failed: %s", cudaGetErrorString(e));
        return LNV_ERR_CUDA;
    }
    pl->triples = (int64_t)h[0];
    pl->triples_up = (int64_t)h[3];
    pl->push_scan = (int64_t)h[1];
    pl->pull_cand = (int64_t)h[2];
    pl->mode = pl->push_scan <= pl->pull_cand ? 0 : (B->symmetric ? 2 : 1);
    {
        // Prefer the row-group kernels when their tables fit a third of the free
        // device memory.
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        const size_t budget = free_b / 3;
        lnv_status gs = group_plan_build(ctx, pl, 4, budget, false, false);
        // dense position table when most candidates hit, hit lists otherwise
        if (gs == LNV_OK) {
            const bool dense = pl->grp.candidates > 0 && 2 * pl->grp.hits >= pl->grp.candidates;
            gs = group_plan_build(ctx, pl, 4, budget, dense, !dense);
            if (gs == LNV_OK) pl->mode = dense ? 3 : 4;
        }
        else if (gs != LNV_ERR_UNSUPPORTED) {
            plan_free(pl);
            return gs;
        }
    }
    if (pl->mode == 2) {
        lnv_status is = plan_pull_items(pl);
        if (is != LNV_OK) {
            plan_free(pl);
            return is;
        }
    }
    *out = pl;
    return LNV_OK;
}

// work items of the merge-join pull: (row, first slot) per 64 / 128 outputs
lnv_status plan_pull_items(lnv_plan *pl)
{
    const lnv_pattern *C = pl->C;
    if (pl->items64) return LNV_OK;
    {
        for (int chunk : {64, 128}) {
            std::vector<int2> items;
            for (int64_t r = 0; r < C->n; ++r) {
                const int64_t nc = C->h_row_ptr[r + 1] - C->h_row_ptr[r];
                for (int64_t s0 = 0; s0 < nc; s0 += chunk) items.push_back(make_int2((int)r, (int)s0));
            }
            int2 *d = nullptr;
            if (!items.empty()) {
                cudaError_t e2 = cudaMalloc(&d, sizeof(int2) * items.size());
                if (e2 == cudaSuccess)
                    e2 = cudaMemcpy(d, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
                if (e2 != cudaSuccess) {
                    cudaFree(d);
                    set_error("plan work items: %s", cudaGetErrorString(e2));
                    return e2 == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA;
                }
            }
            if (chunk == 64) {
                pl->items64 = d;
                pl->n_items64 = (int64_t)items.size();
            } else {
                pl->items128 = d;
                pl->n_items128 = (int64_t)items.size();
            }
        }
    }
    return LNV_OK;
}

lnv_status plan_set_kernel(lnv_ctx *ctx, lnv_plan *pl, int kernel)
{
    LNV_ARG(pl && kernel >= 0 && kernel < LNV_NUM_KERNELS, "kernel must be 0..13");
    if (kernel == 2) {
        if (!pl->B->symmetric) {
            set_error("the merge-join pull needs a symmetric B pattern");
            return LNV_ERR_UNSUPPORTED;
        }
        LNV_TRY(plan_pull_items(pl));
    }
    if (kernel == 9 || kernel == 12) {
        // 8-row group tables with the dense position table; the kernel reads
        // op(B) = B^T only (rows of the stored B_jk)
        if (!pl->trans_b) {
            set_error("kernels 9 and 12 need a product with op(B) = B^T");
            return LNV_ERR_UNSUPPORTED;
        }
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        LNV_TRY(group_plan_build_into(ctx, pl, 8, free_b / 3, true, false, pl->tc));
        LNV_TRY(umma_prepare(ctx, pl));
    } else if (kernel == 10) {
        // 7-row group tables with the dense position table (either op(B))
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        tile_plan_free(&pl->tt);
        LNV_TRY(group_plan_build_into(ctx, pl, kTc9G, free_b / 3, true, false, pl->tc));
        LNV_TRY(umma_prepare(ctx, pl));
    } else if (kernel == 11 || kernel == 13) {
        // kernel 9's 8-row tables (either op(B)), then each 32-column tile's k list
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        LNV_TRY(group_plan_build_into(ctx, pl, 8, free_b / 3, true, false, pl->tc));
        LNV_TRY(umma_prepare(ctx, pl));
        LNV_TRY(tile_plan_build(ctx, pl, free_b / 3));
    } else if (kernel == 7) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        LNV_TRY(triple_plan_build(ctx, pl, free_b / 3));
    } else if (kernel >= 3) {
        // build the row-group form this kernel reads, if missing
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        LNV_TRY(group_plan_build(ctx, pl, 4, free_b / 3, kernel != 4, kernel == 4));
    }
    pl->mode = kernel;
    return LNV_OK;
}

lnv_status plan_set_split(lnv_ctx *ctx, lnv_plan *pl, int on)
{
    on = on && pl->sym1 ? 1 : 0;
    if (pl->split == on) return LNV_OK;
    pl->split = on;
    // the row-group lists order J by the split: rebuild the forms present
    GroupPlan &gp = pl->grp;
    if (gp.G == 0) return LNV_OK;
    const bool dense = gp.bidx != nullptr, sparse = gp.hk != nullptr;
    group_plan_free(&gp);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
    return group_plan_build(ctx, pl, 4, free_b / 3, dense, sparse);
}

void plan_trim(lnv_plan *plan)
{
    if (plan->mode != 7) triple_plan_free(&plan->tri);
    if (plan->mode < 9) group_plan_free(&plan->tc);
    if (plan->mode != 11 && plan->mode != 13) tile_plan_free(&plan->tt);
    GroupPlan &gp = plan->grp;
    const bool dense = plan->mode == 3 || plan->mode == 5 || plan->mode == 6 || plan->mode == 8,
               sparse = plan->mode == 4;
    if (!dense && !sparse) {
        group_plan_free(&gp);
        return;
    }
    if (!dense && gp.bidx) {
        cudaFree(gp.bidx);
        gp.bidx = nullptr;
    }
    if (!sparse && gp.hk) {
        cudaFree(gp.hk); cudaFree(gp.hp);
        gp.hk = nullptr; gp.hp = nullptr;
    }
}

void plan_free(lnv_plan *plan)
{
    if (!plan) return;
    cudaFree(plan->items64);
    cudaFree(plan->items128);
    group_plan_free(&plan->grp);
    tile_plan_free(&plan->tt);
    group_plan_free(&plan->tc);
    triple_plan_free(&plan->tri);
    delete plan;
}

lnv_status multiply(lnv_ctx *ctx, const lnv_plan *plan, int nsf, lnv_prec prec, const void *A,
                    const void *B, void *C)
{
    return multiply2(ctx, plan, nsf, prec, A, B, nullptr, C, nullptr);
}

lnv_status mirror_lower(lnv_ctx *ctx, const lnv_pattern *P, int nsf, lnv_prec prec, void *vals)
{
    const int64_t n = P->nnzb * (int64_t)nsf * nsf;
    if (n == 0) return LNV_OK;
    if (!P->symmetric || !P->tr) {
        set_error("mirroring needs a symmetric pattern");
        return LNV_ERR_PATTERN;
    }
    if (prec == LNV_FP64) return mirror_launch<double>(ctx, P, nsf, (double *)vals);
    return mirror_launch<float>(ctx, P, nsf, (float *)vals);
}

lnv_status multiply2(lnv_ctx *ctx, const lnv_plan *plan, int nsf, lnv_prec prec, const void *A,
                     const void *B1, const void *B2, void *C1, void *C2)
{
    LNV_ARG(ctx && plan && A && B1 && C1 && (B2 == nullptr) == (C2 == nullptr), "null pointer");
    LNV_ARG(prec == LNV_FP64 || prec == LNV_FP32, "unknown precision");
    // With a symmetric first output the kernels may skip its lower triangle
    // (they form it only where that is free); it is mirrored afterwards.
    if (prec == LNV_FP64) LNV_TRY(dispatch_nsf<double>(ctx, plan, nsf, A, B1, B2, C1, C2));
    else LNV_TRY(dispatch_nsf<float>(ctx, plan, nsf, A, B1, B2, C1, C2));
    if (plan->sym1 && plan->split) LNV_TRY(mirror_lower(ctx, plan->C, nsf, prec, C1));
    return LNV_OK;
}

}  // namespace lnv
