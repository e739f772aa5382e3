// Symbolic phase of the listed-triple product kernel.
//
// For C = mask_C(op(A) op(B)) every block C_ij is a sum over the k with both
// op(A)_ik and op(B)_kj stored.  This pass lists, once per plan, those pairs
// of storage positions for every block of C, k ascending, so the numeric
// kernel neither searches B's rows nor multiplies blocks that are absent.
// The blocks of C are ordered by groups of four consecutive rows, and inside
// a group by the length of their lists, longest first (ties: by column, then
// row).  The numeric kernel runs eight blocks per warp and a warp lasts as
// long as its longest list, so lists of like length keep its lanes busy: on
// the products whose lists vary with the distance |r_i - r_j| (T = SX, U = SY
// and X = LS, Y = LH), column order left a third of the lanes idle.  Every
// block still sums its own list in k order, so the order changes no result.
#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

#include "lnv_impl.cuh"

namespace lnv {
namespace {

constexpr int kTripleGroup = 4;

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *__restrict__ a, int64_t lo, int64_t hi,
                                                   int32_t key)
{
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Count (tri == nullptr) or list the triples of each item.  op(A) and op(B)
// have the patterns of A and B (a transposed operand has a symmetric
// pattern); a transposed operand's block is read at the transpose position.
__global__ void k_triples(int64_t n_items, const int32_t *__restrict__ item_cb,
                          const int32_t *__restrict__ c_row, const int32_t *__restrict__ c_col,
                          const int64_t *__restrict__ a_rp, const int32_t *__restrict__ a_col,
                          const int64_t *__restrict__ a_tr, const int64_t *__restrict__ b_rp,
                          const int32_t *__restrict__ b_col, const int64_t *__restrict__ b_tr, int ta,
                          int tb, int64_t *cnt, const int64_t *__restrict__ t_off, int2 *tri)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_items) return;
    const int32_t cb = item_cb[t];
    const int32_t i = c_row[cb], j = c_col[cb];
    int64_t c = 0, w = tri ? t_off[t] : 0;
    for (int64_t q = a_rp[i]; q < a_rp[i + 1]; ++q) {
        const int32_t k = a_col[q];
        const int64_t be = b_rp[k + 1];
        const int64_t p = lower_bound_i32(b_col, b_rp[k], be, j);
        if (p < be && b_col[p] == j) {
            if (tri) tri[w + c] = make_int2((int32_t)(ta ? a_tr[q] : q), (int32_t)(tb ? b_tr[p] : p));
            ++c;
        }
    }
    if (!tri) cnt[t] = c;
}

}  // namespace

void triple_plan_free(TriplePlan *tp)
{
    cudaFree(tp->item_cb);
    cudaFree(tp->t_off);
    cudaFree(tp->tri);
    cudaFree(tp->up);
    *tp = TriplePlan();
}

lnv_status triple_plan_build(lnv_ctx *ctx, lnv_plan *pl, size_t budget_bytes)
{
    TriplePlan &tp = pl->tri;
    if (tp.tri || (tp.t_off && pl->triples == 0)) return LNV_OK;
    const lnv_pattern *A = pl->A, *B = pl->B, *C = pl->C;
    if (A->nnzb >= ((int64_t)1 << 31) || B->nnzb >= ((int64_t)1 << 31) || C->nnzb >= ((int64_t)1 << 31)) {
        set_error("triple-list plan: 2^31 or more blocks in an operand");
        return LNV_ERR_UNSUPPORTED;
    }
    const size_t need = sizeof(int2) * (size_t)pl->triples + (sizeof(int64_t) * 2 + sizeof(int32_t)) * (size_t)(C->nnzb + 1);
    if (need > budget_bytes) {
        set_error("triple-list plan needs %zu bytes, over the %zu budget", need, budget_bytes);
        return LNV_ERR_UNSUPPORTED;
    }
    // first order: groups of rows, then column, then row (host, from C's
    // pattern); the lengths counted in this order then reorder each group
    LNV_TRY(pattern_host_cols(ctx, C));
    const int64_t n = C->n, G = kTripleGroup, ng = (n + G - 1) / G;
    std::vector<int32_t> items((size_t)C->nnzb);
    {
        const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t)
            th.emplace_back([&, t] {
                std::vector<int64_t> cur(G);
                for (int64_t g = t; g < ng; g += nth) {
                    const int64_t r0 = g * G, r1 = std::min(n, r0 + G);
                    int64_t w = C->h_row_ptr[r0];
                    for (int64_t r = r0; r < r1; ++r) cur[r - r0] = C->h_row_ptr[r];
                    // merge the rows' sorted column lists; ties go to the lower row
                    for (;;) {
                        int best = -1;
                        int32_t bc = 0;
                        for (int64_t r = r0; r < r1; ++r) {
                            const int64_t q = cur[r - r0];
                            if (q < C->h_row_ptr[r + 1] && (best < 0 || C->h_col[q] < bc)) {
                                best = (int)(r - r0);
                                bc = C->h_col[q];
                            }
                        }
                        if (best < 0) break;
                        items[(size_t)w++] = (int32_t)cur[best]++;
                    }
                }
            });
        for (auto &x : th) x.join();
    }
    size_t bytes = 0;
    cudaError_t e = cudaMalloc(&tp.item_cb, sizeof(int32_t) * std::max<size_t>(1, items.size()));
    if (e == cudaSuccess) e = cudaMalloc(&tp.t_off, sizeof(int64_t) * (size_t)(C->nnzb + 1));
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(tp.item_cb, items.data(), sizeof(int32_t) * items.size(), cudaMemcpyHostToDevice);
    int64_t *cnt = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(int64_t) * std::max<int64_t>(1, C->nnzb));
    if (e != cudaSuccess) {
        cudaFree(cnt);
        triple_plan_free(&tp);
        set_error("triple-list plan: allocation failed (%s)", cudaGetErrorString(e));
        return LNV_ERR_OOM;
    }
    bytes += sizeof(int32_t) * items.size() + sizeof(int64_t) * (size_t)(C->nnzb + 1);
    tp.n_items = C->nnzb;
    const unsigned nb = (unsigned)((C->nnzb + 255) / 256);
    lnv_status s = LNV_OK;
    if (C->nnzb > 0) {
        k_triples<<<nb, 256, 0, ctx->stream>>>(C->nnzb, tp.item_cb, C->row, C->col, A->row_ptr, A->col, A->tr,
                                               B->row_ptr, B->col, B->tr, pl->trans_a, pl->trans_b, cnt,
                                               nullptr, nullptr);
        if (cudaGetLastError() != cudaSuccess) s = LNV_ERR_CUDA;
        count_launch();
    }
    if (s == LNV_OK && C->nnzb > 0) {
        // order each group's items by list length, longest first (stable:
        // equal lengths keep the column order), and the counts with them
        std::vector<int64_t> c_h((size_t)C->nnzb), c_o((size_t)C->nnzb);
        if (cudaMemcpyAsync(c_h.data(), cnt, sizeof(int64_t) * c_h.size(), cudaMemcpyDeviceToHost,
                            ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            s = LNV_ERR_CUDA;
        } else {
            std::vector<int32_t> sorted(items.size());
            const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
            std::vector<std::thread> th;
            for (int t = 0; t < nth; ++t)
                th.emplace_back([&, t] {
                    std::vector<int64_t> ord;
                    for (int64_t g = t; g < ng; g += nth) {
                        const int64_t q0 = C->h_row_ptr[g * G], q1 = C->h_row_ptr[std::min(n, g * G + G)];
                        ord.resize((size_t)(q1 - q0));
                        for (int64_t q = q0; q < q1; ++q) ord[(size_t)(q - q0)] = q;
                        std::stable_sort(ord.begin(), ord.end(),
                                         [&](int64_t a, int64_t b) { return c_h[(size_t)a] > c_h[(size_t)b]; });
                        for (int64_t q = q0; q < q1; ++q) {
                            sorted[(size_t)q] = items[(size_t)ord[(size_t)(q - q0)]];
                            c_o[(size_t)q] = c_h[(size_t)ord[(size_t)(q - q0)]];
                        }
                    }
                });
            for (auto &x : th) x.join();
            items.swap(sorted);
            if (cudaMemcpyAsync(tp.item_cb, items.data(), sizeof(int32_t) * items.size(), cudaMemcpyHostToDevice,
                                ctx->stream) != cudaSuccess ||
                cudaMemcpyAsync(cnt, c_o.data(), sizeof(int64_t) * c_o.size(), cudaMemcpyHostToDevice,
                                ctx->stream) != cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess)
                s = LNV_ERR_CUDA;
        }
    }
    if (s == LNV_OK) s = scan_exclusive(ctx->stream, cnt, C->nnzb, tp.t_off);
    int64_t total = 0;
    if (s == LNV_OK && cudaMemcpyAsync(&total, tp.t_off + C->nnzb, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                       ctx->stream) != cudaSuccess)
        s = LNV_ERR_CUDA;
    if (s == LNV_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) s = LNV_ERR_CUDA;
    if (s == LNV_OK && total != pl->triples) {
        set_error("triple-list plan: %lld triples listed, %lld counted", (long long)total, (long long)pl->triples);
        s = LNV_ERR_PATTERN;
    }
    if (s == LNV_OK && total > 0) {
        if (cudaMalloc(&tp.tri, sizeof(int2) * (size_t)total) != cudaSuccess) {
            set_error("triple-list plan: allocation of %lld triples failed", (long long)total);
            s = LNV_ERR_OOM;
        } else {
            bytes += sizeof(int2) * (size_t)total;
            k_triples<<<nb, 256, 0, ctx->stream>>>(C->nnzb, tp.item_cb, C->row, C->col, A->row_ptr, A->col,
                                                   A->tr, B->row_ptr, B->col, B->tr, pl->trans_a, pl->trans_b,
                                                   nullptr, tp.t_off, tp.tri);
            if (cudaGetLastError() != cudaSuccess) s = LNV_ERR_CUDA;
            count_launch();
            if (s == LNV_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) s = LNV_ERR_CUDA;
        }
    }
    cudaFree(cnt);
    if (s == LNV_OK && pl->sym1) {
        // the items of C's upper triangle (col >= row), in item order
        std::vector<int32_t> row_of((size_t)C->nnzb);
        for (int64_t r = 0; r < n; ++r)
            for (int64_t q = C->h_row_ptr[r]; q < C->h_row_ptr[r + 1]; ++q) row_of[(size_t)q] = (int32_t)r;
        std::vector<int32_t> up;
        up.reserve(items.size() / 2 + 1);
        for (size_t t = 0; t < items.size(); ++t)
            if (C->h_col[(size_t)items[t]] >= row_of[(size_t)items[t]]) up.push_back((int32_t)t);
        tp.n_up = (int64_t)up.size();
        if (!up.empty()) {
            if (cudaMalloc(&tp.up, sizeof(int32_t) * up.size()) != cudaSuccess ||
                cudaMemcpy(tp.up, up.data(), sizeof(int32_t) * up.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
                set_error("triple-list plan: allocation of the upper-triangle items failed");
                s = LNV_ERR_OOM;
            }
            bytes += sizeof(int32_t) * up.size();
        }
    }
    if (s != LNV_OK) {
        if (s == LNV_ERR_CUDA) set_error("triple-list plan: kernel failed");
        triple_plan_free(&tp);
        return s;
    }
    tp.bytes = bytes;
    return LNV_OK;
}

}  // namespace lnv
