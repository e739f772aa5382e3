// Symbolic phase of the row-group product kernel.
//
// Each output row's products share nothing with the next row in a one-row
// kernel, so every block op(B)_kj is fetched once per row that uses it.
// Spatially close atoms have consecutive indices in a cell-ordered system, so
// taking G consecutive rows together lets one fetch of op(B)_kj serve every
// row of the group that holds A_ik.  This pass lists, per group, the k's and
// j's the group touches and a 16-bit position table of op(B)_kj, so the
// numeric kernel neither searches nor walks B's rows.  It runs once per plan.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include "lnv_impl.cuh"

namespace lnv {
namespace {

// bidx[k_local][j_local] of one group per CTA.
__global__ void k_bidx(const int64_t *__restrict__ k_off, const int32_t *__restrict__ k_list,
                       const int64_t *__restrict__ j_off, const int32_t *__restrict__ j_list,
                       const int64_t *__restrict__ bidx_off, const int64_t *__restrict__ b_rp,
                       const int32_t *__restrict__ b_col, int trans_b, uint16_t *bidx)
{
    const int64_t g = blockIdx.x;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    uint16_t *out = bidx + bidx_off[g];
    const int64_t nj_pad = (nj + 7) & ~int64_t(7);  // rows padded to 16 bytes
    for (int64_t t = threadIdx.x; t < nk * nj; t += blockDim.x) {
        const int64_t kl = t / nj, jl = t - kl * nj;
        const int32_t k = k_list[kb + kl], j = j_list[jb + jl];
        // op(B)_kj: B^T -> block (j, k) in row j; B -> block (k, j) in row k
        const int32_t row = trans_b ? j : k, key = trans_b ? k : j;
        int64_t lo = b_rp[row], hi = b_rp[row + 1];
        const int64_t r0 = lo;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (b_col[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        const bool found = lo < b_rp[row + 1] && b_col[lo] == key;
        out[kl * nj_pad + jl] = found ? (uint16_t)(lo - r0) : (uint16_t)0xFFFF;
    }
}

// The same table j-major (the tensor-core kernel's form): bidx[j_local][k_local],
// rows of nk_pad entries (a multiple of 4, so a thread reads the offsets of
// four consecutive k's in one 8-byte load).
__global__ void k_bidx_t(const int64_t *__restrict__ k_off, const int32_t *__restrict__ k_list,
                         const int64_t *__restrict__ j_off, const int32_t *__restrict__ j_list,
                         const int64_t *__restrict__ bidx_off, const int64_t *__restrict__ b_rp,
                         const int32_t *__restrict__ b_col, int trans_b, uint16_t *bidx)
{
    const int64_t g = blockIdx.x;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    uint16_t *out = bidx + bidx_off[g];
    const int64_t nk_pad = (nk + 3) & ~int64_t(3);
    for (int64_t t = threadIdx.x; t < nk * nj; t += blockDim.x) {
        const int64_t jl = t / nk, kl = t - jl * nk;
        const int32_t k = k_list[kb + kl], j = j_list[jb + jl];
        const int32_t row = trans_b ? j : k, key = trans_b ? k : j;
        int64_t lo = b_rp[row], hi = b_rp[row + 1];
        const int64_t r0 = lo;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (b_col[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        const bool found = lo < b_rp[row + 1] && b_col[lo] == key;
        out[jl * nk_pad + kl] = found ? (uint16_t)(lo - r0) : (uint16_t)0xFFFF;
    }
}

// Hit lists: per (group, j) the k's of the group's K with op(B)_kj stored.
// fill == nullptr: count into cnt[j_entry]; else write hk / hp at hoff.
__global__ void k_hits(const int64_t *__restrict__ k_off, const int32_t *__restrict__ k_list,
                       const int64_t *__restrict__ j_off, const int32_t *__restrict__ j_list,
                       const int64_t *__restrict__ b_rp, const int32_t *__restrict__ b_col,
                       int trans_b, int64_t *cnt, const int64_t *__restrict__ hoff, uint16_t *hk,
                       int32_t *hp)
{
    const int64_t g = blockIdx.x;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    for (int64_t jl = threadIdx.x; jl < nj; jl += blockDim.x) {
        const int32_t j = j_list[jb + jl];
        int64_t c = 0, w = hp ? hoff[jb + jl] : 0;
        for (int64_t kl = 0; kl < nk; ++kl) {
            const int32_t k = k_list[kb + kl];
            const int32_t row = trans_b ? j : k, key = trans_b ? k : j;
            int64_t lo = b_rp[row], hi = b_rp[row + 1];
            while (lo < hi) {
                const int64_t mid = lo + ((hi - lo) >> 1);
                if (b_col[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            if (lo < b_rp[row + 1] && b_col[lo] == key) {
                if (hp) {
                    hk[w + c] = (uint16_t)kl;
                    hp[w + c] = (int32_t)lo;
                }
                ++c;
            }
        }
        if (!hp) cnt[jb + jl] = c;
    }
}

template <typename X>
lnv_status upload(const std::vector<X> &h, X **d, size_t *bytes)
{
    *d = nullptr;
    if (h.empty()) return LNV_OK;
    LNV_CUDA(cudaMalloc(d, sizeof(X) * h.size()));
    LNV_CUDA(cudaMemcpy(*d, h.data(), sizeof(X) * h.size(), cudaMemcpyHostToDevice));
    *bytes += sizeof(X) * h.size();
    return LNV_OK;
}

}  // namespace

lnv_status pattern_host_cols(lnv_ctx *ctx, const lnv_pattern *p)
{
    if ((int64_t)p->h_col.size() == p->nnzb) return LNV_OK;
    p->h_col.resize(p->nnzb);
    if (p->nnzb > 0) {
        LNV_CUDA(cudaMemcpyAsync(p->h_col.data(), p->col, sizeof(int32_t) * p->nnzb,
                                 cudaMemcpyDeviceToHost, ctx->stream));
        LNV_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return LNV_OK;
}

void group_plan_free(GroupPlan *gp)
{
    cudaFree(gp->k_off); cudaFree(gp->k_list); cudaFree(gp->apos);
    cudaFree(gp->j_off); cudaFree(gp->j_list); cudaFree(gp->cpos);
    cudaFree(gp->bidx_off); cudaFree(gp->bidx);
    cudaFree(gp->hoff); cudaFree(gp->hk); cudaFree(gp->hp);
    cudaFree(gp->jsplit);
    cudaFree(gp->items);
    *gp = GroupPlan();
}

// Lists (K, J, apos, cpos) and hit counts of the row groups: built once per plan
// into gp (the plan's 4-row tables, or the 8-row tables of kernel 9).
static lnv_status group_plan_lists(lnv_ctx *ctx, lnv_plan *pl, int G, size_t budget_bytes, GroupPlan &gp)
{
    const lnv_pattern *A = pl->A, *B = pl->B, *C = pl->C;
    if (B->max_row >= 0xFFFF) {
        set_error("row-group plan: B rows longer than 65534 blocks");
        return LNV_ERR_UNSUPPORTED;
    }
    LNV_TRY(pattern_host_cols(ctx, A));
    LNV_TRY(pattern_host_cols(ctx, C));
    const int64_t n = C->n;
    const int64_t ng = (n + G - 1) / G;
    std::vector<int64_t> nk(ng), nj(ng);
    std::vector<std::vector<int32_t>> Ks(ng), Js(ng);
    auto unite = [&](const lnv_pattern *P, int64_t r0, int64_t r1, std::vector<int32_t> &out) {
        out.clear();
        for (int64_t r = r0; r < r1; ++r)
            out.insert(out.end(), P->h_col.begin() + P->h_row_ptr[r], P->h_col.begin() + P->h_row_ptr[r + 1]);
        std::sort(out.begin(), out.end());
        out.erase(std::unique(out.begin(), out.end()), out.end());
    };
    const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    {
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t)
            th.emplace_back([&, t] {
                for (int64_t g = t; g < ng; g += nth) {
                    const int64_t r0 = g * G, r1 = std::min(n, r0 + G);
                    unite(A, r0, r1, Ks[g]);
                    unite(C, r0, r1, Js[g]);
                    nk[g] = (int64_t)Ks[g].size();
                    nj[g] = (int64_t)Js[g].size();
                }
            });
        for (auto &x : th) x.join();
    }
    // the tensor-core kernel's tables: spatial J order, j-major position
    // table, CTA work items
    const bool jmajor = &gp == &pl->tc;
    std::vector<int64_t> k_off(ng + 1, 0), j_off(ng + 1, 0), b_off(ng + 1, 0);
    int max_k = 0, max_j = 0;
    for (int64_t g = 0; g < ng; ++g) {
        k_off[g + 1] = k_off[g] + nk[g];
        j_off[g + 1] = j_off[g] + nj[g];
        b_off[g + 1] = b_off[g] + (jmajor ? nj[g] * ((nk[g] + 3) & ~int64_t(3)) : nk[g] * ((nj[g] + 7) & ~int64_t(7)));
        max_k = std::max<int>(max_k, (int)nk[g]);
        max_j = std::max<int>(max_j, (int)nj[g]);
    }
    const size_t need = (sizeof(int32_t) * (1 + G) + sizeof(int64_t)) * (size_t)(k_off[ng] + j_off[ng]);
    if (need > budget_bytes) {
        set_error("row-group lists need %zu bytes, over the %zu budget", need, budget_bytes);
        return LNV_ERR_UNSUPPORTED;
    }
    // symmetric first output: the upper part of J (j >= the group's first row)
    // comes first, and jsplit[g] (a multiple of 8) is where the rest starts
    const bool split = pl->sym1 && pl->split && &gp == &pl->grp;
    std::vector<int32_t> jsplit(split ? ng : 0);
    std::vector<int32_t> k_list(k_off[ng]), j_list(j_off[ng]);
    std::vector<int32_t> apos((size_t)k_off[ng] * G, -1), cpos((size_t)j_off[ng] * G, -1);
    {
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t)
            th.emplace_back([&, t] {
                for (int64_t g = t; g < ng; g += nth) {
                    const int64_t r0 = g * G, r1 = std::min(n, r0 + G);
                    std::copy(Ks[g].begin(), Ks[g].end(), k_list.begin() + k_off[g]);
                    std::copy(Js[g].begin(), Js[g].end(), j_list.begin() + j_off[g]);
                    for (int64_t r = r0; r < r1; ++r) {
                        const int m = (int)(r - r0);
                        for (int64_t q = A->h_row_ptr[r]; q < A->h_row_ptr[r + 1]; ++q) {
                            const int64_t kl = std::lower_bound(Ks[g].begin(), Ks[g].end(), A->h_col[q]) - Ks[g].begin();
                            apos[(size_t)(k_off[g] + kl) * G + m] = (int32_t)q;
                        }
                        for (int64_t q = C->h_row_ptr[r]; q < C->h_row_ptr[r + 1]; ++q) {
                            const int64_t jl = std::lower_bound(Js[g].begin(), Js[g].end(), C->h_col[q]) - Js[g].begin();
                            cpos[(size_t)(j_off[g] + jl) * G + m] = (int32_t)q;
                        }
                    }
                    // Order J by the set of the group's rows whose C row holds j (then by
                    // index): consecutive columns then need the same rows, so a kernel
                    // can skip the rows that no column of a set keeps.  With a split,
                    // the columns j >= r0 come first.  The tensor-core tables keep J in
                    // atom order: with cell-ordered atoms, spatially compact chunks.
                    if (!jmajor) {
                        const int64_t nj_g = nj[g];
                        std::vector<int32_t> key(nj_g), perm(nj_g);
                        int64_t n_hi = 0;
                        for (int64_t jl = 0; jl < nj_g; ++jl) {
                            int cm = 0;
                            for (int m = 0; m < G; ++m)
                                if (cpos[(size_t)(j_off[g] + jl) * G + m] >= 0) cm |= 1 << m;
                            const bool hi = split && j_list[j_off[g] + jl] >= r0;
                            n_hi += hi ? 1 : 0;
                            key[jl] = cm | (hi ? 1 << G : 0);
                            perm[jl] = (int32_t)jl;
                        }
                        if (split) jsplit[g] = (int32_t)std::min<int64_t>(nj_g, (n_hi + 7) & ~int64_t(7));
                        std::stable_sort(perm.begin(), perm.end(),
                                         [&](int32_t a, int32_t b) { return key[a] > key[b]; });
                        std::vector<int32_t> jl_new(nj_g), cp_new((size_t)nj_g * G);
                        for (int64_t t = 0; t < nj_g; ++t) {
                            jl_new[t] = j_list[j_off[g] + perm[t]];
                            for (int m = 0; m < G; ++m)
                                cp_new[(size_t)t * G + m] = cpos[(size_t)(j_off[g] + perm[t]) * G + m];
                        }
                        std::copy(jl_new.begin(), jl_new.end(), j_list.begin() + j_off[g]);
                        std::copy(cp_new.begin(), cp_new.end(), cpos.begin() + (size_t)j_off[g] * G);
                    }
                    std::vector<int32_t>().swap(Ks[g]);
                    std::vector<int32_t>().swap(Js[g]);
                }
            });
        for (auto &x : th) x.join();
    }
    gp.G = G;
    gp.n_groups = ng;
    gp.jmajor = jmajor ? 1 : 0;
    gp.max_k = max_k;
    gp.max_j = max_j;
    gp.candidates = b_off[ng];
    gp.max_j_hi = gp.max_j_lo = 0;
    for (int64_t g = 0; g < (int64_t)jsplit.size(); ++g) {
        gp.max_j_hi = std::max<int>(gp.max_j_hi, jsplit[g]);
        gp.max_j_lo = std::max<int>(gp.max_j_lo, (int)(nj[g] - jsplit[g]));
    }
    size_t bytes = 0;
    lnv_status s = LNV_OK;
    if (split) s = upload(jsplit, &gp.jsplit, &bytes);
    if (s == LNV_OK) s = upload(k_off, &gp.k_off, &bytes);
    if (s == LNV_OK) s = upload(k_list, &gp.k_list, &bytes);
    if (s == LNV_OK) s = upload(apos, &gp.apos, &bytes);
    if (s == LNV_OK) s = upload(j_off, &gp.j_off, &bytes);
    if (s == LNV_OK) s = upload(j_list, &gp.j_list, &bytes);
    if (s == LNV_OK) s = upload(cpos, &gp.cpos, &bytes);
    if (s == LNV_OK) s = upload(b_off, &gp.bidx_off, &bytes);
    if (s == LNV_OK && jmajor) {
        // CTA work items of the tensor-core kernel: (group, first column) per
        // kTcCols (kTc9Cols) columns of J, ordered by that first column's atom, then by
        // group, so that the CTAs running at one time cover nearby columns
        // (and share the rows of op(B) they gather) across many groups
        const int cols = G == kTc9G ? kTc9Cols : kTcCols;
        std::vector<std::pair<std::pair<uint64_t, int64_t>, int2>> it;
        for (int64_t g = 0; g < ng; ++g)
            for (int64_t c0 = 0; c0 < nj[g]; c0 += cols)
                it.push_back({{(uint64_t)j_list[j_off[g] + c0], g}, make_int2((int)g, (int)c0)});
        std::sort(it.begin(), it.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
        std::vector<int2> items(it.size());
        for (size_t q = 0; q < it.size(); ++q) items[q] = it[q].second;
        gp.n_items = (int64_t)items.size();
        s = upload(items, &gp.items, &bytes);
    }
    // hit counts per (group, j) -> offsets of the hit lists
    if (s == LNV_OK && j_off[ng] > 0) {
        int64_t *cnt = nullptr;
        cudaError_t e = cudaMalloc(&cnt, sizeof(int64_t) * (size_t)j_off[ng]);
        if (e == cudaSuccess) e = cudaMalloc(&gp.hoff, sizeof(int64_t) * (size_t)(j_off[ng] + 1));
        if (e == cudaSuccess) {
            k_hits<<<(unsigned)ng, 128, 0, ctx->stream>>>(gp.k_off, gp.k_list, gp.j_off, gp.j_list, B->row_ptr,
                                                         B->col, pl->trans_b, cnt, nullptr, nullptr, nullptr);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            s = scan_exclusive(ctx->stream, cnt, j_off[ng], gp.hoff);
            if (s == LNV_OK)
                e = cudaMemcpy(&gp.hits, gp.hoff + j_off[ng], sizeof(int64_t), cudaMemcpyDeviceToHost);
            bytes += sizeof(int64_t) * (size_t)(j_off[ng] + 1);
        }
        cudaFree(cnt);
        if (s == LNV_OK && e != cudaSuccess) {
            set_error("row-group hit counts: %s", cudaGetErrorString(e));
            s = e == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA;
        }
    }
    if (s != LNV_OK) {
        group_plan_free(&gp);
        return s;
    }
    gp.bytes = bytes;
    return LNV_OK;
}

// Build the lists (once) and the requested forms: the dense 16-bit position
// table and / or the hit lists.  Each form is checked against the budget.
lnv_status group_plan_build_into(lnv_ctx *ctx, lnv_plan *pl, int G, size_t budget_bytes, bool dense, bool sparse,
                                 GroupPlan &gp)
{
    if (gp.G != 0 && gp.G != G) group_plan_free(&gp);
    if (gp.G == 0) LNV_TRY(group_plan_lists(ctx, pl, G, budget_bytes, gp));
    const lnv_pattern *B = pl->B;
    const int64_t ng = gp.n_groups;
    if (dense && !gp.bidx && gp.candidates > 0) {
        const size_t need = sizeof(uint16_t) * (size_t)gp.candidates;
        if (need > budget_bytes) {
            set_error("row-group position table needs %zu bytes, over the %zu budget", need, budget_bytes);
            return LNV_ERR_UNSUPPORTED;
        }
        LNV_CUDA(cudaMalloc(&gp.bidx, need));
        LNV_CUDA(cudaMemsetAsync(gp.bidx, 0xFF, need, ctx->stream));
        if (gp.jmajor)
            k_bidx_t<<<(unsigned)ng, 256, 0, ctx->stream>>>(gp.k_off, gp.k_list, gp.j_off, gp.j_list, gp.bidx_off,
                                                            B->row_ptr, B->col, pl->trans_b, gp.bidx);
        else
            k_bidx<<<(unsigned)ng, 256, 0, ctx->stream>>>(gp.k_off, gp.k_list, gp.j_off, gp.j_list, gp.bidx_off,
                                                          B->row_ptr, B->col, pl->trans_b, gp.bidx);
        LNV_LAUNCHED();
        LNV_CUDA(cudaStreamSynchronize(ctx->stream));
        gp.bytes += need;
    }
    if (sparse && !gp.hk && gp.hits > 0) {
        const size_t need = (sizeof(uint16_t) + sizeof(int32_t)) * (size_t)gp.hits;
        if (need > budget_bytes) {
            set_error("row-group hit lists need %zu bytes, over the %zu budget", need, budget_bytes);
            return LNV_ERR_UNSUPPORTED;
        }
        LNV_CUDA(cudaMalloc(&gp.hk, sizeof(uint16_t) * (size_t)gp.hits));
        LNV_CUDA(cudaMalloc(&gp.hp, sizeof(int32_t) * (size_t)gp.hits));
        k_hits<<<(unsigned)ng, 128, 0, ctx->stream>>>(gp.k_off, gp.k_list, gp.j_off, gp.j_list, B->row_ptr, B->col,
                                                     pl->trans_b, nullptr, gp.hoff, gp.hk, gp.hp);
        LNV_LAUNCHED();
        LNV_CUDA(cudaStreamSynchronize(ctx->stream));
        gp.bytes += need;
    }
    return LNV_OK;
}

lnv_status group_plan_build(lnv_ctx *ctx, lnv_plan *pl, int G, size_t budget_bytes, bool dense, bool sparse)
{
    return group_plan_build_into(ctx, pl, G, budget_bytes, dense, sparse, pl->grp);
}

}  // namespace lnv
