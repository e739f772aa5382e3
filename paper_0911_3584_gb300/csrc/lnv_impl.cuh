// Internal declarations shared by the liblnv translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/lnv.h"

namespace lnv {

void set_error(const char *fmt, ...);

// Status helpers: every host routine returns lnv_status and records a message.
#define LNV_CUDA(call)                                                               \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ::lnv::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                    \
            return e_ == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA;     \
        }                                                                            \
    } while (0)

#define LNV_TRY(expr)                       \
    do {                                    \
        lnv_status s_ = (expr);             \
        if (s_ != LNV_OK) return s_;        \
    } while (0)

#define LNV_ARG(cond, msg)                                   \
    do {                                                     \
        if (!(cond)) {                                       \
            ::lnv::set_error("invalid argument: %s", msg);   \
            return LNV_ERR_ARG;                              \
        }                                                    \
    } while (0)

// Launch check after a kernel<<<>>>; also counts the library's kernel launches.
void count_launch();
#define LNV_LAUNCHED()                   \
    do {                                 \
        ::lnv::count_launch();           \
        LNV_CUDA(cudaGetLastError());    \
    } while (0)

// Maximum blocks in one pattern row (bitonic row sort in shared memory).
constexpr int kMaxRow = 16384;

// Raise a kernel's dynamic shared-memory limit once (not inside every launch,
// so that launches can be captured in CUDA graphs).
cudaError_t ensure_smem(const void *kernel, size_t bytes);
// Ask for the largest shared-memory carveout for a kernel (once per device),
// so that shared memory does not cap the CTAs resident per SM.
cudaError_t prefer_smem(const void *kernel);

}  // namespace lnv

struct lnv_ctx {
    int device;
    cudaStream_t stream;
    int sm_count;
    size_t smem_optin;
    // device status word: set to 1 by a kernel whose bounded device-side wait
    // ran out (read and cleared by lnv_ctx_device_status)
    int *dev_status = nullptr;
    unsigned long long wait_ns = 1000000000ull;  // limit of one device-side wait
    double *scratch = nullptr;  // reduction partials of lnv_vec_dot (grown on demand)
    size_t scratch_n = 0;
    void *prod_scratch = nullptr;  // product of lnv_bsr_multiply with beta != 0 (grown on demand)
    size_t prod_scratch_bytes = 0;
};

struct lnv_pattern {
    int64_t n = 0;
    int64_t nnzb = 0;
    int64_t *row_ptr = nullptr;  // device, n+1
    int32_t *col = nullptr;      // device, nnzb
    int32_t *row = nullptr;      // device, nnzb: row of each block
    int64_t *tr = nullptr;       // device, nnzb: position of the transpose block or -1
    int symmetric = 0;
    int max_row = 0;             // longest row (host copy)
    std::vector<int64_t> h_row_ptr;  // host copy of row_ptr (for planning and tuning)
    mutable std::vector<int32_t> h_col;  // host copy of col, filled on demand by the planner
};

// Row-group plan of a product (see group.cu): rows are taken G at a time; for
// group g, K = sorted union of A's rows, J = sorted union of C's rows,
// apos[k][m] / cpos[j][m] the positions of (row m, k) in A and (row m, j) in
// C (-1 if absent), and bidx[k][j] the offset of op(B)_kj inside its B row
// (B's row j when op(B) = B^T, row k otherwise; 0xFFFF if absent), rows of
// the table padded to a multiple of 8 entries.
struct GroupPlan {
    int G = 0;
    int64_t n_groups = 0;
    int64_t *k_off = nullptr;    // [n_groups + 1]
    int32_t *k_list = nullptr;   // [sum |K|]
    int32_t *apos = nullptr;     // [sum |K|][G]
    int64_t *j_off = nullptr;    // [n_groups + 1]
    int32_t *j_list = nullptr;   // [sum |J|]
    int32_t *cpos = nullptr;     // [sum |J|][G]
    int64_t *bidx_off = nullptr; // [n_groups + 1]
    uint16_t *bidx = nullptr;    // [sum |K| |J|]  (dense table; may be absent)
    // sparse form: for each (group, j) the hits k (ascending) with op(B)_kj stored
    int64_t *hoff = nullptr;     // [sum |J| + 1]
    uint16_t *hk = nullptr;      // [hits] k position in the group's K list
    int32_t *hp = nullptr;       // [hits] block index of op(B)_kj's stored block
    int64_t hits = 0, candidates = 0;
    int max_k = 0, max_j = 0;
    // plans whose first output is symmetric: J lists first the columns j >= the
    // group's first row (the upper part, padded with lower columns to a
    // multiple of 8), then the rest; jsplit[g] is where the rest starts
    int32_t *jsplit = nullptr;   // [n_groups] or absent
    int max_j_hi = 0, max_j_lo = 0;
    // the tensor-core kernel's form: J in atom order (spatial order for
    // cell-ordered atoms), bidx j-major (bidx[j][k], rows of nk_pad(g) entries, a
    // multiple of 4) and the CTA work items (group, first column of J) of
    // kTcCols (kTc9Cols for 7-row groups) columns each, sorted by the key of
    // the item's first column
    int jmajor = 0;
    int apos_op = 0;             // apos holds op(A)'s stored block (transposed through tr)
    int2 *items = nullptr;       // [n_items]
    int64_t n_items = 0;
    size_t bytes = 0;
};

// Columns j per CTA of the tensor-core kernel (two 128-row tiles of 32 atoms).
constexpr int kTcCols = 64;
// Its NSF = 9 form (kernel 10): groups of 7 rows (N = 63 of 64), one tile of
// 14 columns (M = 126 of 128) per CTA.
constexpr int kTc9G = 7;
constexpr int kTc9Cols = 14;

// Tile plan of kernel 11 (umma_tile.cu), built from the 8-row tables in tc:
// one work item per 32 columns of a group's J, with the item's own k list
// (the k's at which any of its columns holds op(B)_kj, padded with empty
// entries to a multiple of 4).  Per listed k: B's row start (block index of
// row k; op(B) = B only) and the op(A) positions of the group's 8 rows; per
// item a j-major table of 16-bit offsets of op(B)_kj in its stored row
// (0xFFFF: absent), [32 columns][its k count].
struct TilePlan {
    int64_t n_items = 0;
    int2 *items = nullptr;       // [n_items] (group, first column of J)
    int64_t *ck_off = nullptr;   // [n_items + 1] the item's range of listed k's
    int32_t *ck_brow = nullptr;  // [listed]
    int32_t *ck_apos = nullptr;  // [listed][8]
    uint16_t *ck_tab = nullptr;  // [listed * 32]
    // plans with a symmetric first output: the items holding a column j >=
    // the group's first row (the first output formed on its upper triangle)
    int32_t *up = nullptr;
    int64_t n_up = 0;
    int64_t listed = 0;
    const int2 *src = nullptr;   // tc.items the plan was built from
    size_t bytes = 0;
};

// Triple-list plan of a product (see triples.cu): C's blocks as work items,
// ordered by groups of 4 rows, then by list length inside the group; for
// each item the contributing (op(A)_ik, op(B)_kj) storage positions, k
// ascending.
struct TriplePlan {
    int64_t n_items = 0;
    int32_t *item_cb = nullptr;  // [n_items]     C block of the item
    int64_t *t_off = nullptr;    // [n_items + 1] item's range in tri
    int2 *tri = nullptr;         // [triples]     (A block, B block) storage positions
    // plans with a symmetric first output: the items of C's blocks with
    // col >= row, in item order (the first output formed on its upper triangle)
    int32_t *up = nullptr;       // [n_up] item indices
    int64_t n_up = 0;
    size_t bytes = 0;
};

struct lnv_plan {
    const lnv_pattern *A, *B, *C;
    int trans_a, trans_b;
    // C1 (the first output) is symmetric, on a symmetric pattern; with split,
    // the kernels that can form only its blocks with col >= row do so and the
    // rest is mirrored from them (split = 0: C1 is formed whole)
    int sym1 = 0, split = 0;
    // 0 push (row gather into a shared-memory row accumulator), 1 pull with a
    // binary search per k, 2 pull with a merge-join walk (symmetric B pattern),
    // 3 row groups with a dense position table, 4 row groups with hit lists,
    // 5 row groups with per-warp lists, 6 row groups on tensor cores, 7
    // listed triples per output block, 8 kernel 5 with warp slices of half
    // the width, 9 8-row groups on the tcgen05 tensor cores (tables in tc),
    // 10 its NSF = 9 form, 11 tcgen05 tiles of 32 columns over their own k
    // lists (tables in tc and tt), 12 and 13 the single-pass TF32 forms of 9
    // and 11
    int mode;
    GroupPlan grp;
    GroupPlan tc;  // 8-row groups of the tensor-core kernels (9, 11; 7-row groups for 10)
    TilePlan tt;   // kernel 11's per-tile k lists
    TriplePlan tri;
    // work items (row, first output slot) of the merge-join pull, for 64 and
    // 128 outputs per CTA (device arrays)
    int2 *items64 = nullptr, *items128 = nullptr;
    int64_t n_items64 = 0, n_items128 = 0;
    int64_t triples;     // contributing block triples
    int64_t triples_up;  // those of C's blocks with col >= row
    int64_t push_scan;   // B blocks a push kernel scans
    int64_t pull_cand;   // (k, j) candidates a pull kernel tests
    int max_a_row, max_c_row;
};

namespace lnv {

// Pattern internals (pattern.cu)
lnv_status pattern_build_impl(lnv_ctx *ctx, const double *pos, int n_seg, const int64_t *seg_off,
                              const double *cells, double cutoff, lnv_pattern **out);
lnv_status pattern_finish(lnv_ctx *ctx, lnv_pattern *p, bool sort_rows);
lnv_status pattern_validate(lnv_ctx *ctx, const lnv_pattern *p);
// Block values carried from one pattern onto another of the same atoms (zeros
// where `from` has no block).
lnv_status pattern_remap(lnv_ctx *ctx, const lnv_pattern *from, const lnv_pattern *to, int nsf, lnv_prec prec,
                         const void *from_vals, void *to_vals);
void pattern_free(lnv_pattern *p);
// Upper triangle (col >= row) of P as its own pattern, and for every block
// (i, j) of P the position of (min(i,j), max(i,j)) in it.
lnv_status pattern_upper(lnv_ctx *ctx, const lnv_pattern *P, lnv_pattern **out);
lnv_status pattern_upper_map(lnv_ctx *ctx, const lnv_pattern *P, const lnv_pattern *U, int64_t *map_dev);
// position map of every block of `sub` inside `super` (both sorted), -1 if absent
lnv_status pattern_submap(lnv_ctx *ctx, const lnv_pattern *sub, const lnv_pattern *super,
                          int64_t *map_dev);

// Product internals (mult.cu)
// flags: LNV_TRANS_A, LNV_TRANS_B, LNV_SYM_C (the first output of the plan's
// products is symmetric; C's pattern must be symmetric)
lnv_status plan_create(lnv_ctx *ctx, const lnv_pattern *A, const lnv_pattern *B,
                       const lnv_pattern *C, int flags, lnv_plan **out);
// The strict lower triangle of a matrix on the symmetric pattern P set from its
// upper one: vals[p] = vals[tr p]^T for every block p = (i, j), j < i, and the
// diagonal blocks made symmetric from their upper elements.
lnv_status mirror_lower(lnv_ctx *ctx, const lnv_pattern *P, int nsf, lnv_prec prec, void *vals);
void plan_free(lnv_plan *plan);
// Free the row-group tables the plan's current kernel does not use.
void plan_trim(lnv_plan *plan);
lnv_status plan_set_kernel(lnv_ctx *ctx, lnv_plan *pl, int kernel);
// Form a symmetric first output on one triangle (on = 1) or whole (0); the
// row-group lists, whose column order follows the setting, are rebuilt.
lnv_status plan_set_split(lnv_ctx *ctx, lnv_plan *pl, int on);
// Row-group plan (group.cu); returns LNV_ERR_UNSUPPORTED when the table would
// not fit the budget or a B row is too long for 16-bit offsets.
lnv_status group_plan_build(lnv_ctx *ctx, lnv_plan *pl, int G, size_t budget_bytes, bool dense,
                            bool sparse);
lnv_status group_plan_build_into(lnv_ctx *ctx, lnv_plan *pl, int G, size_t budget_bytes, bool dense, bool sparse,
                                 GroupPlan &gp);
// Kernel 9 (umma.cu): C = mask(op(A) B^T) on 8-row groups, tcgen05 tensor
// cores, FP32 values, NSF = 4.
// onepass: kernel 12, the single-pass TF32 form (below the FP32-level bound).
lnv_status launch_umma(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B, void *C,
                       bool onepass = false);
// Finish kernel 9's or 10's tables after they are built (op(A) positions for A^T).
lnv_status umma_prepare(lnv_ctx *ctx, lnv_plan *pl);
// Kernel 10 (umma9.cu): C = mask(op(A) op(B)) on 7-row groups, tcgen05 tensor
// cores, FP32 values, NSF = 9.
lnv_status launch_umma9(lnv_ctx *ctx, const lnv_plan *pl, bool ta, bool tb, const void *A, const void *B, void *C);
// Kernel 11 (umma_tile.cu): C = mask(op(A) op(B)) on 32-column tiles of
// 8-row groups over each tile's own k list, tcgen05 tensor cores, FP32
// values, NSF = 4, either op(B).  upper: only the tiles holding a column j >=
// the group's first row (a symmetric output formed on its upper triangle).
// onepass: kernel 13, the single-pass TF32 form (below the FP32-level bound).
lnv_status launch_umma_tile(lnv_ctx *ctx, const lnv_plan *pl, bool ta, bool tb, bool upper, const void *A,
                            const void *B, void *C, bool onepass = false);
// Build kernel 11's tile plan from the plan's 8-row tables (tc, finished by
// umma_prepare); LNV_ERR_UNSUPPORTED over the budget.
lnv_status tile_plan_build(lnv_ctx *ctx, lnv_plan *pl, size_t budget_bytes);
void tile_plan_free(TilePlan *tt);
lnv_status scan_exclusive(cudaStream_t st, const int64_t *in, int64_t n, int64_t *out);
void group_plan_free(GroupPlan *gp);
// Triple-list plan (triples.cu); LNV_ERR_UNSUPPORTED when it would not fit the budget.
lnv_status triple_plan_build(lnv_ctx *ctx, lnv_plan *pl, size_t budget_bytes);
void triple_plan_free(TriplePlan *tp);
lnv_status pattern_host_cols(lnv_ctx *ctx, const lnv_pattern *p);
lnv_status multiply(lnv_ctx *ctx, const lnv_plan *plan, int nsf, lnv_prec prec, const void *A,
                    const void *B, void *C);
// Two products sharing A and the patterns of B and C: C1 = A B1, C2 = A B2.
lnv_status multiply2(lnv_ctx *ctx, const lnv_plan *plan, int nsf, lnv_prec prec, const void *A,
                     const void *B1, const void *B2, void *C1, void *C2);

// Vectors on value arrays (minimize.cu): out = a x + b y (x, y not read when
// their factor is 0); *out_dev = x.y in FP64 (fixed-order reduction)
lnv_status vec_axpby(lnv_ctx *ctx, lnv_prec prec, int64_t n, double a, const void *x, double b, const void *y,
                     void *out);
lnv_status vec_dot(lnv_ctx *ctx, lnv_prec prec, int64_t n, const void *x, const void *y, double *out_dev);
// out = (x + x^T) / 2 for values on the symmetric block pattern P (out != x)
lnv_status sym_blocks(lnv_ctx *ctx, lnv_prec prec, const lnv_pattern *P, int nsf, const void *x, void *out);

// Traces and gradient (trace_grad.cu)
lnv_status trace_rows(lnv_ctx *ctx, const lnv_pattern *P, int nsf, lnv_prec prec, int nterms,
                      const void *const *A, const void *const *B, double *row_part);
lnv_status reduce_rows(lnv_ctx *ctx, const double *row_part, int64_t n, int nterms, int n_seg,
                       const int64_t *seg_off_dev, double *out, int stride, int offset);
lnv_status lnv_combine(lnv_ctx *ctx, int n_seg, double *out);
// W is stored on the upper triangle of L's pattern: block (i, j) of L's
// pattern reads W at w_map[p], transposed when j < i.
lnv_status grad_assemble(lnv_ctx *ctx, const lnv_pattern *PL, const int64_t *sub_LT,
                         const int64_t *w_map, int nsf, lnv_prec prec, const void *U, const void *W,
                         const void *Q, void *G);
// dN_e/dL = 12 (T - V) on L's pattern, T = SLS read through sub_LT, V = S Z.
lnv_status grad_ne_assemble(lnv_ctx *ctx, const lnv_pattern *PL, const int64_t *sub_LT, int nsf,
                            lnv_prec prec, const void *T, const void *V, void *GN);

}  // namespace lnv
