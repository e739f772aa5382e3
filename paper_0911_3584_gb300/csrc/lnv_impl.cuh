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

}  // namespace lnv

struct lnv_ctx {
    int device;
    cudaStream_t stream;
    int sm_count;
    size_t smem_optin;
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
};

struct lnv_plan {
    const lnv_pattern *A, *B, *C;
    int trans_a, trans_b;
    int mode;            // 0 push (row gather into a shared-memory row accumulator), 1 pull
    int64_t triples;     // contributing block triples
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
void pattern_free(lnv_pattern *p);
// position map of every block of `sub` inside `super` (both sorted), -1 if absent
lnv_status pattern_submap(lnv_ctx *ctx, const lnv_pattern *sub, const lnv_pattern *super,
                          int64_t *map_dev);

// Product internals (mult.cu)
lnv_status plan_create(lnv_ctx *ctx, const lnv_pattern *A, const lnv_pattern *B,
                       const lnv_pattern *C, int flags, lnv_plan **out);
lnv_status multiply(lnv_ctx *ctx, const lnv_plan *plan, int nsf, lnv_prec prec, const void *A,
                    const void *B, void *C);
// Two products sharing A and the patterns of B and C: C1 = A B1, C2 = A B2.
lnv_status multiply2(lnv_ctx *ctx, const lnv_plan *plan, int nsf, lnv_prec prec, const void *A,
                     const void *B1, const void *B2, void *C1, void *C2);

// Traces and gradient (trace_grad.cu)
lnv_status trace_rows(lnv_ctx *ctx, const lnv_pattern *P, int nsf, lnv_prec prec, int nterms,
                      const void *const *A, const void *const *B, double *row_part);
lnv_status reduce_rows(lnv_ctx *ctx, const double *row_part, int64_t n, int nterms, int n_seg,
                       const int64_t *seg_off_dev, double *out, int stride, int offset);
lnv_status lnv_combine(lnv_ctx *ctx, int n_seg, double *out);
lnv_status grad_assemble(lnv_ctx *ctx, const lnv_pattern *PL, const int64_t *sub_LT, int nsf,
                         lnv_prec prec, const void *U, const void *W, const void *Q, void *G);

}  // namespace lnv
