// The extern "C" surface of liblnv (declared in include/lnv.h).
//
// An LNV evaluation (Sec. 2, Eq. 3) runs, on the context stream:
//   X = L S, Y = L H            push product, one kernel for both (shared A = L)
//   T = S X, U = S Y            push product, one kernel for both (shared A = S);
//                               T = SLS is symmetric: its lower triangle is mirrored
//   Z = L T  masked to R_X      pull product
//   Tr[XY], Tr[ZY], Tr[XX], Tr[ZX] -> E, N_e   (one fused FP64 trace pass)
//   Q = H Z  masked to R_L      pull product
//   W = X^T U^T masked to R_L   (= SL HLS = SLHLS, symmetric: upper triangle only)
//   G = 6(U + U^T) - 4(Q^T + W + Q) on L's pattern
// with R_X = R_L + R_SH and R_T = R_L + 2 R_SH: X, Y, T, U are the exact full
// products (the minimum-image distance obeys the triangle inequality, so A B
// vanishes beyond R_A + R_B), and Z is needed only inside R_X.
#include <atomic>
#include <cmath>
#include <map>
#include <set>
#include <mutex>
#include <utility>
#include <cstdarg>
#include <cstring>
#include <new>

#include "lnv_impl.cuh"

namespace lnv {

static thread_local char g_err[512] = "";
static std::atomic<int64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaError_t ensure_smem(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;  // (kernel, device) -> bytes
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    const std::pair<const void *, int> key(kernel, dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = set.find(key);
    if (it != set.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) set[key] = bytes;
    return e;
}

cudaError_t prefer_smem(const void *kernel)
{
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;  // (kernel, device)
    int dev = 0;
    cudaGetDevice(&dev);
    const std::pair<const void *, int> key(kernel, dev);
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(key)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

}  // namespace lnv

using namespace lnv;

struct lnv_system {
    int nsf = 0;
    lnv_prec prec = LNV_FP64;
    int64_t n = 0;
    int n_seg = 1;
    double r_sh = 0, r_l = 0;
    int64_t *seg_off_dev = nullptr;
    lnv_pattern *P_sh = nullptr, *P_l = nullptr, *P_x = nullptr, *P_t = nullptr;
    lnv_pattern *P_lu = nullptr;  // upper triangle of P_l: W = SLHLS is symmetric
    int64_t *w_map = nullptr;     // block of P_l -> its (min, max) block in P_lu
    lnv_plan *pl_xy = nullptr, *pl_tu = nullptr, *pl_z = nullptr, *pl_q = nullptr, *pl_w = nullptr;
    int64_t *sub_lt = nullptr;  // position in P_t of every block of P_l
    void *own_ws = nullptr;
    size_t own_ws_bytes = 0;
    // device copies of the host arrays of lnv_energy_grad_host (allocated on first use)
    void *io_dev = nullptr;
    // stage timing (lnv_system_profile): events before XY, TU, Z, traces, Q, W, G and at the end
    static constexpr int kStages = 7;
    int profile = 0;
    int profiled_grad = 0;
    cudaEvent_t ev[kStages + 1] = {};
};

namespace {

size_t elem_size(lnv_prec p) { return p == LNV_FP64 ? 8 : 4; }

// Device value arrays start on 16-byte boundaries (NULL passes: optional arrays).
bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
    size_t X, Y, Z, T, U, W, Q, V, rows, total;
};

WsLayout ws_layout(const lnv_system *s, int with_grad)
{
    WsLayout L{};
    const size_t bs = (size_t)s->nsf * s->nsf * elem_size(s->prec);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    L.X = take(s->P_x->nnzb * bs);
    L.Y = take(s->P_x->nnzb * bs);
    L.Z = take(s->P_x->nnzb * bs);
    L.T = take(s->P_t->nnzb * bs);
    L.U = with_grad ? take(s->P_t->nnzb * bs) : 0;
    L.W = with_grad ? take(s->P_lu->nnzb * bs) : 0;
    L.Q = with_grad ? take(s->P_l->nnzb * bs) : 0;
    L.V = take(s->P_l->nnzb * bs);  // S Z for dN_e/dL
    L.rows = take(sizeof(double) * 4 * (size_t)std::max<int64_t>(s->n, 1));
    L.total = off;
    return L;
}

void system_free(lnv_system *s)
{
    if (!s) return;
    plan_free(s->pl_xy); plan_free(s->pl_tu); plan_free(s->pl_z); plan_free(s->pl_q); plan_free(s->pl_w);
    pattern_free(s->P_sh); pattern_free(s->P_l); pattern_free(s->P_x); pattern_free(s->P_t);
    pattern_free(s->P_lu);
    cudaFree(s->w_map);
    cudaFree(s->sub_lt);
    cudaFree(s->seg_off_dev);
    cudaFree(s->own_ws);
    cudaFree(s->io_dev);
    for (auto &e : s->ev)
        if (e) cudaEventDestroy(e);
    delete s;
}

lnv_status set_dev(const lnv_ctx *ctx)
{
    LNV_ARG(ctx, "null context");
    LNV_CUDA(cudaSetDevice(ctx->device));
    return LNV_OK;
}

}  // namespace

extern "C" {

const char *lnv_last_error(void) { return g_err; }

int64_t lnv_launch_count(void) { return g_launches.load(); }

const char *lnv_version(void) { return "liblnv 0.1 (sm_103a)"; }

lnv_status lnv_ctx_create(int device, void *cuda_stream, lnv_ctx **out)
{
    LNV_ARG(out, "null output");
    int ndev = 0;
    LNV_CUDA(cudaGetDeviceCount(&ndev));
    LNV_ARG(device >= 0 && device < ndev, "device index out of range");
    LNV_CUDA(cudaSetDevice(device));
    lnv_ctx *c = new (std::nothrow) lnv_ctx();
    if (!c) {
        set_error("host allocation failed");
        return LNV_ERR_OOM;
    }
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    c->sm_count = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)v;
    cudaError_t e = cudaMalloc(&c->dev_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->dev_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(c->dev_status);
        delete c;
        set_error("context status word: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA;
    }
    *out = c;
    return LNV_OK;
}

lnv_status lnv_ctx_device_status(lnv_ctx *ctx)
{
    LNV_TRY(set_dev(ctx));
    int h = 0;
    LNV_CUDA(cudaMemcpyAsync(&h, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LNV_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h == 0) return LNV_OK;
    LNV_CUDA(cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), ctx->stream));
    LNV_CUDA(cudaStreamSynchronize(ctx->stream));
    set_error("a device-side wait ran out; the outputs of the kernels since the last check are undefined");
    return LNV_ERR_TIMEOUT;
}

lnv_status lnv_ctx_set_wait_limit(lnv_ctx *ctx, uint64_t ns)
{
    LNV_ARG(ctx && ns > 0, "wait limit must be positive");
    ctx->wait_ns = (unsigned long long)ns;
    return LNV_OK;
}

lnv_status lnv_ctx_set_stream(lnv_ctx *ctx, void *cuda_stream)
{
    LNV_ARG(ctx, "null context");
    ctx->stream = (cudaStream_t)cuda_stream;
    return LNV_OK;
}

lnv_status lnv_ctx_destroy(lnv_ctx *ctx)
{
    if (ctx) {
        cudaFree(ctx->scratch);
        cudaFree(ctx->prod_scratch);
        cudaFree(ctx->dev_status);
    }
    delete ctx;
    return LNV_OK;
}

lnv_status lnv_pattern_build(lnv_ctx *ctx, const double *pos_dev, int64_t n_atoms,
                             const double *cell_host, double cutoff, lnv_pattern **out)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(n_atoms >= 0 && n_atoms < INT32_MAX, "n_atoms out of range");
    LNV_ARG(cell_host, "null cell");
    int64_t off[2] = {0, n_atoms};
    return pattern_build_impl(ctx, pos_dev, 1, off, cell_host, cutoff, out);
}

lnv_status lnv_pattern_build_batched(lnv_ctx *ctx, const double *pos_dev, int n_seg,
                                     const int64_t *seg_off_host, const double *cells_host,
                                     double cutoff, lnv_pattern **out)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(n_seg >= 1 && seg_off_host && cells_host, "bad segments");
    LNV_ARG(seg_off_host[n_seg] < INT32_MAX, "too many atoms");
    return pattern_build_impl(ctx, pos_dev, n_seg, seg_off_host, cells_host, cutoff, out);
}

lnv_status lnv_pattern_from_csr(lnv_ctx *ctx, int64_t n, const int64_t *row_ptr_dev,
                                const int32_t *col_dev, lnv_pattern **out)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(out && row_ptr_dev && (n >= 0) && n < INT32_MAX, "bad pattern arguments");
    lnv_pattern *p = new lnv_pattern();
    p->n = n;
    int64_t nnzb = 0;
    cudaError_t e = cudaMemcpyAsync(&nnzb, row_ptr_dev + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && (nnzb < 0 || nnzb >= INT32_MAX)) {
        pattern_free(p);
        set_error("pattern block count %lld out of range", (long long)nnzb);
        return LNV_ERR_PATTERN;
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->row_ptr, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&p->col, sizeof(int32_t) * std::max<int64_t>(nnzb, 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->row_ptr, row_ptr_dev, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && nnzb > 0) {
        LNV_ARG(col_dev, "null columns");
        e = cudaMemcpyAsync(p->col, col_dev, sizeof(int32_t) * nnzb, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    if (e != cudaSuccess) {
        pattern_free(p);
        set_error("pattern copy failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA;
    }
    lnv_status s = pattern_validate(ctx, p);
    if (s == LNV_OK) s = pattern_finish(ctx, p, false);
    if (s != LNV_OK) {
        pattern_free(p);
        return s;
    }
    *out = p;
    return LNV_OK;
}

lnv_status lnv_pattern_info(const lnv_pattern *p, int64_t *n, int64_t *nnzb,
                            const int64_t **row_ptr_dev, const int32_t **col_dev,
                            const int64_t **tr_dev, int *symmetric)
{
    LNV_ARG(p, "null pattern");
    if (n) *n = p->n;
    if (nnzb) *nnzb = p->nnzb;
    if (row_ptr_dev) *row_ptr_dev = p->row_ptr;
    if (col_dev) *col_dev = p->col;
    if (tr_dev) *tr_dev = p->tr;
    if (symmetric) *symmetric = p->symmetric;
    return LNV_OK;
}

lnv_status lnv_pattern_destroy(lnv_pattern *p)
{
    pattern_free(p);
    return LNV_OK;
}

lnv_status lnv_plan_product(lnv_ctx *ctx, const lnv_pattern *A, const lnv_pattern *B,
                            const lnv_pattern *C, int flags, lnv_plan **out)
{
    LNV_TRY(set_dev(ctx));
    return plan_create(ctx, A, B, C, flags, out);
}

lnv_status lnv_plan_info(const lnv_plan *plan, int64_t *triples, int *mode)
{
    LNV_ARG(plan, "null plan");
    if (triples) *triples = plan->triples;
    if (mode) *mode = plan->mode;
    return LNV_OK;
}

lnv_status lnv_plan_set_kernel(lnv_ctx *ctx, lnv_plan *plan, int kernel)
{
    LNV_TRY(set_dev(ctx));
    return plan_set_kernel(ctx, plan, kernel);
}

lnv_status lnv_plan_destroy(lnv_plan *plan)
{
    plan_free(plan);
    return LNV_OK;
}

lnv_status lnv_bsr_multiply(lnv_ctx *ctx, const lnv_plan *plan, int nsf, lnv_prec prec,
                            const void *A_dev, const void *B_dev, void *C_dev, double alpha, double beta)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(plan, "null plan");
    LNV_ARG(aligned16(A_dev) && aligned16(B_dev) && aligned16(C_dev), "value arrays must be 16-byte aligned");
    LNV_ARG(prec == LNV_FP64 || prec == LNV_FP32, "unknown precision");
    const int64_t n = plan->C->nnzb * (int64_t)nsf * nsf;
    if (beta == 0.0) {
        LNV_TRY(multiply(ctx, plan, nsf, prec, A_dev, B_dev, C_dev));
        if (alpha != 1.0) LNV_TRY(vec_axpby(ctx, prec, n, alpha, C_dev, 0.0, nullptr, C_dev));
        return LNV_OK;
    }
    const size_t bytes = (size_t)std::max<int64_t>(n, 1) * elem_size(prec);
    if (ctx->prod_scratch_bytes < bytes) {
        LNV_CUDA(cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->prod_scratch);
        ctx->prod_scratch = nullptr;
        ctx->prod_scratch_bytes = 0;
        LNV_CUDA(cudaMalloc(&ctx->prod_scratch, bytes));
        ctx->prod_scratch_bytes = bytes;
    }
    LNV_TRY(multiply(ctx, plan, nsf, prec, A_dev, B_dev, ctx->prod_scratch));
    return vec_axpby(ctx, prec, n, alpha, ctx->prod_scratch, beta, C_dev, C_dev);
}

lnv_status lnv_trace_product(lnv_ctx *ctx, const lnv_pattern *P, int nsf, lnv_prec prec,
                             const void *A_dev, const void *B_dev, double *scratch_dev,
                             double *out_dev)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(P && A_dev && B_dev && scratch_dev && out_dev, "null pointer");
    LNV_ARG(aligned16(A_dev) && aligned16(B_dev), "value arrays must be 16-byte aligned");
    const void *A[1] = {A_dev}, *B[1] = {B_dev};
    LNV_TRY(trace_rows(ctx, P, nsf, prec, 1, A, B, scratch_dev));
    return reduce_rows(ctx, scratch_dev, P->n, 1, 1, nullptr, out_dev, 1, 0);
}

lnv_status lnv_system_create(lnv_ctx *ctx, int nsf, lnv_prec prec, const double *pos_dev,
                             int64_t n_atoms, int n_seg, const int64_t *seg_off_host,
                             const double *cells_host, double r_sh, double r_l, lnv_system **out)
{
    return lnv_system_create_truncated(ctx, nsf, prec, pos_dev, n_atoms, n_seg, seg_off_host, cells_host, r_sh,
                                       r_l, 0.0, 0.0, out);
}

lnv_status lnv_system_create_truncated(lnv_ctx *ctx, int nsf, lnv_prec prec, const double *pos_dev,
                                       int64_t n_atoms, int n_seg, const int64_t *seg_off_host,
                                       const double *cells_host, double r_sh, double r_l, double r_x,
                                       double r_t, lnv_system **out)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(out && pos_dev && cells_host, "null pointer");
    LNV_ARG(nsf == 1 || nsf == 2 || nsf == 4 || nsf == 9, "NSF must be 1, 2, 4 or 9");
    LNV_ARG(prec == LNV_FP64 || prec == LNV_FP32, "unknown precision");
    LNV_ARG(n_seg >= 1, "n_seg < 1");
    LNV_ARG(r_sh > 0 && r_l > 0, "ranges must be positive");
    if (r_x <= 0.0) r_x = r_l + r_sh;
    if (r_t <= 0.0) r_t = r_l + 2 * r_sh;
    LNV_ARG(r_x >= r_l && r_x <= r_l + r_sh, "r_x must lie in [r_l, r_l + r_sh]");
    LNV_ARG(r_t >= r_l && r_t <= r_l + 2 * r_sh, "r_t must lie in [r_l, r_l + 2 r_sh]");
    std::vector<int64_t> off(n_seg + 1);
    if (n_seg == 1 && !seg_off_host) {
        off[0] = 0;
        off[1] = n_atoms;
    } else {
        LNV_ARG(seg_off_host, "seg_off_host is required for n_seg > 1");
        for (int s = 0; s <= n_seg; ++s) off[s] = seg_off_host[s];
        LNV_ARG(off[n_seg] == n_atoms, "segment offsets must end at n_atoms");
    }
    LNV_ARG(n_atoms >= 0 && n_atoms < INT32_MAX, "n_atoms out of range");
    lnv_system *s = new lnv_system();
    s->nsf = nsf;
    s->prec = prec;
    s->n = n_atoms;
    s->n_seg = n_seg;
    s->r_sh = r_sh;
    s->r_l = r_l;
    lnv_status st = LNV_OK;
#define SYS_TRY(expr)              \
    do {                           \
        st = (expr);               \
        if (st != LNV_OK) {        \
            system_free(s);        \
            return st;             \
        }                          \
    } while (0)
    SYS_TRY(pattern_build_impl(ctx, pos_dev, n_seg, off.data(), cells_host, r_sh, &s->P_sh));
    SYS_TRY(pattern_build_impl(ctx, pos_dev, n_seg, off.data(), cells_host, r_l, &s->P_l));
    SYS_TRY(pattern_build_impl(ctx, pos_dev, n_seg, off.data(), cells_host, r_x, &s->P_x));
    SYS_TRY(pattern_build_impl(ctx, pos_dev, n_seg, off.data(), cells_host, r_t, &s->P_t));
    SYS_TRY(plan_create(ctx, s->P_l, s->P_sh, s->P_x, 0, &s->pl_xy));
    // T = SLS is symmetric when X = LS is exact (L symmetric): only its upper
    // triangle is formed, the lower one mirrored.  With X truncated it is not.
    SYS_TRY(plan_create(ctx, s->P_sh, s->P_x, s->P_t, r_x >= r_l + r_sh ? LNV_SYM_C : 0, &s->pl_tu));
    // Z = L T: T = SLS is symmetric, so L T = L T^T; the transposed form lets
    // the merge-join pull read T's row j in order instead of through tr.
    SYS_TRY(plan_create(ctx, s->P_l, s->P_t, s->P_x, LNV_TRANS_B, &s->pl_z));
    SYS_TRY(plan_create(ctx, s->P_sh, s->P_x, s->P_l, 0, &s->pl_q));
    // W = X^T U^T = SLHLS is symmetric: only its upper triangle is formed
    SYS_TRY(pattern_upper(ctx, s->P_l, &s->P_lu));
    SYS_TRY(plan_create(ctx, s->P_x, s->P_t, s->P_lu, LNV_TRANS_A | LNV_TRANS_B, &s->pl_w));
    cudaError_t e = cudaMalloc(&s->sub_lt, sizeof(int64_t) * std::max<int64_t>(s->P_l->nnzb, 1));
    if (e == cudaSuccess) e = cudaMalloc(&s->w_map, sizeof(int64_t) * std::max<int64_t>(s->P_l->nnzb, 1));
    if (e == cudaSuccess) e = cudaMalloc(&s->seg_off_dev, sizeof(int64_t) * (n_seg + 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->seg_off_dev, off.data(), sizeof(int64_t) * (n_seg + 1), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
        system_free(s);
        set_error("system allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA;
    }
    SYS_TRY(pattern_submap(ctx, s->P_l, s->P_t, s->sub_lt));
    SYS_TRY(pattern_upper_map(ctx, s->P_l, s->P_lu, s->w_map));
#undef SYS_TRY
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        system_free(s);
        set_error("system setup failed: %s", cudaGetErrorString(e));
        return LNV_ERR_CUDA;
    }
    *out = s;
    return LNV_OK;
}

lnv_status lnv_pattern_remap(lnv_ctx *ctx, const lnv_pattern *from, const lnv_pattern *to, int nsf,
                             lnv_prec prec, const void *from_vals_dev, void *to_vals_dev)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(from && to && (to->nnzb == 0 || (from_vals_dev && to_vals_dev)), "null pointer");
    LNV_ARG(nsf == 1 || nsf == 2 || nsf == 4 || nsf == 9, "NSF must be 1, 2, 4 or 9");
    LNV_ARG(prec == LNV_FP64 || prec == LNV_FP32, "unknown precision");
    LNV_ARG(from_vals_dev != to_vals_dev || to->nnzb == 0, "the value arrays must not alias");
    LNV_ARG(aligned16(from_vals_dev) && aligned16(to_vals_dev), "value arrays must be 16-byte aligned");
    return pattern_remap(ctx, from, to, nsf, prec, from_vals_dev, to_vals_dev);
}

lnv_status lnv_system_info(const lnv_system *sys, int *nsf, lnv_prec *prec, int *n_seg)
{
    LNV_ARG(sys, "null system");
    if (nsf) *nsf = sys->nsf;
    if (prec) *prec = sys->prec;
    if (n_seg) *n_seg = sys->n_seg;
    return LNV_OK;
}

lnv_status lnv_system_patterns(const lnv_system *sys, const lnv_pattern **sh, const lnv_pattern **l)
{
    LNV_ARG(sys, "null system");
    if (sh) *sh = sys->P_sh;
    if (l) *l = sys->P_l;
    return LNV_OK;
}

lnv_status lnv_system_workspace_size(const lnv_system *sys, int with_grad, size_t *bytes)
{
    LNV_ARG(sys && bytes, "null pointer");
    *bytes = ws_layout(sys, with_grad).total;
    return LNV_OK;
}

lnv_status lnv_system_triples(const lnv_system *sys, int with_grad, int64_t *triples)
{
    LNV_ARG(sys && triples, "null pointer");
    // X, Y (two products), T (its upper triangle when the lower one is
    // mirrored), Z, then U, Q and W
    const lnv_plan *tu = sys->pl_tu;
    int64_t t = 2 * sys->pl_xy->triples + (tu->sym1 && tu->split ? tu->triples_up : tu->triples) +
                sys->pl_z->triples;
    if (with_grad) t += tu->triples + sys->pl_q->triples + sys->pl_w->triples;
    *triples = t;
    return LNV_OK;
}

lnv_status lnv_system_stage_kernels(const lnv_system *sys, int *k7)
{
    LNV_ARG(sys && k7, "null pointer");
    k7[0] = sys->pl_xy->mode;
    k7[1] = sys->pl_tu->mode;
    k7[2] = sys->pl_z->mode;
    k7[3] = -1;
    k7[4] = sys->pl_q->mode;
    k7[5] = sys->pl_w->mode;
    k7[6] = -1;
    return LNV_OK;
}

lnv_status lnv_system_set_stage_kernel(lnv_ctx *ctx, lnv_system *sys, int stage, int kernel)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(sys, "null system");
    lnv_plan *pl = stage == 0 ? sys->pl_xy : stage == 1 ? sys->pl_tu : stage == 2 ? sys->pl_z
                 : stage == 4 ? sys->pl_q : stage == 5 ? sys->pl_w : nullptr;
    LNV_ARG(pl, "stage must be 0 (XY), 1 (TU), 2 (Z), 4 (Q) or 5 (W)");
    return plan_set_kernel(ctx, pl, kernel);
}

lnv_status lnv_system_set_mirror(lnv_ctx *ctx, lnv_system *sys, int on)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(sys, "null system");
    if (on && !sys->pl_tu->sym1) {
        set_error("T is not symmetric on a system with truncated X");
        return LNV_ERR_UNSUPPORTED;
    }
    return plan_set_split(ctx, sys->pl_tu, on);
}

lnv_status lnv_system_mirror(const lnv_system *sys, int *on)
{
    LNV_ARG(sys && on, "null pointer");
    *on = sys->pl_tu->sym1 && sys->pl_tu->split;
    return LNV_OK;
}

lnv_status lnv_system_autotune(lnv_ctx *ctx, lnv_system *sys, const void *S_dev, const void *H_dev,
                               const void *L_dev, int reps, double *ms_out)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(sys && S_dev && H_dev && L_dev, "null pointer");
    LNV_ARG(aligned16(S_dev) && aligned16(H_dev) && aligned16(L_dev), "value arrays must be 16-byte aligned");
    if (reps < 1) reps = 1;
    // one evaluation fills the intermediates the products read
    const WsLayout wl = ws_layout(sys, 1);
    void *G = nullptr;
    double *out = nullptr;
    LNV_CUDA(cudaMalloc(&G, (size_t)sys->P_l->nnzb * sys->nsf * sys->nsf * elem_size(sys->prec) + 16));
    cudaError_t e = cudaMalloc(&out, sizeof(double) * 6 * (size_t)sys->n_seg);
    if (e != cudaSuccess) {
        cudaFree(G);
        set_error("autotune allocation: %s", cudaGetErrorString(e));
        return LNV_ERR_OOM;
    }
    lnv_status st = lnv_energy_grad(ctx, sys, S_dev, H_dev, L_dev, out, G, nullptr, nullptr, 0);
    unsigned char *ws = (unsigned char *)sys->own_ws;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == LNV_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        set_error("autotune: event creation failed");
        st = LNV_ERR_CUDA;
    }
    struct Stage {
        lnv_plan *pl;
        const void *A, *B1, *B2;
        void *C1, *C2;
    };
    void *X = ws + wl.X, *Y = ws + wl.Y, *Z = ws + wl.Z, *T = ws + wl.T, *U = ws + wl.U;
    void *W = ws + wl.W, *Q = ws + wl.Q;
    Stage stages[5] = {{sys->pl_xy, L_dev, S_dev, H_dev, X, Y},
                       {sys->pl_tu, S_dev, X, Y, T, U},
                       {sys->pl_z, L_dev, T, nullptr, Z, nullptr},
                       {sys->pl_q, H_dev, Z, nullptr, Q, nullptr},
                       {sys->pl_w, X, U, nullptr, W, nullptr}};
    for (int si = 0; si < 5 && st == LNV_OK; ++si) {
        Stage &sg = stages[si];
        const int orig = sg.pl->mode, orig_split = sg.pl->split;
        int best = orig, best_split = orig_split;
        float best_ms = 1e30f;
        for (int k = 0; k < LNV_NUM_KERNELS; ++k)
            if (ms_out) ms_out[si * LNV_NUM_KERNELS + k] = -1.0;
        // a symmetric first output (T): every kernel with the split (its upper
        // triangle, then the mirror) and without (formed whole)
        for (int split = sg.pl->sym1; split >= 0 && st == LNV_OK; --split) {
            st = plan_set_split(ctx, sg.pl, split);
            for (int k : {0, 2, 3, 4, 5, 8, 6, 7, 9, 10, 11}) {
                if (st != LNV_OK) break;
                // tcgen05 kernel: one FP32 product with NSF = 4 and op(B) = B^T
                if (k == 9 && (sys->nsf != 4 || sys->prec != LNV_FP32 || !sg.pl->trans_b || sg.B2)) continue;
                // its NSF = 9 form: FP32 products with NSF = 9
                if (k == 10 && (sys->nsf != 9 || sys->prec != LNV_FP32)) continue;
                // tcgen05 tiles over their own k lists: FP32 products with NSF = 4
                if (k == 11 && (sys->nsf != 4 || sys->prec != LNV_FP32)) continue;
                // per-warp ring kernel: FP32 values, NSF = 4 (elsewhere kernel 5 is kernel 3)
                if (k == 5 && (sys->nsf != 4 || sys->prec != LNV_FP32)) continue;
                // its half-width form: the same cases
                if (k == 8 && (sys->nsf != 4 || sys->prec != LNV_FP32)) continue;
                // tensor-core kernel: FP32 values, NSF = 4 (3xTF32, FP32-level accuracy)
                if (k == 6 && (sys->nsf != 4 || sys->prec != LNV_FP32)) continue;
                // listed triples: NSF = 4 (elsewhere kernel 7 is kernel 0)
                if (k == 7 && sys->nsf != 4) continue;
                if (plan_set_kernel(ctx, sg.pl, k) != LNV_OK) continue;
                lnv_status rs = multiply2(ctx, sg.pl, sys->nsf, sys->prec, sg.A, sg.B1, sg.B2, sg.C1, sg.C2);
                if (rs == LNV_OK && cudaEventRecord(e0, ctx->stream) == cudaSuccess) {
                    for (int r = 0; r < reps && rs == LNV_OK; ++r)
                        rs = multiply2(ctx, sg.pl, sys->nsf, sys->prec, sg.A, sg.B1, sg.B2, sg.C1, sg.C2);
                    float ms = 0.f;
                    if (rs == LNV_OK && cudaEventRecord(e1, ctx->stream) == cudaSuccess &&
                        cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
                        ms /= reps;
                        if (ms_out) {
                            double &slot = ms_out[si * LNV_NUM_KERNELS + k];
                            if (slot < 0 || ms < slot) slot = ms;
                        }
                        if (ms < best_ms) {
                            best_ms = ms;
                            best = k;
                            best_split = split;
                        }
                    }
                }
                if (rs != LNV_OK) st = rs;
            }
        }
        if (st == LNV_OK) st = plan_set_split(ctx, sg.pl, best_split);
        if (st == LNV_OK) st = plan_set_kernel(ctx, sg.pl, best);
        if (st != LNV_OK) {
            plan_set_split(ctx, sg.pl, orig_split);
            plan_set_kernel(ctx, sg.pl, orig);
        }
        if (st == LNV_OK) plan_trim(sg.pl);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(G);
    cudaFree(out);
    return st;
}

lnv_status lnv_system_stage_triples(const lnv_system *sys, int64_t *t7)
{
    LNV_ARG(sys && t7, "null pointer");
    t7[0] = 2 * sys->pl_xy->triples;  // X and Y
    // T (its upper triangle when it is mirrored) and U (U only with the gradient)
    const lnv_plan *tu = sys->pl_tu;
    t7[1] = (tu->sym1 && tu->split ? tu->triples_up : tu->triples) + tu->triples;
    t7[2] = sys->pl_z->triples;
    t7[3] = 0;
    t7[4] = sys->pl_q->triples;
    t7[5] = sys->pl_w->triples;
    t7[6] = 0;
    return LNV_OK;
}

lnv_status lnv_system_destroy(lnv_system *sys)
{
    system_free(sys);
    return LNV_OK;
}

lnv_status lnv_system_profile(lnv_system *sys, int enable)
{
    LNV_ARG(sys, "null system");
    if (enable)
        for (auto &e : sys->ev)
            if (!e) LNV_CUDA(cudaEventCreate(&e));
    sys->profile = enable ? 1 : 0;
    return LNV_OK;
}

lnv_status lnv_system_stage_ms(lnv_system *sys, double *ms)
{
    LNV_ARG(sys && ms, "null pointer");
    LNV_ARG(sys->ev[0], "profiling was never enabled");
    const int last = sys->profiled_grad ? lnv_system::kStages : 4;
    LNV_CUDA(cudaEventSynchronize(sys->ev[last]));
    for (int k = 0; k < lnv_system::kStages; ++k) {
        ms[k] = 0.0;
        if (k < last) {
            float f = 0.f;
            LNV_CUDA(cudaEventElapsedTime(&f, sys->ev[k], sys->ev[k + 1]));
            ms[k] = f;
        }
    }
    return LNV_OK;
}

lnv_status lnv_energy_grad_host(lnv_ctx *ctx, lnv_system *sys, const void *S_host, const void *H_host,
                                const void *L_host, double *out_host, void *G_host)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(sys && S_host && H_host && L_host && out_host, "null pointer");
    const size_t bs = (size_t)sys->nsf * sys->nsf * elem_size(sys->prec);
    const size_t n_sh = align256(bs * (size_t)sys->P_sh->nnzb), n_l = align256(bs * (size_t)sys->P_l->nnzb);
    const size_t n_out = align256(sizeof(double) * 6 * (size_t)sys->n_seg);
    if (!sys->io_dev) {
        // S, H, L, G, out, each on a 256-byte boundary
        cudaError_t e = cudaMalloc(&sys->io_dev, 2 * n_sh + 2 * n_l + n_out);
        if (e != cudaSuccess) {
            sys->io_dev = nullptr;
            set_error("host-evaluation buffers: %s", cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA;
        }
    }
    unsigned char *b = (unsigned char *)sys->io_dev;
    void *S = b, *H = b + n_sh, *L = b + 2 * n_sh, *G = b + 2 * n_sh + n_l;
    double *out = (double *)(b + 2 * n_sh + 2 * n_l);
    const size_t v_sh = bs * (size_t)sys->P_sh->nnzb, v_l = bs * (size_t)sys->P_l->nnzb;
    LNV_CUDA(cudaMemcpyAsync(S, S_host, v_sh, cudaMemcpyHostToDevice, ctx->stream));
    LNV_CUDA(cudaMemcpyAsync(H, H_host, v_sh, cudaMemcpyHostToDevice, ctx->stream));
    LNV_CUDA(cudaMemcpyAsync(L, L_host, v_l, cudaMemcpyHostToDevice, ctx->stream));
    LNV_TRY(lnv_energy_grad(ctx, sys, S, H, L, out, G_host ? G : nullptr, nullptr, nullptr, 0));
    LNV_CUDA(cudaMemcpyAsync(out_host, out, sizeof(double) * 6 * (size_t)sys->n_seg, cudaMemcpyDeviceToHost,
                             ctx->stream));
    if (G_host) LNV_CUDA(cudaMemcpyAsync(G_host, G, v_l, cudaMemcpyDeviceToHost, ctx->stream));
    LNV_CUDA(cudaStreamSynchronize(ctx->stream));
    return LNV_OK;
}

lnv_status lnv_energy_grad(lnv_ctx *ctx, lnv_system *sys, const void *S_dev, const void *H_dev,
                           const void *L_dev, double *out_dev, void *G_dev, void *GN_dev, void *ws_dev,
                           size_t ws_bytes)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(sys && S_dev && H_dev && L_dev && out_dev, "null pointer");
    LNV_ARG(aligned16(S_dev) && aligned16(H_dev) && aligned16(L_dev) && aligned16(G_dev) && aligned16(GN_dev) &&
                aligned16(ws_dev),
            "value arrays and the workspace must be 16-byte aligned");
    const int grad = G_dev != nullptr;
    const WsLayout wl = ws_layout(sys, grad);
    unsigned char *ws = (unsigned char *)ws_dev;
    if (!ws) {
        if (sys->own_ws_bytes < wl.total) {
            cudaFree(sys->own_ws);
            sys->own_ws = nullptr;
            sys->own_ws_bytes = 0;
            // the largest layout (with gradient) so later calls never reallocate
            size_t need = ws_layout(sys, 1).total;
            LNV_CUDA(cudaMalloc(&sys->own_ws, need));
            sys->own_ws_bytes = need;
        }
        ws = (unsigned char *)sys->own_ws;
    } else {
        LNV_ARG(ws_bytes >= wl.total, "workspace smaller than lnv_system_workspace_size");
    }
    void *X = ws + wl.X, *Y = ws + wl.Y, *Z = ws + wl.Z, *T = ws + wl.T;
    void *U = grad ? ws + wl.U : nullptr, *W = grad ? ws + wl.W : nullptr, *Q = grad ? ws + wl.Q : nullptr;
    void *V = ws + wl.V;
    double *rows = (double *)(ws + wl.rows);
    const int nsf = sys->nsf;
    const lnv_prec pr = sys->prec;
    auto mark = [&](int k) -> lnv_status {
        if (sys->profile) LNV_CUDA(cudaEventRecord(sys->ev[k], ctx->stream));
        return LNV_OK;
    };
    sys->profiled_grad = grad;
    LNV_TRY(mark(0));
    // a1: X = L S, Y = L H
    LNV_TRY(multiply2(ctx, sys->pl_xy, nsf, pr, L_dev, S_dev, H_dev, X, Y));
    LNV_TRY(mark(1));
    // a2: T = S X (= SLS), U = S Y (= SLH)
    if (grad) LNV_TRY(multiply2(ctx, sys->pl_tu, nsf, pr, S_dev, X, Y, T, U));
    else LNV_TRY(multiply(ctx, sys->pl_tu, nsf, pr, S_dev, X, T));
    LNV_TRY(mark(2));
    // a3: Z = L T (= LSLS) on R_X
    LNV_TRY(multiply(ctx, sys->pl_z, nsf, pr, L_dev, T, Z));
    LNV_TRY(mark(3));
    // a4: Tr[XY], Tr[ZY], Tr[XX], Tr[ZX] -> E, N_e per system
    const void *ta[4] = {X, Z, X, Z}, *tb[4] = {Y, Y, X, X};
    LNV_TRY(trace_rows(ctx, sys->P_x, nsf, pr, 4, ta, tb, rows));
    LNV_TRY(reduce_rows(ctx, rows, sys->n, 4, sys->n_seg, sys->seg_off_dev, out_dev, 6, 2));
    LNV_TRY(lnv_combine(ctx, sys->n_seg, out_dev));
    LNV_TRY(mark(4));
    if (grad) {
        // a6: Q = H Z (= HLSLS) on R_L;  a5: W = X^T U^T (= SLHLS) on R_L
        LNV_TRY(multiply(ctx, sys->pl_q, nsf, pr, H_dev, Z, Q));
        // V = S Z (= SLSLS) on R_L has the patterns of Q = H Z
        if (GN_dev) LNV_TRY(multiply(ctx, sys->pl_q, nsf, pr, S_dev, Z, V));
        LNV_TRY(mark(5));
        LNV_TRY(multiply(ctx, sys->pl_w, nsf, pr, X, U, W));
        LNV_TRY(mark(6));
        // a7: G = 6(U + U^T) - 4(Q^T + W + Q) on L's pattern
        LNV_TRY(grad_assemble(ctx, sys->P_l, sys->sub_lt, sys->w_map, nsf, pr, U, W, Q, G_dev));
        if (GN_dev) LNV_TRY(grad_ne_assemble(ctx, sys->P_l, sys->sub_lt, nsf, pr, T, V, GN_dev));
        LNV_TRY(mark(7));
    } else if (GN_dev) {
        // a7 (electron count): dN_e/dL = 12 (SLS - SLSLS) on L's pattern
        LNV_TRY(multiply(ctx, sys->pl_q, nsf, pr, S_dev, Z, V));
        LNV_TRY(grad_ne_assemble(ctx, sys->P_l, sys->sub_lt, nsf, pr, T, V, GN_dev));
    }
    return LNV_OK;
}

}  // extern "C"
