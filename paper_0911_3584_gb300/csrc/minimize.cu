// The minimisation of E(L) around the evaluation (Sec. 2): vector kernels on
// L's values and the host loop of a conjugate-gradient search with exact
// cubic line searches.
//
// The paper states the conditions (the electron count N_e = 2 Tr[KS] "easy to
// impose" within the minimisation, weak idempotency through Eq. 3) but prints
// no algorithm.  This loop takes the standard reading:
//   * the electron count is set by a chemical potential mu: the function
//     minimised is the grand potential Omega = E - mu N_e = 2 Tr[K (H - mu S)],
//     the band energy of H' = H - mu S, so one evaluation with H' gives Omega
//     and its gradient dE/dL(H') = dE/dL - mu dN_e/dL;
//   * gradients are the elementwise derivatives on L's stored entries, and the
//     search runs in the Euclidean inner product of those entries;
//   * directions follow Polak-Ribiere with restarts (beta < 0 -> 0, or no
//     descent -> steepest descent);
//   * Omega(L + tD) is a cubic polynomial in t (K is cubic in L), so each line
//     search fits it exactly from its value and slope at 0 and two more
//     evaluations, and takes the positive root of its derivative where the
//     curvature is positive.
// With mu inside a gap of the spectrum of (H, S) and no truncation the
// minimum is the projector on the states below mu.
#include <cmath>
#include <vector>

#include "lnv_impl.cuh"

namespace lnv {
namespace {

constexpr int kDotBlocks = 1216;  // 8 per SM on 152 SMs; fixed, so sums are reproducible
constexpr int kDotThreads = 256;

template <typename T>
__global__ void k_axpby(int64_t n, double a, const T *__restrict__ x, double b, const T *__restrict__ y,
                        T *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double xv = a != 0.0 ? (double)x[i] : 0.0;
        const double yv = b != 0.0 ? (double)y[i] : 0.0;
        out[i] = (T)(a * xv + b * yv);
    }
}

// FP64 partial sums of x.y: grid-stride per thread, then a fixed tree per block.
template <typename T>
__global__ void __launch_bounds__(kDotThreads)
k_dot_partial(int64_t n, const T *__restrict__ x, const T *__restrict__ y, double *__restrict__ part)
{
    __shared__ double red[kDotThreads];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)x[i] * (double)y[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kDotThreads) k_dot_final(const double *__restrict__ part, int np, double *out)
{
    __shared__ double red[kDotThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += kDotThreads) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// out = (x + x^T) / 2 on a symmetric block pattern: block p of out holds the
// mean of block p of x and the transpose of its mirror block tr[p].  out must
// not alias x.
template <typename T>
__global__ void k_sym_blocks(int64_t nnzb, int nsf, const int64_t *__restrict__ tr, const T *__restrict__ x,
                             T *__restrict__ out)
{
    const int bs = nsf * nsf;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnzb * bs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / bs;
        const int r = (int)(e - p * bs), a = r / nsf, b = r % nsf;
        out[e] = (T)(0.5 * ((double)x[e] + (double)x[tr[p] * bs + b * nsf + a]));
    }
}

lnv_status ctx_scratch(lnv_ctx *ctx, size_t n_doubles, double **out)
{
    if (ctx->scratch_n < n_doubles) {
        cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_n = 0;
        LNV_CUDA(cudaMalloc(&ctx->scratch, sizeof(double) * n_doubles));
        ctx->scratch_n = n_doubles;
    }
    *out = ctx->scratch;
    return LNV_OK;
}

unsigned vec_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4864, (n + 255) / 256)); }

}  // namespace

lnv_status sym_blocks(lnv_ctx *ctx, lnv_prec prec, const lnv_pattern *P, int nsf, const void *x, void *out)
{
    const int64_t n = P->nnzb * (int64_t)nsf * nsf;
    if (n == 0) return LNV_OK;
    if (!P->symmetric || !P->tr) {
        set_error("symmetrisation needs a symmetric pattern");
        return LNV_ERR_PATTERN;
    }
    if (prec == LNV_FP64)
        k_sym_blocks<double><<<vec_grid(n), 256, 0, ctx->stream>>>(P->nnzb, nsf, P->tr, (const double *)x,
                                                                  (double *)out);
    else
        k_sym_blocks<float><<<vec_grid(n), 256, 0, ctx->stream>>>(P->nnzb, nsf, P->tr, (const float *)x,
                                                                 (float *)out);
    LNV_LAUNCHED();
    return LNV_OK;
}

lnv_status vec_axpby(lnv_ctx *ctx, lnv_prec prec, int64_t n, double a, const void *x, double b, const void *y,
                     void *out)
{
    if (n <= 0) return LNV_OK;
    if (prec == LNV_FP64)
        k_axpby<double><<<vec_grid(n), 256, 0, ctx->stream>>>(n, a, (const double *)x, b, (const double *)y,
                                                             (double *)out);
    else
        k_axpby<float><<<vec_grid(n), 256, 0, ctx->stream>>>(n, a, (const float *)x, b, (const float *)y,
                                                            (float *)out);
    LNV_LAUNCHED();
    return LNV_OK;
}

// out_dev: one double, written on the context stream.
lnv_status vec_dot(lnv_ctx *ctx, lnv_prec prec, int64_t n, const void *x, const void *y, double *out_dev)
{
    double *part = nullptr;
    LNV_TRY(ctx_scratch(ctx, kDotBlocks + 8, &part));
    if (prec == LNV_FP64)
        k_dot_partial<double><<<kDotBlocks, kDotThreads, 0, ctx->stream>>>(n, (const double *)x, (const double *)y,
                                                                         part);
    else
        k_dot_partial<float><<<kDotBlocks, kDotThreads, 0, ctx->stream>>>(n, (const float *)x, (const float *)y,
                                                                        part);
    LNV_LAUNCHED();
    k_dot_final<<<1, kDotThreads, 0, ctx->stream>>>(part, kDotBlocks, out_dev);
    LNV_LAUNCHED();
    return LNV_OK;
}

}  // namespace lnv

using namespace lnv;

namespace {

lnv_status set_dev(const lnv_ctx *ctx)
{
    LNV_ARG(ctx, "null context");
    LNV_CUDA(cudaSetDevice(ctx->device));
    return LNV_OK;
}

// Host side of the minimisation: device buffers and FP64 scalars.
struct Minimiser {
    lnv_ctx *ctx;
    lnv_system *sys;
    const void *S;
    void *L;
    lnv_prec prec;
    int64_t n;       // stored entries of L
    size_t bytes;    // bytes of one L-sized array
    void *Hp = nullptr;  // H - mu S on the pattern of S and H
    void *G = nullptr, *D = nullptr, *g_old = nullptr, *Lt = nullptr;
    double *dev = nullptr;  // [8] device scalars: out[6], dot
    int evals = 0;

    ~Minimiser()
    {
        cudaFree(Hp); cudaFree(G); cudaFree(D); cudaFree(g_old); cudaFree(Lt); cudaFree(dev);
    }

    lnv_status alloc(size_t h_bytes)
    {
        LNV_CUDA(cudaMalloc(&Hp, std::max<size_t>(h_bytes, 16)));
        for (void **p : {&G, &D, &g_old, &Lt}) LNV_CUDA(cudaMalloc(p, std::max<size_t>(bytes, 16)));
        LNV_CUDA(cudaMalloc(&dev, sizeof(double) * 8));
        return LNV_OK;
    }

    // Omega (the energy of H') and N_e at M, and dOmega/dL into G when asked
    lnv_status eval(const void *M, bool grad, double *Om, double *Ne)
    {
        LNV_TRY(lnv_energy_grad(ctx, sys, S, Hp, M, dev, grad ? G : nullptr, nullptr, nullptr, 0));
        double h[2];
        LNV_CUDA(cudaMemcpyAsync(h, dev, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
        LNV_CUDA(cudaStreamSynchronize(ctx->stream));
        *Om = h[0];
        *Ne = h[1];
        ++evals;
        return LNV_OK;
    }

    lnv_status dot(const void *x, const void *y, double *v)
    {
        LNV_TRY(vec_dot(ctx, prec, n, x, y, dev + 6));
        LNV_CUDA(cudaMemcpyAsync(v, dev + 6, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        LNV_CUDA(cudaStreamSynchronize(ctx->stream));
        return LNV_OK;
    }
};

// values f(t1), f(2 t1) of f(t) = f0 + f1 t + c2 t^2 + c3 t^3 -> (c2, c3)
void fit_cubic(double f0, double f1, double t1, double fa, double fb, double *c2, double *c3)
{
    const double r1 = fa - f0 - f1 * t1, r2 = fb - f0 - 2.0 * f1 * t1;
    *c3 = (r2 - 4.0 * r1) / (4.0 * t1 * t1 * t1);
    *c2 = (r1 - *c3 * t1 * t1 * t1) / (t1 * t1);
}

// smallest t > 0 with slope + 2 c2 t + 3 c3 t^2 = 0 and 2 c2 + 6 c3 t > 0, else 0
double cubic_min(double slope, double c2, double c3)
{
    const double qa = 3.0 * c3, qb = 2.0 * c2, qc = slope;
    double r[2];
    int nr = 0;
    if (qa == 0.0) {
        if (qb != 0.0) r[nr++] = -qc / qb;
    } else {
        const double disc = qb * qb - 4.0 * qa * qc;
        if (disc >= 0.0) {
            const double sq = std::sqrt(disc);
            const double q = -0.5 * (qb + (qb >= 0.0 ? sq : -sq));
            if (q != 0.0) {
                r[nr++] = q / qa;
                r[nr++] = qc / q;
            } else {
                r[nr++] = 0.0;
            }
        }
    }
    double t = 0.0;
    for (int i = 0; i < nr; ++i)
        if (r[i] > 0.0 && 2.0 * c2 + 6.0 * c3 * r[i] > 0.0 && (t == 0.0 || r[i] < t)) t = r[i];
    return t;
}

}  // namespace

extern "C" lnv_status lnv_vec_axpby(lnv_ctx *ctx, lnv_prec prec, int64_t n, double a, const void *x_dev,
                                    double b, const void *y_dev, void *out_dev)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(prec == LNV_FP64 || prec == LNV_FP32, "unknown precision");
    LNV_ARG(n >= 0 && (n == 0 || (out_dev && (a == 0.0 || x_dev) && (b == 0.0 || y_dev))), "null pointer");
    return vec_axpby(ctx, prec, n, a, x_dev, b, y_dev, out_dev);
}

extern "C" lnv_status lnv_vec_dot(lnv_ctx *ctx, lnv_prec prec, int64_t n, const void *x_dev, const void *y_dev,
                                  double *out_dev)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(prec == LNV_FP64 || prec == LNV_FP32, "unknown precision");
    LNV_ARG(n >= 0 && out_dev && (n == 0 || (x_dev && y_dev)), "null pointer");
    return vec_dot(ctx, prec, n, x_dev, y_dev, out_dev);
}

extern "C" lnv_status lnv_minimize(lnv_ctx *ctx, lnv_system *sys, const void *S_dev, const void *H_dev,
                                   void *L_dev, double mu, int max_iter, double tol, double *hist_host,
                                   int *iters_out)
{
    LNV_TRY(set_dev(ctx));
    LNV_ARG(ctx && sys && S_dev && H_dev && L_dev && iters_out, "null pointer");
    LNV_ARG(max_iter >= 0 && tol > 0.0, "max_iter < 0 or tol <= 0");
    LNV_ARG((((uintptr_t)S_dev | (uintptr_t)H_dev | (uintptr_t)L_dev) & 15u) == 0,
            "value arrays must be 16-byte aligned");
    const lnv_pattern *PSH = nullptr, *PL = nullptr;
    LNV_TRY(lnv_system_patterns(sys, &PSH, &PL));
    int nseg = 0, nsf = 0;
    lnv_prec prec = LNV_FP64;
    LNV_TRY(lnv_system_info(sys, &nsf, &prec, &nseg));
    if (nseg != 1) {
        set_error("lnv_minimize: one system per call (this one holds %d)", nseg);
        return LNV_ERR_UNSUPPORTED;
    }
    const size_t es = prec == LNV_FP64 ? 8 : 4;
    const int64_t bs = (int64_t)nsf * nsf;
    Minimiser M{ctx, sys, S_dev, L_dev, prec, PL->nnzb * bs, 0};
    M.bytes = (size_t)M.n * es;
    LNV_TRY(M.alloc((size_t)(PSH->nnzb * bs) * es));
    // H' = H - mu S (S and H share their pattern)
    LNV_TRY(vec_axpby(ctx, prec, PSH->nnzb * bs, 1.0, H_dev, -mu, S_dev, M.Hp));
    // The gradient formula holds for symmetric L (W is formed on one triangle,
    // HLS is read as (SLH)^T), so L and every step are kept exactly symmetric:
    // L is symmetrised once and each gradient projected on symmetric matrices.
    LNV_TRY(sym_blocks(ctx, prec, PL, nsf, L_dev, M.Lt));
    LNV_TRY(vec_axpby(ctx, prec, M.n, 1.0, M.Lt, 0.0, M.Lt, L_dev));
    double Om = 0.0, Ne = 0.0, gg_old = 0.0, t_prev = 0.0;
    int it = 0;
    for (;; ++it) {
        LNV_TRY(M.eval(L_dev, true, &Om, &Ne));
        LNV_TRY(sym_blocks(ctx, prec, PL, nsf, M.G, M.Lt));
        std::swap(M.G, M.Lt);
        double gg = 0.0;
        LNV_TRY(M.dot(M.G, M.G, &gg));
        const double g_rms = std::sqrt(gg / (double)std::max<int64_t>(1, M.n));
        if (hist_host) {
            double *h = hist_host + 5 * it;
            h[0] = Om;
            h[1] = Om + mu * Ne;  // E
            h[2] = Ne;
            h[3] = g_rms;
            h[4] = t_prev;
        }
        if (g_rms <= tol || it >= max_iter) break;
        // Polak-Ribiere direction, restarted when beta < 0 or no descent
        double beta = 0.0;
        if (it > 0 && gg_old > 0.0) {
            double go = 0.0;
            LNV_TRY(M.dot(M.G, M.g_old, &go));
            beta = std::max(0.0, (gg - go) / gg_old);
        }
        LNV_TRY(vec_axpby(ctx, prec, M.n, -1.0, M.G, beta, M.D, M.D));
        double slope = 0.0, dd = 0.0;
        LNV_TRY(M.dot(M.G, M.D, &slope));
        if (!(slope < 0.0)) {
            LNV_TRY(vec_axpby(ctx, prec, M.n, -1.0, M.G, 0.0, M.G, M.D));
            slope = -gg;
        }
        LNV_TRY(M.dot(M.D, M.D, &dd));
        // exact cubic line search along D
        const double t_ref = 0.1 / std::sqrt(std::max(dd, 1e-300));
        const double t1 = t_prev > 1e-3 * t_ref ? t_prev : t_ref;
        double fa, fb, na, nb;
        LNV_TRY(vec_axpby(ctx, prec, M.n, 1.0, L_dev, t1, M.D, M.Lt));
        LNV_TRY(M.eval(M.Lt, false, &fa, &na));
        LNV_TRY(vec_axpby(ctx, prec, M.n, 1.0, L_dev, 2.0 * t1, M.D, M.Lt));
        LNV_TRY(M.eval(M.Lt, false, &fb, &nb));
        double c2, c3;
        fit_cubic(Om, slope, t1, fa, fb, &c2, &c3);
        double t = cubic_min(slope, c2, c3);
        if (t == 0.0) t = 2.0 * t1;   // no minimum ahead: take the farther trial point
        if (t < 1e-8 * t_ref) break;  // Omega differences at rounding: no further progress
        LNV_TRY(vec_axpby(ctx, prec, M.n, 1.0, L_dev, t, M.D, L_dev));
        t_prev = t;
        std::swap(M.G, M.g_old);
        gg_old = gg;
    }
    *iters_out = it;
    return LNV_OK;
}
