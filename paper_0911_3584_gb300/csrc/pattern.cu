// a0: range patterns {(i, j): d_ij^2 < R^2} from positions, with a cell list.
//
// Locality in the method (Sec. 2) is a distance criterion: L_ij = 0 beyond R_L,
// and every product of range-limited matrices is itself range-limited.  The
// pattern of each matrix is therefore a neighbour list.  Atoms are binned into
// boxes of side >= R per segment (one segment per independent system), each
// atom tests the atoms of its 27 (or fewer, for small boxes) neighbouring bins,
// rows are counted, scanned, filled and sorted in shared memory, and the
// transpose map tr[p] = position of (j, i) is found by binary search.
//
// The distance test is the exact FP64 recipe of the header: minimum image
// d - box*rint(d/box) per axis, d^2 = ((dx*dx)+(dy*dy))+(dz*dz), each
// operation a separately rounded IEEE intrinsic (no FMA contraction).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>

#include "lnv_impl.cuh"

namespace lnv {
namespace {

__device__ __forceinline__ double min_image(double d, double box)
{
    double t = __ddiv_rn(d, box);
    double r = rint(t);
    double m = __dmul_rn(box, r);
    return __dsub_rn(d, m);
}

__device__ __forceinline__ double dist2(const double *pi, const double *pj, const double *cell)
{
    double dx = min_image(__dsub_rn(pj[0], pi[0]), cell[0]);
    double dy = min_image(__dsub_rn(pj[1], pi[1]), cell[1]);
    double dz = min_image(__dsub_rn(pj[2], pi[2]), cell[2]);
    double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return __dadd_rn(s, __dmul_rn(dz, dz));
}

struct SegGrid {
    int64_t off0, off1;   // atom range
    double cell[3];
    int nb[3];            // bins per axis
    int64_t bin0;         // first global bin id
};

__device__ __forceinline__ int seg_of(const SegGrid *segs, int n_seg, int64_t i)
{
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].off0 <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int bin_axis(double x, double box, int nb)
{
    double w = x - box * floor(x / box);  // wrapped into [0, box] (binning only)
    int b = (int)floor(w * (double)nb / box);
    return b < 0 ? 0 : (b >= nb ? nb - 1 : b);
}

__global__ void k_bin_atoms(const double *__restrict__ pos, int64_t n, const SegGrid *segs,
                            int n_seg, int32_t *atom_seg, int64_t *atom_bin,
                            unsigned long long *bin_count)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = seg_of(segs, n_seg, i);
    const SegGrid &g = segs[s];
    int bx = bin_axis(pos[3 * i + 0], g.cell[0], g.nb[0]);
    int by = bin_axis(pos[3 * i + 1], g.cell[1], g.nb[1]);
    int bz = bin_axis(pos[3 * i + 2], g.cell[2], g.nb[2]);
    int64_t b = g.bin0 + ((int64_t)bx * g.nb[1] + by) * g.nb[2] + bz;
    atom_seg[i] = s;
    atom_bin[i] = b;
    atomicAdd(&bin_count[b], 1ull);
}

__global__ void k_bin_scatter(const int64_t *__restrict__ atom_bin, int64_t n,
                              const int64_t *__restrict__ bin_start,
                              unsigned long long *bin_fill, int32_t *bin_atoms)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t b = atom_bin[i];
    unsigned long long slot = atomicAdd(&bin_fill[b], 1ull);
    bin_atoms[bin_start[b] + (int64_t)slot] = (int32_t)i;
}

// Neighbouring bins along one axis: b-1, b, b+1 (periodic) when nb >= 3,
// otherwise every bin of the axis once.
__device__ __forceinline__ int axis_bins(int b, int nb, int *out)
{
    if (nb >= 3) {
        out[0] = (b + nb - 1) % nb;
        out[1] = b;
        out[2] = (b + 1) % nb;
        return 3;
    }
    for (int k = 0; k < nb; ++k) out[k] = k;
    return nb;
}

// One thread per atom: count (col == nullptr) or write its neighbours.
__global__ void k_neighbours(const double *__restrict__ pos, int64_t n, const SegGrid *segs,
                             const int32_t *__restrict__ atom_seg,
                             const int64_t *__restrict__ atom_bin,
                             const int64_t *__restrict__ bin_start,
                             const int32_t *__restrict__ bin_atoms, double R2,
                             int64_t *__restrict__ row_cnt, const int64_t *__restrict__ row_ptr,
                             int32_t *__restrict__ col)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SegGrid &g = segs[atom_seg[i]];
    int64_t lb = atom_bin[i] - g.bin0;
    int bz = (int)(lb % g.nb[2]);
    int by = (int)((lb / g.nb[2]) % g.nb[1]);
    int bx = (int)(lb / ((int64_t)g.nb[2] * g.nb[1]));
    int xs[3], ys[3], zs[3];
    int nx = axis_bins(bx, g.nb[0], xs), ny = axis_bins(by, g.nb[1], ys),
        nz = axis_bins(bz, g.nb[2], zs);
    double pi[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    int64_t c = 0;
    int64_t w = col ? row_ptr[i] : 0;
    for (int a = 0; a < nx; ++a)
        for (int b = 0; b < ny; ++b)
            for (int e = 0; e < nz; ++e) {
                int64_t bin = g.bin0 + ((int64_t)xs[a] * g.nb[1] + ys[b]) * g.nb[2] + zs[e];
                for (int64_t q = bin_start[bin]; q < bin_start[bin + 1]; ++q) {
                    int32_t j = bin_atoms[q];
                    double pj[3] = {pos[3 * (int64_t)j], pos[3 * (int64_t)j + 1],
                                    pos[3 * (int64_t)j + 2]};
                    if (dist2(pi, pj, g.cell) < R2) {
                        if (col) col[w + c] = j;
                        ++c;
                    }
                }
            }
    if (!col) row_cnt[i] = c;
}

// Bitonic sort of one row per CTA in shared memory (len <= cap, cap a power of 2).
__global__ void k_sort_rows(const int64_t *__restrict__ row_ptr, int32_t *col)
{
    extern __shared__ int32_t sbuf[];
    int64_t i = blockIdx.x;
    int64_t b = row_ptr[i], e = row_ptr[i + 1];
    int len = (int)(e - b);
    if (len <= 1) return;
    int cap = 1;
    while (cap < len) cap <<= 1;
    for (int t = threadIdx.x; t < cap; t += blockDim.x) sbuf[t] = t < len ? col[b + t] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= cap; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < cap; t += blockDim.x) {
                int u = t ^ j;
                if (u > t) {
                    bool up = (t & k) == 0;
                    int32_t x = sbuf[t], y = sbuf[u];
                    if ((x > y) == up) {
                        sbuf[t] = y;
                        sbuf[u] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < len; t += blockDim.x) col[b + t] = sbuf[t];
}

__global__ void k_row_of(const int64_t *__restrict__ row_ptr, int64_t n, int32_t *row)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) row[p] = (int32_t)i;
}

__device__ __forceinline__ int64_t find_col(const int32_t *col, int64_t lo, int64_t hi, int32_t j)
{
    int64_t end = hi;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && col[lo] == j) ? lo : -1;
}

// Validation of a caller pattern: columns in range and strictly ascending.
__global__ void k_validate(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                           int64_t n, int *bad)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t b = row_ptr[i], e = row_ptr[i + 1];
    if (e < b) {
        atomicOr(bad, 1);
        return;
    }
    for (int64_t p = b; p < e; ++p) {
        int32_t j = col[p];
        if (j < 0 || j >= n || (p > b && col[p - 1] >= j)) {
            atomicOr(bad, 1);
            return;
        }
    }
}

__global__ void k_transpose_map(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                const int32_t *__restrict__ row, int64_t nnzb, int64_t *tr,
                                int *asym)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nnzb) return;
    int32_t i = row[p], j = col[p];
    int64_t q = find_col(col, row_ptr[j], row_ptr[j + 1], i);
    tr[p] = q;
    if (q < 0) atomicOr(asym, 1);
}

__global__ void k_submap(const int64_t *__restrict__ s_rp, const int32_t *__restrict__ s_col,
                         const int32_t *__restrict__ s_row, int64_t nnzb,
                         const int64_t *__restrict__ p_rp, const int32_t *__restrict__ p_col,
                         int64_t *map)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nnzb) return;
    int32_t i = s_row[p];
    map[p] = find_col(p_col, p_rp[i], p_rp[i + 1], s_col[p]);
}

// Values of one pattern carried onto another: block (i, j) of `to` takes
// block (i, j) of `from`, or zeros where `from` has none.
template <typename T>
__global__ void k_remap(int64_t nnzb, int bs, const int32_t *__restrict__ t_row, const int32_t *__restrict__ t_col,
                        const int64_t *__restrict__ f_rp, const int32_t *__restrict__ f_col,
                        const T *__restrict__ f_val, T *__restrict__ t_val)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nnzb) return;
    const int32_t i = t_row[p];
    const int64_t q = find_col(f_col, f_rp[i], f_rp[i + 1], t_col[p]);
    for (int e = 0; e < bs; ++e) t_val[p * bs + e] = q >= 0 ? f_val[q * bs + e] : T(0);
}

// Exclusive scan of int64 counts: out[0..n], out[n] = total.
__global__ void k_scan_block(const int64_t *__restrict__ in, int64_t n, int64_t *out,
                             int64_t *block_sums)
{
    __shared__ int64_t warp_tot[32];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int64_t t = lane < nw ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t pre = wid > 0 ? warp_tot[wid - 1] : 0;
    if (i < n) out[i] = pre + x - v;
    if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = pre + x;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *__restrict__ block_off)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && blockIdx.x > 0) out[i] += block_off[blockIdx.x];
}

}  // namespace

// out must hold n+1 values.
lnv_status scan_exclusive(cudaStream_t st, const int64_t *in, int64_t n, int64_t *out)
{
    const int T = 1024;
    int64_t nb = (n + T - 1) / T;
    if (nb == 0) {
        LNV_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return LNV_OK;
    }
    int64_t *sums = nullptr, *offs = nullptr;
    LNV_CUDA(cudaMalloc(&sums, sizeof(int64_t) * nb));
    LNV_CUDA(cudaMalloc(&offs, sizeof(int64_t) * (nb + 1)));
    k_scan_block<<<(unsigned)nb, T, 0, st>>>(in, n, out, sums);
    LNV_LAUNCHED();
    lnv_status s = LNV_OK;
    if (nb > 1) {
        s = scan_exclusive(st, sums, nb, offs);
        if (s == LNV_OK) {
            k_scan_add<<<(unsigned)nb, T, 0, st>>>(out, n, offs);
            count_launch();
            s = cudaGetLastError() == cudaSuccess ? LNV_OK : LNV_ERR_CUDA;
        }
        // total = offs[nb]
        if (s == LNV_OK)
            LNV_CUDA(cudaMemcpyAsync(out + n, offs + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    } else {
        LNV_CUDA(cudaMemcpyAsync(out + n, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    }
    LNV_CUDA(cudaStreamSynchronize(st));
    cudaFree(sums);
    cudaFree(offs);
    return s;
}

void pattern_free(lnv_pattern *p)
{
    if (!p) return;
    cudaFree(p->row_ptr);
    cudaFree(p->col);
    cudaFree(p->row);
    cudaFree(p->tr);
    delete p;
}

// Given row_ptr and col filled: sort rows (optional), fill row[], tr[], host copies.
lnv_status pattern_finish(lnv_ctx *ctx, lnv_pattern *p, bool sort_rows)
{
    cudaStream_t st = ctx->stream;
    p->h_row_ptr.resize(p->n + 1);
    LNV_CUDA(cudaMemcpyAsync(p->h_row_ptr.data(), p->row_ptr, sizeof(int64_t) * (p->n + 1),
                             cudaMemcpyDeviceToHost, st));
    LNV_CUDA(cudaStreamSynchronize(st));
    p->nnzb = p->h_row_ptr[p->n];
    int64_t mx = 0;
    for (int64_t i = 0; i < p->n; ++i) mx = std::max(mx, p->h_row_ptr[i + 1] - p->h_row_ptr[i]);
    p->max_row = (int)mx;
    if (sort_rows && mx > 1) {
        if (mx > kMaxRow) {
            set_error("pattern row of %lld blocks exceeds the supported %d", (long long)mx, kMaxRow);
            return LNV_ERR_UNSUPPORTED;
        }
        int cap = 1;
        while (cap < mx) cap <<= 1;
        size_t smem = sizeof(int32_t) * cap;
        LNV_CUDA(cudaFuncSetAttribute(k_sort_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        k_sort_rows<<<(unsigned)p->n, 256, smem, st>>>(p->row_ptr, p->col);
        LNV_LAUNCHED();
    }
    int64_t nn = std::max<int64_t>(p->nnzb, 1);
    LNV_CUDA(cudaMalloc(&p->row, sizeof(int32_t) * nn));
    LNV_CUDA(cudaMalloc(&p->tr, sizeof(int64_t) * nn));
    if (p->n > 0) {
        k_row_of<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(p->row_ptr, p->n, p->row);
        LNV_LAUNCHED();
    }
    int *d_asym = nullptr;
    LNV_CUDA(cudaMalloc(&d_asym, sizeof(int)));
    LNV_CUDA(cudaMemsetAsync(d_asym, 0, sizeof(int), st));
    if (p->nnzb > 0) {
        k_transpose_map<<<(unsigned)((p->nnzb + 255) / 256), 256, 0, st>>>(
            p->row_ptr, p->col, p->row, p->nnzb, p->tr, d_asym);
        LNV_LAUNCHED();
    }
    int asym = 0;
    LNV_CUDA(cudaMemcpyAsync(&asym, d_asym, sizeof(int), cudaMemcpyDeviceToHost, st));
    LNV_CUDA(cudaStreamSynchronize(st));
    cudaFree(d_asym);
    p->symmetric = asym ? 0 : 1;
    return LNV_OK;
}

lnv_status pattern_build_impl(lnv_ctx *ctx, const double *pos, int n_seg, const int64_t *seg_off,
                              const double *cells, double cutoff, lnv_pattern **out)
{
    LNV_ARG(out && pos && seg_off && cells && n_seg >= 1, "null pointer or n_seg < 1");
    LNV_ARG(cutoff > 0 && std::isfinite(cutoff), "cutoff must be positive and finite");
    cudaStream_t st = ctx->stream;
    const int64_t n = seg_off[n_seg];
    LNV_ARG(seg_off[0] == 0 && n >= 0, "segment offsets must start at 0");
    std::vector<SegGrid> segs(n_seg);
    int64_t nbins = 0;
    for (int s = 0; s < n_seg; ++s) {
        SegGrid &g = segs[s];
        g.off0 = seg_off[s];
        g.off1 = seg_off[s + 1];
        LNV_ARG(g.off1 >= g.off0, "segment offsets must be non-decreasing");
        for (int d = 0; d < 3; ++d) {
            double box = cells[3 * s + d];
            LNV_ARG(box > 0 && std::isfinite(box), "cell lengths must be positive");
            g.cell[d] = box;
            double nb = std::floor(box / (cutoff * (1.0 + 1e-6)));
            g.nb[d] = (int)std::max(1.0, std::min(nb, 1024.0));
        }
        // At most ~2 bins per atom: fewer, wider bins stay correct (width >= R).
        const double target = std::max(27.0, 2.0 * (double)(g.off1 - g.off0));
        for (int it = 0; it < 64 && (double)g.nb[0] * g.nb[1] * g.nb[2] > target; ++it) {
            int d = (g.nb[0] >= g.nb[1] && g.nb[0] >= g.nb[2]) ? 0 : (g.nb[1] >= g.nb[2] ? 1 : 2);
            g.nb[d] = std::max(1, (int)(g.nb[d] * 0.8));
        }
        g.bin0 = nbins;
        nbins += (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
    }
    lnv_pattern *p = new lnv_pattern();
    p->n = n;
    SegGrid *d_segs = nullptr;
    int32_t *atom_seg = nullptr, *bin_atoms = nullptr;
    int64_t *atom_bin = nullptr, *bin_start = nullptr, *row_cnt = nullptr;
    unsigned long long *bin_count = nullptr;
    int64_t *bin_count64 = nullptr;
    lnv_status s = LNV_OK;
    auto fail = [&](lnv_status e) {
        cudaFree(d_segs); cudaFree(atom_seg); cudaFree(bin_atoms); cudaFree(atom_bin);
        cudaFree(bin_start); cudaFree(row_cnt); cudaFree(bin_count); cudaFree(bin_count64);
        if (e != LNV_OK) pattern_free(p);
        return e;
    };
#define STEP(x)                                   \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) {                  \
            set_error("%s: %s", #x, cudaGetErrorString(e_)); \
            return fail(e_ == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA); \
        }                                         \
    } while (0)
    int64_t nn = std::max<int64_t>(n, 1);
    STEP(cudaMalloc(&d_segs, sizeof(SegGrid) * n_seg));
    STEP(cudaMemcpyAsync(d_segs, segs.data(), sizeof(SegGrid) * n_seg, cudaMemcpyHostToDevice, st));
    STEP(cudaMalloc(&atom_seg, sizeof(int32_t) * nn));
    STEP(cudaMalloc(&atom_bin, sizeof(int64_t) * nn));
    STEP(cudaMalloc(&bin_atoms, sizeof(int32_t) * nn));
    STEP(cudaMalloc(&bin_count, sizeof(unsigned long long) * nbins));
    STEP(cudaMalloc(&bin_count64, sizeof(int64_t) * nbins));
    STEP(cudaMalloc(&bin_start, sizeof(int64_t) * (nbins + 1)));
    STEP(cudaMalloc(&row_cnt, sizeof(int64_t) * nn));
    STEP(cudaMalloc(&p->row_ptr, sizeof(int64_t) * (n + 1)));
    STEP(cudaMemsetAsync(bin_count, 0, sizeof(unsigned long long) * nbins, st));
    unsigned g = (unsigned)((n + 255) / 256);
    if (n > 0) {
        k_bin_atoms<<<g, 256, 0, st>>>(pos, n, d_segs, n_seg, atom_seg, atom_bin, bin_count);
        count_launch();
        STEP(cudaGetLastError());
    }
    STEP(cudaMemcpyAsync(bin_count64, bin_count, sizeof(int64_t) * nbins, cudaMemcpyDeviceToDevice, st));
    s = scan_exclusive(st, bin_count64, nbins, bin_start);
    if (s != LNV_OK) return fail(s);
    STEP(cudaMemsetAsync(bin_count, 0, sizeof(unsigned long long) * nbins, st));
    if (n > 0) {
        k_bin_scatter<<<g, 256, 0, st>>>(atom_bin, n, bin_start, bin_count, bin_atoms);
        count_launch();
        STEP(cudaGetLastError());
        k_neighbours<<<g, 256, 0, st>>>(pos, n, d_segs, atom_seg, atom_bin, bin_start, bin_atoms,
                                         cutoff * cutoff, row_cnt, nullptr, nullptr);
        count_launch();
        STEP(cudaGetLastError());
    }
    s = scan_exclusive(st, row_cnt, n, p->row_ptr);
    if (s != LNV_OK) return fail(s);
    int64_t nnzb = 0;
    STEP(cudaMemcpyAsync(&nnzb, p->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    STEP(cudaStreamSynchronize(st));
    if (nnzb >= (int64_t)INT_MAX) {
        set_error("pattern has %lld blocks; at most 2^31-1 are supported", (long long)nnzb);
        return fail(LNV_ERR_UNSUPPORTED);
    }
    STEP(cudaMalloc(&p->col, sizeof(int32_t) * std::max<int64_t>(nnzb, 1)));
    if (n > 0) {
        k_neighbours<<<g, 256, 0, st>>>(pos, n, d_segs, atom_seg, atom_bin, bin_start, bin_atoms,
                                         cutoff * cutoff, nullptr, p->row_ptr, p->col);
        count_launch();
        STEP(cudaGetLastError());
    }
#undef STEP
    s = pattern_finish(ctx, p, true);
    if (s != LNV_OK) return fail(s);
    fail(LNV_OK);
    *out = p;
    return LNV_OK;
}

// Upper triangle (col >= row) of a pattern, as its own (non-symmetric) pattern.
lnv_status pattern_upper(lnv_ctx *ctx, const lnv_pattern *P, lnv_pattern **out)
{
    LNV_TRY(pattern_host_cols(ctx, P));
    lnv_pattern *u = new lnv_pattern();
    u->n = P->n;
    std::vector<int64_t> rp(P->n + 1, 0);
    std::vector<int32_t> col;
    col.reserve(P->nnzb / 2 + P->n);
    for (int64_t i = 0; i < P->n; ++i) {
        for (int64_t q = P->h_row_ptr[i]; q < P->h_row_ptr[i + 1]; ++q)
            if (P->h_col[q] >= i) col.push_back(P->h_col[q]);
        rp[i + 1] = (int64_t)col.size();
    }
    cudaError_t e = cudaMalloc(&u->row_ptr, sizeof(int64_t) * (P->n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&u->col, sizeof(int32_t) * std::max<size_t>(col.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(u->row_ptr, rp.data(), sizeof(int64_t) * (P->n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !col.empty())
        e = cudaMemcpy(u->col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pattern_free(u);
        set_error("upper pattern: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LNV_ERR_OOM : LNV_ERR_CUDA;
    }
    lnv_status s = pattern_finish(ctx, u, false);
    if (s != LNV_OK) {
        pattern_free(u);
        return s;
    }
    *out = u;
    return LNV_OK;
}

namespace {
// For every block (i, j) of P: position of (min, max) = (i, j) or (j, i) in U.
__global__ void k_upper_map(const int32_t *__restrict__ p_row, const int32_t *__restrict__ p_col, int64_t nnzb,
                            const int64_t *__restrict__ u_rp, const int32_t *__restrict__ u_col, int64_t *map)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nnzb) return;
    const int32_t i = p_row[p], j = p_col[p];
    const int32_t r = i <= j ? i : j, c = i <= j ? j : i;
    map[p] = find_col(u_col, u_rp[r], u_rp[r + 1], c);
}
}  // namespace

lnv_status pattern_upper_map(lnv_ctx *ctx, const lnv_pattern *P, const lnv_pattern *U, int64_t *map_dev)
{
    if (P->nnzb == 0) return LNV_OK;
    k_upper_map<<<(unsigned)((P->nnzb + 255) / 256), 256, 0, ctx->stream>>>(P->row, P->col, P->nnzb,
                                                                          U->row_ptr, U->col, map_dev);
    LNV_LAUNCHED();
    return LNV_OK;
}

lnv_status pattern_submap(lnv_ctx *ctx, const lnv_pattern *sub, const lnv_pattern *super,
                          int64_t *map_dev)
{
    if (sub->nnzb == 0) return LNV_OK;
    k_submap<<<(unsigned)((sub->nnzb + 255) / 256), 256, 0, ctx->stream>>>(
        sub->row_ptr, sub->col, sub->row, sub->nnzb, super->row_ptr, super->col, map_dev);
    LNV_LAUNCHED();
    return LNV_OK;
}

lnv_status pattern_remap(lnv_ctx *ctx, const lnv_pattern *from, const lnv_pattern *to, int nsf, lnv_prec prec,
                         const void *from_vals, void *to_vals)
{
    if (from->n != to->n) {
        set_error("remap between patterns of %lld and %lld atoms", (long long)from->n, (long long)to->n);
        return LNV_ERR_PATTERN;
    }
    if (to->nnzb == 0) return LNV_OK;
    const unsigned grid = (unsigned)((to->nnzb + 255) / 256);
    if (prec == LNV_FP64)
        k_remap<double><<<grid, 256, 0, ctx->stream>>>(to->nnzb, nsf * nsf, to->row, to->col, from->row_ptr,
                                                       from->col, (const double *)from_vals, (double *)to_vals);
    else
        k_remap<float><<<grid, 256, 0, ctx->stream>>>(to->nnzb, nsf * nsf, to->row, to->col, from->row_ptr,
                                                      from->col, (const float *)from_vals, (float *)to_vals);
    LNV_LAUNCHED();
    return LNV_OK;
}

lnv_status pattern_validate(lnv_ctx *ctx, const lnv_pattern *p)
{
    int *bad = nullptr;
    LNV_CUDA(cudaMalloc(&bad, sizeof(int)));
    LNV_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    if (p->n > 0) {
        k_validate<<<(unsigned)((p->n + 255) / 256), 256, 0, ctx->stream>>>(p->row_ptr, p->col, p->n, bad);
        LNV_LAUNCHED();
    }
    int h = 0;
    LNV_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LNV_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaFree(bad);
    if (h) {
        set_error("pattern rows must hold ascending columns in [0, n)");
        return LNV_ERR_PATTERN;
    }
    return LNV_OK;
}

}  // namespace lnv
