// Kernels of the masked block products; instantiated per (precision, NSF) in
// mult_inst_*.cu so that the library compiles in parallel.
#pragma once
#include <type_traits>
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

// ------------------------------------------------------------------ push2

// Row-gather product with warp-owned column slices.  CTA = (row i, column
// chunk [c0, c0 + chunk) of C's row), accumulated in shared memory.  Warp w
// owns a contiguous slice of the chunk's slots.  For each k of A's row i (in
// order), the blocks of B's row k whose column falls in warp w's slice form a
// contiguous sub-range (B's rows are sorted); the CTA finds all sub-range
// bounds with parallel binary searches once per staged k-chunk.  Lanes take
// (block, output row x, product) tasks of the sub-range: within one k every
// column j is distinct, so no two lanes touch one accumulator row, and a
// __syncwarp separates successive k.  Each slot therefore sums its k's in order
// (deterministic) and no CTA-wide barrier is needed inside the k loop.  SYM:
// the first output is symmetric and only its blocks with j >= i are formed
// (a further bound per k marks the diagonal in B's row); the lower triangle
// is mirrored afterwards.
template <typename T, int NSF, int NOUT, bool TA, bool TB, int NW, bool SYM>
__global__ void __launch_bounds__(NW * 32)
k_push2(const int64_t *__restrict__ a_rp, const int32_t *__restrict__ a_col,
        const int64_t *__restrict__ a_tr, const T *__restrict__ a_val,
        const int64_t *__restrict__ b_rp, const int32_t *__restrict__ b_col,
        const int64_t *__restrict__ b_tr, const T *__restrict__ b_val1,
        const T *__restrict__ b_val2, const int64_t *__restrict__ c_rp,
        const int32_t *__restrict__ c_col, T *__restrict__ c_val1, T *__restrict__ c_val2,
        int chunk, int kchunk)
{
    constexpr int BS = NSF * NSF;
    constexpr int NB = NW + 2;  // bounds per k: NW + 1 slice starts, then the diagonal
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *acc = reinterpret_cast<T *>(smem_raw);                      // [NOUT][chunk][BS]
    T *a_s = acc + (size_t)NOUT * chunk * BS;                      // [kchunk][BS]
    int32_t *ccol = reinterpret_cast<int32_t *>(a_s + (size_t)kchunk * BS);  // [chunk]
    int32_t *bnd = ccol + chunk;                                   // [kchunk][NB]
    int32_t *a_k = bnd + (size_t)kchunk * NB;                      // [kchunk]

    const int64_t i = blockIdx.x;
    const int64_t cb = c_rp[i], ce = c_rp[i + 1];
    const int64_t c0 = cb + (int64_t)blockIdx.y * chunk;
    if (c0 >= ce) return;
    const int cn = (int)min((int64_t)chunk, ce - c0);
    const int64_t ab = a_rp[i], ae = a_rp[i + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warp slices of the chunk: [sl0, sl1)
    const int per_w = (cn + NW - 1) / NW;
    const int sl0 = min(cn, warp * per_w), sl1 = min(cn, sl0 + per_w);

    for (int t = threadIdx.x; t < cn; t += blockDim.x) ccol[t] = c_col[c0 + t];
    for (int t = threadIdx.x; t < NOUT * chunk * BS; t += blockDim.x) acc[t] = T(0);

    for (int64_t k0 = ab; k0 < ae; k0 += kchunk) {
        const int kn = (int)min((int64_t)kchunk, ae - k0);
        __syncthreads();
        for (int t = threadIdx.x; t < kn * BS; t += blockDim.x) {
            const int qq = t / BS, e = t - qq * BS;
            const int64_t q = k0 + qq;
            if (TA) {
                const int x = e / NSF, z = e % NSF;
                a_s[t] = a_val[a_tr[q] * BS + z * NSF + x];
            } else {
                a_s[t] = a_val[q * BS + e];
            }
        }
        for (int t = threadIdx.x; t < kn; t += blockDim.x) a_k[t] = a_col[k0 + t];
        __syncthreads();
        // sub-range bounds: bnd[qq][w] = first block of B's row k with column >=
        // the first column of slice w (w = NW: past the chunk's last column;
        // w = NW + 1: column i, the diagonal)
        constexpr int nbw = SYM ? NB : NB - 1;  // the diagonal only when it is used
        for (int t = threadIdx.x; t < kn * nbw; t += blockDim.x) {
            const int qq = t / nbw, w = t - qq * nbw;
            const int32_t k = a_k[qq];
            const int s_w = min(cn, w * per_w);
            const int32_t jkey = w == NW + 1 ? (int32_t)i : s_w < cn ? ccol[s_w] : ccol[cn - 1] + 1;
            const int64_t rb = b_rp[k];
            bnd[qq * NB + w] = (int32_t)(lower_bound_g(b_col, rb, b_rp[k + 1], jkey) - rb);
        }
        __syncthreads();
        if (sl0 >= sl1) continue;
        for (int qq = 0; qq < kn; ++qq) {
            const int32_t k = a_k[qq];
            const int64_t rb = b_rp[k];
            const int64_t lo = rb + bnd[qq * NB + warp], hi = rb + bnd[qq * NB + warp + 1];
            // symmetric first output: its blocks left of the diagonal (j < i) are
            // not formed; those columns take the second product only, if any
            const int64_t pm = SYM ? max(lo, min(hi, rb + bnd[qq * NB + NW + 1])) : lo;
            // tasks (block, row x, product o): the products are separate tasks so
            // that a k's few blocks fill more of the warp's lanes
            const int n1 = (SYM && NOUT == 2) ? (int)(pm - lo) * NSF : 0;
            const int ntask = n1 + (int)(hi - pm) * NSF * NOUT;
            const T *as = a_s + (size_t)qq * BS;
            for (int t = lane; t < ntask; t += 32) {
                int64_t p;
                int x, o;
                if (t < n1) {
                    p = lo + t / NSF;
                    x = t % NSF;
                    o = NOUT - 1;
                } else {
                    const int t2 = t - n1, xo = t2 % (NSF * NOUT);
                    p = pm + t2 / (NSF * NOUT);
                    x = xo / NOUT;
                    o = xo - x * NOUT;
                }
                const int32_t j = __ldg(b_col + p);
                // slot of j inside this warp's slice
                int lo_s = sl0, hi_s = sl1;
                while (lo_s < hi_s) {
                    const int mid = (lo_s + hi_s) >> 1;
                    if (ccol[mid] < j) lo_s = mid + 1;
                    else hi_s = mid;
                }
                if (lo_s >= sl1 || ccol[lo_s] != j) continue;
                const int64_t pb = TB ? b_tr[p] : p;
                T ax[NSF];
#pragma unroll
                for (int z = 0; z < NSF; ++z) ax[z] = as[x * NSF + z];
                {
                    const T *bblk = (NOUT == 1 || o == 0 ? b_val1 : b_val2) + pb * BS;
                    T *ar = acc + ((size_t)o * chunk + lo_s) * BS + x * NSF;
                    T r[NSF];
#pragma unroll
                    for (int y = 0; y < NSF; ++y) r[y] = ar[y];
#pragma unroll
                    for (int z = 0; z < NSF; ++z) {
                        T br[NSF];
                        load_row<T, NSF, TB>(bblk, z, br);
#pragma unroll
                        for (int y = 0; y < NSF; ++y) r[y] = fma(ax[z], br[y], r[y]);
                    }
#pragma unroll
                    for (int y = 0; y < NSF; ++y) ar[y] = r[y];
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NOUT * cn * BS; t += blockDim.x) {
        const int o = t / (cn * BS), r = t - o * cn * BS;
        T *dst = o == 0 ? c_val1 : c_val2;
        dst[c0 * BS + r] = acc[(size_t)o * chunk * BS + r];
    }
}

// ------------------------------------------------------------------ pull2 (merge-join)

// Output-owner product for a symmetric B pattern.  Work item = (row i, first
// output slot); the CTA's threads own outputs start+t, start+t+blockDim, ...
// (OPT of them) and keep them in registers.  For output (i, j) the k's with
// op(B)_kj stored are the columns of B's row j (the pattern is symmetric), so
// each thread walks B's sorted row j forward, galloping to each k of A's row
// i (sorted, staged in shared memory): no per-k search from the row start.
// op(B)_kj is B[p]^T (TB: p is (j, k) in row j) or B[tr p] (block (k, j)).
template <typename T, int NSF, int OPT, bool TA, bool TB>
__global__ void __launch_bounds__(64)
k_pull2(const int2 *__restrict__ items, const int64_t *__restrict__ a_rp,
        const int32_t *__restrict__ a_col, const int64_t *__restrict__ a_tr,
        const T *__restrict__ a_val, const int64_t *__restrict__ b_rp,
        const int32_t *__restrict__ b_col, const int64_t *__restrict__ b_tr,
        const T *__restrict__ b_val, const int64_t *__restrict__ c_rp,
        const int32_t *__restrict__ c_col, T *__restrict__ c_val, int chunk_out, int kchunk)
{
    constexpr int BS = NSF * NSF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *a_s = reinterpret_cast<T *>(smem_raw);                               // [kchunk][BS]
    int32_t *a_k = reinterpret_cast<int32_t *>(a_s + (size_t)kchunk * BS);  // [kchunk]

    const int2 it = items[blockIdx.x];
    const int64_t i = it.x;
    const int64_t cb = c_rp[i], ce = c_rp[i + 1];
    const int64_t ab = a_rp[i], ae = a_rp[i + 1];
    const int64_t s_end = min(ce, cb + (int64_t)it.y + chunk_out);
    int64_t pos[OPT], end[OPT], cpos[OPT];
    T acc[OPT][BS];
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        cpos[o] = cb + it.y + threadIdx.x + (int64_t)o * blockDim.x;
        pos[o] = end[o] = 0;
        if (cpos[o] < s_end) {
            const int32_t j = c_col[cpos[o]];
            pos[o] = b_rp[j];
            end[o] = b_rp[j + 1];
        }
#pragma unroll
        for (int e = 0; e < BS; ++e) acc[o][e] = T(0);
    }
    for (int64_t k0 = ab; k0 < ae; k0 += kchunk) {
        const int kn = (int)min((int64_t)kchunk, ae - k0);
        __syncthreads();
        for (int t = threadIdx.x; t < kn * BS; t += blockDim.x) {
            const int qq = t / BS, e = t - qq * BS;
            const int64_t q = k0 + qq;
            if (TA) {
                const int x = e / NSF, z = e % NSF;
                a_s[t] = a_val[a_tr[q] * BS + z * NSF + x];
            } else {
                a_s[t] = a_val[q * BS + e];
            }
        }
        for (int t = threadIdx.x; t < kn; t += blockDim.x) a_k[t] = a_col[k0 + t];
        __syncthreads();
        for (int qq = 0; qq < kn; ++qq) {
            const int32_t k = a_k[qq];
            const T *as = a_s + (size_t)qq * BS;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (pos[o] >= end[o]) continue;
                pos[o] = gallop_g(b_col, pos[o], end[o], k);
                if (pos[o] >= end[o] || __ldg(b_col + pos[o]) != k) continue;
                const T *bblk = b_val + (TB ? pos[o] : b_tr[pos[o]]) * BS;
#pragma unroll
                for (int z = 0; z < NSF; ++z) {
                    T br[NSF];
                    load_row<T, NSF, TB>(bblk, z, br);
#pragma unroll
                    for (int x = 0; x < NSF; ++x) {
                        const T ax = as[x * NSF + z];
#pragma unroll
                        for (int y = 0; y < NSF; ++y) acc[o][x * NSF + y] = fma(ax, br[y], acc[o][x * NSF + y]);
                    }
                }
                ++pos[o];
            }
        }
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        if (cpos[o] >= s_end) continue;
        T *dst = c_val + cpos[o] * BS;
#pragma unroll
        for (int e = 0; e < BS; ++e) dst[e] = acc[o][e];
    }
}

// ------------------------------------------------------------------ row groups

// Group index and column chunk of a row-group CTA.  The column chunk is the
// fastest grid index, so the CTAs of one group run together and the rows of B
// its K touches are fetched from DRAM about once; groups beyond 65535 go to
// grid.z.
__device__ __forceinline__ int64_t grp_of_block() { return blockIdx.y + (int64_t)blockIdx.z * gridDim.y; }


// Row-group product (plan built by group.cu).  CTA = (group g of G rows, a
// chunk of the group's output columns J).  Lanes form groups of NSF, one per
// output column j; lane r keeps column r of C_(m,j) for the G rows m (and
// NOUT products sharing A) in registers.  For each k of the group's K (A's
// blocks of the G rows staged in shared memory, zero where absent, with a
// bitmask of the rows that hold A_mk), the lane reads the 16-bit position of
// op(B)_kj (coalesced: the table is k-major), fetches its column r of
// op(B)_kj once, and adds A_mk op(B)_kj for every row m in the mask.  Sums
// run over k in ascending order (deterministic).  Outputs (m, j) outside C's
// pattern are discarded at the store.
// Vector helpers: NSF = 4 rows are 16 (FP32) or 32 (FP64) bytes, aligned in
// every value array (blocks of 64 / 128 bytes from a 256-byte aligned base).
template <typename T, int N>
__device__ __forceinline__ void ld_row(const T *__restrict__ p, T (&v)[N], bool global)
{
    if constexpr (N == 4 && sizeof(T) == 4) {
        const float4 q = global ? __ldg(reinterpret_cast<const float4 *>(p)) : *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (N == 4 && sizeof(T) == 8) {
        const double2 q0 = global ? __ldg(reinterpret_cast<const double2 *>(p)) : *reinterpret_cast<const double2 *>(p);
        const double2 q1 = global ? __ldg(reinterpret_cast<const double2 *>(p) + 1) : *(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    } else if constexpr (N == 2 && sizeof(T) == 8) {
        const double2 q = global ? __ldg(reinterpret_cast<const double2 *>(p)) : *reinterpret_cast<const double2 *>(p);
        v[0] = q.x; v[1] = q.y;
    } else if constexpr (N == 2 && sizeof(T) == 4) {
        const float2 q = global ? __ldg(reinterpret_cast<const float2 *>(p)) : *reinterpret_cast<const float2 *>(p);
        v[0] = q.x; v[1] = q.y;
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = global ? __ldg(p + i) : p[i];
    }
}

// The columns [c0, c0 + CW) of op(B)_kj held by one lane: bc[y][z] = op(B)[z][c0 + y].
// op(B) = B^T: op(B)[z][c] = blk[c][z] -> rows c0.. of the stored block.
// op(B) = B:   op(B)[z][c] = blk[z][c] -> a CW-wide slice of every row.
template <typename T, int NSF, int CW, bool TB>
__device__ __forceinline__ void ld_bcols(const T *__restrict__ blk, int c0, T (&bc)[CW][NSF])
{
    constexpr bool VEC = (NSF == 4) || (NSF == 2);
    if constexpr (TB) {
#pragma unroll
        for (int y = 0; y < CW; ++y) {
            if constexpr (VEC) ld_row<T, NSF>(blk + (c0 + y) * NSF, bc[y], true);
            else {
#pragma unroll
                for (int z = 0; z < NSF; ++z) bc[y][z] = __ldg(blk + (c0 + y) * NSF + z);
            }
        }
    } else {
#pragma unroll
        for (int z = 0; z < NSF; ++z) {
            T row[CW];
            if constexpr (VEC && CW == NSF) ld_row<T, NSF>(blk + z * NSF, row, true);
            else {
#pragma unroll
                for (int y = 0; y < CW; ++y) row[y] = __ldg(blk + z * NSF + c0 + y);
            }
#pragma unroll
            for (int y = 0; y < CW; ++y) bc[y][z] = row[y];
        }
    }
}

// acc[x][y] += sum_z A[x][z] * bc[y][z] for the NSF rows x of one A block.
template <typename T, int NSF, int CW, int NOUT>
__device__ __forceinline__ void blk_fma(const T *am, const T (&bc)[NOUT][CW][NSF],
                                        T (&acc)[NOUT][NSF][CW])
{
#pragma unroll
    for (int x = 0; x < NSF; ++x) {
        T a[NSF];
        if constexpr (NSF == 4 || NSF == 2) ld_row<T, NSF>(am + x * NSF, a, false);
        else {
#pragma unroll
            for (int z = 0; z < NSF; ++z) a[z] = am[x * NSF + z];
        }
#pragma unroll
        for (int n = 0; n < NOUT; ++n)
#pragma unroll
            for (int y = 0; y < CW; ++y) {
                T s = acc[n][x][y];
#pragma unroll
                for (int z = 0; z < NSF; ++z) s = fma(a[z], bc[n][y][z], s);
                acc[n][x][y] = s;
            }
    }
}

// Staging helpers shared by the row-group kernels.
// A's blocks of the G rows for k-chunk [k0, k0 + kn): one thread per (k, row)
// block, loaded row by row (16-byte loads for NSF = 4) and stored transposed
// when op(A) = A^T; zero where the row has no block.  msk[kk] gets the rows
// holding A_(m, k).
template <typename T, int NSF, int G, bool TA, typename S, bool MASK = true>
__device__ __forceinline__ void stage_a(S *a_s, uint32_t *msk, const int32_t *__restrict__ apos,
                                        const int64_t *__restrict__ a_tr, const T *__restrict__ a_val,
                                        int64_t kbase, int kn)
{
    constexpr int BS = NSF * NSF;
    for (int t = threadIdx.x; t < kn * G; t += blockDim.x) {
        const int kk = t / G, m = t - kk * G;
        const int32_t q = __ldg(apos + (kbase + kk) * G + m);
        T blk[NSF][NSF];
        if (q >= 0) {
            const T *src = a_val + (TA ? __ldg(a_tr + q) : (int64_t)q) * BS;
#pragma unroll
            for (int x = 0; x < NSF; ++x) {
                if constexpr (NSF == 4 || NSF == 2) ld_row<T, NSF>(src + x * NSF, blk[x], true);
                else {
#pragma unroll
                    for (int z = 0; z < NSF; ++z) blk[x][z] = __ldg(src + x * NSF + z);
                }
            }
        } else {
#pragma unroll
            for (int x = 0; x < NSF; ++x)
#pragma unroll
                for (int z = 0; z < NSF; ++z) blk[x][z] = T(0);
        }
        S *dst = a_s + (size_t)t * BS;
#pragma unroll
        for (int x = 0; x < NSF; ++x)
#pragma unroll
            for (int z = 0; z < NSF; ++z) dst[x * NSF + z] = S(TA ? blk[z][x] : blk[x][z]);
    }
    if (MASK)
        for (int kk = threadIdx.x; kk < kn; kk += blockDim.x) {
            uint32_t mm = 0;
#pragma unroll
            for (int m = 0; m < G; ++m) mm |= (__ldg(apos + (kbase + kk) * G + m) >= 0 ? 1u : 0u) << m;
            msk[kk] = mm;
        }
}

// Position-table tile [kn][jc] of rows padded to a multiple of 8 entries,
// loaded 16 bytes at a time; kflag[kk] = 1 when row kk has a hit.
__device__ __forceinline__ void stage_ix(uint16_t *ixs, int32_t *kflag, const uint16_t *__restrict__ bx,
                                         int64_t k0, int kn, int64_t nj_pad, int64_t j0, int jcn, int jc)
{
    for (int t = threadIdx.x; t < kn; t += blockDim.x) kflag[t] = 0;
    __syncthreads();
    const int vec = jc / 8;
    for (int t = threadIdx.x; t < kn * vec; t += blockDim.x) {
        const int kk = t / vec, v = t - kk * vec;
        const int c = v * 8;
        uint4 w = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        if (c < jcn) w = __ldg(reinterpret_cast<const uint4 *>(bx + (k0 + kk) * nj_pad + j0 + c));
        uint16_t e[8];
        memcpy(e, &w, 16);
        bool any = false;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (c + u >= jcn) e[u] = 0xFFFF;
            any |= e[u] != 0xFFFF;
        }
        memcpy(ixs + kk * jc + c, e, 16);
        if (any) kflag[kk] = 1;
    }
}

// List the flagged k's in order (warp 0, ballot prefix sums): kact[0..n), kact[cap] = n.
__device__ __forceinline__ void compact_k(int32_t *kact, const int32_t *kflag, int kn, int cap)
{
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int base = 0;
    for (int k0 = 0; k0 < kn; k0 += 32) {
        const int kk = k0 + lane;
        const bool f = kk < kn && kflag[kk];
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (f) kact[base + __popc(b & ((1u << lane) - 1u))] = kk;
        base += __popc(b);
    }
    if (lane == 0) kact[cap] = base;
}

// Row-group product (plan built by group.cu).  CTA = (group g of G rows, a
// chunk of the group's output columns J).  NSF / CW lanes share one output
// column j; each keeps columns [c0, c0 + CW) of C_(m,j) for the G rows m (and
// NOUT products sharing A) in registers, for OPT columns j per lane group.
// For each k of the group's K, A's blocks of the G rows (staged in shared
// memory, zero where absent, with a bitmask of the rows holding A_mk) are
// applied to op(B)_kj, fetched once per lane:
//   SPARSE = false: the 16-bit position of op(B)_kj comes from the dense
//     table (a tile staged in shared memory per k-chunk); k's without a hit
//     in the CTA's columns are skipped; the next k's blocks are fetched while
//     the current ones are applied.
//   SPARSE = true: each column walks its own hit list (ascending k), with the
//     next hit's block fetched while the current one is applied.
// Each A row is read once per k and applied to all OPT x NOUT outputs.  Sums
// run over k in ascending order (deterministic).  Outputs (m, j) outside C's
// pattern are discarded at the store.
template <typename T, int NSF, int G, int NOUT, int CW, int OPT, bool TA, bool TB, bool SPARSE>
__global__ void __launch_bounds__(128)
k_grp(const int64_t *__restrict__ k_off, const int32_t *__restrict__ k_list,
      const int32_t *__restrict__ apos, const int64_t *__restrict__ j_off,
      const int32_t *__restrict__ j_list, const int32_t *__restrict__ cpos,
      const int64_t *__restrict__ bidx_off, const uint16_t *__restrict__ bidx,
      const int64_t *__restrict__ hoff, const uint16_t *__restrict__ hk,
      const int32_t *__restrict__ hp, const int64_t *__restrict__ a_tr,
      const T *__restrict__ a_val, const int64_t *__restrict__ b_rp,
      const T *__restrict__ b_val1, const T *__restrict__ b_val2, T *__restrict__ c_val1,
      T *__restrict__ c_val2, int jc, int kchunk, int64_t n_groups, const int32_t *__restrict__ jsplit,
      int part)
{
    static_assert(NOUT == 1 || NOUT == 2, "one or two products");
    static_assert(NSF % CW == 0, "CW divides NSF");
    constexpr int BS = NSF * NSF;
    constexpr int LPJ = NSF / CW;    // lanes per output column
    constexpr int JPW = 32 / LPJ;    // lane groups per warp
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *a_s = reinterpret_cast<T *>(smem_raw);                                    // [kchunk][G][BS]
    int64_t *brow = reinterpret_cast<int64_t *>(a_s + (size_t)kchunk * G * BS);  // [kchunk]
    uint32_t *msk = reinterpret_cast<uint32_t *>(brow + kchunk);                 // [kchunk]
    int32_t *kact = reinterpret_cast<int32_t *>(msk + kchunk);                   // [kchunk + 2]
    int32_t *kflag = kact + kchunk + 2;                                          // [kchunk]
    uint16_t *ixs = reinterpret_cast<uint16_t *>(kflag + kchunk + 2);            // [kchunk][jc]

    const int64_t g = grp_of_block();
    if (g >= n_groups) return;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    const int64_t nj_pad = (nj + 7) & ~int64_t(7);
    // columns [jlo, jhi) of J: all (part 0), the upper part (1) or the rest (2)
    const int64_t jlo = part == 2 ? jsplit[g] : 0, jhi = part == 1 ? jsplit[g] : nj;
    const int64_t j0 = jlo + (int64_t)blockIdx.x * jc;
    if (j0 >= jhi) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int jg = lane / LPJ, c0 = (lane - jg * LPJ) * CW;
    const int groups_cta = (blockDim.x >> 5) * JPW;
    const int jcn = (int)min((int64_t)jc, jhi - j0);
    int col[OPT];
    bool jv[OPT];
    int64_t brj[OPT], ptr[OPT], pend[OPT];
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        col[o] = warp * JPW + jg + o * groups_cta;
        jv[o] = jg < JPW && col[o] < jcn;
        brj[o] = (TB && jv[o]) ? b_rp[j_list[jb + j0 + col[o]]] : 0;
        ptr[o] = (SPARSE && jv[o]) ? hoff[jb + j0 + col[o]] : 0;
        pend[o] = (SPARSE && jv[o]) ? hoff[jb + j0 + col[o] + 1] : 0;
    }
    bool any_col = false;
#pragma unroll
    for (int o = 0; o < OPT; ++o) any_col |= jv[o];

    T acc[OPT][G][NOUT][NSF][CW];
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int m = 0; m < G; ++m)
#pragma unroll
            for (int n = 0; n < NOUT; ++n)
#pragma unroll
                for (int x = 0; x < NSF; ++x)
#pragma unroll
                    for (int y = 0; y < CW; ++y) acc[o][m][n][x][y] = T(0);

    // apply A_mk (all active rows m) to the fetched blocks of the OPT columns
    auto apply = [&](int kc, const T (&bc)[OPT][NOUT][CW][NSF], const bool (&h)[OPT], uint32_t mk) {
        const T *ak = a_s + (size_t)kc * G * BS;
#pragma unroll
        for (int m = 0; m < G; ++m) {
            if (!((mk >> m) & 1u)) continue;
            const T *am = ak + m * BS;
#pragma unroll
            for (int x = 0; x < NSF; ++x) {
                T a[NSF];
                if constexpr (NSF == 4 || NSF == 2) ld_row<T, NSF>(am + x * NSF, a, false);
                else {
#pragma unroll
                    for (int z = 0; z < NSF; ++z) a[z] = am[x * NSF + z];
                }
#pragma unroll
                for (int o = 0; o < OPT; ++o) {
                    if (!h[o]) continue;
#pragma unroll
                    for (int n = 0; n < NOUT; ++n)
#pragma unroll
                        for (int y = 0; y < CW; ++y) {
                            T sacc = acc[o][m][n][x][y];
#pragma unroll
                            for (int z = 0; z < NSF; ++z) sacc = fma(a[z], bc[o][n][y][z], sacc);
                            acc[o][m][n][x][y] = sacc;
                        }
                }
            }
        }
    };
    auto fetch_one = [&](int64_t p, T (&bc)[NOUT][CW][NSF]) {
#pragma unroll
        for (int n = 0; n < NOUT; ++n)
            ld_bcols<T, NSF, CW, TB>((n == 0 ? b_val1 : b_val2) + p * BS, c0, bc[n]);
    };
    // dense: the blocks of active k number q (kact[q]) for every owned column
    auto fetch_dense = [&](int kc, T (&bc)[OPT][NOUT][CW][NSF], bool (&h)[OPT]) {
#pragma unroll
        for (int o = 0; o < OPT; ++o) {
            const uint16_t ix = jv[o] ? ixs[kc * jc + col[o]] : (uint16_t)0xFFFF;
            h[o] = ix != 0xFFFF;
            if (h[o]) fetch_one((TB ? brj[o] : brow[kc]) + ix, bc[o]);
        }
    };

    for (int64_t k0 = 0; k0 < nk; k0 += kchunk) {
        const int kn = (int)min((int64_t)kchunk, nk - k0);
        __syncthreads();
        stage_a<T, NSF, G, TA>(a_s, msk, apos, a_tr, a_val, kb + k0, kn);
        if (!SPARSE) {
            for (int t = threadIdx.x; t < kn; t += blockDim.x) brow[t] = TB ? 0 : b_rp[k_list[kb + k0 + t]];
            stage_ix(ixs, kflag, bidx + bidx_off[g], k0, kn, nj_pad, j0, jcn, jc);
            __syncthreads();
            compact_k(kact, kflag, kn, kchunk);
        }
        __syncthreads();
        if (!any_col) continue;
        if (!SPARSE) {
            const int na = kact[kchunk];
            T bc0[OPT][NOUT][CW][NSF], bc1[OPT][NOUT][CW][NSF];
            bool h0[OPT], h1[OPT];
            // ping-pong over the active k's: the next k's blocks load during this k
            if (na > 0) fetch_dense(kact[0], bc0, h0);
            for (int q = 0; q < na; q += 2) {
                const int ka = kact[q];
                if (q + 1 < na) fetch_dense(kact[q + 1], bc1, h1);
                apply(ka, bc0, h0, msk[ka]);
                if (q + 1 >= na) break;
                const int kb1 = kact[q + 1];
                if (q + 2 < na) fetch_dense(kact[q + 2], bc0, h0);
                apply(kb1, bc1, h1, msk[kb1]);
            }
        } else {
            const int kend = (int)(k0 + kn);
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                T bc0[OPT][NOUT][CW][NSF], bc1[OPT][NOUT][CW][NSF];
                bool hh[OPT];
#pragma unroll
                for (int oo = 0; oo < OPT; ++oo) hh[oo] = oo == o;
                int kl = ptr[o] < pend[o] ? (int)__ldg(hk + ptr[o]) : kend;
                if (kl < kend) fetch_one(__ldg(hp + ptr[o]), bc0[o]);
                while (kl < kend) {
                    const int kc = kl - (int)k0;
                    ++ptr[o];
                    const int kl1 = ptr[o] < pend[o] ? (int)__ldg(hk + ptr[o]) : kend;
                    if (kl1 < kend) fetch_one(__ldg(hp + ptr[o]), bc1[o]);
                    apply(kc, bc0, hh, msk[kc]);
                    kl = kl1;
                    if (kl >= kend) break;
                    const int kc1 = kl - (int)k0;
                    ++ptr[o];
                    const int kl2 = ptr[o] < pend[o] ? (int)__ldg(hk + ptr[o]) : kend;
                    if (kl2 < kend) fetch_one(__ldg(hp + ptr[o]), bc0[o]);
                    apply(kc1, bc1, hh, msk[kc1]);
                    kl = kl2;
                }
            }
        }
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        if (!jv[o]) continue;
#pragma unroll
        for (int m = 0; m < G; ++m) {
            const int32_t pos = cpos[(jb + j0 + col[o]) * G + m];
            if (pos < 0) continue;
#pragma unroll
            for (int n = 0; n < NOUT; ++n) {
                T *dst = (n == 0 ? c_val1 : c_val2) + (int64_t)pos * BS;
#pragma unroll
                for (int x = 0; x < NSF; ++x)
#pragma unroll
                    for (int y = 0; y < CW; ++y) dst[x * NSF + c0 + y] = acc[o][m][n][x][y];
            }
        }
    }
}

// ------------------------------------------------------------------ row groups, per-warp k lists

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}


// Row-group product with independent warps (FP32, NSF = 4, G = 4 rows).
//
// A warp owns one slice of the group's output columns J: OPT sets of eight
// consecutive columns (OPT = 2 for two fused products and 4 for one, or half
// that: a warp then lists only the k's its narrower slice hits, and groups
// with few columns give more warps).  In a set,
// four lanes share a column j and lane r keeps column r of C_(m,j) for the G
// rows m and NOUT products in registers.  Warps share nothing, so there is no
// block-wide barrier: per chunk of KC k's of the group's K, the warp lists
// the k's at which any of its columns holds op(B)_kj (one lane per k, ballot
// compaction).  An entry carries k, a bitmask of the sets that hit, a bitmask
// of the rows m holding A_mk, A's block positions and, per column, the block
// index of op(B)_kj's stored block (-1 at a miss).  For each entry the warp
// copies A's blocks (rows with A_mk only) and the stored rows of op(B)_kj
// (16 bytes per lane, zero-filled at a miss) into a warp-private ring of D
// stages with cp.async, D - 1 entries ahead of the one being multiplied.
// Stored block rows are columns of op(B) when op(B) = B^T, else lanes read
// column r across the four rows of the block; the four rows of a block slot
// are rotated by (jg / 2) so those column reads are free of bank conflicts.
// A is read the same way: rows of op(A), or of the stored block when
// op(A) = A^T.  Sums run over k in ascending order (deterministic).  Outputs
// (m, j) outside C's pattern are discarded at the store.
template <int NOUT, int OPT_, int D, bool TA, bool TB>
struct GwShape {
    static constexpr int G = 4, BS = 16, OPT = OPT_, COLS = 8 * OPT;
    // k's per list chunk: one k per lane (the list is built in one pass of the
    // warp), 30 where 32 would not let eight two-warp CTAs share an SM's 228 KB
    static constexpr int KC = NOUT * OPT == 4 && NOUT == 1 ? 30 : 32;
    // list entry: k | set mask << 16 | row mask << 24, A's four block
    // positions, then op(B)_kj's block index per column (odd size: the
    // strided entry writes are free of bank conflicts)
    static constexpr int EW = 5 + COLS;
    static constexpr int STAGE = G * BS + OPT * NOUT * 8 * BS;     // floats per ring stage
    static constexpr size_t warp_bytes =
        sizeof(float) * D * STAGE + sizeof(int32_t) * (KC * EW + COLS + 1);
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16s(uint32_t dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}

// Resident CTAs per SM a k_gw shape is compiled for: 16 warps of up to 128
// registers.  (24 warps of the half-width shapes, at 80 registers, ran 10-15%
// slower: less room to keep loads in flight.)
template <int NOUT, int OPT, int NW>
constexpr int gw_min_blocks()
{
    return 16 / NW;
}

template <int NOUT, int OPT_, int D, int NW, bool TA, bool TB>
__global__ void __launch_bounds__(NW * 32, gw_min_blocks<NOUT, OPT_, NW>())
k_gw(const int64_t *__restrict__ k_off, const int32_t *__restrict__ apos,
     const int64_t *__restrict__ j_off, const int32_t *__restrict__ j_list,
     const int32_t *__restrict__ cpos, const int64_t *__restrict__ bidx_off,
     const uint16_t *__restrict__ bidx, const int32_t *__restrict__ k_list,
     const int64_t *__restrict__ a_tr, const float *__restrict__ a_val,
     const int64_t *__restrict__ b_rp, const float *__restrict__ b_val1,
     const float *__restrict__ b_val2, float *__restrict__ c_val1, float *__restrict__ c_val2,
     int64_t n_groups, const int32_t *__restrict__ jsplit, int part)
{
    using S = GwShape<NOUT, OPT_, D, TA, TB>;
    constexpr int G = S::G, BS = S::BS, OPT = S::OPT, COLS = S::COLS, KC = S::KC, EW = S::EW;
    // Row layout for the half-width shapes with op(B) = B: lane r keeps row r
    // of C_mj (not column r), so it reads one row of each A block (one 16-byte
    // read instead of four) and every B block whole (four 16-byte reads instead
    // of four 4-byte ones).  It took XY from 1.17 to 1.11 ms; with op(B) = B^T,
    // where the column layout reads B in one 16-byte read, it slowed Z and W.
    constexpr bool ROWL = NOUT * OPT == 2 && !TB;
    constexpr int STAGE = S::STAGE;
    static_assert((D & (D - 1)) == 0, "ring depth is a power of two");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *ring = reinterpret_cast<float *>(smem_raw) + (size_t)warp * D * STAGE;                 // [D][STAGE]
    int32_t *list = reinterpret_cast<int32_t *>(reinterpret_cast<float *>(smem_raw) + (size_t)NW * D * STAGE) +
                    (size_t)warp * (KC * EW + COLS + 1);                                          // [KC][EW]
    int32_t *rowj = list + KC * EW;                                                               // [COLS]

    const int64_t g = grp_of_block();
    if (g >= n_groups) return;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    const int64_t nj_pad = (nj + 7) & ~int64_t(7);
    // columns [jlo, jhi) of J: all (part 0), the upper part (1) or the rest (2)
    const int64_t jlo = part == 2 ? jsplit[g] : 0, jhi = part == 1 ? jsplit[g] : nj;
    const int64_t j0 = jlo + ((int64_t)blockIdx.x * NW + warp) * COLS;
    if (j0 >= jhi) return;
    const int jcn = (int)min((int64_t)COLS, jhi - j0);
    const int jg = lane >> 2, r = lane & 3;
    // op(B) = B^T: row start of the stored row j for each of the warp's columns
    if (TB)
        for (int c = lane; c < COLS; c += 32) rowj[c] = c < jcn ? (int32_t)b_rp[j_list[jb + j0 + c]] : 0;
    const uint16_t *bx = bidx + bidx_off[g];

    // per-lane shared-memory offsets (bytes) inside a ring stage
    const uint32_t ring0 = smem_addr(ring);
    const int rot = jg >> 1;
    const uint32_t b_dst = (uint32_t)(G * BS + jg * BS + ((r + rot) & 3) * 4) * 4u;   // copy of stored row r
    uint32_t b_rd[4];                                                                // stored row z, column r
#pragma unroll
    for (int z = 0; z < 4; ++z) b_rd[z] = (uint32_t)(G * BS + jg * BS + ((z + rot) & 3) * 4 + r) * 4u;
    const uint32_t a_dst = (uint32_t)((lane >> 2) * BS + (lane & 3) * 4) * 4u;
    const float *a_src = a_val + (lane & 3) * 4;
    const float *b_src1 = b_val1 + r * 4, *b_src2 = (NOUT == 2 ? b_val2 : b_val1) + r * 4;
    // need: for each set o, bits (4 o + m) for the rows m whose C row holds one
    // of the set's columns; rows outside it are never multiplied for the set
    uint32_t need = 0;
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        uint32_t cm = 0;
        if (o * 8 + jg < jcn) {
            const int4 cp = __ldg(reinterpret_cast<const int4 *>(cpos + (jb + j0 + o * 8 + jg) * G));
            cm = (cp.x >= 0 ? 1u : 0u) | (cp.y >= 0 ? 2u : 0u) | (cp.z >= 0 ? 4u : 0u) | (cp.w >= 0 ? 8u : 0u);
        }
        need |= __reduce_or_sync(0xffffffffu, cm) << (4 * o);
    }

    float acc[OPT][G][NOUT][4];
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int m = 0; m < G; ++m)
#pragma unroll
            for (int n = 0; n < NOUT; ++n)
#pragma unroll
                for (int x = 0; x < 4; ++x) acc[o][m][n][x] = 0.f;

    for (int64_t k0 = 0; k0 < nk; k0 += KC) {
        const int kn = (int)min((int64_t)KC, nk - k0);
        __syncwarp();
        // list of this chunk's k's that hit any of the warp's columns
        int na = 0;
        for (int kq = 0; kq < kn; kq += 32) {
            const int kk = kq + lane;
            uint32_t om = 0, mk = 0;
            uint32_t ixw[COLS / 2];
            int4 ap = make_int4(-1, -1, -1, -1);
            if (kk < kn) {
                ap = __ldg(reinterpret_cast<const int4 *>(apos + (kb + k0 + kk) * G));
                mk = (ap.x >= 0 ? 1u : 0u) | (ap.y >= 0 ? 2u : 0u) | (ap.z >= 0 ? 4u : 0u) | (ap.w >= 0 ? 8u : 0u);
                const uint16_t *row = bx + (k0 + kk) * nj_pad + j0;
#pragma unroll
                for (int p = 0; p < COLS / 8; ++p) {
                    uint4 v = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
                    if (p * 8 < jcn) {
                        v = __ldg(reinterpret_cast<const uint4 *>(row) + p);
                        if (p * 8 + 8 > jcn) {
                            uint16_t e[8];
                            memcpy(e, &v, 16);
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (p * 8 + u >= jcn) e[u] = 0xFFFF;
                            memcpy(&v, e, 16);
                        }
                    }
                    ixw[p * 4 + 0] = v.x; ixw[p * 4 + 1] = v.y; ixw[p * 4 + 2] = v.z; ixw[p * 4 + 3] = v.w;
                    // a set counts when it holds a block and one of its needed rows has A_mk
                    if ((v.x & v.y & v.z & v.w) != 0xFFFFFFFFu && ((need >> (4 * p)) & mk)) om |= 1u << p;
                }
                uint32_t used = 0;
#pragma unroll
                for (int o = 0; o < OPT; ++o)
                    if ((om >> o) & 1) used |= need >> (4 * o);
                mk &= used;
            }
            const unsigned b = __ballot_sync(0xffffffffu, om != 0);
            if (om) {
                int32_t *e = list + (size_t)(na + __popc(b & ((1u << lane) - 1u))) * EW;
                const int32_t aq[4] = {ap.x, ap.y, ap.z, ap.w};
#pragma unroll
                for (int m = 0; m < G; ++m) {
                    int32_t q = aq[m];
                    if (TA && ((mk >> m) & 1)) q = (int32_t)__ldg(a_tr + q);
                    e[1 + m] = q;
                }
                e[0] = kk | (int)(om << 16) | (int)(mk << 24);
                const int32_t brk = TB ? 0 : (int32_t)b_rp[k_list[kb + k0 + kk]];
#pragma unroll
                for (int c = 0; c < COLS; ++c) {
                    const uint32_t ix = (ixw[c >> 1] >> ((c & 1) * 16)) & 0xFFFFu;
                    e[5 + c] = ix == 0xFFFFu ? -1 : (TB ? rowj[c] : brk) + (int32_t)ix;
                }
            }
            na += __popc(b);
        }
        __syncwarp();

        // copy entry q into ring stage q % D (an empty commit group past the list's end)
        auto issue = [&](int q) {
            if (q < na) {
                const int32_t *e = list + (size_t)q * EW;
                // the entry is the same for every lane: a broadcast keeps the tests warp-uniform
                const int w0 = __shfl_sync(0xffffffffu, e[0], 0);
                const int om = (w0 >> 16) & 0xFF, mk = (w0 >> 24) & 0xF;
                const uint32_t st = ring0 + (uint32_t)((q & (D - 1)) * STAGE * 4);
                if (lane < 16 && ((mk >> (lane >> 2)) & 1))
                    cp_async16s(st + a_dst, a_src + (int64_t)e[1 + (lane >> 2)] * BS, 16);
#pragma unroll
                for (int o = 0; o < OPT; ++o) {
                    if (!((om >> o) & 1)) continue;
                    const int32_t blk = e[5 + o * 8 + jg];
                    const int bytes = blk >= 0 ? 16 : 0;
                    const int64_t off = (int64_t)max(blk, 0) * BS;
                    cp_async16s(st + b_dst + (uint32_t)(o * NOUT * 8 * BS * 4), b_src1 + off, bytes);
                    if (NOUT == 2)
                        cp_async16s(st + b_dst + (uint32_t)((o * NOUT + 1) * 8 * BS * 4), b_src2 + off, bytes);
                }
            }
            cp_async_commit();
        };
#pragma unroll
        for (int q = 0; q < D - 1; ++q) issue(q);
        for (int q = 0; q < na; ++q) {
            issue(q + D - 1);
            cp_async_wait<D - 1>();
            __syncwarp();
            const int w0 = __shfl_sync(0xffffffffu, list[(size_t)q * EW], 0);
            const int om = (w0 >> 16) & 0xFF, mk = (w0 >> 24) & 0xF;
            const unsigned char *st = reinterpret_cast<const unsigned char *>(ring) + (q & (D - 1)) * STAGE * 4;
            if constexpr (ROWL) {
                // bq[o][n][z][y] = op(B)_kj[z][y]: the whole block, four 16-byte reads
                float bq[OPT][NOUT][4][4];
#pragma unroll
                for (int o = 0; o < OPT; ++o) {
                    if (!((om >> o) & 1)) continue;
#pragma unroll
                    for (int n = 0; n < NOUT; ++n) {
                        const unsigned char *blk = st + ((o * NOUT + n) * 8 * BS + G * BS + jg * BS) * 4;
#pragma unroll
                        for (int rr = 0; rr < 4; ++rr) {
                            const float4 v = *reinterpret_cast<const float4 *>(blk + ((rr + rot) & 3) * 16);
                            const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                if (TB) bq[o][n][c][rr] = e[c];  // stored row rr = column rr of op(B)
                                else bq[o][n][rr][c] = e[c];
                            }
                        }
                    }
                }
#pragma unroll
                for (int m = 0; m < G; ++m) {
                    if (!((mk >> m) & 1)) continue;
                    // a[z] = op(A)_mk[r][z]
                    float a[4];
                    if (TA) {
#pragma unroll
                        for (int z = 0; z < 4; ++z) a[z] = *reinterpret_cast<const float *>(st + (m * BS + z * 4 + r) * 4);
                    } else {
                        const float4 v = *reinterpret_cast<const float4 *>(st + (m * BS + r * 4) * 4);
                        a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
                    }
#pragma unroll
                    for (int o = 0; o < OPT; ++o) {
                        if (!((om >> o) & 1) || !((need >> (4 * o + m)) & 1)) continue;
#pragma unroll
                        for (int z = 0; z < 4; ++z)
#pragma unroll
                            for (int n = 0; n < NOUT; ++n)
#pragma unroll
                                for (int y = 0; y < 4; ++y)
                                    acc[o][m][n][y] = fmaf(a[z], bq[o][n][z][y], acc[o][m][n][y]);
                    }
                }
                __syncwarp();
                continue;
            }
            // bv[o][n][z] = op(B)[z][r]
            float bv[OPT][NOUT][4];
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (!((om >> o) & 1)) continue;
#pragma unroll
                for (int n = 0; n < NOUT; ++n) {
                    const unsigned char *slot = st + (o * NOUT + n) * 8 * BS * 4;
                    if (TB) {
                        const float4 v = *reinterpret_cast<const float4 *>(slot + b_dst);
                        bv[o][n][0] = v.x; bv[o][n][1] = v.y; bv[o][n][2] = v.z; bv[o][n][3] = v.w;
                    } else {
#pragma unroll
                        for (int z = 0; z < 4; ++z) bv[o][n][z] = *reinterpret_cast<const float *>(slot + b_rd[z]);
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < G; ++m) {
                if (!((mk >> m) & 1)) continue;
                const float4 *am = reinterpret_cast<const float4 *>(st) + m * 4;
                float a[4][4];  // a[x][z] = op(A)_mk[x][z]
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const float4 v = am[y];
                    if (TA) {
                        a[0][y] = v.x; a[1][y] = v.y; a[2][y] = v.z; a[3][y] = v.w;
                    } else {
                        a[y][0] = v.x; a[y][1] = v.y; a[y][2] = v.z; a[y][3] = v.w;
                    }
                }
#pragma unroll
                for (int o = 0; o < OPT; ++o) {
                    if (!((om >> o) & 1) || !((need >> (4 * o + m)) & 1)) continue;
#pragma unroll
                    for (int z = 0; z < 4; ++z)
#pragma unroll
                        for (int n = 0; n < NOUT; ++n)
#pragma unroll
                            for (int x = 0; x < 4; ++x)
                                acc[o][m][n][x] = fmaf(a[x][z], bv[o][n][z], acc[o][m][n][x]);
                }
            }
            __syncwarp();
        }
        cp_async_wait<0>();
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        if (o * 8 + jg >= jcn) continue;
#pragma unroll
        for (int m = 0; m < G; ++m) {
            const int32_t pos = cpos[(jb + j0 + o * 8 + jg) * G + m];
            if (pos < 0) continue;
#pragma unroll
            for (int n = 0; n < NOUT; ++n) {
                float *dst = (n == 0 ? c_val1 : c_val2) + (int64_t)pos * BS;
                if (ROWL) {
                    *reinterpret_cast<float4 *>(dst + r * 4) =
                        make_float4(acc[o][m][n][0], acc[o][m][n][1], acc[o][m][n][2], acc[o][m][n][3]);
                } else {
#pragma unroll
                    for (int x = 0; x < 4; ++x) dst[x * 4 + r] = acc[o][m][n][x];
                }
            }
        }
    }
}

// ------------------------------------------------------------------ listed triples

// Output-stationary product over listed triples (NSF = 4).  Four lanes own one
// block of C (an item of the triple-list plan) and lane x keeps row x of it
// for the NOUT products in registers.  For each listed (op(A)_ik, op(B)_kj)
// pair, k ascending, the lane reads row x of op(A)_ik and the whole block
// op(B)_kj (the group's four lanes read the same addresses) and adds their
// product; the next pair's blocks are fetched while the current ones are
// applied.  Nothing is multiplied that is absent or discarded.  Items are
// ordered by groups of four rows, then by list length, so a warp's eight
// items end together and its lanes stay busy (the FP64 pipe spends a full
// slot on a partly idle warp instruction).  With sub (not null) the launch covers the
// items sub[0 .. n_items - 1] only (the upper triangle of a symmetric output).
template <typename T, int NOUT, bool TA, bool TB>
__global__ void __launch_bounds__(128)
k_tri(int64_t n_items, const int32_t *__restrict__ sub, const int32_t *__restrict__ item_cb,
      const int64_t *__restrict__ t_off, const int2 *__restrict__ tri, const T *__restrict__ a_val,
      const T *__restrict__ b_val1, const T *__restrict__ b_val2, T *__restrict__ c_val1, T *__restrict__ c_val2)
{
    constexpr int BS = 16;
    const int64_t iq = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2;
    const int x = threadIdx.x & 3;
    if (iq >= n_items) return;
    const int64_t it = sub ? (int64_t)sub[iq] : iq;
    const int64_t t0 = t_off[it], t1 = t_off[it + 1];
    T acc[NOUT][4];
#pragma unroll
    for (int n = 0; n < NOUT; ++n)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[n][y] = T(0);
    // a[z] = op(A)_ik[x][z]; b[n][z][y] = stored block of op(B)_kj, row z
    auto load = [&](int64_t t, T (&a)[4], T (&b)[NOUT][4][4]) {
        const int2 p = __ldg(tri + t);
        const T *ab = a_val + (int64_t)p.x * BS;
        if (TA) {
#pragma unroll
            for (int z = 0; z < 4; ++z) a[z] = __ldg(ab + z * 4 + x);
        } else {
            ld_row<T, 4>(ab + x * 4, a, true);
        }
#pragma unroll
        for (int n = 0; n < NOUT; ++n) {
            const T *bb = (n == 0 ? b_val1 : b_val2) + (int64_t)p.y * BS;
#pragma unroll
            for (int z = 0; z < 4; ++z) ld_row<T, 4>(bb + z * 4, b[n][z], true);
        }
    };
    auto apply = [&](const T (&a)[4], const T (&b)[NOUT][4][4]) {
#pragma unroll
        for (int n = 0; n < NOUT; ++n)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                T s = acc[n][y];
#pragma unroll
                for (int z = 0; z < 4; ++z) s = fma(a[z], TB ? b[n][y][z] : b[n][z][y], s);
                acc[n][y] = s;
            }
    };
    T a0[4], a1[4], b0[NOUT][4][4], b1[NOUT][4][4];
    if (t0 < t1) load(t0, a0, b0);
    for (int64_t t = t0; t < t1; t += 2) {
        if (t + 1 < t1) load(t + 1, a1, b1);
        apply(a0, b0);
        if (t + 1 >= t1) break;
        if (t + 2 < t1) load(t + 2, a0, b0);
        apply(a1, b1);
    }
    const int64_t cb = item_cb[it];
#pragma unroll
    for (int n = 0; n < NOUT; ++n) {
        T *dst = (n == 0 ? c_val1 : c_val2) + cb * BS + x * 4;
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(dst) = make_float4(acc[n][0], acc[n][1], acc[n][2], acc[n][3]);
        } else {
            reinterpret_cast<double2 *>(dst)[0] = make_double2(acc[n][0], acc[n][1]);
            reinterpret_cast<double2 *>(dst)[1] = make_double2(acc[n][2], acc[n][3]);
        }
    }
}

// ------------------------------------------------------------------ row groups on tensor cores

__device__ __forceinline__ uint32_t to_tf32(float f)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(f));
    return r;
}

// D += A (16x4, row) * B (4x8, col), TF32 operands, FP32 accumulation.
__device__ __forceinline__ void mma_tf32_k4(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0)
{
    asm volatile(
        "mma.sync.aligned.m16n8k4.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// Row-group product on tensor cores (FP32 values, NSF = 4, G = 4).  The G rows
// of a group times NSF give M = 16, the tile of one mma.m16n8k4: rows (m, x),
// columns (j, y) for two output columns j, reduction (k, z) over one k.  A's
// blocks of the group are staged in shared memory already split into TF32
// high and low parts (a = hi + lo); each op(B)_kj element is split in
// registers, and hi*hi + hi*lo + lo*hi are accumulated in FP32 (the lo*lo
// term is below FP32 rounding), which keeps FP32-level accuracy.  A warp owns
// NT tiles (2 NT output columns); the position table gives op(B)_kj and a
// warp skips a tile whose four lanes-groups all miss.  Sums run over k in
// ascending order.
template <int NOUT, int NT, bool TA, bool TB>
__global__ void __launch_bounds__(128)
k_gmma(const int64_t *__restrict__ k_off, const int32_t *__restrict__ k_list,
       const int32_t *__restrict__ apos, const int64_t *__restrict__ j_off,
       const int32_t *__restrict__ j_list, const int32_t *__restrict__ cpos,
       const int64_t *__restrict__ bidx_off, const uint16_t *__restrict__ bidx,
       const int64_t *__restrict__ a_tr, const float *__restrict__ a_val,
       const int64_t *__restrict__ b_rp, const float *__restrict__ b_val1,
       const float *__restrict__ b_val2, float *__restrict__ c_val1, float *__restrict__ c_val2,
       int kchunk, int64_t n_groups)
{
    constexpr int G = 4, NSF = 4, BS = 16;
    constexpr int JC = 4 * NT * 2;  // output columns per CTA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *ahi = reinterpret_cast<uint32_t *>(smem_raw);   // [kchunk][G][BS] tf32 high
    uint32_t *alo = ahi + (size_t)kchunk * G * BS;            // [kchunk][G][BS] tf32 low
    int64_t *brow = reinterpret_cast<int64_t *>(alo + (size_t)kchunk * G * BS);  // [kchunk]
    int32_t *kact = reinterpret_cast<int32_t *>(brow + kchunk);                  // [kchunk + 2]
    int32_t *kflag = kact + kchunk + 2;                                          // [kchunk + 2]
    uint16_t *ixs = reinterpret_cast<uint16_t *>(kflag + kchunk + 2);            // [kchunk][JC]

    const int64_t g = grp_of_block();
    if (g >= n_groups) return;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    const int64_t nj_pad = (nj + 7) & ~int64_t(7);
    const int64_t j0 = (int64_t)blockIdx.x * JC;
    if (j0 >= nj) return;
    const int jcn = (int)min((int64_t)JC, nj - j0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane >> 2, tig = lane & 3;  // mma groupID / thread-in-group
    const int wbase = warp * NT * 2;            // first column of this warp
    // the column this lane feeds into B fragments of tile nt: wbase + 2 nt + grp / 4
    int64_t brj[NT];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int c = wbase + 2 * nt + (grp >> 2);
        brj[nt] = (TB && c < jcn) ? b_rp[j_list[jb + j0 + c]] : 0;
    }
    float acc[NOUT][NT][4];
#pragma unroll
    for (int n = 0; n < NOUT; ++n)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[n][nt][e] = 0.f;

    const uint16_t *bx = bidx + bidx_off[g];
    for (int64_t k0 = 0; k0 < nk; k0 += kchunk) {
        const int kn = (int)min((int64_t)kchunk, nk - k0);
        __syncthreads();
        stage_a<float, NSF, G, TA, float, false>(reinterpret_cast<float *>(ahi), nullptr, apos, a_tr, a_val,
                                                 kb + k0, kn);
        __syncthreads();
        // split A into TF32 high and low parts in place (ahi holds the FP32 values)
        for (int t = threadIdx.x; t < kn * G * BS; t += blockDim.x) {
            const float v = __uint_as_float(ahi[t]);
            const uint32_t hi = to_tf32(v);
            ahi[t] = hi;
            alo[t] = to_tf32(v - __uint_as_float(hi));
        }
        for (int t = threadIdx.x; t < kn; t += blockDim.x) brow[t] = TB ? 0 : b_rp[k_list[kb + k0 + t]];
        stage_ix(ixs, kflag, bx, k0, kn, nj_pad, j0, jcn, JC);
        __syncthreads();
        compact_k(kact, kflag, kn, kchunk);
        __syncthreads();
        const int na = kact[kchunk];
        for (int q = 0; q < na; ++q) {
            const int kk = kact[q];
            // A fragment: rows (m, x) = grp and grp + 8, column z = tig
            const uint32_t *ah = ahi + (size_t)kk * G * BS, *al = alo + (size_t)kk * G * BS;
            const uint32_t ah0 = ah[grp * 4 + tig], ah1 = ah[32 + grp * 4 + tig];
            const uint32_t al0 = al[grp * 4 + tig], al1 = al[32 + grp * 4 + tig];
            const int64_t bk = brow[kk];
            // B fragments of every tile first (independent loads), then the MMAs
            float bv[NOUT][NT];
            bool hit[NT];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int c = wbase + 2 * nt + (grp >> 2);
                const uint16_t ix = ixs[kk * JC + c];
                hit[nt] = ix != 0xFFFF;
                const int64_t p = (TB ? brj[nt] : bk) + (hit[nt] ? ix : 0);
                // op(B)_kj[z = tig][y = grp % 4]
                const int off = TB ? ((grp & 3) * NSF + tig) : (tig * NSF + (grp & 3));
#pragma unroll
                for (int n = 0; n < NOUT; ++n)
                    bv[n][nt] = hit[nt] ? __ldg((n == 0 ? b_val1 : b_val2) + p * BS + off) : 0.f;
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                if (!__any_sync(0xffffffffu, hit[nt])) continue;
#pragma unroll
                for (int n = 0; n < NOUT; ++n) {
                    const uint32_t bh = to_tf32(bv[n][nt]);
                    const uint32_t bl = to_tf32(bv[n][nt] - __uint_as_float(bh));
                    mma_tf32_k4(acc[n][nt], ah0, ah1, bh);
                    mma_tf32_k4(acc[n][nt], ah0, ah1, bl);
                    mma_tf32_k4(acc[n][nt], al0, al1, bh);
                }
            }
        }
    }
    // D fragment: rows (m, x) = grp (c0, c1) and grp + 8 (c2, c3); columns
    // (j, y) = 2 tig and 2 tig + 1 of the tile
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int cc = 2 * tig;                     // column in the 8-wide tile
        const int jj = wbase + 2 * nt + (cc >> 2);  // output column
        const int y = cc & 3;
        if (jj >= jcn) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = grp + 8 * h, m = row >> 2, x = row & 3;
            const int32_t pos = cpos[(jb + j0 + jj) * G + m];
            if (pos < 0) continue;
#pragma unroll
            for (int n = 0; n < NOUT; ++n) {
                float *dst = (n == 0 ? c_val1 : c_val2) + (int64_t)pos * BS + x * NSF + y;
                dst[0] = acc[n][nt][2 * h];
                dst[1] = acc[n][nt][2 * h + 1];
            }
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
    LNV_CUDA(ensure_smem((const void *)kern, smem));
    kern<<<(unsigned)PC->n, kThreads, smem, ctx->stream>>>(
        PA->row_ptr, PA->col, PA->tr, (const T *)A, PB->row_ptr, PB->col, PB->tr, (const T *)B,
        PC->row_ptr, PC->col, (T *)C, kchunk);
    LNV_LAUNCHED();
    return LNV_OK;
}

constexpr int kGroupThreads = 128;



template <int NSF>
constexpr int group_cw()
{
    // lanes per output column: NSF / CW (NSF = 4: four lanes, one column each)
    return NSF == 9 ? 3 : (NSF == 4 ? 1 : NSF);
}

// Grid of a row-group launch: (column chunks, groups), groups past 65535 in z.
inline dim3 group_grid(int64_t n_groups, int64_t max_j, int jc)
{
    const int64_t gy = std::min<int64_t>(n_groups, 65535);
    return dim3((unsigned)((max_j + jc - 1) / jc), (unsigned)gy, (unsigned)((n_groups + gy - 1) / gy));
}

// Columns of J a row-group launch covers: part 0 all of them, 1 the upper part
// of a split plan, 2 the rest.  The widest group's count sizes the grid.
inline int group_part_width(const GroupPlan &gp, int part)
{
    return part == 0 ? gp.max_j : part == 1 ? gp.max_j_hi : gp.max_j_lo;
}

template <typename T, int NSF, int G, int NOUT, bool TA, bool TB, bool SPARSE>
lnv_status launch_grp(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1,
                      const void *B2, void *C1, void *C2, int part)
{
    constexpr int BS = NSF * NSF;
    constexpr int CW = group_cw<NSF>();
    constexpr int LPJ = NSF / CW;
    constexpr int OPT = NSF == 4 ? 2 : 1;
    const GroupPlan &gp = pl->grp;
    if (gp.n_groups == 0 || group_part_width(gp, part) == 0) return LNV_OK;
    if (SPARSE ? (!gp.hk && gp.hits > 0) : (!gp.bidx && gp.candidates > 0)) {
        set_error("row-group plan lacks the %s", SPARSE ? "hit lists" : "position table");
        return LNV_ERR_UNSUPPORTED;
    }
    const int jc = (kGroupThreads / 32) * (32 / LPJ) * OPT;
    const size_t per_k = (size_t)G * BS * sizeof(T) + sizeof(int64_t) + sizeof(uint32_t) +
                         2 * sizeof(int32_t) + (SPARSE ? 0 : sizeof(uint16_t) * (size_t)jc);
    int kchunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::max(gp.max_k, 1),
                                                           (SPARSE ? 40 : 32) * 1024 / per_k));
    const size_t smem = (size_t)kchunk * per_k + 128;
    auto kern = k_grp<T, NSF, G, NOUT, CW, OPT, TA, TB, SPARSE>;
    LNV_CUDA(ensure_smem((const void *)kern, smem));
    LNV_CUDA(prefer_smem((const void *)kern));
    kern<<<group_grid(gp.n_groups, group_part_width(gp, part), jc), kGroupThreads, smem, ctx->stream>>>(
        gp.k_off, gp.k_list, gp.apos, gp.j_off, gp.j_list, gp.cpos, gp.bidx_off, gp.bidx, gp.hoff,
        gp.hk, gp.hp, pl->A->tr, (const T *)A, pl->B->row_ptr, (const T *)B1, (const T *)B2,
        (T *)C1, (T *)C2, jc, kchunk, gp.n_groups, gp.jsplit, part);
    LNV_LAUNCHED();
    return LNV_OK;
}

template <int NOUT, int OPT, bool TA, bool TB>
lnv_status launch_gw(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1, const void *B2,
                     void *C1, void *C2, int part)
{
    // ring depth 4 (8 stages for the half-width shapes measured the same)
    constexpr int D = 4, NW = 2;
    using S = GwShape<NOUT, OPT, D, TA, TB>;
    const GroupPlan &gp = pl->grp;
    if (gp.n_groups == 0 || group_part_width(gp, part) == 0) return LNV_OK;
    if (!gp.bidx && gp.candidates > 0) {
        set_error("row-group plan lacks the position table");
        return LNV_ERR_UNSUPPORTED;
    }
    if (gp.max_k > 0xFFFF || pl->B->nnzb >= ((int64_t)1 << 31)) {
        set_error("row-group plan: more than 65535 k's in a group or 2^31 blocks in B");
        return LNV_ERR_UNSUPPORTED;
    }
    const size_t smem = NW * S::warp_bytes;
    constexpr int MINB = gw_min_blocks<NOUT, OPT, NW>();
    static_assert(MINB * (NW * S::warp_bytes + 1024) <= 228 * 1024, "the CTAs of one SM fit its shared memory");
    auto kern = k_gw<NOUT, OPT, D, NW, TA, TB>;
    LNV_CUDA(ensure_smem((const void *)kern, smem));
    LNV_CUDA(prefer_smem((const void *)kern));
    kern<<<group_grid(gp.n_groups, group_part_width(gp, part), NW * S::COLS), NW * 32, smem, ctx->stream>>>(
        gp.k_off, gp.apos, gp.j_off, gp.j_list, gp.cpos, gp.bidx_off, gp.bidx, gp.k_list, pl->A->tr,
        (const float *)A, pl->B->row_ptr, (const float *)B1, (const float *)B2, (float *)C1, (float *)C2,
        gp.n_groups, gp.jsplit, part);
    LNV_LAUNCHED();
    return LNV_OK;
}

template <int NOUT, bool TA, bool TB>
lnv_status launch_gmma(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1,
                       const void *B2, void *C1, void *C2)
{
    constexpr int G = 4, BS = 16, NT = 8, JC = 4 * NT * 2;
    const GroupPlan &gp = pl->grp;
    if (gp.n_groups == 0 || gp.max_j == 0) return LNV_OK;
    if (!gp.bidx) {
        set_error("row-group plan lacks the position table");
        return LNV_ERR_UNSUPPORTED;
    }
    const size_t per_k = 2 * (size_t)G * BS * sizeof(uint32_t) + sizeof(int64_t) + 2 * sizeof(int32_t) +
                         sizeof(uint16_t) * JC;
    int kchunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::max(gp.max_k, 1), (32 * 1024) / per_k));
    const size_t smem = (size_t)kchunk * per_k + 128;
    auto kern = k_gmma<NOUT, NT, TA, TB>;
    LNV_CUDA(ensure_smem((const void *)kern, smem));
    kern<<<group_grid(gp.n_groups, gp.max_j, JC), 128, smem, ctx->stream>>>(
        gp.k_off, gp.k_list, gp.apos, gp.j_off, gp.j_list, gp.cpos, gp.bidx_off, gp.bidx, pl->A->tr,
        (const float *)A, pl->B->row_ptr, (const float *)B1, (const float *)B2, (float *)C1, (float *)C2,
        kchunk, gp.n_groups);
    LNV_LAUNCHED();
    return LNV_OK;
}

// upper1: the first output is formed on its upper triangle only (a plan with
// a symmetric first output and the split on; the caller mirrors the rest).
template <typename T, int NOUT, bool TA, bool TB>
lnv_status launch_tri(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1, const void *B2,
                      void *C1, void *C2, bool upper1)
{
    const TriplePlan &tp = pl->tri;
    if (tp.n_items == 0) return LNV_OK;
    if (!tp.t_off || (!tp.tri && pl->triples > 0)) {
        set_error("plan lacks its triple lists");
        return LNV_ERR_UNSUPPORTED;
    }
    auto run = [&](const int32_t *sub, int64_t n, const void *b1, const void *b2, void *c1, void *c2, auto nout) {
        constexpr int NO = decltype(nout)::value;
        if (n == 0) return;
        k_tri<T, NO, TA, TB><<<(unsigned)((n * 4 + 127) / 128), 128, 0, ctx->stream>>>(
            n, sub, tp.item_cb, tp.t_off, tp.tri, (const T *)A, (const T *)b1, (const T *)b2, (T *)c1, (T *)c2);
    };
    if (upper1 && tp.up) {
        // the symmetric first output on its upper triangle, the second one
        // everywhere
        run(tp.up, tp.n_up, B1, nullptr, C1, nullptr, std::integral_constant<int, 1>{});
        LNV_LAUNCHED();
        if (NOUT == 2) {
            run(nullptr, tp.n_items, B2, nullptr, C2, nullptr, std::integral_constant<int, 1>{});
            LNV_LAUNCHED();
        }
        return LNV_OK;
    }
    run(nullptr, tp.n_items, B1, B2, C1, C2, std::integral_constant<int, NOUT>{});
    LNV_LAUNCHED();
    return LNV_OK;
}

// part: the columns of J to form (see group_part_width), or -1 to choose: on a
// plan whose first output is symmetric (split J), the first output is formed
// on the upper part only (the second, if any, everywhere); the caller then
// mirrors the first output's lower triangle.
template <typename T, int NSF, int NOUT, bool TA, bool TB>
lnv_status launch_group(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1,
                        const void *B2, void *C1, void *C2, int part = -1)
{
    const bool split = part == -1 && pl->sym1 && pl->split && pl->grp.jsplit;
    if (part == -1) part = split && NOUT == 1 ? 1 : 0;
    if constexpr (NSF == 4 && sizeof(T) == 4) {
        if (pl->mode == 6) return launch_gmma<NOUT, TA, TB>(ctx, pl, A, B1, B2, C1, C2);
    }
    if constexpr (NSF == 4 && sizeof(T) == 4) {
        if (pl->mode == 5 || pl->mode == 8) {
            // kernel 8: warp slices of half the width (8 columns for two
            // products, 16 for one)
            const bool half = pl->mode == 8;
            if (B2 && split && NOUT == 2) {
                // the second product alone on the rest: half-width slices either
                // way (they were the faster one-product form on every product
                // measured)
                LNV_TRY(half ? (launch_gw<2, 1, TA, TB>(ctx, pl, A, B1, B2, C1, C2, 1))
                             : (launch_gw<2, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, 1)));
                return launch_gw<1, 2, TA, TB>(ctx, pl, A, B2, nullptr, C2, nullptr, 2);
            }
            if (B2)
                return half ? launch_gw<2, 1, TA, TB>(ctx, pl, A, B1, B2, C1, C2, part)
                            : launch_gw<2, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, part);
            return half ? launch_gw<1, 2, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, part)
                        : launch_gw<1, 4, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, part);
        }
    }
    if (pl->grp.G != 4) {
        set_error("row-group size %d is not built (4 is)", pl->grp.G);
        return LNV_ERR_UNSUPPORTED;
    }
    // Two fused products need two register accumulators per row; for FP64 and
    // for NSF = 9 that exceeds the register file, so they run one at a time.
    if constexpr (NOUT == 2 && (sizeof(T) == 8 || NSF > 4)) {
        LNV_TRY((launch_group<T, NSF, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, split ? 1 : part)));
        return launch_group<T, NSF, 1, TA, TB>(ctx, pl, A, B2, nullptr, C2, nullptr, part);
    } else {
        if (split && NOUT == 2) {
            LNV_TRY((launch_group<T, NSF, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, 1)));
            return launch_group<T, NSF, 1, TA, TB>(ctx, pl, A, B2, nullptr, C2, nullptr, 2);
        }
        if (pl->mode == 4) return launch_grp<T, NSF, 4, NOUT, TA, TB, true>(ctx, pl, A, B1, B2, C1, C2, part);
        return launch_grp<T, NSF, 4, NOUT, TA, TB, false>(ctx, pl, A, B1, B2, C1, C2, part);
    }
}

constexpr int kPush2Warps = 4;

template <typename T, int NSF, int NOUT, bool TA, bool TB>
lnv_status launch_push2(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1,
                        const void *B2, void *C1, void *C2, int sym = 0)
{
    constexpr int BS = NSF * NSF;
    constexpr int NW = kPush2Warps;
    const lnv_pattern *PA = pl->A, *PB = pl->B, *PC = pl->C;
    if (PC->n == 0 || PC->max_row == 0) return LNV_OK;
    // accumulator chunk: 32 KB of shared memory, a multiple of the warp count
    int chunk = (int)((32 * 1024) / ((size_t)NOUT * BS * sizeof(T)));
    chunk = std::max(NW, std::min(chunk, ((PC->max_row + NW - 1) / NW) * NW));
    chunk = (chunk / NW) * NW;
    int kchunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::max(PA->max_row, 1),
                                                            (16 * 1024) / (BS * sizeof(T))));
    size_t smem = (size_t)NOUT * chunk * BS * sizeof(T) + (size_t)kchunk * BS * sizeof(T) +
                  sizeof(int32_t) * ((size_t)chunk + (size_t)kchunk * (NW + 2) + kchunk) + 16;
    auto kern = sym ? k_push2<T, NSF, NOUT, TA, TB, NW, true> : k_push2<T, NSF, NOUT, TA, TB, NW, false>;
    LNV_CUDA(ensure_smem((const void *)kern, smem));
    dim3 grid((unsigned)PC->n, (unsigned)((PC->max_row + chunk - 1) / chunk));
    kern<<<grid, NW * 32, smem, ctx->stream>>>(
        PA->row_ptr, PA->col, PA->tr, (const T *)A, PB->row_ptr, PB->col, PB->tr, (const T *)B1,
        (const T *)B2, PC->row_ptr, PC->col, (T *)C1, (T *)C2, chunk, kchunk);
    LNV_LAUNCHED();
    return LNV_OK;
}

constexpr int kPull2Threads = 64;

template <typename T, int NSF>
constexpr int pull2_opt()
{
    return NSF >= 9 ? 1 : 2;
}

template <typename T, int NSF, bool TA, bool TB>
lnv_status launch_pull2(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B, void *C)
{
    constexpr int BS = NSF * NSF;
    constexpr int OPT = pull2_opt<T, NSF>();
    const int chunk_out = kPull2Threads * OPT;
    const int2 *items = chunk_out == 128 ? pl->items128 : pl->items64;
    const int64_t n_items = chunk_out == 128 ? pl->n_items128 : pl->n_items64;
    if (n_items == 0) return LNV_OK;
    const lnv_pattern *PA = pl->A, *PB = pl->B, *PC = pl->C;
    size_t per_k = BS * sizeof(T) + sizeof(int32_t);
    int kchunk = (int)std::min<size_t>((16 * 1024) / per_k, (size_t)std::max(pl->max_a_row, 1));
    kchunk = std::max(kchunk, 1);
    size_t smem = (size_t)kchunk * per_k + 16;
    auto kern = k_pull2<T, NSF, OPT, TA, TB>;
    LNV_CUDA(ensure_smem((const void *)kern, smem));
    kern<<<(unsigned)n_items, kPull2Threads, smem, ctx->stream>>>(
        items, PA->row_ptr, PA->col, PA->tr, (const T *)A, PB->row_ptr, PB->col, PB->tr,
        (const T *)B, PC->row_ptr, PC->col, (T *)C, chunk_out, kchunk);
    LNV_LAUNCHED();
    return LNV_OK;
}

template <typename T, int NSF, bool TA, bool TB>
lnv_status dispatch_mode(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B1,
                         const void *B2, void *C1, void *C2)
{
    if (pl->mode == 9 || pl->mode == 12) {
        // tcgen05 tensor cores: one product, FP32 values, NSF = 4, op(B) = B^T
        // (12: single pass); other cases run the push kernel, which needs no tables
        if constexpr (NSF == 4 && sizeof(T) == 4 && TB) {
            LNV_TRY(launch_umma(ctx, pl, A, B1, C1, pl->mode == 12));
            if (B2) LNV_TRY(launch_umma(ctx, pl, A, B2, C2, pl->mode == 12));
            return LNV_OK;
        } else {
            if (B2) return launch_push2<T, NSF, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, pl->sym1 && pl->split);
            return launch_push2<T, NSF, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, pl->sym1 && pl->split);
        }
    }
    if (pl->mode == 10) {
        // tcgen05 tensor cores for 9 x 9 blocks: FP32 values, NSF = 9, either
        // transpose; other cases run the push kernel, which needs no tables
        if constexpr (NSF == 9 && sizeof(T) == 4) {
            LNV_TRY(launch_umma9(ctx, pl, TA, TB, A, B1, C1));
            if (B2) LNV_TRY(launch_umma9(ctx, pl, TA, TB, A, B2, C2));
            return LNV_OK;
        } else {
            if (B2) return launch_push2<T, NSF, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, pl->sym1 && pl->split);
            return launch_push2<T, NSF, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, pl->sym1 && pl->split);
        }
    }
    if (pl->mode == 11 || pl->mode == 13) {
        // tcgen05 tiles over their own k lists: FP32 values, NSF = 4, either
        // transpose (13: single pass); a symmetric first output on the tiles of
        // its upper part (mirrored by the caller); other cases run the push kernel
        if constexpr (NSF == 4 && sizeof(T) == 4) {
            const bool one = pl->mode == 13;
            LNV_TRY(launch_umma_tile(ctx, pl, TA, TB, pl->sym1 && pl->split, A, B1, C1, one));
            if (B2) LNV_TRY(launch_umma_tile(ctx, pl, TA, TB, false, A, B2, C2, one));
            return LNV_OK;
        } else {
            if (B2) return launch_push2<T, NSF, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, pl->sym1 && pl->split);
            return launch_push2<T, NSF, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, pl->sym1 && pl->split);
        }
    }
    if (pl->mode == 7) {
        if constexpr (NSF == 4) {
            // two fused FP32 products; FP64 runs them one at a time (registers)
            const bool up = pl->sym1 && pl->split;
            if (B2 && sizeof(T) == 4) return launch_tri<T, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, up);
            LNV_TRY((launch_tri<T, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, up)));
            if (B2) LNV_TRY((launch_tri<T, 1, TA, TB>(ctx, pl, A, B2, nullptr, C2, nullptr, false)));
            return LNV_OK;
        } else {
            // other block sizes: the push kernel, which needs no tables
            if (B2) return launch_push2<T, NSF, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, pl->sym1 && pl->split);
            return launch_push2<T, NSF, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, pl->sym1 && pl->split);
        }
    }
    if (pl->mode >= 3) {
        if (B2) return launch_group<T, NSF, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2);
        return launch_group<T, NSF, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr);
    }
    if (pl->mode == 2) {
        LNV_TRY((launch_pull2<T, NSF, TA, TB>(ctx, pl, A, B1, C1)));
        if (B2) LNV_TRY((launch_pull2<T, NSF, TA, TB>(ctx, pl, A, B2, C2)));
        return LNV_OK;
    }
    if (pl->mode == 0) {
        if (B2) return launch_push2<T, NSF, 2, TA, TB>(ctx, pl, A, B1, B2, C1, C2, pl->sym1 && pl->split);
        return launch_push2<T, NSF, 1, TA, TB>(ctx, pl, A, B1, nullptr, C1, nullptr, pl->sym1 && pl->split);
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
