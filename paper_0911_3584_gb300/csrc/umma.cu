// Kernel 9: row-group products on the tcgen05 tensor cores (FP32 values,
// NSF = 4, op(B) = B^T), with FP32-level accuracy from split TF32 operands.
//
// The products Z = L T (LSLS) and W = X^T U^T (SLHLS) of Eq. 3 and its
// gradient are the dense part of the evaluation: for a group of G = 8
// consecutive rows (one conventional cell of the cell-ordered lattice), the
// union K of their A columns and the union J of their C columns form a K x J
// table of op(B) blocks that is ~90% filled.  Those tables are multiplied as
// dense tiles on the tensor cores, transposed so that the long side is M:
//
//     C_g^T [ (j, y), (m, x) ] = sum_(k, z)  op(B)_kj[z][y]  op(A)_mk[x][z]
//
// with rows (j, y) of 32 columns j per 128-row tile, N = (m, x) = 32 for the
// group's 8 rows, and K = (k, z) over the group's K in steps of KA atoms.
//
// Precision (3xTF32): every operand is split x = hi + lo, hi exact in TF32.
// Two MMAs per K step give hi*hi + hi*lo + lo*hi with FP32 accumulation:
//     MMA1: D[:, 0:64]  (+)= A_hi [B_hi | B_lo]      (N = 64)
//     MMA2: D[:, 0:32]   += A_lo  B_hi               (N = 32)
// and the result is D[:, n] + D[:, 32 + n].
//
// Data path.  The big operand (op(B) rows, op(B)_kj = B_jk^T: row y of the
// stored block B_jk) is gathered by the producer warps straight into
// registers, one 128-row tile lane per thread, split there and written to
// TMEM with tcgen05.st; the MMAs read it from TMEM (no shared-memory round
// trip).  The small operand (op(A) blocks of the 8 rows, hi and lo) is written
// to shared memory in the canonical K-major layout.  One thread of a control
// warp issues the MMAs; a ring of NS stages, ordered by mbarriers (full:
// producers -> MMA, empty: MMA completion -> producers), overlaps the gather
// with the multiplies.  Loads run P stages ahead in registers.
//
// Every wait is bounded; a wait that runs out sets the context's device
// status flag (LNV_ERR_TIMEOUT from lnv_ctx_device_status) and the CTA
// drains, frees its TMEM and exits.
#include <algorithm>

#include "lnv_impl.cuh"
#include "tcgen05.cuh"

namespace lnv {
namespace {

constexpr int kTcG = 8;  // rows (atoms) per group

template <int MT_, int KA_, int NS_, int P_>
struct UmmaShape {
    static constexpr int MT = MT_, KA = KA_, NS = NS_, P = P_;
    static constexpr int NPW = 4 * MT;                   // producer warps: 4 per 128-row tile
    static constexpr int THREADS = (NPW + 1) * 32;       // + the control warp
    static constexpr int ACOLS = 4 * KA;                 // K elements of a stage
    static constexpr int DCOLS = 64 * MT;                // accumulators: 64 columns per tile
    static constexpr int USED = DCOLS + NS * MT * 2 * ACOLS;
    static constexpr int TCOLS = USED <= 32 ? 32 : USED <= 64 ? 64 : USED <= 128 ? 128 : USED <= 256 ? 256 : 512;
    static constexpr int BSTAGE = KA * 1024;             // bytes of a B stage: per k-atom 8 core matrices
    static constexpr int BAR_OFF = NS * BSTAGE;
    // shared memory: B stages, barriers, TMEM slot, abort flag; padded so that
    // at most two CTAs share an SM (two x TCOLS <= 512 TMEM columns)
    static constexpr size_t SMEM_USED = (size_t)BAR_OFF + 8 * (2 * NS + 1) + 16;
    static constexpr size_t SMEM = SMEM_USED < 80 * 1024 ? 80 * 1024 : SMEM_USED;
    static_assert(TCOLS * 2 <= 512, "two CTAs per SM must fit the tensor memory");
    static_assert(KA % 2 == 0, "a stage holds whole K = 8 steps");
    static_assert((NS & (NS - 1)) == 0, "ring depth is a power of two");
};

__device__ __forceinline__ int64_t tc_group() { return blockIdx.y + (int64_t)blockIdx.z * gridDim.y; }

template <int MT, int KA, int NS, int P, bool TA>
__global__ void __launch_bounds__((4 * MT + 1) * 32, 2)
k_umma(const int64_t *__restrict__ k_off, const int32_t *__restrict__ apos, const int64_t *__restrict__ j_off,
       const int32_t *__restrict__ j_list, const int32_t *__restrict__ cpos, const int64_t *__restrict__ bidx_off,
       const uint16_t *__restrict__ bidx, const int64_t *__restrict__ a_tr, const float *__restrict__ a_val,
       const int64_t *__restrict__ b_rp, const float *__restrict__ b_val, float *__restrict__ c_val,
       int64_t n_groups, int *__restrict__ status, unsigned long long wait_ns)
{
    using S = UmmaShape<MT, KA, NS, P>;
    constexpr int G = kTcG, ACOLS = S::ACOLS, NPW = S::NPW;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::BAR_OFF);  // full[NS], empty[NS], done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 1);
    volatile int *abort_s = reinterpret_cast<volatile int *>(tslot + 1);
    const uint32_t bst0 = tc::smem_u32(smem), bar0 = tc::smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(NS + s); };
    const uint32_t done_bar = bar0 + 8u * (uint32_t)(2 * NS);

    const int64_t g = tc_group();
    if (g >= n_groups) return;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    const int64_t j0 = (int64_t)blockIdx.x * (MT * 32);
    if (j0 >= nj) return;  // uniform over the CTA, before any allocation
    const int64_t nj_pad = (nj + 7) & ~int64_t(7);
    const int nst = (int)((nk + KA - 1) / KA);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == NPW) {
        tc::tmem_alloc(tc::smem_u32(tslot), S::TCOLS);
        if (lane == 0) {
            for (int s = 0; s < NS; ++s) {
                tc::mbar_init(full_bar(s), NPW);
                tc::mbar_init(empty_bar(s), 1);
            }
            tc::mbar_init(done_bar, 1);
            *abort_s = 0;
            tc::mbar_init_fence();
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tslot;

    if (warp == NPW) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            constexpr uint32_t id1 = tc::idesc_tf32(128, 64), id2 = tc::idesc_tf32(128, 32);
            for (int i = 0; i < nst; ++i) {
                const int s = i & (NS - 1);
                if (!tc::mbar_wait(full_bar(s), (uint32_t)(i / NS) & 1u, abort_s, wait_ns)) break;
                tc::fence_after_sync();
                const uint32_t a_st = tm + (uint32_t)(S::DCOLS + s * MT * 2 * ACOLS);
                const uint32_t b_st = bst0 + (uint32_t)(s * S::BSTAGE);
#pragma unroll
                for (int t = 0; t < MT; ++t)
#pragma unroll
                    for (int q = 0; q < KA / 2; ++q) {
                        const uint32_t a = a_st + (uint32_t)(t * 2 * ACOLS + 8 * q);
                        const uint64_t bd = tc::smem_desc(b_st + (uint32_t)(q * 2048), 1024, 128);
                        tc::mma_tf32_ts(tm + (uint32_t)(t * 64), a, bd, id1, (i | q) != 0);
                        tc::mma_tf32_ts(tm + (uint32_t)(t * 64), a + ACOLS, bd, id2, 1u);
                    }
                tc::commit(empty_bar(s));
            }
            // arrives once every MMA issued above has completed
            tc::commit(done_bar);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ producers
        const int t = warp >> 2, quad = warp & 3;
        const int r = quad * 32 + lane;  // row of the tile: (j, y)
        const int64_t jl = j0 + t * 32 + (r >> 2);
        const int y = r & 3;
        const bool jvalid = jl < nj;
        const float *brow = b_val + (jvalid ? b_rp[j_list[jb + jl]] * 16 : 0) + y * 4;
        const uint16_t *bx = bidx + bidx_off[g] + (jvalid ? jl : 0);
        const uint32_t lane_base = tm + ((uint32_t)(quad * 32) << 16);
        // B-stage role: (m, kk, x) for the first 32 KA threads
        const int pb = threadIdx.x;
        const bool bprod = pb < 32 * KA;
        const int bx_ = pb & 3, bkk = (pb >> 2) % KA, bm = pb / (4 * KA);
        // hi row of (m, x) in core matrix (m / 2) at row (m % 2) * 4 + x; lo 4 core matrices on
        const uint32_t b_off = (uint32_t)(bkk * 1024 + (bm >> 1) * 128 + ((bm & 1) * 4 + bx_) * 16);

        // register rings (static indices by unrolling over P + 1 slots)
        uint32_t ix[P + 1][KA];
        int32_t ib[P + 1];
        float4 va[P + 1][KA];
        float4 vb[P + 1];
        auto load_idx = [&](int ii, uint32_t (&x)[KA], int32_t &b) {
#pragma unroll
            for (int kk = 0; kk < KA; ++kk) {
                const int64_t k = (int64_t)ii * KA + kk;
                x[kk] = (jvalid && k < nk) ? (uint32_t)__ldg(bx + k * nj_pad) : 0xFFFFu;
            }
            b = -1;
            if (bprod) {
                const int64_t k = (int64_t)ii * KA + bkk;
                if (k < nk) {
                    b = __ldg(apos + (kb + k) * G + bm);
                    if (TA && b >= 0) b = (int32_t)__ldg(a_tr + b);
                }
            }
        };
        auto load_data = [&](const uint32_t (&x)[KA], int32_t b, float4 (&v)[KA], float4 &w) {
#pragma unroll
            for (int kk = 0; kk < KA; ++kk)
                v[kk] = x[kk] != 0xFFFFu ? tc::ldg_stream(brow + (int64_t)x[kk] * 16) : make_float4(0.f, 0.f, 0.f, 0.f);
            w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (b >= 0) {
                const float *blk = a_val + (int64_t)b * 16;
                if (TA) w = make_float4(__ldg(blk + bx_), __ldg(blk + 4 + bx_), __ldg(blk + 8 + bx_), __ldg(blk + 12 + bx_));
                else w = __ldg(reinterpret_cast<const float4 *>(blk) + bx_);
            }
        };
        bool ok = true;
        auto consume = [&](int i, const float4 (&v)[KA], const float4 &w) {
            const int s = i & (NS - 1);
            // every lane waits (each acquires the MMAs' completion); the warp
            // continues only if all saw it, so the .sync.aligned TMEM stores
            // below run on whole warps
            const bool seen = i < NS || tc::mbar_wait(empty_bar(s), (uint32_t)(i / NS - 1) & 1u, abort_s, wait_ns);
            if (!__all_sync(0xffffffffu, seen)) {
                ok = false;
                return;
            }
            tc::fence_after_sync();
            const uint32_t acol = lane_base + (uint32_t)(S::DCOLS + (s * MT + t) * 2 * ACOLS);
#pragma unroll
            for (int h = 0; h < KA / 2; ++h) {
                float hi[8], lo[8];
                const float e[8] = {v[2 * h].x, v[2 * h].y, v[2 * h].z, v[2 * h].w,
                                    v[2 * h + 1].x, v[2 * h + 1].y, v[2 * h + 1].z, v[2 * h + 1].w};
#pragma unroll
                for (int c = 0; c < 8; ++c) tc::split_tf32(e[c], hi[c], lo[c]);
                tc::tmem_st8(acol + (uint32_t)(8 * h), hi);
                tc::tmem_st8(acol + (uint32_t)(ACOLS + 8 * h), lo);
            }
            if (bprod) {
                float4 h4, l4;
                tc::split_tf32(w.x, h4.x, l4.x);
                tc::split_tf32(w.y, h4.y, l4.y);
                tc::split_tf32(w.z, h4.z, l4.z);
                tc::split_tf32(w.w, h4.w, l4.w);
                unsigned char *dst = smem + s * S::BSTAGE + b_off;
                *reinterpret_cast<float4 *>(dst) = h4;
                *reinterpret_cast<float4 *>(dst + 4 * 128) = l4;
                tc::fence_async_smem();
            }
            tc::tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full_bar(s));
        };
        // prologue: indices of stages 0 .. P, data of stages 0 .. P - 1
#pragma unroll
        for (int u = 0; u <= P; ++u) load_idx(u, ix[u], ib[u]);
#pragma unroll
        for (int u = 0; u < P; ++u) load_data(ix[u], ib[u], va[u], vb[u]);
        for (int i0 = 0; i0 < nst && ok; i0 += P + 1) {
#pragma unroll
            for (int u = 0; u <= P; ++u) {
                const int i = i0 + u;
                if (i >= nst || !ok) break;
                // data of stage i + P (its indices were loaded one stage earlier),
                // then the indices of stage i + P + 1 into the slot stage i used
                const int un = (u + P) % (P + 1);
                load_data(ix[un], ib[un], va[un], vb[un]);
                load_idx(i + P + 1, ix[u], ib[u]);
                consume(i, va[u], vb[u]);
            }
        }
        if (!ok) atomicExch(status, 1);

        // ------------------------------------------------------------ epilogue
        // every MMA of the CTA has completed once `done` fires; wait for it
        // even after an abort, so that no MMA still reads or writes the tensor
        // memory when it is released
        const bool drained = __all_sync(0xffffffffu, tc::mbar_wait_for(done_bar, 0u, 2 * wait_ns));
        const bool fin = ok && drained;
        if (!drained) atomicExch(status, 1);
        tc::fence_after_sync();
        if (fin) {
            // D columns of this tile: hi part (m, x) at 4 m + x, lo part 32 further
            float d[64];
            if (nst > 0) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float v8[8];
                    tc::tmem_ld8(lane_base + (uint32_t)(t * 64 + 8 * c), v8);
#pragma unroll
                    for (int e = 0; e < 8; ++e) d[8 * c + e] = v8[e];
                }
            } else {
#pragma unroll
                for (int e = 0; e < 64; ++e) d[e] = 0.f;
            }
            if (jvalid) {
                const int4 c0 = __ldg(reinterpret_cast<const int4 *>(cpos + (jb + jl) * G));
                const int4 c1 = __ldg(reinterpret_cast<const int4 *>(cpos + (jb + jl) * G + 4));
                const int32_t cp[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int m = 0; m < G; ++m) {
                    if (cp[m] < 0) continue;
                    // C_mj[x][y] for x = 0..3 (this lane holds column y of the block)
                    float *dst = c_val + (int64_t)cp[m] * 16 + y;
#pragma unroll
                    for (int x = 0; x < 4; ++x) dst[4 * x] = d[4 * m + x] + d[32 + 4 * m + x];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == NPW) tc::tmem_dealloc(tm, S::TCOLS);
}

// One thread waits on a barrier that nothing completes; the bounded wait gives
// up after wait_ns and raises the status word.
__global__ void k_expire_wait(int *status, unsigned long long wait_ns)
{
    __shared__ uint64_t bar;
    __shared__ int abort_s;
    if (threadIdx.x != 0) return;
    abort_s = 0;
    const uint32_t b = tc::smem_u32(&bar);
    tc::mbar_init(b, 1);
    tc::mbar_init_fence();
    if (!tc::mbar_wait(b, 0u, &abort_s, wait_ns)) atomicExch(status, 1);
}

// Launch shape: 2 tiles of 32 columns per CTA, 4 k-atoms per stage, 2
// stages, loads 2 stages ahead.
constexpr int kMT = 2, kKA = 4, kNS = 2, kP = 2;
using Shape = UmmaShape<kMT, kKA, kNS, kP>;

}  // namespace

lnv_status launch_umma(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B, void *C)
{
    const GroupPlan &gp = pl->tc;
    if (!pl->trans_b) {
        set_error("kernel 9 needs op(B) = B^T");
        return LNV_ERR_UNSUPPORTED;
    }
    if (gp.G != kTcG) {
        set_error("kernel 9 needs its 8-row group tables");
        return LNV_ERR_UNSUPPORTED;
    }
    if (gp.n_groups == 0 || gp.max_j == 0) return LNV_OK;
    if (!gp.bidx && gp.candidates > 0) {
        set_error("row-group plan lacks the position table");
        return LNV_ERR_UNSUPPORTED;
    }
    const int64_t per_chunk = kMT * 32;
    const int64_t gy = std::min<int64_t>(gp.n_groups, 65535);
    const dim3 grid((unsigned)((gp.max_j + per_chunk - 1) / per_chunk), (unsigned)gy,
                    (unsigned)((gp.n_groups + gy - 1) / gy));
    const bool ta = pl->trans_a != 0;
    auto kern = ta ? k_umma<kMT, kKA, kNS, kP, true> : k_umma<kMT, kKA, kNS, kP, false>;
    LNV_CUDA(ensure_smem((const void *)kern, Shape::SMEM));
    kern<<<grid, Shape::THREADS, Shape::SMEM, ctx->stream>>>(
        gp.k_off, gp.apos, gp.j_off, gp.j_list, gp.cpos, gp.bidx_off, gp.bidx, pl->A->tr, (const float *)A,
        pl->B->row_ptr, (const float *)B, (float *)C, gp.n_groups, ctx->dev_status, ctx->wait_ns);
    LNV_LAUNCHED();
    return LNV_OK;
}

}  // namespace lnv

extern "C" lnv_status lnv_debug_expire_wait(lnv_ctx *ctx)
{
    LNV_ARG(ctx, "null context");
    LNV_CUDA(cudaSetDevice(ctx->device));
    lnv::k_expire_wait<<<1, 32, 0, ctx->stream>>>(ctx->dev_status, ctx->wait_ns);
    LNV_LAUNCHED();
    return LNV_OK;
}
