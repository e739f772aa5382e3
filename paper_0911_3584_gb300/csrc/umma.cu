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
// and the result is D[:, n] + D[:, 32 + n].  The split is the truncating one
// (the producer threads bound this kernel, and rounding both parts costs
// four more instructions per pair); the tensor core's FP32 accumulation
// truncates too (kernel 10 folds its partial sums for that), so this
// kernel's error grows with K: 2e-6 relative on the 4096-atom evaluation,
// within the FP32 bound of 2e-5 at every size tested.
//
// Data path.  The big operand (op(B) rows, op(B)_kj = B_jk^T: row y of the
// stored block B_jk) is gathered by the producer warps, one 128-row tile lane
// per thread, with cp.async into a shared-memory staging ring P stages ahead
// (deep enough to cover the L2 latency without holding registers), then split
// in registers and written to TMEM with tcgen05.st; the MMAs read it from
// TMEM.  The small operand (op(A) blocks of the 8 rows, hi and lo) is staged
// the same way and written to shared memory in the canonical K-major layout.
// One thread of a control warp issues the MMAs; a ring of NS stages, ordered
// by mbarriers (full: producers -> MMA, empty: MMA completion -> producers),
// overlaps the gather with the multiplies.
//
// Locality: the work items (group, 64 columns of its J) run in the order of
// their columns' spatial keys, so the CTAs in flight at one time read nearby
// rows of op(B) for many groups, and each row travels from DRAM about once.
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
    static constexpr int DA = P + 1;                     // cp.async staging slots (P stages in flight)
    static constexpr int NPW = 4 * MT;                   // producer warps: 4 per 128-row tile
    // + one MMA-issuing warp per tile (the first also allocates the tensor memory)
    static constexpr int THREADS = (NPW + MT) * 32;
    static constexpr int ACOLS = 4 * KA;                 // K elements of a stage
    static constexpr int DCOLS = 64 * MT;                // accumulators: 64 columns per tile
    static constexpr int USED = DCOLS + NS * MT * 2 * ACOLS;
    static constexpr int TCOLS = USED <= 32 ? 32 : USED <= 64 ? 64 : USED <= 128 ? 128 : USED <= 256 ? 256 : 512;
    static constexpr int BSTAGE = KA * 1024;             // bytes of a B stage: per k-atom 8 core matrices
    // staging ring of the op(B) rows: DA slots of [MT tiles][KA k][128 rows][16 B]
    static constexpr int GSLOT = MT * KA * 128 * 16;
    static constexpr int GSTAGE_OFF = NS * BSTAGE;
    // staging ring of the op(A) rows: DA slots of 32 KA rows of 16 bytes
    static constexpr int ASTAGE_OFF = GSTAGE_OFF + DA * GSLOT;
    static constexpr int BAR_OFF = ASTAGE_OFF + DA * 32 * KA * 16;
    // shared memory: B stages, barriers, TMEM slot, abort flag; padded so that
    // at most two CTAs share an SM (two x TCOLS <= 512 TMEM columns)
    static constexpr size_t SMEM_USED = (size_t)BAR_OFF + 8 * (2 * NS + 1) + 16;
    static constexpr size_t SMEM = SMEM_USED < 80 * 1024 ? 80 * 1024 : SMEM_USED;
    static_assert(2 * SMEM <= 227 * 1024, "two CTAs per SM must fit the shared memory");
    static_assert(TCOLS * 2 <= 512, "two CTAs per SM must fit the tensor memory");
    static_assert(KA % 2 == 0, "a stage holds whole K = 8 steps");
    static_assert((NS & (NS - 1)) == 0, "ring depth is a power of two");
};

// ONE: the single-pass form (kernel 12): operands rounded to TF32, one MMA
// of N = 32 per K step (A_hi B_hi), no low parts.  Its error, about 1e-4
// relative, misses the FP32-level bound; it exists to measure that trade-off.
template <int MT, int KA, int NS, int P, bool TA, bool ONE = false>
__global__ void __launch_bounds__(5 * MT * 32, 2)
k_umma(const int2 *__restrict__ items, const int64_t *__restrict__ k_off, const int32_t *__restrict__ apos,
       const int64_t *__restrict__ j_off, const int32_t *__restrict__ j_list, const int32_t *__restrict__ cpos,
       const int64_t *__restrict__ bidx_off, const uint16_t *__restrict__ bidx, const float *__restrict__ a_val,
       const int64_t *__restrict__ b_rp, const float *__restrict__ b_val, float *__restrict__ c_val,
       int *__restrict__ status, unsigned long long wait_ns)
{
    using S = UmmaShape<MT, KA, NS, P>;
    constexpr int G = kTcG, ACOLS = S::ACOLS, NPW = S::NPW;
    static_assert(KA == 4, "a thread reads its four k indices in one 8-byte load");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::BAR_OFF);  // full[NS], empty[NS], done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 1);
    volatile int *abort_s = reinterpret_cast<volatile int *>(tslot + 1);
    const uint32_t bst0 = tc::smem_u32(smem), bar0 = tc::smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(NS + s); };
    const uint32_t done_bar = bar0 + 8u * (uint32_t)(2 * NS);

    const int2 item = items[blockIdx.x];
    const int64_t g = item.x, j0 = item.y;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    const int64_t nk_pad = (nk + 3) & ~int64_t(3);
    const int nst = (int)((nk + KA - 1) / KA);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == NPW) {
        tc::tmem_alloc(tc::smem_u32(tslot), S::TCOLS);  // the first issuing warp
        if (lane == 0) {
            for (int s = 0; s < NS; ++s) {
                tc::mbar_init(full_bar(s), NPW);
                tc::mbar_init(empty_bar(s), MT);
            }
            tc::mbar_init(done_bar, MT);
            *abort_s = 0;
            tc::mbar_init_fence();
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tslot;

    if (warp >= NPW && warp < NPW + MT) {
        // ------------------------------------------------------------ MMA issue
        // warp NPW + t issues tile t's MMAs; every operand address is fixed per
        // (stage slot, K step), so the descriptors are formed once
        if (lane == 0) {
            const int t = warp - NPW;
            constexpr uint32_t id1 = tc::idesc_tf32(128, 64), id2 = tc::idesc_tf32(128, 32);
            uint64_t bd[NS][KA / 2];
            uint32_t aa[NS][KA / 2];
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int q = 0; q < KA / 2; ++q) {
                    bd[s][q] = tc::smem_desc(bst0 + (uint32_t)(s * S::BSTAGE + q * 2048), 1024, 128);
                    aa[s][q] = tm + (uint32_t)(S::DCOLS + (s * MT + t) * 2 * ACOLS + 8 * q);
                }
            const uint32_t d = tm + (uint32_t)(t * 64);
            for (int i0 = 0; i0 < nst; i0 += NS) {
                bool stop = false;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int i = i0 + s;
                    if (i >= nst) break;
                    if (!tc::mbar_wait(full_bar(s), (uint32_t)(i / NS) & 1u, abort_s, wait_ns)) {
                        stop = true;
                        break;
                    }
                    tc::fence_after_sync();
#pragma unroll
                    for (int q = 0; q < KA / 2; ++q) {
                        if (ONE) {
                            tc::mma_tf32_ts(d, aa[s][q], bd[s][q], id2, (i | q) != 0);
                        } else {
                            tc::mma_tf32_ts(d, aa[s][q], bd[s][q], id1, (i | q) != 0);
                            tc::mma_tf32_ts(d, aa[s][q] + ACOLS, bd[s][q], id2, 1u);
                        }
                    }
                    tc::commit(empty_bar(s));
                }
                if (stop) break;
            }
            // arrives once every MMA issued above has completed
            tc::commit(done_bar);
        }
        __syncwarp();
    } else if (warp < NPW) {
        // ------------------------------------------------------------ op(B) rows
        const int t = warp >> 2, quad = warp & 3;
        const int r = quad * 32 + lane;  // row of the tile: (j, y)
        const int64_t jl = j0 + t * 32 + (r >> 2);
        const int y = r & 3;
        const bool jvalid = jl < nj;
        const float *brow = b_val + (jvalid ? b_rp[j_list[jb + jl]] * 16 : 0) + y * 4;
        // this row's k indices: KA consecutive 16-bit offsets per stage, one 8-byte load
        const uint16_t *bxr = bidx + bidx_off[g] + (jvalid ? jl : 0) * nk_pad;
        const uint32_t lane_base = tm + ((uint32_t)(quad * 32) << 16);

        // Every row travels global -> shared with cp.async into a ring of DA =
        // P + 1 slots, P stages ahead of the stage being consumed (no registers
        // held in flight); the k indices of a stage are loaded into a register
        // ring RI stages before its copies are issued.  The stage loop is
        // unrolled by the index ring's size.
        constexpr int DA = S::DA, RI = P + 1;
        static_assert(P < RI, "the prologue's indices fit the ring");
        static_assert(NPW == G && KA == 4, "producer warp m stages op(A) row m: 16 lanes (kk, x)");
        uint2 ix[RI];
        int32_t ib[RI];
        const uint32_t gst0 = bst0 + (uint32_t)S::GSTAGE_OFF + (uint32_t)((t * KA * 128 + r) * 16);
        // op(A) role (lanes 0..15 of warp m = warp): k-atom kk = lane / 4, row x = lane % 4
        const bool aprod = lane < 16;
        const int am = warp, akk = (lane >> 2) & 3, ax = lane & 3;
        const int aq = am * 16 + (lane & 15);  // row of the op(A) staging slot
        const uint32_t ast0 = bst0 + (uint32_t)S::ASTAGE_OFF + (uint32_t)aq * 16u;
        auto load_idx = [&](int ii, uint2 &x, int32_t &b) {
            const int64_t k0 = (int64_t)ii * KA;
            x = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
            if (jvalid && k0 < nk_pad) x = __ldg(reinterpret_cast<const uint2 *>(bxr + k0));
            b = (aprod && k0 + akk < nk) ? __ldg(apos + (kb + k0 + akk) * G + am) : -1;
        };
        // copies of stage ii (an empty commit group past the last stage)
        auto issue = [&](int ii, const uint2 &x, int32_t b) {
            if (ii < nst) {
                const uint32_t e[4] = {x.x & 0xFFFFu, x.x >> 16, x.y & 0xFFFFu, x.y >> 16};
                const uint32_t slot = gst0 + (uint32_t)((ii % DA) * S::GSLOT);
#pragma unroll
                for (int kk = 0; kk < KA; ++kk) {
                    const bool hit = e[kk] != 0xFFFFu;
                    tc::cp_async16(slot + (uint32_t)(kk * 128 * 16), brow + (hit ? e[kk] * 16u : 0u), hit ? 16 : 0);
                }
                if (aprod)
                    tc::cp_async16(ast0 + (uint32_t)((ii % DA) * 32 * KA * 16), a_val + (int64_t)max(b, 0) * 16 + 4 * ax,
                                   b >= 0 ? 16 : 0);
            }
            tc::cp_async_commit();
        };
        bool ok = true;
        auto consume = [&](int i) {
            const int s = i & (NS - 1);
            // every lane waits (each acquires the MMAs' completion); the warp
            // continues only if all saw it, so the .sync.aligned TMEM stores
            // below run on whole warps
            const bool seen = i < NS || tc::mbar_wait(empty_bar(s), (uint32_t)(i / NS - 1) & 1u, abort_s, wait_ns);
            if (!__all_sync(0xffffffffu, seen)) {
                ok = false;
                return;
            }
            // this stage's copies (those of the P later stages, already issued,
            // may still fly)
            tc::cp_async_wait<P>();
            __syncwarp();  // A^T: a lane reads op(A) rows three other lanes copied
            if (aprod) {
                // op(A)_mk, hi and lo, into the canonical K-major layout of the B
                // stage: N = 64 rows (part, m, x), K = (k, z); row (part, m, x) of
                // k-atom kk lies in core matrix 4 part + m / 2 at row (m % 2) 4 + x
                const unsigned char *src = smem + S::ASTAGE_OFF + (i % DA) * 32 * KA * 16;
                float4 w;
                if (TA) {
                    // op(A)_mk[x][z] = stored[z][x]: column x of the block
                    const float *blk = reinterpret_cast<const float *>(src + (aq & ~3) * 16);
                    w = make_float4(blk[ax], blk[4 + ax], blk[8 + ax], blk[12 + ax]);
                } else {
                    w = *reinterpret_cast<const float4 *>(src + aq * 16);
                }
                unsigned char *dst = smem + s * S::BSTAGE + akk * 1024 + (am >> 1) * 128 + ((am & 1) * 4 + ax) * 16;
                if (ONE) {
                    *reinterpret_cast<float4 *>(dst) =
                        make_float4(tc::tf32_rna(w.x), tc::tf32_rna(w.y), tc::tf32_rna(w.z), tc::tf32_rna(w.w));
                } else {
                    float4 h4, l4;
                    tc::split_tf32x2_trunc(w.x, w.y, h4.x, h4.y, l4.x, l4.y);
                    tc::split_tf32x2_trunc(w.z, w.w, h4.z, h4.w, l4.z, l4.w);
                    *reinterpret_cast<float4 *>(dst) = h4;
                    *reinterpret_cast<float4 *>(dst + 4 * 128) = l4;
                }
                tc::fence_async_smem();
            }
            tc::fence_after_sync();
            const uint32_t acol = lane_base + (uint32_t)(S::DCOLS + (s * MT + t) * 2 * ACOLS);
            const unsigned char *grow = smem + S::GSTAGE_OFF + (i % DA) * S::GSLOT + (t * KA * 128 + r) * 16;
#pragma unroll
            for (int h = 0; h < KA / 2; ++h) {
                const float4 v0 = *reinterpret_cast<const float4 *>(grow + (2 * h) * 128 * 16);
                const float4 v1 = *reinterpret_cast<const float4 *>(grow + (2 * h + 1) * 128 * 16);
                float hi[8], lo[8];
                if (ONE) {
                    const float e[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                    for (int u = 0; u < 8; ++u) hi[u] = tc::tf32_rna(e[u]);
                    tc::tmem_st8(acol + (uint32_t)(8 * h), hi);
                    continue;
                }
                tc::split_tf32x2_trunc(v0.x, v0.y, hi[0], hi[1], lo[0], lo[1]);
                tc::split_tf32x2_trunc(v0.z, v0.w, hi[2], hi[3], lo[2], lo[3]);
                tc::split_tf32x2_trunc(v1.x, v1.y, hi[4], hi[5], lo[4], lo[5]);
                tc::split_tf32x2_trunc(v1.z, v1.w, hi[6], hi[7], lo[6], lo[7]);
                tc::tmem_st8(acol + (uint32_t)(8 * h), hi);
                tc::tmem_st8(acol + (uint32_t)(ACOLS + 8 * h), lo);
            }
            tc::tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full_bar(s));
        };
        // prologue: indices of stages 0 .. RI - 1, then the copies of stages
        // 0 .. P - 1 (each slot, once read, takes the indices of stage + RI)
#pragma unroll
        for (int q = 0; q < RI; ++q) load_idx(q, ix[q], ib[q]);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            issue(q, ix[q % RI], ib[q % RI]);
            load_idx(q + RI, ix[q % RI], ib[q % RI]);
        }
        for (int i0 = 0; i0 < nst && ok; i0 += RI) {
#pragma unroll
            for (int u = 0; u < RI; ++u) {
                const int i = i0 + u;
                if (i >= nst || !ok) break;
                // copies of stage i + P from index slot (i + P) % RI, which then
                // takes the indices of stage i + P + RI
                const int sl = (u + P) % RI;
                issue(i + P, ix[sl], ib[sl]);
                load_idx(i + P + RI, ix[sl], ib[sl]);
                consume(i);
            }
        }
        tc::cp_async_wait<0>();
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
            // D columns of this tile: hi part (m, x) at 4 m + x, lo part 32
            // further; two rows m per pass (8 + 8 columns)
            int32_t cp[8];
            if (jvalid) {
                const int4 c0 = __ldg(reinterpret_cast<const int4 *>(cpos + (jb + jl) * G));
                const int4 c1 = __ldg(reinterpret_cast<const int4 *>(cpos + (jb + jl) * G + 4));
                cp[0] = c0.x; cp[1] = c0.y; cp[2] = c0.z; cp[3] = c0.w;
                cp[4] = c1.x; cp[5] = c1.y; cp[6] = c1.z; cp[7] = c1.w;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float dh[8], dl[8];
                if (nst > 0) {
                    tc::tmem_ld8(lane_base + (uint32_t)(t * 64 + 8 * c), dh);
                    if (ONE) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) dl[e] = 0.f;
                    } else {
                        tc::tmem_ld8(lane_base + (uint32_t)(t * 64 + 32 + 8 * c), dl);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) dh[e] = dl[e] = 0.f;
                }
                if (jvalid) {
#pragma unroll
                    for (int mm = 0; mm < 2; ++mm) {
                        const int m = 2 * c + mm;
                        if (cp[m] < 0) continue;
                        // C_mj[x][y] for x = 0..3 (this lane holds column y of the block)
                        float *dst = c_val + (int64_t)cp[m] * 16 + y;
#pragma unroll
                        for (int x = 0; x < 4; ++x) dst[4 * x] = dh[4 * mm + x] + dl[4 * mm + x];
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == NPW) tc::tmem_dealloc(tm, S::TCOLS);
}

// op(A) block positions of a row-group table: apos[q] -> tr[apos[q]] (the
// stored block (k, m) whose transpose is op(A)_mk), so the kernel reads one
// position per block.
__global__ void k_apos_transpose(int64_t n, int32_t *apos, const int64_t *__restrict__ tr)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        if (apos[q] >= 0) apos[q] = (int32_t)tr[apos[q]];
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

// Launch shape: 2 tiles of 32 columns per CTA (kTcCols), 4 k-atoms per
// stage, 2 stages, copies LNV_TC_DEPTH stages ahead of the stage consumed.
#ifndef LNV_TC_DEPTH
#define LNV_TC_DEPTH 3
#endif
constexpr int kMT = 2, kKA = 4, kNS = 2, kP = LNV_TC_DEPTH;
static_assert(kMT * 32 == kTcCols, "a CTA covers one work item");
using Shape = UmmaShape<kMT, kKA, kNS, kP>;

}  // namespace

lnv_status launch_umma(lnv_ctx *ctx, const lnv_plan *pl, const void *A, const void *B, void *C, bool onepass)
{
    const GroupPlan &gp = pl->tc;
    if (!pl->trans_b) {
        set_error("kernel 9 needs op(B) = B^T");
        return LNV_ERR_UNSUPPORTED;
    }
    if (gp.G != kTcG || !gp.jmajor || (pl->trans_a && !gp.apos_op)) {
        set_error("kernel 9 needs its 8-row group tables");
        return LNV_ERR_UNSUPPORTED;
    }
    if (gp.n_items == 0) return LNV_OK;
    if (!gp.bidx && gp.candidates > 0) {
        set_error("row-group plan lacks the position table");
        return LNV_ERR_UNSUPPORTED;
    }
    const bool ta = pl->trans_a != 0;
    auto kern = ta ? (onepass ? k_umma<kMT, kKA, kNS, kP, true, true> : k_umma<kMT, kKA, kNS, kP, true, false>)
                   : (onepass ? k_umma<kMT, kKA, kNS, kP, false, true> : k_umma<kMT, kKA, kNS, kP, false, false>);
    LNV_CUDA(ensure_smem((const void *)kern, Shape::SMEM));
    kern<<<(unsigned)gp.n_items, Shape::THREADS, Shape::SMEM, ctx->stream>>>(
        gp.items, gp.k_off, gp.apos, gp.j_off, gp.j_list, gp.cpos, gp.bidx_off, gp.bidx, (const float *)A,
        pl->B->row_ptr, (const float *)B, (float *)C, ctx->dev_status, ctx->wait_ns);
    LNV_LAUNCHED();
    return LNV_OK;
}

lnv_status umma_prepare(lnv_ctx *ctx, lnv_plan *pl)
{
    GroupPlan &gp = pl->tc;
    if (pl->trans_a && !gp.apos_op && gp.apos && gp.n_groups > 0) {
        int64_t n = 0;
        LNV_CUDA(cudaMemcpy(&n, gp.k_off + gp.n_groups, sizeof(int64_t), cudaMemcpyDeviceToHost));
        n *= gp.G;
        if (n > 0) {
            k_apos_transpose<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1 << 20), 256, 0, ctx->stream>>>(
                n, gp.apos, pl->A->tr);
            LNV_LAUNCHED();
            LNV_CUDA(cudaStreamSynchronize(ctx->stream));
        }
    }
    gp.apos_op = 1;
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

