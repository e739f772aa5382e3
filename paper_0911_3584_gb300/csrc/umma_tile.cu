// Kernel 11: row-group products on the tcgen05 tensor cores (FP32 values,
// NSF = 4, either op(B)), one tile of 32 output columns of an 8-row group per
// CTA, multiplied over that tile's own list of k's.
//
// Kernel 9 multiplies a group's whole K x J table of op(B) blocks as dense
// tiles, which pays where the table is nearly full (Z = L T and W = X^T U^T
// of Eq. 3: about 95% of the (k, j) pairs present).  For T = S X and U = S Y
// (SLS and SLH) a group's K, the union of its rows' S neighbours, meets each
// column j of the long range R_T = R_L + 2 R_SH in a few k only: a quarter of
// the table is present.  Listing, per tile of 32 columns, only the k's at
// which one of its columns holds a block (padded to whole stages of four)
// raises the useful share of the multiplied blocks on the 4096-atom Si
// workload from 0.10 to 0.16 (Z on kernel 9: 0.32).  Per tile:
//
//     C^T [ (j, y), (m, x) ] = sum_(k listed, z)  op(B)_kj[z][y]  op(A)_mk[x][z]
//
// with M = (j, y) = 128 rows for the tile's 32 columns, N = (m, x) = 32 for
// the group's 8 rows.  Precision, pipeline and epilogue follow kernel 9
// (3xTF32 with the truncating split, FP32 accumulation in tensor memory, a
// cp.async staging ring P stages ahead of two MMA stages, every wait bounded).
// What differs:
//  - one 128-row tile per CTA: four producer warps, one MMA warp, 128 TMEM
//    columns, four CTAs per SM (the shared memory admits no fifth, so the
//    four always find their tensor memory);
//  - op(B) = B: lane (j, y) needs column y of the stored block B_kj.  The four
//    lanes of column j copy the block's four rows (16 bytes each) into their
//    four staging slots, rotated by (j / 2) mod 4, and each lane then reads
//    its column across them; with that rotation the 32 lanes of a warp hit 32
//    different banks;
//  - its tables (TilePlan): per item its k list, B's row start per listed k
//    (op(B) = B), the 8 rows' op(A) positions per listed k, and a j-major
//    table of 16-bit block offsets.
#include <algorithm>
#include <vector>

#include "lnv_impl.cuh"
#include "tcgen05.cuh"

namespace lnv {
namespace {

constexpr int kG = 8;        // rows (atoms) per group: kernel 9's tables
constexpr int kCols = 32;    // output columns per tile (M = 128)
constexpr int kKA = 4;       // k-atoms per stage (K = 16)
constexpr int kNS = 2;       // MMA stages (operand buffers)
#ifndef LNV_TT_DEPTH
#define LNV_TT_DEPTH 3
#endif
constexpr int kP = LNV_TT_DEPTH;      // copies in flight, in stages
constexpr int kDA = kP + 1;           // staging slots
constexpr int kNPW = 4;               // producer warps: one per 32 tile rows
constexpr int kThreads = (kNPW + 1) * 32;
constexpr int kACOLS = 4 * kKA;       // TMEM columns of one part (hi or lo) of a stage
constexpr int kDCOLS = 64;            // accumulator: hi*hi + hi*lo in 0..31, + lo*hi's 32..63 (below)
constexpr int kTCOLS = 128;
static_assert(kDCOLS + kNS * 2 * kACOLS <= kTCOLS, "accumulator and operand stages fit");
constexpr int kBSTAGE = kKA * 1024;             // op(A) operand stage: N = 64 rows (hi, lo) x K = 16
constexpr int kGSLOT = kKA * 128 * 16;          // op(B) staging slot: [k-atom][tile row][16 bytes]
constexpr int kASLOT = 32 * kKA * 16;           // op(A) staging slot: [m][k-atom][x][16 bytes]
constexpr int kGSTAGE_OFF = kNS * kBSTAGE;
constexpr int kASTAGE_OFF = kGSTAGE_OFF + kDA * kGSLOT;
constexpr int kBAR_OFF = kASTAGE_OFF + kDA * kASLOT;
constexpr size_t kSmemUsed = (size_t)kBAR_OFF + 8 * (2 * kNS + 1) + 16;
// padded so that four CTAs share an SM and a fifth does not fit (4 x 128 TMEM
// columns); 1 KB per CTA is reserved by the system
constexpr size_t kSmem = 52 * 1024;
static_assert(kSmemUsed <= kSmem, "shared memory layout fits");
static_assert(4 * (kSmem + 1024) <= 228 * 1024 && 5 * (kSmem + 1024) > 228 * 1024,
              "exactly four CTAs per SM");
static_assert(kKA == 4 && kNPW * 32 == 4 * kCols, "a lane reads its four k offsets in one 8-byte load");

// ONE: the single-pass form (kernel 13): operands rounded to TF32, one MMA of
// N = 32 per K step, no low parts (about 1e-4 relative error: it misses the
// FP32-level bound and is kept to measure that trade-off).
template <bool TA, bool TB, bool ONE>
__global__ void __launch_bounds__(kThreads, 4)
k_umma_tile(const int32_t *__restrict__ sub, const int2 *__restrict__ items, const int64_t *__restrict__ ck_off,
            const int32_t *__restrict__ ck_brow, const int32_t *__restrict__ ck_apos,
            const uint16_t *__restrict__ ck_tab, const int64_t *__restrict__ j_off,
            const int32_t *__restrict__ j_list, const int32_t *__restrict__ cpos, const float *__restrict__ a_val,
            const int64_t *__restrict__ b_rp, const float *__restrict__ b_val, float *__restrict__ c_val,
            int *__restrict__ status, unsigned long long wait_ns)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kBAR_OFF);  // full[NS], empty[NS], done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * kNS + 1);
    volatile int *abort_s = reinterpret_cast<volatile int *>(tslot + 1);
    const uint32_t bst0 = tc::smem_u32(smem), bar0 = tc::smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(kNS + s); };
    const uint32_t done_bar = bar0 + 8u * (uint32_t)(2 * kNS);

    const int64_t it = sub ? (int64_t)sub[blockIdx.x] : (int64_t)blockIdx.x;
    const int2 item = items[it];
    const int64_t g = item.x, j0 = item.y;
    const int64_t c0 = ck_off[it], nkc = ck_off[it + 1] - c0;  // a multiple of kKA
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    const int nst = (int)(nkc / kKA);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == kNPW) {
        tc::tmem_alloc(tc::smem_u32(tslot), kTCOLS);
        if (lane == 0) {
            for (int s = 0; s < kNS; ++s) {
                tc::mbar_init(full_bar(s), kNPW);
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

    if (warp == kNPW) {
        // ------------------------------------------------------------ MMA issue
        // D[:, 0:64] (+)= A_hi [B_hi | B_lo] and D[:, 0:32] += A_lo B_hi per
        // K = 8 step; the operand addresses are fixed per (stage, step)
        if (lane == 0) {
            constexpr uint32_t id1 = tc::idesc_tf32(128, 64), id2 = tc::idesc_tf32(128, 32);
            uint64_t bd[kNS][kKA / 2];
            uint32_t aa[kNS][kKA / 2];
#pragma unroll
            for (int s = 0; s < kNS; ++s)
#pragma unroll
                for (int q = 0; q < kKA / 2; ++q) {
                    bd[s][q] = tc::smem_desc(bst0 + (uint32_t)(s * kBSTAGE + q * 2048), 1024, 128);
                    aa[s][q] = tm + (uint32_t)(kDCOLS + s * 2 * kACOLS + 8 * q);
                }
            for (int i0 = 0; i0 < nst; i0 += kNS) {
                bool stop = false;
#pragma unroll
                for (int s = 0; s < kNS; ++s) {
                    const int i = i0 + s;
                    if (i >= nst) break;
                    if (!tc::mbar_wait(full_bar(s), (uint32_t)(i / kNS) & 1u, abort_s, wait_ns)) {
                        stop = true;
                        break;
                    }
                    tc::fence_after_sync();
#pragma unroll
                    for (int q = 0; q < kKA / 2; ++q) {
                        if (ONE) {
                            tc::mma_tf32_ts(tm, aa[s][q], bd[s][q], id2, (i | q) != 0);
                        } else {
                            tc::mma_tf32_ts(tm, aa[s][q], bd[s][q], id1, (i | q) != 0);
                            tc::mma_tf32_ts(tm, aa[s][q] + kACOLS, bd[s][q], id2, 1u);
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
    } else {
        // ------------------------------------------------------------ producers
        const int r = warp * 32 + lane;  // tile row (j, y)
        const int jl = r >> 2, y = r & 3;
        const int64_t jc = j0 + jl;       // column of the group's J
        const bool jvalid = jc < nj;
        const int rot = (jl >> 1) & 3;
        // op(B) = B^T: this lane copies row y of the stored block B_jk from B's
        // row j; op(B) = B: row y of B_kj from B's row k (given per listed k)
        const float *brow = b_val + (TB && jvalid ? b_rp[j_list[jb + jc]] * 16 : 0) + y * 4;
        const uint16_t *tabr = ck_tab + c0 * kCols + (int64_t)jl * nkc;
        const uint32_t lane_base = tm + ((uint32_t)(warp * 32) << 16);
        // op(A) role: lane -> group row m, k-atom kk, block row x
        const int am = 2 * warp + (lane >> 4), akk = (lane >> 2) & 3, ax = lane & 3;
        const int aq = am * 16 + (lane & 15);  // row of the op(A) staging slot
        const uint32_t ast0 = bst0 + (uint32_t)kASTAGE_OFF + (uint32_t)aq * 16u;
        // op(B) staging: row r of the slot, or (op(B) = B) block row y of
        // column j at its rotated place among column j's four rows
        const uint32_t gdst = TB ? (uint32_t)r * 16u : (uint32_t)(4 * jl + ((y + rot) & 3)) * 16u;
        const uint32_t gst0 = bst0 + (uint32_t)kGSTAGE_OFF + gdst;

        constexpr int RI = kP + 1;
        uint2 ix[RI];
        int4 ibr[RI];
        int32_t ib[RI];
        auto load_idx = [&](int ii, uint2 &x, int4 &br, int32_t &b) {
            x = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
            br = make_int4(0, 0, 0, 0);
            b = -1;
            if (ii < nst) {
                if (jvalid) x = __ldg(reinterpret_cast<const uint2 *>(tabr + (int64_t)ii * kKA));
                if (!TB) br = __ldg(reinterpret_cast<const int4 *>(ck_brow + c0 + (int64_t)ii * kKA));
                b = __ldg(ck_apos + (c0 + (int64_t)ii * kKA + akk) * kG + am);
            }
        };
        // copies of stage ii (an empty commit group past the last stage)
        auto issue = [&](int ii, const uint2 &x, const int4 &br, int32_t b) {
            if (ii < nst) {
                const uint32_t e[4] = {x.x & 0xFFFFu, x.x >> 16, x.y & 0xFFFFu, x.y >> 16};
                const int32_t rb[4] = {br.x, br.y, br.z, br.w};
                const uint32_t slot = gst0 + (uint32_t)((ii % kDA) * kGSLOT);
#pragma unroll
                for (int kk = 0; kk < kKA; ++kk) {
                    const bool hit = e[kk] != 0xFFFFu;
                    const float *src = TB ? brow + (hit ? e[kk] * 16u : 0u)
                                          : b_val + (hit ? ((int64_t)rb[kk] + e[kk]) * 16 + y * 4 : 0);
                    tc::cp_async16(slot + (uint32_t)(kk * 128 * 16), src, hit ? 16 : 0);
                }
                tc::cp_async16(ast0 + (uint32_t)((ii % kDA) * kASLOT), a_val + (int64_t)max(b, 0) * 16 + 4 * ax,
                               b >= 0 ? 16 : 0);
            }
            tc::cp_async_commit();
        };
        bool ok = true;
        auto consume = [&](int i) {
            const int s = i & (kNS - 1);
            const bool seen = i < kNS || tc::mbar_wait(empty_bar(s), (uint32_t)(i / kNS - 1) & 1u, abort_s, wait_ns);
            if (!__all_sync(0xffffffffu, seen)) {
                ok = false;
                return;
            }
            tc::cp_async_wait<kP>();
            __syncwarp();  // lanes read rows that other lanes of the warp copied
            {
                // op(A)_mk, hi and lo, into the canonical K-major layout of the
                // operand stage: row (part, m, x) of k-atom kk in core matrix
                // 4 part + m / 2, row (m % 2) 4 + x
                const unsigned char *src = smem + kASTAGE_OFF + (i % kDA) * kASLOT;
                float4 w;
                if (TA) {
                    const float *blk = reinterpret_cast<const float *>(src + (aq & ~3) * 16);
                    w = make_float4(blk[ax], blk[4 + ax], blk[8 + ax], blk[12 + ax]);
                } else {
                    w = *reinterpret_cast<const float4 *>(src + aq * 16);
                }
                unsigned char *dst = smem + s * kBSTAGE + akk * 1024 + (am >> 1) * 128 + ((am & 1) * 4 + ax) * 16;
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
            const uint32_t acol = lane_base + (uint32_t)(kDCOLS + s * 2 * kACOLS);
            const unsigned char *gs = smem + kGSTAGE_OFF + (i % kDA) * kGSLOT;
#pragma unroll
            for (int h = 0; h < kKA / 2; ++h) {
                float4 v[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int kk = 2 * h + u;
                    if (TB) {
                        v[u] = *reinterpret_cast<const float4 *>(gs + (kk * 128 + r) * 16);
                    } else {
                        // column y of B_kj: element y of its rows z = 0..3
                        const float *c4 = reinterpret_cast<const float *>(gs + (kk * 128 + 4 * jl) * 16) + y;
                        v[u] = make_float4(c4[((0 + rot) & 3) * 4], c4[((1 + rot) & 3) * 4],
                                           c4[((2 + rot) & 3) * 4], c4[((3 + rot) & 3) * 4]);
                    }
                }
                float hi[8], lo[8];
                if (ONE) {
                    const float e[8] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w};
#pragma unroll
                    for (int u = 0; u < 8; ++u) hi[u] = tc::tf32_rna(e[u]);
                    tc::tmem_st8(acol + (uint32_t)(8 * h), hi);
                    continue;
                }
                tc::split_tf32x2_trunc(v[0].x, v[0].y, hi[0], hi[1], lo[0], lo[1]);
                tc::split_tf32x2_trunc(v[0].z, v[0].w, hi[2], hi[3], lo[2], lo[3]);
                tc::split_tf32x2_trunc(v[1].x, v[1].y, hi[4], hi[5], lo[4], lo[5]);
                tc::split_tf32x2_trunc(v[1].z, v[1].w, hi[6], hi[7], lo[6], lo[7]);
                tc::tmem_st8(acol + (uint32_t)(8 * h), hi);
                tc::tmem_st8(acol + (uint32_t)(kACOLS + 8 * h), lo);
            }
            tc::tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full_bar(s));
        };
#pragma unroll
        for (int q = 0; q < RI; ++q) load_idx(q, ix[q], ibr[q], ib[q]);
#pragma unroll
        for (int q = 0; q < kP; ++q) {
            issue(q, ix[q % RI], ibr[q % RI], ib[q % RI]);
            load_idx(q + RI, ix[q % RI], ibr[q % RI], ib[q % RI]);
        }
        for (int i0 = 0; i0 < nst && ok; i0 += RI) {
#pragma unroll
            for (int u = 0; u < RI; ++u) {
                const int i = i0 + u;
                if (i >= nst || !ok) break;
                const int sl = (u + kP) % RI;
                issue(i + kP, ix[sl], ibr[sl], ib[sl]);
                load_idx(i + kP + RI, ix[sl], ibr[sl], ib[sl]);
                consume(i);
            }
        }
        tc::cp_async_wait<0>();
        if (!ok) atomicExch(status, 1);

        // ------------------------------------------------------------ epilogue
        // every MMA has completed once `done` fires; wait for it even after an
        // abort, so that no MMA still uses the tensor memory when it is freed
        const bool drained = __all_sync(0xffffffffu, tc::mbar_wait_for(done_bar, 0u, 2 * wait_ns));
        const bool fin = ok && drained;
        if (!drained) atomicExch(status, 1);
        tc::fence_after_sync();
        if (fin) {
            int32_t cp[8];
            if (jvalid) {
                const int4 p0 = __ldg(reinterpret_cast<const int4 *>(cpos + (jb + jc) * kG));
                const int4 p1 = __ldg(reinterpret_cast<const int4 *>(cpos + (jb + jc) * kG + 4));
                cp[0] = p0.x; cp[1] = p0.y; cp[2] = p0.z; cp[3] = p0.w;
                cp[4] = p1.x; cp[5] = p1.y; cp[6] = p1.z; cp[7] = p1.w;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float dh[8], dl[8];
                if (nst > 0) {
                    tc::tmem_ld8(lane_base + (uint32_t)(8 * c), dh);
                    if (ONE) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) dl[e] = 0.f;
                    } else {
                        tc::tmem_ld8(lane_base + (uint32_t)(32 + 8 * c), dl);
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
    if (warp == kNPW) tc::tmem_dealloc(tm, kTCOLS);
}

// ------------------------------------------------------------------ tile plan

// Warp per item: lane = column c + lane of the group's J.  Walks the group's
// K in order and keeps the k's at which any of the 32 columns holds a block:
// counts them (cnt, rounded up to a multiple of kKA) or writes them (B's row
// start, the op(A) positions and the offsets, padded with empty entries).
__global__ void k_tile_lists(int64_t n_items, const int2 *__restrict__ items, const int64_t *__restrict__ k_off,
                             const int32_t *__restrict__ k_list, const int32_t *__restrict__ apos,
                             const int64_t *__restrict__ j_off, const int64_t *__restrict__ bidx_off,
                             const uint16_t *__restrict__ bidx, const int64_t *__restrict__ b_rp, int trans_b,
                             int64_t *cnt, const int64_t *__restrict__ ck_off, int32_t *ck_brow, int32_t *ck_apos,
                             uint16_t *ck_tab)
{
    const int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (it >= n_items) return;
    const int2 item = items[it];
    const int64_t g = item.x, kb = k_off[g], nk = k_off[g + 1] - kb, nj = j_off[g + 1] - j_off[g];
    const int64_t nk_pad = (nk + 3) & ~int64_t(3);
    const int64_t jc = item.y + lane;
    const bool valid = jc < nj;
    const uint16_t *col = bidx + bidx_off[g] + (valid ? jc : 0) * nk_pad;
    const int64_t c0 = cnt ? 0 : ck_off[it], nkc = cnt ? 0 : ck_off[it + 1] - c0;
    int64_t n = 0;
    for (int64_t k = 0; k < nk; ++k) {
        const uint16_t v = valid ? col[k] : (uint16_t)0xFFFF;
        if (!__any_sync(0xffffffffu, v != 0xFFFF)) continue;
        if (!cnt) {
            const int64_t p = c0 + n;
            if (lane == 0) ck_brow[p] = trans_b ? 0 : (int32_t)b_rp[k_list[kb + k]];
            if (lane < kG) ck_apos[p * kG + lane] = apos[(kb + k) * kG + lane];
            ck_tab[c0 * kCols + (int64_t)lane * nkc + n] = v;
        }
        ++n;
    }
    if (cnt) {
        if (lane == 0) cnt[it] = (n + kKA - 1) / kKA * kKA;
        return;
    }
    for (; n < nkc; ++n) {
        const int64_t p = c0 + n;
        if (lane == 0) ck_brow[p] = 0;
        if (lane < kG) ck_apos[p * kG + lane] = -1;
        ck_tab[c0 * kCols + (int64_t)lane * nkc + n] = 0xFFFF;
    }
}

template <typename X>
cudaError_t upload_vec(const std::vector<X> &h, X **d)
{
    cudaError_t e = cudaMalloc(d, sizeof(X) * std::max<size_t>(1, h.size()));
    if (e == cudaSuccess && !h.empty()) e = cudaMemcpy(*d, h.data(), sizeof(X) * h.size(), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

void tile_plan_free(TilePlan *tt)
{
    cudaFree(tt->items);
    cudaFree(tt->ck_off);
    cudaFree(tt->ck_brow);
    cudaFree(tt->ck_apos);
    cudaFree(tt->ck_tab);
    cudaFree(tt->up);
    *tt = TilePlan();
}

lnv_status tile_plan_build(lnv_ctx *ctx, lnv_plan *pl, size_t budget_bytes)
{
    const GroupPlan &gp = pl->tc;
    TilePlan &tt = pl->tt;
    if (tt.items && tt.src == gp.items) return LNV_OK;
    tile_plan_free(&tt);
    if (gp.G != kG || !gp.jmajor || (pl->trans_a && !gp.apos_op) || (!gp.bidx && gp.candidates > 0)) {
        set_error("kernel 11 needs the 8-row tables with their position table");
        return LNV_ERR_UNSUPPORTED;
    }
    if (pl->A->nnzb >= INT32_MAX || pl->B->nnzb >= INT32_MAX) {
        set_error("kernel 11: more than 2^31 blocks");
        return LNV_ERR_UNSUPPORTED;
    }
    // 32-column items in the order of kernel 9's 64-column ones (spatial)
    const int64_t ng = gp.n_groups;
    std::vector<int64_t> j_off((size_t)ng + 1);
    std::vector<int2> it64((size_t)gp.n_items);
    LNV_CUDA(cudaMemcpy(j_off.data(), gp.j_off, sizeof(int64_t) * j_off.size(), cudaMemcpyDeviceToHost));
    if (!it64.empty())
        LNV_CUDA(cudaMemcpy(it64.data(), gp.items, sizeof(int2) * it64.size(), cudaMemcpyDeviceToHost));
    std::vector<int32_t> j_list((size_t)j_off[ng]);
    if (!j_list.empty())
        LNV_CUDA(cudaMemcpy(j_list.data(), gp.j_list, sizeof(int32_t) * j_list.size(), cudaMemcpyDeviceToHost));
    std::vector<int2> items;
    std::vector<int32_t> up;
    items.reserve(it64.size() * 2);
    for (const int2 &q : it64) {
        const int64_t nj = j_off[q.x + 1] - j_off[q.x];
        for (int64_t c = q.y; c < std::min<int64_t>(nj, (int64_t)q.y + kTcCols); c += kCols) {
            // J is in ascending atom order: the tile's last column is its largest
            const int64_t last = std::min<int64_t>(nj, c + kCols) - 1;
            if (pl->sym1 && j_list[(size_t)(j_off[q.x] + last)] >= (int64_t)q.x * kG)
                up.push_back((int32_t)items.size());
            items.push_back(make_int2(q.x, (int)c));
        }
    }
    tt.n_items = (int64_t)items.size();
    tt.n_up = (int64_t)up.size();
    cudaError_t e = upload_vec(items, &tt.items);
    if (e == cudaSuccess) e = upload_vec(up, &tt.up);
    int64_t *cnt = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(int64_t) * std::max<int64_t>(1, tt.n_items));
    if (e == cudaSuccess) e = cudaMalloc(&tt.ck_off, sizeof(int64_t) * (size_t)(tt.n_items + 1));
    if (e != cudaSuccess) {
        cudaFree(cnt);
        tile_plan_free(&tt);
        set_error("kernel 11 tile plan: allocation failed (%s)", cudaGetErrorString(e));
        return LNV_ERR_OOM;
    }
    const unsigned nb = (unsigned)((tt.n_items * 32 + 127) / 128);
    lnv_status s = LNV_OK;
    if (tt.n_items > 0) {
        k_tile_lists<<<nb, 128, 0, ctx->stream>>>(tt.n_items, tt.items, gp.k_off, gp.k_list, gp.apos, gp.j_off,
                                                 gp.bidx_off, gp.bidx, pl->B->row_ptr, pl->trans_b, cnt, nullptr,
                                                 nullptr, nullptr, nullptr);
        if (cudaGetLastError() != cudaSuccess) s = LNV_ERR_CUDA;
        count_launch();
    }
    if (s == LNV_OK) s = scan_exclusive(ctx->stream, cnt, tt.n_items, tt.ck_off);
    int64_t listed = 0;
    if (s == LNV_OK && (cudaMemcpyAsync(&listed, tt.ck_off + tt.n_items, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                        ctx->stream) != cudaSuccess ||
                        cudaStreamSynchronize(ctx->stream) != cudaSuccess))
        s = LNV_ERR_CUDA;
    cudaFree(cnt);
    const size_t need = (sizeof(int32_t) * (1 + kG) + sizeof(uint16_t) * kCols) * (size_t)listed;
    if (s == LNV_OK && need > budget_bytes) {
        set_error("kernel 11 tile plan needs %zu bytes, over the %zu budget", need, budget_bytes);
        s = LNV_ERR_UNSUPPORTED;
    }
    if (s == LNV_OK && listed > 0) {
        if (cudaMalloc(&tt.ck_brow, sizeof(int32_t) * (size_t)listed) != cudaSuccess ||
            cudaMalloc(&tt.ck_apos, sizeof(int32_t) * kG * (size_t)listed) != cudaSuccess ||
            cudaMalloc(&tt.ck_tab, sizeof(uint16_t) * kCols * (size_t)listed) != cudaSuccess) {
            set_error("kernel 11 tile plan: allocation of %lld listed k's failed", (long long)listed);
            s = LNV_ERR_OOM;
        } else {
            k_tile_lists<<<nb, 128, 0, ctx->stream>>>(tt.n_items, tt.items, gp.k_off, gp.k_list, gp.apos, gp.j_off,
                                                     gp.bidx_off, gp.bidx, pl->B->row_ptr, pl->trans_b, nullptr,
                                                     tt.ck_off, tt.ck_brow, tt.ck_apos, tt.ck_tab);
            if (cudaGetLastError() != cudaSuccess) s = LNV_ERR_CUDA;
            count_launch();
            if (s == LNV_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) s = LNV_ERR_CUDA;
        }
    }
    if (s != LNV_OK) {
        if (s == LNV_ERR_CUDA) set_error("kernel 11 tile plan: kernel failed");
        tile_plan_free(&tt);
        return s;
    }
    tt.listed = listed;
    tt.src = gp.items;
    tt.bytes = sizeof(int2) * items.size() + sizeof(int32_t) * up.size() + sizeof(int64_t) * (items.size() + 1) + need;
    return LNV_OK;
}

lnv_status launch_umma_tile(lnv_ctx *ctx, const lnv_plan *pl, bool ta, bool tb, bool upper, const void *A,
                            const void *B, void *C, bool onepass)
{
    const GroupPlan &gp = pl->tc;
    const TilePlan &tt = pl->tt;
    if (gp.G != kG || !gp.jmajor || (ta && !gp.apos_op) || !tt.items || tt.src != gp.items) {
        set_error("kernel 11 needs its tile plan");
        return LNV_ERR_UNSUPPORTED;
    }
    // 16-byte aligned value arrays: the block rows are 16-byte copies
    if (((uintptr_t)A | (uintptr_t)B) & 15u) {
        set_error("kernel 11 needs 16-byte aligned value arrays");
        return LNV_ERR_UNSUPPORTED;
    }
    const bool sub = upper && pl->sym1;
    const int64_t n = sub ? tt.n_up : tt.n_items;
    if (n == 0) return LNV_OK;
    auto kern = onepass ? (ta ? (tb ? k_umma_tile<true, true, true> : k_umma_tile<true, false, true>)
                              : (tb ? k_umma_tile<false, true, true> : k_umma_tile<false, false, true>))
                        : (ta ? (tb ? k_umma_tile<true, true, false> : k_umma_tile<true, false, false>)
                              : (tb ? k_umma_tile<false, true, false> : k_umma_tile<false, false, false>));
    LNV_CUDA(ensure_smem((const void *)kern, kSmem));
    kern<<<(unsigned)n, kThreads, kSmem, ctx->stream>>>(
        sub ? tt.up : nullptr, tt.items, tt.ck_off, tt.ck_brow, tt.ck_apos, tt.ck_tab, gp.j_off, gp.j_list, gp.cpos,
        (const float *)A, pl->B->row_ptr, (const float *)B, (float *)C, ctx->dev_status, ctx->wait_ns);
    LNV_LAUNCHED();
    return LNV_OK;
}

}  // namespace lnv
