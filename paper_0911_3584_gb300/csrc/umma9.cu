// Kernel 10: row-group products on the tcgen05 tensor cores for NSF = 9
// (s, p and d functions per atom), FP32 values, FP32-level accuracy from
// split TF32 operands.
//
// The same transposed formulation as kernel 9,
//
//     C_g^T [ (j, y), (m, x) ] = sum_(k, z)  op(B)_kj[z][y]  op(A)_mk[x][z],
//
// with shapes fitted to 9 x 9 blocks:
//   M = 128 rows (j, y): 14 columns j of the group's J (126 rows; 2 zero rows);
//   N = 64 rows (m, x): the G = 7 rows m of a group (63; one zero row);
//   K = (k, z) in stages of 8 k-atoms (72 = 9 MMA steps of K = 8).
// Precision (3xTF32): per K step three MMAs of N = 64,
//     H += A_hi B_hi,   LO += A_hi B_lo,   H += A_lo B_hi,
// with every operand rounded to the nearest TF32 value.  The tensor core
// accumulates in FP32 with truncation, a bias that grows with the length of
// the sum (measured on GB300: -3e-5 relative after K = 3600 positive terms).
// So the large part H alternates between two accumulators by stage: once a
// stage's MMAs have completed, the producer threads add its H into FP32
// registers (round to nearest) and zero it.  LO (about 2^-11 of the result)
// keeps one accumulator over the whole K.
// A (the gathered op(B) rows) is split and written to TMEM by the producer
// threads; B (op(A) of the group) is split and written to shared memory in
// the canonical K-major layout.  One CTA per SM holds 3 x 64 + 2 x 144
// TMEM columns (H twice, LO, and two stages of A hi and lo).
//
// Data path.  A 9 x 9 FP32 block is 324 bytes: block p of a value array
// starts on a 16-byte boundary only when p is a multiple of 4.  Each block is
// copied as 21 aligned 16-byte pieces (cp.async, L2 -> shared memory) from
// the 16-byte boundary at or before its start, into a 336-byte slot, so that
// it sits 4 (p mod 4) bytes into the slot; the last piece reads only up to
// the block's end.  Per stage a CTA copies 8 x 14 blocks of op(B) and 8 x 7
// of op(A); eight lanes copy one block (three 16-byte pieces each), so each
// warp instruction moves four contiguous 128-byte runs.  The block positions
// of a stage are looked up two stages ahead into a shared table; copies run
// one stage ahead of the stage being split and stored.
//
// Every wait is bounded.  The producer warps synchronise with named barriers
// that all of them reach the same number of times whatever happens; after a
// wait runs out (or the MMA warp gives up) they skip the remaining work but
// keep reaching the barriers, the CTA drains its MMAs, frees its TMEM and
// raises the context's device status flag.
#include <algorithm>

#include "lnv_impl.cuh"
#include "tcgen05.cuh"

namespace lnv {
namespace {

constexpr int kN = 9;                 // functions per atom
constexpr int kG = kTc9G;             // rows per group (7: N = 63 of 64)
constexpr int kJT = kTc9Cols;         // columns per tile (14: M = 126 of 128)
constexpr int kKA = 8;                // k-atoms per stage
constexpr int kK = kKA * kN;          // 72 K elements per stage
constexpr int kNS = 2;                // TMEM / B-operand stages
constexpr int kDA = 2;                // copy slots (copies one stage ahead)
constexpr int kNBG = kKA * kJT;       // op(B) blocks per stage (112)
constexpr int kNBA = kKA * kG;        // op(A) blocks per stage (56)
constexpr int kNB = kNBG + kNBA;      // 168
constexpr int kSlot = 336;            // bytes per staged block (21 x 16)
constexpr int kSlotF = kSlot / 4;     // 84 floats
constexpr int kPieces = 21;
constexpr int kNPW = 8;               // producer warps
constexpr int kProd = kNPW * 32;      // producer threads (256)
constexpr int kThreads = kProd + 32;  // + the MMA warp
// shared memory layout (bytes)
constexpr int kBst = 128 * kK * 4;                  // one B-operand stage: 128 rows x 72 K (36,864)
constexpr int kOffRaw = kNS * kBst;                 // 73,728
constexpr int kRaw = kNB * kSlot;                   // one copy slot (56,448)
constexpr int kOffTbl = kOffRaw + kDA * kRaw;       // 186,624: block positions, 3 stages x 168
constexpr int kOffJrow = kOffTbl + 3 * kNB * 4;     // 188,640: first block of the tile's op(B) rows
constexpr int kOffBar = kOffJrow + kJT * 4;         // 188,696
constexpr int kSmem = kOffBar + 8 * (2 * kNS + 1) + 16;
static_assert(kOffBar % 8 == 0, "mbarriers are 8-byte aligned");
static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
static_assert(2 * kSmem > 228 * 1024, "one CTA per SM (it holds all 512 TMEM columns)");
// TMEM columns: H of even stages [0, 64), of odd stages [64, 128), LO
// [128, 192); stage s: A_hi [192 + 144 s, + 72), A_lo + 72
constexpr int kDCols = 192;
constexpr int kLoCol = 128;
constexpr int kACols = 2 * kK;
static_assert(kDCols + kNS * kACols <= 512, "tensor memory");

__device__ __forceinline__ void prod_sync() { asm volatile("barrier.sync 1, %0;" ::"n"(kProd) : "memory"); }

__device__ __forceinline__ void tmem_st4(uint32_t taddr, float a, float b, float c, float d)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}



// op(A)_mk[x][z] (hi, lo) of one stage -> B operand rows n = 9 m + x and 64 + n,
// K chunks K4 = AK0 + 4 c (all of K, AK0 = 0..3 over the four thread
// quarters); the K positions are compile-time here.
template <int AK0, bool TA>
__device__ __forceinline__ void opa_pass(unsigned char *bst, const float *raw, const int32_t *tb, int am, int ax,
                                         bool anv, int an)
{
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const int K4 = AK0 + 4 * c;
        if (K4 < kK / 4) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int K = 4 * K4 + e, kk = K / kN, z = K - kk * kN;
                const int b = kNBG + kk * kG + am;
                v[e] = anv ? raw[b * kSlotF + (tb[b] & 3) + (TA ? kN * z + ax : kN * ax + z)] : 0.f;
            }
            float4 h4, l4;
            tc::split_tf32x2(v[0], v[1], h4.x, h4.y, l4.x, l4.y);
            tc::split_tf32x2(v[2], v[3], h4.z, h4.w, l4.z, l4.w);
            unsigned char *dst = bst + K4 * 2048 + (an >> 3) * 128 + (an & 7) * 16;
            *reinterpret_cast<float4 *>(dst) = h4;
            *reinterpret_cast<float4 *>(dst + 1024) = l4;
        }
    }
}

// op(B)_kj[z][y] (hi, lo) of this lane's row (j, y) and the k-atoms 4 HH ..
// 4 HH + 3 of a stage -> TMEM columns 36 HH .. 36 HH + 35 of A hi and A lo.
// Every store starts on a multiple of its width.
template <int HH, bool TB>
__device__ __forceinline__ void gather_pass(uint32_t acol, const float *raw, const int32_t *tb, int jt, int y, bool rv)
{
    float v[36];
#pragma unroll
    for (int kq = 0; kq < 4; ++kq) {
        const int b = (4 * HH + kq) * kJT + jt;
        const float *blk = raw + b * kSlotF + (rv ? (tb[b] & 3) : 0);
#pragma unroll
        for (int z = 0; z < kN; ++z) v[kN * kq + z] = rv ? blk[TB ? kN * y + z : kN * z + y] : 0.f;
    }
    auto st8 = [&](int c0) {
        float h8[8], l8[8];
#pragma unroll
        for (int e = 0; e < 8; e += 2) tc::split_tf32x2(v[c0 + e], v[c0 + e + 1], h8[e], h8[e + 1], l8[e], l8[e + 1]);
        tc::tmem_st8(acol + (uint32_t)c0, h8);
        tc::tmem_st8(acol + (uint32_t)(kK + c0), l8);
    };
    auto st4 = [&](int c0) {
        float h4[4], l4[4];
        tc::split_tf32x2(v[c0], v[c0 + 1], h4[0], h4[1], l4[0], l4[1]);
        tc::split_tf32x2(v[c0 + 2], v[c0 + 3], h4[2], h4[3], l4[2], l4[3]);
        tmem_st4(acol + (uint32_t)c0, h4[0], h4[1], h4[2], h4[3]);
        tmem_st4(acol + (uint32_t)(kK + c0), l4[0], l4[1], l4[2], l4[3]);
    };
    if (HH == 0) {
        st8(0); st8(8); st8(16); st8(24); st4(32);
    } else {
        st4(0); st8(4); st8(12); st8(20); st8(28);
    }
}

// TA: op(A) = A^T (apos already points at the stored block (k, m)).
// TB: op(B) = B^T (op(B)_kj is the stored block (j, k), row j of B).
template <bool TA, bool TB>
__global__ void __launch_bounds__(kThreads, 1)
k_umma9(const int2 *__restrict__ items, const int64_t *__restrict__ k_off, const int32_t *__restrict__ k_list,
        const int32_t *__restrict__ apos, const int64_t *__restrict__ j_off, const int32_t *__restrict__ j_list,
        const int32_t *__restrict__ cpos, const int64_t *__restrict__ bidx_off, const uint16_t *__restrict__ bidx,
        const float *__restrict__ a_val, const int64_t *__restrict__ b_rp, const float *__restrict__ b_val,
        float *__restrict__ c_val, int *__restrict__ status, unsigned long long wait_ns)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);  // full[NS], empty[NS], done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * kNS + 1);
    volatile int *abort_s = reinterpret_cast<volatile int *>(tslot + 1);
    int32_t *tbl = reinterpret_cast<int32_t *>(smem + kOffTbl);
    int32_t *jrow = reinterpret_cast<int32_t *>(smem + kOffJrow);
    const float *rawf = reinterpret_cast<const float *>(smem + kOffRaw);
    const uint32_t s0 = tc::smem_u32(smem), bar0 = tc::smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(kNS + s); };
    const uint32_t done_bar = bar0 + 8u * (uint32_t)(2 * kNS);

    const int2 item = items[blockIdx.x];
    const int64_t g = item.x, j0 = item.y;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    const int64_t nk_pad = (nk + 3) & ~int64_t(3);
    const int nst = (int)((nk + kKA - 1) / kKA);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = threadIdx.x;

    if (warp == kNPW) {
        tc::tmem_alloc(tc::smem_u32(tslot), 512);
        if (lane == 0) {
            for (int s = 0; s < kNS; ++s) {
                tc::mbar_init(full_bar(s), kNPW);
                tc::mbar_init(empty_bar(s), 1);
            }
            tc::mbar_init(done_bar, 1);
            *abort_s = 0;
            tc::mbar_init_fence();
        }
    } else if (t < kJT) {
        // first stored block of op(B) row j for each column of the tile (TB)
        const int64_t jl = j0 + t;
        jrow[t] = (TB && jl < nj) ? (int32_t)b_rp[j_list[jb + jl]] : -1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tslot;

    if (warp == kNPW) {
        // ---------------------------------------------------------------- MMA issue
        if (lane == 0) {
            // the accumulators start zeroed by the producers: every MMA adds
            constexpr uint32_t id = tc::idesc_tf32(128, 64);
            const uint32_t lo = tm + (uint32_t)kLoCol;
            for (int i = 0; i < nst; ++i) {
                const int s = i & 1;
                if (!tc::mbar_wait(full_bar(s), (uint32_t)(i >> 1) & 1u, abort_s, wait_ns)) break;
                tc::fence_after_sync();
                const uint32_t ahi = tm + (uint32_t)(kDCols + s * kACols), h = tm + (uint32_t)(64 * (i & 1));
#pragma unroll
                for (int q = 0; q < kK / 8; ++q) {
                    // B rows 0..63 hold op(A) hi, rows 64..127 lo
                    const uint32_t b0 = s0 + (uint32_t)(s * kBst + q * 4096);
                    const uint64_t bhi = tc::smem_desc(b0, 2048, 128), blo = tc::smem_desc(b0 + 1024, 2048, 128);
                    tc::mma_tf32_ts(h, ahi + 8u * q, bhi, id, 1u);
                    tc::mma_tf32_ts(lo, ahi + 8u * q, blo, id, 1u);
                    tc::mma_tf32_ts(h, ahi + (uint32_t)kK + 8u * q, bhi, id, 1u);
                }
                tc::commit(empty_bar(s));
            }
            tc::commit(done_bar);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- producers
        // position of block t of stage ii's table (op(B) blocks (kk, jt), then
        // op(A) blocks (kk, m)); -1 when absent
        const uint16_t *bx = bidx + bidx_off[g];
        auto lookup = [&](int ii) -> int32_t {
            if (t >= kNB || ii >= nst) return -1;
            if (t < kNBG) {
                const int kk = t / kJT, jt = t - kk * kJT;
                const int64_t kl = (int64_t)ii * kKA + kk, jl = j0 + jt;
                if (kl >= nk || jl >= nj) return -1;
                const uint16_t e = __ldg(bx + jl * nk_pad + kl);
                if (e == 0xFFFFu) return -1;
                const int32_t r0 = TB ? jrow[jt] : (int32_t)__ldg(b_rp + __ldg(k_list + kb + kl));
                return r0 + (int32_t)e;
            }
            const int u = t - kNBG, kk = u / kG, m = u - kk * kG;
            const int64_t kl = (int64_t)ii * kKA + kk;
            return kl < nk ? __ldg(apos + (kb + kl) * kG + m) : -1;
        };
        // copies of stage ii into slot ii % 2: warp w copies blocks 21 w ..
        // 21 w + 20, eight lanes per block, pieces sub, sub + 8, sub + 16
        const int grp = lane >> 3, sub = lane & 7;
        auto issue = [&](int ii) {
            if (ii < nst) {
                const int32_t *tb = tbl + (ii % 3) * kNB;
                const uint32_t slot = s0 + (uint32_t)(kOffRaw + (ii & 1) * kRaw);
#pragma unroll
                for (int rho = 0; rho < 6; ++rho) {
                    const int bl = 4 * rho + grp;
                    if (bl >= 21) break;
                    const int b = 21 * warp + bl;
                    const int32_t pos = tb[b];
                    const char *base = reinterpret_cast<const char *>(b < kNBG ? b_val : a_val);
                    const int sh = pos & 3;
                    const char *src0 = base + (pos >= 0 ? (int64_t)pos * 324 - 4 * sh : 0);
                    const uint32_t dst = slot + (uint32_t)(b * kSlot);
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        const int c = sub + 8 * c3;
                        if (c < kPieces) {
                            const int bytes = pos < 0 ? 0 : (c == kPieces - 1 ? 4 + 4 * sh : 16);
                            tc::cp_async16(dst + 16u * c, pos < 0 ? base : src0 + 16 * c, bytes);
                        }
                    }
                }
            }
            tc::cp_async_commit();
        };

        // op(A) role: row n = t % 64 of the B operand, K chunks K4 = t / 64 + 4 i
        const int an = t & 63, am = an / kN, ax = an - am * kN;
        const bool anv = an < kG * kN;
        const int ak0 = t >> 6;
        // op(B) role: TMEM lane r = 32 (warp % 4) + lane, k-atoms 4 h .. 4 h + 3
        const int q4 = warp & 3, hh = warp >> 2;
        const int r = 32 * q4 + lane, jt = r / kN, y = r - jt * kN;
        const bool rv = r < kJT * kN;
        const uint32_t lane_base = tm + ((uint32_t)(32 * q4) << 16);

        // FP32 sums of the folded H columns 32 hh .. 32 hh + 31 of this lane's row
        float acc[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = 0.f;
        {
            // zero both H accumulators and LO (columns 32 hh .. 32 hh + 31 of each)
            const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int part = 0; part < 3; ++part)
#pragma unroll
                for (int c8 = 0; c8 < 4; ++c8) tc::tmem_st8(lane_base + (uint32_t)(64 * part + 32 * hh + 8 * c8), z8);
            tc::tmem_st_wait();
        }


        auto consume = [&](int i) {
            const int s = i & 1, a = i & 1;
            const int32_t *tb = tbl + (i % 3) * kNB;
            bool seen = true;
            if (i >= kNS) seen = tc::mbar_wait(empty_bar(s), (uint32_t)((i >> 1) - 1) & 1u, abort_s, wait_ns);
            if (!__all_sync(0xffffffffu, seen)) *abort_s = 1;
            tc::cp_async_wait<1>();
            prod_sync();  // every copy of stage i has landed
            if (*abort_s) return;
            tc::fence_after_sync();
            if (i >= kNS) {
                // stage i - 2's MMAs have completed: fold its H (columns 32 hh ..
                // 32 hh + 31 of this warp's lanes) into acc and zero it for stage i
                const uint32_t hcol = lane_base + (uint32_t)(64 * (i & 1) + 32 * hh);
#pragma unroll
                for (int c8 = 0; c8 < 4; ++c8) {
                    float d[8];
                    tc::tmem_ld8(hcol + 8u * c8, d);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[8 * c8 + e] += d[e];
                }
                const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int c8 = 0; c8 < 4; ++c8) tc::tmem_st8(hcol + 8u * c8, z8);
            }
            const float *raw = rawf + a * (kRaw / 4);
            unsigned char *bst = smem + s * kBst;
            switch (ak0) {
            case 0: opa_pass<0, TA>(bst, raw, tb, am, ax, anv, an); break;
            case 1: opa_pass<1, TA>(bst, raw, tb, am, ax, anv, an); break;
            case 2: opa_pass<2, TA>(bst, raw, tb, am, ax, anv, an); break;
            default: opa_pass<3, TA>(bst, raw, tb, am, ax, anv, an); break;
            }
            tc::fence_async_smem();
            const uint32_t acol = lane_base + (uint32_t)(kDCols + s * kACols + 36 * hh);
            if (hh == 0) gather_pass<0, TB>(acol, raw, tb, jt, y, rv);
            else gather_pass<1, TB>(acol, raw, tb, jt, y, rv);
            tc::tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full_bar(s));
        };

        // prologue: positions of stages 0 and 1, copies of stage 0
        {
            const int32_t p0 = lookup(0), p1 = lookup(1);
            if (t < kNB) {
                tbl[t] = p0;
                tbl[kNB + t] = p1;
            }
        }
        prod_sync();
        issue(0);
        for (int i = 0; i < nst; ++i) {
            prod_sync();  // slot (i + 1) % 2 is free, table (i + 1) % 3 is written
            issue(i + 1);
            const int32_t p2 = lookup(i + 2);
            consume(i);
            if (t < kNB && i + 2 < nst) tbl[((i + 2) % 3) * kNB + t] = p2;
        }
        tc::cp_async_wait<0>();
        const bool ok = !*abort_s;
        if (!ok && t == 0) atomicExch(status, 1);

        // ---------------------------------------------------------------- epilogue
        const bool drained = __all_sync(0xffffffffu, tc::mbar_wait_for(done_bar, 0u, 2 * wait_ns));
        if (!drained && lane == 0) atomicExch(status, 1);
        tc::fence_after_sync();
        if (ok && drained) {
            // this warp: TMEM lanes of quarter q4, columns n = 32 hh .. 32 hh + 31
            const int64_t jl = j0 + jt;
            const bool cv = rv && jl < nj;
            auto epi = [&](auto hc) {
                constexpr int H = decltype(hc)::value;
                constexpr int M0 = (32 * H) / kN, M1 = std::min(kG - 1, (32 * H + 31) / kN);
                int32_t cp[M1 - M0 + 1];
#pragma unroll
                for (int m = M0; m <= M1; ++m) cp[m - M0] = cv ? __ldg(cpos + (jb + jl) * kG + m) : -1;
#pragma unroll
                for (int c8 = 0; c8 < 4; ++c8) {
                    // the folded sum plus the last two stages' H and LO
                    float ha[8], hb[8], dl[8];
                    tc::tmem_ld8(lane_base + (uint32_t)(32 * H + 8 * c8), ha);
                    tc::tmem_ld8(lane_base + (uint32_t)(64 + 32 * H + 8 * c8), hb);
                    tc::tmem_ld8(lane_base + (uint32_t)(kLoCol + 32 * H + 8 * c8), dl);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int n = 32 * H + 8 * c8 + e;
                        if (n < kG * kN) {
                            const int m = n / kN, x = n - m * kN;
                            const int32_t p = cp[m - M0];
                            const float v = ((acc[8 * c8 + e] + ha[e]) + hb[e]) + dl[e];
                            if (p >= 0) c_val[(int64_t)p * (kN * kN) + kN * x + y] = v;
                        }
                    }
                }
            };
            if (hh == 0) epi(std::integral_constant<int, 0>{});
            else epi(std::integral_constant<int, 1>{});
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == kNPW) tc::tmem_dealloc(tm, 512);
}

}  // namespace

lnv_status launch_umma9(lnv_ctx *ctx, const lnv_plan *pl, bool ta, bool tb, const void *A, const void *B, void *C)
{
    const GroupPlan &gp = pl->tc;
    if (gp.G != kG || !gp.jmajor || (ta && !gp.apos_op)) {
        set_error("kernel 10 needs its 7-row group tables");
        return LNV_ERR_UNSUPPORTED;
    }
    if (gp.n_items == 0) return LNV_OK;
    if (!gp.bidx && gp.candidates > 0) {
        set_error("row-group plan lacks the position table");
        return LNV_ERR_UNSUPPORTED;
    }
    // 16-byte aligned value arrays (the block copies are 16-byte pieces), and
    // block indices that fit 32 bits
    if (((uintptr_t)A | (uintptr_t)B) & 15u) {
        set_error("kernel 10 needs 16-byte aligned value arrays");
        return LNV_ERR_UNSUPPORTED;
    }
    if (pl->A->nnzb >= INT32_MAX || pl->B->nnzb >= INT32_MAX) {
        set_error("kernel 10: more than 2^31 blocks");
        return LNV_ERR_UNSUPPORTED;
    }
    auto kern = ta ? (tb ? k_umma9<true, true> : k_umma9<true, false>)
                   : (tb ? k_umma9<false, true> : k_umma9<false, false>);
    LNV_CUDA(ensure_smem((const void *)kern, kSmem));
    kern<<<(unsigned)gp.n_items, kThreads, kSmem, ctx->stream>>>(
        gp.items, gp.k_off, gp.k_list, gp.apos, gp.j_off, gp.j_list, gp.cpos, gp.bidx_off, gp.bidx,
        (const float *)A, pl->B->row_ptr, (const float *)B, (float *)C, ctx->dev_status, ctx->wait_ns);
    LNV_LAUNCHED();
    return LNV_OK;
}

}  // namespace lnv
