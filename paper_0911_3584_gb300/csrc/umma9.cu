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
//   K = (k, z) in stages of 4 k-atoms (36, padded with zeros to 5 MMA steps
//   of K = 8).
// Precision (3xTF32): per K step three MMAs of N = 64 into three
// accumulators, each product issued by its own warp,
//     H += A_hi B_hi,   L1 += A_lo B_hi,   L2 += A_hi B_lo,
// with every operand rounded to the nearest TF32 value.  The tensor core
// accumulates in FP32 with truncation, a bias that grows with the length of
// the sum (measured on GB300: -3e-5 relative after K = 3600 positive terms).
// So the large part H alternates between two accumulators every two stages
// (72 K): once those stages' MMAs have completed, the compute threads add
// that H into FP32 registers (round to nearest) and zero it.  L1 and L2 (about 2^-11 of the
// result) keep one accumulator each over the whole K.
// A (the gathered op(B) rows) is split and written to TMEM by the producer
// threads; B (op(A) of the group) is split and written to shared memory in
// the canonical K-major layout.  One CTA per SM holds 4 x 64 + 2 x 80
// TMEM columns (H twice, L1, L2, and two stages of A hi and lo).
//
// Data path.  A 9 x 9 FP32 block is 324 bytes: block p of a value array
// starts on a 16-byte boundary only when p is a multiple of 4.  Per stage a
// CTA stages 4 x 14 blocks of op(B) (rows j of the tile) and 4 x 7 of op(A)
// (rows m of the group).  Along such a row the stored blocks of consecutive
// k mostly follow one another in memory (B's row j and A's row m are sorted
// by k), so each run of them is one bulk copy (cp.async.bulk, the TMA
// engine) of the 16-byte aligned span that holds it, a few per row instead
// of one per block.
//
// Warp roles.  Four copy warps load the blocks' positions two stages ahead
// (raw words in registers, decoded when used), write each block's
// shared-memory offset to the slot's table and issue the copies; the slot's
// "landed" barrier completes when every copy has arrived (bulk copies count
// their bytes on it, the rare tail pieces arrive through
// cp.async.mbarrier.arrive).  kNQ compute warps per TMEM lane quarter wait
// for it, fold, split op(A) into the B-operand stage and split and store
// their rows of op(B) (warp (q, h): rows 32 q .. 32 q + 31, k-atoms h kKW ..
// h kKW + kKW - 1) into TMEM, then release the slot.  Three warps issue the
// MMAs, one per accumulator.  kDA copy slots and two operand stages: copies
// run up to kDA - 1 stages ahead of the stage being split.
//
// Measured on GB300 (Z = L T^T, 4096 atoms, NSF = 9): with the 21 rows of a
// stage spread over four copy warps (two: 20% slower; six: no faster), the
// copy warps' work and the compute warps' work take about 0.9 us per stage
// each; 16-byte cp.async pieces issued by the compute warps themselves, or by
// six copy warps, and one bulk copy per block were each slower.
//
// Every wait is bounded (mbarriers only, no named barriers): after a wait
// runs out, the CTA-wide abort flag makes every other wait give up, the CTA
// drains its MMAs and copies, frees its TMEM and raises the context's device
// status flag.
#include <algorithm>

#include "lnv_impl.cuh"
#include "tcgen05.cuh"

#ifndef LNV_TC9_NQ
#define LNV_TC9_NQ 2
#endif

namespace lnv {
namespace {

constexpr int kN = 9;                 // functions per atom
constexpr int kG = kTc9G;             // rows per group (7: N = 63 of 64)
constexpr int kJT = kTc9Cols;         // columns per tile (14: M = 126 of 128)
#ifndef LNV_TC9_DA
#define LNV_TC9_DA 4
#endif
constexpr int kKA = 4;                // k-atoms per stage
constexpr int kK = kKA * kN;          // 36 K elements per stage
constexpr int kKP = 40;               // K of a stage padded to whole MMA steps (5 x 8)
constexpr int kNS = 2;                // TMEM / B-operand stages
constexpr int kDA = LNV_TC9_DA;       // copy slots (copies kDA - 1 stages ahead)
constexpr int kNBG = kKA * kJT;       // op(B) blocks per stage (56)
constexpr int kNBA = kKA * kG;        // op(A) blocks per stage (28)
constexpr int kNB = kNBG + kNBA;      // 84
constexpr int kRowB = 1408;           // bytes per staged row of 4 blocks (4 x 324 + room for 4 aligned runs)
constexpr int kRowsG = kJT;           // op(B) rows (columns j) per stage
constexpr int kRowsA = kG;            // op(A) rows (rows m) per stage
constexpr int kNQ = LNV_TC9_NQ;       // compute warps per TMEM lane quarter
constexpr int kNPW = 4 * kNQ;         // compute warps (split, TMEM and B-operand stores)
constexpr int kProd = kNPW * 32;      // compute threads
#ifndef LNV_TC9_CP
#define LNV_TC9_CP 4
#endif
constexpr int kCP = LNV_TC9_CP;       // copy warps (block positions, bulk copies)
constexpr int kCT = kCP * 32;         // copy threads
constexpr int kMW = 3;                // MMA warps: hi*hi, lo*hi, hi*lo
constexpr int kThreads = kProd + kCT + 32 * kMW;
constexpr int kKW = kKA / kNQ;        // k-atoms of a stage per producer warp
constexpr int kCW = kKW * kN;         // their A columns
constexpr int kHW = 64 / kNQ;         // H columns a warp folds and writes out
constexpr int kAQ = kProd / 64;       // op(A) chunk classes (K4 mod kAQ)
static_assert(kKA % kNQ == 0 && 64 % kNQ == 0 && kHW % 8 == 0, "producer split");
// shared memory layout (bytes)
constexpr int kBst = 128 * kKP * 4;                 // one B-operand stage: 128 rows x 40 K (20,480)
constexpr int kOffRaw = kNS * kBst;                 // 40,960
constexpr int kRaw = (kRowsG + kRowsA) * kRowB;     // one copy slot (29,568)
constexpr int kOffTbl = kOffRaw + kDA * kRaw;       // each block's float offset in shared memory
constexpr int kOffZero = kOffTbl + kDA * kNB * 4;   // 84 zero floats (absent blocks)
constexpr int kOffJrow = kOffZero + 336;            // first block of the tile's op(B) rows
constexpr int kOffBar = kOffJrow + kJT * 4;
// mbarriers: full[NS], empty[NS], landed[DA], slotfree[DA], done
constexpr int kNBars = 2 * kNS + 2 * kDA + 1;
constexpr int kSmem = kOffBar + 8 * kNBars + 16;
static_assert(kOffBar % 8 == 0 && kOffZero % 16 == 0 && kRowB % 16 == 0, "alignment");
static_assert(kKA * 324 + kKA * 27 <= kRowB, "a row's runs fit its region");
static_assert(kKP % 8 == 0 && kKP >= kK && kKP - kK <= 4, "padded stage K: the pad is one zero K chunk");
static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
static_assert(2 * kSmem > 228 * 1024, "one CTA per SM (it holds all 512 TMEM columns)");
// TMEM columns: H (hi*hi) of stages 4q, 4q + 1 [0, 64), of 4q + 2, 4q + 3 [64, 128),
// L1 (lo*hi) [128, 192), L2 (hi*lo) [192, 256); stage s: A_hi [256 + 80 s,
// + 40), A_lo + 40 (columns 36..39 of each stay zero)
constexpr int kDCols = 256;
constexpr int kL1Col = 128, kL2Col = 192;
constexpr int kACols = 2 * kKP;
static_assert(kDCols + kNS * kACols <= 512, "tensor memory");
static_assert(kDCols % 8 == 0 && kACols % 8 == 0, "stage columns start on multiples of 8");

// tcgen05.st of W = 1, 2, 4 columns (32 lanes x 32 bits)
template <int W>
__device__ __forceinline__ void tmem_stw(uint32_t taddr, const float *v)
{
    if constexpr (W == 1) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "f"(v[0]) : "memory");
    } else if constexpr (W == 2) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "f"(v[0]), "f"(v[1])
                     : "memory");
    } else {
        static_assert(W == 4, "width");
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "f"(v[0]),
                     "f"(v[1]), "f"(v[2]), "f"(v[3])
                     : "memory");
    }
}

// Store columns [C, E) of the values v (v[0] is column C0) as pieces of 8, 4,
// 2 or 1 columns, each starting on a multiple of its width.
template <int C0, int C, int E>
__device__ __forceinline__ void tmem_st_run(uint32_t base, const float *v)
{
    if constexpr (C < E) {
        constexpr int W = (C % 8 == 0 && C + 8 <= E) ? 8 : (C % 4 == 0 && C + 4 <= E) ? 4 : (C % 2 == 0 && C + 2 <= E) ? 2 : 1;
        if constexpr (W == 8) {
            const float(&w)[8] = *reinterpret_cast<const float(*)[8]>(v + (C - C0));
            tc::tmem_st8(base + (uint32_t)C, w);
        } else {
            tmem_stw<W>(base + (uint32_t)C, v + (C - C0));
        }
        tmem_st_run<C0, C + W, E>(base, v);
    }
}

// op(A)_mk[x][z] (hi, lo) of one stage -> B operand rows n = 9 m + x and 64 + n
// (block b of the stage at float offset tb[b] of shared memory),
// K chunks K4 = AK0 + kAQ c (AK0 = 0 .. kAQ - 1 over the thread classes); the
// K positions are compile-time here.
template <int AK0, bool TA>
__device__ __forceinline__ void opa_pass(unsigned char *bst, const float *smf, const int32_t *tb, int am, int ax,
                                         bool anv, int an)
{
#pragma unroll
    for (int c = 0; c < (kK / 4 + kAQ - 1) / kAQ; ++c) {
        const int K4 = AK0 + kAQ * c;
        if (K4 < kK / 4) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int K = 4 * K4 + e, kk = K / kN, z = K - kk * kN;
                const int b = kNBG + kk * kG + am;
                v[e] = anv ? smf[tb[b] + (TA ? kN * z + ax : kN * ax + z)] : 0.f;
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

// op(B)_kj[z][y] (hi, lo) of this lane's row (j, y) and the k-atoms HQ kKW ..
// HQ kKW + kKW - 1 of a stage -> TMEM columns HQ kCW .. HQ kCW + kCW - 1 of A
// hi (at abase) and A lo (abase + 40).
template <int HQ, bool TB>
__device__ __forceinline__ void gather_pass(uint32_t abase, const float *smf, const int32_t *tb, int jt, int y, bool rv)
{
    float v[kCW], h[kCW], l[kCW];
#pragma unroll
    for (int kq = 0; kq < kKW; ++kq) {
        const int b = (HQ * kKW + kq) * kJT + jt;
        const float *blk = smf + (rv ? tb[b] : kOffZero / 4);
#pragma unroll
        for (int z = 0; z < kN; ++z) v[kN * kq + z] = rv ? blk[TB ? kN * y + z : kN * z + y] : 0.f;
    }
#pragma unroll
    for (int e = 0; e + 1 < kCW; e += 2) tc::split_tf32x2(v[e], v[e + 1], h[e], h[e + 1], l[e], l[e + 1]);
    if constexpr (kCW % 2) tc::split_tf32(v[kCW - 1], h[kCW - 1], l[kCW - 1]);
    tmem_st_run<HQ * kCW, HQ * kCW, HQ * kCW + kCW>(abase, h);
    tmem_st_run<HQ * kCW, HQ * kCW, HQ * kCW + kCW>(abase + (uint32_t)kKP, l);
}

// TA: op(A) = A^T (apos already points at the stored block (k, m)).
// TB: op(B) = B^T (op(B)_kj is the stored block (j, k), row j of B).
template <bool TA, bool TB>
__global__ void __launch_bounds__(kThreads, 1)
k_umma9(const int2 *__restrict__ items, const int64_t *__restrict__ k_off, const int32_t *__restrict__ k_list,
        const int32_t *__restrict__ apos, const int64_t *__restrict__ j_off, const int32_t *__restrict__ j_list,
        const int32_t *__restrict__ cpos, const int64_t *__restrict__ bidx_off, const uint16_t *__restrict__ bidx,
        const float *__restrict__ a_val, const int64_t *__restrict__ b_rp, const float *__restrict__ b_val,
        float *__restrict__ c_val, int32_t a_last, int32_t b_last,
        int *__restrict__ status, unsigned long long wait_ns)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + kNBars);
    volatile int *abort_s = reinterpret_cast<volatile int *>(tslot + 1);
    int32_t *tbl = reinterpret_cast<int32_t *>(smem + kOffTbl);
    int32_t *jrow = reinterpret_cast<int32_t *>(smem + kOffJrow);
    const uint32_t s0 = tc::smem_u32(smem), bar0 = tc::smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(kNS + s); };
    auto landed_bar = [&](int a) { return bar0 + 8u * (uint32_t)(2 * kNS + a); };
    auto free_bar = [&](int a) { return bar0 + 8u * (uint32_t)(2 * kNS + kDA + a); };
    const uint32_t done_bar = bar0 + 8u * (uint32_t)(2 * kNS + 2 * kDA);

    const int2 item = items[blockIdx.x];
    const int64_t g = item.x, j0 = item.y;
    const int64_t kb = k_off[g], nk = k_off[g + 1] - kb;
    const int64_t jb = j_off[g], nj = j_off[g + 1] - jb;
    const int64_t nk_pad = (nk + 3) & ~int64_t(3);
    const int nst = (int)((nk + kKA - 1) / kKA);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = threadIdx.x;
    constexpr int kMmaWarp = kNPW + kCP;  // the first MMA warp (it also allocates TMEM)

    if (warp == kMmaWarp) {
        tc::tmem_alloc(tc::smem_u32(tslot), 512);
        if (lane == 0) {
            for (int s = 0; s < kNS; ++s) {
                tc::mbar_init(full_bar(s), kNPW);
                tc::mbar_init(empty_bar(s), kMW);
            }
            for (int a = 0; a < kDA; ++a) {
                // each copy thread arrives twice: once for its table entries,
                // once (through cp.async) when its copies have landed
                tc::mbar_init(landed_bar(a), 2 * kCT);
                tc::mbar_init(free_bar(a), kNPW);
            }
            tc::mbar_init(done_bar, kMW);
            *abort_s = 0;
            tc::mbar_init_fence();
        }
    } else if (t < kJT) {
        // first stored block of op(B) row j for each column of the tile (TB)
        const int64_t jl = j0 + t;
        jrow[t] = (TB && jl < nj) ? (int32_t)b_rp[j_list[jb + jl]] : -1;
    } else if (t >= 32 && t < 32 + 84) {
        reinterpret_cast<float *>(smem + kOffZero)[t - 32] = 0.f;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tslot;

    if (warp >= kMmaWarp) {
        // ---------------------------------------------------------------- MMA issue
        // warp kMmaWarp + 0: H[i % 2] += A_hi B_hi; + 1: L1 += A_lo B_hi;
        // + 2: L2 += A_hi B_lo.  The accumulators start zeroed by the compute
        // warps: every MMA adds.
        if (lane == 0) {
            const int role = warp - kMmaWarp;
            constexpr uint32_t id = tc::idesc_tf32(128, 64);
            for (int i = 0; i < nst; ++i) {
                const int s = i & 1;
                if (!tc::mbar_wait(full_bar(s), (uint32_t)(i >> 1) & 1u, abort_s, wait_ns)) break;
                tc::fence_after_sync();
                const uint32_t a0 = tm + (uint32_t)(kDCols + s * kACols + (role == 1 ? kKP : 0));
                const uint32_t d = tm + (uint32_t)(role == 0 ? 64 * ((i >> 1) & 1) : role == 1 ? kL1Col : kL2Col);
                // B rows 0..63 hold op(A) hi, rows 64..127 lo
                const uint32_t b0 = s0 + (uint32_t)(s * kBst + (role == 2 ? 1024 : 0));
#pragma unroll
                for (int q = 0; q < kKP / 8; ++q)
                    tc::mma_tf32_ts(d, a0 + 8u * q, tc::smem_desc(b0 + (uint32_t)(q * 4096), 2048, 128), id, 1u);
                tc::commit(empty_bar(s));
            }
            tc::commit(done_bar);
        }
        __syncwarp();
    } else if (warp >= kNPW) {
        // ---------------------------------------------------------------- copy warps
        // Per stage 21 rows of kKA blocks: op(B) rows jt (blocks (kk, jt)) and
        // op(A) rows m (blocks (kk, m)), one lane each: row gr (op(B) rows
        // 0..13, then op(A) rows 14..20) goes to copy warp gr % kCP, lane
        // gr / kCP.  The present blocks of a row whose positions follow one
        // another form a run, copied as one bulk copy (cp.async.bulk, the TMA
        // engine) of the aligned span that holds it; each block's table entry
        // is the float offset of its data in shared memory (the zero block
        // when absent).  A run ending with an array's last block is cut at the
        // last 16-byte boundary and its tail copied by a cp.async piece of the
        // remaining bytes, so nothing past the array is read.
        static_assert((kRowsG + kRowsA + kCP - 1) / kCP <= 32, "copy split");
        const uint16_t *bx = bidx + bidx_off[g];
        const int cw = warp - kNPW;
        const int gr = lane * kCP + cw;
        const bool brow = gr < kRowsG, arow = gr >= kRowsG && gr < kRowsG + kRowsA;
        const int rid = brow ? gr : gr - kRowsG;  // jt of an op(B) row, m of an op(A) row
        const bool has_row = brow || arow;
        const char *vbase = reinterpret_cast<const char *>(brow ? b_val : a_val);
        const int32_t last = brow ? b_last : a_last;
        // The loads behind the positions of this lane's row in stage ii are
        // issued two stages ahead into raw words (a load's value is not used
        // until then, so its latency is hidden); positions() decodes them.
        struct Raw {
            uint32_t w[kKA];  // TB op(B) row: two words of 16-bit offsets; op(A): positions
        };
        auto fetch = [&](int ii, Raw &r) {
#pragma unroll
            for (int kk = 0; kk < kKA; ++kk) r.w[kk] = 0xFFFFFFFFu;
            if (!has_row || ii >= nst) return;
            const int64_t k0 = (int64_t)ii * kKA;
            if (brow) {
                const int64_t jl = j0 + rid;
                if (jl >= nj) return;
                if (TB) {
                    // four consecutive 16-bit offsets: one aligned 8-byte load
                    // (rows hold nk_pad, a multiple of 4, entries)
                    static_assert(kKA == 4, "one 8-byte load per stage");
                    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(bx + jl * nk_pad + k0));
                    r.w[0] = v.x;
                    r.w[1] = v.y;
                } else {
#pragma unroll
                    for (int kk = 0; kk < kKA; ++kk) {
                        const int64_t kl = k0 + kk;
                        if (kl < nk) {
                            const uint16_t e = __ldg(bx + jl * nk_pad + kl);
                            if (e != 0xFFFFu) r.w[kk] = (uint32_t)(__ldg(b_rp + __ldg(k_list + kb + kl)) + e);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int kk = 0; kk < kKA; ++kk)
                    if (k0 + kk < nk) r.w[kk] = (uint32_t)__ldg(apos + (kb + k0 + kk) * kG + rid);
            }
        };
        auto positions = [&](int ii, const Raw &r, int32_t (&p)[kKA]) {
            const int64_t k0 = (int64_t)ii * kKA;
            if (brow && TB) {
                const int32_t r0 = jrow[rid];
                const uint32_t e[4] = {r.w[0] & 0xFFFFu, r.w[0] >> 16, r.w[1] & 0xFFFFu, r.w[1] >> 16};
#pragma unroll
                for (int kk = 0; kk < kKA; ++kk)
                    p[kk] = (k0 + kk < nk && e[kk] != 0xFFFFu && r0 >= 0) ? r0 + (int32_t)e[kk] : -1;
            } else {
#pragma unroll
                for (int kk = 0; kk < kKA; ++kk) p[kk] = (int32_t)r.w[kk];  // -1 when absent
            }
        };
        // copies of stage i from the positions p (looked up two stages earlier)
        auto stage = [&](int i, const Raw &raw) -> bool {
            const int a = i % kDA;
            if (i >= kDA && !tc::mbar_wait(free_bar(a), (uint32_t)(i / kDA - 1) & 1u, abort_s, wait_ns)) return false;
            int32_t pn[kKA];
            positions(i, raw, pn);
            int32_t *tb = tbl + a * kNB;
            const uint32_t lb = landed_bar(a);
            if (has_row) {
                const int row = brow ? rid : kRowsG + rid;
                uint32_t cur = s0 + (uint32_t)(kOffRaw + a * kRaw + row * kRowB);
#pragma unroll
                for (int kk = 0; kk < kKA; ++kk) {
                    const int b = brow ? kk * kJT + rid : kNBG + kk * kG + rid;
                    // a run starts at kk when this block is present and its
                    // predecessor is absent or not adjacent in memory
                    if (pn[kk] < 0) {
                        tb[b] = kOffZero / 4;
                        continue;
                    }
                    if (kk > 0 && pn[kk - 1] >= 0 && pn[kk] == pn[kk - 1] + 1) continue;
                    int n = 1;
#pragma unroll
                    for (int q = kk + 1; q < kKA; ++q)
                        if (n == q - kk && pn[q] == pn[kk] + n) ++n;
                    const int32_t p0 = pn[kk];
                    const int sh = p0 & 3;
                    const uint32_t span = (uint32_t)(324 * n + 4 * sh);
                    const char *src = vbase + (int64_t)p0 * 324 - 4 * sh;
                    const int fo = (int)((cur - s0) >> 2) + sh;
#pragma unroll
                    for (int q = kk; q < kKA; ++q)
                        if (q - kk < n) {
                            const int bq = brow ? q * kJT + rid : kNBG + q * kG + rid;
                            tb[bq] = fo + 81 * (q - kk);
                        }
                    const bool tail = p0 + n - 1 == last && (span & 15u) != 0;
                    const uint32_t bulk = tail ? (span & ~15u) : ((span + 15u) & ~15u);
                    if (bulk > 0) {
                        tc::mbar_expect_tx(lb, bulk);
                        tc::bulk_g2s(cur, src, bulk, lb);
                    }
                    if (tail) tc::cp_async16(cur + bulk, src + bulk, (int)(span & 15u));
                    cur += (span + 15u) & ~15u;
                }
            }
            tc::mbar_arrive(lb);           // the table entries (release)
            tc::cp_async_mbar_arrive(lb);  // this thread's tail pieces, once they land
            return true;
        };
        Raw ra, rb;
        fetch(0, ra);
        fetch(1, rb);
        int issued = 0;
        for (int i = 0; i < nst; i += 2) {
            if (!stage(i, ra)) break;
            issued = i + 1;
            fetch(i + 2, ra);
            if (i + 1 >= nst) break;
            if (!stage(i + 1, rb)) break;
            issued = i + 2;
            fetch(i + 3, rb);
        }
        // no copy may still be in flight when the CTA exits: wait (bounded) for
        // the slots of the last kDA stages to be complete
        for (int i = max(0, issued - kDA); i < issued; ++i)
            tc::mbar_wait_for(landed_bar(i % kDA), (uint32_t)(i / kDA) & 1u, wait_ns);
        tc::cp_async_wait<0>();
    } else {
        // ---------------------------------------------------------------- compute warps
        // op(A) role: row n = t % 64 of the B operand, K chunks K4 = t / 64 + kAQ i
        const int an = t & 63, am = an / kN, ax = an - am * kN;
        const bool anv = an < kG * kN;
        const int ak0 = t >> 6;
        // op(B) role: TMEM lane r = 32 (warp % 4) + lane, k-atoms hq kKW ..
        const int q4 = warp & 3, hq = warp >> 2;
        const int r = 32 * q4 + lane, jt = r / kN, y = r - jt * kN;
        const bool rv = r < kJT * kN;
        const uint32_t lane_base = tm + ((uint32_t)(32 * q4) << 16);

        // FP32 sums of the folded H columns hq kHW .. hq kHW + kHW - 1 of this lane's row
        float acc[kHW];
#pragma unroll
        for (int c = 0; c < kHW; ++c) acc[c] = 0.f;
        {
            // zero both H accumulators, L1 and L2 (this warp's kHW columns of each)
            const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int part = 0; part < 4; ++part)
#pragma unroll
                for (int c8 = 0; c8 < kHW / 8; ++c8)
                    tc::tmem_st8(lane_base + (uint32_t)(64 * part + kHW * hq + 8 * c8), z8);
            if (hq == 0) {
                // the pad K columns 36..39 of A hi and lo in both stages
#pragma unroll
                for (int st = 0; st < kNS; ++st)
#pragma unroll
                    for (int part = 0; part < 2; ++part)
                        tmem_stw<4>(lane_base + (uint32_t)(kDCols + st * kACols + part * kKP + kK), z8);
            }
            tc::tmem_st_wait();
            // the pad K chunk (K 36..39) of every B-operand row in both stages
            for (int q = t; q < kNS * 128; q += kProd)
                *reinterpret_cast<float4 *>(smem + (q >> 7) * kBst + (kK / 4) * 2048 + (q & 127) * 16) =
                    make_float4(0.f, 0.f, 0.f, 0.f);
        }

        for (int i = 0; i < nst; ++i) {
            const int s = i & 1, a = i % kDA;
            // the stage's blocks have landed; stage i - 2's MMAs are done
            bool go = tc::mbar_wait(landed_bar(a), (uint32_t)(i / kDA) & 1u, abort_s, wait_ns);
            if (go && i >= kNS) go = tc::mbar_wait(empty_bar(s), (uint32_t)((i >> 1) - 1) & 1u, abort_s, wait_ns);
            if (!__all_sync(0xffffffffu, go)) {
                *abort_s = 1;
                break;
            }
            tc::fence_after_sync();
            const int32_t *tb = tbl + a * kNB;
            if (i >= 4 && (i & 1) == 0) {
                // H alternates every two stages: fold the one stages i - 4 and
                // i - 3 summed into (both done: stage i - 2's MMAs are) into
                // acc, and zero it for stages i and i + 1
                const uint32_t hcol = lane_base + (uint32_t)(64 * ((i >> 1) & 1) + kHW * hq);
#pragma unroll
                for (int c8 = 0; c8 < kHW / 8; ++c8) {
                    float d[8];
                    tc::tmem_ld8(hcol + 8u * c8, d);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[8 * c8 + e] += d[e];
                }
                const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int c8 = 0; c8 < kHW / 8; ++c8) tc::tmem_st8(hcol + 8u * c8, z8);
            }
            const float *smf = reinterpret_cast<const float *>(smem);
            unsigned char *bst = smem + s * kBst;
            switch (ak0) {
            case 0: opa_pass<0, TA>(bst, smf, tb, am, ax, anv, an); break;
            case 1: opa_pass<1 % kAQ, TA>(bst, smf, tb, am, ax, anv, an); break;
            case 2: opa_pass<2 % kAQ, TA>(bst, smf, tb, am, ax, anv, an); break;
            case 3: opa_pass<3 % kAQ, TA>(bst, smf, tb, am, ax, anv, an); break;
            case 4: opa_pass<4 % kAQ, TA>(bst, smf, tb, am, ax, anv, an); break;
            case 5: opa_pass<5 % kAQ, TA>(bst, smf, tb, am, ax, anv, an); break;
            case 6: opa_pass<6 % kAQ, TA>(bst, smf, tb, am, ax, anv, an); break;
            default: opa_pass<7 % kAQ, TA>(bst, smf, tb, am, ax, anv, an); break;
            }
            tc::fence_async_smem();
            const uint32_t abase = lane_base + (uint32_t)(kDCols + s * kACols);
            switch (hq) {
            case 0: gather_pass<0, TB>(abase, smf, tb, jt, y, rv); break;
            case 1: gather_pass<1 % kNQ, TB>(abase, smf, tb, jt, y, rv); break;
            case 2: gather_pass<2 % kNQ, TB>(abase, smf, tb, jt, y, rv); break;
            default: gather_pass<3 % kNQ, TB>(abase, smf, tb, jt, y, rv); break;
            }
            tc::tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(full_bar(s));
                tc::mbar_arrive(free_bar(a));
            }
        }
        const bool ok = !*abort_s;
        if (!ok && t == 0) atomicExch(status, 1);

        // ---------------------------------------------------------------- epilogue
        const bool drained = __all_sync(0xffffffffu, tc::mbar_wait_for(done_bar, 0u, 2 * wait_ns));
        if (!drained && lane == 0) atomicExch(status, 1);
        tc::fence_after_sync();
        if (ok && drained) {
            // this warp: TMEM lanes of quarter q4, columns n = hq kHW .. hq kHW + kHW - 1
            const int64_t jl = j0 + jt;
            const bool cv = rv && jl < nj;
            auto epi = [&](auto hc) {
                constexpr int HQ = decltype(hc)::value;
                constexpr int N0 = kHW * HQ;
                constexpr int M0 = N0 / kN, M1 = std::min(kG - 1, (N0 + kHW - 1) / kN);
                int32_t cp[M1 - M0 + 1];
#pragma unroll
                for (int m = M0; m <= M1; ++m) cp[m - M0] = cv ? __ldg(cpos + (jb + jl) * kG + m) : -1;
#pragma unroll
                for (int c8 = 0; c8 < kHW / 8; ++c8) {
                    // the folded sum plus the H of the stages not yet folded, and L1 + L2
                    float ha[8], hb[8], d1[8], d2[8];
                    tc::tmem_ld8(lane_base + (uint32_t)(N0 + 8 * c8), ha);
                    tc::tmem_ld8(lane_base + (uint32_t)(64 + N0 + 8 * c8), hb);
                    tc::tmem_ld8(lane_base + (uint32_t)(kL1Col + N0 + 8 * c8), d1);
                    tc::tmem_ld8(lane_base + (uint32_t)(kL2Col + N0 + 8 * c8), d2);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int n = N0 + 8 * c8 + e;
                        if (n < kG * kN) {
                            const int m = n / kN, x = n - m * kN;
                            const int32_t p = cp[m - M0];
                            const float v = ((acc[8 * c8 + e] + ha[e]) + hb[e]) + (d1[e] + d2[e]);
                            if (p >= 0) c_val[(int64_t)p * (kN * kN) + kN * x + y] = v;
                        }
                    }
                }
            };
            switch (hq) {
            case 0: epi(std::integral_constant<int, 0>{}); break;
            case 1: epi(std::integral_constant<int, 1 % kNQ>{}); break;
            case 2: epi(std::integral_constant<int, 2 % kNQ>{}); break;
            default: epi(std::integral_constant<int, 3 % kNQ>{}); break;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == kMmaWarp) tc::tmem_dealloc(tm, 512);
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
        (const float *)A, pl->B->row_ptr, (const float *)B, (float *)C, (int32_t)(pl->A->nnzb - 1),
        (int32_t)(pl->B->nnzb - 1), ctx->dev_status, ctx->wait_ns);
    LNV_LAUNCHED();
    return LNV_OK;
}

}  // namespace lnv
