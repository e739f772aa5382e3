// Thin wrappers of the sm_100-family tensor-core instructions (tcgen05), the
// mbarrier operations that order them, and the two descriptors they read.
//
// Conventions (PTX ISA, tcgen05):
//  - Tensor memory (TMEM) is 128 lanes x 512 columns of 32-bit cells per SM.
//    An address is (lane << 16) | column.  A warp reaches only the lanes
//    32 (warp % 4) .. 32 (warp % 4) + 31.
//  - An MMA D[M x N] (+)= A[M x K] B[K x N] of kind::tf32 takes K = 8.  D
//    lives in TMEM (lane = row, one column per element); A comes from TMEM
//    (same layout) or shared memory; B from shared memory, described by a
//    64-bit descriptor.
//  - Shared-memory operands here are K-major without swizzle: "core
//    matrices" of 8 rows x 16 bytes stored as 128 contiguous bytes; the
//    descriptor's leading byte offset (LBO) steps between core matrices
//    along K, the stride byte offset (SBO) between groups of 8 rows.
//  - FP32 operands are read as TF32: the tensor core ignores the low 13
//    bits of the significand (truncation; checked on GB300 against a CPU
//    reference of truncated operands).  The split below hands it values
//    already rounded to TF32, so nothing is truncated.
//
// Every wait below is bounded by a time limit: a wait that runs out raises a
// flag in shared memory that every other wait of the CTA observes, so the
// CTA drains and exits instead of hanging.
#pragma once
#include <cstdint>

namespace lnv {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- TMEM allocation (one warp, all lanes) ----------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- ordering between tcgen05 operations and thread synchronisation --------
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory made visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- mbarriers ----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Test the phase; if it is not complete the thread may sleep (up to 20 us)
// until it completes, so waiting warps do not spin on the issue slots.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(20000)
        : "memory");
    return ok != 0;
}
// Wait for the completion of the barrier phase of the given parity.  Gives up
// (false) when *abort is set by another thread of the CTA, or after limit_ns,
// in which case it sets *abort itself.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, uint64_t limit_ns)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}
// The same without the abort flag (used to drain in-flight MMAs before the
// tensor memory is released).
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
// Add `bytes` to the transfer count the barrier's current phase waits for.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bulk copy global -> shared memory of this CTA (the TMA engine, no tensor
// map): both addresses 16-byte aligned, bytes a multiple of 16; its bytes
// count toward the barrier's transfer count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst_smem, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst_smem),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Arrive on the barrier once every cp.async this thread issued so far has
// landed (the arrival is not counted in advance: the barrier's count includes it).
__device__ __forceinline__ void cp_async_mbar_arrive(uint32_t bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
// Arrive on the barrier once every tcgen05 operation this thread issued so far
// has completed.
__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// ---- descriptors ----------------------------------------------------------------
// Shared-memory matrix descriptor: K-major, no swizzle, start address and the
// two core-matrix strides in bytes (multiples of 16).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, dense, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- MMA ---------------------------------------------------------------------
// D (+)= A B with A in TMEM at a_tmem (M = 128 lanes, 8 columns), B described
// by b_desc; accumulate != 0 adds to D, else overwrites it.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// ---- TMEM <-> registers (32 lanes x 32 bits, 8 columns per call) --------------
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// load 8 columns and wait for them (the values are usable on return)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "r"(taddr)
        : "memory");
}

// ---- operand split for 3xTF32 --------------------------------------------------
// x = hi + lo + r with hi = x rounded to the nearest TF32 value, lo = x - hi
// (exact in FP32) rounded to the nearest TF32 value, |r| <= 2^-22 |x|.  Both
// roundings are to nearest: truncation (what the tensor core applies to FP32
// operands) leaves lo, and the dropped lo*lo term, with the sign of x, an
// error that adds up over long sums instead of cancelling.
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(x - hi);
}
// The same for two values at once (one packed FP32 subtraction; x - hi is
// exact, so its rounding mode does not matter).
__device__ __forceinline__ void split_tf32x2(float x0, float x1, float &h0, float &h1, float &l0, float &l1)
{
    h0 = tf32_rna(x0);
    h1 = tf32_rna(x1);
    unsigned long long x, h, l;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(x0), "f"(x1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(h) : "f"(h0), "f"(h1));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(l) : "l"(x), "l"(h));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l0), "=f"(l1) : "l"(l));
    l0 = tf32_rna(l0);
    l1 = tf32_rna(l1);
}
// The cheaper split of kernels whose producer threads are bound by their
// instruction count: hi = x with the low 13 significand bits cleared, lo = x
// - hi exact in FP32 (the tensor core then truncates lo to TF32: lo and the
// dropped lo*lo term carry the sign of x, a bias of about 2^-21 relative).
__device__ __forceinline__ void split_tf32x2_trunc(float x0, float x1, float &h0, float &h1, float &l0, float &l1)
{
    h0 = __uint_as_float(__float_as_uint(x0) & 0xFFFFE000u);
    h1 = __uint_as_float(__float_as_uint(x1) & 0xFFFFE000u);
    unsigned long long x, h, l;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(x0), "f"(x1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(h) : "f"(h0), "f"(h1));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(l) : "l"(x), "l"(h));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l0), "=f"(l1) : "l"(l));
}


// 16-byte asynchronous copy global -> shared (zero-filled when src_bytes = 0),
// its commit group and wait (up to N groups of this thread still in flight).
__device__ __forceinline__ void cp_async16(uint32_t dst_smem, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst_smem), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace tc
}  // namespace lnv
