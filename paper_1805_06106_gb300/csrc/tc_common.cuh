// Blackwell (sm_103a) tensor-core building blocks in inline PTX: mbarriers, 1D bulk copies
// (TMA engine), tensor memory allocation, shared-memory matrix descriptors and tcgen05.mma of
// kind::tf32 with FP32 accumulation in tensor memory.
//
// Operand layout used throughout ("K-major, no swizzle"): a tile of R rows x W columns (W a
// multiple of 8, 4-byte elements) is stored as core matrices of 8 rows x 16 bytes, each core
// matrix 128 contiguous bytes (row r of the core at byte 16 r).  The core holding rows
// 8g..8g+7 and columns 4h..4h+3 starts at byte h * 128 + g * SBO, with SBO >= W * 32 (a larger
// SBO pads the row groups apart, which spreads row-group writes over more banks).  An MMA step
// over columns 8s..8s+7 then reads the descriptor (start + 256 s, LBO = 128, SBO).
//
// Split-TF32 ("3xTF32") products: x = hi + lo with hi = rna_tf32(x), lo = rna_tf32(x - hi);
// a b ~= a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in FP32 by the tensor cores.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qbx {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------- mbarriers

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity; gives up (returns false) after `limit` clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1D bulk copy global -> shared (TMA engine); both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Makes this thread's generic-proxy shared-memory writes visible to the tensor cores.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------- tensor memory

// Whole warp: allocates ncols (power of two, 32..512) columns; the address lands in *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Whole warp: 32 lanes (TMEM lanes taddr.lane .. +31) x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- MMA

// Shared-memory matrix descriptor, K-major without swizzle (layout in the header comment).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family
    return d;                // base offset 0, absolute LBO mode, no swizzle
}

// Instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] x B[smem]^T; issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives on `bar` once every tcgen05 operation this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// ---------------------------------------------------------------- split TF32

// x rounded to TF32 (10 explicit significand bits), to nearest with ties away from zero: half a TF32 unit
// in the last place (bit 12) is added to the bit pattern and the 13 low bits are cleared.  The sign bit
// is apart from the magnitude, so this rounds the magnitude; a carry out of the significand moves into
// the exponent (the next power of two), and an infinity stays infinite.  The same result as
// cvt.rna.tf32.f32 for every finite or infinite input, in two integer operations.
__device__ __forceinline__ float tf32_rna(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(x - hi);
}

// from FP64: hi carries the leading 11 bits, lo the next 11 (both exact tf32 values)
__device__ __forceinline__ void split_tf32(double x, float &hi, float &lo)
{
    hi = tf32_rna((float)x);
    lo = tf32_rna((float)(x - (double)hi));
}

// byte offset of element (row, col) in a K-major no-swizzle tile with row-group stride sbo
__host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int col, uint32_t sbo)
{
    return (uint32_t)(col >> 2) * 128u + (uint32_t)(row >> 3) * sbo + (uint32_t)(row & 7) * 16u +
           (uint32_t)(col & 3) * 4u;
}

// Compensated FP32 accumulation (a double-float sum): hi + lo carries the running sum of FP32 terms to
// about 2^-44 of the sum of their magnitudes.  Each step is Knuth's TwoSum (t + err == hi + x exactly)
// with the error added into lo; six FP32 operations, no FP64 instruction.
__device__ __forceinline__ void df_add(float &hi, float &lo, float x)
{
    const float t = hi + x;
    const float bp = t - hi;
    const float err = (hi - (t - bp)) + (x - bp);
    hi = t;
    lo += err;
}

constexpr long long WAIT_LIMIT = 4000000000LL;  // clock cycles (about two seconds) before a wait gives up

}  // namespace tc
}  // namespace qbx
