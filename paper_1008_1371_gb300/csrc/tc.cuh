// tc.cuh -- 5th-generation tensor-core (tcgen05) building blocks for sm_103a,
// and the exact FP64 <-> BF16-slice conversions of the split-precision form.
//
// Operands live in shared memory in the no-swizzle K-major "core matrix"
// layout: a core matrix is 8 rows x 8 BF16 (16 bytes per row, 128 contiguous
// bytes); the descriptor's leading-byte offset is the stride between core
// matrices along K (128 B here) and its stride-byte offset the stride between
// 8-row groups.  Accumulators live in tensor memory (TMEM), 128 lanes x 32-bit
// columns, one lane per output row.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hsvd {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), the
// descriptor version bit of this architecture, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// K-major, 128-byte swizzle: rows of 64 BF16 (128 B), 8-row atoms of 1024 B,
// the 16-byte chunk index XOR the row within the atom; tiles 1024-B aligned.
// The start address advances by 32 B per K step of 16.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// byte offset of element (r, k), 0 <= k < 64, in a 128B-swizzled tile
__host__ __device__ __forceinline__ uint32_t sw128_offset(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1));
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of an R x KT operand tile in the core-matrix layout
__host__ __device__ __forceinline__ uint32_t core_offset(int r, int k, int KT) {
    return (uint32_t)((((r >> 3) * (KT >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7)) * 2u;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                    uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_addr(mbar)));
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;"); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes));
}
// Bounded wait for the phase with the given parity; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t max_iter = (1u << 26)) {
    uint32_t ok = 0;
    for (uint32_t it = 0; it < max_iter; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(mbar)), "r"(parity));
        if (ok) return true;
    }
    return false;
}
// 1-D bulk copy global -> shared (TMA), completion counted on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar))
        : "memory");
}
// 16 consecutive 32-bit TMEM columns of this thread's lane (32x32b shape).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 8 consecutive 32-bit TMEM columns of this thread's lane (32x32b shape).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// ---- split precision ---------------------------------------------------------
// A finite double x with |x| < 2^E is cut into kSlices balanced base-128 digits:
//   x 2^-E ~ V 2^-55,  V = trunc(x 2^(55-E)),  V = sum_k q_k 128^(8-k),
//   q_k in [-64, 64],  so  x 2^-E = sum_k q_k 2^(-6-7(k-1)) + r,  |r| < 2^-55.
// The digits come from x's integer mantissa (integer arithmetic only: the FP64
// pipe of this GPU is narrow).  Slice k is the BF16 number q_k 2^(-6-7(k-1)),
// exact (|q_k| <= 64 has at most 7 significant bits).
constexpr int kSlices = 8;

// exponent E with |x| < 2^E for a finite nonzero x (E = ilogb(x) + 1); zero and
// subnormals give a very small value
__device__ __forceinline__ int exp_bound(double x) {
    const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
    return ex == 0 ? -2000 : ex - 1022;
}

// BF16 bits of q 2^(-6-7(k-1)), |q| <= 64
__device__ __forceinline__ uint16_t digit_bits(int q, int k) {
    if (!q) return 0;
    const uint32_t sign = q < 0 ? 0x8000u : 0u;
    const uint32_t a = (uint32_t)(q < 0 ? -q : q);
    const int msb = 31 - __clz((int)a);
    const uint32_t biased = (uint32_t)(msb - 6 - 7 * (k - 1) + 127);
    const uint32_t mant = (a << (7 - msb)) & 0x7Fu;
    return (uint16_t)(sign | (biased << 7) | mant);
}

// slices of x 2^-E (the caller guarantees |x| < 2^E); out[k-1] = slice k
__device__ __forceinline__ void split_slices(double x, int E, uint16_t (&out)[kSlices]) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    long long V = 0;
    if (ex != 0) {
        const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = (ex - 1023) - E + 3;  // <= 2
        uint64_t F = 0;
        if (sh >= 0) F = M << sh;
        else if (sh > -64) F = M >> (-sh);
        V = (b >> 63) ? -(long long)F : (long long)F;
    }
#pragma unroll
    for (int k = kSlices; k >= 2; --k) {
        int d = (int)(V & 127);
        if (d >= 64) d -= 128;
        V = (V - d) >> 7;
        out[k - 1] = digit_bits(d, k);
    }
    out[0] = digit_bits((int)V, 1);
}

// Products S_a S_b with a + b = d (d = 2..9) accumulate in accumulator d - 2:
// integers in units 2^(-12-7(d-2)) of at most K (d-1) 2^12 <= 2^24 for
// K <= 512, exact in FP32.  Recombination: H = sum_{d<=5} I_d 2^(7(5-d)) (units
// 2^-33), L = sum_{d>=6} I_d 2^(7(9-d)) (units 2^-61), both exact in 64-bit
// integers and in FP64; value = 2^-61 (H 2^28 + L) 2^escale with one rounding.
__device__ __forceinline__ double combine8(const float (&d)[8], int escale) {
    long long I[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) I[k] = __float2ll_rn(ldexpf(d[k], 12 + 7 * k));
    const long long H = (I[0] << 21) + (I[1] << 14) + (I[2] << 7) + I[3];
    const long long L = (I[4] << 21) + (I[5] << 14) + (I[6] << 7) + I[7];
    const double v = fma((double)H, 268435456.0, (double)L);
    return ldexp(v, escale - 61);
}

}  // namespace tc
}  // namespace hsvd
