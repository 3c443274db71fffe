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
#include <cuda_bf16.h>

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
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}
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
// Hint: bring the 128-byte line holding p into L2.
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
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

// 8 TMEM columns without the wait: the caller issues tmem_wait_ld() and then
// reg_dep8() on every destination before using it (the empty asm makes the
// uses depend on the wait)
__device__ __forceinline__ void tmem_ld8_raw(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld4_raw(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
__device__ __forceinline__ void reg_dep4(uint32_t (&r)[4]) {
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void reg_dep8(uint32_t (&r)[8]) {
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

// ---- thread-block clusters -------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_peer(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_u32(uint32_t caddr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(caddr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_s32(uint32_t caddr, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(caddr), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Bulk copy from this CTA's shared memory into another CTA of the cluster
// (dst and mbar are shared::cluster addresses from map_peer); the bytes are
// counted on the destination's mbarrier.  16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_s2peer(uint32_t dst_cluster, uint32_t src_cta, uint32_t bytes,
                                            uint32_t mbar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_cluster),
        "r"(src_cta), "r"(bytes), "r"(mbar_cluster)
        : "memory");
}
// Commit of this thread's earlier products to the mbarrier at the same offset
// in every CTA of cta_mask (one arrival each).
__device__ __forceinline__ void commit_multicast(uint64_t *mbar, uint16_t cta_mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_addr(mbar)),
        "h"(cta_mask));
}
__device__ __forceinline__ void fence_proxy_async_cluster() {
    asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
}

// ---- split precision ---------------------------------------------------------
// A finite double x with |x| < 2^E is cut into kSlices balanced base-128 digits:
//   x 2^-E ~ V 2^-55,  V = trunc(x 2^(55-E)),  |V| < 2^55,
//   V = sum_k q_k 128^(8-k),  q_2..q_8 in [-64, 63],  q_1 in [-64, 64],
//   so  x 2^-E = sum_k q_k 2^(1-7k) + r,  |r| < 2^-55.
// The digits need no carry loop: W = V + B with B = 64 sum_{j<7} 128^j has
// plain base-128 digits q_k + 64 in its low 49 bits and q_1 = floor(W / 2^49).
// Integer arithmetic only (the FP64 pipe of this GPU is narrow).  Slice k is
// the BF16 number q_k 2^(1-7k), exact (|q_k| <= 64).
constexpr int kSlices = 8;
constexpr long long kDigitBias = 64LL * 4432676798593LL;  // 64 (128^7 - 1) / 127

// exponent E with |x| < 2^E for a finite nonzero x (E = ilogb(x) + 1); zero and
// subnormals give a very small value
__device__ __forceinline__ int exp_bound(double x) {
    const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
    return ex == 0 ? -2000 : ex - 1022;
}

// W = V + B for x 2^-E (the caller guarantees |x| < 2^E)
__device__ __forceinline__ long long digit_word(double x, int E) {
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
    return V + kDigitBias;
}

// Two slices (k of elements lo and hi, adjacent along K) as one 32-bit word,
// built two at a time in BF16x2: with u = q + 64 in [0, 128], the BF16 bit
// pattern 0x4300 + u is the number 128 + u (the exponent of 128 makes the ULP
// 1; u = 128 carries into the exponent and reads 256), and one packed FMA
// (128 + u) 2^e - 192 2^e = q 2^e, e = 1 - 7k, is exact, so no rounding.
__device__ __forceinline__ uint32_t slice_pair(long long Wlo, long long Whi, int k) {
    uint32_t ulo, uhi;
    if (k == 1) {
        ulo = (uint32_t)((int)(Wlo >> 49) + 64);
        uhi = (uint32_t)((int)(Whi >> 49) + 64);
    } else {
        const int sh = 7 * (kSlices - k);
        ulo = (uint32_t)(Wlo >> sh) & 127u;
        uhi = (uint32_t)(Whi >> sh) & 127u;
    }
    const uint32_t packed = (ulo | (uhi << 16)) + 0x43004300u;
    const uint32_t sc = (uint32_t)(128 - 7 * k) << 7;                   // BF16 2^(1-7k)
    const uint32_t off = 0x8000u | ((uint32_t)(135 - 7 * k) << 7) | 0x40u;  // BF16 -1.5 2^(8-7k)
    const __nv_bfloat162 r = __hfma2(*reinterpret_cast<const __nv_bfloat162 *>(&packed),
                                     __halves2bfloat162(__ushort_as_bfloat16((unsigned short)sc),
                                                        __ushort_as_bfloat16((unsigned short)sc)),
                                     __halves2bfloat162(__ushort_as_bfloat16((unsigned short)off),
                                                        __ushort_as_bfloat16((unsigned short)off)));
    return *reinterpret_cast<const uint32_t *>(&r);
}

// All eight slices of two elements (as slice_pair for k = 1..8) from 32-bit
// halves of W: h = W >> 28 (|W| < 2^56, so h fits 32 bits) holds digits 1..4
// (q_1 = h >> 21 arithmetically, the others 7-bit fields), the low 28 bits of
// W hold digits 5..8.  The two elements' digits are paired by a byte permute.
__device__ __forceinline__ void slice_pairs8(long long W0, long long W1, uint32_t (&out)[kSlices]) {
    const int h0 = (int)(W0 >> 28), h1 = (int)(W1 >> 28);
    const uint32_t l0 = (uint32_t)W0 & 0x0FFFFFFFu, l1 = (uint32_t)W1 & 0x0FFFFFFFu;
    uint32_t u0[kSlices], u1[kSlices];
    u0[0] = (uint32_t)((h0 >> 21) + 64);
    u1[0] = (uint32_t)((h1 >> 21) + 64);
    u0[1] = ((uint32_t)h0 >> 14) & 127u;
    u1[1] = ((uint32_t)h1 >> 14) & 127u;
    u0[2] = ((uint32_t)h0 >> 7) & 127u;
    u1[2] = ((uint32_t)h1 >> 7) & 127u;
    u0[3] = (uint32_t)h0 & 127u;
    u1[3] = (uint32_t)h1 & 127u;
    u0[4] = l0 >> 21;
    u1[4] = l1 >> 21;
    u0[5] = (l0 >> 14) & 127u;
    u1[5] = (l1 >> 14) & 127u;
    u0[6] = (l0 >> 7) & 127u;
    u1[6] = (l1 >> 7) & 127u;
    u0[7] = l0 & 127u;
    u1[7] = l1 & 127u;
#pragma unroll
    for (int k = 1; k <= kSlices; ++k) {
        const uint32_t packed = __byte_perm(u0[k - 1], u1[k - 1], 0x5410) + 0x43004300u;
        const uint32_t sc = (uint32_t)(128 - 7 * k) << 7;
        const uint32_t off = 0x8000u | ((uint32_t)(135 - 7 * k) << 7) | 0x40u;
        const __nv_bfloat162 r = __hfma2(*reinterpret_cast<const __nv_bfloat162 *>(&packed),
                                         __halves2bfloat162(__ushort_as_bfloat16((unsigned short)sc),
                                                            __ushort_as_bfloat16((unsigned short)sc)),
                                         __halves2bfloat162(__ushort_as_bfloat16((unsigned short)off),
                                                            __ushort_as_bfloat16((unsigned short)off)));
        out[k - 1] = *reinterpret_cast<const uint32_t *>(&r);
    }
}

// Products S_a S_b with a + b = d (d = 2..9) accumulate in accumulator d - 2:
// integers in units 2^(2-7d) of magnitude at most K (d-1) 2^12 <= 2^24 for
// K <= 512, exact in FP32.  Recombination in integers: H = sum_{d<=5} I_d
// 2^(7(5-d)) (units 2^-33), L = sum_{d>=6} I_d 2^(7(9-d)) (units 2^-61),
// T = H 2^28 + L exactly (128 bits), value = T 2^(escale-61) rounded once to
// nearest even.  No FP64 instruction on the normal-range path.
__device__ __forceinline__ double combine_ints(const long long (&I)[8], int escale);

// v 2^e as a double, exactly, for an integer |v| < 2^53 whose scaled value is
// a normal number (the caller checks the range): the bits are assembled.
__device__ __forceinline__ double exact_scaled(long long v, int e) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int lz = __clzll((long long)a);               // >= 11
    const unsigned long long mant = a << (lz - 11);     // leading one at bit 52
    const unsigned long long ex = (unsigned long long)(63 - lz + e + 1022);
    return __longlong_as_double((long long)(sgn | (mant + (ex << 52))));  // the leading one adds 1
}

// T 2^(escale - 61), T = sum_k I_k 2^(7 (7 - k)), rounded once.  With
// H = sum_{k<4} I_k 2^(7 (3 - k)) and L = sum_{k>=4} I_k 2^(7 (7 - k)) (both
// below 2^53 in magnitude), T = H 2^28 + L: the two scaled halves are exact
// doubles and one FP64 addition rounds their sum correctly.  Scales where a
// half could leave the normal range take the 128-bit integer path.
__device__ __forceinline__ double combine_halves(const long long (&I)[8], int escale) {
    const int sc = escale - 61;
    if (sc < -1000 || sc > 900) return combine_ints(I, escale);
    const long long H = (I[0] << 21) + (I[1] << 14) + (I[2] << 7) + I[3];
    const long long L = (I[4] << 21) + (I[5] << 14) + (I[6] << 7) + I[7];
    return exact_scaled(H, sc + 28) + exact_scaled(L, sc);
}

__device__ __forceinline__ double combine8(const float (&d)[8], int escale) {
    long long I[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) I[k] = (long long)__float2int_rn(d[k] * __int_as_float((127 + 12 + 7 * k) << 23));
    return combine_halves(I, escale);
}

// The same rounding for accumulators whose integers are at most 2^22 in
// magnitude (at most 128 terms per accumulation: |I_d| <= (d - 1) 128 64^2 <=
// 2^22, the update's case).  The integer is read from the bits of an exact
// FP32 add: with M = 1.5 2^23 in the accumulator's unit, d + M lies in
// [2^23, 2^24] units, where consecutive integers are consecutive bit patterns,
// so bits(d + M) - bits(M) = I with no conversion instruction.
__device__ __forceinline__ double combine8_small(const float (&d)[8], int escale) {
    long long I[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int mb = ((127 + 11 - 7 * k) << 23) | 0x400000;  // 1.5 2^(11 - 7k) = 1.5 2^23 units of 2^-(12+7k)
        I[k] = (long long)(__float_as_int(d[k] + __int_as_float(mb)) - mb);
    }
    return combine_halves(I, escale);
}

__device__ __forceinline__ double combine_ints(const long long (&I)[8], int escale) {
    const long long H = (I[0] << 21) + (I[1] << 14) + (I[2] << 7) + I[3];
    const long long L = (I[4] << 21) + (I[5] << 14) + (I[6] << 7) + I[7];
    // T = H 2^28 + L as hi:lo (two's complement, 128 bits)
    const unsigned long long lo = ((unsigned long long)H << 28) + (unsigned long long)L;
    const long long carry = (unsigned long long)lo < ((unsigned long long)H << 28) ? 1 : 0;
    const long long hi = (H >> 36) + (L >> 63) + carry;
    if (hi == 0 && lo == 0) return 0.0;
    const bool neg = hi < 0;
    unsigned long long ahi = (unsigned long long)hi, alo = lo;
    if (neg) {  // |T|
        alo = ~alo + 1ull;
        ahi = ~ahi + (alo == 0 ? 1ull : 0ull);
    }
    // most significant bit position of |T| (< 75)
    const int msb = ahi ? 127 - __clzll((long long)ahi) : 63 - __clzll((long long)alo);
    unsigned long long mant;
    int e2 = msb;
    if (msb <= 52) {
        mant = alo << (52 - msb);
    } else {
        const int sh = msb - 52;  // 1..22: |T| < 2^75
        const unsigned long long keep = (alo >> sh) | (ahi << (64 - sh));
        const unsigned long long rem = alo & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        mant = keep + ((rem > half || (rem == half && (keep & 1ull))) ? 1ull : 0ull);
        if (mant >> 53) {
            mant >>= 1;
            ++e2;
        }
    }
    const int biased = e2 + escale - 61 + 1023;
    if (biased <= 0 || biased >= 2047) {  // outside the normal range: FP64 arithmetic
        const double v = ldexp((double)mant, e2 - 52);
        return ldexp(neg ? -v : v, escale - 61);
    }
    return __longlong_as_double((long long)((neg ? (1ull << 63) : 0ull) | ((unsigned long long)biased << 52) |
                                            (mant & 0xFFFFFFFFFFFFFull)));
}

}  // namespace tc
}  // namespace hsvd
