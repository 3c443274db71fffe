// precision.cu -- the split-precision form of the blocked method: the pivot
// Gram blocks and the G / V updates as BF16-slice products on the tcgen05
// tensor cores (Ozaki-style splitting), exact FP32 accumulation in tensor
// memory and an exact integer recombination into FP64.  Everything else
// (rotation angles, tanh / cosh, the test of Eq. 2.3, the column norms of the
// finalisation) stays in FP64.  Pivot blocks are 128 x 128 (block width 64).
//
// Splitting (tc.cuh): a row or column of an operand with |x| < 2^E is written
// as 8 balanced base-128 digits, x 2^-E = sum_k q_k 2^(1-7k) + r with
// |q_k| <= 64 and |r| < 2^-55; slice k is the exact BF16 number q_k 2^(1-7k).  The 36 products of slices a, b with a + b <= 9 run on the
// tensor cores; those with a + b = d accumulate in TMEM accumulator d - 2,
// where every partial sum is an integer below 2^24 in its unit (at most 512
// rows per accumulation), so the FP32 accumulation is exact.  The eight
// accumulators are recombined in 64-bit integers and rounded once to FP64.
// What is left out (products with a + b >= 10, the digits' remainder r) is
// below 2^-53 of the operands' scale per term.
//
// TMEM holds 512 columns per SM: eight accumulators of 64 columns.  Outputs
// are therefore formed 128 x 64 at a time (M = 128 lanes, N = 64).
//
// Update balancing: X W = (X D^-1)(D W) with D = diag(2^d_k), d_k from the
// column norms of G's panel, so a small column of a graded G keeps its
// relative precision; V's rows use D = I.
#include "hsvd_internal.cuh"
#include "tc.cuh"

namespace hsvd {
namespace {

using namespace tc;

constexpr int NNX = 128;             // pivot block order 2b
constexpr int kThrX = 256;           // eight warps: two per TMEM lane quarter
constexpr int kThrU = 544;           // update: the products warp and sixteen producer warps
constexpr int kThrG = 544;           // Gram: the products warp and sixteen splitting warps
constexpr int kGramK = 512;          // rows of G per Gram CTA pair (exactness window)
constexpr int kGramKT = 32;          // rows per shared-memory tile of the Gram
constexpr int kGramBufs = 2;         // Gram tiles in flight (96 KB each)
constexpr int kUpdKT = 32;           // k per shared-memory tile of the update
constexpr int kUpdRows = 64;         // rows of G or V per update item (N)
constexpr int kN = 64;               // MMA N
constexpr uint32_t kTmemCols = 512;  // eight accumulators of 64 columns
constexpr uint32_t kWaitIter = 1u << 26;

__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The 36 slice products of one K step (16 k) as 12 instructions.  Slice a of
// A (at a_base + (a - 1) a_stride) meets B slices 1 .. 9 - a, which lie side
// by side along N (slice b at b_base + (b - 1) b_stride, b_stride = 8 core
// groups of sbo bytes, so one descriptor with a uniform group stride covers
// several): one product with N = 64 nb covers b = b1 .. b1 + nb - 1 and writes
// accumulators a + b1 - 2 .. a + b1 + nb - 3, adjacent in TMEM.  Large N keeps
// the tensor core near its peak; 36 products with N = 64 ran at 0.42 of it.
// `first`: the first K step of an accumulation (slice 1 initialises all eight
// accumulators; the later products add to them).
__device__ __forceinline__ void issue_products(uint32_t tmem, uint32_t a_base, uint32_t a_stride, uint32_t b_base,
                                               uint32_t b_stride, uint32_t koff, uint32_t sbo, bool first) {
    const uint64_t da0 = smem_desc(a_base + koff, 128, sbo);
#pragma unroll
    for (int a = 1; a <= kSlices; ++a) {
        const uint64_t da = da0 + (uint64_t)(a - 1) * (a_stride >> 4);
#pragma unroll
        for (int b1 = 1; a + b1 <= kSlices + 1; b1 += 4) {
            const int nb = (kSlices + 2 - a - b1) < 4 ? (kSlices + 2 - a - b1) : 4;
            const uint64_t db = smem_desc(b_base + (uint32_t)(b1 - 1) * b_stride + koff, 128, sbo);
            mma(tmem + (uint32_t)(a + b1 - 2) * kN, da, db, idesc_bf16(NNX, kN * nb), (first && a == 1) ? 0u : 1u);
        }
    }
}

__device__ __forceinline__ void bar_named(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// this thread's lane and 4 columns [c0, c0+4) of all eight accumulators
__device__ __forceinline__ void read_accs4(uint32_t tmem, int lane_base, int c0, float (&v)[8][4]) {
    uint32_t r[8][4];
#pragma unroll
    for (int acc = 0; acc < 8; ++acc) tmem_ld4_raw(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(acc * kN + c0), r[acc]);
    tmem_wait_ld();
#pragma unroll
    for (int acc = 0; acc < 8; ++acc) {
        reg_dep4(r[acc]);
#pragma unroll
        for (int j = 0; j < 4; ++j) v[acc][j] = __uint_as_float(r[acc][j]);
    }
}

// this thread's lane and 8 columns [c0, c0+8) of all eight accumulators: the
// eight loads are issued back to back and waited for once
__device__ __forceinline__ void read_accs(uint32_t tmem, int lane_base, int c0, float (&v)[8][8]) {
    uint32_t r[8][8];
#pragma unroll
    for (int acc = 0; acc < 8; ++acc) tmem_ld8_raw(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(acc * kN + c0), r[acc]);
    tmem_wait_ld();
#pragma unroll
    for (int acc = 0; acc < 8; ++acc) {
        reg_dep8(r[acc]);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[acc][j] = __uint_as_float(r[acc][j]);
    }
}

// ---------------------------------------------------------------- Gram
// Two CTAs per (pair, split): CTA h forms columns [64 h, 64 h + 64) of the
// partial A_P over rows [512 split, 512 split + 512) of the panel
// P = [G_I G_J] (m x 128): A = P^T (128 x K, K-major), B = columns
// [64 h, 64 h + 64) of the same tile, written a second time with the eight
// slices side by side (the wide products of issue_products).  The two CTAs
// form a cluster: each splits only its own 64 columns (into its A and B
// regions) and bulk-copies its A part into the peer's A region, so every
// column is split once.  Warp-specialised pipeline over 32-row tiles,
// kGramBufs in flight:
//   - warps 1..16 wait until the products that last read a buffer are done
//     in both CTAs (mbarrier `empty`, one commit from each), split the own
//     columns of the tile into it (values loaded one tile ahead), send the A
//     part to the peer and arrive on `full` expecting the peer's A part;
//   - warp 0, lane 0 waits on `full`, issues the tile's 24 products and
//     commits them to `empty` in both CTAs.
// Every wait is bounded; after a failure each role still passes the same
// barriers and the kernel reports HSVD_ERR_CUDA.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThrG, 1)
k_gram_x(const double *__restrict__ G, int64_t rows, int64_t ldg, const int *__restrict__ col0, int ksplit,
         double *__restrict__ part, int *__restrict__ status, int ahead) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr uint32_t kSliceBytes = NNX * kGramKT * 2;     // one slice of a tile, all columns (8 KB)
    constexpr uint32_t kHalfBytes = kN * kGramKT * 2;       // one slice, this CTA's columns (4 KB)
    constexpr uint32_t kBOff = kSlices * kSliceBytes;       // the B copy after the A slices
    constexpr uint32_t kBufBytes = kBOff + kSlices * kHalfBytes;  // one tile (96 KB)
    constexpr int kProd = kThrG - 32;                       // splitting threads (warps 1..16)
    __shared__ int Ecol[NNX];
    __shared__ __align__(8) uint64_t full[kGramBufs], empty[kGramBufs];
    __shared__ uint32_t tbase;
    __shared__ int s_fail;
    const uint32_t half = cluster_rank(), peer = half ^ 1u;
    const int pair = (blockIdx.x >> 1) / ksplit, split = (blockIdx.x >> 1) % ksplit;
    const int64_t r0 = (int64_t)split * kGramK, r1 = min(rows, r0 + kGramK);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cI = col0[2 * pair], cJ = col0[2 * pair + 1];
    auto colptr = [&](int c) { return G + (int64_t)(c < NNX / 2 ? cI + c : cJ + c - NNX / 2) * ldg; };
    cluster_sync();  // both CTAs run before either writes into the other
    // exponents of the own columns over the split's rows, into both CTAs
    for (int c = kN * (int)half + warp; c < kN * (int)half + kN; c += kThrG / 32) {
        const double *g = colptr(c);
        int e = -2000;
        int64_t r = r0 + lane;
        for (; r + 15 * 32 < r1; r += 16 * 32) {  // sixteen loads in flight per lane
            double x[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) x[u] = g[r + u * 32];
#pragma unroll
            for (int u = 0; u < 16; ++u) e = max(e, exp_bound(x[u]));
        }
        for (; r < r1; r += 32) e = max(e, exp_bound(g[r]));
        e = warp_max_i(e);
        if (lane == 0) {
            e = e < -1000 ? 0 : e;
            Ecol[c] = e;
            st_cluster_s32(map_peer(smem_addr(&Ecol[c]), peer), e);
        }
    }
    if (tid == 0) {
        s_fail = 0;
        for (int b = 0; b < kGramBufs; ++b) {
            mbar_init(&full[b], 1);   // the splitters' arrival (expecting the peer's A part)
            mbar_init(&empty[b], 2);  // the products' commits of both CTAs
        }
    }
    if (warp == 0) tmem_alloc(&tbase, kTmemCols);
    fence_before();
    cluster_sync();  // exponents exchanged, barriers of both CTAs initialised
    fence_after();
    const uint32_t tmem = tbase;
    const int ntiles = (int)((r1 - r0 + kGramKT - 1) / kGramKT);
    // the use-th fill of a buffer (tile t is fill t / kGramBufs of buffer t % kGramBufs)
    auto wait1 = [&](uint64_t *mb, int tile) {
        if (!s_fail && !mbar_wait(mb, (uint32_t)((tile / kGramBufs) & 1), kWaitIter)) s_fail = 1;
    };
    if (warp > 0) {
        // ------------------------------------------------ splitters
        // a thread splits four consecutive rows of one column per tile: warp
        // (8 column groups x 2 halves of the tile's 32 rows), lane -> column
        // (lane >> 2) of the group and rows 4 (lane & 3) .. + 3 of the half;
        // each slice is one 8-byte store (two adjacent words of a core row)
        const int pw = warp - 1, ptid = tid - 32, cbase = kN * (int)half;
        static_assert(kProd == kN * (kGramKT / 4), "one row quad of one column per thread");
        const int c = cbase + (pw >> 1) * 8 + (lane >> 2), k = (pw & 1) * 16 + 4 * (lane & 3);
        const double *gcol = colptr(c);
        const uint32_t off = core_offset(c, k, kGramKT), offb = kBOff + core_offset(c - cbase, k, kGramKT);
        auto load_tile = [&](int t, double (&x)[4]) {
            const int64_t row = r0 + (int64_t)t * kGramKT + k;
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = row + u < r1 ? gcol[row + u] : 0.0;
        };
        double cur[4];
        if (ntiles > 0) load_tile(0, cur);
        // the panel of the CTA `ahead` blocks later (the next wave's CTA in the
        // same place) into L2, a few lines per tile, so that its column
        // exponents and tiles read L2 rather than DRAM
        const int nblk = (int)blockIdx.x + ahead;
        const double *pf_col = nullptr;
        int64_t pf_r0 = 0, pf_r1 = 0;
        if (ahead > 0 && nblk < (int)gridDim.x) {
            const int npair = (nblk >> 1) / ksplit, nsplit_i = (nblk >> 1) % ksplit, nh = nblk & 1;
            const int cc2 = kN * nh + ptid % kN;
            const int ci2 = col0[2 * npair], cj2 = col0[2 * npair + 1];
            pf_col = G + (int64_t)(cc2 < NNX / 2 ? ci2 + cc2 : cj2 + cc2 - NNX / 2) * ldg;
            pf_r0 = (int64_t)nsplit_i * kGramK;
            pf_r1 = min(rows, pf_r0 + kGramK);
        }
        for (int t = 0; t < ntiles; ++t) {
            const int b = t % kGramBufs;
            if (pf_col) {  // 512 threads x one 128-byte line per tile: 64 columns x 8 lines per tile
                const int64_t row = pf_r0 + ((int64_t)t * (kProd / kN) + ptid / kN) * 16;
                if (row < pf_r1) prefetch_l2(pf_col + row);
            }
            // the products of tile t - kGramBufs read buffer b
            if (ptid == 0 && t >= kGramBufs) wait1(&empty[b], t - kGramBufs);
            bar_named(1, kProd);
            if (!s_fail) {
                unsigned char *buf = smem + (uint32_t)b * kBufBytes;
                const int e = Ecol[c];
                uint32_t s01[kSlices], s23[kSlices];
                slice_pairs8(digit_word(cur[0], e), digit_word(cur[1], e), s01);
                slice_pairs8(digit_word(cur[2], e), digit_word(cur[3], e), s23);
#pragma unroll
                for (int sl = 0; sl < kSlices; ++sl) {
                    const uint2 v = make_uint2(s01[sl], s23[sl]);
                    *reinterpret_cast<uint2 *>(buf + off + (uint32_t)sl * kSliceBytes) = v;
                    *reinterpret_cast<uint2 *>(buf + offb + (uint32_t)sl * kHalfBytes) = v;
                }
            }
            fence_proxy_async();
            bar_named(1, kProd);
            if (ptid < kSlices && !s_fail) {
                // the own columns of every A slice (4 KB each) into the peer's
                // buffer, one copy per lane; lane 0 arrives expecting the peer's part
                const uint32_t lsrc = smem_addr(smem) + (uint32_t)b * kBufBytes + (uint32_t)half * kHalfBytes +
                                      (uint32_t)ptid * kSliceBytes;
                bulk_s2peer(map_peer(lsrc, peer), lsrc, kHalfBytes, map_peer(smem_addr(&full[b]), peer));
                if (ptid == 0) mbar_expect_tx(&full[b], kSlices * kHalfBytes);
            }
            if (t + 1 < ntiles) load_tile(t + 1, cur);
        }
    } else {
        // ------------------------------------------------ products (warp 0, lane 0)
        if (lane == 0) {
            const uint32_t sbo = (kGramKT / 8) * 128;
            static_assert(kHalfBytes == (kN / 8) * (kGramKT / 8) * 128, "B slices side by side along N");
            for (int t = 0; t < ntiles; ++t) {
                const int b = t % kGramBufs;
                wait1(&full[b], t);
                if (s_fail) continue;
                fence_after();
                const uint32_t base = smem_addr(smem) + (uint32_t)b * kBufBytes;
                for (int ks = 0; ks < kGramKT / 16; ++ks)
                    issue_products(tmem, base, kSliceBytes, base + kBOff, kHalfBytes, ks * 256, sbo, t == 0 && ks == 0);
                commit_multicast(&empty[b], 0x3);
            }
            if (ntiles > 0) wait1(&empty[(ntiles - 1) % kGramBufs], ntiles - 1);
        }
        __syncwarp();
    }
    __syncthreads();
    fence_after();
    if (!s_fail) {
        // warps 1..16: lane c = row of A_P (TMEM lane quarter warp % 4), the
        // four warps of a quarter take 16 TMEM columns each
        if (warp > 0) {
            const int q = warp & 3, c = 32 * q + lane, h2 = (warp - 1) >> 2;
            constexpr int kCols = kN / 4;
            double *out = part + ((size_t)pair * ksplit + split) * NNX * NNX;
            for (int c0 = kCols * h2; c0 < kCols * h2 + kCols; c0 += 8) {
                float v[8][8];
                read_accs(tmem, 32 * q, c0, v);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float d[8];
#pragma unroll
                    for (int a = 0; a < 8; ++a) d[a] = v[a][j];
                    const int col = kN * (int)half + c0 + j;
                    out[c + (size_t)col * NNX] = combine8(d, Ecol[c] + Ecol[col]);
                }
            }
        }
    } else if (tid == 0 && status) {
        atomicExch(status, HSVD_ERR_CUDA);
    }
    fence_before();
    cluster_sync();  // no CTA leaves while its peer may still write into it
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- W' slices
// The A operand of the transposed update, W'^T (128 x 128, K-major), for G rows
// (W' = D W_P) and for V rows (W' = W_P), in four k quarters of 32, with
// per-column exponents F_j.  A cluster of eight CTAs per rotated pair: CTA
// (which, quarter) forms one 128 x 32 tile of slices.  The column exponents of
// both kinds are formed once per pair, each CTA taking 16 columns and writing
// them into every CTA of the cluster.
// wsl layout: [pair][which][quarter][slice][128 x 32 core-matrix tile]
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(kThrX)
k_wprep_x(const double *__restrict__ Wp, const int *__restrict__ dexp, const int *__restrict__ rotated,
          uint16_t *__restrict__ wsl, int *__restrict__ wexp, unsigned long long *__restrict__ upd_count) {
    const int pair = blockIdx.x >> 3;
    const int rank = (int)cluster_rank(), which = (rank >> 2) & 1, q = rank & 3;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (!rotated[pair]) return;  // the whole cluster leaves together
    if (tid == 0 && upd_count && rank == 0) atomicAdd(upd_count, 1ull);
    __shared__ int dg[NNX], Fk[2][NNX];
    const double *W = Wp + (size_t)pair * NNX * NNX;  // W(k, j) at k + j * 128
    for (int k = tid; k < NNX; k += kThrX) dg[k] = dexp[(size_t)pair * NNX + k];
    cluster_sync();  // every CTA running before any remote write
    // columns [16 rank, 16 rank + 16): F_j for G rows (with d_k) and for V rows
    for (int j = NNX / 8 * rank + warp; j < NNX / 8 * (rank + 1); j += kThrX / 32) {
        int eg = -2000, ev = -2000;
        for (int k = lane; k < NNX; k += 32) {
            const int e = exp_bound(W[k + (size_t)j * NNX]);
            eg = max(eg, e + dg[k]);
            ev = max(ev, e);
        }
        eg = warp_max_i(eg);
        ev = warp_max_i(ev);
        if (lane < 8) {
            const int fg = eg < -1000 ? 0 : eg, fv = ev < -1000 ? 0 : ev;
            st_cluster_s32(map_peer(smem_addr(&Fk[0][j]), (uint32_t)lane), fg);
            st_cluster_s32(map_peer(smem_addr(&Fk[1][j]), (uint32_t)lane), fv);
        }
    }
    cluster_sync();
    const int *F = Fk[which];
    if (q == 0)
        for (int j = tid; j < NNX; j += kThrX) wexp[((size_t)pair * 2 + which) * NNX + j] = F[j];
    constexpr size_t kTile = (size_t)NNX * kUpdKT;  // elements per slice tile
    uint16_t *dst = wsl + (((size_t)pair * 2 + which) * 4 + q) * kSlices * kTile;
    // a warp step covers one 8 (j) x 8 (k) core matrix: lane -> j (lane >> 2),
    // k pair 2 (lane & 3)
    const int jj = lane >> 2, kp = 2 * (lane & 3);
    for (int core = warp; core < (NNX / 8) * (kUpdKT / 8); core += kThrX / 32) {
        const int j = (core / (kUpdKT / 8)) * 8 + jj, kk = (core % (kUpdKT / 8)) * 8 + kp;
        const int k = q * kUpdKT + kk;
        const int dk0 = which == 0 ? dg[k] : 0, dk1 = which == 0 ? dg[k + 1] : 0;
        const double w0 = W[k + (size_t)j * NNX], w1 = W[k + 1 + (size_t)j * NNX];
        const long long d0 = digit_word(w0, F[j] - dk0);
        const long long d1 = digit_word(w1, F[j] - dk1);
        const uint32_t off = core_offset(j, kk, kUpdKT) >> 1;
        uint32_t sw[kSlices];
        slice_pairs8(d0, d1, sw);
#pragma unroll
        for (int s = 0; s < kSlices; ++s) *reinterpret_cast<uint32_t *>(dst + s * kTile + off) = sw[s];
    }
}

// ---------------------------------------------------------------- update
// Items (pair, 64-row chunk of G or of V): Out = X W_P in place, computed
// transposed, Out^T = W'^T X'^T: A = W'^T (128 x 128 from k_wprep_x, bulk
// copies per k quarter), B = X' (the chunk's 64 rows, K-major over the panel's
// 128 columns), split per row after balancing.  D is 128 (columns j) x 64 (rows).
// Warp-specialised pipeline over the flat sequence of k-quarter tiles of the
// CTA's items, A and B tiles double-buffered:
//   - warps 1..16 (producers) wait until the products that last read a
//     buffer are done (mbarrier `empty`), start the bulk copy of the A tile
//     and split the B tile (its values loaded while the previous tile was
//     split), then arrive on `full` (two arrivals: the copy's expect-tx and
//     the split); the next item's block is prefetched into L2 one item ahead;
//   - warp 0, lane 0 waits on `full`, issues the 24 products of the tile and
//     commits them to `empty`;
//   - after the producers have filled the first tile of item i + 1, warps
//     1..16 form item i's epilogue (TMEM -> FP64) while warp 0 waits, then
//     warp 0 issues item i + 1's products: the eight accumulators take all of
//     TMEM, so only the epilogue waits for the tensor cores.
// Every wait is bounded; after a failure each role still passes the same
// barriers (no deadlock) and the kernel reports HSVD_ERR_CUDA.
struct UpdItem {
    double *M;
    int64_t ld, rows, r0;
    int pair, which, cI, cJ;
};


__global__ void __launch_bounds__(kThrU, 1)
k_update_x(double *__restrict__ X, int64_t rowsX, int64_t ldx, double *__restrict__ Y, int64_t rowsY, int64_t ldy,
           int npairs, const int *__restrict__ col0, const uint16_t *__restrict__ wsl,
           const int *__restrict__ wexp, const int *__restrict__ dexp, const int *__restrict__ rotated,
           int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr uint32_t kATile = NNX * kUpdKT * 2;       // one slice of W'^T (8 KB)
    constexpr uint32_t kBTile = kUpdRows * kUpdKT * 2;  // one slice of X' (4 KB)
    constexpr uint32_t kABuf = kSlices * kATile, kBBuf = kSlices * kBTile;
    constexpr int kProd = kThrU - 32;                   // producer threads (warps 1..)
    constexpr int kTiles = NNX / kUpdKT;                // k quarters per item
    unsigned char *As = smem;                // two A buffers
    unsigned char *Bs = smem + 2 * kABuf;    // two B buffers
    __shared__ int Erow[2][kUpdRows], Fcol[2][NNX], dk[2][NNX];
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ uint32_t tbase;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t chunksX = (rowsX + kUpdRows - 1) / kUpdRows;
    const int64_t chunks = chunksX + (Y ? (rowsY + kUpdRows - 1) / kUpdRows : 0);
    const int64_t items = (int64_t)npairs * chunks;
    if (tid == 0) {
        s_fail = 0;
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 2);   // the copy's expect-tx arrival and the split's arrival
            mbar_init(&empty[b], 1);  // the products' commit
        }
    }
    if (warp == 0) tmem_alloc(&tbase, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    const uint32_t sbo = (kUpdKT / 8) * 128;
    static_assert(kBTile == (kUpdRows / 8) * (kUpdKT / 8) * 128, "B slices side by side along N");

    auto next_item = [&](int64_t from) -> int64_t {
        for (int64_t it = from; it < items; it += gridDim.x)
            if (rotated[it / chunks]) return it;
        return -1;
    };
    auto describe = [&](int64_t it) {
        UpdItem d;
        d.pair = (int)(it / chunks);
        const int64_t chunk = it % chunks;
        d.which = chunk < chunksX ? 0 : 1;
        d.M = d.which == 0 ? X : Y;
        d.ld = d.which == 0 ? ldx : ldy;
        d.rows = d.which == 0 ? rowsX : rowsY;
        d.r0 = (d.which == 0 ? chunk : chunk - chunksX) * kUpdRows;
        d.cI = col0[2 * d.pair];
        d.cJ = col0[2 * d.pair + 1];
        return d;
    };
    // bounded wait by one thread; the caller follows it with a barrier
    auto wait1 = [&](uint64_t *mb, int64_t use) {
        if (!s_fail && !mbar_wait(mb, (uint32_t)((use >> 1) & 1), kWaitIter)) s_fail = 1;
    };

    // item i's epilogue, warps 1..16: lane j = output column, the four warps
    // of a TMEM lane quarter take rows [16 h2, 16 h2 + 16); glast = the item's
    // last tile.  Warp 0 passes the barriers only.
    auto epilogue = [&](const UpdItem &d, int slot, int64_t glast) {
        if (tid == 0) wait1(&empty[glast & 1], glast);
        bar_named(2, kThrU);
        fence_after();
        if (!s_fail && warp > 0) {
            const int qd = warp & 3, j = 32 * qd + lane, h2 = (warp - 1) >> 2;
            const int jj = j < NNX / 2 ? d.cI + j : d.cJ + j - NNX / 2;
            constexpr int kCols = kN / 4;
            // a thread's values are consecutive rows of one column: stored two
            // at a time (16 B) where the column start allows it
            double *col = d.M + (int64_t)jj * d.ld;
            const bool vec = ((reinterpret_cast<uintptr_t>(col) & 15u) == 0);
            for (int c0 = kCols * h2; c0 < kCols * h2 + kCols; c0 += 4) {
                float v[8][4];
                read_accs4(tmem, 32 * qd, c0, v);
#pragma unroll
                for (int t = 0; t < 4; t += 2) {
                    const int i = c0 + t;
                    const int64_t row = d.r0 + i;
                    float d0[8], d1[8];
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        d0[a] = v[a][t];
                        d1[a] = v[a][t + 1];
                    }
                    const double x0 = combine8_small(d0, Erow[slot][i] + Fcol[slot][j]);
                    const double x1 = combine8_small(d1, Erow[slot][i + 1] + Fcol[slot][j]);
                    if (vec && row + 1 < d.rows) {
                        *reinterpret_cast<double2 *>(col + row) = make_double2(x0, x1);
                    } else {
                        if (row < d.rows) col[row] = x0;
                        if (row + 1 < d.rows) col[row + 1] = x1;
                    }
                }
            }
        }
        fence_before();
        bar_named(2, kThrU);
        fence_after();
    };
    auto epilogue_barriers = [&](int64_t glast) {
        if (tid == 0) wait1(&empty[glast & 1], glast);
        bar_named(2, kThrU);
        fence_after();
        fence_before();
        bar_named(2, kThrU);
        fence_after();
    };

    int64_t g_end = -1;  // last tile of the last item
    if (warp > 0) {
        // ------------------------------------------------ producers
        const int ptid = tid - 32, pw = warp - 1;
        const int rr = lane >> 2, kp = 2 * (lane & 3);
        // a warp splits two 8 x 8 core matrices of a tile: lane -> row rr of
        // the core, k pair kp
        constexpr int kCoresPerWarp = (kUpdRows / 8) * (kUpdKT / 8) / (kProd / 32);
        static_assert(kCoresPerWarp * (kProd / 32) == (kUpdRows / 8) * (kUpdKT / 8), "update split mapping");
        auto colof = [](const UpdItem &d, int k) { return k < NNX / 2 ? d.cI + k : d.cJ + k - NNX / 2; };
        // this lane's 16 values of an item: tile q, core ci, elements k, k + 1
        auto load_item = [&](const UpdItem &d, double (&x)[kTiles][kCoresPerWarp][2]) {
#pragma unroll
            for (int q = 0; q < kTiles; ++q)
#pragma unroll
                for (int ci = 0; ci < kCoresPerWarp; ++ci) {
                    const int core = pw + ci * (kProd / 32);
                    const int i = (core / (kUpdKT / 8)) * 8 + rr, k = q * kUpdKT + (core % (kUpdKT / 8)) * 8 + kp;
                    const int64_t row = d.r0 + i;
                    x[q][ci][0] = row < d.rows ? d.M[row + (int64_t)colof(d, k) * d.ld] : 0.0;
                    x[q][ci][1] = row < d.rows ? d.M[row + (int64_t)colof(d, k + 1) * d.ld] : 0.0;
                }
        };
        // the item's 64 x 128 block into L2: 128 columns x four 128-byte lines
        auto prefetch_item = [&](const UpdItem &d) {
            const int k = ptid >> 2;
            const int64_t row = d.r0 + (ptid & 3) * 16;
            if (row < d.rows) prefetch_l2(d.M + row + (int64_t)colof(d, k) * d.ld);
        };
        int64_t it = next_item(blockIdx.x), itp = -1;
        int ii = 0;
        int64_t g = 0;
        while (it >= 0) {
            const int slot = ii & 1;
            const int64_t itn = next_item(it + gridDim.x);
            const UpdItem cur = describe(it);
            double xv[kTiles][kCoresPerWarp][2];
            load_item(cur, xv);
            if (itn >= 0) prefetch_item(describe(itn));
            for (int k = ptid; k < NNX; k += kProd) {
                dk[slot][k] = cur.which == 0 ? dexp[(size_t)cur.pair * NNX + k] : 0;
                Fcol[slot][k] = wexp[((size_t)cur.pair * 2 + cur.which) * NNX + k];
            }
            if (ptid < kUpdRows) Erow[slot][ptid] = -2000;
            bar_named(1, kProd);
            // row exponents from the loaded values: a lane holds 8 columns of
            // each of its two rows; the four lanes of a row group (same rr)
            // combine by shuffles, and four warps per row by shared atomics
#pragma unroll
            for (int ci = 0; ci < kCoresPerWarp; ++ci) {
                const int core = pw + ci * (kProd / 32);
                const int i = (core / (kUpdKT / 8)) * 8 + rr;
                int ex = -2000;
#pragma unroll
                for (int q = 0; q < kTiles; ++q) {
                    const int k = q * kUpdKT + (core % (kUpdKT / 8)) * 8 + kp;
                    ex = max(ex, exp_bound(xv[q][ci][0]) - dk[slot][k]);
                    ex = max(ex, exp_bound(xv[q][ci][1]) - dk[slot][k + 1]);
                }
                ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, 1));
                ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, 2));
                if ((lane & 3) == 0 && cur.r0 + i < cur.rows) atomicMax(&Erow[slot][i], ex);
            }
            bar_named(1, kProd);
            if (ptid < kUpdRows && Erow[slot][ptid] < -1000) Erow[slot][ptid] = 0;
            bar_named(1, kProd);
#pragma unroll
            for (int q = 0; q < kTiles; ++q, ++g) {
                const int b = (int)(g & 1);
                // the products that last read buffer b (tile g - 2) are done
                if (ptid == 0) {
                    if (g >= 2) wait1(&empty[b], g - 2);
                    if (!s_fail) {
                        mbar_expect_tx(&full[b], kABuf);
                        bulk_g2s(As + b * kABuf,
                                 wsl + (((size_t)cur.pair * 2 + cur.which) * 4 + q) * kSlices * NNX * kUpdKT, kABuf,
                                 &full[b]);
                    }
                }
                bar_named(1, kProd);
                unsigned char *Bb = Bs + b * kBBuf;
#pragma unroll
                for (int ci = 0; ci < kCoresPerWarp; ++ci) {
                    const int core = pw + ci * (kProd / 32);
                    const int i = (core / (kUpdKT / 8)) * 8 + rr, kk = (core % (kUpdKT / 8)) * 8 + kp;
                    const int k = q * kUpdKT + kk;
                    const long long w0 = digit_word(xv[q][ci][0], Erow[slot][i] + dk[slot][k]);
                    const long long w1 = digit_word(xv[q][ci][1], Erow[slot][i] + dk[slot][k + 1]);
                    const uint32_t off = core_offset(i, kk, kUpdKT);
                    uint32_t sw[kSlices];
                    slice_pairs8(w0, w1, sw);
#pragma unroll
                    for (int sl = 0; sl < kSlices; ++sl) *reinterpret_cast<uint32_t *>(Bb + sl * kBTile + off) = sw[sl];
                }
                fence_proxy_async();
                bar_named(1, kProd);
                if (ptid == 0 && !s_fail) mbar_arrive(&full[b]);
                // item ii - 1's epilogue once item ii's first tile is on its way
                if (q == 0 && ii > 0) epilogue(describe(itp), (ii - 1) & 1, g - 1);
            }
            itp = it;
            ++ii;
            it = itn;
        }
        if (ii > 0) epilogue(describe(itp), (ii - 1) & 1, g - 1);
        g_end = g - 1;
    } else {
        // ------------------------------------------------ warp 0: products
        // (warp 0 passes the epilogue's barriers: TMEM is reused after it)
        int64_t it = next_item(blockIdx.x);
        int ii = 0;
        int64_t g = 0;
        while (it >= 0) {
            for (int q = 0; q < kTiles; ++q, ++g) {
                if (q == 0 && ii > 0) epilogue_barriers(g - 1);
                const int b = (int)(g & 1);
                if (lane == 0) {
                    wait1(&full[b], g);
                    if (!s_fail) {
                        fence_after();
                        const uint32_t ab = smem_addr(As + b * kABuf), bb = smem_addr(Bs + b * kBBuf);
                        for (int ks = 0; ks < kUpdKT / 16; ++ks)
                            issue_products(tmem, ab, kATile, bb, kBTile, ks * 256, sbo, q == 0 && ks == 0);
                        commit(&empty[b]);
                    }
                }
                __syncwarp();
            }
            ++ii;
            it = next_item(it + gridDim.x);
        }
        if (ii > 0) epilogue_barriers(g - 1);
        g_end = g - 1;
    }
    __syncthreads();
    if (s_fail && tid == 0) {
        // let the copies and products already issued finish (bounded) before TMEM is freed
        for (int64_t gg = g_end > 1 ? g_end - 1 : 0; gg <= g_end; ++gg) {
            mbar_wait(&full[gg & 1], (uint32_t)((gg >> 1) & 1), kWaitIter);
            mbar_wait(&empty[gg & 1], (uint32_t)((gg >> 1) & 1), kWaitIter);
        }
        if (status) atomicExch(status, HSVD_ERR_CUDA);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// Full 2b x 2b A_P from the split-precision Gram partials (upper triangle,
// exactly symmetric): the kernel-level entry point's assembly.
__global__ void k_assemble_x(const double *__restrict__ part, int ksplit, double *__restrict__ A) {
    const int pair = blockIdx.x;
    for (int e = threadIdx.x; e < NNX * NNX; e += blockDim.x) {
        const int x = e % NNX, y = e / NNX, lo = min(x, y), hi = max(x, y);
        const double *pp = part + (size_t)pair * ksplit * NNX * NNX + lo + (size_t)hi * NNX;
        double v = 0.0;
        for (int s = 0; s < ksplit; ++s) v += pp[(size_t)s * NNX * NNX];
        A[(size_t)pair * NNX * NNX + e] = v;
    }
}

}  // namespace

size_t precision_wsl_elems(int npairs) { return (size_t)npairs * 2 * 4 * kSlices * NNX * kUpdKT; }
int precision_gram_ksplit(int64_t rows) { return (int)((rows + kGramK - 1) / kGramK); }

cudaError_t launch_gram_x(const double *G, int64_t rows, int64_t ldg, int npairs, const int *col0, double *part,
                          int *status, cudaStream_t st) {
    const int ksplit = precision_gram_ksplit(rows);
    const size_t smem = (size_t)kGramBufs * kSlices * (NNX + kN) * kGramKT * 2;
    cudaError_t e = cudaFuncSetAttribute(k_gram_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one CTA per SM: the CTA an SM count later runs in the next wave
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ahead = sms & ~1;
    k_gram_x<<<npairs * ksplit * 2, kThrG, smem, st>>>(G, rows, ldg, col0, ksplit, part, status, ahead);
    return cudaGetLastError();
}

cudaError_t launch_assemble_x(int npairs, const double *part, int ksplit, double *A, cudaStream_t st) {
    k_assemble_x<<<npairs, 256, 0, st>>>(part, ksplit, A);
    return cudaGetLastError();
}

cudaError_t launch_wprep_x(int npairs, const double *Wp, const int *dexp, const int *rotated, uint16_t *wsl,
                           int *wexp, unsigned long long *upd_count, cudaStream_t st) {
    k_wprep_x<<<npairs * 8, kThrX, 0, st>>>(Wp, dexp, rotated, wsl, wexp, upd_count);
    return cudaGetLastError();
}

cudaError_t launch_update_x(double *X, int64_t rowsX, int64_t ldx, double *Y, int64_t rowsY, int64_t ldy,
                            int npairs, const int *col0, const uint16_t *wsl, const int *wexp, const int *dexp,
                            const int *rotated, int *status, cudaStream_t st) {
    // two A tiles (2 x 64 KB) and two B tiles (2 x 32 KB): one CTA per SM, each
    // holding all 512 TMEM columns for its whole life
    const size_t smem = (size_t)2 * kSlices * (NNX + kUpdRows) * kUpdKT * 2;
    static_assert((size_t)2 * kSlices * (NNX + kUpdRows) * kUpdKT * 2 <= (size_t)200 * 1024, "update smem");
    cudaError_t e = cudaFuncSetAttribute(k_update_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t chunks = (rowsX + kUpdRows - 1) / kUpdRows + (Y ? (rowsY + kUpdRows - 1) / kUpdRows : 0);
    const int64_t items = (int64_t)npairs * chunks;
    const unsigned grid = (unsigned)(items < sms ? items : sms);
    k_update_x<<<grid, kThrU, smem, st>>>(X, rowsX, ldx, Y, rowsY, ldy, npairs, col0, wsl, wexp, dexp, rotated,
                                          status);
    return cudaGetLastError();
}

namespace {
// The bounded wait of the tensor-core kernels, run out on purpose: an
// mbarrier that nothing arrives at, waited on for `iters` polls.  out[0] = 1 if
// the wait gave up (the path the kernels take to report HSVD_ERR_CUDA instead
// of hanging), 0 if it completed.
__global__ void k_diag_wait(uint32_t iters, int *out) {
    __shared__ __align__(8) uint64_t mb;
    if (threadIdx.x == 0) mbar_init(&mb, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool done = mbar_wait(&mb, 0, iters);
        out[0] = done ? 0 : 1;
        if (!done) mbar_arrive(&mb);  // complete the phase before the CTA leaves
    }
}
}  // namespace

cudaError_t launch_diag_wait(uint32_t iters, int *out, cudaStream_t st) {
    k_diag_wait<<<1, 32, 0, st>>>(iters, out);
    return cudaGetLastError();
}

}  // namespace hsvd
