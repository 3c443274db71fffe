// precision.cu -- the split-precision form of the blocked method: the pivot
// Gram blocks and the G / V updates as BF16-slice products on the tcgen05
// tensor cores (Ozaki-style splitting), exact FP32 accumulation in tensor
// memory and an exact integer recombination into FP64.  Everything else
// (rotation angles, tanh / cosh, the test of Eq. 2.3, the column norms of the
// finalisation) stays in FP64.  Pivot blocks are 128 x 128 (block width 64).
//
// Splitting (tc.cuh): a row or column of an operand with |x| < 2^E is written
// as 8 balanced base-128 digits, x 2^-E = sum_k q_k 2^(-6-7(k-1)) + r with
// |q_k| <= 64 and |r| < 2^-55; slice k is the exact BF16 number
// q_k 2^(-6-7(k-1)).  The 36 products of slices a, b with a + b <= 9 run on the
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
constexpr int kGramK = 512;          // rows of G per Gram CTA (exactness window)
constexpr int kGramKT = 64;          // rows per shared-memory tile of the Gram
constexpr int kUpdKT = 32;           // k per shared-memory tile of the update
constexpr int kUpdRows = 64;         // rows of G or V per update item (N)
constexpr int kN = 64;               // MMA N
constexpr uint32_t kTmemCols = 512;  // eight accumulators of 64 columns

__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The 36 slice products of one K step (16 k): slice s of A at a_base + s *
// a_stride bytes, of B at b_base + s * b_stride; koff selects the K step.
__device__ __forceinline__ void issue_products(uint32_t tmem, uint32_t a_base, uint32_t a_stride, uint32_t b_base,
                                               uint32_t b_stride, uint32_t koff, uint32_t sbo, uint32_t idesc,
                                               int (&inited)[8]) {
    for (int a = 1; a <= kSlices; ++a)
        for (int b = 1; a + b <= kSlices + 1; ++b) {
            const int acc = a + b - 2;
            const uint64_t da = smem_desc(a_base + (a - 1) * a_stride + koff, 128, sbo);
            const uint64_t db = smem_desc(b_base + (b - 1) * b_stride + koff, 128, sbo);
            mma(tmem + (uint32_t)acc * kN, da, db, idesc, (uint32_t)inited[acc]);
            inited[acc] = 1;
        }
}

// this thread's lane (row of D) and 8 columns [c0, c0+8) of all eight accumulators
__device__ __forceinline__ void read_accs(uint32_t tmem, int lane_base, int c0, float (&v)[8][8]) {
#pragma unroll
    for (int acc = 0; acc < 8; ++acc) tmem_ld8(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(acc * kN + c0), v[acc]);
}

// ---------------------------------------------------------------- Gram
// CTA (pair, split, half): columns [64 h, 64 h + 64) of the partial A_P over
// rows [512 split, 512 split + 512) of the panel P = [G_I G_J] (m x 128).
// A = P^T (128 x K, K-major); B = rows [64 h, 64 h + 64) of the same tile.
__global__ void __launch_bounds__(kThrX, 1)
k_gram_x(const double *__restrict__ G, int64_t rows, int64_t ldg, const int *__restrict__ col0, int ksplit,
         double *__restrict__ part, int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint16_t *sl = reinterpret_cast<uint16_t *>(smem);  // kSlices x (128 x 64)
    __shared__ int Ecol[NNX];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ int s_fail;
    constexpr uint32_t kSliceBytes = NNX * kGramKT * 2;
    const int half = blockIdx.x & 1;
    const int pair = (blockIdx.x >> 1) / ksplit, split = (blockIdx.x >> 1) % ksplit;
    const int64_t r0 = (int64_t)split * kGramK, r1 = min(rows, r0 + kGramK);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cI = col0[2 * pair], cJ = col0[2 * pair + 1];
    for (int c = warp; c < NNX; c += kThrX / 32) {
        const double *g = G + (int64_t)(c < NNX / 2 ? cI + c : cJ + c - NNX / 2) * ldg;
        int e = -2000;
        for (int64_t r = r0 + lane; r < r1; r += 32) e = max(e, exp_bound(g[r]));
        e = warp_max_i(e);
        if (lane == 0) Ecol[c] = e < -1000 ? 0 : e;
    }
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&mbar, 1);
    }
    if (warp == 0) tmem_alloc(&tbase, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    const uint32_t idesc = idesc_bf16(NNX, kN);
    const uint32_t sbo = (kGramKT / 8) * 128;
    const uint32_t b_off = core_offset(kN * half, 0, kGramKT);
    int inited[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t phase = 0;
    for (int64_t t0 = r0; t0 < r1; t0 += kGramKT) {
        for (int e = tid; e < kGramKT * NNX; e += kThrX) {
            const int r = e % kGramKT, c = e / kGramKT;
            const int64_t row = t0 + r;
            const double x = row < r1 ? G[row + (int64_t)(c < NNX / 2 ? cI + c : cJ + c - NNX / 2) * ldg] : 0.0;
            uint16_t s[kSlices];
            split_slices(x, Ecol[c], s);
            const uint32_t off = core_offset(c, r, kGramKT) >> 1;
#pragma unroll
            for (int k = 0; k < kSlices; ++k) sl[k * (NNX * kGramKT) + off] = s[k];
        }
        fence_proxy_async();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            const uint32_t base = smem_addr(sl);
            for (int ks = 0; ks < kGramKT / 16; ++ks)
                issue_products(tmem, base, kSliceBytes, base + b_off, kSliceBytes, ks * 256, sbo, idesc, inited);
            commit(&mbar);
        }
        if (!mbar_wait(&mbar, phase)) atomicExch(&s_fail, 1);
        phase ^= 1;
        fence_after();
        __syncthreads();
        if (s_fail) break;
    }
    if (!s_fail) {
        // lane c = row of A_P; warp group h2 takes TMEM columns [32 h2, 32 h2 + 32)
        const int q = warp & 3, c = 32 * q + lane, h2 = warp >> 2;
        double *out = part + ((size_t)pair * ksplit + split) * NNX * NNX;
        for (int c0 = 32 * h2; c0 < 32 * h2 + 32; c0 += 8) {
            float v[8][8];
            read_accs(tmem, 32 * q, c0, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float d[8];
#pragma unroll
                for (int a = 0; a < 8; ++a) d[a] = v[a][j];
                const int col = kN * half + c0 + j;
                out[c + (size_t)col * NNX] = combine8(d, Ecol[c] + Ecol[col]);
            }
        }
    } else if (tid == 0 && status) {
        atomicExch(status, HSVD_ERR_CUDA);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- W' slices
// One CTA per rotated pair: the A operand of the transposed update, W'^T
// (128 x 128, K-major), for G rows (W' = D W_P) and for V rows (W' = W_P), in
// four k quarters of 32, with per-column exponents F_j.
// wsl layout: [pair][which][quarter][slice][128 x 32 core-matrix tile]
__global__ void __launch_bounds__(kThrX)
k_wprep_x(const double *__restrict__ Wp, const int *__restrict__ dexp, const int *__restrict__ rotated,
          uint16_t *__restrict__ wsl, int *__restrict__ wexp, unsigned long long *__restrict__ upd_count) {
    const int pair = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (!rotated[pair]) return;
    if (tid == 0 && upd_count) atomicAdd(upd_count, 1ull);
    __shared__ int dk[NNX], F[2][NNX];
    const double *W = Wp + (size_t)pair * NNX * NNX;  // W(k, j) at k + j * 128
    for (int k = tid; k < NNX; k += kThrX) dk[k] = dexp[(size_t)pair * NNX + k];
    __syncthreads();
    for (int j = warp; j < NNX; j += kThrX / 32) {
        int e0 = -2000, e1 = -2000;
        for (int k = lane; k < NNX; k += 32) {
            const int e = exp_bound(W[k + (size_t)j * NNX]);
            e0 = max(e0, e + dk[k]);
            e1 = max(e1, e);
        }
        e0 = warp_max_i(e0);
        e1 = warp_max_i(e1);
        if (lane == 0) {
            F[0][j] = e0 < -1000 ? 0 : e0;
            F[1][j] = e1 < -1000 ? 0 : e1;
        }
    }
    __syncthreads();
    for (int e = tid; e < 2 * NNX; e += kThrX) wexp[(size_t)pair * 2 * NNX + e] = F[e / NNX][e % NNX];
    constexpr size_t kTile = (size_t)NNX * kUpdKT;  // elements per slice tile
    for (int e = tid; e < 2 * NNX * NNX; e += kThrX) {
        const int which = e / (NNX * NNX), rem = e % (NNX * NNX);
        const int k = rem % NNX, j = rem / NNX;  // consecutive threads: consecutive k (coalesced reads)
        const double w = W[k + (size_t)j * NNX];
        uint16_t s[kSlices];
        split_slices(w, which == 0 ? F[0][j] - dk[k] : F[1][j], s);
        const int q = k / kUpdKT, kk = k % kUpdKT;
        uint16_t *dst = wsl + (((size_t)pair * 2 + which) * 4 + q) * kSlices * kTile;
        const uint32_t off = core_offset(j, kk, kUpdKT) >> 1;
#pragma unroll
        for (int s_ = 0; s_ < kSlices; ++s_) dst[s_ * kTile + off] = s[s_];
    }
}

// ---------------------------------------------------------------- update
// Items (pair, 64-row chunk of G or of V): Out = X W_P in place, computed
// transposed, Out^T = W'^T X'^T: A = W'^T (128 x 128 from k_wprep_x, bulk
// copies per k quarter), B = X' (the chunk's 64 rows, K-major over the panel's
// 128 columns), split per row after balancing.  D is 128 (columns j) x 64 (rows).
__global__ void __launch_bounds__(kThrX, 1)
k_update_x(double *__restrict__ X, int64_t rowsX, int64_t ldx, double *__restrict__ Y, int64_t rowsY, int64_t ldy,
           int npairs, const int *__restrict__ col0, const uint16_t *__restrict__ wsl,
           const int *__restrict__ wexp, const int *__restrict__ dexp, const int *__restrict__ rotated,
           int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr uint32_t kATile = NNX * kUpdKT * 2;       // one slice of W'^T (8 KB)
    constexpr uint32_t kBTile = kUpdRows * kUpdKT * 2;  // one slice of X' (4 KB)
    uint16_t *As = reinterpret_cast<uint16_t *>(smem);  // kSlices A tiles
    uint16_t *Bs = As + kSlices * NNX * kUpdKT;         // kSlices B tiles
    __shared__ int Erow[kUpdRows], Fcol[NNX], dk[NNX];
    __shared__ __align__(8) uint64_t mbar_a, mbar_m;
    __shared__ uint32_t tbase;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t chunksX = (rowsX + kUpdRows - 1) / kUpdRows;
    const int64_t chunks = chunksX + (Y ? (rowsY + kUpdRows - 1) / kUpdRows : 0);
    const int64_t items = (int64_t)npairs * chunks;
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&mbar_a, 1);
        mbar_init(&mbar_m, 1);
    }
    if (warp == 0) tmem_alloc(&tbase, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    const uint32_t idesc = idesc_bf16(NNX, kN);
    const uint32_t sbo = (kUpdKT / 8) * 128;
    uint32_t phase_a = 0, phase_m = 0;
    for (int64_t item = blockIdx.x; item < items && !s_fail; item += gridDim.x) {
        const int pair = (int)(item / chunks);
        const int64_t chunk = item % chunks;
        if (!rotated[pair]) continue;
        const int which = chunk < chunksX ? 0 : 1;
        double *M = which == 0 ? X : Y;
        const int64_t ld = which == 0 ? ldx : ldy, rows = which == 0 ? rowsX : rowsY;
        const int64_t r0 = (which == 0 ? chunk : chunk - chunksX) * kUpdRows;
        const int cI = col0[2 * pair], cJ = col0[2 * pair + 1];
        for (int k = tid; k < NNX; k += kThrX) {
            dk[k] = which == 0 ? dexp[(size_t)pair * NNX + k] : 0;
            Fcol[k] = wexp[((size_t)pair * 2 + which) * NNX + k];
        }
        if (tid < kUpdRows) Erow[tid] = -2000;
        __syncthreads();
        {   // row exponents of X' = X D^-1 (four threads per row)
            const int i = tid & (kUpdRows - 1), part4 = tid >> 6;
            const int64_t row = r0 + i;
            int e = -2000;
            if (row < rows)
                for (int k = part4 * 32; k < part4 * 32 + 32; ++k) {
                    const int col = k < NNX / 2 ? cI + k : cJ + k - NNX / 2;
                    e = max(e, exp_bound(M[row + (int64_t)col * ld]) - dk[k]);
                }
            atomicMax(&Erow[i], e);
        }
        __syncthreads();
        int inited[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int q = 0; q < NNX / kUpdKT; ++q) {
            if (tid == 0) {
                mbar_expect_tx(&mbar_a, kSlices * kATile);
                bulk_g2s(As, wsl + (((size_t)pair * 2 + which) * 4 + q) * kSlices * NNX * kUpdKT, kSlices * kATile,
                         &mbar_a);
            }
            for (int e = tid; e < kUpdRows * kUpdKT; e += kThrX) {
                const int i = e % kUpdRows, kk = e / kUpdRows, k = q * kUpdKT + kk;
                const int64_t row = r0 + i;
                const int col = k < NNX / 2 ? cI + k : cJ + k - NNX / 2;
                const double x = row < rows ? M[row + (int64_t)col * ld] : 0.0;
                uint16_t s[kSlices];
                split_slices(x, (Erow[i] < -1000 ? 0 : Erow[i]) + dk[k], s);
                const uint32_t off = core_offset(i, kk, kUpdKT) >> 1;
#pragma unroll
                for (int s_ = 0; s_ < kSlices; ++s_) Bs[s_ * (kUpdRows * kUpdKT) + off] = s[s_];
            }
            fence_proxy_async();
            if (!mbar_wait(&mbar_a, phase_a)) atomicExch(&s_fail, 1);
            phase_a ^= 1;
            fence_before();
            __syncthreads();
            fence_after();
            if (s_fail) break;
            if (tid == 0) {
                for (int ks = 0; ks < kUpdKT / 16; ++ks)
                    issue_products(tmem, smem_addr(As), kATile, smem_addr(Bs), kBTile, ks * 256, sbo, idesc, inited);
                commit(&mbar_m);
            }
            if (!mbar_wait(&mbar_m, phase_m)) atomicExch(&s_fail, 1);
            phase_m ^= 1;
            fence_after();
            __syncthreads();
            if (s_fail) break;
        }
        if (s_fail) break;
        {   // epilogue: lane j = output column, warp group h2 = rows [32 h2, 32 h2 + 32)
            const int qd = warp & 3, j = 32 * qd + lane, h2 = warp >> 2;
            const int jj = j < NNX / 2 ? cI + j : cJ + j - NNX / 2;
            for (int c0 = 32 * h2; c0 < 32 * h2 + 32; c0 += 8) {
                float v[8][8];
                read_accs(tmem, 32 * qd, c0, v);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int i = c0 + t;
                    const int64_t row = r0 + i;
                    if (row >= rows) continue;
                    float d[8];
#pragma unroll
                    for (int a = 0; a < 8; ++a) d[a] = v[a][t];
                    M[row + (int64_t)jj * ld] = combine8(d, (Erow[i] < -1000 ? 0 : Erow[i]) + Fcol[j]);
                }
            }
        }
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (s_fail && tid == 0 && status) atomicExch(status, HSVD_ERR_CUDA);
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
    const size_t smem = (size_t)kSlices * NNX * kGramKT * 2;
    cudaError_t e = cudaFuncSetAttribute(k_gram_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_x<<<npairs * ksplit * 2, kThrX, smem, st>>>(G, rows, ldg, col0, ksplit, part, status);
    return cudaGetLastError();
}

cudaError_t launch_assemble_x(int npairs, const double *part, int ksplit, double *A, cudaStream_t st) {
    k_assemble_x<<<npairs, 256, 0, st>>>(part, ksplit, A);
    return cudaGetLastError();
}

cudaError_t launch_wprep_x(int npairs, const double *Wp, const int *dexp, const int *rotated, uint16_t *wsl,
                           int *wexp, unsigned long long *upd_count, cudaStream_t st) {
    k_wprep_x<<<npairs, kThrX, 0, st>>>(Wp, dexp, rotated, wsl, wexp, upd_count);
    return cudaGetLastError();
}

cudaError_t launch_update_x(double *X, int64_t rowsX, int64_t ldx, double *Y, int64_t rowsY, int64_t ldy,
                            int npairs, const int *col0, const uint16_t *wsl, const int *wexp, const int *dexp,
                            const int *rotated, int *status, cudaStream_t st) {
    // 96 KB of operands, requested as 120 KB so that two CTAs never share an
    // SM: each holds all 512 TMEM columns for its whole life
    const size_t smem = (size_t)120 * 1024;
    static_assert((size_t)kSlices * (NNX + kUpdRows) * kUpdKT * 2 <= (size_t)120 * 1024, "update smem");
    cudaError_t e = cudaFuncSetAttribute(k_update_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t chunks = (rowsX + kUpdRows - 1) / kUpdRows + (Y ? (rowsY + kUpdRows - 1) / kUpdRows : 0);
    const int64_t items = (int64_t)npairs * chunks;
    const unsigned grid = (unsigned)(items < sms ? items : sms);
    k_update_x<<<grid, kThrX, smem, st>>>(X, rowsX, ldx, Y, rowsY, ldy, npairs, col0, wsl, wexp, dexp, rotated,
                                          status);
    return cudaGetLastError();
}

}  // namespace hsvd
