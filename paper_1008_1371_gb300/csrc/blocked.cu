// blocked.cu -- one step of the blocked one-sided hyperbolic Jacobi method
// (Sec. 5 block-oriented method, Sec. 6 full-block variant), as three kernels:
//
//   k_gram    A_P = [G_I G_J]^T [G_I G_J] for every block pair of the step
//             (Sec. 2 pivot block, Sec. 5 blocking).  Split over rows into
//             partial blocks so the whole GPU works on the 3 distinct b x b
//             blocks (I,I), (I,J), (J,J) of each pair.  FP64 DFMA register
//             tiles fed from shared memory: on this GPU the FP64 pipe (about
//             2 DFMA per clock per SM) is the bound by two orders of magnitude,
//             and FP64 mma.sync measured slower than DFMA, so neither tensor
//             cores nor TMA staging can help this kernel.
//   (the inner solve of each pair, between the two, is in solve_cluster.cu)
//   k_update  [G_I G_J] <- [G_I G_J] W_P and [V_I V_J] <- [V_I V_J] W_P in
//             place (Eq. 2.1), one CTA per (pair, row chunk), skipped for pairs
//             that did not rotate.
#include "hsvd_internal.cuh"

namespace hsvd {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramKS = 32;  // rows per shared-memory slice

// Partial b x b block C = X^T Y over rows [r0, r1) of the split.
template <int B>
__global__ void __launch_bounds__(kGramThreads)
k_gram(const double *__restrict__ G, int64_t rows, int64_t ldg, int npairs,
       const int *__restrict__ col0, int nsplit, int64_t rows_per, double *__restrict__ part) {
    constexpr int TM = B / 16;  // outputs per thread along each axis
    __shared__ double Xs[kGramKS][B + 1];
    __shared__ double Ys[kGramKS][B + 1];
    const int idx = blockIdx.x;
    const int split = idx % nsplit;
    const int blk = (idx / nsplit) % 3;
    const int pair = idx / (3 * nsplit);
    const int x0 = col0[2 * pair + (blk == 2 ? 1 : 0)];
    const int y0 = col0[2 * pair + (blk >= 1 ? 1 : 0)];
    if (x0 < 0) return;  // a visit the skip mask removed
    const int64_t r0 = (int64_t)split * rows_per;
    const int64_t r1 = min(rows, r0 + rows_per);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = 0.0;

    for (int64_t rb = r0; rb < r1; rb += kGramKS) {
        // coalesced loads: consecutive threads take consecutive rows of a column
        for (int e = tid; e < kGramKS * B; e += kGramThreads) {
            const int r = e % kGramKS, c = e / kGramKS;
            const int64_t row = rb + r;
            const bool in = row < r1;
            Xs[r][c] = in ? G[row + (int64_t)(x0 + c) * ldg] : 0.0;
            Ys[r][c] = in ? G[row + (int64_t)(y0 + c) * ldg] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < kGramKS; ++r) {
            double a[TM], b[TM];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = Xs[r][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < TM; ++j) b[j] = Ys[r][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *out = part + (size_t)idx * B * B;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) out[(tx + 16 * i) + (size_t)(ty + 16 * j) * B] = acc[i][j];
}

template <int NN>
__global__ void __launch_bounds__(256)
k_assemble(const double *__restrict__ part, int nsplit, double *__restrict__ A) {
    for (int e = threadIdx.x; e < NN * NN; e += 256)
        A[(size_t)blockIdx.x * NN * NN + e] = assemble_entry<NN>(part, nsplit, blockIdx.x, e);
}

constexpr int kUpdThreads = 256;
constexpr int kUpdRows = 32;

// Out[R x NN] = X[R x NN] * W_P for one row chunk of a block-column pair, in
// place.  Thread (r = tid % 32, g = tid / 32) computes row r, columns g + 8j.
// W_P is streamed through shared memory in column tiles of at most 64.  The
// kernel is bound by the FP64 pipe of each SM, so the CTAs loop over
// (pair, 32-row chunk) items: every SM gets the same number of items, within
// one, whatever the grid.
template <int NN>
__global__ void __launch_bounds__(kUpdThreads, 4)
k_update(double *__restrict__ X, int64_t rowsX, int64_t ldx, double *__restrict__ Y, int64_t rowsY,
         int64_t ldy, int npairs, const int *__restrict__ col0, const double *__restrict__ Wp,
         const int *__restrict__ rotated, unsigned long long *__restrict__ upd_count) {
    constexpr int B = NN / 2;
    constexpr int CT = NN < 64 ? NN : 64;  // output column tile
    constexpr int PER = CT / 8;
    extern __shared__ __align__(16) double sm[];
    double *Xs = sm;                 // [NN][kUpdRows]
    double *Ws = Xs + NN * kUpdRows;  // [NN][CT]
    const int64_t chunksX = (rowsX + kUpdRows - 1) / kUpdRows;
    const int64_t chunksY = Y ? (rowsY + kUpdRows - 1) / kUpdRows : 0;
    const int64_t chunks = chunksX + chunksY;
    const int64_t items = (int64_t)npairs * chunks;
    const int tid = threadIdx.x, r = tid % kUpdRows, g = tid / kUpdRows;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int pair = (int)(item / chunks);
        const int64_t chunk = item % chunks;
        if (!rotated[pair]) continue;
        double *M;
        int64_t ld, rows, r0;
        if (chunk < chunksX) { M = X; ld = ldx; rows = rowsX; r0 = chunk * kUpdRows; }
        else { M = Y; ld = ldy; rows = rowsY; r0 = (chunk - chunksX) * kUpdRows; }
        const int cI = col0[2 * pair], cJ = col0[2 * pair + 1];
        __syncthreads();  // previous item done with Xs / Ws
        for (int e = tid; e < NN * kUpdRows; e += kUpdThreads) {
            const int rr = e % kUpdRows, k = e / kUpdRows;
            const int64_t row = r0 + rr;
            const int col = (k < B) ? (cI + k) : (cJ + k - B);
            Xs[k * kUpdRows + rr] = row < rows ? M[row + (int64_t)col * ld] : 0.0;
        }
        const double *Wpp = Wp + (size_t)pair * NN * NN;
        const int64_t row = r0 + r;
        for (int c0 = 0; c0 < NN; c0 += CT) {
            __syncthreads();
            for (int e = tid; e < NN * CT; e += kUpdThreads) {
                const int cc = e % CT, k = e / CT;
                Ws[k * CT + cc] = Wpp[k + (size_t)(c0 + cc) * NN];
            }
            __syncthreads();
            double acc[PER];
#pragma unroll
            for (int j = 0; j < PER; ++j) acc[j] = 0.0;
#pragma unroll 8
            for (int k = 0; k < NN; ++k) {
                const double a = Xs[k * kUpdRows + r];
#pragma unroll
                for (int j = 0; j < PER; ++j) acc[j] = fma(a, Ws[k * CT + g + 8 * j], acc[j]);
            }
            if (row < rows) {
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    const int oc = c0 + g + 8 * j;
                    const int col = (oc < B) ? (cI + oc) : (cJ + oc - B);
                    M[row + (int64_t)col * ld] = acc[j];
                }
            }
        }
        if (upd_count && tid == 0 && chunk == 0) atomicAdd(upd_count, 1ull);
    }
}

template <int NN>
size_t update_smem() {
    constexpr int CT = NN < 64 ? NN : 64;
    return ((size_t)NN * kUpdRows + (size_t)NN * CT) * sizeof(double);
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    }
    return sms;
}

template <int NN>
cudaError_t update_impl(double *X, int64_t rowsX, int64_t ldx, double *Y, int64_t rowsY, int64_t ldy,
                        int npairs, const int *col0, const double *Wp, const int *rotated,
                        unsigned long long *upd_count, cudaStream_t st) {
    const size_t smem = update_smem<NN>();
    cudaError_t e = cudaFuncSetAttribute(k_update<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update<NN>, kUpdThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t chunks = (rowsX + kUpdRows - 1) / kUpdRows + (Y ? (rowsY + kUpdRows - 1) / kUpdRows : 0);
    const int64_t items = (int64_t)npairs * chunks;
    const int64_t slots = (int64_t)num_sms() * (per_sm < 1 ? 1 : per_sm);
    const unsigned grid = (unsigned)(items < slots ? items : slots);
    k_update<NN><<<grid, kUpdThreads, smem, st>>>(X, rowsX, ldx, Y, rowsY, ldy, npairs, col0, Wp, rotated,
                                                  upd_count);
    return cudaGetLastError();
}

}  // namespace

int gram_nsplit(int64_t rows, int npairs) {
    // The kernel is bound by the FP64 pipe of each SM, so what matters is an
    // even number of work items per SM: at most one resident wave (4 CTAs per
    // SM), at least 32 rows per item.  The row split fixes the order of the
    // partial sums, so results are reproducible on one GPU model.
    const int64_t slots = 4 * (int64_t)num_sms();
    int64_t s = slots / (3 * (int64_t)npairs);
    const int64_t maxs = (rows + 31) / 32;
    if (s > maxs) s = maxs;
    return (int)(s < 1 ? 1 : s);
}

cudaError_t launch_gram(const double *G, int64_t rows, int64_t ldg, int b, int npairs, const int *col0,
                        int nsplit, double *part, cudaStream_t st) {
    int64_t rows_per = (rows + nsplit - 1) / nsplit;
    rows_per = (rows_per + 7) / 8 * 8;
    const unsigned grid = (unsigned)(npairs * 3 * nsplit);
    switch (b) {
        case 16: k_gram<16><<<grid, kGramThreads, 0, st>>>(G, rows, ldg, npairs, col0, nsplit, rows_per, part); break;
        case 32: k_gram<32><<<grid, kGramThreads, 0, st>>>(G, rows, ldg, npairs, col0, nsplit, rows_per, part); break;
        case 64: k_gram<64><<<grid, kGramThreads, 0, st>>>(G, rows, ldg, npairs, col0, nsplit, rows_per, part); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_assemble(int b, int npairs, const double *part, int nsplit, double *A, cudaStream_t st) {
    switch (b) {
        case 16: k_assemble<32><<<npairs, 256, 0, st>>>(part, nsplit, A); break;
        case 32: k_assemble<64><<<npairs, 256, 0, st>>>(part, nsplit, A); break;
        case 64: k_assemble<128><<<npairs, 256, 0, st>>>(part, nsplit, A); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_update(double *X, int64_t rows, int64_t ldx, double *Y, int64_t rowsY, int64_t ldy, int b,
                          int npairs, const int *col0, const double *Wp, const int *rotated,
                          unsigned long long *upd_count, cudaStream_t st) {
    switch (b) {
        case 16: return update_impl<32>(X, rows, ldx, Y, rowsY, ldy, npairs, col0, Wp, rotated, upd_count, st);
        case 32: return update_impl<64>(X, rows, ldx, Y, rowsY, ldy, npairs, col0, Wp, rotated, upd_count, st);
        case 64: return update_impl<128>(X, rows, ldx, Y, rowsY, ldy, npairs, col0, Wp, rotated, upd_count, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hsvd
