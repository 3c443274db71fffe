// qr.cu -- the shortening front end for tall factors (Sec. 1): G = Q R by
// Householder reflections, the HSVD of the square R, and U = Q [U_R; 0].
// R V = U_R Sigma gives G V = Q R V = (Q [U_R; 0]) Sigma with the same J-unitary
// V, and Householder QR is column-wise backward stable, so relative accuracy
// for column-scaled factors carries over.  One sweep of the blocked method on
// the m x n factor costs 2 n^2 (4m + 2n) flops, on R 12 n^3; the QR and the
// application of Q cost about 4 m n^2 once.
//
// Blocked QR with panels of width kQB (compact WY form, H_1 ... H_w =
// I - V T V^T, T upper triangular):
//   k_qr_panel   factors one panel column by column (reflector as in LAPACK's
//                dlarfg: beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta,
//                v = x / (alpha - beta) below the unit diagonal).  One CTA.
//   k_qr_vtc     partial products V^T C over row splits (C: the trailing
//                columns, V itself for T, or U when Q is applied).
//   k_qr_tbuild  T from tau and V^T V (T_jj = tau_j,
//                T_{0:j,j} = -tau_j T_{0:j,0:j} V_{:,0:j}^T v_j): the partials
//                summed by one thread per entry, the recurrence by one warp.
//   k_qr_tz      Z = op(T) (sum of the partials): op = T^T for the
//                factorisation (Q^T C), T for applying Q.
//   k_qr_update  C -= V Z.
// Every product is an FP64 FMA chain (the library is compiled without
// floating-point contraction).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "hsvd_internal.cuh"

namespace cg = cooperative_groups;

namespace hsvd {
namespace {

constexpr int kQB = 32;         // panel width
constexpr int kPanelThreads = 256;
constexpr int kVtcThreads = 256;
constexpr int kVtcRows = 32;    // rows per shared-memory slice

// V's entry (i, a) for the panel starting at column j0: zero above the
// diagonal, one on it, the stored reflector below
__device__ __forceinline__ double v_entry(const double *__restrict__ A, int64_t lda, int64_t i, int j0, int a) {
    const int64_t d = (int64_t)j0 + a;
    if (i < d) return 0.0;
    if (i == d) return 1.0;
    return A[i + d * lda];
}

// One CTA factors columns j0 .. j0 + w - 1 of A over rows j0 .. m - 1.  For
// column j: one pass forms x^T x and x^T a_c over the rows below j for the
// later panel columns c, a block reduction gives beta, tau and w_c = v^T a_c,
// and a second pass stores v and updates the later columns.
__global__ void __launch_bounds__(kPanelThreads)
k_qr_panel(double *__restrict__ A, int64_t lda, int64_t m, int j0, int w, double *__restrict__ tau) {
    __shared__ double red[kPanelThreads / 32][kQB];
    __shared__ double sw[kQB];   // w_c of the current column
    __shared__ double s_scale, s_tau;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int jj = 0; jj < w; ++jj) {
        const int64_t j = (int64_t)j0 + jj;
        const double *x = A + j * lda;
        // pass A: acc[0] = sum x_i^2, acc[c] = sum x_i a_{i, j + c} (rows i > j)
        double acc[kQB];
#pragma unroll
        for (int c = 0; c < kQB; ++c) acc[c] = 0.0;
        for (int64_t i = j + 1 + tid; i < m; i += kPanelThreads) {
            const double xi = x[i];
            double val[kQB];
#pragma unroll
            for (int c = 1; c < kQB; ++c)
                if (jj + c < w) val[c] = A[i + (j + c) * lda];
            acc[0] = fma(xi, xi, acc[0]);
#pragma unroll
            for (int c = 1; c < kQB; ++c)
                if (jj + c < w) acc[c] = fma(xi, val[c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < kQB; ++c) {
            double v = acc[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][c] = v;
        }
        __syncthreads();
        if (tid < kQB) {
            double s = 0.0;
            for (int q = 0; q < kPanelThreads / 32; ++q) s += red[q][tid];
            red[0][tid] = s;  // warp 0's row is read only below, after the barrier
        }
        __syncthreads();
        if (tid == 0) {
            const double alpha = x[j], xnorm2 = red[0][0];
            double t = 0.0, scale = 0.0, beta = alpha;
            if (xnorm2 > 0.0) {
                beta = -copysign(sqrt(fma(alpha, alpha, xnorm2)), alpha);
                t = (beta - alpha) / beta;
                scale = 1.0 / (alpha - beta);
            }
            s_tau = t;
            s_scale = scale;
            tau[j] = t;
            A[j + j * lda] = beta;
        }
        __syncthreads();
        const double t = s_tau, scale = s_scale;
        if (tid > 0 && tid < kQB && jj + tid < w) {
            const int c = tid;  // w_c = a_{j, j+c} + scale * sum_{i>j} x_i a_{i, j+c}
            sw[c] = fma(scale, red[0][c], A[j + (j + c) * lda]);
        }
        __syncthreads();
        // pass B: v below the diagonal, then a_c -= tau w_c v for the later
        // columns; a row's loads are all issued before its stores
        double *xm = A + j * lda;
        for (int64_t i = j + 1 + tid; i < m; i += kPanelThreads) {
            const double vi = xm[i] * scale;
            double val[kQB];
#pragma unroll
            for (int c = 1; c < kQB; ++c)
                if (jj + c < w) val[c] = A[i + (j + c) * lda];
            xm[i] = vi;
#pragma unroll
            for (int c = 1; c < kQB; ++c)
                if (jj + c < w) A[i + (j + c) * lda] = fma(-t * sw[c], vi, val[c]);
        }
        if (tid > 0 && tid < kQB && jj + tid < w) {  // row j: v_j = 1
            double *ac = A + (j + tid) * lda;
            ac[j] = fma(-t, sw[tid], ac[j]);
        }
        __syncthreads();
    }
}

// The same panel factorisation on a cluster of kPanelCl CTAs that keep the
// panel in shared memory: CTA r holds rows j0 + r rp .. j0 + (r+1) rp - 1
// (column-major, stride rp).  Per column, every CTA reduces its rows' part of
// x^T x and x^T a_c and writes it, with the diagonal row when it owns it, into
// every CTA (double-buffered by column parity); after one cluster barrier
// every CTA sums the same partials in the same order, forms beta, tau, w_c
// itself and updates its own rows.  The panel goes back to A at the end.
constexpr int kPanelCl = 16;
constexpr int kPanelClMaxRows = 832;  // rows per CTA kept in shared memory: 32 x 832 doubles = 208 KB

// Sum over the warp of 32 per-lane values v[0..31]; lane l receives the sum of
// v[l] (a butterfly that halves the values a lane carries at each level: 31
// shuffles instead of 32 x 5).
__device__ __forceinline__ double warp_transpose_sum(double (&v)[kQB], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool hi = lane & o;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const double send = hi ? v[i] : v[i + o];
            const double keep = hi ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// The same panel factorisation on a cluster of kPanelCl CTAs: CTA r owns rows
// j0 + r rp .. j0 + (r+1) rp - 1, kept in shared memory (column-major, stride
// rp) when SMEM, else worked on in place in A.  Per column, every CTA reduces
// its rows' part of x^T x and x^T a_c and writes it, with the diagonal row
// when it owns it, into every CTA (double-buffered by column parity); after
// one cluster barrier every CTA sums the same partials in the same order,
// forms beta, tau, w_c itself and updates its own rows.
template <bool SMEM>
__global__ void __launch_bounds__(kPanelThreads)
k_qr_panel_cl(double *__restrict__ A, int64_t lda, int64_t m, int j0, int w, int rp, double *__restrict__ tau) {
    extern __shared__ __align__(16) double P[];  // [kQB][rp] when SMEM
    __shared__ double red[2][kPanelCl][kQB];     // partial sums from every CTA
    __shared__ double drow[2][kQB];              // the diagonal row of the column
    __shared__ double wred[kPanelThreads / 32][kQB];
    __shared__ double s_beta, s_tau, s_scale, sw[kQB];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = (int64_t)j0 + (int64_t)rank * rp;
    const int64_t left = m - row0;
    const int nrows = left <= 0 ? 0 : (left < rp ? (int)left : rp);
    double *const Ab = A + row0 + (int64_t)j0 * lda;
    auto at = [&](int c, int i) -> double & { return SMEM ? P[c * rp + i] : Ab[i + (int64_t)c * lda]; };
    if (SMEM)
        for (int e = tid; e < kQB * rp; e += kPanelThreads) {
            const int c = e / rp, i = e % rp;
            P[e] = (c < w && i < nrows) ? Ab[i + (int64_t)c * lda] : 0.0;
        }
    cluster.sync();  // every CTA loaded and running before any remote write
    for (int jj = 0; jj < w; ++jj) {
        const int buf = jj & 1;
        // local rows strictly below the diagonal row j0 + jj
        const int64_t below = (int64_t)j0 + jj + 1 - row0;
        const int first = below <= 0 ? 0 : (below < rp ? (int)below : rp);
        double acc[kQB];
#pragma unroll
        for (int c = 0; c < kQB; ++c) acc[c] = 0.0;
        for (int i = first + tid; i < nrows; i += kPanelThreads) {
            const double x = at(jj, i);
#pragma unroll
            for (int c = 0; c < kQB; ++c)
                if (c >= jj && c < w) acc[c] = fma(x, at(c, i), acc[c]);
        }
        const double mine = warp_transpose_sum(acc, lane);  // this warp's sum for column `lane`
        wred[warp][lane] = mine;
        __syncthreads();
        const int64_t dl = (int64_t)j0 + jj - row0;  // the diagonal row, local index
        const bool own_diag = dl >= 0 && dl < nrows;
        if (tid < kQB) {
            double ssum = 0.0;
            for (int q = 0; q < kPanelThreads / 32; ++q) ssum += wred[q][tid];
            const double dv = own_diag ? at(tid, (int)dl) : 0.0;
            for (int r = 0; r < kPanelCl; ++r) {
                *cluster.map_shared_rank(&red[buf][rank][tid], r) = ssum;
                if (own_diag) *cluster.map_shared_rank(&drow[buf][tid], r) = dv;
            }
        }
        cluster.sync();
        // every CTA: the same sums in the same order
        if (tid < kQB) {
            double tot = 0.0;
            for (int r = 0; r < kPanelCl; ++r) tot += red[buf][r][tid];
            wred[0][tid] = tot;
        }
        __syncthreads();
        if (tid == 0) {
            const double alpha = drow[buf][jj], xnorm2 = wred[0][jj];
            double t = 0.0, scale = 0.0, beta = alpha;
            if (xnorm2 > 0.0) {
                beta = -copysign(sqrt(fma(alpha, alpha, xnorm2)), alpha);
                t = (beta - alpha) / beta;
                scale = 1.0 / (alpha - beta);
            }
            s_beta = beta;
            s_tau = t;
            s_scale = scale;
            if (rank == 0) tau[j0 + jj] = t;
        }
        if (tid > jj && tid < w) sw[tid] = wred[0][tid];  // the dot; w_c is formed after the barrier
        __syncthreads();
        const double t = s_tau, scale = s_scale;
        if (tid > jj && tid < w) sw[tid] = fma(scale, sw[tid], drow[buf][tid]);
        __syncthreads();
        for (int i = first + tid; i < nrows; i += kPanelThreads) {
            const double v = at(jj, i) * scale;
            if constexpr (SMEM) {
                at(jj, i) = v;
#pragma unroll
                for (int c = 0; c < kQB; ++c)
                    if (c > jj && c < w) at(c, i) = fma(-t * sw[c], v, at(c, i));
            } else {  // global memory: a row's loads are all issued before its stores
                double val[kQB];
#pragma unroll
                for (int c = 0; c < kQB; ++c)
                    if (c > jj && c < w) val[c] = at(c, i);
                at(jj, i) = v;
#pragma unroll
                for (int c = 0; c < kQB; ++c)
                    if (c > jj && c < w) at(c, i) = fma(-t * sw[c], v, val[c]);
            }
        }
        if (own_diag) {
            if (tid == 0) at(jj, (int)dl) = s_beta;
            if (tid > jj && tid < w) at(tid, (int)dl) = fma(-t, sw[tid], at(tid, (int)dl));
        }
        __syncthreads();
    }
    if (SMEM)
        for (int e = tid; e < kQB * rp; e += kPanelThreads) {
            const int c = e / rp, i = e % rp;
            if (c < w && i < nrows) Ab[i + (int64_t)c * lda] = P[e];
        }
    cluster.sync();  // no CTA leaves while another may still read its partials
}

// part[s][a][c] = sum over the rows of split s (from j0 on) of V(i, a) C(i, c0 + c),
// a < w, c < ncols; C is V itself (c_is_v) or a plain matrix.
__global__ void __launch_bounds__(kVtcThreads)
k_qr_vtc(const double *__restrict__ A, int64_t lda, int64_t m, int j0, int w, const double *__restrict__ C,
         int64_t ldc, int c0, int ncols, int c_is_v, int nsplit, int64_t rows_per, double *__restrict__ part) {
    __shared__ double Vs[kVtcRows][kQB + 1];
    __shared__ double Cs[kVtcRows][kQB + 1];
    const int tile = blockIdx.x, split = blockIdx.y;
    const int ct0 = tile * kQB;
    const int64_t r0 = (int64_t)j0 + (int64_t)split * rows_per;
    const int64_t r1 = m < r0 + rows_per ? m : r0 + rows_per;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t rb = r0; rb < r1; rb += kVtcRows) {
        for (int e = tid; e < kVtcRows * kQB; e += kVtcThreads) {
            const int rr = e % kVtcRows, k = e / kVtcRows;
            const int64_t i = rb + rr;
            const bool in = i < r1;
            Vs[rr][k] = (in && k < w) ? v_entry(A, lda, i, j0, k) : 0.0;
            const int c = ct0 + k;
            double cv = 0.0;
            if (in && c < ncols) cv = c_is_v ? v_entry(A, lda, i, j0, c) : C[i + (int64_t)(c0 + c) * ldc];
            Cs[rr][k] = cv;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kVtcRows; ++rr) {
            const double v0 = Vs[rr][ty], v1 = Vs[rr][ty + 16];
            const double x0 = Cs[rr][tx], x1 = Cs[rr][tx + 16];
            acc[0][0] = fma(v0, x0, acc[0][0]);
            acc[0][1] = fma(v0, x1, acc[0][1]);
            acc[1][0] = fma(v1, x0, acc[1][0]);
            acc[1][1] = fma(v1, x1, acc[1][1]);
        }
        __syncthreads();
    }
    double *pp = part + (size_t)split * kQB * ncols;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int a = ty + 16 * u, c = ct0 + tx + 16 * v;
            if (a < w && c < ncols) pp[(size_t)a * ncols + c] = acc[u][v];
        }
}

// T of the panel from tau and Y = V^T V (the sum of the partials), one warp:
// lane r holds row r of T; column j is formed from column j of Y.
__global__ void __launch_bounds__(kQB * kQB)
k_qr_tbuild(const double *__restrict__ part, int nsplit, int w, const double *__restrict__ tau_j0,
            double *__restrict__ T) {
    __shared__ double Ts[kQB][kQB + 1];
    __shared__ double Y[kQB][kQB + 1];
    // every entry of Y = V^T V (the sum of the partials) by its own thread
    {
        const int a = threadIdx.x / kQB, c = threadIdx.x % kQB;
        double s = 0.0;
        if (a < w && c < w)
            for (int q = 0; q < nsplit; ++q) s += part[(size_t)q * kQB * w + (size_t)a * w + c];
        Y[a][c] = s;
        Ts[a][c] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int r = threadIdx.x;
    for (int j = 0; j < w; ++j) {
        const double tj = tau_j0[j];
        if (r < j) {  // T_{r,j} = -tau_j sum_{k=r}^{j-1} T_{r,k} y_k, y_k = v_k^T v_j
            double s = 0.0;
            for (int k = r; k < j; ++k) s = fma(Ts[r][k], Y[k][j], s);
            Ts[r][j] = -tj * s;
        }
        if (r == j) Ts[r][j] = tj;
        __syncwarp();
    }
    for (int c = 0; c < kQB; ++c) T[r * kQB + c] = Ts[r][c];
}

// Z[a][c] = sum_b op(T)[a][b] X[b][c], X the sum of the partials; op = T^T
// when trans (the factorisation applies H^T), T otherwise (Q applied).
__global__ void k_qr_tz(const double *__restrict__ part, int nsplit, int w, int ncols, const double *__restrict__ T,
                        int trans, double *__restrict__ Z) {
    __shared__ double Xs[kQB][kQB + 1];
    __shared__ double Ts[kQB][kQB + 1];
    const int ct0 = blockIdx.x * kQB, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int a = ty; a < kQB; a += 8) {
        const int c = ct0 + tx;
        double s = 0.0;
        if (a < w && c < ncols)
            for (int q = 0; q < nsplit; ++q) s += part[(size_t)q * kQB * ncols + (size_t)a * ncols + c];
        Xs[a][tx] = s;
        Ts[a][tx] = T[a * kQB + tx];
    }
    __syncthreads();
    for (int a = ty; a < w; a += 8) {
        const int c = ct0 + tx;
        if (c >= ncols) continue;
        double s = 0.0;
        for (int b = 0; b < w; ++b) s = fma(trans ? Ts[b][a] : Ts[a][b], Xs[b][tx], s);
        Z[(size_t)a * ncols + c] = s;
    }
}

// C(i, c0 + c) -= sum_a V(i, a) Z[a][c] for rows i >= j0; one CTA per (row
// chunk of 64, column tile of 32)
__global__ void __launch_bounds__(256)
k_qr_update(double *__restrict__ C, int64_t ldc, int64_t m, int c0, int ncols, const double *__restrict__ A,
            int64_t lda, int j0, int w, const double *__restrict__ Z) {
    __shared__ double Vs[kQB][64];
    __shared__ double Zs[kQB][kQB];
    const int64_t r0 = (int64_t)j0 + (int64_t)blockIdx.x * 64;
    const int ct0 = blockIdx.y * kQB;
    const int tid = threadIdx.x;
    for (int e = tid; e < kQB * 64; e += 256) {
        const int a = e / 64, rr = e % 64;
        const int64_t i = r0 + rr;
        Vs[a][rr] = (i < m && a < w) ? v_entry(A, lda, i, j0, a) : 0.0;
    }
    for (int e = tid; e < kQB * kQB; e += 256) {
        const int a = e / kQB, c = e % kQB;
        Zs[a][c] = (a < w && ct0 + c < ncols) ? Z[(size_t)a * ncols + ct0 + c] : 0.0;
    }
    __syncthreads();
    const int rr = tid & 63, cg = tid >> 6;  // 64 rows x 4 column groups of 8
    const int64_t i = r0 + rr;
    if (i >= m) return;
    double s[8], old[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = 0.0;
    for (int a = 0; a < w; ++a) {
        const double v = Vs[a][rr];
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] = fma(v, Zs[a][cg * 8 + k], s[k]);
    }
    // every load before any store (the columns of C are disjoint)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int c = ct0 + cg * 8 + k;
        old[k] = c < ncols ? C[i + (int64_t)(c0 + c) * ldc] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int c = ct0 + cg * 8 + k;
        if (c < ncols) C[i + (int64_t)(c0 + c) * ldc] = old[k] - s[k];
    }
}

// the panel on a 16-CTA cluster: rows in shared memory when they fit, else in
// place in A
template <bool SMEM>
cudaError_t launch_panel_cl(double *A, int64_t lda, int64_t m, int j0, int w, int rp, double *tau, cudaStream_t st) {
    const size_t smem = SMEM ? (size_t)kQB * rp * sizeof(double) : 0;
    cudaError_t e = cudaFuncSetAttribute(k_qr_panel_cl<SMEM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_qr_panel_cl<SMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kPanelCl);
    cfg.blockDim = dim3(kPanelThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kPanelCl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;  // launch only what the GPU can hold at once
    e = cudaOccupancyMaxActiveClusters(&clusters, k_qr_panel_cl<SMEM>, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    return cudaLaunchKernelEx(&cfg, k_qr_panel_cl<SMEM>, A, lda, m, j0, w, rp, tau);
}

cudaError_t panel_cluster(double *A, int64_t lda, int64_t m, int j0, int w, double *tau, cudaStream_t st) {
    const int64_t L = m - j0;
    const int rp = (int)((L + kPanelCl - 1) / kPanelCl);
    if (L < 2 * kPanelCl) return cudaErrorInvalidValue;
    return rp <= kPanelClMaxRows ? launch_panel_cl<true>(A, lda, m, j0, w, rp, tau, st)
                                 : launch_panel_cl<false>(A, lda, m, j0, w, rp, tau, st);
}

int qr_nsplit(int64_t rows) {
    const int64_t s = (rows + 255) / 256;  // at least 256 rows per split
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, 64));
}

// Applies H_panel^T (trans) or H_panel to columns c0 .. c0 + ncols - 1 of C,
// in chunks of kMaxCols columns (workspace: part, Z).
constexpr int kMaxCols = 2048;
cudaError_t apply_panel(double *A, int64_t lda, int64_t m, int j0, int w, const double *T, int trans, double *C,
                        int64_t ldc, int c0, int ncols, double *part, double *Z, cudaStream_t st) {
    const int64_t rows = m - j0;
    const int nsplit = qr_nsplit(rows);
    const int64_t rows_per = (rows + nsplit - 1) / nsplit;
    for (int cb = 0; cb < ncols; cb += kMaxCols) {
        const int nc = std::min(kMaxCols, ncols - cb);
        const dim3 g1((nc + kQB - 1) / kQB, nsplit);
        k_qr_vtc<<<g1, kVtcThreads, 0, st>>>(A, lda, m, j0, w, C, ldc, c0 + cb, nc, 0, nsplit, rows_per, part);
        k_qr_tz<<<(nc + kQB - 1) / kQB, 256, 0, st>>>(part, nsplit, w, nc, T, trans, Z);
        const dim3 g2((unsigned)((rows + 63) / 64), (nc + kQB - 1) / kQB);
        k_qr_update<<<g2, 256, 0, st>>>(C, ldc, m, c0 + cb, nc, A, lda, j0, w, Z);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t qr_workspace_doubles(int64_t n) {
    const int64_t panels = (n + kQB - 1) / kQB;
    const int64_t cols = std::min<int64_t>(n, kMaxCols);  // widest column chunk
    return (size_t)panels * kQB * kQB             // T of every panel
           + (size_t)n                            // tau
           + (size_t)64 * kQB * cols              // partials (at most 64 row splits)
           + (size_t)kQB * cols;                  // Z
}

namespace {
// R (n x n, ldr) <- the upper triangle of A, zeros below; U (m x n, ldu) <-
// [U_R; 0] from U_R (n x n, ldur)
__global__ void k_qr_extract_r(const double *__restrict__ A, int64_t lda, int64_t n, double *__restrict__ R,
                               int64_t ldr) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e % n, j = e / n;
    R[i + j * ldr] = i <= j ? A[i + j * lda] : 0.0;
}
__global__ void k_qr_embed_u(const double *__restrict__ UR, int64_t ldur, int64_t m, int64_t n,
                             double *__restrict__ U, int64_t ldu) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * n) return;
    const int64_t i = e % m, j = e / m;
    U[i + j * ldu] = i < n ? UR[i + j * ldur] : 0.0;
}
}  // namespace

cudaError_t qr_extract_r(const double *A, int64_t lda, int64_t n, double *R, int64_t ldr, cudaStream_t st) {
    const int64_t total = n * n;
    k_qr_extract_r<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(A, lda, n, R, ldr);
    return cudaGetLastError();
}

cudaError_t qr_embed_u(const double *UR, int64_t ldur, int64_t m, int64_t n, double *U, int64_t ldu,
                       cudaStream_t st) {
    const int64_t total = m * n;
    k_qr_embed_u<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(UR, ldur, m, n, U, ldu);
    return cudaGetLastError();
}

// A (m x n, lda) <- R in the upper triangle and the reflectors below it; T of
// every panel into ws.  m >= n.
cudaError_t qr_factor(double *A, int64_t lda, int64_t m, int64_t n, double *ws, cudaStream_t st,
                      long long *launches) {
    const int64_t panels = (n + kQB - 1) / kQB;
    double *Tall = ws, *tau = Tall + (size_t)panels * kQB * kQB;
    double *part = tau + n, *Z = part + (size_t)64 * kQB * std::min<int64_t>(n, kMaxCols);
    for (int64_t p = 0; p < panels; ++p) {
        const int j0 = (int)(p * kQB), w = (int)std::min<int64_t>(kQB, n - j0);
        double *T = Tall + (size_t)p * kQB * kQB;
        if (panel_cluster(A, lda, m, j0, w, tau, st) != cudaSuccess) {
            cudaGetLastError();  // clear a refused cluster launch; the one-CTA kernel does the panel
            k_qr_panel<<<1, kPanelThreads, 0, st>>>(A, lda, m, j0, w, tau);
        }
        // T from V^T V
        const int64_t rows = m - j0;
        const int nsplit = qr_nsplit(rows);
        const int64_t rows_per = (rows + nsplit - 1) / nsplit;
        k_qr_vtc<<<dim3(1, nsplit), kVtcThreads, 0, st>>>(A, lda, m, j0, w, nullptr, 0, 0, w, 1, nsplit, rows_per,
                                                          part);
        k_qr_tbuild<<<1, kQB * kQB, 0, st>>>(part, nsplit, w, tau + j0, T);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches += 3;
        const int nt = (int)(n - j0 - w);
        if (nt > 0) {
            e = apply_panel(A, lda, m, j0, w, T, 1, A, lda, j0 + w, nt, part, Z, st);
            if (e != cudaSuccess) return e;
            *launches += 3 * ((nt + kMaxCols - 1) / kMaxCols);
        }
    }
    return cudaSuccess;
}

// U (m x ncols, ldu; ncols = 0: n) holds [U_R; 0] on entry; U <- Q U with the
// reflectors in A and the T factors in ws (as left by qr_factor).  The
// workspace holds partials for min(n, 2048) columns, so U is taken in chunks
// of that many columns.
cudaError_t qr_apply_q(double *A, int64_t lda, int64_t m, int64_t n, double *ws, double *U, int64_t ldu,
                       cudaStream_t st, long long *launches, int64_t ncols) {
    const int64_t panels = (n + kQB - 1) / kQB;
    double *Tall = ws, *tau = Tall + (size_t)panels * kQB * kQB;
    const int64_t wcols = std::min<int64_t>(n, kMaxCols);
    double *part = tau + n, *Z = part + (size_t)64 * kQB * wcols;
    if (ncols <= 0) ncols = n;
    for (int64_t c0 = 0; c0 < ncols; c0 += wcols) {
        const int nc = (int)std::min<int64_t>(wcols, ncols - c0);
        for (int64_t p = panels - 1; p >= 0; --p) {
            const int j0 = (int)(p * kQB), w = (int)std::min<int64_t>(kQB, n - j0);
            const cudaError_t e = apply_panel(A, lda, m, j0, w, Tall + (size_t)p * kQB * kQB, 0, U, ldu, (int)c0,
                                              nc, part, Z, st);
            if (e != cudaSuccess) return e;
            *launches += 3;
        }
    }
    return cudaSuccess;
}

}  // namespace hsvd
