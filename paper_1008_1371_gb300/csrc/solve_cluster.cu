// solve_cluster.cu -- the inner pivot-block solve of the blocked method
// (Sec. 5 block-oriented / Sec. 6 full-block) on a thread-block cluster.
//
// One pivot pair (I, J) of an outer step has a 2b x 2b pivot block A_P that is
// J-orthogonalised by inner steps of disjoint 2x2 rotations.  On this GPU the
// FP64 pipe of a single SM is narrow (about 2 DFMA per clock), and an outer
// step only has n/(2b) pairs, so one CTA per pair leaves most SMs idle.  Here
// a cluster of C CTAs shares one pair: CTA r owns rows [r R, r R + R) of the
// stored matrix S (S = A or A^T) and of the accumulated W_P, R = 2b / C.
//
// One inner step A <- R^T A R (reading of the paper: the two one-sided halves
// alternate order from step to step):
//   1. the owner of the stored row holding a_pq writes it into every CTA of
//      the cluster through distributed shared memory;      cluster barrier
//      every CTA computes (t, c) of every pair (Sec. 2 rotation, test of
//      Eq. 2.3) from its replica of the diagonal;

//   2. every CTA mixes columns p, q of its own rows of S and of W (the column
//      update of Alg. 4.5), updates the replicated diagonal by Eq. 2.6, and
//      scatters its rows of S transposed into the owners' receive buffers;
//                                                           cluster barrier
//   3. every CTA mixes columns p, q of its received rows (the other half of
//      R^T A R) and writes Eq. 2.6's diagonal and the zeros of the pair.
// Parameters and pair lists are double-buffered by step parity, so two
// barriers per step suffice.  The arithmetic is the oracle's, element for
// element, so the result is bit-identical to it.
#include <cooperative_groups.h>

#include "hsvd_internal.cuh"

namespace cg = cooperative_groups;

namespace hsvd {
namespace {

constexpr int kClThreads = 256;

template <int NN>
struct ClusterOf {
    static constexpr int C = NN == 32 ? 4 : 8;
};

template <int NN, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kClThreads)
k_solve_cluster(const double *__restrict__ part, int nsplit, int full_part, double *__restrict__ A_io,
                const int8_t *__restrict__ sgn_cols, const int *__restrict__ col0,
                const int8_t *__restrict__ sgn_direct, double tol, int mode, int max_passes,
                const int *__restrict__ tab_full, const int *__restrict__ tab_cross,
                double *__restrict__ Wout, int *__restrict__ rotated,
                unsigned long long *__restrict__ rot_count, int *__restrict__ status, int *__restrict__ dexp,
                const int *__restrict__ visit, float *__restrict__ trace) {
    constexpr int H = NN / 2, R = NN / C, LD = NN + 1, B = NN / 2;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int pair = blockIdx.x / C;
    const int row0 = rank * R;
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) double sm[];
    double *Sa = sm;               // [R][LD] stored rows (current or receive)
    double *Sb = Sa + R * LD;      // [R][LD]
    double *Wl = Sb + R * LD;      // [R][NN] own rows of W_P
    __shared__ double D[NN];
    __shared__ int sg[NN];
    __shared__ int P[2][H], Q[2][H], Hy[2][H], Rot[2][H];
    __shared__ double T[2][H], Cc[2][H], Apq[2][H];
    __shared__ int s_flag;
    __shared__ double tr_max[C], tr_sum[C], tr_red[2][kClThreads / 32];

    // initial state: own rows of A_P, the whole diagonal, W = I.  A_P comes from
    // the three-block partials of the FP64 Gram, from full 2b x 2b partials of
    // the split-precision Gram (upper triangle, so A_P is exactly symmetric),
    // or from A_io.
    auto entry = [&](int x, int y) -> double {
        if (!part) return A_io[(size_t)pair * NN * NN + x + y * NN];
        if (!full_part) return assemble_entry<NN>(part, nsplit, pair, x + y * NN);
        const int lo = x < y ? x : y, hi = x < y ? y : x;
        const double *pp = part + (size_t)pair * nsplit * NN * NN + lo + (size_t)hi * NN;
        double v = 0.0;
        for (int s = 0; s < nsplit; ++s) v += pp[(size_t)s * NN * NN];
        return v;
    };
    if (tid == 0) s_flag = 0;
    for (int x = tid; x < NN; x += kClThreads) {
        if (sgn_direct) sg[x] = sgn_direct[(size_t)pair * NN + x];
        else sg[x] = sgn_cols[col0[2 * pair + (x >= B)] + (x % B)];
        D[x] = entry(x, x);
        // column-norm exponents for the balancing of the split-precision update
        if (dexp && rank == 0) dexp[(size_t)pair * NN + x] = D[x] > 0.0 ? (ilogb(D[x]) >> 1) : 0;
    }
    for (int e = tid; e < R * NN; e += kClThreads) {
        const int x = e / NN, y = e % NN;
        const int gx = row0 + x;
        Sa[x * LD + y] = entry(gx, y);
        Wl[x * NN + y] = (gx == y) ? 1.0 : 0.0;
    }
    double *S = Sa, *Rv = Sb;
    int transposed = 0;  // 0: S holds rows of A, 1: rows of A^T
    cluster.sync();      // every CTA initialised before any remote write
    // visit record for the learned form: the I x J block of A_P scaled by the
    // diagonal (max and sum of squares of a_ij / sqrt(a_ii a_jj)), reduced into
    // rank 0; the block means of the diagonal and the hyperbolic fraction
    float rec_meanI = 0.f, rec_meanJ = 0.f, rec_hyp = 0.f;
    if (trace) {
        double lmax = 0.0, lsum = 0.0;
        for (int e = tid; e < R * NN; e += kClThreads) {
            const int x = e / NN, y = e % NN, gx = row0 + x;
            if (gx < B && y >= B) {
                const double dd = D[gx] * D[y];
                const double sc = dd > 0.0 ? fabs(Sa[x * LD + y]) / sqrt(dd) : 0.0;
                lmax = fmax(lmax, sc);
                lsum = fma(sc, sc, lsum);
            }
        }
        lmax = warp_max(lmax);
        lsum = warp_sum(lsum);
        if ((tid & 31) == 0) {
            tr_red[0][tid >> 5] = lmax;
            tr_red[1][tid >> 5] = lsum;
        }
        __syncthreads();
        if (tid == 0) {
            double mx = 0.0, sm2 = 0.0;
            for (int w = 0; w < kClThreads / 32; ++w) {
                mx = fmax(mx, tr_red[0][w]);
                sm2 += tr_red[1][w];
            }
            *cluster.map_shared_rank(&tr_max[rank], 0) = mx;
            *cluster.map_shared_rank(&tr_sum[rank], 0) = sm2;
            if (rank == 0) {
                double mi = 0.0, mj = 0.0;
                int pi = 0, pj = 0;
                for (int x = 0; x < B; ++x) {
                    mi += D[x];
                    mj += D[B + x];
                    pi += sg[x] > 0;
                    pj += sg[B + x] > 0;
                }
                rec_meanI = (float)(mi / B);
                rec_meanJ = (float)(mj / B);
                rec_hyp = (float)(pi * (B - pj) + (B - pi) * pj) / (float)(B * B);
            }
        }
    }

    int total = 0, step = 0, err = 0;
    const int npass = (mode == 0) ? max_passes : 1;
    for (int pass = 0; pass < npass && !err; ++pass) {
        int pass_rot = 0;
        const int nsteps = (mode == 1) ? H : NN;
        for (int s = 0; s < nsteps; ++s, ++step) {
            const int buf = step & 1;
            const int *tab = (mode == 1) ? (tab_cross + (size_t)s * H * 2) : (tab_full + (size_t)s * H * 2);
            if (tid < H) {
                P[buf][tid] = tab[2 * tid];
                Q[buf][tid] = tab[2 * tid + 1];
            }
            __syncthreads();
            // 1. the owner of a_pq broadcasts it to the cluster; every CTA then
            //    computes (t, c) for every pair itself (Sec. 2 rotation, test of
            //    Eq. 2.3) from the replicated diagonal: the same operands and
            //    operations everywhere, so the same bits
            if (tid < H) {
                const int k = tid, p = P[buf][k], q = Q[buf][k];
                const int orow = transposed ? q : p, ocol = transposed ? p : q;
                if (orow / R == rank) {
                    const double apq = S[(orow - row0) * LD + ocol];
                    for (int r = 0; r < C; ++r) *cluster.map_shared_rank(&Apq[buf][k], r) = apq;
                }
            }
            cluster.sync();
            if (tid < H) {
                const int k = tid, p = P[buf][k], q = Q[buf][k];
                const double apq = Apq[buf][k], app = D[p], aqq = D[q];
                const int hyp = (sg[p] == sg[q]) ? -1 : 1;
                double t = 0.0, c = 1.0;
                int rot = 0;
                if (!pair_passes(app, aqq, apq, tol)) {
                    if (rotation_params(app, aqq, apq, hyp, t, c)) rot = 1;
                    else s_flag = HSVD_ERR_RANK;
                }
                T[buf][k] = t;
                Cc[buf][k] = c;
                Hy[buf][k] = hyp;
                Rot[buf][k] = rot;
            }
            __syncthreads();
            if (s_flag) { err = 1; break; }
            // 2. first half on own rows of S, W rows, diagonal (Eq. 2.6), transpose-scatter
            for (int e = tid; e < R * H; e += kClThreads) {
                const int x = e / H, k = e % H;
                if (!Rot[buf][k]) continue;
                const int p = P[buf][k], q = Q[buf][k];
                const double t = T[buf][k], c = Cc[buf][k], ht = Hy[buf][k] < 0 ? -t : t;
                double *row = S + x * LD;
                const double a = row[p], b = row[q];
                row[p] = fma(ht, b, a) * c;
                row[q] = fma(t, a, b) * c;
                double *wr = Wl + x * NN;
                const double wa = wr[p], wb = wr[q];
                wr[p] = fma(ht, wb, wa) * c;
                wr[q] = fma(t, wa, wb) * c;
            }
            if (tid < H && Rot[buf][tid]) {
                const int p = P[buf][tid], q = Q[buf][tid];
                const double t = T[buf][tid], ht = Hy[buf][tid] < 0 ? -t : t, apq = Apq[buf][tid];
                D[p] = fma(ht, apq, D[p]);
                D[q] = fma(t, apq, D[q]);
            }
            __syncthreads();
            for (int e = tid; e < R * NN; e += kClThreads) {
                const int x = e / NN, y = e % NN;
                const int dst = y / R;
                double *rv = cluster.map_shared_rank(Rv, dst);
                rv[(y - dst * R) * LD + (row0 + x)] = S[x * LD + y];
            }
            cluster.sync();
            { double *tmp = S; S = Rv; Rv = tmp; }
            transposed ^= 1;
            // 3. second half on the received rows, then the pair's own entries
            for (int e = tid; e < R * H; e += kClThreads) {
                const int x = e / H, k = e % H;
                if (!Rot[buf][k]) continue;
                const int p = P[buf][k], q = Q[buf][k];
                const double t = T[buf][k], c = Cc[buf][k], ht = Hy[buf][k] < 0 ? -t : t;
                double *row = S + x * LD;
                const double a = row[p], b = row[q];
                row[p] = fma(ht, b, a) * c;
                row[q] = fma(t, a, b) * c;
            }
            __syncthreads();
            if (tid < H && Rot[buf][tid]) {
                const int p = P[buf][tid], q = Q[buf][tid];
                if (p / R == rank) {
                    S[(p - row0) * LD + p] = D[p];
                    S[(p - row0) * LD + q] = 0.0;
                }
                if (q / R == rank) {
                    S[(q - row0) * LD + q] = D[q];
                    S[(q - row0) * LD + p] = 0.0;
                }
            }
            pass_rot += __syncthreads_count(tid < H && Rot[buf][tid]);
        }
        total += pass_rot;
        if (pass_rot == 0) break;
    }
    // outputs: own rows of W (column-major W_P), and A_P when asked for
    double *wo = Wout + (size_t)pair * NN * NN;
    for (int e = tid; e < R * NN; e += kClThreads) {
        const int x = e / NN, y = e % NN;
        wo[(row0 + x) + (size_t)y * NN] = Wl[x * NN + y];
    }
    if (!part) {
        double *ao = A_io + (size_t)pair * NN * NN;
        for (int e = tid; e < R * NN; e += kClThreads) {
            const int x = e / NN, y = e % NN;
            const int gx = row0 + x;
            if (transposed) ao[y + (size_t)gx * NN] = S[x * LD + y];  // stored row gx is column gx of A
            else ao[gx + (size_t)y * NN] = S[x * LD + y];
        }
    }
    if (rank == 0 && tid == 0) {
        rotated[pair] = total;
        if (rot_count && total) atomicAdd(rot_count, (unsigned long long)total);
        if (s_flag && status) atomicExch(status, s_flag);
    }
    cluster.sync();  // no CTA leaves while others may still write into it
    if (trace && rank == 0 && tid == 0) {
        double mx = 0.0, sm2 = 0.0;
        for (int r = 0; r < C; ++r) {
            mx = fmax(mx, tr_max[r]);
            sm2 += tr_sum[r];
        }
        float *rec = trace + (size_t)visit[pair] * HSVD_TRACE_FIELDS;
        rec[0] = (float)mx;
        rec[1] = (float)sqrt(sm2);
        rec[2] = (float)total;
        rec[3] = rec_meanI;
        rec[4] = rec_meanJ;
        rec[5] = rec_hyp;
    }
}

template <int NN>
cudaError_t solve_cluster_impl(int npairs, const double *part, int nsplit, int full_part, double *A,
                               const int8_t *sgn_cols, const int *col0, const int8_t *sgn_direct, double tol,
                               int mode, int max_passes, const int *tab_full, const int *tab_cross, double *Wp,
                               int *rotated, unsigned long long *rot_count, int *status, int *dexp,
                               const int *visit, float *trace, cudaStream_t st) {
    constexpr int C = ClusterOf<NN>::C, R = NN / C;
    const size_t smem = (size_t)(2 * R * (NN + 1) + R * NN) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_solve_cluster<NN, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_solve_cluster<NN, C><<<npairs * C, kClThreads, smem, st>>>(part, nsplit, full_part, A, sgn_cols, col0,
                                                                 sgn_direct, tol, mode, max_passes, tab_full,
                                                                 tab_cross, Wp, rotated, rot_count, status, dexp,
                                                                 visit, trace);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_solve(int b, int npairs, const double *part, int nsplit, double *A, const int8_t *sgn_cols,
                         const int *col0, const int8_t *sgn_direct, double tol, int mode, int max_passes,
                         const int *tab_full, const int *tab_cross, double *Wp, int *rotated,
                         unsigned long long *rot_count, int *status, cudaStream_t st, int full_part, int *dexp,
                         const int *visit, float *trace) {
    switch (b) {
        case 16: return solve_cluster_impl<32>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct, tol,
                                               mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                               status, dexp, visit, trace, st);
        case 32: return solve_cluster_impl<64>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct, tol,
                                               mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                               status, dexp, visit, trace, st);
        case 64: return solve_cluster_impl<128>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct,
                                                tol, mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                                status, dexp, visit, trace, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hsvd
