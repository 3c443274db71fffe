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
//   1. the owner of the stored row holding a_pq computes (t, c) for the pair
//      (Sec. 2 rotation, test of Eq. 2.3) and writes them into every CTA of
//      the cluster through distributed shared memory;      cluster barrier
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
                unsigned long long *__restrict__ rot_count, int *__restrict__ status, int *__restrict__ dexp) {
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
            // 1. rotation parameters by the owner of a_pq, broadcast to the cluster
            if (tid < H) {
                const int k = tid, p = P[buf][k], q = Q[buf][k];
                const int orow = transposed ? q : p, ocol = transposed ? p : q;
                if (orow / R == rank) {
                    const double apq = S[(orow - row0) * LD + ocol];
                    const double app = D[p], aqq = D[q];
                    const int hyp = (sg[p] == sg[q]) ? -1 : 1;
                    double t = 0.0, c = 1.0;
                    int rot = 0, bad = 0;
                    if (!pair_passes(app, aqq, apq, tol)) {
                        if (rotation_params(app, aqq, apq, hyp, t, c)) rot = 1;
                        else bad = 1;
                    }
                    for (int r = 0; r < C; ++r) {
                        *cluster.map_shared_rank(&T[buf][k], r) = t;
                        *cluster.map_shared_rank(&Cc[buf][k], r) = c;
                        *cluster.map_shared_rank(&Apq[buf][k], r) = apq;
                        *cluster.map_shared_rank(&Hy[buf][k], r) = hyp;
                        *cluster.map_shared_rank(&Rot[buf][k], r) = rot;
                        if (bad) *cluster.map_shared_rank(&s_flag, r) = HSVD_ERR_RANK;
                    }
                }
            }
            cluster.sync();
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
            int nr = 0;
            for (int k = 0; k < H; ++k) nr += Rot[buf][k];
            pass_rot += nr;
            __syncthreads();
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
}

template <int NN>
cudaError_t solve_cluster_impl(int npairs, const double *part, int nsplit, int full_part, double *A,
                               const int8_t *sgn_cols, const int *col0, const int8_t *sgn_direct, double tol,
                               int mode, int max_passes, const int *tab_full, const int *tab_cross, double *Wp,
                               int *rotated, unsigned long long *rot_count, int *status, int *dexp,
                               cudaStream_t st) {
    constexpr int C = ClusterOf<NN>::C, R = NN / C;
    const size_t smem = (size_t)(2 * R * (NN + 1) + R * NN) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_solve_cluster<NN, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_solve_cluster<NN, C><<<npairs * C, kClThreads, smem, st>>>(part, nsplit, full_part, A, sgn_cols, col0,
                                                                 sgn_direct, tol, mode, max_passes, tab_full,
                                                                 tab_cross, Wp, rotated, rot_count, status, dexp);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_solve(int b, int npairs, const double *part, int nsplit, double *A, const int8_t *sgn_cols,
                         const int *col0, const int8_t *sgn_direct, double tol, int mode, int max_passes,
                         const int *tab_full, const int *tab_cross, double *Wp, int *rotated,
                         unsigned long long *rot_count, int *status, cudaStream_t st, int full_part, int *dexp) {
    switch (b) {
        case 16: return solve_cluster_impl<32>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct, tol,
                                               mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                               status, dexp, st);
        case 32: return solve_cluster_impl<64>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct, tol,
                                               mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                               status, dexp, st);
        case 64: return solve_cluster_impl<128>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct,
                                                tol, mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                                status, dexp, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hsvd
