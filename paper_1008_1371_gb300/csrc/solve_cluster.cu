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
// barriers per step suffice.
//
// All three kernels here apply scaled rotations (hsvd_internal.cuh): they
// keep S = diag(s)^-1 A diag(s)^-1 and W = Wh diag(s), so a rotation costs two
// FMAs per element pair instead of two FMAs and two multiplies, which halves
// the FP64 work of the inner solve; the true a_pq of a test is (s_p s_q) S_pq,
// and the outputs are the true A_P (diagonal from Eq. 2.6) and W_P.  The
// element operations and their order are those of the exact CPU model of the
// kernels (oracle/inner_model.c), so the results are bit-identical to it.
#include <cooperative_groups.h>

#include <vector>

#include "hsvd_internal.cuh"

namespace cg = cooperative_groups;

namespace hsvd {
namespace {

constexpr int kClThreads = 256;
constexpr int kCrossThreads = kClThreads + 32;  // cross pass: 8 mixing warps + the look-ahead warp

// the mixing threads' barrier: barrier 1 among the last n threads of the CTA
// (warps 1..) when warp 0 runs ahead, else the whole CTA
template <bool LA>
__device__ __forceinline__ void mix_sync(int n) {
    if (LA) asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
    else __syncthreads();
}

template <int NN>
struct ClusterOf {
    static constexpr int C = NN == 32 ? 4 : 8;
};

// CTAs per pivot block of the cross pass (the pass of every step but the first)
template <int NN>
struct CrossClusterOf {
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
                const int *__restrict__ visit, float *__restrict__ trace, double tstop, int *__restrict__ tbig) {
    constexpr int H = NN / 2, R = NN / C, LD = NN + 1, B = NN / 2;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int pair = blockIdx.x / C;
    const int row0 = rank * R;
    const int tid = threadIdx.x;

    if (col0 && col0[2 * pair] < 0) {  // a visit the skip mask removed: the whole cluster leaves
        if (rank == 0 && tid == 0) rotated[pair] = 0;
        return;
    }
    extern __shared__ __align__(16) double sm[];
    double *Sa = sm;               // [R][LD] stored rows (current or receive)
    double *Sb = Sa + R * LD;      // [R][LD]
    double *Wl = Sb + R * LD;      // [R][NN] own rows of W_P
    __shared__ double D[NN];
    __shared__ int sg[NN];
    __shared__ int P[2][H], Q[2][H], Hy[2][H], Rot[2][H];
    __shared__ double T[2][H], Cc[2][H], Qv[2][H], Apq[2][H];  // Apq: the true a_pq
    __shared__ double Sc[NN], Rc[NN];  // column scales of the stored block and their reciprocals
    __shared__ double Al[H], Be[H];    // the step's scaled-rotation coefficients
    __shared__ int s_renorm;
    __shared__ int s_flag;
    __shared__ int s_big;  // a rotation had |t| > tstop (Eq. 4.2 code (11)_2)
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
    if (tid == 0) {
        s_flag = 0;
        s_big = 0;
        s_renorm = 0;
    }
    for (int x = tid; x < NN; x += kClThreads) {
        if (sgn_direct) sg[x] = sgn_direct[(size_t)pair * NN + x];
        else sg[x] = sgn_cols[col0[2 * pair + (x >= B)] + (x % B)];
        D[x] = entry(x, x);
        Sc[x] = 1.0;
        Rc[x] = 1.0;
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
                const double apq = (Sc[p] * Sc[q]) * Apq[buf][k], app = D[p], aqq = D[q];  // true a_pq
                const int hyp = (sg[p] == sg[q]) ? -1 : 1;
                double t, c, qv;
                const int d = pair_decision_fast(app, aqq, apq, hyp, tol, t, c, qv);
                const int rot = d == 1;
                if (d == 2) s_flag = HSVD_ERR_RANK;
                if (rot && fabs(t) > tstop) s_big = 1;
                T[buf][k] = t;
                Cc[buf][k] = c;
                Qv[buf][k] = qv;
                Apq[buf][k] = apq;
                Hy[buf][k] = hyp;
                Rot[buf][k] = rot;
                if (rot) {  // the step's coefficients from its starting scales
                    const double ht = hyp < 0 ? -t : t;
                    Al[k] = ht * (Sc[q] * Rc[p]);
                    Be[k] = t * (Sc[p] * Rc[q]);
                }
            }
            __syncthreads();
            if (s_flag) { err = 1; break; }
            // 2. first half on own rows of S, W rows, diagonal (Eq. 2.6), transpose-scatter;
            //    a thread keeps one pair (its rotation in registers) and walks rows
            static_assert(kClThreads % H == 0, "whole rows per pass");
            if (Rot[buf][tid % H]) {
                const int k = tid % H, p = P[buf][k], q = Q[buf][k];
                const double al = Al[k], be = Be[k];
                for (int x = tid / H; x < R; x += kClThreads / H) {
                    double *row = S + x * LD;
                    const double a = row[p], b = row[q];
                    row[p] = fma(al, b, a);
                    row[q] = fma(be, a, b);
                    double *wr = Wl + x * NN;
                    const double wa = wr[p], wb = wr[q];
                    wr[p] = fma(al, wb, wa);
                    wr[q] = fma(be, wa, wb);
                }
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
            if (Rot[buf][tid % H]) {
                const int k = tid % H, p = P[buf][k], q = Q[buf][k];
                const double al = Al[k], be = Be[k];
                for (int x = tid / H; x < R; x += kClThreads / H) {
                    double *row = S + x * LD;
                    const double a = row[p], b = row[q];
                    row[p] = fma(al, b, a);
                    row[q] = fma(be, a, b);
                }
            }
            __syncthreads();
            if (tid < H && Rot[buf][tid]) {
                const int p = P[buf][tid], q = Q[buf][tid];
                if (p / R == rank) {
                    S[(p - row0) * LD + p] = 0.0;
                    S[(p - row0) * LD + q] = 0.0;
                }
                if (q / R == rank) {
                    S[(q - row0) * LD + q] = 0.0;
                    S[(q - row0) * LD + p] = 0.0;
                }
                const double c = Cc[buf][tid], qv = Qv[buf][tid];
                Sc[p] = Sc[p] * c;
                Sc[q] = Sc[q] * c;
                Rc[p] = Rc[p] * qv;
                Rc[q] = Rc[q] * qv;
                if (scale_out_of_range(Sc[p]) || scale_out_of_range(Sc[q])) s_renorm = 1;
            }
            pass_rot += __syncthreads_count(tid < H && Rot[buf][tid]);
            if (s_renorm) {  // scales out of range: the block back to s = r = 1
                for (int e = tid; e < R * NN; e += kClThreads) {
                    const int x = e / NN, y = e % NN;
                    S[x * LD + y] = (Sc[row0 + x] * Sc[y]) * S[x * LD + y];
                    Wl[x * NN + y] = Wl[x * NN + y] * Sc[y];
                }
                __syncthreads();
                for (int x = tid; x < NN; x += kClThreads) Sc[x] = Rc[x] = 1.0;
                if (tid == 0) s_renorm = 0;
                __syncthreads();
            }
        }
        total += pass_rot;
        if (pass_rot == 0) break;
    }
    // outputs: own rows of W (column-major W_P), and A_P when asked for
    double *wo = Wout + (size_t)pair * NN * NN;
    for (int e = tid; e < R * NN; e += kClThreads) {
        const int x = e / NN, y = e % NN;
        wo[(row0 + x) + (size_t)y * NN] = Wl[x * NN + y] * Sc[y];
    }
    if (!part) {
        // true values (s_x s_y) S_xy, the diagonal from D
        double *ao = A_io + (size_t)pair * NN * NN;
        for (int e = tid; e < R * NN; e += kClThreads) {
            const int x = e / NN, y = e % NN;
            const int gx = row0 + x;
            const double v = gx == y ? D[gx] : (Sc[gx] * Sc[y]) * S[x * LD + y];
            if (transposed) ao[y + (size_t)gx * NN] = v;  // stored row gx is column gx of A
            else ao[gx + (size_t)y * NN] = v;
        }
    }
    if (rank == 0 && tid == 0) {
        rotated[pair] = total;
        if (rot_count && total) atomicAdd(rot_count, (unsigned long long)total);
        if (s_flag && status) atomicExch(status, s_flag);
        if (tbig && s_big) atomicOr(tbig, 1);
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

// The cross pass (block-oriented mode, Sec. 5: the pairs (k, h + (k + s) mod h)
// of the off-diagonal block, h = b, s = 0..h-1) without transposes.  CTA r of
// the cluster owns the pairs k in [r P, r P + P), P = h / C: their fixed rows
// k and their current partner rows h + (k + s) mod h.  Both halves of
// R^T A R touch only a pair's two rows (the row mix) and, inside every row,
// the two columns of each pair (the column mix), so a step is local once the
// CTA knows every pair's (t, c).  From step s to s + 1 pair k takes pair
// k + 1's partner row: inside the CTA that is a ring of P + 1 row slots, and
// across the cluster every CTA hands its first pair's partner row to the
// previous CTA.  The next step's a_pq lies in the owner's fixed row, so the
// owner computes that pair's (t, c) as soon as its rows are updated and writes
// them into every CTA; one cluster barrier per step.  The element operations
// and their order (column mix first on even steps, row mix first on odd
// steps, Eq. 2.6 on the diagonal, zeros at the pair) are the oracle's, so the
// result is bit-identical to it and to k_solve_cluster.
template <int NN, int C, bool LA>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(LA ? kCrossThreads : kClThreads, 3)
k_solve_cross(const double *__restrict__ part, int nsplit, int full_part, double *__restrict__ A_io,
              const int8_t *__restrict__ sgn_cols, const int *__restrict__ col0,
              const int8_t *__restrict__ sgn_direct, double tol, double *__restrict__ Wout,
              int *__restrict__ rotated, unsigned long long *__restrict__ rot_count, int *__restrict__ status,
              int *__restrict__ dexp, const int *__restrict__ visit, float *__restrict__ trace, double tstop,
              int *__restrict__ tbig) {
    constexpr int h = NN / 2, P = h / C, RW = NN / C, B = NN / 2;
    constexpr int kT = LA ? kCrossThreads : kClThreads;
    static_assert(P * C == h && RW * C == NN, "the pairs and rows split evenly over the cluster");
    static_assert(!LA || P <= 32, "the look-ahead warp has one lane per owned pair");
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int pair = blockIdx.x / C;
    const int tid = threadIdx.x;
    const int k0 = rank * P;        // first pair owned
    const int w0 = rank * RW;       // first row of W owned
    if (col0 && col0[2 * pair] < 0) {  // a visit the skip mask removed: the whole cluster leaves
        if (rank == 0 && tid == 0) rotated[pair] = 0;
        return;
    }

    extern __shared__ __align__(16) double sm[];
    double *fix = sm;                 // [P][NN]    rows k0 .. k0 + P - 1
    double *mov = fix + P * NN;       // [P + 1][NN] partner rows, ring
    double *Wl = mov + (P + 1) * NN;  // [RW][NN]   rows w0 .. w0 + RW - 1 of W_P
    __shared__ double D[NN];
    __shared__ int sg[NN];
    __shared__ double T[2][h], Cc[2][h], Qv[2][h], Apq[2][h];  // Apq: the true a_pq
    __shared__ int Fl[2][h];          // bit 0: rotate, bit 1: rank deficient
    __shared__ double Sc[NN], Rc[NN];  // column scales of the stored block and their reciprocals
    __shared__ double Al[h], Be[h];    // the step's scaled-rotation coefficients
    __shared__ int s_renorm;
    __shared__ double tr_max[C], tr_sum[C], tr_red[2][kT / 32];
    __shared__ int s_first[C];        // per CTA: first step with a pair failing Eq. 2.3 on A_P
    __shared__ int s_own;
    __shared__ int s_tot[2];          // rotations counted by warps 0 and 1
    static_assert(h <= 64, "the rotation count lives in warps 0 and 1");

    auto entry = [&](int x, int y) -> double {
        if (!part) return A_io[(size_t)pair * NN * NN + x + y * NN];
        if (!full_part) return assemble_entry<NN>(part, nsplit, pair, x + y * NN);
        const int lo = x < y ? x : y, hi = x < y ? y : x;
        const double *pp = part + (size_t)pair * nsplit * NN * NN + lo + (size_t)hi * NN;
        double v = 0.0;
        for (int s = 0; s < nsplit; ++s) v += pp[(size_t)s * NN * NN];
        return v;
    };
    for (int x = tid; x < NN; x += kT) {
        if (sgn_direct) sg[x] = sgn_direct[(size_t)pair * NN + x];
        else sg[x] = sgn_cols[col0[2 * pair + (x >= B)] + (x % B)];
        D[x] = entry(x, x);
        Sc[x] = 1.0;
        Rc[x] = 1.0;
        if (dexp && rank == 0) dexp[(size_t)pair * NN + x] = D[x] > 0.0 ? (ilogb(D[x]) >> 1) : 0;
    }
    if (tid == 0) {
        s_own = h;
        s_renorm = 0;
    }
    for (int e = tid; e < P * NN; e += kT) {
        const int kl = e / NN, y = e % NN;
        fix[kl * NN + y] = entry(k0 + kl, y);
    }
    for (int e = tid; e < RW * NN; e += kT) {
        const int x = e / NN, y = e % NN;
        Wl[x * NN + y] = (w0 + x == y) ? 1.0 : 0.0;
    }
    __syncthreads();
    // Steps before the first one holding a pair that fails Eq. 2.3 on A_P as
    // it stands rotate nothing and change nothing: the pass starts there.
    // Pair k meets partner h + j at step (j - k) mod h; every CTA tests its
    // own rows' cross entries, and the cluster takes the minimum.
    for (int e = tid; e < P * h; e += kT) {
        const int kl = e / h, j = e % h, k = k0 + kl;
        if (!pair_passes(D[k], D[h + j], fix[kl * NN + h + j], tol)) atomicMin(&s_own, (j - k + h) % h);
    }
    __syncthreads();
    // visit record: the I x J block (rows k < h are the fixed rows) scaled by the diagonal
    float rec_meanI = 0.f, rec_meanJ = 0.f, rec_hyp = 0.f;
    double rec_max = 0.0, rec_sum = 0.0;
    if (trace) {
        double lmax = 0.0, lsum = 0.0;
        for (int e = tid; e < P * h; e += kT) {
            const int kl = e / h, y = h + e % h, x = k0 + kl;
            const double dd = D[x] * D[y];
            const double sc = dd > 0.0 ? fabs(fix[kl * NN + y]) / sqrt(dd) : 0.0;
            lmax = fmax(lmax, sc);
            lsum = fma(sc, sc, lsum);
        }
        lmax = warp_max(lmax);
        lsum = warp_sum(lsum);
        if ((tid & 31) == 0) {
            tr_red[0][tid >> 5] = lmax;
            tr_red[1][tid >> 5] = lsum;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 0; w < kT / 32; ++w) {
                rec_max = fmax(rec_max, tr_red[0][w]);
                rec_sum += tr_red[1][w];
            }
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
    cluster.sync();  // every CTA initialised before any remote write
    if (trace && tid == 0) {
        *cluster.map_shared_rank(&tr_max[rank], 0) = rec_max;
        *cluster.map_shared_rank(&tr_sum[rank], 0) = rec_sum;
    }
    if (tid < C) *cluster.map_shared_rank(&s_first[rank], tid) = s_own;
    cluster.sync();
    int s0 = h;
    for (int r = 0; r < C; ++r) s0 = min(s0, s_first[r]);
    // partner rows of the starting step (the last one when nothing fails):
    // pair k with row h + (k + s) mod h in ring slot (kl + s) mod (P + 1)
    {
        const int sl = min(s0, h - 1);
        for (int e = tid; e < P * NN; e += kT) {
            const int kl = e / NN, y = e % NN;
            mov[((kl + sl) % (P + 1)) * NN + y] = entry(h + (k0 + kl + sl) % h, y);
        }
    }
    __syncthreads();
    // (t, c) of the owned pairs for step s into every CTA (buffer s & 1)
    auto put_params = [&](int s, int k, double t, double c, double qv, double apq, int fl) {
        const int b = s & 1;
        for (int r = 0; r < C; ++r) {
            *cluster.map_shared_rank(&T[b][k], r) = t;
            *cluster.map_shared_rank(&Cc[b][k], r) = c;
            *cluster.map_shared_rank(&Qv[b][k], r) = qv;
            *cluster.map_shared_rank(&Apq[b][k], r) = apq;
            *cluster.map_shared_rank(&Fl[b][k], r) = fl;
        }
    };
    auto params_out = [&](int s) {
        if (tid < P) {
            const int kl = tid, k = k0 + kl, p = k, q = h + (k + s) % h;
            const double apq = (Sc[p] * Sc[q]) * fix[kl * NN + q];  // true a_pq
            const double app = D[p], aqq = D[q];
            const int hyp = (sg[p] == sg[q]) ? -1 : 1;
            double t, c, qv;
            const int fl = pair_decision_fast(app, aqq, apq, hyp, tol, t, c, qv);
            put_params(s, k, t, c, qv, apq, fl);
        }
    };
    if (s0 < h) params_out(s0);
    cluster.sync();

    // Warp 0 works one step ahead: at the top of step s lane kl < P reads the
    // four entries of its rows (k, q_k) in the columns (j, q') of pair
    // j = k + 1 and the diagonal values a_kk, a_q'q', forms the step-s values
    // of a_kq' and of the two diagonal entries with the same operations as the
    // bulk update below, and computes the (t, c) of pair (k, q') for step
    // s + 1 while warps 1..8 update the rows (named barrier 1).
    // Without the look-ahead (LA = false) every warp mixes and the owners
    // compute the next parameters after the update.
    constexpr int kMixThreads = LA ? kT - 32 : kT;
    const int warp = tid >> 5, lane = tid & 31;
    int total = 0, bad = 0, s_end = h - 1;
    int big = 0;  // a rotation of pair tid had |t| > tstop (Eq. 4.2 code (11)_2)
    const int mt = LA ? tid - 32 : tid;  // mixing thread index (warps 1.. with the look-ahead)
    for (int s = s0; s < h; ++s) {
        const int b = s & 1;
        auto slot = [&](int kl) { return (kl + s) % (P + 1); };
        // scales out of range after the last step: the block back to s = r = 1
        if (s_renorm) {
            for (int e = tid; e < (2 * P + RW) * NN; e += kT) {
                const int r = e / NN, y = e % NN;
                if (r < 2 * P) {
                    const int kl = r < P ? r : r - P, x = r < P ? k0 + kl : h + (k0 + kl + s) % h;
                    double *row = r < P ? fix + kl * NN : mov + slot(kl) * NN;
                    row[y] = (Sc[x] * Sc[y]) * row[y];
                } else {
                    Wl[(r - 2 * P) * NN + y] = Wl[(r - 2 * P) * NN + y] * Sc[y];
                }
            }
            __syncthreads();
            for (int x = tid; x < NN; x += kT) Sc[x] = Rc[x] = 1.0;
            if (tid == 0) s_renorm = 0;
            __syncthreads();
        }
        double nx_t = 0.0, nx_c = 1.0, nx_qv = 1.0, nx_apq = 0.0;
        int nx_fl = 0;
        double e_kj = 0.0, e_kq = 0.0, e_qj = 0.0, e_qq = 0.0, d_k = 0.0, d_q = 0.0, s_k = 1.0, s_q = 1.0;
        const bool ahead = LA && warp == 0 && lane < P && s + 1 < h;
        if (ahead) {
            const int kl = lane, k = k0 + kl, j = (k + 1) % h, q2 = h + (j + s) % h;
            const double *rk = fix + kl * NN, *rq = mov + ((kl + s) % (P + 1)) * NN;
            e_kj = rk[j];
            e_kq = rk[q2];
            e_qj = rq[j];
            e_qq = rq[q2];
            d_k = D[k];
            d_q = D[q2];
            s_k = Sc[k];
            s_q = Sc[q2];
        }
        // the step's coefficients from its starting scales (alpha by threads
        // [0, h), beta by [h, 2h): two FP64 instructions per warp)
        if (mt >= 0 && mt < 2 * h && (Fl[b][mt % h] & 1)) {
            const int j = mt % h, p = j, q = h + (j + s) % h;
            const double t = T[b][j];
            if (mt < h) Al[j] = ((sg[p] == sg[q]) ? -t : t) * (Sc[q] * Rc[p]);
            else Be[j] = t * (Sc[p] * Rc[q]);
        }
        // every CTA sees every pair's flags: the same decision everywhere
        const int f = tid < h ? Fl[b][tid] : 0;
        if (tbig && (f & 1) && fabs(T[b][tid]) > tstop) big = 1;
        bad = __syncthreads_or(f & 2);
        if (bad) {
            s_end = s;
            break;
        }
        // the step's rotations, counted by the warps holding the flags (one
        // CTA barrier per step instead of two); lane 0 of warp w keeps warp
        // w's count
        if (warp * 32 < h) total += __popc(__ballot_sync(0xffffffffu, f & 1));
        if (LA && warp == 0) {
            if (ahead) {
                const int kl = lane, k = k0 + kl, j = (k + 1) % h, q2 = h + (j + s) % h, qk = h + (k + s) % h;
                const int fk = Fl[b][k] & 1, fj = Fl[b][j] & 1;
                const double tk = T[b][k], htk = (sg[k] == sg[qk]) ? -tk : tk;
                const double tj = T[b][j];
                const double alk = fk ? Al[k] : 0.0, bej = fj ? Be[j] : 0.0;
                double v;
                if ((s & 1) == 0) {  // column mix (pair j), then row mix (pair k)
                    double r1 = e_kq, r2 = e_qq;
                    if (fj) {
                        r1 = fma(bej, e_kj, e_kq);
                        r2 = fma(bej, e_qj, e_qq);
                    }
                    v = fk ? fma(alk, r2, r1) : r1;
                } else {  // row mix (pair k), then column mix (pair j)
                    double u1 = e_kj, u2 = e_kq;
                    if (fk) {
                        u1 = fma(alk, e_qj, e_kj);
                        u2 = fma(alk, e_qq, e_kq);
                    }
                    v = fj ? fma(bej, u1, u2) : u2;
                }
                const double app = fk ? fma(htk, Apq[b][k], d_k) : d_k;
                const double aqq = fj ? fma(tj, Apq[b][j], d_q) : d_q;
                // the step's new scales of rows k and q2 (as the update phase forms them)
                const double sk = fk ? s_k * Cc[b][k] : s_k, sq = fj ? s_q * Cc[b][j] : s_q;
                const double apq = (sk * sq) * v;
                const int hyp = (sg[k] == sg[q2]) ? -1 : 1;
                nx_fl = pair_decision_fast(app, aqq, apq, hyp, tol, nx_t, nx_c, nx_qv);
                nx_apq = apq;
            }
        } else {
            // The column mix on every owned row of A (and of W): pair j's columns
            // j and h + (j + s) mod h.  A thread keeps one pair (its rotation in
            // registers) and walks rows; consecutive threads take consecutive
            // pairs, so a warp's loads of one row are consecutive words.
            auto col_mix = [&](bool with_w) {
                static_assert(kMixThreads % h == 0, "whole rows per pass");
                const int j = mt % h;
                if (!(Fl[b][j] & 1)) return;
                const int p = j, q = h + (j + s) % h;
                const double al = Al[j], be = Be[j];
                const int nrows = 2 * P + (with_w ? RW : 0);
                for (int r = mt / h; r < nrows; r += kMixThreads / h) {
                    double *row = r < P ? fix + r * NN : (r < 2 * P ? mov + slot(r - P) * NN : Wl + (r - 2 * P) * NN);
                    const double a = row[p], bb = row[q];
                    row[p] = fma(al, bb, a);
                    row[q] = fma(be, a, bb);
                }
            };
            // The row mix of every owned pair: rows k and its partner, every
            // column; a thread keeps one pair and walks columns.  With W, also
            // W's column mix (as in col_mix, on W's rows only).
            auto row_mix = [&](bool with_w) {
                static_assert(kMixThreads % P == 0, "threads split evenly over the owned pairs");
                constexpr int TP = kMixThreads / P;  // threads per owned pair
                const int kl = mt / TP, k = k0 + kl;
                if (Fl[b][k] & 1) {
                    const double al = Al[k], be = Be[k];
                    double *rp = fix + kl * NN, *rq = mov + slot(kl) * NN;
                    for (int y = mt % TP; y < NN; y += TP) {
                        const double a = rp[y], bb = rq[y];
                        rp[y] = fma(al, bb, a);
                        rq[y] = fma(be, a, bb);
                    }
                }
                if (!with_w) return;
                const int j = mt % h;
                if (!(Fl[b][j] & 1)) return;
                const int pw = j, qw = h + (j + s) % h;
                const double al = Al[j], be = Be[j];
                for (int x = mt / h; x < RW; x += kMixThreads / h) {
                    double *row = Wl + x * NN;
                    const double a = row[pw], bb = row[qw];
                    row[pw] = fma(al, bb, a);
                    row[qw] = fma(be, a, bb);
                }
            };
            if ((s & 1) == 0) {
                col_mix(true);
                mix_sync<LA>(kMixThreads);
                row_mix(false);
            } else {
                row_mix(true);
                mix_sync<LA>(kMixThreads);
                col_mix(false);
            }
            mix_sync<LA>(kMixThreads);
            // Eq. 2.6 on the replicated diagonal and the owned pairs' own
            // stored entries to 0 (threads [0, h)), the new scales (threads
            // [h, 2h)) and their reciprocals (threads [2h, 3h)) of the rotated
            // rows: three warp groups, so that no warp's chain of FP64
            // instructions (one issues every 64 cycles) holds up the step
            static_assert(kMixThreads >= 3 * h, "three groups of h mixing threads");
            if (mt < 3 * h && (Fl[b][mt % h] & 1)) {
                const int j = mt % h, p = j, q = h + (j + s) % h;
                if (mt < h) {
                    const double t = T[b][j], ht = (sg[p] == sg[q]) ? -t : t, apq = Apq[b][j];
                    D[p] = fma(ht, apq, D[p]);
                    D[q] = fma(t, apq, D[q]);
                    if (p >= k0 && p < k0 + P) {
                        const int kl = p - k0;
                        double *rp = fix + kl * NN, *rq = mov + slot(kl) * NN;
                        rp[p] = 0.0;
                        rp[q] = 0.0;
                        rq[q] = 0.0;
                        rq[p] = 0.0;
                    }
                } else if (mt < 2 * h) {
                    const double c = Cc[b][j];
                    Sc[p] = Sc[p] * c;
                    Sc[q] = Sc[q] * c;
                    if (scale_out_of_range(Sc[p]) || scale_out_of_range(Sc[q])) s_renorm = 1;
                } else {
                    const double qv = Qv[b][j];
                    Rc[p] = Rc[p] * qv;
                    Rc[q] = Rc[q] * qv;
                }
            }
        }
        __syncthreads();
        if (s + 1 < h) {
            // hand the first pair's partner row to the previous CTA (its last
            // pair's row at step s + 1, in the slot that is free during step s)
            const int dst = (rank + C - 1) % C;
            double *src = mov + slot(0) * NN;
            double *rdst = cluster.map_shared_rank(mov, dst) + ((P + s) % (P + 1)) * NN;
            for (int y = tid; y < NN; y += kT) rdst[y] = src[y];
            if (!LA) params_out(s + 1);
            if (ahead) put_params(s + 1, k0 + lane, nx_t, nx_c, nx_qv, nx_apq, nx_fl);
        }
        cluster.sync();
    }
    // outputs: own rows of W (column-major W_P), and A_P when asked for
    double *wo = Wout + (size_t)pair * NN * NN;
    for (int e = tid; e < RW * NN; e += kT) {
        const int x = e / NN, y = e % NN;
        wo[(w0 + x) + (size_t)y * NN] = Wl[x * NN + y] * Sc[y];
    }
    if (!part) {
        // rows where the pass ended: fixed rows k, partner rows h + (k + s_end) mod h;
        // true values (s_x s_y) S_xy, the diagonal from D
        double *ao = A_io + (size_t)pair * NN * NN;
        for (int e = tid; e < P * NN; e += kT) {
            const int kl = e / NN, y = e % NN, k = k0 + kl, x = h + (k + s_end) % h;
            ao[k + (size_t)y * NN] = k == y ? D[k] : (Sc[k] * Sc[y]) * fix[kl * NN + y];
            ao[x + (size_t)y * NN] = x == y ? D[x] : (Sc[x] * Sc[y]) * mov[((kl + s_end) % (P + 1)) * NN + y];
        }
    }
    if (lane == 0 && warp * 32 < h) s_tot[warp] = total;
    cluster.sync();
    const int any_big = tbig ? __syncthreads_or(big) : 0;
    if (rank == 0 && tid == 0) {
        total = 0;
        for (int w = 0; w * 32 < h; ++w) total += s_tot[w];
        rotated[pair] = total;
        if (rot_count && total) atomicAdd(rot_count, (unsigned long long)total);
        if (bad && status) atomicExch(status, HSVD_ERR_RANK);
        if (any_big) atomicOr(tbig, 1);
        if (trace) {
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
}

// One ring table entry of the full pass: the pair (lo, hi) of a slot at a
// step, the row buffers holding rows lo and hi in the owning CTA's pool, and
// whether row lo (else row hi) arrived from the previous slot.
__device__ __forceinline__ int ring_buf_lo(int4 e) { return e.z & 0xff; }
__device__ __forceinline__ int ring_buf_hi(int4 e) { return (e.z >> 8) & 0xff; }

// The full pass (every pair of the 2b columns once, in the modulus order of
// Sec. 2: the first visit of a block pair in a sweep of the block-oriented
// method, Sec. 5) without transposes.  Step s pairs a with c - a (mod 2b);
// from one step to the next every pair keeps one of its two rows and takes
// the row that leaves the previous pair, so the b pairs form a ring of slots
// in which one row per slot moves on by one slot per step.  The host table
// (fill_ring) gives, per step and slot, the pair, which of its rows arrived
// and the pool buffers of both.  CTA r of the cluster owns slots
// [r P, r P + P) and holds both rows of each, in a pool of 2P + 1 row buffers
// (one free to receive); per step the row leaving its last slot is written
// into the next CTA's free buffer, the only exchange of rows.  Both halves of
// R^T A R are then local, as in the cross pass.  The entry a_lo,hi of a pair
// is read from row lo (as the transposing kernel reads it), so the (t, c) of
// a pair is formed by the CTA holding row lo at the end of the previous step:
// the slot's own CTA, or the previous one when row lo is the row crossing
// over.  The element operations and their order (column mix first on even
// steps, row mix first on odd steps, Eq. 2.6 on the diagonal, zeros at the
// pair) are those of k_solve_cluster in one-pass mode: the same bits.
template <int NN, int C, bool LA>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(LA ? kCrossThreads : kClThreads, 3)
k_solve_ring(const double *__restrict__ part, int nsplit, int full_part, double *__restrict__ A_io,
             const int8_t *__restrict__ sgn_cols, const int *__restrict__ col0,
             const int8_t *__restrict__ sgn_direct, double tol, const int4 *__restrict__ ring,
             double *__restrict__ Wout, int *__restrict__ rotated, unsigned long long *__restrict__ rot_count,
             int *__restrict__ status, int *__restrict__ dexp, const int *__restrict__ visit,
             float *__restrict__ trace, double tstop, int *__restrict__ tbig) {
    constexpr int h = NN / 2, P = h / C, RW = NN / C, B = NN / 2, NBUF = 2 * P + 1;
    constexpr int kT = LA ? kCrossThreads : kClThreads;
    static_assert(P * C == h && RW * C == NN, "the slots and rows split evenly over the cluster");
    static_assert(!LA || P + 1 <= 32, "the look-ahead warp has one lane per pair it forms");
    static_assert(NBUF <= 255, "buffer indices fit the table's byte fields");
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int pair = blockIdx.x / C;
    const int tid = threadIdx.x;
    const int k0 = rank * P;   // first slot owned
    const int w0 = rank * RW;  // first row of W owned
    if (col0 && col0[2 * pair] < 0) {  // a visit the skip mask removed: the whole cluster leaves
        if (rank == 0 && tid == 0) rotated[pair] = 0;
        return;
    }

    extern __shared__ __align__(16) double sm[];
    double *pool = sm;               // [NBUF][NN] rows of A: both rows of every owned slot, one free
    double *Wl = pool + NBUF * NN;   // [RW][NN] rows w0 .. w0 + RW - 1 of W_P
    __shared__ double D[NN];
    __shared__ int sg[NN];
    __shared__ double T[2][h], Cc[2][h], Qv[2][h], Apq[2][h];  // Apq: the true a_pq
    __shared__ int Fl[2][h];         // bit 0: rotate, bit 1: rank deficient
    __shared__ double Sc[NN], Rc[NN];  // column scales of the stored block and their reciprocals
    __shared__ double Al[h], Be[h];    // the step's scaled-rotation coefficients
    __shared__ int s_tot[2];           // rotations counted by warps 0 and 1
    static_assert(h <= 64, "the rotation count lives in warps 0 and 1");
    __shared__ int s_renorm;
    __shared__ int4 tb[3][h];        // ring table rows of steps s, s + 1, s + 2 (at step % 3)
    __shared__ double tr_max[C], tr_sum[C], tr_red[2][kT / 32];

    auto entry = [&](int x, int y) -> double {
        if (!part) return A_io[(size_t)pair * NN * NN + x + y * NN];
        if (!full_part) return assemble_entry<NN>(part, nsplit, pair, x + y * NN);
        const int lo = x < y ? x : y, hi = x < y ? y : x;
        const double *pp = part + (size_t)pair * nsplit * NN * NN + lo + (size_t)hi * NN;
        double v = 0.0;
        for (int s = 0; s < nsplit; ++s) v += pp[(size_t)s * NN * NN];
        return v;
    };
    for (int x = tid; x < NN; x += kT) {
        if (sgn_direct) sg[x] = sgn_direct[(size_t)pair * NN + x];
        else sg[x] = sgn_cols[col0[2 * pair + (x >= B)] + (x % B)];
        D[x] = entry(x, x);
        Sc[x] = 1.0;
        Rc[x] = 1.0;
        if (dexp && rank == 0) dexp[(size_t)pair * NN + x] = D[x] > 0.0 ? (ilogb(D[x]) >> 1) : 0;
    }
    if (tid == 0) s_renorm = 0;
    for (int e = tid; e < 2 * h; e += kT) tb[e / h][e % h] = ring[e];
    __syncthreads();
    // rows of the owned slots at step 0, W = I
    for (int e = tid; e < 2 * P * NN; e += kT) {
        const int r = e / NN, y = e % NN;
        const int4 t = tb[0][k0 + (r >> 1)];
        const int x = (r & 1) ? t.y : t.x, bf = (r & 1) ? ring_buf_hi(t) : ring_buf_lo(t);
        pool[bf * NN + y] = entry(x, y);
    }
    for (int e = tid; e < RW * NN; e += kT) {
        const int x = e / NN, y = e % NN;
        Wl[x * NN + y] = (w0 + x == y) ? 1.0 : 0.0;
    }
    __syncthreads();
    // visit record for the learned form: the I x J block of A_P scaled by the
    // diagonal over the rows this CTA holds, reduced into rank 0
    float rec_meanI = 0.f, rec_meanJ = 0.f, rec_hyp = 0.f;
    double rec_max = 0.0, rec_sum = 0.0;
    if (trace) {
        double lmax = 0.0, lsum = 0.0;
        for (int e = tid; e < 2 * P * B; e += kT) {
            const int r = e / B, y = B + e % B;
            const int4 t = tb[0][k0 + (r >> 1)];
            const int x = (r & 1) ? t.y : t.x, bf = (r & 1) ? ring_buf_hi(t) : ring_buf_lo(t);
            if (x >= B) continue;
            const double dd = D[x] * D[y];
            const double sc = dd > 0.0 ? fabs(pool[bf * NN + y]) / sqrt(dd) : 0.0;
            lmax = fmax(lmax, sc);
            lsum = fma(sc, sc, lsum);
        }
        lmax = warp_max(lmax);
        lsum = warp_sum(lsum);
        if ((tid & 31) == 0) {
            tr_red[0][tid >> 5] = lmax;
            tr_red[1][tid >> 5] = lsum;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 0; w < kT / 32; ++w) {
                rec_max = fmax(rec_max, tr_red[0][w]);
                rec_sum += tr_red[1][w];
            }
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
    cluster.sync();  // every CTA initialised before any remote write
    if (trace && tid == 0) {
        *cluster.map_shared_rank(&tr_max[rank], 0) = rec_max;
        *cluster.map_shared_rank(&tr_sum[rank], 0) = rec_sum;
    }
    // (t, c) of a pair into every CTA (buffer s & 1)
    auto put_params = [&](int s, int k, double t, double c, double qv, double apq, int fl) {
        const int b = s & 1;
        for (int r = 0; r < C; ++r) {
            *cluster.map_shared_rank(&T[b][k], r) = t;
            *cluster.map_shared_rank(&Cc[b][k], r) = c;
            *cluster.map_shared_rank(&Qv[b][k], r) = qv;
            *cluster.map_shared_rank(&Apq[b][k], r) = apq;
            *cluster.map_shared_rank(&Fl[b][k], r) = fl;
        }
    };
    // Lane l <= P forms the step-s pair of slot k0 + l (l = P: the next CTA's
    // first slot) when this CTA holds its row lo at the end of step s - 1:
    // row lo stays in slot k0 + l, or arrives from slot k0 + l - 1 (local for
    // l >= 1; for l = P, this CTA's last slot).
    auto forms = [&](int s, int l) -> bool {
        const int4 e = tb[s % 3][(k0 + l) % h];
        const bool lo_arr = e.w & 1;
        return l < P ? !(lo_arr && l == 0) : lo_arr;
    };
    // step 0: every CTA forms the pairs of its own slots
    if (tid < P) {
        const int k = k0 + tid;
        const int4 e = tb[0][k];
        const double apq = (Sc[e.x] * Sc[e.y]) * pool[ring_buf_lo(e) * NN + e.y];
        const int hyp = (sg[e.x] == sg[e.y]) ? -1 : 1;
        double t, c, qv;
        const int fl = pair_decision_fast(D[e.x], D[e.y], apq, hyp, tol, t, c, qv);
        put_params(0, k, t, c, qv, apq, fl);
    }
    cluster.sync();

    // Warp 0 works one step ahead (LA): lane l reads, at the top of step s,
    // the four entries of the rows of pair i (the slot holding row lo of the
    // step-(s+1) pair) in the columns of pair j (the slot holding its row hi)
    // and the two diagonal values, forms their step-s values with the
    // operations of the bulk update and the (t, c) of the step-(s+1) pair,
    // while warps 1.. update the rows (named barrier 1).
    constexpr int kMixThreads = LA ? kT - 32 : kT;
    const int warp = tid >> 5, lane = tid & 31;
    int total = 0, bad = 0, s_end = NN - 1;
    int big = 0;  // a rotation of pair tid had |t| > tstop (Eq. 4.2 code (11)_2)
    const int mt = LA ? tid - 32 : tid;  // mixing thread index (warps 1.. with the look-ahead)
    for (int s = 0; s < NN; ++s) {
        const int b = s & 1;
        const int4 *cur = tb[s % 3];
        // scales out of range after the last step: the block back to s = r = 1
        if (s_renorm) {
            for (int e = tid; e < (2 * P + RW) * NN; e += kT) {
                const int r = e / NN, y = e % NN;
                if (r < 2 * P) {
                    const int4 t = cur[k0 + (r >> 1)];
                    const int x = (r & 1) ? t.y : t.x, bf = (r & 1) ? ring_buf_hi(t) : ring_buf_lo(t);
                    pool[bf * NN + y] = (Sc[x] * Sc[y]) * pool[bf * NN + y];
                } else {
                    Wl[(r - 2 * P) * NN + y] = Wl[(r - 2 * P) * NN + y] * Sc[y];
                }
            }
            __syncthreads();
            for (int x = tid; x < NN; x += kT) Sc[x] = Rc[x] = 1.0;
            if (tid == 0) s_renorm = 0;
            __syncthreads();
        }
        double nx_t = 0.0, nx_c = 1.0, nx_qv = 1.0, nx_apq = 0.0;
        int nx_fl = 0;
        double e_pp = 0.0, e_pq = 0.0, e_qp = 0.0, e_qq = 0.0, d_lo = 0.0, d_hi = 0.0, s_lo = 1.0, s_hi = 1.0;
        int si = 0, sj = 0;
        bool lo_p = false, hi_p = false, trig_i = false, trig_j = false, trig_n = false;
        const bool ahead = LA && warp == 0 && lane <= P && s + 1 < NN && forms(s + 1, lane);
        if (ahead) {
            const int k = (k0 + lane) % h;
            const int4 ne = tb[(s + 1) % 3][k];
            const bool lo_arr = ne.w & 1;
            si = lo_arr ? (k + h - 1) % h : k;
            sj = lo_arr ? k : (k + h - 1) % h;
            const int4 fi = cur[si], fj = cur[sj];
            const double *rp = pool + ring_buf_lo(fi) * NN, *rq = pool + ring_buf_hi(fi) * NN;
            e_pp = rp[fj.x];
            e_pq = rp[fj.y];
            e_qp = rq[fj.x];
            e_qq = rq[fj.y];
            d_lo = D[ne.x];
            d_hi = D[ne.y];
            s_lo = Sc[ne.x];
            s_hi = Sc[ne.y];
            lo_p = ne.x == fi.x;  // row lo is pair i's first row
            hi_p = ne.y == fj.x;  // column hi is pair j's first column
            trig_i = sg[fi.x] == sg[fi.y];
            trig_j = sg[fj.x] == sg[fj.y];
            trig_n = sg[ne.x] == sg[ne.y];
        }
        // the step's coefficients from its starting scales (alpha by threads
        // [0, h), beta by [h, 2h))
        if (mt >= 0 && mt < 2 * h && (Fl[b][mt % h] & 1)) {
            const int j = mt % h, p = cur[j].x, q = cur[j].y;
            const double t = T[b][j];
            if (mt < h) Al[j] = ((sg[p] == sg[q]) ? -t : t) * (Sc[q] * Rc[p]);
            else Be[j] = t * (Sc[p] * Rc[q]);
        }
        // every CTA sees every pair's flags: the same decision everywhere
        const int f = tid < h ? Fl[b][tid] : 0;
        if (tbig && (f & 1) && fabs(T[b][tid]) > tstop) big = 1;
        bad = __syncthreads_or(f & 2);
        if (bad) {
            s_end = s;
            break;
        }
        // the step's rotations, counted by the warps holding the flags (one
        // CTA barrier per step instead of two); lane 0 of warp w keeps warp
        // w's count
        if (warp * 32 < h) total += __popc(__ballot_sync(0xffffffffu, f & 1));
        if (LA && warp == 0) {
            if (ahead) {
                const int ri = Fl[b][si] & 1, rj = Fl[b][sj] & 1;
                const double ti = T[b][si], hti = trig_i ? -ti : ti;
                const double tj = T[b][sj], htj = trig_j ? -tj : tj;
                const double ali = ri ? Al[si] : 0.0, bei = ri ? Be[si] : 0.0;
                const double alj = rj ? Al[sj] : 0.0, bej = rj ? Be[sj] : 0.0;
                double v;
                if ((s & 1) == 0) {  // column mix (pair j) of rows p_i, q_i, then row mix (pair i)
                    double up = hi_p ? e_pp : e_pq, uq = hi_p ? e_qp : e_qq;
                    if (rj) {
                        up = hi_p ? fma(alj, e_pq, e_pp) : fma(bej, e_pp, e_pq);
                        uq = hi_p ? fma(alj, e_qq, e_qp) : fma(bej, e_qp, e_qq);
                    }
                    v = lo_p ? up : uq;
                    if (ri) v = lo_p ? fma(ali, uq, up) : fma(bei, up, uq);
                } else {  // row mix (pair i) in columns p_j, q_j, then column mix (pair j)
                    double wp = lo_p ? e_pp : e_qp, wq = lo_p ? e_pq : e_qq;
                    if (ri) {
                        wp = lo_p ? fma(ali, e_qp, e_pp) : fma(bei, e_pp, e_qp);
                        wq = lo_p ? fma(ali, e_qq, e_pq) : fma(bei, e_pq, e_qq);
                    }
                    v = hi_p ? wp : wq;
                    if (rj) v = hi_p ? fma(alj, wq, wp) : fma(bej, wp, wq);
                }
                // Eq. 2.6 on the two diagonal entries, the step's new scales of the two rows
                const double app = ri ? fma(lo_p ? hti : ti, Apq[b][si], d_lo) : d_lo;
                const double aqq = rj ? fma(hi_p ? htj : tj, Apq[b][sj], d_hi) : d_hi;
                const double sl = ri ? s_lo * Cc[b][si] : s_lo, sh = rj ? s_hi * Cc[b][sj] : s_hi;
                const double apq = (sl * sh) * v;
                nx_fl = pair_decision_fast(app, aqq, apq, trig_n ? -1 : 1, tol, nx_t, nx_c, nx_qv);
                nx_apq = apq;
            }
        } else {
            // the column mix on every held row of A (and of W): a thread keeps
            // one pair (its rotation in registers) and walks rows
            auto col_mix = [&](bool with_w) {
                static_assert(kMixThreads % h == 0, "whole rows per pass");
                const int j = mt % h;
                if (!(Fl[b][j] & 1)) return;
                const int p = cur[j].x, q = cur[j].y;
                const double al = Al[j], be = Be[j];
                const int nrows = 2 * P + (with_w ? RW : 0);
                for (int r = mt / h; r < nrows; r += kMixThreads / h) {
                    double *row;
                    if (r < 2 * P) {
                        const int4 e = cur[k0 + (r >> 1)];
                        row = pool + ((r & 1) ? ring_buf_hi(e) : ring_buf_lo(e)) * NN;
                    } else {
                        row = Wl + (r - 2 * P) * NN;
                    }
                    const double a = row[p], bb = row[q];
                    row[p] = fma(al, bb, a);
                    row[q] = fma(be, a, bb);
                }
            };
            // the row mix of every owned slot's pair, every column; with W,
            // also W's column mix
            auto row_mix = [&](bool with_w) {
                static_assert(kMixThreads % P == 0, "threads split evenly over the owned slots");
                constexpr int TP = kMixThreads / P;  // threads per owned slot
                const int kl = mt / TP, k = k0 + kl;
                if (Fl[b][k] & 1) {
                    const int4 e = cur[k];
                    const double al = Al[k], be = Be[k];
                    double *rp = pool + ring_buf_lo(e) * NN, *rq = pool + ring_buf_hi(e) * NN;
                    for (int y = mt % TP; y < NN; y += TP) {
                        const double a = rp[y], bb = rq[y];
                        rp[y] = fma(al, bb, a);
                        rq[y] = fma(be, a, bb);
                    }
                }
                if (!with_w) return;
                const int j = mt % h;
                if (!(Fl[b][j] & 1)) return;
                const int pw = cur[j].x, qw = cur[j].y;
                const double al = Al[j], be = Be[j];
                for (int x = mt / h; x < RW; x += kMixThreads / h) {
                    double *row = Wl + x * NN;
                    const double a = row[pw], bb = row[qw];
                    row[pw] = fma(al, bb, a);
                    row[qw] = fma(be, a, bb);
                }
            };
            if ((s & 1) == 0) {
                col_mix(true);
                mix_sync<LA>(kMixThreads);
                row_mix(false);
            } else {
                row_mix(true);
                mix_sync<LA>(kMixThreads);
                col_mix(false);
            }
            mix_sync<LA>(kMixThreads);
            // Eq. 2.6 on the replicated diagonal and the owned pairs' own
            // stored entries to 0, the new scales and their reciprocals of
            // the rotated rows, in three warp groups (as in the cross pass)
            static_assert(kMixThreads >= 3 * h, "three groups of h mixing threads");
            if (mt < 3 * h && (Fl[b][mt % h] & 1)) {
                const int j = mt % h;
                const int4 e = cur[j];
                const int p = e.x, q = e.y;
                if (mt < h) {
                    const double t = T[b][j], ht = (sg[p] == sg[q]) ? -t : t, apq = Apq[b][j];
                    D[p] = fma(ht, apq, D[p]);
                    D[q] = fma(t, apq, D[q]);
                    if (j >= k0 && j < k0 + P) {
                        double *rp = pool + ring_buf_lo(e) * NN, *rq = pool + ring_buf_hi(e) * NN;
                        rp[p] = 0.0;
                        rp[q] = 0.0;
                        rq[q] = 0.0;
                        rq[p] = 0.0;
                    }
                } else if (mt < 2 * h) {
                    const double c = Cc[b][j];
                    Sc[p] = Sc[p] * c;
                    Sc[q] = Sc[q] * c;
                    if (scale_out_of_range(Sc[p]) || scale_out_of_range(Sc[q])) s_renorm = 1;
                } else {
                    const double qv = Qv[b][j];
                    Rc[p] = Rc[p] * qv;
                    Rc[q] = Rc[q] * qv;
                }
            }
        }
        __syncthreads();
        if (s + 1 < NN) {
            const int4 *nxt = tb[(s + 1) % 3];
            // the row leaving the last owned slot: the row arriving in slot
            // k0 + P at step s + 1, into its buffer in the next CTA
            {
                const int4 en = nxt[(k0 + P) % h];
                const bool lo_arr = en.w & 1;
                const int mv = lo_arr ? en.x : en.y, dbf = lo_arr ? ring_buf_lo(en) : ring_buf_hi(en);
                const int4 el = cur[k0 + P - 1];
                const int sbf = el.x == mv ? ring_buf_lo(el) : ring_buf_hi(el);
                double *rdst = cluster.map_shared_rank(pool, (rank + 1) % C) + dbf * NN;
                const double *src = pool + sbf * NN;
                for (int y = tid; y < NN; y += kT) rdst[y] = src[y];
            }
            if (!LA && tid <= P && forms(s + 1, tid)) {
                // row lo of the step-(s+1) pair, where it is at step s
                const int k = (k0 + tid) % h;
                const int4 e = nxt[k];
                const int4 fl = cur[(e.w & 1) ? (k + h - 1) % h : k];
                const int bf = fl.x == e.x ? ring_buf_lo(fl) : ring_buf_hi(fl);
                const double apq = (Sc[e.x] * Sc[e.y]) * pool[bf * NN + e.y];
                const int hyp = (sg[e.x] == sg[e.y]) ? -1 : 1;
                double t, c, qv;
                const int fd = pair_decision_fast(D[e.x], D[e.y], apq, hyp, tol, t, c, qv);
                put_params(s + 1, k, t, c, qv, apq, fd);
            }
            if (ahead) put_params(s + 1, (k0 + lane) % h, nx_t, nx_c, nx_qv, nx_apq, nx_fl);
            // the table row of step s + 2 into the slot of step s - 1
            if (s + 2 < NN)
                for (int e = tid; e < h; e += kT) tb[(s + 2) % 3][e] = ring[(size_t)(s + 2) * h + e];
        }
        cluster.sync();
    }
    // outputs: own rows of W (column-major W_P), and A_P when asked for
    double *wo = Wout + (size_t)pair * NN * NN;
    for (int e = tid; e < RW * NN; e += kT) {
        const int x = e / NN, y = e % NN;
        wo[(w0 + x) + (size_t)y * NN] = Wl[x * NN + y] * Sc[y];
    }
    if (!part) {
        // the rows of the owned slots where the pass ended: true values
        // (s_x s_y) S_xy, the diagonal from D
        double *ao = A_io + (size_t)pair * NN * NN;
        const int4 *at = tb[s_end % 3];
        for (int e = tid; e < 2 * P * NN; e += kT) {
            const int r = e / NN, y = e % NN;
            const int4 t = at[k0 + (r >> 1)];
            const int x = (r & 1) ? t.y : t.x, bf = (r & 1) ? ring_buf_hi(t) : ring_buf_lo(t);
            ao[x + (size_t)y * NN] = x == y ? D[x] : (Sc[x] * Sc[y]) * pool[bf * NN + y];
        }
    }
    if (lane == 0 && warp * 32 < h) s_tot[warp] = total;
    cluster.sync();
    const int any_big = tbig ? __syncthreads_or(big) : 0;
    if (rank == 0 && tid == 0) {
        total = 0;
        for (int w = 0; w * 32 < h; ++w) total += s_tot[w];
        rotated[pair] = total;
        if (rot_count && total) atomicAdd(rot_count, (unsigned long long)total);
        if (bad && status) atomicExch(status, HSVD_ERR_RANK);
        if (any_big) atomicOr(tbig, 1);
        if (trace) {
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
}

template <int NN>
cudaError_t solve_cluster_impl(int npairs, const double *part, int nsplit, int full_part, double *A,
                               const int8_t *sgn_cols, const int *col0, const int8_t *sgn_direct, double tol,
                               int mode, int max_passes, const int *tab_full, const int *tab_cross, double *Wp,
                               int *rotated, unsigned long long *rot_count, int *status, int *dexp,
                               const int *visit, float *trace, double tstop, int *tbig, cudaStream_t st) {
    constexpr int C = ClusterOf<NN>::C, R = NN / C;
    if (mode == 1) {
        constexpr int CX = CrossClusterOf<NN>::C, P = NN / 2 / CX, RX = NN / CX;
        const size_t smem_x = (size_t)(P * NN + (P + 1) * NN + RX * NN) * sizeof(double);
        // the look-ahead warp pays at b = 64 (measured), not at b <= 32
        constexpr bool LA = NN >= 128;
        constexpr int threads = LA ? kCrossThreads : kClThreads;
        cudaError_t e = cudaFuncSetAttribute(k_solve_cross<NN, CX, LA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_x);
        if (e != cudaSuccess) return e;
        k_solve_cross<NN, CX, LA><<<npairs * CX, threads, smem_x, st>>>(part, nsplit, full_part, A, sgn_cols, col0,
                                                                     sgn_direct, tol, Wp, rotated, rot_count,
                                                                     status, dexp, visit, trace, tstop, tbig);
        return cudaGetLastError();
    }
    if (mode == 2) {
        constexpr int CX = CrossClusterOf<NN>::C, P = NN / 2 / CX, RX = NN / CX;
        const size_t smem_r = (size_t)((2 * P + 1) * NN + RX * NN) * sizeof(double);
        constexpr bool LA = NN >= 128;
        constexpr int threads = LA ? kCrossThreads : kClThreads;
        const int4 *ring = reinterpret_cast<const int4 *>(tab_full + (size_t)NN * (NN / 2) * 2);
        cudaError_t e = cudaFuncSetAttribute(k_solve_ring<NN, CX, LA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_r);
        if (e != cudaSuccess) return e;
        k_solve_ring<NN, CX, LA><<<npairs * CX, threads, smem_r, st>>>(part, nsplit, full_part, A, sgn_cols, col0,
                                                                    sgn_direct, tol, ring, Wp, rotated, rot_count,
                                                                    status, dexp, visit, trace, tstop, tbig);
        return cudaGetLastError();
    }
    const size_t smem = (size_t)(2 * R * (NN + 1) + R * NN) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_solve_cluster<NN, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_solve_cluster<NN, C><<<npairs * C, kClThreads, smem, st>>>(part, nsplit, full_part, A, sgn_cols, col0,
                                                                 sgn_direct, tol, mode, max_passes, tab_full,
                                                                 tab_cross, Wp, rotated, rot_count, status, dexp,
                                                                 visit, trace, tstop, tbig);
    return cudaGetLastError();
}

}  // namespace

// Cluster size of the ring kernel for block width b (CrossClusterOf).
static int ring_cluster(int b) { return b == 16 ? 4 : 8; }

size_t ring_table_ints(int b) { return (size_t)(2 * b) * b * 4; }

// The ring of the full pass (k_solve_ring): step 0's slots are the modulus
// pairs of step 0 in their order; at every later step the pair holding one
// row of slot k and one row of slot k - 1 (cyclically) takes slot k, the row
// from slot k - 1 being the one that moved.  Rows keep their pool buffer
// while they move inside a CTA; a row crossing into the next CTA takes that
// CTA's free buffer, and the buffer it leaves becomes the sender's free one.
// Entry [s][k] = {lo, hi, buf_lo | buf_hi << 8, lo arrived}.
bool fill_ring(int b, int *tab) {
    if (b != 16 && b != 32 && b != 64) return false;
    const int nn = 2 * b, h = b, C = ring_cluster(b), P = h / C;
    std::vector<int> slot_lo(h), slot_hi(h), where(nn), buf(nn), freeb(C, 2 * P);
    std::vector<int> nlo(h, -1), nhi(h), narr(h);
    for (int k = 0; k < h; ++k) {
        int lo, hi;
        modulus_pair(nn, 0, k, lo, hi);
        slot_lo[k] = lo;
        slot_hi[k] = hi;
        buf[lo] = 2 * (k % P);
        buf[hi] = 2 * (k % P) + 1;
        int *e = tab + 4 * k;
        e[0] = lo;
        e[1] = hi;
        e[2] = buf[lo] | (buf[hi] << 8);
        e[3] = 0;
    }
    for (int s = 1; s < nn; ++s) {
        for (int k = 0; k < h; ++k) {
            where[slot_lo[k]] = k;
            where[slot_hi[k]] = k;
            nlo[k] = -1;
        }
        for (int j = 0; j < h; ++j) {
            int lo, hi;
            modulus_pair(nn, s, j, lo, hi);
            const int kl = where[lo], kh = where[hi];
            int k, arr;
            if ((kl + h - 1) % h == kh) { k = kl; arr = 0; }       // row hi came from slot k - 1
            else if ((kh + h - 1) % h == kl) { k = kh; arr = 1; }  // row lo came from slot k - 1
            else return false;
            if (nlo[k] >= 0) return false;
            nlo[k] = lo;
            nhi[k] = hi;
            narr[k] = arr;
        }
        // rows crossing into CTA r's first slot take its free buffer; the
        // buffer the crossing row leaves in CTA r - 1 becomes that CTA's free one
        std::vector<int> nfree(C);
        for (int r = 0; r < C; ++r) {
            const int k = r * P, mv = narr[k] ? nlo[k] : nhi[k];
            nfree[(r + C - 1) % C] = buf[mv];
            buf[mv] = freeb[r];
        }
        freeb = nfree;
        for (int k = 0; k < h; ++k) {
            slot_lo[k] = nlo[k];
            slot_hi[k] = nhi[k];
            int *e = tab + 4 * ((size_t)s * h + k);
            e[0] = nlo[k];
            e[1] = nhi[k];
            e[2] = buf[nlo[k]] | (buf[nhi[k]] << 8);
            e[3] = narr[k];
        }
    }
    return true;
}

cudaError_t launch_solve(int b, int npairs, const double *part, int nsplit, double *A, const int8_t *sgn_cols,
                         const int *col0, const int8_t *sgn_direct, double tol, int mode, int max_passes,
                         const int *tab_full, const int *tab_cross, double *Wp, int *rotated,
                         unsigned long long *rot_count, int *status, cudaStream_t st, int full_part, int *dexp,
                         const int *visit, float *trace, double tstop, int *tbig) {
    switch (b) {
        case 16: return solve_cluster_impl<32>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct, tol,
                                               mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                               status, dexp, visit, trace, tstop, tbig, st);
        case 32: return solve_cluster_impl<64>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct, tol,
                                               mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                               status, dexp, visit, trace, tstop, tbig, st);
        case 64: return solve_cluster_impl<128>(npairs, part, nsplit, full_part, A, sgn_cols, col0, sgn_direct,
                                                tol, mode, max_passes, tab_full, tab_cross, Wp, rotated, rot_count,
                                                status, dexp, visit, trace, tstop, tbig, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hsvd
