// pw_core.cuh -- the per-factor body of the pointwise one-sided hyperbolic
// Jacobi method (Sec. 2, Alg. 4.5), shared by the single-factor kernel
// (pointwise.cu) and the persistent batched kernel (batched.cu).
//
// A group of NT threads (a whole CTA, or an aligned part of one that
// synchronises on its own named barrier `bar`) owns one factor for all sweeps.  G (column-major, rows
// padded to a multiple of 32) and the accumulated transformation W (the paper's
// V^{-T}, Eq. 2.1) sit wherever the caller put them: shared memory when they
// fit, otherwise global memory (L2-resident at these sizes).  A step of the
// modified modulus strategy (Sec. 2) has n'/2 disjoint pairs; warp w takes
// pairs w, w + NT/32, ...  For each pair the warp recomputes a_ii, a_jj, a_ij
// from the current columns (lane l owns rows l, l+32, ...; xor-butterfly
// reduction, so every lane holds the same sums), applies the test of Eq. 2.3,
// computes (t, c) redundantly in all lanes (uniform control flow, no divergence
// between the two rotation kinds inside a warp) and updates its two columns of
// G and of W with the FMA form of Alg. 4.5.  One group barrier separates
// steps.  The convergence check is the bit-or reduction of Eq. 4.2 held in two
// shared words: the sweep's rotation count (code (00)_2 when it is zero) and,
// with the tangent threshold T on, a flag set by any rotation with |t| > T
// (code (11)_2); a sweep that rotated without setting it is code (01)_2 and
// also ends the iteration.  No host round trip is needed between sweeps.
//
// Columns are never moved: positions map to columns through pos[] (Sec. 4).
// Before the first sweep positions are grouped J+ then J- (Alg. 4.2 assumes
// J = diag(I_p, -I_{n-p})); with sorting on they are then ordered by
// d = ||g||^2, decreasing in the J+ part and increasing in the J- part, ties in
// current order (Sec. 4, Sort_Diagonal), again after every sweep.  An odd n is
// bordered with one unit column in a fresh row (Eq. 4.1).
#pragma once

#include "hsvd_internal.cuh"

namespace hsvd {

// the factor's working arrays: G (m_pad x n_pad), W (n_pad x n_pad), and the
// per-column arrays d (doubles), pos, newpos, sg (ints), all n_pad long
struct PwArrays {
    double *G;
    double *W;
    double *d;
    int *pos;
    int *newpos;
    int *sg;
};

// a_pp, a_qq, a_pq of columns gp, gq (length len, a multiple of 32): lane l
// sums rows l, l + 32, ... in order; four loads are issued ahead of their
// FMAs so that columns in global memory stream (same arithmetic either way)
__device__ __forceinline__ void pw_dots(const double *__restrict__ gp, const double *__restrict__ gq, int len,
                                        int lane, double &app, double &aqq, double &apq) {
    constexpr int U = 4;
    int i = lane;
    for (; i + (U - 1) * kWarp < len; i += U * kWarp) {
        double x[U], y[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            x[u] = gp[i + u * kWarp];
            y[u] = gq[i + u * kWarp];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            app = fma(x[u], x[u], app);
            aqq = fma(y[u], y[u], aqq);
            apq = fma(x[u], y[u], apq);
        }
    }
    for (; i < len; i += kWarp) {
        const double x = gp[i], y = gq[i];
        app = fma(x, x, app);
        aqq = fma(y, y, aqq);
        apq = fma(x, y, apq);
    }
}

// the column update of Alg. 4.5 on columns gp, gq (distinct), same loads-ahead scheme
__device__ __forceinline__ void pw_rotate(double *__restrict__ gp, double *__restrict__ gq, int len, int lane,
                                          double ht, double t, double c) {
    constexpr int U = 4;
    int i = lane;
    for (; i + (U - 1) * kWarp < len; i += U * kWarp) {
        double x[U], y[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            x[u] = gp[i + u * kWarp];
            y[u] = gq[i + u * kWarp];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            gp[i + u * kWarp] = fma(ht, y[u], x[u]) * c;
            gq[i + u * kWarp] = fma(t, x[u], y[u]) * c;
        }
    }
    for (; i < len; i += kWarp) {
        const double x = gp[i], y = gq[i];
        gp[i] = fma(ht, y, x) * c;
        gq[i] = fma(t, x, y) * c;
    }
}

// barrier of a group of NT threads (NT a multiple of 32; id 0 with NT equal
// to the CTA size is __syncthreads)
template <int NT>
__device__ __forceinline__ void grp_sync(int bar) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(NT) : "memory");
}

// shared scalars of a group
struct PwScalars {
    int rot, err, bad, big;
    unsigned long long total;
};

template <int NT>
__device__ void pw_reorder(const PwArrays &sh, int m_pad, int n_pad, int use_d, int bar) {
    constexpr int kW = NT / kWarp;
    const int tid = threadIdx.x & (NT - 1), lane = tid & 31, warp = tid >> 5;
    if (use_d) {
        for (int j = warp; j < n_pad; j += kW) {
            const double *g = sh.G + (size_t)j * m_pad;
            double s = 0.0;
            for (int i = lane; i < m_pad; i += kWarp) s = fma(g[i], g[i], s);
            s = warp_sum(s);
            if (lane == 0) sh.d[j] = s;
        }
    }
    grp_sync<NT>(bar);
    int nplus = 0;
    for (int a = 0; a < n_pad; ++a) nplus += sh.sg[sh.pos[a]] > 0;
    for (int a = tid; a < n_pad; a += NT) {
        const int col = sh.pos[a];
        const int grp = sh.sg[col];
        const double key = use_d ? sh.d[col] : 0.0;
        int rank = 0;
        for (int b = 0; b < n_pad; ++b) {
            const int cb = sh.pos[b];
            if (sh.sg[cb] != grp || b == a) continue;
            const double kb = use_d ? sh.d[cb] : 0.0;
            const bool before = (grp > 0) ? (kb > key) : (kb < key);
            if (before || (kb == key && b < a)) ++rank;
        }
        sh.newpos[(grp > 0 ? 0 : nplus) + rank] = col;
    }
    grp_sync<NT>(bar);
    for (int a = tid; a < n_pad; a += NT) sh.pos[a] = sh.newpos[a];
    grp_sync<NT>(bar);
}

// Solves one factor; every thread of the group calls it.  Writes status, sweeps,
// the rotation count and the stop rule (HSVD_STOP_*) through out_status /
// out_sweeps / out_rot / out_rule (thread 0; out_rule may be null).  tstop > 0
// is the tangent threshold of the early stop (Sec. 2), 0 turns it off.
template <int NT>
__device__ void pw_solve(const double *__restrict__ G, int64_t ldg, int m, int n, const int8_t *__restrict__ J,
                         int m_pad, int n_pad, double tol, double tstop, int max_sweeps, int sort,
                         const PwArrays &sh, PwScalars &sc, double *__restrict__ sigma, double *__restrict__ U,
                         int64_t ldu, double *__restrict__ V, int64_t ldv, int *out_status, int *out_sweeps,
                         long long *out_rot, int *out_rule, int bar) {
    constexpr int kW = NT / kWarp;
    const int tid = threadIdx.x & (NT - 1), lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        sc.rot = 0;
        sc.err = 0;
        sc.bad = 0;
        sc.big = 0;
        sc.total = 0;
    }
    grp_sync<NT>(bar);

    // load and border (Eq. 4.1): pad columns are unit vectors in fresh rows
    int bad = 0;
    for (int j = warp; j < n_pad; j += kW) {
        double *g = sh.G + (size_t)j * m_pad;
        for (int i = lane; i < m_pad; i += kWarp) {
            double v = 0.0;
            if (j < n) {
                if (i < m) v = G[i + (int64_t)j * ldg];
            } else if (i == m + (j - n)) {
                v = 1.0;
            }
            bad |= !isfinite(v);
            g[i] = v;
        }
    }
    for (int64_t e = tid; e < (int64_t)n_pad * n_pad; e += NT) {
        const int64_t i = e % n_pad, j = e / n_pad;
        sh.W[e] = (i == j) ? 1.0 : 0.0;
    }
    if (bad) atomicOr(&sc.bad, 1);
    for (int j = tid; j < n_pad; j += NT) {
        const int sj = (j < n) ? (int)J[j] : 1;
        sh.sg[j] = sj > 0 ? 1 : -1;
        if (sj != 1 && sj != -1) atomicOr(&sc.bad, 2);
    }
    grp_sync<NT>(bar);
    if (sc.bad) {
        const int b = sc.bad;
        grp_sync<NT>(bar);
        if (tid == 0) {
            *out_status = (b & 2) ? HSVD_ERR_ARG : HSVD_ERR_NONFINITE;
            *out_sweeps = 0;
            *out_rot = 0;
            if (out_rule) *out_rule = HSVD_STOP_NONE;
        }
        return;
    }
    // initial positions: J+ columns in index order, then J- columns
    for (int j = tid; j < n_pad; j += NT) {
        int before = 0;
        for (int i = 0; i < j; ++i) before += (sh.sg[i] > 0) == (sh.sg[j] > 0);
        int nplus = 0;
        if (sh.sg[j] < 0)
            for (int i = 0; i < n_pad; ++i) nplus += sh.sg[i] > 0;
        sh.pos[(sh.sg[j] > 0 ? 0 : nplus) + before] = j;
    }
    grp_sync<NT>(bar);
    if (sort) pw_reorder<NT>(sh, m_pad, n_pad, 1, bar);

    long long rot_total = 0;
    int sweep = 0, status = HSVD_NOT_CONVERGED, rule = HSVD_STOP_NONE;
    const int half = n_pad / 2;
    for (sweep = 1; sweep <= max_sweeps; ++sweep) {
        for (int s = 0; s < n_pad; ++s) {
            // A warp takes the pairs k = warp, warp + kW, ... in batches of up
            // to 32: the dots of every pair of the batch, then lane j computes
            // pair j's rotation, then the column updates.  Pairs of a step are
            // disjoint, so this is the same as one pair after the other.  The
            // dots are reduced four pairs at a time: a butterfly that halves
            // the values a lane carries at the first two levels (lanes with bit
            // 4 clear keep pairs 0-1, bit 3 clear the first of those), then sums
            // the eight lanes that hold the same pair; 18 shuffle-adds for four
            // pairs instead of 15 per pair.
            for (int k0 = warp; k0 < half; k0 += 32 * kW) {
                const int nbatch = min(32, (half - k0 + kW - 1) / kW);
                double my_app = 0.0, my_aqq = 0.0, my_apq = 0.0;
                int my_p = 0, my_q = 0;
                if (lane < nbatch) {
                    int a, b;
                    modulus_pair(n_pad, s, k0 + lane * kW, a, b);
                    my_p = sh.pos[a];
                    my_q = sh.pos[b];
                }
                for (int j0 = 0; j0 < nbatch; j0 += 4) {
                    double v[12];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        double app = 0.0, aqq = 0.0, apq = 0.0;
                        if (j0 + u < nbatch) {
                            const int p = __shfl_sync(0xffffffffu, my_p, j0 + u);
                            const int q = __shfl_sync(0xffffffffu, my_q, j0 + u);
                            pw_dots(sh.G + (size_t)p * m_pad, sh.G + (size_t)q * m_pad, m_pad, lane, app, aqq, apq);
                        }
                        v[3 * u] = app;
                        v[3 * u + 1] = aqq;
                        v[3 * u + 2] = apq;
                    }
                    const bool h16 = lane & 16, h8 = lane & 8;
                    double w[6], x[3];
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        const double send = h16 ? v[i] : v[6 + i];
                        w[i] = (h16 ? v[6 + i] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const double send = h8 ? w[i] : w[3 + i];
                        x[i] = (h8 ? w[3 + i] : w[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        x[i] += __shfl_xor_sync(0xffffffffu, x[i], 4);
                        x[i] += __shfl_xor_sync(0xffffffffu, x[i], 2);
                        x[i] += __shfl_xor_sync(0xffffffffu, x[i], 1);
                    }
                    // lanes 8u .. 8u + 7 hold pair j0 + u; lane j0 + u takes it
                    const int src = 8 * ((lane - j0) & 3);
                    const double s0 = __shfl_sync(0xffffffffu, x[0], src);
                    const double s1 = __shfl_sync(0xffffffffu, x[1], src);
                    const double s2 = __shfl_sync(0xffffffffu, x[2], src);
                    if (lane >= j0 && lane < j0 + 4) {
                        my_app = s0;
                        my_aqq = s1;
                        my_apq = s2;
                    }
                }
                double my_t = 0.0, my_c = 1.0;
                int my_rot = 0;
                const int my_hyp = (sh.sg[my_p] == sh.sg[my_q]) ? -1 : 1;
                if (lane < nbatch) {
                    const int d = pair_decision(my_app, my_aqq, my_apq, my_hyp, tol, my_t, my_c);
                    my_rot = d == 1;
                    if (d == 2) atomicExch(&sc.err, HSVD_ERR_RANK);
                }
                const unsigned rmask = __ballot_sync(0xffffffffu, my_rot);
                if (tstop > 0.0 && __any_sync(0xffffffffu, my_rot && fabs(my_t) > tstop) && lane == 0)
                    sc.big = 1;
                for (int j = 0; j < nbatch; ++j) {
                    if (!((rmask >> j) & 1u)) continue;
                    const double t = __shfl_sync(0xffffffffu, my_t, j), c = __shfl_sync(0xffffffffu, my_c, j);
                    const int hyp = __shfl_sync(0xffffffffu, my_hyp, j);
                    const int p = __shfl_sync(0xffffffffu, my_p, j), q = __shfl_sync(0xffffffffu, my_q, j);
                    const double ht = hyp < 0 ? -t : t;
                    pw_rotate(sh.G + (size_t)p * m_pad, sh.G + (size_t)q * m_pad, m_pad, lane, ht, t, c);
                    pw_rotate(sh.W + (size_t)p * n_pad, sh.W + (size_t)q * n_pad, n_pad, lane, ht, t, c);
                }
                if (lane == 0 && rmask) {
                    atomicAdd(&sc.rot, __popc(rmask));
                    rot_total += __popc(rmask);
                }
            }
            grp_sync<NT>(bar);
            if (sc.err) break;
        }
        if (sc.err) {
            status = sc.err;
            break;
        }
        const int nrot = sc.rot, big = sc.big;
        grp_sync<NT>(bar);
        if (tid == 0) {
            sc.rot = 0;
            sc.big = 0;
        }
        if (nrot == 0 || (tstop > 0.0 && !big)) {  // (00)_2 or (01)_2 of Eq. 4.2
            status = HSVD_OK;
            rule = nrot == 0 ? HSVD_STOP_ORTHO : HSVD_STOP_TANGENT;
            break;
        }
        if (sort) pw_reorder<NT>(sh, m_pad, n_pad, 1, bar);
        else grp_sync<NT>(bar);
    }
    if (sweep > max_sweeps) sweep = max_sweeps;
    grp_sync<NT>(bar);

    // finalisation (Sec. 2): sigma_j = ||g_j||, u_j = g_j / sigma_j, V = W
    if (status == HSVD_OK || status == HSVD_NOT_CONVERGED) {
        for (int j = warp; j < n; j += kW) {
            const double *g = sh.G + (size_t)j * m_pad;
            double mx = 0.0;
            for (int i = lane; i < m; i += kWarp) mx = fmax(mx, fabs(g[i]));
            mx = warp_max(mx);
            int e;
            const double scl = pow2_scale_for(mx, e);
            double ss = 0.0;
            for (int i = lane; i < m; i += kWarp) {
                const double v = g[i] * scl;
                ss = fma(v, v, ss);
            }
            ss = warp_sum(ss);
            const double sj = ldexp(sqrt(ss), e);
            if (lane == 0) {
                sigma[j] = sj;
                if (!(sj > 0.0)) atomicExch(&sc.err, HSVD_ERR_RANK);
                if (!isfinite(sj)) atomicExch(&sc.err, HSVD_ERR_NONFINITE);
            }
            if (U)
                for (int i = lane; i < m; i += kWarp) U[i + (int64_t)j * ldu] = g[i] / sj;
            if (V)
                for (int i = lane; i < n; i += kWarp) V[i + (int64_t)j * ldv] = sh.W[i + (size_t)j * n_pad];
        }
        grp_sync<NT>(bar);
        if (sc.err) status = sc.err;
    }
    if (lane == 0 && rot_total) atomicAdd(&sc.total, (unsigned long long)rot_total);
    grp_sync<NT>(bar);
    if (tid == 0) {
        *out_status = status;
        *out_sweeps = sweep;
        *out_rot = (long long)sc.total;
        if (out_rule) *out_rule = status == HSVD_OK ? rule : HSVD_STOP_NONE;
    }
    grp_sync<NT>(bar);
}

// rows of G's working copy: m plus the bordering row of an odd n, rounded up to 32
__host__ __device__ inline int pw_rows_pad(int64_t m, int64_t n) {
    const int64_t n_pad = n + (n & 1);
    const int64_t rows = m + (n_pad - n);
    return (int)((rows + 31) / 32 * 32);
}

// shared bytes of the per-column arrays (d, pos, newpos, sg)
__host__ __device__ inline size_t pw_aux_bytes(int64_t n_pad) {
    return (size_t)n_pad * (sizeof(double) + 3 * sizeof(int));
}

}  // namespace hsvd
