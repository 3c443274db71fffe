// pointwise.cu -- the pointwise one-sided hyperbolic Jacobi method (Sec. 2,
// Alg. 4.5) for a factor small enough to live in one SM's shared memory.
//
// One CTA of 1024 threads owns the whole problem for all sweeps: G sits in
// shared memory (column-major, rows padded to a multiple of 32), the
// accumulated transformation W (the paper's V^{-T}, Eq. 2.1) in global memory
// (L2-resident at these sizes).  A step of the modified modulus strategy
// (Sec. 2) has n'/2 disjoint pairs; warp w takes pairs w, w+32, ...  For each
// pair the warp recomputes a_ii, a_jj, a_ij from the current columns (lane l
// owns rows l, l+32, ...; xor-butterfly reduction, so every lane holds the
// same sums), applies the test of Eq. 2.3, computes (t, c) redundantly in all
// lanes (uniform control flow, no divergence between the two rotation kinds
// inside a warp) and updates its two columns of G and of W with the FMA form
// of Alg. 4.5.  One __syncthreads separates steps.  The convergence check is a
// shared counter (the bit-or reduction of Eq. 4.2 collapses to "any rotation
// in this sweep"), so no host round trip is needed between sweeps.
//
// Columns are never moved: positions map to columns through pos[] (Sec. 4).
// Before the first sweep positions are grouped J+ then J- (Alg. 4.2 assumes
// J = diag(I_p, -I_{n-p})); with sorting on they are then ordered by
// d = ||g||^2, decreasing in the J+ part and increasing in the J- part, ties in
// current order (Sec. 4, Sort_Diagonal), again after every sweep.  An odd n is
// bordered with one unit column in a fresh row (Eq. 4.1).
#include "hsvd_internal.cuh"

namespace hsvd {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / kWarp;

// shared layout: G (m_pad * n_pad doubles) | d (n_pad doubles) | pos, newpos (ints) | sg (ints)
struct PwShared {
    double *G;
    double *d;
    int *pos;
    int *newpos;
    int *sg;
};

__device__ void pw_reorder(const PwShared &sh, int m_pad, int n_pad, int use_d) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (use_d) {
        for (int j = warp; j < n_pad; j += kWarps) {
            const double *g = sh.G + (size_t)j * m_pad;
            double s = 0.0;
            for (int i = lane; i < m_pad; i += kWarp) s = fma(g[i], g[i], s);
            s = warp_sum(s);
            if (lane == 0) sh.d[j] = s;
        }
    }
    __syncthreads();
    int nplus = 0;
    for (int a = 0; a < n_pad; ++a) nplus += sh.sg[sh.pos[a]] > 0;
    for (int a = tid; a < n_pad; a += kThreads) {
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
    __syncthreads();
    for (int a = tid; a < n_pad; a += kThreads) sh.pos[a] = sh.newpos[a];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1)
k_pointwise(const double *__restrict__ G, int64_t ldg, int m, int n, const int8_t *__restrict__ J,
            int m_pad, int n_pad, double tol, int max_sweeps, int sort, double *__restrict__ W,
            double *__restrict__ sigma, double *__restrict__ U, int64_t ldu, double *__restrict__ V,
            int64_t ldv, int *__restrict__ out, long long *__restrict__ rot_out) {
    extern __shared__ __align__(16) double smem[];
    PwShared sh;
    sh.G = smem;
    sh.d = sh.G + (size_t)m_pad * n_pad;
    sh.pos = reinterpret_cast<int *>(sh.d + n_pad);
    sh.newpos = sh.pos + n_pad;
    sh.sg = sh.newpos + n_pad;
    __shared__ int s_rot, s_err, s_bad;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) { s_rot = 0; s_err = 0; s_bad = 0; }
    __syncthreads();

    // load and border (Eq. 4.1): pad columns are unit vectors in fresh rows
    int bad = 0;
    for (int j = warp; j < n_pad; j += kWarps) {
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
    for (int64_t e = tid; e < (int64_t)n_pad * n_pad; e += kThreads) {
        const int64_t i = e % n_pad, j = e / n_pad;
        W[e] = (i == j) ? 1.0 : 0.0;
    }
    if (bad) atomicOr(&s_bad, 1);
    for (int j = tid; j < n_pad; j += kThreads) {
        const int sj = (j < n) ? (int)J[j] : 1;
        sh.sg[j] = sj > 0 ? 1 : -1;
        if (sj != 1 && sj != -1) atomicOr(&s_bad, 2);
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            out[0] = (s_bad & 2) ? HSVD_ERR_ARG : HSVD_ERR_NONFINITE;
            out[1] = 0;
            *rot_out = 0;
        }
        return;
    }
    // initial positions: J+ columns in index order, then J- columns
    for (int j = tid; j < n_pad; j += kThreads) {
        int before = 0;
        for (int i = 0; i < j; ++i) before += (sh.sg[i] > 0) == (sh.sg[j] > 0);
        int nplus = 0;
        if (sh.sg[j] < 0)
            for (int i = 0; i < n_pad; ++i) nplus += sh.sg[i] > 0;
        sh.pos[(sh.sg[j] > 0 ? 0 : nplus) + before] = j;
    }
    __syncthreads();
    if (sort) pw_reorder(sh, m_pad, n_pad, 1);

    long long rot_total = 0;
    int sweep = 0, status = HSVD_NOT_CONVERGED;
    const int half = n_pad / 2;
    for (sweep = 1; sweep <= max_sweeps; ++sweep) {
        for (int s = 0; s < n_pad; ++s) {
            for (int k = warp; k < half; k += kWarps) {
                int a, b;
                modulus_pair(n_pad, s, k, a, b);
                const int p = sh.pos[a], q = sh.pos[b];
                double *gp = sh.G + (size_t)p * m_pad, *gq = sh.G + (size_t)q * m_pad;
                double app = 0.0, aqq = 0.0, apq = 0.0;
                for (int i = lane; i < m_pad; i += kWarp) {
                    const double x = gp[i], y = gq[i];
                    app = fma(x, x, app);
                    aqq = fma(y, y, aqq);
                    apq = fma(x, y, apq);
                }
                app = warp_sum(app);
                aqq = warp_sum(aqq);
                apq = warp_sum(apq);
                if (pair_passes(app, aqq, apq, tol)) continue;
                const int hyp = (sh.sg[p] == sh.sg[q]) ? -1 : 1;
                double t, c;
                if (!rotation_params(app, aqq, apq, hyp, t, c)) {
                    if (lane == 0) atomicExch(&s_err, HSVD_ERR_RANK);
                    continue;
                }
                const double ht = hyp < 0 ? -t : t;
                for (int i = lane; i < m_pad; i += kWarp) {
                    const double x = gp[i], y = gq[i];
                    gp[i] = fma(ht, y, x) * c;
                    gq[i] = fma(t, x, y) * c;
                }
                double *wp = W + (size_t)p * n_pad, *wq = W + (size_t)q * n_pad;
                for (int i = lane; i < n_pad; i += kWarp) {
                    const double x = wp[i], y = wq[i];
                    wp[i] = fma(ht, y, x) * c;
                    wq[i] = fma(t, x, y) * c;
                }
                if (lane == 0) { atomicAdd(&s_rot, 1); ++rot_total; }
            }
            __syncthreads();
            if (s_err) break;
        }
        if (s_err) { status = s_err; break; }
        const int nrot = s_rot;
        __syncthreads();
        if (tid == 0) s_rot = 0;
        if (nrot == 0) { status = HSVD_OK; break; }
        if (sort) pw_reorder(sh, m_pad, n_pad, 1);
        else __syncthreads();
    }
    if (sweep > max_sweeps) sweep = max_sweeps;
    __syncthreads();

    // finalisation (Sec. 2): sigma_j = ||g_j||, u_j = g_j / sigma_j, V = W
    if (status == HSVD_OK || status == HSVD_NOT_CONVERGED) {
        for (int j = warp; j < n; j += kWarps) {
            const double *g = sh.G + (size_t)j * m_pad;
            double mx = 0.0;
            for (int i = lane; i < m; i += kWarp) mx = fmax(mx, fabs(g[i]));
            mx = warp_max(mx);
            int e;
            const double sc = pow2_scale_for(mx, e);
            double ss = 0.0;
            for (int i = lane; i < m; i += kWarp) {
                const double v = g[i] * sc;
                ss = fma(v, v, ss);
            }
            ss = warp_sum(ss);
            const double sj = ldexp(sqrt(ss), e);
            if (lane == 0) {
                sigma[j] = sj;
                if (!(sj > 0.0)) atomicExch(&s_err, HSVD_ERR_RANK);
                if (!isfinite(sj)) atomicExch(&s_err, HSVD_ERR_NONFINITE);
            }
            if (U)
                for (int i = lane; i < m; i += kWarp) U[i + (int64_t)j * ldu] = g[i] / sj;
            if (V)
                for (int i = lane; i < n; i += kWarp) V[i + (int64_t)j * ldv] = W[i + (size_t)j * n_pad];
        }
        __syncthreads();
        if (s_err) status = s_err;
    }
    // per-warp rotation counts
    __shared__ long long s_total;
    if (tid == 0) s_total = 0;
    __syncthreads();
    if (lane == 0 && rot_total) atomicAdd(reinterpret_cast<unsigned long long *>(&s_total),
                                          (unsigned long long)rot_total);
    __syncthreads();
    if (tid == 0) {
        out[0] = status;
        out[1] = sweep;
        *rot_out = s_total;
    }
}

}  // namespace

static int64_t pw_m_pad(int64_t m, int64_t n) {
    const int64_t n_pad = n + (n & 1);
    const int64_t rows = m + (n_pad - n);
    return (rows + 31) / 32 * 32;
}

size_t pointwise_smem_bytes(int64_t m_pad, int64_t n_pad) {
    return (size_t)m_pad * n_pad * sizeof(double) + (size_t)n_pad * (sizeof(double) + 3 * sizeof(int));
}

bool pointwise_fits(int64_t m, int64_t n) {
    const int64_t n_pad = n + (n & 1);
    return n_pad <= 2048 && pointwise_smem_bytes(pw_m_pad(m, n), n_pad) <= 200 * 1024;
}

cudaError_t launch_pointwise(const double *G, int64_t ldg, int m, int n, const int8_t *J,
                             double tol, int max_sweeps, int sort, double *Wws, double *sigma,
                             double *U, int64_t ldu, double *V, int64_t ldv, int *dev_out,
                             long long *dev_rot, cudaStream_t st) {
    const int n_pad = n + (n & 1);
    const int m_pad = (int)pw_m_pad(m, n);
    const size_t smem = pointwise_smem_bytes(m_pad, n_pad);
    cudaError_t e = cudaFuncSetAttribute(k_pointwise, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_pointwise<<<1, kThreads, smem, st>>>(G, ldg, m, n, J, m_pad, n_pad, tol, max_sweeps, sort, Wws,
                                           sigma, U, ldu, V, ldv, dev_out, dev_rot);
    return cudaGetLastError();
}

}  // namespace hsvd
