// prep.cu -- bordering, column reordering and finalisation for the blocked
// method.  All of it is O((m + n) n) memory traffic, a vanishing share of a
// sweep (Sec. 5 reports the non-step routines well below 0.1% of the time).
#include "hsvd_internal.cuh"

namespace hsvd {
namespace {

constexpr int kThreads = 256;

// Working copy bordered as in Eq. 4.1: columns n..n_pad-1 are unit vectors in
// the fresh rows m..m+(n_pad-n)-1, rows up to m_pad are zero.  W = I, working
// position k holds input column perm[k] = k, pads carry sign +1.
__global__ void k_load_pad(const double *__restrict__ G, int64_t ldg, int64_t m, int64_t n,
                           const int8_t *__restrict__ J, double *__restrict__ Gw, int64_t m_pad,
                           int64_t n_pad, double *__restrict__ Ww, int64_t ldw, int *__restrict__ perm,
                           int8_t *__restrict__ sgn, int *__restrict__ status) {
    const int64_t j = blockIdx.x;
    int bad = 0;
    for (int64_t i = threadIdx.x; i < m_pad; i += kThreads) {
        double v = 0.0;
        if (j < n) {
            if (i < m) v = G[i + j * ldg];
        } else if (i == m + (j - n)) {
            v = 1.0;
        }
        bad |= !isfinite(v);
        Gw[i + j * m_pad] = v;
    }
    for (int64_t i = threadIdx.x; i < ldw; i += kThreads) Ww[i + j * ldw] = (i == j) ? 1.0 : 0.0;
    if (threadIdx.x == 0) {
        perm[j] = (int)j;
        const int8_t sj = (j < n) ? J[j] : (int8_t)1;
        sgn[j] = sj > 0 ? (int8_t)1 : (int8_t)-1;
        if (sj != 1 && sj != -1) atomicExch(status, HSVD_ERR_ARG);
    }
    if (bad) atomicExch(status, HSVD_ERR_NONFINITE);
}

// d_k = ||g_k||^2 (one warp per column)
__global__ void k_col_norms2(const double *__restrict__ Gw, int64_t m_pad, int64_t n_pad,
                             double *__restrict__ d) {
    const int64_t k = (int64_t)blockIdx.x * (kThreads / kWarp) + threadIdx.x / kWarp;
    const int lane = threadIdx.x & 31;
    if (k >= n_pad) return;
    const double *g = Gw + k * m_pad;
    double s = 0.0;
    for (int64_t i = lane; i < m_pad; i += kWarp) s = fma(g[i], g[i], s);
    s = warp_sum(s);
    if (lane == 0) d[k] = s;
}

// New order of the working positions (Sec. 4, Sort_Diagonal): the J+ part first,
// then the J- part; with sort != 0 the J+ part by d decreasing and the J- part
// by d increasing; equal keys keep their current order.  newpos[k] = current
// position of the column that goes to position k.  One thread per position,
// rank by counting (O(n^2) comparisons, spread over the whole GPU).
__global__ void k_sort_positions(const double *__restrict__ d, const int8_t *__restrict__ sgn, int64_t n_pad,
                                 int sort, int *__restrict__ newpos) {
    constexpr int kTile = 2048;
    __shared__ double sd[kTile];
    __shared__ int8_t ss[kTile];
    const int64_t a = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool act = a < n_pad;
    const int grp = act ? sgn[a] : 0;
    const double key = (act && sort) ? d[a] : 0.0;
    // keys between +0 and +inf compare as their bit patterns (integer
    // instructions; an FP64 comparison issues at the FP64 rate): the same
    // order and the same ties as the floating-point comparison
    constexpr unsigned long long kInf = 0x7FF0000000000000ull;
    const unsigned long long kbits = (unsigned long long)__double_as_longlong(key);
    int64_t rank = 0, nplus = 0;
    for (int64_t t0 = 0; t0 < n_pad; t0 += kTile) {
        const int len = (int)min((int64_t)kTile, n_pad - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += kThreads) {
            sd[i] = sort ? d[t0 + i] : 0.0;
            ss[i] = sgn[t0 + i];
        }
        __syncthreads();
        if (!act) continue;
        for (int i = 0; i < len; ++i) {
            const int gb = ss[i];
            nplus += gb > 0;
            const int64_t b = t0 + i;
            if (gb != grp || b == a) continue;
            const double kb = sd[i];
            const unsigned long long bbits = (unsigned long long)__double_as_longlong(kb);
            bool before, tie;
            if (kbits <= kInf && bbits <= kInf) {
                before = (grp > 0) ? (bbits > kbits) : (bbits < kbits);
                tie = bbits == kbits;
            } else {
                before = (grp > 0) ? (kb > key) : (kb < key);
                tie = kb == key;
            }
            if (before || (tie && b < a)) ++rank;
        }
    }
    if (act) newpos[(grp > 0 ? 0 : nplus) + rank] = (int)a;
}

__global__ void k_permute(const double *__restrict__ Gw, double *__restrict__ Gt, int64_t m_pad,
                          const double *__restrict__ Ww, double *__restrict__ Wt, int64_t ldw,
                          const int *__restrict__ perm, int *__restrict__ perm_t,
                          const int8_t *__restrict__ sgn, int8_t *__restrict__ sgn_t,
                          const int *__restrict__ newpos) {
    const int64_t k = blockIdx.x;
    const int64_t src = newpos[k];
    const double2 *gs = reinterpret_cast<const double2 *>(Gw + src * m_pad);
    double2 *gd = reinterpret_cast<double2 *>(Gt + k * m_pad);
    for (int64_t i = threadIdx.x; i < m_pad / 2; i += kThreads) gd[i] = gs[i];
    const double2 *ws = reinterpret_cast<const double2 *>(Ww + src * ldw);
    double2 *wd = reinterpret_cast<double2 *>(Wt + k * ldw);
    for (int64_t i = threadIdx.x; i < ldw / 2; i += kThreads) wd[i] = ws[i];
    if (threadIdx.x == 0) {
        perm_t[k] = perm[src];
        sgn_t[k] = sgn[src];
    }
}

// sigma_j = ||g_k||_2 (exact power-of-two scaling, no over/underflow),
// u_j = g_k / sigma_j, v_j = w_k, j = perm[k] (Sec. 2 finalisation, results in
// input column order).
__global__ void k_finalize(const double *__restrict__ Gw, int64_t m_pad, const double *__restrict__ Ww,
                           int64_t ldw, const int *__restrict__ perm, int64_t n_pad, int64_t m, int64_t n,
                           double *__restrict__ sigma, double *__restrict__ U, int64_t ldu,
                           double *__restrict__ V, int64_t ldv, int *__restrict__ status) {
    const int64_t k = blockIdx.x;
    const int64_t j = perm[k];
    if (j >= n) return;
    __shared__ double red[kThreads / kWarp];
    __shared__ double s_sig;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *g = Gw + k * m_pad;
    double mx = 0.0;
    for (int64_t i = tid; i < m; i += kThreads) mx = fmax(mx, fabs(g[i]));
    mx = warp_max(mx);
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int w = 0; w < kThreads / kWarp; ++w) v = fmax(v, red[w]);
        s_sig = v;
    }
    __syncthreads();
    int e;
    const double sc = pow2_scale_for(s_sig, e);
    __syncthreads();
    double ss = 0.0;
    for (int64_t i = tid; i < m; i += kThreads) {
        const double v = g[i] * sc;
        ss = fma(v, v, ss);
    }
    ss = warp_sum(ss);
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int w = 0; w < kThreads / kWarp; ++w) v += red[w];
        const double sj = ldexp(sqrt(v), e);
        s_sig = sj;
        sigma[j] = sj;
        if (!(sj > 0.0)) atomicExch(status, HSVD_ERR_RANK);
        if (!isfinite(sj)) atomicExch(status, HSVD_ERR_NONFINITE);
    }
    __syncthreads();
    const double sj = s_sig;
    if (U)
        for (int64_t i = tid; i < m; i += kThreads) U[i + j * ldu] = g[i] / sj;
    if (V)
        for (int64_t i = tid; i < n; i += kThreads) V[i + j * ldv] = Ww[i + k * ldw];
}

}  // namespace

cudaError_t launch_load_pad(const double *G, int64_t ldg, int64_t m, int64_t n, const int8_t *J, double *Gw,
                            int64_t m_pad, int64_t n_pad, double *Ww, int64_t ldw, int *perm, int8_t *sgn,
                            int *status, cudaStream_t st) {
    k_load_pad<<<(unsigned)n_pad, kThreads, 0, st>>>(G, ldg, m, n, J, Gw, m_pad, n_pad, Ww, ldw, perm, sgn, status);
    return cudaGetLastError();
}

cudaError_t launch_reorder(double *Gw, double *Gt, int64_t m_pad, double *Ww, double *Wt, int64_t ldw,
                           int64_t n_pad, int *perm, int *perm_t, int8_t *sgn, int8_t *sgn_t, double *d,
                           int *newpos, int sort, cudaStream_t st) {
    if (sort) {
        const int wpb = kThreads / kWarp;
        k_col_norms2<<<(unsigned)((n_pad + wpb - 1) / wpb), kThreads, 0, st>>>(Gw, m_pad, n_pad, d);
    }
    k_sort_positions<<<(unsigned)((n_pad + kThreads - 1) / kThreads), kThreads, 0, st>>>(d, sgn, n_pad, sort,
                                                                                         newpos);
    k_permute<<<(unsigned)n_pad, kThreads, 0, st>>>(Gw, Gt, m_pad, Ww, Wt, ldw, perm, perm_t, sgn, sgn_t, newpos);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(Gw, Gt, sizeof(double) * m_pad * n_pad, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(Ww, Wt, sizeof(double) * ldw * n_pad, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(perm, perm_t, sizeof(int) * n_pad, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(sgn, sgn_t, n_pad, cudaMemcpyDeviceToDevice, st);
}

cudaError_t launch_finalize(const double *Gw, int64_t m_pad, const double *Ww, int64_t ldw, const int *perm,
                            int64_t n_pad, int64_t m, int64_t n, double *sigma, double *U, int64_t ldu, double *V,
                            int64_t ldv, int *status, cudaStream_t st) {
    k_finalize<<<(unsigned)n_pad, kThreads, 0, st>>>(Gw, m_pad, Ww, ldw, perm, n_pad, m, n, sigma, U, ldu, V, ldv,
                                                     status);
    return cudaGetLastError();
}

}  // namespace hsvd
