// hypqr.cu -- the hyperbolic QR factorisation that shortens a wide factor
// (Sec. 1: a G whose transpose is tall is reduced by a hyperbolic QR of G^T,
// and V is premultiplied by the transformation).
//
// A = G^T (n x m, n > m) with signature S = J is reduced by J-orthogonal
// Householder reflectors H = I - beta v v^T S (H^T S H = S on the rows they
// touch) with row interchanges, and columns chosen on the trailing J-Gram
// C = X^T S X (X the trailing rows k.. of the remaining columns) by the
// Bunch-Parlett rule, alpha_bp = (1 + sqrt 17) / 8:
//   1 x 1 when the largest |C_jj| is at least alpha_bp times the largest
//     |C_ij|: that column moves to position k and is reduced to R_kk e_k;
//   2 x 2 otherwise: the columns x, y of the largest |C_ij| move to k, k + 1;
//     z = x + tau y (tau = +-1 so that |z^T S z| = |C_xx + C_yy| + 2 |C_xy|)
//     is reduced at row k, then y's rows k+1.. at row k + 1; R gets a full
//     2 x 2 diagonal block.
// A reduction of z at row r: if S_r is not the sign of gamma = z^T S z (rows
// r..), row r is interchanged with the row of that sign holding the largest
// |z_i| (ties: the smallest i); alpha = -sign(z_r) sqrt|gamma| keeps the
// J-norm, v = z - alpha e_r, beta = 2 / (v^T S v) = 1 / (S_r sqrt|gamma|
// (sqrt|gamma| + |z_r|)).  gamma = 0 means A^T J A is singular: HSVD_ERR_RANK.
//
// On the GPU the trailing J-Gram is kept as an m x m matrix: formed once, and
// after every finished row r downdated by S_r w_r w_r^T (w_r row r of the
// transformed A), since the reflectors and interchanges leave the J-Gram of
// the rows they touch unchanged.  The pivot choice reads it; gamma, tau and the
// reflectors are computed from the columns themselves.  One round per
// reflector: select (one CTA: pivot, column swaps, z, interchange, v, beta),
// apply (one CTA per column), finish (R's entries of the step), downdate (the
// trailing J-Gram, with per-CTA maxima for the next pivot).  The position and
// phase live on the device; the host launches m rounds.
//
// Afterwards T A C = [R; 0] with T^T Jh T = J (T the product of the
// interchanges and reflectors, Jh the signature after the interchanges), so
// G J G^T = F Jh_1 F^T with the square F = C R^T (m x m), whose HSVD
// F V_F = U Sigma gives V = T^T [V_F; 0]: G V = U Sigma and V^T J V = Jh_1.
#include <cuda_runtime.h>

#include <vector>

#include "hsvd_internal.cuh"

namespace hsvd {
namespace {

constexpr int kSelThreads = 1024;
constexpr int kColThreads = 256;
constexpr int kDownThreads = 256;
constexpr int kDownGrid = 304;
constexpr int kTile = 32;

struct HqState {
    int k;      // first column of the current step
    int phase;  // 0: first (or only) reflector of the step, 1: the second of a 2 x 2 step
    int s;      // size of the current step (1 or 2)
    int r0;     // row of the current reflector
    int bad;    // gamma = 0 (A^T J A singular): HSVD_ERR_RANK
    int done;   // every column reduced
    double alpha;
};

// per-CTA maxima of the trailing J-Gram: |diagonal| with its index, |off-diagonal| with (r, q), r < q
struct HqMax {
    double dmax, omax;
    int di, r, q, pad;
};

__device__ __forceinline__ HqMax hq_none() {
    HqMax m;
    m.dmax = -1.0;
    m.omax = -1.0;
    m.di = m.r = m.q = 0x7fffffff;
    m.pad = 0;
    return m;
}

__device__ __forceinline__ void hq_merge(HqMax &a, const HqMax &b) {
    if (b.dmax > a.dmax || (b.dmax == a.dmax && b.di < a.di)) {
        a.dmax = b.dmax;
        a.di = b.di;
    }
    if (b.omax > a.omax || (b.omax == a.omax && (b.q < a.q || (b.q == a.q && b.r < a.r)))) {
        a.omax = b.omax;
        a.r = b.r;
        a.q = b.q;
    }
}

__device__ __forceinline__ HqMax hq_shfl(const HqMax &a, int o) {
    HqMax b;
    b.dmax = __shfl_xor_sync(0xffffffffu, a.dmax, o);
    b.omax = __shfl_xor_sync(0xffffffffu, a.omax, o);
    b.di = __shfl_xor_sync(0xffffffffu, a.di, o);
    b.r = __shfl_xor_sync(0xffffffffu, a.r, o);
    b.q = __shfl_xor_sync(0xffffffffu, a.q, o);
    b.pad = 0;
    return b;
}

// the maximum entries (i, j >= k) seen by the CTA's threads into its slot
// (NT threads in a 1-D or 2-D block, whole warps)
template <int NT>
__device__ void hq_block_max(HqMax a, HqMax *out) {
    __shared__ HqMax red[NT / 32];
    const int lt = (int)(threadIdx.x + threadIdx.y * blockDim.x);
    for (int o = 16; o > 0; o >>= 1) hq_merge(a, hq_shfl(a, o));
    if ((lt & 31) == 0) red[lt >> 5] = a;
    __syncthreads();
    if (lt == 0) {
        HqMax t = red[0];
        for (int w = 1; w < NT / 32; ++w) hq_merge(t, red[w]);
        *out = t;
    }
}

__device__ __forceinline__ void hq_see(HqMax &a, int i, int j, double v) {
    const double av = fabs(v);
    if (i == j) {
        if (av > a.dmax || (av == a.dmax && i < a.di)) {
            a.dmax = av;
            a.di = i;
        }
    } else if (i < j) {  // the upper triangle stands for both
        if (av > a.omax || (av == a.omax && (j < a.q || (j == a.q && i < a.r)))) {
            a.omax = av;
            a.r = i;
            a.q = j;
        }
    }
}

// A (n x m, column-major) = G^T, G m x n (ldg)
__global__ void k_hq_transpose(const double *__restrict__ G, int64_t ldg, int m, int n, double *__restrict__ A) {
    __shared__ double t[kTile][kTile + 1];
    const int i0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;  // i: row of G (< m), j: column of G (< n)
    for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
        const int i = i0 + threadIdx.x, j = j0 + y;
        t[y][threadIdx.x] = (i < m && j < n) ? G[i + (int64_t)j * ldg] : 0.0;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
        const int j = j0 + threadIdx.x, i = i0 + y;  // A(j, i) = G(i, j)
        if (i < m && j < n) A[j + (int64_t)i * n] = t[threadIdx.x][y];
    }
}

// C = A^T S A (m x m, full symmetric), 32 x 32 tiles, and the per-CTA maxima
__global__ void __launch_bounds__(kTile * 8)
k_hq_gram(const double *__restrict__ A, int n, int m, const int8_t *__restrict__ s, double *__restrict__ C,
          HqMax *__restrict__ mx) {
    __shared__ double ta[kTile][kTile + 1], tb[kTile][kTile + 1];
    const int i0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r0 = 0; r0 < n; r0 += kTile) {
        for (int y = ty; y < kTile; y += 8) {
            const int r = r0 + tx;
            const double sg = (r < n) ? (double)s[r] : 0.0;
            ta[y][tx] = (r < n && i0 + y < m) ? A[r + (int64_t)(i0 + y) * n] * sg : 0.0;
            tb[y][tx] = (r < n && j0 + y < m) ? A[r + (int64_t)(j0 + y) * n] : 0.0;
        }
        __syncthreads();
        for (int u = 0; u < 4; ++u) {
            const int jy = ty + 8 * u;
#pragma unroll 8
            for (int r = 0; r < kTile; ++r) acc[u] = fma(ta[tx][r], tb[jy][r], acc[u]);
        }
        __syncthreads();
    }
    HqMax a = hq_none();
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + tx, j = j0 + ty + 8 * u;
        if (i < m && j < m) {
            C[i + (int64_t)j * m] = acc[u];
            hq_see(a, i, j, acc[u]);
        }
    }
    hq_block_max<kTile * 8>(a, &mx[blockIdx.x + blockIdx.y * gridDim.x]);
}

// swaps columns a and b of X (rows 0..rows-1, ld)
__device__ void swap_cols(double *X, int64_t ld, int rows, int a, int b) {
    if (a == b) return;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const double t = X[i + (int64_t)a * ld];
        X[i + (int64_t)a * ld] = X[i + (int64_t)b * ld];
        X[i + (int64_t)b * ld] = t;
    }
}

// One reflector's set-up (one CTA): at phase 0 the pivot choice and column
// swaps of a new step, then z, gamma, the row interchange, v and beta.
__global__ void __launch_bounds__(kSelThreads)
k_hq_select(double *__restrict__ A, int n, int m, int8_t *__restrict__ s, double *__restrict__ C,
            const HqMax *__restrict__ mx, int nmx, int *__restrict__ cperm, double *__restrict__ z,
            double *__restrict__ Vr, double *__restrict__ beta, int *__restrict__ rswap, int8_t *__restrict__ bsize,
            HqState *__restrict__ st) {
    __shared__ double red[kSelThreads / 32][3];
    __shared__ int s_choice[3];
    __shared__ double s_sc[4];  // gamma, tau
    __shared__ int s_ip;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (st->done || st->bad) return;
    const int k = st->k;
    if (st->phase == 0) {
        if (k >= m) {
            if (tid == 0) st->done = 1;
            return;
        }
        // pivot choice on the trailing J-Gram
        __shared__ HqMax mred[kSelThreads / 32];
        HqMax a = hq_none();
        for (int i = tid; i < nmx; i += kSelThreads) hq_merge(a, mx[i]);
        for (int o = 16; o > 0; o >>= 1) hq_merge(a, hq_shfl(a, o));
        if (lane == 0) mred[warp] = a;
        __syncthreads();
        if (tid == 0) {
            HqMax t = mred[0];
            for (int w = 1; w < kSelThreads / 32; ++w) hq_merge(t, mred[w]);
            const double alpha_bp = (1.0 + sqrt(17.0)) / 8.0;
            if (k == m - 1 || !(t.omax > 0.0) || t.dmax >= alpha_bp * t.omax) {
                s_choice[0] = (t.di >= k && t.di < m) ? 1 : 0;
                s_choice[1] = t.di;
            } else {
                s_choice[0] = (t.r >= k && t.q < m && t.r < t.q) ? 2 : 0;
                s_choice[1] = t.r;
                s_choice[2] = t.q;
            }
        }
        __syncthreads();
        const int sz = s_choice[0];
        if (sz == 0) {  // no finite pivot left
            if (tid == 0) st->bad = 1;
            return;
        }
        // columns to positions k (and k + 1): W, the rows and columns of C, the permutation
        auto swap_both = [&](int a0, int b0) {
            swap_cols(A, n, n, a0, b0);
            swap_cols(C, m, m, a0, b0);
            __syncthreads();
            if (a0 != b0)
                for (int j = tid; j < m; j += kSelThreads) {
                    const double t = C[a0 + (int64_t)j * m];
                    C[a0 + (int64_t)j * m] = C[b0 + (int64_t)j * m];
                    C[b0 + (int64_t)j * m] = t;
                }
            if (tid == 0 && a0 != b0) {
                const int t = cperm[a0];
                cperm[a0] = cperm[b0];
                cperm[b0] = t;
            }
            __syncthreads();
        };
        if (sz == 1) {
            swap_both(k, s_choice[1]);
        } else {
            const int pr = s_choice[1], pq = s_choice[2];
            swap_both(k, pr);
            swap_both(k + 1, pq == k ? pr : pq);
        }
        const double *x = A + (int64_t)k * n, *y = A + (int64_t)(k + 1) * n;
        double tau = 0.0;
        if (sz == 2) {
            // tau from the J-norms and J-product of x and y over rows k..
            double gx = 0.0, gy = 0.0, d = 0.0;
            for (int i = k + tid; i < n; i += kSelThreads) {
                const double sg = (double)s[i];
                gx = fma(sg * x[i], x[i], gx);
                gy = fma(sg * y[i], y[i], gy);
                d = fma(sg * x[i], y[i], d);
            }
            for (int o = 16; o > 0; o >>= 1) {
                gx += __shfl_xor_sync(0xffffffffu, gx, o);
                gy += __shfl_xor_sync(0xffffffffu, gy, o);
                d += __shfl_xor_sync(0xffffffffu, d, o);
            }
            if (lane == 0) {
                red[warp][0] = gx;
                red[warp][1] = gy;
                red[warp][2] = d;
            }
            __syncthreads();
            if (tid == 0) {
                double a0 = 0.0, a1 = 0.0, a2 = 0.0;
                for (int w = 0; w < kSelThreads / 32; ++w) {
                    a0 += red[w][0];
                    a1 += red[w][1];
                    a2 += red[w][2];
                }
                s_sc[1] = ((a0 + a1 >= 0.0) == (a2 >= 0.0)) ? 1.0 : -1.0;
            }
            __syncthreads();
            tau = s_sc[1];
        }
        for (int i = tid; i < n; i += kSelThreads) z[i] = i < k ? 0.0 : (sz == 2 ? fma(tau, y[i], x[i]) : x[i]);
        if (tid == 0) {
            st->s = sz;
            st->r0 = k;
            bsize[k] = (int8_t)sz;
            if (sz == 2) bsize[k + 1] = 0;
        }
        __syncthreads();
    } else {
        // the second reflector of a 2 x 2 step: y's rows k + 1..
        const double *y = A + (int64_t)(k + 1) * n;
        for (int i = tid; i < n; i += kSelThreads) z[i] = i <= k ? 0.0 : y[i];
        if (tid == 0) st->r0 = k + 1;
        __syncthreads();
    }
    const int r0 = st->phase == 0 ? k : k + 1;
    // gamma = z^T S z over rows r0..
    double g = 0.0;
    for (int i = r0 + tid; i < n; i += kSelThreads) g = fma((double)s[i] * z[i], z[i], g);
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if (lane == 0) red[warp][0] = g;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kSelThreads / 32; ++w) t += red[w][0];
        s_sc[0] = t;
    }
    __syncthreads();
    const double gamma = s_sc[0];
    if (!(gamma != 0.0)) {
        if (tid == 0) st->bad = 1;
        return;
    }
    const int sg = gamma > 0.0 ? 1 : -1;
    // the row interchange when S_r0 is not the sign of gamma: the row of that
    // sign with the largest |z_i|, ties to the smallest i
    if (s[r0] != sg) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int i = r0 + 1 + tid; i < n; i += kSelThreads)
            if (s[i] == sg && (fabs(z[i]) > best || (fabs(z[i]) == best && i < bi))) {
                best = fabs(z[i]);
                bi = i;
            }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) {
            red[warp][0] = best;
            red[warp][1] = (double)bi;
        }
        __syncthreads();
        if (tid == 0) {
            double b = -1.0;
            int i2 = 0x7fffffff;
            for (int w = 0; w < kSelThreads / 32; ++w) {
                const int wi = (int)red[w][1];
                if (red[w][0] > b || (red[w][0] == b && wi < i2)) {
                    b = red[w][0];
                    i2 = wi;
                }
            }
            s_ip = (i2 > r0 && i2 < n) ? i2 : -1;
        }
        __syncthreads();
        const int ip = s_ip;
        if (ip < 0) {
            if (tid == 0) st->bad = 1;
            return;
        }
        for (int j = tid; j < m; j += kSelThreads) {
            const double t = A[r0 + (int64_t)j * n];
            A[r0 + (int64_t)j * n] = A[ip + (int64_t)j * n];
            A[ip + (int64_t)j * n] = t;
        }
        if (tid == 0) {
            const double tz = z[r0];
            z[r0] = z[ip];
            z[ip] = tz;
            const int8_t ts = s[r0];
            s[r0] = s[ip];
            s[ip] = ts;
            rswap[r0] = ip;
        }
        __syncthreads();
    } else if (tid == 0) {
        rswap[r0] = r0;
    }
    __syncthreads();
    // alpha, v (zero above r0) and beta
    const double root = sqrt(fabs(gamma));
    const double zr = z[r0];
    const double alpha = zr >= 0.0 ? -root : root;
    double *v = Vr + (int64_t)r0 * n;
    for (int i = tid; i < n; i += kSelThreads) v[i] = i < r0 ? 0.0 : (i == r0 ? zr - alpha : z[i]);
    if (tid == 0) {
        const double vsv = 2.0 * (double)s[r0] * root * (root + fabs(zr));
        beta[r0] = 2.0 / vsv;
        st->alpha = alpha;
    }
}

// y <- y - beta (v^T S y) v over rows r0.. for every column c >= k (one CTA per column)
__global__ void __launch_bounds__(kColThreads)
k_hq_apply(double *__restrict__ A, int n, int m, const int8_t *__restrict__ s, const double *__restrict__ Vr,
           const double *__restrict__ beta, const HqState *__restrict__ st) {
    __shared__ double red[kColThreads / 32];
    if (st->done || st->bad) return;
    const int k = st->k, r0 = st->r0;
    const int c = k + (int)blockIdx.x;
    if (c >= m) return;
    const double *v = Vr + (int64_t)r0 * n;
    double *y = A + (int64_t)c * n;
    const int tid = threadIdx.x;
    double d = 0.0;
    for (int i = r0 + tid; i < n; i += kColThreads) d = fma((double)s[i] * v[i], y[i], d);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((tid & 31) == 0) red[tid >> 5] = d;
    __syncthreads();
    if (tid < 32) {
        double t = tid < kColThreads / 32 ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (tid == 0) red[0] = t;
    }
    __syncthreads();
    const double f = beta[r0] * red[0];
    for (int i = r0 + tid; i < n; i += kColThreads) y[i] = fma(-f, v[i], y[i]);
}

// R's entries of the step and the next position (one CTA); `downdate` gets the rows to remove
__global__ void k_hq_finish(double *__restrict__ A, int n, HqState *__restrict__ st, int *__restrict__ drows) {
    if (st->done || st->bad) {
        if (threadIdx.x == 0) drows[0] = 0;
        return;
    }
    const int k = st->k, sz = st->s, ph = st->phase;
    double *x = A + (int64_t)k * n, *y = A + (int64_t)(k + 1) * n;
    __syncthreads();
    if (sz == 1) {
        for (int i = k + (int)threadIdx.x; i < n; i += blockDim.x) x[i] = i == k ? st->alpha : 0.0;
    } else if (ph == 1) {
        for (int i = k + 2 + (int)threadIdx.x; i < n; i += blockDim.x) {
            x[i] = 0.0;
            y[i] = 0.0;
        }
        if (threadIdx.x == 0) y[k + 1] = st->alpha;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sz == 1) {
            drows[0] = 1;  // remove row k; the step is done
            drows[1] = k;
            st->k = k + 1;
            st->phase = 0;
        } else if (ph == 0) {
            drows[0] = 0;  // the second reflector comes first
            st->phase = 1;
        } else {
            drows[0] = 2;  // remove rows k and k + 1
            drows[1] = k;
            st->k = k + 2;
            st->phase = 0;
        }
    }
}

// the trailing J-Gram without the finished rows: C_ij -= S_r A(r, i) A(r, j),
// i, j >= first remaining column; per-CTA maxima of the new trailing block
__global__ void __launch_bounds__(kDownThreads)
k_hq_downdate(const double *__restrict__ A, int n, int m, const int8_t *__restrict__ s, double *__restrict__ C,
              const int *__restrict__ drows, const HqState *__restrict__ st, HqMax *__restrict__ mx) {
    const int nr = drows[0];
    HqMax a = hq_none();
    if (nr > 0) {
        const int r = drows[1], c0 = r + nr, nt = m - c0;
        const double s0 = (double)s[r], s1 = nr == 2 ? (double)s[r + 1] : 0.0;
        const int64_t total = (int64_t)nt * nt;
        for (int64_t e = (int64_t)blockIdx.x * kDownThreads + threadIdx.x; e < total;
             e += (int64_t)gridDim.x * kDownThreads) {
            const int i = c0 + (int)(e % nt), j = c0 + (int)(e / nt);
            double v = C[i + (int64_t)j * m];
            v = fma(-s0 * A[r + (int64_t)i * n], A[r + (int64_t)j * n], v);
            if (nr == 2) v = fma(-s1 * A[r + 1 + (int64_t)i * n], A[r + 1 + (int64_t)j * n], v);
            C[i + (int64_t)j * m] = v;
            hq_see(a, i, j, v);
        }
    }
    hq_block_max<kDownThreads>(a, &mx[blockIdx.x]);
    (void)st;
}

// F (m x m) = C R^T: F(cperm[j], l) = R(l, j), R the block upper triangle of A's first m rows
__global__ void k_hq_form_f(const double *__restrict__ A, int n, int m, const int *__restrict__ cperm,
                            const int8_t *__restrict__ bsize, double *__restrict__ F) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int l = (int)(e % m), j = (int)(e / m);
    const bool in_r = l <= j || (l == j + 1 && bsize[j] == 2);
    F[cperm[j] + (int64_t)l * m] = in_r ? A[l + (int64_t)j * n] : 0.0;
}

// X (n x c, ldx) <- H_k^T X = X - beta_k S v_k (v_k^T X), then the row
// interchange of step k, with the signature S of step k (one CTA per column)
__global__ void __launch_bounds__(kColThreads)
k_hq_apply_t(double *__restrict__ X, int64_t ldx, int n, int c, int k, const double *__restrict__ Vr,
             const double *__restrict__ beta, const int *__restrict__ rswap, const int8_t *__restrict__ s) {
    __shared__ double red[kColThreads / 32];
    const int j = blockIdx.x, tid = threadIdx.x;
    if (j >= c) return;
    const double *v = Vr + (int64_t)k * n;
    double *y = X + (int64_t)j * ldx;
    double d = 0.0;
    for (int i = k + tid; i < n; i += kColThreads) d = fma(v[i], y[i], d);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((tid & 31) == 0) red[tid >> 5] = d;
    __syncthreads();
    if (tid < 32) {
        double t = tid < kColThreads / 32 ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (tid == 0) red[0] = t;
    }
    __syncthreads();
    const double f = beta[k] * red[0];
    for (int i = k + tid; i < n; i += kColThreads) y[i] = fma(-(double)s[i] * f, v[i], y[i]);
    __syncthreads();
    const int ip = rswap[k];
    if (tid == 0 && ip != k) {
        const double t = y[k];
        y[k] = y[ip];
        y[ip] = t;
    }
}

// the signature of step k from that of step k + 1: undo step k's interchange
__global__ void k_hq_unswap_sign(int8_t *__restrict__ s, const int *__restrict__ rswap, int k) {
    const int ip = rswap[k];
    if (ip != k) {
        const int8_t t = s[k];
        s[k] = s[ip];
        s[ip] = t;
    }
}

// V (n x m, ldv) <- [V_F; 0]
__global__ void k_hq_embed(const double *__restrict__ VF, int m, int n, double *__restrict__ V, int64_t ldv) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * m) return;
    const int i = (int)(e % n), j = (int)(e / n);
    V[i + (int64_t)j * ldv] = i < m ? VF[i + (int64_t)j * m] : 0.0;
}

}  // namespace

size_t hypqr_state_bytes() { return sizeof(HqState); }
// per-CTA maxima: the Gram's tiles or the downdate's CTAs, whichever is more
size_t hypqr_mx_bytes(int64_t m) {
    const int64_t tiles = ((m + kTile - 1) / kTile) * ((m + kTile - 1) / kTile);
    return sizeof(HqMax) * (size_t)(tiles > kDownGrid ? tiles : kDownGrid);
}

// The hyperbolic QR of A = G^T (G m x n, m < n) and F = C R^T.  Outputs, all
// device: F (m x m), Jh (n signs after the interchanges; Jh_1 = the first m);
// the reflectors stay in the workspace `hq` for hypqr_apply_tt.  Returns
// HSVD_OK, HSVD_ERR_RANK or HSVD_ERR_CUDA.
int hypqr_factor(const double *G, int64_t m64, int64_t n64, int64_t ldg, const int8_t *J, HypQr &hq, double *F,
                 cudaStream_t st, long long *launches) {
    const int m = (int)m64, n = (int)n64;
    HqState *state = static_cast<HqState *>(hq.state);
    HqMax *mx = static_cast<HqMax *>(hq.mx);
    auto ck = [](cudaError_t e) { return e == cudaSuccess; };
    std::vector<int> p((size_t)m);
    for (int j = 0; j < m; ++j) p[(size_t)j] = j;
    HqState s0 = {};
    if (!ck(cudaMemcpyAsync(hq.cperm, p.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st)) ||
        !ck(cudaMemcpyAsync(state, &s0, sizeof s0, cudaMemcpyHostToDevice, st)) ||
        !ck(cudaMemcpyAsync(hq.s, J, (size_t)n, cudaMemcpyDeviceToDevice, st)) ||
        !ck(cudaMemsetAsync(hq.Vr, 0, sizeof(double) * (size_t)n * m, st)))
        return HSVD_ERR_CUDA;
    k_hq_transpose<<<dim3((m + kTile - 1) / kTile, (n + kTile - 1) / kTile), dim3(kTile, 8), 0, st>>>(G, ldg, m, n,
                                                                                                     hq.A);
    const dim3 gg((m + kTile - 1) / kTile, (m + kTile - 1) / kTile);
    const int nmx0 = (int)(gg.x * gg.y);  // the Gram's maxima, one per tile (hypqr_mx_bytes)
    k_hq_gram<<<gg, dim3(kTile, 8), 0, st>>>(hq.A, n, m, hq.s, hq.C, mx);
    if (!ck(cudaGetLastError())) return HSVD_ERR_CUDA;
    long long nl = 2;
    // m rounds, one reflector each
    for (int r = 0; r < m; ++r) {
        k_hq_select<<<1, kSelThreads, 0, st>>>(hq.A, n, m, hq.s, hq.C, mx, r == 0 ? nmx0 : kDownGrid, hq.cperm, hq.z,
                                               hq.Vr, hq.beta, hq.rswap, hq.bsize, state);
        k_hq_apply<<<m, kColThreads, 0, st>>>(hq.A, n, m, hq.s, hq.Vr, hq.beta, state);
        k_hq_finish<<<1, 256, 0, st>>>(hq.A, n, state, hq.drows);
        k_hq_downdate<<<kDownGrid, kDownThreads, 0, st>>>(hq.A, n, m, hq.s, hq.C, hq.drows, state, mx);
        if (!ck(cudaGetLastError())) return HSVD_ERR_CUDA;
        nl += 4;
    }
    k_hq_form_f<<<(unsigned)(((int64_t)m * m + 255) / 256), 256, 0, st>>>(hq.A, n, m, hq.cperm, hq.bsize, F);
    HqState fin = {};
    if (!ck(cudaGetLastError()) || !ck(cudaMemcpyAsync(&fin, state, sizeof fin, cudaMemcpyDeviceToHost, st)) ||
        !ck(cudaStreamSynchronize(st)))
        return HSVD_ERR_CUDA;
    if (launches) *launches += nl + 1;
    if (fin.bad) return HSVD_ERR_RANK;
    return fin.done || fin.k >= m ? HSVD_OK : HSVD_ERR_CUDA;
}

// V (n x m, ldv) <- T^T [V_F; 0], V_F (m x m): the reflectors in reverse order,
// each with the signature of its step (recovered from the final one by
// undoing the later interchanges; hq.s is consumed).
int hypqr_apply_tt(HypQr &hq, int64_t m64, int64_t n64, const double *VF, double *V, int64_t ldv, cudaStream_t st,
                   long long *launches) {
    const int m = (int)m64, n = (int)n64;
    k_hq_embed<<<(unsigned)(((int64_t)n * m + 255) / 256), 256, 0, st>>>(VF, m, n, V, ldv);
    for (int k = m - 1; k >= 0; --k) {
        k_hq_apply_t<<<m, kColThreads, 0, st>>>(V, ldv, n, m, k, hq.Vr, hq.beta, hq.rswap, hq.s);
        k_hq_unswap_sign<<<1, 1, 0, st>>>(hq.s, hq.rswap, k);
    }
    if (launches) *launches += 1 + 2 * (long long)m;
    return cudaGetLastError() == cudaSuccess ? HSVD_OK : HSVD_ERR_CUDA;
}

}  // namespace hsvd
