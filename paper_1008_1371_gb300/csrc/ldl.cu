// ldl.cu -- the symmetric indefinite factorisation that turns an eigenproblem
// of a symmetric M into an HSVD (Sec. 1): M = P L D L^T P^T with complete
// (Bunch-Parlett) pivoting, D block diagonal with 1 x 1 and 2 x 2 blocks, and
// then G = P L B, J = diag(sign), B = diag(sqrt|d|) on 1 x 1 blocks and
// Q sqrt|Lambda| on a 2 x 2 block D_k = Q Lambda Q^T, so that M = G J G^T.
// The HSVD G V = U Sigma then gives M = U (Sigma^2 J) U^T: the eigenvalues of
// M are sigma_j^2 J_jj with eigenvectors u_j.
//
// Pivoting (Bunch and Parlett): with alpha = (1 + sqrt(17)) / 8,
// mu0 = max |a_ij| and mu1 = max |a_ii| over the trailing matrix, a 1 x 1 pivot
// on the largest diagonal entry if mu1 >= alpha mu0, else a 2 x 2 pivot on the
// rows and columns (r, q) of the largest off-diagonal entry.
//
// Unblocked and right-looking on the full symmetric trailing matrix:
//   k_ldl_pivot   one CTA: reduces the per-CTA maxima of the last update,
//                 chooses the pivot, swaps it into place (rows and columns of
//                 the trailing matrix, rows of the finished L) and records the
//                 D block;
//   k_ldl_update  the rank-1 or rank-2 update of the trailing matrix, with the
//                 maxima of the updated entries per CTA for the next pivot;
//   k_ldl_lstore  the pivot column(s) below the block become L = W D^-1, and
//                 the position moves on.
// The position k and the step size live on the device; the host launches n
// rounds and the ones past the end return at once.
#include <cuda_runtime.h>

#include <vector>

#include "hsvd_internal.cuh"

namespace hsvd {
namespace {

constexpr int kPivThreads = 1024;
constexpr int kUpdThreads = 256;

struct LdlState {
    int k;       // first column of the current step
    int s;       // its size (1 or 2; 0 once k reaches n)
    int bad;     // a non-finite entry (or no pivot found): HSVD_ERR_RANK
    int rank;    // columns factored: n, or the step at which the trailing matrix was zero
    double d[4];  // the step's D block, row-major
};

// per-CTA maxima of the trailing matrix: |diagonal| with its index, |off-diagonal| with (r, q)
struct LdlMax {
    double dmax, omax;
    int di, r, q, pad;
};

__device__ __forceinline__ void max_merge(LdlMax &a, const LdlMax &b) {
    // larger magnitude first, ties to the smaller index
    if (b.dmax > a.dmax || (b.dmax == a.dmax && b.di < a.di)) {
        a.dmax = b.dmax;
        a.di = b.di;
    }
    if (b.omax > a.omax || (b.omax == a.omax && (b.r < a.r || (b.r == a.r && b.q < a.q)))) {
        a.omax = b.omax;
        a.r = b.r;
        a.q = b.q;
    }
}

__device__ __forceinline__ LdlMax max_none() {
    LdlMax m;
    m.dmax = -1.0;
    m.omax = -1.0;
    m.di = m.r = m.q = 0x7fffffff;
    m.pad = 0;
    return m;
}

// swaps index a and b (both >= k) of the trailing symmetric matrix, and rows a, b of L's columns < k
__device__ void sym_swap(double *M, int64_t ld, int n, int k, int a, int b) {
    if (a == b) return;
    const int tid = threadIdx.x;
    // rows a, b in every column j (columns < k hold L; columns >= k the trailing matrix)
    for (int j = tid; j < n; j += blockDim.x) {
        if (j == a || j == b) continue;
        double *c = M + (int64_t)j * ld;
        const double t = c[a];
        c[a] = c[b];
        c[b] = t;
    }
    __syncthreads();
    // columns a, b in the trailing rows (the matrix is kept whole and symmetric)
    for (int i = k + tid; i < n; i += blockDim.x) {
        if (i == a || i == b) continue;
        double *ca = M + (int64_t)a * ld, *cb = M + (int64_t)b * ld;
        const double t = ca[i];
        ca[i] = cb[i];
        cb[i] = t;
    }
    if (tid == 0) {
        double *ca = M + (int64_t)a * ld, *cb = M + (int64_t)b * ld;
        const double t = ca[a];  // the two diagonal entries
        ca[a] = cb[b];
        cb[b] = t;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPivThreads)
k_ldl_pivot(double *__restrict__ M, int64_t ld, int n, LdlState *__restrict__ st, const LdlMax *__restrict__ mx,
            int nmx, int *__restrict__ perm, double *__restrict__ Dblk, int8_t *__restrict__ bsize) {
    __shared__ LdlMax red[kPivThreads / 32];
    __shared__ int s_choice[4];  // s, first, second
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = st->k;
    if (k >= n || st->bad) {  // done, or stopped at a zero pivot
        if (tid == 0) {
            st->s = 0;
            st->k = n;
        }
        return;
    }
    LdlMax a = max_none();
    for (int i = tid; i < nmx; i += kPivThreads) max_merge(a, mx[i]);
    for (int o = 16; o > 0; o >>= 1) {
        LdlMax b;
        b.dmax = __shfl_xor_sync(0xffffffffu, a.dmax, o);
        b.omax = __shfl_xor_sync(0xffffffffu, a.omax, o);
        b.di = __shfl_xor_sync(0xffffffffu, a.di, o);
        b.r = __shfl_xor_sync(0xffffffffu, a.r, o);
        b.q = __shfl_xor_sync(0xffffffffu, a.q, o);
        max_merge(a, b);
    }
    if (lane == 0) red[warp] = a;
    __syncthreads();
    if (tid == 0) {
        LdlMax t = red[0];
        for (int w = 1; w < kPivThreads / 32; ++w) max_merge(t, red[w]);
        const double alpha = (1.0 + sqrt(17.0)) / 8.0;
        const double mu0 = fmax(t.dmax, t.omax), mu1 = t.dmax;
        if (t.di >= k && t.di < n && mu0 == 0.0) {
            // the trailing matrix is zero: M has rank k (the postprocessing of a
            // singular M keeps the k columns found so far)
            s_choice[0] = -1;
        } else if (k == n - 1 || t.omax <= 0.0 || mu1 >= alpha * mu0) {
            s_choice[0] = 1;
            s_choice[1] = t.di;
        } else {
            s_choice[0] = 2;
            s_choice[1] = t.r < t.q ? t.r : t.q;
            s_choice[2] = t.r < t.q ? t.q : t.r;
        }
        // no valid pivot (NaN or Inf in the trailing matrix): stop with an error
        const bool valid = s_choice[0] == -1 ||
                           (s_choice[0] == 1 ? (s_choice[1] >= k && s_choice[1] < n)
                                             : (s_choice[1] >= k && s_choice[2] < n && s_choice[1] < s_choice[2]));
        if (!valid) s_choice[0] = 0;
    }
    __syncthreads();
    const int s = s_choice[0];
    if (s == -1) {
        if (tid == 0) {
            st->rank = k;
            st->s = 0;
            st->k = n;
        }
        return;
    }
    if (s == 0) {
        if (tid == 0) {
            st->bad = 1;
            st->s = 0;
            st->k = n;
        }
        return;
    }
    if (s == 1) {
        const int p = s_choice[1];
        sym_swap(M, ld, n, k, k, p);
        if (tid == 0) {
            const int t = perm[k];
            perm[k] = perm[p];
            perm[p] = t;
        }
    } else {
        const int r = s_choice[1], q = s_choice[2];  // r < q, both >= k
        // r -> k, then q -> k + 1 (q cannot be k: r < q and r >= k)
        sym_swap(M, ld, n, k, k, r);
        if (tid == 0) {
            const int t = perm[k];
            perm[k] = perm[r];
            perm[r] = t;
        }
        __syncthreads();
        const int q2 = (q == k) ? r : q;  // where q's index went after the first swap
        sym_swap(M, ld, n, k, k + 1, q2);
        if (tid == 0) {
            const int t = perm[k + 1];
            perm[k + 1] = perm[q2];
            perm[q2] = t;
        }
    }
    __syncthreads();
    // the D block; the pivot columns below it stay unscaled (W) for the update
    // and become L in k_ldl_lstore
    double *ck = M + (int64_t)k * ld;
    if (s == 1) {
        const double d = ck[k];
        if (tid == 0) {
            st->s = 1;
            st->d[0] = d;
            if (d == 0.0) st->bad = 1;
            Dblk[4 * k] = d;
            bsize[k] = 1;
        }
    } else {
        double *ck1 = M + (int64_t)(k + 1) * ld;
        const double d00 = ck[k], d01 = ck[k + 1], d11 = ck1[k + 1];
        if (tid == 0) {
            st->s = 2;
            st->d[0] = d00;
            st->d[1] = d01;
            st->d[2] = d01;
            st->d[3] = d11;
            if (fma(d00, d11, -d01 * d01) == 0.0) st->bad = 1;
            Dblk[4 * k] = d00;
            Dblk[4 * k + 1] = d01;
            Dblk[4 * k + 2] = d01;
            Dblk[4 * k + 3] = d11;
            bsize[k] = 2;
            bsize[k + 1] = 0;
        }
    }
}

// The trailing update for the step just pivoted: a_ij -= W_i D^-1 W_j^T for
// i, j >= k + s, W_i = (a_ik [, a_i,k+1]) the unscaled pivot columns.  The
// pivot columns become L = W D^-1 afterwards (k_ldl_lstore), once every CTA
// of this kernel has read them.
__global__ void __launch_bounds__(kUpdThreads)
k_ldl_update(double *__restrict__ M, int64_t ld, int n, const LdlState *__restrict__ st, LdlMax *__restrict__ mx) {
    __shared__ LdlMax red[kUpdThreads / 32];
    const int k = st->k, s = st->s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    LdlMax a = max_none();
    if (s > 0 && k < n && !st->bad) {
        const int t0 = k + s, nt = n - t0;
        const double *ck = M + (int64_t)k * ld, *ck1 = M + (int64_t)(k + 1) * ld;
        // D^-1 (1 x 1 or 2 x 2)
        double i00, i01 = 0.0, i11 = 0.0;
        if (s == 1) {
            i00 = 1.0 / st->d[0];
        } else {
            const double det = fma(st->d[0], st->d[3], -st->d[1] * st->d[1]);
            i00 = st->d[3] / det;
            i01 = -st->d[1] / det;
            i11 = st->d[0] / det;
        }
        const int64_t total = (int64_t)nt * nt;
        for (int64_t e = (int64_t)blockIdx.x * kUpdThreads + tid; e < total; e += (int64_t)gridDim.x * kUpdThreads) {
            const int i = t0 + (int)(e % nt), j = t0 + (int)(e / nt);
            double v;
            if (s == 1) {
                const double li = ck[i] * i00;
                v = fma(-li, ck[j], M[i + (int64_t)j * ld]);
            } else {
                const double wi0 = ck[i], wi1 = ck1[i];
                const double li0 = fma(wi0, i00, wi1 * i01), li1 = fma(wi0, i01, wi1 * i11);
                v = fma(-li0, ck[j], fma(-li1, ck1[j], M[i + (int64_t)j * ld]));
            }
            M[i + (int64_t)j * ld] = v;
            const double av = fabs(v);
            if (i == j) {
                if (av > a.dmax || (av == a.dmax && i < a.di)) {
                    a.dmax = av;
                    a.di = i;
                }
            } else if (i > j) {  // the lower triangle stands for both
                if (av > a.omax || (av == a.omax && (j < a.r || (j == a.r && i < a.q)))) {
                    a.omax = av;
                    a.r = j;
                    a.q = i;
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        LdlMax b;
        b.dmax = __shfl_xor_sync(0xffffffffu, a.dmax, o);
        b.omax = __shfl_xor_sync(0xffffffffu, a.omax, o);
        b.di = __shfl_xor_sync(0xffffffffu, a.di, o);
        b.r = __shfl_xor_sync(0xffffffffu, a.r, o);
        b.q = __shfl_xor_sync(0xffffffffu, a.q, o);
        max_merge(a, b);
    }
    if (lane == 0) red[warp] = a;
    __syncthreads();
    if (tid == 0) {
        LdlMax t = red[0];
        for (int w = 1; w < kUpdThreads / 32; ++w) max_merge(t, red[w]);
        mx[blockIdx.x] = t;
    }
}

// After the update: the pivot column(s) below the block become L = W D^-1,
// and the state moves to the next step.
__global__ void k_ldl_lstore(double *__restrict__ M, int64_t ld, int n, LdlState *__restrict__ st) {
    const int k = st->k, s = st->s;
    if (s == 0 || k >= n) return;
    double *ck = M + (int64_t)k * ld, *ck1 = M + (int64_t)(k + 1) * ld;
    if (!st->bad) {
        double i00, i01 = 0.0, i11 = 0.0;
        if (s == 1) {
            i00 = 1.0 / st->d[0];
        } else {
            const double det = fma(st->d[0], st->d[3], -st->d[1] * st->d[1]);
            i00 = st->d[3] / det;
            i01 = -st->d[1] / det;
            i11 = st->d[0] / det;
        }
        for (int i = k + s + (int)threadIdx.x; i < n; i += blockDim.x) {
            if (s == 1) {
                ck[i] = ck[i] * i00;
            } else {
                const double wi0 = ck[i], wi1 = ck1[i];
                ck[i] = fma(wi0, i00, wi1 * i01);
                ck1[i] = fma(wi0, i01, wi1 * i11);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) st->k = k + s;
}

// maxima of the whole matrix before the first pivot
__global__ void __launch_bounds__(kUpdThreads)
k_ldl_max0(const double *__restrict__ M, int64_t ld, int n, LdlMax *__restrict__ mx, LdlState *__restrict__ st) {
    __shared__ LdlMax red[kUpdThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    LdlMax a = max_none();
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * kUpdThreads + tid; e < total; e += (int64_t)gridDim.x * kUpdThreads) {
        const int i = (int)(e % n), j = (int)(e / n);
        const double av = fabs(M[i + (int64_t)j * ld]);
        if (!(av <= 1.7976931348623157e308)) atomicExch(&st->bad, 1);  // NaN or Inf in M
        if (i == j) {
            if (av > a.dmax || (av == a.dmax && i < a.di)) {
                a.dmax = av;
                a.di = i;
            }
        } else if (i > j) {
            if (av > a.omax || (av == a.omax && (j < a.r || (j == a.r && i < a.q)))) {
                a.omax = av;
                a.r = j;
                a.q = i;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        LdlMax b;
        b.dmax = __shfl_xor_sync(0xffffffffu, a.dmax, o);
        b.omax = __shfl_xor_sync(0xffffffffu, a.omax, o);
        b.di = __shfl_xor_sync(0xffffffffu, a.di, o);
        b.r = __shfl_xor_sync(0xffffffffu, a.r, o);
        b.q = __shfl_xor_sync(0xffffffffu, a.q, o);
        max_merge(a, b);
    }
    if (lane == 0) red[warp] = a;
    __syncthreads();
    if (tid == 0) {
        LdlMax t = red[0];
        for (int w = 1; w < kUpdThreads / 32; ++w) max_merge(t, red[w]);
        mx[blockIdx.x] = t;
    }
}

// G = P L B (column-major n x n) and J from the factors: column j of L is the
// unit lower triangle; a 1 x 1 block scales its column by sqrt|d|, a 2 x 2 block
// D = Q diag(l1, l2) Q^T (Jacobi rotation, l1 > 0 > l2 for a 2 x 2 pivot) maps
// its two columns by Q diag(sqrt|l1|, sqrt|l2|).  Position i of the factored
// matrix holds original index perm[i]: G(perm[i], j) = (L B)(i, j).
__global__ void k_ldl_form_g(const double *__restrict__ M, int64_t ld, int n, const int *__restrict__ perm,
                             const double *__restrict__ Dblk, const int8_t *__restrict__ bsize,
                             double *__restrict__ G, int64_t ldg, int8_t *__restrict__ J,
                             const LdlState *__restrict__ st) {
    const int j = blockIdx.x;  // one CTA per column of G
    if (j >= st->rank) {       // past the rank of a singular M: no column, no sign
        for (int i = threadIdx.x; i < n; i += blockDim.x) G[i + (int64_t)j * ldg] = 0.0;
        if (threadIdx.x == 0) J[j] = 0;
        return;
    }
    const int bs = bsize[j];
    int b0 = j;                  // first column of j's block
    if (bs == 0) b0 = j - 1;
    const int size = bsize[b0];
    double c0, c1, sgn;          // column j of G = c0 * L(:, b0) + c1 * L(:, b0 + 1)
    if (size == 1) {
        const double d = Dblk[4 * b0];
        c0 = sqrt(fabs(d));
        c1 = 0.0;
        sgn = d > 0.0 ? 1.0 : -1.0;
    } else {
        const double a = Dblk[4 * b0], b = Dblk[4 * b0 + 1], c = Dblk[4 * b0 + 3];
        // the symmetric 2 x 2 Schur decomposition (a Jacobi rotation, t = tan phi
        // the smaller root): with Q = [cs sn; -sn cs], Q^T D Q = diag(a - t b, c + t b)
        double t = 0.0;
        if (b != 0.0) {
            const double zeta = (c - a) / (2.0 * b);
            t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
        }
        const double cs = 1.0 / sqrt(fma(t, t, 1.0)), sn = t * cs;
        const double l1 = fma(-t, b, a), l2 = fma(t, b, c);
        // columns: q1 = (cs, -sn), q2 = (sn, cs)
        if (j == b0) {
            c0 = cs * sqrt(fabs(l1));
            c1 = -sn * sqrt(fabs(l1));
            sgn = l1 > 0.0 ? 1.0 : -1.0;
        } else {
            c0 = sn * sqrt(fabs(l2));
            c1 = cs * sqrt(fabs(l2));
            sgn = l2 > 0.0 ? 1.0 : -1.0;
        }
    }
    const double *L0 = M + (int64_t)b0 * ld, *L1 = M + (int64_t)(b0 + 1) * ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        // L(i, b0) is 1 on the diagonal, 0 above, the stored column below the block
        double l0 = 0.0, l1v = 0.0;
        if (i == b0) l0 = 1.0;
        else if (i > b0 + (size - 1)) l0 = L0[i];
        if (size == 2) {
            if (i == b0 + 1) l1v = 1.0;
            else if (i > b0 + 1) l1v = L1[i];
        }
        G[perm[i] + (int64_t)j * ldg] = fma(c0, l0, c1 * l1v);
    }
    if (threadIdx.x == 0) J[j] = sgn > 0.0 ? 1 : -1;
}

constexpr int kUpdGrid = 608;

}  // namespace

// M (n x n, ldm, device, symmetric; read-only) -> G (n x n, ldg, device) and
// J (n, device) with M = G J G^T.  A singular M stops once the trailing matrix
// is zero: *rank (may be NULL) receives the columns factored, and G's columns
// and J's entries past it are zero.  Returns HSVD_OK or HSVD_ERR_RANK (a
// non-finite entry).
int ldl_factor(const double *M, int64_t n, int64_t ldm, double *G, int64_t ldg, int8_t *J, cudaStream_t st,
               long long *launches, int64_t *rank) {
    double *W = nullptr, *Dblk = nullptr;
    int *perm = nullptr;
    int8_t *bsize = nullptr;
    LdlState *state = nullptr;
    LdlMax *mx = nullptr;
    int rc = HSVD_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == HSVD_OK) rc = HSVD_ERR_CUDA;
        return e == cudaSuccess;
    };
    if (!ok(cudaMallocAsync((void **)&W, sizeof(double) * n * n, st)) ||
        !ok(cudaMallocAsync((void **)&Dblk, sizeof(double) * 4 * n, st)) ||
        !ok(cudaMallocAsync((void **)&perm, sizeof(int) * n, st)) ||
        !ok(cudaMallocAsync((void **)&bsize, (size_t)n, st)) ||
        !ok(cudaMallocAsync((void **)&state, sizeof(LdlState), st)) ||
        !ok(cudaMallocAsync((void **)&mx, sizeof(LdlMax) * kUpdGrid, st))) {
        rc = HSVD_ERR_NOMEM;
    }
    if (rc == HSVD_OK) {
        std::vector<int> p((size_t)n);
        for (int64_t i = 0; i < n; ++i) p[(size_t)i] = (int)i;
        LdlState s0 = {};
        s0.rank = (int)n;
        ok(cudaMemcpy2DAsync(W, sizeof(double) * n, M, sizeof(double) * ldm, sizeof(double) * n, n,
                             cudaMemcpyDeviceToDevice, st));
        ok(cudaMemcpyAsync(perm, p.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        ok(cudaMemcpyAsync(state, &s0, sizeof s0, cudaMemcpyHostToDevice, st));
        ok(cudaMemsetAsync(bsize, 1, (size_t)n, st));
        k_ldl_max0<<<kUpdGrid, kUpdThreads, 0, st>>>(W, n, (int)n, mx, state);
        ok(cudaGetLastError());
        // every step takes one or two columns: n (pivot, update, store) rounds
        // cover the worst case, rounds past the end return at once
        for (int64_t t = 0; t < n && rc == HSVD_OK; ++t) {
            k_ldl_pivot<<<1, kPivThreads, 0, st>>>(W, n, (int)n, state, mx, kUpdGrid, perm, Dblk, bsize);
            k_ldl_update<<<kUpdGrid, kUpdThreads, 0, st>>>(W, n, (int)n, state, mx);
            k_ldl_lstore<<<1, 256, 0, st>>>(W, n, (int)n, state);
            ok(cudaGetLastError());
        }
        k_ldl_form_g<<<(unsigned)n, 256, 0, st>>>(W, n, (int)n, perm, Dblk, bsize, G, ldg, J, state);
        ok(cudaGetLastError());
        LdlState fin = {};
        if (ok(cudaMemcpyAsync(&fin, state, sizeof fin, cudaMemcpyDeviceToHost, st)) &&
            ok(cudaStreamSynchronize(st)) && fin.bad)
            rc = HSVD_ERR_RANK;
        if (rank) *rank = fin.rank;
        if (launches) *launches += 2 + 3 * n;
    }
    if (W) cudaFreeAsync(W, st);
    if (Dblk) cudaFreeAsync(Dblk, st);
    if (perm) cudaFreeAsync(perm, st);
    if (bsize) cudaFreeAsync(bsize, st);
    if (state) cudaFreeAsync(state, st);
    if (mx) cudaFreeAsync(mx, st);
    return rc;
}

}  // namespace hsvd
