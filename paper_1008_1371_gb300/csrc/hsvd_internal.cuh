// hsvd_internal.cuh -- device helpers and cross-file declarations of the GB300
// hyperbolic SVD library.  Everything here is internal; the public C ABI is
// include/hsvd.h.
//
// The whole library is compiled with -fmad=false: every fused multiply-add is
// written out as fma(), so the rounding of each formula is the one stated in
// its comment (the parenthesised terms of Eq. 2.4 / 2.5 use one FMA, Sec. 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>

#include "../../include/hsvd.h"

namespace hsvd {

constexpr int kWarp = 32;

// Relative orthogonality test (Eq. 2.3): a pair is left alone when
// |a_ij| < tol sqrt(a_ii a_jj), and also when a_ij == 0 exactly (exactly
// orthogonal columns, e.g. a zero or bordering column, are never rotated).
__device__ __forceinline__ bool pair_passes(double aii, double ajj, double aij, double tol) {
    return aij == 0.0 || fabs(aij) < tol * sqrt(aii * ajj);
}

// Rotation annihilating a_ij (Sec. 2, Eq. 2.2).  hyp = -1 trigonometric
// (equal signs in J), +1 hyperbolic.  The update it defines is
//   g_i' = (g_i + hyp t g_j) c,   g_j' = (t g_i + g_j) c        (Alg. 4.5).
// Requiring a_ij' = 0 gives a_ij (1 + hyp t^2) + t (a_ii + hyp a_jj) = 0; t is
// its smaller root, written through zeta so that nothing overflows:
//   trig: zeta = (a_jj - a_ii)/(2 a_ij), t = sign(zeta)/(|zeta| + sqrt(zeta^2+1)),
//         c = 1/sqrt(1 + t^2)
//   hyp:  zeta = -(a_ii + a_jj)/(2 a_ij), t = sign(zeta)/(|zeta| + sqrt(zeta^2-1)),
//         c = 1/sqrt((1 - t)(1 + t))
// sign(0) = +1.  Returns false (t = 0, c = 1) when a hyperbolic pair has
// |zeta| <= 1: no J-unitary rotation exists, the pair is rank deficient.
// qv = 1/c as computed before the division (the scaled inner solve keeps it).
__device__ __forceinline__ bool rotation_params(double aii, double ajj, double aij, int hyp,
                                                double &t, double &c, double &qv) {
    if (hyp < 0) {
        const double zeta = (ajj - aii) / (2.0 * aij);
        double tt = 1.0 / (fabs(zeta) + sqrt(zeta * zeta + 1.0));
        if (zeta < 0.0) tt = -tt;
        t = tt;
        qv = sqrt(1.0 + tt * tt);
        c = 1.0 / qv;
        return true;
    }
    const double zeta = -(aii + ajj) / (2.0 * aij);
    if (!(fabs(zeta) > 1.0)) {
        t = 0.0;
        c = 1.0;
        qv = 1.0;
        return false;
    }
    double tt = 1.0 / (fabs(zeta) + sqrt(zeta * zeta - 1.0));
    if (zeta < 0.0) tt = -tt;
    t = tt;
    qv = sqrt((1.0 - tt) * (1.0 + tt));
    c = 1.0 / qv;
    return true;
}

// The test of Eq. 2.3, then the rotation of Sec. 2 for a pair that fails it.
// Returns 0 (the pair passes), 1 (rotate with t, c; qv = 1/c) or 2 (rank
// deficient); t = 0, c = qv = 1 unless it returns 1.  Late in the iteration
// most pairs pass, so the rotation's divides and square roots are skipped.
__device__ __forceinline__ int pair_decision(double aii, double ajj, double aij, int hyp, double tol,
                                             double &t, double &c, double &qv) {
    t = 0.0;
    c = 1.0;
    qv = 1.0;
    if (pair_passes(aii, ajj, aij, tol)) return 0;
    double tt, cc, qq;
    if (!rotation_params(aii, ajj, aij, hyp, tt, cc, qq)) return 2;
    t = tt;
    c = cc;
    qv = qq;
    return 1;
}
__device__ __forceinline__ int pair_decision(double aii, double ajj, double aij, int hyp, double tol,
                                             double &t, double &c) {
    double qv;
    return pair_decision(aii, ajj, aij, hyp, tol, t, c, qv);
}

// The same decision with the test and the rotation evaluated side by side
// (their square roots and divides overlap, the rotation is discarded when the
// pair passes): for a thread whose chain is the critical path whatever the
// outcome (the look-ahead warp of the cross pass).  Same results.
__device__ __forceinline__ int pair_decision_eager(double aii, double ajj, double aij, int hyp, double tol,
                                                   double &t, double &c, double &qv) {
    const bool passes = pair_passes(aii, ajj, aij, tol);
    double tt, cc, qq;
    const bool ok = rotation_params(aii, ajj, aij, hyp, tt, cc, qq);
    t = 0.0;
    c = 1.0;
    qv = 1.0;
    if (passes) return 0;
    if (!ok) return 2;
    t = tt;
    c = cc;
    qv = qq;
    return 1;
}

// Scaled rotations of the inner solve: the kernels keep S = diag(s)^-1 A
// diag(s)^-1 and W = Wh diag(s) with column scales s (reciprocals r), so a
// rotation costs two FMAs per element pair, x_p' = x_p + alpha x_q,
// x_q' = beta x_p + x_q, with alpha = ht (s_q r_p), beta = t (s_p r_q); then
// s <- s c and r <- r qv for p and q.  A scale whose binary exponent leaves
// [-kScaleExp, kScaleExp] sends the block back to s = r = 1 before the next step.
constexpr int kScaleExp = 8;
__device__ __forceinline__ bool scale_out_of_range(double s) { return abs(ilogb(s)) > kScaleExp; }

// k-th pivot pair (a < b) of step `s` of the modified modulus strategy on r
// indices (Sec. 2): the pairs with a + b = c (mod r), c = (r - 1 + s) mod r,
// plus (c/2, c/2 + r/2) for even c.  Slots are ordered by their smaller index.
__host__ __device__ __forceinline__ void modulus_pair(int r, int s, int k, int &a, int &b) {
    const int c = (r - 1 + (s % r)) % r;
    if (c & 1) {
        const int low = (c + 1) / 2;  // pairs (k, c - k), k < low
        if (k < low) { a = k; b = c - k; }
        else { a = c + 1 + (k - low); b = c + r - a; }
    } else {
        const int low = c / 2;
        if (k < low) { a = k; b = c - k; }
        else if (k == low) { a = c / 2; b = c / 2 + r / 2; }
        else { a = c + 1 + (k - low - 1); b = c + r - a; }
    }
    if (a > b) { const int x = a; a = b; b = x; }
}

// Scaled Euclidean norm pieces: x * 2^-e with 2^e >= max|x| is exact, so the
// scaled sum of squares equals the plain one without over- or underflow.
__device__ __forceinline__ double pow2_scale_for(double maxabs, int &e) {
    if (maxabs == 0.0 || !isfinite(maxabs)) { e = 0; return 1.0; }
    frexp(maxabs, &e);
    return ldexp(1.0, -e);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// A_P element e = x + y NN of pair `pair` from the three partial blocks
// (I,I) | (I,J) / (J,I) = (I,J)^T | (J,J), each summed over the row splits in
// split order.  A_P comes out exactly symmetric.
template <int NN>
__device__ __forceinline__ double assemble_entry(const double *__restrict__ part, int nsplit, int pair, int e) {
    constexpr int B = NN / 2;
    const int x = e % NN, y = e / NN;
    int blk, bx = x % B, by = y % B;
    if (x < B && y < B) blk = 0;
    else if (x >= B && y >= B) blk = 2;
    else {
        blk = 1;
        if (x >= B) { const int z = bx; bx = by; by = z; }
    }
    const double *pp = part + ((size_t)pair * 3 + blk) * nsplit * B * B + bx + (size_t)by * B;
    double v = 0.0;
    for (int s = 0; s < nsplit; ++s) v += pp[(size_t)s * B * B];
    return v;
}

// ---- launchers implemented in the .cu files --------------------------------

// pointwise.cu: one CTA solves one factor held in shared memory.
size_t pointwise_smem_bytes(int64_t m_pad, int64_t n_pad);
// True for device or managed memory (the kernels may read and write it);
// false for host memory, pinned or not, for NULL, and when no GPU answers.
bool is_device_ptr(const void *p);
// Every non-NULL pointer of the list is device memory.  The device-only entry
// points refuse host pointers with HSVD_ERR_ARG instead of launching kernels
// on them.
bool all_device(std::initializer_list<const void *> ps);

bool pointwise_fits(int64_t m, int64_t n);
// dev_out: status, sweeps, stop rule (HSVD_STOP_*); tstop = 0: strict stop only
cudaError_t launch_pointwise(const double *G, int64_t ldg, int m, int n, const int8_t *J,
                             double tol, double tstop, int max_sweeps, int sort, double *Wws,
                             double *sigma, double *U, int64_t ldu, double *V, int64_t ldv,
                             int *dev_out, long long *dev_rot, cudaStream_t st);

// blocked.cu: the three kernels of one step of the blocked method.
int gram_nsplit(int64_t rows, int npairs);
cudaError_t launch_gram(const double *G, int64_t rows, int64_t ldg, int b, int npairs,
                        const int *col0, int nsplit, double *part, cudaStream_t st);
// solve_cluster.cu: the inner pivot-block solve.  tab_full holds the modulus
// pairs of the 2b columns (2b steps of b pairs, 2 ints each) followed by the
// ring table of the full pass (ring_table_ints(b) ints, fill_ring).
size_t ring_table_ints(int b);
// false if the ring of the full pass cannot be formed (not for b = 16, 32, 64)
bool fill_ring(int b, int *tab);
cudaError_t launch_solve(int b, int npairs, const double *part, int nsplit, double *A,
                         const int8_t *sgn_cols, const int *col0, const int8_t *sgn_direct,
                         double tol, int mode, int max_passes, const int *tab_full,
                         const int *tab_cross, double *Wp, int *rotated,
                         unsigned long long *rot_count, int *status, cudaStream_t st,
                         int full_part = 0, int *dexp = nullptr, const int *visit = nullptr,
                         float *trace = nullptr, double tstop = 0.0, int *tbig = nullptr);
// precision.cu: the bounded mbarrier wait run out on purpose (a diagnostic)
cudaError_t launch_diag_wait(uint32_t iters, int *out, cudaStream_t st);

// qr.cu: the shortening front end (Householder QR of a tall factor)
size_t qr_workspace_doubles(int64_t n);
// A <- R (upper triangle) and the reflectors (below); ws: qr_workspace_doubles(n)
cudaError_t qr_factor(double *A, int64_t lda, int64_t m, int64_t n, double *ws, cudaStream_t st,
                      long long *launches);
// U (m x n) <- Q U, Q from the reflectors in A and the T factors in ws
// U (m x ncols, ldu) <- Q U; ncols = 0 means n
cudaError_t qr_apply_q(double *A, int64_t lda, int64_t m, int64_t n, double *ws, double *U, int64_t ldu,
                       cudaStream_t st, long long *launches, int64_t ncols = 0);
cudaError_t qr_extract_r(const double *A, int64_t lda, int64_t n, double *R, int64_t ldr, cudaStream_t st);
cudaError_t qr_embed_u(const double *UR, int64_t ldur, int64_t m, int64_t n, double *U, int64_t ldu,
                       cudaStream_t st);

// hypqr.cu: the hyperbolic QR of G^T for a wide G (m < n).  Device buffers,
// filled by the caller: A, Vr (n x m), C (m x m), z (n), beta (m), cperm,
// rswap (m), drows (4), s (n), bsize (m), state and mx (hypqr_state_bytes,
// hypqr_mx_bytes).
struct HypQr {
    double *A, *C, *Vr, *z, *beta;
    int *cperm, *rswap, *drows;
    int8_t *s, *bsize;
    void *state, *mx;
};
size_t hypqr_state_bytes();
size_t hypqr_mx_bytes(int64_t m);
// F = C R^T (m x m) from T G^T C = [R; 0]; hq.s ends as Jh (the first m: the
// signature of F).  HSVD_OK, HSVD_ERR_RANK (G J G^T singular) or HSVD_ERR_CUDA.
int hypqr_factor(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, HypQr &hq, double *F,
                 cudaStream_t st, long long *launches);
// V (n x m, ldv) <- T^T [V_F; 0]; consumes hq.s
int hypqr_apply_tt(HypQr &hq, int64_t m, int64_t n, const double *VF, double *V, int64_t ldv, cudaStream_t st,
                   long long *launches);

// ldl.cu: M = G J G^T by Bunch-Parlett pivoting (device arrays)
int ldl_factor(const double *M, int64_t n, int64_t ldm, double *G, int64_t ldg, int8_t *J, cudaStream_t st,
               long long *launches, int64_t *rank);

// learned form (learned.cu)
cudaError_t launch_features(const float *trace, const int8_t *prev_skip, const int *tab, int nvis, int b, int nb,
                            int sweep, int max_sweeps, double tol, float *X, cudaStream_t st);
cudaError_t launch_mlp_infer(const float *params, const float *X, int n, float *logits, int8_t *skip,
                             float logit_tau, cudaStream_t st);
cudaError_t launch_export(const float *X, const float *trace, int nvis, float *out, cudaStream_t st);
// visit table of a masked sweep: skipped visits become (-1, -1)
cudaError_t launch_mask_table(const int *outer, const int8_t *skip, int nvis, int *tab, int *kept, cudaStream_t st);
cudaError_t launch_assemble(int b, int npairs, const double *part, int nsplit, double *A, cudaStream_t st);
cudaError_t launch_update(double *X, int64_t rows, int64_t ldx, double *Y, int64_t rowsY,
                          int64_t ldy, int b, int npairs, const int *col0, const double *Wp,
                          const int *rotated, unsigned long long *upd_count, cudaStream_t st);

// precision.cu: split-precision (BF16 slices on tcgen05) Gram and update, b = 64.
size_t precision_wsl_elems(int npairs);
int precision_gram_ksplit(int64_t rows);
cudaError_t launch_gram_x(const double *G, int64_t rows, int64_t ldg, int npairs, const int *col0, double *part,
                          int *status, cudaStream_t st);
cudaError_t launch_assemble_x(int npairs, const double *part, int ksplit, double *A, cudaStream_t st);
cudaError_t launch_wprep_x(int npairs, const double *Wp, const int *dexp, const int *rotated, uint16_t *wsl,
                           int *wexp, unsigned long long *upd_count, cudaStream_t st);
cudaError_t launch_update_x(double *X, int64_t rowsX, int64_t ldx, double *Y, int64_t rowsY, int64_t ldy,
                            int npairs, const int *col0, const uint16_t *wsl, const int *wexp, const int *dexp,
                            const int *rotated, int *status, cudaStream_t st);

// prep.cu: bordering, reordering, finalisation.
cudaError_t launch_load_pad(const double *G, int64_t ldg, int64_t m, int64_t n, const int8_t *J,
                            double *Gw, int64_t m_pad, int64_t n_pad, double *Ww, int64_t ldw,
                            int *perm, int8_t *sgn, int *status, cudaStream_t st);
cudaError_t launch_reorder(double *Gw, double *Gt, int64_t m_pad, double *Ww, double *Wt,
                           int64_t ldw, int64_t n_pad, int *perm, int *perm_t, int8_t *sgn,
                           int8_t *sgn_t, double *d, int *newpos, int sort, cudaStream_t st);
cudaError_t launch_finalize(const double *Gw, int64_t m_pad, const double *Ww, int64_t ldw,
                            const int *perm, int64_t n_pad, int64_t m, int64_t n, double *sigma,
                            double *U, int64_t ldu, double *V, int64_t ldv, int *status,
                            cudaStream_t st);

}  // namespace hsvd
