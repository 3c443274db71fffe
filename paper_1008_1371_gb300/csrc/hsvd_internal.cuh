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


// Bit-level conversions (integer operations only, no floating-point
// instruction) for the rotation parameters below.
// Unbiased binary exponent field of x (-1023 for 0 and subnormals, 1024 for
// infinities and NaN).
__device__ __forceinline__ int exp_field(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1023; }
// x 2^-e rounded toward zero to single precision; x normal and x 2^-e in the
// normal single range (the caller checks both).
__device__ __forceinline__ float f32_scaled(double x, int e) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned ex = (unsigned)((int)((hi >> 20) & 0x7ff) - 1023 - e + 127);
    return __uint_as_float((hi & 0x80000000u) | (ex << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
// f 2^e exactly in double precision; f a normal single, the result normal.
__device__ __forceinline__ double f64_scaled(float f, int e) {
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (unsigned)((int)((b >> 23) & 0xff) - 127 + e + 1023);
    return __hiloint2double((int)((b & 0x80000000u) | (ex << 20) | ((b & 0x7fffffu) >> 3)), (int)(b << 29));
}
__device__ __forceinline__ double neg_bits(double x) {
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000u, __double2loint(x));
}

// Relative orthogonality test (Eq. 2.3): a pair is left alone when
// |a_ij| < tol sqrt(a_ii a_jj), and also when a_ij == 0 exactly (exactly
// orthogonal columns, e.g. a zero or bordering column, are never rotated).
// The same decision as that expression, with few double-precision
// instructions: where all four operands are normal with binary exponents in
// +-500 (+-200 for tol) and a_ii, a_jj > 0, the ratio r = a_ij^2 /
// (tol^2 a_ii a_jj) is estimated from the exponents and the 23-bit truncated
// mantissas (relative error below 2^-20) and decides whenever it is outside
// 1 +- 2^-16; the expression's three roundings move its threshold by less
// than 2^-51, so both agree there.  Every other case evaluates the
// expression.
__device__ __forceinline__ bool pair_passes(double aii, double ajj, double aij, double tol) {
    const unsigned ha = (unsigned)__double2hiint(aij) & 0x7fffffffu, h1 = (unsigned)__double2hiint(aii),
                   h2 = (unsigned)__double2hiint(ajj), ht = (unsigned)__double2hiint(tol);
    const int ea = (int)(ha >> 20) - 1023, e1 = (int)(h1 >> 20) - 1023, e2 = (int)(h2 >> 20) - 1023,
              et = (int)(ht >> 20) - 1023;  // a_ii, a_jj, tol: the sign bit makes these out of range
    if (ea >= -500 && ea <= 500 && e1 >= -500 && e1 <= 500 && e2 >= -500 && e2 <= 500 && et >= -200 && et <= 200) {
        const int k = 2 * ea - 2 * et - e1 - e2;
        if (k >= 5) return false;
        if (k <= -3) return true;
        const float ma = f32_scaled(aij, ea), m1 = f32_scaled(aii, e1), m2 = f32_scaled(ajj, e2),
                    mt = f32_scaled(tol, et);
        const float lm = __fmul_rn(__fmul_rn(ma, ma), __int_as_float((127 + k) << 23));
        const float rm = __fmul_rn(__fmul_rn(mt, mt), __fmul_rn(m1, m2));
        if (lm < __fmul_rn(rm, 1.0f - 1.52587890625e-05f)) return true;
        if (lm > __fmul_rn(rm, 1.0f + 1.52587890625e-05f)) return false;
    }
    return aij == 0.0 || fabs(aij) < tol * sqrt(aii * ajj);
}

// c = 1/sqrt(1 - hyp t^2) to about half an ulp from an estimate c0: one
// Newton step on c^2 (1 - hyp t^2) = 1 whose residual (1 - c0^2) + hyp (c0 t)^2
// is formed from t itself by FMAs.  1/sqrt(x) with x = 1 - hyp t^2 rounded
// first, as two correctly rounded operations, leans upward for small t
// (c^2 (1 - hyp t^2) - 1 averages about +u for t^2 between u and 2^-30), a
// bias that about 10^5 rotations per column at n = 4096 turned into a
// relative +1.2e-12 on the large sigma.
__device__ __forceinline__ double cosine_step(double t, int hyp, double c0) {
    const double s = c0 * t;
    return fma(0.5 * c0, fma(hyp < 0 ? neg_bits(s) : s, s, fma(neg_bits(c0), c0, 1.0)), c0);
}
// qv = 1/c from an estimate q0 by one Newton step, so that c qv - 1 is an
// unbiased rounding error (the scaled inner solve multiplies by c and by qv)
__device__ __forceinline__ double reciprocal_step(double c, double q0) {
    return fma(q0, fma(neg_bits(c), q0, 1.0), q0);
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
// c by cosine_step, qv = 1/c by reciprocal_step (the scaled inner solve keeps
// qv).
__device__ __forceinline__ bool rotation_params(double aii, double ajj, double aij, int hyp,
                                                double &t, double &c, double &qv) {
    if (hyp < 0) {
        const double zeta = (ajj - aii) / (2.0 * aij);
        double tt = 1.0 / (fabs(zeta) + sqrt(zeta * zeta + 1.0));
        if (zeta < 0.0) tt = -tt;
        t = tt;
        const double q0 = sqrt(1.0 + tt * tt);
        c = cosine_step(tt, hyp, 1.0 / q0);
        qv = reciprocal_step(c, q0);
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
    const double q0 = sqrt((1.0 - tt) * (1.0 + tt));
    c = cosine_step(tt, hyp, 1.0 / q0);
    qv = reciprocal_step(c, q0);
    return true;
}

// The test of Eq. 2.3, then the rotation of Sec. 2 (rotation_params) for a
// pair that fails it: the one-sided pointwise kernels, whose rotations are
// the oracle's bit for bit (a tangent threshold of Eq. 4.2 then stops them
// at the oracle's sweep).  Returns 0 (the pair passes), 1 (rotate with t, c)
// or 2 (rank deficient); t = 0, c = 1 unless it returns 1.
__device__ __forceinline__ int pair_decision(double aii, double ajj, double aij, int hyp, double tol,
                                             double &t, double &c) {
    t = 0.0;
    c = 1.0;
    if (pair_passes(aii, ajj, aij, tol)) return 0;
    double tt, cc, qq;
    if (!rotation_params(aii, ajj, aij, hyp, tt, cc, qq)) return 2;
    t = tt;
    c = cc;
    return 1;
}

// The rotation of rotation_params with few double-precision instructions.
// On this part one warp issues a double-precision instruction every 64
// cycles (a single-precision or integer one every few), and the rotation of
// the next step is the critical path of the inner solve's steps, so:
//   - zeta and a first t in single precision, from a_ij and b scaled by
//     2^-e(a_ij) (b = a_jj - a_ii trigonometric, a_ii + a_jj hyperbolic);
//   - two Newton steps in double precision on f(t) = a_ij (t^2 + sg) + b t
//     (sg = -1 trigonometric, +1 hyperbolic: the equation of rotation_params,
//     whose smaller root is t), with 1/f' from single precision;
//   - x = 1 - hyp t^2, y = 1/sqrt(x) by one Newton step
//     y <- y + (y/2)(1 - x y^2) from the single-precision 1/sqrt(x), then c
//     from y by cosine_step (the residual from t itself) and qv from x c by
//     reciprocal_step.
// t and c agree with rotation_params' to a few units in the last place (other
// bits).  The single-precision start needs a_ij normal with |e(a_ij)| < 800,
// b = 0 (trigonometric only) or normal with 2^-100 <= |b / a_ij| < 2^101, and
// a hyperbolic pair with |zeta| >= 2 (|b| >= 4 |a_ij|, which also settles the
// rank test); every other pair takes rotation_params.
__device__ __forceinline__ bool rotation_params_fast(double aii, double ajj, double aij, int hyp, double &t,
                                                     double &c, double &qv) {
    const bool trig = hyp < 0;
    const double b = trig ? ajj - aii : aii + ajj;
    const int E = exp_field(aij), eb = exp_field(b);
    const unsigned long long abits = (unsigned long long)__double_as_longlong(aij) & 0x7fffffffffffffffull;
    const unsigned long long bbits = (unsigned long long)__double_as_longlong(b) & 0x7fffffffffffffffull;
    bool fast = E > -800 && E < 800;
    if (bbits == 0) fast = fast && trig;
    else fast = fast && eb > -1023 && eb < 1024 && eb - E >= -100 && eb - E <= 100;
    if (fast && !trig) fast = bbits >= abits + (2ull << 52);  // |b| >= 4 |a_ij|
    if (!fast) return rotation_params(aii, ajj, aij, hyp, t, c, qv);
    const float af = f32_scaled(aij, E);
    const float bf = bbits == 0 ? 0.0f : f32_scaled(b, E);
    const float z = __fdiv_rn(trig ? bf : -bf, __fmul_rn(2.0f, af));  // zeta
    const float az = fabsf(z);
    float tf;
    if (az <= 1048576.0f) {
        const float r = trig ? __fadd_rn(__fmul_rn(az, az), 1.0f) : __fsub_rn(__fmul_rn(az, az), 1.0f);
        tf = __fdiv_rn(1.0f, __fadd_rn(az, __fsqrt_rn(r)));
    } else {
        tf = __fdiv_rn(0.5f, az);
    }
    if (z < 0.0f) tf = -tf;
    // 1/f'(t) 2^E in single precision, f'(t) = 2 a_ij t + b: |f'| >= 2 |a_ij| at the root
    const float gf = __fdiv_rn(1.0f, __fadd_rn(__fmul_rn(__fmul_rn(2.0f, af), tf), bf));
    const double ngd = neg_bits(f64_scaled(gf, -E));
    const double sa = trig ? neg_bits(aij) : aij;
    double tt = f64_scaled(tf, 0);
#pragma unroll
    for (int it = 0; it < 2; ++it) tt = fma(fma(fma(aij, tt, b), tt, sa), ngd, tt);
    const double x = fma(tt, trig ? tt : neg_bits(tt), 1.0);
    const float r0 = __fdiv_rn(1.0f, __fsqrt_rn(f32_scaled(x, 0)));
    double y = f64_scaled(r0, 0);
    y = fma(f64_scaled(r0, -1), fma(neg_bits(x * y), y, 1.0), y);
    t = tt;
    c = cosine_step(tt, hyp, y);
    qv = reciprocal_step(c, x * c);
    return true;
}

// The test of Eq. 2.3, then the rotation of Sec. 2 (rotation_params_fast) for
// a pair that fails it.  Returns 0 (the pair passes), 1 (rotate with t, c;
// qv = 1/c) or 2 (rank deficient); t = 0, c = qv = 1 unless it returns 1.
// Late in the iteration most pairs pass and the rotation is skipped;
// evaluating it eagerly gains nothing on a warp whose double-precision
// instructions issue one at a time.
__device__ __forceinline__ int pair_decision_fast(double aii, double ajj, double aij, int hyp, double tol,
                                                  double &t, double &c, double &qv) {
    t = 0.0;
    c = 1.0;
    qv = 1.0;
    if (pair_passes(aii, ajj, aij, tol)) return 0;
    double tt, cc, qq;
    if (!rotation_params_fast(aii, ajj, aij, hyp, tt, cc, qq)) return 2;
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
// (a scale is a product of cosines and their reciprocals, always normal:
// its exponent field is ilogb, read with integer operations)
__device__ __forceinline__ bool scale_out_of_range(double s) { return abs(exp_field(s)) > kScaleExp; }

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
