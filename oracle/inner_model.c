/*
 * inner_model.c -- exact CPU model of the library's inner-solve kernels
 * (the J-orthogonalisation of one pivot block, Sec. 5 / Sec. 6).
 *
 * TEST INFRASTRUCTURE ONLY, and NOT the oracle.  The oracle's inner solve
 * (orc_inner_solve in hsvd_oracle.c) applies one rotation at a time, in the
 * paper's row-cyclic order.  This file instead reproduces, operation for
 * operation, what the library's cluster kernels compute, so that a test can
 * compare them bit for bit; a second test bounds this model against the
 * oracle.  It shares no code with the CUDA library: it is written from the
 * kernels' documented arithmetic; the pivot table and, outside the range of
 * M5, the rotation come from the oracle (orc_modulus_pairs, orc_rotation).
 *
 * The model's choices where the paper leaves the implementation open:
 *   M1  Pair order: the steps of the parallel strategy inside the block --
 *       the modified modulus strategy over the 2b indices for a full pass,
 *       (k, b + ((k + s) mod b)) at step s for the cross pass -- with all
 *       pairs of a step tested on the step's starting values and rotated at
 *       once (they are disjoint).
 *   M2  The two one-sided halves of R^T A R alternate their order from step
 *       to step: the step's rotations mix the rows of a row-major copy S of
 *       the block, S is transposed, and the rows are mixed again, so S holds
 *       the transpose of the block after an odd number of steps.  (The
 *       kernels transpose once per step this way.)
 *   M3  After the mixing, a rotated pair's diagonal values take Eq. 2.6
 *       with the step's starting a_pq (a replicated vector d), and the
 *       stored (p, q), (q, p), (p, p), (q, q) become 0.
 *   M4  Scaled rotations: the kernels store S = diag(s)^-1 A diag(s)^-1 and
 *       W = Wh diag(s), with column scales s (and their reciprocals r) that
 *       start at 1.  A rotation (t, c) of pair (p, q), with q = 1/c computed
 *       as in the rotation, becomes x_p' = x_p + alpha x_q,
 *       x_q' = beta x_p + x_q on the stored values, alpha = ht (s_q r_p),
 *       beta = t (s_p r_q) (two FMAs per element pair instead of two FMAs
 *       and two multiplies), and s_p, s_q <- s c, r_p, r_q <- r q.  The
 *       test of Eq. 2.3 reads a_pq = (s_p s_q) S_pq.  When an updated scale
 *       has a binary exponent beyond +-8 the whole block is brought back to s = r = 1
 *       (S_xy <- (s_x s_y) S_xy, Wh_xy <- Wh_xy s_y) before the next step.
 *       At the end, W = Wh diag(s) and A_xy = (s_x s_y) S_xy off the
 *       diagonal, d on it.
 *   M5  Rotation parameters with few double-precision operations (the
 *       kernels' rotation is the critical path of a step, and one warp issues
 *       one double-precision instruction per 64 cycles): zeta and a first t
 *       in single precision from a_ij and b scaled by 2^-e(a_ij) (b = a_jj -
 *       a_ii trigonometric, a_ii + a_jj hyperbolic), truncated to 23
 *       fraction bits; two Newton steps in double precision on f(t) =
 *       a_ij (t^2 + sg) + b t (sg = -1 trigonometric, +1 hyperbolic), the
 *       equation of Sec. 2 whose smaller root is the oracle's t, with 1/f'
 *       from single precision; y = 1/sqrt(x), x = 1 - hyp t^2, by one Newton
 *       step y <- y + (y/2)(1 - x y^2) from the single-precision 1/sqrt(x),
 *       then c from y by the oracle's unbiased cosine step (the residual
 *       (1 - y^2) + hyp (y t)^2 formed from t); q = 1/c by one Newton step
 *       q <- q + q (1 - c q) from x c (so that c q - 1, which the running
 *       scales s and r = 1/s accumulate, is an unbiased rounding error).  Pairs outside the range of the single-precision start
 *       (a_ij subnormal or beyond 2^+-800, |b/a_ij| beyond 2^+-100, a
 *       hyperbolic |zeta| < 2) take the oracle's orc_rotation and q from
 *       sqrt(1 - hyp t^2) refined as the reciprocal of c.  t and c agree with the oracle's to a few
 *       units in the last place (a test pins both to the exact root).
 *
 * Build: compiled into the oracle's shared object by oracle.py (gcc -O2
 * -ffp-contract=off: every fused multiply-add is an explicit fma()).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MDL_OK 0
#define MDL_ARG (-1)
#define MDL_RANK (-2)

int orc_rotation(double aii, double ajj, double aij, int hyp, double *t, double *c);
void orc_modulus_pairs(int r, int nsteps, int *pairs);

/* the scaled column update (M4) on two vectors of length m */
static void mdl_rotate_cols(int m, double *x, double *y, double alpha, double beta)
{
    for (int i = 0; i < m; ++i) {
        const double xi = x[i], yi = y[i];
        x[i] = fma(alpha, yi, xi);
        y[i] = fma(beta, xi, yi);
    }
}

/* the step's scaled rotations (M4) on every row x of the row-major nn x nn
 * matrix S: entries p, q of the row */
static void mdl_mix_rows(int nn, double *S, int h, const int *P, const int *Q, const double *AL,
                         const double *BE, const int *rot)
{
    for (int x = 0; x < nn; ++x)
        for (int k = 0; k < h; ++k) {
            if (!rot[k]) continue;
            double *row = S + (int64_t)x * nn;
            const double a = row[P[k]], b = row[Q[k]];
            row[P[k]] = fma(AL[k], b, a);
            row[Q[k]] = fma(BE[k], a, b);
        }
}

/* M5: c from an estimate c0 by one Newton step on c^2 (1 - hyp t^2) = 1 with
 * the residual (1 - c0^2) + hyp (c0 t)^2 formed from t (as the oracle's
 * orc_cosine), and q = 1/c from an estimate q0 by one Newton step */
static double mdl_cosine_step(double t, int hyp, double c0)
{
    const double s = c0 * t;
    return fma(0.5 * c0, fma(hyp < 0 ? -s : s, s, fma(-c0, c0, 1.0)), c0);
}
static double mdl_reciprocal_step(double c, double q0) { return fma(q0, fma(-c, q0, 1.0), q0); }

/* q = 1/c as the kernels form it beside the oracle's c: sqrt(x) refined */
static double mdl_inv_c(double t, double c, int hyp)
{
    const double q0 = hyp < 0 ? sqrt(1.0 + t * t) : sqrt((1.0 - t) * (1.0 + t));
    return mdl_reciprocal_step(c, q0);
}

/* M5: bit-level conversions (no rounding but the stated truncation) */
static uint64_t mdl_bits(double x)
{
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
}
static double mdl_from_bits(uint64_t u)
{
    double x;
    memcpy(&x, &u, 8);
    return x;
}
static int mdl_exp_field(double x) { return (int)((mdl_bits(x) >> 52) & 0x7ff) - 1023; }
/* x 2^-e truncated to single precision (x normal, the result normal) */
static float mdl_f32_scaled(double x, int e)
{
    const uint64_t u = mdl_bits(x);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t ex = (uint32_t)((int)((hi >> 20) & 0x7ff) - 1023 - e + 127);
    const uint32_t b = (hi & 0x80000000u) | (ex << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    float f;
    memcpy(&f, &b, 4);
    return f;
}
/* f 2^e exactly (f a normal single, the result normal) */
static double mdl_f64_scaled(float f, int e)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    const uint32_t ex = (uint32_t)((int)((b >> 23) & 0xff) - 127 + e + 1023);
    const uint32_t hi = (b & 0x80000000u) | (ex << 20) | ((b & 0x7fffffu) >> 3);
    return mdl_from_bits(((uint64_t)hi << 32) | (uint64_t)(uint32_t)(b << 29));
}
static double mdl_neg(double x) { return mdl_from_bits(mdl_bits(x) ^ 0x8000000000000000ull); }

/* M5: the rotation (t, c) and q = 1/c of a pair that fails Eq. 2.3; returns
 * nonzero for a rank-deficient hyperbolic pair (as orc_rotation) */
int mdl_rotation(double aii, double ajj, double aij, int hyp, double *t, double *c, double *q)
{
    const int trig = hyp < 0;
    const double b = trig ? ajj - aii : aii + ajj;
    const int E = mdl_exp_field(aij), eb = mdl_exp_field(b);
    const uint64_t abits = mdl_bits(aij) & 0x7fffffffffffffffull, bbits = mdl_bits(b) & 0x7fffffffffffffffull;
    int fast = E > -800 && E < 800;
    if (bbits == 0)
        fast = fast && trig;
    else
        fast = fast && eb > -1023 && eb < 1024 && eb - E >= -100 && eb - E <= 100;
    if (fast && !trig) fast = bbits >= abits + (2ull << 52); /* |b| >= 4 |a_ij| */
    if (!fast) {
        const int st = orc_rotation(aii, ajj, aij, hyp, t, c);
        *q = st == 0 ? mdl_inv_c(*t, *c, hyp) : 1.0;
        return st;
    }
    const float af = mdl_f32_scaled(aij, E);
    const float bf = bbits == 0 ? 0.0f : mdl_f32_scaled(b, E);
    const float two_af = 2.0f * af;
    const float z = (trig ? bf : -bf) / two_af; /* zeta */
    const float az = fabsf(z);
    float tf;
    if (az <= 1048576.0f) {
        const float zz = az * az;
        const float r = trig ? zz + 1.0f : zz - 1.0f;
        const float den = az + sqrtf(r);
        tf = 1.0f / den;
    } else {
        tf = 0.5f / az;
    }
    if (z < 0.0f) tf = -tf;
    const float fp = two_af * tf; /* f'(t) 2^-E = 2 a_ij t + b, scaled */
    const float gf = 1.0f / (fp + bf);
    const double ngd = mdl_neg(mdl_f64_scaled(gf, -E));
    const double sa = trig ? mdl_neg(aij) : aij;
    double tt = mdl_f64_scaled(tf, 0);
    for (int it = 0; it < 2; ++it) tt = fma(fma(fma(aij, tt, b), tt, sa), ngd, tt);
    const double x = fma(tt, trig ? tt : mdl_neg(tt), 1.0);
    const float sx = sqrtf(mdl_f32_scaled(x, 0));
    const float r0 = 1.0f / sx;
    double y = mdl_f64_scaled(r0, 0);
    y = fma(mdl_f64_scaled(r0, -1), fma(mdl_neg(x * y), y, 1.0), y);
    *t = tt;
    *c = mdl_cosine_step(tt, hyp, y);
    *q = mdl_reciprocal_step(*c, x * *c);
    return 0;
}

/* Model of the inner solve of one pivot block (nn x nn column-major,
 * symmetric, signs sgn).  mode 0: full passes until one rotates nothing or
 * max_passes ran; 1: one cross pass; 2: one full pass.  Outputs as for
 * orc_inner_solve: A <- the final block (A itself, not its transpose), W the
 * accumulated transformation, rotation count, passes, largest |t|. */
int mdl_inner_solve(int nn, double *A, const int8_t *sgn, double tol, int mode,
                    int max_passes, double *W, int64_t *nrot_out, int *passes_out, double *tmax_out)
{
    if (nn < 2 || (nn % 2) || max_passes < 1 || mode < 0 || mode > 2) return MDL_ARG;
    const int h = nn / 2;
    int *pairs = (int *)malloc(sizeof(int) * (size_t)nn * (size_t)h * 2);
    int *P = (int *)malloc(sizeof(int) * h), *Q = (int *)malloc(sizeof(int) * h);
    double *T = (double *)malloc(sizeof(double) * h), *C = (double *)malloc(sizeof(double) * h);
    double *QV = (double *)malloc(sizeof(double) * h);
    int *H = (int *)malloc(sizeof(int) * h), *rot = (int *)malloc(sizeof(int) * h);
    double *S = (double *)malloc(sizeof(double) * (size_t)nn * nn);
    double *St = (double *)malloc(sizeof(double) * (size_t)nn * nn);
    double *d = (double *)malloc(sizeof(double) * nn);
    double *apq = (double *)malloc(sizeof(double) * h);
    double *sc = (double *)malloc(sizeof(double) * nn), *rc = (double *)malloc(sizeof(double) * nn);
    double *AL = (double *)malloc(sizeof(double) * h), *BE = (double *)malloc(sizeof(double) * h);
    double tmax = 0.0;
    orc_modulus_pairs(nn, nn, pairs);
    memset(W, 0, sizeof(double) * (size_t)nn * nn);
    for (int i = 0; i < nn; ++i) W[i + (int64_t)i * nn] = 1.0;
    for (int x = 0; x < nn; ++x)
        for (int y = 0; y < nn; ++y) S[(int64_t)x * nn + y] = A[x + (int64_t)y * nn];
    for (int x = 0; x < nn; ++x) {
        d[x] = A[x + (int64_t)x * nn];
        sc[x] = 1.0;
        rc[x] = 1.0;
    }
    int transposed = 0; /* 0: S = A, 1: S = A^T (M2) */
    int status = MDL_OK, npass = 0;
    int64_t nrot_total = 0;
    const int npass_max = (mode == 0) ? max_passes : 1;
    for (int pass = 0; pass < npass_max; ++pass) {
        ++npass;
        int64_t nrot_pass = 0;
        const int nsteps = (mode == 1) ? h : nn;
        for (int s = 0; s < nsteps; ++s) {
            for (int k = 0; k < h; ++k) { /* M1 */
                int a, b;
                if (mode == 1) {
                    a = k;
                    b = h + ((k + s) % h);
                } else {
                    a = pairs[(s * h + k) * 2];
                    b = pairs[(s * h + k) * 2 + 1];
                }
                P[k] = a < b ? a : b;
                Q[k] = a < b ? b : a;
            }
            for (int k = 0; k < h; ++k) {
                const int p = P[k], q = Q[k];
                const double a_pq = (sc[p] * sc[q]) * (transposed ? S[(int64_t)q * nn + p] : S[(int64_t)p * nn + q]);
                apq[k] = a_pq;
                H[k] = (sgn[p] == sgn[q]) ? -1 : 1;
                T[k] = 0.0;
                C[k] = 1.0;
                QV[k] = 1.0;
                rot[k] = 0;
                if (a_pq == 0.0 || fabs(a_pq) < tol * sqrt(d[p] * d[q])) continue; /* Eq. 2.3 */
                if (mdl_rotation(d[p], d[q], a_pq, H[k], &T[k], &C[k], &QV[k]) != 0) { /* M5 */
                    status = MDL_RANK;
                    goto out;
                }
                rot[k] = 1;
                ++nrot_pass;
                if (fabs(T[k]) > tmax) tmax = fabs(T[k]);
            }
            for (int k = 0; k < h; ++k) { /* M4: coefficients from the step's starting scales */
                if (!rot[k]) continue;
                const int p = P[k], q = Q[k];
                const double ht = H[k] < 0 ? -T[k] : T[k];
                AL[k] = ht * (sc[q] * rc[p]);
                BE[k] = T[k] * (sc[p] * rc[q]);
            }
            /* M2: one half on the rows of S, transpose, the other half */
            mdl_mix_rows(nn, S, h, P, Q, AL, BE, rot);
            for (int x = 0; x < nn; ++x)
                for (int y = 0; y < nn; ++y) St[(int64_t)y * nn + x] = S[(int64_t)x * nn + y];
            memcpy(S, St, sizeof(double) * (size_t)nn * nn);
            transposed ^= 1;
            mdl_mix_rows(nn, S, h, P, Q, AL, BE, rot);
            int renorm = 0;
            for (int k = 0; k < h; ++k) { /* M3, M4 */
                if (!rot[k]) continue;
                const int p = P[k], q = Q[k];
                const double ht = H[k] < 0 ? -T[k] : T[k];
                d[p] = fma(ht, apq[k], d[p]);
                d[q] = fma(T[k], apq[k], d[q]);
                S[(int64_t)p * nn + p] = 0.0;
                S[(int64_t)q * nn + q] = 0.0;
                S[(int64_t)p * nn + q] = 0.0;
                S[(int64_t)q * nn + p] = 0.0;
                const double qv = QV[k];
                sc[p] = sc[p] * C[k];
                sc[q] = sc[q] * C[k];
                rc[p] = rc[p] * qv;
                rc[q] = rc[q] * qv;
                if (abs(ilogb(sc[p])) > 8 || abs(ilogb(sc[q])) > 8) renorm = 1;
            }
            for (int k = 0; k < h; ++k) /* W <- W R */
                if (rot[k]) mdl_rotate_cols(nn, W + (int64_t)P[k] * nn, W + (int64_t)Q[k] * nn, AL[k], BE[k]);
            if (renorm) {
                for (int x = 0; x < nn; ++x)
                    for (int y = 0; y < nn; ++y) S[(int64_t)x * nn + y] = (sc[x] * sc[y]) * S[(int64_t)x * nn + y];
                for (int y = 0; y < nn; ++y)
                    for (int x = 0; x < nn; ++x) W[x + (int64_t)y * nn] = W[x + (int64_t)y * nn] * sc[y];
                for (int x = 0; x < nn; ++x) sc[x] = rc[x] = 1.0;
            }
        }
        nrot_total += nrot_pass;
        if (nrot_pass == 0) break;
    }
out:
    for (int x = 0; x < nn; ++x)
        for (int y = 0; y < nn; ++y)
            A[x + (int64_t)y * nn] =
                x == y ? d[x] : (sc[x] * sc[y]) * (transposed ? S[(int64_t)y * nn + x] : S[(int64_t)x * nn + y]);
    for (int y = 0; y < nn; ++y)
        for (int x = 0; x < nn; ++x) W[x + (int64_t)y * nn] = W[x + (int64_t)y * nn] * sc[y];
    if (nrot_out) *nrot_out = nrot_total;
    if (passes_out) *passes_out = npass;
    if (tmax_out) *tmax_out = tmax;
    free(pairs); free(P); free(Q); free(T); free(C); free(QV); free(H); free(rot);
    free(S); free(St); free(d); free(apq); free(sc); free(rc); free(AL); free(BE);
    return status;
}
