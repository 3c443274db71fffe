/*
 * hsvd_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * one-sided Jacobi hyperbolic SVD (Novakovic & Singer, "A GPU-based hyperbolic
 * SVD algorithm").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, import or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library; the two are written independently from the paper.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (contraction off, so every
 * fused multiply-add in here is one written as fma() on purpose).
 *
 * Storage is column-major FP64 throughout, zero-based indices (Sec. 4).
 *
 * What each function follows:
 *   orc_rotation       -- rotation parameters from a 2x2 pivot block
 *                         (Sec. 2, Eq. 2.2, the theta/t definitions, Eq. 2.6).
 *   orc_modulus_pairs  -- the modified modulus pivot strategy as the stepper
 *                         of Alg. 4.3 / Alg. 4.4 (Sec. 2 text on the strategy).
 *   orc_set_threads    -- threads of the OpenMP modulus-parallel mode
 *   orc_hsvd           -- pointwise one-sided hyperbolic Jacobi (Eq. 2.1,
 *                         Eq. 2.3 test, Eq. 2.4/2.5 updates in the unified
 *                         form of Alg. 4.5, Sec. 2 stopping rule), with the
 *                         row-cyclic order or the modulus order and optional
 *                         diagonal sorting (Sec. 4, Sort_Diagonal); optional
 *                         early stop at the tangent threshold T_eps (Sec. 2)
 *                         through the convergence statistic of Eq. 4.2.
 *   orc_inner_solve    -- J-orthogonalisation of one 2b x 2b pivot block A_P by
 *                         rotations applied one at a time as R^T A R (Sec. 5
 *                         block-oriented method, Sec. 6 full-block variant),
 *                         row-cyclic inner order (Sec. 5) or, on request, the
 *                         pairs of the parallel strategy (R9).
 *   orc_sym_factor     -- symmetric indefinite factorisation M = G J G^T with
 *                         complete (Bunch-Parlett) pivoting (Sec. 1: M given
 *                         explicitly is factored first).
 *   orc_block_hsvd     -- blocked one-sided method: modulus strategy over block
 *                         columns, Gram block, inner solve, G/V update
 *                         (Sec. 5 block-oriented description, Eq. 2.1).
 *   orc_hyp_qr         -- hyperbolic (J-orthogonal) Householder QR of a tall
 *                         matrix (Sec. 1: a factor whose transpose is tall is
 *                         shortened by the hyperbolic QR of its transpose),
 *                         reading R15 below; orc_hyp_qr_apply_tt applies the
 *                         transformation's transpose.
 *   orc_wide_hsvd      -- HSVD of a wide factor through that QR (Sec. 1: the
 *                         HSVD of the square R^T, then V premultiplied by the
 *                         transformation).
 *
 * Readings of the paper where it is silent or garbled:
 *   R1  theta as printed in Sec. 2 has the sign of `hyp' flipped against the
 *       update of Alg. 4.5; requiring a'_ij = 0 under that update gives
 *       theta = 2 a_ij / (-a_ii - hyp a_jj).  Eq. 2.6 agrees with this form.
 *   R2  t is the smaller root of the zeroing quadratic (|phi| <= pi/4),
 *       written through zeta so nothing overflows:
 *         trigonometric  zeta = (a_jj - a_ii) / (2 a_ij),
 *                        t = sign(zeta) / (|zeta| + sqrt(zeta^2 + 1)),
 *                        c = 1 / sqrt(1 + t^2)
 *         hyperbolic     zeta = -(a_ii + a_jj) / (2 a_ij),
 *                        t = sign(zeta) / (|zeta| + sqrt(zeta^2 - 1)),
 *                        c = 1 / sqrt((1 - t)(1 + t)).
 *       sign(0) is +1.  |zeta| <= 1 in the hyperbolic case means the pair is
 *       numerically rank deficient: status ORC_RANK, nothing is rotated.
 *   R3  Alg. 4.4 as printed steps out of range with zero-based indices; the
 *       threshold that reproduces the strategy described in Sec. 2 (r steps,
 *       r/2 disjoint pairs per step, pairs (i, i+r/2) twice, next quasi-sweep
 *       starting with the assignment reversed) is  ip + jp > r - 2.
 *   R4  Sorting (Sec. 4): the J = +1 part by d decreasing, the J = -1 part by
 *       d increasing, equal keys keep their current relative order.
 *   R5  A sweep counts every sweep run, including the final one in which no
 *       pair rotates (Sec. 2 stopping rule).
 *   R7  Inside a pivot block the diagonal is carried by Eq. 2.6 (as Sec. 4
 *       carries d for the pointwise method) rather than recomputed.
 *   R9  Inner pair order.  Sec. 5 gives the block-oriented method a
 *       row-cyclic inner order, one rotation at a time; that is the default
 *       (order 0).  Order 1 takes the pairs of the parallel strategy of
 *       Sec. 2 (modified modulus over the 2b indices of the block; for the
 *       cross pass k paired with b + ((k + s) mod b) at step s), still one
 *       rotation at a time, so that a parallel implementation can be
 *       compared with it pair for pair.
 *   R6  A pair with a_ij == 0 exactly is orthogonal and is never rotated (the
 *       strict test of Eq. 2.3 would otherwise "rotate" a zero column by the
 *       identity for ever).  A zero column (sigma_j = 0) is rank deficiency,
 *       which the paper excludes (Sec. 1): status ORC_RANK.
 *   R14 The tangent threshold (Sec. 2, T_eps = sqrt(eps)/2) is optional and
 *       off by default (tstop = 0): only a sweep without rotations ends the
 *       iteration.  With tstop > 0 every applied rotation contributes the
 *       code of Eq. 4.2 -- (11)_2 if |t| > tstop, (01)_2 otherwise -- to a
 *       bitwise-or over the sweep (for the blocked method the tangents are
 *       those of the inner rotations); (00)_2 (no rotation) stops as before,
 *       (01)_2 also stops, after that sweep, and (11)_2 goes on.  Pairs that
 *       pass Eq. 2.3 compute no tangent and contribute nothing.  The sweep
 *       count includes the sweep that stopped.
 *   R15 Sec. 1 names the hyperbolic QR factorisation of G^T for a wide G but
 *       does not define it.  Here: J-orthogonal Householder reflectors
 *       I - beta v v^T S, pivots chosen on the trailing J-Gram by the
 *       Bunch-Parlett rule (1 x 1 on the largest |J-norm^2|, else a 2 x 2
 *       block reduced through z = x +- y and then y), a row interchange when
 *       the pivot row's sign is not that of the reduced J-norm^2.  A zero
 *       trailing J-Gram is ORC_RANK.  With J = I this is Householder QR with
 *       column pivoting on the largest trailing norm.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_ARG (-1)
#define ORC_RANK (-2)
#define ORC_NONFINITE (-3)

/* how the iteration ended (R14) */
#define ORC_STOP_NONE 0    /* not converged, or an error          */
#define ORC_STOP_ORTHO 1   /* a sweep without rotations, Eq. 2.3  */
#define ORC_STOP_TANGENT 2 /* every tangent of a sweep <= tstop   */

/* Eq. 4.2: the convergence code of one applied rotation with tangent t */
static int conv_code(double t, double tstop)
{
    return (tstop > 0.0 && fabs(t) <= tstop) ? 1 : 3;
}

/* ------------------------------------------------------------------------ */
/* Rotation parameters (Sec. 2, Eq. 2.2; readings R1, R2).                    */
/* hyp = -1: trigonometric (equal signs in J), +1: hyperbolic.                */
/* The rotation applied to a column pair is                                   */
/*   g_i' = (g_i + hyp*t*g_j) * c,   g_j' = (t*g_i + g_j) * c   (Alg. 4.5).   */
/* ------------------------------------------------------------------------ */
/* c = 1/sqrt(1 - hyp t^2) to about half a unit in the last place, from an
 * estimate c0: one Newton step on c^2 (1 - hyp t^2) = 1 whose residual is
 * formed from t itself, (1 - c0^2) + hyp (c0 t)^2, by fused multiply-adds.
 * 1/sqrt(x) with x = 1 - hyp t^2 rounded first, as two correctly rounded
 * operations, leans upward for small t: c^2 (1 - hyp t^2) - 1 averages about
 * +u over the rotations with t^2 between u and 2^-30 (the rounding of x
 * before the square root, and the square root's before the division).  A
 * column takes about 10^5 rotations at n = 4096, and that bias became a
 * relative +1.2e-12 on every large sigma, measured against LAPACK's
 * eigenvalues of the pencil (G^T G, J). */
static double orc_cosine(double t, int hyp, double c0)
{
    const double s = c0 * t;
    return fma(0.5 * c0, fma(hyp < 0 ? -s : s, s, fma(-c0, c0, 1.0)), c0);
}

int orc_rotation(double aii, double ajj, double aij, int hyp, double *t, double *c)
{
    double zeta, tt;
    if (hyp < 0) {
        zeta = (ajj - aii) / (2.0 * aij);
        tt = 1.0 / (fabs(zeta) + sqrt(zeta * zeta + 1.0));
        if (zeta < 0.0) tt = -tt;
        *t = tt;
        *c = orc_cosine(tt, -1, 1.0 / sqrt(1.0 + tt * tt));
        return ORC_OK;
    }
    zeta = -(aii + ajj) / (2.0 * aij);
    if (!(fabs(zeta) > 1.0)) {
        *t = 0.0;
        *c = 1.0;
        return ORC_RANK;
    }
    tt = 1.0 / (fabs(zeta) + sqrt(zeta * zeta - 1.0));
    if (zeta < 0.0) tt = -tt;
    *t = tt;
    *c = orc_cosine(tt, 1, 1.0 / sqrt((1.0 - tt) * (1.0 + tt)));
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Modified modulus strategy (Sec. 2; Alg. 4.3 and Alg. 4.4 with R3).        */
/* r even.  pairs[(s*(r/2) + k)*2 + {0,1}] = pivot pair of task k at step s,  */
/* for s = 0 .. nsteps-1 (nsteps may exceed r: the stepper just continues).   */
/* ------------------------------------------------------------------------ */
void orc_modulus_pairs(int r, int nsteps, int *pairs)
{
    int half = r / 2;
    int *ip = (int *)malloc(sizeof(int) * half), *jp = (int *)malloc(sizeof(int) * half);
    int *ib = (int *)malloc(sizeof(int) * half), *jb = (int *)malloc(sizeof(int) * half);
    for (int k = 0; k < half; ++k) { /* Alg. 4.3: antidiagonal start */
        ip[k] = k;
        ib[k] = k;
        jp[k] = r - k - 1;
        jb[k] = jp[k];
    }
    for (int s = 0; s < nsteps; ++s) {
        for (int k = 0; k < half; ++k) {
            pairs[(s * half + k) * 2 + 0] = ib[k];
            pairs[(s * half + k) * 2 + 1] = jb[k];
        }
        for (int k = 0; k < half; ++k) { /* Alg. 4.4 with threshold r-2 */
            if (ip[k] + jp[k] > r - 2) {
                ip[k] = ip[k] + 1;
                if (ip[k] == jp[k]) {
                    ip[k] = ip[k] - half;
                    jp[k] = ip[k];
                }
                ib[k] = ip[k];
            } else {
                jp[k] = jp[k] + 1;
                jb[k] = jp[k];
            }
        }
    }
    free(ip); free(jp); free(ib); free(jb);
}

/* ------------------------------------------------------------------------ */
/* Small helpers (plain loops).                                               */
/* ------------------------------------------------------------------------ */
static double dot(int64_t m, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += x[i] * y[i];
    return s;
}

/* Euclidean norm with the scale / sum-of-squares recurrence of the reference
 * BLAS dnrm2, so no intermediate overflows or underflows. */
static double nrm2(int64_t m, const double *x)
{
    double scale = 0.0, ssq = 1.0;
    for (int64_t i = 0; i < m; ++i) {
        if (x[i] != 0.0) {
            double a = fabs(x[i]);
            if (scale < a) {
                ssq = 1.0 + ssq * (scale / a) * (scale / a);
                scale = a;
            } else {
                ssq += (a / scale) * (a / scale);
            }
        }
    }
    return scale * sqrt(ssq);
}

/* Column update of Alg. 4.5 (Eq. 2.4 / 2.5): the parenthesised term with one
 * fused multiply-add (Sec. 2), then the scaling by c. */
static void rotate_cols(int64_t m, double *x, double *y, int hyp, double t, double c)
{
    double ht = hyp < 0 ? -t : t;
    for (int64_t i = 0; i < m; ++i) {
        double xi = x[i], yi = y[i];
        x[i] = fma(ht, yi, xi) * c;
        y[i] = fma(t, xi, yi) * c;
    }
}

static int all_finite(int64_t m, int64_t n, const double *G, int64_t ld)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i)
            if (!isfinite(G[i + j * ld])) return 0;
    return 1;
}

/* Sorting permutation (Sec. 4, Sort_Diagonal; reading R4).  pos[] lists the
 * columns in their current order; on return it lists them sorted, J+ part by
 * d decreasing then J- part by d increasing, equal keys in current order.
 * Written as a plain stable insertion sort. */
static void sort_positions(int n, int *pos, const double *d, const int8_t *sgn)
{
    int *tmp = (int *)malloc(sizeof(int) * n);
    int np = 0;
    for (int k = 0; k < n; ++k)
        if (sgn[pos[k]] > 0) tmp[np++] = pos[k];
    int nm = np;
    for (int k = 0; k < n; ++k)
        if (sgn[pos[k]] < 0) tmp[nm++] = pos[k];
    for (int k = 1; k < np; ++k) { /* decreasing d */
        int v = tmp[k], x = k - 1;
        while (x >= 0 && d[tmp[x]] < d[v]) { tmp[x + 1] = tmp[x]; --x; }
        tmp[x + 1] = v;
    }
    for (int k = np + 1; k < n; ++k) { /* increasing d */
        int v = tmp[k], x = k - 1;
        while (x >= np && d[tmp[x]] > d[v]) { tmp[x + 1] = tmp[x]; --x; }
        tmp[x + 1] = v;
    }
    memcpy(pos, tmp, sizeof(int) * n);
    free(tmp);
}

/* Finalisation (Sec. 2): sigma_j = ||g_j||, u_j = g_j / sigma_j, V = W. */
static void finalise(int64_t m, int64_t n, const double *Gw, const double *W,
                     double *sigma, double *U, int64_t ldu, double *V, int64_t ldv)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = nrm2(m, Gw + j * m);
        sigma[j] = s;
        if (U)
            for (int64_t i = 0; i < m; ++i) U[i + j * ldu] = Gw[i + j * m] / s;
        if (V)
            for (int64_t i = 0; i < n; ++i) V[i + j * ldv] = W[i + j * n];
    }
}

/* One pivot pair of the pointwise method: Gram entries recomputed from the
 * current columns, the relative orthogonality test (Eq. 2.3), and if it fails
 * the rotation of the G and W columns (Alg. 4.5). */
static int pointwise_pair(int64_t mw, int64_t nw, double *Gw, double *W, const int8_t *sgn,
                          double tol, int pi, int pj, int64_t *nrot, double tstop, int *cd)
{
    double *gi = Gw + (int64_t)pi * mw, *gj = Gw + (int64_t)pj * mw;
    double aii = dot(mw, gi, gi), ajj = dot(mw, gj, gj), aij = dot(mw, gi, gj);
    if (aij == 0.0 || fabs(aij) < tol * sqrt(aii * ajj)) return ORC_OK; /* Eq. 2.3, R6 */
    int hyp = (sgn[pi] == sgn[pj]) ? -1 : 1;
    double t, c;
    if (orc_rotation(aii, ajj, aij, hyp, &t, &c) != ORC_OK) return ORC_RANK;
    rotate_cols(mw, gi, gj, hyp, t, c);
    rotate_cols(nw, W + (int64_t)pi * nw, W + (int64_t)pj * nw, hyp, t, c);
    ++*nrot;
    *cd |= conv_code(t, tstop);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Pointwise one-sided hyperbolic Jacobi (Eq. 2.1 - 2.5, Alg. 4.5).           */
/*   order 0: row-cyclic (i < j, i outer), the sequential comparison method   */
/*            of Sec. 5;                                                      */
/*   order 1: modified modulus strategy (Sec. 2), pairs of a step applied one */
/*            after the other (they are disjoint, so this equals applying     */
/*            them at once), positions mapped to columns through the current  */
/*            permutation (Sec. 4: columns are never moved).                  */
/* For order 1 the columns are first grouped J+ then J- (Alg. 4.2 assumes     */
/* J = diag(I_p, -I_{n-p})), odd n gets one bordering column (Eq. 4.1).       */
/* sort != 0 sorts the positions before the first sweep and after each sweep  */
/* (Alg. 4.1).  tstop > 0 adds the tangent-threshold stop (R14); *stop_rule  */
/* (may be NULL) receives ORC_STOP_*.  Returns ORC_OK, ORC_NOT_CONVERGED,     */
/* ORC_RANK, ORC_NONFINITE or ORC_ARG; sigma, U (m x n, ldu) and V (n x n,    */
/* ldv; either may be NULL) are written in input column order.                */
/* ------------------------------------------------------------------------ */
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the modulus-parallel mode (OpenMP builds; 0 = the runtime's
 * default).  Returns the number of threads that will be used, 1 without
 * OpenMP. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_hsvd(int64_t m, int64_t n, const double *G, int64_t ldg, const int8_t *J,
             double tol, int max_sweeps, int order, int sort,
             double *sigma, double *U, int64_t ldu, double *V, int64_t ldv,
             int *sweeps, int64_t *rotations, double tstop, int *stop_rule)
{
    if (stop_rule) *stop_rule = ORC_STOP_NONE;
    if (m < n || n < 1 || ldg < m || max_sweeps < 1 || !(tol > 0.0) || !(tstop >= 0.0)) return ORC_ARG;
    for (int64_t j = 0; j < n; ++j)
        if (J[j] != 1 && J[j] != -1) return ORC_ARG;
    if (!all_finite(m, n, G, ldg)) return ORC_NONFINITE;

    /* working copy, bordered with one unit column in a fresh row if the
     * modulus strategy needs an even order (Eq. 4.1) */
    int64_t nw = (order == 1 && (n % 2)) ? n + 1 : n;
    int64_t mw = m + (nw - n);
    double *Gw = (double *)calloc((size_t)(mw * nw), sizeof(double));
    double *W = (double *)calloc((size_t)(nw * nw), sizeof(double));
    int8_t *sgn = (int8_t *)malloc((size_t)nw);
    double *d = (double *)malloc(sizeof(double) * (size_t)nw);
    int *pos = (int *)malloc(sizeof(int) * (size_t)nw);
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) Gw[i + j * mw] = G[i + j * ldg];
        sgn[j] = J[j];
    }
    for (int64_t j = n; j < nw; ++j) {
        Gw[(m + (j - n)) + j * mw] = 1.0;
        sgn[j] = 1;
    }
    for (int64_t j = 0; j < nw; ++j) W[j + j * nw] = 1.0;

    int *pairs = NULL;
    if (order == 1) {
        pairs = (int *)malloc(sizeof(int) * (size_t)(nw * nw));
        orc_modulus_pairs((int)nw, (int)nw, pairs);
        int k = 0; /* J+ first, J- after, each in input order */
        for (int64_t j = 0; j < nw; ++j) if (sgn[j] > 0) pos[k++] = (int)j;
        for (int64_t j = 0; j < nw; ++j) if (sgn[j] < 0) pos[k++] = (int)j;
    } else {
        for (int64_t j = 0; j < nw; ++j) pos[j] = (int)j;
    }

    int status = ORC_NOT_CONVERGED, sw = 0;
    int64_t nrot_total = 0;
    if (order == 1 && sort) {
        for (int64_t j = 0; j < nw; ++j) d[j] = dot(mw, Gw + j * mw, Gw + j * mw);
        sort_positions((int)nw, pos, d, sgn);
    }
    int rule = ORC_STOP_NONE;
    for (sw = 1; sw <= max_sweeps; ++sw) {
        int64_t nrot = 0;
        int st = ORC_OK, cd = 0;
        if (order == 1) {
            /* the pairs of a step are disjoint, so the step's pairs may run in
             * any order or at once: with OpenMP they are spread over the
             * host's threads (same arithmetic per pair, the same result) */
            const int64_t half = nw / 2;
            for (int64_t s = 0; s < nw && st == ORC_OK; ++s) {
                int64_t step_rot = 0;
                int step_st = ORC_OK, step_cd = 0;
#pragma omp parallel for schedule(static) reduction(+ : step_rot) reduction(min : step_st) reduction(| : step_cd) if (nw >= 64)
                for (int64_t k = 0; k < half; ++k) {
                    const int a = pairs[(s * half + k) * 2], b = pairs[(s * half + k) * 2 + 1];
                    int64_t r = 0;
                    int c = 0;
                    const int sk = pointwise_pair(mw, nw, Gw, W, sgn, tol, pos[a < b ? a : b], pos[a < b ? b : a], &r,
                                                  tstop, &c);
                    step_rot += r;
                    step_cd |= c;
                    if (sk < step_st) step_st = sk;
                }
                nrot += step_rot;
                cd |= step_cd;
                st = step_st;
            }
        } else {
            for (int64_t i = 0; i < nw - 1 && st == ORC_OK; ++i)
                for (int64_t j = i + 1; j < nw && st == ORC_OK; ++j)
                    st = pointwise_pair(mw, nw, Gw, W, sgn, tol, (int)i, (int)j, &nrot, tstop, &cd);
        }
        if (st != ORC_OK) {
            status = st;
            goto done;
        }
        nrot_total += nrot;
        if (cd == 0 || cd == 1) { /* (00)_2 or (01)_2 of Eq. 4.2 */
            status = ORC_OK;
            rule = cd == 0 ? ORC_STOP_ORTHO : ORC_STOP_TANGENT;
            break;
        }
        if (order == 1 && sort) {
            for (int64_t j = 0; j < nw; ++j) d[j] = dot(mw, Gw + j * mw, Gw + j * mw);
            sort_positions((int)nw, pos, d, sgn);
        }
    }
    if (sw > max_sweeps) sw = max_sweeps;
    if (!all_finite(mw, nw, Gw, mw)) status = ORC_NONFINITE;
done:
    if (status == ORC_OK || status == ORC_NOT_CONVERGED) {
        /* drop the bordering row/column: the unit column never rotates */
        double *Gc = (double *)malloc(sizeof(double) * (size_t)(m * n));
        double *Wc = (double *)malloc(sizeof(double) * (size_t)(n * n));
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t i = 0; i < m; ++i) Gc[i + j * m] = Gw[i + j * mw];
            for (int64_t i = 0; i < n; ++i) Wc[i + j * n] = W[i + j * nw];
        }
        finalise(m, n, Gc, Wc, sigma, U, ldu, V, ldv);
        for (int64_t j = 0; j < n; ++j)
            if (!(sigma[j] > 0.0)) status = ORC_RANK;
        free(Gc);
        free(Wc);
    }
    if (sweeps) *sweeps = sw;
    if (rotations) *rotations = nrot_total;
    if (stop_rule && status == ORC_OK) *stop_rule = rule;
    free(Gw); free(W); free(sgn); free(d); free(pos); free(pairs);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Inner solve: J-orthogonalisation of a pivot block A_P (nn x nn, nn even,   */
/* symmetric on entry, column-major, ld = nn) with signs sgn[nn] (Sec. 5      */
/* block-oriented method, Sec. 6 full-block variant).  Rotations are applied  */
/* one at a time, each as the symmetric two-sided update A <- R^T A R of the  */
/* plane rotation R of its pair (p, q), p < q (Eq. 2.1 / 2.2 on the pivot     */
/* block), see rotate_block:                                                  */
/*   - the test of Eq. 2.3 on (a_pp, a_qq, a_pq) (R6: a_pq == 0 is never      */
/*     rotated); if it fails, (t, c) from orc_rotation, hyp from the signs;   */
/*   - the diagonal is carried by Eq. 2.6 (R7), a_pq becomes 0;               */
/*   - W <- W R: columns p, q of W as in Alg. 4.5.                           */
/* Pair order (`order'):                                                      */
/*   0 row-cyclic: the inner order of the block-oriented method (Sec. 5):     */
/*     p outer, q inner, over the pairs the mode visits;                      */
/*   1 the parallel order: the steps of the modified modulus strategy over    */
/*     the nn indices (Sec. 2, Alg. 4.3/4.4), or for the cross pass the steps */
/*     s = 0 .. h-1 pairing k with h + ((k + s) mod h), h = nn/2; the         */
/*     disjoint pairs of a step are applied one after the other in ascending */
/*     order of their smaller index (they touch disjoint rows and columns,    */
/*     so their rotation parameters do not depend on that order).            */
/* Modes:                                                                     */
/*   0 full-block: passes over all pairs p < q until a pass rotates nothing   */
/*     or max_passes passes ran (Sec. 6);                                     */
/*   1 cross pass: one pass over the pairs of the off-diagonal block,         */
/*     p < h <= q (Sec. 5, every step of a sweep after the first);            */
/*   2 one pass over all pairs p < q (Sec. 5, the first step of a sweep).     */
/* On return A holds R^T A R for the product R of the applied rotations, W    */
/* (nn x nn) that product (starting from I); *tmax_out (may be NULL) the     */
/* largest |t| applied (0 if none).                                           */
/* ------------------------------------------------------------------------ */

/* One rotation of the pivot block: for every other index x the entries       */
/* (x, p), (x, q) take the column update of Alg. 4.5, and (p, x), (q, x) the  */
/* same values (the row update of R^T on a symmetric matrix); a_pp and a_qq   */
/* follow Eq. 2.6 with the a_pq before the rotation; a_pq = a_qp = 0.         */
static void rotate_block(int nn, double *A, double *W, int p, int q, int hyp, double t, double c)
{
    const double apq = A[p + (int64_t)q * nn];
    const double ht = hyp < 0 ? -t : t;
    for (int x = 0; x < nn; ++x) {
        if (x == p || x == q) continue;
        const double axp = A[x + (int64_t)p * nn], axq = A[x + (int64_t)q * nn];
        const double np_ = fma(ht, axq, axp) * c;
        const double nq_ = fma(t, axp, axq) * c;
        A[x + (int64_t)p * nn] = np_;
        A[p + (int64_t)x * nn] = np_;
        A[x + (int64_t)q * nn] = nq_;
        A[q + (int64_t)x * nn] = nq_;
    }
    A[p + (int64_t)p * nn] = fma(ht, apq, A[p + (int64_t)p * nn]);
    A[q + (int64_t)q * nn] = fma(t, apq, A[q + (int64_t)q * nn]);
    A[p + (int64_t)q * nn] = 0.0;
    A[q + (int64_t)p * nn] = 0.0;
    rotate_cols(nn, W + (int64_t)p * nn, W + (int64_t)q * nn, hyp, t, c);
}

/* Test and, if it fails, rotation of one pair; returns ORC_OK or ORC_RANK. */
static int inner_pair(int nn, double *A, double *W, const int8_t *sgn, double tol, int p, int q,
                      int64_t *nrot, double *tmax)
{
    const double apq = A[p + (int64_t)q * nn];
    const double app = A[p + (int64_t)p * nn], aqq = A[q + (int64_t)q * nn];
    if (apq == 0.0 || fabs(apq) < tol * sqrt(app * aqq)) return ORC_OK; /* Eq. 2.3, R6 */
    const int hyp = (sgn[p] == sgn[q]) ? -1 : 1;
    double t, c;
    if (orc_rotation(app, aqq, apq, hyp, &t, &c) != ORC_OK) return ORC_RANK;
    rotate_block(nn, A, W, p, q, hyp, t, c);
    ++*nrot;
    if (fabs(t) > *tmax) *tmax = fabs(t);
    return ORC_OK;
}

int orc_inner_solve(int nn, double *A, const int8_t *sgn, double tol, int mode, int order,
                    int max_passes, double *W, int64_t *nrot_out, int *passes_out, double *tmax_out)
{
    if (nn < 2 || (nn % 2) || max_passes < 1 || mode < 0 || mode > 2 || order < 0 || order > 1) return ORC_ARG;
    const int h = nn / 2;
    int *pairs = NULL;
    if (order == 1 && mode != 1) {
        pairs = (int *)malloc(sizeof(int) * (size_t)nn * (size_t)h * 2);
        orc_modulus_pairs(nn, nn, pairs);
    }
    int *step_p = (int *)malloc(sizeof(int) * (size_t)h), *step_q = (int *)malloc(sizeof(int) * (size_t)h);
    memset(W, 0, sizeof(double) * (size_t)nn * nn);
    for (int i = 0; i < nn; ++i) W[i + (int64_t)i * nn] = 1.0;
    double tmax = 0.0;
    int64_t nrot_total = 0;
    int status = ORC_OK, npass = 0;
    const int npass_max = (mode == 0) ? max_passes : 1;
    for (int pass = 0; pass < npass_max && status == ORC_OK; ++pass) {
        ++npass;
        int64_t nrot = 0;
        if (order == 0) {
            /* row-cyclic: p outer, q inner; the cross pass keeps p < h <= q */
            for (int p = 0; p < (mode == 1 ? h : nn - 1) && status == ORC_OK; ++p)
                for (int q = (mode == 1 ? h : p + 1); q < nn && status == ORC_OK; ++q)
                    status = inner_pair(nn, A, W, sgn, tol, p, q, &nrot, &tmax);
        } else {
            const int nsteps = (mode == 1) ? h : nn;
            for (int s = 0; s < nsteps && status == ORC_OK; ++s) {
                /* the step's pairs (p < q), applied in ascending order of p */
                for (int k = 0; k < h; ++k) {
                    int a, b;
                    if (mode == 1) {
                        a = k;
                        b = h + ((k + s) % h);
                    } else {
                        a = pairs[(s * h + k) * 2];
                        b = pairs[(s * h + k) * 2 + 1];
                    }
                    step_p[k] = a < b ? a : b;
                    step_q[k] = a < b ? b : a;
                }
                for (int k = 1; k < h; ++k) { /* insertion sort by p */
                    const int pk = step_p[k], qk = step_q[k];
                    int x = k - 1;
                    while (x >= 0 && step_p[x] > pk) {
                        step_p[x + 1] = step_p[x];
                        step_q[x + 1] = step_q[x];
                        --x;
                    }
                    step_p[x + 1] = pk;
                    step_q[x + 1] = qk;
                }
                for (int k = 0; k < h && status == ORC_OK; ++k)
                    status = inner_pair(nn, A, W, sgn, tol, step_p[k], step_q[k], &nrot, &tmax);
            }
        }
        nrot_total += nrot;
        if (nrot == 0) break;
    }
    if (nrot_out) *nrot_out = nrot_total;
    if (passes_out) *passes_out = npass;
    if (tmax_out) *tmax_out = tmax;
    free(pairs);
    free(step_p);
    free(step_q);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Blocked one-sided hyperbolic Jacobi (Sec. 5 block-oriented method; the     */
/* transformation of a pivot block applied to G_P and V_P from the right,     */
/* Eq. 2.1).  Columns are bordered (Eq. 4.1) to a multiple of 2b with unit    */
/* columns in fresh rows (sign +1), grouped J+ then J-, optionally sorted     */
/* (reading R4) before the first sweep and after each sweep, and the columns  */
/* are physically reordered to follow that order.  Each sweep runs nb steps   */
/* of the modulus strategy over the nb = n'/b block columns; each pair        */
/* (I, J) of a step forms A_P = [G_I G_J]^T [G_I G_J] (plain triple loop),    */
/* calls orc_inner_solve (inner_mode 0: full-block with inner_max_passes;     */
/* inner_mode 1: block-oriented -- whole block in the first step of a sweep,  */
/* cross pass afterwards; inner_order 0 row-cyclic, 1 the parallel order),    */
/* and, if any inner rotation was applied, updates                            */
/* [G_I G_J] <- [G_I G_J] W_P and [V_I V_J] <- [V_I V_J] W_P (plain triple    */
/* loops).  Stops after a sweep with no rotation, or (tstop > 0, R14) after a  */
/* sweep whose inner tangents are all <= tstop.  Outputs in input order.      */
/* ------------------------------------------------------------------------ */
int orc_block_hsvd(int64_t m, int64_t n, const double *G, int64_t ldg, const int8_t *J,
                   int b, double tol, int max_sweeps, int inner_mode, int inner_max_passes,
                   int inner_order, int sort, double *sigma, double *U, int64_t ldu, double *V, int64_t ldv,
                   int *sweeps, int64_t *rotations, double tstop, int *stop_rule)
{
    if (stop_rule) *stop_rule = ORC_STOP_NONE;
    if (m < n || n < 1 || ldg < m || b < 1 || max_sweeps < 1 || !(tol > 0.0) || !(tstop >= 0.0) ||
        inner_order < 0 || inner_order > 1)
        return ORC_ARG;
    for (int64_t j = 0; j < n; ++j)
        if (J[j] != 1 && J[j] != -1) return ORC_ARG;
    if (!all_finite(m, n, G, ldg)) return ORC_NONFINITE;
    int64_t nw = ((n + 2 * b - 1) / (2 * b)) * (2 * b);
    int64_t mw = m + (nw - n);
    int nb = (int)(nw / b), nn = 2 * b;
    double *Gw = (double *)calloc((size_t)(mw * nw), sizeof(double));
    double *W = (double *)calloc((size_t)(nw * nw), sizeof(double));
    double *Gt = (double *)malloc(sizeof(double) * (size_t)(mw * nw));
    double *Wt = (double *)malloc(sizeof(double) * (size_t)(nw * nw));
    int8_t *sgn = (int8_t *)malloc((size_t)nw), *sgt = (int8_t *)malloc((size_t)nw);
    int *col = (int *)malloc(sizeof(int) * (size_t)nw), *colt = (int *)malloc(sizeof(int) * (size_t)nw);
    int *pos = (int *)malloc(sizeof(int) * (size_t)nw);
    double *d = (double *)malloc(sizeof(double) * (size_t)nw);
    double *A = (double *)malloc(sizeof(double) * nn * nn), *Wp = (double *)malloc(sizeof(double) * nn * nn);
    double *Pan = (double *)malloc(sizeof(double) * (size_t)(mw > nw ? mw : nw) * nn);
    int8_t *ps = (int8_t *)malloc(nn);
    int *pairs = (int *)malloc(sizeof(int) * (size_t)nb * nb);
    orc_modulus_pairs(nb, nb, pairs);

    /* bordered copy; col[k] = input column held at working position k */
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) Gt[i + j * mw] = G[i + j * ldg];
        for (int64_t i = m; i < mw; ++i) Gt[i + j * mw] = 0.0;
        sgt[j] = J[j];
    }
    for (int64_t j = n; j < nw; ++j) {
        for (int64_t i = 0; i < mw; ++i) Gt[i + j * mw] = 0.0;
        Gt[(m + (j - n)) + j * mw] = 1.0;
        sgt[j] = 1;
    }
    {
        int k = 0;
        for (int64_t j = 0; j < nw; ++j) if (sgt[j] > 0) pos[k++] = (int)j;
        for (int64_t j = 0; j < nw; ++j) if (sgt[j] < 0) pos[k++] = (int)j;
    }
    if (sort) {
        for (int64_t j = 0; j < nw; ++j) d[j] = dot(mw, Gt + j * mw, Gt + j * mw);
        sort_positions((int)nw, pos, d, sgt);
    }
    for (int64_t k = 0; k < nw; ++k) {
        memcpy(Gw + k * mw, Gt + (int64_t)pos[k] * mw, sizeof(double) * (size_t)mw);
        sgn[k] = sgt[pos[k]];
        col[k] = pos[k];
        W[(int64_t)pos[k] + k * nw] = 1.0; /* W holds V's columns for the working order */
    }

    int status = ORC_NOT_CONVERGED, sw, rule = ORC_STOP_NONE;
    int64_t nrot_total = 0;
    for (sw = 1; sw <= max_sweeps; ++sw) {
        int64_t nrot = 0;
        int cd = 0; /* Eq. 4.2 over the sweep: the inner tangents */
        for (int s = 0; s < nb; ++s) {
            for (int k = 0; k < nb / 2; ++k) {
                int a = pairs[(s * (nb / 2) + k) * 2], bb = pairs[(s * (nb / 2) + k) * 2 + 1];
                int I = a < bb ? a : bb, Jb = a < bb ? bb : a;
                int cidx[2] = {I * b, Jb * b};
                /* A_P = G_P^T G_P (plain triple loop) */
                for (int y = 0; y < nn; ++y) {
                    const double *gy = Gw + (int64_t)(cidx[y / b] + y % b) * mw;
                    ps[y] = sgn[cidx[y / b] + y % b];
                    for (int x = 0; x < nn; ++x) {
                        const double *gx = Gw + (int64_t)(cidx[x / b] + x % b) * mw;
                        A[x + y * nn] = dot(mw, gx, gy);
                    }
                }
                int mode = (inner_mode == 0) ? 0 : (s == 0 ? 2 : 1);
                int64_t nr = 0;
                double tmax = 0.0;
                int st = orc_inner_solve(nn, A, ps, tol, mode, inner_order, inner_max_passes, Wp, &nr, NULL, &tmax);
                if (st != ORC_OK) { status = st; goto done; }
                if (nr == 0) continue;
                nrot += nr;
                cd |= conv_code(tmax, tstop); /* the block's largest tangent decides its code */
                /* [G_I G_J] <- [G_I G_J] W_P and [V_I V_J] <- [V_I V_J] W_P */
                for (int which = 0; which < 2; ++which) {
                    double *M = which ? W : Gw;
                    int64_t rows = which ? nw : mw;
                    for (int y = 0; y < nn; ++y)
                        for (int64_t i = 0; i < rows; ++i) {
                            double acc = 0.0;
                            for (int x = 0; x < nn; ++x)
                                acc += M[i + (int64_t)(cidx[x / b] + x % b) * rows] * Wp[x + y * nn];
                            Pan[i + (int64_t)y * rows] = acc;
                        }
                    for (int y = 0; y < nn; ++y)
                        memcpy(M + (int64_t)(cidx[y / b] + y % b) * rows, Pan + (int64_t)y * rows,
                               sizeof(double) * (size_t)rows);
                }
            }
        }
        nrot_total += nrot;
        if (cd == 0 || cd == 1) { /* (00)_2 or (01)_2 of Eq. 4.2 */
            status = ORC_OK;
            rule = cd == 0 ? ORC_STOP_ORTHO : ORC_STOP_TANGENT;
            break;
        }
        if (sort) {
            for (int64_t k = 0; k < nw; ++k) { d[k] = dot(mw, Gw + k * mw, Gw + k * mw); pos[k] = (int)k; }
            sort_positions((int)nw, pos, d, sgn);
            memcpy(Gt, Gw, sizeof(double) * (size_t)(mw * nw));
            memcpy(Wt, W, sizeof(double) * (size_t)(nw * nw));
            memcpy(sgt, sgn, (size_t)nw);
            memcpy(colt, col, sizeof(int) * (size_t)nw);
            for (int64_t k = 0; k < nw; ++k) {
                memcpy(Gw + k * mw, Gt + (int64_t)pos[k] * mw, sizeof(double) * (size_t)mw);
                memcpy(W + k * nw, Wt + (int64_t)pos[k] * nw, sizeof(double) * (size_t)nw);
                sgn[k] = sgt[pos[k]];
                col[k] = colt[pos[k]];
            }
        }
    }
    if (sw > max_sweeps) sw = max_sweeps;
    if (!all_finite(mw, nw, Gw, mw)) status = ORC_NONFINITE;
done:
    if (status == ORC_OK || status == ORC_NOT_CONVERGED) {
        /* back to input order; drop the bordering */
        double *Gc = (double *)malloc(sizeof(double) * (size_t)(m * n));
        double *Wc = (double *)malloc(sizeof(double) * (size_t)(n * n));
        for (int64_t k = 0; k < nw; ++k) {
            int j = col[k];
            if (j >= n) continue;
            for (int64_t i = 0; i < m; ++i) Gc[i + (int64_t)j * m] = Gw[i + k * mw];
            for (int64_t i = 0; i < n; ++i) Wc[i + (int64_t)j * n] = W[i + k * nw];
        }
        finalise(m, n, Gc, Wc, sigma, U, ldu, V, ldv);
        for (int64_t j = 0; j < n; ++j)
            if (!(sigma[j] > 0.0)) status = ORC_RANK;
        free(Gc);
        free(Wc);
    }
    if (sweeps) *sweeps = sw;
    if (rotations) *rotations = nrot_total;
    if (stop_rule && status == ORC_OK) *stop_rule = rule;
    free(Gw); free(W); free(Gt); free(Wt); free(sgn); free(sgt); free(col); free(colt);
    free(pos); free(d); free(A); free(Wp); free(Pan); free(ps); free(pairs);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Symmetric indefinite factorisation (Sec. 1: M given explicitly is first    */
/* factored as M = G J G^T).  Complete pivoting after Bunch and Parlett: with */
/* alpha = (1 + sqrt 17) / 8, mu0 = max |a_ij| and mu1 = max |a_ii| over the  */
/* trailing matrix, a 1 x 1 pivot on the largest diagonal entry when          */
/* mu1 >= alpha mu0, else a 2 x 2 pivot on the rows and columns of the        */
/* largest off-diagonal entry (ties: the smallest indices, column first).     */
/* The pivot is swapped to position k (rows and columns of the trailing       */
/* matrix, rows of the finished L); with W the pivot column(s) and D the      */
/* block, L = W D^-1 and the trailing matrix loses L D L^T = W D^-1 W^T.      */
/* G = P L B: B = sqrt|d| on a 1 x 1 block, Q sqrt|Lambda| on a 2 x 2 block    */
/* D = Q Lambda Q^T (a Jacobi rotation with the smaller angle), J = the signs. */
/* The whole symmetric matrix is kept; every product is an explicit fma.      */
/* R16 (postprocessing of a singular M): when the whole trailing matrix is   */
/* zero after r steps, M = G J G^T holds with the first r columns of G (full */
/* column rank) and r signs; the columns and signs past r are returned as     */
/* zeros and *rank_out (may be NULL) = r.  Returns ORC_OK, ORC_RANK (a non-   */
/* finite entry) or ORC_ARG.  perm (may be NULL) receives the original index */
/* held at each position.                                                    */
/* ------------------------------------------------------------------------ */
static void orc_sym_swap(int n, double *A, int k, int a, int b)
{
    if (a == b) return;
    for (int j = 0; j < n; ++j) { /* rows a, b in every column but a and b */
        if (j == a || j == b) continue;
        double t = A[a + (int64_t)j * n];
        A[a + (int64_t)j * n] = A[b + (int64_t)j * n];
        A[b + (int64_t)j * n] = t;
    }
    for (int i = k; i < n; ++i) { /* columns a, b in the trailing rows but a and b */
        if (i == a || i == b) continue;
        double t = A[i + (int64_t)a * n];
        A[i + (int64_t)a * n] = A[i + (int64_t)b * n];
        A[i + (int64_t)b * n] = t;
    }
    double t = A[a + (int64_t)a * n];
    A[a + (int64_t)a * n] = A[b + (int64_t)b * n];
    A[b + (int64_t)b * n] = t;
}

int orc_sym_factor(int64_t n64, const double *M, int64_t ldm, double *G, int64_t ldg, int8_t *J, int *perm_out,
                   int *rank_out)
{
    if (n64 < 1 || ldm < n64 || ldg < n64 || n64 > (1 << 20)) return ORC_ARG;
    if (!all_finite(n64, n64, M, ldm)) return ORC_RANK;
    const int n = (int)n64;
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *D = (double *)calloc((size_t)4 * n, sizeof(double));
    int *perm = (int *)malloc(sizeof(int) * (size_t)n);
    int8_t *bs = (int8_t *)malloc((size_t)n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) A[i + (int64_t)j * n] = M[i + (int64_t)j * ldm];
    for (int i = 0; i < n; ++i) { perm[i] = i; bs[i] = 1; }
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;
    int status = ORC_OK;
    int k = 0;
    while (k < n) {
        /* the largest |diagonal| and |off-diagonal| entries of the trailing matrix */
        double dmax = -1.0, omax = -1.0;
        int di = -1, r = -1, q = -1;
        for (int j = k; j < n; ++j) {
            const double ad = fabs(A[j + (int64_t)j * n]);
            if (ad > dmax) { dmax = ad; di = j; }
            for (int i = j + 1; i < n; ++i) {
                const double ao = fabs(A[i + (int64_t)j * n]);
                if (ao > omax) { omax = ao; r = j; q = i; }
            }
        }
        const double mu0 = dmax > omax ? dmax : omax;
        if (mu0 == 0.0) break; /* R16: the trailing matrix is zero, M has rank k */
        int s;
        if (k == n - 1 || omax <= 0.0 || dmax >= alpha * mu0) {
            s = 1;
            if (di < 0) { status = ORC_RANK; break; } /* NaN everywhere */
            orc_sym_swap(n, A, k, k, di);
            int t = perm[k]; perm[k] = perm[di]; perm[di] = t;
        } else {
            s = 2;
            orc_sym_swap(n, A, k, k, r); /* r < q, so q stays where it is */
            int t = perm[k]; perm[k] = perm[r]; perm[r] = t;
            orc_sym_swap(n, A, k, k + 1, q);
            t = perm[k + 1]; perm[k + 1] = perm[q]; perm[q] = t;
        }
        double *wk = A + (int64_t)k * n, *wk1 = A + (int64_t)(k + 1) * n;
        double i00, i01 = 0.0, i11 = 0.0;
        if (s == 1) {
            const double d = wk[k];
            D[4 * k] = d;
            bs[k] = 1;
            if (d == 0.0) { status = ORC_RANK; break; }
            i00 = 1.0 / d;
        } else {
            const double d00 = wk[k], d01 = wk[k + 1], d11 = wk1[k + 1];
            D[4 * k] = d00; D[4 * k + 1] = d01; D[4 * k + 2] = d01; D[4 * k + 3] = d11;
            bs[k] = 2;
            bs[k + 1] = 0;
            const double det = fma(d00, d11, -d01 * d01);
            if (det == 0.0) { status = ORC_RANK; break; }
            i00 = d11 / det;
            i01 = -d01 / det;
            i11 = d00 / det;
        }
        /* trailing matrix minus W D^-1 W^T, then the pivot columns become L */
        for (int j = k + s; j < n; ++j)
            for (int i = k + s; i < n; ++i) {
                double v;
                if (s == 1) {
                    const double li = wk[i] * i00;
                    v = fma(-li, wk[j], A[i + (int64_t)j * n]);
                } else {
                    const double li0 = fma(wk[i], i00, wk1[i] * i01), li1 = fma(wk[i], i01, wk1[i] * i11);
                    v = fma(-li0, wk[j], fma(-li1, wk1[j], A[i + (int64_t)j * n]));
                }
                A[i + (int64_t)j * n] = v;
            }
        for (int i = k + s; i < n; ++i) {
            if (s == 1) {
                wk[i] = wk[i] * i00;
            } else {
                const double w0 = wk[i], w1 = wk1[i];
                wk[i] = fma(w0, i00, w1 * i01);
                wk1[i] = fma(w0, i01, w1 * i11);
            }
        }
        k += s;
    }
    const int rank = k < n ? k : n;
    if (status == ORC_OK) {
        for (int j = 0; j < n; ++j) {
            if (j >= rank) { /* past the rank: no column, no sign */
                for (int i = 0; i < n; ++i) G[i + (int64_t)j * ldg] = 0.0;
                J[j] = 0;
                continue;
            }
            const int b0 = bs[j] == 0 ? j - 1 : j, size = bs[b0];
            double c0, c1, sgn;
            if (size == 1) {
                const double d = D[4 * b0];
                c0 = sqrt(fabs(d));
                c1 = 0.0;
                sgn = d > 0.0 ? 1.0 : -1.0;
            } else {
                const double a = D[4 * b0], b = D[4 * b0 + 1], c = D[4 * b0 + 3];
                double t = 0.0;
                if (b != 0.0) {
                    const double zeta = (c - a) / (2.0 * b);
                    t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
                }
                const double cs = 1.0 / sqrt(fma(t, t, 1.0)), sn = t * cs;
                const double l1 = fma(-t, b, a), l2 = fma(t, b, c);
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
            for (int i = 0; i < n; ++i) {
                double l0 = 0.0, l1v = 0.0;
                if (i == b0) l0 = 1.0;
                else if (i > b0 + (size - 1)) l0 = A[i + (int64_t)b0 * n];
                if (size == 2) {
                    if (i == b0 + 1) l1v = 1.0;
                    else if (i > b0 + 1) l1v = A[i + (int64_t)(b0 + 1) * n];
                }
                G[perm[i] + (int64_t)j * ldg] = fma(c0, l0, c1 * l1v);
            }
            J[j] = sgn > 0.0 ? 1 : -1;
        }
        if (perm_out)
            for (int i = 0; i < n; ++i) perm_out[i] = perm[i];
        if (rank_out) *rank_out = rank;
    }
    free(A); free(D); free(perm); free(bs);
    return status;
}

/* ------------------------------------------------------------------------ */
/* orc_hyp_qr -- hyperbolic QR of a tall A (n x m, n >= m) with signature J  */
/* (Sec. 1: a factor G whose transpose is tall is shortened by the           */
/* hyperbolic QR of G^T; the HSVD then runs on the square R^T).  Reading    */
/* R15: J-orthogonal Householder reflectors H = I - beta v v^T S with S the */
/* current signature, pivots chosen on the trailing J-Gram C = X^T S X (X   */
/* the trailing rows k..n-1 of the remaining columns) by the Bunch-Parlett   */
/* rule, alpha = (1 + sqrt 17) / 8:                                          */
/*   1 x 1 (the largest |C_jj| >= alpha times the largest |C_ij|, i != j):  */
/*     that column moves to position k and is reduced to R_kk e_k;          */
/*   2 x 2 otherwise: the columns x, y of the largest |C_ij| move to k, k+1; */
/*     z = x + tau y (tau = +-1 so that |z^T S z| = |C_xx + C_yy| + 2|C_xy|) */
/*     is reduced at row k, then y's rows k+1.. at row k+1, each reflector  */
/*     applied to every remaining column, x included; R gets a full 2 x 2   */
/*     diagonal block.                                                       */
/* A reduction of a vector z at row k: if S_k is not sign(gamma), gamma =   */
/* z^T S z over rows k.., row k is interchanged with the row i > k of that   */
/* sign with the largest |z_i| (ties: smallest i); then alpha = -sign(z_k)  */
/* sqrt|gamma| (the J-norm is kept: alpha^2 S_k = gamma), v = z - alpha e_k, */
/* v^T S v = 2 S_k sqrt|gamma| (sqrt|gamma| + |z_k|), beta = 2 / v^T S v.   */
/* With T = H_{m-1} P_{m-1} ... H_0 P_0 (P_k the row interchanges) and C   */
/* the column permutation:  T A C = [R; 0],  T^T Jh T = J  (Jh = J after   */
/* the interchanges), so A C = Q [R; 0] with Q = T^-1 and Q^T J Q = Jh,   */
/* and C^T (A^T J A) C = R^T Jh_1 R with Jh_1 the first m entries of Jh.   */
/* A zero trailing J-Gram (A^T J A singular) returns ORC_RANK.  With J = I  */
/* every pivot is 1 x 1 and this is Householder QR with column pivoting.    */
/* Outputs: R (m x m, ldr; block upper triangular), Jh (n signs), cperm (m: */
/* the original column at each position), and, each may be NULL, the       */
/* reflectors V (n x m, ldv; v_k in rows k..n-1 of column k in the row      */
/* order of step k, zero above), beta (m), rswap (m: the row interchanged    */
/* with row k at step k) and bsize (m: 1 for a 1 x 1 pivot, 2 and 0 for the  */
/* two positions of a 2 x 2 pivot).                                          */
/* ------------------------------------------------------------------------ */
static double hq_sdot(int n, int k, const int8_t *s, const double *x, const double *y)
{
    double acc = 0.0;
    for (int i = k; i < n; ++i) acc += s[i] > 0 ? x[i] * y[i] : -(x[i] * y[i]);
    return acc;
}

static void hq_swap_cols(int n, double *W, int a, int b)
{
    if (a == b) return;
    for (int i = 0; i < n; ++i) {
        const double t = W[i + (int64_t)a * n];
        W[i + (int64_t)a * n] = W[i + (int64_t)b * n];
        W[i + (int64_t)b * n] = t;
    }
}

/* reduce z (rows k..n-1, a work vector) at row k: the row interchange, then */
/* the reflector applied to the columns c0..m-1 of W                         */
static int hq_reduce(int n, int m, double *W, int8_t *s, double *z, int k, int c0, double *v,
                     double *alpha_out, double *beta_out, int *rswap_out)
{
    const double gamma = hq_sdot(n, k, s, z, z);
    if (!(gamma != 0.0)) return ORC_RANK;
    const int8_t sg = gamma > 0.0 ? 1 : -1;
    int ip = k;
    if (s[k] != sg) {
        double xbest = -1.0;
        for (int i = k + 1; i < n; ++i)
            if (s[i] == sg && fabs(z[i]) > xbest) { xbest = fabs(z[i]); ip = i; }
        if (ip == k) return ORC_RANK; /* cannot happen for gamma != 0 */
        for (int j = 0; j < m; ++j) {
            const double t = W[k + (int64_t)j * n];
            W[k + (int64_t)j * n] = W[ip + (int64_t)j * n];
            W[ip + (int64_t)j * n] = t;
        }
        const double tz = z[k]; z[k] = z[ip]; z[ip] = tz;
        const int8_t t = s[k]; s[k] = s[ip]; s[ip] = t;
    }
    *rswap_out = ip;
    const double root = sqrt(fabs(gamma));
    const double alpha = z[k] >= 0.0 ? -root : root;
    for (int i = 0; i < n; ++i) v[i] = i < k ? 0.0 : z[i];
    v[k] = z[k] - alpha;
    const double vsv = 2.0 * (double)s[k] * root * (root + fabs(z[k]));
    const double beta = 2.0 / vsv;
    for (int j = c0; j < m; ++j) {
        double *y = W + (int64_t)j * n;
        double vsy = 0.0;
        for (int i = k; i < n; ++i) vsy += s[i] > 0 ? v[i] * y[i] : -(v[i] * y[i]);
        const double f = beta * vsy;
        for (int i = k; i < n; ++i) y[i] -= f * v[i];
    }
    *alpha_out = alpha;
    *beta_out = beta;
    return ORC_OK;
}

int orc_hyp_qr(int64_t n64, int64_t m64, const double *A, int64_t lda, const int8_t *J, double *R, int64_t ldr,
               int8_t *Jh, int *cperm, double *Vr, int64_t ldv, double *beta_out, int *rswap_out, int *bsize_out)
{
    if (m64 < 1 || n64 < m64 || lda < n64 || ldr < m64 || n64 > (1 << 24)) return ORC_ARG;
    if (Vr && ldv < n64) return ORC_ARG;
    const int n = (int)n64, m = (int)m64;
    for (int i = 0; i < n; ++i)
        if (J[i] != 1 && J[i] != -1) return ORC_ARG;
    if (!all_finite(n, m, A, lda)) return ORC_NONFINITE;
    double *W = (double *)malloc(sizeof(double) * (size_t)n * m);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *bt = (double *)malloc(sizeof(double) * (size_t)m);
    int8_t *s = (int8_t *)malloc((size_t)n);
    int *cp = (int *)malloc(sizeof(int) * (size_t)m);
    int *rs = (int *)malloc(sizeof(int) * (size_t)m);
    int *bs = (int *)malloc(sizeof(int) * (size_t)m);
    for (int j = 0; j < m; ++j) {
        cp[j] = j;
        for (int i = 0; i < n; ++i) W[i + (int64_t)j * n] = A[i + (int64_t)j * lda];
    }
    for (int i = 0; i < n; ++i) s[i] = J[i];
    if (Vr)
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < n; ++i) Vr[i + (int64_t)j * ldv] = 0.0;
    const double alpha_bp = (1.0 + sqrt(17.0)) / 8.0;
    int status = ORC_OK;
    int k = 0;
    while (k < m && status == ORC_OK) {
        /* the trailing J-Gram: largest |diagonal| and |off-diagonal| entries */
        int jp = -1, pr = -1, pq = -1;
        double gbest = -1.0, obest = -1.0;
        for (int j = k; j < m; ++j) {
            const double *xj = W + (int64_t)j * n;
            const double g = hq_sdot(n, k, s, xj, xj);
            if (fabs(g) > gbest) { gbest = fabs(g); jp = j; }
            for (int i = k; i < j; ++i) {
                const double o = fabs(hq_sdot(n, k, s, W + (int64_t)i * n, xj));
                if (o > obest) { obest = o; pr = i; pq = j; }
            }
        }
        double alpha = 0.0, beta = 0.0;
        int ip = k;
        if (k == m - 1 || !(obest > 0.0) || gbest >= alpha_bp * obest) {
            if (!(gbest > 0.0)) { status = ORC_RANK; break; }
            hq_swap_cols(n, W, k, jp);
            { const int t = cp[k]; cp[k] = cp[jp]; cp[jp] = t; }
            double *x = W + (int64_t)k * n;
            for (int i = 0; i < n; ++i) z[i] = i < k ? 0.0 : x[i];
            status = hq_reduce(n, m, W, s, z, k, k, v, &alpha, &beta, &ip);
            if (status != ORC_OK) break;
            x[k] = alpha;
            for (int i = k + 1; i < n; ++i) x[i] = 0.0;
            bt[k] = beta; rs[k] = ip; bs[k] = 1;
            if (Vr)
                for (int i = k; i < n; ++i) Vr[i + (int64_t)k * ldv] = v[i];
            k += 1;
        } else {
            /* columns pr < pq to positions k, k + 1 */
            hq_swap_cols(n, W, k, pr);
            { const int t = cp[k]; cp[k] = cp[pr]; cp[pr] = t; }
            const int q2 = pq == k ? pr : pq;
            hq_swap_cols(n, W, k + 1, q2);
            { const int t = cp[k + 1]; cp[k + 1] = cp[q2]; cp[q2] = t; }
            double *x = W + (int64_t)k * n, *y = W + (int64_t)(k + 1) * n;
            const double gx = hq_sdot(n, k, s, x, x), gy = hq_sdot(n, k, s, y, y), d = hq_sdot(n, k, s, x, y);
            const double tau = ((gx + gy >= 0.0) == (d >= 0.0)) ? 1.0 : -1.0;
            for (int i = 0; i < n; ++i) z[i] = i < k ? 0.0 : x[i] + tau * y[i];
            status = hq_reduce(n, m, W, s, z, k, k, v, &alpha, &beta, &ip);
            if (status != ORC_OK) break;
            bt[k] = beta; rs[k] = ip; bs[k] = 2;
            if (Vr)
                for (int i = k; i < n; ++i) Vr[i + (int64_t)k * ldv] = v[i];
            for (int i = 0; i < n; ++i) z[i] = i <= k ? 0.0 : y[i];
            double alpha2 = 0.0;
            status = hq_reduce(n, m, W, s, z, k + 1, k, v, &alpha2, &beta, &ip);
            if (status != ORC_OK) break;
            bt[k + 1] = beta; rs[k + 1] = ip; bs[k + 1] = 0;
            if (Vr)
                for (int i = k + 1; i < n; ++i) Vr[i + (int64_t)(k + 1) * ldv] = v[i];
            y[k + 1] = alpha2;
            for (int i = k + 2; i < n; ++i) { x[i] = 0.0; y[i] = 0.0; }
            k += 2;
        }
    }
    if (status == ORC_OK) {
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i)
                R[i + (int64_t)j * ldr] = (i <= j || (i == j + 1 && bs[j] == 2)) ? W[i + (int64_t)j * n] : 0.0;
        for (int i = 0; i < n; ++i) Jh[i] = s[i];
        for (int j = 0; j < m; ++j) cperm[j] = cp[j];
        for (int j = 0; j < m; ++j) {
            if (beta_out) beta_out[j] = bt[j];
            if (rswap_out) rswap_out[j] = rs[j];
            if (bsize_out) bsize_out[j] = bs[j];
        }
    }
    free(W); free(v); free(z); free(bt); free(s); free(cp); free(rs); free(bs);
    return status;
}

/* X (n x c, ldx) <- T^T X with T = H_{m-1} P_{m-1} ... H_0 P_0 from           */
/* orc_hyp_qr: T^T = P_0 H_0^T P_1 H_1^T ... P_{m-1} H_{m-1}^T, applied right */
/* to left.  H_k^T = I - beta_k S_k v_k v_k^T, where S_k, the signature at    */
/* step k, is recovered from the final Jh by undoing the later interchanges. */
/* With X = [V_F; 0], V_F the HSVD right factor of the square F = C R^T,     */
/* the result V satisfies G V = U Sigma and V^T J V = Jh_1 for G = A^T.       */
int orc_hyp_qr_apply_tt(int64_t n64, int64_t m64, const double *Vr, int64_t ldv, const double *beta,
                        const int *rswap, const int8_t *Jh, double *X, int64_t ldx, int64_t c64)
{
    if (m64 < 1 || n64 < m64 || ldv < n64 || ldx < n64 || c64 < 0) return ORC_ARG;
    const int n = (int)n64, m = (int)m64, c = (int)c64;
    int8_t *s = (int8_t *)malloc((size_t)n);
    for (int i = 0; i < n; ++i) s[i] = Jh[i];
    for (int k = m - 1; k >= 0; --k) {
        const double *v = Vr + (int64_t)k * ldv;
        for (int j = 0; j < c; ++j) {
            double *y = X + (int64_t)j * ldx;
            double vy = 0.0;
            for (int i = k; i < n; ++i) vy += v[i] * y[i];
            const double f = beta[k] * vy;
            for (int i = k; i < n; ++i) y[i] -= s[i] > 0 ? f * v[i] : -(f * v[i]);
        }
        const int ip = rswap[k];
        if (ip != k) {
            for (int j = 0; j < c; ++j) {
                double *y = X + (int64_t)j * ldx;
                const double t = y[k]; y[k] = y[ip]; y[ip] = t;
            }
            const int8_t t = s[k]; s[k] = s[ip]; s[ip] = t;
        }
    }
    free(s);
    return ORC_OK;
}

/* HSVD of a wide factor G (m x n, m < n is the case it is for; m <= n) with   */
/* signature J (n), through the hyperbolic QR of A = G^T (Sec. 1):           */
/*   A C = Q [R; 0]  gives  G J G^T = F Jh_1 F^T  with F = C R^T (m x m),    */
/*   F V_F = U Sigma (orc_hsvd, row-cyclic or modulus order),                 */
/*   V = T^T [V_F; 0]  (n x m):  G V = U Sigma,  V^T J V = Jh_1.               */
/* sigma, U (m x m) and Jout (m signs, lambda_j = sigma_j^2 Jout_j) follow    */
/* F's columns; V may be NULL.                                                 */
int orc_wide_hsvd(int64_t m64, int64_t n64, const double *G, int64_t ldg, const int8_t *J, double tol,
                  int max_sweeps, int order, double *sigma, double *U, int64_t ldu, double *V, int64_t ldv,
                  int8_t *Jout, int *sweeps)
{
    if (m64 < 1 || n64 < m64 || ldg < m64 || n64 > (1 << 24)) return ORC_ARG;
    if ((U && ldu < m64) || (V && ldv < n64)) return ORC_ARG;
    const int m = (int)m64, n = (int)n64;
    double *A = (double *)calloc((size_t)n * m, sizeof(double));
    double *R = (double *)malloc(sizeof(double) * (size_t)m * m);
    double *F = (double *)malloc(sizeof(double) * (size_t)m * m);
    double *VF = (double *)malloc(sizeof(double) * (size_t)m * m);
    double *Vr = (double *)malloc(sizeof(double) * (size_t)n * m);
    double *beta = (double *)malloc(sizeof(double) * (size_t)m);
    int *rswap = (int *)malloc(sizeof(int) * (size_t)m);
    int *cperm = (int *)malloc(sizeof(int) * (size_t)m);
    int8_t *Jh = (int8_t *)malloc((size_t)n);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) A[j + (int64_t)i * n] = G[i + (int64_t)j * ldg];
    int status = orc_hyp_qr(n, m, A, n, J, R, m, Jh, cperm, Vr, n, beta, rswap, NULL);
    if (status == ORC_OK) {
        for (int j = 0; j < m; ++j)
            for (int l = 0; l < m; ++l) F[cperm[j] + (int64_t)l * m] = R[l + (int64_t)j * m];
        int64_t rots = 0;
        status = orc_hsvd(m, m, F, m, Jh, tol, max_sweeps, order, 0, sigma, U, ldu, VF, m, sweeps, &rots, 0.0, NULL);
    }
    if (status == ORC_OK || status == ORC_NOT_CONVERGED) {
        for (int i = 0; i < m; ++i) Jout[i] = Jh[i];
        if (V) {
            for (int j = 0; j < m; ++j)
                for (int i = 0; i < n; ++i) V[i + (int64_t)j * ldv] = i < m ? VF[i + (int64_t)j * m] : 0.0;
            orc_hyp_qr_apply_tt(n, m, Vr, n, beta, rswap, Jh, V, ldv, m);
        }
    }
    free(A); free(R); free(F); free(VF); free(Vr); free(beta); free(rswap); free(cperm); free(Jh);
    return status;
}
