/*
 * hsvd.h -- C ABI of the GB300 (sm_103a) one-sided Jacobi hyperbolic SVD.
 *
 * Problem (Sec. 1, Eq. 1.1): for a real m x n factor G, m >= n, of full column
 * rank and a signature J = diag(+-1), compute
 *
 *     G V = U Sigma,   U^T U = I,   V^T J V = J,   Sigma = diag(sigma) > 0,
 *
 * so that M = G J G^T = U (Sigma^2 J) U^T (Sec. 1): lambda_j = sigma_j^2 J_jj.
 * V is the accumulated product of the J-unitary rotations applied to G's
 * columns (Eq. 2.1, the paper's V^{-T}); the paper's right hyperbolic singular
 * vectors are J V J (Sec. 2).
 *
 * Conventions shared by every entry point:
 *  - Matrices are column-major FP64 with a leading dimension >= rows.
 *  - Outputs are in INPUT column order: sigma[j], U(:,j), V(:,j) belong to the
 *    column that started as G(:,j), and keep its sign J[j] (the paper also
 *    returns results in the original column order, Sec. 4).  Sort them if you
 *    need lambda in order.
 *  - Memory: for hsvd_solve / hsvd_solve_ex / hsvd_solve_batched every array
 *    argument is either a device pointer (cudaMalloc / PyTorch CUDA memory of
 *    the current device) or a host pointer (pageable or pinned); all arrays of
 *    one call must be of the same kind.  With host arrays the library copies
 *    the inputs in and the results out on `stream` and returns after the copy
 *    back.  The caller owns every array; the library allocates only its own
 *    workspace (stream-ordered, released before return) and never keeps a
 *    pointer after return.  G is read-only.  A call that mixes the kinds
 *    returns HSVD_ERR_ARG.  Every other entry point takes device arrays only
 *    and returns HSVD_ERR_ARG, before any allocation or launch, when one of
 *    its arrays is host memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  With
 *    device arrays the call still synchronises `stream` once per sweep to read
 *    the convergence flag, and before returning.
 *  - Return value: one of the HSVD_* status codes below.  No exception or
 *    abort crosses the ABI.  Outputs are written for HSVD_OK and
 *    HSVD_NOT_CONVERGED only.
 */
#ifndef HSVD_H
#define HSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define HSVD_OK 0
#define HSVD_NOT_CONVERGED 1   /* max_sweeps reached; outputs hold the last iterate   */
#define HSVD_ERR_ARG (-1)      /* bad size, leading dimension, signature or option      */
#define HSVD_ERR_RANK (-2)     /* a hyperbolic pair with |zeta| <= 1, or a zero column:
                                  G (or G J G^T) is numerically rank deficient, Sec. 1 */
#define HSVD_ERR_NONFINITE (-3) /* NaN or Inf in G or produced during the sweep         */
#define HSVD_ERR_CUDA (-4)     /* a CUDA runtime call failed                            */
#define HSVD_ERR_NOMEM (-5)    /* workspace allocation failed                           */

/* Methods. */
#define HSVD_METHOD_AUTO 0      /* pointwise for n < 32 (measured faster only there),
                                   else blocked                                        */
#define HSVD_METHOD_POINTWISE 1 /* column-pair rotations (Alg. 4.5), one CTA per factor */
#define HSVD_METHOD_BLOCKED 2   /* block-column pairs (Sec. 5 block-oriented method)    */

/* Inner pivot-block solve of the blocked method. */
#define HSVD_INNER_ORIENTED 0 /* Sec. 5: whole block in the first step of a sweep,
                                 then one pass over the off-diagonal block only */
#define HSVD_INNER_FULL 1     /* Sec. 6: diagonalise the pivot block (passes until
                                 no inner rotation, at most inner_max_passes) */

#define HSVD_SORT_AUTO (-1)

/* Schedule of a sweep of the blocked method.  Either way a sweep is one CUDA
 * graph and every visit does the same arithmetic, so the results are the same
 * bit for bit. */
#define HSVD_SCHEDULE_AUTO 0  /* pairs, or steps with opts.profile                 */
#define HSVD_SCHEDULE_STEPS 1 /* the steps of the pivot strategy one after the other:
                                 Gram of all pairs, inner solves, updates            */
#define HSVD_SCHEDULE_PAIRS 2 /* every block-pair visit on its own: its Gram waits
                                 only for the updates that last wrote its two block
                                 columns, so one visit's latency-bound inner solve
                                 overlaps other visits' Gram and update work        */

/* Stopping (Sec. 2).  The iteration always stops after a sweep in which every
 * pair passed the test of Eq. 2.3 (no rotation).  With opts.tstop != 0 it also
 * stops after a sweep whose applied rotations all had |t| <= T (the
 * convergence statistic of Eq. 4.2 reduced to (01)_2): quadratic convergence
 * has set in and the confirming sweep is saved.  For the blocked method the
 * tangents are those of the inner (pivot-block) rotations.  HSVD_TSTOP_PAPER
 * is the paper's T_eps = sqrt(eps)/2 with eps = 2^-52; a negative tstop
 * selects it. */
#define HSVD_TSTOP_PAPER 7.450580596923828125e-9 /* 2^-27 */

/* Shortening (Sec. 1) of a tall factor: G = Q R by Householder reflections,
 * the HSVD of the square R, U = Q [U_R; 0]; V and Sigma are R's.  One sweep
 * then costs 12 n^3 flops instead of 2 n^2 (4m + 2n). */
#define HSVD_SHORTEN_AUTO 0   /* when 4m >= 5n                                     */
#define HSVD_SHORTEN_NEVER 1
#define HSVD_SHORTEN_ALWAYS 2 /* whenever m > n                                    */

#define HSVD_STOP_NONE 0    /* not converged, or an error                      */
#define HSVD_STOP_ORTHO 1   /* a sweep without rotations (every pair passed)   */
#define HSVD_STOP_TANGENT 2 /* a sweep whose tangents were all <= T            */

/* Learned form: per-visit features and the MLP 8 -> 64 -> 64 -> 1 (ReLU, ReLU,
 * logit).  Parameter vector (FP32 master values; weights are rounded to BF16
 * where the network runs, accumulation is FP32): W1[64][8], b1[64],
 * W2[64][64], b2[64], w3[64], b3. */
#define HSVD_MLP_FEATURES 8
#define HSVD_MLP_PARAMS 4801
#define HSVD_TRACE_FIELDS 8

/* Arithmetic of the blocked method's Gram and update products. */
#define HSVD_PRECISION_FP64 0   /* FP64 FMA                                             */
#define HSVD_PRECISION_BF16X8 1 /* split precision: each FP64 operand as 8 BF16 slices
                                   (balanced 7-bit digits), the 36 leading slice
                                   products on the tensor cores with exact FP32
                                   accumulation, recombined exactly into FP64; rotation
                                   angles, the test of Eq. 2.3 and the norms stay FP64.
                                   Requires block_w = 64 (0 selects it).             */

typedef struct hsvd_opts {
    double tol;           /* relative orthogonality threshold of Eq. 2.3;
                             <= 0 selects n * 2^-53                                   */
    int max_sweeps;       /* <= 0 selects 30                                           */
    int method;           /* HSVD_METHOD_*                                             */
    int block_w;          /* block width b of the blocked method: 16, 32 or 64; 0=auto */
    int inner_mode;       /* HSVD_INNER_*                                              */
    int inner_max_passes; /* cap for HSVD_INNER_FULL; <= 0 selects 8                   */
    int sort;             /* 1: diagonal sorting before the first sweep and after each
                             sweep (Sec. 4): J+ part by ||g||^2 decreasing, J- part
                             increasing; 0: no sorting; HSVD_SORT_AUTO: sorting for the
                             pointwise method and the split-precision form (without
                             skip_model or trace_out), none for FP64 blocked          */
    int profile;          /* nonzero: time every kernel with CUDA events (hsvd_info)   */
    int precision;        /* HSVD_PRECISION_FP64 or HSVD_PRECISION_BF16X8              */
    const float *skip_model; /* learned form (blocked method, sort = 0): HSVD_MLP_PARAMS
                             floats, host or device; NULL = plain sweeps              */
    double skip_tau;      /* learned form: a visit is skipped when the predicted
                             probability that it rotates is below skip_tau; <= 0
                             selects 0.5                                              */
    float *trace_out;     /* blocked method, sort = 0: device array receiving training
                             rows (HSVD_MLP_FEATURES features, then the label 1/0:
                             the visit rotated) for every block-pair visit of every
                             sweep after the first; NULL = none                       */
    int64_t trace_cap;    /* rows available at trace_out                               */
    double tstop;         /* tangent threshold T of the early stop: 0 (default) = off,
                             < 0 = HSVD_TSTOP_PAPER, else T itself (0 < T <= 1)       */
    int schedule;         /* HSVD_SCHEDULE_* (blocked method); with the pair schedule
                             opts.profile reports only the sweep total, in ms_other  */
    int shorten;          /* HSVD_SHORTEN_*                                            */
    int8_t *jout;         /* wide factor (m < n): receives the m signs of the result,
                             lambda_j = sigma_j^2 jout_j (same kind of memory as G);
                             may be NULL; unused for m >= n                           */
    int reserved[2];      /* must be zero                                              */
} hsvd_opts;

typedef struct hsvd_info {
    int sweeps;           /* sweeps run, including the final one without rotations     */
    int method;           /* method actually used                                      */
    int block_w;          /* block width actually used (1 for pointwise)               */
    int status;           /* same as the return value                                  */
    int64_t rotations;    /* rotations applied (inner rotations for the blocked method) */
    int64_t pair_updates; /* blocked method: pivot pairs whose panels were updated     */
    int64_t kernel_launches; /* kernels of this library launched by the call           */
    double ms_gram;       /* with opts.profile: summed CUDA-event time of the Gram      */
    double ms_solve;      /*   kernels, the inner-solve kernels, the update kernels,    */
    double ms_update;     /*   and of everything else (bordering, reordering,           */
    double ms_other;      /*   finalisation; the pointwise kernel counts as "solve")   */
    int64_t pair_visits;  /* blocked method: block-pair visits whose Gram was formed    */
    int masked_sweeps;    /* learned form: sweeps run with a skip mask                  */
    int judge_sweeps;     /* learned form: full sweeps run after a masked sweep without
                             rotations                                                  */
    int64_t trace_rows;   /* rows written to trace_out                                 */
    int stop_rule;        /* HSVD_STOP_*: which rule ended the iteration               */
    int shortened;        /* 1: a tall factor was shortened by a QR first, 2: a wide
                             one by the hyperbolic QR of its transpose              */
    double ms_host_graph; /* blocked method: host wall time spent capturing and
                             instantiating sweep graphs (one per call, plus one per
                             masked sweep of the learned form)                      */
} hsvd_info;

/* Fills *opts with the defaults (tol = n 2^-53 at call time, 30 sweeps, auto
 * method and block width, block-oriented inner solve, HSVD_SORT_AUTO). */
void hsvd_default_opts(hsvd_opts *opts);

/*
 * hsvd_solve -- the HSVD of one factor (Sec. 1, Eq. 1.1) by the one-sided
 * hyperbolic Jacobi method (Sec. 2): sweeps of the modified modulus strategy
 * (Sec. 2) until a sweep in which every pair passes the relative
 * orthogonality test |a_ij| < tol sqrt(a_ii a_jj) (Eq. 2.3, Sec. 2 stopping
 * rule).
 *   G      m x n, leading dimension ldg >= m, m >= n >= 1          (input)
 *   J      n signs, each +1 or -1 (int8)                              (input)
 *   tol    <= 0 selects n * 2^-53; max_sweeps <= 0 selects 30
 *   sigma  n                                                          (output)
 *   U      m x n, ldu >= m, may be NULL                               (output)
 *   V      n x n, ldv >= n, may be NULL                               (output)
 *   sweeps may be NULL; receives the number of sweeps run
 * Sizes up to n = 2^24 and m = 2^31 are accepted (device memory permitting).
 * A wide factor (m < n, m <= 2^24) is shortened first, as Sec. 1 prescribes,
 * by a hyperbolic QR of G^T: T G^T C = [R; 0] with J-orthogonal Householder
 * reflectors and row interchanges (T^T Jh T = J) and Bunch-Parlett column
 * pivoting on the trailing J-Gram; the square F = C R^T (m x m) with the
 * signature Jh_1 (the first m of Jh) satisfies G J G^T = F Jh_1 F^T, and its
 * HSVD F V_F = U Sigma gives V = T^T [V_F; 0].  Then sigma has m entries, U is
 * m x m (ldu >= m), V is n x m (ldv >= n) with G V = U Sigma and
 * V^T J V = Jh_1; the m signs Jh_1 go to hsvd_opts.jout (hsvd_solve_ex), so
 * the eigenvalues of M = G J G^T are sigma_j^2 jout_j.  G J G^T singular
 * returns HSVD_ERR_RANK.
 */
int hsvd_solve(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J,
               double tol, int max_sweeps, double *sigma, double *U, int64_t ldu,
               double *V, int64_t ldv, int *sweeps, void *stream);

/* hsvd_solve with explicit options (opts may be NULL for the defaults) and an
 * optional info record. */
int hsvd_solve_ex(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J,
                  double *sigma, double *U, int64_t ldu, double *V, int64_t ldv,
                  const hsvd_opts *opts, hsvd_info *info, void *stream);

/* Human-readable name of a status code (static string, never NULL). */
const char *hsvd_status_string(int status);

/*
 * Pivot strategy (Sec. 2, Alg. 4.3 / 4.4): the modified modulus strategy on r
 * indices, r even, 2 <= r <= 65536.  Writes nsteps * (r/2) pairs (i, j), i < j,
 * as pairs[2*(s*(r/2)+k) + {0,1}]: step s (0-based, taken modulo r) holds the
 * pairs with i + j = (r - 1 + s) mod r (mod r), plus (c/2, c/2 + r/2) when that
 * residue c is even.  Host memory.  Returns HSVD_ERR_ARG on bad r.
 */
int hsvd_modulus_pairs(int r, int nsteps, int *pairs);

/*
 * The ring that the full pass of the inner solve follows (Sec. 2 modulus
 * order on the 2b columns of a pivot block, Sec. 5 first visit): from one
 * step to the next each pair keeps one row and takes the row leaving the
 * previous pair, so the b pairs form a ring of slots.  Writes 2b steps x b
 * slots x 4 ints (8 b^2 ints), entry [s][k] =
 * {lo, hi, buf_lo | buf_hi << 8, lo_arrived}: the pair (lo < hi) of slot k at
 * step s (as a set, step s's pairs are those of hsvd_modulus_pairs(2b, ...)
 * step s), the row buffers of lo and hi in the pool of the slot's owning CTA
 * (slots split evenly over 4 CTAs at b = 16, 8 otherwise; 2P + 1 buffers for
 * P slots), and 1 if row lo (else row hi) came from slot k - 1 (always 0 at
 * step 0).  Host memory, host computation, no GPU needed.  b in {16, 32, 64};
 * HSVD_ERR_ARG otherwise or for a NULL tab.
 */
int hsvd_ring_table(int b, int *tab);

/*
 * Kernel-level entry points of the blocked method, exposed so each kernel can
 * be checked on its own.  All pointers are device pointers; the call is
 * stream-ordered (no synchronisation); the caller owns all memory.  The pair
 * table col0 lives in device memory and is not read on the host: every block
 * [col0, col0 + b) must lie inside the columns of G (or X), and the two blocks
 * of a pair must not overlap; the Python binding checks this before the call.
 *
 * hsvd_pivot_gram: A_P = [G_I G_J]^T [G_I G_J] for npairs block-column pairs
 * (Sec. 2 pivot block A_P, blocked as in Sec. 5).  G has `rows` rows (a
 * multiple of 64), leading dimension ldg; col0[2k], col0[2k+1] are the first
 * columns of blocks I and J of pair k (device int array).  A receives npairs
 * (2b x 2b) column-major blocks, A + k*(2b)^2.  b in {16, 32, 64}.
 */
int hsvd_pivot_gram(const double *G, int64_t rows, int64_t ldg, int b, int npairs,
                    const int *col0, double *A, void *stream);

/*
 * hsvd_pivot_solve: J-orthogonalise npairs pivot blocks A (each 2b x 2b,
 * overwritten by W^T A W) with signs sgn (npairs x 2b int8, device) by
 * two-sided rotations (Sec. 5 block method; Sec. 6 full-block), writing the
 * transformation W (npairs x (2b)^2) and rotated[k] = number of rotations.
 * mode: 0 passes over all index pairs until none rotates (at most max_passes),
 * 1 one pass over the off-diagonal block only, 2 one pass over all pairs.
 * Returns HSVD_ERR_RANK through *status_dev (device int, may be NULL) when a
 * hyperbolic pair has |zeta| <= 1.
 */
int hsvd_pivot_solve(int b, int npairs, double *A, const int8_t *sgn, double tol, int mode,
                     int max_passes, double *W, int *rotated, int *status_dev, void *stream);

/*
 * hsvd_pivot_update: [X_I X_J] <- [X_I X_J] W_k in place for every pair k with
 * rotated[k] != 0 (Eq. 2.1 applied to a block-column pair).  X has `rows` rows
 * (a multiple of 32), leading dimension ldx.
 */
int hsvd_pivot_update(double *X, int64_t rows, int64_t ldx, int b, int npairs, const int *col0,
                      const double *W, const int *rotated, void *stream);

/*
 * Split-precision kernel-level entry points (HSVD_PRECISION_BF16X8, b = 64),
 * the counterparts of hsvd_pivot_gram and hsvd_pivot_update: same operands,
 * device pointers, stream-ordered, the caller owns the outputs; here `rows` may
 * be any count >= 1.  They allocate
 * their scratch (partials, slices) stream-ordered and free it before return.
 * hsvd_pivot_update_x: dexp (npairs x 128 ints, device, may be NULL for none)
 * are the balancing exponents d_k of X W = (X 2^-d)(2^d W).
 */
int hsvd_pivot_gram_x(const double *G, int64_t rows, int64_t ldg, int npairs, const int *col0, double *A,
                      void *stream);
int hsvd_pivot_update_x(double *X, int64_t rows, int64_t ldx, int npairs, const int *col0, const double *W,
                        const int *rotated, const int *dexp, void *stream);

/*
 * hsvd_solve_pointwise_noalloc -- the pointwise solver (HSVD_METHOD_POINTWISE)
 * without any allocation, for callers that cannot allocate device memory: code
 * running while another allocator owns the device, real-time or certified
 * code that forbids allocation after start-up, memory-capped contexts.  The
 * paper has no counterpart; it is an interface choice of this library.
 *
 * Its scratch (the accumulated transformation W, three status ints -- status,
 * sweeps, stop rule -- and a 64-bit rotation count) is a fixed device array
 * inside the library, sized for n <= HSVD_NOALLOC_MAX_N, that every GPU which
 * loads the library holds until the process exits (about 195 KB).  156 is the
 * largest n whose square factor (m = n) fits one SM's shared memory, which the
 * pointwise kernel needs anyway.
 * The caller passes inputs and outputs as DEVICE pointers with the meanings of
 * hsvd_solve; sort != 0 selects diagonal sorting (Sec. 4).  The call launches
 * on `stream`, then waits for it to read the status; it calls no cudaMalloc,
 * cudaFree or other allocating routine.  n > HSVD_NOALLOC_MAX_N, or a factor
 * whose G does not fit one SM's shared memory (m x n FP64 up to about 200 KB),
 * returns HSVD_ERR_ARG.  The first call on a device (and the first after a
 * cudaDeviceReset) looks up the array's device address (cudaGetSymbolAddress)
 * with that device current: make that first call before any stream capture.
 * Every call on a device shares the one array, so calls that overlap on the GPU
 * (other streams, other host threads) race: issue them one after the other.
 * Nothing has to be cleared between calls: the kernel writes every scratch
 * word before it reads it.
 */
#define HSVD_NOALLOC_MAX_N 156
int hsvd_solve_pointwise_noalloc(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J,
                                 double tol, int max_sweeps, int sort, double *sigma, double *U,
                                 int64_t ldu, double *V, int64_t ldv, int *sweeps, void *stream);

/*
 * hsvd_shorten_qr -- the shortening QR on its own (kernel-level entry point):
 * G (m x n, ldg, device, m >= n >= 1, read-only) = Q R with R (n x n, ldr,
 * device) upper triangular, R_jj = -sign(alpha) ||x|| as in LAPACK's dgeqrf,
 * and, if Q is not NULL, the thin Q (m x n, ldq, device) with orthonormal
 * columns.  Workspace is allocated and freed on `stream`; returns after the
 * results are complete.
 */
int hsvd_shorten_qr(const double *G, int64_t m, int64_t n, int64_t ldg, double *R, int64_t ldr, double *Q,
                    int64_t ldq, void *stream);

/*
 * hsvd_diag_wait_timeout -- a diagnostic of failure detection without a GPU
 * fault: runs the bounded mbarrier wait of the tensor-core kernels on a
 * barrier that nothing arrives at, with a short poll limit.  Returns HSVD_OK
 * when the wait gave up as designed (the kernels then report HSVD_ERR_CUDA
 * instead of hanging) and the context stays usable, else HSVD_ERR_CUDA.
 */
int hsvd_diag_wait_timeout(void *stream);

/*
 * hsvd_sym_factor -- the symmetric indefinite factorisation that turns an
 * eigenproblem into an HSVD (Sec. 1): M (n x n, ldm, device, symmetric; only
 * read) = G J G^T with G (n x n, ldg, device) and J (n signs, device, int8),
 * from M = P L D L^T P^T with complete (Bunch-Parlett) pivoting, D of 1 x 1 and
 * 2 x 2 blocks.  A singular M is postprocessed (Sec. 1): the factorisation
 * stops once the trailing matrix is zero, and M = G_r J_r G_r^T with the first
 * r columns of G (full column rank) and r signs; the columns and signs past r
 * are zero, and *rank (may be NULL) receives r.  Returns HSVD_ERR_RANK for a
 * non-finite entry, HSVD_ERR_ARG for bad sizes or host pointers.  Returns after
 * the results are complete.
 *
 * hsvd_sym_eig -- the eigendecomposition M = U diag(lambda) U^T through the
 * factorisation and the HSVD of G (opts and info as for hsvd_solve_ex; NULL
 * opts = defaults): lambda[j] = sigma_j^2 J_jj with eigenvector U(:, j) (n x n,
 * ldu, device; may be NULL).  For a singular M of rank r the HSVD of the
 * n x r factor G_r (shortened by QR) gives the first r pairs; lambda[r..n-1]
 * are zero with eigenvectors spanning the orthogonal complement of range(G_r)
 * (the last n - r columns of the Q of a QR of U(:, 0..r-1)).  Device arrays
 * only.
 */
int hsvd_sym_factor(const double *M, int64_t n, int64_t ldm, double *G, int64_t ldg, int8_t *J, int64_t *rank,
                    void *stream);
int hsvd_sym_eig(const double *M, int64_t n, int64_t ldm, double *lambda, double *U, int64_t ldu,
                 const hsvd_opts *opts, hsvd_info *info, void *stream);

/*
 * Batched form: many independent factors of mixed sizes in one persistent
 * launch (a captured CUDA graph), each solved by the pointwise method
 * (Sec. 2, Alg. 4.5) with diagonal sorting (Sec. 4).  Factors are dispatched
 * largest first from one work queue; a CTA of 1024 threads solves one large
 * factor at a time and splits into groups of 512 or 256 threads for smaller
 * ones.  The group width of each size bucket (n < 40, < 72, < 128, < 192, and
 * larger) is picked by an autotuner that times the candidate widths on a
 * sample of the call's factors (two sweeps each) the first time a device sees
 * a set of buckets, and reuses that choice afterwards.
 */
typedef struct hsvd_batch_opts {
    double tol;      /* <= 0: n_k 2^-53 for factor k                                */
    int max_sweeps;  /* <= 0 selects 30                                             */
    int sort;        /* nonzero (default): diagonal sorting (Sec. 4)                */
    int group_width; /* 0 (default): autotuned per size bucket; 256, 512 or 1024:
                        that width for every factor                                 */
    int use_graph;   /* nonzero (default): the launch is captured as a CUDA graph  */
    double tstop;    /* tangent threshold of the early stop, as hsvd_opts.tstop    */
    int cta_threads; /* 0 or 1024 (default): CTAs of 1024 threads (groups of 1024,
                        512, 256); 512: CTAs of 512 threads with twice the
                        registers a thread (groups of 512, 256; group_width must
                        not exceed it)                                              */
    int reserved;    /* must be zero                                                */
} hsvd_batch_opts;

typedef struct hsvd_batch_info {
    int grid;             /* CTAs of the persistent launch (one per SM)            */
    int tuned;            /* 1: the autotuner ran in this call, 2: its cached
                             choice was used, 0: group_width was given              */
    int bucket_width[5];  /* group width used per size bucket                      */
    int max_sweeps_run;   /* largest sweep count over the factors                  */
    int64_t rotations;    /* rotations applied, all factors                        */
    int64_t kernel_launches; /* kernels of this library launched by the solve (1) */
    int64_t resident[3];  /* factors with G and W in shared memory, with G only,
                             with neither                                           */
    double ms_kernel;     /* CUDA-event time of the batched launch                 */
    double ms_tune;       /* CUDA-event time of the autotuner's sample runs        */
    int64_t tangent_stops; /* factors whose iteration ended at the tangent threshold */
    int cta_threads;      /* threads of the launch's CTAs                           */
} hsvd_batch_info;

/* Fills *opts with the defaults above. */
void hsvd_default_batch_opts(hsvd_batch_opts *opts);

/*
 * hsvd_solve_batched -- `count` independent HSVDs (Sec. 1, Eq. 1.1).  The
 * arrays G, m, n, ldg, J, sigma, U, V, sweeps and status are HOST arrays with
 * `count` entries.  The matrices they point to are all device pointers or all
 * host pointers (then staged through device copies, one copy per matrix).
 * Factor k: G[k] is m[k] x n[k] with leading dimension ldg[k], m >= n >= 1,
 * n <= 2048, m <= 4096; J[k] holds n[k] signs (int8, +-1); sigma[k] receives
 * n[k] values; U[k] (m[k] x n[k], leading dimension m[k]) and V[k] (n[k] x
 * n[k], leading dimension n[k]) may be NULL, and U or V itself may be NULL for
 * none at all.  sweeps and status (may be NULL) receive each factor's sweep
 * count and status code.  The call returns after the results are complete:
 * HSVD_OK if every factor converged, otherwise the first error code met
 * (or HSVD_NOT_CONVERGED); argument errors return HSVD_ERR_ARG before any work.
 */
int hsvd_solve_batched(int64_t count, const double *const *G, const int64_t *m, const int64_t *n,
                       const int64_t *ldg, const int8_t *const *J, double tol, int max_sweeps,
                       double *const *sigma, double *const *U, double *const *V, int *sweeps, int *status,
                       void *stream);

/* hsvd_solve_batched with options (NULL: defaults) and an optional report. */
int hsvd_solve_batched_ex(int64_t count, const double *const *G, const int64_t *m, const int64_t *n,
                          const int64_t *ldg, const int8_t *const *J, double *const *sigma, double *const *U,
                          double *const *V, int *sweeps, int *status, const hsvd_batch_opts *opts,
                          hsvd_batch_info *info, void *stream);

/*
 * Learned-form network kernels (device pointers, stream-ordered; the paper has
 * no counterpart: the network and its features are this library's additions).
 * hsvd_mlp_forward: logits[s] = net(X[s]) for n samples (X: n x 8 floats,
 *   row-major).
 * hsvd_mlp_grad: gradient of the mean binary cross-entropy with logits,
 *   mean(softplus(z) - y z), with respect to the parameter vector (the BF16
 *   rounding of the weights is treated as the identity); loss (device float,
 *   may be NULL) receives the mean loss.  Deterministic: fixed summation order.
 * hsvd_mlp_adam: one Adam step (Kingma and Ba) at step count t >= 1 on the
 *   parameter vector with moment vectors m and v.
 */
int hsvd_mlp_forward(const float *params, const float *X, int64_t n, float *logits, void *stream);
int hsvd_mlp_grad(const float *params, const float *X, const float *y, int64_t n, float *grad, float *loss,
                  void *stream);
int hsvd_mlp_adam(float *params, float *m, float *v, const float *grad, int t, float lr, float beta1, float beta2,
                  float eps, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HSVD_H */
