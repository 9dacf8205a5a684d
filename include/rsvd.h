/*
 * gb300-rsvd: truncated, randomized and exact SVD / PCA of tall zero-mean
 * matrices (m >> n) on one GB300 GPU (sm_103a), after the methods compared in
 * arXiv:1906.12085 ("Tutorial: Complexity analysis of Singular Value
 * Decomposition and its variants").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are ROW-MAJOR and dense; a row is one example (Sec. 2.2, the
 *   "each row of A represents an example" case).  A is m x n with m >= n.
 * - Every matrix / vector pointer is a caller-owned DEVICE pointer unless a
 *   parameter says otherwise.  The plan owns only its workspace.
 * - Calls are asynchronous on the plan's CUDA stream (the stream passed to
 *   rsvd_plan_create; NULL means the legacy default stream).  Argument errors
 *   are returned immediately; numerical conditions found on the device
 *   (Cholesky breakdown, Jacobi non-convergence, K > k) are accumulated in a
 *   device status word that rsvd_plan_sync() and pca_threshold() return.
 * - Element types follow the plan's dtype:
 *     RSVD_F64 : A, Omega, U, V are double;
 *     RSVD_F32 : A, Omega, U, V are float;
 *     RSVD_BF16: A holds bfloat16 codes (2 bytes, e.g. from rsvd_quantize);
 *                Omega, U, V are float;
 *     RSVD_FP8_E4M3: A holds e4m3 codes (1 byte) and rsvd takes the column
 *                scales s (the matrix is A diag(s)); Omega, U, V are float;
 *   singular values S are always double.
 * - Outputs are sorted by descending singular value.  Sign convention: the
 *   largest-magnitude entry of every right singular vector v_i is positive
 *   (u_i is flipped with it).
 * - Centring (Sec. 1 assumption that each feature has zero mean): by default
 *   every solve works on the centred matrix A - 1 mu^T (mu = column means) and
 *   records ||A - 1 mu^T||_F^2 (Eq. sumeigen).  rsvd and svd_truncated_krylov
 *   never write A: the means are subtracted inside the products.  svd_exact
 *   centres A IN PLACE.  RSVD_FLAG_NO_CENTER takes A as already centred
 *   (mu = 0) but still records ||A||_F^2.
 * - Plans are not thread-safe: one plan serves one solve at a time.
 */
#ifndef GB300_RSVD_H
#define GB300_RSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RSVD_F64 = 0,      /* float64 storage and arithmetic                       */
    RSVD_F32 = 1,      /* float32 storage, float32 products with float32 sums   */
    RSVD_BF16 = 2,     /* bfloat16 storage of A (precision form, rsvd only)     */
    RSVD_FP8_E4M3 = 3  /* e4m3 storage of A with per-column scales (rsvd only)  */
} rsvd_dtype;

typedef enum {
    RSVD_OK = 0,
    RSVD_ERR_ARG = -1,          /* invalid argument (sizes, NULL pointers, method)     */
    RSVD_ERR_OOM = -2,          /* device workspace allocation failed                  */
    RSVD_ERR_CHOL = -3,         /* Cholesky breakdown even after the shifted retry, or a
                                   final basis that failed its orthonormality check     */
    RSVD_ERR_NOCONV = -4,       /* a Jacobi solver hit its sweep cap                   */
    RSVD_ERR_TIMEOUT = -5,      /* a bounded device wait gave up (a product pipeline)  */
    RSVD_ERR_CUDA = -6,         /* a CUDA runtime call or kernel launch failed         */
    RSVD_ERR_UNSUPPORTED = -8,  /* size or dtype outside what this build implements    */
    RSVD_ERR_REDUCE = -9,       /* rsvd_sharded: the caller's reduction reported failure */
    RSVD_WARN_K_GT_k = 1,       /* the threshold t is not reached within the k values  */
    RSVD_WARN_RANK_DEFICIENT = 2 /* numerically rank-deficient input: a basis Cholesky
                                   needed its shift or removed dependent columns, or a
                                   Gram-route sigma_i fell to ~0; results are valid and
                                   the bases passed their orthonormality check          */
} rsvd_status;

/* svd_exact methods */
enum {
    RSVD_EXACT_GRAM = 0,        /* Sec. 2.3 / 3.1.3: A^T A, eigen-decomposition, u_i = A v_i / sigma_i */
    RSVD_EXACT_QR_JACOBI = 1    /* A = QR (CholeskyQR2), one-sided Jacobi SVD of R, U = Q U_R        */
};

/* plan flags */
enum {
    RSVD_FLAG_NO_CENTER = 1,     /* A is already centred (mu = 0)                                     */
    RSVD_FLAG_GKL_TWO_PASS = 2,  /* svd_truncated_krylov reads A twice per step (see there)           */
    RSVD_FLAG_SMALL_F32 = 4,     /* RSVD_BF16 / RSVD_FP8_E4M3: small SVD of B without the float64
                                    refinement (float32 rotations, float64 Rayleigh quotients)       */
    RSVD_FLAG_SMALL_FP64 = 8     /* RSVD_F32 rsvd / block Krylov: add the float64 refinement of the
                                    small SVD of B (default for BF16 / e4m3; see rsvd)               */
};

typedef struct rsvd_plan *rsvd_plan_t;

/*
 * Create a plan for m x n matrices (m >= n >= 1), target rank k, oversampling
 * p (sketch width l = k + p <= n) and q power iterations (Sec. 3.1.2: l is the
 * width of G, q plays the role of i).  The plan allocates its device
 * workspace once (cudaMalloc) and launches everything on `cuda_stream`
 * (a cudaStream_t, may be NULL).  For svd_exact the plan needs n <= 112 (the
 * n x n eigen / SVD problem is solved in one CTA's shared memory), or n <= 4096
 * for its Gram route (see svd_exact); for rsvd
 * l <= 288 (RSVD_F32, RSVD_BF16, RSVD_FP8_E4M3) or l <= 112 (RSVD_F64).  Above
 * l = 128 the tensor-core products run on column slices of at most 128 and the
 * l x l Cholesky and Jacobi blocks live in the plan's workspace, solved by an
 * 8-CTA thread-block cluster once they exceed one SM's shared memory.  Returns RSVD_ERR_ARG on inconsistent sizes, RSVD_ERR_UNSUPPORTED
 * for a dtype this build does not implement, RSVD_ERR_OOM if the workspace
 * cannot be allocated.  On error *plan is set to NULL.
 */
rsvd_status rsvd_plan_create(rsvd_plan_t *plan, int64_t m, int64_t n, int k, int p, int q,
                             rsvd_dtype dtype, void *cuda_stream);

/* Free the plan and its workspace (synchronises the plan's stream first). NULL is a no-op. */
rsvd_status rsvd_plan_destroy(rsvd_plan_t plan);

/* Bytes of device workspace owned by the plan (used for HBM admission). 0 for NULL. */
size_t rsvd_plan_workspace_bytes(rsvd_plan_t plan);

/* Set RSVD_FLAG_* bits for subsequent solves. */
rsvd_status rsvd_plan_set_flags(rsvd_plan_t plan, unsigned flags);

/* Wait for the plan's stream; return the device status of the last solve
 * (RSVD_OK, RSVD_WARN_RANK_DEFICIENT, RSVD_ERR_CHOL, RSVD_ERR_NOCONV, RSVD_ERR_TIMEOUT or
 * RSVD_ERR_CUDA; errors take precedence over the warning) and clear it. */
rsvd_status rsvd_plan_sync(rsvd_plan_t plan);

/*
 * Randomized PCA (Sec. 3.1.2, steps 2-7, with the power step re-orthonormalised
 * after each half step):
 *   Y = A Omega;  Q = orth(Y);
 *   repeat q times: Z = A^T Q, Q_Z = orth(Z), Y = A Q_Z, Q = orth(Y);
 *   T = A^T Q (= B^T with B = Q^T A);  T = Vt Sigma W^T;  U = Q W.
 * orth() is CholeskyQR2 (R_ii > 0), which in exact arithmetic equals the
 * Householder QR the step list names.  Bases stored in float32 (every dtype but
 * RSVD_F64) factor their float32 Gram matrix first; when that Cholesky breaks
 * down (a basis with condition number beyond ~1e4, as steep spectra and power
 * steps produce), the Gram matrix is formed again from the float32 basis with
 * float64 products and sums and factored in float64, so every direction the
 * float32 basis resolves is kept; exactly dependent columns (rank(A) < l) then
 * take the shift 11 (rows l + l(l+1)) u tr(G) of shifted CholeskyQR in float64.
 * Float64 bases remove a column whose Cholesky pivot is below l u of its squared
 * norm (it lies in the span of the columns before it) and replace it by a
 * pseudo-random column that the next pass orthonormalises.  Both are reported as
 * RSVD_WARN_RANK_DEFICIENT.  After the last CholeskyQR2 of Q and of T's factor
 * Q_T, max |Q^T Q - I| is checked on the device against 2e-5 (float32 bases) or
 * 1e-12 (float64); a basis beyond it makes the solve RSVD_ERR_CHOL, never a
 * silent result.
 *   A      : m x n, row-major, read only (centred on the fly).
 *   col_scales : n floats (device) for RSVD_FP8_E4M3 plans, NULL otherwise.
 * RSVD_BF16 plans (n a multiple of 8, l <= 288) solve for the stored bfloat16
 * matrix exactly as given: the products with A run on the tensor cores with
 * float32 accumulation, the small operand of the sketch and power products
 * rounded to bfloat16 and the basis of T = A^T Q split into three bfloat16
 * terms (float32-accurate); the column means enter as exact rank-1
 * corrections; the Cholesky of CholeskyQR2 (final basis and T) runs in
 * float64, the single-pass re-orthonormalisations of the power steps in
 * float32.  The small SVD of B (the SVD of T's factor R, Sec. 3.1.2 step 6) is
 * taken in float64: a float32 one-sided Jacobi start, then two Newton-type
 * float64 refinement steps (Ogita and Aishima's refinement of the SVD by matrix
 * products) that make U_R, W and sigma float64-accurate for the singular values
 * above 1e-5 sigma_1 (smaller ones lie beneath the float32 accuracy of T and keep
 * the start's absolute accuracy); about 0.5 ms at l = 288.  RSVD_FLAG_SMALL_F32
 * skips the refinement (float32 rotations, float64 Rayleigh-quotient values);
 * RSVD_FLAG_SMALL_FP64 adds it to RSVD_F32 single solves, which otherwise use
 * that float32 form (their stated tolerance, 1e-5 sigma_1, needs no more).
 * RSVD_FP8_E4M3 plans (n a multiple of 16, l <= 288) solve for A diag(s): the
 * sketch and power products run on e4m3 operands (the small operand diag(s) Z
 * and the basis Q quantised per column with their own scales, which the
 * epilogues multiply back); the Rayleigh-Ritz product runs on the exact
 * bfloat16 copy of the codes with the three-term basis (float32-accurate), in
 * 2mn bytes of extra workspace; the rest as for bfloat16.
 * svd_exact, svd_truncated_krylov and batches take RSVD_F32 / RSVD_F64 plans.
 *   Omega  : n x l Gaussian test matrix (caller-drawn), row-major.
 *   S      : k doubles; U : m x k; V : n x k (row-major).
 */
rsvd_status rsvd(rsvd_plan_t plan, void *A, const float *col_scales, const void *Omega,
                 double *S, void *U, void *V);

/*
 * Row-sharded randomized PCA (Sec. 3.1.2 over a row-block partition of A; the
 * paper runs one process).  Rank r of N holds the rows A_r of A = [A_1; ...; A_N]
 * (m_total rows in all) and calls rsvd_sharded with its own plan, created with
 * m = its row count (m >= n), the same n, k, p, q and dtype (RSVD_F32 or RSVD_F64)
 * on every rank, and the same Omega.  Every product with A stays on the rank;
 * what the method sums over rows is reduced across ranks by `allreduce`, a host
 * function that must replace values[0 .. count) by their elementwise sum over all
 * ranks (in rank-independent order, so that every rank receives the same numbers)
 * and return 0 (anything else ends the solve with RSVD_ERR_REDUCE):
 *   the column sums (n; the means follow), ||A - 1 mu^T||_F^2 (1), the Gram
 *   matrix of every CholeskyQR pass and of the final basis (lp x lp, lp = l
 *   rounded up to 16), Z = A^T Q of every power step and T = A^T Q (n x lp).
 * The small steps after a reduction (CholeskyQR of Z and T, the SVD of R, V) run
 * on every rank from the same numbers.  The reduced Gram matrices are factored in
 * float64 with the breakdown shift; the fallback tiers of rsvd's CholeskyQR (which
 * re-read the whole basis) are not used, so steep spectra that need them return
 * RSVD_WARN_RANK_DEFICIENT or RSVD_ERR_CHOL here.
 *   A     : this rank's m x n rows, read only.   Omega : n x l, as for rsvd.
 *   S     : k doubles and V : n x k, the same on every rank.
 *   U     : this rank's m x k rows of U.
 * Direct launches with a stream synchronisation at every reduction (no graph).
 * The first call allocates max(n, lp) x lp doubles of staging with cudaMalloc.
 * Status as for rsvd (read with rsvd_plan_sync).
 */
typedef int (*rsvd_allreduce_fn)(double *values, int64_t count, void *ctx);
rsvd_status rsvd_sharded(rsvd_plan_t plan, int64_t m_total, void *A, const void *Omega, double *S, void *U,
                         void *V, rsvd_allreduce_fn allreduce, void *ctx);

/*
 * All n singular triplets of A (Sec. 2.1 definition).
 *   method RSVD_EXACT_GRAM: the paper's "Truncated SVD" route (Sec. 2.3 and the
 *     step list of Sec. 3.1.3): G = A^T A, cyclic Jacobi eigen-decomposition,
 *     sigma_i = sqrt(lambda_i), u_i = A v_i / sigma_i (columns with
 *     sigma_i <= n * eps * sigma_1 are returned as zero vectors).
 *   method RSVD_EXACT_QR_JACOBI: A = Q R by CholeskyQR2, R = U_R Sigma V^T by
 *     one-sided Jacobi, U = Q U_R (backward stable; no squaring of cond(A)).
 *   S : n doubles; U : m x n; V : n x n.  dtype RSVD_F64 or RSVD_F32.
 * Sizes: n <= 112 for both methods (the n x n problem in one CTA's shared memory);
 * the Gram route also takes 112 < n <= 4096 (the k = n regime of the paper's
 * experiments, Sec. 4): G = A^T A (float32 plans on the tensor cores when n is a
 * multiple of 16), then a float64 eigen-decomposition on the whole GPU --
 * Householder tridiagonalisation, bisection, inverse iteration (Gram-Schmidt
 * inside clusters of eigenvalues closer than 1e-8 max|lambda|, at most 512 of
 * them, else RSVD_ERR_NOCONV) and back-transformation.  Its first call on a plan
 * allocates ~6 n^2 doubles of workspace with cudaMalloc.  RSVD_ERR_UNSUPPORTED
 * beyond these sizes.
 */
rsvd_status svd_exact(rsvd_plan_t plan, void *A, int method, double *S, void *U, void *V);

/*
 * Truncated SVD by Golub-Kahan-Lanczos bidiagonalisation with full
 * reorthogonalisation (classical Gram-Schmidt applied twice against every
 * previous basis vector) for `steps` steps from the start vector v1 (n
 * floats for RSVD_F32, n doubles for RSVD_F64; normalised internally):
 *   u_j = (A v_j - beta_{j-1} u_{j-1}) reorthogonalised / alpha_j,
 *   v_{j+1} = (A^T u_j - alpha_j v_j) reorthogonalised / beta_j,
 * then the SVD of the steps x steps upper bidiagonal B (alpha on the
 * diagonal, beta above) by one-sided Jacobi, B = X Sigma Y^T, and the leading
 * k Ritz triplets: S k doubles, U = U_s X (m x k), V = V_s Y (n x k).
 * This is the Krylov route of the library; the paper's own Krylov method
 * (Sec. 3.1.1, a block power basis) is a different algorithm.
 * Float32 plans read A once per step: g = (A - 1 mu^T) v_j and x = (A - 1 mu^T)^T g
 * come from the same rows, and A^T u_j is recovered by linearity from the stored
 * A^T u_i (i < j) and the summed reorthogonalisation coefficients; the recovery
 * multiplies the rounding of x by ||x|| / alpha_j, so a step whose ||x|| exceeds
 * 16 alpha_j max_i alpha_i also reads A a second time (decided on the device).
 * RSVD_FLAG_GKL_TWO_PASS (and float64 plans) always read A twice per step.
 * Requires k <= steps <= n and steps <= 160 (RSVD_F32) / 112 (RSVD_F64)
 * (RSVD_ERR_UNSUPPORTED otherwise).  The first call on a plan allocates the
 * Lanczos workspace (steps x m + (steps+1) x n elements and small buffers)
 * with cudaMalloc; later calls with no more steps reuse it.
 */
rsvd_status svd_truncated_krylov(rsvd_plan_t plan, void *A, const void *v1, int steps,
                                 double *S, void *U, void *V);

/*
 * Block Krylov method (Sec. 3.1.1): the Rayleigh-Ritz approximation of the
 * leading k singular triplets from the block Krylov space
 *   span [H(0) | H(1) | ... | H(i)],  H(0) = A Omega,  H(j) = A (A^T H(j-1)),
 * of W = (i + 1) b columns (Omega n x b Gaussian, caller-drawn):
 *   Q = orth([H(0) | ... | H(i)]);  T = A^T Q (= B^T);  T = Vt Sigma W^T;  U = Q W.
 * The plan comes from rsvd_plan_create_block_krylov (block width b, i =
 * `iters`); rsvd() and batches reject such plans, and rsvd_block_krylov
 * rejects the others (RSVD_ERR_ARG).
 * The basis is built block by block and never from the power blocks
 * themselves, which become nearly dependent as they converge: block j is the
 * part of A A^T (block j-1) orthogonal to the blocks before it (block classical
 * Gram-Schmidt, applied twice), orthonormalised by SVQB -- the eigen-
 * decomposition G = V diag(lam) V^T of its Gram matrix, X V diag(lam)^{-1/2}
 * -- then projected once more and finished by CholeskyQR2.  In exact arithmetic
 * this spans the same space as the step list; directions of a block whose
 * eigenvalue lam is below 2u lam_1 (u the unit roundoff of the element type)
 * are not resolved by the block's rounding and are replaced by pseudo-random
 * ones (SplitMix64, fixed seed), which keeps Q orthonormal on rank-deficient
 * or fast-decaying spectra and only enlarges the space searched.  The products
 * with A and Omega are those of rsvd(); the Rayleigh-Ritz steps are rsvd()'s
 * at width W, except that an RSVD_F32 plan factors T by CholeskyQR2 in float64
 * (its Gram matrices accumulated in float64 from the float32 T): T's Ritz
 * values span the whole Krylov space, far below what a float32 Gram resolves.
 *   A     : m x n row-major, read only (centred on the fly unless RSVD_FLAG_NO_CENTER).
 *   Omega : n x b; S : k doubles; U : m x k; V : n x k.
 * Element types as for rsvd() with RSVD_F32 / RSVD_F64 (the only dtypes).
 * Limits: k <= W <= n, b <= 112 (the block's Gram eigen-decomposition runs in
 * one CTA), W <= 288 (RSVD_F32) or 112 (RSVD_F64); RSVD_ERR_UNSUPPORTED
 * beyond them, RSVD_ERR_ARG for inconsistent sizes.  Launches run directly on
 * the plan's stream (no graph capture); statuses as for rsvd().
 */
rsvd_status rsvd_plan_create_block_krylov(rsvd_plan_t *plan, int64_t m, int64_t n, int k, int b, int iters,
                                          rsvd_dtype dtype, void *cuda_stream);
rsvd_status rsvd_block_krylov(rsvd_plan_t plan, void *A, const void *Omega, double *S, void *U, void *V);

/*
 * Sec. 2.4 cumulative explained variance: the minimal K with
 *   sum_{i<=K} sigma_i^2 >= t * ||A||_F^2
 * over the singular values of the plan's last solve, with the denominator
 * from Eq. (sumeigen).  Synchronises the stream and writes K to the HOST int
 * *K.  If the values returned by the last solve do not reach t, *K is their
 * count and the result is RSVD_WARN_K_GT_k.  t must lie in (0, 1].
 */
rsvd_status pca_threshold(rsvd_plan_t plan, double t, int *K);

/*
 * svd_exact_gram_static: svd_exact with method RSVD_EXACT_GRAM for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is an
 * interface addition, not a method.
 *
 * Who needs it: code that runs where device memory is owned by someone else
 * or where cudaMalloc / cudaFree are not allowed -- a plugin inside a host
 * framework that hands out memory only from its own pool, a process under a
 * hard device-memory budget fixed at start-up, or a latency-critical loop
 * that must not hit cudaMalloc's and cudaFree's implicit device-wide
 * synchronisation.  Such a caller still passes A, S, U and V; the entry point
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Scratch: a file-scope 12 MiB static device array.  Every GPU that loads the
 * library holds it until process exit.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the one array, which keeps the previous call's contents: the status word is
 * cleared at the start of every call, and calls that overlap on the GPU (two
 * streams, two host threads) race and must be serialised by the caller.
 *
 * Arguments: A m x n row-major (centred in place, as svd_exact does), S n
 * doubles, U m x n, V n x n (float64 for RSVD_F64, float32 for RSVD_F32),
 * cuda_stream a cudaStream_t (may be NULL).  Limit: n <= 64 (any m >= n);
 * larger n returns RSVD_ERR_UNSUPPORTED.  The call synchronises the stream
 * and returns RSVD_OK, RSVD_ERR_NOCONV (Jacobi sweep cap), RSVD_ERR_ARG or
 * RSVD_ERR_CUDA.  Results equal svd_exact's Gram route on the same input.
 */
rsvd_status svd_exact_gram_static(void *A, int64_t m, int64_t n, rsvd_dtype dtype, double *S, void *U, void *V,
                                  void *cuda_stream);

/*
 * Process-wide cap on the sweeps of the Jacobi solvers (the one-sided SVD of R and
 * of the Lanczos bidiagonal, the two-sided eigen-decompositions of the Gram route
 * and of block Krylov's SVQB); cap 0 restores the defaults (40 and 50 sweeps).  A
 * solver that reaches the cap before a sweep without rotations sets
 * RSVD_ERR_NOCONV.  Applies to launches issued afterwards: a CUDA graph a plan
 * captured earlier keeps the cap it was captured with.  RSVD_ERR_ARG for cap < 0.
 */
rsvd_status rsvd_set_jacobi_sweep_cap(int cap);

/* Host copy of ||A||_F^2 (after centring) recorded by the last solve; synchronises. */
rsvd_status rsvd_plan_fro2(rsvd_plan_t plan, double *fro2);

/*
 * Tracing: per-stage CUDA-event timing.  When enabled, the plan records a
 * pair of events on its stream around every kernel group of a stage; the
 * read call synchronises the stream, writes the summed milliseconds and the
 * number of timed groups per stage (arrays of `nstages` entries, host
 * memory) since the previous read, and clears them.  Stages:
 */
enum {
    RSVD_STAGE_CENTER = 0,  /* column means, centring, ||A||_F^2                      */
    RSVD_STAGE_AX = 1,      /* products A X with X skinny (sketch, power step, U)     */
    RSVD_STAGE_ATX = 2,     /* products A^T X (power step, T = A^T Q, Gram of A)      */
    RSVD_STAGE_ORTH = 3,    /* CholeskyQR2 of the m-row and n-row blocks              */
    RSVD_STAGE_SMALL = 4,   /* small SVD / eigen problems (Jacobi), K selection       */
    RSVD_STAGE_FINISH = 5,  /* Ritz vectors, sign convention, output copies           */
    RSVD_STAGE_COUNT = 6
};
rsvd_status rsvd_plan_profile(rsvd_plan_t plan, int enable);
rsvd_status rsvd_plan_profile_read(rsvd_plan_t plan, double *ms, int *groups, int nstages);

/* Process-wide number of kernels this library has launched (all plans). */
uint64_t rsvd_launch_count(void);

/* Static description of a status code. */
const char *rsvd_status_string(rsvd_status s);

/*
 * Storage of the precision form (BF16 / FP8 e4m3 matrices; the paper works in
 * float64 throughout and has no counterpart).  A: m x n float32 (lda >= n,
 * device).  Aq: m x n row-major codes (device; 2 bytes per entry for
 * RSVD_BF16, 1 byte for RSVD_FP8_E4M3).
 *   RSVD_BF16     : the nearest bfloat16 value, ties to even.
 *   RSVD_FP8_E4M3 : col_scales (n floats, device) receive s_j = amax_j / 448
 *                   (float32 division; 1 for an all-zero column) and Aq the
 *                   nearest OCP e4m3 value (bias 7, 3 mantissa bits, no
 *                   infinities) of the float32 quotient a_ij / s_j, ties to
 *                   even, magnitudes above 448 saturated to 448.
 * The stored matrix is then exactly Aq (bfloat16) or Aq diag(s) (e4m3).
 * Asynchronous on cuda_stream; no workspace (col_scales also holds the
 * column maxima while they are reduced).  RSVD_ERR_ARG for NULL pointers or
 * bad sizes, RSVD_ERR_UNSUPPORTED for other dtypes.
 */
rsvd_status rsvd_quantize(const float *A, int64_t m, int64_t n, int64_t lda, rsvd_dtype dtype, void *Aq,
                          float *col_scales, void *cuda_stream);

/* ====================================================================
 * Batching and serving.  The paper has no counterpart: these run many
 * independent randomized PCA problems (Sec. 3.1.2) at once.  Each problem
 * executes exactly the kernels and arithmetic of a single rsvd() call, so its
 * result does not depend on what it was batched or served with.
 * ==================================================================== */

/* Device workspace bytes a plan of these sizes needs, a multiple of 256 (no
 * allocation, no GPU work).  Same argument rules and errors as rsvd_plan_create. */
rsvd_status rsvd_workspace_query(int64_t m, int64_t n, int k, int p, int q, rsvd_dtype dtype, size_t *bytes);

/* rsvd_plan_create on caller-owned device memory: `workspace` (256-byte
 * aligned, at least rsvd_workspace_query bytes) is carved, not allocated, and
 * is cleared with an asynchronous memset on `cuda_stream`; the call neither
 * allocates device memory nor synchronises.  The caller keeps the workspace
 * alive until rsvd_plan_destroy and frees it afterwards.  RSVD_ERR_ARG for a
 * NULL, misaligned or short workspace. */
rsvd_status rsvd_plan_create_in(rsvd_plan_t *plan, int64_t m, int64_t n, int k, int p, int q, rsvd_dtype dtype,
                                void *cuda_stream, void *workspace, size_t bytes);

/*
 * Batched small solves: `count` (1..RSVD_BATCH_MAX) problems whose plans share
 * dtype (RSVD_F32 or RSVD_F64), l = k + p <= 128 and q (m, n, k may differ;
 * plans distinct); RSVD_ERR_UNSUPPORTED otherwise.  A run solves
 * every problem in lockstep: each problem's products run on its own plan's
 * stream; each small dense step (Cholesky of the CholeskyQR2 Gram matrices,
 * Jacobi SVD of R, the float64 refinement) is one launch over all problems on
 * `cuda_stream`, which waits for the problems' streams and which they wait
 * for.  On a non-legacy stream the whole run is captured into one CUDA graph
 * on first use and replayed while the argument pointers and plan flags repeat
 * (the plans' streams must then be non-legacy too).  rsvd_batch_run takes
 * arrays of `count` device pointers with the meaning and layout of rsvd()'s
 * arguments (col_scales NULL); it is asynchronous.  rsvd_batch_sync waits and
 * returns the first failing status (statuses: `count` host ints or NULL).
 * Afterwards pca_threshold works on each plan as after rsvd().  The batch
 * object owns only its tables and events; the plans stay the caller's.
 */
#define RSVD_BATCH_MAX 256
typedef struct rsvd_batch *rsvd_batch_t;
rsvd_status rsvd_batch_create(rsvd_batch_t *batch, int count, rsvd_plan_t const *plans, void *cuda_stream);
rsvd_status rsvd_batch_run(rsvd_batch_t batch, void *const *A, const void *const *Omega, double *const *S,
                           void *const *U, void *const *V);
rsvd_status rsvd_batch_sync(rsvd_batch_t batch, int *statuses);
rsvd_status rsvd_batch_destroy(rsvd_batch_t batch);

/*
 * Autotuner of the products' launch shape (float32 plans on the tensor-core
 * path): the number of persistent CTAs of Y = A X and of Z = A^T X.  The tiles
 * and their order of summation do not depend on it, so results are bitwise the
 * same under every choice; only the sharing of the GPU between concurrent
 * problems changes.  Runs `concurrency` (1..64) copies of the plan's problem on A and
 * Omega (the caller's plan plus concurrency-1 temporary plans, as one lockstep
 * batch like rsvd_batch_run) under each candidate decomposition, keeps the one
 * with the smallest median batch time over three runs, and records it in a
 * process-wide table keyed by (ceil(log2 m), n, l rounded up to 16): the plan
 * and every plan created later in that bucket (rsvd_plan_create,
 * rsvd_plan_create_in, the serving loop) use it.  Synchronises; allocates and
 * frees temporary device memory; the plan's outputs of the last solve are not
 * kept (solve again before pca_threshold).  nn_ctas / tn_ctas (host, may be
 * NULL) receive the choice, 0 meaning the default (one CTA per SM).  Other plans: RSVD_OK with the current (default)
 * choice.  rsvd_tune_lookup returns RSVD_OK and the recorded choice for a
 * bucket, RSVD_ERR_ARG when there is none; rsvd_tune_clear empties the table.
 */
rsvd_status rsvd_autotune(rsvd_plan_t plan, void *A, const void *Omega, int concurrency, int *nn_ctas,
                          int *tn_ctas);
rsvd_status rsvd_tune_lookup(int64_t m, int64_t n, int k, int p, int *nn_ctas, int *tn_ctas);
void rsvd_tune_clear(void);

/*
 * Serving loop: continuous batching of randomized PCA requests.
 *   rsvd_server_create: one device arena of `hbm_bytes` (cudaMalloc'd once)
 *     holds every admitted request's plan workspace; at most `max_inflight`
 *     batches run at once, each of at most `max_batch` requests, on streams
 *     of the server's own.
 *   rsvd_server_submit: queue request `id` (A m x n, Omega n x (k+p), S k
 *     doubles, U m x k, V n x k: caller-owned device memory that must stay
 *     valid until the request completes; t is the Sec. 2.4 threshold).
 *     RSVD_ERR_OOM if its workspace can never fit the arena; argument errors
 *     as rsvd_plan_create.  Does not block.
 *   rsvd_server_poll: retire finished batches (frees their arena space),
 *     admit queued requests in arrival order while the arena and the batch
 *     slots allow (the oldest waiting request is never overtaken; consecutive
 *     queued requests of the same l and q share a batch), launch them, and
 *     write up to `max_out` completions to `out`.  Returns the number written,
 *     or a negative rsvd_status on a CUDA error.  Does not block.
 *   rsvd_server_pending: requests queued or running.
 * Times are host milliseconds since rsvd_server_create: submit (the call),
 * start (admission and launch), done (the device finished the request's
 * batch, from CUDA events).  One host thread drives a server.
 */
typedef struct rsvd_server *rsvd_server_t;
typedef struct {
    int64_t id;
    int status;  /* rsvd_status of the solve, RSVD_WARN_K_GT_k when t is not reached within k */
    int K;       /* Sec. 2.4 K */
    int batch;   /* requests in the batch it ran in */
    double submit_ms, start_ms, done_ms;
} rsvd_completion;
rsvd_status rsvd_server_create(rsvd_server_t *server, size_t hbm_bytes, int max_batch, int max_inflight);
rsvd_status rsvd_server_submit(rsvd_server_t server, int64_t id, int64_t m, int64_t n, int k, int p, int q,
                               double t, const float *A, const float *Omega, double *S, float *U, float *V);
/* rsvd_server_submit for a stored matrix of any rsvd storage type: RSVD_F32,
 * RSVD_BF16 or RSVD_FP8_E4M3 (with its n column scales; NULL otherwise).
 * Omega, U, V are float.  Requests batch only with requests of the same type;
 * the precision forms' batches (and float32 batches with l > 128) run their
 * solves concurrently (one stream per request) rather than in lockstep. */
rsvd_status rsvd_server_submit_ex(rsvd_server_t server, int64_t id, int64_t m, int64_t n, int k, int p, int q,
                                  rsvd_dtype dtype, double t, const void *A, const float *col_scales,
                                  const float *Omega, double *S, float *U, float *V);
int rsvd_server_poll(rsvd_server_t server, rsvd_completion *out, int max_out);
int rsvd_server_pending(rsvd_server_t server);
rsvd_status rsvd_server_destroy(rsvd_server_t server);

#ifdef __cplusplus
}
#endif
#endif /* GB300_RSVD_H */
