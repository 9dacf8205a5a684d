/*
 * FP64 CPU oracle for the tall-skinny SVD / PCA methods of arXiv:1906.12085.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA library
 * shares no code, header, table or helper with it.
 *
 * Conventions: every matrix is row-major float64; m >= n (tall).  Return
 * value 0 on success, negative on error, positive for a warning.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_OOM = -2, ORC_ERR_NOCONV = -4,
       ORC_ERR_BREAKDOWN = -7, ORC_WARN_K_GT_COUNT = 1 };

/* Sec. 1 assumption (zero mean per feature) and Eq. (sumeigen):
 * mu_j = mean_i a_ij, A <- A - 1 mu^T, fro2 = sum_ij a_ij^2 of the centred A. */
int orc_center(int64_t m, int64_t n, double *A, double *mu, double *fro2);

/* Householder QR, thin: Y (m x n) = Q R with R_ii >= 0.  Q m x n, R n x n (may be NULL). */
int orc_qr(int64_t m, int64_t n, const double *Y, double *Q, double *R);

/* Sec. 2.1 definition A = U Sigma V^T, computed by Householder bidiagonalisation
 * followed by implicit-shift QR on the bidiagonal (Golub-Reinsch 1970).
 * S: n values, descending, >= 0.  U: m x n, V: n x n (either may be NULL). */
int orc_svd(int64_t m, int64_t n, const double *A, double *S, double *U, double *V);

/* Cyclic two-sided Jacobi eigensolver of a symmetric n x n matrix.
 * lam descending; V n x n with eigenvectors as columns.  *sweeps (may be NULL). */
int orc_eig_jacobi(int64_t n, const double *G, double *lam, double *V, int *sweeps);

/* Sec. 2.3 / Sec. 3.1.3 "Truncated SVD" (Gram route): G = A^T A, eig(G),
 * sigma_i = sqrt(lambda_i), u_i = A v_i / sigma_i.  U m x n, V n x n. */
int orc_svd_gram(int64_t m, int64_t n, const double *A, double *S, double *U, double *V);

/* Sec. 3.1.2 randomized PCA with the given Gaussian test matrix Omega (n x l):
 * Y = A Omega, Q = qr(Y); q times { Z = A^T Q, Q_Z = qr(Z), Y = A Q_Z, Q = qr(Y) };
 * T = A^T Q; T = Vt Sigma W^T (so B = Q^T A = W Sigma Vt^T); U = Q W.
 * Outputs the leading k triplets: S k, U m x k, V n x k. */
int orc_rsvd(int64_t m, int64_t n, const double *A, int64_t l, int q,
             const double *Omega, int64_t k, double *S, double *U, double *V);

/* Sec. 3.1.1 block Krylov method with the given Gaussian test matrix Omega (n x l):
 * H(0) = A Omega, H(j) = A (A^T H(j-1)) (j = 1..iters, every block re-orthonormalised
 * before it feeds the next), H = [H(0) | ... | H(iters)] (m x (iters+1) l),
 * Q = qr(H), T = A^T Q = Vt Sigma W^T, U = Q W.  Requires (iters+1) l <= n.
 * Outputs the leading k triplets: S k, U m x k, V n x k. */
int orc_block_krylov(int64_t m, int64_t n, const double *A, int64_t l, int iters,
                     const double *Omega, int64_t k, double *S, double *U, double *V);

/* Golub-Kahan-Lanczos bidiagonalisation with full reorthogonalisation
 * (classical Gram-Schmidt applied twice), `steps` steps from the start
 * vector v1 (length n), followed by the SVD of the steps x steps bidiagonal.
 * alpha, beta: steps values each (may be NULL).  S k, U m x k, V n x k. */
int orc_gkl(int64_t m, int64_t n, const double *A, const double *v1, int steps,
            int64_t k, double *S, double *U, double *V, double *alpha, double *beta);

/* Sec. 2.4 cumulative explained variance: minimal K with
 * sum_{i<=K} sigma_i^2 >= t * fro2 (Eq. sumeigen gives the denominator).
 * If the `count` known values never reach it, K = count and the return is
 * ORC_WARN_K_GT_COUNT. */
int orc_pca_threshold(int64_t count, const double *sigma, double fro2, double t, int64_t *K);

/* Make the largest-|entry| component of each column of V positive, flipping
 * the matching column of U (sign convention of all oracle outputs). */
void orc_sign_normalize(int64_t m, int64_t n, int64_t k, double *U, double *V);

/* ---- Storage formats of the precision form ----
 * bfloat16: the float32 value rounded to the nearest bfloat16 (8 exponent
 * bits, 7 stored mantissa bits), ties to the even mantissa.
 * e4m3 (OCP FP8 "E4M3FN": bias 7, 3 mantissa bits, no infinities, NaN =
 * S.1111.111, largest finite 448): per column j the scale s_j = amax_j / 448
 * computed in float32 (s_j = 1 for an all-zero column), the quotient
 * a / s_j rounded to float32, then the nearest e4m3 value with ties to the
 * even code, magnitudes above 448 saturated to 448. */
uint16_t orc_bf16_encode(float x);
double orc_bf16_decode(uint16_t b);
uint8_t orc_e4m3_encode(float x);
double orc_e4m3_decode(uint8_t c);
/* A float32 m x n (lda) -> codes m x n (row-major) and n column scales. */
void orc_quantize_bf16(int64_t m, int64_t n, const float *A, int64_t lda, uint16_t *out);
void orc_quantize_e4m3(int64_t m, int64_t n, const float *A, int64_t lda, uint8_t *out, float *scales);

#ifdef __cplusplus
}
#endif
#endif
