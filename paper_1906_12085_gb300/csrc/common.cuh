// Internal declarations shared by the CUDA translation units of gb300-rsvd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsvd.h"

namespace gbr {

// Bits of the device status word (OR-ed by kernels, read by rsvd_plan_sync).
enum StatusBits : int {
    ST_CHOL = 1,      // Cholesky breakdown after the shifted retry
    ST_NOCONV = 2,    // Jacobi sweep cap reached
    ST_SHIFT = 4,     // shifted Cholesky was needed (warning: rank deficient)
    ST_RANKDEF = 8,   // a singular value fell below n*eps*sigma_1, or a float64 basis column
                      // was removed and refilled (warning: rank deficient)
    ST_TIMEOUT = 16,  // a bounded device wait gave up (pipeline stalled)
    ST_ORTH = 32,     // a final basis failed the orthonormality check max|Q^T Q - I| <= tol
};

// Orthonormality bound of the final bases (max |Q^T Q - I|, checked on the device after the
// last CholeskyQR2): float32 bases 2e-5 (a basis this close to orthonormal moves no Ritz
// value by more than ~1e-5 relative), float64 bases 1e-12.
constexpr double kOrthTolF32 = 2e-5;
constexpr double kOrthTolF64 = 1e-12;

// Largest l (or n for svd_exact) whose l x l working set fits one CTA's shared memory.
constexpr int kSmallMaxF64 = 112;
// Largest l of a float32 batched or lockstep-served solve (the batched small kernels
// keep their l x l blocks in shared memory).
constexpr int kSmallMaxF32 = 128;
// Largest l of a single float32 / bfloat16 / e4m3 randomized solve: above the shared-
// memory sizes the Cholesky and Jacobi keep their l x l blocks in a global scratch
// (on an 8-CTA cluster), and the products run on column slices (N <= 128 per launch;
// the bfloat16 / e4m3 A Z product up to 256, the one-term bfloat16 A^T Q up to 192).
constexpr int kRsvdMaxL = 288;
// The float32 tensor-core products take N <= 128 output columns per launch; wider
// products run as ceil(N / 128) launches on column slices of this width (a multiple
// of 16).
inline int column_slice(int N) {
    const int k = (N + 127) / 128;
    return ((N + k - 1) / k + 15) / 16 * 16;
}
// Largest Lanczos step count whose bidiagonal SVD fits one CTA in float32.
constexpr int kGklMaxStepsF32 = 160;

// Count of kernel launches issued by the library (reported by rsvd_launch_count).
void note_launch(int count = 1);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the finaliser applied to seed + (i + 1) * gamma.  The
// counter-based source of the columns that replace removed basis directions.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// ---------------------------------------------------------------- centring
// mu = column means of A (m x n, ld), A <- A - 1 mu^T, *fro2 = ||A||_F^2 (float64).
// part: scratch of centre_partials(m, n) doubles.
template <typename T>
cudaError_t center_columns(T *A, int64_t m, int64_t n, int64_t lda, bool subtract, double *mu,
                           double *fro2, double *part, cudaStream_t s);
int64_t center_partials(int64_t m, int64_t n);
// mu = column means (float64) and mu_t = the same in T, zero padded to npad entries (A read only).
template <typename T>
cudaError_t column_means(const T *A, int64_t m, int64_t n, int64_t lda, double *mu, T *mu_t, int64_t npad,
                         double *part, cudaStream_t s);
// *fro2 = ||A - 1 mu^T||_F^2 (mu may be NULL: ||A||_F^2), A read only.
template <typename T>
cudaError_t centered_fro2(const T *A, int64_t m, int64_t n, int64_t lda, const double *mu, double *fro2, double *part,
                          cudaStream_t s);
// out[c] = sum_r X[r][c] (dsum: float64 copy, cols entries; part: center_partials(rows, cols))
template <typename T>
cudaError_t column_sums(const T *X, int64_t rows, int64_t cols, int64_t ld, double *dsum, T *out, double *part,
                        cudaStream_t s);
// *out = sum of count doubles (fixed order)
cudaError_t sum_f64(const double *x, int64_t count, double *out, cudaStream_t s);
// Column means from column sums over all row blocks of a row-sharded A: sum[i] *= inv_m
// (in place) and mu_t = the means in T, zero-padded to npad.
template <typename T>
cudaError_t scale_means(double *sum, int64_t n, int64_t npad, double inv_m, T *mu_t, cudaStream_t s);
// C[r][c] -= (x ? x[r] : 1) * y[c] for r < rows, c < cols
template <typename T>
cudaError_t rank1_sub(T *C, int64_t rows, int64_t cols, int64_t ldc, const T *x, const T *y, cudaStream_t s);
// c[j] = sum_k mu[k] B[k][j], j < N (float64 accumulation)
template <typename T>
cudaError_t vecmat(const T *mu, const T *B, int64_t K, int64_t N, int64_t ldb, T *c, cudaStream_t s);

// ---------------------------------------------------------------- products
// C (M x N) = A (M x K) * B (K x N); all row-major with leading dimensions.
template <typename T>
cudaError_t gemm_nn(int64_t M, int64_t N, int64_t K, const T *A, int64_t lda, const T *B, int64_t ldb,
                    T *C, int64_t ldc, cudaStream_t s);

// C (N x L) = A^T B with A rows x N (lda) and B rows x L (ldb): split over row
// chunks into `part`, then summed in chunk order (deterministic).
template <typename T>
cudaError_t gemm_tn(int64_t rows, int64_t N, int64_t L, const T *A, int64_t lda, const T *B, int64_t ldb,
                    T *C, int64_t ldc, T *part, int64_t part_elems, cudaStream_t s);
// scratch elements gemm_tn needs for these sizes
int64_t gemm_tn_partials(int64_t rows, int64_t N, int64_t L);

// ---------------------------------------------------------- small dense
// Upper Cholesky R^T R = G (+ shift) of the leading l x l block of G (ldg), then
// R^{-1}, arithmetic in Tk.  Writes R, Rinv (float64, l x l dense, ld l) and
// Rinv_c (element type Tc, lp x lp, zero padded).  The role selects what a
// breakdown (a pivot that is not positive and finite) does:
//   kCholPlain    : retry once with the shift 11 (rows*l + l(l+1)) u tr(G) (shifted
//                   CholeskyQR, ST_SHIFT); on a second breakdown set ST_CHOL and return
//                   R = 0, R^{-1} = I;
//   kCholFirst    : a float64 fallback follows: write *fb = 1 and leave R, Rinv and
//                   Rinv_c to it; on success write *fb = 0.  With float32 arithmetic and a
//                   scratch of chol_scratch_bytes(l, 8) bytes, a breakdown is first retried
//                   in float64 on the same G (kCholRetry, in the scratch), and *fb = 1 only
//                   when that breaks down too;
//   kCholFallback : return at once unless *fb is set; otherwise as kCholPlain (G is then
//                   the float64 Gram matrix of gram64_fb);
//   kCholDeflate  : never shift: a pivot <= kDeflateRel l G_kk (G_kk the diagonal of G)
//                   removes column k -- R_kk = 1, the rest of row and column k of R zero --
//                   and sets fb[k] = 1 and fb[l] = 1 (fb: l + 1 ints, cleared first); X R^{-1}
//                   then keeps column k of X, which the caller replaces.
// Matrices whose two l x l blocks exceed one SM's shared memory (l > 112 in float64,
// l > 128 in float32) live in `scratch` (chol_scratch_bytes(l, sizeof(Tk)) bytes of
// device memory), which may be NULL otherwise.
enum CholRole : int { kCholPlain = 0, kCholFirst = 1, kCholFallback = 2, kCholDeflate = 3, kCholRetry = 4 };
// relative pivot below which kCholDeflate removes a column, per column of the block: the
// float64 unit roundoff, i.e. a column whose squared distance from the span of the previous
// ones is below l u of its squared norm, the rounding level of its float64 Gram matrix
constexpr double kDeflateRel = 0x1.0p-53;
template <typename TG, typename Tk, typename Tc>
cudaError_t chol_inv(const TG *G, int64_t ldg, int l, int64_t rows, double unit_roundoff, double *R,
                     double *Rinv, Tc *Rinv_c, int lp, int *status, cudaStream_t s, void *scratch = nullptr,
                     int *fb = nullptr, int role = kCholPlain);
size_t chol_scratch_bytes(int l, size_t tk);

// The fallback of CholeskyQR after a breakdown of the float32 Gram matrix, one launch: the
// float64 Gram matrix G (l x l upper triangle, ldg) = X^T X of X rows x l (ld, float32), every
// product and sum in float64 (CUDA cores), split over row chunks into `part`
// (gram64_partials(rows, l) doubles) and summed in chunk order by the last CTA (`count`: a
// zeroed counter of the job, left zero), which then factors G as chol_inv does with `role`
// kCholFallback (shift; R, Rinv, Rc, lp, status, shift coefficient `coef`) or kCholDeflate
// (removed columns flagged in dflag, l ints), its matrices in the global scratch gws
// (chol_scratch_bytes(l, 8) bytes).  Returns at once unless *fb is set.
struct G64Job {
    const float *X;
    int64_t rows, ld;
    double *part, *G;
    const int *fb;
    unsigned *count;
    double coef;
    double *R, *Rinv;
    float *Rc;
    int lp;
    int *status;
    double *gws;
    int role;
    int *dflag;
};
int64_t gram64_partials(int64_t rows, int l);
cudaError_t gram64_fb(const G64Job &job, int l, int64_t ldg, cudaStream_t s);
// the same for `count` jobs of one l (device table, one launch)
cudaError_t gram64_fb_batched(const G64Job *tab, int count, int64_t max_rows, int l, int64_t ldg, cudaStream_t s);
// The basis of a fallback pass: Q (rows x l, ld, float32) = X R^{-1} to ~2^-48 relative
// (Rinv: float64 l x l upper triangular, ld l), rounded once; the columns flagged in dflag
// (may be NULL) are replaced by uniform entries in [-sqrt(3/rows), sqrt(3/rows)) from
// SplitMix64 with `seed` (as bk_fill).  Returns at once unless *fb is set and, when `need`
// is given, *need too (an intermediate basis: only when a column was removed).  X and Q
// must not overlap.
struct Rinv64Job {
    const float *X;
    int64_t rows, ld;
    const double *Rinv;
    float *Q;
    const int *fb;
    const int *dflag;
    uint64_t seed;
    const int *need;
};
cudaError_t rinv64_fb(const Rinv64Job &job, int l, cudaStream_t s);

// ST_ORTH into *status when max_{i<=j<l} |G_ij - delta_ij| > tol (or is not a number), G the
// upper triangle of the Gram matrix Q^T Q of a basis (ldg).
template <typename T>
cudaError_t orth_check(const T *G, int l, int64_t ldg, double tol, int *status, cudaStream_t s);

// Process-wide sweep cap of the Jacobi solvers (0: the defaults).
void set_sweep_cap(int cap);

// R = R2 * R1 for upper-triangular l x l float64 matrices (ld l).
cudaError_t trmm_upper(const double *R2, const double *R1, double *R, int l, cudaStream_t s);

// One-sided Jacobi SVD of the l x l float64 matrix R (ld l), arithmetic in Ta:
// R W = U_R diag(sig).  Outputs sorted descending: sig (l doubles), U_R and W
// in element type To (lp x lp, zero padded, ld lp).
// Above one SM's shared memory (float32: l > 160; float64: l > 112) X and V live in
// `scratch` (jacobi_scratch_bytes(l, sizeof(Ta)) bytes), l <= 288 (float32).
template <typename Ta, typename To>
cudaError_t jacobi_osvd(const double *R, int l, int lp, double *sig, To *UR, To *W, int *status,
                        cudaStream_t s, void *scratch = nullptr);
size_t jacobi_scratch_bytes(int l, size_t ta);

// Float64 Rayleigh-quotient refinement of the singular values returned by
// jacobi_osvd: sig[i] = u_i^T R w_i / (||u_i|| ||w_i||) (R upper triangular or
// bidiagonal, l x l, ld l; UR, W ld lp).
template <typename To>
cudaError_t sv_refine(const double *R, int l, int lp, const To *UR, const To *W, double *sig, cudaStream_t s);

// Float64 SVD of R from the float32 jacobi_osvd result: two Newton-type refinement steps
// (Ogita-Aishima) built from l x l float64 products update U_R and W (lp x lp float32,
// in place: rounded back at the end) and give sig, the float64 singular values,
// descending.  ws: svd_refine64_bytes(l) bytes; l <= 4096.
size_t svd_refine64_bytes(int l);
cudaError_t svd_refine64(const double *R, int l, int lp, float *UR, float *W, double *sig, double *ws,
                         cudaStream_t s);

// ------------------------------------------------------ bfloat16 precision form
// Y (m x N) = A Z - 1 c^T with A m x n bfloat16 (lda), Z given as Zt (N x n
// bfloat16, ldz); c (N floats) may be NULL.  n, lda, ldz multiples of 8.
cudaError_t tc16_gemm_nn(int64_t m, int n, int N, const void *A, int64_t lda, const void *Zt, int64_t ldz, float *Y,
                         int64_t ldy, const float *c, int *status, cudaStream_t s);
// C (ncols x N) = A^T (Q_1 + .. + Q_nq) - mu qsum^T with A rows x ncols bfloat16 and
// nq (1 or 3) bfloat16 terms Q_i rows x N (ldq); mu (ncols floats) / qsum (N doubles)
// optional.  part: tc16_gemm_tn_partials floats.
int64_t tc16_gemm_tn_partials(int64_t rows, int ncols, int N);
cudaError_t tc16_gemm_tn(int64_t rows, int ncols, int N, const void *A, int64_t lda, const void *const *Q, int nq,
                         int64_t ldq, float *C, int64_t ldc, float *part, int64_t part_elems, const float *mu,
                         const double *qsum, int *status, cudaStream_t s, const float *cs = nullptr);
// e4m3 forms (A and the small operand as e4m3 codes, float32 accumulation):
//   Y = (A Zq) diag(ts) - 1 c^T                     (ts, c: N floats, optional)
//   C = diag(cs) (A^T Qq) diag(qs) - mu qsum^T      (cs: ncols, qs: N floats; mu, qsum optional)
// n and the leading dimensions multiples of 16.
cudaError_t tc8_gemm_nn(int64_t m, int n, int N, const void *A, int64_t lda, const void *Zt, int64_t ldz, float *Y,
                        int64_t ldy, const float *ts, const float *c, int *status, cudaStream_t s);
int64_t tc8_gemm_tn_partials(int64_t rows, int ncols, int N);
cudaError_t tc8_gemm_tn(int64_t rows, int ncols, int N, const void *A, int64_t lda, const void *Q, int64_t ldq,
                        float *C, int64_t ldc, float *part, int64_t part_elems, const float *cs, const float *qs,
                        const float *mu, const double *qsum, int *status, cudaStream_t s);
// column statistics of a bfloat16 matrix (psum / psq: colstats16_chunks(m) x n doubles, colv: n doubles)
int64_t colstats16_chunks(int64_t m);
cudaError_t colstats16(const void *A, int64_t m, int64_t n, int64_t lda, bool center, double *mu, float *mu_f,
                       double *fro2, double *psum, double *psq, double *colv, cudaStream_t s);
// Zt = round(Z)^T padded to lp rows; c = mu^T Zt^T (when mu and c are given)
cudaError_t to_bf16_t(const float *Z, int64_t n, int l, int64_t ldzin, int lp, void *Zt, int64_t ldz,
                      const double *mu, float *c, cudaStream_t s);
// Q -> nq (1 or 3) bfloat16 terms and their column sums qsum (part: split_bf16_chunks(rows) x lp doubles)
int64_t split_bf16_chunks(int64_t rows);
int64_t q_chunk_rows(int64_t rows);
cudaError_t split_bf16(const float *Q, int64_t rows, int lp, int nq, void *Q1, void *Q2, void *Q3, double *part,
                       double *qsum, cudaStream_t s);

// e4m3 counterparts (the stored matrix is A_q diag(scales); see k_prec.cu)
cudaError_t colstats8(const void *A, int64_t m, int64_t n, int64_t lda, bool center, const float *scales, double *mu,
                      float *mu_f, double *fro2, double *psum, double *psq, double *colv, cudaStream_t s);
cudaError_t prep8_small(const float *Z, int64_t n, int l, int64_t ldzin, int lp, const float *scales,
                        const double *mu, void *Zqt, int64_t ldz, float *t, float *c, cudaStream_t s);
// mpart: split_bf16_chunks(rows) x lp floats, part: split_bf16_chunks(rows) x lp doubles
cudaError_t prep8_q(const float *Q, int64_t rows, int lp, void *Qq, float *u, float *mpart, double *part,
                    double *qsum, cudaStream_t s);
cudaError_t e4m3_to_bf16(const void *A, int64_t count, void *B, cudaStream_t s);

// Serving interface of plan.cu (used by server.cu): a batch context on stream bs
// for up to `cap` problems, and one launch of a batch (float32: lockstep; the
// bfloat16 / e4m3 forms: concurrent solves on the problems' streams) followed, per
// problem, by the Sec. 2.4 K selection and an asynchronous copy of three ints
// (status bits, K, reached) to host_out + 3 i (pinned memory).
struct ServeBatch;
ServeBatch *serve_batch_new(cudaStream_t bs, int cap);
void serve_batch_free(ServeBatch *b);
rsvd_status serve_batch_launch(ServeBatch *b, int count, rsvd_plan_t const *plans, const void *const *A,
                               const float *const *sc, const float *const *Om, double *const *S, float *const *U,
                               float *const *V, const double *t, int *host_out);
rsvd_status serve_status(int bits, int reached);

// Batched forms: one launch solves `count` independent problems of the same l, lp;
// problem b takes its pointers from the device table entry b (one CTA per problem,
// sv_refine one CTA per (value, problem)).  Same arithmetic as the single forms,
// so a problem's result does not depend on the batch it is solved in.
struct CholTab {
    const void *G;     // TG, l x l (ldg)
    double *R, *Rinv;  // l x l
    void *Rc;          // Tc, lp x lp
    int *status;
    double coef;       // chol_shift_coef(rows, l, u) of the arithmetic that may shift
    const double *G64; // float64 Gram matrix of the fallback (kCholFallback), or NULL
    int *fb;           // fallback flag (kCholFirst / kCholFallback), or NULL
    double *ws64;      // scratch of the float64 retry of kCholFirst (chol_scratch_bytes(l, 8)), or NULL
};
struct JacTab {
    const double *R;   // l x l
    double *sig;       // l
    void *UR, *W;      // To, lp x lp
    int *status;
};
double chol_shift_coef(int64_t rows, int l, double unit_roundoff);
template <typename TG, typename Tk, typename Tc>
cudaError_t chol_inv_batched(const CholTab *tab, int count, int64_t ldg, int l, int lp, cudaStream_t s,
                             int role = kCholPlain);
template <typename Ta, typename To>
cudaError_t jacobi_osvd_batched(const JacTab *tab, int count, int l, int lp, cudaStream_t s);
template <typename To>
cudaError_t sv_refine_batched(const JacTab *tab, int count, int l, int lp, cudaStream_t s);

// Cyclic (parallel-ordered) two-sided Jacobi eigen-decomposition of the n x n
// symmetric float64 matrix G (ld n): lam descending (n doubles), V (n x n, ld n).
cudaError_t jacobi_eig(const double *G, int n, double *lam, double *V, int *status, cudaStream_t s);
// The same in float32 arithmetic (inputs and outputs float64), rotating a pair only when
// |g_pq| also exceeds floor_rel * max_i g_ii (n <= 112).
cudaError_t jacobi_eig_f32(const double *G, int n, double *lam, double *V, int *status, cudaStream_t s,
                           double floor_rel);

// Symmetric eigen-decomposition of the n x n float64 matrix A (row-major, both triangles;
// overwritten) beyond one CTA (n <= kGramMaxN): lam descending (n doubles), V (n x n, column
// i = eigenvector i).  Householder tridiagonalisation (a cooperative persistent launch with
// bounded grid barriers: ST_TIMEOUT if one gives up), bisection, inverse iteration,
// Gram-Schmidt inside clusters of eigenvalues closer than 1e-8 max|lam| (ST_NOCONV for a
// cluster of more than 512), back-transformation.  ws: eigh_workspace_bytes(n) bytes.
constexpr int kGramMaxN = 4096;
size_t eigh_workspace_bytes(int n);
cudaError_t eigh_large(double *A, int n, double *lam, double *V, int *status, void *ws, cudaStream_t s);
// G64 (n x n, both triangles) = the upper triangle of Gs (ldg) in float64
template <typename T>
cudaError_t symmetrize(const T *Gs, int64_t ldg, int n, double *G64, cudaStream_t s);
// gram_finish for any n (a multi-CTA grid)
template <typename T>
cudaError_t gram_scale(const double *lam, const double *V, int n, double *sig, T *Vs, int *status, cudaStream_t s);

// Vs[:, i] = V[:, i] / sigma_i (zero column when sigma_i <= n eps sigma_1), sigma_i = sqrt(max(lam_i,0)).
template <typename T>
cudaError_t gram_finish(const double *lam, const double *V, int n, double *sig, T *Vs, int *status,
                        cudaStream_t s);

// For each column j < cols of Vt (rows x cols, ld): if its largest-|entry|
// (first one) is negative, negate that column of Vt and of W (wrows, ldw).
template <typename T>
cudaError_t sign_normalize(T *Vt, int64_t rows, int cols, int64_t ldv, T *W, int64_t wrows, int64_t ldw,
                           cudaStream_t s);

// dst[r * ldd + c] = src[r * lds + c] for r < rows, c < cols; zero for cols <= c < cols_pad.
template <typename Ts, typename Td>
cudaError_t copy2d(const Ts *src, int64_t lds, Td *dst, int64_t ldd, int64_t rows, int64_t cols,
                   int64_t cols_pad, cudaStream_t s);

// dst[i] = src[i] for i < count (float64)
cudaError_t copy_f64(const double *src, double *dst, int64_t count, cudaStream_t s);

// K selection (Sec. 2.4 with Eq. sumeigen): *K = minimal count with
// sum sigma_i^2 >= t * fro2; *reached = 0 if not reached within count.
cudaError_t pca_select(const double *sigma, int count, const double *fro2, double t, int *K, int *reached,
                       cudaStream_t s);

// ------------------------------------------------------ tensor-core path
// true when the driver exposes TMA descriptor encoding (cuTensorMapEncodeTiled)
bool tc_available();
// th / tl (N x ldt) = tf32 hi / lo split of Z^T for Z rows x cols row-major (ldz); zero beyond.
cudaError_t tc_split_transpose(const float *Z, int64_t rows, int cols, int64_t ldz, int N, float *th, float *tl,
                               int64_t ldt, cudaStream_t s);
// Y (m x N) = (A - 1 mu^T) Z with Z given as its transposed tf32 split (N x ldb each);
// 3xTF32 on tcgen05.  N in {16, 32, ..., 128}; A, lda*4 and ldb*4 16-byte aligned.
// mu (optional, 16-byte aligned, zero padded to a multiple of 32): column means
// subtracted on the fly.  ctas > 0 caps the persistent grid (tuning; 0 = one CTA per SM).
// upper_b: B is upper triangular (K = N), so a column slice of Y needs only the first
// (end of the slice) columns of A and rows of B.
// ssq (optional, tc_gemm_nn_grid(m, ctas) doubles): per-CTA
// sums of the squared centred entries, i.e. ||A - 1 mu^T||_F^2 in parts.
cudaError_t tc_gemm_nn(int64_t m, int n, int N, const float *A, int64_t lda, const float *Bth, const float *Btl,
                       int64_t ldb, float *Y, int64_t ldy, int *status, cudaStream_t s, const float *mu = nullptr,
                       double *ssq = nullptr, int ctas = 0, bool upper_b = false);
int tc_gemm_nn_grid(int64_t m, int ctas = 0);
// C (ncols x N, ldc) = (A - 1 mu^T)^T Q for A rows x ncols (lda) and Q rows x N (ldq), 3xTF32 on
// tcgen05, split over row chunks into `part` (tc_gemm_tn_partials elements) and
// summed in chunk order.  N in {16, ..., 128}; pointers and leading dimensions 16-byte
// aligned; mu optional (zero padded to a multiple of 128).  upper_c: only the upper
// triangle of C is wanted (a Gram matrix, A = Q, ncols = N): a column slice of C is
// computed for the rows up to its end.
// chk (optional): C is the Gram matrix of a basis of chk_l columns; ST_ORTH goes into *chk when
// an entry of its upper triangle differs from the identity's by more than chk_tol (col0: the
// global index of this call's first column, for column slices).
// Qth, Qtl (optional): Q's transposed tf32 split (tc_split_transpose of Q, N x ldqt, ldqt >= rows,
// 16-byte aligned): the small operand is then read by TMA in the MMA's layout and the kernel's
// workers split only A (about a quarter less time at N = 64).
cudaError_t tc_gemm_tn(int64_t rows, int ncols, int N, const float *A, int64_t lda, const float *Q, int64_t ldq,
                       float *C, int64_t ldc, float *part, int64_t part_elems, int *status, cudaStream_t s,
                       const float *mu = nullptr, int ctas = 0, bool upper_c = false, int *chk = nullptr,
                       int chk_l = 0, double chk_tol = 0.0, int col0 = 0, const float *Qth = nullptr,
                       const float *Qtl = nullptr, int64_t ldqt = 0);
int64_t tc_gemm_tn_partials(int64_t rows, int ncols, int N);
// C (N x N, ldc) = X^T X for a basis X (rows x N, ldx; N in {16, 32, 48, 64}; X and ldx*4
// 16-byte aligned): one pass over X, each 32-row stage split once into tf32 hi / lo and
// transposed into one tile [X_hi^T; X_lo^T] whose product with itself (one 128 x 128 MMA
// per K slice) carries the three products of the 3xTF32 sum; per-CTA partials in `part`
// (tc_gram_partials elements), summed in chunk order.  chk / chk_l / chk_tol as tc_gemm_tn.
cudaError_t tc_gram(int64_t rows, int N, const float *X, int64_t ldx, float *C, int64_t ldc, float *part,
                    int64_t part_elems, int *status, cudaStream_t s, int *chk = nullptr, int chk_l = 0,
                    double chk_tol = 0.0);
int64_t tc_gram_partials(int64_t rows, int N);

// ------------------------------------------------------ block Krylov (Sec. 3.1.1)
// B ((jl + l) x lp, ld lp): rows below jl negated in place (they hold C = H^T Y),
// rows jl..jl+l-1 set to [I_l 0]; then H[:, :jl+l] B = Y - H[:, :jl] C when
// H[:, jl:jl+l] holds Y.
template <typename T>
cudaError_t bk_proj_matrix(T *B, int jl, int l, int lp, cudaStream_t s);
// SVQB scaling of a block's Gram eigen-decomposition (lam descending, V l x l,
// column i = eigenvector i): M (lp x lp) = V diag(lam)^{-1/2} on the columns with
// lam_c > tau lam_0, zero columns elsewhere, flag[c] = 1 for those (lp ints).
template <typename T>
cudaError_t svqb_scale(const double *lam, const double *V, int l, int lp, double tau, T *M, int *flag,
                       cudaStream_t s);
// The flagged columns c < l of X (m x lp, ld lp) <- uniform entries in
// [-sqrt(3/m), sqrt(3/m)) from a counter-based generator (SplitMix64) and `seed`.
template <typename T>
cudaError_t bk_fill(T *X, int64_t m, int l, int lp, const int *flag, uint64_t seed, cudaStream_t s);

// ------------------------------------------------------ Golub-Kahan-Lanczos
// y = (A - 1 mu^T) v - beta[0] * uprev (beta / uprev / mu may be NULL)
template <typename T>
cudaError_t gkl_gemv_n(const T *A, int64_t m, int n, int64_t lda, const T *v, const T *beta, const T *uprev, T *y,
                       cudaStream_t s, const T *mu = nullptr);
// z = (A - 1 mu^T)^T u - alpha[0] * vprev (alpha / vprev / mu may be NULL);
// part: gkl_gemv_chunks(m, n) * (n + 1) float64 scratch
// (y, when given, also receives (A - 1 mu^T)^T u; gate, when given, must be non-zero for the launches to run)
template <typename T>
cudaError_t gkl_gemv_t(const T *A, int64_t m, int n, int64_t lda, const T *u, const T *alpha, const T *vprev, T *z,
                       double *part, cudaStream_t s, const T *mu = nullptr, T *y = nullptr, const int *gate = nullptr);
// The one-pass step (float32): w = g - beta uprev and x = (A - 1 mu^T)^T g for g = (A - 1 mu^T) v,
// one read of A; part: gkl_gemv_nt_chunks(m) * (n + 1) doubles.  cudaErrorInvalidValue when
// gkl_one_pass_ok fails (n % 4, n > 4096, alignment).
bool gkl_one_pass_ok(int64_t m, int n, int64_t lda, const void *A);
int64_t gkl_gemv_nt_chunks(int64_t m);
cudaError_t gkl_gemv_nt(const float *A, int64_t m, int n, int64_t lda, const float *v, const float *beta,
                        const float *uprev, float *w, float *x, double *part, cudaStream_t s, const float *mu);
// y_j = (x - beta_{j-1} y_{j-1} - sum_{i<j} coef_i y_i) / alpha_j into row j of Y (ld n),
// z = y_j - alpha_j v_j, flag = whether gemv_t must recompute them (j <= 1024).
cudaError_t gkl_recover(const float *x, float *Y, int j, int n, const float *beta, const float *coef,
                        const float *alpha, const float *vj, float *z, int *flag, cudaStream_t s);
int64_t gkl_gemv_chunks(int64_t m, int n);
int64_t gkl_reorth_blocks(int64_t len);
// (ctot, when given, receives the sum of the two passes' coefficients)
template <typename T>
cudaError_t gkl_reorth_normalize(const T *Bt, int64_t ld, int cnt, T *w, int64_t len, T *coef, T *part, T *sq,
                                 T *nrm, T *out, int *status, cudaStream_t s, T *ctot = nullptr);
template <typename T>
cudaError_t gkl_bidiag(const T *alpha, const T *beta, int steps, double *B, cudaStream_t s);

}  // namespace gbr
