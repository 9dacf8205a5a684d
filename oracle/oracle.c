/*
 * FP64 CPU oracle — TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain loops, float64 throughout, no BLAS.  Each routine follows either the
 * plain definition of the quantity (SVD, eigen-decomposition, Frobenius norm)
 * or the step list of arXiv:1906.12085 in the paper's order.  OpenMP is used
 * only to spread independent output entries over cores; every dot product
 * and sum is still taken in index order.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define AT(M, i, j, ld) (M)[(size_t)(i) * (size_t)(ld) + (size_t)(j)]

static double *dalloc(size_t count) { return (double *)calloc(count ? count : 1, sizeof(double)); }

/* ---------------------------------------------------------------- products */

/* C (m x n) = A (m x kk) * B (kk x n); each C_ij summed over p in order. */
static void mm_nn(int64_t m, int64_t kk, int64_t n, const double *A, int64_t lda,
                  const double *B, int64_t ldb, double *C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++) {
        double *c = &AT(C, i, 0, ldc);
        for (int64_t j = 0; j < n; j++) c[j] = 0.0;
        for (int64_t p = 0; p < kk; p++) {
            const double a = AT(A, i, p, lda);
            const double *b = &AT(B, p, 0, ldb);
            for (int64_t j = 0; j < n; j++) c[j] += a * b[j];
        }
    }
}

/* C (n x l) = A^T B with A stored kk x n and B stored kk x l; each C_ij summed over p in order. */
static void mm_tn(int64_t kk, int64_t n, int64_t l, const double *A, int64_t lda,
                  const double *B, int64_t ldb, double *C, int64_t ldc) {
    const int64_t blk = 32;
#pragma omp parallel for schedule(dynamic)
    for (int64_t c0 = 0; c0 < n; c0 += blk) {
        const int64_t c1 = c0 + blk < n ? c0 + blk : n;
        for (int64_t c = c0; c < c1; c++)
            for (int64_t j = 0; j < l; j++) AT(C, c, j, ldc) = 0.0;
        for (int64_t p = 0; p < kk; p++) {
            const double *b = &AT(B, p, 0, ldb);
            for (int64_t c = c0; c < c1; c++) {
                const double a = AT(A, p, c, lda);
                double *out = &AT(C, c, 0, ldc);
                for (int64_t j = 0; j < l; j++) out[j] += a * b[j];
            }
        }
    }
}

/* ---------------------------------------------------------------- centring */

int orc_center(int64_t m, int64_t n, double *A, double *mu, double *fro2) {
    if (m <= 0 || n <= 0 || !A) return ORC_ERR_ARG;
    double *mean = mu ? mu : dalloc((size_t)n);
    if (!mean) return ORC_ERR_OOM;
    for (int64_t j = 0; j < n; j++) mean[j] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) mean[j] += AT(A, i, j, n);
    for (int64_t j = 0; j < n; j++) mean[j] /= (double)m;
    double f = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) {
            AT(A, i, j, n) -= mean[j];
            f += AT(A, i, j, n) * AT(A, i, j, n);
        }
    if (fro2) *fro2 = f;
    if (!mu) free(mean);
    return ORC_OK;
}

/* ------------------------------------------------------------ Householder */

/* Householder vector for x (len entries, stride): on return v (len) and beta
 * such that (I - beta v v^T) x = -s ||x|| e_1, s = sign(x_0) (sign(0) = +1).
 * Returns the new leading entry. */
static double house(int64_t len, const double *x, int64_t stride, double *v, double *beta) {
    double nrm = 0.0;
    for (int64_t i = 0; i < len; i++) nrm += x[i * stride] * x[i * stride];
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < len; i++) v[i] = x[i * stride];
    if (nrm == 0.0) {
        *beta = 0.0;
        return 0.0;
    }
    const double s = x[0] >= 0.0 ? 1.0 : -1.0;
    v[0] = x[0] + s * nrm;
    double vtv = 0.0;
    for (int64_t i = 0; i < len; i++) vtv += v[i] * v[i];
    *beta = 2.0 / vtv;
    return -s * nrm;
}

/* W[r0.., c0..c1) <- (I - beta v v^T) W[r0.., c0..c1): reflector on rows r0..r0+len-1. */
static void reflect_rows(double *W, int64_t ld, int64_t r0, int64_t len, int64_t c0, int64_t c1,
                         const double *v, double beta) {
    if (beta == 0.0) return;
#pragma omp parallel for schedule(static) if (len * (c1 - c0) > 65536)
    for (int64_t c = c0; c < c1; c++) {
        double w = 0.0;
        for (int64_t i = 0; i < len; i++) w += v[i] * AT(W, r0 + i, c, ld);
        w *= beta;
        for (int64_t i = 0; i < len; i++) AT(W, r0 + i, c, ld) -= w * v[i];
    }
}

/* W[r0..r1, c0..] <- W[r0..r1, c0..] (I - beta v v^T): reflector on columns c0..c0+len-1. */
static void reflect_cols(double *W, int64_t ld, int64_t r0, int64_t r1, int64_t c0, int64_t len,
                         const double *v, double beta) {
    if (beta == 0.0) return;
#pragma omp parallel for schedule(static) if ((r1 - r0) * len > 65536)
    for (int64_t r = r0; r < r1; r++) {
        double w = 0.0;
        for (int64_t j = 0; j < len; j++) w += AT(W, r, c0 + j, ld) * v[j];
        w *= beta;
        for (int64_t j = 0; j < len; j++) AT(W, r, c0 + j, ld) -= w * v[j];
    }
}

int orc_qr(int64_t m, int64_t n, const double *Y, double *Q, double *R) {
    if (m < n || n <= 0 || !Y || !Q) return ORC_ERR_ARG;
    double *W = dalloc((size_t)m * n), *V = dalloc((size_t)m * n), *beta = dalloc((size_t)n);
    if (!W || !V || !beta) { free(W); free(V); free(beta); return ORC_ERR_OOM; }
    memcpy(W, Y, sizeof(double) * (size_t)m * n);
    /* reflector j stored in V[j.., j] (column j, rows j..m-1) */
    double *v = dalloc((size_t)m);
    for (int64_t j = 0; j < n; j++) {
        const double lead = house(m - j, &AT(W, j, j, n), n, v, &beta[j]);
        reflect_rows(W, n, j, m - j, j, n, v, beta[j]);
        if (beta[j] != 0.0) AT(W, j, j, n) = lead;
        for (int64_t i = j; i < m; i++) AT(V, i, j, n) = v[i - j];
    }
    /* thin Q = H_0 ... H_{n-1} [I_n; 0], applied right to left */
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) AT(Q, i, j, n) = (i == j) ? 1.0 : 0.0;
    for (int64_t j = n - 1; j >= 0; j--) {
        for (int64_t i = j; i < m; i++) v[i - j] = AT(V, i, j, n);
        reflect_rows(Q, n, j, m - j, 0, n, v, beta[j]);
    }
    /* sign convention R_ii >= 0 */
    for (int64_t j = 0; j < n; j++) {
        if (AT(W, j, j, n) < 0.0) {
            for (int64_t c = j; c < n; c++) AT(W, j, c, n) = -AT(W, j, c, n);
            for (int64_t i = 0; i < m; i++) AT(Q, i, j, n) = -AT(Q, i, j, n);
        }
    }
    if (R)
        for (int64_t i = 0; i < n; i++)
            for (int64_t c = 0; c < n; c++) AT(R, i, c, n) = (c >= i) ? AT(W, i, c, n) : 0.0;
    free(v); free(W); free(V); free(beta);
    return ORC_OK;
}

/* -------------------------------------------------------------- Golub-Reinsch */

/* Givens pair with c*y + s*z = r, -s*y + c*z = 0. */
static void givens(double y, double z, double *c, double *s, double *r) {
    const double h = hypot(y, z);
    if (h == 0.0) { *c = 1.0; *s = 0.0; *r = 0.0; return; }
    *c = y / h; *s = z / h; *r = h;
}

/* columns a, b of M (rows x ld): (M_a, M_b) <- (c M_a + s M_b, -s M_a + c M_b) */
static void rot_cols(double *M, int64_t rows, int64_t ld, int64_t a, int64_t b, double c, double s) {
    if (!M) return;
    for (int64_t i = 0; i < rows; i++) {
        const double x = AT(M, i, a, ld), y = AT(M, i, b, ld);
        AT(M, i, a, ld) = c * x + s * y;
        AT(M, i, b, ld) = -s * x + c * y;
    }
}

/* Implicit-shift QR iteration on the upper bidiagonal (d, e), accumulating the
 * left rotations into the columns of U (m x n) and the right ones into V (n x n):
 * Golub-Kahan SVD step with a Wilkinson shift, plus the zero-diagonal chases. */
static int bidiag_qr(int64_t n, double *d, double *e, int64_t m, double *U, double *V) {
    const double eps = DBL_EPSILON;
    double anorm = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double r = fabs(d[i]) + (i < n - 1 ? fabs(e[i]) : 0.0);
        if (r > anorm) anorm = r;
    }
    const double tol = eps * anorm;
    const int64_t maxit = 75 * n + 100;
    int64_t iter = 0;
    int64_t hi = n - 1;
    while (hi > 0) {
        for (int64_t i = 0; i < hi; i++)
            if (fabs(e[i]) <= tol) e[i] = 0.0;
        if (e[hi - 1] == 0.0) { hi--; continue; }
        int64_t lo = hi - 1;
        while (lo > 0 && e[lo - 1] != 0.0) lo--;
        /* a negligible diagonal entry splits the block after its superdiagonal is chased out */
        int64_t z = -1;
        for (int64_t i = lo; i <= hi; i++)
            if (fabs(d[i]) <= tol) { z = i; break; }
        if (z >= 0) {
            d[z] = 0.0;
            double c, s, r;
            if (z < hi) {
                /* rotate rows j and z (j = z+1..hi) to remove the entry of row z */
                double bulge = e[z];
                e[z] = 0.0;
                for (int64_t j = z + 1; j <= hi; j++) {
                    givens(d[j], bulge, &c, &s, &r);
                    d[j] = r;
                    if (j < hi) { bulge = -s * e[j]; e[j] = c * e[j]; }
                    rot_cols(U, m, n, j, z, c, s);
                }
            } else {
                /* d[hi] = 0: rotate columns j and hi (j = hi-1..lo) to remove e[hi-1] */
                double bulge = e[hi - 1];
                e[hi - 1] = 0.0;
                for (int64_t j = hi - 1; j >= lo; j--) {
                    givens(d[j], bulge, &c, &s, &r);
                    d[j] = r;
                    if (j > lo) { bulge = -s * e[j - 1]; e[j - 1] = c * e[j - 1]; }
                    rot_cols(V, n, n, j, hi, c, s);
                }
            }
            continue;
        }
        if (++iter > maxit) return ORC_ERR_NOCONV;
        /* Wilkinson shift: eigenvalue of the trailing 2x2 of B^T B closer to its last entry */
        const double dm = d[hi - 1], dn = d[hi], em = e[hi - 1];
        const double fm = (hi - 1 > lo) ? e[hi - 2] : 0.0;
        const double t11 = dm * dm + fm * fm, t12 = dm * em, t22 = dn * dn + em * em;
        const double delta = 0.5 * (t11 - t22);
        double mu = t22;
        if (t12 != 0.0) {
            const double sg = delta >= 0.0 ? 1.0 : -1.0;
            mu = t22 - t12 * t12 / (delta + sg * hypot(delta, t12));
        }
        double y = d[lo] * d[lo] - mu, zz = d[lo] * e[lo];
        for (int64_t k = lo; k < hi; k++) {
            double c, s, r;
            givens(y, zz, &c, &s, &r);
            if (k > lo) e[k - 1] = r;
            double f = c * d[k] + s * e[k];
            e[k] = -s * d[k] + c * e[k];
            double bulge = s * d[k + 1];
            d[k + 1] = c * d[k + 1];
            d[k] = f;
            rot_cols(V, n, n, k, k + 1, c, s);
            givens(d[k], bulge, &c, &s, &r);
            d[k] = r;
            f = c * e[k] + s * d[k + 1];
            d[k + 1] = -s * e[k] + c * d[k + 1];
            e[k] = f;
            if (k < hi - 1) {
                const double b2 = s * e[k + 1];
                e[k + 1] = c * e[k + 1];
                y = e[k];
                zz = b2;
            }
            rot_cols(U, m, n, k, k + 1, c, s);
        }
    }
    return ORC_OK;
}

/* order singular values descending (non-negative), permuting the columns of U and V */
static void sort_desc(int64_t n, double *S, int64_t mu, int64_t ldu, double *U, int64_t mv, int64_t ldv, double *V) {
    for (int64_t i = 0; i < n; i++) {
        int64_t best = i;
        for (int64_t j = i + 1; j < n; j++)
            if (S[j] > S[best]) best = j;
        if (best != i) {
            double t = S[i]; S[i] = S[best]; S[best] = t;
            if (U)
                for (int64_t r = 0; r < mu; r++) {
                    t = AT(U, r, i, ldu); AT(U, r, i, ldu) = AT(U, r, best, ldu); AT(U, r, best, ldu) = t;
                }
            if (V)
                for (int64_t r = 0; r < mv; r++) {
                    t = AT(V, r, i, ldv); AT(V, r, i, ldv) = AT(V, r, best, ldv); AT(V, r, best, ldv) = t;
                }
        }
    }
}

int orc_svd(int64_t m, int64_t n, const double *A, double *S, double *U, double *V) {
    if (m < n || n <= 0 || !A || !S) return ORC_ERR_ARG;
    double *W = dalloc((size_t)m * n), *d = dalloc((size_t)n), *e = dalloc((size_t)n);
    double *vl = dalloc((size_t)m * n), *bl = dalloc((size_t)n);
    double *vr = dalloc((size_t)n * n), *br = dalloc((size_t)n), *v = dalloc((size_t)m);
    double *Uw = dalloc((size_t)m * n), *Vw = dalloc((size_t)n * n);
    if (!W || !d || !e || !vl || !bl || !vr || !br || !v || !Uw || !Vw) {
        free(W); free(d); free(e); free(vl); free(bl); free(vr); free(br); free(v); free(Uw); free(Vw);
        return ORC_ERR_OOM;
    }
    memcpy(W, A, sizeof(double) * (size_t)m * n);
    /* Householder bidiagonalisation: W = Ub B Vb^T, B upper bidiagonal */
    for (int64_t j = 0; j < n; j++) {
        double lead = house(m - j, &AT(W, j, j, n), n, v, &bl[j]);
        reflect_rows(W, n, j, m - j, j, n, v, bl[j]);
        if (bl[j] != 0.0) AT(W, j, j, n) = lead;
        for (int64_t i = j; i < m; i++) AT(vl, i, j, n) = v[i - j];
        d[j] = AT(W, j, j, n);
        if (j < n - 2) {
            lead = house(n - j - 1, &AT(W, j, j + 1, n), 1, v, &br[j]);
            reflect_cols(W, n, j, m, j + 1, n - j - 1, v, br[j]);
            if (br[j] != 0.0) AT(W, j, j + 1, n) = lead;
            for (int64_t c = j + 1; c < n; c++) AT(vr, j, c, n) = v[c - j - 1];
        }
        if (j < n - 1) e[j] = AT(W, j, j + 1, n);
    }
    /* Ub = H_0 ... H_{n-1} [I_n; 0] and Vb = P_0 ... P_{n-3}, applied right to left */
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) AT(Uw, i, j, n) = (i == j) ? 1.0 : 0.0;
    for (int64_t j = n - 1; j >= 0; j--) {
        for (int64_t i = j; i < m; i++) v[i - j] = AT(vl, i, j, n);
        reflect_rows(Uw, n, j, m - j, 0, n, v, bl[j]);
    }
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) AT(Vw, i, j, n) = (i == j) ? 1.0 : 0.0;
    for (int64_t j = n - 3; j >= 0; j--) {
        for (int64_t c = j + 1; c < n; c++) v[c - j - 1] = AT(vr, j, c, n);
        reflect_rows(Vw, n, j + 1, n - j - 1, 0, n, v, br[j]);
    }
    int st = bidiag_qr(n, d, e, m, Uw, Vw);
    for (int64_t i = 0; i < n; i++)
        if (d[i] < 0.0) {
            d[i] = -d[i];
            for (int64_t r = 0; r < n; r++) AT(Vw, r, i, n) = -AT(Vw, r, i, n);
        }
    sort_desc(n, d, m, n, Uw, n, n, Vw);
    for (int64_t i = 0; i < n; i++) S[i] = d[i];
    if (U) memcpy(U, Uw, sizeof(double) * (size_t)m * n);
    if (V) memcpy(V, Vw, sizeof(double) * (size_t)n * n);
    free(W); free(d); free(e); free(vl); free(bl); free(vr); free(br); free(v); free(Uw); free(Vw);
    return st;
}

/* ------------------------------------------------------------------- Jacobi */

int orc_eig_jacobi(int64_t n, const double *G, double *lam, double *V, int *sweeps) {
    if (n <= 0 || !G || !lam) return ORC_ERR_ARG;
    double *a = dalloc((size_t)n * n), *v = dalloc((size_t)n * n);
    if (!a || !v) { free(a); free(v); return ORC_ERR_OOM; }
    memcpy(a, G, sizeof(double) * (size_t)n * n);
    for (int64_t i = 0; i < n; i++) AT(v, i, i, n) = 1.0;
    const double rel = 1e-15;
    const int maxsweep = 50;
    int sw = 0, converged = 0;
    for (sw = 0; sw < maxsweep; sw++) {
        int rotated = 0;
        for (int64_t p = 0; p < n - 1; p++)
            for (int64_t q = p + 1; q < n; q++) {
                const double apq = AT(a, p, q, n);
                const double app = AT(a, p, p, n), aqq = AT(a, q, q, n);
                if (fabs(apq) <= rel * sqrt(fabs(app * aqq)) || apq == 0.0) continue;
                rotated = 1;
                /* J = [c s; -s c] in (p, q) with (J^T a J)_pq = 0 */
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int64_t r = 0; r < n; r++) { /* a <- a J */
                    const double x = AT(a, r, p, n), y = AT(a, r, q, n);
                    AT(a, r, p, n) = c * x - s * y;
                    AT(a, r, q, n) = s * x + c * y;
                }
                for (int64_t r = 0; r < n; r++) { /* a <- J^T a */
                    const double x = AT(a, p, r, n), y = AT(a, q, r, n);
                    AT(a, p, r, n) = c * x - s * y;
                    AT(a, q, r, n) = s * x + c * y;
                }
                for (int64_t r = 0; r < n; r++) { /* v <- v J */
                    const double x = AT(v, r, p, n), y = AT(v, r, q, n);
                    AT(v, r, p, n) = c * x - s * y;
                    AT(v, r, q, n) = s * x + c * y;
                }
            }
        if (!rotated) { converged = 1; break; }
    }
    for (int64_t i = 0; i < n; i++) lam[i] = AT(a, i, i, n);
    sort_desc(n, lam, 0, 0, NULL, n, n, v);
    if (V) memcpy(V, v, sizeof(double) * (size_t)n * n);
    if (sweeps) *sweeps = sw;
    free(a); free(v);
    return converged ? ORC_OK : ORC_ERR_NOCONV;
}

/* ---------------------------------------------------------------- Gram route */

int orc_svd_gram(int64_t m, int64_t n, const double *A, double *S, double *U, double *V) {
    if (m < n || n <= 0 || !A || !S) return ORC_ERR_ARG;
    double *G = dalloc((size_t)n * n), *lam = dalloc((size_t)n), *Vw = dalloc((size_t)n * n);
    if (!G || !lam || !Vw) { free(G); free(lam); free(Vw); return ORC_ERR_OOM; }
    mm_tn(m, n, n, A, n, A, n, G, n);                 /* step 1: A^T A */
    int st = orc_eig_jacobi(n, G, lam, Vw, NULL);     /* step 2: eigen-decomposition */
    for (int64_t i = 0; i < n; i++) S[i] = sqrt(lam[i] > 0.0 ? lam[i] : 0.0); /* step 3 */
    if (U) {                                           /* step 4: u_i = A v_i / sigma_i */
        mm_nn(m, n, n, A, n, Vw, n, U, n);
        for (int64_t i = 0; i < m; i++)
            for (int64_t j = 0; j < n; j++) AT(U, i, j, n) = S[j] > 0.0 ? AT(U, i, j, n) / S[j] : 0.0;
    }
    if (V) memcpy(V, Vw, sizeof(double) * (size_t)n * n);
    free(G); free(lam); free(Vw);
    return st;
}

/* ------------------------------------------------------------ randomized PCA */

int orc_rsvd(int64_t m, int64_t n, const double *A, int64_t l, int q,
             const double *Omega, int64_t k, double *S, double *U, double *V) {
    if (l <= 0 || l > n || n > m || k <= 0 || k > l || q < 0 || !A || !Omega || !S) return ORC_ERR_ARG;
    double *Y = dalloc((size_t)m * l), *Q = dalloc((size_t)m * l), *Z = dalloc((size_t)n * l);
    double *Qz = dalloc((size_t)n * l), *T = dalloc((size_t)n * l), *sg = dalloc((size_t)l);
    double *Vt = dalloc((size_t)n * l), *W = dalloc((size_t)l * l), *Ut = dalloc((size_t)m * l);
    int st = ORC_ERR_OOM;
    if (!Y || !Q || !Z || !Qz || !T || !sg || !Vt || !W || !Ut) goto done;
    mm_nn(m, n, l, A, n, Omega, l, Y, l);                    /* H(0) = A G */
    if ((st = orc_qr(m, l, Y, Q, NULL))) goto done;
    for (int it = 0; it < q; it++) {                          /* H(i) = A (A^T H(i-1)), re-orthonormalised */
        mm_tn(m, n, l, A, n, Q, l, Z, l);
        if ((st = orc_qr(n, l, Z, Qz, NULL))) goto done;
        mm_nn(m, n, l, A, n, Qz, l, Y, l);
        if ((st = orc_qr(m, l, Y, Q, NULL))) goto done;
    }
    mm_tn(m, n, l, A, n, Q, l, T, l);                        /* T = A^T Q */
    if ((st = orc_svd(n, l, T, sg, Vt, W)) < 0) goto done;   /* T = Vt Sigma W^T */
    mm_nn(m, l, l, Q, l, W, l, Ut, l);                       /* U = Q W */
    orc_sign_normalize(m, n, l, Ut, Vt);
    for (int64_t i = 0; i < k; i++) S[i] = sg[i];
    if (U)
        for (int64_t r = 0; r < m; r++)
            for (int64_t j = 0; j < k; j++) AT(U, r, j, k) = AT(Ut, r, j, l);
    if (V)
        for (int64_t r = 0; r < n; r++)
            for (int64_t j = 0; j < k; j++) AT(V, r, j, k) = AT(Vt, r, j, l);
done:
    free(Y); free(Q); free(Z); free(Qz); free(T); free(sg); free(Vt); free(W); free(Ut);
    return st;
}

/* Sec. 3.1.1 (block Krylov): H(0) = A G, H(j) = A (A^T H(j-1)) for j = 1..iters,
 * H = [H(0) | ... | H(iters)], Q = qr(H), T = A^T Q = Vt Sigma W^T, U = Q W.  Each
 * block is re-orthonormalised before it feeds the next (its span, and so the span
 * of H, is that of the printed chain in exact arithmetic); the blocks are kept as
 * the columns of H, whose Householder QR then gives the basis. */
int orc_block_krylov(int64_t m, int64_t n, const double *A, int64_t l, int iters,
                     const double *Omega, int64_t k, double *S, double *U, double *V) {
    const int64_t w = (int64_t)(iters + 1) * l;
    if (l <= 0 || iters < 0 || w > n || n > m || k <= 0 || k > w || !A || !Omega || !S) return ORC_ERR_ARG;
    double *Y = dalloc((size_t)m * l), *Qb = dalloc((size_t)m * l), *Z = dalloc((size_t)n * l);
    double *Qz = dalloc((size_t)n * l), *H = dalloc((size_t)m * w), *Q = dalloc((size_t)m * w);
    double *T = dalloc((size_t)n * w), *sg = dalloc((size_t)w), *Vt = dalloc((size_t)n * w);
    double *W = dalloc((size_t)w * w), *Ut = dalloc((size_t)m * w);
    int st = ORC_ERR_OOM;
    if (!Y || !Qb || !Z || !Qz || !H || !Q || !T || !sg || !Vt || !W || !Ut) goto done;
    mm_nn(m, n, l, A, n, Omega, l, Y, l);                      /* H(0) = A G */
    if ((st = orc_qr(m, l, Y, Qb, NULL))) goto done;
    for (int j = 0; j <= iters; j++) {
        if (j > 0) {                                           /* H(j) = A (A^T H(j-1)) */
            mm_tn(m, n, l, A, n, Qb, l, Z, l);
            if ((st = orc_qr(n, l, Z, Qz, NULL))) goto done;
            mm_nn(m, n, l, A, n, Qz, l, Y, l);
            if ((st = orc_qr(m, l, Y, Qb, NULL))) goto done;
        }
        for (int64_t r = 0; r < m; r++)                        /* block j of H */
            for (int64_t c = 0; c < l; c++) AT(H, r, (int64_t)j * l + c, w) = AT(Qb, r, c, l);
    }
    if ((st = orc_qr(m, w, H, Q, NULL))) goto done;            /* Q = qr(H) */
    mm_tn(m, n, w, A, n, Q, w, T, w);                          /* T = A^T Q */
    if ((st = orc_svd(n, w, T, sg, Vt, W)) < 0) goto done;     /* T = Vt Sigma W^T */
    mm_nn(m, w, w, Q, w, W, w, Ut, w);                         /* U = Q W */
    orc_sign_normalize(m, n, w, Ut, Vt);
    for (int64_t i = 0; i < k; i++) S[i] = sg[i];
    if (U)
        for (int64_t r = 0; r < m; r++)
            for (int64_t j = 0; j < k; j++) AT(U, r, j, k) = AT(Ut, r, j, w);
    if (V)
        for (int64_t r = 0; r < n; r++)
            for (int64_t j = 0; j < k; j++) AT(V, r, j, k) = AT(Vt, r, j, w);
done:
    free(Y); free(Qb); free(Z); free(Qz); free(H); free(Q); free(T); free(sg); free(Vt); free(W); free(Ut);
    return st;
}

/* ------------------------------------------------------ Golub-Kahan-Lanczos */

/* w <- w - B (B^T w), twice (classical Gram-Schmidt applied twice), B rows x cnt, ld */
static void cgs2(int64_t rows, int64_t cnt, const double *B, int64_t ld, double *w) {
    if (cnt <= 0) return;
    double *c = dalloc((size_t)cnt);
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t j = 0; j < cnt; j++) {
            double s = 0.0;
            for (int64_t i = 0; i < rows; i++) s += AT(B, i, j, ld) * w[i];
            c[j] = s;
        }
        for (int64_t i = 0; i < rows; i++) {
            double s = 0.0;
            for (int64_t j = 0; j < cnt; j++) s += AT(B, i, j, ld) * c[j];
            w[i] -= s;
        }
    }
    free(c);
}

static double nrm2(int64_t len, const double *x) {
    double s = 0.0;
    for (int64_t i = 0; i < len; i++) s += x[i] * x[i];
    return sqrt(s);
}

int orc_gkl(int64_t m, int64_t n, const double *A, const double *v1, int steps,
            int64_t k, double *S, double *U, double *V, double *alpha, double *beta) {
    if (steps <= 0 || steps > n || n > m || k <= 0 || k > steps || !A || !v1 || !S) return ORC_ERR_ARG;
    const int64_t s = steps;
    double *Ub = dalloc((size_t)m * s), *Vb = dalloc((size_t)n * (s + 1));
    double *al = dalloc((size_t)s), *be = dalloc((size_t)s);
    double *u = dalloc((size_t)m), *w = dalloc((size_t)n), *x = dalloc((size_t)n);
    double *Bd = dalloc((size_t)s * s), *sg = dalloc((size_t)s), *X = dalloc((size_t)s * s), *Yr = dalloc((size_t)s * s);
    double *Uk = dalloc((size_t)m * s), *Vk = dalloc((size_t)n * s);
    int st = ORC_ERR_OOM;
    if (!Ub || !Vb || !al || !be || !u || !w || !x || !Bd || !sg || !X || !Yr || !Uk || !Vk) goto done;
    {
        const double nv = nrm2(n, v1);
        if (nv == 0.0) { st = ORC_ERR_ARG; goto done; }
        for (int64_t i = 0; i < n; i++) AT(Vb, i, 0, s + 1) = v1[i] / nv;
    }
    for (int64_t j = 0; j < s; j++) {
        /* u = A v_j - beta_{j-1} u_{j-1}, reorthogonalised against u_0..u_{j-1} */
        for (int64_t i = 0; i < n; i++) x[i] = AT(Vb, i, j, s + 1);
        mm_nn(m, n, 1, A, n, x, 1, u, 1);
        if (j > 0)
            for (int64_t i = 0; i < m; i++) u[i] -= be[j - 1] * AT(Ub, i, j - 1, s);
        cgs2(m, j, Ub, s, u);
        al[j] = nrm2(m, u);
        if (al[j] == 0.0) { st = ORC_ERR_BREAKDOWN; goto done; }
        for (int64_t i = 0; i < m; i++) AT(Ub, i, j, s) = u[i] / al[j];
        /* w = A^T u_j - alpha_j v_j, reorthogonalised against v_0..v_j */
        for (int64_t i = 0; i < m; i++) u[i] = AT(Ub, i, j, s);
        mm_tn(m, n, 1, A, n, u, 1, w, 1);
        for (int64_t i = 0; i < n; i++) w[i] -= al[j] * AT(Vb, i, j, s + 1);
        cgs2(n, j + 1, Vb, s + 1, w);
        be[j] = nrm2(n, w);
        if (be[j] == 0.0 && j < s - 1) { st = ORC_ERR_BREAKDOWN; goto done; }
        for (int64_t i = 0; i < n; i++) AT(Vb, i, j + 1, s + 1) = be[j] != 0.0 ? w[i] / be[j] : 0.0;
    }
    /* A V_s = U_s B_s with B_s upper bidiagonal (alpha on the diagonal, beta above) */
    for (int64_t j = 0; j < s; j++) {
        AT(Bd, j, j, s) = al[j];
        if (j + 1 < s) AT(Bd, j, j + 1, s) = be[j];
    }
    if ((st = orc_svd(s, s, Bd, sg, X, Yr)) < 0) goto done;
    mm_nn(m, s, s, Ub, s, X, s, Uk, s);            /* left Ritz vectors U_s X */
    mm_nn(n, s, s, Vb, s + 1, Yr, s, Vk, s);       /* right Ritz vectors V_s Y */
    orc_sign_normalize(m, n, s, Uk, Vk);
    for (int64_t i = 0; i < k; i++) S[i] = sg[i];
    if (U)
        for (int64_t r = 0; r < m; r++)
            for (int64_t j = 0; j < k; j++) AT(U, r, j, k) = AT(Uk, r, j, s);
    if (V)
        for (int64_t r = 0; r < n; r++)
            for (int64_t j = 0; j < k; j++) AT(V, r, j, k) = AT(Vk, r, j, s);
    if (alpha) memcpy(alpha, al, sizeof(double) * (size_t)s);
    if (beta) memcpy(beta, be, sizeof(double) * (size_t)s);
done:
    free(Ub); free(Vb); free(al); free(be); free(u); free(w); free(x);
    free(Bd); free(sg); free(X); free(Yr); free(Uk); free(Vk);
    return st;
}

/* ------------------------------------------------------------ K selection */

int orc_pca_threshold(int64_t count, const double *sigma, double fro2, double t, int64_t *K) {
    if (count <= 0 || !sigma || !K || !(fro2 > 0.0)) return ORC_ERR_ARG;
    double acc = 0.0;
    for (int64_t i = 0; i < count; i++) {
        acc += sigma[i] * sigma[i];
        if (acc >= t * fro2) { *K = i + 1; return ORC_OK; }
    }
    *K = count;
    return ORC_WARN_K_GT_COUNT;
}

void orc_sign_normalize(int64_t m, int64_t n, int64_t k, double *U, double *V) {
    for (int64_t j = 0; j < k; j++) {
        int64_t best = 0;
        for (int64_t i = 1; i < n; i++)
            if (fabs(AT(V, i, j, k)) > fabs(AT(V, best, j, k))) best = i;
        if (AT(V, best, j, k) < 0.0) {
            for (int64_t i = 0; i < n; i++) AT(V, i, j, k) = -AT(V, i, j, k);
            if (U)
                for (int64_t i = 0; i < m; i++) AT(U, i, j, k) = -AT(U, i, j, k);
        }
    }
}


/* ------------------------------------------------ precision-form storage formats
 * Written from the format definitions: every finite value of the target format
 * is enumerated (or bracketed) and the nearest one is chosen by an exact
 * comparison in float64, ties to the even code. */

static double bf16_value(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

double orc_bf16_decode(uint16_t b) { return bf16_value(b); }

uint16_t orc_bf16_encode(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if (x != x) return (uint16_t)((u >> 16) | 0x0040u);  /* NaN stays NaN (quiet) */
    /* the two bfloat16 values bracketing x: the truncation toward zero and the
     * next one away from zero (same sign); both exact in float64 */
    const uint16_t lo = (uint16_t)(u >> 16);
    const uint16_t hi = (uint16_t)(lo + 1);
    if ((u & 0xFFFFu) == 0) return lo;                    /* exactly representable */
    const double v = (double)x, a = bf16_value(lo);
    /* the upper neighbour as if the exponent range were unbounded (IEEE rounding:
     * a value nearer 2^128 than the largest finite bfloat16 overflows to infinity) */
    const double b = ((hi & 0x7FFFu) == 0x7F80u) ? (x < 0.f ? -ldexp(1.0, 128) : ldexp(1.0, 128)) : bf16_value(hi);
    const double da = fabs(v - a), db = fabs(b - v);
    if (da < db) return lo;
    if (db < da) return hi;
    return (lo & 1u) ? hi : lo;                           /* tie: even mantissa */
}

static double e4m3_value(uint8_t c) {
    const int s = c >> 7, e = (c >> 3) & 15, mt = c & 7;
    double v;
    if (e == 0) v = ldexp((double)mt, -9);               /* subnormal: m * 2^-9 */
    else v = ldexp(1.0 + mt / 8.0, e - 7);
    return s ? -v : v;
}

double orc_e4m3_decode(uint8_t c) {
    if ((c & 0x7F) == 0x7F) return NAN;
    return e4m3_value(c);
}

uint8_t orc_e4m3_encode(float x) {
    if (x != x) return 0x7F;
    const double v = fabs((double)x);
    const uint8_t sign = signbit(x) ? 0x80 : 0x00;   /* a zero result keeps the sign of x */
    if (v >= 448.0) return (uint8_t)(sign | 0x7E);        /* saturate to the largest finite */
    int best = 0;
    double bd = v;                                        /* distance to code 0 (value 0) */
    for (int c = 1; c <= 0x7E; c++) {                     /* every non-negative finite code */
        const double d = fabs(e4m3_value((uint8_t)c) - v);
        if (d < bd || (d == bd && (c & 1) == 0 && (best & 1) == 1)) {
            bd = d;
            best = c;
        }
    }
    return (uint8_t)(sign | best);
}

void orc_quantize_bf16(int64_t m, int64_t n, const float *A, int64_t lda, uint16_t *out) {
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) out[i * n + j] = orc_bf16_encode(A[i * lda + j]);
}

void orc_quantize_e4m3(int64_t m, int64_t n, const float *A, int64_t lda, uint8_t *out, float *scales) {
    for (int64_t j = 0; j < n; j++) {
        float amax = 0.f;
        for (int64_t i = 0; i < m; i++) {
            const float a = fabsf(A[i * lda + j]);
            if (a > amax) amax = a;
        }
        volatile float s = amax > 0.f ? amax / 448.0f : 1.0f;   /* float32 division */
        scales[j] = s;
    }
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) {
            volatile float q = A[i * lda + j] / scales[j];        /* rounded to float32 */
            out[i * n + j] = orc_e4m3_encode(q);
        }
}
