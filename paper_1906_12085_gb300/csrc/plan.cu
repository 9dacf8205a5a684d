// Plan object, solver sequencing and the C ABI declared in include/rsvd.h.
//
// Every step of every solve is a kernel of this library launched on the
// plan's stream; the host only sequences launches and reads back status / K.
#include <cuda_runtime.h>
#include <float.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "common.cuh"

using namespace gbr;

namespace {
std::atomic<uint64_t> g_launches{0};
}
void gbr::note_launch(int count) { g_launches.fetch_add((uint64_t)count, std::memory_order_relaxed); }

struct rsvd_plan {
    int64_t m = 0, n = 0;
    int k = 0, p = 0, q = 0, l = 0, lp = 0;  // lp: l padded to a multiple of 16 (zero columns)
    int lpc = 0;                             // widest basis the workspace is sized for (lp, or Wp below)
    // block Krylov plans (Sec. 3.1.1): bk_blocks = i + 1 blocks of l = b columns, W = bk_blocks * l
    // columns in all, Wp = lpc = W padded to a multiple of 16; 0 for the other plans
    int bk_blocks = 0;
    int nx = 0;                              // n if svd_exact is supported (n <= kSmallMaxF64), else 0
    int wide = 0;                            // width of the m-row work buffers
    rsvd_dtype dtype = RSVD_F32;
    cudaStream_t stream = nullptr;
    unsigned flags = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = true;     // false: the workspace belongs to the caller (rsvd_plan_create_in)
    // carved workspace
    double *mu = nullptr, *fro2 = nullptr, *cpart = nullptr;
    void *mu_t = nullptr;        // column means in the element type, zero padded to npad
    int64_t npad = 0;
    double *ssq = nullptr;       // per-CTA partial sums of squares from the sketch product
    void *cvec = nullptr;        // rank-1 correction vectors (CUDA-core fallback)
    double *dsum = nullptr;
    void *Y = nullptr, *Qb = nullptr, *Tmp = nullptr;   // m x wide
    void *Ob = nullptr, *Z = nullptr, *Qz = nullptr, *Tn = nullptr, *Vt = nullptr, *Tmpn = nullptr;  // n x max(lp, nx)
    void *part = nullptr;
    int64_t part_elems = 0;
    void *G = nullptr, *Rinv_c = nullptr, *UR = nullptr, *Wm = nullptr;  // s x s, s = max(lp, nx)
    double *G64 = nullptr, *R1 = nullptr, *R1i = nullptr, *R2 = nullptr, *R2i = nullptr, *Rt = nullptr;
    double *lam = nullptr, *Vfull = nullptr, *sig = nullptr;
    int *status = nullptr, *Kdev = nullptr;
    // CholeskyQR fallback of the float32 bases: breakdown flag of the current factorisation and
    // the split-K partials of the float64 Gram matrix (not used by float64 plans)
    int *fb = nullptr;             // fallback flag of the current factorisation (float32 bases)
    int *dflag = nullptr;          // columns removed by kCholDeflate in the current factorisation (sq ints)
    double *g64part = nullptr;
    unsigned *g64count = nullptr;  // CTA counter of the float64 Gram reduction (kept zero between uses)
    uint64_t nfact = 0;            // factorisations of the current solve (seeds of the column refills)
    void *chol_ws = nullptr, *jac_ws = nullptr;  // global l x l blocks of the small solvers (large l only)
    double *ref64 = nullptr;                     // float64 refinement of the small SVD (float32 storage types)
    void *Hk = nullptr;                          // block Krylov basis, m x Wp
    int *bk_flag = nullptr;                      // block Krylov: directions of a block to refill (lp ints)
    // float32 block Krylov plans: float64 copies of T and its CholeskyQR2 bases (n x Wp) and
    // the split-K partials of their float64 Gram products
    double *t64 = nullptr, *q64a = nullptr, *q64b = nullptr, *part64 = nullptr;
    int64_t part64_elems = 0;
    int last_count = 0;
    // tensor-core path (float32): transposed tf32 split of the small operand, split-K partials
    bool tc = false;
    int nn_ctas = 0, tn_ctas = 0;  // work decomposition of the products (0: defaults; see rsvd_autotune)
    int64_t ldt = 0;          // leading dimension of Bth / Btl (>= max(n, wide), multiple of 4)
    float *Bth = nullptr, *Btl = nullptr;
    float *tcpart = nullptr;
    int64_t tcpart_elems = 0;
    // bfloat16 precision form (dtype RSVD_BF16): A is stored as bfloat16, the m-row and
    // n-row work blocks stay float32; these hold the bfloat16 operands of the products
    void *Ztb = nullptr;                       // lp x ldzb: the small operand of A X, transposed
    int64_t ldzb = 0;
    void *Qb1 = nullptr, *Qb2 = nullptr, *Qb3 = nullptr;   // m x lp: terms of Q for A^T Q
    float *mu_f = nullptr, *c16 = nullptr;    // means (float), mean correction of A X
    double *qsum = nullptr, *qpart = nullptr;  // column sums of the Q terms and their partials
    double *psum = nullptr, *psq = nullptr, *colv = nullptr;  // column statistics scratch
    float *part16 = nullptr;
    int64_t part16_elems = 0;
    // e4m3 form (dtype RSVD_FP8_E4M3): e4m3 operands of the sketch / power products and the
    // bfloat16 copy of the stored codes for the float32-accurate Rayleigh-Ritz product
    void *Zq8 = nullptr, *Qq8 = nullptr, *A16 = nullptr;
    int64_t ldz8 = 0;
    float *t8 = nullptr, *u8 = nullptr, *mpart8 = nullptr, *part8 = nullptr;
    int64_t part8_elems = 0;
    // Golub-Kahan-Lanczos workspace, allocated on the first Krylov solve and grown with `steps`
    void *gkl_ws = nullptr;
    int gkl_cap = 0;
    // Gram route beyond one CTA (n > kSmallMaxF64), allocated on the first such svd_exact
    void *gram_ws = nullptr;
    // row-sharded solves: float64 staging of the partial sums (device, allocated on the first
    // rsvd_sharded) and the host buffer the caller's reduction works on
    double *shard_ws = nullptr;
    std::vector<double> shard_host;
    // CUDA graph of the last rsvd solve, replayed while the caller's pointers and flags repeat
    cudaGraphExec_t graph = nullptr;
    const void *gkey[7] = {};
    unsigned gflags = 0;
    uint64_t glaunches = 0;
    // tracing: event pairs recorded around stage groups while profiling is on
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_stage;
    size_t ev_used = 0;
};

namespace {

size_t esize(rsvd_dtype d) { return d == RSVD_F64 ? 8 : 4; }

struct Carver {
    size_t off = 0;
    char *base = nullptr;
    void *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

void carve(rsvd_plan *P, Carver &c) {
    const size_t es = esize(P->dtype);
    const int64_t m = P->m, n = P->n;
    const int64_t sq = P->lpc > P->nx ? P->lpc : P->nx;  // small square side
    const int64_t nw = sq;                               // width of the n-row buffers
    P->mu = (double *)c.take(sizeof(double) * n);
    P->fro2 = (double *)c.take(sizeof(double));
    {
        int64_t cp = center_partials(m, n);
        const int64_t cq = center_partials(m, P->wide);
        P->cpart = (double *)c.take(sizeof(double) * (cp > cq ? cp : cq));
    }
    P->npad = round_up(n, 128);
    P->mu_t = c.take(es * P->npad);
    P->ssq = (double *)c.take(sizeof(double) * 2048);
    P->cvec = c.take(es * P->wide);
    P->dsum = (double *)c.take(sizeof(double) * (P->wide > n ? P->wide : n));
    // Y and Tmp also hold the transposed split of the basis for the products with A (prod_tn)
    P->Y = c.take(es * round_up(m, 4) * P->wide);
    P->Qb = c.take(es * m * P->wide);
    P->Tmp = c.take(es * round_up(m, 4) * P->wide);
    P->Ob = c.take(es * n * nw);
    P->Z = c.take(es * n * nw);
    P->Qz = c.take(es * n * nw);
    P->Tn = c.take(es * n * nw);
    P->Vt = c.take(es * n * nw);
    P->Tmpn = c.take(es * n * nw);
    // split-K scratch: the largest of the products the solvers issue
    int64_t pe = 0;
    auto upd = [&](int64_t rows, int64_t N, int64_t L) {
        const int64_t e = gemm_tn_partials(rows, N, L);
        if (e > pe) pe = e;
    };
    upd(m, n, P->lpc);         // Z = A^T Q, T = A^T Q
    upd(m, P->lpc, P->lpc);    // Gram of Y
    upd(n, P->lpc, P->lpc);    // Gram of Z, T
    upd(m, P->lp, P->lp);
    for (int j = 1; j < P->bk_blocks; j++) upd(m, (int64_t)j * P->l, P->lp);  // block Krylov projections
    if (P->nx) {
        upd(m, P->nx, P->nx);  // A^T A and Gram of A
    }
    P->part_elems = pe;
    P->part = c.take(es * (pe > 0 ? pe : 1));
    P->G = c.take(es * sq * sq);
    P->Rinv_c = c.take(es * sq * sq);
    P->UR = c.take(es * sq * sq);
    P->Wm = c.take(es * sq * sq);
    P->G64 = (double *)c.take(sizeof(double) * sq * sq);
    P->R1 = (double *)c.take(sizeof(double) * sq * sq);
    P->R1i = (double *)c.take(sizeof(double) * sq * sq);
    P->R2 = (double *)c.take(sizeof(double) * sq * sq);
    P->R2i = (double *)c.take(sizeof(double) * sq * sq);
    P->Rt = (double *)c.take(sizeof(double) * sq * sq);
    P->lam = (double *)c.take(sizeof(double) * sq);
    P->Vfull = (double *)c.take(sizeof(double) * sq * sq);
    P->sig = (double *)c.take(sizeof(double) * (n > sq ? n : sq));
    P->status = (int *)c.take(sizeof(int));
    P->Kdev = (int *)c.take(2 * sizeof(int));
    P->fb = (int *)c.take(sizeof(int));
    P->dflag = (int *)c.take(sizeof(int) * (sq + 1));
    if (P->dtype != RSVD_F64) {  // float64 Gram partials of the widest block the factorisations see
        const int wmax = (int)sq;
        int64_t ge = 0;
        for (int w = 64; w < wmax + 64; w += 64) {  // the partials depend on w through its 64-column tiles
            const int64_t e = gram64_partials(m > n ? m : n, w < wmax ? w : wmax);
            if (e > ge) ge = e;
        }
        P->g64part = (double *)c.take(sizeof(double) * ge);
        P->g64count = (unsigned *)c.take(sizeof(unsigned));
    }
    // l x l blocks of the Cholesky beyond one SM's shared memory (float64 sizing); float32 bases
    // always: the float64 fallback factorisation runs in this scratch
    if (P->lpc > kSmallMaxF64 || P->dtype != RSVD_F64)
        P->chol_ws = c.take(chol_scratch_bytes((int)sq, sizeof(double)));
    if (P->lpc > 160)           // and of the float32 Jacobi
        P->jac_ws = c.take(jacobi_scratch_bytes(P->lpc, sizeof(float)));
    if (P->dtype != RSVD_F64) P->ref64 = (double *)c.take(svd_refine64_bytes((int)P->lpc));
    if (P->bk_blocks) {
        P->Hk = c.take(es * m * P->lpc);
        P->bk_flag = (int *)c.take(sizeof(int) * P->lpc);
        if (P->dtype == RSVD_F32) {
            P->t64 = (double *)c.take(sizeof(double) * n * P->lpc);
            P->q64a = (double *)c.take(sizeof(double) * n * P->lpc);
            P->q64b = (double *)c.take(sizeof(double) * n * P->lpc);
            P->part64_elems = gemm_tn_partials(n, P->lpc, P->lpc);
            P->part64 = (double *)c.take(sizeof(double) * (P->part64_elems > 0 ? P->part64_elems : 1));
        }
    }
    if (P->dtype == RSVD_FP8_E4M3) {
        P->ldz8 = round_up(n, 16);
        P->Zq8 = c.take((size_t)P->lp * P->ldz8);
        P->Qq8 = c.take((size_t)m * P->lp);
        P->A16 = c.take(2 * (size_t)m * n);
        P->t8 = (float *)c.take(sizeof(float) * P->lp);
        P->u8 = (float *)c.take(sizeof(float) * P->lp);
        P->mpart8 = (float *)c.take(sizeof(float) * split_bf16_chunks(m) * P->lp);
        P->part8_elems = tc8_gemm_tn_partials(m, (int)n, P->lp);
        P->part8 = (float *)c.take(sizeof(float) * P->part8_elems);
    }
    if (P->dtype == RSVD_BF16 || P->dtype == RSVD_FP8_E4M3) {
        P->ldzb = round_up(n, 8);
        P->Ztb = c.take(2 * P->lp * P->ldzb);
        P->Qb1 = c.take(2 * m * P->lp);
        P->Qb2 = c.take(2 * m * P->lp);
        P->Qb3 = c.take(2 * m * P->lp);
        P->mu_f = (float *)c.take(sizeof(float) * n);
        P->c16 = (float *)c.take(sizeof(float) * P->lp);
        P->qsum = (double *)c.take(sizeof(double) * P->lp);
        P->qpart = (double *)c.take(sizeof(double) * split_bf16_chunks(m) * P->lp);
        P->psum = (double *)c.take(sizeof(double) * colstats16_chunks(m) * n);
        P->psq = (double *)c.take(sizeof(double) * colstats16_chunks(m) * n);
        P->colv = (double *)c.take(sizeof(double) * n);
        P->part16_elems = tc16_gemm_tn_partials(m, (int)n, P->lp);
        P->part16 = (float *)c.take(sizeof(float) * P->part16_elems);
    }
    if (P->tc) {
        P->ldt = round_up(n > P->wide ? n : P->wide, 4);
        P->Bth = (float *)c.take(sizeof(float) * P->lpc * P->ldt);
        P->Btl = (float *)c.take(sizeof(float) * P->lpc * P->ldt);
        int64_t te = 0;
        auto tupd = [&](int64_t rows, int64_t ncols, int N) {
            const int64_t e = tc_gemm_tn_partials(rows, (int)ncols, N);
            if (e > te) te = e;
        };
        tupd(m, n, P->lpc);
        tupd(m, P->lpc, P->lpc);
        tupd(m, P->lp, P->lp);
        for (int j = 1; j < P->bk_blocks; j++) tupd(m, (int64_t)j * P->l, P->lp);
        P->tcpart_elems = te;
        P->tcpart = (float *)c.take(sizeof(float) * te);
    }
}

// The small SVD of B in float64 (refinement of the float32 Jacobi start): BF16 / e4m3
// plans unless RSVD_FLAG_SMALL_F32, float32 plans when RSVD_FLAG_SMALL_FP64.
bool small_fp64(const rsvd_plan *P) {
    if (P->dtype == RSVD_BF16 || P->dtype == RSVD_FP8_E4M3) return !(P->flags & RSVD_FLAG_SMALL_F32);
    return P->dtype == RSVD_F32 && (P->flags & RSVD_FLAG_SMALL_FP64) && P->ref64;
}

// Records a pair of events around a stage group when tracing is enabled.
struct Span {
    rsvd_plan *P;
    int stage;
    size_t idx = (size_t)-1;
    Span(rsvd_plan *P_, int stage_) : P(P_), stage(stage_) {
        if (!P->prof) return;
        if (P->ev.size() < P->ev_used + 2) {
            for (int i = 0; i < 64; i++) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                P->ev.push_back(e);
            }
            P->ev_stage.resize(P->ev.size() / 2);
        }
        idx = P->ev_used;
        P->ev_used += 2;
        cudaEventRecord(P->ev[idx], P->stream);
    }
    ~Span() {
        if (idx == (size_t)-1) return;
        cudaEventRecord(P->ev[idx + 1], P->stream);
        P->ev_stage[idx / 2] = stage;
    }
};

#define CK(...)                                        \
    do {                                               \
        cudaError_t e_ = (__VA_ARGS__);                \
        if (e_ != cudaSuccess) return RSVD_ERR_CUDA;   \
    } while (0)

template <typename T> constexpr double unit_roundoff();
template <> constexpr double unit_roundoff<float>() { return FLT_EPSILON / 2; }
template <> constexpr double unit_roundoff<double>() { return DBL_EPSILON / 2; }

// Products with the skinny operand on the right.  The float32 plan uses the
// tcgen05 3xTF32 kernels when TMA can address the operands (16-byte aligned
// pointers and rows) and the CUDA-core kernels otherwise; float64 always uses
// the CUDA-core kernels.
inline bool al16(const void *p, int64_t ld, size_t es) {
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && ((ld * (int64_t)es) & 15) == 0;
}

// Y (rows x N) = (X - 1 mu^T) B, B row-major K x N (ldb), N = lp.  mu (element type,
// padded) may be NULL.  When fro2 is given it receives ||X - 1 mu^T||_F^2.
// upper_b: B is upper triangular (the inverse Cholesky factor of CholeskyQR; K = lp).
template <typename T>
cudaError_t prod_nn(rsvd_plan *P, int64_t rows, int64_t K, const T *X, int64_t ldx, const T *B, int64_t ldb, T *Y,
                    int64_t ldy, const T *mu = nullptr, double *fro2 = nullptr, bool upper_b = false) {
    if constexpr (sizeof(T) == 4) {
        if (P->tc && al16(X, ldx, 4) && (ldy % 4) == 0 && K <= P->ldt) {
            cudaError_t e = tc_split_transpose(B, K, P->lp, ldb, P->lp, P->Bth, P->Btl, P->ldt, P->stream);
            if (e == cudaSuccess)
                e = tc_gemm_nn(rows, (int)K, P->lp, X, ldx, P->Bth, P->Btl, P->ldt, Y, ldy, P->status, P->stream, mu,
                               fro2 ? P->ssq : nullptr, P->nn_ctas, upper_b && K == P->lp);
            if (e == cudaSuccess && fro2) e = sum_f64(P->ssq, tc_gemm_nn_grid(rows, P->nn_ctas), fro2, P->stream);
            if (e != cudaErrorInvalidValue) return e;
            cudaGetLastError();
        }
    }
    cudaError_t e = cudaSuccess;
    if (fro2) e = centered_fro2<T>(X, rows, K, ldx, mu ? P->mu : nullptr, fro2, P->cpart, P->stream);
    if (e == cudaSuccess) e = gemm_nn<T>(rows, P->lp, K, X, ldx, B, ldb, Y, ldy, P->stream);
    if (e == cudaSuccess && mu) {  // exact rank-1 correction: Y -= 1 (mu^T B)
        e = vecmat<T>(mu, B, K, P->lp, ldb, (T *)P->cvec, P->stream);
        if (e == cudaSuccess) e = rank1_sub<T>(Y, rows, P->lp, ldy, nullptr, (T *)P->cvec, P->stream);
    }
    return e;
}

// C (ncols x N) = (X - 1 mu^T)^T Q with X rows x ncols (ldx), Q rows x N (ldq), N = lp.
// gram: X = Q and only the upper triangle of C is wanted (CholeskyQR's Gram matrix).
// chk_l > 0 (with gram): C = Q^T Q of a basis of chk_l columns, checked against the identity
// (ST_ORTH beyond the element type's bound; fused into the product's reduction when it runs
// on the tensor cores).
// presplit: Y and Tmp are free (a product with A after the basis Q was formed): on the tensor
// cores Q's transposed tf32 split is written there first and the kernel reads it by TMA.
template <typename T>
cudaError_t prod_tn(rsvd_plan *P, int64_t rows, int64_t ncols, const T *X, int64_t ldx, const T *Q, int64_t ldq,
                    T *C, int64_t ldc, const T *mu = nullptr, bool gram = false, int chk_l = 0,
                    bool presplit = false) {
    const double tol = sizeof(T) == 4 ? kOrthTolF32 : kOrthTolF64;
    if constexpr (sizeof(T) == 4) {
        // the Gram matrix of a basis of at most 64 columns: one split per stage serves both
        // operands (tc_gram)
        if (P->tc && X == Q && ldx == ldq && ncols == P->lp && P->lp <= 64 && al16(X, ldx, 4) &&
            tc_gram_partials(rows, P->lp) <= P->tcpart_elems) {
            cudaError_t e = tc_gram(rows, P->lp, X, ldx, C, ldc, P->tcpart, P->tcpart_elems, P->status, P->stream,
                                    chk_l ? P->status : nullptr, chk_l, tol);
            if (e != cudaErrorInvalidValue) return e;
            cudaGetLastError();
        }
        if (P->tc && al16(X, ldx, 4) && al16(Q, ldq, 4) &&
            tc_gemm_tn_partials(rows, (int)ncols, P->lp) <= P->tcpart_elems) {
            float *qth = nullptr, *qtl = nullptr;
            const int64_t ldqt = round_up(rows, 4);
            if (presplit && rows <= P->m && P->lp <= P->wide) {
                qth = (float *)P->Y;
                qtl = (float *)P->Tmp;
                const cudaError_t e = tc_split_transpose(Q, rows, P->lp, ldq, P->lp, qth, qtl, ldqt, P->stream);
                if (e != cudaSuccess) return e;
            }
            cudaError_t e = tc_gemm_tn(rows, (int)ncols, P->lp, X, ldx, Q, ldq, C, ldc, P->tcpart, P->tcpart_elems,
                                       P->status, P->stream, mu, P->tn_ctas, gram && X == Q && ncols == P->lp,
                                       chk_l ? P->status : nullptr, chk_l, tol, 0, qth, qtl, ldqt);
            if (e != cudaErrorInvalidValue) return e;
            cudaGetLastError();
        }
    }
    cudaError_t e = gemm_tn<T>(rows, ncols, P->lp, X, ldx, Q, ldq, C, ldc, (T *)P->part, P->part_elems, P->stream);
    if (e == cudaSuccess && chk_l) e = orth_check<T>(C, chk_l, ldc, tol, P->status, P->stream);
    if (e == cudaSuccess && mu) {  // exact rank-1 correction: C -= mu (1^T Q)
        e = column_sums<T>(Q, rows, P->lp, ldq, P->dsum, (T *)P->cvec, P->cpart, P->stream);
        if (e == cudaSuccess) e = rank1_sub<T>(C, ncols, P->lp, ldc, mu, (T *)P->cvec, P->stream);
    }
    return e;
}

// The Cholesky of one CholeskyQR pass, R^T R = G with G the Gram matrix of X (rows x w, ld)
// already in P->G.  Float32 bases (every dtype but float64): the float32 factorisation
// (float64 arithmetic when f64) of the float32 Gram matrix; when it breaks down (a basis
// with cond(X) beyond ~1e4, whose float32 Gram matrix is no longer positive definite) the
// Gram matrix is formed again from the float32 X with float64 products and sums and
// factored in float64 (mixed-precision CholeskyQR: it resolves every direction the float32
// data carries; its shift, 11 (rows w + w(w+1)) u64 tr(G), only for exactly dependent
// columns).  The basis of such a pass is then formed as X R^{-1} in float64 too (rinv64_fb in
// cqr), so its error no longer grows with cond(X) times the product's rounding.  The
// fallback launches return at once when the first factorisation succeeded.
// A float32 Cholesky that breaks down is first retried in float64 arithmetic on the same
// float32 Gram matrix (inside the same launch): its rounding, ~l u32 relative to the pivots,
// exceeds the small positive pivots of moderately conditioned bases at large l (measured:
// pivot 263 of 288 at -2.2e-5 G_kk on the 1048576 x 4096 i^-1.5 sketch), which the float64
// arithmetic resolves; only a Gram matrix that is itself indefinite reaches the float64 Gram.
// Float64 bases whose R is not kept (deflate): columns with a pivot below l u64 of their
// squared norm are removed (kCholDeflate) and refilled by the caller; a factorisation whose R
// is kept (T, and A in svd_exact) shifts instead.
template <typename T>
rsvd_status chol_pass(rsvd_plan *P, const T *X, int64_t rows, int w, int ld, bool f64, double *R, double *Ri,
                      T *Ric, bool deflate) {
    // float32 bases whose R is not kept: the float64 fallback removes dependent columns
    // (kCholDeflate; rinv64_fb refills them) instead of shifting
    cudaStream_t s = P->stream;
    const double u64 = DBL_EPSILON / 2;
    if constexpr (sizeof(T) == 4) {
        const float *G = (const float *)P->G;
        if (f64)
            CK(chol_inv<float, double, float>(G, ld, w, rows, u64, R, Ri, Ric, ld, P->status, s, P->chol_ws, P->fb,
                                              kCholFirst));
        else CK(chol_inv<float, float, float>(G, ld, w, rows, u64, R, Ri, Ric, ld, P->status, s, P->chol_ws, P->fb,
                                              kCholFirst));
        const G64Job job = {X,  rows, ld,  P->g64part, P->G64,    P->fb, P->g64count, chol_shift_coef(rows, w, u64),
                            R,  Ri,   Ric, ld,         P->status, (double *)P->chol_ws, deflate ? kCholDeflate : kCholFallback,
                            P->dflag};
        CK(gram64_fb(job, w, ld, s));  // float64 Gram matrix and Cholesky, after a breakdown only
    } else {
        CK(chol_inv<double, double, double>((const double *)P->G, ld, w, rows, u64, R, Ri, Ric, ld, P->status, s,
                                            P->chol_ws, deflate ? P->dflag : nullptr,
                                            deflate ? kCholDeflate : kCholPlain));
    }
    return RSVD_OK;
}

uint64_t refill_seed(rsvd_plan *P) { return 0x2D0C4A5E1ull + 0x9E3779B97F4A7C15ull * ++P->nfact; }

// The columns of a float64 basis that kCholDeflate removed (P->dflag) are replaced by pseudo-
// random ones (SplitMix64 from a per-factorisation seed), which the next CholeskyQR pass
// orthonormalises against the rest.
template <typename T>
rsvd_status refill(rsvd_plan *P, T *Q, int64_t rows, int w, int ld) {
    if constexpr (sizeof(T) == 8) CK(bk_fill<T>(Q, rows, w, ld, P->dflag, refill_seed(P), P->stream));
    return RSVD_OK;
}

// Orthonormality check of a final basis Q (rows x w, ld): G = Q^T Q (upper triangle) and
// ST_ORTH when max |G - I| exceeds the bound of the element type (kOrthTolF32 / F64).
template <typename T>
rsvd_status check_basis(rsvd_plan *P, const T *Q, int64_t rows, int w, int ld) {
    T *G = (T *)P->G;
    if (ld == P->lp) {
        CK(prod_tn<T>(P, rows, ld, Q, ld, Q, ld, G, ld, nullptr, true, w));
    } else {
        CK(gemm_tn<T>(rows, ld, ld, Q, ld, Q, ld, G, ld, (T *)P->part, P->part_elems, P->stream));
        CK(orth_check<T>(G, w, ld, sizeof(T) == 4 ? kOrthTolF32 : kOrthTolF64, P->status, P->stream));
    }
    return RSVD_OK;
}

// CholeskyQR of X (rows x w, ld) with one or two passes: Qo = X R^{-1}.
// Pass 1: R1 = chol(X^T X), Q1 = X R1^{-1}.  Pass 2 (CholeskyQR2): R2 = chol(Q1^T Q1),
// Qo = Q1 R2^{-1}, and R = R2 R1 is written to Rt when want_r.  One pass leaves Qo
// well conditioned (||Qo^T Qo - I|| ~ u cond(X)^2) with exactly the range of X, which
// is all an intermediate power-iteration basis needs; the final basis and the
// factorisation of T use two passes.
template <typename T>
rsvd_status cqr(rsvd_plan *P, const T *X, int64_t rows, int w, int ld, T *Qo, T *Tmp, bool want_r, int passes = 2) {
    cudaStream_t s = P->stream;
    T *G = (T *)P->G, *Ric = (T *)P->Rinv_c, *part = (T *)P->part;
    const bool skinny = ld == P->lp;  // the l-wide blocks of the randomized solver
    rsvd_status st;
    T *Q1 = passes == 2 ? Tmp : Qo;
    // the precision forms factor the Gram matrices of CholeskyQR2 (the final basis and
    // T) in float64; the single-pass re-orthonormalisations inside the power
    // iteration, like the float32 path's, in float32
    const bool f64 = (P->dtype == RSVD_BF16 || P->dtype == RSVD_FP8_E4M3) && passes == 2;
    if (skinny) CK(prod_tn<T>(P, rows, ld, X, ld, X, ld, G, ld, nullptr, true));
    else CK(gemm_tn<T>(rows, ld, ld, X, ld, X, ld, G, ld, part, P->part_elems, s));
    const bool defl = !want_r;  // bases: remove and refill dependent columns (float32: in the fallback only)
    if ((st = chol_pass<T>(P, X, rows, w, ld, f64, P->R1, P->R1i, Ric, defl))) return st;
    if (skinny) CK(prod_nn<T>(P, rows, ld, X, ld, Ric, ld, Q1, ld, nullptr, nullptr, true));
    else CK(gemm_nn<T>(rows, ld, ld, X, ld, Ric, ld, Q1, ld, s));
    // after a fallback: the basis X R^{-1} to float64 accuracy, removed columns refilled (an
    // intermediate basis only carries a range: there only when a column was removed)
    if (sizeof(T) == 4)
        CK(rinv64_fb({(const float *)X, rows, ld, P->R1i, (float *)Q1, P->fb, defl ? P->dflag : nullptr,
                      refill_seed(P), passes == 2 ? nullptr : P->dflag + w}, w, s));
    else if (defl && (st = refill<T>(P, Q1, rows, w, ld))) return st;
    if (passes == 1) return RSVD_OK;
    if (skinny) CK(prod_tn<T>(P, rows, ld, Q1, ld, Q1, ld, G, ld, nullptr, true));
    else CK(gemm_tn<T>(rows, ld, ld, Q1, ld, Q1, ld, G, ld, part, P->part_elems, s));
    if ((st = chol_pass<T>(P, Q1, rows, w, ld, f64, P->R2, P->R2i, Ric, defl))) return st;
    if (skinny) CK(prod_nn<T>(P, rows, ld, Q1, ld, Ric, ld, Qo, ld, nullptr, nullptr, true));
    else CK(gemm_nn<T>(rows, ld, ld, Q1, ld, Ric, ld, Qo, ld, s));
    if (sizeof(T) == 4)
        CK(rinv64_fb({(const float *)Q1, rows, ld, P->R2i, (float *)Qo, P->fb, defl ? P->dflag : nullptr,
                      refill_seed(P), nullptr}, w, s));
    else if (defl && (st = refill<T>(P, Qo, rows, w, ld))) return st;
    if (want_r) CK(trmm_upper(P->R2, P->R1, P->Rt, w, s));
    return RSVD_OK;
}

template <typename T>
rsvd_status cqr2(rsvd_plan *P, const T *X, int64_t rows, int w, int ld, T *Qo, T *Tmp, bool want_r) {
    return cqr<T>(P, X, rows, w, ld, Qo, Tmp, want_r, 2);
}

template <typename T>
rsvd_status center(rsvd_plan *P, T *A) {
    CK(center_columns<T>(A, P->m, P->n, P->n, !(P->flags & RSVD_FLAG_NO_CENTER), P->mu, P->fro2, P->cpart,
                         P->stream));
    return RSVD_OK;
}

// CholeskyQR2 of the float32 T (rows x w, ld) in float64: the Gram matrices are
// accumulated in float64 from the float32 entries (every product exact), so they
// stay positive semidefinite to float64 rounding and the factorisation holds up
// to cond(T) ~ 1e8 (with the breakdown shift beyond).  Qo = float32 Q_T, Rt = R.
rsvd_status cqr2_f64(rsvd_plan *P, const float *X, int64_t rows, int w, int ld, float *Qo) {
    cudaStream_t s = P->stream;
    const double u = DBL_EPSILON / 2;
    double *T = P->t64, *Q1 = P->q64a, *Q2 = P->q64b;
    CK(copy2d<float, double>(X, ld, T, ld, rows, ld, ld, s));
    CK(gemm_tn<double>(rows, ld, ld, T, ld, T, ld, P->G64, ld, P->part64, P->part64_elems, s));
    CK(chol_inv<double, double, double>(P->G64, ld, w, rows, u, P->R1, P->R1i, P->Vfull, ld, P->status, s,
                                        P->chol_ws));
    CK(gemm_nn<double>(rows, ld, ld, T, ld, P->Vfull, ld, Q1, ld, s));
    CK(gemm_tn<double>(rows, ld, ld, Q1, ld, Q1, ld, P->G64, ld, P->part64, P->part64_elems, s));
    CK(chol_inv<double, double, double>(P->G64, ld, w, rows, u, P->R2, P->R2i, P->Vfull, ld, P->status, s,
                                        P->chol_ws));
    CK(gemm_nn<double>(rows, ld, ld, Q1, ld, P->Vfull, ld, Q2, ld, s));
    CK(trmm_upper(P->R2, P->R1, P->Rt, w, s));
    CK(copy2d<double, float>(Q2, ld, Qo, ld, rows, ld, ld, s));
    return RSVD_OK;
}

// The Rayleigh-Ritz steps shared by Sec. 3.1.1 and Sec. 3.1.2 for an orthonormal
// basis Q (m x lp, the plan's current l and lp): T = (A - 1 mu^T)^T Q (= B^T),
// T = Q_T R (CholeskyQR2), R = U_R Sigma W^T (one-sided Jacobi, singular values
// refined in float64), V = Q_T U_R, U = Q W; the leading k triplets.  The float32
// block Krylov solve factors T in float64 (cqr2_f64): its Ritz values span the
// whole Krylov space, far below what a float32 Gram matrix of T resolves.
template <typename T>
rsvd_status ritz_from_t(rsvd_plan *P, const T *Q, double *S, T *U, T *V);

template <typename T>
rsvd_status ritz(rsvd_plan *P, const T *A, const T *mu, const T *Q, double *S, T *U, T *V) {
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n;
    const int l = P->l, lp = P->lp, k = P->k;
    T *Qz = (T *)P->Qz, *Tn = (T *)P->Tn, *Vt = (T *)P->Vt, *Tmpn = (T *)P->Tmpn;
    rsvd_status st;
    {
        Span sp(P, RSVD_STAGE_ORTH);
        if ((st = check_basis<T>(P, Q, m, l, lp))) return st;                  // Q^T Q = I
    }
    {
        Span sp(P, RSVD_STAGE_ATX);
        CK(prod_tn<T>(P, m, n, A, n, Q, lp, Tn, lp, mu, false, 0, !P->bk_blocks));  // T = A^T Q  (= B^T)
    }
    return ritz_from_t<T>(P, Q, S, U, V);
}

// The Rayleigh-Ritz steps after T = (A - 1 mu^T)^T Q (in P->Tn): the SVD of B = T^T
// through T = Q_T R, R = U_R Sigma W^T, then V = Q_T U_R and U = Q W.
template <typename T>
rsvd_status ritz_from_t(rsvd_plan *P, const T *Q, double *S, T *U, T *V) {
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n;
    const int l = P->l, lp = P->lp, k = P->k;
    T *Qz = (T *)P->Qz, *Tn = (T *)P->Tn, *Vt = (T *)P->Vt, *Tmpn = (T *)P->Tmpn;
    rsvd_status st;
    T *UR = (T *)P->UR, *W = (T *)P->Wm;
    {
        Span sp(P, RSVD_STAGE_SMALL);
        if constexpr (sizeof(T) == 4) {
            if (P->bk_blocks) {
                if ((st = cqr2_f64(P, (const float *)Tn, n, l, lp, (float *)Qz))) return st;   // T = Q_T R
            } else if ((st = cqr2<T>(P, Tn, n, l, lp, Qz, Tmpn, true))) {
                return st;
            }
        } else if ((st = cqr2<T>(P, Tn, n, l, lp, Qz, Tmpn, true))) {
            return st;
        }
        if ((st = check_basis<T>(P, Qz, n, l, lp))) return st;                // Q_T^T Q_T = I
        CK(jacobi_osvd<T, T>(P->Rt, l, lp, P->sig, UR, W, P->status, s, P->jac_ws));     // R = U_R Sigma W^T
        if constexpr (sizeof(T) == 4) {
            if (small_fp64(P)) CK(svd_refine64(P->Rt, l, lp, (float *)UR, (float *)W, P->sig, P->ref64, s));
            else CK(sv_refine<T>(P->Rt, l, lp, UR, W, P->sig, s));                 // sigma_i = u_i^T R w_i (float64)
        } else {
            CK(sv_refine<T>(P->Rt, l, lp, UR, W, P->sig, s));
        }
    }
    {
        Span sp(P, RSVD_STAGE_FINISH);
        CK(gemm_nn<T>(n, lp, lp, Qz, lp, UR, lp, Vt, lp, s));                 // Vt = Q_T U_R
        CK(sign_normalize<T>(Vt, n, l, lp, W, l, lp, s));
        CK(gemm_nn<T>(m, k, lp, Q, lp, W, lp, U, k, s));                      // U = Q W (leading k)
        CK(copy2d<T, T>(Vt, lp, V, k, n, k, k, s));
        CK(copy_f64(P->sig, S, k, s));
    }
    P->last_count = k;
    return RSVD_OK;
}

// Sec. 3.1.2 with re-orthonormalised power steps; see rsvd() in include/rsvd.h.
template <typename T>
rsvd_status run_rsvd(rsvd_plan *P, T *A, const T *Omega, double *S, T *U, T *V) {
    cudaStream_t s = P->stream;
    P->nfact = 0;
    const int64_t m = P->m, n = P->n;
    const int l = P->l, lp = P->lp;
    T *Y = (T *)P->Y, *Q = (T *)P->Qb, *Tmp = (T *)P->Tmp;
    T *Ob = (T *)P->Ob, *Z = (T *)P->Z, *Qz = (T *)P->Qz, *Tmpn = (T *)P->Tmpn;
    rsvd_status st;
    // A is read only: its column means mu are subtracted inside every product with A
    const bool centred = !(P->flags & RSVD_FLAG_NO_CENTER);
    const T *mu = centred ? (const T *)P->mu_t : nullptr;
    {
        Span sp(P, RSVD_STAGE_CENTER);
        if (centred) CK(column_means<T>(A, m, n, n, P->mu, (T *)P->mu_t, P->npad, P->cpart, s));
        else CK(cudaMemsetAsync(P->mu, 0, sizeof(double) * n, s));
    }
    CK(copy2d<T, T>(Omega, l, Ob, lp, n, l, lp, s));                          // G padded to lp columns
    {
        Span sp(P, RSVD_STAGE_AX);
        CK(prod_nn<T>(P, m, n, A, n, Ob, lp, Y, lp, mu, P->fro2));             // H(0) = A G, ||A||_F^2
    }
    // re-orthonormalisation after every half step; one CholeskyQR pass for the
    // intermediate bases, two for the final one (see cqr)
    {
        Span sp(P, RSVD_STAGE_ORTH);
        if ((st = cqr<T>(P, Y, m, l, lp, Q, Tmp, false, P->q > 0 ? 1 : 2))) return st;  // Q = orth(H)
    }
    for (int it = 0; it < P->q; it++) {                                      // H(i) = A (A^T H(i-1))
        const bool last = it == P->q - 1;
        {
            Span sp(P, RSVD_STAGE_ATX);
            CK(prod_tn<T>(P, m, n, A, n, Q, lp, Z, lp, mu, false, 0, true));
        }
        {
            Span sp(P, RSVD_STAGE_ORTH);
            if ((st = cqr<T>(P, Z, n, l, lp, Qz, Tmpn, false, 1))) return st;
        }
        {
            Span sp(P, RSVD_STAGE_AX);
            CK(prod_nn<T>(P, m, n, A, n, Qz, lp, Y, lp, mu));
        }
        {
            Span sp(P, RSVD_STAGE_ORTH);
            if ((st = cqr<T>(P, Y, m, l, lp, Q, Tmp, false, last ? 2 : 1))) return st;
        }
    }
    return ritz<T>(P, A, mu, Q, S, U, V);
}

// ---------------------------------------------------------------- row-sharded solve
// Sec. 3.1.2 over a row-block partition A = [A_1; ...; A_N] (one rank per block, this plan
// holding A_r): every product with A is local (Y_r = (A_r - 1 mu^T) Omega, Y_r = (A_r - 1
// mu^T) Z, U_r = Q_r W) and the quantities summed over rows are reduced across ranks by
// the caller's function on the host: the column sums (mu), ||A - 1 mu^T||_F^2, the Gram
// matrices Y^T Y = sum_r Y_r^T Y_r of every CholeskyQR pass and the final check,
// Z = sum_r (A_r - 1 mu^T)^T Q_r and T = sum_r (A_r - 1 mu^T)^T Q_r.  Everything n x l
// or l x l after a reduction (the factorisations of Z and T, the SVD of R, V) is computed
// by every rank from identical inputs.  The reduced Gram matrices are factored in float64
// (shift on breakdown); the fallback tiers of the single-GPU CholeskyQR, which re-read the
// whole basis, are not available here.

struct Reducer {
    rsvd_allreduce_fn fn;
    void *ctx;
};

// dev (count doubles, device) <- its sum over all ranks (through the host; synchronises)
rsvd_status shard_reduce(rsvd_plan *P, const Reducer &r, double *dev, int64_t count) {
    cudaStream_t s = P->stream;
    P->shard_host.resize((size_t)count);
    CK(cudaMemcpyAsync(P->shard_host.data(), dev, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (r.fn(P->shard_host.data(), count, r.ctx) != 0) return RSVD_ERR_REDUCE;
    CK(cudaMemcpyAsync(dev, P->shard_host.data(), sizeof(double) * count, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return RSVD_OK;
}

// X (rows x cols, ld, element type T) <- its sum over all ranks, staged in float64
template <typename T>
rsvd_status shard_reduce_mat(rsvd_plan *P, const Reducer &r, T *X, int64_t rows, int64_t cols, int64_t ld) {
    CK(copy2d<T, double>(X, ld, P->shard_ws, cols, rows, cols, cols, P->stream));
    rsvd_status st = shard_reduce(P, r, P->shard_ws, rows * cols);
    if (st) return st;
    CK(copy2d<double, T>(P->shard_ws, cols, X, ld, rows, cols, cols, P->stream));
    return RSVD_OK;
}

// The global Gram matrix of the distributed basis X (local rows x lp) in P->shard_ws (float64)
template <typename T>
rsvd_status shard_gram(rsvd_plan *P, const Reducer &r, const T *X) {
    const int lp = P->lp;
    T *G = (T *)P->G;
    CK(prod_tn<T>(P, P->m, lp, X, lp, X, lp, G, lp, nullptr, false));
    CK(copy2d<T, double>(G, lp, P->shard_ws, lp, lp, lp, lp, P->stream));
    return shard_reduce(P, r, P->shard_ws, (int64_t)lp * lp);
}

// CholeskyQR (one or two passes) of the distributed basis X: Qo_r = X_r R^{-1} with R the
// Cholesky factor of the reduced Gram matrix (float64, shifted on breakdown)
template <typename T>
rsvd_status shard_cqr(rsvd_plan *P, const Reducer &r, int64_t m_total, const T *X, T *Qo, T *Tmp, int passes) {
    cudaStream_t s = P->stream;
    const int l = P->l, lp = P->lp;
    const double u64 = DBL_EPSILON / 2;
    T *Ric = (T *)P->Rinv_c;
    rsvd_status st;
    const T *in = X;
    for (int pass = 0; pass < passes; pass++) {
        T *out = pass == passes - 1 ? Qo : Tmp;
        if ((st = shard_gram<T>(P, r, in))) return st;
        double *R = pass == 0 ? P->R1 : P->R2, *Ri = pass == 0 ? P->R1i : P->R2i;
        CK(chol_inv<double, double, T>(P->shard_ws, lp, l, m_total, u64, R, Ri, Ric, lp, P->status, s,
                                       P->chol_ws));
        CK(prod_nn<T>(P, P->m, lp, in, lp, Ric, lp, out, lp, nullptr, nullptr, true));
        in = out;
    }
    return RSVD_OK;
}

template <typename T>
rsvd_status run_rsvd_sharded(rsvd_plan *P, int64_t m_total, const T *A, const T *Omega, double *S, T *U, T *V,
                             const Reducer &r) {
    cudaStream_t s = P->stream;
    P->nfact = 0;
    const int64_t m = P->m, n = P->n;
    const int l = P->l, lp = P->lp;
    T *Y = (T *)P->Y, *Q = (T *)P->Qb, *Tmp = (T *)P->Tmp;
    T *Ob = (T *)P->Ob, *Z = (T *)P->Z, *Qz = (T *)P->Qz, *Tmpn = (T *)P->Tmpn, *Tn = (T *)P->Tn;
    rsvd_status st;
    const bool centred = !(P->flags & RSVD_FLAG_NO_CENTER);
    const T *mu = centred ? (const T *)P->mu_t : nullptr;
    if (centred) {
        CK(column_sums<T>(A, m, n, n, P->mu, (T *)P->mu_t, P->cpart, s));        // local column sums
        if ((st = shard_reduce(P, r, P->mu, n))) return st;                       // over all rows
        CK(scale_means<T>(P->mu, n, P->npad, 1.0 / (double)m_total, (T *)P->mu_t, s));
    } else {
        CK(cudaMemsetAsync(P->mu, 0, sizeof(double) * n, s));
    }
    CK(copy2d<T, T>(Omega, l, Ob, lp, n, l, lp, s));
    CK(prod_nn<T>(P, m, n, A, n, Ob, lp, Y, lp, mu, P->fro2));                   // Y_r, ||A_r - 1 mu^T||_F^2
    if ((st = shard_reduce(P, r, P->fro2, 1))) return st;
    if ((st = shard_cqr<T>(P, r, m_total, Y, Q, Tmp, P->q > 0 ? 1 : 2))) return st;
    for (int it = 0; it < P->q; it++) {
        const bool last = it == P->q - 1;
        CK(prod_tn<T>(P, m, n, A, n, Q, lp, Z, lp, mu, false, 0, true));          // Z_r
        if ((st = shard_reduce_mat<T>(P, r, Z, n, lp, lp))) return st;           // Z
        if ((st = cqr<T>(P, Z, n, l, lp, Qz, Tmpn, false, 1))) return st;        // same on every rank
        CK(prod_nn<T>(P, m, n, A, n, Qz, lp, Y, lp, mu));
        if ((st = shard_cqr<T>(P, r, m_total, Y, Q, Tmp, last ? 2 : 1))) return st;
    }
    if ((st = shard_gram<T>(P, r, Q))) return st;                                // Q^T Q = I (global)
    CK(orth_check<double>(P->shard_ws, l, lp, sizeof(T) == 4 ? kOrthTolF32 : kOrthTolF64, P->status, s));
    CK(prod_tn<T>(P, m, n, A, n, Q, lp, Tn, lp, mu, false, 0, true));             // T_r
    if ((st = shard_reduce_mat<T>(P, r, Tn, n, lp, lp))) return st;              // T = A^T Q
    return ritz_from_t<T>(P, Q, S, U, V);
}

// The plan's basis width switched for the Rayleigh-Ritz steps of a block Krylov solve.
struct Width {
    rsvd_plan *P;
    int l0, lp0;
    Width(rsvd_plan *P_, int l, int lp) : P(P_), l0(P_->l), lp0(P_->lp) {
        P->l = l;
        P->lp = lp;
    }
    ~Width() {
        P->l = l0;
        P->lp = lp0;
    }
};

// Sec. 3.1.1 block Krylov method; see rsvd_block_krylov() in include/rsvd.h.  The basis
// of the Krylov space [H(0) | ... | H(i)] is built block by block (block classical
// Gram-Schmidt applied twice, each block orthonormalised by SVQB and CholeskyQR2), so
// it is never formed from nearly dependent power blocks; the Rayleigh-Ritz steps are
// those of the randomized method at width W = (i + 1) b.
template <typename T>
rsvd_status run_block_krylov(rsvd_plan *P, T *A, const T *Omega, double *S, T *U, T *V) {
    cudaStream_t s = P->stream;
    P->nfact = 0;
    const int64_t m = P->m, n = P->n;
    const int b = P->l, lp = P->lp, nb = P->bk_blocks, Wp = P->lpc;
    T *Y = (T *)P->Y, *Qb = (T *)P->Qb, *Tmp = (T *)P->Tmp, *H = (T *)P->Hk;
    T *Ob = (T *)P->Ob, *Z = (T *)P->Z, *Qz = (T *)P->Qz, *Tmpn = (T *)P->Tmpn;
    T *Bp = (T *)P->UR, *M = (T *)P->Wm, *G = (T *)P->G;
    rsvd_status st;
    const bool centred = !(P->flags & RSVD_FLAG_NO_CENTER);
    const T *mu = centred ? (const T *)P->mu_t : nullptr;
    // eigenvalues of a block's Gram matrix below tau lam_1 are not resolved by its
    // rounding (float32: 2^-23); their directions are replaced by random ones
    const double tau = 2.0 * unit_roundoff<T>();
    const uint64_t seed = 0x190612085ull;
    {
        Span sp(P, RSVD_STAGE_CENTER);
        if (centred) CK(column_means<T>(A, m, n, n, P->mu, (T *)P->mu_t, P->npad, P->cpart, s));
        else CK(cudaMemsetAsync(P->mu, 0, sizeof(double) * n, s));
    }
    // Out = X - H_j (H_j^T X) for the first jl columns H_j of the basis: X is copied into
    // the next b columns of H so that one product H[:, :jl+b] [-C; I] applies it
    auto project = [&](const T *X, int jl, T *Out) -> cudaError_t {
        cudaError_t e = copy2d<T, T>(X, lp, H + jl, Wp, m, b, b, s);
        if (e == cudaSuccess) e = prod_tn<T>(P, m, jl, H, Wp, X, lp, Bp, lp);        // C = H_j^T X
        if (e == cudaSuccess) e = bk_proj_matrix<T>(Bp, jl, b, lp, s);               // [-C; I]
        if (e == cudaSuccess) e = prod_nn<T>(P, m, jl + b, H, Wp, Bp, lp, Out, lp);  // X - H_j C
        return e;
    };
    // SVQB (Stathopoulos and Wu, 2002): X^T X = V diag(lam) V^T, Out = X V diag(lam)^{-1/2}
    // on the resolved directions, random columns on the others
    auto svqb = [&](const T *X, T *Out, uint64_t sd) -> cudaError_t {
        cudaError_t e = prod_tn<T>(P, m, lp, X, lp, X, lp, G, lp);                   // the full Gram matrix
        if (e == cudaSuccess) e = copy2d<T, double>(G, lp, P->G64, b, b, b, b, s);
        // float32 plans: float32 Jacobi that leaves pairs below 2^-30 max_i g_ii alone, far below
        // the 2u lam_1 refill threshold (the float64 one in one CTA took ~14 ms per 96 x 96 block)
        if (e == cudaSuccess)
            e = sizeof(T) == 4 ? jacobi_eig_f32(P->G64, b, P->lam, P->Vfull, P->status, s, 0x1.0p-30)
                               : jacobi_eig(P->G64, b, P->lam, P->Vfull, P->status, s);
        if (e == cudaSuccess) e = svqb_scale<T>(P->lam, P->Vfull, b, lp, tau, M, P->bk_flag, s);
        if (e == cudaSuccess) e = prod_nn<T>(P, m, lp, X, lp, M, lp, Out, lp);
        if (e == cudaSuccess) e = bk_fill<T>(Out, m, b, lp, P->bk_flag, sd, s);
        return e;
    };
    CK(copy2d<T, T>(Omega, b, Ob, lp, n, b, lp, s));                          // G padded to lp columns
    {
        Span sp(P, RSVD_STAGE_AX);
        CK(prod_nn<T>(P, m, n, A, n, Ob, lp, Y, lp, mu, P->fro2));             // H(0) = A G, ||A||_F^2
    }
    {
        Span sp(P, RSVD_STAGE_ORTH);
        CK(svqb(Y, Tmp, seed));
        if ((st = cqr<T>(P, Tmp, m, b, lp, Qb, Y, false, 2))) return st;
        CK(copy2d<T, T>(Qb, lp, H, Wp, m, b, b, s));
    }
    for (int j = 1; j < nb; j++) {                // block j spans the new directions of A A^T (block j-1)
        const int jl = j * b;
        {
            Span sp(P, RSVD_STAGE_ATX);
            CK(prod_tn<T>(P, m, n, A, n, Qb, lp, Z, lp, mu));
        }
        {
            Span sp(P, RSVD_STAGE_ORTH);
            if ((st = cqr<T>(P, Z, n, b, lp, Qz, Tmpn, false, 1))) return st;
        }
        {
            Span sp(P, RSVD_STAGE_AX);
            CK(prod_nn<T>(P, m, n, A, n, Qz, lp, Y, lp, mu));
        }
        {
            Span sp(P, RSVD_STAGE_ORTH);
            CK(project(Y, jl, Tmp));
            CK(project(Tmp, jl, Y));
            CK(svqb(Y, Tmp, seed + (uint64_t)j));
            CK(project(Tmp, jl, Y));
            if ((st = cqr<T>(P, Y, m, b, lp, Qb, Tmp, false, 2))) return st;
            CK(copy2d<T, T>(Qb, lp, H + jl, Wp, m, b, b, s));
        }
    }
    Width wd(P, nb * b, Wp);
    return ritz<T>(P, A, mu, H, S, U, V);
}

// Sec. 3.1.2 on a bfloat16-stored A (precision form).  The products with A take
// bfloat16 operands on the tensor cores with float32 accumulation: the small operand
// of the sketch and power products is rounded to bfloat16 (it only spans the
// subspace), the basis Q of the Rayleigh-Ritz product T = A^T Q is split into three
// bfloat16 terms (float32-accurate against the stored A); the column means enter as
// exact rank-1 corrections of each product.  The Cholesky of CholeskyQR2 (final basis
// and T) runs in float64, that of the single-pass power-step bases in float32; the SVD
// of R is a one-sided Jacobi whose values are recomputed in float64.
rsvd_status run_rsvd_bf16(rsvd_plan *P, const void *A, const float *Omega, double *S, float *U, float *V) {
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n;
    const int l = P->l, lp = P->lp, k = P->k;
    float *Y = (float *)P->Y, *Q = (float *)P->Qb, *Tmp = (float *)P->Tmp;
    float *Z = (float *)P->Z, *Qz = (float *)P->Qz, *Tn = (float *)P->Tn, *Vt = (float *)P->Vt;
    float *Tmpn = (float *)P->Tmpn;
    const bool centred = !(P->flags & RSVD_FLAG_NO_CENTER);
    rsvd_status st;
    {
        Span sp(P, RSVD_STAGE_CENTER);
        CK(colstats16(A, m, n, n, centred, P->mu, P->mu_f, P->fro2, P->psum, P->psq, P->colv, s));
    }
    const double *mu = centred ? P->mu : nullptr;
    const float *muf = centred ? P->mu_f : nullptr;
    const void *q1[3] = {P->Qb1, P->Qb2, P->Qb3};
    auto ax = [&](const float *Zs, int64_t ldzs) -> rsvd_status {  // Y = (A - 1 mu^T) round(Zs)
        Span sp(P, RSVD_STAGE_AX);
        CK(to_bf16_t(Zs, n, l, ldzs, lp, P->Ztb, P->ldzb, mu, P->c16, s));
        CK(tc16_gemm_nn(m, (int)n, lp, A, n, P->Ztb, P->ldzb, Y, lp, mu ? P->c16 : nullptr, P->status, s));
        return RSVD_OK;
    };
    auto atx = [&](int nq, float *Out) -> rsvd_status {  // Out = (A - 1 mu^T)^T (sum of the nq terms of Q)
        Span sp(P, RSVD_STAGE_ATX);
        CK(split_bf16(Q, m, lp, nq, P->Qb1, P->Qb2, P->Qb3, P->qpart, P->qsum, s));
        CK(tc16_gemm_tn(m, (int)n, lp, A, n, q1, nq, lp, Out, lp, P->part16, P->part16_elems, muf,
                        muf ? P->qsum : nullptr, P->status, s));
        return RSVD_OK;
    };
    if ((st = ax(Omega, l))) return st;
    {
        Span sp(P, RSVD_STAGE_ORTH);
        if ((st = cqr<float>(P, Y, m, l, lp, Q, Tmp, false, P->q > 0 ? 1 : 2))) return st;
    }
    for (int it = 0; it < P->q; it++) {
        const bool last = it == P->q - 1;
        if ((st = atx(1, Z))) return st;
        {
            Span sp(P, RSVD_STAGE_ORTH);
            if ((st = cqr<float>(P, Z, n, l, lp, Qz, Tmpn, false, 1))) return st;
        }
        if ((st = ax(Qz, lp))) return st;
        {
            Span sp(P, RSVD_STAGE_ORTH);
            if ((st = cqr<float>(P, Y, m, l, lp, Q, Tmp, false, last ? 2 : 1))) return st;
        }
    }
    {
        Span sp(P, RSVD_STAGE_ORTH);
        if ((st = check_basis<float>(P, Q, m, l, lp))) return st;
    }
    if ((st = atx(3, Tn))) return st;  // T = A^T Q, float32-accurate
    float *UR = (float *)P->UR, *W = (float *)P->Wm;
    {
        Span sp(P, RSVD_STAGE_SMALL);
        if ((st = cqr2<float>(P, Tn, n, l, lp, Qz, Tmpn, true))) return st;
        if ((st = check_basis<float>(P, Qz, n, l, lp))) return st;
        // float32 rotations (the float64 rate of this GPU is 1/58 of float32: a float64
        // Jacobi of l = 112 takes ~50 ms), then the float64 refinement built from l x l
        // products over all SMs (or float64 Rayleigh-quotient values only)
        CK(jacobi_osvd<float, float>(P->Rt, l, lp, P->sig, UR, W, P->status, s, P->jac_ws));
        if (small_fp64(P)) CK(svd_refine64(P->Rt, l, lp, UR, W, P->sig, P->ref64, s));
        else CK(sv_refine<float>(P->Rt, l, lp, UR, W, P->sig, s));
    }
    {
        Span sp(P, RSVD_STAGE_FINISH);
        CK(gemm_nn<float>(n, lp, lp, Qz, lp, UR, lp, Vt, lp, s));
        CK(sign_normalize<float>(Vt, n, l, lp, W, l, lp, s));
        CK(gemm_nn<float>(m, k, lp, Q, lp, W, lp, U, k, s));
        CK(copy2d<float, float>(Vt, lp, V, k, n, k, k, s));
        CK(copy_f64(P->sig, S, k, s));
    }
    P->last_count = k;
    return RSVD_OK;
}

// Sec. 3.1.2 on an e4m3-stored A = A_q diag(s) (precision form).  The sketch and power
// products take e4m3 operands (kind::f8f6f4, float32 accumulation): the small operand
// diag(s) Z and the basis Q are quantised per column with their own scales, which the
// epilogues multiply back; the Rayleigh-Ritz product T = A^T Q runs on the exact
// bfloat16 copy of the codes with Q split into three bfloat16 terms and diag(s)
// applied to the sum.  Means, CholeskyQR and the small SVD as for bfloat16.
rsvd_status run_rsvd_fp8(rsvd_plan *P, const void *A, const float *sc, const float *Omega, double *S, float *U,
                         float *V) {
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n;
    const int l = P->l, lp = P->lp, k = P->k;
    float *Y = (float *)P->Y, *Q = (float *)P->Qb, *Tmp = (float *)P->Tmp;
    float *Z = (float *)P->Z, *Qz = (float *)P->Qz, *Tn = (float *)P->Tn, *Vt = (float *)P->Vt;
    float *Tmpn = (float *)P->Tmpn;
    const bool centred = !(P->flags & RSVD_FLAG_NO_CENTER);
    rsvd_status st;
    {
        Span sp(P, RSVD_STAGE_CENTER);
        CK(colstats8(A, m, n, n, centred, sc, P->mu, P->mu_f, P->fro2, P->psum, P->psq, P->colv, s));
    }
    const double *mu = centred ? P->mu : nullptr;
    const float *muf = centred ? P->mu_f : nullptr;
    auto ax = [&](const float *Zs, int64_t ldzs) -> rsvd_status {  // Y = (A - 1 mu^T) Z_eff
        Span sp(P, RSVD_STAGE_AX);
        CK(prep8_small(Zs, n, l, ldzs, lp, sc, mu, P->Zq8, P->ldz8, P->t8, P->c16, s));
        CK(tc8_gemm_nn(m, (int)n, lp, A, n, P->Zq8, P->ldz8, Y, lp, P->t8, mu ? P->c16 : nullptr, P->status, s));
        return RSVD_OK;
    };
    auto atx = [&](float *Out) -> rsvd_status {  // Out = (A - 1 mu^T)^T Q_eff
        Span sp(P, RSVD_STAGE_ATX);
        CK(prep8_q(Q, m, lp, P->Qq8, P->u8, P->mpart8, P->qpart, P->qsum, s));
        CK(tc8_gemm_tn(m, (int)n, lp, A, n, P->Qq8, lp, Out, lp, P->part8, P->part8_elems, sc, P->u8, muf,
                       muf ? P->qsum : nullptr, P->status, s));
        return RSVD_OK;
    };
    if ((st = ax(Omega, l))) return st;
    {
        Span sp(P, RSVD_STAGE_ORTH);
        if ((st = cqr<float>(P, Y, m, l, lp, Q, Tmp, false, P->q > 0 ? 1 : 2))) return st;
    }
    for (int it = 0; it < P->q; it++) {
        const bool last = it == P->q - 1;
        if ((st = atx(Z))) return st;
        {
            Span sp(P, RSVD_STAGE_ORTH);
            if ((st = cqr<float>(P, Z, n, l, lp, Qz, Tmpn, false, 1))) return st;
        }
        if ((st = ax(Qz, lp))) return st;
        {
            Span sp(P, RSVD_STAGE_ORTH);
            if ((st = cqr<float>(P, Y, m, l, lp, Q, Tmp, false, last ? 2 : 1))) return st;
        }
    }
    {
        Span sp(P, RSVD_STAGE_ORTH);
        if ((st = check_basis<float>(P, Q, m, l, lp))) return st;
    }
    {
        Span sp(P, RSVD_STAGE_ATX);  // T = A^T Q, float32-accurate, on the bfloat16 copy of the codes
        const void *q3[3] = {P->Qb1, P->Qb2, P->Qb3};
        CK(e4m3_to_bf16(A, m * n, P->A16, s));
        CK(split_bf16(Q, m, lp, 3, P->Qb1, P->Qb2, P->Qb3, P->qpart, P->qsum, s));
        CK(tc16_gemm_tn(m, (int)n, lp, P->A16, n, q3, 3, lp, Tn, lp, P->part16, P->part16_elems, muf,
                        muf ? P->qsum : nullptr, P->status, s, sc));
    }
    float *UR = (float *)P->UR, *W = (float *)P->Wm;
    {
        Span sp(P, RSVD_STAGE_SMALL);
        if ((st = cqr2<float>(P, Tn, n, l, lp, Qz, Tmpn, true))) return st;
        if ((st = check_basis<float>(P, Qz, n, l, lp))) return st;
        CK(jacobi_osvd<float, float>(P->Rt, l, lp, P->sig, UR, W, P->status, s, P->jac_ws));
        if (small_fp64(P)) CK(svd_refine64(P->Rt, l, lp, UR, W, P->sig, P->ref64, s));
        else CK(sv_refine<float>(P->Rt, l, lp, UR, W, P->sig, s));
    }
    {
        Span sp(P, RSVD_STAGE_FINISH);
        CK(gemm_nn<float>(n, lp, lp, Qz, lp, UR, lp, Vt, lp, s));
        CK(sign_normalize<float>(Vt, n, l, lp, W, l, lp, s));
        CK(gemm_nn<float>(m, k, lp, Q, lp, W, lp, U, k, s));
        CK(copy2d<float, float>(Vt, lp, V, k, n, k, k, s));
        CK(copy_f64(P->sig, S, k, s));
    }
    P->last_count = k;
    return RSVD_OK;
}

// Sec. 2.3 / Sec. 3.1.3 Gram route, and the CholeskyQR2 + one-sided Jacobi route.
template <typename T>
rsvd_status run_exact(rsvd_plan *P, T *A, int method, double *S, T *U, T *V) {
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n;
    const int nn = (int)n;
    rsvd_status st;
    {
        Span sp(P, RSVD_STAGE_CENTER);
        if ((st = center<T>(P, A))) return st;
    }
    if (method == RSVD_EXACT_GRAM) {
        T *G = (T *)P->G, *Vs = (T *)P->UR;
        {
            Span sp(P, RSVD_STAGE_ATX);
            CK(gemm_tn<T>(m, n, n, A, n, A, n, G, n, (T *)P->part, P->part_elems, s));  // step 1: A^T A
        }
        {
            Span sp(P, RSVD_STAGE_SMALL);
            CK(copy2d<T, double>(G, n, P->G64, n, n, n, n, s));
            CK(jacobi_eig(P->G64, nn, P->lam, P->Vfull, P->status, s));              // step 2: eigen-decomposition
            CK(gram_finish<T>(P->lam, P->Vfull, nn, P->sig, Vs, P->status, s));       // step 3: sigma = sqrt(lambda)
        }
        {
            Span sp(P, RSVD_STAGE_AX);
            CK(gemm_nn<T>(m, n, n, A, n, Vs, n, U, n, s));                            // step 4: u_i = A v_i / sigma_i
        }
        Span sp(P, RSVD_STAGE_FINISH);
        CK(copy2d<double, T>(P->Vfull, n, V, n, n, n, n, s));
    } else {
        T *Qw = (T *)P->Qb, *Tmp = (T *)P->Tmp, *UR = (T *)P->UR, *W = (T *)P->Wm;
        {
            Span sp(P, RSVD_STAGE_ORTH);
            if ((st = cqr2<T>(P, A, m, nn, nn, Qw, Tmp, true))) return st;           // A = Q R
            if ((st = check_basis<T>(P, Qw, m, nn, nn))) return st;
        }
        {
            Span sp(P, RSVD_STAGE_SMALL);
            if (sizeof(T) == 8) CK(jacobi_osvd<double, T>(P->Rt, nn, nn, P->sig, UR, W, P->status, s));
            else CK(jacobi_osvd<float, T>(P->Rt, nn, nn, P->sig, UR, W, P->status, s));
            CK(sv_refine<T>(P->Rt, nn, nn, UR, W, P->sig, s));
        }
        Span sp(P, RSVD_STAGE_FINISH);
        CK(gemm_nn<T>(m, n, n, Qw, n, UR, n, U, n, s));                               // U = Q U_R
        CK(copy2d<T, T>(W, n, V, n, n, n, n, s));
    }
    {
        Span sp(P, RSVD_STAGE_FINISH);
        CK(sign_normalize<T>(V, n, nn, n, U, m, n, s));
        CK(copy_f64(P->sig, S, n, s));
    }
    P->last_count = nn;
    return RSVD_OK;
}

// The Gram route (Sec. 2.3, Sec. 3.1.3) for n beyond one CTA, the k = n regime of the
// paper's experiments (Sec. 4): G = A^T A (float32 plans on the tensor cores when TMA can
// address A, else CUDA cores), eigen-decomposition in float64 (eigh_large),
// sigma = sqrt(lambda), U = A V Sigma^{-1}.  The workspace (G and V in float64, V Sigma^{-1}
// in the element type, the solver's scratch, the Gram product's partials) is allocated on
// the first call.
struct GramBufs {
    double *G64, *V64, *lam;
    void *Vs, *eig, *part;
    int64_t part_elems;
};

GramBufs gram_carve(rsvd_plan *P, char *base, size_t *bytes) {
    const int64_t n = P->n, m = P->m;
    const size_t es = esize(P->dtype);
    Carver c;
    c.base = base;
    GramBufs b;
    b.G64 = (double *)c.take(sizeof(double) * n * n);
    b.V64 = (double *)c.take(sizeof(double) * n * n);
    b.lam = (double *)c.take(sizeof(double) * n);
    b.Vs = c.take(es * n * n);
    b.eig = c.take(eigh_workspace_bytes((int)n));
    int64_t pe = gemm_tn_partials(m, n, n);
    if (P->dtype == RSVD_F32 && n % 16 == 0) {  // the tensor-core Gram: column slices up to the diagonal
        const int w = column_slice((int)n);
        for (int64_t c0 = 0; c0 < n; c0 += w) {
            const int wn = (int)std::min<int64_t>(w, n - c0);
            pe = std::max(pe, tc_gemm_tn_partials(m, (int)std::min<int64_t>(c0 + wn, n), wn));
        }
    }
    b.part_elems = pe;
    b.part = c.take(es * (pe > 0 ? pe : 1));
    *bytes = c.off;
    return b;
}

template <typename T>
rsvd_status run_exact_large(rsvd_plan *P, T *A, double *S, T *U, T *V) {
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n;
    const int nn = (int)n;
    size_t bytes = 0;
    gram_carve(P, nullptr, &bytes);
    if (!P->gram_ws) {
        if (cudaMalloc(&P->gram_ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            P->gram_ws = nullptr;
            return RSVD_ERR_OOM;
        }
    }
    const GramBufs b = gram_carve(P, (char *)P->gram_ws, &bytes);
    rsvd_status st;
    {
        Span sp(P, RSVD_STAGE_CENTER);
        if ((st = center<T>(P, A))) return st;
    }
    {
        Span sp(P, RSVD_STAGE_ATX);  // step 1: G = A^T A (upper triangle), widened to float64, both triangles
        T *Gs = (T *)b.Vs;           // the n x n buffer of V Sigma^{-1}, free until step 3
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (P->tc && n % 16 == 0 && al16(A, n, 4)) {
                const cudaError_t e = tc_gemm_tn(m, nn, nn, A, n, A, n, Gs, n, (float *)b.part, b.part_elems,
                                                 P->status, s, nullptr, 0, true);
                if (e == cudaSuccess) done = true;
                else if (e != cudaErrorInvalidValue) return RSVD_ERR_CUDA;
                else cudaGetLastError();
            }
        }
        if (!done) CK(gemm_tn<T>(m, n, n, A, n, A, n, Gs, n, (T *)b.part, b.part_elems, s));
        CK(symmetrize<T>(Gs, n, nn, b.G64, s));
    }
    {
        Span sp(P, RSVD_STAGE_SMALL);  // step 2: eigen-decomposition; step 3: sigma = sqrt(lambda)
        CK(eigh_large(b.G64, nn, b.lam, b.V64, P->status, b.eig, s));
        CK(gram_scale<T>(b.lam, b.V64, nn, P->sig, (T *)b.Vs, P->status, s));
    }
    {
        Span sp(P, RSVD_STAGE_AX);  // step 4: u_i = A v_i / sigma_i
        CK(gemm_nn<T>(m, n, n, A, n, (const T *)b.Vs, n, U, n, s));
    }
    {
        Span sp(P, RSVD_STAGE_FINISH);
        CK(copy2d<double, T>(b.V64, n, V, n, n, n, n, s));
        CK(sign_normalize<T>(V, n, nn, n, U, m, n, s));
        CK(copy_f64(P->sig, S, n, s));
    }
    P->last_count = nn;
    return RSVD_OK;
}

// Golub-Kahan-Lanczos with full reorthogonalisation (CGS2), then the SVD of the
// steps x steps bidiagonal and the Ritz vectors; see svd_truncated_krylov().
struct GklBufs {
    void *Ut, *Vt, *w, *z, *part, *coef, *sq, *alpha, *beta, *nrm, *X, *Y;
    double *B, *gpart;
    // the one-pass form (float32): x = A^T A v, the stored y_i = A^T u_i, the summed CGS2
    // coefficients, the second-pass flag and the fused product's partials
    float *x1, *Yr, *ctot;
    int *flag;
    double *ntpart;
};

GklBufs gkl_carve(rsvd_plan *P, int steps, char *base, size_t *bytes) {
    const size_t es = esize(P->dtype);
    const int64_t m = P->m, n = P->n;
    const int64_t sp = round_up(steps, 16);
    const int64_t nblk = std::max(gkl_reorth_blocks(m), gkl_reorth_blocks(n));
    Carver c;
    c.base = base;
    GklBufs b;
    b.Ut = c.take(es * steps * m);
    b.Vt = c.take(es * (steps + 1) * n);
    b.w = c.take(es * m);
    b.z = c.take(es * n);
    b.part = c.take(es * nblk * (steps + 1));
    b.gpart = (double *)c.take(sizeof(double) * gkl_gemv_chunks(m, (int)n) * (n + 1));
    b.coef = c.take(es * (steps + 1));
    b.sq = c.take(es * nblk);
    b.alpha = c.take(es * steps);
    b.beta = c.take(es * steps);
    b.nrm = c.take(es * 2);
    b.X = c.take(es * sp * sp);
    b.Y = c.take(es * sp * sp);
    b.B = (double *)c.take(sizeof(double) * steps * steps);
    b.x1 = (float *)c.take(sizeof(float) * n);
    b.Yr = (float *)c.take(sizeof(float) * steps * n);
    b.ctot = (float *)c.take(sizeof(float) * (steps + 1));
    b.flag = (int *)c.take(sizeof(int));
    b.ntpart = (double *)c.take(sizeof(double) * gkl_gemv_nt_chunks(m) * (n + 1));
    *bytes = c.off;
    return b;
}

template <typename T>
rsvd_status run_gkl(rsvd_plan *P, T *A, const T *v1, int steps, double *S, T *U, T *V) {
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n;
    const int k = P->k, sp = (int)round_up(steps, 16);
    size_t bytes = 0;
    gkl_carve(P, steps, nullptr, &bytes);
    if (steps > P->gkl_cap) {
        if (P->gkl_ws) {
            cudaStreamSynchronize(s);
            cudaFree(P->gkl_ws);
            P->gkl_ws = nullptr;
            P->gkl_cap = 0;
        }
        if (cudaMalloc(&P->gkl_ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            return RSVD_ERR_OOM;
        }
        P->gkl_cap = steps;
    }
    GklBufs b = gkl_carve(P, steps, (char *)P->gkl_ws, &bytes);
    T *Ut = (T *)b.Ut, *Vt = (T *)b.Vt, *w = (T *)b.w, *z = (T *)b.z, *part = (T *)b.part, *coef = (T *)b.coef;
    T *sq = (T *)b.sq, *alpha = (T *)b.alpha, *beta = (T *)b.beta, *nrm = (T *)b.nrm;
    // A is read only: the column means are subtracted inside the products
    const bool centred = !(P->flags & RSVD_FLAG_NO_CENTER);
    const T *mu = centred ? (const T *)P->mu_t : nullptr;
    {
        Span sp_(P, RSVD_STAGE_CENTER);
        if (centred) CK(column_means<T>(A, m, n, n, P->mu, (T *)P->mu_t, P->npad, P->cpart, s));
        CK(centered_fro2<T>(A, m, n, n, centred ? P->mu : nullptr, P->fro2, P->cpart, s));
    }
    {   // v_1 = v1 / ||v1||
        Span sp_(P, RSVD_STAGE_ORTH);
        CK(copy2d<T, T>(v1, 1, z, 1, n, 1, 1, s));
        CK(gkl_reorth_normalize<T>(Vt, n, 0, z, n, coef, part, sq, nrm, Vt, P->status, s));
    }
    // float32: one read of A per step (A^T u_j recovered by linearity, a gated second pass
    // where the recovery would lose accuracy), unless RSVD_FLAG_GKL_TWO_PASS
    bool one = false;
    if constexpr (sizeof(T) == 4)
        one = !(P->flags & RSVD_FLAG_GKL_TWO_PASS) && gkl_one_pass_ok(m, (int)n, n, A) &&
              (reinterpret_cast<uintptr_t>(Vt) & 15) == 0 && n % 4 == 0 &&
              (!mu || (reinterpret_cast<uintptr_t>(mu) & 15) == 0) && steps <= 1024;
    for (int j = 0; j < steps; j++) {
        {
            Span sp_(P, RSVD_STAGE_AX);   // w = A v_j - beta_{j-1} u_{j-1}  (and x = A^T (A v_j) in one pass)
            if constexpr (sizeof(T) == 4) {
                if (one)
                    CK(gkl_gemv_nt(A, m, (int)n, n, Vt + (int64_t)j * n, j ? beta + j - 1 : nullptr,
                                   j ? Ut + (int64_t)(j - 1) * m : nullptr, w, b.x1, b.ntpart, s, mu));
            }
            if (!one)
                CK(gkl_gemv_n<T>(A, m, (int)n, n, Vt + (int64_t)j * n, j ? beta + j - 1 : nullptr,
                                 j ? Ut + (int64_t)(j - 1) * m : nullptr, w, s, mu));
        }
        {
            Span sp_(P, RSVD_STAGE_ORTH);  // CGS2 against u_0..u_{j-1}; alpha_j = ||w||; u_j = w / alpha_j
            CK(gkl_reorth_normalize<T>(Ut, m, j, w, m, coef, part, sq, alpha + j, Ut + (int64_t)j * m, P->status, s,
                                       one ? (T *)b.ctot : nullptr));
        }
        {
            Span sp_(P, RSVD_STAGE_ATX);  // z = A^T u_j - alpha_j v_j
            if constexpr (sizeof(T) == 4) {
                if (one) {
                    CK(gkl_recover(b.x1, b.Yr, j, (int)n, beta, b.ctot, alpha, Vt + (int64_t)j * n, z, b.flag, s));
                    CK(gkl_gemv_t<T>(A, m, (int)n, n, Ut + (int64_t)j * m, alpha + j, Vt + (int64_t)j * n, z, b.gpart,
                                     s, mu, b.Yr + (int64_t)j * n, b.flag));
                }
            }
            if (!one)
                CK(gkl_gemv_t<T>(A, m, (int)n, n, Ut + (int64_t)j * m, alpha + j, Vt + (int64_t)j * n, z, b.gpart, s,
                                 mu));
        }
        {
            Span sp_(P, RSVD_STAGE_ORTH);  // CGS2 against v_0..v_j; beta_j = ||z||; v_{j+1} = z / beta_j
            CK(gkl_reorth_normalize<T>(Vt, n, j + 1, z, n, coef, part, sq, beta + j, Vt + (int64_t)(j + 1) * n,
                                       P->status, s));
        }
    }
    T *X = (T *)b.X, *Y = (T *)b.Y;
    {
        Span sp_(P, RSVD_STAGE_SMALL);  // B = X Sigma Y^T (one-sided Jacobi on the dense bidiagonal)
        CK(gkl_bidiag<T>(alpha, beta, steps, b.B, s));
        if (sizeof(T) == 8) CK(jacobi_osvd<double, T>(b.B, steps, sp, P->sig, X, Y, P->status, s));
        else CK(jacobi_osvd<float, T>(b.B, steps, sp, P->sig, X, Y, P->status, s));
        CK(sv_refine<T>(b.B, steps, sp, X, Y, P->sig, s));
    }
    {
        Span sp_(P, RSVD_STAGE_FINISH);  // Ritz vectors U_s X, V_s Y (leading k)
        CK(gemm_tn<T>(steps, m, k, Ut, m, X, sp, U, k, (T *)P->part, P->part_elems, s));
        CK(gemm_tn<T>(steps, n, k, Vt, n, Y, sp, V, k, (T *)P->part, P->part_elems, s));
        CK(sign_normalize<T>(V, n, k, k, U, m, k, s));
        CK(copy_f64(P->sig, S, k, s));
    }
    P->last_count = k;
    return RSVD_OK;
}

rsvd_status rsvd_direct(rsvd_plan_t P, void *A, const float *sc, const void *Omega, double *S, void *U, void *V) {
    if (P->dtype == RSVD_FP8_E4M3) return run_rsvd_fp8(P, A, sc, (const float *)Omega, S, (float *)U, (float *)V);
    if (P->dtype == RSVD_BF16) return run_rsvd_bf16(P, A, (const float *)Omega, S, (float *)U, (float *)V);
    if (P->dtype == RSVD_F32) return run_rsvd<float>(P, (float *)A, (const float *)Omega, S, (float *)U, (float *)V);
    return run_rsvd<double>(P, (double *)A, (const double *)Omega, S, (double *)U, (double *)V);
}

void drop_graph(rsvd_plan *P) {
    if (P->graph) cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
}

// ------------------------------------------------------------------ batching
// Several independent randomized PCA problems of the same l, lp, q and dtype
// solved in lockstep: each problem's products run on its own plan's stream, and
// at every small dense step (Cholesky of a Gram matrix, Jacobi SVD of R, the
// float64 refinement) the streams join on the batch stream, one batched launch
// solves that step for every problem, and the streams fork again.  Every
// problem runs exactly the kernels (and arithmetic) of a single solve.
struct BatchCtx {
    cudaStream_t bs = nullptr;
    std::vector<cudaEvent_t> ev;  // cap join events + 1 fork event
    cudaEvent_t up = nullptr;     // the last direct-mode table upload (the host table is reused)
    bool up_pending = false;
    void *dtab = nullptr, *htab = nullptr;
    size_t tab_bytes = 0;
    int cap = 0;
    ~BatchCtx() {
        if (up) cudaEventDestroy(up);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (dtab) cudaFree(dtab);
        if (htab) cudaFreeHost(htab);
    }
    // tables: 4 CholTab blocks (rows m / n x pass 1 / 2), one JacTab block and 6 G64Job blocks
    // (which block x pass 1 / 2: the float64 Gram fallback), `count` entries each
    static size_t bytes_for(int count) {
        return (4 * sizeof(CholTab) + sizeof(JacTab) + 6 * sizeof(G64Job)) * (size_t)count;
    }
    cudaError_t reserve(int count) {
        if (count <= cap) return cudaSuccess;
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        if (dtab) cudaFree(dtab);
        if (htab) cudaFreeHost(htab);
        dtab = htab = nullptr;
        cap = 0;
        if (!up && cudaEventCreateWithFlags(&up, cudaEventDisableTiming) != cudaSuccess) return cudaErrorMemoryAllocation;
        ev.resize(count + 1);
        for (auto &e : ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return cudaErrorMemoryAllocation;
        tab_bytes = bytes_for(count);
        if (cudaMalloc(&dtab, tab_bytes) != cudaSuccess) return cudaErrorMemoryAllocation;
        if (cudaMallocHost(&htab, tab_bytes) != cudaSuccess) return cudaErrorMemoryAllocation;
        cap = count;
        return cudaSuccess;
    }
    CholTab *chol(int variant, int count, bool dev) {
        return reinterpret_cast<CholTab *>((char *)(dev ? dtab : htab)) + (size_t)variant * count;
    }
    JacTab *jac(int count, bool dev) {
        return reinterpret_cast<JacTab *>((char *)(dev ? dtab : htab) + 4 * sizeof(CholTab) * (size_t)count);
    }
    G64Job *g64(int variant, int count, bool dev) {
        return reinterpret_cast<G64Job *>((char *)(dev ? dtab : htab) +
                                          (4 * sizeof(CholTab) + sizeof(JacTab)) * (size_t)count) +
               (size_t)variant * count;
    }
};

cudaError_t join(BatchCtx &C, int count, rsvd_plan *const *Ps) {
    for (int i = 0; i < count; i++) {
        if (Ps[i]->stream == C.bs) continue;
        if (cudaEventRecord(C.ev[i], Ps[i]->stream) != cudaSuccess) return cudaErrorUnknown;
        if (cudaStreamWaitEvent(C.bs, C.ev[i], 0) != cudaSuccess) return cudaErrorUnknown;
    }
    return cudaSuccess;
}

cudaError_t fork(BatchCtx &C, int count, rsvd_plan *const *Ps) {
    if (cudaEventRecord(C.ev[count], C.bs) != cudaSuccess) return cudaErrorUnknown;
    for (int i = 0; i < count; i++)
        if (Ps[i]->stream != C.bs && cudaStreamWaitEvent(Ps[i]->stream, C.ev[count], 0) != cudaSuccess)
            return cudaErrorUnknown;
    return cudaSuccess;
}

enum { BQ_Y = 0, BQ_Z = 1, BQ_T = 2 };  // which l-wide block a batched CholeskyQR works on

// Batched form of cqr(): the same products per problem, one batched Cholesky per pass.
template <typename T>
rsvd_status bcqr(BatchCtx &C, int count, rsvd_plan *const *Ps, int which, int passes, bool want_r) {
    const int lp = Ps[0]->lp, l = Ps[0]->l;
    auto bufs = [&](rsvd_plan *P, T *&X, T *&Qo, T *&Tmp, int64_t &rows) {
        if (which == BQ_Y) { X = (T *)P->Y; Qo = (T *)P->Qb; Tmp = (T *)P->Tmp; rows = P->m; }
        else { X = which == BQ_Z ? (T *)P->Z : (T *)P->Tn; Qo = (T *)P->Qz; Tmp = (T *)P->Tmpn; rows = P->n; }
    };
    const int rv = which == BQ_Y ? 0 : 2;  // table block: rows m (0, 1) or rows n (2, 3)
    int64_t max_rows = 0;
    for (int i = 0; i < count; i++) max_rows = std::max(max_rows, which == BQ_Y ? Ps[i]->m : Ps[i]->n);
    for (int pass = 0; pass < passes; pass++) {
        for (int i = 0; i < count; i++) {
            rsvd_plan *P = Ps[i];
            T *X, *Qo, *Tmp;
            int64_t rows;
            bufs(P, X, Qo, Tmp, rows);
            const T *src = pass == 0 ? X : Tmp;
            CK(prod_tn<T>(P, rows, lp, src, lp, src, lp, (T *)P->G, lp));
        }
        CK(join(C, count, Ps));
        const CholTab *tab = C.chol(rv + pass, count, true);
        if constexpr (sizeof(T) == 4) {  // the float32 factorisation, and on a breakdown the float64 one (chol_pass)
            CK(chol_inv_batched<float, float, float>(tab, count, lp, l, lp, C.bs, kCholFirst));
            CK(gram64_fb_batched(C.g64(2 * which + pass, count, true), count, max_rows, l, lp, C.bs));
        } else {  // float64: bases remove dependent columns (refilled below), T shifts (chol_pass)
            CK(chol_inv_batched<T, T, T>(tab, count, lp, l, lp, C.bs, want_r ? kCholPlain : kCholDeflate));
            // (the float64 deflation flags are each problem's dflag: table field fb, see the table fill)
        }
        CK(fork(C, count, Ps));
        for (int i = 0; i < count; i++) {
            rsvd_plan *P = Ps[i];
            T *X, *Qo, *Tmp;
            int64_t rows;
            bufs(P, X, Qo, Tmp, rows);
            const T *src = pass == 0 ? X : Tmp;
            T *dst = (pass == passes - 1) ? Qo : Tmp;
            CK(prod_nn<T>(P, rows, lp, src, lp, (const T *)P->Rinv_c, lp, dst, lp, nullptr, nullptr, true));
            if (sizeof(T) == 4)
                CK(rinv64_fb({(const float *)src, rows, lp, pass ? P->R2i : P->R1i, (float *)dst, P->fb,
                              want_r ? nullptr : P->dflag, refill_seed(P), passes == 2 ? nullptr : P->dflag + l},
                             l, P->stream));
            if (sizeof(T) == 8 && !want_r) {
                const rsvd_status rs = refill<T>(P, dst, rows, l, lp);
                if (rs) return rs;
            }
            if (pass == 1 && want_r) CK(trmm_upper(P->R2, P->R1, P->Rt, l, P->stream));
        }
    }
    return RSVD_OK;
}

// The steps of run_rsvd for `count` problems (see there for the step list).
template <typename T>
rsvd_status run_rsvd_batch(BatchCtx &C, int count, rsvd_plan *const *Ps, T *const *A, const T *const *Om,
                           double *const *S, T *const *U, T *const *V, bool capturing) {
    const int l = Ps[0]->l, lp = Ps[0]->lp, q = Ps[0]->q;
    const double u = DBL_EPSILON / 2;  // shifts are applied in float64 only (chol_pass)
    CK(C.reserve(count));
    if (C.up_pending) {  // the previous upload must have read the host table before it is rewritten
        CK(cudaEventSynchronize(C.up));
        C.up_pending = false;
    }
    for (int i = 0; i < count; i++) {
        rsvd_plan *P = Ps[i];
        for (int pass = 0; pass < 2; pass++) {
            double *R = pass ? P->R2 : P->R1, *Ri = pass ? P->R2i : P->R1i;
            // fb: the fallback flag (float32 plans) or the deflation flags (float64 plans)
            int *fbt = sizeof(T) == 8 ? P->dflag : P->fb;
            C.chol(pass, count, false)[i] = {P->G, R, Ri, P->Rinv_c, P->status, chol_shift_coef(P->m, l, u),
                                              P->G64, fbt, (double *)P->chol_ws};
            C.chol(2 + pass, count, false)[i] = {P->G, R, Ri, P->Rinv_c, P->status, chol_shift_coef(P->n, l, u),
                                                  P->G64, fbt, (double *)P->chol_ws};
        }
        if constexpr (sizeof(T) == 4) {  // the float64 Gram fallback of each (block, pass): its source block
            const float *src[6] = {(const float *)P->Y, (const float *)P->Tmp, (const float *)P->Z,
                                   (const float *)P->Tmpn, (const float *)P->Tn, (const float *)P->Tmpn};
            for (int v = 0; v < 6; v++) {
                const int64_t rows = v < 2 ? P->m : P->n;
                const int pass = v & 1;
                C.g64(v, count, false)[i] = {src[v],      rows,          lp,        P->g64part,
                                             P->G64,      P->fb,         P->g64count, chol_shift_coef(rows, l, u),
                                             pass ? P->R2 : P->R1, pass ? P->R2i : P->R1i, (float *)P->Rinv_c, lp,
                                             P->status,   (double *)P->chol_ws, v >= 4 ? kCholFallback : kCholDeflate,
                                             P->dflag};
            }
        }
        C.jac(count, false)[i] = {P->Rt, P->sig, P->UR, P->Wm, P->status};
    }
    CK(cudaMemcpyAsync(C.dtab, C.htab, BatchCtx::bytes_for(count), cudaMemcpyHostToDevice, C.bs));
    if (!capturing) {
        CK(cudaEventRecord(C.up, C.bs));
        C.up_pending = true;
    }
    CK(fork(C, count, Ps));
    for (int i = 0; i < count; i++) {  // means, padded Omega, sketch H(0) = A G with ||A||_F^2
        rsvd_plan *P = Ps[i];
        P->nfact = 0;
        const bool centred = !(P->flags & RSVD_FLAG_NO_CENTER);
        if (centred) CK(column_means<T>(A[i], P->m, P->n, P->n, P->mu, (T *)P->mu_t, P->npad, P->cpart, P->stream));
        else CK(cudaMemsetAsync(P->mu, 0, sizeof(double) * P->n, P->stream));
        CK(copy2d<T, T>(Om[i], l, (T *)P->Ob, lp, P->n, l, lp, P->stream));
        CK(prod_nn<T>(P, P->m, P->n, A[i], P->n, (T *)P->Ob, lp, (T *)P->Y, lp,
                      centred ? (const T *)P->mu_t : nullptr, P->fro2));
    }
    rsvd_status st;
    if ((st = bcqr<T>(C, count, Ps, BQ_Y, q > 0 ? 1 : 2, false))) return st;
    for (int it = 0; it < q; it++) {
        const bool last = it == q - 1;
        for (int i = 0; i < count; i++) {
            rsvd_plan *P = Ps[i];
            const T *mu = (P->flags & RSVD_FLAG_NO_CENTER) ? nullptr : (const T *)P->mu_t;
            CK(prod_tn<T>(P, P->m, P->n, A[i], P->n, (T *)P->Qb, lp, (T *)P->Z, lp, mu, false, 0, true));
        }
        if ((st = bcqr<T>(C, count, Ps, BQ_Z, 1, false))) return st;
        for (int i = 0; i < count; i++) {
            rsvd_plan *P = Ps[i];
            const T *mu = (P->flags & RSVD_FLAG_NO_CENTER) ? nullptr : (const T *)P->mu_t;
            CK(prod_nn<T>(P, P->m, P->n, A[i], P->n, (T *)P->Qz, lp, (T *)P->Y, lp, mu));
        }
        if ((st = bcqr<T>(C, count, Ps, BQ_Y, last ? 2 : 1, false))) return st;
    }
    // orthonormality checks of the final bases (check_basis), per problem on its own stream
    auto bcheck = [&](int which) -> rsvd_status {
        for (int i = 0; i < count; i++) {
            rsvd_plan *P = Ps[i];
            const rsvd_status st = check_basis<T>(P, which == BQ_Y ? (const T *)P->Qb : (const T *)P->Qz,
                                                  which == BQ_Y ? P->m : P->n, l, lp);
            if (st) return st;
        }
        return RSVD_OK;
    };
    if ((st = bcheck(BQ_Y))) return st;
    for (int i = 0; i < count; i++) {  // T = A^T Q
        rsvd_plan *P = Ps[i];
        const T *mu = (P->flags & RSVD_FLAG_NO_CENTER) ? nullptr : (const T *)P->mu_t;
        CK(prod_tn<T>(P, P->m, P->n, A[i], P->n, (T *)P->Qb, lp, (T *)P->Tn, lp, mu, false, 0, true));
    }
    if ((st = bcqr<T>(C, count, Ps, BQ_T, 2, true))) return st;  // T = Q_T R
    if ((st = bcheck(BQ_T))) return st;
    CK(join(C, count, Ps));
    CK(jacobi_osvd_batched<T, T>(C.jac(count, true), count, l, lp, C.bs));
    CK(sv_refine_batched<T>(C.jac(count, true), count, l, lp, C.bs));
    CK(fork(C, count, Ps));
    for (int i = 0; i < count; i++) {
        rsvd_plan *P = Ps[i];
        const int k = P->k;
        cudaStream_t s = P->stream;
        CK(gemm_nn<T>(P->n, lp, lp, (T *)P->Qz, lp, (T *)P->UR, lp, (T *)P->Vt, lp, s));
        CK(sign_normalize<T>((T *)P->Vt, P->n, l, lp, (T *)P->Wm, l, lp, s));
        CK(gemm_nn<T>(P->m, k, lp, (T *)P->Qb, lp, (T *)P->Wm, lp, U[i], k, s));
        CK(copy2d<T, T>((T *)P->Vt, lp, V[i], k, P->n, k, k, s));
        CK(copy_f64(P->sig, S[i], k, s));
        P->last_count = k;
    }
    CK(join(C, count, Ps));
    return RSVD_OK;
}

rsvd_status batch_direct(BatchCtx &C, int count, rsvd_plan *const *Ps, void *const *A, const void *const *Om,
                         double *const *S, void *const *U, void *const *V, bool capturing = false) {
    if (Ps[0]->dtype == RSVD_F32)
        return run_rsvd_batch<float>(C, count, Ps, (float *const *)A, (const float *const *)Om, S,
                                     (float *const *)U, (float *const *)V, capturing);
    return run_rsvd_batch<double>(C, count, Ps, (double *const *)A, (const double *const *)Om, S,
                                  (double *const *)U, (double *const *)V, capturing);
}

// Maps the device status bits of a solve onto the ABI status.
rsvd_status status_from_bits(int st) {
    if (st & (ST_CHOL | ST_ORTH)) return RSVD_ERR_CHOL;
    if (st & ST_NOCONV) return RSVD_ERR_NOCONV;
    if (st & ST_TIMEOUT) return RSVD_ERR_TIMEOUT;
    if (st & (ST_SHIFT | ST_RANKDEF)) return RSVD_WARN_RANK_DEFICIENT;
    return RSVD_OK;
}

// Process-wide table of tuned product decompositions (rsvd_autotune), keyed by
// (ceil(log2 m), n, lp).
struct TuneKey {
    int lgm;
    int64_t n;
    int lp;
    bool operator<(const TuneKey &o) const { return std::tie(lgm, n, lp) < std::tie(o.lgm, o.n, o.lp); }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;

TuneKey tune_key(int64_t m, int64_t n, int lp) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) < m) b++;
    return {b, n, lp};
}

// Validates the sizes and fills the plan's shape fields and workspace size.
rsvd_status plan_init(rsvd_plan *P, int64_t m, int64_t n, int k, int p, int q, rsvd_dtype dtype, void *cuda_stream) {
    if (m < 1 || n < 1 || m < n || k < 1 || p < 0 || q < 0) return RSVD_ERR_ARG;
    if ((int64_t)k + p > n) return RSVD_ERR_ARG;
    if (dtype != RSVD_F32 && dtype != RSVD_F64 && dtype != RSVD_BF16 && dtype != RSVD_FP8_E4M3)
        return RSVD_ERR_UNSUPPORTED;
    if (k + p > (dtype == RSVD_F64 ? kSmallMaxF64 : kRsvdMaxL)) return RSVD_ERR_UNSUPPORTED;
    // TMA rows of 16-byte multiples: n % 8 (bfloat16), n % 16 (e4m3)
    if (dtype == RSVD_BF16 && (n % 8 || !tc_available())) return RSVD_ERR_UNSUPPORTED;
    if (dtype == RSVD_FP8_E4M3 && (n % 16 || !tc_available())) return RSVD_ERR_UNSUPPORTED;
    P->m = m;
    P->n = n;
    P->k = k;
    P->p = p;
    P->q = q;
    P->l = k + p;
    P->lp = (int)round_up(P->l, 16);
    P->lpc = P->lp;
    P->nx = n <= kSmallMaxF64 && (dtype == RSVD_F32 || dtype == RSVD_F64) ? (int)n : 0;
    P->wide = P->lp > P->nx ? P->lp : P->nx;
    P->dtype = dtype;
    P->stream = (cudaStream_t)cuda_stream;
    P->tc = dtype != RSVD_F64 && tc_available();
    if (P->tc) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(tune_key(m, n, P->lp));
        if (it != g_tune.end()) {
            P->nn_ctas = it->second.first;
            P->tn_ctas = it->second.second;
        }
    }
    Carver c;
    carve(P, c);
    P->ws_bytes = c.off;
    return RSVD_OK;
}

// Block Krylov plan: blocks of b columns, iters + 1 of them (W = (iters + 1) b).
rsvd_status bk_plan_init(rsvd_plan *P, int64_t m, int64_t n, int k, int b, int iters, rsvd_dtype dtype,
                         void *cuda_stream) {
    if (m < 1 || n < 1 || m < n || k < 1 || b < 1 || iters < 0) return RSVD_ERR_ARG;
    const int64_t W = (int64_t)(iters + 1) * b;
    if (k > W || W > n) return RSVD_ERR_ARG;
    if (dtype != RSVD_F32 && dtype != RSVD_F64) return RSVD_ERR_UNSUPPORTED;
    // a block's Gram eigen-decomposition runs in one CTA's shared memory; the Rayleigh-Ritz
    // steps at width W have the randomized method's limits
    if (round_up(b, 16) > kSmallMaxF64) return RSVD_ERR_UNSUPPORTED;
    if (W > (dtype == RSVD_F64 ? kSmallMaxF64 : kRsvdMaxL)) return RSVD_ERR_UNSUPPORTED;
    P->m = m;
    P->n = n;
    P->k = k;
    P->p = 0;
    P->q = iters;
    P->l = b;
    P->lp = (int)round_up(b, 16);
    P->bk_blocks = iters + 1;
    P->lpc = (int)round_up(W, 16);
    P->nx = n <= kSmallMaxF64 ? (int)n : 0;
    P->wide = P->lpc > P->nx ? P->lpc : P->nx;
    P->dtype = dtype;
    P->stream = (cudaStream_t)cuda_stream;
    P->tc = dtype == RSVD_F32 && tc_available();
    Carver c;
    carve(P, c);
    P->ws_bytes = c.off;
    return RSVD_OK;
}

// Allocates, carves and clears the workspace of an initialised plan.
rsvd_status plan_alloc(rsvd_plan *P) {
    if (cudaMalloc(&P->ws, P->ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        return RSVD_ERR_OOM;
    }
    Carver c2;
    c2.base = (char *)P->ws;
    carve(P, c2);
    if (cudaMemsetAsync(P->ws, 0, P->ws_bytes, P->stream) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) {
        cudaFree(P->ws);
        P->ws = nullptr;
        return RSVD_ERR_CUDA;
    }
    return RSVD_OK;
}

}  // namespace

namespace gbr {

struct ServeBatch {
    BatchCtx ctx;
};

ServeBatch *serve_batch_new(cudaStream_t bs, int cap) {
    ServeBatch *b = new (std::nothrow) ServeBatch();
    if (!b) return nullptr;
    b->ctx.bs = bs;
    if (b->ctx.reserve(cap) != cudaSuccess) {
        delete b;
        return nullptr;
    }
    return b;
}

void serve_batch_free(ServeBatch *b) { delete b; }

rsvd_status serve_batch_launch(ServeBatch *b, int count, rsvd_plan *const *plans, const void *const *A,
                               const float *const *sc, const float *const *Om, double *const *S, float *const *U,
                               float *const *V, const double *t, int *host_out) {
    const rsvd_dtype dt = plans[0]->dtype;
    if ((dt == RSVD_F32 || dt == RSVD_F64) && plans[0]->l <= kSmallMaxF32) {  // lockstep batch
        const rsvd_status st = batch_direct(b->ctx, count, plans, (void *const *)A, (const void *const *)Om, S,
                                            (void *const *)U, (void *const *)V);
        if (st != RSVD_OK) return st;
    } else {  // precision forms and large l: every problem's solve on its own stream, then joined
        CK(b->ctx.reserve(count));
        CK(fork(b->ctx, count, plans));
        for (int i = 0; i < count; i++) {
            const rsvd_status st = rsvd_direct(plans[i], const_cast<void *>(A[i]), sc ? sc[i] : nullptr, Om[i], S[i],
                                               U[i], V[i]);
            if (st != RSVD_OK) return st;
        }
        CK(join(b->ctx, count, plans));
    }
    cudaStream_t bs = b->ctx.bs;
    for (int i = 0; i < count; i++) {  // K selection and the three result words per problem
        rsvd_plan *P = plans[i];
        CK(pca_select(P->sig, P->k, P->fro2, t[i], P->Kdev, P->Kdev + 1, bs));
        CK(cudaMemcpyAsync(host_out + 3 * i, P->status, sizeof(int), cudaMemcpyDeviceToHost, bs));
        CK(cudaMemcpyAsync(host_out + 3 * i + 1, P->Kdev, 2 * sizeof(int), cudaMemcpyDeviceToHost, bs));
    }
    return RSVD_OK;
}

rsvd_status serve_status(int bits, int reached) {
    const rsvd_status st = status_from_bits(bits);
    return st >= RSVD_OK && !reached ? RSVD_WARN_K_GT_k : st;  // errors first, then the K warning
}

}  // namespace gbr

extern "C" {

rsvd_status rsvd_workspace_query(int64_t m, int64_t n, int k, int p, int q, rsvd_dtype dtype, size_t *bytes) {
    if (!bytes) return RSVD_ERR_ARG;
    *bytes = 0;
    rsvd_plan P;
    const rsvd_status st = plan_init(&P, m, n, k, p, q, dtype, nullptr);
    if (st != RSVD_OK) return st;
    *bytes = (size_t)round_up((int64_t)P.ws_bytes, 256);
    return RSVD_OK;
}

rsvd_status rsvd_plan_create_in(rsvd_plan_t *plan, int64_t m, int64_t n, int k, int p, int q, rsvd_dtype dtype,
                                void *cuda_stream, void *workspace, size_t bytes) {
    if (!plan) return RSVD_ERR_ARG;
    *plan = nullptr;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return RSVD_ERR_ARG;
    rsvd_plan *P = new (std::nothrow) rsvd_plan();
    if (!P) return RSVD_ERR_OOM;
    rsvd_status st = plan_init(P, m, n, k, p, q, dtype, cuda_stream);
    if (st == RSVD_OK && bytes < P->ws_bytes) st = RSVD_ERR_ARG;
    if (st != RSVD_OK) {
        delete P;
        return st;
    }
    P->ws = workspace;
    P->ws_owned = false;
    Carver c2;
    c2.base = (char *)P->ws;
    carve(P, c2);
    if (cudaMemsetAsync(P->ws, 0, P->ws_bytes, P->stream) != cudaSuccess) {
        delete P;
        return RSVD_ERR_CUDA;
    }
    *plan = P;
    return RSVD_OK;
}

rsvd_status rsvd_plan_create(rsvd_plan_t *plan, int64_t m, int64_t n, int k, int p, int q, rsvd_dtype dtype,
                             void *cuda_stream) {
    if (!plan) return RSVD_ERR_ARG;
    *plan = nullptr;
    rsvd_plan *P = new (std::nothrow) rsvd_plan();
    if (!P) return RSVD_ERR_OOM;
    rsvd_status st = plan_init(P, m, n, k, p, q, dtype, cuda_stream);
    if (st == RSVD_OK) st = plan_alloc(P);
    if (st != RSVD_OK) {
        delete P;
        return st;
    }
    *plan = P;
    return RSVD_OK;
}

rsvd_status rsvd_plan_create_block_krylov(rsvd_plan_t *plan, int64_t m, int64_t n, int k, int b, int iters,
                                          rsvd_dtype dtype, void *cuda_stream) {
    if (!plan) return RSVD_ERR_ARG;
    *plan = nullptr;
    rsvd_plan *P = new (std::nothrow) rsvd_plan();
    if (!P) return RSVD_ERR_OOM;
    rsvd_status st = bk_plan_init(P, m, n, k, b, iters, dtype, cuda_stream);
    if (st == RSVD_OK) st = plan_alloc(P);
    if (st != RSVD_OK) {
        delete P;
        return st;
    }
    *plan = P;
    return RSVD_OK;
}

rsvd_status rsvd_block_krylov(rsvd_plan_t P, void *A, const void *Omega, double *S, void *U, void *V) {
    if (!P || !A || !Omega || !S || !U || !V || !P->bk_blocks) return RSVD_ERR_ARG;
    if (P->dtype == RSVD_F32)
        return run_block_krylov<float>(P, (float *)A, (const float *)Omega, S, (float *)U, (float *)V);
    return run_block_krylov<double>(P, (double *)A, (const double *)Omega, S, (double *)U, (double *)V);
}

rsvd_status rsvd_plan_destroy(rsvd_plan_t P) {
    if (!P) return RSVD_OK;
    cudaStreamSynchronize(P->stream);
    for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
    drop_graph(P);
    if (P->gkl_ws) cudaFree(P->gkl_ws);
    if (P->gram_ws) cudaFree(P->gram_ws);
    if (P->shard_ws) cudaFree(P->shard_ws);
    if (P->ws_owned) cudaFree(P->ws);
    delete P;
    return RSVD_OK;
}

size_t rsvd_plan_workspace_bytes(rsvd_plan_t P) { return P ? P->ws_bytes : 0; }

rsvd_status rsvd_set_jacobi_sweep_cap(int cap) {
    if (cap < 0) return RSVD_ERR_ARG;
    set_sweep_cap(cap);
    return RSVD_OK;
}

rsvd_status rsvd_plan_set_flags(rsvd_plan_t P, unsigned flags) {
    if (!P || (flags & ~(unsigned)(RSVD_FLAG_NO_CENTER | RSVD_FLAG_GKL_TWO_PASS | RSVD_FLAG_SMALL_F32 |
                                   RSVD_FLAG_SMALL_FP64)))
        return RSVD_ERR_ARG;
    P->flags = flags;
    return RSVD_OK;
}

rsvd_status rsvd_plan_sync(rsvd_plan_t P) {
    if (!P) return RSVD_ERR_ARG;
    int st = 0;
    if (cudaMemcpyAsync(&st, P->status, sizeof(int), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess)
        return RSVD_ERR_CUDA;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return RSVD_ERR_CUDA;
    if (cudaMemsetAsync(P->status, 0, sizeof(int), P->stream) != cudaSuccess) return RSVD_ERR_CUDA;
    return status_from_bits(st);
}

rsvd_status rsvd(rsvd_plan_t P, void *A, const float *col_scales, const void *Omega, double *S, void *U, void *V) {
    if (!P || !A || !Omega || !S || !U || !V || P->bk_blocks) return RSVD_ERR_ARG;
    if ((col_scales != nullptr) != (P->dtype == RSVD_FP8_E4M3)) return RSVD_ERR_ARG;  // e4m3 needs its scales
    // Tracing records events between launches and the legacy stream cannot be captured:
    // both run the launches directly.
    if (P->prof || P->stream == nullptr) return rsvd_direct(P, A, col_scales, Omega, S, U, V);
    const void *key[7] = {A, Omega, S, U, V, P, col_scales};
    bool hit = P->graph && P->gflags == P->flags;
    for (int i = 0; hit && i < 7; i++) hit = P->gkey[i] == key[i];
    if (!hit) {
        drop_graph(P);
        cudaGraph_t g = nullptr;
        const uint64_t before = rsvd_launch_count();
        if (cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cudaGetLastError();
            return rsvd_direct(P, A, col_scales, Omega, S, U, V);
        }
        const rsvd_status st = rsvd_direct(P, A, col_scales, Omega, S, U, V);
        const cudaError_t ce = cudaStreamEndCapture(P->stream, &g);
        const uint64_t captured = rsvd_launch_count() - before;
        g_launches.fetch_sub(captured, std::memory_order_relaxed);  // captured, not yet executed
        if (st != RSVD_OK || ce != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st != RSVD_OK ? st : RSVD_ERR_CUDA;
        }
        cudaError_t ie = cudaGraphInstantiate(&P->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            P->graph = nullptr;
            cudaGetLastError();
            return rsvd_direct(P, A, col_scales, Omega, S, U, V);
        }
        for (int i = 0; i < 7; i++) P->gkey[i] = key[i];
        P->gflags = P->flags;
        P->glaunches = captured;
    }
    if (cudaGraphLaunch(P->graph, P->stream) != cudaSuccess) return RSVD_ERR_CUDA;
    note_launch((int)P->glaunches);
    P->last_count = P->k;
    return RSVD_OK;
}

rsvd_status rsvd_sharded(rsvd_plan_t P, int64_t m_total, void *A, const void *Omega, double *S, void *U, void *V,
                         rsvd_allreduce_fn allreduce, void *ctx) {
    if (!P || !A || !Omega || !S || !U || !V || !allreduce || P->bk_blocks || m_total < P->m) return RSVD_ERR_ARG;
    if (P->dtype != RSVD_F32 && P->dtype != RSVD_F64) return RSVD_ERR_UNSUPPORTED;
    if (!P->shard_ws) {
        const size_t bytes = sizeof(double) * (size_t)std::max<int64_t>(P->n, P->lp) * P->lp;
        if (cudaMalloc(&P->shard_ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            P->shard_ws = nullptr;
            return RSVD_ERR_OOM;
        }
    }
    const Reducer r{allreduce, ctx};
    if (P->dtype == RSVD_F32)
        return run_rsvd_sharded<float>(P, m_total, (const float *)A, (const float *)Omega, S, (float *)U, (float *)V,
                                       r);
    return run_rsvd_sharded<double>(P, m_total, (const double *)A, (const double *)Omega, S, (double *)U,
                                    (double *)V, r);
}

}  // extern "C"

struct rsvd_batch {
    std::vector<rsvd_plan *> plans;
    cudaStream_t stream = nullptr;
    BatchCtx ctx;
    cudaGraphExec_t graph = nullptr;
    std::vector<const void *> key;
    std::vector<unsigned> kflags;
    uint64_t glaunches = 0;
};

extern "C" {

rsvd_status rsvd_batch_create(rsvd_batch_t *batch, int count, rsvd_plan_t const *plans, void *cuda_stream) {
    if (!batch) return RSVD_ERR_ARG;
    *batch = nullptr;
    if (count < 1 || count > RSVD_BATCH_MAX || !plans) return RSVD_ERR_ARG;
    for (int i = 0; i < count; i++) {
        const rsvd_plan *P = plans[i];
        if (!P || P->bk_blocks) return RSVD_ERR_ARG;
        if (P->dtype != plans[0]->dtype || P->l != plans[0]->l || P->q != plans[0]->q) return RSVD_ERR_ARG;
        if (P->dtype != RSVD_F32 && P->dtype != RSVD_F64) return RSVD_ERR_UNSUPPORTED;
        if (P->l > kSmallMaxF32) return RSVD_ERR_UNSUPPORTED;  // batched small kernels: l x l in shared memory
        for (int j = 0; j < i; j++)
            if (plans[j] == P) return RSVD_ERR_ARG;
    }
    rsvd_batch *B = new (std::nothrow) rsvd_batch();
    if (!B) return RSVD_ERR_OOM;
    B->plans.assign(plans, plans + count);
    B->stream = (cudaStream_t)cuda_stream;
    B->ctx.bs = B->stream;
    if (B->ctx.reserve(count) != cudaSuccess) {
        delete B;
        return RSVD_ERR_OOM;
    }
    *batch = B;
    return RSVD_OK;
}

rsvd_status rsvd_batch_run(rsvd_batch_t B, void *const *A, const void *const *Omega, double *const *S,
                           void *const *U, void *const *V) {
    if (!B || !A || !Omega || !S || !U || !V) return RSVD_ERR_ARG;
    const int count = (int)B->plans.size();
    bool direct = B->stream == nullptr;
    std::vector<const void *> key;
    std::vector<unsigned> kflags;
    for (int i = 0; i < count; i++) {
        if (!A[i] || !Omega[i] || !S[i] || !U[i] || !V[i]) return RSVD_ERR_ARG;
        rsvd_plan *P = B->plans[i];
        if (P->stream == nullptr || P->prof) direct = true;
        key.insert(key.end(), {A[i], Omega[i], S[i], U[i], V[i]});
        kflags.push_back(P->flags);
    }
    rsvd_plan *const *Ps = B->plans.data();
    if (direct) {
        if (B->graph) cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
        return batch_direct(B->ctx, count, Ps, A, Omega, S, U, V);
    }
    if (!(B->graph && key == B->key && kflags == B->kflags)) {
        if (B->graph) cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
        cudaGraph_t g = nullptr;
        const uint64_t before = rsvd_launch_count();
        if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cudaGetLastError();
            return batch_direct(B->ctx, count, Ps, A, Omega, S, U, V);
        }
        const rsvd_status st = batch_direct(B->ctx, count, Ps, A, Omega, S, U, V, true);
        const cudaError_t ce = cudaStreamEndCapture(B->stream, &g);
        const uint64_t captured = rsvd_launch_count() - before;
        g_launches.fetch_sub(captured, std::memory_order_relaxed);
        if (st != RSVD_OK || ce != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st != RSVD_OK ? st : RSVD_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&B->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            B->graph = nullptr;
            cudaGetLastError();
            return batch_direct(B->ctx, count, Ps, A, Omega, S, U, V);
        }
        B->key = key;
        B->kflags = kflags;
        B->glaunches = captured;
    }
    if (cudaGraphLaunch(B->graph, B->stream) != cudaSuccess) return RSVD_ERR_CUDA;
    note_launch((int)B->glaunches);
    for (rsvd_plan *P : B->plans) P->last_count = P->k;
    return RSVD_OK;
}

rsvd_status rsvd_batch_sync(rsvd_batch_t B, int *statuses) {
    if (!B) return RSVD_ERR_ARG;
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return RSVD_ERR_CUDA;
    rsvd_status worst = RSVD_OK;
    for (size_t i = 0; i < B->plans.size(); i++) {
        const rsvd_status st = rsvd_plan_sync(B->plans[i]);
        if (statuses) statuses[i] = st;
        if ((st < RSVD_OK && worst >= RSVD_OK) || (st > RSVD_OK && worst == RSVD_OK)) worst = st;  // errors first
    }
    return worst;
}

rsvd_status rsvd_batch_destroy(rsvd_batch_t B) {
    if (!B) return RSVD_OK;
    cudaStreamSynchronize(B->stream);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    delete B;
    return RSVD_OK;
}

rsvd_status rsvd_autotune(rsvd_plan_t P, void *A, const void *Omega, int concurrency, int *nn_out, int *tn_out) {
    if (!P || !A || !Omega || concurrency < 1 || concurrency > 64 || P->bk_blocks) return RSVD_ERR_ARG;
    if (nn_out) *nn_out = P->nn_ctas;
    if (tn_out) *tn_out = P->tn_ctas;
    if (P->dtype != RSVD_F32 || !P->tc || P->l > kSmallMaxF32) return RSVD_OK;  // tunes through lockstep batches (l <= 128)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RSVD_ERR_CUDA;
    const int cand[][2] = {{0, 0}, {sms / 2, sms / 2}, {sms / 4, sms / 4}, {sms / 2, 0}, {0, sms / 2}};
    const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
    rsvd_status st = RSVD_OK;
    std::vector<rsvd_plan *> plans{P};
    std::vector<cudaStream_t> streams;
    cudaStream_t bs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    char *out = nullptr;
    const size_t sb = round_up(sizeof(double) * P->k, 256), ub = round_up(sizeof(float) * P->m * P->k, 256),
                 vb = round_up(sizeof(float) * P->n * P->k, 256);
    std::vector<void *> Av(concurrency, A), Ov(concurrency, const_cast<void *>(Omega)), Uv, Vv;
    std::vector<double *> Sv;
    float best_ms = 3.4e38f;
    int best = 0;
    {
        BatchCtx ctx;
        bool ok = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
                  cudaMalloc(&out, (sb + ub + vb) * concurrency) == cudaSuccess;
        for (int i = 1; ok && i < concurrency; i++) {
            cudaStream_t x = nullptr;
            rsvd_plan_t Q = nullptr;
            ok = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) == cudaSuccess;
            if (ok) streams.push_back(x);
            ok = ok && rsvd_plan_create(&Q, P->m, P->n, P->k, P->p, P->q, P->dtype, x) == RSVD_OK;
            if (ok) plans.push_back(Q);
        }
        ctx.bs = bs;
        ok = ok && ctx.reserve(concurrency) == cudaSuccess;
        for (int i = 0; ok && i < concurrency; i++) {
            char *b = out + (sb + ub + vb) * i;
            Sv.push_back((double *)b);
            Uv.push_back(b + sb);
            Vv.push_back(b + sb + ub);
        }
        for (int c = 0; ok && c < ncand; c++) {
            for (rsvd_plan *X : plans) {
                X->nn_ctas = cand[c][0];
                X->tn_ctas = cand[c][1];
            }
            float ms[3];
            for (int r = 0; ok && r < 4; r++) {  // one warm-up, three timed
                ok = cudaEventRecord(e0, bs) == cudaSuccess &&
                     batch_direct(ctx, concurrency, plans.data(), Av.data(), (const void *const *)Ov.data(),
                                  Sv.data(), Uv.data(), Vv.data()) == RSVD_OK &&
                     cudaEventRecord(e1, bs) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
                if (ok && r > 0) ok = cudaEventElapsedTime(&ms[r - 1], e0, e1) == cudaSuccess;
            }
            if (!ok) break;
            std::sort(ms, ms + 3);
            if (ms[1] < best_ms) {
                best_ms = ms[1];
                best = c;
            }
        }
        if (!ok) st = RSVD_ERR_CUDA;
        for (size_t i = 1; i < plans.size(); i++) rsvd_plan_destroy(plans[i]);
    }
    for (cudaStream_t x : streams) cudaStreamDestroy(x);
    if (bs) cudaStreamDestroy(bs);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    cudaMemsetAsync(P->status, 0, sizeof(int), P->stream);
    P->nn_ctas = cand[best][0];
    P->tn_ctas = cand[best][1];
    if (st == RSVD_OK) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[tune_key(P->m, P->n, P->lp)] = {P->nn_ctas, P->tn_ctas};
    }
    if (nn_out) *nn_out = P->nn_ctas;
    if (tn_out) *tn_out = P->tn_ctas;
    P->last_count = 0;
    return st;
}

rsvd_status rsvd_tune_lookup(int64_t m, int64_t n, int k, int p, int *nn_ctas, int *tn_ctas) {
    if (m < 1 || n < 1 || k < 1 || p < 0) return RSVD_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(tune_key(m, n, (int)round_up(k + p, 16)));
    if (it == g_tune.end()) return RSVD_ERR_ARG;
    if (nn_ctas) *nn_ctas = it->second.first;
    if (tn_ctas) *tn_ctas = it->second.second;
    return RSVD_OK;
}

void rsvd_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

rsvd_status svd_exact(rsvd_plan_t P, void *A, int method, double *S, void *U, void *V) {
    if (!P || !A || !S || !U || !V) return RSVD_ERR_ARG;
    if (method != RSVD_EXACT_GRAM && method != RSVD_EXACT_QR_JACOBI) return RSVD_ERR_ARG;
    if (P->dtype != RSVD_F32 && P->dtype != RSVD_F64) return RSVD_ERR_UNSUPPORTED;
    if (!P->nx) {  // beyond one CTA: the Gram route's float64 eigensolver on the whole GPU
        if (method != RSVD_EXACT_GRAM || P->n > kGramMaxN) return RSVD_ERR_UNSUPPORTED;
        if (P->dtype == RSVD_F32) return run_exact_large<float>(P, (float *)A, S, (float *)U, (float *)V);
        return run_exact_large<double>(P, (double *)A, S, (double *)U, (double *)V);
    }
    if (P->dtype == RSVD_F32) return run_exact<float>(P, (float *)A, method, S, (float *)U, (float *)V);
    return run_exact<double>(P, (double *)A, method, S, (double *)U, (double *)V);
}

rsvd_status svd_truncated_krylov(rsvd_plan_t P, void *A, const void *v1, int steps, double *S, void *U, void *V) {
    if (!P || !A || !v1 || !S || !U || !V) return RSVD_ERR_ARG;
    if (steps < P->k || steps > P->n || steps < 1) return RSVD_ERR_ARG;
    if (P->dtype != RSVD_F32 && P->dtype != RSVD_F64) return RSVD_ERR_UNSUPPORTED;
    if (steps > (P->dtype == RSVD_F64 ? kSmallMaxF64 : kGklMaxStepsF32)) return RSVD_ERR_UNSUPPORTED;
    if (P->dtype == RSVD_F32)
        return run_gkl<float>(P, (float *)A, (const float *)v1, steps, S, (float *)U, (float *)V);
    return run_gkl<double>(P, (double *)A, (const double *)v1, steps, S, (double *)U, (double *)V);
}

rsvd_status pca_threshold(rsvd_plan_t P, double t, int *K) {
    if (!P || !K || !(t > 0.0) || t > 1.0) return RSVD_ERR_ARG;
    if (P->last_count <= 0) return RSVD_ERR_ARG;
    int host[2] = {0, 0};
    if (pca_select(P->sig, P->last_count, P->fro2, t, P->Kdev, P->Kdev + 1, P->stream) != cudaSuccess)
        return RSVD_ERR_CUDA;
    if (cudaMemcpyAsync(host, P->Kdev, 2 * sizeof(int), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess)
        return RSVD_ERR_CUDA;
    rsvd_status st = rsvd_plan_sync(P);
    *K = host[0];
    if (st != RSVD_OK) return st;
    return host[1] ? RSVD_OK : RSVD_WARN_K_GT_k;
}

rsvd_status rsvd_plan_fro2(rsvd_plan_t P, double *fro2) {
    if (!P || !fro2) return RSVD_ERR_ARG;
    if (cudaMemcpyAsync(fro2, P->fro2, sizeof(double), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess)
        return RSVD_ERR_CUDA;
    return cudaStreamSynchronize(P->stream) == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

rsvd_status rsvd_plan_profile(rsvd_plan_t P, int enable) {
    if (!P) return RSVD_ERR_ARG;
    P->prof = enable != 0;
    return RSVD_OK;
}

rsvd_status rsvd_plan_profile_read(rsvd_plan_t P, double *ms, int *groups, int nstages) {
    if (!P || !ms || !groups || nstages < 1) return RSVD_ERR_ARG;
    for (int i = 0; i < nstages; i++) { ms[i] = 0.0; groups[i] = 0; }
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return RSVD_ERR_CUDA;
    for (size_t i = 0; i + 1 < P->ev_used; i += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, P->ev[i], P->ev[i + 1]) != cudaSuccess) return RSVD_ERR_CUDA;
        const int st = P->ev_stage[i / 2];
        if (st >= 0 && st < nstages) { ms[st] += t; groups[st] += 1; }
    }
    P->ev_used = 0;
    return RSVD_OK;
}

uint64_t rsvd_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *rsvd_status_string(rsvd_status s) {
    switch (s) {
        case RSVD_OK: return "ok";
        case RSVD_ERR_ARG: return "invalid argument";
        case RSVD_ERR_OOM: return "device allocation failed";
        case RSVD_ERR_CHOL: return "Cholesky breakdown";
        case RSVD_ERR_NOCONV: return "Jacobi did not converge";
        case RSVD_ERR_TIMEOUT: return "device wait timed out";
        case RSVD_ERR_CUDA: return "CUDA error";
        case RSVD_ERR_UNSUPPORTED: return "unsupported size or dtype";
        case RSVD_ERR_REDUCE: return "the reduction over ranks failed";
        case RSVD_WARN_K_GT_k: return "threshold not reached within the returned values";
        case RSVD_WARN_RANK_DEFICIENT: return "numerically rank-deficient input or basis (handled; bases checked)";
    }
    return "unknown status";
}

}  // extern "C"
