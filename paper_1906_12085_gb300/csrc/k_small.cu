// Small dense problems solved inside one CTA's shared memory:
//   chol_inv    : shifted Cholesky + triangular inverse (the QR step of Sec. 3.1.2
//                 done as CholeskyQR2; float64 arithmetic)
//   jacobi_osvd : one-sided (Hestenes) Jacobi SVD of an l x l factor (the SVD of
//                 T = A^T Q in Sec. 3.1.2 step 6, after T = Q_T R)
//   jacobi_eig  : two-sided Jacobi eigen-decomposition of A^T A (Sec. 2.3 and
//                 Sec. 3.1.3 step 2)
// plus the elementwise finishing kernels (sigma = sqrt(lambda), u_i = A v_i /
// sigma_i scaling, sign convention, K selection of Sec. 2.4).
//
// Jacobi rotations use the round-robin ("circle") parallel ordering: in each
// of the L-1 rounds of a sweep the L/2 index pairs are disjoint, so one warp
// rotates one pair without synchronising with the others.
#include <float.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"

namespace gbr {
namespace {

// Sweep caps of the Jacobi solvers (rsvd_set_jacobi_sweep_cap): 0 means the defaults, 40
// sweeps for the one-sided SVD and 50 for the two-sided eigen-decomposition.
std::atomic<int> g_sweep_cap{0};
int sweep_cap(int dflt) {
    const int c = g_sweep_cap.load(std::memory_order_relaxed);
    return c > 0 ? c : dflt;
}

__device__ __forceinline__ int rr_pos(int k, int r, int L) {
    // position k of round r in the circle method: player 0 fixed, the rest rotate
    // (k - 1 + r < 2 (L - 1), so one conditional subtraction replaces the modulo)
    if (k == 0) return 0;
    int x = k - 1 + r;
    if (x >= L - 1) x -= L - 1;
    return 1 + x;
}

// Jacobi rotation (c, s) annihilating gamma for column norms^2 alpha, beta:
// zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t.
__device__ __forceinline__ void jrot(float al, float be, float ga, float &c, float &s, float &t) {
    // zeta and t only choose the angle (fast division is enough); c comes from the
    // reciprocal square root: a rotation scaled by (1 + O(eps)) keeps the two columns
    // (and the two accumulated V columns) orthogonal, only their norms move, and the
    // V columns are renormalised at the end
    const float zeta = __fdividef(be - al, 2.f * ga);
    const float z2 = fmaf(zeta, zeta, 1.f);
    const float root = z2 < 1e30f ? z2 * rsqrtf(z2) : fabsf(zeta);  // sqrt(1 + zeta^2)
    t = copysignf(1.f, zeta) * __fdividef(1.f, fabsf(zeta) + root);
    c = rsqrtf(fmaf(t, t, 1.f));
    s = c * t;
}
__device__ __forceinline__ void jrot(double al, double be, double ga, double &c, double &s, double &t) {
    const double zeta = (be - al) / (2.0 * ga);
    t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    s = c * t;
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = FLT_EPSILON; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };

// Synchronisation of the small solvers: one CTA (__syncthreads), or the CTAs of a
// thread-block cluster (hardware cluster barrier with release / acquire, which also orders the
// global-memory columns between the CTAs).
struct CtaSync {
    static constexpr bool size_is_one = true;
    static __device__ __forceinline__ void sync() { __syncthreads(); }
    static __device__ __forceinline__ int rank() { return 0; }
    static __device__ __forceinline__ int size() { return 1; }
};
struct ClusterSync {
    static constexpr bool size_is_one = false;
    static __device__ __forceinline__ void sync() {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    static __device__ __forceinline__ int rank() {
        unsigned r;
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
        return (int)r;
    }
    static __device__ __forceinline__ int size() {
        unsigned r;
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
        return (int)r;
    }
};

// ------------------------------------------------------------ Cholesky + inverse
// Upper Cholesky R^T R = G and the inverse X = R^{-1} of an l x l matrix in one
// CTA of 256 threads, blocked by 16-column panels (NP = ceil(l / 16) panels, the
// matrix padded to 16 NP with the identity).  Arithmetic in Tk, in shared memory.
//   Cholesky, panel p (rows / columns o = 16 p .. o + 15), right-looking:
//     (1) one warp factors the diagonal block D = R_pp^T R_pp with each column in
//         the registers of one lane (row k of R broadcast through shared memory):
//         for k = 0..15, R_kk = sqrt(D_kk), R_kc = D_kc / R_kk (c > k),
//         D_ic -= R_ki R_kc (k < i <= c);
//     (2) every column c right of the panel solves R_pp^T x = A[o..o+15][c]
//         (forward substitution) for the panel rows of R;
//     (3) rank-16 update of the trailing upper triangle:
//         A[i][c] -= sum_k R[o+k][i] R[o+k][c].
//   Inverse, row blocks p = NP-1 .. 0 (back substitution by blocks):
//     T = delta_pb I - sum_{p<q<=b} R_pq X_qb for every column block b >= p, then
//     X_pb = R_pp^{-1} T by back substitution inside the block (rows 15..0).
// The reciprocal pivots 1 / R_kk come from the reciprocal square root, so no
// step waits on a division.  Three barriers per panel for the factor, two per
// row block for the inverse.
template <typename Tk>
struct CholSmem {
    Tk *A, *X, *rdiag;
    int S;  // row stride of A and X
};

// A and X in shared memory, or (GM: matrices too large for one SM) with the pivots in
// the global scratch gws (2 LL S + LL elements, then the trace and breakdown flag).
template <typename Tk, bool GM>
__device__ __forceinline__ CholSmem<Tk> chol_smem(int LL, Tk *gws) {
    extern __shared__ __align__(16) unsigned char smraw[];
    CholSmem<Tk> m;
    m.S = LL + (sizeof(Tk) == 4 ? 16 : 1);
    if constexpr (GM) {
        m.A = gws;
        m.X = gws + (size_t)LL * m.S;
        m.rdiag = gws + 2 * (size_t)LL * m.S;
    } else {
        m.A = reinterpret_cast<Tk *>(smraw);
        m.X = m.A + (size_t)LL * m.S;
        m.rdiag = m.X + (size_t)LL * m.S;
    }
    return m;
}

// The float64 retry of a float32 first attempt (kCholRetry), kept out of line so that the
// float32 kernels' own code is generated as if it were absent.
template <typename TG, typename Tc>
__device__ __noinline__ void chol_retry64(const TG *G, int64_t ldg, int l, double shift_coef, double *R, double *Rinv,
                                          Tc *Rinv_c, int lp, int *status, double *ws64, int *fb);

template <typename TG, typename Tk, typename Tc, bool GM = false>
__device__ __forceinline__ void chol_inv_body(const TG *__restrict__ G, int64_t ldg, int l, double shift_coef,
                                              double *__restrict__ R, double *__restrict__ Rinv,
                                              Tc *__restrict__ Rinv_c, int lp, int *__restrict__ status,
                                              Tk *gws = nullptr, int *fb = nullptr, int role = kCholPlain,
                                              double *ws64 = nullptr) {
    // GM: the matrices, the pivots and the breakdown flag in the global scratch, the work
    // shared by the CTAs of a cluster (cluster barriers between the phases)
    using Sync = typename std::conditional<GM, ClusterSync, CtaSync>::type;
    // the fallback runs only after a breakdown of the first attempt (every thread reads the flag)
    if (role == kCholFallback && *reinterpret_cast<volatile int *>(fb) == 0) return;
    // kCholDeflate (float64 only, compiled out of the other forms): pivots <= tau G_kk remove
    // their column (flags in fb[0..l-1])
    constexpr bool kCanDeflate = std::is_same<Tk, double>::value;
    const bool deflate = kCanDeflate && role == kCholDeflate;
    const double tau = deflate ? kDeflateRel * l : 0.0;
    const int NP = (l + 15) >> 4, LL = 16 * NP;
    const CholSmem<Tk> sm = chol_smem<Tk, GM>(LL, gws);
    Tk *A = sm.A, *X = sm.X, *rdiag = sm.rdiag;
    const int S = sm.S;
    __shared__ double trace_s;
    __shared__ int bad_s;
    double *tracep = &trace_s;
    int *badp = &bad_s;
    if constexpr (GM) {
        tracep = reinterpret_cast<double *>(gws + 2 * (size_t)LL * S + ((LL + 1) & ~1));
        badp = reinterpret_cast<int *>(tracep + 1);
    }
    volatile int *bad = badp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, tx = tid & 15, ty = tid >> 4;
    const int rank = Sync::rank(), nct = Sync::size();
    const int gt = rank * 256 + tid, gnt = nct * 256;
    int used = 0;  // 0: plain, 1: shifted, 2: breakdown fallback (R = 0, R^{-1} = I)
    if (deflate)  // the flags and, after them, the word that says whether any column was removed
        for (int i = gt; i <= l; i += gnt) fb[i] = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        if (attempt == 1 && rank == 0 && warp == 0) {  // trace for the shift (only after a breakdown)
            double tr = 0.0;
            for (int i = lane; i < l; i += 32) tr += (double)G[(int64_t)i * ldg + i];
            tr = warp_sum(tr);
            if (lane == 0) *tracep = tr;
        }
        if (rank == 0 && tid == 0) *bad = 0;
        Sync::sync();
        const Tk sh = attempt == 1 ? (Tk)(shift_coef * *reinterpret_cast<volatile double *>(tracep)) : Tk(0);
        for (int idx = gt; idx < LL * LL; idx += gnt) {  // upper triangle (the lower one is never read)
            const int i = idx / LL, j = idx % LL;
            if (j < i) continue;
            Tk v;
            if (i < l && j < l) v = attempt == 2 ? Tk(i == j ? 1 : 0) : (Tk)G[(int64_t)i * ldg + j];
            else v = Tk(i == j ? 1 : 0);
            if (i == j && i < l) v += sh;
            A[i * S + j] = v;
        }
        Sync::sync();
        for (int p = 0; p < NP; p++) {
            const int o = 16 * p;
            if (rank == 0 && warp == 0) {  // (1) diagonal block: lane c (and c + 16) holds column o + c in registers
                const int c = lane & 15;
                Tk col[16];
#pragma unroll
                for (int i = 0; i < 16; i++) col[i] = A[(o + i) * S + o + c];
                Tk *rowk = X;  // row k of R_pp (X is free until the inverse)
                bool ok = true;
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    const Tk d = __shfl_sync(0xffffffffu, col[k], k);  // D_kk, the same in every lane
                    if (kCanDeflate && deflate) {  // a dependent column: R_kk = 1, R_kc = 0, panel row k zero
                        const double g0 = o + k < l ? (double)G[(int64_t)(o + k) * ldg + o + k] : 1.0;
                        const bool dep = !((double)d > tau * g0 && d < Tk(3.0e38));
                        const Tk rinv = dep ? Tk(0) : rsq(d);
                        col[k] = c == k ? (dep ? Tk(1) : d * rinv) : (c > k ? col[k] * rinv : col[k]);
                        if (lane < 16) rowk[c] = col[k];
                        if (lane == 0) {
                            rdiag[o + k] = rinv;
                            if (dep && o + k < l) {
                                fb[o + k] = 1;
                                fb[l] = 1;
                                atomicOr(status, (int)ST_RANKDEF);
                            }
                        }
                        __syncwarp();
#pragma unroll
                        for (int i = k + 1; i < 16; i++) {
                            const Tk rki = rowk[i];
                            if (c >= i) col[i] -= rki * col[k];
                        }
                        __syncwarp();
                        continue;
                    }
                    ok = ok && d > Tk(0) && d < Tk(3.0e38);  // after a breakdown the remaining steps are discarded
                    const Tk rinv = rsq(ok ? d : Tk(1));
                    col[k] = c == k ? d * rinv : (c > k ? col[k] * rinv : col[k]);  // R_kc for c >= k
                    if (lane < 16) rowk[c] = col[k];
                    if (lane == 0) rdiag[o + k] = rinv;
                    __syncwarp();
#pragma unroll
                    for (int i = k + 1; i < 16; i++) {
                        const Tk rki = rowk[i];
                        if (c >= i) col[i] -= rki * col[k];
                    }
                    __syncwarp();
                }
                if (!ok) {
                    if (lane == 0) *bad = 1;
                } else if (lane < 16) {
#pragma unroll
                    for (int i = 0; i < 16; i++) A[(o + i) * S + o + c] = col[i];
                }
            }
            Sync::sync();
            if (*bad) break;
            // (2) panel rows right of the block: R_pp^T x = a for every column c
            for (int c = o + 16 + gt; c < LL; c += gnt) {
                Tk x[16];
#pragma unroll
                for (int k = 0; k < 16; k++) x[k] = A[(o + k) * S + c];
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    x[k] *= rdiag[o + k];
#pragma unroll
                    for (int i = k + 1; i < 16; i++) x[i] -= A[(o + k) * S + o + i] * x[k];
                }
#pragma unroll
                for (int k = 0; k < 16; k++) A[(o + k) * S + c] = x[k];
            }
            Sync::sync();
            // (3) trailing update, blocks p < a <= b
            if constexpr (!GM) {
                for (int a = p + 1; a < NP; a++) {
                    const int i = 16 * a + ty;
                    Tk ri[16];
#pragma unroll
                    for (int k = 0; k < 16; k++) ri[k] = A[(o + k) * S + i];
                    for (int b = a; b < NP; b++) {
                        const int c = 16 * b + tx;
                        Tk acc = A[i * S + c];
#pragma unroll
                        for (int k = 0; k < 16; k++) acc -= ri[k] * A[(o + k) * S + c];
                        A[i * S + c] = acc;
                    }
                }
            } else {  // the triangle of blocks dealt round-robin to the CTAs
                const int na = NP - p - 1, ntri = na * (na + 1) / 2;
                for (int t = rank; t < ntri; t += nct) {
                    int a = p + 1, rem = t;
                    while (rem >= NP - a) {
                        rem -= NP - a;
                        a++;
                    }
                    const int i = 16 * a + ty, c = 16 * (a + rem) + tx;
                    Tk acc = A[i * S + c];
#pragma unroll
                    for (int k = 0; k < 16; k++) acc -= A[(o + k) * S + i] * A[(o + k) * S + c];
                    A[i * S + c] = acc;
                }
            }
            Sync::sync();
        }
        if (!*bad) {
            if (attempt > 0 && rank == 0 && tid == 0) atomicOr(status, attempt == 1 ? (int)ST_SHIFT : (int)ST_CHOL);
            used = attempt;
            break;
        }
        if (role == kCholFirst || role == kCholRetry) {
            if constexpr (!std::is_same<Tk, double>::value) {
                // the float32 arithmetic broke down (its rounding, ~l u of the pivots, can exceed a
                // small positive pivot): factor the same Gram matrix again in float64, in the
                // global scratch, with the CTAs of this launch
                if (ws64) {
                    Sync::sync();
                    chol_retry64<TG, Tc>(G, ldg, l, shift_coef, R, Rinv, Rinv_c, lp, status, ws64, fb);
                    return;
                }
            }
            // breakdown: the float64 Gram matrix and Cholesky take over
            if (rank == 0 && tid == 0) *fb = 1;
            return;
        }
        Sync::sync();
    }
    if ((role == kCholFirst || role == kCholRetry) && rank == 0 && tid == 0) *fb = 0;
    if (kCanDeflate && deflate) {  // a removed column: zero above the diagonal, unit pivot for the inverse
        for (int idx = gt; idx < LL * LL; idx += gnt) {
            const int i = idx / LL, j = idx % LL;
            if (j < l && i < j && reinterpret_cast<volatile int *>(fb)[j]) A[i * S + j] = Tk(0);
        }
        Sync::sync();
        for (int i = gt; i < l; i += gnt)
            if (reinterpret_cast<volatile int *>(fb)[i]) rdiag[i] = Tk(1);
        Sync::sync();
    }
    for (int idx = gt; idx < l * l; idx += gnt) {
        const int i = idx / l, j = idx % l;
        R[idx] = (used < 2 && j >= i) ? (double)A[i * S + j] : 0.0;
    }
    // inverse by row blocks, bottom up
    for (int p = NP - 1; p >= 0; p--) {
        const int o = 16 * p;
        // T = delta I - sum_{p<q<=b} R_pq X_qb for column blocks b >= p (written into X)
        for (int b = p + rank; b < NP; b += nct) {
            const int i = o + ty, c = 16 * b + tx;
            Tk acc = (b == p && ty == tx) ? Tk(1) : Tk(0);
            for (int q = p + 1; q <= b; q++) {
#pragma unroll
                for (int k = 0; k < 16; k++) acc -= A[i * S + 16 * q + k] * X[(16 * q + k) * S + c];
            }
            X[i * S + c] = acc;
        }
        Sync::sync();
        // X_pb = R_pp^{-1} T: back substitution inside the block, one thread per column
        for (int c = o + gt; c < LL; c += gnt) {
            Tk x[16];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = X[(o + k) * S + c];
#pragma unroll
            for (int k = 15; k >= 0; k--) {
                x[k] *= rdiag[o + k];
#pragma unroll
                for (int i = 0; i < k; i++) x[i] -= A[(o + i) * S + o + k] * x[k];
            }
#pragma unroll
            for (int k = 0; k < 16; k++) X[(o + k) * S + c] = x[k];
        }
        Sync::sync();
    }
    for (int idx = gt; idx < l * l; idx += gnt) {
        const int i = idx / l, j = idx % l;
        Rinv[idx] = j >= i ? (double)X[i * S + j] : 0.0;
    }
    for (int idx = gt; idx < lp * lp; idx += gnt) {
        const int i = idx / lp, j = idx % lp;
        Rinv_c[idx] = (i < l && j < l && j >= i) ? (Tc)X[i * S + j] : Tc(0);
    }
}

template <typename TG, typename Tc>
__device__ __noinline__ void chol_retry64(const TG *G, int64_t ldg, int l, double shift_coef, double *R, double *Rinv,
                                          Tc *Rinv_c, int lp, int *status, double *ws64, int *fb) {
    chol_inv_body<TG, double, Tc, true>(G, ldg, l, shift_coef, R, Rinv, Rinv_c, lp, status, ws64, fb, kCholRetry);
}

// ------------------------------------------------ float64 Gram of a float32 block
// 64 x 64 output tiles of the upper triangle (tile pairs ti <= tj), row chunks split over
// gridDim.y; each CTA stages 32 rows of both column tiles in shared memory and accumulates
// 4 x 4 outputs per thread in row order.  The sums are float-float pairs on the FP32 units
// (GB300's float64 rate is ~1/58 of its float32 rate): every product of two float32 values
// is split exactly into p + e (p = fl(ab), e = fma(a, b, -p)), p is added to the running
// sum by an error-free two-sum (Knuth) and the errors are gathered in a second float32
// word: ~2^-48 relative per sum, like a float64 accumulation.  Intrinsics with explicit
// rounding keep the compiler from fusing the steps.
constexpr int G64_TILE = 64, G64_ROWS = 32;

struct G64Split {
    int nt;            // column tiles
    int pairs;         // tile pairs ti <= tj
    int64_t chunks;    // row chunks
    int64_t rpc;       // rows per chunk
    int64_t cap;       // bound of `chunks` that grows with the rows (buffer and grid sizes)
};

__host__ __device__ inline G64Split g64_split(int64_t rows, int l) {
    G64Split sp;
    sp.nt = (l + G64_TILE - 1) / G64_TILE;
    sp.pairs = sp.nt * (sp.nt + 1) / 2;
    int64_t chunks = (304 + sp.pairs - 1) / sp.pairs;
    const int64_t maxc = (rows + 255) / 256;
    if (chunks > maxc) chunks = maxc;
    if (chunks < 1) chunks = 1;
    sp.cap = chunks;
    const int64_t rpc = ((rows + chunks - 1) / chunks + G64_ROWS - 1) / G64_ROWS * G64_ROWS;
    sp.rpc = rpc;
    sp.chunks = (rows + rpc - 1) / rpc;
    return sp;
}

// The CTAs of one job count themselves out on J.count; the last one sums the partials in
// chunk order into G (deterministic), resets the counter and factors G in float64 (the
// Cholesky body with its matrices in the global scratch J.gws, one CTA).
// (hi, lo) += a b: the product split exactly (p + e), p added by an error-free two-sum, the
// rounding errors gathered in lo (explicit rounding intrinsics: no contraction)
__device__ __forceinline__ void ff_madd(float &hi, float &lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(hi, p);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

template <bool TAB>
__global__ void __launch_bounds__(256) gram64_kernel(G64Job job, const G64Job *__restrict__ tab, int l, int64_t ldg) {
    const G64Job J = TAB ? tab[blockIdx.z] : job;
    if (*reinterpret_cast<const volatile int *>(J.fb) == 0) return;
    const G64Split sp = g64_split(J.rows, l);
    const int64_t chunk = blockIdx.y;
    if (chunk >= sp.chunks || (int)blockIdx.x >= sp.pairs) return;
    const unsigned total = (unsigned)(sp.chunks * sp.pairs);
    int ti = 0, p = blockIdx.x;
    while (p >= sp.nt - ti) {
        p -= sp.nt - ti;
        ti++;
    }
    const int tj = ti + p;
    __shared__ float xa[G64_ROWS][G64_TILE + 1], xb[G64_ROWS][G64_TILE + 1];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float sh[4][4], sl[4][4];  // float-float sums: value sh + sl
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) sh[i][j] = sl[i][j] = 0.f;
    const int64_t rb = chunk * sp.rpc, re = min(J.rows, rb + sp.rpc);
    for (int64_t r0 = rb; r0 < re; r0 += G64_ROWS) {
#pragma unroll
        for (int v = 0; v < G64_ROWS * G64_TILE / 256; v++) {
            const int e = tid + 256 * v, rr = e / G64_TILE, cc = e % G64_TILE;
            const int64_t gr = r0 + rr;
            const int ca = G64_TILE * ti + cc, cb = G64_TILE * tj + cc;
            xa[rr][cc] = (gr < re && ca < l) ? J.X[gr * J.ld + ca] : 0.f;
            xb[rr][cc] = (gr < re && cb < l) ? J.X[gr * J.ld + cb] : 0.f;
        }
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < G64_ROWS; k++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = xa[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = xb[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) ff_madd(sh[i][j], sl[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    const int LT = G64_TILE * sp.nt;
    double *out = J.part + chunk * (int64_t)LT * LT;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            out[(int64_t)(G64_TILE * ti + ty * 4 + i) * LT + G64_TILE * tj + tx * 4 + j] =
                (double)sh[i][j] + (double)sl[i][j];
    // G[i][j] (i <= j < l) = sum of the chunk partials in chunk order, by the last CTA
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(J.count, 1u) == total - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int idx = tid; idx < l * l; idx += 256) {
        const int i = idx / l, j = idx % l;
        if (j < i) continue;
        double sum = 0.0;
        for (int64_t c = 0; c < sp.chunks; c++)
            sum += reinterpret_cast<const volatile double *>(J.part)[c * LT * LT + (int64_t)i * LT + j];
        J.G[(int64_t)i * ldg + j] = sum;
    }
    if (tid == 0) *J.count = 0u;
    __threadfence();
    __syncthreads();
    chol_inv_body<double, double, float, true>(J.G, ldg, l, J.coef, J.R, J.Rinv, J.Rc, J.lp, J.status, J.gws,
                                               J.role == kCholDeflate ? J.dflag : const_cast<int *>(J.fb), J.role);
}

// Q (rows x l, ld) = X R^{-1} to ~2^-48 relative, rounded once to float32; Rinv the float64
// l x l upper-triangular inverse (ld l), split into float32 words rh + rl.  Float-float sums
// as in gram64_kernel: x rh exactly as p + e, x rl rounded (its error is 2^-48 of the
// term).  64 x 64 output tiles over a fixed grid; the K range of a tile stops at its last
// column (Rinv is upper triangular).
template <bool TAB>
__global__ void __launch_bounds__(256) rinv64_kernel(Rinv64Job job, const Rinv64Job *__restrict__ tab, int l) {
    const Rinv64Job J = TAB ? tab[blockIdx.z] : job;
    if (*reinterpret_cast<const volatile int *>(J.fb) == 0) return;
    if (J.need && *reinterpret_cast<const volatile int *>(J.need) == 0) return;
    __shared__ float xs[G64_TILE][G64_ROWS + 1], rsh[G64_ROWS][G64_TILE + 1], rsl[G64_ROWS][G64_TILE + 1];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int ct = (l + G64_TILE - 1) / G64_TILE;
    const int64_t rt = (J.rows + G64_TILE - 1) / G64_TILE;
    for (int64_t t = blockIdx.x; t < rt * ct; t += gridDim.x) {
        const int64_t r0 = (t / ct) * G64_TILE;
        const int c0 = (int)(t % ct) * G64_TILE;
        const int kend = min(l, c0 + G64_TILE);
        float sh[4][4], sl[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) sh[i][j] = sl[i][j] = 0.f;
        for (int k0 = 0; k0 < kend; k0 += G64_ROWS) {
#pragma unroll
            for (int v = 0; v < G64_TILE * G64_ROWS / 256; v++) {
                const int e = tid + 256 * v;
                const int xr = e / G64_ROWS, xk = e % G64_ROWS;  // X tile: 64 rows x 32 k
                const int64_t gr = r0 + xr;
                xs[xr][xk] = (gr < J.rows && k0 + xk < l) ? J.X[gr * J.ld + k0 + xk] : 0.f;
                const int rk = e / G64_TILE, rc = e % G64_TILE;  // Rinv tile: 32 k x 64 cols
                const double r = (k0 + rk < l && c0 + rc < l) ? J.Rinv[(int64_t)(k0 + rk) * l + c0 + rc] : 0.0;
                const float rh = __double2float_rn(r);
                rsh[rk][rc] = rh;
                rsl[rk][rc] = __double2float_rn(r - (double)rh);
            }
            __syncthreads();
#pragma unroll 2
            for (int k = 0; k < G64_ROWS; k++) {
                float a[4], bh[4], bl[4];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = xs[ty * 4 + i][k];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    bh[j] = rsh[k][tx * 4 + j];
                    bl[j] = rsl[k][tx * 4 + j];
                }
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        ff_madd(sh[i][j], sl[i][j], a[i], bh[j]);
                        sl[i][j] = __fmaf_rn(a[i], bl[j], sl[i][j]);
                    }
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int64_t r = r0 + ty * 4 + i;
            if (r >= J.rows) break;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int c = c0 + tx * 4 + j;
                if (c >= l) continue;
                if (J.dflag && J.dflag[c]) {  // a removed column: pseudo-random entries (as bk_fill)
                    const double u01 = (double)(splitmix64(J.seed, (uint64_t)(r * J.ld + c)) >> 11) * 0x1.0p-53;
                    J.Q[r * J.ld + c] = (float)(sqrt(3.0 / (double)J.rows) * (2.0 * u01 - 1.0));
                } else {
                    J.Q[r * J.ld + c] = __double2float_rn((double)sh[i][j] + (double)sl[i][j]);
                }
            }
        }
    }
}


template <typename TG, typename Tk, typename Tc, bool GM>
__global__ void __launch_bounds__(256, 1) chol_inv_kernel(const TG *__restrict__ G, int64_t ldg, int l,
                                                          double shift_coef, double *__restrict__ R,
                                                          double *__restrict__ Rinv, Tc *__restrict__ Rinv_c, int lp,
                                                          int *__restrict__ status, Tk *__restrict__ gws, int *fb,
                                                          int role, double *ws64) {
    chol_inv_body<TG, Tk, Tc, GM>(G, ldg, l, shift_coef, R, Rinv, Rinv_c, lp, status, gws, fb, role, ws64);
}

// One CTA per problem of a batch; problem b's pointers and shift are tab[b] (the fallback
// role factors tab[b].G64).
template <typename TG, typename Tk, typename Tc>
__global__ void __launch_bounds__(256, 1) chol_inv_batch_kernel(const CholTab *__restrict__ tab, int64_t ldg, int l,
                                                                int lp, int role) {
    const CholTab t = tab[blockIdx.x];
    const TG *G = static_cast<const TG *>(role == kCholFallback ? static_cast<const void *>(t.G64) : t.G);
    chol_inv_body<TG, Tk, Tc>(G, ldg, l, t.coef, t.R, t.Rinv, static_cast<Tc *>(t.Rc), lp, t.status, nullptr, t.fb,
                              role, t.ws64);
}

// ST_ORTH when max_{i <= j < l} |G_ij - delta_ij| > tol (or not a number): one CTA.
template <typename T>
__device__ __forceinline__ void orth_check_body(const T *__restrict__ G, int l, int64_t ldg, double tol,
                                                int *__restrict__ status) {
    bool bad = false;
    for (int idx = threadIdx.x; idx < l * l; idx += blockDim.x) {
        const int i = idx / l, j = idx % l;
        if (j < i) continue;
        const double e = fabs((double)G[(int64_t)i * ldg + j] - (i == j ? 1.0 : 0.0));
        bad = bad || !(e <= tol);  // also catches NaN
    }
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(status, (int)ST_ORTH);
}

template <typename T>
__global__ void orth_check_kernel(const T *__restrict__ G, int l, int64_t ldg, double tol, int *__restrict__ status) {
    orth_check_body<T>(G, l, ldg, tol, status);
}


__global__ void trmm_upper_kernel(const double *__restrict__ R2, const double *__restrict__ R1, double *__restrict__ R,
                                  int l) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= l * l) return;
    const int i = idx / l, j = idx % l;
    double s = 0.0;
    for (int k = i; k <= j; k++) s += R2[i * l + k] * R1[k * l + j];
    R[idx] = j >= i ? s : 0.0;
}

// ------------------------------------------------------------ one-sided Jacobi
// Blocked one-sided (Hestenes) Jacobi.  The columns of X (= R at the start) and
// of the accumulated rotation V are cut into nb blocks of BW columns.  A sweep
// pairs the blocks in the round-robin order (nb - 1 block rounds, nb / 2 disjoint
// block pairs each); warp w holds the 2 BW columns of its block pair, X and V,
// in registers, NR rows per lane (row i = lane + 32 r), and rotates every
// column pair between the two blocks (BW rounds of BW disjoint pairs; in the
// first block round also the pairs inside each block, BW - 1 rounds) without
// leaving the warp.  One round of BW pairs:
//   gamma_j = x_p . x_q : per-lane partial sums, then a reduce-scatter over the
//                         warp (lane group g ends with the total of pair g);
//   each group computes its rotation from gamma and the tracked squared norms
//   alpha = ||x_p||^2, beta = ||x_q||^2 (rotate when |gamma| > tol sqrt(alpha beta)),
//   c, s and t gamma go to every lane, which rotates its rows of x_p, x_q, v_p,
//   v_q and updates alpha -= t gamma, beta += t gamma (exact for the rotation
//   that zeroes gamma).
// The squared norms are recomputed from the columns whenever a block pair is
// loaded.  The sweep order covers every column pair once; sweeps repeat until
// one rotates nothing.
template <int BW>
__device__ __forceinline__ int rs_index(int lane) {  // pair held by this lane after the reduce-scatter
    return BW == 8 ? ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)
                   : ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
}
template <int BW>
__device__ __forceinline__ int rs_owner(int j) {  // lowest lane holding pair j
    return BW == 8 ? ((j >> 2) & 1) * 16 + ((j >> 1) & 1) * 8 + (j & 1) * 4 : ((j >> 1) & 1) * 16 + (j & 1) * 8;
}

// warp sums of BW per-lane values; lane ends with the total of value rs_index(lane)
template <typename Ta, int BW>
__device__ __forceinline__ Ta reduce_scatter(const Ta (&g)[BW], int lane) {
    Ta h[BW / 2];
    const bool b16 = lane & 16;
#pragma unroll
    for (int j = 0; j < BW / 2; j++) {
        const Ta send = b16 ? g[j] : g[j + BW / 2];
        const Ta keep = b16 ? g[j + BW / 2] : g[j];
        h[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    Ta k[BW / 4];
    const bool b8 = lane & 8;
#pragma unroll
    for (int j = 0; j < BW / 4; j++) {
        const Ta send = b8 ? h[j] : h[j + BW / 4];
        const Ta keep = b8 ? h[j + BW / 4] : h[j];
        k[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    Ta v;
    if constexpr (BW == 8) {
        const bool b4 = lane & 4;
        const Ta send = b4 ? k[0] : k[1];
        v = (b4 ? k[1] : k[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
    } else {
        v = k[0];
        v += __shfl_xor_sync(0xffffffffu, v, 4);
    }
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

// (c, s, t gamma) of the rotation annihilating gamma, or (1, 0, 0) below the
// threshold |gamma| > tol sqrt(alpha beta) (compared squared: tol2 = tol^2)
template <typename Ta>
__device__ __forceinline__ void jrot_t(Ta al, Ta be, Ta ga, Ta tol2, Ta &c, Ta &s, Ta &d, bool &rot) {
    c = Ta(1);
    s = Ta(0);
    d = Ta(0);
    if (ga != Ta(0) && ga * ga > tol2 * (al * be)) {
        Ta t;
        jrot(al, be, ga, c, s, t);
        d = t * ga;
        rot = true;
    }
}

// Pair j of round rd: kind 0 crosses the blocks (column j of the first with
// column (j + rd) mod BW of the second); kind 1 pairs columns inside each block
// (circle method on BW columns, BW / 2 pairs per block).
template <int BW>
__device__ __forceinline__ void bj_pair(int kind, int rd, int j, int &p, int &q) {
    if (kind == 0) {
        p = j;
        q = BW + (j + rd) % BW;
    } else {
        const int k = j % (BW / 2), off = j < BW / 2 ? 0 : BW;
        const int a = rr_pos(k, rd, BW), b = rr_pos(BW - 1 - k, rd, BW);
        p = off + min(a, b);
        q = off + max(a, b);
    }
}

template <typename Ta, int BW, int NR>
__device__ __forceinline__ void bj_round(int kind, int rd, Ta (&x)[2 * BW][NR], Ta (&v)[2 * BW][NR],
                                         Ta (&nr)[2 * BW], Ta tol2, int lane, bool &rot) {
    Ta g[BW];
#pragma unroll
    for (int j = 0; j < BW; j++) {
        int p, q;
        bj_pair<BW>(kind, rd, j, p, q);
        Ta a = Ta(0);
#pragma unroll
        for (int r = 0; r < NR; r++) a = fma(x[p][r], x[q][r], a);
        g[j] = a;
    }
    const Ta ga = reduce_scatter<Ta, BW>(g, lane);
    const int mine = rs_index<BW>(lane);
    Ta al = Ta(0), be = Ta(0);
#pragma unroll
    for (int j = 0; j < BW; j++) {
        int p, q;
        bj_pair<BW>(kind, rd, j, p, q);
        if (j == mine) {
            al = nr[p];
            be = nr[q];
        }
    }
    Ta c, s, d;
    jrot_t(al, be, ga, tol2, c, s, d, rot);
#pragma unroll
    for (int j = 0; j < BW; j++) {
        int p, q;
        bj_pair<BW>(kind, rd, j, p, q);
        const int src = rs_owner<BW>(j);
        const Ta cj = __shfl_sync(0xffffffffu, c, src), sj = __shfl_sync(0xffffffffu, s, src);
        const Ta dj = __shfl_sync(0xffffffffu, d, src);
#pragma unroll
        for (int r = 0; r < NR; r++) {
            const Ta xp = x[p][r], xq = x[q][r];
            x[p][r] = cj * xp - sj * xq;
            x[q][r] = sj * xp + cj * xq;
            const Ta vp = v[p][r], vq = v[q][r];
            v[p][r] = cj * vp - sj * vq;
            v[q][r] = sj * vp + cj * vq;
        }
        nr[p] -= dj;
        nr[q] += dj;
    }
}

// X, V: Lc columns of L rows each (column c at X + c L); rows >= L of a lane are zero.
// Warp w takes block pairs w, w + nwarps, ... of each block round.
// trk: the squared column norms, recomputed from the columns at the start of
// every sweep and carried (updated by the rotations) from block round to block round.
// The block pairs of a round go to the warps of all CTAs of the group (warp w of CTA
// r is warp r * nwarps + w).  rotated: one int in shared memory (CtaSync) or
// max_sweeps zeroed counters in global memory (ClusterSync).
template <typename Ta, int BW, int NR, typename Sync>
__device__ __forceinline__ bool bj_sweeps(Ta *X, Ta *V, Ta *trk, int l, int L, int nb, int max_sweeps,
                                          int *rotated) {
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int warp = Sync::rank() * nwarps + (threadIdx.x >> 5), gwarps = Sync::size() * nwarps;
    const Ta tol = (Ta)(sqrt((double)l) * Eps<Ta>::v), tol2 = tol * tol;
    Ta x[2 * BW][NR], v[2 * BW][NR], nr[2 * BW];
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
        bool rot = false;
        for (int p = warp; p < nb * BW; p += gwarps) {
            Ta ss = Ta(0);
#pragma unroll
            for (int r = 0; r < NR; r++) {
                const int i = lane + 32 * r;
                const Ta xv = i < L ? X[p * L + i] : Ta(0);
                ss = fma(xv, xv, ss);
            }
            ss = warp_sum(ss);
            if (lane == 0) trk[p] = ss;
        }
        Sync::sync();
        for (int br = 0; br < nb - 1; br++) {
          for (int bp = warp; bp < nb / 2; bp += gwarps) {
            const int A = rr_pos(bp, br, nb), B = rr_pos(nb - 1 - bp, br, nb);
#pragma unroll
            for (int c = 0; c < 2 * BW; c++) {
                const int col = (c < BW ? A * BW + c : B * BW + c - BW);
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    const int i = lane + 32 * r;
                    x[c][r] = i < L ? X[col * L + i] : Ta(0);
                    v[c][r] = i < L ? V[col * L + i] : Ta(0);
                }
                nr[c] = trk[col];
            }
            if (br == 0) {
#pragma unroll
                for (int rd = 0; rd < BW - 1; rd++) bj_round<Ta, BW, NR>(1, rd, x, v, nr, tol2, lane, rot);
            }
#pragma unroll
            for (int rd = 0; rd < BW; rd++) bj_round<Ta, BW, NR>(0, rd, x, v, nr, tol2, lane, rot);
#pragma unroll
            for (int c = 0; c < 2 * BW; c++) {
                const int col = (c < BW ? A * BW + c : B * BW + c - BW);
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    const int i = lane + 32 * r;
                    if (i < L) {
                        X[col * L + i] = x[c][r];
                        V[col * L + i] = v[c][r];
                    }
                }
                if (lane == 0) trk[col] = nr[c];
            }
          }
            Sync::sync();
        }
        if constexpr (Sync::size_is_one) {
            if (threadIdx.x == 0) *rotated = 0;
            __syncthreads();
            if (__any_sync(0xffffffffu, rot) && lane == 0) *rotated = 1;
            __syncthreads();
            if (!*rotated) return true;
        } else {
            if (__any_sync(0xffffffffu, rot) && lane == 0) atomicAdd(rotated + sweep, 1);
            Sync::sync();
            if (*reinterpret_cast<volatile int *>(rotated + sweep) == 0) return true;
        }
    }
    return false;
}

// Columns of the blocked sweep: nb blocks of BW (nb even, nb BW >= l).
__host__ __device__ constexpr int bj_blocks(int l, int bw) { return 2 * ((l + 2 * bw - 1) / (2 * bw)); }

// X and V in shared memory, or (gws != NULL: too large for one SM) in the global
// scratch gws (2 Lc L elements, L2-resident); the per-column arrays in shared memory.
template <typename Ta, typename To, int BW, int NR>
__device__ __forceinline__ void jacobi_osvd_body(const double *__restrict__ R, int l, int lp, double *__restrict__ sig,
                                                 To *__restrict__ UR, To *__restrict__ W, int *__restrict__ status,
                                                 int max_sweeps, Ta *gws) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = l + (l & 1);
    const int nb = bj_blocks(l, BW), Lc = nb * BW;
    // NR >= 6 (more than 160 rows) is only used with the global scratch, by the CTAs of
    // a cluster: X, V, the tracked norms and the per-sweep rotation counters in gws
    constexpr bool GM = NR >= 6;
    using Sync = typename std::conditional<GM, ClusterSync, CtaSync>::type;
    Ta *X = GM ? gws : reinterpret_cast<Ta *>(smraw);  // X[p * L + i]: column p of the rotated matrix (Lc columns)
    Ta *V = X + (size_t)Lc * L;                        // V[p * L + i]: column p of the accumulated rotation
    double *nrm = GM ? reinterpret_cast<double *>(smraw)
                     : reinterpret_cast<double *>(V + (size_t)Lc * L + (((size_t)Lc * L) & 1));
    int *perm = reinterpret_cast<int *>(nrm + L);
    __shared__ int rotated;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int gt = Sync::rank() * nt + tid, gnt = Sync::size() * nt;
    for (int idx = gt; idx < Lc * L; idx += gnt) {
        const int p = idx / L, i = idx % L;
        X[idx] = (p < l && i < l) ? (Ta)R[i * l + p] : Ta(0);
        V[idx] = (p == i) ? Ta(1) : Ta(0);
    }
    Ta *trk = GM ? V + (size_t)Lc * L : reinterpret_cast<Ta *>(perm + L) + L;  // (shared: after vn)
    int *rotcnt = GM ? reinterpret_cast<int *>(trk + Lc) : &rotated;
    if (GM && Sync::rank() == 0 && tid < max_sweeps) rotcnt[tid] = 0;
    Sync::sync();
    // rotate when |x_p . x_q| > tol ||x_p|| ||x_q||, tol = sqrt(l) eps: the converged
    // columns are then orthogonal to sqrt(l) eps (an l eps threshold leaves l eps)
    const bool converged = bj_sweeps<Ta, BW, NR, Sync>(X, V, trk, l, L, nb, max_sweeps, rotcnt);
    if (GM && Sync::rank() != 0) return;  // the first CTA sorts and writes the results
    if (!converged && tid == 0) atomicOr(status, (int)ST_NOCONV);
    Ta *nrm_t = reinterpret_cast<Ta *>(nrm);
    for (int p = warp; p < l; p += nw) {
        Ta s = 0;
        for (int i = lane; i < l; i += 32) s += X[p * L + i] * X[p * L + i];
        s = warp_sum(s);
        if (lane == 0) nrm_t[p] = sqrt(s);
    }
    __syncthreads();
    // descending order, stable in the column index: rank of column p among all columns
    for (int p = tid; p < l; p += nt) {
        const Ta v = nrm_t[p];
        int rank = 0;
        for (int j = 0; j < l; j++) {
            const Ta w = nrm_t[j];
            rank += (w > v) || (w == v && j < p);
        }
        perm[rank] = p;
    }
    __syncthreads();
    // the accumulated rotations are orthogonal up to rounding; renormalise their columns
    Ta *vn = reinterpret_cast<Ta *>(perm + L);  // L entries after perm (see the launcher's size)
    for (int p = warp; p < l; p += nw) {
        Ta s = 0;
        for (int i = lane; i < l; i += 32) s += V[p * L + i] * V[p * L + i];
        s = warp_sum(s);
        if (lane == 0) vn[p] = Ta(1) / sqrt(s);
    }
    __syncthreads();
    for (int o = tid; o < l; o += nt) sig[o] = (double)nrm_t[perm[o]];
    for (int idx = tid; idx < lp * lp; idx += nt) {
        const int i = idx / lp, o = idx % lp;
        To u = To(0), w = To(0);
        if (i < l && o < l) {
            const int p = perm[o];
            const Ta sp = nrm_t[p];
            u = sp > Ta(0) ? (To)(X[p * L + i] / sp) : To(0);
            w = (To)(V[p * L + i] * vn[p]);
        }
        UR[idx] = u;
        W[idx] = w;
    }
}

// MAXT threads at most (MAXT / 32 warps), so that the 4 BW NR column registers fit
template <typename Ta, typename To, int BW, int NR, int MAXT>
__global__ void __launch_bounds__(MAXT) jacobi_osvd_kernel(const double *__restrict__ R, int l, int lp,
                                                           double *__restrict__ sig, To *__restrict__ UR,
                                                           To *__restrict__ W, int *__restrict__ status,
                                                           int max_sweeps, Ta *gws) {
    jacobi_osvd_body<Ta, To, BW, NR>(R, l, lp, sig, UR, W, status, max_sweeps, gws);
}

template <typename Ta, typename To, int BW, int NR, int MAXT>
__global__ void __launch_bounds__(MAXT) jacobi_osvd_batch_kernel(const JacTab *__restrict__ tab, int l, int lp,
                                                                 int max_sweeps) {
    const JacTab t = tab[blockIdx.x];
    jacobi_osvd_body<Ta, To, BW, NR>(t.R, l, lp, t.sig, static_cast<To *>(t.UR), static_cast<To *>(t.W), t.status,
                                     max_sweeps, nullptr);
}

// sig[i] = x_i^T R w_i / (||x_i|| ||w_i||) in float64 for the columns x_i of UR and
// w_i of W (ld lp): the Rayleigh quotient of the Jacobi singular vectors, whose
// error is quadratic in the vectors' error.  One block per singular value.
template <typename To>
__device__ __forceinline__ void sv_refine_body(const double *__restrict__ R, int l, int lp, const To *__restrict__ UR,
                                               const To *__restrict__ W, double *__restrict__ sig, int i) {
    __shared__ double red[3][32];
    double acc = 0.0, nx = 0.0, nw = 0.0;
    for (int r = threadIdx.x; r < l; r += blockDim.x) {
        double rw = 0.0;
        for (int c = r; c < l; c++) rw += R[r * l + c] * (double)W[c * lp + i];   // R upper triangular or bidiagonal
        const double x = (double)UR[r * lp + i];
        acc += x * rw;
        nx += x * x;
        const double w = (double)W[r * lp + i];
        nw += w * w;
    }
    acc = warp_sum(acc);
    nx = warp_sum(nx);
    nw = warp_sum(nw);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][wid] = acc; red[1][wid] = nx; red[2][wid] = nw; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, x = 0.0, w = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) { a += red[0][k]; x += red[1][k]; w += red[2][k]; }
        if (x > 0.0 && w > 0.0) sig[i] = fabs(a) / sqrt(x * w);
    }
}

template <typename To>
__global__ void sv_refine_kernel(const double *__restrict__ R, int l, int lp, const To *__restrict__ UR,
                                 const To *__restrict__ W, double *__restrict__ sig) {
    sv_refine_body<To>(R, l, lp, UR, W, sig, blockIdx.x);
}

// blockIdx.x: singular value, blockIdx.y: problem of the batch
template <typename To>
__global__ void sv_refine_batch_kernel(const JacTab *__restrict__ tab, int l, int lp) {
    const JacTab t = tab[blockIdx.y];
    sv_refine_body<To>(t.R, l, lp, static_cast<const To *>(t.UR), static_cast<const To *>(t.W), t.sig, blockIdx.x);
}

// ------------------------------------------------------------ two-sided Jacobi
// Arithmetic in Tm (float64 for the Gram route; float32 for the block Gram matrices of
// SVQB).  A pair is rotated when |g_pq| > rel sqrt(|g_pp g_qq|) and |g_pq| > floor_rel *
// max_i g_ii: the floor (0 for the Gram route) stops rotations among directions far
// below what the caller resolves, which a relative test alone never finishes in float32.
template <typename Tm>
__global__ void __launch_bounds__(1024) jacobi_eig_kernel(const double *__restrict__ G, int n,
                                                          double *__restrict__ lam, double *__restrict__ Vout,
                                                          int *__restrict__ status, int max_sweeps,
                                                          double floor_rel) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = n + (n & 1);
    Tm *M = reinterpret_cast<Tm *>(smraw);  // n x n, row-major
    Tm *Vt = M + n * n;                     // Vt[p * n + i] = V[i][p]
    Tm *cs = Vt + n * n;                    // per pair: c, s
    int *pq = reinterpret_cast<int *>(cs + L + (L & 1));  // per pair: p, q (or -1)
    int *perm = pq + L;
    __shared__ int rotated;
    __shared__ Tm floor_s;
    const int tid = threadIdx.x, nt = blockDim.x, np = L / 2;
    for (int idx = tid; idx < n * n; idx += nt) {
        M[idx] = (Tm)G[idx];
        Vt[idx] = (idx / n == idx % n) ? Tm(1) : Tm(0);
    }
    const Tm rel = sizeof(Tm) == 8 ? Tm(1e-15) : (Tm)(sqrt((double)n) * FLT_EPSILON);
    if (tid == 0) {
        double dmax = 0.0;
        for (int i = 0; i < n; i++) dmax = fmax(dmax, G[(int64_t)i * n + i]);
        floor_s = (Tm)(floor_rel * dmax);
    }
    bool converged = false;
    __syncthreads();
    const Tm floor_v = floor_s;
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < L - 1; r++) {
            for (int pr = tid; pr < np; pr += nt) {
                const int a = rr_pos(pr, r, L), b = rr_pos(L - 1 - pr, r, L);
                int p = min(a, b), q = max(a, b);
                Tm c = 1, s = 0;
                if (q < n) {
                    const Tm apq = M[p * n + q], app = M[p * n + p], aqq = M[q * n + q];
                    // sqrt of each diagonal entry: their product overflows float32 for column
                    // norms above ~4e9, which would stop every rotation
                    if (apq != Tm(0) && fabs(apq) > rel * (sqrt(fabs(app)) * sqrt(fabs(aqq))) &&
                        fabs(apq) > floor_v) {
                        const Tm theta = (aqq - app) / (Tm(2) * apq);
                        const Tm t = (theta >= Tm(0) ? Tm(1) : Tm(-1)) / (fabs(theta) + sqrt(Tm(1) + theta * theta));
                        c = Tm(1) / sqrt(Tm(1) + t * t);
                        s = t * c;
                        rotated = 1;
                    } else {
                        p = -1;
                    }
                } else {
                    p = -1;
                }
                cs[2 * pr] = c;
                cs[2 * pr + 1] = s;
                pq[2 * pr] = p;
                pq[2 * pr + 1] = q;
            }
            __syncthreads();
            // M <- M J and V <- V J (columns p, q of every active pair)
            for (int idx = tid; idx < np * n; idx += nt) {
                const int pr = idx / n, i = idx % n, p = pq[2 * pr];
                if (p < 0) continue;
                const int q = pq[2 * pr + 1];
                const Tm c = cs[2 * pr], s = cs[2 * pr + 1];
                const Tm x = M[i * n + p], y = M[i * n + q];
                M[i * n + p] = c * x - s * y;
                M[i * n + q] = s * x + c * y;
                const Tm vx = Vt[p * n + i], vy = Vt[q * n + i];
                Vt[p * n + i] = c * vx - s * vy;
                Vt[q * n + i] = s * vx + c * vy;
            }
            __syncthreads();
            // M <- J^T M (rows p, q)
            for (int idx = tid; idx < np * n; idx += nt) {
                const int pr = idx / n, j = idx % n, p = pq[2 * pr];
                if (p < 0) continue;
                const int q = pq[2 * pr + 1];
                const Tm c = cs[2 * pr], s = cs[2 * pr + 1];
                const Tm x = M[p * n + j], y = M[q * n + j];
                M[p * n + j] = c * x - s * y;
                M[q * n + j] = s * x + c * y;
            }
            __syncthreads();
            for (int pr = tid; pr < np; pr += nt) {
                const int p = pq[2 * pr];
                if (p < 0) continue;
                const int q = pq[2 * pr + 1];
                M[p * n + q] = Tm(0);
                M[q * n + p] = Tm(0);
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) { converged = true; break; }
    }
    if (!converged && tid == 0) atomicOr(status, (int)ST_NOCONV);
    if (tid == 0) {
        for (int i = 0; i < n; i++) perm[i] = i;
        for (int i = 0; i < n; i++) {
            int best = i;
            for (int j = i + 1; j < n; j++)
                if (M[perm[j] * n + perm[j]] > M[perm[best] * n + perm[best]]) best = j;
            const int t = perm[i]; perm[i] = perm[best]; perm[best] = t;
        }
    }
    __syncthreads();
    for (int o = tid; o < n; o += nt) lam[o] = (double)M[perm[o] * n + perm[o]];
    for (int idx = tid; idx < n * n; idx += nt) {
        const int i = idx / n, o = idx % n;
        Vout[idx] = (double)Vt[perm[o] * n + i];
    }
}

template <typename T>
__global__ void gram_finish_kernel(const double *__restrict__ lam, const double *__restrict__ V, int n,
                                   double *__restrict__ sig, T *__restrict__ Vs, int *__restrict__ status) {
    __shared__ double thr;
    if (threadIdx.x == 0) {
        const double s1 = sqrt(fmax(lam[0], 0.0));
        thr = (double)n * DBL_EPSILON * s1;
        int rd = 0;
        for (int i = 0; i < n; i++)
            if (!(sqrt(fmax(lam[i], 0.0)) > thr)) rd = 1;
        if (rd) atomicOr(status, (int)ST_RANKDEF);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) sig[i] = sqrt(fmax(lam[i], 0.0));
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int j = idx % n;
        const double s = sqrt(fmax(lam[j], 0.0));
        Vs[idx] = s > thr ? (T)(V[idx] / s) : T(0);
    }
}

template <typename T>
__global__ void sign_normalize_kernel(T *__restrict__ Vt, int64_t rows, int64_t ldv, T *__restrict__ W,
                                      int64_t wrows, int64_t ldw) {
    __shared__ double bv[32];
    __shared__ int64_t bi[32];
    __shared__ int flip;
    const int j = blockIdx.x;
    double best = -1.0;
    int64_t bidx = 0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
        const double a = fabs((double)Vt[r * ldv + j]);
        if (a > best) { best = a; bidx = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) { bv[w] = best; bi[w] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = bv[0];
        int64_t i0 = bi[0];
        for (int k = 1; k < nw; k++)
            if (bv[k] > b || (bv[k] == b && bi[k] < i0)) { b = bv[k]; i0 = bi[k]; }
        flip = Vt[i0 * ldv + j] < T(0);
    }
    __syncthreads();
    if (!flip) return;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) Vt[r * ldv + j] = -Vt[r * ldv + j];
    for (int64_t r = threadIdx.x; r < wrows; r += blockDim.x) W[r * ldw + j] = -W[r * ldw + j];
}

template <typename Ts, typename Td>
__global__ void copy2d_kernel(const Ts *__restrict__ src, int64_t lds, Td *__restrict__ dst, int64_t ldd,
                              int64_t rows, int64_t cols, int64_t cols_pad) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols_pad) return;
    const int64_t r = idx / cols_pad, c = idx % cols_pad;
    dst[r * ldd + c] = c < cols ? (Td)src[r * lds + c] : Td(0);
}

__global__ void copy_f64_kernel(const double *__restrict__ src, double *__restrict__ dst, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = src[i];
}

__global__ void pca_select_kernel(const double *__restrict__ sigma, int count, const double *__restrict__ fro2,
                                  double t, int *__restrict__ K, int *__restrict__ reached) {
    if (threadIdx.x != 0) return;
    const double target = t * (*fro2);
    double acc = 0.0;
    for (int i = 0; i < count; i++) {
        acc += sigma[i] * sigma[i];
        if (acc >= target) { *K = i + 1; *reached = 1; return; }
    }
    *K = count;
    *reached = 0;
}

// shared memory of the blocked Cholesky: A and X (16 NP rows of stride S) and the pivots
template <typename Tk>
size_t chol_smem_bytes(int l) {
    const int LL = 16 * ((l + 15) / 16), S = LL + (sizeof(Tk) == 4 ? 16 : 1);
    return sizeof(Tk) * (2 * (size_t)LL * S + LL);
}

}  // namespace

int64_t gram64_partials(int64_t rows, int l) {
    const G64Split sp = g64_split(rows, l);
    return sp.cap * (int64_t)(G64_TILE * sp.nt) * (G64_TILE * sp.nt);
}

cudaError_t gram64_fb(const G64Job &job, int l, int64_t ldg, cudaStream_t s) {
    if (l < 1 || !job.fb || !job.count || !job.gws) return cudaErrorInvalidValue;
    const G64Split sp = g64_split(job.rows, l);
    gram64_kernel<false><<<dim3(sp.pairs, (unsigned)sp.chunks, 1), 256, 0, s>>>(job, nullptr, l, ldg);
    note_launch();
    return cudaGetLastError();
}

cudaError_t gram64_fb_batched(const G64Job *tab, int count, int64_t max_rows, int l, int64_t ldg, cudaStream_t s) {
    if (count < 1) return cudaSuccess;
    const G64Split sp = g64_split(max_rows, l);  // the chunk bound grows with the rows: enough for every job
    G64Job none = {};
    // a job's CTAs beyond its own chunk count return before counting themselves out
    gram64_kernel<true><<<dim3(sp.pairs, (unsigned)sp.cap, count), 256, 0, s>>>(none, tab, l, ldg);
    note_launch();
    return cudaGetLastError();
}

cudaError_t rinv64_fb(const Rinv64Job &job, int l, cudaStream_t s) {
    if (l < 1 || !job.fb) return cudaErrorInvalidValue;
    rinv64_kernel<false><<<dim3(304, 1, 1), 256, 0, s>>>(job, nullptr, l);
    note_launch();
    return cudaGetLastError();
}

void set_sweep_cap(int cap) { g_sweep_cap.store(cap > 0 ? cap : 0, std::memory_order_relaxed); }

size_t chol_scratch_bytes(int l, size_t tk) {
    const int LL = 16 * ((l + 15) / 16), S = LL + (tk == 4 ? 16 : 1);
    return tk * (2 * (size_t)LL * S + ((LL + 1) & ~1)) + 2 * sizeof(double);  // A, X, pivots, trace, flag
}

template <typename TG, typename Tk, typename Tc>
cudaError_t chol_inv(const TG *G, int64_t ldg, int l, int64_t rows, double u, double *R, double *Rinv, Tc *Rinv_c,
                     int lp, int *status, cudaStream_t s, void *scratch, int *fb, int role) {
    if (role != kCholPlain && !fb) return cudaErrorInvalidValue;
    // the float64 retry of a float32 first attempt: the scratch holds a float64 l x l pair
    double *ws64 = (role == kCholFirst && sizeof(Tk) == 4) ? static_cast<double *>(scratch) : nullptr;
    const double coef = chol_shift_coef(rows, l, u);
    size_t smem = chol_smem_bytes<Tk>(l);
    Tk *gws = nullptr;
    if (smem > 227 * 1024) {  // matrices and pivots in the global scratch
        if (!scratch) return cudaErrorInvalidValue;
        gws = static_cast<Tk *>(scratch);
        smem = 0;
    }
    if (gws) {  // a cluster of 8 CTAs
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(8);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 8;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, chol_inv_kernel<TG, Tk, Tc, true>, G, ldg, l, coef, R, Rinv, Rinv_c, lp, status, gws,
                           fb, role, ws64);
    } else {
        cudaFuncSetAttribute(chol_inv_kernel<TG, Tk, Tc, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        chol_inv_kernel<TG, Tk, Tc, false><<<1, 256, smem, s>>>(G, ldg, l, coef, R, Rinv, Rinv_c, lp, status, nullptr,
                                                                fb, role, ws64);
    }
    note_launch();
    return cudaGetLastError();
}

template <typename TG, typename Tk, typename Tc>
cudaError_t chol_inv_batched(const CholTab *tab, int count, int64_t ldg, int l, int lp, cudaStream_t s, int role) {
    if (count < 1) return cudaSuccess;
    const size_t smem = chol_smem_bytes<Tk>(l);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(chol_inv_batch_kernel<TG, Tk, Tc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    chol_inv_batch_kernel<TG, Tk, Tc><<<count, 256, smem, s>>>(tab, ldg, l, lp, role);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t orth_check(const T *G, int l, int64_t ldg, double tol, int *status, cudaStream_t s) {
    orth_check_kernel<T><<<1, 256, 0, s>>>(G, l, ldg, tol, status);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t orth_check<float>(const float *, int, int64_t, double, int *, cudaStream_t);
template cudaError_t orth_check<double>(const double *, int, int64_t, double, int *, cudaStream_t);

double chol_shift_coef(int64_t rows, int l, double u) { return 11.0 * ((double)rows * l + (double)l * (l + 1)) * u; }

cudaError_t trmm_upper(const double *R2, const double *R1, double *R, int l, cudaStream_t s) {
    trmm_upper_kernel<<<(l * l + 255) / 256, 256, 0, s>>>(R2, R1, R, l);
    note_launch();
    return cudaGetLastError();
}

// Block width and rows per lane of the blocked Jacobi for an l x l factor:
// 8-column blocks for float32 of 65..128 columns, else 4 (register budget);
// rows per lane ceil(L / 32).
template <typename Ta>
void jacobi_shape(int l, int &bw, int &nr) {
    const int L = l + (l & 1);
    nr = (L + 31) / 32;
    bw = (sizeof(Ta) == 4 && l > 64 && L <= 128) ? 8 : 4;
}

template <typename Ta>
size_t jacobi_smem(int l, int bw) {
    const int L = l + (l & 1);
    const size_t cells = (size_t)bj_blocks(l, bw) * bw * L;
    // X, V (cells each), norms (L doubles), permutation (L ints), column scales (L x Ta),
    // tracked squared norms (nb bw x Ta)
    return sizeof(Ta) * (2 * cells + 1) + sizeof(double) * L + sizeof(int) * L + sizeof(double) * L +
           sizeof(double) * (size_t)bj_blocks(l, bw) * bw + 16;
}

// the per-column arrays only (X and V in the global scratch)
template <typename Ta>
size_t jacobi_smem_small(int l, int bw) {
    const int L = l + (l & 1);
    return sizeof(double) * L + sizeof(int) * L + sizeof(double) * L + sizeof(double) * (size_t)bj_blocks(l, bw) * bw +
           16;
}

template <typename Ta, typename To, int BW, int NR>
void launch_jacobi(const JacTab *tab, int count, const double *R, int l, int lp, double *sig, To *UR, To *W,
                   int *status, cudaStream_t s, Ta *gws) {
    // float64, the 8-wide blocks and 5 or more rows per lane need up to 255 registers: 8 warps; else 16
    constexpr int MAXT = (sizeof(Ta) == 8 || BW == 8 || NR >= 5) ? 256 : 512;
    const size_t smem = gws ? jacobi_smem_small<Ta>(l, BW) : jacobi_smem<Ta>(l, BW);
    const int threads = 32 * std::min(bj_blocks(l, BW) / 2, MAXT / 32);
    if (tab) {
        cudaFuncSetAttribute(jacobi_osvd_batch_kernel<Ta, To, BW, NR, MAXT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        jacobi_osvd_batch_kernel<Ta, To, BW, NR, MAXT><<<count, threads, smem, s>>>(tab, l, lp, sweep_cap(40));
    } else if (gws) {  // a cluster of up to 8 CTAs (one warp per block pair where possible)
        auto kern = jacobi_osvd_kernel<Ta, To, BW, NR, MAXT>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int pairs = bj_blocks(l, BW) / 2;
        const int csize = std::max(1, std::min(8, (pairs + MAXT / 32 - 1) / (MAXT / 32)));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)csize);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, kern, R, l, lp, sig, UR, W, status, sweep_cap(40), gws);
    } else {
        cudaFuncSetAttribute(jacobi_osvd_kernel<Ta, To, BW, NR, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        jacobi_osvd_kernel<Ta, To, BW, NR, MAXT><<<1, threads, smem, s>>>(R, l, lp, sig, UR, W, status,
                                                                          sweep_cap(40), gws);
    }
}

template <typename Ta, typename To>
cudaError_t jacobi_dispatch(const JacTab *tab, int count, const double *R, int l, int lp, double *sig, To *UR,
                            To *W, int *status, cudaStream_t s, void *scratch) {
    int bw, nr;
    jacobi_shape<Ta>(l, bw, nr);
    Ta *gws = nullptr;
    if (nr >= 6) {  // X and V in the global scratch (single problems only)
        if (tab || !scratch) return cudaErrorInvalidValue;
        gws = static_cast<Ta *>(scratch);
    }
    if (nr > (sizeof(Ta) == 8 ? 4 : 9) || (!gws && jacobi_smem<Ta>(l, bw) > 227 * 1024)) return cudaErrorInvalidValue;
    if constexpr (sizeof(Ta) == 4) {
        if (bw == 8) {
            switch (nr) {
                case 3: launch_jacobi<Ta, To, 8, 3>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
                default: launch_jacobi<Ta, To, 8, 4>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
            }
            note_launch();
            return cudaGetLastError();
        }
    }
    switch (nr) {
        case 1: launch_jacobi<Ta, To, 4, 1>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
        case 2: launch_jacobi<Ta, To, 4, 2>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
        case 3: launch_jacobi<Ta, To, 4, 3>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
        case 4: launch_jacobi<Ta, To, 4, 4>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
        default:
            if constexpr (sizeof(Ta) == 4) {
                switch (nr) {
                    case 5: launch_jacobi<Ta, To, 4, 5>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
                    case 6: launch_jacobi<Ta, To, 4, 6>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
                    case 7: launch_jacobi<Ta, To, 4, 7>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
                    case 8: launch_jacobi<Ta, To, 4, 8>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
                    default: launch_jacobi<Ta, To, 4, 9>(tab, count, R, l, lp, sig, UR, W, status, s, gws); break;
                }
            }
            break;
    }
    note_launch();
    return cudaGetLastError();
}

size_t jacobi_scratch_bytes(int l, size_t ta) {
    const int L = l + (l & 1);
    const int bw = (ta == 4 && l > 64 && L <= 128) ? 8 : 4;
    const size_t lc = (size_t)bj_blocks(l, bw) * bw;
    return ta * (2 * lc * L + lc) + 64 * sizeof(int);  // X, V, tracked norms, rotation counters
}

template <typename Ta, typename To>
cudaError_t jacobi_osvd(const double *R, int l, int lp, double *sig, To *UR, To *W, int *status, cudaStream_t s,
                        void *scratch) {
    return jacobi_dispatch<Ta, To>(nullptr, 1, R, l, lp, sig, UR, W, status, s, scratch);
}

template <typename Ta, typename To>
cudaError_t jacobi_osvd_batched(const JacTab *tab, int count, int l, int lp, cudaStream_t s) {
    if (count < 1) return cudaSuccess;
    return jacobi_dispatch<Ta, To>(tab, count, nullptr, l, lp, nullptr, nullptr, nullptr, nullptr, s, nullptr);
}

template <typename To>
cudaError_t sv_refine_batched(const JacTab *tab, int count, int l, int lp, cudaStream_t s) {
    if (count < 1) return cudaSuccess;
    sv_refine_batch_kernel<To><<<dim3(l, count), 128, 0, s>>>(tab, l, lp);
    note_launch();
    return cudaGetLastError();
}

template <typename To>
cudaError_t sv_refine(const double *R, int l, int lp, const To *UR, const To *W, double *sig, cudaStream_t s) {
    sv_refine_kernel<To><<<l, 128, 0, s>>>(R, l, lp, UR, W, sig);
    note_launch();
    return cudaGetLastError();
}
template cudaError_t sv_refine<float>(const double *, int, int, const float *, const float *, double *, cudaStream_t);
template cudaError_t sv_refine_batched<float>(const JacTab *, int, int, int, cudaStream_t);
template cudaError_t sv_refine_batched<double>(const JacTab *, int, int, int, cudaStream_t);
template cudaError_t jacobi_osvd_batched<float, float>(const JacTab *, int, int, int, cudaStream_t);
template cudaError_t jacobi_osvd_batched<double, double>(const JacTab *, int, int, int, cudaStream_t);
template cudaError_t chol_inv_batched<float, float, float>(const CholTab *, int, int64_t, int, int, cudaStream_t, int);
template cudaError_t chol_inv_batched<double, double, double>(const CholTab *, int, int64_t, int, int, cudaStream_t,
                                                              int);
template cudaError_t chol_inv_batched<double, double, float>(const CholTab *, int, int64_t, int, int, cudaStream_t,
                                                             int);
template cudaError_t sv_refine<double>(const double *, int, int, const double *, const double *, double *,
                                       cudaStream_t);

template <typename Tm>
cudaError_t jacobi_eig_t(const double *G, int n, double *lam, double *V, int *status, cudaStream_t s,
                         double floor_rel) {
    const int L = n + (n & 1);
    const size_t smem = sizeof(Tm) * (2 * (size_t)n * n + L + (L & 1)) + sizeof(int) * (2 * L) + 16;
    if (n < 1 || smem > 227 * 1024) return cudaErrorInvalidValue;  // one CTA holds M and V
    const cudaError_t e = cudaFuncSetAttribute(jacobi_eig_kernel<Tm>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
    jacobi_eig_kernel<Tm><<<1, 1024, smem, s>>>(G, n, lam, V, status, sweep_cap(50), floor_rel);
    note_launch();
    return cudaGetLastError();
}

cudaError_t jacobi_eig(const double *G, int n, double *lam, double *V, int *status, cudaStream_t s) {
    return jacobi_eig_t<double>(G, n, lam, V, status, s, 0.0);
}

cudaError_t jacobi_eig_f32(const double *G, int n, double *lam, double *V, int *status, cudaStream_t s,
                           double floor_rel) {
    return jacobi_eig_t<float>(G, n, lam, V, status, s, floor_rel);
}

template <typename T>
cudaError_t gram_finish(const double *lam, const double *V, int n, double *sig, T *Vs, int *status,
                        cudaStream_t s) {
    gram_finish_kernel<T><<<1, 256, 0, s>>>(lam, V, n, sig, Vs, status);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sign_normalize(T *Vt, int64_t rows, int cols, int64_t ldv, T *W, int64_t wrows, int64_t ldw,
                           cudaStream_t s) {
    if (cols <= 0) return cudaSuccess;
    sign_normalize_kernel<T><<<cols, 256, 0, s>>>(Vt, rows, ldv, W, wrows, ldw);
    note_launch();
    return cudaGetLastError();
}

template <typename Ts, typename Td>
cudaError_t copy2d(const Ts *src, int64_t lds, Td *dst, int64_t ldd, int64_t rows, int64_t cols, int64_t cols_pad,
                   cudaStream_t s) {
    const int64_t total = rows * cols_pad;
    if (total <= 0) return cudaSuccess;
    copy2d_kernel<Ts, Td><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols, cols_pad);
    note_launch();
    return cudaGetLastError();
}

cudaError_t copy_f64(const double *src, double *dst, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    copy_f64_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, s>>>(src, dst, count);
    note_launch();
    return cudaGetLastError();
}

cudaError_t pca_select(const double *sigma, int count, const double *fro2, double t, int *K, int *reached,
                       cudaStream_t s) {
    pca_select_kernel<<<1, 32, 0, s>>>(sigma, count, fro2, t, K, reached);
    note_launch();
    return cudaGetLastError();
}

#define INST_CHOL(TG, TK, TC)                                                                                   \
    template cudaError_t chol_inv<TG, TK, TC>(const TG *, int64_t, int, int64_t, double, double *, double *, TC *, \
                                              int, int *, cudaStream_t, void *, int *, int);
INST_CHOL(float, float, float)
INST_CHOL(float, double, float)
INST_CHOL(double, double, double)
INST_CHOL(double, double, float)
template cudaError_t jacobi_osvd<float, float>(const double *, int, int, double *, float *, float *, int *,
                                               cudaStream_t, void *);
template cudaError_t jacobi_osvd<double, float>(const double *, int, int, double *, float *, float *, int *,
                                                cudaStream_t, void *);
template cudaError_t jacobi_osvd<double, double>(const double *, int, int, double *, double *, double *, int *,
                                                 cudaStream_t, void *);
template cudaError_t gram_finish<float>(const double *, const double *, int, double *, float *, int *, cudaStream_t);
template cudaError_t gram_finish<double>(const double *, const double *, int, double *, double *, int *,
                                         cudaStream_t);
template cudaError_t sign_normalize<float>(float *, int64_t, int, int64_t, float *, int64_t, int64_t, cudaStream_t);
template cudaError_t sign_normalize<double>(double *, int64_t, int, int64_t, double *, int64_t, int64_t,
                                            cudaStream_t);
#define INST_COPY(TS, TD)                                                                                      \
    template cudaError_t copy2d<TS, TD>(const TS *, int64_t, TD *, int64_t, int64_t, int64_t, int64_t, cudaStream_t);
INST_COPY(float, float)
INST_COPY(double, double)
INST_COPY(float, double)
INST_COPY(double, float)

}  // namespace gbr
