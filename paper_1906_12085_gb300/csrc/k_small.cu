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

#include "common.cuh"

namespace gbr {
namespace {

__device__ __forceinline__ int rr_pos(int k, int r, int L) {
    // position k of round r in the circle method: player 0 fixed, the rest rotate
    return k == 0 ? 0 : 1 + ((k - 1 + r) % (L - 1));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = FLT_EPSILON; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };

// ------------------------------------------------------------ Cholesky + inverse
// Right-looking upper Cholesky R^T R = G with one barrier per column: the
// scaled row j of R goes to a separate buffer, so the trailing update (which
// reads the unscaled row j of the working matrix) never races with it.  The
// inverse solves R x = e_c column by column, one column per thread, with no
// barriers (R is read-only by then).  Arithmetic in Tk.
template <typename TG, typename Tk, typename Tc>
__global__ void chol_inv_kernel(const TG *__restrict__ G, int64_t ldg, int l, double shift_coef,
                                double *__restrict__ R, double *__restrict__ Rinv, Tc *__restrict__ Rinv_c, int lp,
                                int *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Tk *M = reinterpret_cast<Tk *>(smraw);  // l x l working matrix (upper triangle)
    Tk *Rs = M + l * l;                     // l x l factor R (upper), then its inverse in place by columns
    __shared__ double trace;
    const int tid = threadIdx.x, nt = blockDim.x;
    int used = 0;  // 0: plain, 1: shifted, 2: breakdown fallback (R = 0, R^{-1} = I)
    for (int attempt = 0; attempt < 3; attempt++) {
        for (int idx = tid; idx < l * l; idx += nt) {
            const int i = idx / l, j = idx % l;
            M[idx] = attempt == 2 ? Tk(i == j ? 1 : 0) : (Tk)G[(int64_t)min(i, j) * ldg + max(i, j)];
            Rs[idx] = Tk(0);
        }
        __syncthreads();
        if (tid == 0) {
            double tr = 0.0;
            for (int i = 0; i < l; i++) tr += (double)M[i * l + i];
            trace = tr;
        }
        __syncthreads();
        if (attempt == 1) {  // shifted CholeskyQR: G + s I with s = 11 (rows l + l(l+1)) u tr(G)
            const Tk sh = (Tk)(shift_coef * trace);
            for (int i = tid; i < l; i += nt) M[i * l + i] += sh;
            __syncthreads();
        }
        bool bad = false;
        for (int j = 0; j < l; j++) {
            const Tk d = M[j * l + j];
            if (!(d > Tk(0)) || !isfinite((double)d)) { bad = true; break; }  // uniform: every thread reads d
            const Tk rinv = Tk(1) / sqrt(d), dinv = Tk(1) / d;
            for (int c = j + tid; c < l; c += nt) Rs[j * l + c] = M[j * l + c] * rinv;
            const int nr = l - j - 1;
            for (int idx = tid; idx < nr * nr; idx += nt) {
                const int r = j + 1 + idx / nr, c = j + 1 + idx % nr;
                if (c >= r) M[r * l + c] -= M[j * l + r] * M[j * l + c] * dinv;
            }
            __syncthreads();
        }
        if (!bad) {
            if (attempt > 0 && tid == 0) atomicOr(status, attempt == 1 ? (int)ST_SHIFT : (int)ST_CHOL);
            used = attempt;
            break;
        }
        __syncthreads();
    }
    for (int idx = tid; idx < l * l; idx += nt) R[idx] = used < 2 ? (double)Rs[idx] : 0.0;
    __syncthreads();
    // column c of R^{-1}: back substitution R x = e_c (rows c..0), written over column c of Rs
    Tk *X = M;  // reuse: X[i * l + c]
    for (int c = tid; c < l; c += nt) {
        for (int i = 0; i < l; i++) X[i * l + c] = Tk(0);
        for (int k = c; k >= 0; k--) {
            Tk acc = (k == c) ? Tk(1) : Tk(0);
            for (int t = k + 1; t <= c; t++) acc -= Rs[k * l + t] * X[t * l + c];
            X[k * l + c] = acc / Rs[k * l + k];
        }
    }
    __syncthreads();
    for (int idx = tid; idx < l * l; idx += nt) {
        const int i = idx / l, j = idx % l;
        Rinv[idx] = j >= i ? (double)X[idx] : 0.0;
    }
    for (int idx = tid; idx < lp * lp; idx += nt) {
        const int i = idx / lp, j = idx % lp;
        Rinv_c[idx] = (i < l && j < l && j >= i) ? (Tc)X[i * l + j] : Tc(0);
    }
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
template <typename Ta, typename To>
__global__ void __launch_bounds__(1024) jacobi_osvd_kernel(const double *__restrict__ R, int l, int lp,
                                                           double *__restrict__ sig, To *__restrict__ UR,
                                                           To *__restrict__ W, int *__restrict__ status,
                                                           int max_sweeps, int gsize) {
    // gsize lanes (16 or 32) rotate one column pair; a warp holds 32 / gsize pairs
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = l + (l & 1);
    Ta *X = reinterpret_cast<Ta *>(smraw);  // X[p * L + i]: column p of the rotated matrix
    Ta *V = X + L * L;                       // V[p * L + i]: column p of the accumulated rotation
    double *nrm = reinterpret_cast<double *>(V + L * L + ((L * L) & 1));
    int *perm = reinterpret_cast<int *>(nrm + L);
    __shared__ int rotated;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int gl = lane % gsize, gpw = 32 / gsize;               // lane in group, groups per warp
    const int grp = warp * gpw + lane / gsize, ngrp = nw * gpw;
    const unsigned gmask = gsize == 32 ? 0xffffffffu : (0xffffu << (lane & 16));
    for (int idx = tid; idx < L * L; idx += nt) {
        const int p = idx / L, i = idx % L;
        X[idx] = (p < l && i < l) ? (Ta)R[i * l + p] : Ta(0);
        V[idx] = (p == i) ? Ta(1) : Ta(0);
    }
    // rotate when |x_p . x_q| > tol ||x_p|| ||x_q||
    const Ta tol = (Ta)((double)l * Eps<Ta>::v);
    int sweep = 0;
    bool converged = false;
    __syncthreads();
    for (; sweep < max_sweeps; sweep++) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < L - 1; r++) {
            for (int pr0 = 0; pr0 < L / 2; pr0 += ngrp) {
                const int pr = pr0 + grp;
                const bool act = pr < L / 2;
                int p = 0, q = 1;
                if (act) {
                    const int a = rr_pos(pr, r, L), b = rr_pos(L - 1 - pr, r, L);
                    p = min(a, b);
                    q = max(a, b);
                }
                const bool live = act && q < l;
                Ta al = 0, be = 0, ga = 0;
                if (live)
                    for (int i = gl; i < l; i += gsize) {
                        const Ta xp = X[p * L + i], xq = X[q * L + i];
                        al += xp * xp;
                        be += xq * xq;
                        ga += xp * xq;
                    }
                // three interleaved reductions inside the group
                for (int o = gsize >> 1; o > 0; o >>= 1) {
                    const Ta a1 = __shfl_xor_sync(gmask, al, o);
                    const Ta b1 = __shfl_xor_sync(gmask, be, o);
                    const Ta g1 = __shfl_xor_sync(gmask, ga, o);
                    al += a1;
                    be += b1;
                    ga += g1;
                }
                if (live && ga != Ta(0) && fabs(ga) > tol * sqrt(al * be)) {
                    const Ta zeta = (be - al) / (Ta(2) * ga);
                    const Ta t = (zeta >= Ta(0) ? Ta(1) : Ta(-1)) / (fabs(zeta) + sqrt(Ta(1) + zeta * zeta));
                    const Ta c = Ta(1) / sqrt(Ta(1) + t * t), s = c * t;
                    for (int i = gl; i < L; i += gsize) {
                        const Ta xp = X[p * L + i], xq = X[q * L + i];
                        X[p * L + i] = c * xp - s * xq;
                        X[q * L + i] = s * xp + c * xq;
                        const Ta vp = V[p * L + i], vq = V[q * L + i];
                        V[p * L + i] = c * vp - s * vq;
                        V[q * L + i] = s * vp + c * vq;
                    }
                    if (gl == 0) rotated = 1;
                }
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) { converged = true; break; }
    }
    if (!converged && tid == 0) atomicOr(status, (int)ST_NOCONV);
    for (int p = warp; p < l; p += nw) {
        Ta s = 0;
        for (int i = lane; i < l; i += 32) s += X[p * L + i] * X[p * L + i];
        s = warp_sum(s);
        if (lane == 0) nrm[p] = sqrt((double)s);
    }
    __syncthreads();
    if (tid == 0) {  // descending order, stable in the column index
        for (int i = 0; i < l; i++) perm[i] = i;
        for (int i = 0; i < l; i++) {
            int best = i;
            for (int j = i + 1; j < l; j++)
                if (nrm[perm[j]] > nrm[perm[best]]) best = j;
            const int t = perm[i]; perm[i] = perm[best]; perm[best] = t;
        }
    }
    __syncthreads();
    for (int o = tid; o < l; o += nt) sig[o] = nrm[perm[o]];
    for (int idx = tid; idx < lp * lp; idx += nt) {
        const int i = idx / lp, o = idx % lp;
        To u = To(0), w = To(0);
        if (i < l && o < l) {
            const int p = perm[o];
            const double sp = nrm[p];
            u = sp > 0.0 ? (To)((double)X[p * L + i] / sp) : To(0);
            w = (To)V[p * L + i];
        }
        UR[idx] = u;
        W[idx] = w;
    }
}

// ------------------------------------------------------------ two-sided Jacobi
__global__ void __launch_bounds__(1024) jacobi_eig_kernel(const double *__restrict__ G, int n,
                                                          double *__restrict__ lam, double *__restrict__ Vout,
                                                          int *__restrict__ status, int max_sweeps) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = n + (n & 1);
    double *M = reinterpret_cast<double *>(smraw);  // n x n, row-major
    double *Vt = M + n * n;                         // Vt[p * n + i] = V[i][p]
    double *cs = Vt + n * n;                        // per pair: c, s
    int *pq = reinterpret_cast<int *>(cs + L);      // per pair: p, q (or -1)
    int *perm = pq + L;
    __shared__ int rotated;
    const int tid = threadIdx.x, nt = blockDim.x, np = L / 2;
    for (int idx = tid; idx < n * n; idx += nt) {
        M[idx] = G[idx];
        Vt[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
    }
    const double rel = 1e-15;
    bool converged = false;
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < L - 1; r++) {
            for (int pr = tid; pr < np; pr += nt) {
                const int a = rr_pos(pr, r, L), b = rr_pos(L - 1 - pr, r, L);
                int p = min(a, b), q = max(a, b);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = M[p * n + q], app = M[p * n + p], aqq = M[q * n + q];
                    if (apq != 0.0 && fabs(apq) > rel * sqrt(fabs(app * aqq))) {
                        const double theta = (aqq - app) / (2.0 * apq);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                        c = 1.0 / sqrt(1.0 + t * t);
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
                const double c = cs[2 * pr], s = cs[2 * pr + 1];
                const double x = M[i * n + p], y = M[i * n + q];
                M[i * n + p] = c * x - s * y;
                M[i * n + q] = s * x + c * y;
                const double vx = Vt[p * n + i], vy = Vt[q * n + i];
                Vt[p * n + i] = c * vx - s * vy;
                Vt[q * n + i] = s * vx + c * vy;
            }
            __syncthreads();
            // M <- J^T M (rows p, q)
            for (int idx = tid; idx < np * n; idx += nt) {
                const int pr = idx / n, j = idx % n, p = pq[2 * pr];
                if (p < 0) continue;
                const int q = pq[2 * pr + 1];
                const double c = cs[2 * pr], s = cs[2 * pr + 1];
                const double x = M[p * n + j], y = M[q * n + j];
                M[p * n + j] = c * x - s * y;
                M[q * n + j] = s * x + c * y;
            }
            __syncthreads();
            for (int pr = tid; pr < np; pr += nt) {
                const int p = pq[2 * pr];
                if (p < 0) continue;
                const int q = pq[2 * pr + 1];
                M[p * n + q] = 0.0;
                M[q * n + p] = 0.0;
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
    for (int o = tid; o < n; o += nt) lam[o] = M[perm[o] * n + perm[o]];
    for (int idx = tid; idx < n * n; idx += nt) {
        const int i = idx / n, o = idx % n;
        Vout[idx] = Vt[perm[o] * n + i];
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

}  // namespace

template <typename TG, typename Tk, typename Tc>
cudaError_t chol_inv(const TG *G, int64_t ldg, int l, int64_t rows, double u, double *R, double *Rinv, Tc *Rinv_c,
                     int lp, int *status, cudaStream_t s) {
    const size_t smem = sizeof(Tk) * 2 * (size_t)l * l;
    cudaFuncSetAttribute(chol_inv_kernel<TG, Tk, Tc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const double coef = 11.0 * ((double)rows * l + (double)l * (l + 1)) * u;
    chol_inv_kernel<TG, Tk, Tc><<<1, 256, smem, s>>>(G, ldg, l, coef, R, Rinv, Rinv_c, lp, status);
    note_launch();
    return cudaGetLastError();
}

cudaError_t trmm_upper(const double *R2, const double *R1, double *R, int l, cudaStream_t s) {
    trmm_upper_kernel<<<(l * l + 255) / 256, 256, 0, s>>>(R2, R1, R, l);
    note_launch();
    return cudaGetLastError();
}

template <typename Ta, typename To>
cudaError_t jacobi_osvd(const double *R, int l, int lp, double *sig, To *UR, To *W, int *status, cudaStream_t s) {
    const int L = l + (l & 1);
    const size_t smem = sizeof(Ta) * (2 * (size_t)L * L + 1) + sizeof(double) * L + sizeof(int) * L + 16;
    cudaFuncSetAttribute(jacobi_osvd_kernel<Ta, To>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int gsize = l <= 64 ? 16 : 32;
    int threads = (L / 2) * gsize;
    threads = threads < 64 ? 64 : threads > 1024 ? 1024 : (threads + 31) / 32 * 32;
    jacobi_osvd_kernel<Ta, To><<<1, threads, smem, s>>>(R, l, lp, sig, UR, W, status, 40, gsize);
    note_launch();
    return cudaGetLastError();
}

cudaError_t jacobi_eig(const double *G, int n, double *lam, double *V, int *status, cudaStream_t s) {
    const int L = n + (n & 1);
    const size_t smem = sizeof(double) * (2 * (size_t)n * n + L) + sizeof(int) * (2 * L) + 16;
    cudaFuncSetAttribute(jacobi_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    jacobi_eig_kernel<<<1, 1024, smem, s>>>(G, n, lam, V, status, 50);
    note_launch();
    return cudaGetLastError();
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
                                              int, int *, cudaStream_t);
INST_CHOL(float, float, float)
INST_CHOL(double, double, double)
template cudaError_t jacobi_osvd<float, float>(const double *, int, int, double *, float *, float *, int *,
                                               cudaStream_t);
template cudaError_t jacobi_osvd<double, float>(const double *, int, int, double *, float *, float *, int *,
                                                cudaStream_t);
template cudaError_t jacobi_osvd<double, double>(const double *, int, int, double *, double *, double *, int *,
                                                 cudaStream_t);
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
