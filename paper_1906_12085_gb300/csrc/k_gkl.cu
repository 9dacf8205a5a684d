// Golub-Kahan-Lanczos bidiagonalisation with full reorthogonalisation: the
// HBM-bound kernels of svd_truncated_krylov.
//
// One step j (alpha, beta and every reorthogonalisation coefficient stay in
// device memory; the host only launches):
//   w  = A v_j - beta_{j-1} u_{j-1}          gemv_n     (one read of A)
//   w -= U (U^T w), twice (CGS2)             multi_dot + multi_axpy (reads of U)
//   alpha_j = ||w||, u_j = w / alpha_j       multi_axpy (norm fused) + scale_store
//   z  = A^T u_j - alpha_j v_j               gemv_t + colsum_sub (one read of A)
//   z -= V (V^T z), twice; beta_j = ||z||; v_{j+1} = z / beta_j
// The one-pass form (float32) reads A once per step: gemv_nt forms g = A v_j and
// x = A^T g from the same rows, and A^T u_j is recovered by linearity,
//   y_j = A^T u_j = (x - beta_{j-1} y_{j-1} - sum_i c_i y_i) / alpha_j,
// from the stored y_i = A^T u_i and the summed CGS2 coefficients c_i; the recovery
// multiplies the rounding of x by ||x|| / alpha_j, so a step whose
// ||x|| / (alpha_j max_i alpha_i) exceeds kRecoverBound runs gemv_t after all (gated on a
// device flag).
// The Krylov bases are stored transposed (U^T: steps x m, V^T: (steps+1) x n)
// so every basis vector is contiguous.
#include "common.cuh"

namespace gbr {
namespace {

constexpr int GT = 256;

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; static constexpr int n = 4; };
template <> struct V4<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ T warp_red(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// y[r] = A[r] . v - (beta ? beta[0] : 0) * uprev[r]; one warp per row, v staged in shared memory.
// With mu, the centred product (A - 1 mu^T) v = A v - (mu . v) is formed (each block
// recomputes mu . v from shared memory).
template <typename T, bool VEC>
__global__ void __launch_bounds__(GT) gemv_n_kernel(const T *__restrict__ A, int64_t m, int n, int64_t lda,
                                                    const T *__restrict__ v, const T *__restrict__ beta,
                                                    const T *__restrict__ uprev, T *__restrict__ y,
                                                    const T *__restrict__ mu) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *vs = reinterpret_cast<T *>(sm_raw);
    __shared__ double mred[GT / 32];
    double mv = 0.0;
    for (int c = threadIdx.x; c < n; c += GT) {
        vs[c] = v[c];
        if (mu) mv += (double)mu[c] * (double)v[c];
    }
    mv = warp_red(mv);
    if ((threadIdx.x & 31) == 0) mred[threadIdx.x >> 5] = mv;
    __syncthreads();
    double mvt = 0.0;
    for (int k = 0; k < GT / 32; k++) mvt += mred[k];
    const T mdot = (T)mvt;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (GT / 32);
    const T b = beta ? beta[0] : T(0);
    for (int64_t r = (int64_t)blockIdx.x * (GT / 32) + (threadIdx.x >> 5); r < m; r += warps) {
        const T *row = A + r * lda;
        T acc = T(0);
        if constexpr (VEC) {
            using V = typename V4<T>::type;
            constexpr int E = V4<T>::n;
#pragma unroll 4
            for (int c = lane * E; c < n; c += 32 * E) {
                const V a = *reinterpret_cast<const V *>(row + c);
                const T *pa = reinterpret_cast<const T *>(&a);
#pragma unroll
                for (int e = 0; e < E; e++) acc += pa[e] * vs[c + e];
            }
        } else {
            for (int c = lane; c < n; c += 32) acc += row[c] * vs[c];
        }
        acc = warp_red(acc) - mdot;
        if (lane == 0) y[r] = uprev ? acc - b * uprev[r] : acc;
    }
}

// part[chunk][c] = sum over the chunk's rows of u[r] A[r][c]; block = (chunk, column block of GT*E columns).
// Products are summed in the element type over 32-row groups and the group sums
// in float64, so the 1M-row sums keep float64-level accumulation error at the
// cost of one float64 add per 32 rows.
template <typename T, bool VEC>
__global__ void __launch_bounds__(GT) gemv_t_kernel(const T *__restrict__ A, int64_t m, int n, int64_t lda,
                                                    const T *__restrict__ u, int64_t rpc, double *__restrict__ part,
                                                    double *__restrict__ usum, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    constexpr int E = VEC ? V4<T>::n : 1;
    const int64_t r0 = (int64_t)blockIdx.x * rpc;
    const int64_t r1 = min(m, r0 + rpc);
    const int c0 = (blockIdx.y * GT + threadIdx.x) * E;
    if (usum && blockIdx.y == 0) {  // sum of u over the chunk (for the mean correction), whole block
        __shared__ double ured[GT / 32];
        double su = 0.0;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += GT) su += (double)u[r];
        su = warp_red(su);
        if ((threadIdx.x & 31) == 0) ured[threadIdx.x >> 5] = su;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < GT / 32; k++) t += ured[k];
            usum[blockIdx.x] = t;
        }
    }
    if (c0 >= n) return;
    double acc[E];
#pragma unroll
    for (int e = 0; e < E; e++) acc[e] = 0.0;
    for (int64_t g = r0; g < r1; g += 32) {
        const int64_t ge = min(r1, g + 32);
        T sub[E];
#pragma unroll
        for (int e = 0; e < E; e++) sub[e] = T(0);
#pragma unroll 8
        for (int64_t r = g; r < ge; r++) {
            const T ur = u[r];
            if constexpr (VEC) {
                using V = typename V4<T>::type;
                const V a = *reinterpret_cast<const V *>(A + r * lda + c0);
                const T *pa = reinterpret_cast<const T *>(&a);
#pragma unroll
                for (int e = 0; e < E; e++) sub[e] += ur * pa[e];
            } else {
                sub[0] += ur * A[r * lda + c0];
            }
        }
#pragma unroll
        for (int e = 0; e < E; e++) acc[e] += (double)sub[e];
    }
#pragma unroll
    for (int e = 0; e < E; e++)
        if (c0 + e < n) part[(int64_t)blockIdx.x * n + c0 + e] = acc[e];
}

// z[c] = sum_k part[k][c] - (alpha ? alpha[0] : 0) * vprev[c]; 8 row groups x 32 columns per block, fixed order
// (y, when given, receives the sum itself; gate, when given, must be set for the kernel to run)
template <typename T>
__global__ void colsum_sub_kernel(const double *__restrict__ part, int64_t chunks, int n, const T *__restrict__ alpha,
                                  const T *__restrict__ vprev, T *__restrict__ z, const T *__restrict__ mu,
                                  const double *__restrict__ usum, T *__restrict__ y, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ double red[8][33];
    __shared__ double usr[8];
    const int cx = threadIdx.x & 31, gy = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cx;
    double s = 0.0;
    if (c < n)
        for (int64_t k = gy; k < chunks; k += 8) s += part[k * n + c];
    red[gy][cx] = s;
    if (mu && cx == 0) {
        double su = 0.0;
        for (int64_t k = gy; k < chunks; k += 8) su += usum[k];
        usr[gy] = su;
    }
    __syncthreads();
    if (gy == 0 && c < n) {
        double t = red[0][cx];
        for (int g = 1; g < 8; g++) t += red[g][cx];
        if (mu) {
            double su = usr[0];
            for (int g = 1; g < 8; g++) su += usr[g];
            t -= (double)mu[c] * su;
        }
        z[c] = alpha ? (T)(t - (double)alpha[0] * (double)vprev[c]) : (T)t;
        if (y) y[c] = (T)t;
    }
}

// ---------------------------------------------------------------- one pass over A
// A CTA takes a chunk of rows R at a time: every thread loads NV float4 of each row (its
// columns c = 4 (tid + GT k)), forms its share of the R row dots with v, one CTA-wide
// reduction gives g_r = (a_r - mu) . v, w_r = g_r - beta uprev_r is stored, and the same
// registers accumulate a_rc g_r into the column partials (float32 over 32 rows, float64
// beyond), with sum_r g_r kept for the mean correction of x = (A - 1 mu^T)^T g.
template <int NV, int R>
__global__ void __launch_bounds__(GT) gemv_nt_kernel(const float *__restrict__ A, int64_t m, int n, int64_t lda,
                                                     const float *__restrict__ v, const float *__restrict__ beta,
                                                     const float *__restrict__ uprev, float *__restrict__ w,
                                                     const float *__restrict__ mu, int64_t rpc,
                                                     double *__restrict__ part, double *__restrict__ gsum) {
    __shared__ float red[GT / 32][R];
    __shared__ float gr[R];
    __shared__ double mred[GT / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float4 vr[NV];
    bool on[NV];
    double mv = 0.0;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        const int c = 4 * (tid + GT * k);
        on[k] = c < n;
        vr[k] = on[k] ? *reinterpret_cast<const float4 *>(v + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (mu && on[k]) {
            const float4 mk = *reinterpret_cast<const float4 *>(mu + c);
            mv += (double)mk.x * vr[k].x + (double)mk.y * vr[k].y + (double)mk.z * vr[k].z + (double)mk.w * vr[k].w;
        }
    }
    mv = warp_red(mv);
    if (lane == 0) mred[wid] = mv;
    __syncthreads();
    double mvt = 0.0;
#pragma unroll
    for (int k = 0; k < GT / 32; k++) mvt += mred[k];
    const float mdot = (float)mvt;
    const float b = beta ? beta[0] : 0.f;
    const int64_t r0 = (int64_t)blockIdx.x * rpc, r1 = min(m, r0 + rpc);
    float4 sub[NV];
    double acc[NV][4];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        sub[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.0;
    }
    double gs = 0.0;
    int since = 0;
    for (int64_t rb = r0; rb < r1; rb += R) {
        float4 a[R][NV];
        float d[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const bool rin = rb + r < r1;
            d[r] = 0.f;
#pragma unroll
            for (int k = 0; k < NV; k++) {
                a[r][k] = (rin && on[k]) ? *reinterpret_cast<const float4 *>(A + (rb + r) * lda + 4 * (tid + GT * k))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                d[r] += a[r][k].x * vr[k].x + a[r][k].y * vr[k].y + a[r][k].z * vr[k].z + a[r][k].w * vr[k].w;
            }
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            const float t = warp_red(d[r]);
            if (lane == 0) red[wid][r] = t;
        }
        __syncthreads();
        if (tid < R) {
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < GT / 32; k++) t += red[k][tid];
            t -= mdot;
            gr[tid] = t;
            if (rb + tid < r1) {
                w[rb + tid] = uprev ? t - b * uprev[rb + tid] : t;
                gs += (double)t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; r++) {
            const float g = rb + r < r1 ? gr[r] : 0.f;
#pragma unroll
            for (int k = 0; k < NV; k++) {
                sub[k].x += a[r][k].x * g;
                sub[k].y += a[r][k].y * g;
                sub[k].z += a[r][k].z * g;
                sub[k].w += a[r][k].w * g;
            }
        }
        since += R;
        if (since >= 32) {
#pragma unroll
            for (int k = 0; k < NV; k++) {
                acc[k][0] += sub[k].x;
                acc[k][1] += sub[k].y;
                acc[k][2] += sub[k].z;
                acc[k][3] += sub[k].w;
                sub[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            since = 0;
        }
    }
#pragma unroll
    for (int k = 0; k < NV; k++) {
        acc[k][0] += sub[k].x;
        acc[k][1] += sub[k].y;
        acc[k][2] += sub[k].z;
        acc[k][3] += sub[k].w;
        if (on[k]) {
            double *pp = part + (int64_t)blockIdx.x * n + 4 * (tid + GT * k);
            pp[0] = acc[k][0];
            pp[1] = acc[k][1];
            pp[2] = acc[k][2];
            pp[3] = acc[k][3];
        }
    }
    // sum of g over the chunk (threads 0 .. R-1 hold their rows' shares)
    gs = warp_red(gs);
    if (tid == 0) gsum[blockIdx.x] = gs;
}

// The recovery of y_j = A^T u_j (one CTA): ||x||, y_j = (x - beta y_{j-1} - sum_{i<j} c_i y_i) / alpha_j
// (Y: rows of the stored y_i, ld n), z = y_j - alpha_j v_j; flag = 1 when
// ||x|| / (alpha_j max_{i<=j} alpha_i) > kRecoverBound (or alpha_j is not positive): the
// caller's gated gemv_t then recomputes z and y_j from A.
constexpr double kRecoverBound = 16.0;
__global__ void __launch_bounds__(1024) recover_kernel(const float *__restrict__ x, float *__restrict__ Y, int j, int n,
                                                       const float *__restrict__ beta, const float *__restrict__ coef,
                                                       const float *__restrict__ alpha, const float *__restrict__ vj,
                                                       float *__restrict__ z, int *__restrict__ flag) {
    __shared__ double red[32];
    __shared__ float cs[1024];
    const float aj = alpha[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) cs[i] = coef[i];
    double x2 = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) x2 += (double)x[c] * x[c];
    x2 = warp_red(x2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
        float amax = 0.f;
        for (int i = 0; i <= j; i++) amax = fmaxf(amax, alpha[i]);
        const bool bad = !(aj > 0.f) || sqrt(t) > kRecoverBound * (double)aj * (double)amax;
        *flag = bad ? 1 : 0;
    }
    const float b = j > 0 ? beta[j - 1] : 0.f;
    const float inv = aj > 0.f ? 1.f / aj : 0.f;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        float t = x[c];
        if (j > 0) t -= b * Y[(int64_t)(j - 1) * n + c];
        for (int i = 0; i < j; i++) t -= cs[i] * Y[(int64_t)i * n + c];
        const float y = t * inv;
        Y[(int64_t)j * n + c] = y;
        z[c] = y - aj * vj[c];
    }
}

// part[b][i] = sum over rows of block b of Bt[i][r] w[r], i < cnt (Bt cnt x len, ld).
// Four basis vectors per sweep (independent accumulators); warp sums land in
// shared memory and are combined once at the end, in warp order.
// part[b][i] = sum over block b's rows r of Bt[i][r] w[r].  VEC: warp k takes the
// vectors i = k, k + 8, ... (two at a time), each lane a strided run of E-wide loads
// over the block's rows, with w staged in shared memory; one warp reduction per
// vector.  Scalar form for lengths or strides that are not multiples of E.
template <typename T, bool VEC>
__global__ void __launch_bounds__(GT) multi_dot_kernel(const T *__restrict__ Bt, int64_t ld, int cnt,
                                                       const T *__restrict__ w, int64_t len, int64_t rpb,
                                                       T *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *ws = reinterpret_cast<T *>(sm_raw);  // rpb entries of w
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int nr = (int)(min(len, r0 + rpb) - r0);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int r = threadIdx.x; r < nr; r += GT) ws[r] = w[r0 + r];
    __syncthreads();
    if constexpr (VEC) {
        using V = typename V4<T>::type;
        constexpr int E = V4<T>::n;
        for (int i = wid; i < cnt; i += 2 * (GT / 32)) {
            const int i2 = i + GT / 32;
            const bool two = i2 < cnt;
            const T *b1 = Bt + (int64_t)i * ld + r0;
            const T *b2 = Bt + (int64_t)(two ? i2 : i) * ld + r0;
            T a1 = T(0), a2 = T(0);
#pragma unroll 8
            for (int r = lane * E; r < nr; r += 32 * E) {
                const V x = *reinterpret_cast<const V *>(ws + r);
                const V u1 = *reinterpret_cast<const V *>(b1 + r);
                const V u2 = *reinterpret_cast<const V *>(b2 + r);
                const T *px = reinterpret_cast<const T *>(&x);
                const T *p1 = reinterpret_cast<const T *>(&u1);
                const T *p2 = reinterpret_cast<const T *>(&u2);
#pragma unroll
                for (int e = 0; e < E; e++) {
                    a1 += p1[e] * px[e];
                    a2 += p2[e] * px[e];
                }
            }
            a1 = warp_red(a1);
            a2 = warp_red(a2);
            if (lane == 0) {
                part[(int64_t)blockIdx.x * cnt + i] = a1;
                if (two) part[(int64_t)blockIdx.x * cnt + i2] = a2;
            }
        }
    } else {
        for (int i = wid; i < cnt; i += GT / 32) {
            const T *b1 = Bt + (int64_t)i * ld + r0;
            T a1 = T(0);
            for (int r = lane; r < nr; r += 32) a1 += b1[r] * ws[r];
            a1 = warp_red(a1);
            if (lane == 0) part[(int64_t)blockIdx.x * cnt + i] = a1;
        }
    }
}

// coef[i] = sum_b part[b][i] (fixed order), one warp per i
template <typename T>
__global__ void sum_parts_kernel(const T *__restrict__ part, int64_t nblk, int cnt, T *__restrict__ coef) {
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= cnt) return;
    T s = T(0);
    for (int64_t b = lane; b < nblk; b += 32) s += part[b * cnt + i];
    s = warp_red(s);
    if (lane == 0) coef[i] = s;
}

// w[r] -= sum_i coef[i] Bt[i][r]; sq[b] = sum over the block's rows of w[r]^2 (after the update).
// VEC: a thread owns E consecutive rows, so the loop over i runs E independent chains
// with its loads issued ahead.
template <typename T, bool VEC>
__global__ void __launch_bounds__(GT) multi_axpy_kernel(const T *__restrict__ Bt, int64_t ld, int cnt,
                                                        const T *__restrict__ coef, T *__restrict__ w, int64_t len,
                                                        int64_t rpb, T *__restrict__ sq) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *cs = reinterpret_cast<T *>(sm_raw);
    __shared__ T red[GT / 32];
    for (int i = threadIdx.x; i < cnt; i += GT) cs[i] = coef[i];
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = min(len, r0 + rpb);
    T s2 = T(0);
    if constexpr (VEC) {
        using V = typename V4<T>::type;
        constexpr int E = V4<T>::n;
        for (int64_t r = r0 + (int64_t)threadIdx.x * E; r < r1; r += (int64_t)GT * E) {
            V xv = *reinterpret_cast<const V *>(w + r);
            T *x = reinterpret_cast<T *>(&xv);
#pragma unroll 8
            for (int i = 0; i < cnt; i++) {
                const V bv = *reinterpret_cast<const V *>(Bt + (int64_t)i * ld + r);
                const T *pb = reinterpret_cast<const T *>(&bv);
                const T c = cs[i];
#pragma unroll
                for (int e = 0; e < E; e++) x[e] -= c * pb[e];
            }
            *reinterpret_cast<V *>(w + r) = xv;
#pragma unroll
            for (int e = 0; e < E; e++) s2 += x[e] * x[e];
        }
    } else {
        for (int64_t r = r0 + threadIdx.x; r < r1; r += GT) {
            T x = w[r];
            for (int i = 0; i < cnt; i++) x -= cs[i] * Bt[(int64_t)i * ld + r];
            w[r] = x;
            s2 += x * x;
        }
    }
    s2 = warp_red(s2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = red[0];
        for (int k = 1; k < GT / 32; k++) t += red[k];
        sq[blockIdx.x] = t;
    }
}

// nrm[0] = sqrt(sum_b sq[b]) (fixed order); out[r] = w[r] / nrm[0] in a second kernel
template <typename T>
__global__ void norm_kernel(const T *__restrict__ sq, int64_t nblk, T *__restrict__ nrm) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) s += (double)sq[b];
    s = warp_red(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
        nrm[0] = (T)sqrt(t);
    }
}

template <typename T>
__global__ void scale_store_kernel(const T *__restrict__ w, int64_t len, const T *__restrict__ nrm,
                                   T *__restrict__ out, int *__restrict__ status) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const T d = nrm[0];
    if (r == 0 && !(d > T(0))) atomicOr(status, (int)ST_RANKDEF);
    if (r < len) out[r] = d > T(0) ? w[r] / d : T(0);
}

// dense s x s upper bidiagonal (float64): diag alpha, superdiag beta[0..s-2]
template <typename T>
__global__ void bidiag_kernel(const T *__restrict__ alpha, const T *__restrict__ beta, int s, double *__restrict__ B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= s * s) return;
    const int i = idx / s, j = idx % s;
    B[idx] = j == i ? (double)alpha[i] : (j == i + 1 ? (double)beta[i] : 0.0);
}

}  // namespace

// Rows per chunk of A^T u: small enough that the (chunk, column block) grid fills
// about two waves of 8 blocks on every SM, at least 256 rows so each thread keeps
// a long run of independent loads.  Partials cost 8 (n + 1) bytes per chunk.
static int64_t gemv_t_rpc(int64_t m, int n) {
    if (m < 4096) return 64;
    const int64_t colblocks = ceil_div(n, GT * 4);
    const int64_t want = ceil_div(2 * 8 * 152, colblocks);
    const int64_t rpc = round_up(ceil_div(m, want), 32);
    return rpc < 256 ? 256 : rpc;
}

int64_t gkl_gemv_chunks(int64_t m, int n) { return ceil_div(m, gemv_t_rpc(m, n)); }

template <typename T>
cudaError_t gkl_gemv_n(const T *A, int64_t m, int n, int64_t lda, const T *v, const T *beta, const T *uprev, T *y,
                       cudaStream_t s, const T *mu) {
    constexpr int E = V4<T>::n;
    const bool vec = (n % E == 0) && (lda % E == 0) && ((uintptr_t)A % 16 == 0);
    int64_t blocks = ceil_div(m, GT / 32);
    if (blocks > 152 * 8) blocks = 152 * 8;
    const size_t smem = sizeof(T) * (size_t)n;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(gemv_n_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(gemv_n_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (vec) gemv_n_kernel<T, true><<<(unsigned)blocks, GT, smem, s>>>(A, m, n, lda, v, beta, uprev, y, mu);
    else gemv_n_kernel<T, false><<<(unsigned)blocks, GT, smem, s>>>(A, m, n, lda, v, beta, uprev, y, mu);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t gkl_gemv_t(const T *A, int64_t m, int n, int64_t lda, const T *u, const T *alpha, const T *vprev, T *z,
                       double *part, cudaStream_t s, const T *mu, T *y, const int *gate) {
    constexpr int E = V4<T>::n;
    const bool vec = (n % E == 0) && (lda % E == 0) && ((uintptr_t)A % 16 == 0);
    const int64_t rpc = gemv_t_rpc(m, n);
    const int64_t chunks = ceil_div(m, rpc);
    const int cols_per_block = GT * (vec ? E : 1);
    dim3 grid((unsigned)chunks, (unsigned)ceil_div(n, cols_per_block));
    double *usum = mu ? part + chunks * n : nullptr;  // chunks extra entries after the column partials
    if (vec) gemv_t_kernel<T, true><<<grid, GT, 0, s>>>(A, m, n, lda, u, rpc, part, usum, gate);
    else gemv_t_kernel<T, false><<<grid, GT, 0, s>>>(A, m, n, lda, u, rpc, part, usum, gate);
    colsum_sub_kernel<T><<<(unsigned)ceil_div(n, 32), 256, 0, s>>>(part, chunks, n, alpha, vprev, z, mu, usum, y,
                                                                  gate);
    note_launch(2);
    return cudaGetLastError();
}

// Rows per chunk of the one-pass product: two CTAs per SM, whole groups of 32 rows.
static int64_t gemv_nt_rpc(int64_t m) { return round_up(ceil_div(m, 2 * 152), 32); }
int64_t gkl_gemv_nt_chunks(int64_t m) { return ceil_div(m, gemv_nt_rpc(m)); }

bool gkl_one_pass_ok(int64_t m, int n, int64_t lda, const void *A) {
    return n % 4 == 0 && lda % 4 == 0 && n <= 4 * GT * 4 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 && m >= 1;
}

cudaError_t gkl_gemv_nt(const float *A, int64_t m, int n, int64_t lda, const float *v, const float *beta,
                        const float *uprev, float *w, float *x, double *part, cudaStream_t s, const float *mu) {
    if (!gkl_one_pass_ok(m, n, lda, A) || (reinterpret_cast<uintptr_t>(v) & 15) ||
        (mu && (reinterpret_cast<uintptr_t>(mu) & 15)))
        return cudaErrorInvalidValue;
    const int64_t rpc = gemv_nt_rpc(m);
    const int64_t chunks = ceil_div(m, rpc);
    double *gsum = part + chunks * n;
    const int nv = (n + 4 * GT - 1) / (4 * GT);
    const dim3 grid((unsigned)chunks);
    switch (nv) {
        case 1: gemv_nt_kernel<1, 8><<<grid, GT, 0, s>>>(A, m, n, lda, v, beta, uprev, w, mu, rpc, part, gsum); break;
        case 2: gemv_nt_kernel<2, 8><<<grid, GT, 0, s>>>(A, m, n, lda, v, beta, uprev, w, mu, rpc, part, gsum); break;
        case 3: gemv_nt_kernel<3, 4><<<grid, GT, 0, s>>>(A, m, n, lda, v, beta, uprev, w, mu, rpc, part, gsum); break;
        default: gemv_nt_kernel<4, 4><<<grid, GT, 0, s>>>(A, m, n, lda, v, beta, uprev, w, mu, rpc, part, gsum); break;
    }
    colsum_sub_kernel<float><<<(unsigned)ceil_div(n, 32), 256, 0, s>>>(part, chunks, n, nullptr, nullptr, x, mu, gsum,
                                                                       nullptr, nullptr);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t gkl_recover(const float *x, float *Y, int j, int n, const float *beta, const float *coef,
                        const float *alpha, const float *vj, float *z, int *flag, cudaStream_t s) {
    if (j > 1024) return cudaErrorInvalidValue;
    recover_kernel<<<1, 1024, 0, s>>>(x, Y, j, n, beta, coef, alpha, vj, z, flag);
    note_launch();
    return cudaGetLastError();
}

// Rows per block of the Gram-Schmidt kernels: 2048, or fewer for short vectors (the n-long
// V side), so that a pass over a basis spreads over about two blocks per SM; a multiple of
// 128 (32 E-wide loads per warp row for float32 and float64).
constexpr int64_t kReorthRows = 2048;
int64_t gkl_reorth_rows(int64_t len) {
    const int64_t r = round_up(ceil_div(len, 2 * 152), 128);
    return r < 128 ? 128 : (r > kReorthRows ? kReorthRows : r);
}
int64_t gkl_reorth_blocks(int64_t len) { return ceil_div(len, gkl_reorth_rows(len)); }

// w <- w - B (B^T w) twice (classical Gram-Schmidt, twice) against the first cnt rows of
// Bt (cnt x len, ld); then nrm[0] = ||w|| and out = w / nrm[0].  coef: cnt scratch,
// part: blocks * max(cnt, 1) scratch, sq: blocks scratch (blocks = gkl_reorth_blocks(len)).
// (elementwise sum of two coefficient vectors: the total CGS2 coefficient of each basis vector)
template <typename T>
__global__ void coef_add_kernel(const T *__restrict__ c, int cnt, T *__restrict__ tot, bool first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) tot[i] = first ? c[i] : tot[i] + c[i];
}

template <typename T>
cudaError_t gkl_reorth_normalize(const T *Bt, int64_t ld, int cnt, T *w, int64_t len, T *coef, T *part, T *sq,
                                 T *nrm, T *out, int *status, cudaStream_t s, T *ctot) {
    constexpr int E = V4<T>::n;
    const int64_t rpb = gkl_reorth_rows(len);  // a multiple of 32 E
    const int64_t nblk = ceil_div(len, rpb);
    // E-wide loads need every vector (and w) to start on a 16-byte boundary and whole E-groups
    const bool vec = ld % E == 0 && len % E == 0 && (reinterpret_cast<uintptr_t>(Bt) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(w) & 15) == 0;
    const size_t smem_c = sizeof(T) * (size_t)(cnt > 0 ? cnt : 1);
    const size_t smem_d = sizeof(T) * (size_t)rpb;
    for (int pass = 0; pass < 2 && cnt > 0; pass++) {
        if (vec) multi_dot_kernel<T, true><<<(unsigned)nblk, GT, smem_d, s>>>(Bt, ld, cnt, w, len, rpb, part);
        else multi_dot_kernel<T, false><<<(unsigned)nblk, GT, smem_d, s>>>(Bt, ld, cnt, w, len, rpb, part);
        sum_parts_kernel<T><<<(unsigned)ceil_div(cnt, 8), 256, 0, s>>>(part, nblk, cnt, coef);
        if (ctot) {
            coef_add_kernel<T><<<(unsigned)ceil_div(cnt, 256), 256, 0, s>>>(coef, cnt, ctot, pass == 0);
            note_launch();
        }
        if (vec) multi_axpy_kernel<T, true><<<(unsigned)nblk, GT, smem_c, s>>>(Bt, ld, cnt, coef, w, len, rpb, sq);
        else multi_axpy_kernel<T, false><<<(unsigned)nblk, GT, smem_c, s>>>(Bt, ld, cnt, coef, w, len, rpb, sq);
        note_launch(3);
    }
    if (cnt == 0) {  // norm only
        if (vec) multi_axpy_kernel<T, true><<<(unsigned)nblk, GT, smem_c, s>>>(Bt, ld, 0, coef, w, len, rpb, sq);
        else multi_axpy_kernel<T, false><<<(unsigned)nblk, GT, smem_c, s>>>(Bt, ld, 0, coef, w, len, rpb, sq);
        note_launch();
    }
    norm_kernel<T><<<1, 1024, 0, s>>>(sq, nblk, nrm);
    scale_store_kernel<T><<<(unsigned)ceil_div(len, 256), 256, 0, s>>>(w, len, nrm, out, status);
    note_launch(2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gkl_bidiag(const T *alpha, const T *beta, int steps, double *B, cudaStream_t s) {
    bidiag_kernel<T><<<(unsigned)ceil_div((int64_t)steps * steps, 256), 256, 0, s>>>(alpha, beta, steps, B);
    note_launch();
    return cudaGetLastError();
}

#define INST_GKL(T)                                                                                                  \
    template cudaError_t gkl_gemv_n<T>(const T *, int64_t, int, int64_t, const T *, const T *, const T *, T *,        \
                                       cudaStream_t, const T *);                                                     \
    template cudaError_t gkl_gemv_t<T>(const T *, int64_t, int, int64_t, const T *, const T *, const T *, T *,       \
                                       double *, cudaStream_t, const T *, T *, const int *);                         \
    template cudaError_t gkl_reorth_normalize<T>(const T *, int64_t, int, T *, int64_t, T *, T *, T *, T *, T *,     \
                                                 int *, cudaStream_t, T *);                                          \
    template cudaError_t gkl_bidiag<T>(const T *, const T *, int, double *, cudaStream_t);
INST_GKL(float)
INST_GKL(double)

}  // namespace gbr
