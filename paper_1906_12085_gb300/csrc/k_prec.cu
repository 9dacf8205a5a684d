// Element-wise and reduction kernels of the bfloat16 precision form (the
// products themselves are in k_tc16.cu):
//   colstats16 : column means mu of the stored bfloat16 matrix and
//                ||A - 1 mu^T||_F^2 = sum_j (sum_i a_ij^2 - m mu_j^2), float64
//                accumulation in a fixed order;
//   to_bf16_t  : Zt (lp x n bfloat16) = round(Z)^T, rows l..lp-1 zero, and the
//                mean correction c = mu^T round(Z) of the sketch / power products;
//   split_bf16 : Q (m x lp float32) -> one bfloat16 term, or three whose sum
//                carries Q to float32 accuracy (hi = round(Q), mid = round(Q - hi),
//                lo = round(Q - hi - mid), each difference exact in float32), and
//                the column sums of the terms (compensated float32 per thread, then
//                float64) for the mean correction.
// and their e4m3 counterparts (the stored matrix is A_q diag(s)):
//   colstats8  : means and ||A - 1 mu^T||_F^2 of A_q diag(s);
//   prep8_small: Zq = e4m3(diag(s) Z diag(1/t)) transposed, t_j = amax_i |s_i Z_ij| / 448,
//                and c_j = t_j sum_i (mu_i / s_i) Zq_ij (the product uses exactly
//                Z_eff = diag(1/s) Zq diag(t), so c = mu^T Z_eff);
//   prep8_q    : Qq = e4m3(Q diag(1/u)), u_j = amax_r |Q_rj| / 448, and
//                qsum_j = u_j sum_r Qq_rj (code sums exact in integers);
//   e4m3_to_bf16: the codes as bfloat16 (exact: every e4m3 value is a bfloat16).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace gbr {
namespace {

__device__ __forceinline__ float bf(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ uint16_t rbf(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// partial column sums / sums of squares over row chunks: 32 columns x 8 row groups per block
__global__ void colstats16_kernel(const uint16_t *__restrict__ A, int64_t m, int64_t n, int64_t lda, int64_t rpb,
                                  double *__restrict__ psum, double *__restrict__ psq) {
    __shared__ double rs[8][33], rq[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * 32 + tx;
    const int64_t r0 = (int64_t)blockIdx.y * rpb, r1 = min(m, r0 + rpb);
    double s = 0.0, q = 0.0;
    if (c < n) {
        for (int64_t g = r0 + ty * 32; g < r1; g += 8 * 32) {  // 32-row groups in float32, then float64
            float fs = 0.f, fq = 0.f;
            const int64_t ge = min(r1, g + 32);
#pragma unroll 8
            for (int64_t r = g; r < ge; r++) {
                const float a = bf(A[r * lda + c]);
                fs += a;
                fq = fmaf(a, a, fq);
            }
            s += fs;
            q += fq;
        }
    }
    rs[ty][tx] = s;
    rq[ty][tx] = q;
    __syncthreads();
    if (ty == 0 && c < n) {
        for (int k = 1; k < 8; k++) {
            s += rs[k][tx];
            q += rq[k][tx];
        }
        psum[(int64_t)blockIdx.y * n + c] = s;
        psq[(int64_t)blockIdx.y * n + c] = q;
    }
}

// mu_j, float copy, and colv_j = sum_i a_ij^2 - m mu_j^2 (chunks summed in order)
__global__ void colstats16_finish(const double *__restrict__ psum, const double *__restrict__ psq, int nch,
                                  int64_t m, int64_t n, bool center, double *__restrict__ mu, float *__restrict__ mu_f,
                                  double *__restrict__ colv) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s = 0.0, q = 0.0;
    for (int k = 0; k < nch; k++) {
        s += psum[(int64_t)k * n + c];
        q += psq[(int64_t)k * n + c];
    }
    const double mj = center ? s / (double)m : 0.0;  // without centring: mu = 0, ||A||_F^2
    mu[c] = mj;
    mu_f[c] = (float)mj;
    colv[c] = q - (double)m * mj * mj;
}

// Zt[j][i] = round(Z[i][j]) for j < l, 0 for l <= j < lp (i < n; ldz >= n)
__global__ void to_bf16_t_kernel(const float *__restrict__ Z, int64_t n, int l, int64_t ldzin, int lp,
                                 uint16_t *__restrict__ Zt, int64_t ldz) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)lp * n) return;
    const int j = (int)(idx / n);
    const int64_t i = idx % n;
    Zt[(int64_t)j * ldz + i] = j < l ? rbf(Z[i * ldzin + j]) : (uint16_t)0;
}

// c[j] = sum_i mu_i Zt[j][i] (float64, fixed order), one warp per j
__global__ void mean_corr_kernel(const double *__restrict__ mu, const uint16_t *__restrict__ Zt, int64_t n,
                                 int64_t ldz, int lp, float *__restrict__ c) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= lp) return;
    double s = 0.0;
    for (int64_t i = lane; i < n; i += 32) s += mu[i] * (double)bf(Zt[(int64_t)j * ldz + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) c[j] = (float)s;
}

// The per-column passes over Q (rows x lp) run 256 threads per (row chunk, group of
// up to 128 columns: blockIdx.y) as G = 256 / CW row groups of CW = the group's
// width rounded up to 32 columns.  jj: column within the group, j: column of Q.
struct QLayout {
    int j, jj, ry, G, cw;
    bool ok;
};
__device__ __forceinline__ QLayout q_layout(int lp) {
    QLayout q;
    const int j0 = blockIdx.y * 128, wid = min(128, lp - j0);
    q.cw = (wid + 31) & ~31;
    q.G = 256 / q.cw;
    q.jj = threadIdx.x % q.cw;
    q.ry = threadIdx.x / q.cw;
    q.j = j0 + q.jj;
    q.ok = q.jj < wid && q.ry < q.G;
    return q;
}

// s + c += x with the rounding error of every addition carried in c (Neumaier):
// |s + c - sum x| stays at float32 rounding of the total, not of every step
__device__ __forceinline__ void nsum(float &s, float &c, float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

// Q (rows x lp) -> nq bfloat16 terms; per row chunk the column sums of the terms
// (compensated float32 per thread, float64 across the row groups in a fixed order)
__global__ void split_bf16_kernel(const float *__restrict__ Q, int64_t rows, int lp, int nq, uint16_t *__restrict__ Q1,
                                  uint16_t *__restrict__ Q2, uint16_t *__restrict__ Q3, int64_t rpb,
                                  double *__restrict__ part) {
    __shared__ double red[256];
    const QLayout ql = q_layout(lp);
    const int j = ql.j, ry = ql.ry, G = ql.G;
    const int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min(rows, r0 + rpb);
    float s = 0.f, c = 0.f;
    if (ql.ok) {
        for (int64_t r = r0 + ry; r < r1; r += G) {
            const float x = Q[r * lp + j];
            const uint16_t h = rbf(x);
            Q1[r * lp + j] = h;
            nsum(s, c, bf(h));
            if (nq == 3) {
                const float d1 = x - bf(h);          // exact
                const uint16_t mid = rbf(d1);
                const float d2 = d1 - bf(mid);       // exact
                const uint16_t lo = rbf(d2);
                Q2[r * lp + j] = mid;
                Q3[r * lp + j] = lo;
                nsum(s, c, bf(mid));
                nsum(s, c, bf(lo));
            }
        }
    }
    red[threadIdx.x] = (double)s + (double)c;
    __syncthreads();
    if (ry == 0 && ql.ok) {
        double a = red[ql.jj];
        for (int g = 1; g < G; g++) a += red[g * ql.cw + ql.jj];
        part[(int64_t)blockIdx.x * lp + j] = a;
    }
}

// qsum[j] = sum over chunks: one warp per column, lane-strided partial sums in
// chunk order, then a fixed shuffle tree
__global__ void sum_rows_kernel(const double *__restrict__ part, int nch, int lp, double *__restrict__ qsum) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= lp) return;
    double s = 0.0;
    for (int k = lane; k < nch; k += 32) s += part[(int64_t)k * lp + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) qsum[j] = s;
}

// ------------------------------------------------------------------ e4m3
// value of an e4m3 code (finite codes only): normal 2^(e-7) (1 + m/8), subnormal m 2^-9
__device__ __forceinline__ float f8(uint8_t c) {
    const uint32_t e = (c >> 3) & 15u, mt = c & 7u, sg = (uint32_t)(c & 0x80u) << 24;
    if (e) return __uint_as_float(sg | ((e + 120u) << 23) | (mt << 20));
    return __uint_as_float(sg | __float_as_uint((float)mt * 0.001953125f));  // m * 2^-9
}

__device__ __forceinline__ uint8_t e4m3(float x) {
    unsigned short d;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(0.f), "f"(x));
    return (uint8_t)(d & 0xFF);
}

// 4 consecutive columns per thread (one 4-byte load per row; n and lda multiples of 4)
__global__ void colstats8_kernel(const uint8_t *__restrict__ A, int64_t m, int64_t n, int64_t lda, int64_t rpb,
                                 double *__restrict__ psum, double *__restrict__ psq) {
    __shared__ double rs[8][128], rq[8][128];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * 128 + 4 * tx;
    const int64_t r0 = (int64_t)blockIdx.y * rpb, r1 = min(m, r0 + rpb);
    double s[4] = {0.0, 0.0, 0.0, 0.0}, q[4] = {0.0, 0.0, 0.0, 0.0};
    if (c < n) {
        for (int64_t g = r0 + ty * 32; g < r1; g += 8 * 32) {
            float fs[4] = {0.f, 0.f, 0.f, 0.f}, fq[4] = {0.f, 0.f, 0.f, 0.f};
            const int64_t ge = min(r1, g + 32);
#pragma unroll 8
            for (int64_t r = g; r < ge; r++) {
                const uint32_t w = *reinterpret_cast<const uint32_t *>(A + r * lda + c);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const float a = f8((uint8_t)(w >> (8 * e)));
                    fs[e] += a;
                    fq[e] = fmaf(a, a, fq[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                s[e] += fs[e];
                q[e] += fq[e];
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
        rs[ty][4 * tx + e] = s[e];
        rq[ty][4 * tx + e] = q[e];
    }
    __syncthreads();
    if (ty == 0 && c < n) {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            double a = rs[0][4 * tx + e], b = rq[0][4 * tx + e];
            for (int k = 1; k < 8; k++) {
                a += rs[k][4 * tx + e];
                b += rq[k][4 * tx + e];
            }
            psum[(int64_t)blockIdx.y * n + c + e] = a;
            psq[(int64_t)blockIdx.y * n + c + e] = b;
        }
    }
}

// the statistics of column j scaled by s_j
__global__ void colstats8_finish(const double *__restrict__ psum, const double *__restrict__ psq, int nch, int64_t m,
                                 int64_t n, bool center, const float *__restrict__ sc, double *__restrict__ mu,
                                 float *__restrict__ mu_f, double *__restrict__ colv) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s = 0.0, q = 0.0;
    for (int k = 0; k < nch; k++) {
        s += psum[(int64_t)k * n + c];
        q += psq[(int64_t)k * n + c];
    }
    const double sj = (double)sc[c];
    const double mq = center ? s / (double)m : 0.0;   // mean of the codes' values
    mu[c] = sj * mq;
    mu_f[c] = (float)(sj * mq);
    colv[c] = sj * sj * (q - (double)m * mq * mq);
}

// one block per column j < lp: t_j, the codes of column j (row j of Zqt), c_j
__global__ void prep8_small_kernel(const float *__restrict__ Z, int64_t n, int l, int64_t ldzin,
                                   const float *__restrict__ sc, const double *__restrict__ mu,
                                   uint8_t *__restrict__ Zqt, int64_t ldz, float *__restrict__ t, float *__restrict__ c) {
    __shared__ float rmax[32];
    __shared__ double rsum[32];
    const int j = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint8_t *row = Zqt + (int64_t)j * ldz;
    if (j >= l) {  // padding rows
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) row[i] = 0;
        if (threadIdx.x == 0) {
            t[j] = 1.f;
            if (c) c[j] = 0.f;
        }
        return;
    }
    float mx = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf(sc[i] * Z[i * ldzin + j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) rmax[wid] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < nw; w++) mx = fmaxf(mx, rmax[w]);
    const float tj = mx > 0.f ? __fdiv_rn(mx, 448.f) : 1.f;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint8_t q = e4m3(__fdiv_rn(sc[i] * Z[i * ldzin + j], tj));
        row[i] = q;
        if (mu) acc += mu[i] / (double)sc[i] * (double)f8(q);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rsum[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        t[j] = tj;
        if (c) {
            double a = 0.0;
            for (int w = 0; w < nw; w++) a += rsum[w];
            c[j] = (float)(a * (double)tj);
        }
    }
}

// column maxima of Q (rows x lp), partial over row chunks
__global__ void colmax_q_kernel(const float *__restrict__ Q, int64_t rows, int lp, int64_t rpb,
                                float *__restrict__ part) {
    __shared__ float red[256];
    const QLayout ql = q_layout(lp);
    const int j = ql.j, ry = ql.ry, G = ql.G;
    const int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min(rows, r0 + rpb);
    float mx = 0.f;
    if (ql.ok)
        for (int64_t r = r0 + ry; r < r1; r += G) mx = fmaxf(mx, fabsf(Q[r * lp + j]));
    red[threadIdx.x] = mx;
    __syncthreads();
    if (ry == 0 && ql.ok) {
        for (int g = 1; g < G; g++) mx = fmaxf(mx, red[g * ql.cw + ql.jj]);
        part[(int64_t)blockIdx.x * lp + j] = mx;
    }
}

__global__ void colmax_finish(const float *__restrict__ part, int nch, int lp, float *__restrict__ u) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= lp) return;
    float mx = 0.f;
    for (int k = 0; k < nch; k++) mx = fmaxf(mx, part[(int64_t)k * lp + j]);
    u[j] = mx > 0.f ? __fdiv_rn(mx, 448.f) : 1.f;
}

// an e4m3 code's value in units of 2^-9 (every finite e4m3 value is an integer
// multiple of 2^-9, at most 448 = 229376 units)
__device__ __forceinline__ int f8_units(uint8_t q) {
    const int e = (q >> 3) & 15, mt = q & 7;
    const int v = e ? (8 + mt) << (e - 1) : mt;
    return (q & 0x80) ? -v : v;
}

// Qq = e4m3(Q / u) and per row chunk the column sums of u_j Qq_rj (the code sums are
// exact integers; one rounding, the product with u_j, in float64)
__global__ void quant_q_kernel(const float *__restrict__ Q, int64_t rows, int lp, const float *__restrict__ u,
                               uint8_t *__restrict__ Qq, int64_t rpb, double *__restrict__ part) {
    __shared__ long long red[256];
    const QLayout ql = q_layout(lp);
    const int j = ql.j, ry = ql.ry, G = ql.G;
    const int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min(rows, r0 + rpb);
    long long s = 0;
    if (ql.ok) {
        const float uj = u[j];
        for (int64_t r = r0 + ry; r < r1; r += G) {
            const uint8_t q = e4m3(__fdiv_rn(Q[r * lp + j], uj));
            Qq[r * lp + j] = q;
            s += f8_units(q);
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if (ry == 0 && ql.ok) {
        for (int g = 1; g < G; g++) s += red[g * ql.cw + ql.jj];
        part[(int64_t)blockIdx.x * lp + j] = (double)s * 0.001953125 * (double)u[j];
    }
}

// 16 codes per thread (one 16-byte load, two 16-byte stores); a scalar tail
__global__ void e4m3_to_bf16_kernel(const uint8_t *__restrict__ A, int64_t total, uint16_t *__restrict__ B) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16;
    if (i + 16 <= total) {
        const uint4 v = *reinterpret_cast<const uint4 *>(A + i);
        const uint8_t *c = reinterpret_cast<const uint8_t *>(&v);
        uint32_t o[8];
#pragma unroll
        for (int k = 0; k < 8; k++) o[k] = (uint32_t)rbf(f8(c[2 * k])) | ((uint32_t)rbf(f8(c[2 * k + 1])) << 16);
        *reinterpret_cast<uint4 *>(B + i) = make_uint4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<uint4 *>(B + i + 8) = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
        for (int64_t j = i; j < total; j++) B[j] = rbf(f8(A[j]));
    }
}

}  // namespace

cudaError_t colstats8(const void *A, int64_t m, int64_t n, int64_t lda, bool center, const float *scales, double *mu,
                      float *mu_f, double *fro2, double *psum, double *psq, double *colv, cudaStream_t s) {
    const int64_t nch = colstats16_chunks(m);
    const int64_t rpb = round_up(ceil_div(m, nch), 32);
    const int64_t ch = ceil_div(m, rpb);
    if (n % 4 || lda % 4 || (reinterpret_cast<uintptr_t>(A) & 3)) return cudaErrorInvalidValue;
    colstats8_kernel<<<dim3((unsigned)ceil_div(n, 128), (unsigned)ch), 256, 0, s>>>(static_cast<const uint8_t *>(A),
                                                                                    m, n, lda, rpb, psum, psq);
    colstats8_finish<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(psum, psq, (int)ch, m, n, center, scales, mu, mu_f,
                                                                colv);
    note_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return sum_f64(colv, n, fro2, s);
}

cudaError_t prep8_small(const float *Z, int64_t n, int l, int64_t ldzin, int lp, const float *scales,
                        const double *mu, void *Zqt, int64_t ldz, float *t, float *c, cudaStream_t s) {
    prep8_small_kernel<<<lp, 256, 0, s>>>(Z, n, l, ldzin, scales, mu, static_cast<uint8_t *>(Zqt), ldz, t, c);
    note_launch();
    return cudaGetLastError();
}

cudaError_t prep8_q(const float *Q, int64_t rows, int lp, void *Qq, float *u, float *mpart, double *part,
                    double *qsum, cudaStream_t s) {
    const int64_t rpb = q_chunk_rows(rows);
    const int64_t nch = ceil_div(rows, rpb);
    const dim3 grid((unsigned)nch, (unsigned)ceil_div(lp, 128));
    colmax_q_kernel<<<grid, 256, 0, s>>>(Q, rows, lp, rpb, mpart);
    colmax_finish<<<(unsigned)ceil_div(lp, 128), 128, 0, s>>>(mpart, (int)nch, lp, u);
    quant_q_kernel<<<grid, 256, 0, s>>>(Q, rows, lp, u, static_cast<uint8_t *>(Qq), rpb, part);
    sum_rows_kernel<<<(unsigned)ceil_div(lp, 8), 256, 0, s>>>(part, (int)nch, lp, qsum);
    note_launch(4);
    return cudaGetLastError();
}

cudaError_t e4m3_to_bf16(const void *A, int64_t count, void *B, cudaStream_t s) {
    if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return cudaErrorInvalidValue;
    e4m3_to_bf16_kernel<<<(unsigned)ceil_div(ceil_div(count, 16), 256), 256, 0, s>>>(
        static_cast<const uint8_t *>(A), count, static_cast<uint16_t *>(B));
    note_launch();
    return cudaGetLastError();
}

int64_t colstats16_chunks(int64_t m) { return ceil_div(m, 4096) < 1024 ? ceil_div(m, 4096) : 1024; }

cudaError_t colstats16(const void *A, int64_t m, int64_t n, int64_t lda, bool center, double *mu, float *mu_f,
                       double *fro2, double *psum, double *psq, double *colv, cudaStream_t s) {
    const int64_t nch = colstats16_chunks(m);
    const int64_t rpb = round_up(ceil_div(m, nch), 32);
    const int64_t ch = ceil_div(m, rpb);
    colstats16_kernel<<<dim3((unsigned)ceil_div(n, 32), (unsigned)ch), 256, 0, s>>>(
        static_cast<const uint16_t *>(A), m, n, lda, rpb, psum, psq);
    colstats16_finish<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(psum, psq, (int)ch, m, n, center, mu, mu_f, colv);
    note_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return sum_f64(colv, n, fro2, s);
}

cudaError_t to_bf16_t(const float *Z, int64_t n, int l, int64_t ldzin, int lp, void *Zt, int64_t ldz,
                      const double *mu, float *c, cudaStream_t s) {
    const int64_t total = (int64_t)lp * n;
    to_bf16_t_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(Z, n, l, ldzin, lp, static_cast<uint16_t *>(Zt),
                                                                    ldz);
    note_launch();
    if (mu && c) {
        mean_corr_kernel<<<(unsigned)ceil_div(lp, 8), 256, 0, s>>>(mu, static_cast<const uint16_t *>(Zt), n, ldz, lp,
                                                                    c);
        note_launch();
    }
    return cudaGetLastError();
}

// rows per chunk of the passes over Q: about four chunks per SM, multiples of 32 rows
int64_t q_chunk_rows(int64_t rows) { return round_up(std::max<int64_t>(ceil_div(rows, 4 * 152), 32), 32); }
int64_t split_bf16_chunks(int64_t rows) { return ceil_div(rows, q_chunk_rows(rows)); }

cudaError_t split_bf16(const float *Q, int64_t rows, int lp, int nq, void *Q1, void *Q2, void *Q3, double *part,
                       double *qsum, cudaStream_t s) {
    const int64_t rpb = q_chunk_rows(rows);
    const int64_t nch = ceil_div(rows, rpb);
    split_bf16_kernel<<<dim3((unsigned)nch, (unsigned)ceil_div(lp, 128)), 256, 0, s>>>(Q, rows, lp, nq,
                                                                                    static_cast<uint16_t *>(Q1),
                                                    static_cast<uint16_t *>(Q2), static_cast<uint16_t *>(Q3), rpb,
                                                    part);
    sum_rows_kernel<<<(unsigned)ceil_div(lp, 8), 256, 0, s>>>(part, (int)nch, lp, qsum);
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace gbr
