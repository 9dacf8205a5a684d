// Column centring and squared Frobenius norm (Sec. 1 zero-mean assumption;
// Eq. (sumeigen): sum_i lambda_i = ||A||_F^2 = sum_ij a_ij^2).
//
// HBM-bound: pass 1 reads A once (column sums), pass 2 reads and writes A
// once (subtract the mean, accumulate squares).  Each block owns a contiguous
// slab of rows, so every load is a coalesced row segment; threads own
// 16-byte column groups.  Sums run in the element type over 32-row groups and
// are then promoted to float64 (float64 throughput on GB300 is ~1/64 of
// float32, so per-element float64 adds would bound the kernel); the cross-block
// reductions are float64 in a fixed order, so results are deterministic.
#include "common.cuh"

namespace gbr {
namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 32;  // rows summed in the element type before promotion

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

template <typename V, typename T>
__device__ __forceinline__ void unpack(const V &v, T *x);
template <> __device__ __forceinline__ void unpack(const float4 &v, float *x) { x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
template <> __device__ __forceinline__ void unpack(const double2 &v, double *x) { x[0] = v.x; x[1] = v.y; }
template <typename V, typename T>
__device__ __forceinline__ V pack(const T *x);
template <> __device__ __forceinline__ float4 pack(const float *x) { return make_float4(x[0], x[1], x[2], x[3]); }
template <> __device__ __forceinline__ double2 pack(const double *x) { return make_double2(x[0], x[1]); }

// part[chunk * n + c] = sum over the chunk's rows of A[r][c]
template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) colsum_kernel(const T *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                                                          int64_t rows_per_chunk, double *__restrict__ part) {
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r1 = min(m, r0 + rows_per_chunk);
    for (int64_t c0 = (int64_t)threadIdx.x * VEC; c0 < n; c0 += (int64_t)kThreads * VEC) {
        double acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; v++) acc[v] = 0.0;
        for (int64_t g = r0; g < r1; g += kGroup) {
            const int64_t e = min(r1, g + kGroup);
            T sub[VEC];
#pragma unroll
            for (int v = 0; v < VEC; v++) sub[v] = T(0);
#pragma unroll 8
            for (int64_t r = g; r < e; r++) {
                T x[VEC];
                if constexpr (VEC > 1) {
                    using V = typename Vec<T>::type;
                    unpack(*reinterpret_cast<const V *>(A + r * lda + c0), x);
                } else {
                    x[0] = A[r * lda + c0];
                }
#pragma unroll
                for (int v = 0; v < VEC; v++) sub[v] += x[v];
            }
#pragma unroll
            for (int v = 0; v < VEC; v++) acc[v] += (double)sub[v];
        }
#pragma unroll
        for (int v = 0; v < VEC; v++) part[(int64_t)blockIdx.x * n + c0 + v] = acc[v];
    }
}

// one warp per column: lanes sum interleaved chunks, then a fixed xor tree
__global__ void colmean_kernel(const double *__restrict__ part, int64_t chunks, int64_t n, int64_t m,
                               double *__restrict__ mu) {
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    double s = 0.0;
    for (int64_t k = lane; k < chunks; k += 32) s += part[k * n + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) mu[c] = s / (double)m;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// A <- A - mu (if subtract); sq[chunk] = sum over the chunk of a_ij^2
template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) center_sq_kernel(T *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                                                             int64_t rows_per_chunk, const double *__restrict__ mu,
                                                             int subtract, double *__restrict__ sq, int write = 1) {
    __shared__ double red[kThreads / 32];
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r1 = min(m, r0 + rows_per_chunk);
    double acc = 0.0;
    for (int64_t c0 = (int64_t)threadIdx.x * VEC; c0 < n; c0 += (int64_t)kThreads * VEC) {
        T mv[VEC];
#pragma unroll
        for (int v = 0; v < VEC; v++) mv[v] = subtract ? (T)mu[c0 + v] : T(0);
        for (int64_t g = r0; g < r1; g += kGroup) {
            const int64_t e = min(r1, g + kGroup);
            T sub = T(0);
#pragma unroll 8
            for (int64_t r = g; r < e; r++) {
                T x[VEC];
                if constexpr (VEC > 1) {
                    using V = typename Vec<T>::type;
                    V *p = reinterpret_cast<V *>(A + r * lda + c0);
                    unpack(*p, x);
#pragma unroll
                    for (int v = 0; v < VEC; v++) x[v] -= mv[v];
                    if (subtract && write) *p = pack<V>(x);
                } else {
                    x[0] = A[r * lda + c0] - mv[0];
                    if (subtract && write) A[r * lda + c0] = x[0];
                }
#pragma unroll
                for (int v = 0; v < VEC; v++) sub += x[v] * x[v];
            }
            acc += (double)sub;
        }
    }
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) sq[blockIdx.x] = t;
}

__global__ void sum_kernel(const double *__restrict__ x, int64_t count, double *__restrict__ out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc += x[i];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) *out = t;
}

template <typename T>
__global__ void mean_copy_kernel(const double *__restrict__ mu, int64_t n, int64_t npad, T *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npad) out[i] = i < n ? (T)mu[i] : T(0);
}

// sum[i] *= inv_m (column sums over all row blocks -> means), out = the means in T, padded
template <typename T>
__global__ void scale_means_kernel(double *__restrict__ sum, int64_t n, int64_t npad, double inv_m,
                                   T *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i < n) {
        const double mu = sum[i] * inv_m;
        sum[i] = mu;
        out[i] = (T)mu;
    } else {
        out[i] = T(0);
    }
}

// C[r][c] -= (x ? x[r] : 1) * y[c]
template <typename T>
__global__ void rank1_sub_kernel(T *__restrict__ C, int64_t rows, int64_t cols, int64_t ldc, const T *__restrict__ x,
                                 const T *__restrict__ y) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t r = idx / cols, c = idx % cols;
    C[r * ldc + c] -= (x ? x[r] : T(1)) * y[c];
}

// c[j] = sum_k mu[k] B[k][j] (j < N), one thread per j
template <typename T>
__global__ void vecmat_kernel(const T *__restrict__ mu, const T *__restrict__ B, int64_t K, int64_t N, int64_t ldb,
                              T *__restrict__ c) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s = 0.0;
    for (int64_t k = 0; k < K; k++) s += (double)mu[k] * (double)B[k * ldb + j];
    c[j] = (T)s;
}

int64_t chunk_rows(int64_t m) {
    // about four blocks per SM on a 152-SM part, at least one 32-row group each
    int64_t r = ceil_div(m, 608);
    return r < kGroup ? kGroup : round_up(r, kGroup);
}

}  // namespace

int64_t center_partials(int64_t m, int64_t n) {
    const int64_t chunks = ceil_div(m, chunk_rows(m));
    return chunks * n + chunks;
}

template <typename T>
cudaError_t center_columns(T *A, int64_t m, int64_t n, int64_t lda, bool subtract, double *mu, double *fro2,
                           double *part, cudaStream_t s) {
    const int64_t rpc = chunk_rows(m);
    const int64_t chunks = ceil_div(m, rpc);
    double *colpart = part, *sq = part + chunks * n;
    constexpr int V = Vec<T>::n;
    const bool vec = (n % V == 0) && (lda % V == 0) && ((uintptr_t)A % 16 == 0);
    if (subtract) {
        if (vec) colsum_kernel<T, V><<<(unsigned)chunks, kThreads, 0, s>>>(A, m, n, lda, rpc, colpart);
        else colsum_kernel<T, 1><<<(unsigned)chunks, kThreads, 0, s>>>(A, m, n, lda, rpc, colpart);
        colmean_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, s>>>(colpart, chunks, n, m, mu);
        note_launch(2);
    } else {
        cudaMemsetAsync(mu, 0, sizeof(double) * n, s);
    }
    if (vec) center_sq_kernel<T, V><<<(unsigned)chunks, kThreads, 0, s>>>(A, m, n, lda, rpc, mu, subtract, sq);
    else center_sq_kernel<T, 1><<<(unsigned)chunks, kThreads, 0, s>>>(A, m, n, lda, rpc, mu, subtract, sq);
    sum_kernel<<<1, 1024, 0, s>>>(sq, chunks, fro2);
    note_launch(2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t column_means(const T *A, int64_t m, int64_t n, int64_t lda, double *mu, T *mu_t, int64_t npad,
                         double *part, cudaStream_t s) {
    const int64_t rpc = chunk_rows(m);
    const int64_t chunks = ceil_div(m, rpc);
    constexpr int V = Vec<T>::n;
    const bool vec = (n % V == 0) && (lda % V == 0) && ((uintptr_t)A % 16 == 0);
    if (vec) colsum_kernel<T, V><<<(unsigned)chunks, kThreads, 0, s>>>(A, m, n, lda, rpc, part);
    else colsum_kernel<T, 1><<<(unsigned)chunks, kThreads, 0, s>>>(A, m, n, lda, rpc, part);
    colmean_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, s>>>(part, chunks, n, m, mu);
    mean_copy_kernel<T><<<(unsigned)ceil_div(npad, 256), 256, 0, s>>>(mu, n, npad, mu_t);
    note_launch(3);
    return cudaGetLastError();
}

template <typename T>
cudaError_t column_sums(const T *X, int64_t rows, int64_t cols, int64_t ld, double *dsum, T *out, double *part,
                        cudaStream_t s) {
    const int64_t rpc = chunk_rows(rows);
    const int64_t chunks = ceil_div(rows, rpc);
    constexpr int V = Vec<T>::n;
    const bool vec = (cols % V == 0) && (ld % V == 0) && ((uintptr_t)X % 16 == 0);
    if (vec) colsum_kernel<T, V><<<(unsigned)chunks, kThreads, 0, s>>>(X, rows, cols, ld, rpc, part);
    else colsum_kernel<T, 1><<<(unsigned)chunks, kThreads, 0, s>>>(X, rows, cols, ld, rpc, part);
    colmean_kernel<<<(unsigned)ceil_div(cols, 8), 256, 0, s>>>(part, chunks, cols, 1, dsum);
    mean_copy_kernel<T><<<(unsigned)ceil_div(cols, 256), 256, 0, s>>>(dsum, cols, cols, out);
    note_launch(3);
    return cudaGetLastError();
}

template <typename T>
cudaError_t centered_fro2(const T *A, int64_t m, int64_t n, int64_t lda, const double *mu, double *fro2, double *part,
                          cudaStream_t s) {
    const int64_t rpc = chunk_rows(m);
    const int64_t chunks = ceil_div(m, rpc);
    double *sq = part + chunks * n;
    constexpr int V = Vec<T>::n;
    const bool vec = (n % V == 0) && (lda % V == 0) && ((uintptr_t)A % 16 == 0);
    T *Aw = const_cast<T *>(A);  // read only: write = 0
    if (vec) center_sq_kernel<T, V><<<(unsigned)chunks, kThreads, 0, s>>>(Aw, m, n, lda, rpc, mu, mu != nullptr, sq, 0);
    else center_sq_kernel<T, 1><<<(unsigned)chunks, kThreads, 0, s>>>(Aw, m, n, lda, rpc, mu, mu != nullptr, sq, 0);
    sum_kernel<<<1, 1024, 0, s>>>(sq, chunks, fro2);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t sum_f64(const double *x, int64_t count, double *out, cudaStream_t s) {
    sum_kernel<<<1, 1024, 0, s>>>(x, count, out);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t rank1_sub(T *C, int64_t rows, int64_t cols, int64_t ldc, const T *x, const T *y, cudaStream_t s) {
    const int64_t total = rows * cols;
    if (total <= 0) return cudaSuccess;
    rank1_sub_kernel<T><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(C, rows, cols, ldc, x, y);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t scale_means(double *sum, int64_t n, int64_t npad, double inv_m, T *mu_t, cudaStream_t s) {
    scale_means_kernel<T><<<(unsigned)ceil_div(npad, 256), 256, 0, s>>>(sum, n, npad, inv_m, mu_t);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t vecmat(const T *mu, const T *B, int64_t K, int64_t N, int64_t ldb, T *c, cudaStream_t s) {
    vecmat_kernel<T><<<(unsigned)ceil_div(N, 128), 128, 0, s>>>(mu, B, K, N, ldb, c);
    note_launch();
    return cudaGetLastError();
}

#define INST_CENTER(T)                                                                                            \
    template cudaError_t column_means<T>(const T *, int64_t, int64_t, int64_t, double *, T *, int64_t, double *,    \
                                         cudaStream_t);                                                           \
    template cudaError_t centered_fro2<T>(const T *, int64_t, int64_t, int64_t, const double *, double *, double *, \
                                          cudaStream_t);                                                          \
    template cudaError_t column_sums<T>(const T *, int64_t, int64_t, int64_t, double *, T *, double *,              \
                                        cudaStream_t);                                                            \
    template cudaError_t rank1_sub<T>(T *, int64_t, int64_t, int64_t, const T *, const T *, cudaStream_t);          \
    template cudaError_t vecmat<T>(const T *, const T *, int64_t, int64_t, int64_t, T *, cudaStream_t);            \
    template cudaError_t scale_means<T>(double *, int64_t, int64_t, double, T *, cudaStream_t);
INST_CENTER(float)
INST_CENTER(double)

template cudaError_t center_columns<float>(float *, int64_t, int64_t, int64_t, bool, double *, double *, double *,
                                           cudaStream_t);
template cudaError_t center_columns<double>(double *, int64_t, int64_t, int64_t, bool, double *, double *, double *,
                                            cudaStream_t);

}  // namespace gbr
