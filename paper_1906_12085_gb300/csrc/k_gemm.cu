// Tall-skinny products on CUDA cores (float32 / float64):
//   gemm_nn : C = A B        (Y = A Omega, Y = A Z, Q = Y R^{-1}, U = Q W; Sec. 3.1.2 steps 2-3, 7)
//   gemm_tn : C = A^T B      (Z = A^T Q, T = A^T Q, Gram matrices; Sec. 3.1.2 steps 3-5, Sec. 3.1.3 step 1)
//
// Both share one register-tiled core: a 128 x 64 output tile per 256-thread
// CTA, 8 x 4 outputs per thread, a 16-deep K slab staged in shared memory
// with the next slab prefetched into registers while the current one is
// consumed.  gemm_tn splits the long K (= rows of A, up to millions) into row
// chunks; each chunk writes its own partial tile and a second kernel sums the
// partials in chunk order, so results are bitwise reproducible.
#include "common.cuh"

namespace gbr {
namespace {

constexpr int BM = 128, BN = 64, BK = 16, NT = 256;
constexpr int PAD = 4;

template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static constexpr int n = 4; };
template <> struct V16<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ float fmat(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
struct Tile {
    T a[BK][BM + PAD];  // a[k][i] = op(A)(m0 + i, k0 + k)
    T b[BK][BN + PAD];  // b[k][j] = B(k0 + k, n0 + j)
};

// Register staging for one K slab: A slab BM x BK, B slab BK x BN.
template <typename T>
struct Stage {
    static constexpr int VE = V16<T>::n;
    static constexpr int NA = BM * BK / VE / NT;  // vectors of the A slab per thread
    static constexpr int NB = BK * BN / VE / NT;
    T a[NA][VE];
    T b[NB][VE];
};

// Load the A slab. TRANS = false: A is M x K row-major (slab rows m0.., cols k0..).
// TRANS = true: A is K x M row-major and op(A) = A^T (slab rows k0.., cols m0..).
template <typename T, bool TRANS>
__device__ __forceinline__ void load_a(Stage<T> &st, const T *__restrict__ A, int64_t lda, int64_t M, int64_t K,
                                       int64_t m0, int64_t k0, bool fast) {
    constexpr int VE = V16<T>::n;
    using V = typename V16<T>::type;
#pragma unroll
    for (int v = 0; v < Stage<T>::NA; v++) {
        const int idx = threadIdx.x + v * NT;
        int r, c;  // position inside the stored slab (row-major in memory order)
        if (!TRANS) { r = idx / (BK / VE); c = (idx % (BK / VE)) * VE; }   // BM rows x BK cols
        else        { r = idx / (BM / VE); c = (idx % (BM / VE)) * VE; }   // BK rows x BM cols
        const int64_t gr = (TRANS ? k0 : m0) + r, gc = (TRANS ? m0 : k0) + c;
        const int64_t rmax = TRANS ? K : M, cmax = TRANS ? M : K;
        if (fast) {
            const V x = *reinterpret_cast<const V *>(A + gr * lda + gc);
            const T *px = reinterpret_cast<const T *>(&x);
#pragma unroll
            for (int e = 0; e < VE; e++) st.a[v][e] = px[e];
        } else {
#pragma unroll
            for (int e = 0; e < VE; e++)
                st.a[v][e] = (gr < rmax && gc + e < cmax) ? A[gr * lda + gc + e] : T(0);
        }
    }
}

template <typename T>
__device__ __forceinline__ void load_b(Stage<T> &st, const T *__restrict__ B, int64_t ldb, int64_t K, int64_t N,
                                       int64_t k0, int64_t n0, bool fast) {
    constexpr int VE = V16<T>::n;
    using V = typename V16<T>::type;
#pragma unroll
    for (int v = 0; v < Stage<T>::NB; v++) {
        const int idx = threadIdx.x + v * NT;
        const int r = idx / (BN / VE), c = (idx % (BN / VE)) * VE;
        const int64_t gr = k0 + r, gc = n0 + c;
        if (fast) {
            const V x = *reinterpret_cast<const V *>(B + gr * ldb + gc);
            const T *px = reinterpret_cast<const T *>(&x);
#pragma unroll
            for (int e = 0; e < VE; e++) st.b[v][e] = px[e];
        } else {
#pragma unroll
            for (int e = 0; e < VE; e++) st.b[v][e] = (gr < K && gc + e < N) ? B[gr * ldb + gc + e] : T(0);
        }
    }
}

template <typename T, bool TRANS>
__device__ __forceinline__ void store_stage(Tile<T> &t, const Stage<T> &st) {
    constexpr int VE = V16<T>::n;
#pragma unroll
    for (int v = 0; v < Stage<T>::NA; v++) {
        const int idx = threadIdx.x + v * NT;
        if (!TRANS) {
            const int r = idx / (BK / VE), c = (idx % (BK / VE)) * VE;
#pragma unroll
            for (int e = 0; e < VE; e++) t.a[c + e][r] = st.a[v][e];
        } else {
            const int r = idx / (BM / VE), c = (idx % (BM / VE)) * VE;
#pragma unroll
            for (int e = 0; e < VE; e++) t.a[r][c + e] = st.a[v][e];
        }
    }
#pragma unroll
    for (int v = 0; v < Stage<T>::NB; v++) {
        const int idx = threadIdx.x + v * NT;
        const int r = idx / (BN / VE), c = (idx % (BN / VE)) * VE;
#pragma unroll
        for (int e = 0; e < VE; e++) t.b[r][c + e] = st.b[v][e];
    }
}

// C tile (rows m0.., cols n0..) = sum over k in [kbeg, kend) of op(A)(i, k) B(k, j).
// Thread layout: 8 warps as 4 x 2 warp tiles of 32 x 32; lane -> 8 rows x 4 cols.
template <typename T, bool TRANS>
__device__ __forceinline__ void tile_product(T acc[8][4], Tile<T> &t, const T *__restrict__ A, int64_t lda,
                                             const T *__restrict__ B, int64_t ldb, int64_t M, int64_t N,
                                             int64_t m0, int64_t n0, int64_t kbeg, int64_t kend) {
    constexpr int VE = V16<T>::n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tr = (warp >> 1) * 32 + (lane >> 3) * 8;
    const int tc = (warp & 1) * 32 + (lane & 7) * 4;
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = T(0);
    const bool a_al = (lda % VE == 0) && ((uintptr_t)A % 16 == 0);
    const bool b_al = (ldb % VE == 0) && ((uintptr_t)B % 16 == 0);
    const int64_t Kdim = kend;  // global bound of the K index
    Stage<T> st;
    int64_t k0 = kbeg;
    if (k0 >= kend) return;
    auto fast_a = [&](int64_t kk) {
        return a_al && (TRANS ? (kk + BK <= Kdim && m0 + BM <= M) : (m0 + BM <= M && kk + BK <= Kdim));
    };
    auto fast_b = [&](int64_t kk) { return b_al && kk + BK <= Kdim && n0 + BN <= N; };
    load_a<T, TRANS>(st, A, lda, M, Kdim, m0, k0, fast_a(k0));
    load_b<T>(st, B, ldb, Kdim, N, k0, n0, fast_b(k0));
    for (; k0 < kend; k0 += BK) {
        store_stage<T, TRANS>(t, st);
        __syncthreads();
        const int64_t kn = k0 + BK;
        if (kn < kend) {
            load_a<T, TRANS>(st, A, lda, M, Kdim, m0, kn, fast_a(kn));
            load_b<T>(st, B, ldb, Kdim, N, kn, n0, fast_b(kn));
        }
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            T a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; i++) a[i] = t.a[kk][tr + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = t.b[kk][tc + j];
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmat(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void store_tile(const T acc[8][4], T *__restrict__ C, int64_t ldc, int64_t M, int64_t N,
                                           int64_t m0, int64_t n0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = m0 + (warp >> 1) * 32 + (lane >> 3) * 8;
    const int64_t c0 = n0 + (warp & 1) * 32 + (lane & 7) * 4;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int64_t r = r0 + i;
        if (r >= M) break;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (c0 + j < N) C[r * ldc + c0 + j] = acc[i][j];
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) gemm_nn_kernel(int64_t M, int64_t N, int64_t K, const T *__restrict__ A,
                                                     int64_t lda, const T *__restrict__ B, int64_t ldb,
                                                     T *__restrict__ C, int64_t ldc) {
    __shared__ __align__(16) Tile<T> t;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    T acc[8][4];
    tile_product<T, false>(acc, t, A, lda, B, ldb, M, N, m0, n0, 0, K);
    store_tile<T>(acc, C, ldc, M, N, m0, n0);
}

// part[chunk] (N x L dense) = A[rows of chunk]^T B[rows of chunk]; if out_ld > 0 the
// single chunk writes straight to out.
template <typename T>
__global__ void __launch_bounds__(NT) gemm_tn_kernel(int64_t rows, int64_t N, int64_t L, const T *__restrict__ A,
                                                     int64_t lda, const T *__restrict__ B, int64_t ldb,
                                                     int64_t rows_per_chunk, T *__restrict__ out, int64_t out_ld) {
    __shared__ __align__(16) Tile<T> t;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    const int64_t kb = (int64_t)blockIdx.z * rows_per_chunk;
    const int64_t ke = min(rows, kb + rows_per_chunk);
    T acc[8][4];
    tile_product<T, true>(acc, t, A, lda, B, ldb, N, L, m0, n0, kb, ke);
    if (out_ld > 0) store_tile<T>(acc, out, out_ld, N, L, m0, n0);
    else store_tile<T>(acc, out + (int64_t)blockIdx.z * N * L, L, N, L, m0, n0);
}

// C[i][j] = sum_{s < chunks} part[s][i][j], in chunk order.
template <typename T>
__global__ void reduce_chunks_kernel(const T *__restrict__ part, int64_t chunks, int64_t N, int64_t L,
                                     T *__restrict__ C, int64_t ldc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * L) return;
    const int64_t stride = N * L;
    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
    int64_t c = 0;
    for (; c + 4 <= chunks; c += 4) {
        s0 += part[(c + 0) * stride + idx];
        s1 += part[(c + 1) * stride + idx];
        s2 += part[(c + 2) * stride + idx];
        s3 += part[(c + 3) * stride + idx];
    }
    for (; c < chunks; c++) s0 += part[c * stride + idx];
    C[(idx / L) * ldc + idx % L] = (s0 + s1) + (s2 + s3);
}

struct SplitK {
    int64_t chunks, rows_per_chunk;
};

SplitK choose_split(int64_t rows, int64_t N, int64_t L) {
    const int64_t tiles = ceil_div(N, BM) * ceil_div(L, BN);
    const int64_t target = 304;  // two CTAs per SM on 152 SMs
    int64_t chunks = ceil_div(target, tiles);
    const int64_t min_rows = 256;
    const int64_t max_chunks = ceil_div(rows, min_rows);
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    int64_t rpc = round_up(ceil_div(rows, chunks), BK);
    chunks = ceil_div(rows, rpc);
    return {chunks, rpc};
}

}  // namespace

int64_t gemm_tn_partials(int64_t rows, int64_t N, int64_t L) {
    const SplitK sk = choose_split(rows, N, L);
    return sk.chunks > 1 ? sk.chunks * N * L : 0;
}

template <typename T>
cudaError_t gemm_nn(int64_t M, int64_t N, int64_t K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C,
                    int64_t ldc, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)ceil_div(M, BM), (unsigned)ceil_div(N, BN));
    gemm_nn_kernel<T><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t gemm_tn(int64_t rows, int64_t N, int64_t L, const T *A, int64_t lda, const T *B, int64_t ldb, T *C,
                    int64_t ldc, T *part, int64_t part_elems, cudaStream_t s) {
    if (N <= 0 || L <= 0) return cudaSuccess;
    const SplitK sk = choose_split(rows, N, L);
    dim3 grid((unsigned)ceil_div(N, BM), (unsigned)ceil_div(L, BN), (unsigned)sk.chunks);
    if (sk.chunks == 1) {
        gemm_tn_kernel<T><<<grid, NT, 0, s>>>(rows, N, L, A, lda, B, ldb, sk.rows_per_chunk, C, ldc);
        note_launch();
        return cudaGetLastError();
    }
    if (part == nullptr || part_elems < sk.chunks * N * L) return cudaErrorInvalidValue;
    gemm_tn_kernel<T><<<grid, NT, 0, s>>>(rows, N, L, A, lda, B, ldb, sk.rows_per_chunk, part, 0);
    reduce_chunks_kernel<T><<<(unsigned)ceil_div(N * L, 256), 256, 0, s>>>(part, sk.chunks, N, L, C, ldc);
    note_launch(2);
    return cudaGetLastError();
}

template cudaError_t gemm_nn<float>(int64_t, int64_t, int64_t, const float *, int64_t, const float *, int64_t,
                                    float *, int64_t, cudaStream_t);
template cudaError_t gemm_nn<double>(int64_t, int64_t, int64_t, const double *, int64_t, const double *, int64_t,
                                     double *, int64_t, cudaStream_t);
template cudaError_t gemm_tn<float>(int64_t, int64_t, int64_t, const float *, int64_t, const float *, int64_t,
                                    float *, int64_t, float *, int64_t, cudaStream_t);
template cudaError_t gemm_tn<double>(int64_t, int64_t, int64_t, const double *, int64_t, const double *, int64_t,
                                     double *, int64_t, double *, int64_t, cudaStream_t);

}  // namespace gbr
