// bfloat16 and e4m3 tall-skinny products of the precision form on tcgen05
// (kind::f16 / kind::f8f6f4, float32 accumulation in tensor memory).  The stored bfloat16 matrix A is an
// exact operand; the small operand is bfloat16 too: rounded from float32 for
// the power-iteration products (only its span matters there), or split into
// three bfloat16 terms whose sum carries the float32 value (the
// Rayleigh-Ritz product, float32-accurate against the stored A).
//
//   tc16_gemm_nn : Y (m x N) = A (m x n) Z (n x N) - 1 c^T      (c: N floats or NULL)
//                  A and Zt (Z transposed, N x n) are K-major: TMA boxes of 64
//                  K elements (one 128-byte swizzled row) x rows.
//   tc16_gemm_tn : C (n x N) = A^T (Q_1 + ... + Q_nb) - mu (1^T Q)  (mu, qsum optional)
//                  A and Q are used as stored (row-major): both operands are
//                  MN-major; split-K over row chunks into float32 partials that a
//                  second kernel sums in chunk order.
//
// Both kernels are persistent and warp-specialised: warp 0 issues the TMA loads
// of a ring of shared-memory stages, one thread of warp 1 issues the MMAs into
// one of two TMEM accumulators, warps 2-5 drain the other accumulator.  Every
// wait is bounded; a stalled pipeline sets ST_TIMEOUT instead of hanging.
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace gbr {
namespace {

using namespace tc;

constexpr int TM = 128;                  // MMA M
constexpr int THR = 192;                 // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int NEPI = 128;
constexpr uint32_t A_ST = TM * 128;      // 16 KB of A per stage (NN: 128 rows; TN: 128 columns)

// Element-size traits (ESZ bytes per element: 2 bfloat16, 1 e4m3).  A stage holds
// 128 bytes of K per row in NN (one swizzled row), and in TN TN_BK rows of the
// 128-column A tile as MN atoms of 128 bytes (QW elements); each MMA consumes KMMA
// K elements (32 bytes of a K-major row, or KMMA rows of an MN-major atom).
template <int ESZ>
struct Elt;
template <>
struct Elt<2> {
    static constexpr int NN_BK = 64, TN_BK = 64, KMMA = 16, QW = 64, A_ATOMS = 2;
    static constexpr uint32_t ATOM = 64 * 128;       // one MN atom over the stage's 64 rows
    static constexpr uint32_t LBO = ATOM;            // byte stride between MN-adjacent atoms
    static constexpr uint32_t Q_ROOM = 2 * ATOM;     // two atoms of room per Q operand (see TN16)
};
template <>
struct Elt<1> {
    static constexpr int NN_BK = 128, TN_BK = 128, KMMA = 32, QW = 128, A_ATOMS = 1;
    static constexpr uint32_t ATOM = 128 * 128;      // the single MN atom over the stage's 128 rows
    static constexpr uint32_t LBO = 1024;            // unused with one atom; equal to SBO, so both stride readings agree
    static constexpr uint32_t Q_ROOM = ATOM;
};

template <int ESZ>
__host__ __device__ constexpr uint32_t idesc_e(int M, int N, bool a_mn, bool b_mn) {
    return ESZ == 2 ? idesc_bf16(M, N, a_mn, b_mn) : idesc_e4m3(M, N, a_mn, b_mn);
}

template <int ESZ>
__device__ __forceinline__ void mma_e(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (ESZ == 2) mma_bf16(d, a, b, idesc, acc);
    else mma_e4m3(d, a, b, idesc, acc);
}
// TN: stages accumulated in one TMEM accumulator before it is drained and added (IEEE
// float32) to the partial: the tensor core's accumulation error grows with the number of
// accumulation steps, 4 stages (256 rows) bound it.
constexpr int SUBK = 4;

template <int S>
struct Bars16 {
    uint64_t full[S], empty[S];
    uint64_t acc_full[2], acc_empty[2];
    uint32_t tmem;
    int abort_flag;
};

__device__ __forceinline__ bool wait16(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (*abort_flag) return false;
    if (mbar_wait(bar, parity)) return true;
    *abort_flag = 1;
    return false;
}

constexpr int cmin(int a, int b) { return a < b ? a : b; }

// ======================================================================= NN
template <int N, int ESZ>
struct NN16 {
    // two accumulators of N float32 columns: 256 TMEM columns up to N = 128, 512 above
    static constexpr uint32_t ACS = N > 128 ? 256 : 128;  // column stride of the accumulators
    static constexpr uint32_t TC = 2 * ACS;
    static constexpr uint32_t B_ST = N * 128;
    static constexpr uint32_t STAGE = A_ST + B_ST;
    static constexpr int S = cmin(8, (int)((200 * 1024) / STAGE));
    static constexpr uint32_t NEED = S * STAGE + 1024 + sizeof(Bars16<S>) + 64;
    static constexpr uint32_t SMEM = NEED > 120 * 1024 ? NEED : 120 * 1024;  // one CTA per SM (owns TMEM)
};

template <int N, int ESZ>
__global__ void __launch_bounds__(THR, 1)
    tc16_nn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t m, int n,
                   float *__restrict__ Y, int64_t ldy, const float *__restrict__ ts, const float *__restrict__ c,
                   int *__restrict__ status) {
    using C = NN16<N, ESZ>;
    constexpr int BK = Elt<ESZ>::NN_BK;
    constexpr int S = C::S;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;
    uint8_t *sB = sA + S * A_ST;
    Bars16<S> *bar = reinterpret_cast<Bars16<S> *>(sB + S * C::B_ST);
    volatile int *abort_flag = &bar->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (m + TM - 1) / TM;
    const int nkb = (n + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&bar->full[s], 1);
            mbar_init(&bar->empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bar->acc_full[b], 1);
            mbar_init(&bar->acc_empty[b], NEPI);
        }
        bar->abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&bar->tmem, C::TC);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bar->tmem;

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            uint32_t g = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x)
                for (int kb = 0; kb < nkb; kb++, g++) {
                    const int s = g % S;
                    if (!(ok = wait16(&bar->empty[s], ((g / S) & 1) ^ 1, abort_flag))) break;
                    mbar_arrive_expect_tx(&bar->full[s], C::STAGE);
                    tma_load_2d(sA + s * A_ST, &tmA, kb * BK, (int32_t)(t * TM), &bar->full[s]);
                    tma_load_2d(sB + s * C::B_ST, &tmB, kb * BK, 0, &bar->full[s]);
                }
            for (uint32_t k = g > (uint32_t)S ? g - S : 0; k < g; k++) mbar_wait(&bar->full[k % S], (k / S) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_e<ESZ>(TM, N, false, false);
            uint32_t g = 0, it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x, it++) {
                const uint32_t b = it & 1;
                if (!(ok = wait16(&bar->acc_empty[b], ((it >> 1) & 1) ^ 1, abort_flag))) break;
                tc_fence_after();
                const uint32_t d = tmem + b * C::ACS;
                for (int kb = 0; kb < nkb; kb++, g++) {
                    const int s = g % S;
                    if (!(ok = wait16(&bar->full[s], (g / S) & 1, abort_flag))) break;
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < 4; kk++)  // 32 bytes of K per MMA
                        mma_e<ESZ>(d, sdesc_kmajor_sw128(sA + s * A_ST, kk * 32),
                                   sdesc_kmajor_sw128(sB + s * C::B_ST, kk * 32), idesc, (kb | kk) ? 1u : 0u);
                    mma_commit(&bar->empty[s]);
                }
                if (ok) mma_commit(&bar->acc_full[b]);
            }
        }
    } else {
        const int q = warp & 3;  // TMEM lane quarter of this warp
        uint32_t it = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
            const uint32_t b = it & 1;
            if (!wait16(&bar->acc_full[b], (it >> 1) & 1, abort_flag)) break;
            tc_fence_after();
            const int64_t row = t * TM + q * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + b * C::ACS + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                if (row < m) {
                    float *p = Y + row * ldy + c0;
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        if (c0 + j < N) p[j] = (ts ? v[j] * ts[c0 + j] : v[j]) - (c ? c[c0 + j] : 0.f);
                }
            }
            tc_fence_before();
            mbar_arrive(&bar->acc_empty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TC);
    }
    if (threadIdx.x == 0 && bar->abort_flag) atomicOr(status, (int)ST_TIMEOUT);
}

// ======================================================================= TN
// Tile (chunk, column tile): D (128 columns of A x N) = sum over the chunk's rows
// of A[r][c] Q_i[r][j].  Stage layout: A as two MN atoms (columns c0..c0+63 and
// c0+64..c0+127) of 64 rows each; every Q_i as ceil(N/64) MN atoms of 64 rows.
template <int N, int NB, int ESZ>
struct TN16 {
    using E = Elt<ESZ>;
    static constexpr int NA = (N + E::QW - 1) / E::QW;  // MN atoms of one Q operand loaded by TMA
    // bfloat16: two atoms of room per operand up to N = 128, so the MMA's reads of one operand
    // stay inside its own 16 KB under either assignment of the two descriptor strides; wider
    // operands (N > 128, one term) take NA atoms at the atom stride the A operand already uses
    static constexpr uint32_t Q_ST = NA * E::ATOM > E::Q_ROOM ? NA * E::ATOM : E::Q_ROOM;
    // two accumulators of N float32 columns: 256 TMEM columns up to N = 128, 512 above
    static constexpr uint32_t ACS = N > 128 ? 256 : 128;
    static constexpr uint32_t TC = 2 * ACS;
    static constexpr uint32_t STAGE = A_ST + NB * Q_ST;
    static constexpr int S = cmin(8, (int)((200 * 1024) / STAGE));
    static constexpr uint32_t NEED = S * STAGE + 1024 + sizeof(Bars16<S>) + 64;
    static constexpr uint32_t SMEM = NEED > 120 * 1024 ? NEED : 120 * 1024;
};

template <int N, int NB, int ESZ>
__global__ void __launch_bounds__(THR, 1)
    tc16_tn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmQ1,
                   const __grid_constant__ CUtensorMap tmQ2, const __grid_constant__ CUtensorMap tmQ3, int64_t rows,
                   int ncols, int64_t rpc, int nchunks, float *__restrict__ part, int *__restrict__ status) {
    using C = TN16<N, NB, ESZ>;
    using E = Elt<ESZ>;
    constexpr int BK = E::TN_BK;
    constexpr int S = C::S;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    Bars16<S> *bar = reinterpret_cast<Bars16<S> *>(base + S * C::STAGE);
    volatile int *abort_flag = &bar->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntn = (ncols + TM - 1) / TM;
    const int64_t ntiles = (int64_t)ntn * nchunks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&bar->full[s], 1);
            mbar_init(&bar->empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bar->acc_full[b], 1);
            mbar_init(&bar->acc_empty[b], NEPI);
        }
        bar->abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&bar->tmem, C::TC);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bar->tmem;

    auto tile = [&](int64_t t, int64_t &r0, int64_t &r1, int &c0) {
        const int64_t chunk = t / ntn;
        c0 = (int)(t % ntn) * TM;
        r0 = chunk * rpc;
        r1 = r0 + rpc < rows ? r0 + rpc : rows;
    };

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmQ1);
            if (NB > 1) {
                tma_prefetch_desc(&tmQ2);
                tma_prefetch_desc(&tmQ3);
            }
            uint32_t g = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
                int64_t r0, r1;
                int c0;
                tile(t, r0, r1, c0);
                const int nkb = (int)((r1 - r0 + BK - 1) / BK);
                for (int kb = 0; kb < nkb; kb++, g++) {
                    const int s = g % S;
                    if (!(ok = wait16(&bar->empty[s], ((g / S) & 1) ^ 1, abort_flag))) break;
                    uint8_t *st = base + s * C::STAGE;
                    const int32_t y = (int32_t)(r0 + kb * BK);
                    // bytes the boxes below bring
                    mbar_arrive_expect_tx(&bar->full[s], (E::A_ATOMS + NB * C::NA) * E::ATOM);
#pragma unroll
                    for (int a = 0; a < E::A_ATOMS; a++)
                        tma_load_2d(st + a * E::ATOM, &tmA, c0 + a * E::QW, y, &bar->full[s]);
#pragma unroll
                    for (int i = 0; i < NB; i++) {
                        const CUtensorMap *mq = i == 0 ? &tmQ1 : i == 1 ? &tmQ2 : &tmQ3;
#pragma unroll
                        for (int a = 0; a < C::NA; a++)
                            tma_load_2d(st + A_ST + i * C::Q_ST + a * E::ATOM, mq, a * E::QW, y, &bar->full[s]);
                    }
                }
            }
            for (uint32_t k = g > (uint32_t)S ? g - S : 0; k < g; k++) mbar_wait(&bar->full[k % S], (k / S) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_e<ESZ>(TM, N, true, true);
            uint32_t g = 0, it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
                int64_t r0, r1;
                int c0;
                tile(t, r0, r1, c0);
                const int nkb = (int)((r1 - r0 + BK - 1) / BK);
                for (int k0 = 0; ok && k0 < nkb; k0 += SUBK, it++) {
                    const int k1 = k0 + SUBK < nkb ? k0 + SUBK : nkb;
                    const uint32_t b = it & 1;
                    if (!(ok = wait16(&bar->acc_empty[b], ((it >> 1) & 1) ^ 1, abort_flag))) break;
                    tc_fence_after();
                    const uint32_t d = tmem + b * C::ACS;
                    for (int kb = k0; kb < k1; kb++, g++) {
                        const int s = g % S;
                        if (!(ok = wait16(&bar->full[s], (g / S) & 1, abort_flag))) break;
                        tc_fence_after();
                        const uint8_t *st = base + s * C::STAGE;
#pragma unroll
                        for (int kk = 0; kk < BK / E::KMMA; kk++) {  // KMMA rows = KMMA / 8 K atoms of 1024 bytes
                            const uint32_t off = kk * E::KMMA * 128;
                            const uint64_t ad = sdesc_mn_sw128(st, off, E::LBO, 1024);
#pragma unroll
                            for (int i = 0; i < NB; i++)
                                mma_e<ESZ>(d, ad, sdesc_mn_sw128(st + A_ST + i * C::Q_ST, off, E::LBO, 1024), idesc,
                                           ((kb - k0) | kk | i) ? 1u : 0u);
                        }
                        mma_commit(&bar->empty[s]);
                    }
                    if (ok) mma_commit(&bar->acc_full[b]);
                }
            }
        }
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            int64_t r0, r1;
            int c0;
            tile(t, r0, r1, c0);
            const int nkb = (int)((r1 - r0 + BK - 1) / BK);
            const int64_t chunk = t / ntn;
            const int cc = c0 + q * 32 + lane;
            float acc[N];  // the tile's sum over its sub-chunks (IEEE float32 adds, fixed order)
            for (int k0 = 0; k0 < nkb; k0 += SUBK, it++) {
                const uint32_t b = it & 1;
                if (!(ok = wait16(&bar->acc_full[b], (it >> 1) & 1, abort_flag))) break;
                tc_fence_after();
#pragma unroll
                for (int j0 = 0; j0 < N; j0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + b * C::ACS + ((uint32_t)(q * 32) << 16) + (uint32_t)j0, v);
#pragma unroll
                    for (int j = 0; j < 16; j++) acc[j0 + j] = k0 > 0 ? acc[j0 + j] + v[j] : v[j];
                }
                tc_fence_before();
                mbar_arrive(&bar->acc_empty[b]);
            }
            if (ok && cc < ncols) {
                float *p = part + (chunk * ncols + cc) * (int64_t)N;
#pragma unroll
                for (int j = 0; j < N; j += 4)
                    *reinterpret_cast<float4 *>(p + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TC);
    }
    if (threadIdx.x == 0 && bar->abort_flag) atomicOr(status, (int)ST_TIMEOUT);
}

// out[c][j] = cs[c] qs[j] (sum over chunks, in order, of part[chunk][c][j]) - mu[c] qsum[j]
// (cs, qs, mu optional); one thread per (c, j)
__global__ void sum16_kernel(const float *__restrict__ part, int nchunks, int ncols, int N, float *__restrict__ out,
                             int64_t ldo, const float *__restrict__ cs, const float *__restrict__ qs,
                             const float *__restrict__ mu, const double *__restrict__ qsum) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ncols * N) return;
    const int c = (int)(idx / N), j = (int)(idx % N);
    double s = 0.0;
    for (int k = 0; k < nchunks; k++) s += (double)part[((int64_t)k * ncols + c) * N + j];
    if (cs) s *= (double)cs[c];
    if (qs) s *= (double)qs[j];
    if (mu) s -= (double)mu[c] * qsum[j];
    out[(int64_t)c * ldo + j] = (float)s;
}

int sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

struct Split16 {
    int64_t rpc;
    int chunks;
};

// Row chunks of A^T Q: at least two waves of (chunk, column tile) tiles, the count of
// chunks chosen (up to twice that) so the last wave is as full as possible; at least
// four stages per tile.
Split16 split16(int64_t rows, int ncols, int bk) {
    const int64_t ntn = ceil_div(ncols, TM), nsm = sms();
    const int64_t maxc = ceil_div(rows, 4 * bk);
    int64_t c0 = ceil_div(2 * nsm, ntn), chunks = c0;
    double best = -1.0;
    for (int64_t c = c0; c <= 2 * c0 && c <= maxc; c++) {
        const int64_t t = c * ntn;
        const double eff = (double)t / (double)(ceil_div(t, nsm) * nsm);
        if (eff > best + 1e-9) {
            best = eff;
            chunks = c;
        }
    }
    if (chunks > maxc) chunks = maxc;
    if (chunks < 1) chunks = 1;
    const int64_t rpc = round_up(ceil_div(rows, chunks), bk);
    return {rpc, (int)ceil_div(rows, rpc)};
}

template <int N, int ESZ>
cudaError_t launch16_nn(const CUtensorMap &a, const CUtensorMap &b, int64_t m, int n, float *Y, int64_t ldy,
                        const float *ts, const float *c, int *status, cudaStream_t s) {
    using C = NN16<N, ESZ>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tc16_nn_kernel<N, ESZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        attr = true;
    }
    const int64_t tiles = ceil_div(m, TM);
    const int grid = (int)(tiles < sms() ? tiles : sms());
    tc16_nn_kernel<N, ESZ><<<grid, THR, C::SMEM, s>>>(a, b, m, n, Y, ldy, ts, c, status);
    note_launch();
    return cudaGetLastError();
}

template <int N, int NB, int ESZ>
cudaError_t launch16_tn(const CUtensorMap &a, const CUtensorMap *q, int64_t rows, int ncols, Split16 sp, float *part,
                        int *status, cudaStream_t s) {
    using C = TN16<N, NB, ESZ>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tc16_tn_kernel<N, NB, ESZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        attr = true;
    }
    const int64_t tiles = ceil_div(ncols, TM) * sp.chunks;
    const int grid = (int)(tiles < sms() ? tiles : sms());
    tc16_tn_kernel<N, NB, ESZ><<<grid, THR, C::SMEM, s>>>(a, q[0], q[1], q[2], rows, ncols, sp.rpc, sp.chunks, part,
                                                           status);
    note_launch();
    return cudaGetLastError();
}

template <int ESZ>
cudaError_t gemm_nn_e(int64_t m, int n, int N, const void *A, int64_t lda, const void *Zt, int64_t ldz, float *Y,
                      int64_t ldy, const float *ts, const float *c, int *status, cudaStream_t s) {
    if (N > 256 && N % 16 == 0) {  // column slices of up to 256 (A read once per slice)
        const int k = (N + 255) / 256, w = ((N + k - 1) / k + 15) / 16 * 16;
        for (int c0 = 0; c0 < N; c0 += w) {
            const cudaError_t e =
                gemm_nn_e<ESZ>(m, n, w < N - c0 ? w : N - c0, A, lda, static_cast<const uint8_t *>(Zt) + c0 * ldz * ESZ,
                               ldz, Y + c0, ldy, ts ? ts + c0 : nullptr, c ? c + c0 : nullptr, status, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (N % 16 || N < 16 || N > 256) return cudaErrorInvalidValue;
    constexpr int BK = Elt<ESZ>::NN_BK;
    CUtensorMap ma, mb;
    if (!tc_make_map(&ma, A, ESZ, m, n, lda, TM, BK, true) || !tc_make_map(&mb, Zt, ESZ, N, n, ldz, N, BK, true))
        return cudaErrorInvalidValue;
    switch (N) {
        case 16: return launch16_nn<16, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 32: return launch16_nn<32, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 48: return launch16_nn<48, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 64: return launch16_nn<64, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 80: return launch16_nn<80, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 96: return launch16_nn<96, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 112: return launch16_nn<112, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 128: return launch16_nn<128, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 144: return launch16_nn<144, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 160: return launch16_nn<160, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 176: return launch16_nn<176, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 192: return launch16_nn<192, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 208: return launch16_nn<208, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 224: return launch16_nn<224, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 240: return launch16_nn<240, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
        case 256: return launch16_nn<256, ESZ>(ma, mb, m, n, Y, ldy, ts, c, status, s);
    }
    return cudaErrorInvalidValue;
}

template <int ESZ>
cudaError_t gemm_tn_e(int64_t rows, int ncols, int N, const void *A, int64_t lda, const void *const *Q, int nq,
                      int64_t ldq, float *C, int64_t ldc, float *part, int64_t part_elems, const float *cs,
                      const float *qs, const float *mu, const double *qsum, int *status, cudaStream_t s) {
    using E = Elt<ESZ>;
    // one bfloat16 term: up to 192 columns per launch (the epilogue holds N sums per thread)
    const int wmax = (ESZ == 2 && nq == 1) ? 192 : 128;
    if (N > wmax && N % 16 == 0) {  // column slices of the Q terms and C (A read once per slice)
        const int kq = (N + wmax - 1) / wmax, w = ((N + kq - 1) / kq + 15) / 16 * 16;
        for (int c0 = 0; c0 < N; c0 += w) {
            const void *qs_[3];
            for (int i = 0; i < nq && i < 3; i++) qs_[i] = static_cast<const uint8_t *>(Q[i]) + c0 * ESZ;
            const cudaError_t e = gemm_tn_e<ESZ>(rows, ncols, w < N - c0 ? w : N - c0, A, lda, qs_, nq, ldq, C + c0,
                                                 ldc, part, part_elems, cs, qs ? qs + c0 : nullptr, mu,
                                                 qsum ? qsum + c0 : nullptr, status, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (N % 16 || N < 16 || N > wmax || (nq != 1 && nq != 3) || (ESZ == 1 && nq != 1)) return cudaErrorInvalidValue;
    const Split16 sp = split16(rows, ncols, E::TN_BK);
    if (!part || part_elems < (int64_t)sp.chunks * ncols * N) return cudaErrorInvalidValue;
    CUtensorMap ma, mq[3];
    if (!tc_make_map(&ma, A, ESZ, rows, ncols, lda, E::TN_BK, E::QW, true)) return cudaErrorInvalidValue;
    for (int i = 0; i < 3; i++)
        if (!tc_make_map(&mq[i], Q[i < nq ? i : 0], ESZ, rows, N, ldq, E::TN_BK, E::QW, true))
            return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
#define TN16_CASE(NN)                                                                                   \
    case NN:                                                                                            \
        e = nq == 1 ? launch16_tn<NN, 1, ESZ>(ma, mq, rows, ncols, sp, part, status, s)                 \
                    : launch16_tn<NN, ESZ == 2 ? 3 : 1, ESZ>(ma, mq, rows, ncols, sp, part, status, s); \
        break;
    switch (N) {
        TN16_CASE(16)
        TN16_CASE(32)
        TN16_CASE(48)
        TN16_CASE(64)
        TN16_CASE(80)
        TN16_CASE(96)
        TN16_CASE(112)
        TN16_CASE(128)
    }
#undef TN16_CASE
    if constexpr (ESZ == 2) {  // one term, N > 128
        switch (N) {
            case 144: e = launch16_tn<144, 1, 2>(ma, mq, rows, ncols, sp, part, status, s); break;
            case 160: e = launch16_tn<160, 1, 2>(ma, mq, rows, ncols, sp, part, status, s); break;
            case 176: e = launch16_tn<176, 1, 2>(ma, mq, rows, ncols, sp, part, status, s); break;
            case 192: e = launch16_tn<192, 1, 2>(ma, mq, rows, ncols, sp, part, status, s); break;
        }
    }
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)ncols * N;
    sum16_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(part, sp.chunks, ncols, N, C, ldc, cs, qs, mu, qsum);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t tc16_gemm_nn(int64_t m, int n, int N, const void *A, int64_t lda, const void *Zt, int64_t ldz, float *Y,
                         int64_t ldy, const float *c, int *status, cudaStream_t s) {
    return gemm_nn_e<2>(m, n, N, A, lda, Zt, ldz, Y, ldy, nullptr, c, status, s);
}

cudaError_t tc8_gemm_nn(int64_t m, int n, int N, const void *A, int64_t lda, const void *Zt, int64_t ldz, float *Y,
                        int64_t ldy, const float *ts, const float *c, int *status, cudaStream_t s) {
    return gemm_nn_e<1>(m, n, N, A, lda, Zt, ldz, Y, ldy, ts, c, status, s);
}

int64_t tc16_gemm_tn_partials(int64_t rows, int ncols, int N) {
    const Split16 sp = split16(rows, ncols, Elt<2>::TN_BK);
    return (int64_t)sp.chunks * ncols * N;
}

int64_t tc8_gemm_tn_partials(int64_t rows, int ncols, int N) {
    const Split16 sp = split16(rows, ncols, Elt<1>::TN_BK);
    return (int64_t)sp.chunks * ncols * N;
}

cudaError_t tc16_gemm_tn(int64_t rows, int ncols, int N, const void *A, int64_t lda, const void *const *Q, int nq,
                         int64_t ldq, float *C, int64_t ldc, float *part, int64_t part_elems, const float *mu,
                         const double *qsum, int *status, cudaStream_t s, const float *cs) {
    return gemm_tn_e<2>(rows, ncols, N, A, lda, Q, nq, ldq, C, ldc, part, part_elems, cs, nullptr, mu, qsum, status,
                        s);
}

cudaError_t tc8_gemm_tn(int64_t rows, int ncols, int N, const void *A, int64_t lda, const void *Q, int64_t ldq,
                        float *C, int64_t ldc, float *part, int64_t part_elems, const float *cs, const float *qs,
                        const float *mu, const double *qsum, int *status, cudaStream_t s) {
    const void *q3[3] = {Q, Q, Q};
    return gemm_tn_e<1>(rows, ncols, N, A, lda, q3, 1, ldq, C, ldc, part, part_elems, cs, qs, mu, qsum, status, s);
}

}  // namespace gbr
