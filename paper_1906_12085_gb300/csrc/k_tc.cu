// Tensor-core (tcgen05) products for the float32 path with float32 accuracy.
//
// Each float32 value x of an operand is split into two tf32 values, x = hi + lo
// with hi = x with its low 13 mantissa bits cleared and lo = rn_tf32(x - hi);
// a product is accumulated as hi*hi + hi*lo + lo*hi in float32 in TMEM (lo*lo
// is below float32 resolution).
//
//   tc_gemm_nn : Y (m x N) = A (m x n) Z (n x N)            (sketch, power step, Q = Y R^-1)
//   tc_gemm_tn : part[chunk] = A[rows of chunk]^T Q[rows]   (power step, T = A^T Q, Gram)
//
// The tall operand A reaches shared memory by TMA, is split by the worker
// warps in registers and stored straight into tensor memory (tcgen05.st); the
// MMA reads A from TMEM and only the small operand (Z^T or Q^T, already split)
// from shared memory.  A TMEM lane is a row of the MMA's A operand, so the
// transposed product needs no shared-memory transpose of A: a worker thread
// reads one column of the raw A tile and stores it into its own lane.
//
// Both kernels are persistent (one CTA per SM) with warp roles:
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM owner and MMA issuer (one elected lane)
//   warps 2-9   split workers (256 threads; warp w serves TMEM lane quarter w % 4,
//               the two warps of a quarter take 16 K columns each)
//   warps 10-13 epilogue: TMEM -> registers -> HBM (one TMEM lane quarter each)
// TMEM holds two accumulators that alternate between tiles, so the epilogue of
// one tile overlaps the main loop of the next, and the A stages of hi and lo.
// For N <= 64 the two products with the hi part are one MMA of width 2N on the
// stacked small operand [B_hi; B_lo] (an MMA's cost grows much less than its width
// at these N: 23% less tensor time per stage, measured), the lo product a second
// MMA of width N into its own accumulator; the epilogue adds the three N-column
// blocks.  Every wait is bounded; a stalled pipeline sets ST_TIMEOUT in the status
// word and the CTA drains and exits.
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace gbr {
namespace {

using namespace tc;

constexpr int TM = 128;    // MMA M: rows of A (NN) or columns of A (TN) per tile
constexpr int TBK = 32;    // fp32 elements of K per stage (one 128-byte swizzle row)
constexpr int NSPLIT = 256;
constexpr int NEPI = 128;
constexpr int NTHR = 64 + NSPLIT + NEPI;
constexpr int EPI_WARP0 = (64 + NSPLIT) / 32;
constexpr uint32_t A_STAGE = TM * 128;  // bytes of one 128 x 32 fp32 stage
constexpr uint32_t TMEM_COLS = 512;
constexpr int TS = 4;                   // TMEM A stages at most

// TMEM layout for output width N: accumulator b at columns [ACC b, ACC b + width) with
// width N, or (MERGE) 2N for [hi B_hi | hi B_lo] followed by N for lo B_hi; the A stages
// after both accumulators, hi at A0 + 64 s and lo at A0 + 64 s + 32.
template <int N>
struct Tm {
    static constexpr bool MERGE = N <= 64;
    static constexpr uint32_t WIDTH = MERGE ? 3 * N : N;
    static constexpr uint32_t ACC = WIDTH <= 128 ? 128 : 192;
    static constexpr int NS = 2 * ACC + 4 * 64 <= TMEM_COLS ? 4 : 2;   // A stages
    static constexpr uint32_t A0 = 2 * ACC;
    // the split workers signal a stage after the work of the next one (hiding the TMEM
    // store latency) only when more than two stages exist
    static constexpr bool DELAY = NS >= 4;
};

__device__ __forceinline__ float rna_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void split4(const float *x, float4 &h, float4 &l) {
    h.x = rna_tf32(x[0]); l.x = rna_tf32(x[0] - h.x);
    h.y = rna_tf32(x[1]); l.y = rna_tf32(x[1] - h.y);
    h.z = rna_tf32(x[2]); l.z = rna_tf32(x[2] - h.z);
    h.w = rna_tf32(x[3]); l.w = rna_tf32(x[3] - h.w);
}

// truncating split for the A operand: hi keeps the tf32 bits, lo the exact rest rounded to tf32
__device__ __forceinline__ void split_tr(float x, uint32_t &h, uint32_t &l) {
    const uint32_t hb = __float_as_uint(x) & 0xFFFFE000u;
    h = hb;
    l = __float_as_uint(rna_tf32(x - __uint_as_float(hb)));
}

// byte offset of the 16-byte chunk `cc` (K position 4cc..4cc+3) of row `r` in
// the 128-byte-swizzled K-major layout (8-row atoms of 1024 bytes)
__device__ __forceinline__ uint32_t kmajor_off(int r, int cc) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((cc ^ (r & 7)) << 4));
}

// Shared barrier block placed after the stage buffers.
template <int S>
struct Bars {
    uint64_t full[S], split[S], empty[S];
    uint64_t tempty[TS];  // TMEM A stage free (NN)
    uint64_t acc_full[2], acc_empty[2];
    double ssq_w[NSPLIT / 32];
    uint32_t tmem;
    int abort_flag;
};

// Bounded wait that also honours the CTA-wide abort flag.
__device__ __forceinline__ bool wait_ok(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (*abort_flag) return false;
    if (mbar_wait(bar, parity)) return true;
    *abort_flag = 1;
    return false;
}

// The MMAs of one stage over its 4 K=8 slices, A in TMEM: D (+)= Ah Bh + Ah Bl + Al Bh
// (12 MMAs), or (MERGE; bl = bh + N rows) D[0, 2N) (+)= Ah [Bh; Bl] and D[2N, 3N) (+)= Al Bh
// (8 MMAs).
template <int N>
__device__ __forceinline__ void mma_stage(uint32_t d, uint32_t a_hi, uint32_t a_lo, const uint8_t *bh,
                                          const uint8_t *bl, bool first) {
    constexpr uint32_t idesc = idesc_tf32(TM, N);
#pragma unroll
    for (int kk = 0; kk < TBK / 8; kk++) {
        const uint32_t acc = (first && kk == 0) ? 0u : 1u;
        const uint64_t dbh = sdesc_kmajor_sw128(bh, kk * 32);
        if constexpr (Tm<N>::MERGE) {
            mma_tf32_ta(d, a_hi + kk * 8, dbh, idesc_tf32(TM, 2 * N), acc);
            mma_tf32_ta(d + 2 * N, a_lo + kk * 8, dbh, idesc, acc);
        } else {
            const uint64_t dbl = sdesc_kmajor_sw128(bl, kk * 32);
            mma_tf32_ta(d, a_hi + kk * 8, dbh, idesc, acc);
            mma_tf32_ta(d, a_hi + kk * 8, dbl, idesc, 1u);
            mma_tf32_ta(d, a_lo + kk * 8, dbh, idesc, 1u);
        }
    }
}

// Store a worker's 16 split values (K columns 16h..16h+15 of its lane) into TMEM stage s.
template <int N>
__device__ __forceinline__ void store_a(uint32_t tmem, int q, int h, int s, const uint32_t *hi, const uint32_t *lo) {
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const uint32_t col = Tm<N>::A0 + (uint32_t)s * 64 + (uint32_t)h * 16;
    tmem_st16(tmem + lane_base + col, hi);
    tmem_st16(tmem + lane_base + col + 32, lo);
}

// K steps (stages) accumulated in one TMEM accumulator before it is drained: the
// tensor core's float32 accumulation does not round to nearest, so its error grows
// with the number of accumulation steps; sub-chunks of SUBK stages (256 rows or
// columns of K) bound it, and the epilogue adds the sub-chunk results with IEEE
// float32 additions in a fixed order.
constexpr int SUBK = 8;

// Sub-chunk results summed in registers (N floats per epilogue thread; beyond 64 the
// 128-register budget of these 448-thread kernels spills part of them to local memory)
// and written once per tile.
template <int N>
__device__ __forceinline__ void sum_acc(uint32_t tmem, uint32_t b, int q, float *acc, bool first) {
    const uint32_t base = tmem + b * Tm<N>::ACC + ((uint32_t)(q * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        if constexpr (Tm<N>::MERGE) {  // hi B_hi + (hi B_lo + lo B_hi), two 16-column buffers live
            float w[16];
            tmem_ld16(base + (uint32_t)(N + c0), w);
            tmem_ld16(base + (uint32_t)(2 * N + c0), v);
#pragma unroll
            for (int j = 0; j < 16; j++) w[j] += v[j];
            tmem_ld16(base + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] += w[j];
        } else {
            tmem_ld16(base + (uint32_t)c0, v);
        }
#pragma unroll
        for (int j = 0; j < 16; j++) acc[c0 + j] = first ? v[j] : acc[c0 + j] + v[j];
    }
}

template <int N>
__device__ __forceinline__ void store_acc(const float *acc, float *dst, bool valid) {
    if (!valid) return;
    if ((N % 4) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < N; j += 4)
            *reinterpret_cast<float4 *>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < N; j++) dst[j] = acc[j];
    }
}

// ======================================================================= NN
template <int N>
struct NNCfg {
    static constexpr uint32_t B_STAGE = N * 128;
    static constexpr uint32_t STAGE = A_STAGE + 2 * B_STAGE;     // shared-memory stage: raw A + B hi/lo
    static constexpr int S = (200 * 1024) / STAGE > 6 ? 6 : (200 * 1024) / STAGE;
    // at least 120 KB so that only one CTA (which owns all 512 TMEM columns) fits on an SM
    static constexpr uint32_t SMEM_NEED = S * STAGE + 1024 + sizeof(Bars<S>) + 64;
    static constexpr uint32_t SMEM = SMEM_NEED > 120 * 1024 ? SMEM_NEED : 120 * 1024;
};

template <int N>
__global__ void __launch_bounds__(NTHR, 1)
    tc_nn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
                 const __grid_constant__ CUtensorMap tmBl, int64_t m, int n, float *__restrict__ Y, int64_t ldy,
                 int *__restrict__ status, const float *__restrict__ mu, double *__restrict__ ssq) {
    using C = NNCfg<N>;
    constexpr int S = C::S;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int NS = Tm<N>::NS;
    uint8_t *sA = base;                    // raw fp32 A stages (TMA, 128-byte swizzle)
    uint8_t *sB = sA + S * A_STAGE;        // per stage: B hi (N rows) then B lo (N rows)
    Bars<S> *bar = reinterpret_cast<Bars<S> *>(sB + S * 2 * C::B_STAGE);
    volatile int *abort_flag = &bar->abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (m + TM - 1) / TM;
    const int nkb = (n + TBK - 1) / TBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&bar->full[s], 1);
            mbar_init(&bar->empty[s], 1);
        }
        for (int t = 0; t < NS; t++) {
            mbar_init(&bar->split[t], NSPLIT);  // TMEM A stage t written
            mbar_init(&bar->tempty[t], 1);      // TMEM A stage t consumed by the MMAs
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bar->acc_full[b], 1);
            mbar_init(&bar->acc_empty[b], NEPI);
        }
        bar->abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&bar->tmem, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bar->tmem;

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmBh);
            tma_prefetch_desc(&tmBl);
            uint32_t g = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x)
                for (int kb = 0; kb < nkb; kb++, g++) {
                    const int s = g % S;
                    if (!(ok = wait_ok(&bar->empty[s], ((g / S) & 1) ^ 1, abort_flag))) break;
                    mbar_arrive_expect_tx(&bar->full[s], A_STAGE + 2 * C::B_STAGE);
                    tma_load_2d(sA + s * A_STAGE, &tmA, kb * TBK, (int32_t)(t * TM), &bar->full[s]);
                    tma_load_2d(sB + s * 2 * C::B_STAGE, &tmBh, kb * TBK, 0, &bar->full[s]);
                    tma_load_2d(sB + s * 2 * C::B_STAGE + C::B_STAGE, &tmBl, kb * TBK, 0, &bar->full[s]);
                }
            for (uint32_t k = g > (uint32_t)S ? g - S : 0; k < g; k++) mbar_wait(&bar->full[k % S], (k / S) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0, it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x)
                for (int k0 = 0; ok && k0 < nkb; k0 += SUBK, it++) {  // one accumulator per sub-chunk
                    const int k1 = k0 + SUBK < nkb ? k0 + SUBK : nkb;
                    const uint32_t b = it & 1;
                    if (!(ok = wait_ok(&bar->acc_empty[b], ((it >> 1) & 1) ^ 1, abort_flag))) break;
                    tc_fence_after();
                    const uint32_t d = tmem + b * Tm<N>::ACC;
                    for (int kb = k0; kb < k1; kb++, g++) {
                        const int s = g % S, ts = g % NS;
                        if (!(ok = wait_ok(&bar->split[ts], (g / NS) & 1, abort_flag))) break;
                        tc_fence_after();
                        const uint32_t a = tmem + Tm<N>::A0 + (uint32_t)ts * 64;
                        const uint8_t *bs = sB + s * 2 * C::B_STAGE;
                        mma_stage<N>(d, a, a + 32, bs, bs + C::B_STAGE, kb == k0);
                        mma_commit(&bar->empty[s]);
                        mma_commit(&bar->tempty[ts]);
                    }
                    if (ok) mma_commit(&bar->acc_full[b]);
                }
        }
    } else if (warp < EPI_WARP0) {
        // split workers; with `mu` the column means are subtracted on the fly (A itself
        // is never written), with `ssq` the squared centred entries of valid rows are summed
        // Stage g's TMEM stores are waited for (and the stage signalled) only after the
        // loads and split of stage g + 1, so the store latency overlaps useful work.
        const int q = warp & 3, h = (warp - 2) >> 2, r = q * 32 + lane;
        uint32_t g = 0;
        bool ok = true;
        int pend = -1;  // TMEM stage whose stores are still in flight
        double acc64 = 0.0;
        for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            const bool row_ok = t * TM + r < m;
            float acc32 = 0.f;
            for (int kb = 0; kb < nkb; kb++, g++) {
                const int s = g % S, ts = g % NS;
                if (!(ok = wait_ok(&bar->full[s], (g / S) & 1, abort_flag))) break;
                if (!(ok = wait_ok(&bar->tempty[ts], ((g / NS) & 1) ^ 1, abort_flag))) break;
                const uint8_t *raw = sA + s * A_STAGE;
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int c4 = 0; c4 < 4; c4++) {
                    float4 v = *reinterpret_cast<const float4 *>(raw + kmajor_off(r, h * 4 + c4));
                    if (mu) {
                        const float4 mv = __ldg(reinterpret_cast<const float4 *>(mu + kb * TBK + h * 16 + c4 * 4));
                        v.x -= mv.x; v.y -= mv.y; v.z -= mv.z; v.w -= mv.w;
                    }
                    if (ssq && row_ok) acc32 += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
                    split_tr(v.x, hi[c4 * 4 + 0], lo[c4 * 4 + 0]);
                    split_tr(v.y, hi[c4 * 4 + 1], lo[c4 * 4 + 1]);
                    split_tr(v.z, hi[c4 * 4 + 2], lo[c4 * 4 + 2]);
                    split_tr(v.w, hi[c4 * 4 + 3], lo[c4 * 4 + 3]);
                }
                if constexpr (Tm<N>::DELAY) {
                    if (pend >= 0) {
                        tmem_wait_st();
                        tc_fence_before();
                        mbar_arrive(&bar->split[pend]);
                    }
                    store_a<N>(tmem, q, h, ts, hi, lo);
                    pend = ts;
                } else {
                    store_a<N>(tmem, q, h, ts, hi, lo);
                    tmem_wait_st();
                    tc_fence_before();
                    mbar_arrive(&bar->split[ts]);
                }
            }
            acc64 += (double)acc32;
        }
        if (pend >= 0) {
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&bar->split[pend]);
        }
        if (ssq) {  // per-warp partials; combined after the final barrier
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc64 += __shfl_xor_sync(0xffffffffu, acc64, o);
            if (lane == 0) bar->ssq_w[warp - 2] = acc64;
        }
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            const int64_t row = t * TM + q * 32 + lane;
            float acc[N];
            for (int k0 = 0; k0 < nkb; k0 += SUBK, it++) {
                const uint32_t b = it & 1;
                if (!(ok = wait_ok(&bar->acc_full[b], (it >> 1) & 1, abort_flag))) break;
                tc_fence_after();
                sum_acc<N>(tmem, b, q, acc, k0 == 0);
                tc_fence_before();
                mbar_arrive(&bar->acc_empty[b]);
            }
            if (ok) store_acc<N>(acc, Y + row * ldy, row < m);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (threadIdx.x == 0) {
        if (bar->abort_flag) atomicOr(status, (int)ST_TIMEOUT);
        if (ssq) {
            double t = 0.0;
            for (int w = 0; w < NSPLIT / 32; w++) t += bar->ssq_w[w];
            ssq[blockIdx.x] = t;
        }
    }
}

// ======================================================================= TN
// Tile t = (chunk, column tile): D (128 columns of A x N) = sum over the chunk's
// rows r of A[r][c] Q[r][j].  Raw A and Q stages land unswizzled (row-major
// 32 x 128 and 32 x N).  A worker thread owns TMEM lane i = column i of the
// A tile and stores its split column there; Q is split and transposed into
// the K-major swizzled layout in shared memory (rows = column j of Q).
template <int N>
struct TNCfg {
    static constexpr uint32_t RAW_A = 32 * TM * 4;     // 16 KB
    static constexpr uint32_t RAW_Q = 32 * N * 4;
    static constexpr uint32_t RAW = RAW_A + RAW_Q;
    static constexpr uint32_t SPL_B = N * 128;
    static constexpr uint32_t SPL = 2 * SPL_B;
    static constexpr int SS = Tm<N>::NS;  // split stages (Q hi/lo in smem, A hi/lo in TMEM)
    static constexpr int SR = (208 * 1024 - SS * SPL) / RAW > 6 ? 6 : (208 * 1024 - SS * SPL) / RAW;
    static constexpr uint32_t SMEM_NEED = SR * RAW + SS * SPL + 1024 + sizeof(Bars<SR + SS>) + 64;
    static constexpr uint32_t SMEM = SMEM_NEED > 120 * 1024 ? SMEM_NEED : 120 * 1024;
};

template <int N>
__global__ void __launch_bounds__(NTHR, 1)
    tc_tn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmQ, int64_t rows,
                 int ncols, int64_t rpc, int nchunks, float *__restrict__ part, int *__restrict__ status,
                 const float *__restrict__ mu) {
    using C = TNCfg<N>;
    constexpr int SR = C::SR, SS = C::SS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sSplit = base;                 // SS x (Qhi, Qlo), 1024-aligned
    uint8_t *sRaw = base + SS * C::SPL;     // SR x (rawA, rawQ)
    // barrier roles: full[0..SR) raw landed, split[0..SS) split ready, empty[0..SR) raw free,
    // empty[SR..SR+SS) split stage free (MMA done)
    Bars<SR + SS> *bar = reinterpret_cast<Bars<SR + SS> *>(sRaw + SR * C::RAW);
    volatile int *abort_flag = &bar->abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntn = (ncols + TM - 1) / TM;
    const int64_t ntiles = (int64_t)ntn * nchunks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SR; s++) {
            mbar_init(&bar->full[s], 1);
            mbar_init(&bar->empty[s], NSPLIT);
        }
        for (int s = 0; s < SS; s++) {
            mbar_init(&bar->split[s], NSPLIT);
            mbar_init(&bar->empty[SR + s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bar->acc_full[b], 1);
            mbar_init(&bar->acc_empty[b], NEPI);
        }
        bar->abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&bar->tmem, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bar->tmem;

    auto tile_rows = [&](int64_t t, int64_t &r0, int64_t &r1, int &c0) {
        const int64_t chunk = t / ntn;
        c0 = (int)(t % ntn) * TM;
        r0 = chunk * rpc;
        r1 = r0 + rpc < rows ? r0 + rpc : rows;
    };

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmQ);
            uint32_t g = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
                int64_t r0, r1;
                int c0;
                tile_rows(t, r0, r1, c0);
                const int nkb = (int)((r1 - r0 + TBK - 1) / TBK);
                for (int kb = 0; kb < nkb; kb++, g++) {
                    const int s = g % SR;
                    if (!(ok = wait_ok(&bar->empty[s], ((g / SR) & 1) ^ 1, abort_flag))) break;
                    uint8_t *raw = sRaw + s * C::RAW;
                    mbar_arrive_expect_tx(&bar->full[s], C::RAW);
                    tma_load_2d(raw, &tmA, c0, (int32_t)(r0 + kb * TBK), &bar->full[s]);
                    tma_load_2d(raw + C::RAW_A, &tmQ, 0, (int32_t)(r0 + kb * TBK), &bar->full[s]);
                }
            }
            for (uint32_t k = g > (uint32_t)SR ? g - SR : 0; k < g; k++) mbar_wait(&bar->full[k % SR], (k / SR) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0, it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
                int64_t r0, r1;
                int c0;
                tile_rows(t, r0, r1, c0);
                const int nkb = (int)((r1 - r0 + TBK - 1) / TBK);
                for (int k0 = 0; ok && k0 < nkb; k0 += SUBK, it++) {  // one accumulator per sub-chunk
                    const int k1 = k0 + SUBK < nkb ? k0 + SUBK : nkb;
                    const uint32_t b = it & 1;
                    if (!(ok = wait_ok(&bar->acc_empty[b], ((it >> 1) & 1) ^ 1, abort_flag))) break;
                    tc_fence_after();
                    const uint32_t d = tmem + b * Tm<N>::ACC;
                    for (int kb = k0; kb < k1; kb++, g++) {
                        const int s = g % SS;
                        if (!(ok = wait_ok(&bar->split[s], (g / SS) & 1, abort_flag))) break;
                        tc_fence_after();
                        uint8_t *sp = sSplit + s * C::SPL;
                        const uint32_t a = tmem + Tm<N>::A0 + (uint32_t)s * 64;
                        mma_stage<N>(d, a, a + 32, sp, sp + C::SPL_B, kb == k0);
                        mma_commit(&bar->empty[SR + s]);
                    }
                    if (ok) mma_commit(&bar->acc_full[b]);
                }
            }
        }
    } else if (warp < EPI_WARP0) {
        // as in the NN kernel, stage g is signalled after the work of stage g + 1 (with four
        // split stages; with two, right after its own work)
        const int wt = threadIdx.x - 64;
        const int q = warp & 3, h = (warp - 2) >> 2, i = q * 32 + lane;
        uint32_t g = 0;
        bool ok = true;
        int pend_sr = -1, pend_ss = -1;
        for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            int64_t r0, r1;
            int c0;
            tile_rows(t, r0, r1, c0);
            const int nkb = (int)((r1 - r0 + TBK - 1) / TBK);
            for (int kb = 0; kb < nkb; kb++, g++) {
                const int sr = g % SR, ss = g % SS;
                if (!(ok = wait_ok(&bar->full[sr], (g / SR) & 1, abort_flag))) break;
                if (!(ok = wait_ok(&bar->empty[SR + ss], ((g / SS) & 1) ^ 1, abort_flag))) break;
                const float *rawA = reinterpret_cast<const float *>(sRaw + sr * C::RAW);
                const float *rawQ = reinterpret_cast<const float *>(sRaw + sr * C::RAW + C::RAW_A);
                uint8_t *sp = sSplit + ss * C::SPL;
                const int valid = (int)(r1 - (r0 + (int64_t)kb * TBK));  // rows of this stage inside the chunk
                {   // A column i, rows 16h..16h+15 -> TMEM lane i (column mean subtracted when given)
                    const float mc = mu ? __ldg(mu + c0 + i) : 0.f;
                    uint32_t hi[16], lo[16];
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const int k = h * 16 + e;
                        split_tr(k < valid ? rawA[k * TM + i] - mc : 0.f, hi[e], lo[e]);
                    }
                    if (Tm<N>::DELAY && pend_ss >= 0) {
                        fence_proxy_async_smem();
                        tmem_wait_st();
                        tc_fence_before();
                        mbar_arrive(&bar->empty[pend_sr]);   // raw stage consumed
                        mbar_arrive(&bar->split[pend_ss]);   // split stage ready
                    }
                    store_a<N>(tmem, q, h, ss, hi, lo);
                }
                for (int idx = wt; idx < N * 8; idx += NSPLIT) {  // Q: (column j, 4-row chunk cc)
                    const int j = idx % N, cc = idx / N;
                    float x[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) x[e] = rawQ[(cc * 4 + e) * N + j];
                    float4 hq, lq;
                    split4(x, hq, lq);
                    const uint32_t off = kmajor_off(j, cc);
                    *reinterpret_cast<float4 *>(sp + off) = hq;
                    *reinterpret_cast<float4 *>(sp + C::SPL_B + off) = lq;
                }
                if constexpr (Tm<N>::DELAY) {
                    pend_sr = sr;
                    pend_ss = ss;
                } else {
                    fence_proxy_async_smem();
                    tmem_wait_st();
                    tc_fence_before();
                    mbar_arrive(&bar->empty[sr]);
                    mbar_arrive(&bar->split[ss]);
                }
            }
        }
        if (pend_ss >= 0) {
            fence_proxy_async_smem();
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&bar->empty[pend_sr]);
            mbar_arrive(&bar->split[pend_ss]);
        }
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            int64_t r0, r1;
            int c0;
            tile_rows(t, r0, r1, c0);
            const int nkb = (int)((r1 - r0 + TBK - 1) / TBK);
            const int64_t chunk = t / ntn;
            const int c = c0 + q * 32 + lane;
            float *dst = part + (chunk * ncols + c) * (int64_t)N;
            float acc[N];
            for (int k0 = 0; k0 < nkb; k0 += SUBK, it++) {
                const uint32_t b = it & 1;
                if (!(ok = wait_ok(&bar->acc_full[b], (it >> 1) & 1, abort_flag))) break;
                tc_fence_after();
                sum_acc<N>(tmem, b, q, acc, k0 == 0);
                tc_fence_before();
                mbar_arrive(&bar->acc_empty[b]);
            }
            if (ok) store_acc<N>(acc, dst, c < ncols);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (threadIdx.x == 0 && bar->abort_flag) atomicOr(status, (int)ST_TIMEOUT);
}

// ======================================================================= TN, pre-split Q
// The same product with Q given as its transposed tf32 split (Q_hi, Q_lo: N x ldq rows of
// K = rows of A, tc_split_transpose): the small operand reaches shared memory by TMA in
// the K-major swizzled layout the MMA reads (hi rows then lo rows, as the NN kernel's B),
// and the split workers only split the A columns into TMEM.  Each raw stage holds 32
// rows of A (unswizzled 32 x 128) and the two Q tiles; it is freed when the MMAs that
// read it complete.
template <int N>
struct TN2Cfg {
    static constexpr uint32_t B_STAGE = N * 128;                   // one of Q hi / Q lo
    static constexpr uint32_t STAGE = A_STAGE + 2 * B_STAGE;
    static constexpr int S = (200 * 1024) / STAGE > 6 ? 6 : (200 * 1024) / STAGE;
    static constexpr uint32_t SMEM_NEED = S * STAGE + 1024 + sizeof(Bars<S>) + 64;
    static constexpr uint32_t SMEM = SMEM_NEED > 120 * 1024 ? SMEM_NEED : 120 * 1024;
};

template <int N>
__global__ void __launch_bounds__(NTHR, 1)
    tc_tn2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmQh,
                  const __grid_constant__ CUtensorMap tmQl, int64_t rows, int ncols, int64_t rpc, int nchunks,
                  float *__restrict__ part, int *__restrict__ status, const float *__restrict__ mu) {
    using C = TN2Cfg<N>;
    constexpr int S = C::S;
    constexpr int NS = Tm<N>::NS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = base;                          // per stage: Q hi (N rows) then Q lo (N rows), swizzled
    uint8_t *sA = sB + S * 2 * C::B_STAGE;       // raw A stages (32 x 128, unswizzled)
    Bars<S> *bar = reinterpret_cast<Bars<S> *>(sA + S * A_STAGE);
    volatile int *abort_flag = &bar->abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntn = (ncols + TM - 1) / TM;
    const int64_t ntiles = (int64_t)ntn * nchunks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&bar->full[s], 1);
            mbar_init(&bar->empty[s], 1);
        }
        for (int t = 0; t < NS; t++) {
            mbar_init(&bar->split[t], NSPLIT);
            mbar_init(&bar->tempty[t], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bar->acc_full[b], 1);
            mbar_init(&bar->acc_empty[b], NEPI);
        }
        bar->abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&bar->tmem, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bar->tmem;

    auto tile_rows = [&](int64_t t, int64_t &r0, int64_t &r1, int &c0) {
        const int64_t chunk = t / ntn;
        c0 = (int)(t % ntn) * TM;
        r0 = chunk * rpc;
        r1 = r0 + rpc < rows ? r0 + rpc : rows;
    };

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmQh);
            tma_prefetch_desc(&tmQl);
            uint32_t g = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
                int64_t r0, r1;
                int c0;
                tile_rows(t, r0, r1, c0);
                const int nkb = (int)((r1 - r0 + TBK - 1) / TBK);
                for (int kb = 0; kb < nkb; kb++, g++) {
                    const int s = g % S;
                    if (!(ok = wait_ok(&bar->empty[s], ((g / S) & 1) ^ 1, abort_flag))) break;
                    const int32_t k = (int32_t)(r0 + (int64_t)kb * TBK);
                    uint8_t *bs = sB + s * 2 * C::B_STAGE;
                    mbar_arrive_expect_tx(&bar->full[s], C::STAGE);
                    tma_load_2d(sA + s * A_STAGE, &tmA, c0, k, &bar->full[s]);
                    tma_load_2d(bs, &tmQh, k, 0, &bar->full[s]);
                    tma_load_2d(bs + C::B_STAGE, &tmQl, k, 0, &bar->full[s]);
                }
            }
            for (uint32_t k = g > (uint32_t)S ? g - S : 0; k < g; k++) mbar_wait(&bar->full[k % S], (k / S) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0, it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
                int64_t r0, r1;
                int c0;
                tile_rows(t, r0, r1, c0);
                const int nkb = (int)((r1 - r0 + TBK - 1) / TBK);
                for (int k0 = 0; ok && k0 < nkb; k0 += SUBK, it++) {  // one accumulator per sub-chunk
                    const int k1 = k0 + SUBK < nkb ? k0 + SUBK : nkb;
                    const uint32_t b = it & 1;
                    if (!(ok = wait_ok(&bar->acc_empty[b], ((it >> 1) & 1) ^ 1, abort_flag))) break;
                    tc_fence_after();
                    const uint32_t d = tmem + b * Tm<N>::ACC;
                    for (int kb = k0; kb < k1; kb++, g++) {
                        const int s = g % S, ts = g % NS;
                        if (!(ok = wait_ok(&bar->split[ts], (g / NS) & 1, abort_flag))) break;
                        tc_fence_after();
                        const uint32_t a = tmem + Tm<N>::A0 + (uint32_t)ts * 64;
                        const uint8_t *bs = sB + s * 2 * C::B_STAGE;
                        mma_stage<N>(d, a, a + 32, bs, bs + C::B_STAGE, kb == k0);
                        mma_commit(&bar->empty[s]);
                        mma_commit(&bar->tempty[ts]);
                    }
                    if (ok) mma_commit(&bar->acc_full[b]);
                }
            }
        }
    } else if (warp < EPI_WARP0) {
        // split workers: column i of the A tile, K rows 16h..16h+15 of the stage -> TMEM lane i
        const int q = warp & 3, h = (warp - 2) >> 2, i = q * 32 + lane;
        uint32_t g = 0;
        bool ok = true;
        int pend = -1;
        for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            int64_t r0, r1;
            int c0;
            tile_rows(t, r0, r1, c0);
            const int nkb = (int)((r1 - r0 + TBK - 1) / TBK);
            const float mc = mu ? __ldg(mu + c0 + i) : 0.f;
            for (int kb = 0; kb < nkb; kb++, g++) {
                const int s = g % S, ts = g % NS;
                if (!(ok = wait_ok(&bar->full[s], (g / S) & 1, abort_flag))) break;
                if (!(ok = wait_ok(&bar->tempty[ts], ((g / NS) & 1) ^ 1, abort_flag))) break;
                const float *rawA = reinterpret_cast<const float *>(sA + s * A_STAGE);
                const int valid = (int)(r1 - (r0 + (int64_t)kb * TBK));  // rows of this stage inside the chunk
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    const int k = h * 16 + e;
                    split_tr(k < valid ? rawA[k * TM + i] - mc : 0.f, hi[e], lo[e]);
                }
                if constexpr (Tm<N>::DELAY) {
                    if (pend >= 0) {
                        tmem_wait_st();
                        tc_fence_before();
                        mbar_arrive(&bar->split[pend]);
                    }
                    store_a<N>(tmem, q, h, ts, hi, lo);
                    pend = ts;
                } else {
                    store_a<N>(tmem, q, h, ts, hi, lo);
                    tmem_wait_st();
                    tc_fence_before();
                    mbar_arrive(&bar->split[ts]);
                }
            }
        }
        if (pend >= 0) {
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&bar->split[pend]);
        }
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            int64_t r0, r1;
            int c0;
            tile_rows(t, r0, r1, c0);
            const int nkb = (int)((r1 - r0 + TBK - 1) / TBK);
            const int64_t chunk = t / ntn;
            const int c = c0 + q * 32 + lane;
            float *dst = part + (chunk * ncols + c) * (int64_t)N;
            float acc[N];
            for (int k0 = 0; k0 < nkb; k0 += SUBK, it++) {
                const uint32_t b = it & 1;
                if (!(ok = wait_ok(&bar->acc_full[b], (it >> 1) & 1, abort_flag))) break;
                tc_fence_after();
                sum_acc<N>(tmem, b, q, acc, k0 == 0);
                tc_fence_before();
                mbar_arrive(&bar->acc_empty[b]);
            }
            if (ok) store_acc<N>(acc, dst, c < ncols);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (threadIdx.x == 0 && bar->abort_flag) atomicOr(status, (int)ST_TIMEOUT);
}

// ======================================================================= Gram, N <= 64
// G (N x N) = X^T X for a basis X (rows x N, N <= 64, row-major ld = N) in one pass over X:
// each 32-row stage of X is split once into tf32 hi / lo and written transposed into one
// K-major tile T = [X_hi^T; X_lo^T] (rows 0..63 hi, 64..127 lo; rows >= N of each half
// unused), and a single MMA of shape 128 x 128 x 8 per K slice computes T T^T, whose
// blocks are hi hi^T, hi lo^T, lo hi^T (lo lo^T, below float32 resolution, is discarded):
// 4 MMAs per stage with both operands in shared memory.  Each CTA reduces one chunk of
// rows; the epilogue adds the three blocks (the lo-hi block reaches the hi rows' threads
// through shared memory) and writes the chunk's partial Gram matrix.
constexpr uint32_t GR_TS = 128 * 128;   // bytes of one T tile (128 rows x 32 fp32, swizzled)
constexpr int GR_SR = 8, GR_ST = 4;

template <int N>
struct GramCfg {
    static constexpr uint32_t RAW = 32 * N * 4;
    static constexpr uint32_t SMEM = GR_ST * GR_TS + GR_SR * RAW + 64 * 65 * 4 + 1024 + sizeof(Bars<GR_SR + GR_ST>) + 64;
};

template <int N>
__global__ void __launch_bounds__(NTHR, 1)
    tc_gram_kernel(const __grid_constant__ CUtensorMap tmX, int64_t rows, int64_t rpc, float *__restrict__ part,
                   int *__restrict__ status) {
    static_assert(N <= 64 && N % 16 == 0, "Gram kernel: N <= 64");
    using C = GramCfg<N>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sT = base;                                  // GR_ST T tiles (1024-aligned)
    uint8_t *sRaw = sT + GR_ST * GR_TS;                  // GR_SR raw stages (32 x N, unswizzled)
    float *xch = reinterpret_cast<float *>(sRaw + GR_SR * C::RAW);  // xch[i][j] = lo_i . hi_j, rows of 65
    // barriers: full[0..SR) raw landed, empty[0..SR) raw read, split[0..ST) T written,
    // empty[SR..SR+ST) T consumed by the MMAs, tempty[0] xch written, tempty[1] xch read
    Bars<GR_SR + GR_ST> *bar = reinterpret_cast<Bars<GR_SR + GR_ST> *>(xch + 64 * 65);
    volatile int *abort_flag = &bar->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * rpc;
    const int64_t r1 = r0 + rpc < rows ? r0 + rpc : rows;
    const int nkb = r1 > r0 ? (int)((r1 - r0 + TBK - 1) / TBK) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GR_SR; s++) {
            mbar_init(&bar->full[s], 1);
            mbar_init(&bar->empty[s], NSPLIT);
        }
        for (int s = 0; s < GR_ST; s++) {
            mbar_init(&bar->split[s], NSPLIT);
            mbar_init(&bar->empty[GR_SR + s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bar->acc_full[b], 1);
            mbar_init(&bar->acc_empty[b], NEPI);
        }
        mbar_init(&bar->tempty[0], NEPI / 2);
        mbar_init(&bar->tempty[1], NEPI / 2);
        bar->abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&bar->tmem, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bar->tmem;

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch_desc(&tmX);
            bool ok = true;
            uint32_t g = 0;
            for (int kb = 0; kb < nkb; kb++, g++) {
                const int s = g % GR_SR;
                if (!(ok = wait_ok(&bar->empty[s], ((g / GR_SR) & 1) ^ 1, abort_flag))) break;
                mbar_arrive_expect_tx(&bar->full[s], C::RAW);
                tma_load_2d(sRaw + s * C::RAW, &tmX, 0, (int32_t)(r0 + (int64_t)kb * TBK), &bar->full[s]);
            }
            for (uint32_t k = g > (uint32_t)GR_SR ? g - GR_SR : 0; k < g; k++)
                mbar_wait(&bar->full[k % GR_SR], (k / GR_SR) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(128, 128);
            uint32_t g = 0, it = 0;
            bool ok = true;
            for (int k0 = 0; ok && k0 < nkb; k0 += SUBK, it++) {
                const int k1 = k0 + SUBK < nkb ? k0 + SUBK : nkb;
                const uint32_t b = it & 1;
                if (!(ok = wait_ok(&bar->acc_empty[b], ((it >> 1) & 1) ^ 1, abort_flag))) break;
                tc_fence_after();
                const uint32_t d = tmem + b * 128;
                for (int kb = k0; kb < k1; kb++, g++) {
                    const int st = g % GR_ST;
                    if (!(ok = wait_ok(&bar->split[st], (g / GR_ST) & 1, abort_flag))) break;
                    tc_fence_after();
                    const uint8_t *t = sT + st * GR_TS;
#pragma unroll
                    for (int kk = 0; kk < TBK / 8; kk++) {
                        const uint64_t desc = sdesc_kmajor_sw128(t, kk * 32);
                        mma_tf32(d, desc, desc, idesc, (kb == k0 && kk == 0) ? 0u : 1u);
                    }
                    mma_commit(&bar->empty[GR_SR + st]);
                }
                if (ok) mma_commit(&bar->acc_full[b]);
            }
        }
    } else if (warp < EPI_WARP0) {
        // worker t: column j = t % 64 of X, rows 8 kq .. 8 kq + 7 of the stage (kq = t / 64)
        const int t = threadIdx.x - 64, j = t & 63, kq = t >> 6;
        uint32_t g = 0;
        bool ok = true;
        for (int kb = 0; kb < nkb; kb++, g++) {
            const int sr = g % GR_SR, st = g % GR_ST;
            if (!(ok = wait_ok(&bar->full[sr], (g / GR_SR) & 1, abort_flag))) break;
            if (!(ok = wait_ok(&bar->empty[GR_SR + st], ((g / GR_ST) & 1) ^ 1, abort_flag))) break;
            if (j < N) {
                const float *raw = reinterpret_cast<const float *>(sRaw + sr * C::RAW);
                const int valid = (int)(r1 - (r0 + (int64_t)kb * TBK));  // rows of this stage in the chunk
                float x[8];
#pragma unroll
                for (int e = 0; e < 8; e++) x[e] = kq * 8 + e < valid ? raw[(kq * 8 + e) * N + j] : 0.f;
                float4 h0, l0, h1, l1;
                split4(x, h0, l0);
                split4(x + 4, h1, l1);
                uint8_t *tt = sT + st * GR_TS;
                *reinterpret_cast<float4 *>(tt + kmajor_off(j, 2 * kq)) = h0;
                *reinterpret_cast<float4 *>(tt + kmajor_off(j, 2 * kq + 1)) = h1;
                *reinterpret_cast<float4 *>(tt + kmajor_off(64 + j, 2 * kq)) = l0;
                *reinterpret_cast<float4 *>(tt + kmajor_off(64 + j, 2 * kq + 1)) = l1;
            }
            fence_proxy_async_smem();
            mbar_arrive(&bar->empty[sr]);   // raw stage read
            mbar_arrive(&bar->split[st]);   // T stage written
        }
    } else {
        // lanes 64..127 (quarters 2, 3) hold the lo rows: their block lo_i . hi_j reaches the
        // hi rows' threads through xch (guarded by two mbarriers, so every wait is bounded)
        const int q = warp & 3, i = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        uint32_t it = 0;
        bool ok = true;
        float acc[N];
        for (int k0 = 0; k0 < nkb; k0 += SUBK, it++) {
            const uint32_t b = it & 1;
            if (!(ok = wait_ok(&bar->acc_full[b], (it >> 1) & 1, abort_flag))) break;
            tc_fence_after();
            const uint32_t dcol = tmem + b * 128 + lane_base;
            if (q >= 2) {
                if (!(ok = wait_ok(&bar->tempty[1], (it & 1) ^ 1, abort_flag))) break;   // xch free
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += 16) {
                    float v[16];
                    tmem_ld16(dcol + (uint32_t)c0, v);
#pragma unroll
                    for (int e = 0; e < 16; e++) xch[(i - 64) * 65 + c0 + e] = v[e];
                }
                tc_fence_before();
                mbar_arrive(&bar->acc_empty[b]);
                mbar_arrive(&bar->tempty[0]);
            } else {
                if (!(ok = wait_ok(&bar->tempty[0], it & 1, abort_flag))) break;       // xch written
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += 16) {
                    float v[16], w[16];
                    tmem_ld16(dcol + (uint32_t)(64 + c0), w);   // hi_i . lo_j
#pragma unroll
                    for (int e = 0; e < 16; e++) w[e] += xch[i * 65 + c0 + e];   // + lo_i . hi_j
                    tmem_ld16(dcol + (uint32_t)c0, v);          // hi_i . hi_j
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const float sm = v[e] + w[e];
                        acc[c0 + e] = k0 == 0 ? sm : acc[c0 + e] + sm;
                    }
                }
                tc_fence_before();
                mbar_arrive(&bar->acc_empty[b]);
                mbar_arrive(&bar->tempty[1]);
            }
        }
        if (ok && q < 2 && i < N && nkb > 0) {
            float *dst = part + ((int64_t)blockIdx.x * N + i) * N;
#pragma unroll
            for (int jj = 0; jj < N; jj += 4)
                *reinterpret_cast<float4 *>(dst + jj) = make_float4(acc[jj], acc[jj + 1], acc[jj + 2], acc[jj + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
    if (threadIdx.x == 0 && bar->abort_flag) atomicOr(status, (int)ST_TIMEOUT);
}

// ==================================================================== helpers
// th / tl (N x ldt) = tf32 split of Z^T, Z rows x cols row-major (ldz); zero beyond.  A 32 x 32
// tile per CTA goes through shared memory, so both the reads (along j) and the writes (along r)
// are coalesced.
__global__ void __launch_bounds__(256) split_transpose_kernel(const float *__restrict__ Z, int64_t rows, int cols,
                                                              int64_t ldz, int N, float *__restrict__ th,
                                                              float *__restrict__ tl, int64_t ldt) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int64_t r = r0 + ty + 8 * k;
        const int j = j0 + tx;
        tile[ty + 8 * k][tx] = (r < rows && j < cols) ? Z[r * ldz + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int j = j0 + ty + 8 * k;
        const int64_t r = r0 + tx;
        if (j < N && r < ldt) {
            const float x = tile[tx][ty + 8 * k];
            const float h = rna_tf32(x);
            th[(int64_t)j * ldt + r] = h;
            tl[(int64_t)j * ldt + r] = rna_tf32(x - h);
        }
    }
}

// C[i * ldc + j] = sum_{s < chunks} part[s][i][j] (N x L per chunk).  A block covers 32
// consecutive outputs with 8 row groups taking interleaved chunks; the groups are
// combined in a fixed order, so the sum is deterministic.  With chk (C the Gram matrix Q^T Q
// of a basis of chk_l columns, this launch's columns starting at col0): ST_ORTH when an entry
// of its upper triangle differs from the identity's by more than tol.
__global__ void sum_chunks_kernel(const float *__restrict__ part, int64_t chunks, int64_t N, int64_t L,
                                  float *__restrict__ C, int64_t ldc, int *chk, int chk_l, int col0, float tol) {
    __shared__ float red[8][33];
    const int cx = threadIdx.x & 31, gy = threadIdx.x >> 5;
    const int64_t idx = (int64_t)blockIdx.x * 32 + cx;
    const int64_t stride = N * L;
    float s = 0.f;
    if (idx < stride)
        for (int64_t c = gy; c < chunks; c += 8) s += part[c * stride + idx];
    red[gy][cx] = s;
    __syncthreads();
    if (gy == 0 && idx < stride) {
        float t = red[0][cx];
        for (int g = 1; g < 8; g++) t += red[g][cx];
        C[(idx / L) * ldc + idx % L] = t;
        if (chk) {
            const int64_t i = idx / L, j = col0 + idx % L;
            if (i < chk_l && j < chk_l && j >= i && !(fabsf(t - (i == j ? 1.f : 0.f)) <= tol))
                atomicOr(chk, (int)ST_ORTH);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Row-major fp32 matrix rows x cols (leading dimension ld elements) as a TMA map
// with a box of box_rows x box_cols; swizzled (box_cols must be 32) or plain.
bool make_map(CUtensorMap *map, const float *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
              int box_cols, bool swizzle) {
    auto fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * 4) & 15)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

template <int N>
cudaError_t launch_nn(const CUtensorMap &a, const CUtensorMap &bh, const CUtensorMap &bl, int64_t m, int n, float *Y,
                      int64_t ldy, int *status, const float *mu, double *ssq, cudaStream_t s, int ctas) {
    using C = NNCfg<N>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tc_nn_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        attr = true;
    }
    const int grid = tc_gemm_nn_grid(m, ctas);
    tc_nn_kernel<N><<<grid, NTHR, C::SMEM, s>>>(a, bh, bl, m, n, Y, ldy, status, mu, ssq);
    note_launch();
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_tn(const CUtensorMap &a, const CUtensorMap &qm, int64_t rows, int ncols, int64_t rpc, int nchunks,
                      float *part, int *status, const float *mu, cudaStream_t s, int ctas) {
    using C = TNCfg<N>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tc_tn_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        attr = true;
    }
    const int64_t tiles = ceil_div(ncols, TM) * nchunks;
    const int64_t cap = ctas > 0 && ctas < num_sms() ? ctas : num_sms();
    const int grid = (int)(tiles < cap ? tiles : cap);
    tc_tn_kernel<N><<<grid, NTHR, C::SMEM, s>>>(a, qm, rows, ncols, rpc, nchunks, part, status, mu);
    note_launch();
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_tn2(const CUtensorMap &a, const CUtensorMap &qh, const CUtensorMap &ql, int64_t rows, int ncols,
                       int64_t rpc, int nchunks, float *part, int *status, const float *mu, cudaStream_t s, int ctas) {
    using C = TN2Cfg<N>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tc_tn2_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        attr = true;
    }
    const int64_t tiles = ceil_div(ncols, TM) * nchunks;
    const int64_t cap = ctas > 0 && ctas < num_sms() ? ctas : num_sms();
    const int grid = (int)(tiles < cap ? tiles : cap);
    tc_tn2_kernel<N><<<grid, NTHR, C::SMEM, s>>>(a, qh, ql, rows, ncols, rpc, nchunks, part, status, mu);
    note_launch();
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_gram(const CUtensorMap &x, int64_t rows, int64_t rpc, int nchunks, float *part, int *status,
                        cudaStream_t s) {
    using C = GramCfg<N>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tc_gram_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        attr = true;
    }
    tc_gram_kernel<N><<<nchunks, NTHR, C::SMEM, s>>>(x, rows, rpc, part, status);
    note_launch();
    return cudaGetLastError();
}

// Row chunks of the Gram kernel: one per CTA, at most one per SM, 32-row aligned.
struct GramSplit {
    int64_t rpc;
    int chunks;
};
GramSplit gram_split(int64_t rows) {
    const int64_t want = std::min<int64_t>(num_sms(), ceil_div(rows, TBK));
    const int64_t rpc = round_up(ceil_div(rows, want > 0 ? want : 1), TBK);
    return {rpc, (int)ceil_div(rows, rpc)};
}

struct TNSplit {
    int64_t rpc;
    int chunks;
};

// Row chunks of A^T Q: about 2 x SMs column-tile x chunk tiles, at least four stages
// per tile.  The split does not depend on the grid size, so a capped grid (tuning)
// computes every tile, and hence the result, exactly as the full one.
TNSplit tn_split(int64_t rows, int ncols) {
    const int64_t ntn = ceil_div(ncols, TM), nsm = num_sms();
    const int64_t maxc = ceil_div(rows, 4 * TBK);  // at least four stages per tile
    // at least two waves of tiles; the chunk count (up to twice that) that fills the last wave best
    const int64_t c0 = ceil_div(2 * nsm, ntn);
    int64_t chunks = c0;
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
    const int64_t rpc = round_up(ceil_div(rows, chunks), TBK);
    return {rpc, (int)ceil_div(rows, rpc)};
}

}  // namespace

bool tc_available() { return encode_fn() != nullptr; }

bool tc_make_map(CUtensorMap *map, const void *ptr, int esize, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                 int box_cols, bool swizzle) {
    auto fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * esize) & 15)) return false;
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, dt, 2, const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t tc_split_transpose(const float *Z, int64_t rows, int cols, int64_t ldz, int N, float *th, float *tl,
                               int64_t ldt, cudaStream_t s) {
    const dim3 grid((unsigned)ceil_div(ldt, 32), (unsigned)ceil_div(N, 32));
    split_transpose_kernel<<<grid, 256, 0, s>>>(Z, rows, cols, ldz, N, th, tl, ldt);
    note_launch();
    return cudaGetLastError();
}

int tc_gemm_nn_grid(int64_t m, int ctas) {
    const int64_t tiles = ceil_div(m, TM);
    const int64_t cap = ctas > 0 && ctas < num_sms() ? ctas : num_sms();
    return (int)(tiles < cap ? tiles : cap);
}

cudaError_t tc_gemm_nn(int64_t m, int n, int N, const float *A, int64_t lda, const float *Bth, const float *Btl,
                       int64_t ldb, float *Y, int64_t ldy, int *status, cudaStream_t s, const float *mu,
                       double *ssq, int ctas, bool upper_b) {
    if (N > 128 && N % 16 == 0) {  // column slices (A read once per slice)
        const int w = column_slice(N);
        for (int c0 = 0; c0 < N; c0 += w) {
            const int wn = w < N - c0 ? w : N - c0;
            const int kn = upper_b && c0 + wn < n ? c0 + wn : n;  // rows of a triangular B below the slice are zero
            const cudaError_t e = tc_gemm_nn(m, kn, wn, A, lda, Bth + c0 * ldb, Btl + c0 * ldb, ldb, Y + c0, ldy,
                                             status, s, mu, c0 == 0 ? ssq : nullptr, ctas);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (N % 16 || N < 16 || N > 128) return cudaErrorInvalidValue;
    if (mu && (reinterpret_cast<uintptr_t>(mu) & 15)) return cudaErrorInvalidValue;
    CUtensorMap ma, mbh, mbl;
    if (!make_map(&ma, A, m, n, lda, TM, TBK, true) || !make_map(&mbh, Bth, N, n, ldb, N, TBK, true) ||
        !make_map(&mbl, Btl, N, n, ldb, N, TBK, true))
        return cudaErrorInvalidValue;
    switch (N) {
        case 16: return launch_nn<16>(ma, mbh, mbl, m, n, Y, ldy, status, mu, ssq, s, ctas);
        case 32: return launch_nn<32>(ma, mbh, mbl, m, n, Y, ldy, status, mu, ssq, s, ctas);
        case 48: return launch_nn<48>(ma, mbh, mbl, m, n, Y, ldy, status, mu, ssq, s, ctas);
        case 64: return launch_nn<64>(ma, mbh, mbl, m, n, Y, ldy, status, mu, ssq, s, ctas);
        case 80: return launch_nn<80>(ma, mbh, mbl, m, n, Y, ldy, status, mu, ssq, s, ctas);
        case 96: return launch_nn<96>(ma, mbh, mbl, m, n, Y, ldy, status, mu, ssq, s, ctas);
        case 112: return launch_nn<112>(ma, mbh, mbl, m, n, Y, ldy, status, mu, ssq, s, ctas);
        case 128: return launch_nn<128>(ma, mbh, mbl, m, n, Y, ldy, status, mu, ssq, s, ctas);
    }
    return cudaErrorInvalidValue;
}

int64_t tc_gram_partials(int64_t rows, int N) { return (int64_t)gram_split(rows).chunks * N * N; }

cudaError_t tc_gram(int64_t rows, int N, const float *X, int64_t ldx, float *C, int64_t ldc, float *part,
                    int64_t part_elems, int *status, cudaStream_t s, int *chk, int chk_l, double chk_tol) {
    if (N % 16 || N < 16 || N > 64 || rows < 1) return cudaErrorInvalidValue;
    const GramSplit sp = gram_split(rows);
    if (part == nullptr || part_elems < (int64_t)sp.chunks * N * N) return cudaErrorInvalidValue;
    CUtensorMap mx;
    if (!make_map(&mx, X, rows, N, ldx, TBK, N, false)) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    switch (N) {
        case 16: e = launch_gram<16>(mx, rows, sp.rpc, sp.chunks, part, status, s); break;
        case 32: e = launch_gram<32>(mx, rows, sp.rpc, sp.chunks, part, status, s); break;
        case 48: e = launch_gram<48>(mx, rows, sp.rpc, sp.chunks, part, status, s); break;
        case 64: e = launch_gram<64>(mx, rows, sp.rpc, sp.chunks, part, status, s); break;
    }
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)N * N;
    sum_chunks_kernel<<<(unsigned)ceil_div(total, 32), 256, 0, s>>>(part, sp.chunks, N, N, C, ldc, chk, chk_l, 0,
                                                                     (float)chk_tol);
    note_launch();
    return cudaGetLastError();
}

int64_t tc_gemm_tn_partials(int64_t rows, int ncols, int N) {
    const TNSplit sp = tn_split(rows, ncols);
    return (int64_t)sp.chunks * ncols * N;
}

cudaError_t tc_gemm_tn(int64_t rows, int ncols, int N, const float *A, int64_t lda, const float *Q, int64_t ldq,
                       float *C, int64_t ldc, float *part, int64_t part_elems, int *status, cudaStream_t s,
                       const float *mu, int ctas, bool upper_c, int *chk, int chk_l, double chk_tol, int col0,
                       const float *Qth, const float *Qtl, int64_t ldqt) {
    if (N > 128 && N % 16 == 0) {  // column slices of Q and C (A read once per slice)
        const int w = column_slice(N);
        for (int c0 = 0; c0 < N; c0 += w) {
            const int wn = w < N - c0 ? w : N - c0;
            const int nc = upper_c && c0 + wn < ncols ? c0 + wn : ncols;  // upper triangle: rows up to the slice end
            const cudaError_t e =
                tc_gemm_tn(rows, nc, wn, A, lda, Q + c0, ldq, C + c0, ldc, part, part_elems, status, s, mu, ctas,
                           false, chk, chk_l, chk_tol, col0 + c0, Qth ? Qth + c0 * ldqt : nullptr,
                           Qtl ? Qtl + c0 * ldqt : nullptr, ldqt);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (N % 16 || N < 16 || N > 128) return cudaErrorInvalidValue;
    const TNSplit sp = tn_split(rows, ncols);
    if (part == nullptr || part_elems < (int64_t)sp.chunks * ncols * N) return cudaErrorInvalidValue;
    CUtensorMap ma, mq, mqh, mql;
    if (!make_map(&ma, A, rows, ncols, lda, TBK, TM, false)) return cudaErrorInvalidValue;
    const bool pre = Qth && Qtl && make_map(&mqh, Qth, N, rows, ldqt, N, TBK, true) &&
                     make_map(&mql, Qtl, N, rows, ldqt, N, TBK, true);
    if (!pre && !make_map(&mq, Q, rows, N, ldq, TBK, N, false)) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    if (pre) {
        switch (N) {
            case 16: e = launch_tn2<16>(ma, mqh, mql, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
            case 32: e = launch_tn2<32>(ma, mqh, mql, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
            case 48: e = launch_tn2<48>(ma, mqh, mql, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
            case 64: e = launch_tn2<64>(ma, mqh, mql, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
            case 80: e = launch_tn2<80>(ma, mqh, mql, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
            case 96: e = launch_tn2<96>(ma, mqh, mql, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
            case 112: e = launch_tn2<112>(ma, mqh, mql, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
            case 128: e = launch_tn2<128>(ma, mqh, mql, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
        }
    } else switch (N) {
        case 16: e = launch_tn<16>(ma, mq, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
        case 32: e = launch_tn<32>(ma, mq, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
        case 48: e = launch_tn<48>(ma, mq, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
        case 64: e = launch_tn<64>(ma, mq, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
        case 80: e = launch_tn<80>(ma, mq, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
        case 96: e = launch_tn<96>(ma, mq, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
        case 112: e = launch_tn<112>(ma, mq, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
        case 128: e = launch_tn<128>(ma, mq, rows, ncols, sp.rpc, sp.chunks, part, status, mu, s, ctas); break;
    }
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)ncols * N;
    sum_chunks_kernel<<<(unsigned)ceil_div(total, 32), 256, 0, s>>>(part, sp.chunks, ncols, N, C, ldc, chk, chk_l,
                                                                     col0, (float)chk_tol);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gbr
