// Storage formats of the precision form: float32 A -> bfloat16 or OCP e4m3
// with per-column scales (round to nearest even; e4m3 saturating at 448).
//   bfloat16 : one conversion per element (cvt.rn.bf16x2.f32).
//   e4m3     : amax_j over each column (one read of A), s_j = amax_j / 448 in
//              float32 (1 for an all-zero column), then the e4m3 code of the
//              float32 quotient a / s_j (cvt.rn.satfinite.e4m3x2.f32; a second
//              read of A).  Both roundings are IEEE, so the codes are a
//              function of the input bits alone.
#include "common.cuh"

namespace gbr {
namespace {

// per-column max |a| (float bits of non-negative floats order like unsigned ints)
__global__ void colamax_kernel(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda, int64_t rpb,
                               unsigned *__restrict__ amax) {
    __shared__ float red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * 32 + tx;
    const int64_t r0 = (int64_t)blockIdx.y * rpb, r1 = min(m, r0 + rpb);
    float mx = 0.f;
    if (c < n)
        for (int64_t r = r0 + ty; r < r1; r += 8) mx = fmaxf(mx, fabsf(A[r * lda + c]));
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && c < n) {
        for (int k = 1; k < 8; k++) mx = fmaxf(mx, red[k][tx]);
        atomicMax(amax + c, __float_as_uint(mx));
    }
}

// in place: amax bits -> scale s_j = amax_j / 448 (IEEE division), 1 for a zero column
__global__ void scales_kernel(float *__restrict__ s, int64_t n) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float a = __uint_as_float(reinterpret_cast<unsigned *>(s)[j]);
    s[j] = a > 0.f ? __fdiv_rn(a, 448.f) : 1.f;
}

__device__ __forceinline__ unsigned short e4m3x2(float hi, float lo) {
    unsigned short d;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
    return d;  // hi in the upper byte, lo in the lower byte
}

__device__ __forceinline__ unsigned bf16x2(float hi, float lo) {
    unsigned d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// one thread per pair of consecutive elements of a row (n even) or per element
template <bool E4M3>
__global__ void quant_kernel(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                             const float *__restrict__ s, void *__restrict__ out) {
    const int64_t half = (n + 1) / 2;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * half) return;
    const int64_t r = idx / half, c = 2 * (idx % half);
    const float a0 = A[r * lda + c];
    const bool two = c + 1 < n;
    const float a1 = two ? A[r * lda + c + 1] : 0.f;
    if constexpr (E4M3) {
        const unsigned short d = e4m3x2(__fdiv_rn(a1, two ? s[c + 1] : 1.f), __fdiv_rn(a0, s[c]));
        unsigned char *o = static_cast<unsigned char *>(out) + r * n + c;
        o[0] = (unsigned char)(d & 0xFF);
        if (two) o[1] = (unsigned char)(d >> 8);
    } else {
        const unsigned d = bf16x2(a1, a0);
        unsigned short *o = static_cast<unsigned short *>(out) + r * n + c;
        o[0] = (unsigned short)(d & 0xFFFF);
        if (two) o[1] = (unsigned short)(d >> 16);
    }
}

}  // namespace

cudaError_t quantize(const float *A, int64_t m, int64_t n, int64_t lda, bool e4m3, void *out, float *scales,
                     cudaStream_t s) {
    if (e4m3) {
        if (cudaMemsetAsync(scales, 0, sizeof(float) * n, s) != cudaSuccess) return cudaErrorUnknown;
        const int64_t cb = ceil_div(n, 32);
        int64_t rb = ceil_div(4 * 152, cb);
        if (rb < 1) rb = 1;
        const int64_t rpb = round_up(ceil_div(m, rb), 8);
        colamax_kernel<<<dim3((unsigned)cb, (unsigned)ceil_div(m, rpb)), 256, 0, s>>>(
            A, m, n, lda, rpb, reinterpret_cast<unsigned *>(scales));
        scales_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(scales, n);
        note_launch(2);
    }
    const int64_t total = m * ((n + 1) / 2);
    if (e4m3) quant_kernel<true><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(A, m, n, lda, scales, out);
    else quant_kernel<false><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(A, m, n, lda, nullptr, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gbr

extern "C" rsvd_status rsvd_quantize(const float *A, int64_t m, int64_t n, int64_t lda, rsvd_dtype dtype, void *Aq,
                                     float *col_scales, void *cuda_stream) {
    if (!A || !Aq || m < 1 || n < 1 || lda < n) return RSVD_ERR_ARG;
    if (dtype != RSVD_BF16 && dtype != RSVD_FP8_E4M3) return RSVD_ERR_UNSUPPORTED;
    if (dtype == RSVD_FP8_E4M3 && !col_scales) return RSVD_ERR_ARG;
    if (gbr::ceil_div(m * ((n + 1) / 2), 256) > 0x7FFFFFFFLL) return RSVD_ERR_UNSUPPORTED;
    const cudaError_t e = gbr::quantize(A, m, n, lda, dtype == RSVD_FP8_E4M3, Aq, col_scales,
                                        (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}
