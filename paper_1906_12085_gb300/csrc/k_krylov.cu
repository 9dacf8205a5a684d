// Small kernels of the block Krylov method (Sec. 3.1.1) beyond those it shares
// with the randomized one: the coefficient matrix of a block Gram-Schmidt
// projection, the scaling of a block's Gram eigen-decomposition (SVQB) and the
// random refill of the directions a block has lost.
#include <math.h>

#include "common.cuh"

namespace gbr {
namespace {

// B (rows 0..jl-1) = -C in place; B (rows jl..jl+l-1) = [I_l 0]; ld lp.
template <typename T>
__global__ void bk_proj_matrix_kernel(T *__restrict__ B, int jl, int l, int lp) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)(jl + l) * lp) return;
    const int r = (int)(idx / lp), c = (int)(idx % lp);
    if (r < jl) B[idx] = -B[idx];
    else B[idx] = (c == r - jl) ? T(1) : T(0);
}

// lam descending (l doubles), V column i = eigenvector i (l x l, ld l).  A column
// c < l is kept when lam_c > tau * lam_0 (and lam_0 > 0): M[:, c] = V[:, c] /
// sqrt(lam_c); otherwise M[:, c] = 0 and flag[c] = 1.  M is lp x lp (ld lp), zero
// outside the leading l x l block; flag[c] = 0 for c >= l.
template <typename T>
__global__ void svqb_scale_kernel(const double *__restrict__ lam, const double *__restrict__ V, int l, int lp,
                                  double tau, T *__restrict__ M, int *__restrict__ flag) {
    const double l0 = lam[0];
    for (int idx = threadIdx.x; idx < lp * lp; idx += blockDim.x) {
        const int r = idx / lp, c = idx % lp;
        const bool keep = c < l && l0 > 0.0 && lam[c] > tau * l0;
        M[idx] = (keep && r < l) ? (T)(V[r * l + c] / sqrt(lam[c])) : T(0);
        if (r == 0) flag[c] = (c < l && !keep) ? 1 : 0;
    }
}

// X[r, c] = scale * (2 u - 1), u uniform in [0, 1) from counter r * lp + c, for
// the flagged columns c < l of X (m x lp, ld lp).
template <typename T>
__global__ void bk_fill_kernel(T *__restrict__ X, int64_t m, int l, int lp, const int *__restrict__ flag,
                               uint64_t seed, double scale) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * lp) return;
    const int c = (int)(idx % lp);
    if (c >= l || !flag[c]) return;
    const double u = (double)(splitmix64(seed, (uint64_t)idx) >> 11) * 0x1.0p-53;
    X[idx] = (T)(scale * (2.0 * u - 1.0));
}

}  // namespace

template <typename T>
cudaError_t bk_proj_matrix(T *B, int jl, int l, int lp, cudaStream_t s) {
    const int64_t total = (int64_t)(jl + l) * lp;
    if (total <= 0) return cudaSuccess;
    bk_proj_matrix_kernel<T><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(B, jl, l, lp);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t svqb_scale(const double *lam, const double *V, int l, int lp, double tau, T *M, int *flag,
                       cudaStream_t s) {
    svqb_scale_kernel<T><<<1, 256, 0, s>>>(lam, V, l, lp, tau, M, flag);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t bk_fill(T *X, int64_t m, int l, int lp, const int *flag, uint64_t seed, cudaStream_t s) {
    const int64_t total = m * lp;
    if (total <= 0) return cudaSuccess;
    // columns of unit expected norm: E[(2u - 1)^2] = 1/3
    const double scale = sqrt(3.0 / (double)m);
    bk_fill_kernel<T><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(X, m, l, lp, flag, seed, scale);
    note_launch();
    return cudaGetLastError();
}

#define INST_BK(T)                                                                                          \
    template cudaError_t bk_proj_matrix<T>(T *, int, int, int, cudaStream_t);                               \
    template cudaError_t svqb_scale<T>(const double *, const double *, int, int, double, T *, int *,        \
                                       cudaStream_t);                                                       \
    template cudaError_t bk_fill<T>(T *, int64_t, int, int, const int *, uint64_t, cudaStream_t);
INST_BK(float)
INST_BK(double)

}  // namespace gbr
