// Float64 SVD of the small factor R = U_R Sigma W^T (the SVD of B, Sec. 3.1.2 step 6)
// from a float32 start.  The float32 one-sided Jacobi supplies U_R and W (orthonormal and
// diagonalising to ~1e-6); a Newton-type iteration built only from l x l float64
// products -- the refinement of Ogita and Aishima (iterative refinement for the singular
// value decomposition based on matrix multiplication, J. Comput. Appl. Math., 2020) --
// then corrects them.  One step:
//   P = U^T U,  Q = W^T W,  T = U^T R W,   s_i = 2 T_ii / (P_ii + Q_ii),
//   U <- U (I + F),  W <- W (I + G),
// where F + F^T = I - P and G + G^T = I - Q restore orthonormality to first order and,
// for i != j, the pair (F_ij, G_ij) removes the off-diagonal T_ij, T_ji to first order:
//   -s_j F_ij + s_i G_ij = a_ij = -T_ij - (I - P)_ij s_j
//    s_i F_ij - s_j G_ij = b_ij = -T_ji - (I - Q)_ij s_j.
// Every step squares the relative off-diagonal size of the last one, so two steps take a
// float32 start to float64 accuracy.  The 2 x 2 system is solved only for pairs whose
// magnitudes differ by more than 4 max(|a_ij|, |b_ij|) (which keeps |F_ij|, |G_ij| below
// ~1/4) and by more than the rounding level 4 l u s_max.  Closer pairs form a cluster:
// F_ij = (I - P)_ij / 2 and G_ij from the first equation alone, which turns W into
// alignment with U inside the cluster.  Values below 1e-5 s_max -- beneath the float32
// accuracy of T = A^T Q that R factors -- are only re-orthonormalised and keep the
// float32 start's absolute accuracy.
#include <cfloat>

#include "common.cuh"

namespace gbr {
namespace {

constexpr int RT = 16;                     // output tile edge of the float64 products
constexpr double kTinyRel = 1e-5;          // values below kTinyRel s_max are not refined
constexpr int kRefineSteps = 2;

struct Prod64 {
    const double *A, *B, *D;
    double *C;
    int ta;
};
struct Prod64Set {
    Prod64 p[3];
};

// C = D + op(A) B for l x l row-major matrices (op(A) = A^T when ta; D may be null),
// one 16 x 16 tile of C per CTA, product blockIdx.z of the set.
__global__ void __launch_bounds__(RT *RT) prod64_kernel(Prod64Set set, int l) {
    __shared__ double as[RT][RT + 1];  // as[i][k] = op(A)(row0 + i, k0 + k)
    __shared__ double bs[RT][RT + 1];  // bs[k][j] = B(k0 + k, col0 + j)
    const Prod64 pr = set.p[blockIdx.z];
    const int tx = threadIdx.x % RT, ty = threadIdx.x / RT;
    const int row0 = blockIdx.y * RT, col0 = blockIdx.x * RT;
    double acc = 0.0;
    for (int k0 = 0; k0 < l; k0 += RT) {
        if (pr.ta) {  // op(A)(row0 + tx, k0 + ty) = A[k0 + ty][row0 + tx]: coalesced in tx
            const int ak = k0 + ty, ar = row0 + tx;
            as[tx][ty] = (ak < l && ar < l) ? pr.A[(int64_t)ak * l + ar] : 0.0;
        } else {
            const int ar = row0 + ty, ak = k0 + tx;
            as[ty][tx] = (ak < l && ar < l) ? pr.A[(int64_t)ar * l + ak] : 0.0;
        }
        {
            const int bk = k0 + ty, bc = col0 + tx;
            bs[ty][tx] = (bk < l && bc < l) ? pr.B[(int64_t)bk * l + bc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RT; k++) acc = fma(as[ty][k], bs[k][tx], acc);
        __syncthreads();
    }
    const int r = row0 + ty, c = col0 + tx;
    if (r < l && c < l) pr.C[(int64_t)r * l + c] = (pr.D ? pr.D[(int64_t)r * l + c] : 0.0) + acc;
}

// U = U_R, W = W (float32, lp x lp) widened to l x l float64
__global__ void refine_load_kernel(const float *__restrict__ UR, const float *__restrict__ Wf, int l, int lp,
                                   double *__restrict__ U, double *__restrict__ W) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < l * l; idx += gridDim.x * blockDim.x) {
        const int i = idx / l, o = idx % l;
        U[idx] = (double)UR[(int64_t)i * lp + o];
        W[idx] = (double)Wf[(int64_t)i * lp + o];
    }
}

__device__ __forceinline__ double sv_est(const double *P, const double *Q, const double *T, int l, int i) {
    const int64_t d = (int64_t)i * l + i;
    return 2.0 * T[d] / (P[d] + Q[d]);
}

// F, G of one refinement step; sig (the current estimates s_i) written by the diagonal.
__global__ void __launch_bounds__(256) refine_step_kernel(const double *__restrict__ P, const double *__restrict__ Q,
                                                          const double *__restrict__ T, int l, double *__restrict__ F,
                                                          double *__restrict__ G, double *__restrict__ sig) {
    __shared__ double red[8];
    double mx = 0.0;
    for (int i = threadIdx.x; i < l; i += blockDim.x) mx = fmax(mx, fabs(sv_est(P, Q, T, l, i)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    double smax = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) smax = fmax(smax, red[w]);
    const double tau = kTinyRel * smax, rnd = 4.0 * l * (0.5 * DBL_EPSILON) * smax;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < l * l; idx += gridDim.x * blockDim.x) {
        const int i = idx / l, j = idx % l;
        const double si = sv_est(P, Q, T, l, i);
        if (i == j) {
            F[idx] = 0.5 * (1.0 - P[idx]);
            G[idx] = 0.5 * (1.0 - Q[idx]);
            sig[i] = si;
            continue;
        }
        const double sj = sv_est(P, Q, T, l, j);
        const double ru = -P[idx], sv = -Q[idx];  // (I - P)_ij, (I - Q)_ij
        const double tij = T[idx], tji = T[(int64_t)j * l + i];
        const double a = -tij - ru * sj, b = -tji - sv * sj;
        const bool tiny_i = fabs(si) <= tau, tiny_j = fabs(sj) <= tau;
        const bool clus = (tiny_i && tiny_j) || fabs(fabs(si) - fabs(sj)) <= fmax(4.0 * fmax(fabs(a), fabs(b)), rnd);
        double f, g;
        if (!clus) {
            const double det = sj * sj - si * si;
            f = (-sj * a - si * b) / det;
            g = (-si * a - sj * b) / det;
        } else {
            f = 0.5 * ru;
            g = (tiny_i || tiny_j) ? 0.5 * sv : (-tij - 0.5 * ru * sj) / si;
        }
        F[idx] = f;
        G[idx] = g;
    }
}

// sig descending (stable in the index), |s| with the sign moved into U's column; U_R, W
// rounded back to float32 (lp x lp, zero beyond l).
__global__ void refine_store_kernel(const double *__restrict__ U, const double *__restrict__ W, int l, int lp,
                                    double *__restrict__ sig, float *__restrict__ UR, float *__restrict__ Wf) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double *s = reinterpret_cast<double *>(smraw);
    int *perm = reinterpret_cast<int *>(s + l);
    for (int p = threadIdx.x; p < l; p += blockDim.x) s[p] = sig[p];
    __syncthreads();
    for (int p = threadIdx.x; p < l; p += blockDim.x) {
        const double v = fabs(s[p]);
        int rank = 0;
        for (int j = 0; j < l; j++) {
            const double w = fabs(s[j]);
            rank += (w > v) || (w == v && j < p);
        }
        perm[rank] = p;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < l; o += blockDim.x) sig[o] = fabs(s[perm[o]]);
    for (int idx = threadIdx.x; idx < lp * lp; idx += blockDim.x) {
        const int i = idx / lp, o = idx % lp;
        float u = 0.f, w = 0.f;
        if (i < l && o < l) {
            const int p = perm[o];
            const double sg = s[p] < 0.0 ? -1.0 : 1.0;
            u = (float)(sg * U[(int64_t)i * l + p]);
            w = (float)W[(int64_t)i * l + p];
        }
        UR[idx] = u;
        Wf[idx] = w;
    }
}

cudaError_t prod64(const Prod64Set &set, int count, int l, cudaStream_t s) {
    const unsigned t = (unsigned)((l + RT - 1) / RT);
    prod64_kernel<<<dim3(t, t, (unsigned)count), RT * RT, 0, s>>>(set, l);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

size_t svd_refine64_bytes(int l) { return sizeof(double) * 10 * (size_t)l * l; }

cudaError_t svd_refine64(const double *R, int l, int lp, float *UR, float *W, double *sig, double *ws,
                         cudaStream_t s) {
    if (l < 1 || l > 4096 || lp < l || !ws) return cudaErrorInvalidValue;
    const size_t ll = (size_t)l * l;
    double *U0 = ws, *W0 = ws + ll, *U1 = ws + 2 * ll, *W1 = ws + 3 * ll;
    double *P = ws + 4 * ll, *Q = ws + 5 * ll, *M1 = ws + 6 * ll, *T = ws + 7 * ll, *F = ws + 8 * ll,
           *G = ws + 9 * ll;
    const unsigned grid = (unsigned)std::min<size_t>((ll + 255) / 256, 1024);
    refine_load_kernel<<<grid, 256, 0, s>>>(UR, W, l, lp, U0, W0);
    note_launch();
    cudaError_t e = cudaGetLastError();
    for (int it = 0; it < kRefineSteps && e == cudaSuccess; it++) {
        Prod64Set a = {};
        a.p[0] = Prod64{U0, U0, nullptr, P, 1};   // P = U^T U
        a.p[1] = Prod64{W0, W0, nullptr, Q, 1};   // Q = W^T W
        a.p[2] = Prod64{U0, R, nullptr, M1, 1};   // M1 = U^T R
        if ((e = prod64(a, 3, l, s)) != cudaSuccess) break;
        Prod64Set b = {};
        b.p[0] = Prod64{M1, W0, nullptr, T, 0};   // T = U^T R W
        if ((e = prod64(b, 1, l, s)) != cudaSuccess) break;
        refine_step_kernel<<<grid, 256, 0, s>>>(P, Q, T, l, F, G, sig);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        Prod64Set c = {};
        c.p[0] = Prod64{U0, F, U0, U1, 0};        // U (I + F)
        c.p[1] = Prod64{W0, G, W0, W1, 0};        // W (I + G)
        if ((e = prod64(c, 2, l, s)) != cudaSuccess) break;
        std::swap(U0, U1);
        std::swap(W0, W1);
    }
    if (e != cudaSuccess) return e;
    const size_t smem = (sizeof(double) + sizeof(int)) * (size_t)l;
    refine_store_kernel<<<1, 1024, smem, s>>>(U0, W0, l, lp, sig, UR, W);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gbr
