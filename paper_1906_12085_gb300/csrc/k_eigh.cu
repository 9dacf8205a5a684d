// Symmetric eigen-decomposition of an n x n float64 matrix beyond one CTA: the
// eigen-decomposition step of the Gram route (Sec. 2.3, Sec. 3.1.3 step 2) for the
// k = n regime of the paper's experiments (n up to a few thousand, Sec. 4).
//
//   G = H T H^T   Householder tridiagonalisation (H = H_0 ... H_{n-3}), one
//                 cooperative persistent launch: per column a reflector built by one
//                 CTA, p = tau B v by all CTAs, B -= v w^T + w v^T with
//                 w = p - (tau/2)(p^T v) v; bounded grid barriers between the phases;
//   T z = lam z   eigenvalues by bisection on Sturm counts (one thread per value),
//                 eigenvectors by inverse iteration with a tridiagonal LU factorisation
//                 with partial pivoting (one thread per vector), Gram-Schmidt inside
//                 clusters of nearly equal values;
//   V = H Z       the reflectors applied to Z in reverse order, each CTA owning a
//                 stripe of columns.
// Everything in float64 (the Gram matrix is formed in the element type of the plan).
#include <float.h>

#include "common.cuh"

namespace gbr {
namespace {

constexpr int ET = 256;                   // threads per CTA
constexpr unsigned kSpinLimit = 1u << 23; // polls of a grid barrier before it gives up (~1 s)

// Bounded grid-wide barrier of a cooperative launch (all CTAs resident): the last CTA to
// arrive resets the counter and advances the generation; the others poll the generation.
// A CTA that polls kSpinLimit times sets ST_TIMEOUT and returns false; its caller ends
// the kernel (the other CTAs then give up at their next barrier).  Every thread fences on
// both sides; data another CTA wrote is read with ld.global.cg (L2, never a stale L1 line).
__device__ bool grid_sync(unsigned *count, unsigned *gen, int *status) {
    __shared__ int s_ok;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vg = gen;
        const unsigned g = *vg;
        __threadfence();
        int ok = 1;
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            unsigned it = 0;
            while (*vg == g) {
                if (++it > kSpinLimit) {
                    ok = 0;
                    atomicOr(status, (int)ST_TIMEOUT);
                    break;
                }
                if (it > 4096) __nanosleep(64);  // a tight poll first: most waits are a few microseconds
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    __threadfence();
    return s_ok != 0;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the CTA (every thread receives it)
__device__ double block_sum(double v) {
    __shared__ double red[ET / 32];
    __shared__ double tot;
    v = warp_sum_d(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < ET / 32; i++) s += red[i];
        tot = s;
    }
    __syncthreads();
    return tot;
}

// Householder tridiagonalisation of the symmetric A (n x n, row-major, both triangles).
// Step j reduces column / row j: x = A[j][j+1:], H_j = I - tau_j v v^T with v[0] = 1 and
// H_j x = beta e_1 (beta = -sign(x_0) ||x||).  On exit d (n) and e (n - 1) hold T, row j
// of A (columns j+1..) holds v_j and tau[j] its scale.  Work arrays: vb, p (n doubles),
// part (gridDim.x doubles), bar (2 unsigned, zero).
__global__ void __launch_bounds__(ET) tridiag_kernel(double *__restrict__ A, int n, double *__restrict__ d,
                                                     double *__restrict__ e, double *__restrict__ tau,
                                                     double *__restrict__ vb, double *__restrict__ p,
                                                     double *__restrict__ part, unsigned *bar, int *status) {
    __shared__ double s_tau, s_k;
    const int tid = threadIdx.x, lane = tid & 31;
    const int gw = blockIdx.x * (ET / 32) + (tid >> 5), nw = gridDim.x * (ET / 32);
    for (int j = 0; j + 2 < n; j++) {
        const int s = n - j - 1;
        const double *x = A + (int64_t)j * n + j + 1;
        // (A) the reflector, by CTA 0
        if (blockIdx.x == 0) {
            double ss = 0.0;
            for (int i = 1 + tid; i < s; i += ET) {
                const double xi = __ldcg(x + i);
                ss += xi * xi;
            }
            const double sig2 = block_sum(ss);
            const double alpha = __ldcg(x);
            double t, beta, scale;
            if (sig2 == 0.0) {
                t = 0.0;
                beta = alpha;
                scale = 0.0;
            } else {
                const double nrm = sqrt(alpha * alpha + sig2);
                beta = alpha >= 0.0 ? -nrm : nrm;
                t = (beta - alpha) / beta;
                scale = 1.0 / (alpha - beta);
            }
            for (int i = tid; i < s; i += ET) vb[i] = i == 0 ? 1.0 : __ldcg(x + i) * scale;
            __syncthreads();
            for (int i = tid; i < s; i += ET) A[(int64_t)j * n + j + 1 + i] = __ldcg(vb + i);
            if (tid == 0) {
                d[j] = __ldcg(A + (int64_t)j * n + j);
                e[j] = beta;
                tau[j] = t;
            }
        }
        if (!grid_sync(bar, bar + 1, status)) return;
        if (tid == 0) s_tau = __ldcg(tau + j);
        __syncthreads();
        const double t = s_tau;
        if (t != 0.0) {
            // (B) p = tau B v (a warp per row), and this CTA's share of p^T v
            double dot = 0.0;
            for (int i = gw; i < s; i += nw) {
                const double *row = A + (int64_t)(j + 1 + i) * n + j + 1;
                double acc = 0.0;
#pragma unroll 8
                for (int c = lane; c < s; c += 32) acc += __ldcg(row + c) * __ldcg(vb + c);
                acc = warp_sum_d(acc) * t;
                if (lane == 0) {
                    p[i] = acc;
                    dot += acc * __ldcg(vb + i);
                }
            }
            const double bs = block_sum(dot);
            if (tid == 0) part[blockIdx.x] = bs;
            if (!grid_sync(bar, bar + 1, status)) return;
            // (C) w = p - (tau/2)(p^T v) v;  B -= v w^T + w v^T
            if (tid == 0) {
                double ptv = 0.0;
                for (unsigned b = 0; b < gridDim.x; b++) ptv += __ldcg(part + b);
                s_k = 0.5 * t * ptv;
            }
            __syncthreads();
            const double K = s_k;
            for (int i = gw; i < s; i += nw) {  // a warp per row, the lanes along the row
                const double vi = __ldcg(vb + i), wi = __ldcg(p + i) - K * vi;
                double *row = A + (int64_t)(j + 1 + i) * n + j + 1;
#pragma unroll 8
                for (int c = lane; c < s; c += 32) {
                    const double vc = __ldcg(vb + c), wc = __ldcg(p + c) - K * vc;
                    row[c] = __ldcg(row + c) - (vi * wc + wi * vc);
                }
            }
        }
        if (!grid_sync(bar, bar + 1, status)) return;
    }
    if (blockIdx.x == 0 && tid == 0) {  // the last 2 x 2 (or 1 x 1) block
        if (n >= 2) {
            d[n - 2] = __ldcg(A + (int64_t)(n - 2) * n + n - 2);
            e[n - 2] = __ldcg(A + (int64_t)(n - 2) * n + n - 1);
            tau[n - 2] = 0.0;
        }
        d[n - 1] = __ldcg(A + (int64_t)(n - 1) * n + n - 1);
    }
}

// lam[t] = the (t+1)-th largest eigenvalue of T (d, e), by multisection inside the Gershgorin
// interval: eight lanes per eigenvalue, each counting the eigenvalues below one of eight
// interior points of the bracket, which then shrinks 9-fold (about seventeen rounds to
// reach 2u of its end points; fewer float64 divisions in all than 32 points per round).  The count of eigenvalues below x is the number of negative
// pivots of the LDL^T factorisation of T - x I (Sylvester's law of inertia); pivots
// smaller than pivmin in magnitude become -pivmin.
__device__ __forceinline__ int sturm_below(const double *__restrict__ d, const double *__restrict__ e, int n,
                                           double x, double pivmin) {
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    int cnt = q < 0.0;
    for (int k = 1; k < n; k++) {
        const double ek = e[k - 1];
        q = (d[k] - x) - (ek * ek) / q;
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
    }
    return cnt;
}

__global__ void bisect_kernel(const double *__restrict__ d, const double *__restrict__ e, int n,
                              double *__restrict__ lam) {
    constexpr int G = 8;  // lanes per eigenvalue: G interior points, the bracket shrinks (G + 1)-fold
    const int lane = threadIdx.x & 31, sub = lane % G;
    const unsigned gmask = ((1u << G) - 1u) << (lane / G * G);
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (t >= n) return;  // whole groups of G lanes leave together
    double lo = DBL_MAX, hi = -DBL_MAX, emax2 = 0.0;
    for (int k = sub; k < n; k += G) {
        const double r = (k > 0 ? fabs(e[k - 1]) : 0.0) + (k + 1 < n ? fabs(e[k]) : 0.0);
        lo = fmin(lo, d[k] - r);
        hi = fmax(hi, d[k] + r);
        if (k + 1 < n) emax2 = fmax(emax2, e[k] * e[k]);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(gmask, lo, o));
        hi = fmax(hi, __shfl_xor_sync(gmask, hi, o));
        emax2 = fmax(emax2, __shfl_xor_sync(gmask, emax2, o));
    }
    const double pivmin = DBL_MIN * fmax(1.0, emax2);
    const double span = fmax(fabs(lo), fabs(hi));
    lo -= 2.0 * DBL_EPSILON * span + pivmin;
    hi += 2.0 * DBL_EPSILON * span + pivmin;
    const int a = n - 1 - t;  // ascending index of the wanted value
    const int base = lane / G * G;
    for (int it = 0; it < 128; it++) {
        if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) break;
        const double x = lo + (hi - lo) * (double)(sub + 1) / (double)(G + 1);
        const unsigned below = (__ballot_sync(gmask, sturm_below(d, e, n, x, pivmin) <= a) >> base) & ((1u << G) - 1u);
        // the counts grow with x: the points at or below lambda_a form a prefix
        const int jj = 31 - __clz(below);  // -1 when no point is
        const double xj = __shfl_sync(gmask, x, base + (jj < 0 ? 0 : jj));
        const double xn = __shfl_sync(gmask, x, base + (jj + 1 > G - 1 ? G - 1 : jj + 1));
        const double nlo = jj >= 0 ? xj : lo, nhi = jj < G - 1 ? xn : hi;
        if (!(nlo > lo || nhi < hi)) break;  // no progress representable
        lo = nlo;
        hi = nhi;
    }
    if (sub == 0) lam[t] = 0.5 * (lo + hi);
}

// Inverse iteration for eigenvalue lam[t]: (T - lam I) x = b solved by Gaussian elimination
// with partial pivoting on the tridiagonal (at most two superdiagonals appear in U), three
// iterations from a pseudo-random start, x normalised each time.  Column t of Z (n x n,
// row-major, ld ldz) receives the vector; U0, U1, U2 (n x ldz each) are the scratch of U,
// laid out [k][t] like Z so that the threads' accesses coalesce.
__global__ void inviter_kernel(const double *__restrict__ d, const double *__restrict__ e, const double *__restrict__ lam,
                               int n, double *__restrict__ Z, int64_t ldz, double *__restrict__ U0,
                               double *__restrict__ U1, double *__restrict__ U2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double lt = lam[t];
    // replacement of an exactly zero pivot: u ||T|| (||T|| = the largest |eigenvalue|)
    const double tiny = DBL_EPSILON * fmax(fmax(fabs(lam[0]), fabs(lam[n - 1])), DBL_MIN);
    auto Zk = [&](int k) -> double & { return Z[(int64_t)k * ldz + t]; };
    // start vector: uniform in [-1, 1) from a counter-based generator
    for (int k = 0; k < n; k++) {
        const double u = (double)(splitmix64(0x5EED0F1Bull + (uint64_t)t, (uint64_t)k) >> 11) * 0x1.0p-53;
        Zk(k) = 2.0 * u - 1.0;
    }
    for (int it = 0; it < 3; it++) {
        // forward elimination: row k carries (r0, r1, r2) in columns k, k+1, k+2, and b_k
        double r0 = d[0] - lt, r1 = n > 1 ? e[0] : 0.0, r2 = 0.0, rb = Zk(0);
        for (int k = 0; k + 1 < n; k++) {
            const double c = e[k];                              // row k+1: (c, a, cn) in columns k, k+1, k+2
            const double a = d[k + 1] - lt, cn = k + 2 < n ? e[k + 1] : 0.0, bn = Zk(k + 1);
            double u0, u1, u2, ub, n0, n1, nb;
            if (fabs(r0) >= fabs(c)) {                          // pivot on row k
                const double piv = r0 != 0.0 ? r0 : tiny;
                const double m = c / piv;
                u0 = piv; u1 = r1; u2 = r2; ub = rb;
                n0 = a - m * r1; n1 = cn - m * r2; nb = bn - m * rb;
            } else {                                            // rows k and k+1 interchanged
                const double m = r0 / c;
                u0 = c; u1 = a; u2 = cn; ub = bn;
                n0 = r1 - m * a; n1 = r2 - m * cn; nb = rb - m * bn;
            }
            U0[(int64_t)k * ldz + t] = u0;
            U1[(int64_t)k * ldz + t] = u1;
            U2[(int64_t)k * ldz + t] = u2;
            Zk(k) = ub;
            r0 = n0; r1 = n1; r2 = 0.0; rb = nb;
        }
        // back substitution (the last row has only its diagonal)
        double x2 = 0.0, x1 = rb / (r0 != 0.0 ? r0 : tiny);
        Zk(n - 1) = x1;
        double nrm2 = x1 * x1;
        for (int k = n - 2; k >= 0; k--) {
            const double u0 = U0[(int64_t)k * ldz + t], u1 = U1[(int64_t)k * ldz + t], u2 = U2[(int64_t)k * ldz + t];
            const double x0 = (Zk(k) - u1 * x1 - u2 * x2) / (u0 != 0.0 ? u0 : tiny);
            Zk(k) = x0;
            nrm2 += x0 * x0;
            x2 = x1;
            x1 = x0;
        }
        const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
        for (int k = 0; k < n; k++) Zk(k) *= inv;
    }
}

// Inverse iteration leaves the vectors of eigenvalues closer than ~u ||T|| / gap from
// orthogonal.  Gram-Schmidt (applied twice) inside each cluster of consecutive eigenvalues
// closer than kClusterGap ||T||: the CTA whose index starts a cluster orthonormalises its
// vectors in order.  Clusters of more than kClusterMax vectors set ST_NOCONV.
constexpr double kClusterGap = 1e-8;
constexpr int kClusterMax = 512;
__global__ void __launch_bounds__(ET) cluster_mgs_kernel(const double *__restrict__ lam, int n,
                                                         double *__restrict__ Z, int64_t ldz, int *status) {
    const int t0 = blockIdx.x;
    if (t0 + 1 >= n) return;
    const double gap = kClusterGap * fmax(fabs(lam[0]), fabs(lam[n - 1]));
    if (t0 > 0 && lam[t0 - 1] - lam[t0] < gap) return;  // not the start of a cluster
    int t1 = t0;
    while (t1 + 1 < n && lam[t1] - lam[t1 + 1] < gap) t1++;
    if (t1 == t0) return;
    if (t1 - t0 + 1 > kClusterMax) {
        if (threadIdx.x == 0) atomicOr(status, (int)ST_NOCONV);
        return;
    }
    for (int j = t0 + 1; j <= t1; j++) {
        for (int pass = 0; pass < 2; pass++)
            for (int i = t0; i < j; i++) {
                double s = 0.0;
                for (int k = threadIdx.x; k < n; k += ET) s += Z[(int64_t)k * ldz + i] * Z[(int64_t)k * ldz + j];
                const double dot = block_sum(s);
                for (int k = threadIdx.x; k < n; k += ET) Z[(int64_t)k * ldz + j] -= dot * Z[(int64_t)k * ldz + i];
                __syncthreads();
            }
        double s = 0.0;
        for (int k = threadIdx.x; k < n; k += ET) s += Z[(int64_t)k * ldz + j] * Z[(int64_t)k * ldz + j];
        const double nrm2 = block_sum(s);
        const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
        for (int k = threadIdx.x; k < n; k += ET) Z[(int64_t)k * ldz + j] *= inv;
        __syncthreads();
    }
}

// V = H_0 ... H_{n-3} Z: for j = n-3 .. 0, rows j+1.. of Z <- (I - tau_j v_j v_j^T) rows j+1..,
// v_j in row j of A (columns j+1..).  A CTA owns BC columns, kept in shared memory for the
// whole sweep (n x BC doubles); thread (ty, tx) handles column c0 + tx and the rows congruent
// to ty modulo ET / BC.
template <int BC>
__global__ void __launch_bounds__(ET) backtransform_kernel(const double *__restrict__ A, const double *__restrict__ tau,
                                                           int n, double *__restrict__ Z, int64_t ldz) {
    extern __shared__ __align__(16) double zs[];  // n x BC
    constexpr int RY = ET / BC;
    __shared__ double red[RY][BC + 1];
    const int tx = threadIdx.x % BC, ty = threadIdx.x / BC;
    const int c0 = blockIdx.x * BC, c = c0 + tx;
    const bool on = c < n;
    for (int i = ty; i < n; i += RY) zs[i * BC + tx] = on ? Z[(int64_t)i * ldz + c] : 0.0;
    __syncthreads();
    for (int j = n - 3; j >= 0; j--) {
        const double t = tau[j];
        if (t == 0.0) continue;  // uniform across the CTA
        const double *v = A + (int64_t)j * n + j + 1;
        const int s = n - j - 1;
        double acc = 0.0;
        for (int i = ty; i < s; i += RY) acc += v[i] * zs[(j + 1 + i) * BC + tx];
        red[ty][tx] = acc;
        __syncthreads();
        double y = 0.0;
#pragma unroll 8
        for (int r = 0; r < RY; r++) y += red[r][tx];
        y *= t;
        for (int i = ty; i < s; i += RY) zs[(j + 1 + i) * BC + tx] -= y * v[i];
        __syncthreads();
    }
    if (on)
        for (int i = ty; i < n; i += RY) Z[(int64_t)i * ldz + c] = zs[i * BC + tx];
}

// sig = sqrt(max(lam, 0)); Vs[:, i] = V[:, i] / sig_i, for n beyond one CTA.  An eigenvalue of
// the float64 Gram matrix is resolved only to ~n eps lam_1, so a sigma_i below
// sqrt(n eps) sigma_1 is indistinguishable from zero: its column of Vs (and so u_i) is zero
// and ST_RANKDEF is set.
template <typename T>
__global__ void gram_scale_kernel(const double *__restrict__ lam, const double *__restrict__ V, int n,
                                  double *__restrict__ sig, T *__restrict__ Vs, int *__restrict__ status) {
    const double thr = sqrt((double)n * DBL_EPSILON) * sqrt(fmax(lam[0], 0.0));
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) {
        sig[idx] = sqrt(fmax(lam[idx], 0.0));
        if (!(sig[idx] > thr)) atomicOr(status, (int)ST_RANKDEF);
    }
    if (idx >= (int64_t)n * n) return;
    const int j = (int)(idx % n);
    const double s = sqrt(fmax(lam[j], 0.0));
    Vs[idx] = s > thr ? (T)(V[idx] / s) : T(0);
}

}  // namespace

size_t eigh_workspace_bytes(int n) {
    const size_t nn = (size_t)n * n, n8 = ((size_t)n + 31) / 32 * 32;
    // U0, U1, U2 (n x n each), d, e, tau, vb, p (n each), part (up to 1024), barrier
    return sizeof(double) * (3 * nn + 5 * n8 + 1024) + 256;
}

cudaError_t eigh_large(double *A, int n, double *lam, double *V, int *status, void *ws, cudaStream_t s) {
    if (n < 1 || !ws) return cudaErrorInvalidValue;
    const size_t nn = (size_t)n * n, n8 = ((size_t)n + 31) / 32 * 32;
    double *w = static_cast<double *>(ws);
    double *U0 = w, *U1 = U0 + nn, *U2 = U1 + nn;
    double *d = U2 + nn, *e = d + n8, *tau = e + n8, *vb = tau + n8, *p = vb + n8;
    double *part = p + n8;
    unsigned *bar = reinterpret_cast<unsigned *>(part + 1024);
    cudaError_t err = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0, occ = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tridiag_kernel, ET, 0)) != cudaSuccess) return err;
    if (occ < 1) return cudaErrorInvalidValue;
    const int grid = sms < 1024 ? sms : 1024;  // one CTA per SM: every CTA is resident
    {
        void *args[] = {&A, &n, &d, &e, &tau, &vb, &p, &part, &bar, &status};
        if ((err = cudaLaunchCooperativeKernel((const void *)tridiag_kernel, dim3(grid), dim3(ET), args, 0, s)) !=
            cudaSuccess)
            return err;
        note_launch();
    }
    // eigenvalues (descending), eigenvectors of T in V, clusters, then V = H Z in place
    bisect_kernel<<<(unsigned)ceil_div((int64_t)n * 8, 256), 256, 0, s>>>(d, e, n, lam);
    note_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    double *Z = V;
    const int64_t ldz = n;
    inviter_kernel<<<(n + 127) / 128, 128, 0, s>>>(d, e, lam, n, Z, ldz, U0, U1, U2);
    note_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    cluster_mgs_kernel<<<n, ET, 0, s>>>(lam, n, Z, ldz, status);
    note_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // the widest stripe whose n x BC doubles fit one SM's shared memory
    const size_t sm8 = sizeof(double) * (size_t)n * 8, sm4 = sizeof(double) * (size_t)n * 4;
    if (sm8 <= 200 * 1024) {
        cudaFuncSetAttribute(backtransform_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm8);
        backtransform_kernel<8><<<(n + 7) / 8, ET, sm8, s>>>(A, tau, n, Z, ldz);
    } else {
        cudaFuncSetAttribute(backtransform_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm4);
        backtransform_kernel<4><<<(n + 3) / 4, ET, sm4, s>>>(A, tau, n, Z, ldz);
    }
    note_launch();
    return cudaGetLastError();
}

// G64 (n x n, both triangles) = the upper triangle of Gs (ldg) widened to float64
template <typename T>
__global__ void symmetrize_kernel(const T *__restrict__ Gs, int64_t ldg, int n, double *__restrict__ G64) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    G64[idx] = i <= j ? (double)Gs[(int64_t)i * ldg + j] : (double)Gs[(int64_t)j * ldg + i];
}

template <typename T>
cudaError_t symmetrize(const T *Gs, int64_t ldg, int n, double *G64, cudaStream_t s) {
    symmetrize_kernel<T><<<(unsigned)ceil_div((int64_t)n * n, 256), 256, 0, s>>>(Gs, ldg, n, G64);
    note_launch();
    return cudaGetLastError();
}
template cudaError_t symmetrize<float>(const float *, int64_t, int, double *, cudaStream_t);
template cudaError_t symmetrize<double>(const double *, int64_t, int, double *, cudaStream_t);

template <typename T>
cudaError_t gram_scale(const double *lam, const double *V, int n, double *sig, T *Vs, int *status, cudaStream_t s) {
    const int64_t tot = (int64_t)n * n;
    gram_scale_kernel<T><<<(unsigned)ceil_div(tot, 256), 256, 0, s>>>(lam, V, n, sig, Vs, status);
    note_launch();
    return cudaGetLastError();
}
template cudaError_t gram_scale<float>(const double *, const double *, int, double *, float *, int *, cudaStream_t);
template cudaError_t gram_scale<double>(const double *, const double *, int, double *, double *, int *, cudaStream_t);

}  // namespace gbr
