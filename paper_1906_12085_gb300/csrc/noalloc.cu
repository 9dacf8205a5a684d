// svd_exact_gram_static: the Gram route of svd_exact with every piece of
// device scratch taken from one file-scope static array instead of a plan's
// cudaMalloc'd workspace.  The kernels are the library's own (centring, the
// split-K A^T A product with its chunk partials, the Jacobi eigensolver, the
// finishing and sign kernels); only where their scratch lives differs.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = 12u << 20;  // 12 MiB per device, held until process exit
constexpr int kMaxN = 64;
constexpr int kMaxDevices = 64;

// The scratch itself.  Host code must not pass `g_scratch` to a kernel: on the
// host that name is only a stand-in, not a device address.  Its device address
// is looked up once per device with cudaGetSymbolAddress (below).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up on first use.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

struct Bump {
    char *base;
    size_t off = 0;
    void *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

struct Slices {
    int *status;
    double *mu, *fro2, *cpart, *G64, *lam, *Vfull, *sig;
    void *G, *Vs, *part;
    int64_t part_elems;
};

template <typename T>
Slices carve(char *base, int64_t m, int64_t n, size_t *used) {
    Bump b{base};
    Slices s;
    s.status = (int *)b.take(sizeof(int));
    s.mu = (double *)b.take(sizeof(double) * n);
    s.fro2 = (double *)b.take(sizeof(double));
    s.cpart = (double *)b.take(sizeof(double) * gbr::center_partials(m, n));
    s.G = b.take(sizeof(T) * n * n);
    s.G64 = (double *)b.take(sizeof(double) * n * n);
    s.lam = (double *)b.take(sizeof(double) * n);
    s.Vfull = (double *)b.take(sizeof(double) * n * n);
    s.Vs = b.take(sizeof(T) * n * n);
    s.sig = (double *)b.take(sizeof(double) * n);
    s.part_elems = gbr::gemm_tn_partials(m, n, n);
    s.part = b.take(sizeof(T) * (s.part_elems > 0 ? s.part_elems : 1));
    *used = b.off;
    return s;
}

#define CKE(...)                                       \
    do {                                               \
        if ((__VA_ARGS__) != cudaSuccess) return RSVD_ERR_CUDA; \
    } while (0)

template <typename T>
rsvd_status run(T *A, int64_t m, int64_t n, double *S, T *U, T *V, cudaStream_t st) {
    void *addr = nullptr;
    if (scratch_address(&addr) != cudaSuccess) return RSVD_ERR_CUDA;
    size_t used = 0;
    carve<T>(nullptr, m, n, &used);
    if (used > kScratchBytes) return RSVD_ERR_UNSUPPORTED;
    Slices s = carve<T>((char *)addr, m, n, &used);
    const int nn = (int)n;
    CKE(cudaMemsetAsync(s.status, 0, sizeof(int), st));  // the only slice that must start at zero
    CKE(gbr::center_columns<T>(A, m, n, n, true, s.mu, s.fro2, s.cpart, st));
    CKE(gbr::gemm_tn<T>(m, n, n, A, n, A, n, (T *)s.G, n, (T *)s.part, s.part_elems, st));
    CKE(gbr::copy2d<T, double>((T *)s.G, n, s.G64, n, n, n, n, st));
    CKE(gbr::jacobi_eig(s.G64, nn, s.lam, s.Vfull, s.status, st));
    CKE(gbr::gram_finish<T>(s.lam, s.Vfull, nn, s.sig, (T *)s.Vs, s.status, st));
    CKE(gbr::gemm_nn<T>(m, n, n, A, n, (T *)s.Vs, n, U, n, st));
    CKE(gbr::copy2d<double, T>(s.Vfull, n, V, n, n, n, n, st));
    CKE(gbr::sign_normalize<T>(V, n, nn, n, U, m, n, st));
    CKE(gbr::copy_f64(s.sig, S, n, st));
    int h = 0;
    CKE(cudaMemcpyAsync(&h, s.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKE(cudaStreamSynchronize(st));
    if (h & gbr::ST_NOCONV) return RSVD_ERR_NOCONV;
    return RSVD_OK;
}

}  // namespace

extern "C" rsvd_status svd_exact_gram_static(void *A, int64_t m, int64_t n, rsvd_dtype dtype, double *S, void *U,
                                             void *V, void *cuda_stream) {
    if (!A || !S || !U || !V || n < 1 || m < n) return RSVD_ERR_ARG;
    if (n > kMaxN) return RSVD_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (dtype == RSVD_F64) return run<double>((double *)A, m, n, S, (double *)U, (double *)V, st);
    if (dtype == RSVD_F32) return run<float>((float *)A, m, n, S, (float *)U, (float *)V, st);
    return RSVD_ERR_UNSUPPORTED;
}
