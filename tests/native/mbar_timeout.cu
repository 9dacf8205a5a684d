// The bounded mbarrier wait of the product kernels (tc_ptx.cuh) made to run out, GPU-safely:
// one CTA waits with a short cap on a barrier that nothing arrives at and reports the status
// bit the product kernels set when a wait gives up (ST_TIMEOUT); it then waits on a second
// barrier that one of its threads completes, which must succeed.  No TMA copy, MMA or
// tensor-memory allocation is outstanding in this kernel.  Prints: cuda error, status of the
// abandoned wait, result of the completed wait, elapsed nanoseconds of the abandoned wait.
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "tc_ptx.cuh"

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void wait_kernel(long long *out, unsigned cap) {
    __shared__ uint64_t never, once;
    if (threadIdx.x == 0) {
        gbr::tc::mbar_init(&never, 1);
        gbr::tc::mbar_init(&once, 1);
        gbr::tc::mbar_fence_init();
    }
    __syncthreads();
    const unsigned long long t0 = now_ns();
    const bool ok_never = gbr::tc::mbar_wait(&never, 0, cap);
    const unsigned long long t1 = now_ns();
    __syncthreads();
    if (threadIdx.x == 0) gbr::tc::mbar_arrive(&once);
    const bool ok_once = gbr::tc::mbar_wait(&once, 0, cap);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = ok_never ? 0 : (long long)gbr::ST_TIMEOUT;
        out[1] = ok_once ? 1 : 0;
        out[2] = (long long)(t1 - t0);
    }
}

int main(int argc, char **argv) {
    const unsigned cap = argc > 1 ? (unsigned)atoi(argv[1]) : 256u;
    long long *d = nullptr, h[3] = {-1, -1, -1};
    if (cudaMalloc(&d, sizeof h) != cudaSuccess) return 2;
    cudaMemset(d, 0xff, sizeof h);
    wait_kernel<<<1, 64>>>(d, cap);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    printf("%d %lld %lld %lld\n", (int)e, h[0], h[1], h[2]);
    return e == cudaSuccess ? 0 : 1;
}
