// Instantiation unit: 2D compressible Euler (midpoint RK2) and the wave-speed
// reduction that fixes its time step at set_state (for every storage type).
#include "launch.cuh"

namespace swept {

const OpTable *optable_euler() { return Launch<EulerOp>::table(); }

// a = max over points of max(|u| + c, |v| + c), c = sqrt(gamma p / rho), from
// planes 0-3 = (rho, m, q, E), in binary64 (a binary32 or bfloat16 state is
// widened exactly first). Positive doubles order like their bit patterns, so
// the block maxima combine with an integer atomicMax (exact, order-free).
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return (double)v; }
__device__ __forceinline__ double widen(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <class T>
__global__ void __launch_bounds__(256) wavespeed_kernel(const T *U, size_t np, double gamma,
                                                        unsigned long long *out) {
    const double gm1 = gamma - 1.0;
    double amax = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < np;
         p += (size_t)gridDim.x * blockDim.x) {
        const double r = widen(U[p]), m = widen(U[np + p]), q = widen(U[2 * np + p]),
                     E = widen(U[3 * np + p]);
        const double iv = __ddiv_rn(1.0, r);
        const double u = __dmul_rn(m, iv), v = __dmul_rn(q, iv);
        const double ke = __dmul_rn(0.5, __fma_rn(m, u, __dmul_rn(q, v)));
        const double pr = __dmul_rn(gm1, __dsub_rn(E, ke));
        const double c = __dsqrt_rn(__dmul_rn(__dmul_rn(gamma, pr), iv));
        const double su = __dadd_rn(fabs(u), c), sv = __dadd_rn(fabs(v), c);
        const double s = su > sv ? su : sv;
        amax = s > amax ? s : amax;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, amax, off);
        amax = o > amax ? o : amax;
    }
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = red[w] > b ? red[w] : b;
        atomicMax(out, (unsigned long long)__double_as_longlong(b));
    }
}

cudaError_t euler_wavespeed(const void *state, int esize, int nx, int ny, double gamma,
                            unsigned long long *d_scratch, double *a_out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_scratch, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const size_t np = (size_t)nx * ny;
    int blocks = (int)((np + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (esize == 8)
        wavespeed_kernel<<<blocks, 256, 0, st>>>((const double *)state, np, gamma, d_scratch);
    else if (esize == 4)
        wavespeed_kernel<<<blocks, 256, 0, st>>>((const float *)state, np, gamma, d_scratch);
    else
        wavespeed_kernel<<<blocks, 256, 0, st>>>((const __nv_bfloat16 *)state, np, gamma,
                                                 d_scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned long long bits = 0;
    e = cudaMemcpyAsync(&bits, d_scratch, sizeof(bits), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    double a;
    memcpy(&a, &bits, sizeof(a));
    *a_out = a;
    return cudaSuccess;
}

}  // namespace swept
