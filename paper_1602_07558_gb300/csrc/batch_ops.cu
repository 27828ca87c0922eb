// Instantiation unit: the batched kernels of heat FP64, the hash test update and
// Euler FP64, and the per-grid wave-speed reduction that fixes each Euler
// grid's time step. The compensated binary32 forms (built for several tile
// sides) have units of their own: batch_heat_kahan.cu, batch_euler_kahan.cu.
#include "batch.cuh"

namespace swept {
const BatchTable *batchtable_heat() { return BatchLaunch<HeatOp>::table(); }
const BatchTable *batchtable_hash() { return BatchLaunch<HashOp>::table(); }
const BatchTable *batchtable_euler() { return BatchLaunch<EulerOp>::table(); }

namespace {

__device__ __forceinline__ double widen_b(double v) { return v; }
__device__ __forceinline__ double widen_b(float v) { return (double)v; }
__device__ __forceinline__ double widen_b(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// blockIdx.y = grid; the blocks of a grid stride over its points. Each grid's
// a = max over its points of max(|u| + c, |v| + c), c = sqrt(gamma p / rho),
// with the operations of the single-grid reduction; positive doubles order
// like their bit patterns, so the maxima combine with an integer atomicMax.
template <class T>
__global__ void __launch_bounds__(256) batch_wavespeed_kernel(const GridDesc *grids,
                                                              const T *state, double gamma,
                                                              unsigned long long *out) {
    const GridDesc gd = grids[blockIdx.y];
    const size_t np = (size_t)gd.G.nx * gd.G.ny;
    const T *U = state + gd.state_off;
    const double gm1 = gamma - 1.0;
    double amax = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < np;
         p += (size_t)gridDim.x * blockDim.x) {
        const double r = widen_b(U[p]), m = widen_b(U[np + p]), q = widen_b(U[2 * np + p]),
                     E = widen_b(U[3 * np + p]);
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
        atomicMax(out + blockIdx.y, (unsigned long long)__double_as_longlong(b));
    }
}

}  // namespace

cudaError_t batch_euler_wavespeed(const GridDesc *d_grids, int count, const void *state,
                                  int esize, double gamma, unsigned long long *d_out,
                                  cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_out, 0, (size_t)count * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const dim3 grid(8, count);   // 8 blocks per grid (the largest grids have ~260k points)
    if (esize == 8)
        batch_wavespeed_kernel<<<grid, 256, 0, st>>>(d_grids, (const double *)state, gamma, d_out);
    else if (esize == 4)
        batch_wavespeed_kernel<<<grid, 256, 0, st>>>(d_grids, (const float *)state, gamma, d_out);
    else
        batch_wavespeed_kernel<<<grid, 256, 0, st>>>(d_grids, (const __nv_bfloat16 *)state, gamma,
                                                     d_out);
    return cudaGetLastError();
}
}  // namespace swept
