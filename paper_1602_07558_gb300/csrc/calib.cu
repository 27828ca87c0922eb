// Rate measurements for the roofline: the FP64 pipe (fused multiply-add and
// add chains, several chain counts and occupancies, the maximum taken), the
// FP32 pipe (fused multiply-add chains) and shared memory (conflict-free 4-byte
// loads, one wavefront per warp instruction), each timed with CUDA events on
// the caller's stream, best of five launches after a warm-up.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/swept2d.h"

namespace {

constexpr int kIters = 1024;

template <int CH>
__global__ void __launch_bounds__(256) dfma_chains(double *out, double a, double b) {
    double x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = threadIdx.x + i;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = __fma_rn(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s = __dadd_rn(s, x[i]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same 8 chains on `active` lanes of every warp (the others skip the loop):
// the FP64 pipe's time per warp instruction with few lanes busy.
__global__ void __launch_bounds__(256) dfma_lanes(double *out, double a, double b, int active) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x + i;
    if ((int)(threadIdx.x & 31) < active) {
        for (int it = 0; it < kIters; ++it) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = __fma_rn(x[i], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s = __dadd_rn(s, x[i]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void __launch_bounds__(256) dadd_chains(double *out, double a, double b) {
    double x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = threadIdx.x + i;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = __dadd_rn(x[i], (it & 1) ? a : b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s = __dadd_rn(s, x[i]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ffma_chains(double *out, float a, float b) {
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = threadIdx.x + i;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = __fmaf_rn(x[i], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s = __fadd_rn(s, x[i]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Each warp reads 8 rows of 32 consecutive words per round (lane l reads bank
// l: one wavefront per instruction); the loads are volatile, so every one is
// issued, and the running sums keep them live.
constexpr int kSmemWords = 4096;   // 16 KB
__device__ __forceinline__ float lds_volatile(const float *p) {
    float v;
    asm volatile("ld.volatile.shared.f32 %0, [%1];\n"
                 : "=f"(v)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}
__global__ void __launch_bounds__(256) lds_stream(double *out, int rounds) {
    __shared__ float sh[kSmemWords];
    for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) sh[i] = (float)(i & 7);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int row = warp * 8;
    for (int it = 0; it < rounds; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            acc[u] = __fadd_rn(acc[u], lds_volatile(&sh[((row + u) & 127) * 32 + lane]));
        row += 64;
    }
    float s = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) s = __fadd_rn(s, acc[u]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best time (ms) of five launches after a warm-up.
template <class F>
int best_ms(cudaStream_t st, F &&launch, float *best) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SWEPT2D_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SWEPT2D_ECUDA;
    }
    int rc = SWEPT2D_OK;
    *best = 1e30f;
    for (int rep = 0; rep < 6 && rc == SWEPT2D_OK; ++rep) {
        cudaEventRecord(e0, st);
        launch();
        if (cudaGetLastError() != cudaSuccess) rc = SWEPT2D_ECUDA;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = SWEPT2D_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < *best) *best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int swept2d_measure_peaks(void *stream, double *out, int nout) {
    if (!out || nout < 1) return SWEPT2D_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, max_blocks = sms * 8;
    double *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)max_blocks * threads * sizeof(double)) != cudaSuccess)
        return SWEPT2D_ENOMEM;
    double fp64 = 0.0, fp32 = 0.0, smem = 0.0, warp32 = 0.0, warp1 = 0.0;
    int rc = SWEPT2D_OK;
    float ms = 0.f;
    // FP64: chains x blocks per SM, fused multiply-add and add
    const int per_sm[3] = {2, 4, 8};
    for (int k = 0; k < 3 && rc == SWEPT2D_OK; ++k) {
        const int blocks = sms * per_sm[k];
        const double lanes = (double)blocks * threads * kIters;
        if ((rc = best_ms(st, [&] { dfma_chains<4><<<blocks, threads, 0, st>>>(buf, 0.999, 1e-3); }, &ms)) == 0)
            fp64 = fmax(fp64, lanes * 4 / (ms * 1e-3));
        if (rc == 0 && (rc = best_ms(st, [&] { dfma_chains<8><<<blocks, threads, 0, st>>>(buf, 0.999, 1e-3); }, &ms)) == 0)
            fp64 = fmax(fp64, lanes * 8 / (ms * 1e-3));
        if (rc == 0 && (rc = best_ms(st, [&] { dfma_chains<16><<<blocks, threads, 0, st>>>(buf, 0.999, 1e-3); }, &ms)) == 0)
            fp64 = fmax(fp64, lanes * 16 / (ms * 1e-3));
        if (rc == 0 && (rc = best_ms(st, [&] { dadd_chains<8><<<blocks, threads, 0, st>>>(buf, 0.25, -0.25); }, &ms)) == 0)
            fp64 = fmax(fp64, lanes * 8 / (ms * 1e-3));
    }
    if (rc == SWEPT2D_OK && nout > 1) {
        const int blocks = sms * 8;
        if ((rc = best_ms(st, [&] { ffma_chains<<<blocks, threads, 0, st>>>(buf, 0.999f, 1e-3f); }, &ms)) == 0)
            fp32 = (double)blocks * threads * kIters * 16 / (ms * 1e-3);
    }
    if (rc == SWEPT2D_OK && nout > 2) {
        const int blocks = sms * 8, rounds = 4096;
        if ((rc = best_ms(st, [&] { lds_stream<<<blocks, threads, 0, st>>>(buf, rounds); }, &ms)) == 0)
            smem = (double)blocks * (threads / 32) * rounds * 8 / (ms * 1e-3);   // warp loads = wavefronts
    }
    if (rc == SWEPT2D_OK && nout > 3) {
        const int blocks = sms * 8;
        const double winstr = (double)blocks * (threads / 32) * kIters * 8;
        if ((rc = best_ms(st, [&] { dfma_lanes<<<blocks, threads, 0, st>>>(buf, 0.999, 1e-3, 32); }, &ms)) == 0)
            warp32 = winstr / (ms * 1e-3);
        if (rc == 0 && (rc = best_ms(st, [&] { dfma_lanes<<<blocks, threads, 0, st>>>(buf, 0.999, 1e-3, 1); }, &ms)) == 0)
            warp1 = winstr / (ms * 1e-3);
    }
    cudaFree(buf);
    if (rc != SWEPT2D_OK) return rc;
    out[0] = fp64;
    if (nout > 1) out[1] = fp32;
    if (nout > 2) out[2] = smem;
    if (nout > 3) out[3] = warp32;
    if (nout > 4) out[4] = warp1;
    return SWEPT2D_OK;
}

extern "C" int swept2d_measure_fp64_rate(void *stream, double *ops_per_s) {
    if (!ops_per_s) return SWEPT2D_EINVAL;
    return swept2d_measure_peaks(stream, ops_per_s, 1);
}
