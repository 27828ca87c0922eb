// FP64 issue-rate measurement for the roofline: independent fused multiply-add
// chains, eight per thread, enough blocks to fill every SM several times.
#include <cuda_runtime.h>

#include "../../include/swept2d.h"

namespace {

constexpr int kIters = 2048;

__global__ void __launch_bounds__(256) dfma_chains(double *out, double a, double b) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x + i;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = __fma_rn(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s = __dadd_rn(s, x[i]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int swept2d_measure_fp64_rate(void *stream, double *ops_per_s) {
    if (!ops_per_s) return SWEPT2D_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    double *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return SWEPT2D_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int rc = SWEPT2D_OK;
    for (int rep = 0; rep < 6 && rc == SWEPT2D_OK; ++rep) {
        cudaEventRecord(e0, st);
        dfma_chains<<<blocks, threads, 0, st>>>(buf, 0.999, 1e-3);
        if (cudaGetLastError() != cudaSuccess) rc = SWEPT2D_ECUDA;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = SWEPT2D_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;   // first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc == SWEPT2D_OK) *ops_per_s = (double)blocks * threads * kIters * 8 / (best * 1e-3);
    return rc;
}
