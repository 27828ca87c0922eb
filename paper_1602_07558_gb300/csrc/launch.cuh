// Host-side launchers of the kernels in kernels.cuh, one table per point update.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "kernels.cuh"

namespace swept {

// Function table of one point update (filled in by an instantiation unit).
struct OpTable {
    int nv, nst, esize;
    size_t (*smem_bytes)(int n);   // dynamic shared memory of a swept block with tile n
    cudaError_t (*naive)(const Geom &, const double *c, const void *in, void *out, u64 g,
                         cudaStream_t);
    cudaError_t (*up)(const Geom &, const double *c, const void *state, void *up, int o, u64 g0,
                      cudaStream_t);
    cudaError_t (*bridge)(const Geom &, const double *c, const void *up, void *br, u64 g0,
                          cudaStream_t);
    cudaError_t (*octahedron)(const Geom &, const double *c, const void *br, void *up, int o,
                              u64 g0, cudaStream_t);
    cudaError_t (*down)(const Geom &, const double *c, const void *br, void *state, int o, u64 g0,
                        cudaStream_t);
};

constexpr int kBlock = 256;

template <class Op>
inline size_t swept_smem_bytes(int n) {
    return (size_t)(2 * Op::NV + Op::AUX) * (n + 2) * (n + 2) * sizeof(typename Op::S);
}

// Raise the dynamic shared-memory limit of a kernel when it needs more than
// the default 48 KB (the attribute is per kernel and per device).
template <class K>
inline cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class Op>
struct Launch {
    typedef typename Op::S S;
    static cudaError_t naive(const Geom &G, const double *c, const void *in, void *out, u64 g,
                             cudaStream_t st) {
        if constexpr (std::is_same<Op, HeatOp>::value) {
            // rows per warp: as many as keep about 32 warps per SM in flight
            const long long chunks = (G.nx + 30) / 31;
            int rows = 32;
            while (rows > 1 && chunks * ((G.ny + rows - 1) / rows) < 152LL * 32) rows >>= 1;
            const int warps = (G.ny + rows - 1) / rows;
            dim3 grid((unsigned)chunks, (warps + 7) / 8);
            const Op op(c);
            switch (rows) {
                case 32: naive_heat_kernel<32><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                case 16: naive_heat_kernel<16><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                case 8: naive_heat_kernel<8><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                case 4: naive_heat_kernel<4><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                case 2: naive_heat_kernel<2><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                default: naive_heat_kernel<1><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
            }
        } else {
            dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
            naive_kernel<Op><<<grid, kBlock, 0, st>>>(Op(c), G, (const S *)in, (S *)out, g);
        }
        return cudaGetLastError();
    }
    static cudaError_t up(const Geom &G, const double *c, const void *state, void *up, int o,
                          u64 g0, cudaStream_t st) {
        const size_t sm = swept_smem_bytes<Op>(G.n);
        cudaError_t e = allow_smem(up_kernel<Op>, sm);
        if (e != cudaSuccess) return e;
        up_kernel<Op><<<dim3(G.T, G.Q), kBlock, sm, st>>>(Op(c), G, (const S *)state, (S *)up, o,
                                                          g0);
        return cudaGetLastError();
    }
    static cudaError_t bridge(const Geom &G, const double *c, const void *up, void *br, u64 g0,
                              cudaStream_t st) {
        const size_t sm = swept_smem_bytes<Op>(G.n);
        cudaError_t e = allow_smem(bridge_kernel<Op>, sm);
        if (e != cudaSuccess) return e;
        bridge_kernel<Op><<<dim3(G.T, G.Q, 2), kBlock, sm, st>>>(Op(c), G, (const S *)up, (S *)br,
                                                                 g0);
        return cudaGetLastError();
    }
    static cudaError_t octahedron(const Geom &G, const double *c, const void *br, void *up, int o,
                                  u64 g0, cudaStream_t st) {
        const size_t sm = swept_smem_bytes<Op>(G.n);
        cudaError_t e = allow_smem(octahedron_kernel<Op>, sm);
        if (e != cudaSuccess) return e;
        octahedron_kernel<Op><<<dim3(G.T, G.Q), kBlock, sm, st>>>(Op(c), G, (const S *)br,
                                                                  (S *)up, o, g0);
        return cudaGetLastError();
    }
    static cudaError_t down(const Geom &G, const double *c, const void *br, void *state, int o,
                            u64 g0, cudaStream_t st) {
        const size_t sm = swept_smem_bytes<Op>(G.n);
        cudaError_t e = allow_smem(down_kernel<Op>, sm);
        if (e != cudaSuccess) return e;
        down_kernel<Op><<<dim3(G.T, G.Q), kBlock, sm, st>>>(Op(c), G, (const S *)br, (S *)state,
                                                            o, g0);
        return cudaGetLastError();
    }
    static const OpTable *table() {
        static const OpTable t = {Op::NV, Op::NST, (int)sizeof(S), &swept_smem_bytes<Op>,
                                  &naive, &up, &bridge, &octahedron, &down};
        return &t;
    }
};

// Defined in the instantiation units.
const OpTable *optable_heat();
const OpTable *optable_euler();
const OpTable *optable_increment();
const OpTable *optable_hash();
const OpTable *optable_leveltag();
const OpTable *optable_wide2();

// Euler helpers (euler.cu): the max wave speed of planes 0-3 of a state.
cudaError_t euler_wavespeed(const double *state, int nx, int ny, double gamma,
                            unsigned long long *d_scratch, double *a_out, cudaStream_t st);

}  // namespace swept
