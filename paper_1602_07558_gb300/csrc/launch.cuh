// Host-side launchers of the kernels in kernels.cuh, one table per point update.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "kernels.cuh"

namespace swept {

// Launch shape of the swept kernels: threads per block (64, 128 or 256) and
// whether the bridge and downward-pyramid blocks stage their input panels in
// shared memory by TMA (else they prefetch each level with cp.async).
struct Tuning {
    int threads = 256;
    bool stage = false;
};

// Function table of one point update (filled in by an instantiation unit).
struct OpTable {
    int nv, nst, esize;
    size_t (*smem_bytes)(int n);   // largest dynamic shared memory of a swept block, tile n
    cudaError_t (*naive)(const Geom &, const double *c, const void *in, void *out, u64 g,
                         cudaStream_t);
    cudaError_t (*up)(const Geom &, const double *c, const void *state, void *up, int o, u64 g0,
                      cudaStream_t);
    // err: device word set to nonzero if a bounded wait gave up (may be NULL);
    // tn: launch shape (threads per block, panel staging)
    cudaError_t (*bridge)(const Geom &, const double *c, const void *up, void *br, u64 g0,
                          int *err, const Tuning &tn, cudaStream_t);
    cudaError_t (*octahedron)(const Geom &, const double *c, const void *br, void *up, int o,
                              u64 g0, int *err, const Tuning &tn, cudaStream_t);
    cudaError_t (*down)(const Geom &, const double *c, const void *br, void *state, int o, u64 g0,
                        int *err, const Tuning &tn, cudaStream_t);
    bool default_stage;
    size_t (*smem_for)(int n, bool stage);   // largest swept block's shared memory
    // the whole swept part of an advance (H half cycles) as one persistent
    // launch; sched: T*Q phase counters followed by the queue counter, zeroed
    cudaError_t (*persistent)(const Geom &, const double *c, void *state, void *up, void *br,
                              int *sched, int H, u64 g0, int *err, const Tuning &, int first,
                              long long spin_limit, unsigned *trace, cudaStream_t);
    int max_threads;              // largest block of the launch-per-phase swept kernels
    int max_persistent_threads;   // largest block of the persistent kernel
};

constexpr int kBlock = 256;

// Dynamic shared memory of each swept kernel: the up kernel stages nothing,
// the bridge stages 2 input panels (and packs smaller levels' aux values), the
// octahedron and the final down 4. The persistent kernel takes the largest.
template <class Op>
inline size_t up_smem(int n) { return smem_plan<Op>(n, 0, false).total; }
template <class Op>
inline size_t bridge_smem(int n, bool stage) { return smem_plan<Op>(n, 2, stage, true).total; }
template <class Op>
inline size_t down_smem(int n, bool stage) { return smem_plan<Op>(n, 4, stage).total; }
template <class Op>
inline size_t swept_smem_bytes(int n) { return down_smem<Op>(n, Op::STAGE); }
template <class Op>
inline size_t swept_smem_for(int n, bool stage) { return down_smem<Op>(n, stage); }

// Updates whose swept kernels are also built for fixed tile sides 16, 32 and 64
// (the tile side then a compile-time constant: see fixed_tile). The binary32 /
// bfloat16 forms are bound by instruction issue, where the constant pitches
// save the address arithmetic of every shared-memory access; the FP64 forms
// are bound by the FP64 pipe and keep one instantiation.
template <class Op>
struct FixedTiles : std::false_type {};
template <class SS>
struct FixedTiles<HeatKahanOp<SS>> : std::true_type {};
template <class SS>
struct FixedTiles<EulerKahanOp<SS>> : std::true_type {};

// Calls f(std::integral_constant<int, NC>) with NC = n when the update has an
// instantiation for tile side n, else NC = 0 (tile side read at run time).
template <class Op, class F>
inline cudaError_t with_tile(int n, F &&f) {
    if constexpr (FixedTiles<Op>::value) {
        switch (n) {
            case 16: return f(std::integral_constant<int, 16>());
            case 32: return f(std::integral_constant<int, 32>());
            case 64: return f(std::integral_constant<int, 64>());
            default: break;
        }
    }
    return f(std::integral_constant<int, 0>());
}

// Blocks of a persistent launch: every block that fits at once, but no more
// than 3 per tile (one half cycle's two bridges and octahedron of every tile
// can then run together). The items are handed out in order, so a block
// beyond that would only take an item of a later phase and poll its
// neighbourhood flags, adding traffic to the flags and the queue that the
// items on the critical path wait behind (small grids, where the tiles are
// fewer than the SMs).
inline long long persistent_grid(int per_sm, int nsm, long long ntiles, long long nitems) {
    long long grid = (long long)(per_sm > 0 ? per_sm : 1) * nsm;
    if (grid > 3 * ntiles) grid = 3 * ntiles;
    if (grid > nitems) grid = nitems;
    return grid > 0 ? grid : 1;
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
        } else if constexpr (std::is_same<Op, HeatKahanOp<float>>::value ||
                             std::is_same<Op, HeatKahanOp<__nv_bfloat16>>::value) {
            const long long chunks = (G.nx + 31) / 32;
            int rows = 16;
            while (rows > 1 && chunks * ((G.ny + rows - 1) / rows) < 152LL * 32) rows >>= 1;
            const int warps = (G.ny + rows - 1) / rows;
            dim3 grid((unsigned)chunks, (warps + 7) / 8);
            const Op op(c);
            switch (rows) {
                case 16: naive_heat_kahan_kernel<S, 16><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                case 8: naive_heat_kahan_kernel<S, 8><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                case 4: naive_heat_kahan_kernel<S, 4><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                case 2: naive_heat_kahan_kernel<S, 2><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
                default: naive_heat_kahan_kernel<S, 1><<<grid, kBlock, 0, st>>>(op, G, (const S *)in, (S *)out); break;
            }
        } else {
            dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
            naive_kernel<Op><<<grid, kBlock, 0, st>>>(Op(c), G, (const S *)in, (S *)out, g);
        }
        return cudaGetLastError();
    }
    static cudaError_t up(const Geom &G, const double *c, const void *state, void *up, int o,
                          u64 g0, cudaStream_t st) {
        const size_t sm = up_smem<Op>(G.n);
        return with_tile<Op>(G.n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            cudaError_t e = allow_smem(up_kernel<Op, NC>, sm);
            if (e != cudaSuccess) return e;
            up_kernel<Op, NC><<<dim3(G.T, G.Q), kBlock, sm, st>>>(Op(c), G, (const S *)state,
                                                                  (S *)up, o, g0);
            return cudaGetLastError();
        });
    }
    template <bool STG>
    static cudaError_t bridge_t(const Geom &G, const double *c, const void *up, void *br, u64 g0,
                                int *err, int threads, cudaStream_t st) {
        const size_t sm = bridge_smem<Op>(G.n, STG);
        return with_tile<Op>(G.n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            cudaError_t e = allow_smem(bridge_kernel<Op, STG, NC>, sm);
            if (e != cudaSuccess) return e;
            bridge_kernel<Op, STG, NC><<<dim3(G.T, G.Q, 2), threads, sm, st>>>(
                Op(c), G, (const S *)up, (S *)br, g0, err);
            return cudaGetLastError();
        });
    }
    // A bridge's levels are thin rectangles (W + H = n), and its block is
    // smaller than a pyramid's, so bridges take at most 256 threads (128 for
    // the wave update): more, smaller blocks share an SM (the 4096² FP64 heat
    // bridge at n = 64: five blocks of 256 per SM, 1.44 ms per launch, against
    // four of 512, 1.48 ms; the 1024² wave bridge at n = 32: 82 against 86 µs
    // with 128 threads; the Euler bridges measured slower at 128).
    static constexpr int kMaxBridgeThreads = std::is_same<Op, WaveOp>::value ? 128 : 256;
    static cudaError_t bridge(const Geom &G, const double *c, const void *up, void *br, u64 g0,
                              int *err, const Tuning &tn, cudaStream_t st) {
        const int thr = tn.threads > kMaxBridgeThreads ? kMaxBridgeThreads : tn.threads;
        return tn.stage ? bridge_t<true>(G, c, up, br, g0, err, thr, st)
                        : bridge_t<false>(G, c, up, br, g0, err, thr, st);
    }
    template <bool STG>
    static cudaError_t octahedron_t(const Geom &G, const double *c, const void *br, void *up,
                                    int o, u64 g0, int *err, int threads, cudaStream_t st) {
        const size_t sm = down_smem<Op>(G.n, STG);
        return with_tile<Op>(G.n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            cudaError_t e = allow_smem(octahedron_kernel<Op, STG, NC>, sm);
            if (e != cudaSuccess) return e;
            octahedron_kernel<Op, STG, NC><<<dim3(G.T, G.Q), threads, sm, st>>>(
                Op(c), G, (const S *)br, (S *)up, o, g0, err);
            return cudaGetLastError();
        });
    }
    static cudaError_t octahedron(const Geom &G, const double *c, const void *br, void *up, int o,
                                  u64 g0, int *err, const Tuning &tn, cudaStream_t st) {
        return tn.stage ? octahedron_t<true>(G, c, br, up, o, g0, err, tn.threads, st)
                        : octahedron_t<false>(G, c, br, up, o, g0, err, tn.threads, st);
    }
    template <bool STG>
    static cudaError_t down_t(const Geom &G, const double *c, const void *br, void *state, int o,
                              u64 g0, int *err, int threads, cudaStream_t st) {
        const size_t sm = down_smem<Op>(G.n, STG);
        return with_tile<Op>(G.n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            cudaError_t e = allow_smem(down_kernel<Op, STG, NC>, sm);
            if (e != cudaSuccess) return e;
            down_kernel<Op, STG, NC><<<dim3(G.T, G.Q), threads, sm, st>>>(
                Op(c), G, (const S *)br, (S *)state, o, g0, err);
            return cudaGetLastError();
        });
    }
    static cudaError_t down(const Geom &G, const double *c, const void *br, void *state, int o,
                            u64 g0, int *err, const Tuning &tn, cudaStream_t st) {
        return tn.stage ? down_t<true>(G, c, br, state, o, g0, err, tn.threads, st)
                        : down_t<false>(G, c, br, state, o, g0, err, tn.threads, st);
    }
    template <bool STG>
    static cudaError_t persistent_t(const Geom &G, const double *c, void *state, void *upp,
                                    void *br, int *sched, int H, u64 g0, int *err, int threads,
                                    int first, long long spin_limit, unsigned *trace,
                                    cudaStream_t st) {
        const size_t sm = down_smem<Op>(G.n, STG);
        return with_tile<Op>(G.n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            const auto kern = persistent_kernel<Op, STG, NC>;
            cudaError_t e = allow_smem(kern, sm);
            if (e != cudaSuccess) return e;
            int per_sm = 0, dev = 0, nsm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm)) !=
                cudaSuccess)
                return e;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            const int NT = G.T * G.Q;
            const long long grid = persistent_grid(per_sm, nsm, NT, persistent_items(NT, H));
            kern<<<(int)grid, threads, sm, st>>>(Op(c), G, (S *)state, (S *)upp, (S *)br, sched,
                                                 sched + NT, H, g0, err, first, spin_limit, trace);
            return cudaGetLastError();
        });
    }
    static cudaError_t persistent(const Geom &G, const double *c, void *state, void *upp,
                                  void *br, int *sched, int H, u64 g0, int *err,
                                  const Tuning &tn, int first, long long spin_limit,
                                  unsigned *trace, cudaStream_t st) {
        return tn.stage ? persistent_t<true>(G, c, state, upp, br, sched, H, g0, err, tn.threads,
                                             first, spin_limit, trace, st)
                        : persistent_t<false>(G, c, state, upp, br, sched, H, g0, err, tn.threads,
                                              first, spin_limit, trace, st);
    }
    static const OpTable *table() {
        static const OpTable t = {Op::NV,      Op::NST,     (int)sizeof(S), &swept_smem_bytes<Op>,
                                  &naive,      &up,         &bridge,        &octahedron,
                                  &down,       Op::STAGE,   &swept_smem_for<Op>, &persistent,
                                  SweptBounds<Op>::kThreads, kMaxPersistentThreads};
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
const OpTable *optable_wave();
const OpTable *optable_heat_kahan_f32();
const OpTable *optable_heat_kahan_bf16();
const OpTable *optable_euler_kahan_f32();
const OpTable *optable_euler_kahan_bf16();

// Euler helper (op_euler.cu): the max wave speed of planes 0-3 of a state whose
// elements are esize bytes (8 binary64, 4 binary32, 2 bfloat16).
cudaError_t euler_wavespeed(const void *state, int esize, int nx, int ny, double gamma,
                            unsigned long long *d_scratch, double *a_out, cudaStream_t st);

}  // namespace swept
