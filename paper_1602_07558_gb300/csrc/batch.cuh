// Batched kernels: many independent periodic grids of uneven sizes advanced
// together, one launch per swept phase (or per naive sub-step) over the tiles
// (or blocks) of every grid. Grids that use the same tile side n form a class;
// a class's launches cover all of its grids' tiles, listed in a tile table
// (tile -> grid). Each block looks up its grid's descriptor and runs the same
// per-tile bodies as the single-grid kernels, on that grid's slice of the
// pooled state and panel buffers.
#pragma once
#include "launch.cuh"

namespace swept {

struct GridDesc {
    Geom G;                 // the grid's geometry (tile side n of its class)
    long long state_off;    // first element of the grid's state in the pooled state
    long long panel_off;    // first element of the grid's panel slots in each pool
    double c[8];            // the point update's constants for this grid (Euler's
                            // depend on the grid's own state and spacing)
};
// Tile and block tables hold (grid index, tile or block index within the grid).

// NC > 0: every grid of the launch's class has tile side NC (see fixed_tile).
template <class Op, int NC = 0>
__global__ void __launch_bounds__(kMaxSweptThreads) batch_up_kernel(const GridDesc *grids,
                                                                    const int2 *tile_grid,
                                                                    const typename Op::S *state,
                                                                    typename Op::S *up, int o,
                                                                    u64 g0) {
    const int2 e = tile_grid[blockIdx.x];
    const GridDesc gd = grids[e.x];
    const int J = e.y / gd.G.T, I = e.y - J * gd.G.T;
    up_tile(Op(gd.c), fixed_tile<NC>(gd.G), state + gd.state_off, up + gd.panel_off, o, g0, I, J);
}

template <class Op, bool STG, int NC = 0>
__global__ void __launch_bounds__(kMaxSweptThreads) batch_bridge_kernel(const GridDesc *grids,
                                                                        const int2 *tile_grid,
                                                                        const typename Op::S *up,
                                                                        typename Op::S *br, u64 g0,
                                                                        int *err) {
    const int2 e = tile_grid[blockIdx.x];
    const GridDesc gd = grids[e.x];
    const int J = e.y / gd.G.T, I = e.y - J * gd.G.T;
    bridge_tile<Op, STG>(Op(gd.c), fixed_tile<NC>(gd.G), up + gd.panel_off, br + gd.panel_off,
                         g0, err, I, J, blockIdx.y == 1);
}

template <class Op, bool STG, int NC = 0>
__global__ void __launch_bounds__(kMaxSweptThreads) batch_octahedron_kernel(
    const GridDesc *grids, const int2 *tile_grid, const typename Op::S *br, typename Op::S *up,
    int o, u64 g0, int *err) {
    const int2 e = tile_grid[blockIdx.x];
    const GridDesc gd = grids[e.x];
    const int J = e.y / gd.G.T, I = e.y - J * gd.G.T;
    octahedron_tile<Op, STG>(Op(gd.c), fixed_tile<NC>(gd.G), br + gd.panel_off,
                             up + gd.panel_off, o, g0, err, I, J);
}

template <class Op, bool STG, int NC = 0>
__global__ void __launch_bounds__(kMaxSweptThreads) batch_down_kernel(
    const GridDesc *grids, const int2 *tile_grid, const typename Op::S *br, typename Op::S *state,
    int o, u64 g0, int *err) {
    const int2 e = tile_grid[blockIdx.x];
    const GridDesc gd = grids[e.x];
    const int J = e.y / gd.G.T, I = e.y - J * gd.G.T;
    down_tile<Op, STG>(Op(gd.c), fixed_tile<NC>(gd.G), br + gd.panel_off, state + gd.state_off,
                       o, g0, err, I, J);
}

// Persistent form over every tile of a class: the tile table lists each
// grid's tiles consecutively, so a grid's phase counters start at the table
// index of its tile 0.
struct GridTiles {
    const GridDesc *grids;
    const int2 *tiles;
    __device__ __forceinline__ TileAt operator()(int t) const {
        const int2 e = tiles[t];
        const GridDesc gd = grids[e.x];
        TileAt w;
        w.G = gd.G;
        w.soff = gd.state_off;
        w.poff = gd.panel_off;
        w.J = e.y / gd.G.T;
        w.I = e.y - w.J * gd.G.T;
        w.base = t - e.y;
        w.c = grids[e.x].c;
        return w;
    }
};

template <class Op, bool STG, int NC = 0>
__global__ void __launch_bounds__(256) batch_persistent_kernel(
    const GridDesc *grids, const int2 *tile_grid, int ntiles, int n, typename Op::S *state,
    typename Op::S *up, typename Op::S *br, int *stage, int *queue, int H, u64 g0, int *err) {
    // the update's constants come from each item's grid (TileAt::c)
    persistent_loop<Op, STG, NC>(Op(grids[0].c), GridTiles{grids, tile_grid}, ntiles, n, state,
                                 up, br, stage, queue, H, g0, err, 0, kPersistSpinLimit);
}

// One persistent launch over every tile class: each class's items (its own tile
// table, counters, tile side and number of half cycles) follow the previous
// class's in one order, handed out by a 64-bit counter. A class's items depend
// only on that class's earlier items, all handed out before them, so the
// lowest unfinished item can always run, as in one class's launch; the
// classes overlap where one class's last phases and the next one's first
// items share the GPU.
struct ClassRun {
    const int2 *tiles;      // the class's tile table
    int *stage;             // its per-tile item counters (zeroed)
    int ntiles, n, H;       // tiles, tile side, half cycles
    long long first;        // its first item in the launch's order
};
constexpr int kMaxClassRuns = 16;
// passed by value (a kernel parameter, so a captured graph keeps its own copy)
struct ClassRuns {
    ClassRun r[kMaxClassRuns];
    int count;
};

template <class Op, bool STG, int NC>
__device__ __forceinline__ bool class_item(const GridDesc *grids, const ClassRun &c,
                                           typename Op::S *state, typename Op::S *up,
                                           typename Op::S *br, u64 g0, int *err, int item) {
    return persistent_item<Op, STG, NC>(Op(grids[0].c), GridTiles{grids, c.tiles}, c.ntiles, c.n,
                                        state, up, br, c.stage, c.H, g0, err, item,
                                        kPersistSpinLimit, nullptr);
}

template <class Op, bool STG>
__global__ void __launch_bounds__(256) batch_persistent_all_kernel(
    const GridDesc *grids, const ClassRuns runs, long long nitems, typename Op::S *state,
    typename Op::S *up, typename Op::S *br, unsigned long long *queue, u64 g0, int *err) {
    __shared__ long long s_item;
    __shared__ ClassRun s_run;
    for (;;) {
        if (threadIdx.x == 0) {
            long long it = (long long)atomicAdd(queue, 1ULL);
            if (ld_relaxed(err)) it = nitems;        // another block's failure ends this one
            int c = 0;
            while (c + 1 < runs.count && it >= runs.r[c + 1].first) ++c;
            s_item = it;
            s_run = runs.r[c];
        }
        __syncthreads();
        const long long it = s_item;
        if (it >= nitems) return;
        const ClassRun c = s_run;
        const int item = (int)(it - c.first);
        bool ok;
        if constexpr (FixedTiles<Op>::value) {
            switch (c.n) {
                case 16: ok = class_item<Op, STG, 16>(grids, c, state, up, br, g0, err, item); break;
                case 32: ok = class_item<Op, STG, 32>(grids, c, state, up, br, g0, err, item); break;
                case 64: ok = class_item<Op, STG, 64>(grids, c, state, up, br, g0, err, item); break;
                default: ok = class_item<Op, STG, 0>(grids, c, state, up, br, g0, err, item); break;
            }
        } else {
            ok = class_item<Op, STG, 0>(grids, c, state, up, br, g0, err, item);
        }
        if (!ok) return;
    }
}

// One sub-step of every grid in a block table: block b covers a 32 x 8 patch of
// its grid (the same per-point update as the single-grid naive kernel).
template <class Op>
__global__ void __launch_bounds__(256) batch_naive_kernel(const GridDesc *grids,
                                                          const int2 *block_grid,
                                                          const typename Op::S *in,
                                                          typename Op::S *out, u64 g) {
    typedef typename Op::S S;
    const int2 e = block_grid[blockIdx.x];
    const GridDesc gd = grids[e.x];
    const Op op(gd.c);
    const int nbx = (gd.G.nx + 31) / 32;
    const int by = e.y / nbx, bx = e.y - by * nbx;
    const int x = bx * 32 + (threadIdx.x & 31);
    const int y = by * 8 + (threadIdx.x >> 5);
    if (x >= gd.G.nx || y >= gd.G.ny) return;
    const size_t plane = (size_t)gd.G.nx * gd.G.ny;
    GlobalAcc<S> acc(in + gd.state_off, plane, gd.G.nx, gd.G.ny, x, y);
    S res[Op::NV];
    op((int)(g % Op::NST), g, acc, res);
    S *o = out + gd.state_off + (size_t)y * gd.G.nx + x;
#pragma unroll
    for (int v = 0; v < Op::NV; ++v) o[v * plane] = res[v];
}

// Launch functions of one point update for the batch.
struct BatchTable {
    int nv, nst, esize;
    bool default_stage;
    size_t (*smem_for)(int n, bool stage);
    // (every kernel takes its grid's constants from the grid table)
    cudaError_t (*naive)(const GridDesc *, const int2 *block_grid, int nblocks, const void *in,
                         void *out, u64 g, cudaStream_t);
    cudaError_t (*up)(const GridDesc *, const int2 *tile_grid, int ntiles, int n,
                      const void *state, void *up, int o, u64 g0, cudaStream_t);
    cudaError_t (*bridge)(const GridDesc *, const int2 *tile_grid, int ntiles, int n,
                          const void *up, void *br, u64 g0, int *err, const Tuning &,
                          cudaStream_t);
    cudaError_t (*octahedron)(const GridDesc *, const int2 *tile_grid, int ntiles, int n,
                              const void *br, void *up, int o, u64 g0, int *err, const Tuning &,
                              cudaStream_t);
    cudaError_t (*down)(const GridDesc *, const int2 *tile_grid, int ntiles, int n,
                        const void *br, void *state, int o, u64 g0, int *err, const Tuning &,
                        cudaStream_t);
    // all H half cycles of a class as one persistent launch; sched: ntiles
    // phase counters followed by the queue counter, zeroed
    cudaError_t (*persistent)(const GridDesc *, const int2 *tile_grid, int ntiles, int n,
                              void *state, void *up, void *br, int *sched, int H, u64 g0,
                              int *err, const Tuning &, cudaStream_t);
    // every class's half cycles as one persistent launch (runs: the classes in
    // item order, counters zeroed; queue: 64-bit counter, zeroed)
    cudaError_t (*persistent_all)(const GridDesc *, const ClassRuns &runs, long long nitems,
                                  long long total_tiles, int max_n, void *state, void *up,
                                  void *br, unsigned long long *queue, u64 g0, int *err,
                                  const Tuning &, cudaStream_t);
};

template <class Op>
struct BatchLaunch {
    typedef typename Op::S S;
    static cudaError_t naive(const GridDesc *d, const int2 *bg, int nblocks, const void *in,
                             void *out, u64 g, cudaStream_t st) {
        batch_naive_kernel<Op><<<nblocks, kBlock, 0, st>>>(d, bg, (const S *)in, (S *)out, g);
        return cudaGetLastError();
    }
    static cudaError_t up(const GridDesc *d, const int2 *tg, int ntiles, int n, const void *state,
                          void *upp, int o, u64 g0, cudaStream_t st) {
        const size_t sm = up_smem<Op>(n);
        return with_tile<Op>(n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            cudaError_t e = allow_smem(batch_up_kernel<Op, NC>, sm);
            if (e != cudaSuccess) return e;
            batch_up_kernel<Op, NC><<<ntiles, kBlock, sm, st>>>(d, tg, (const S *)state, (S *)upp,
                                                                o, g0);
            return cudaGetLastError();
        });
    }
    template <bool STG>
    static cudaError_t bridge_t(const GridDesc *d, const int2 *tg, int ntiles, int n,
                                const void *upp, void *br, u64 g0, int *err, int threads,
                                cudaStream_t st) {
        const size_t sm = bridge_smem<Op>(n, STG);
        return with_tile<Op>(n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            cudaError_t e = allow_smem(batch_bridge_kernel<Op, STG, NC>, sm);
            if (e != cudaSuccess) return e;
            batch_bridge_kernel<Op, STG, NC><<<dim3(ntiles, 2), threads, sm, st>>>(
                d, tg, (const S *)upp, (S *)br, g0, err);
            return cudaGetLastError();
        });
    }
    static cudaError_t bridge(const GridDesc *d, const int2 *tg, int ntiles, int n,
                              const void *upp, void *br, u64 g0, int *err, const Tuning &tn,
                              cudaStream_t st) {
        return tn.stage ? bridge_t<true>(d, tg, ntiles, n, upp, br, g0, err, tn.threads, st)
                        : bridge_t<false>(d, tg, ntiles, n, upp, br, g0, err, tn.threads, st);
    }
    template <bool STG>
    static cudaError_t oct_t(const GridDesc *d, const int2 *tg, int ntiles, int n, const void *br,
                             void *upp, int o, u64 g0, int *err, int threads, cudaStream_t st) {
        const size_t sm = down_smem<Op>(n, STG);
        return with_tile<Op>(n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            cudaError_t e = allow_smem(batch_octahedron_kernel<Op, STG, NC>, sm);
            if (e != cudaSuccess) return e;
            batch_octahedron_kernel<Op, STG, NC><<<ntiles, threads, sm, st>>>(
                d, tg, (const S *)br, (S *)upp, o, g0, err);
            return cudaGetLastError();
        });
    }
    static cudaError_t octahedron(const GridDesc *d, const int2 *tg, int ntiles, int n,
                                  const void *br, void *upp, int o, u64 g0, int *err,
                                  const Tuning &tn, cudaStream_t st) {
        return tn.stage ? oct_t<true>(d, tg, ntiles, n, br, upp, o, g0, err, tn.threads, st)
                        : oct_t<false>(d, tg, ntiles, n, br, upp, o, g0, err, tn.threads, st);
    }
    template <bool STG>
    static cudaError_t down_t(const GridDesc *d, const int2 *tg, int ntiles, int n, const void *br,
                              void *state, int o, u64 g0, int *err, int threads, cudaStream_t st) {
        const size_t sm = down_smem<Op>(n, STG);
        return with_tile<Op>(n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            cudaError_t e = allow_smem(batch_down_kernel<Op, STG, NC>, sm);
            if (e != cudaSuccess) return e;
            batch_down_kernel<Op, STG, NC><<<ntiles, threads, sm, st>>>(d, tg, (const S *)br,
                                                                        (S *)state, o, g0, err);
            return cudaGetLastError();
        });
    }
    static cudaError_t down(const GridDesc *d, const int2 *tg, int ntiles, int n, const void *br,
                            void *state, int o, u64 g0, int *err, const Tuning &tn,
                            cudaStream_t st) {
        return tn.stage ? down_t<true>(d, tg, ntiles, n, br, state, o, g0, err, tn.threads, st)
                        : down_t<false>(d, tg, ntiles, n, br, state, o, g0, err, tn.threads, st);
    }
    template <bool STG>
    static cudaError_t persistent_t(const GridDesc *d, const int2 *tg, int ntiles, int n,
                                    void *state, void *upp, void *br, int *sched, int H, u64 g0,
                                    int *err, int threads, cudaStream_t st) {
        const size_t sm = down_smem<Op>(n, STG);
        return with_tile<Op>(n, [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            const auto kern = batch_persistent_kernel<Op, STG, NC>;
            cudaError_t e = allow_smem(kern, sm);
            if (e != cudaSuccess) return e;
            int per_sm = 0, dev = 0, nsm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm)) !=
                cudaSuccess)
                return e;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            const long long grid =
                persistent_grid(per_sm, nsm, ntiles, persistent_items(ntiles, H));
            kern<<<(int)grid, threads, sm, st>>>(d, tg, ntiles, n, (S *)state, (S *)upp, (S *)br,
                                                 sched, sched + ntiles, H, g0, err);
            return cudaGetLastError();
        });
    }
    static cudaError_t persistent(const GridDesc *d, const int2 *tg, int ntiles, int n,
                                  void *state, void *upp, void *br, int *sched, int H, u64 g0,
                                  int *err, const Tuning &tn, cudaStream_t st) {
        return tn.stage ? persistent_t<true>(d, tg, ntiles, n, state, upp, br, sched, H, g0, err,
                                             tn.threads, st)
                        : persistent_t<false>(d, tg, ntiles, n, state, upp, br, sched, H, g0,
                                              err, tn.threads, st);
    }
    template <bool STG>
    static cudaError_t persistent_all_t(const GridDesc *d, const ClassRuns &runs,
                                        long long nitems, long long tiles, int max_n,
                                        void *state, void *upp, void *br,
                                        unsigned long long *queue, u64 g0, int *err, int threads,
                                        cudaStream_t st) {
        const size_t sm = down_smem<Op>(max_n, STG);   // the largest class's block
        const auto kern = batch_persistent_all_kernel<Op, STG>;
        cudaError_t e = allow_smem(kern, sm);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, nsm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm)) !=
            cudaSuccess)
            return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const long long grid = persistent_grid(per_sm, nsm, tiles, nitems);
        kern<<<(int)grid, threads, sm, st>>>(d, runs, nitems, (S *)state, (S *)upp, (S *)br,
                                             queue, g0, err);
        return cudaGetLastError();
    }
    static cudaError_t persistent_all(const GridDesc *d, const ClassRuns &runs, long long nitems,
                                      long long tiles, int max_n, void *state, void *upp,
                                      void *br, unsigned long long *queue, u64 g0, int *err,
                                      const Tuning &tn, cudaStream_t st) {
        return tn.stage ? persistent_all_t<true>(d, runs, nitems, tiles, max_n, state, upp, br,
                                                 queue, g0, err, tn.threads, st)
                        : persistent_all_t<false>(d, runs, nitems, tiles, max_n, state, upp, br,
                                                  queue, g0, err, tn.threads, st);
    }
    static const BatchTable *table() {
        static const BatchTable t = {Op::NV, Op::NST, (int)sizeof(S), Op::STAGE,
                                     &swept_smem_for<Op>, &naive, &up, &bridge, &octahedron,
                                     &down, &persistent, &persistent_all};
        return &t;
    }
};

const BatchTable *batchtable_heat();
const BatchTable *batchtable_heat_kahan_f32();
const BatchTable *batchtable_heat_kahan_bf16();
const BatchTable *batchtable_hash();
const BatchTable *batchtable_euler();
const BatchTable *batchtable_euler_kahan_f32();
const BatchTable *batchtable_euler_kahan_bf16();

// Maximum wave speed of planes 0-3 of every grid of a pooled state whose
// elements are esize bytes, into d_out[grid] (bit patterns of positive doubles).
cudaError_t batch_euler_wavespeed(const GridDesc *d_grids, int count, const void *state,
                                  int esize, double gamma, unsigned long long *d_out,
                                  cudaStream_t st);

}  // namespace swept
