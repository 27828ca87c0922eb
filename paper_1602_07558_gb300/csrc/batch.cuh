// Batched kernels: many independent periodic grids of uneven sizes advanced
// together, one launch per swept phase (or per naive sub-step) over the tiles
// (or blocks) of every grid. Grids that use the same tile side n form a class;
// a class's launches cover all of its grids' tiles, listed in a tile table
// (tile -> grid). Each block looks up its grid's descriptor and runs the same
// per-tile bodies as the single-grid kernels, on that grid's slice of the
// pooled state and panel buffers.
#pragma once
#include <algorithm>
#include <type_traits>

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

// One persistent launch over every tile class. Every block takes the classes
// in order; within a class its teams (TeamOf<T>: T threads with their own
// barrier and shared-memory slice, or the whole block) each take the class's
// items, one at a time, from the class's own counter, and run them as that
// class's own launch would (its tile table, counters, tile side and number of
// half cycles; the tile side fixed at compile time for 16, 32 and 64). A block
// goes on to the next class once its teams find the class's counter past its
// last item, so the classes overlap at the class boundaries. An item waits
// only for the same class's earlier items, handed out before it and held by
// teams that never wait at a block barrier while they hold an item, so the
// lowest unfinished item can always run, as in one class's launch.
struct ClassRun {
    const int2 *tiles;      // the class's tile table
    int *stage;             // its per-tile item counters, then its item counter (zeroed)
    int ntiles, n, H;       // tiles, tile side, half cycles
};
constexpr int kMaxClassRuns = 16;
// passed by value (a kernel parameter, so a captured graph keeps its own copy)
struct ClassRuns {
    ClassRun r[kMaxClassRuns];
    int count;
};

// Threads of the one-launch kernel's blocks, and the team that runs one item
// of a class with tile side n (0: the whole block). Small tiles, whose levels
// are short, run several per block: heat in binary32 / bfloat16 one warp per
// tile-16 item and four per tile-32 item; the other updates two warps per
// tile-16 item (their tile-16 slice is 4x larger). Larger tiles take the block.
constexpr int kOneLaunchThreads = 256;
template <class Op>
__host__ __device__ constexpr int one_launch_team(int n) {
    if constexpr (std::is_same<Op, HeatKahanOp<float>>::value ||
                  std::is_same<Op, HeatKahanOp<__nv_bfloat16>>::value)
        return n <= 16 ? 32 : (n <= 32 ? 128 : 0);
    else
        return n <= 16 ? 64 : 0;
}
// Shared memory of a one-launch block for a class of tile side n: its teams'
// slices, or one swept block.
template <class Op, bool STG>
inline size_t one_launch_class_smem(int n) {
    const int T = one_launch_team<Op>(n);
    return T ? (size_t)(kOneLaunchThreads / T) * team_slice<Op, STG>(n) : down_smem<Op>(n, STG);
}

template <class Op, bool STG, int NC, class Tm>
__device__ __forceinline__ bool run_class(const GridDesc *grids, const ClassRun &c,
                                          typename Op::S *state, typename Op::S *up,
                                          typename Op::S *br, u64 g0, int *err) {
    __shared__ int s_item[kMaxTeams];
    int &mine = s_item[Tm::index()];
    const int nitems = (int)persistent_items(c.ntiles, c.H);
    int *queue = c.stage + c.ntiles;
    for (;;) {
        if (Tm::rank() == 0) {
            const int it = atomicAdd(queue, 1);
            mine = ld_relaxed(err) ? nitems : it;     // another team's failure ends this one
        }
        Tm::sync();
        const int item = mine;
        if (item >= nitems) return true;
        if (!persistent_item<Op, STG, NC, Tm>(Op(grids[0].c), GridTiles{grids, c.tiles},
                                              c.ntiles, c.n, state, up, br, c.stage, c.H, g0,
                                              err, item, kPersistSpinLimit, nullptr))
            return false;
    }
}

// The team for tile side N (a compile-time case of the class's side)
template <class Op, bool STG, int N>
__device__ __forceinline__ bool run_class_n(const GridDesc *grids, const ClassRun &c,
                                            typename Op::S *state, typename Op::S *up,
                                            typename Op::S *br, u64 g0, int *err) {
    constexpr int NC = FixedTiles<Op>::value ? N : 0;
    constexpr int T = one_launch_team<Op>(N);
    if constexpr (T > 0 && T < kOneLaunchThreads)
        return run_class<Op, STG, NC, TeamOf<T>>(grids, c, state, up, br, g0, err);
    else
        return run_class<Op, STG, NC, BlockTeam>(grids, c, state, up, br, g0, err);
}

template <class Op, bool STG>
__global__ void __launch_bounds__(kOneLaunchThreads) batch_persistent_all_kernel(
    const GridDesc *grids, const ClassRuns runs, typename Op::S *state, typename Op::S *up,
    typename Op::S *br, u64 g0, int *err) {
    for (int k = 0; k < runs.count; ++k) {
        const ClassRun c = runs.r[k];
        bool ok;
        switch (c.n) {
            case 16: ok = run_class_n<Op, STG, 16>(grids, c, state, up, br, g0, err); break;
            case 32: ok = run_class_n<Op, STG, 32>(grids, c, state, up, br, g0, err); break;
            case 64: ok = run_class_n<Op, STG, 64>(grids, c, state, up, br, g0, err); break;
            default:
                ok = run_class<Op, STG, 0, BlockTeam>(grids, c, state, up, br, g0, err);
                break;
        }
        // every team of the block leaves the class before the team shape changes
        if (__syncthreads_or(!ok)) return;
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
    // order, each class's counters and item counter zeroed)
    cudaError_t (*persistent_all)(const GridDesc *, const ClassRuns &runs, long long total_tiles,
                                  void *state, void *up, void *br, u64 g0, int *err,
                                  const Tuning &, cudaStream_t);
    // dynamic shared memory of the one-launch kernel's blocks (largest class)
    size_t (*one_launch_smem)(const int *tile_sides, int count, bool stage);
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
    static size_t one_launch_smem_t(const int *sides, int count) {
        size_t sm = 0;
        for (int i = 0; i < count; ++i) sm = std::max(sm, one_launch_class_smem<Op, STG>(sides[i]));
        return sm;
    }
    static size_t one_launch_smem(const int *sides, int count, bool stage) {
        return stage ? one_launch_smem_t<true>(sides, count) : one_launch_smem_t<false>(sides, count);
    }
    template <bool STG>
    static cudaError_t persistent_all_t(const GridDesc *d, const ClassRuns &runs, long long tiles,
                                        void *state, void *upp, void *br, u64 g0, int *err,
                                        cudaStream_t st) {
        int sides[kMaxClassRuns];
        for (int i = 0; i < runs.count; ++i) sides[i] = runs.r[i].n;
        const size_t sm = one_launch_smem_t<STG>(sides, runs.count);
        const auto kern = batch_persistent_all_kernel<Op, STG>;
        cudaError_t e = allow_smem(kern, sm);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, nsm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOneLaunchThreads,
                                                               sm)) != cudaSuccess)
            return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const long long grid = persistent_grid(per_sm, nsm, tiles, 3 * tiles);
        kern<<<(int)grid, kOneLaunchThreads, sm, st>>>(d, runs, (S *)state, (S *)upp, (S *)br, g0,
                                                       err);
        return cudaGetLastError();
    }
    static cudaError_t persistent_all(const GridDesc *d, const ClassRuns &runs, long long tiles,
                                      void *state, void *upp, void *br, u64 g0, int *err,
                                      const Tuning &tn, cudaStream_t st) {
        return tn.stage ? persistent_all_t<true>(d, runs, tiles, state, upp, br, g0, err, st)
                        : persistent_all_t<false>(d, runs, tiles, state, upp, br, g0, err, st);
    }
    static const BatchTable *table() {
        static const BatchTable t = {Op::NV, Op::NST, (int)sizeof(S), Op::STAGE,
                                     &swept_smem_for<Op>, &naive, &up, &bridge, &octahedron,
                                     &down, &persistent, &persistent_all, &one_launch_smem};
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
