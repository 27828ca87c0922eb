// C ABI of the batched form (declared in include/swept2d.h): many independent
// periodic grids of uneven sizes, all advanced by the same number of steps.
//
// Grids that share a tile side n form a class. For each class the schedule of
// one swept advance is the single-grid one (Up, then per half cycle the bridge
// launch and the octahedron, a final Down, a naive tail), each launch covering
// every tile of every grid of the class. Grids created with tile 0 only ever
// take naive steps. A naive tail with an odd number of sub-steps ends in the
// second state copy, from which the class's grids are copied back, so the
// pooled state stays in the first copy between calls.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/swept2d.h"
#include "batch.cuh"

using swept::BatchTable;
using swept::GridDesc;

namespace {

struct BatchClass {
    int n = 0;                 // tile side (0: naive-only grids)
    swept::Tuning tune;        // launch shape of this class's swept kernels
    std::vector<int> members;  // grid indices
    std::vector<int2> tiles;   // (grid, tile) for the swept launches
    std::vector<int2> blocks;  // (grid, 32x8 block) for the naive tail
    int2 *d_tiles = nullptr, *d_blocks = nullptr;
    int *d_sched = nullptr;    // persistent form: phase counters + queue counter
};

struct BatchGraph {
    long long nsteps;
    int mode;
    void *state;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    long long kernels;
    bool swaps_state;
};

thread_local std::string g_batch_create_err;

}  // namespace

struct swept2d_batch {
    int count = 0, op = 0, dtype = 0;
    const BatchTable *bt = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<GridDesc> grids;
    GridDesc *d_grids = nullptr;
    std::vector<BatchClass> classes;
    std::vector<int2> all_blocks;
    int2 *d_all_blocks = nullptr;
    void *state = nullptr, *state2 = nullptr, *up = nullptr, *br = nullptr;
    size_t state_bytes = 0, panel_bytes = 0;
    long long cells = 0;
    int *errword = nullptr;
    double consts[8] = {0};
    double params[8] = {0};
    int nparams = 0;
    std::vector<double> wavespeed, dt;          // Euler: per grid, fixed at set_state
    unsigned long long *d_amax = nullptr;       // Euler: per-grid wave-speed scratch
    long long substeps = 0, launches = 0;
    bool has_state = false;
    swept::Tuning tune;
    std::vector<BatchGraph> graphs;
    std::string err;
};

namespace {

int bfail(swept2d_batch *b, int code, const std::string &msg) {
    if (b) b->err = msg;
    return code;
}
int bcuda(swept2d_batch *b, cudaError_t e, const char *where) {
    return bfail(b, SWEPT2D_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

const BatchTable *batch_table(int op, int dtype) {
    if (op == SWEPT2D_OP_HEAT && dtype == SWEPT2D_F64) return swept::batchtable_heat();
    if (op == SWEPT2D_OP_HEAT_KAHAN && dtype == SWEPT2D_F32) return swept::batchtable_heat_kahan_f32();
    if (op == SWEPT2D_OP_HEAT_KAHAN && dtype == SWEPT2D_BF16) return swept::batchtable_heat_kahan_bf16();
    if (op == SWEPT2D_OP_HASH && dtype == SWEPT2D_U64) return swept::batchtable_hash();
    if (op == SWEPT2D_OP_EULER_RK2 && dtype == SWEPT2D_F64) return swept::batchtable_euler();
    if (op == SWEPT2D_OP_EULER_KAHAN && dtype == SWEPT2D_F32) return swept::batchtable_euler_kahan_f32();
    if (op == SWEPT2D_OP_EULER_KAHAN && dtype == SWEPT2D_BF16)
        return swept::batchtable_euler_kahan_bf16();
    return nullptr;
}

void batch_free(swept2d_batch *b) {
    for (auto &c : b->classes) {
        if (c.d_tiles) cudaFree(c.d_tiles);
        if (c.d_blocks) cudaFree(c.d_blocks);
        if (c.d_sched) cudaFree(c.d_sched);
    }
    for (void *p : {(void *)b->d_grids, (void *)b->d_all_blocks, b->state, b->state2, b->up, b->br,
                    (void *)b->errword, (void *)b->d_amax})
        if (p) cudaFree(p);
    for (auto &g : b->graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaGraphDestroy(g.graph);
    }
}

template <class F>
int blaunch(swept2d_batch *b, const char *what, F &&f) {
    cudaError_t e = f();
    if (e != cudaSuccess) return bcuda(b, e, what);
    b->launches += 1;
    return SWEPT2D_OK;
}

// `count` naive sub-steps of one block table from `cur` ping-ponging with
// `other`; returns (through *cur) where the result is.
int batch_naive(swept2d_batch *b, const int2 *d_blocks, int nblocks, long long count, u64 g,
                void **cur, void **other) {
    for (long long s = 0; s < count; ++s) {
        void *in = *cur, *out = *other;
        int rc = blaunch(b, "batched naive kernel", [&] {
            return b->bt->naive(b->d_grids, d_blocks, nblocks, in, out, g + s, b->stream);
        });
        if (rc) return rc;
        std::swap(*cur, *other);
    }
    return SWEPT2D_OK;
}

// The one-launch persistent form's tile sides (classes that take swept steps)
// and its staging: the batch-wide tuning's (swept2d_batch_set_tuning), dropped
// if the staged blocks do not fit. Returns false if not even unstaged blocks
// fit.
bool one_launch_shape(const swept2d_batch *b, bool *stage, long long *tiles) {
    int sides[swept::kMaxClassRuns], count = 0;
    *tiles = 0;
    for (const auto &c : b->classes)
        if (c.n && count < swept::kMaxClassRuns) {
            sides[count++] = c.n;
            *tiles += (long long)c.tiles.size();
        }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    *stage = b->tune.stage && b->bt->one_launch_smem(sides, count, true) <= (size_t)optin;
    return b->bt->one_launch_smem(sides, count, *stage) <= (size_t)optin;
}

int batch_run(swept2d_batch *b, long long total, int mode) {
    const bool persistent = (mode & SWEPT2D_PERSISTENT) != 0;
    const bool one_launch = (mode & SWEPT2D_ONE_LAUNCH) != 0;
    mode &= ~(SWEPT2D_PERSISTENT | SWEPT2D_ONE_LAUNCH);
    const u64 g_start = (u64)b->substeps;
    if (mode == SWEPT2D_NAIVE) {
        void *cur = b->state, *other = b->state2;
        int rc = batch_naive(b, b->d_all_blocks, (int)b->all_blocks.size(), total, g_start, &cur,
                             &other);
        if (rc) return rc;
        b->state = cur;
        b->state2 = other;
        b->substeps += total;
        return SWEPT2D_OK;
    }
    if (persistent && one_launch) {
        // every class's half cycles in one launch; the tails follow per class
        swept::ClassRuns runs{};
        for (auto &c : b->classes) {
            const long long H = c.n > 0 ? total / (c.n / 2) : 0;
            if (H <= 0) continue;
            const int nt = (int)c.tiles.size();
            cudaError_t e = cudaMemsetAsync(c.d_sched, 0, ((size_t)nt + 1) * sizeof(int), b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "persistent schedule reset");
            swept::ClassRun &r = runs.r[runs.count++];
            r.tiles = c.d_tiles;
            r.stage = c.d_sched;
            r.ntiles = nt;
            r.n = c.n;
            r.H = (int)H;
        }
        if (runs.count > 0) {
            bool stage = false;
            long long tiles = 0;
            one_launch_shape(b, &stage, &tiles);
            swept::Tuning tn = b->tune;
            tn.stage = stage;
            int rc = blaunch(b, "batched one-launch persistent kernel", [&] {
                return b->bt->persistent_all(b->d_grids, runs, tiles, b->state, b->up, b->br,
                                             g_start, b->errword, tn, b->stream);
            });
            if (rc) return rc;
        }
    }
    for (auto &c : b->classes) {
        long long H = 0, rem = total;
        if (c.n > 0) {
            const int half = c.n / 2;
            H = total / half;
            rem = total - H * half;
        }
        const int nt = (int)c.tiles.size();
        if (H > 0 && persistent && one_launch) {
            // (run above, with every other class)
        } else if (H > 0 && persistent) {
            cudaError_t e = cudaMemsetAsync(c.d_sched, 0, ((size_t)nt + 1) * sizeof(int), b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "persistent schedule reset");
            int rc = blaunch(b, "batched persistent kernel", [&] {
                return b->bt->persistent(b->d_grids, c.d_tiles, nt, c.n, b->state, b->up, b->br,
                                         c.d_sched, (int)H, g_start, b->errword, c.tune,
                                         b->stream);
            });
            if (rc) return rc;
        } else if (H > 0) {
            const int half = c.n / 2;
            int rc = blaunch(b, "batched up kernel", [&] {
                return b->bt->up(b->d_grids, c.d_tiles, nt, c.n, b->state, b->up, 0, g_start,
                                 b->stream);
            });
            if (rc) return rc;
            for (long long j = 0; j < H; ++j) {
                const u64 g0 = g_start + (u64)j * half;
                const int o = (j & 1) ? half : 0;
                rc = blaunch(b, "batched bridge kernel", [&] {
                    return b->bt->bridge(b->d_grids, c.d_tiles, nt, c.n, b->up, b->br, g0,
                                         b->errword, c.tune, b->stream);
                });
                if (rc) return rc;
                if (j + 1 < H)
                    rc = blaunch(b, "batched octahedron kernel", [&] {
                        return b->bt->octahedron(b->d_grids, c.d_tiles, nt, c.n, b->br, b->up, o,
                                                 g0, b->errword, c.tune, b->stream);
                    });
                else
                    rc = blaunch(b, "batched down kernel", [&] {
                        return b->bt->down(b->d_grids, c.d_tiles, nt, c.n, b->br, b->state, o, g0,
                                           b->errword, c.tune, b->stream);
                    });
                if (rc) return rc;
            }
        }
        if (rem > 0) {
            void *cur = b->state, *other = b->state2;
            const u64 gt = g_start + (u64)(total - rem);
            int rc = batch_naive(b, c.d_blocks, (int)c.blocks.size(), rem, gt, &cur, &other);
            if (rc) return rc;
            if (cur != b->state) {   // odd tail: bring the class's grids back
                for (int gi : c.members) {
                    const GridDesc &gd = b->grids[gi];
                    const size_t bytes = (size_t)b->bt->nv * gd.G.nx * gd.G.ny * b->bt->esize;
                    const size_t off = (size_t)gd.state_off * b->bt->esize;
                    cudaError_t e = cudaMemcpyAsync((char *)b->state + off, (char *)cur + off, bytes,
                                                    cudaMemcpyDeviceToDevice, b->stream);
                    if (e != cudaSuccess) return bcuda(b, e, "tail copy");
                }
            }
        }
    }
    b->substeps += total;
    return SWEPT2D_OK;
}

int batch_graph_advance(swept2d_batch *b, long long nsteps, int mode) {
    for (auto &g : b->graphs) {
        if (g.nsteps == nsteps && g.mode == mode && g.state == b->state) {
            cudaError_t e = cudaGraphLaunch(g.exec, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "graph launch");
            b->substeps += nsteps * b->bt->nst;
            b->launches += g.kernels;
            if (g.swaps_state) std::swap(b->state, b->state2);
            return SWEPT2D_OK;
        }
    }
    BatchGraph g{};
    g.nsteps = nsteps;
    g.mode = mode;
    g.state = b->state;
    const long long sub0 = b->substeps, l0 = b->launches;
    void *s0 = b->state, *s0b = b->state2;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "graph capture begin");
    int rc = batch_run(b, nsteps * b->bt->nst, mode);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->stream, &graph);
    g.kernels = b->launches - l0;
    g.swaps_state = b->state != s0;
    b->substeps = sub0;
    b->launches = l0;
    b->state = s0;
    b->state2 = s0b;
    if (rc != SWEPT2D_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return bcuda(b, e, "graph capture end");
    g.graph = graph;
    if ((e = cudaGraphInstantiate(&g.exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return bcuda(b, e, "graph instantiate");
    }
    if (b->graphs.size() >= 4) {
        cudaGraphExecDestroy(b->graphs.front().exec);
        cudaGraphDestroy(b->graphs.front().graph);
        b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back(g);
    return batch_graph_advance(b, nsteps, mode);
}

}  // namespace

extern "C" {

int swept2d_batch_create(swept2d_batch_t **out, int count, const int *nx, const int *ny,
                         const int *tile, int op, const double *params, int nparams, int dtype,
                         void *stream) {
    if (!out) return SWEPT2D_EINVAL;
    *out = nullptr;
    g_batch_create_err.clear();
    auto reject = [&](const std::string &m) {
        g_batch_create_err = m;
        return SWEPT2D_EINVAL;
    };
    if (count < 1 || !nx || !ny || !tile) return reject("need count >= 1 and nx, ny, tile arrays");
    const BatchTable *bt = batch_table(op, dtype);
    if (!bt)
        return reject("op/dtype not supported by the batch (heat F64, heat_kahan F32/BF16, hash "
                      "U64, euler_rk2 F64, euler_kahan F32/BF16)");
    if ((op == SWEPT2D_OP_HEAT || op == SWEPT2D_OP_HEAT_KAHAN) && (nparams < 1 || !params))
        return reject("heat needs params {r}");
    const bool euler = op == SWEPT2D_OP_EULER_RK2 || op == SWEPT2D_OP_EULER_KAHAN;
    if (euler && (nparams < 3 || nparams == 4 || nparams > 5 || !params))
        return reject("euler needs params {gamma, cfl, kappa[, lx, ly]}");
    if (nparams > 8) return reject("at most 8 params");
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    for (int i = 0; i < count; ++i) {
        if (nx[i] < 1 || ny[i] < 1) return reject("grid sizes must be >= 1");
        const int n = tile[i];
        if (n != 0 && (n < 4 || (n & 1) || nx[i] % n || ny[i] % n))
            return reject("tile " + std::to_string(n) + " of grid " + std::to_string(i) +
                          " must be 0, or even, >= 4 and divide its nx and ny");
        if (n != 0 && bt->smem_for(n, false) > (size_t)optin) return reject("tile too large");
    }
    swept2d_batch *b = new (std::nothrow) swept2d_batch();
    if (!b) return SWEPT2D_ENOMEM;
    b->count = count;
    b->op = op;
    b->dtype = dtype;
    b->bt = bt;
    b->stream = (cudaStream_t)stream;
    b->tune.threads = 256;
    b->tune.stage = bt->default_stage;
    if (nparams > 0 && !euler) b->consts[0] = params[0];
    b->nparams = nparams;
    for (int i = 0; i < nparams; ++i) b->params[i] = params[i];
    if (euler) {
        b->wavespeed.assign(count, 0.0);
        b->dt.assign(count, 0.0);
    }
    // grids, classes (by tile side), pooled offsets
    long long soff = 0, poff = 0;
    for (int i = 0; i < count; ++i) {
        GridDesc gd{};
        const int n = tile[i];
        gd.G.nx = nx[i];
        gd.G.ny = ny[i];
        gd.G.n = n;
        gd.G.T = n ? nx[i] / n : 0;
        gd.G.Q = n ? ny[i] / n : 0;
        gd.G.PS = n ? swept::panel_stride(n) : 0;
        gd.state_off = soff;
        gd.panel_off = poff;
        for (int k = 0; k < 8; ++k) gd.c[k] = b->consts[k];   // Euler's: at set_state
        soff += (long long)bt->nv * nx[i] * ny[i];
        poff += (long long)gd.G.T * gd.G.Q * 4 * bt->nv * gd.G.PS;
        b->cells += (long long)nx[i] * ny[i];
        b->grids.push_back(gd);
        BatchClass *cls = nullptr;
        for (auto &c : b->classes)
            if (c.n == n) cls = &c;
        if (!cls) {
            b->classes.emplace_back();
            cls = &b->classes.back();
            cls->n = n;
            cls->tune = b->tune;
        }
        cls->members.push_back(i);
        for (int t = 0; t < gd.G.T * gd.G.Q; ++t) cls->tiles.push_back(make_int2(i, t));
        const int nb = ((nx[i] + 31) / 32) * ((ny[i] + 7) / 8);
        for (int k = 0; k < nb; ++k) {
            cls->blocks.push_back(make_int2(i, k));
            b->all_blocks.push_back(make_int2(i, k));
        }
    }
    b->state_bytes = (size_t)soff * bt->esize;
    b->panel_bytes = (size_t)poff * bt->esize;
    cudaError_t e = cudaSuccess;
    auto dev_copy = [&](auto **dst, const auto &vec) {
        using T = typename std::remove_reference<decltype(vec)>::type::value_type;
        if (vec.empty()) return cudaSuccess;
        cudaError_t r = cudaMalloc((void **)dst, vec.size() * sizeof(T));
        if (r != cudaSuccess) return r;
        return cudaMemcpy(*dst, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice);
    };
    if ((e = dev_copy(&b->d_grids, b->grids)) != cudaSuccess ||
        (e = dev_copy(&b->d_all_blocks, b->all_blocks)) != cudaSuccess)
        goto fail;
    for (auto &c : b->classes)
        if ((e = dev_copy(&c.d_tiles, c.tiles)) != cudaSuccess ||
            (e = dev_copy(&c.d_blocks, c.blocks)) != cudaSuccess)
            goto fail;
    if (euler && (e = cudaMalloc(&b->d_amax, (size_t)count * sizeof(unsigned long long))) !=
                     cudaSuccess)
        goto fail;
    if ((e = cudaMalloc(&b->state, b->state_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&b->state2, b->state_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&b->errword, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(b->errword, 0, sizeof(int))) != cudaSuccess)
        goto fail;
    if (b->panel_bytes &&
        ((e = cudaMalloc(&b->up, b->panel_bytes)) != cudaSuccess ||
         (e = cudaMalloc(&b->br, b->panel_bytes)) != cudaSuccess))
        goto fail;
    *out = b;
    return SWEPT2D_OK;
fail:
    g_batch_create_err = std::string("batch allocation: ") + cudaGetErrorString(e);
    batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? SWEPT2D_ENOMEM : SWEPT2D_ECUDA;
}

int swept2d_batch_set_state(swept2d_batch_t *b, const void *src, int src_is_device) {
    if (!b) return SWEPT2D_EINVAL;
    if (!src) return bfail(b, SWEPT2D_EINVAL, "set_state: src is NULL");
    cudaError_t e = cudaMemcpyAsync(b->state, src, b->state_bytes,
                                    src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "set_state copy");
    if ((e = cudaMemsetAsync(b->errword, 0, sizeof(int), b->stream)) != cudaSuccess)
        return bcuda(b, e, "set_state error word");
    if (!src_is_device && (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        return bcuda(b, e, "set_state sync");
    b->substeps = 0;
    if (b->op == SWEPT2D_OP_EULER_RK2 || b->op == SWEPT2D_OP_EULER_KAHAN) {
        // each grid's a and dt from its own state, and its constants (formed in
        // binary64 as for a single grid), into the grid table
        const double gamma = b->params[0], cfl = b->params[1], kappa = b->params[2];
        const double lx = b->nparams >= 5 ? b->params[3] : 1.0;
        const double ly = b->nparams >= 5 ? b->params[4] : 1.0;
        if ((e = swept::batch_euler_wavespeed(b->d_grids, b->count, b->state, b->bt->esize, gamma,
                                              b->d_amax, b->stream)) != cudaSuccess)
            return bcuda(b, e, "wave speed");
        b->launches += 1;
        std::vector<unsigned long long> bits(b->count);
        if ((e = cudaMemcpyAsync(bits.data(), b->d_amax, bits.size() * sizeof(bits[0]),
                                 cudaMemcpyDeviceToHost, b->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
            return bcuda(b, e, "wave speed copy");
        for (int i = 0; i < b->count; ++i) {
            GridDesc &gd = b->grids[i];
            double a;
            std::memcpy(&a, &bits[i], sizeof a);
            const double dx = lx / gd.G.nx, dy = ly / gd.G.ny;
            const double hmin = dx < dy ? dx : dy;
            b->wavespeed[i] = a;
            b->dt[i] = (cfl * hmin) / a;
            gd.c[0] = gamma - 1.0;
            gd.c[1] = 0.5 / dx;
            gd.c[2] = 0.5 / dy;
            gd.c[3] = (kappa * a) / dx;
            gd.c[4] = (kappa * a) / dy;
            gd.c[5] = 0.5 * b->dt[i];
            gd.c[6] = b->dt[i];
        }
        if ((e = cudaMemcpyAsync(b->d_grids, b->grids.data(), b->grids.size() * sizeof(GridDesc),
                                 cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
            return bcuda(b, e, "grid table copy");
    }
    b->has_state = true;
    return SWEPT2D_OK;
}

int swept2d_batch_advance(swept2d_batch_t *b, long long nsteps, int mode) {
    if (!b) return SWEPT2D_EINVAL;
    if (nsteps < 0) return bfail(b, SWEPT2D_EINVAL, "advance: nsteps < 0");
    if (!b->has_state) return bfail(b, SWEPT2D_ESTATE, "advance: no state set");
    const bool graph = (mode & SWEPT2D_GRAPH) != 0;
    const int persistent = mode & SWEPT2D_PERSISTENT;
    const int one_launch = mode & SWEPT2D_ONE_LAUNCH;
    mode &= ~(SWEPT2D_GRAPH | SWEPT2D_PERSISTENT | SWEPT2D_ONE_LAUNCH);
    if (mode != SWEPT2D_SWEPT && mode != SWEPT2D_NAIVE) return bfail(b, SWEPT2D_EINVAL, "advance: bad mode");
    if (one_launch && !persistent)
        return bfail(b, SWEPT2D_EINVAL, "advance: the one-launch form needs SWEPT2D_PERSISTENT");
    if (persistent) {
        if (mode != SWEPT2D_SWEPT) return bfail(b, SWEPT2D_EINVAL, "advance: persistent needs the swept mode");
        int swept_classes = 0;
        for (auto &c : b->classes) swept_classes += c.n ? 1 : 0;
        if (one_launch && swept_classes > swept::kMaxClassRuns)
            return bfail(b, SWEPT2D_EINVAL, "advance: the one-launch form takes at most 16 classes");
        if (one_launch) {
            bool stage = false;
            long long tiles = 0;
            if (!one_launch_shape(b, &stage, &tiles))
                return bfail(b, SWEPT2D_EINVAL, "advance: the one-launch blocks do not fit in shared memory");
        }
        for (auto &c : b->classes) {
            if (!c.n) continue;
            if (c.tune.threads > 256 && !one_launch)
                return bfail(b, SWEPT2D_EINVAL, "advance: the persistent form takes at most 256 threads");
            const long long H = nsteps * b->bt->nst / (c.n / 2);
            if (swept::persistent_items((long long)c.tiles.size(), H) >= (1LL << 31))
                return bfail(b, SWEPT2D_EINVAL, "advance: too many work items for one persistent launch");
            if (!c.d_sched) {
                cudaError_t e = cudaMalloc(&c.d_sched, (c.tiles.size() + 1) * sizeof(int));
                if (e != cudaSuccess) return bcuda(b, e, "persistent schedule allocation");
            }
        }
        mode |= persistent | one_launch;
    }
    if (graph) {
        if (!b->stream) return bfail(b, SWEPT2D_EINVAL, "advance: graph mode needs a created stream");
        if (b->op == SWEPT2D_OP_HASH)
            return bfail(b, SWEPT2D_EINVAL, "advance: graph mode is not offered for the hash update");
        return batch_graph_advance(b, nsteps, mode);
    }
    return batch_run(b, nsteps * b->bt->nst, mode);
}

int swept2d_batch_get_state(swept2d_batch_t *b, void *dst, int dst_is_device) {
    if (!b) return SWEPT2D_EINVAL;
    if (!dst) return bfail(b, SWEPT2D_EINVAL, "get_state: dst is NULL");
    if (!b->has_state) return bfail(b, SWEPT2D_ESTATE, "get_state: no state set");
    cudaError_t e = cudaMemcpyAsync(dst, b->state, b->state_bytes,
                                    dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "get_state copy");
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bcuda(b, e, "get_state sync");
    int flag = 0;
    if ((e = cudaMemcpy(&flag, b->errword, sizeof flag, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bcuda(b, e, "get_state error word");
    if (flag) return bfail(b, SWEPT2D_ETIMEOUT, "a kernel's bounded wait gave up; state unspecified");
    return SWEPT2D_OK;
}

// Captured graphs hold the launch shapes they were captured with: drop them
// when a class's tuning changes.
static int drop_graphs(swept2d_batch *b) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "tuning sync");
    for (auto &g : b->graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaGraphDestroy(g.graph);
    }
    b->graphs.clear();
    return SWEPT2D_OK;
}

int swept2d_batch_set_tuning(swept2d_batch_t *b, int threads, int stage) {
    if (!b) return SWEPT2D_EINVAL;
    if (threads != 32 && threads != 64 && threads != 128 && threads != 256 && threads != 512)
        return bfail(b, SWEPT2D_EINVAL, "set_tuning: threads must be 32, 64, 128, 256 or 512");
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    for (auto &c : b->classes)
        if (c.n && b->bt->smem_for(c.n, stage != 0) > (size_t)optin)
            return bfail(b, SWEPT2D_EINVAL, "set_tuning: staged panels do not fit");
    const int rc = drop_graphs(b);
    if (rc) return rc;
    b->tune.threads = threads;
    b->tune.stage = stage != 0;
    for (auto &c : b->classes) c.tune = b->tune;
    return SWEPT2D_OK;
}

int swept2d_batch_set_class_tuning(swept2d_batch_t *b, int tile, int threads, int stage) {
    if (!b) return SWEPT2D_EINVAL;
    if (threads != 32 && threads != 64 && threads != 128 && threads != 256 && threads != 512)
        return bfail(b, SWEPT2D_EINVAL, "set_class_tuning: threads must be 32, 64, 128, 256 or 512");
    for (auto &c : b->classes) {
        if (c.n != tile || tile == 0) continue;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            optin = 227 * 1024;
        if (b->bt->smem_for(c.n, stage != 0) > (size_t)optin)
            return bfail(b, SWEPT2D_EINVAL, "set_class_tuning: staged panels do not fit");
        const int rc = drop_graphs(b);
        if (rc) return rc;
        c.tune.threads = threads;
        c.tune.stage = stage != 0;
        return SWEPT2D_OK;
    }
    return bfail(b, SWEPT2D_EINVAL, "set_class_tuning: no class with that tile");
}

int swept2d_batch_destroy(swept2d_batch_t *b) {
    if (!b) return SWEPT2D_OK;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
    return SWEPT2D_OK;
}

const char *swept2d_batch_last_error(const swept2d_batch_t *b) {
    if (!b) return g_batch_create_err.empty() ? "invalid batch (NULL)" : g_batch_create_err.c_str();
    return b->err.c_str();
}

int swept2d_batch_query_grid(const swept2d_batch_t *b, int grid, int what, double *out) {
    if (!b || !out || grid < 0 || grid >= b->count) return SWEPT2D_EINVAL;
    const GridDesc &gd = b->grids[grid];
    switch (what) {
        case SWEPT2D_Q_DT: *out = b->dt.empty() ? 0.0 : b->dt[grid]; break;
        case SWEPT2D_Q_WAVESPEED: *out = b->wavespeed.empty() ? 0.0 : b->wavespeed[grid]; break;
        case SWEPT2D_Q_CELLS: *out = (double)gd.G.nx * gd.G.ny; break;
        default: return SWEPT2D_EINVAL;
    }
    return SWEPT2D_OK;
}

int swept2d_batch_query(const swept2d_batch_t *b, int what, double *out) {
    if (!b || !out) return SWEPT2D_EINVAL;
    switch (what) {
        case SWEPT2D_Q_SUBSTEPS: *out = (double)b->substeps; break;
        case SWEPT2D_Q_LAUNCHES: *out = (double)b->launches; break;
        case SWEPT2D_Q_STATE_BYTES: *out = (double)b->state_bytes; break;
        case SWEPT2D_Q_PANEL_BYTES: *out = (double)b->panel_bytes; break;
        case SWEPT2D_Q_CELLS: *out = (double)b->cells; break;
        default: return SWEPT2D_EINVAL;
    }
    return SWEPT2D_OK;
}

}  // extern "C"
