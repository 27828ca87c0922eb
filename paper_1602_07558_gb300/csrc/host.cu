// C ABI of libswept2d.so (declared in include/swept2d.h): handle management,
// argument checks and the launch schedule of Algorithm 4 on one GPU.
//
// Schedule of one swept advance of S sub-steps with tile n (h = n/2):
//   H = S / h half cycles, r = S - H h remaining sub-steps.
//   half cycle 0 (frame o = 0):  Up(state)  -> up panels
//   each half cycle j:           Bridge(x and y, one launch)  -> bridge panels
//   between half cycles j, j+1:  Octahedron = Down(j) + Up(j+1)  -> up panels
//   after the last half cycle:   Down -> state (frame (H mod 2) h, periodic wrap)
//   then r naive sub-steps.
// The frame offset alternates 0, h, 0, ... (the paper's shift by half a tile
// after each half cycle, Section 4); on one GPU a frame is only an index offset.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/swept2d.h"
#include "launch.cuh"

using swept::Geom;
using swept::OpTable;

struct TimedLaunch {
    int kind;
    cudaEvent_t start, stop;
};

// One captured advance: replaying it is valid while the state buffer, the step
// count and the mode are the same (and, for the hash update, whose arithmetic
// reads the sub-step index, the starting sub-step).
struct GraphEntry {
    long long nsteps;
    int mode;
    void *state;
    long long g_start;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    long long substeps_advanced;
    long long kernels;
    bool swaps_state;
};

struct swept2d {
    int nx = 0, ny = 0, nv = 0, nst = 0, n = 0, op = 0, dtype = 0, esize = 0;
    Geom G{};
    const OpTable *ops = nullptr;
    cudaStream_t stream = nullptr;
    void *state = nullptr, *state2 = nullptr, *up = nullptr, *br = nullptr;
    unsigned long long *scratch8 = nullptr;
    int *errword = nullptr;   // set by a kernel whose bounded wait gave up
    int *sched = nullptr;     // persistent form: T*Q phase counters + queue counter
    unsigned *trace = nullptr;   // persistent form: caller's per-item cycle record (or none)
    long long trace_items = 0;
    swept::Tuning tune;
    size_t state_bytes = 0, panel_bytes = 0, smem_bytes = 0;
    double consts[8] = {0};
    double params[8] = {0};
    int nparams = 0;
    double dt = 0.0, wavespeed = 0.0;
    long long substeps = 0;
    long long launches = 0;
    bool has_state = false;
    bool timing = false;
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
    std::vector<GraphEntry> graphs;
    long long k_launches[SWEPT2D_K_COUNT] = {0};
    double k_ms[SWEPT2D_K_COUNT] = {0};
    std::string err;
};

namespace {

// Message of the last failed swept2d_create on this thread (no handle exists then).
thread_local std::string g_create_err;

int fail(swept2d *h, int code, const char *fmt, const char *detail = nullptr) {
    if (h) {
        char buf[512];
        snprintf(buf, sizeof buf, fmt, detail ? detail : "");
        h->err = buf;
    }
    return code;
}

int cuda_fail(swept2d *h, cudaError_t e, const char *where) {
    if (h) h->err = std::string(where) + ": " + cudaGetErrorString(e);
    return SWEPT2D_ECUDA;
}

cudaEvent_t take_event(swept2d *h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Fold finished timed launches into the per-kind totals (synchronises).
int collect_timing(swept2d *h) {
    if (h->timed.empty()) return SWEPT2D_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "timing sync");
    for (auto &t : h->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
            h->k_launches[t.kind] += 1;
            h->k_ms[t.kind] += ms;
        }
        h->event_pool.push_back(t.start);
        h->event_pool.push_back(t.stop);
    }
    h->timed.clear();
    return SWEPT2D_OK;
}

// Run one launch (a callable returning cudaError_t) of a given kind.
template <class F>
int launch(swept2d *h, int kind, const char *what, F &&f) {
    TimedLaunch t{kind, nullptr, nullptr};
    if (h->timing) {
        t.start = take_event(h);
        t.stop = take_event(h);
        cudaEventRecord(t.start, h->stream);
    }
    cudaError_t e = f();
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    h->launches += 1;
    if (h->timing) {
        cudaEventRecord(t.stop, h->stream);
        h->timed.push_back(t);
        if (h->timed.size() >= 4096) return collect_timing(h);
    }
    return SWEPT2D_OK;
}

const OpTable *table_for(int op, int dtype) {
    switch (op) {
        case SWEPT2D_OP_HEAT_KAHAN:
            return dtype == SWEPT2D_F32 ? swept::optable_heat_kahan_f32()
                 : dtype == SWEPT2D_BF16 ? swept::optable_heat_kahan_bf16() : nullptr;
        case SWEPT2D_OP_EULER_KAHAN:
            return dtype == SWEPT2D_F32 ? swept::optable_euler_kahan_f32()
                 : dtype == SWEPT2D_BF16 ? swept::optable_euler_kahan_bf16() : nullptr;
        case SWEPT2D_OP_HEAT: return swept::optable_heat();
        case SWEPT2D_OP_EULER_RK2: return swept::optable_euler();
        case SWEPT2D_OP_INCREMENT: return swept::optable_increment();
        case SWEPT2D_OP_HASH: return swept::optable_hash();
        case SWEPT2D_OP_LEVELTAG: return swept::optable_leveltag();
        case SWEPT2D_OP_WIDE2: return swept::optable_wide2();
        case SWEPT2D_OP_WAVE: return swept::optable_wave();
        default: return nullptr;
    }
}

bool dtype_ok(int op, int dtype) {
    if (op == SWEPT2D_OP_HASH || op == SWEPT2D_OP_WIDE2) return dtype == SWEPT2D_U64;
    if (op == SWEPT2D_OP_HEAT_KAHAN || op == SWEPT2D_OP_EULER_KAHAN)
        return dtype == SWEPT2D_F32 || dtype == SWEPT2D_BF16;
    return dtype == SWEPT2D_F64;
}

void free_all(swept2d *h) {
    if (h->state) cudaFree(h->state);
    if (h->state2) cudaFree(h->state2);
    if (h->up) cudaFree(h->up);
    if (h->br) cudaFree(h->br);
    if (h->scratch8) cudaFree(h->scratch8);
    if (h->errword) cudaFree(h->errword);
    if (h->sched) cudaFree(h->sched);
    for (auto &t : h->timed) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    for (auto &g : h->graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaGraphDestroy(g.graph);
    }
    h->graphs.clear();
    h->state = h->state2 = h->up = h->br = nullptr;
    h->scratch8 = nullptr;
    h->errword = nullptr;
    h->sched = nullptr;
}

int naive_substeps(swept2d *h, long long count) {
    for (long long s = 0; s < count; ++s) {
        const u64 g = (u64)h->substeps;
        int rc = launch(h, SWEPT2D_K_NAIVE, "naive kernel", [&] {
            return h->ops->naive(h->G, h->consts, h->state, h->state2, g, h->stream);
        });
        if (rc) return rc;
        std::swap(h->state, h->state2);
        h->substeps += 1;
    }
    return SWEPT2D_OK;
}

int swept_substeps(swept2d *h, long long total, bool persistent) {
    const int half = h->n / 2;
    const long long H = total / half;
    const long long rem = total - H * half;
    if (H > 0 && persistent) {
        const u64 g_start = (u64)h->substeps;
        const size_t nsched = (size_t)h->G.T * h->G.Q + 1;
        cudaError_t e = cudaMemsetAsync(h->sched, 0, nsched * sizeof(int), h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "persistent schedule reset");
        int rc = launch(h, SWEPT2D_K_OCTAHEDRON, "persistent kernel", [&] {
            return h->ops->persistent(h->G, h->consts, h->state, h->up, h->br, h->sched, (int)H,
                                      g_start, h->errword, h->tune, 0,
                                      swept::kPersistSpinLimit, h->trace, h->stream);
        });
        if (rc) return rc;
        h->substeps += H * half;
    } else if (H > 0) {
        const u64 g_start = (u64)h->substeps;
        int rc = launch(h, SWEPT2D_K_UP, "up kernel", [&] {
            return h->ops->up(h->G, h->consts, h->state, h->up, 0, g_start, h->stream);
        });
        if (rc) return rc;
        for (long long j = 0; j < H; ++j) {
            const u64 g0 = g_start + (u64)j * half;
            const int o = (j & 1) ? half : 0;
            rc = launch(h, SWEPT2D_K_BRIDGE, "bridge kernel", [&] {
                return h->ops->bridge(h->G, h->consts, h->up, h->br, g0, h->errword, h->tune,
                                      h->stream);
            });
            if (rc) return rc;
            if (j + 1 < H) {
                rc = launch(h, SWEPT2D_K_OCTAHEDRON, "octahedron kernel", [&] {
                    return h->ops->octahedron(h->G, h->consts, h->br, h->up, o, g0, h->errword,
                                              h->tune, h->stream);
                });
            } else {
                rc = launch(h, SWEPT2D_K_DOWN, "down kernel", [&] {
                    return h->ops->down(h->G, h->consts, h->br, h->state, o, g0, h->errword,
                                        h->tune, h->stream);
                });
            }
            if (rc) return rc;
        }
        h->substeps += H * half;
    }
    return naive_substeps(h, rem);
}

int run_advance(swept2d *h, long long total, int mode) {
    const bool persistent = (mode & SWEPT2D_PERSISTENT) != 0;
    mode &= ~SWEPT2D_PERSISTENT;
    return mode == SWEPT2D_SWEPT ? swept_substeps(h, total, persistent) : naive_substeps(h, total);
}

// Advance through a captured CUDA graph of the whole launch sequence.
int graph_advance(swept2d *h, long long nsteps, int mode) {
    const long long g_key = h->op == SWEPT2D_OP_HASH ? h->substeps : 0;
    for (auto &g : h->graphs) {
        if (g.nsteps == nsteps && g.mode == mode && g.state == h->state && g.g_start == g_key) {
            cudaError_t e = cudaGraphLaunch(g.exec, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
            h->substeps += g.substeps_advanced;
            h->launches += g.kernels;
            if (g.swaps_state) std::swap(h->state, h->state2);
            return SWEPT2D_OK;
        }
    }
    GraphEntry g{};
    g.nsteps = nsteps;
    g.mode = mode;
    g.state = h->state;
    g.g_start = g_key;
    const long long sub0 = h->substeps, l0 = h->launches;
    void *s0 = h->state, *s0b = h->state2;
    const bool timing = h->timing;
    h->timing = false;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        h->timing = timing;
        return cuda_fail(h, e, "graph capture begin");
    }
    int rc = run_advance(h, nsteps * h->nst, mode);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    h->timing = timing;
    // the capture ran nothing: undo the host bookkeeping, then replay it below
    g.substeps_advanced = h->substeps - sub0;
    g.kernels = h->launches - l0;
    g.swaps_state = h->state != s0;
    h->substeps = sub0;
    h->launches = l0;
    h->state = s0;
    h->state2 = s0b;
    if (rc != SWEPT2D_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "graph capture end");
    g.graph = graph;
    if ((e = cudaGraphInstantiate(&g.exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(h, e, "graph instantiate");
    }
    if (h->graphs.size() >= 8) {
        cudaGraphExecDestroy(h->graphs.front().exec);
        cudaGraphDestroy(h->graphs.front().graph);
        h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(g);
    return graph_advance(h, nsteps, mode);
}

}  // namespace

extern "C" {

int swept2d_create(swept2d_t **out, int nx, int ny, int nvars, int nstages, int tile, int op,
                   const double *params, int nparams, int dtype, void *stream) {
    if (!out) return SWEPT2D_EINVAL;
    *out = nullptr;
    swept2d *h = new (std::nothrow) swept2d();
    if (!h) return SWEPT2D_ENOMEM;
    auto bail = [&](int code) {
        g_create_err = h->err;
        free_all(h);
        delete h;
        return code;
    };
    if (op < 0 || op > SWEPT2D_OP_EULER_KAHAN) { fail(h, 0, "unknown op"); return bail(SWEPT2D_EINVAL); }
    if (!dtype_ok(op, dtype)) { fail(h, 0, "dtype does not match the op"); return bail(SWEPT2D_EINVAL); }
    const OpTable *t = table_for(op, dtype);
    if (!t) { fail(h, 0, "unknown op"); return bail(SWEPT2D_EINVAL); }
    if (nx < 1 || ny < 1) { fail(h, 0, "nx and ny must be >= 1"); return bail(SWEPT2D_EINVAL); }
    if (nvars != t->nv || nstages != t->nst) {
        fail(h, 0, "nvars/nstages do not match the op");
        return bail(SWEPT2D_EINVAL);
    }
    if (nparams < 0 || nparams > 8 || (nparams > 0 && !params)) {
        fail(h, 0, "bad params");
        return bail(SWEPT2D_EINVAL);
    }
    if (tile != 0) {
        if (tile < 4 || (tile & 1) || nx % tile || ny % tile) {
            fail(h, 0, "tile must be even, >= 4 and divide nx and ny");
            return bail(SWEPT2D_EINVAL);
        }
        const size_t sm = t->smem_for(tile, false);
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            optin = 227 * 1024;
        if (sm > (size_t)optin) {
            fail(h, 0, "tile too large for shared memory");
            return bail(SWEPT2D_EINVAL);
        }
        h->smem_bytes = t->smem_for(tile, t->default_stage);
        if (h->smem_bytes > (size_t)optin) {   // staging does not fit: prefetch per level
            h->tune.stage = false;
            h->smem_bytes = sm;
        }
    }
    h->nx = nx; h->ny = ny; h->nv = nvars; h->nst = nstages; h->n = tile; h->op = op;
    h->dtype = dtype; h->esize = t->esize; h->ops = t;
    h->tune.threads = 256;
    h->tune.stage = t->default_stage;
    h->stream = (cudaStream_t)stream;
    h->nparams = nparams;
    for (int i = 0; i < nparams; ++i) h->params[i] = params[i];
    // op constants
    switch (op) {
        case SWEPT2D_OP_HEAT:
        case SWEPT2D_OP_HEAT_KAHAN:
            if (nparams < 1) { fail(h, 0, "heat needs params {r}"); return bail(SWEPT2D_EINVAL); }
            h->consts[0] = params[0];
            break;
        case SWEPT2D_OP_WAVE:
            if (nparams < 1) { fail(h, 0, "wave needs params {C}"); return bail(SWEPT2D_EINVAL); }
            h->consts[0] = params[0] * params[0];
            break;
        case SWEPT2D_OP_EULER_RK2:
        case SWEPT2D_OP_EULER_KAHAN:
            if (nparams < 3) {
                fail(h, 0, "euler needs params {gamma, cfl, kappa[, lx, ly]}");
                return bail(SWEPT2D_EINVAL);
            }
            if (nparams == 4) { fail(h, 0, "euler: give both lx and ly"); return bail(SWEPT2D_EINVAL); }
            break;
        default: break;
    }
    h->G.nx = nx; h->G.ny = ny; h->G.n = tile;
    h->G.T = tile ? nx / tile : 0; h->G.Q = tile ? ny / tile : 0;
    h->G.PS = tile ? swept::panel_stride(tile) : 0;
    h->state_bytes = (size_t)nvars * nx * ny * t->esize;
    cudaError_t e;
    if ((e = cudaMalloc(&h->state, h->state_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&h->state2, h->state_bytes)) != cudaSuccess) {
        cuda_fail(h, e, "state allocation");
        return bail(e == cudaErrorMemoryAllocation ? SWEPT2D_ENOMEM : SWEPT2D_ECUDA);
    }
    if (tile) {
        h->panel_bytes = (size_t)h->G.T * h->G.Q * 4 * nvars * h->G.PS * t->esize;
        if ((e = cudaMalloc(&h->up, h->panel_bytes)) != cudaSuccess ||
            (e = cudaMalloc(&h->br, h->panel_bytes)) != cudaSuccess) {
            cuda_fail(h, e, "panel allocation");
            return bail(e == cudaErrorMemoryAllocation ? SWEPT2D_ENOMEM : SWEPT2D_ECUDA);
        }
    }
    if ((e = cudaMalloc(&h->scratch8, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&h->errword, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(h->errword, 0, sizeof(int))) != cudaSuccess) {
        cuda_fail(h, e, "scratch allocation");
        return bail(SWEPT2D_ECUDA);
    }
    g_create_err.clear();
    *out = h;
    return SWEPT2D_OK;
}

int swept2d_set_state(swept2d_t *h, const void *src, int src_is_device) {
    if (!h) return SWEPT2D_EINVAL;
    if (!src) return fail(h, SWEPT2D_EINVAL, "set_state: src is NULL");
    cudaError_t e = cudaMemcpyAsync(h->state, src, h->state_bytes,
                                    src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state copy");
    if (!src_is_device && (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "set_state sync");
    h->substeps = 0;
    if ((e = cudaMemsetAsync(h->errword, 0, sizeof(int), h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "set_state error word");
    if (h->op == SWEPT2D_OP_EULER_RK2 || h->op == SWEPT2D_OP_EULER_KAHAN) {
        const double gamma = h->params[0], cfl = h->params[1], kappa = h->params[2];
        const double lx = h->nparams >= 5 ? h->params[3] : 1.0;
        const double ly = h->nparams >= 5 ? h->params[4] : 1.0;
        const double dx = lx / h->nx, dy = ly / h->ny;
        double a = 0.0;
        int rc = launch(h, SWEPT2D_K_REDUCE, "wave speed", [&] {
            return swept::euler_wavespeed(h->state, h->esize, h->nx, h->ny, gamma,
                                          h->scratch8, &a, h->stream);
        });
        if (rc) return rc;
        const double hmin = dx < dy ? dx : dy;
        h->wavespeed = a;
        h->dt = (cfl * hmin) / a;
        h->consts[0] = gamma - 1.0;
        h->consts[1] = 0.5 / dx;
        h->consts[2] = 0.5 / dy;
        h->consts[3] = (kappa * a) / dx;
        h->consts[4] = (kappa * a) / dy;
        h->consts[5] = 0.5 * h->dt;
        h->consts[6] = h->dt;
    }
    h->has_state = true;
    return SWEPT2D_OK;
}

// Checks and scratch of the persistent form for H half cycles: the staged
// shared-memory plan must fit, the work items must fit an int, and the phase
// counters (T*Q + 1 ints) are allocated on first use.
static int persistent_prepare(swept2d *h, long long H) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    if (h->ops->smem_for(h->n, h->tune.stage) > (size_t)optin)
        return fail(h, SWEPT2D_EINVAL, "advance: the persistent form's shared memory does not fit");
    if (swept::persistent_items((long long)h->G.T * h->G.Q, H) >= (1LL << 31))
        return fail(h, SWEPT2D_EINVAL, "advance: too many work items for one persistent launch");
    if (!h->sched) {
        cudaError_t e = cudaMalloc(&h->sched, ((size_t)h->G.T * h->G.Q + 1) * sizeof(int));
        if (e != cudaSuccess) return cuda_fail(h, e, "persistent schedule allocation");
    }
    return SWEPT2D_OK;
}

int swept2d_selftest_wait_timeout(swept2d_t *h, long long spin_limit) {
    if (!h) return SWEPT2D_EINVAL;
    if (h->n == 0) return fail(h, SWEPT2D_EINVAL, "selftest: needs a handle created with a tile");
    if (spin_limit < 1) return fail(h, SWEPT2D_EINVAL, "selftest: spin_limit < 1");
    if (h->tune.threads > h->ops->max_persistent_threads)
        return fail(h, SWEPT2D_EINVAL, "selftest: the persistent form takes at most 512 threads per block");
    int rc = persistent_prepare(h, 1);
    if (rc) return rc;
    const int NT = h->G.T * h->G.Q;
    cudaError_t e = cudaMemsetAsync(h->sched, 0, ((size_t)NT + 1) * sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "selftest schedule reset");
    // one half cycle with the NT first-phase items skipped: every item taken
    // waits for a phase-1 counter that nothing releases
    rc = launch(h, SWEPT2D_K_OCTAHEDRON, "persistent kernel (wait-timeout self-test)", [&] {
        return h->ops->persistent(h->G, h->consts, h->state, h->up, h->br, h->sched, 1,
                                  (u64)h->substeps, h->errword, h->tune, NT, spin_limit,
                                  nullptr, h->stream);
    });
    if (rc) return rc;
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "selftest sync");
    int flag = 0;
    if ((e = cudaMemcpy(&flag, h->errword, sizeof flag, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(h, e, "selftest error word");
    if ((e = cudaMemset(h->errword, 0, sizeof(int))) != cudaSuccess)
        return cuda_fail(h, e, "selftest error word reset");
    if (flag == 2)
        return fail(h, SWEPT2D_ETIMEOUT, "selftest: the persistent kernel's neighbourhood wait gave up, as intended");
    return fail(h, SWEPT2D_ESTATE, "selftest: the persistent kernel did not report a timed-out wait");
}

int swept2d_advance(swept2d_t *h, long long nsteps, int mode) {
    if (!h) return SWEPT2D_EINVAL;
    if (nsteps < 0) return fail(h, SWEPT2D_EINVAL, "advance: nsteps < 0");
    if (!h->has_state) return fail(h, SWEPT2D_ESTATE, "advance: no state set");
    const bool graph = (mode & SWEPT2D_GRAPH) != 0;
    const int persistent = mode & SWEPT2D_PERSISTENT;
    mode &= ~(SWEPT2D_GRAPH | SWEPT2D_PERSISTENT);
    if (mode != SWEPT2D_SWEPT && mode != SWEPT2D_NAIVE) return fail(h, SWEPT2D_EINVAL, "advance: bad mode");
    if (mode == SWEPT2D_SWEPT && h->n == 0)
        return fail(h, SWEPT2D_EINVAL, "advance: swept mode needs a tile (created with tile 0)");
    if (persistent) {
        if (mode != SWEPT2D_SWEPT) return fail(h, SWEPT2D_EINVAL, "advance: persistent needs the swept mode");
        if (h->tune.threads > h->ops->max_persistent_threads)
            return fail(h, SWEPT2D_EINVAL, "advance: the persistent form takes at most 512 threads per block");
        const long long H = nsteps * h->nst / (h->n / 2);
        const int rc = persistent_prepare(h, H);
        if (rc) return rc;
        if (h->trace && swept::persistent_items((long long)h->G.T * h->G.Q, H) > h->trace_items)
            return fail(h, SWEPT2D_EINVAL, "advance: the trace buffer holds fewer items than this advance has");
        mode |= persistent;
    }
    if (graph) {
        if (!h->stream) return fail(h, SWEPT2D_EINVAL, "advance: graph mode needs a created stream");
        return graph_advance(h, nsteps, mode);
    }
    return run_advance(h, nsteps * h->nst, mode);
}

int swept2d_get_state(swept2d_t *h, void *dst, int dst_is_device) {
    if (!h) return SWEPT2D_EINVAL;
    if (!dst) return fail(h, SWEPT2D_EINVAL, "get_state: dst is NULL");
    if (!h->has_state) return fail(h, SWEPT2D_ESTATE, "get_state: no state set");
    cudaError_t e = cudaMemcpyAsync(dst, h->state, h->state_bytes,
                                    dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_state copy");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "get_state sync");
    int flag = 0;
    if ((e = cudaMemcpy(&flag, h->errword, sizeof flag, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(h, e, "get_state error word");
    if (flag == 2)
        return fail(h, SWEPT2D_ETIMEOUT, "the persistent kernel's bounded wait for its tile neighbourhood gave up; the state is unspecified");
    if (flag) return fail(h, SWEPT2D_ETIMEOUT, "a kernel's bounded wait for its panel copies gave up; the state is unspecified");
    return SWEPT2D_OK;
}

int swept2d_destroy(swept2d_t *h) {
    if (!h) return SWEPT2D_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return SWEPT2D_OK;
}

const char *swept2d_last_error(const swept2d_t *h) {
    if (!h) return g_create_err.empty() ? "invalid handle (NULL)" : g_create_err.c_str();
    return h->err.c_str();
}

int swept2d_query(const swept2d_t *h, int what, double *out) {
    if (!h || !out) return SWEPT2D_EINVAL;
    switch (what) {
        case SWEPT2D_Q_DT: *out = h->dt; break;
        case SWEPT2D_Q_WAVESPEED: *out = h->wavespeed; break;
        case SWEPT2D_Q_SUBSTEPS: *out = (double)h->substeps; break;
        case SWEPT2D_Q_LAUNCHES: *out = (double)h->launches; break;
        case SWEPT2D_Q_STATE_BYTES: *out = (double)h->state_bytes; break;
        case SWEPT2D_Q_PANEL_BYTES: *out = (double)h->panel_bytes; break;
        case SWEPT2D_Q_SMEM_BYTES: *out = (double)h->smem_bytes; break;
        case SWEPT2D_Q_CELLS: *out = (double)h->nx * h->ny; break;
        case SWEPT2D_Q_THREADS: *out = h->tune.threads; break;
        case SWEPT2D_Q_STAGE: *out = h->tune.stage ? 1.0 : 0.0; break;
        default: return SWEPT2D_EINVAL;
    }
    return SWEPT2D_OK;
}

int swept2d_set_tuning(swept2d_t *h, int threads, int stage) {
    if (!h) return SWEPT2D_EINVAL;
    if (threads != 32 && threads != 64 && threads != 128 && threads != 256 && threads != 512)
        return fail(h, SWEPT2D_EINVAL, "set_tuning: threads must be 32, 64, 128, 256 or 512");
    if (h->n == 0) return fail(h, SWEPT2D_EINVAL, "set_tuning: naive-only handle");
    const size_t sm = h->ops->smem_for(h->n, stage != 0);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    if (sm > (size_t)optin) return fail(h, SWEPT2D_EINVAL, "set_tuning: staged panels do not fit");
    if (h->tune.threads != threads || h->tune.stage != (stage != 0)) {
        // captured graphs hold the old launch shape: drop them
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "set_tuning sync");
        for (auto &g : h->graphs) {
            cudaGraphExecDestroy(g.exec);
            cudaGraphDestroy(g.graph);
        }
        h->graphs.clear();
    }
    h->tune.threads = threads;
    h->tune.stage = stage != 0;
    h->smem_bytes = sm;
    return SWEPT2D_OK;
}

int swept2d_set_trace(swept2d_t *h, void *device_buffer, long long items) {
    if (!h) return SWEPT2D_EINVAL;
    if ((device_buffer == nullptr) != (items == 0) || items < 0)
        return fail(h, SWEPT2D_EINVAL, "set_trace: give a buffer and its item count, or NULL and 0");
    // captured graphs hold the old pointer: drop them
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_trace sync");
    for (auto &g : h->graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaGraphDestroy(g.graph);
    }
    h->graphs.clear();
    h->trace = (unsigned *)device_buffer;
    h->trace_items = items;
    return SWEPT2D_OK;
}

int swept2d_set_timing(swept2d_t *h, int on) {
    if (!h) return SWEPT2D_EINVAL;
    int rc = collect_timing(h);
    if (rc) return rc;
    h->timing = on != 0;
    for (int k = 0; k < SWEPT2D_K_COUNT; ++k) {
        h->k_launches[k] = 0;
        h->k_ms[k] = 0.0;
    }
    return SWEPT2D_OK;
}

int swept2d_kernel_stats(swept2d_t *h, int kind, long long *launches, double *total_ms) {
    if (!h || kind < 0 || kind >= SWEPT2D_K_COUNT || !launches || !total_ms) return SWEPT2D_EINVAL;
    int rc = collect_timing(h);
    if (rc) return rc;
    *launches = h->k_launches[kind];
    *total_ms = h->k_ms[kind];
    return SWEPT2D_OK;
}

}  // extern "C"
