// Allocation-free swept advance of the heat equation (FP64).
//
// Who needs this: callers that must not allocate device memory at the point
// where they advance a grid -- for example a host application that owns every
// device allocation through its own fixed pool and forbids cudaMalloc outside
// it, a plugin running under such an application, or a latency-critical loop
// where cudaMalloc/cudaFree would add their implicit device-wide
// synchronisation. They pass their own input and output buffers; the only
// other device memory this path touches is the file-scope array below, which
// the CUDA runtime sets up when it loads this library's device code.
//
// The schedule and the kernels are the same as swept2d_advance's swept mode
// (Up, then per half cycle the x/y Bridge launch and the Octahedron, a final
// Down, then the remaining sub-steps with the naive kernel), so the result is
// bit for bit that of a handle created with op SWEPT2D_OP_HEAT and advanced
// with SWEPT2D_SWEPT from the same input.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "../../include/swept2d.h"
#include "launch.cuh"

namespace {

constexpr size_t kScratchBytes = SWEPT2D_STATIC_SCRATCH_BYTES;

// Shared by every call on a device and kept until the process exits. Holds the
// two panel buffers and, when the step count leaves a naive tail, one state
// copy for its ping-pong. Nothing in it has to start at zero: every element a
// call reads was written earlier in that same call.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

void set_err(char *err, int errlen, const char *msg) {
    if (err && errlen > 0) {
        strncpy(err, msg, (size_t)errlen - 1);
        err[errlen - 1] = '\0';
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of g_scratch on the current device. In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up on every
// call, with the caller's device current: a cached address would outlive a
// cudaDeviceReset or a switch to another context on the same device, after
// which the module is loaded again at another address.
int scratch_address(void **out, char *err, int errlen) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        set_err(err, errlen, e != cudaSuccess ? cudaGetErrorString(e)
                                              : "cudaGetSymbolAddress returned NULL");
        return SWEPT2D_ECUDA;
    }
    *out = p;
    return SWEPT2D_OK;
}

}  // namespace

extern "C" int swept2d_heat_advance_static(const double *u_in, double *u_out, int nx, int ny,
                                           int tile, double r, long long nsteps, void *stream,
                                           char *err, int errlen) {
    set_err(err, errlen, "");
    if (!u_in || !u_out) {
        set_err(err, errlen, "u_in and u_out must be device pointers");
        return SWEPT2D_EINVAL;
    }
    if (nx < 1 || ny < 1 || nsteps < 0) {
        set_err(err, errlen, "need nx, ny >= 1 and nsteps >= 0");
        return SWEPT2D_EINVAL;
    }
    if (tile < 4 || (tile & 1) || nx % tile || ny % tile) {
        set_err(err, errlen, "tile must be even, >= 4 and divide nx and ny");
        return SWEPT2D_EINVAL;
    }
    const size_t state_bytes = (size_t)nx * ny * sizeof(double);
    const char *in_b = (const char *)u_in, *out_b = (const char *)u_out;
    if (in_b < out_b + state_bytes && out_b < in_b + state_bytes) {
        set_err(err, errlen, "u_in and u_out must not overlap");
        return SWEPT2D_EINVAL;
    }
    const size_t smem = swept::optable_heat()->smem_for(tile, false);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    if (smem > (size_t)optin) {
        set_err(err, errlen, "tile too large for shared memory");
        return SWEPT2D_EINVAL;
    }
    swept::Geom G;
    G.nx = nx; G.ny = ny; G.n = tile;
    G.T = nx / tile; G.Q = ny / tile;
    G.PS = swept::panel_stride(tile);
    const size_t panel_bytes = (size_t)G.T * G.Q * 4 * G.PS * sizeof(double);
    const int half = tile / 2;
    const long long H = nsteps / half, rem = nsteps - H * half;
    const size_t need = 2 * align256(panel_bytes) + (rem > 0 ? align256(state_bytes) : 0);
    if (need > kScratchBytes) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "grid needs %zu bytes of scratch; the static scratch holds %zu bytes",
                 need, kScratchBytes);
        set_err(err, errlen, msg);
        return SWEPT2D_EINVAL;
    }
    void *base = nullptr;
    int rc = scratch_address(&base, err, errlen);
    if (rc != SWEPT2D_OK) return rc;
    char *sb = (char *)base;
    void *up = sb;
    void *br = sb + align256(panel_bytes);
    double *tmp = (double *)(sb + 2 * align256(panel_bytes));

    const swept::OpTable *t = swept::optable_heat();
    const double consts[8] = {r, 0, 0, 0, 0, 0, 0, 0};
    const swept::Tuning tn;   // 256 threads, per-level prefetch (the handle path's heat default)
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    auto check = [&](cudaError_t ce, const char *what) {
        if (ce != cudaSuccess) {
            char msg[200];
            snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(ce));
            set_err(err, errlen, msg);
            return false;
        }
        return true;
    };
    // The tail's ping-pong is arranged so that its last sub-step lands in u_out.
    if (H == 0) {
        if (rem == 0) {
            e = cudaMemcpyAsync(u_out, u_in, state_bytes, cudaMemcpyDeviceToDevice, st);
            return check(e, "copy") ? SWEPT2D_OK : SWEPT2D_ECUDA;
        }
        const double *src = u_in;
        for (long long i = 0; i < rem; ++i) {
            double *dst = ((rem - 1 - i) % 2 == 0) ? u_out : tmp;
            if (!check(t->naive(G, consts, src, dst, (u64)i, st), "naive kernel")) return SWEPT2D_ECUDA;
            src = dst;
        }
        return SWEPT2D_OK;
    }
    double *swept_dst = (rem % 2 == 1) ? tmp : u_out;
    if (!check(t->up(G, consts, u_in, up, 0, 0, st), "up kernel")) return SWEPT2D_ECUDA;
    for (long long j = 0; j < H; ++j) {
        const u64 g0 = (u64)j * half;
        const int o = (j & 1) ? half : 0;
        if (!check(t->bridge(G, consts, up, br, g0, nullptr, tn, st), "bridge kernel")) return SWEPT2D_ECUDA;
        if (j + 1 < H) {
            if (!check(t->octahedron(G, consts, br, up, o, g0, nullptr, tn, st), "octahedron kernel"))
                return SWEPT2D_ECUDA;
        } else {
            if (!check(t->down(G, consts, br, swept_dst, o, g0, nullptr, tn, st), "down kernel"))
                return SWEPT2D_ECUDA;
        }
    }
    const double *src = swept_dst;
    for (long long i = 0; i < rem; ++i) {
        double *dst = (src == tmp) ? u_out : tmp;
        if (!check(t->naive(G, consts, src, dst, (u64)(H * half + i), st), "naive kernel"))
            return SWEPT2D_ECUDA;
        src = dst;
    }
    return SWEPT2D_OK;
}
