// Kernels of the swept rule (Sections 3-4) and of the naive per-sub-step path.
//
// Geometry (tile side n, h = n/2, T x Q tiles, frame offset o in {0, h}).
// For one half cycle whose first sub-step is g0, every point at level t in
// 1..h is computed by exactly one component (Algorithms 1, 2, 3, 5):
//   Up(I,J)       frame (o, o):        local square [t, n-t)^2
//   y-bridge(I,J) frame (o, o+h):      x in [t, n-t), y in [h-t, h+t)   (Algorithm 2)
//   x-bridge(I,J) frame (o+h, o):      x in [h-t, h+t), y in [t, n-t)   (Algorithm 3)
//   Down(I,J)     frame (o+h, o+h):    [h-t, h+t)^2                     (Algorithm 5)
// The four counts (n-2t)^2 + 2 * 2t(n-2t) + (2t)^2 = n^2 partition each level.
//
// Panels (Section 3, "triangular sides"): per tile slot, side (N=0, S=1, W=2,
// E=3) and value plane, a packed array of PS = n^2/2 + n elements holding the
// 2-wide edge strip of each level k = 0..h-1 as two lines (d = 0 outermost,
// d = 1 inner) of L elements, line d at offset off(k) + d L:
//   up panels     L = n - 2k,  off(k) = 2k(n-k+1)   (16, 12, 8, 4 for n = 8)
//   bridge panels L = 2k + 2,  off(k) = 2k(k+1)     (4, 8, 12, 16 for n = 8)
// Up panel of Up(I,J) in its local (a, b):   N (k+p, k+d), S (k+p, n-1-k-d),
//                                            W (k+d, k+p), E (n-1-k-d, k+p)
// y-bridge(I,J) writes slot (I,J) sides W, E (local (a, b) of the bridge):
//    W (k+d, h-k+p)  [carries the south corner], E (n-1-k-d, h-k-2+p)  [north corner]
// x-bridge(I,J) writes slot (I,J) sides N, S:
//    N (h-k-2+p, k+d) [west corner],             S (h-k+p, n-1-k-d)    [east corner]
// so the downward pyramid's ring at level k is the pinwheel of Algorithm 5:
// west side <- E of y-bridge(I,J), east <- W of y-bridge(I+1,J),
// north <- S of x-bridge(I,J), south <- N of x-bridge(I,J+1).
//
// Shared memory per block: two level buffers (Algorithm 1's U and D), each NV
// planes of (n+2) x (n+2) with the tile at offset (1, 1), plus Op::AUX planes of
// the same shape for point updates that stage partial results (heat: pair sums).
#pragma once
#include <cuda_runtime.h>

#include "ops.cuh"

namespace swept {

struct Geom {
    int nx, ny;   // grid
    int n;        // tile side
    int T, Q;     // tiles along x and y
    int PS;       // panel elements per (slot, side, plane) = n*n/2 + n
};

__device__ __forceinline__ int wrap_add(int a, int d, int m) {
    int r = a + d;
    return r >= m ? r - m : (r < 0 ? r + m : r);
}

// Asynchronous global -> shared copy of one element (cp.async, no register
// staging) so that the next level's panel loads overlap the current level's
// arithmetic; async_wait() waits for this thread's copies (a __syncthreads()
// afterwards publishes them to the block).
template <class S>
__device__ __forceinline__ void async_copy(S *smem_dst, const S *gmem_src) {
    static_assert(sizeof(S) == 4 || sizeof(S) == 8 || sizeof(S) == 16, "cp.async size");
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem_src),
                 "n"((int)sizeof(S)));
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void async_wait() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Neighbourhood accessor into a shared-memory level buffer; p points at the
// centre point in plane 0.
template <class S>
struct SmemAcc {
    const S *p;
    int P, plane;
    __device__ __forceinline__ S operator()(int dx, int dy, int v) const {
        return p[v * plane + dy * P + dx];
    }
};

// Neighbourhood accessor into the global state with periodic wrap.
template <class S>
struct GlobalAcc {
    const S *base;
    size_t plane;
    int nx, ny, x, y;
    __device__ __forceinline__ S operator()(int dx, int dy, int v) const {
        const int xx = wrap_add(x, dx, nx), yy = wrap_add(y, dy, ny);
        return base[v * plane + (size_t)yy * nx + xx];
    }
};

// Apply the point update on the local rectangle [x0, x0+W) x [y0, y0+H) of the
// level buffer src, writing dst. Threads take consecutive points of the
// rectangle so that warps stay full.
template <class Op>
__device__ __forceinline__ void compute_rect(const Op &op, int stage, u64 g,
                                             const typename Op::S *src, typename Op::S *dst,
                                             typename Op::S * /*aux*/, int P, int x0, int y0,
                                             int W, int H) {
    typedef typename Op::S S;
    const int plane = P * P, cnt = W * H;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int yy = e / W, xx = e - yy * W;
        const int off = (y0 + yy + 1) * P + (x0 + xx + 1);
        SmemAcc<S> acc{src + off, P, plane};
        S out[Op::NV];
        op(stage, g, acc, out);
#pragma unroll
        for (int v = 0; v < Op::NV; ++v) dst[v * plane + off] = out[v];
    }
}

// Heat: the east+south pair sum Pr(x, y) = u(x+1, y) + u(x, y+1) of a point is
// the west+north pair sum of its south-east neighbour (x+1, y+1), so it is
// formed once for [x0-1, x0+W) x [y0-1, y0+H) into the aux buffer (pass 1),
// and each point then needs s = Pr(x, y) + Pr(x-1, y-1) and two fused
// multiply-adds (pass 2): about 4.1 FP64 operations per point instead of 5,
// with the same roundings as HeatOp::operator() (the pair sums commute).
__device__ __forceinline__ void compute_rect(const HeatOp &op, int, u64, const double *src,
                                             double *dst, double *aux, int P, int x0, int y0,
                                             int W, int H) {
    const int W1 = W + 1, cnt1 = W1 * (H + 1);
    for (int e = threadIdx.x; e < cnt1; e += blockDim.x) {
        const int yy = e / W1, xx = e - yy * W1;
        const int off = (y0 + yy) * P + (x0 + xx);      // point (x0-1+xx, y0-1+yy)
        aux[off] = __dadd_rn(src[off + 1], src[off + P]);
    }
    __syncthreads();
    const int cnt = W * H;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int yy = e / W, xx = e - yy * W;
        const int off = (y0 + yy + 1) * P + (x0 + xx + 1);
        const double c = src[off];
        const double sum = __dadd_rn(aux[off], aux[off - P - 1]);
        dst[off] = __fma_rn(op.r, __fma_rn(-4.0, c, sum), c);
    }
}

// Local coordinates of element (d, p) of an up panel side at level k.
__device__ __forceinline__ void up_panel_xy(int side, int n, int k, int d, int p, int &a, int &b) {
    switch (side) {
        case 0: a = k + p; b = k + d; break;
        case 1: a = k + p; b = n - 1 - k - d; break;
        case 2: a = k + d; b = k + p; break;
        default: a = n - 1 - k - d; b = k + p; break;
    }
}

// Write level k of the 4 up panels of the tile held in cur to slot `slot`.
template <class S, int NV>
__device__ __forceinline__ void write_up_panels(const S *cur, int P, const Geom &G, int k,
                                                S *up, int slot) {
    const int n = G.n, L = n - 2 * k, L2 = 2 * L, plane = P * P;
    const size_t off = (size_t)2 * k * (n - k + 1);
    for (int e = threadIdx.x; e < 4 * L2; e += blockDim.x) {
        const int side = e / L2, r = e - side * L2, d = r >= L, p = r - d * L;
        int a, b;
        up_panel_xy(side, n, k, d, p, a, b);
        S *dst = up + ((size_t)slot * 4 + side) * NV * G.PS + off + d * L + p;
#pragma unroll
        for (int v = 0; v < NV; ++v) dst[(size_t)v * G.PS] = cur[v * plane + (b + 1) * P + (a + 1)];
    }
}

// ---------------------------------------------------------------- naive path
// One sub-step over the whole grid: out = St(in) at every point.
template <class Op>
__global__ void __launch_bounds__(256) naive_kernel(Op op, Geom G, const typename Op::S *in,
                                                    typename Op::S *out, u64 g) {
    typedef typename Op::S S;
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= G.nx || y >= G.ny) return;
    const size_t plane = (size_t)G.nx * G.ny;
    GlobalAcc<S> acc{in, plane, G.nx, G.ny, x, y};
    S res[Op::NV];
    op((int)(g % Op::NST), g, acc, res);
    const size_t p = (size_t)y * G.nx + x;
#pragma unroll
    for (int v = 0; v < Op::NV; ++v) out[v * plane + p] = res[v];
}

// Heat, naive path: each warp walks down a chunk of 31 columns over ROWS rows
// (32 on large grids, fewer on small ones so that enough warps run); lane l
// holds column x = 31 c + l - 1 (lane 0 only supplies the pair sum
// of the column to the left). The east+south pair sum of row y-1 moves one lane
// to the right with a shuffle and is the west+north pair sum at row y, so a
// point costs about 4.1 FP64 operations, with the roundings of HeatOp.
template <int ROWS>
__global__ void __launch_bounds__(256) naive_heat_kernel(HeatOp op, Geom G, const double *in,
                                                         double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = blockIdx.x * 31 + lane - 1;
    if (x < 0) x += G.nx;
    const bool active = lane > 0 && x < G.nx;
    if (x >= G.nx) x %= G.nx;            // idle lanes read valid memory, store nothing
    const int xe = x + 1 == G.nx ? 0 : x + 1;
    const int y0 = (blockIdx.y * 8 + warp) * ROWS;
    if (y0 >= G.ny) return;               // whole warp leaves together
    const int y1 = min(y0 + ROWS, G.ny);
    const size_t nx = G.nx;
    int ym = y0 - 1;
    if (ym < 0) ym += G.ny;
    double c = in[(size_t)y0 * nx + x];
    double pp = __dadd_rn(in[(size_t)ym * nx + xe], c);   // Pr(x, y0-1)
    for (int y = y0; y < y1; ++y) {
        const int ys = y + 1 == G.ny ? 0 : y + 1;
        const double sd = in[(size_t)ys * nx + x];
        const double pc = __dadd_rn(in[(size_t)y * nx + xe], sd);   // Pr(x, y)
        const double q = __shfl_up_sync(0xffffffffu, pp, 1);         // Pr(x-1, y-1)
        const double res = __fma_rn(op.r, __fma_rn(-4.0, c, __dadd_rn(pc, q)), c);
        if (active) out[(size_t)y * nx + x] = res;
        pp = pc;
        c = sd;
    }
}

// ------------------------------------------------------- UpwardPyramid (Alg. 1)
// Shared body: tile at level 0 of half cycle g0 is in buffer 0; builds levels
// 1..h-1 and writes the up panels of levels 0..h-1 to slot `slot`.
template <class Op>
__device__ __forceinline__ void up_body(const Op &op, const Geom &G, typename Op::S *buf0,
                                        typename Op::S *buf1, typename Op::S *aux, int P, u64 g0,
                                        typename Op::S *up, int slot, int first_parity) {
    typedef typename Op::S S;
    const int n = G.n, h = n / 2;
    for (int k = 0; k < h; ++k) {
        const int par = (first_parity + k) & 1;
        const S *cur = par ? buf1 : buf0;
        S *nxt = par ? buf0 : buf1;
        write_up_panels<S, Op::NV>(cur, P, G, k, up, slot);
        if (k + 1 < h) {
            const u64 g = g0 + k;
            compute_rect(op, (int)(g % Op::NST), g, cur, nxt, aux, P, k + 1, k + 1,
                         n - 2 * k - 2, n - 2 * k - 2);
        }
        __syncthreads();
    }
}

// K1: first upward pyramid of an advance, frame offset o, reading the state.
template <class Op>
__global__ void __launch_bounds__(256) up_kernel(Op op, Geom G, const typename Op::S *state,
                                                 typename Op::S *up, int o, u64 g0) {
    typedef typename Op::S S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = G.n, P = n + 2, plane = P * P;
    S *buf0 = reinterpret_cast<S *>(smem_raw);
    S *buf1 = buf0 + Op::NV * plane;
    S *aux = buf1 + Op::NV * plane;
    const int I = blockIdx.x, J = blockIdx.y;
    const size_t gplane = (size_t)G.nx * G.ny;
    const int x0 = o + I * n, y0 = o + J * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int b = e / n, a = e - b * n;
        int x = x0 + a; x -= x >= G.nx ? G.nx : 0;
        int y = y0 + b; y -= y >= G.ny ? G.ny : 0;
#pragma unroll
        for (int v = 0; v < Op::NV; ++v)
            buf0[v * plane + (b + 1) * P + (a + 1)] = state[v * gplane + (size_t)y * G.nx + x];
    }
    __syncthreads();
    up_body(op, G, buf0, buf1, aux, P, g0, up, J * G.T + I, 0);
}

// ------------------------------------------- Bridges (Algorithms 2 and 3)
// blockIdx.z == 0: longitudinal (y-) bridge between Up(I,J) and Up(I,J+1),
// frame (o, o+h); blockIdx.z == 1: latitudinal (x-) bridge between Up(I,J)
// and Up(I+1,J), frame (o+h, o). Both run levels 1..h-1 of half cycle g0.
// In "along/across" coordinates (u along the bridge, w across it) the two are
// the same; (x, y) = (u, w) for the y-bridge and (w, u) for the x-bridge.
template <class Op>
__global__ void __launch_bounds__(256) bridge_kernel(Op op, Geom G, const typename Op::S *up,
                                                     typename Op::S *br, u64 g0) {
    typedef typename Op::S S;
    constexpr int NV = Op::NV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = G.n, h = n / 2, P = n + 2, plane = P * P;
    S *bufs[2];
    bufs[0] = reinterpret_cast<S *>(smem_raw);
    bufs[1] = bufs[0] + NV * plane;
    S *aux = bufs[1] + NV * plane;
    const int I = blockIdx.x, J = blockIdx.y;
    const bool xb = blockIdx.z == 1;
    const int slot = J * G.T + I;
    // low tile: Up(I,J); high tile: Up(I,J+1) or Up(I+1,J)
    const int hi_slot = xb ? (J * G.T + (I + 1 == G.T ? 0 : I + 1))
                           : ((J + 1 == G.Q ? 0 : J + 1) * G.T + I);
    // the low tile's panel facing the bridge (S or E) and the high tile's (N or W)
    const int lo_side = xb ? 3 : 1, hi_side = xb ? 2 : 0;
    // output sides: y-bridge W (low-u) / E (high-u); x-bridge N (low-u) / S (high-u)
    const int out_lo = xb ? 0 : 2, out_hi = xb ? 1 : 3;
    // across-offset of each output line start: y-bridge W starts at h-k (south
    // corner), E at h-k-2 (north corner); x-bridge N at h-k-2 (west), S at h-k (east)
    const int lo_w_shift = xb ? -2 : 0, hi_w_shift = xb ? 0 : -2;

    // prefetch the input strips of level 0 into buffer 0
    auto load_strips = [&](int k, S *dst) {
        const int L = n - 2 * k, L2 = 2 * L;
        const size_t off = (size_t)2 * k * (n - k + 1);
        for (int e = threadIdx.x; e < 2 * L2; e += blockDim.x) {
            const int which = e >= L2, r = e - which * L2, d = r >= L, p = r - d * L;
            const int uu = k + p;
            const int ww = which ? h + k + d : h - 1 - k - d;
            const int x = xb ? ww : uu, y = xb ? uu : ww;
            const S *src = up + ((size_t)(which ? hi_slot : slot) * 4 + (which ? hi_side : lo_side)) * NV * G.PS +
                           off + d * L + p;
#pragma unroll
            for (int v = 0; v < NV; ++v)
                async_copy(dst + v * plane + (y + 1) * P + (x + 1), src + (size_t)v * G.PS);
        }
        async_commit();
    };
    load_strips(0, bufs[0]);
    async_wait();
    __syncthreads();
    for (int k = 0; k < h; ++k) {
        S *cur = bufs[k & 1];
        S *nxt = bufs[(k + 1) & 1];
        // bridge panels of level k
        {
            const int L = 2 * k + 2, L2 = 2 * L;
            const size_t off = (size_t)2 * k * (k + 1);
            for (int e = threadIdx.x; e < 2 * L2; e += blockDim.x) {
                const int which = e >= L2, r = e - which * L2, d = r >= L, p = r - d * L;
                const int uu = which ? n - 1 - k - d : k + d;
                const int ww = h - k + (which ? hi_w_shift : lo_w_shift) + p;
                const int x = xb ? ww : uu, y = xb ? uu : ww;
                S *dst = br + ((size_t)slot * 4 + (which ? out_hi : out_lo)) * NV * G.PS + off + d * L + p;
#pragma unroll
                for (int v = 0; v < NV; ++v) dst[(size_t)v * G.PS] = cur[v * plane + (y + 1) * P + (x + 1)];
            }
        }
        if (k + 1 < h) {
            load_strips(k + 1, nxt);   // disjoint from the rectangle computed below
            const u64 g = g0 + k;
            const int u0 = k + 1, uw = n - 2 * k - 2, w0 = h - k - 1, ww = 2 * k + 2;
            if (xb)
                compute_rect(op, (int)(g % Op::NST), g, cur, nxt, aux, P, w0, u0, ww, uw);
            else
                compute_rect(op, (int)(g % Op::NST), g, cur, nxt, aux, P, u0, w0, uw, ww);
            async_wait();
        }
        __syncthreads();
    }
}

// --------------------------------------------- DownwardPyramid (Algorithm 5)
// Down(I,J) in frame (o+h, o+h): levels 1..h of half cycle g0 from the bridge
// panels. Ends with the full tile at level h in buffer (h & 1).
template <class Op>
__device__ __forceinline__ void down_body(const Op &op, const Geom &G, typename Op::S *buf0,
                                          typename Op::S *buf1, typename Op::S *aux, int P,
                                          const typename Op::S *br, u64 g0) {
    typedef typename Op::S S;
    constexpr int NV = Op::NV;
    const int n = G.n, h = n / 2, plane = P * P;
    const int I = blockIdx.x, J = blockIdx.y;
    const int slot = J * G.T + I;
    const int east = J * G.T + (I + 1 == G.T ? 0 : I + 1);
    const int south = (J + 1 == G.Q ? 0 : J + 1) * G.T + I;
    auto load_ring = [&](int k, S *dst) {
        const int L = 2 * k + 2, L2 = 2 * L;
        const size_t off = (size_t)2 * k * (k + 1);
        for (int e = threadIdx.x; e < 4 * L2; e += blockDim.x) {
            const int side = e / L2, r = e - side * L2, d = r >= L, p = r - d * L;
            int x, y, src_slot, src_side;
            switch (side) {
                case 0:  // west side <- E panel of y-bridge(I,J)
                    x = h - 1 - k - d; y = h - k - 2 + p; src_slot = slot; src_side = 3; break;
                case 1:  // east side <- W panel of y-bridge(I+1,J)
                    x = h + k + d; y = h - k + p; src_slot = east; src_side = 2; break;
                case 2:  // north side <- S panel of x-bridge(I,J)
                    x = h - k + p; y = h - 1 - k - d; src_slot = slot; src_side = 1; break;
                default:  // south side <- N panel of x-bridge(I,J+1)
                    x = h - k - 2 + p; y = h + k + d; src_slot = south; src_side = 0; break;
            }
            const S *src = br + ((size_t)src_slot * 4 + src_side) * NV * G.PS + off + d * L + p;
#pragma unroll
            for (int v = 0; v < NV; ++v)
                async_copy(dst + v * plane + (y + 1) * P + (x + 1), src + (size_t)v * G.PS);
        }
        async_commit();
    };
    load_ring(0, buf0);
    async_wait();
    __syncthreads();
    for (int k = 0; k < h; ++k) {
        S *cur = (k & 1) ? buf1 : buf0;
        S *nxt = (k & 1) ? buf0 : buf1;
        if (k + 1 < h) load_ring(k + 1, nxt);   // disjoint from the square computed below
        const u64 g = g0 + k;
        compute_rect(op, (int)(g % Op::NST), g, cur, nxt, aux, P, h - k - 1, h - k - 1,
                     2 * k + 2, 2 * k + 2);
        async_wait();
        __syncthreads();
    }
}

// K3: octahedron = Down of half cycle g0 (frame o+h) fused with the Up of half
// cycle g0+h in the same tile and frame; writes the next up panels.
template <class Op>
__global__ void __launch_bounds__(256) octahedron_kernel(Op op, Geom G, const typename Op::S *br,
                                                         typename Op::S *up, int o, u64 g0) {
    typedef typename Op::S S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = G.n, h = n / 2, P = n + 2, plane = P * P;
    S *buf0 = reinterpret_cast<S *>(smem_raw);
    S *buf1 = buf0 + Op::NV * plane;
    S *aux = buf1 + Op::NV * plane;
    down_body(op, G, buf0, buf1, aux, P, br, g0);
    // Down(I,J) in frame o+h is Up(I,J) of frame h when o = 0, and Up(I+1,J+1)
    // of frame 0 when o = h.
    int I = blockIdx.x, J = blockIdx.y;
    if (o != 0) {
        I = I + 1 == G.T ? 0 : I + 1;
        J = J + 1 == G.Q ? 0 : J + 1;
    }
    up_body(op, G, buf0, buf1, aux, P, g0 + h, up, J * G.T + I, h & 1);
}

// K4: final Down of an advance; writes the tile at level h to the state.
template <class Op>
__global__ void __launch_bounds__(256) down_kernel(Op op, Geom G, const typename Op::S *br,
                                                   typename Op::S *state, int o, u64 g0) {
    typedef typename Op::S S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = G.n, h = n / 2, P = n + 2, plane = P * P;
    S *buf0 = reinterpret_cast<S *>(smem_raw);
    S *buf1 = buf0 + Op::NV * plane;
    S *aux = buf1 + Op::NV * plane;
    down_body(op, G, buf0, buf1, aux, P, br, g0);
    const S *fin = (h & 1) ? buf1 : buf0;
    const size_t gplane = (size_t)G.nx * G.ny;
    const int x0 = o + h + blockIdx.x * n, y0 = o + h + blockIdx.y * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int b = e / n, a = e - b * n;
        int x = x0 + a; x -= x >= G.nx ? G.nx : 0;
        int y = y0 + b; y -= y >= G.ny ? G.ny : 0;
#pragma unroll
        for (int v = 0; v < Op::NV; ++v)
            state[v * gplane + (size_t)y * G.nx + x] = fin[v * plane + (b + 1) * P + (a + 1)];
    }
}

}  // namespace swept
