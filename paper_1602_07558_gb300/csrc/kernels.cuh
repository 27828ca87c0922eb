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
// E=3) and value plane, a packed array of n^2/2 + n elements (stride PS, padded
// to 16 bytes) holding the
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
// planes of (n+2) x (n+2) with the tile at offset (1, 1), or one for the updates
// computed in place (one_buffer), plus Op::AUX planes of scratch values that a
// level packs for its own rectangle (heat and wave: pair sums; Euler: the
// primitives; see aux_elems). With staging (template flag STG) a block also
// gets its whole input panel set (every level) in shared memory, brought in by
// TMA bulk copies at block start on one mbarrier, so the level loop touches no
// global memory for its inputs; without it, the panel strips are copied with
// cp.async. The tile bodies run on a team of threads (BlockTeam: the block;
// TeamOf<T>: a team of T threads with its own barrier and shared-memory slice).
#pragma once
#include <cuda_runtime.h>

#include "ops.cuh"

namespace swept {

struct Geom {
    int nx, ny;   // grid
    int n;        // tile side
    int T, Q;     // tiles along x and y
    int PS;       // panel stride per (slot, side, plane): n*n/2 + n rounded up to a
                  // multiple of 8 elements, so every panel starts on 16 bytes
};

__host__ __device__ inline int panel_stride(int n) { return ((n * n / 2 + n) + 7) & ~7; }

// The geometry a swept kernel works with: NC > 0 fixes the tile side at compile
// time (the launch picks such an instantiation only when G.n == NC), so every
// shared-memory pitch and plane offset of the inlined level code is a constant
// and folds into the load and store instructions; NC = 0 keeps G.n.
template <int NC>
__device__ __forceinline__ Geom fixed_tile(const Geom &G) {
    Geom g = G;
    if constexpr (NC > 0) g.n = NC;
    return g;
}

// Updates whose levels are computed in place in one level buffer.
template <class Op>
__host__ __device__ constexpr bool one_buffer() { return Op::INPLACE || Op::INPLACE_AFTER_AUX; }

// Row pitch of a level's packed flux planes (Euler): W + 2, or W + 4 when
// (W + 2) / 2 is even: an odd half-pitch keeps the 32 points of a column-pair
// walk on 32 banks (4-byte fluxes).
__host__ __device__ constexpr int flux_pitch(int W) { return ((W + 2) & 3) == 0 ? W + 4 : W + 2; }

// Elements of one aux plane of a swept block. A level packs its aux values for
// the rectangle it computes, grown by one: pair sums (heat, wave) with row
// pitch W + 1 over H + 1 rows, fluxes (Euler) with row pitch flux_pitch(W) over
// H + 2 rows. A bridge's levels (W + H = n) need at most (n/2 + 1)^2 and
// (n/2 + 3)^2; the pyramids' largest level is the whole n x n tile.
template <class Op>
__host__ __device__ inline size_t aux_elems(int n, bool bridge) {
    const size_t h = (size_t)n / 2;
    if constexpr (Op::INPLACE_AFTER_AUX)
        return bridge ? (h + 1) * (h + 1) : (size_t)(n + 1) * (n + 1);
    else
        return bridge ? (h + 3) * (h + 3) : (size_t)flux_pitch(n) * (n + 2);
}

// Dynamic shared memory of a swept block: level buffers (+ aux planes), then
// (when staged) the block's input panels, then an mbarrier. `bridge`: the plan
// of a bridge block, whose levels are smaller than the tile.
struct SmemPlan {
    size_t stage_off, bar_off, total;
};
// The downward pyramid's staged panels in two parts: rings 0..k1-1, then
// rings k1..h-1, brought in by a second bulk copy once the first part's rings
// are in the level buffer, so the staging area holds the larger part, not the
// whole panel set. k1 makes the parts most even among the levels whose ring
// offset 2 k1 (k1 + 1) starts on 16 bytes; 0: one part (no such level).
template <class S>
__host__ __device__ inline int stage_split(int n) {
    const int h = n / 2, ps = panel_stride(n);
    int best = 0, best_span = ps;
    for (int k = 1; k < h; ++k) {
        const int off = 2 * k * (k + 1);
        if ((off * (int)sizeof(S)) % 16) continue;
        const int span = off > ps - off ? off : ps - off;
        if (span < best_span) {
            best = k;
            best_span = span;
        }
    }
    return best;
}
// Elements of one (side, plane) slot of the downward pyramid's staging area.
template <class S>
__host__ __device__ inline int stage_span(int n) {
    const int k1 = stage_split<S>(n), ps = panel_stride(n);
    if (!k1) return ps;
    const int off = 2 * k1 * (k1 + 1);
    return off > ps - off ? off : ps - off;
}

template <class Op>
__host__ __device__ inline SmemPlan smem_plan(int n, int stage_segments, bool staged,
                                              bool bridge = false) {
    typedef typename Op::S S;
    const size_t P = (size_t)n + 2;
    const size_t levels = ((size_t)(one_buffer<Op>() ? 1 : 2) * Op::NV * P * P +
                           (size_t)Op::AUX * aux_elems<Op>(n, bridge)) * sizeof(S);
    SmemPlan pl;
    pl.stage_off = (levels + 15) & ~(size_t)15;
    // the downward pyramid (4 segments) stages its panels in two parts
    const size_t span = stage_segments == 4 ? (size_t)stage_span<S>(n) : (size_t)panel_stride(n);
    const size_t stage = staged ? (size_t)stage_segments * Op::NV * span * sizeof(S) : 0;
    pl.bar_off = (pl.stage_off + stage + 7) & ~(size_t)7;
    pl.total = pl.bar_off + (staged && stage_segments ? 16 : 0);   // two mbarriers
    return pl;
}

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
    if constexpr (sizeof(S) == 4 || sizeof(S) == 8 || sizeof(S) == 16) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem_src),
                     "n"((int)sizeof(S)));
    } else {
        *smem_dst = *gmem_src;       // 2-byte elements: cp.async has no 2-byte form
    }
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void async_wait() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---- TMA bulk copies (global -> shared) completed on an mbarrier.
// All waits are bounded: after kSpinLimit polls the block records a timeout in
// the error word (if any) and gives up instead of hanging.
constexpr long long kSpinLimit = 1LL << 22;

// Largest block of the launch-per-phase swept kernels (their register use stays
// far below the 128 a 512-thread block leaves each thread); the naive and the
// persistent kernels take at most 256.
constexpr int kMaxSweptThreads = 512;

// Largest block of the persistent kernel (it needs no more registers a thread
// than the launch-per-phase kernels).
constexpr int kMaxPersistentThreads = 512;

// Launch bounds of the single-grid swept kernels per update: the largest block
// and the blocks per SM its registers must allow. The FP64 heat kernels keep
// to 32 registers a thread (four 512-thread blocks' worth), so that three
// blocks of up to 512 threads per SM at tile 64, or eight of 256 at tile 32,
// are never short of registers; the other updates may use more.
template <class Op>
struct SweptBounds {
    static constexpr int kThreads = kMaxSweptThreads, kMinBlocks = 1;
};
template <>
struct SweptBounds<HeatOp> {
    static constexpr int kThreads = kMaxSweptThreads, kMinBlocks = 4;
};
// The compensated Euler kernels keep to 64 registers (two 512-thread blocks'
// worth), so three 256-thread blocks per SM are never short of registers.
template <class SS>
struct SweptBounds<EulerKahanOp<SS>> {
    static constexpr int kThreads = kMaxSweptThreads, kMinBlocks = 2;
};

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_inval(unsigned long long *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// The threads that run one tile work item: the whole block (BlockTeam: every
// kernel of the single-grid and per-class paths), or one of the block's teams
// of T threads (TeamOf<T>: the one-launch batch kernel, whose blocks, sized for
// the largest tile class, run several small tiles at once). rank() and size()
// take the place of threadIdx.x and blockDim.x, sync() of the block barrier
// (a warp barrier, or a named barrier per team), index() picks the team's
// slice of shared memory.
struct BlockTeam {
    static constexpr int kSize = 0;
    __device__ __forceinline__ static unsigned rank() { return threadIdx.x; }
    __device__ __forceinline__ static unsigned size() { return blockDim.x; }
    __device__ __forceinline__ static int index() { return 0; }
    __device__ __forceinline__ static void sync() { __syncthreads(); }
    __device__ __forceinline__ static int sync_or(int p) { return __syncthreads_or(p); }
};
constexpr int kMaxTeams = 15;   // named barriers 1..15 (0 is the block's)
template <int T>
struct TeamOf {
    static_assert(T >= 32 && T % 32 == 0, "a team is whole warps");
    static constexpr int kSize = T;
    __device__ __forceinline__ static unsigned rank() { return threadIdx.x % T; }
    __device__ __forceinline__ static unsigned size() { return T; }
    __device__ __forceinline__ static int index() { return (int)threadIdx.x / T; }
    __device__ __forceinline__ static void sync() {
        if constexpr (T == 32)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;\n" ::"r"(1 + index()), "n"(T) : "memory");
    }
    __device__ __forceinline__ static int sync_or(int p) {
        if constexpr (T == 32) {
            __syncwarp();
            return __any_sync(0xffffffffu, p);
        } else {
            int r;
            asm volatile(
                "{\n .reg .pred q, o;\n setp.ne.s32 q, %1, 0;\n"
                " bar.red.or.pred o, %2, %3, q;\n selp.s32 %0, 1, 0, o;\n}\n"
                : "=r"(r)
                : "r"(p), "r"(1 + index()), "n"(T)
                : "memory");
            return r;
        }
    }
};

// A team's slice of the block's dynamic shared memory at tile side n: the
// largest swept block's plan (four staged panel segments when STG), rounded
// up to 128 bytes; the whole of it for a BlockTeam.
template <class Op, bool STG>
__host__ __device__ inline size_t team_slice(int n) {
    return (smem_plan<Op>(n, 4, STG).total + 127) & ~(size_t)127;
}
template <class Op, bool STG, class Tm>
__device__ __forceinline__ unsigned char *team_smem(int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (Tm::kSize == 0)
        return smem_raw;
    else
        return smem_raw + (size_t)Tm::index() * team_slice<Op, STG>(n);
}

// Every thread of the team waits for phase 0 of `bar`; returns false (the same
// for the whole team) if the wait gave up, after recording it in *err.
template <class Tm = BlockTeam>
__device__ __forceinline__ bool block_wait_bulk(unsigned long long *bar, int *err) {
    bool ok = false;
    for (long long it = 0; it < kSpinLimit && !ok; ++it) ok = mbar_try_wait(bar, 0);
    const int bad = Tm::sync_or(!ok);
    if (bad) {
        if (Tm::rank() == 0) {
            if (err) atomicExch(err, 1);
            for (long long it = 0; it < kSpinLimit; ++it)   // let copies in flight land
                if (mbar_try_wait(bar, 0)) break;
        }
        Tm::sync();
        return false;
    }
    return true;
}

// Threads take consecutive points of a W-wide rectangle (point e = t, t + T,
// t + 2T, ... in row order, T = blockDim), so warps stay full; the (column,
// row) of the next point follows by adding (T mod W, T div W) with a carry,
// so a level costs two reciprocal divisions per thread, not one per point.
// q = floor(e / d) for 0 <= e < 2^20 and 1 <= d <= 2^10 via a binary32
// reciprocal: (e + 1/2) / d is at least 1/(2d) away from an integer, far more
// than the two roundings' error, so the truncation is exact.
__device__ __forceinline__ int div_small(int e, float rd) {
    return (int)(((float)e + 0.5f) * rd);
}
// The reciprocal div_small takes: an approximate binary32 reciprocal (within 2
// ulp, 2^-22 relative) keeps the truncation exact for e < 2^20, since the
// total relative error (under 1.25 * 2^-22) times (e + 1/2) / d stays below the
// 1/(2d) margin.
__device__ __forceinline__ float recip_small(int d) { return __fdividef(1.0f, (float)d); }

struct LinearWalk {
    int xx, yy, dq, dr;
    __device__ __forceinline__ LinearWalk(int W, int t, int T) {
        const float rw = recip_small(W);
        yy = div_small(t, rw);
        xx = t - yy * W;
        dq = div_small(T, rw);
        dr = T - dq * W;
    }
    __device__ __forceinline__ void next(int W) {
        xx += dr;
        yy += dq;
        if (xx >= W) {
            xx -= W;
            ++yy;
        }
    }
};

// Visit every point (xx, yy) of a W x H rectangle (W even), threads taking
// consecutive points. Tall rectangles narrower than a warp are taken in
// column-pair order (x = 2p + (q & 1), y = q >> 1 for the q-th point of pair
// p): with a row pitch whose half is odd (P = n + 2, n a multiple of 4) the 32
// consecutive points of a pair fall on 32 different banks, where row order maps
// several short rows onto the same banks. Other rectangles are taken in row
// order. (The shape rule is where a bank-count model of both orders at the
// stencil's five offsets favours column pairs for 4-byte elements; 8- and
// 2-byte elements measured no faster, and take row order: PAIRS = false.)
template <bool PAIRS, class Tm = BlockTeam, class F>
__device__ __forceinline__ void for_each_point(int W, int H, F &&f) {
    if (PAIRS && W < 32 && (H >= 14 || (W <= 10 && H >= 6))) {
        for (LinearWalk w(2 * H, (int)Tm::rank(), (int)Tm::size()); w.yy < (W >> 1);
             w.next(2 * H))
            f(2 * w.yy + (w.xx & 1), w.xx >> 1);
    } else {
        for (LinearWalk w(W, (int)Tm::rank(), (int)Tm::size()); w.yy < H; w.next(W)) f(w.xx, w.yy);
    }
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

// Neighbourhood accessor into the global state with periodic wrap; the three
// wrapped rows and columns are formed once per point.
template <class S>
struct GlobalAcc {
    const S *base;
    size_t plane;
    size_t row[3];
    int col[3];
    __device__ __forceinline__ GlobalAcc(const S *b, size_t pl, int nx, int ny, int x, int y)
        : base(b), plane(pl) {
        row[0] = (size_t)wrap_add(y, -1, ny) * nx;
        row[1] = (size_t)y * nx;
        row[2] = (size_t)wrap_add(y, 1, ny) * nx;
        col[0] = wrap_add(x, -1, nx);
        col[1] = x;
        col[2] = wrap_add(x, 1, nx);
    }
    __device__ __forceinline__ S operator()(int dx, int dy, int v) const {
        return base[v * plane + row[dy + 1] + col[dx + 1]];
    }
};

// Apply the point update on the local rectangle [x0, x0+W) x [y0, y0+H) of the
// level buffer src, writing dst. Threads take consecutive points of the
// rectangle so that warps stay full.
template <class Tm = BlockTeam, class Op>
__device__ __forceinline__ void compute_rect(const Op &op, int stage, u64 g,
                                             const typename Op::S *src, typename Op::S *dst,
                                             typename Op::S * /*aux*/, int P, int x0, int y0,
                                             int W, int H) {
    typedef typename Op::S S;
    const int plane = P * P;
    if (W <= 0) return;
    for (LinearWalk w(W, (int)Tm::rank(), (int)Tm::size()); w.yy < H; w.next(W)) {
        const int off = (y0 + w.yy + 1) * P + (x0 + w.xx + 1);
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
// Pass 2 reads only the centre and the pair sums, so it may write the level in
// place (src == dst); `mid` runs after the barrier between the passes, when
// no neighbour value of the level is read any more. The pair sums of a level
// are packed with row pitch W + 1 (entry e of pass 1 at aux[e]), so the aux
// buffer needs only the largest (W + 1)(H + 1) of the block's levels.
template <class Tm = BlockTeam, class Mid>
__device__ __forceinline__ void compute_rect_mid(const HeatOp &op, int, u64, const double *src,
                                                 double *dst, double *aux, int P, int x0, int y0,
                                                 int W, int H, Mid &&mid) {
    // (FP64-pipe bound: the per-point decode by reciprocal keeps independent
    // points per thread visible to the scheduler better than a carried walk)
    const int W1 = W + 1, cnt1 = W1 * (H + 1);
    const float rw1 = recip_small(W1), rw = recip_small(W);
    for (int e = Tm::rank(); e < cnt1; e += Tm::size()) {
        const int yy = div_small(e, rw1), xx = e - yy * W1;
        const int off = (y0 + yy) * P + (x0 + xx);      // point (x0-1+xx, y0-1+yy)
        aux[e] = __dadd_rn(src[off + 1], src[off + P]);
    }
    Tm::sync();
    mid();
    const int cnt = W * H;
    for (int e = Tm::rank(); e < cnt; e += Tm::size()) {
        const int yy = div_small(e, rw), xx = e - yy * W;
        const int off = (y0 + yy + 1) * P + (x0 + xx + 1);
        const int a = e + yy;                            // Pr(x-1, y-1); Pr(x, y) at a + W + 2
        const double c = src[off];
        const double sum = __dadd_rn(aux[a + W1 + 1], aux[a]);
        dst[off] = __fma_rn(op.r, __fma_rn(-4.0, c, sum), c);
    }
}

// Reduced-precision heat: each thread updates a column strip of up to R
// points of the rectangle. All of the strip's loads (R + 2 centre-column
// values, R compensations, R east and R west values: 4 per point instead of 6)
// are issued before its R independent updates, so they overlap, and the index
// walk runs once per strip; full strips take a path without per-row guards.
// Same values as HeatKahanOp::operator().
template <class SS, int R, bool FULL>
__device__ __forceinline__ void heat_kahan_strip(const HeatKahanOp<SS> &op,
                                                 const SS *__restrict__ src, SS *__restrict__ dst,
                                                 int P, int plane, int off, int rows) {
    typedef Store<SS> St;
    float u[R + 2], cv[R], ue[R], uw[R];
#pragma unroll
    for (int r = 0; r < R + 2; ++r)              // u[r]: row r - 1 of the strip, -1 .. rows
        u[r] = (FULL || r <= rows + 1) ? St::ld(src[off + (r - 1) * P]) : 0.0f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int o = off + r * P;
        const bool in = FULL || r < rows;
        cv[r] = in ? St::ld(src[plane + o]) : 0.0f;
        ue[r] = in ? St::ld(src[o + 1]) : 0.0f;
        uw[r] = in ? St::ld(src[o - 1]) : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (FULL || r < rows)
            op.update(u[r + 1], cv[r], ue[r], u[r + 2], uw[r], u[r], dst[off + r * P],
                      dst[plane + off + r * P]);
}

template <class Tm, int R, class SS>
__device__ __forceinline__ void heat_kahan_rect(const HeatKahanOp<SS> &op,
                                                const SS *__restrict__ src, SS *__restrict__ dst,
                                                int P, int x0, int y0, int W, int H) {
    const int plane = P * P;
    const int nb = (H + R - 1) / R;
    for (LinearWalk w(W, (int)Tm::rank(), (int)Tm::size()); w.yy < nb; w.next(W)) {
        const int yb = w.yy * R;
        const int rows = H - yb;
        const int off = (y0 + yb + 1) * P + (x0 + w.xx + 1);
        if (rows >= R)
            heat_kahan_strip<SS, R, true>(op, src, dst, P, plane, off, R);
        else
            heat_kahan_strip<SS, R, false>(op, src, dst, P, plane, off, rows);
    }
}
// Strips of 4 points at tile 64, of 2 on smaller tiles, whose short levels
// have fewer strips to share among the threads (measured: the 1,024-grid
// batch at tiles 16 and 32 247 -> 262 G updates/s with strips of 2, the 2048²
// grid at tile 64 421 -> 410 with strips of 2 and 379 with strips of 8).
template <class Tm = BlockTeam, class SS>
__device__ __forceinline__ void compute_rect(const HeatKahanOp<SS> &op, int, u64,
                                             const SS *__restrict__ src, SS *__restrict__ dst,
                                             SS *, int P, int x0, int y0, int W, int H) {
    if (W <= 0 || H <= 0) return;
    if (P > 34)
        heat_kahan_rect<Tm, 4>(op, src, dst, P, x0, y0, W, H);
    else
        heat_kahan_rect<Tm, 2>(op, src, dst, P, x0, y0, W, H);
}

// Euler: the primitives (u, v, p, E + p) of every point of the rectangle grown
// by one are formed once per level into 4 aux planes (pass 1: one division and
// one evaluation of the pressure per point), and each point then forms the
// fluxes of its 4 neighbours from their primitives and conserved values (pass
// 2): F1-F3 at its east and west neighbours, G1-G3 at its south and north
// ones (one or two operations each), F0 = m and G0 = q being the level's own
// values. A point's primitives serve its 4 neighbours instead of being
// recomputed by each of them, and 4 planes (instead of 8 flux planes) keep the
// block small enough for two (FP64) or three (binary32) blocks per SM at
// n = 32. Same values as EulerOp::operator() (each flux is the same sequence
// of operations on the same operands).
// The aux planes of a level are packed: row pitch A = flux_pitch(W), plane
// pitch A (H + 2), so the aux buffer needs only the largest such rectangle of
// the block's levels (a bridge's levels are far smaller than a tile).
template <class Tm = BlockTeam>
__device__ __forceinline__ void compute_rect(const EulerOp &op, int stage, u64, const double *src,
                                             double *dst, double *aux, int P, int x0, int y0,
                                             int W, int H) {
    const int plane = P * P, w0 = stage == 0 ? 0 : 4;
    if (W <= 0 || H <= 0) return;
    const int A = flux_pitch(W), fp = A * (H + 2);
    for_each_point<false, Tm>(W + 2, H + 2, [&](int xx, int yy) {
        const int off = (y0 + yy) * P + (x0 + xx);     // point (x0-1+xx, y0-1+yy)
        const int a = yy * A + xx;
        double u, v, pr, Ep;
        op.prims(src[w0 * plane + off], src[(w0 + 1) * plane + off],
                 src[(w0 + 2) * plane + off], src[(w0 + 3) * plane + off], u, v, pr, Ep);
        aux[a] = u;
        aux[fp + a] = v;
        aux[2 * fp + a] = pr;
        aux[3 * fp + a] = Ep;
    });
    Tm::sync();
    for_each_point<false, Tm>(W, H, [&](int xx, int yy) {
        const int off = (y0 + yy + 1) * P + (x0 + xx + 1);
        const int a = (yy + 1) * A + xx + 1;
        const double *M = src + (w0 + 1) * plane + off, *Q = src + (w0 + 2) * plane + off;
        double FE[4], FW[4], GS[4], GN[4];
        op.xflux_p(M[1], Q[1], aux[a + 1], aux[2 * fp + a + 1], aux[3 * fp + a + 1], FE);
        op.xflux_p(M[-1], Q[-1], aux[a - 1], aux[2 * fp + a - 1], aux[3 * fp + a - 1], FW);
        op.yflux_p(M[P], Q[P], aux[fp + a + A], aux[2 * fp + a + A], aux[3 * fp + a + A], GS);
        op.yflux_p(M[-P], Q[-P], aux[fp + a - A], aux[2 * fp + a - A], aux[3 * fp + a - A], GN);
        FE[0] = M[1];
        FW[0] = M[-1];
        GS[0] = Q[P];
        GN[0] = Q[-P];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const double *Wc = src + (w0 + c) * plane + off;
            double res;
            op.combine(stage, c, Wc[0], Wc[1], Wc[-1], Wc[P], Wc[-P], __dsub_rn(FE[c], FW[c]),
                       __dsub_rn(GS[c], GN[c]), src[c * plane + off], res);
            // (in place, src == dst: the passed-through plane is already there)
            if (stage == 0) {
                if (src != dst) dst[c * plane + off] = src[c * plane + off];
                dst[(4 + c) * plane + off] = res;
            } else {
                dst[c * plane + off] = res;
                if (src != dst) dst[(4 + c) * plane + off] = src[(4 + c) * plane + off];
            }
        }
    });
}

// Euler in binary32 with reduced-precision storage: the same two passes as
// EulerOp (binary32 primitives of the grown rectangle in the aux planes, then
// the per-point fluxes and combination). Same values as
// EulerKahanOp::operator().
template <class Tm = BlockTeam, class SS>
__device__ __forceinline__ void compute_rect(const EulerKahanOp<SS> &op, int stage, u64,
                                             const SS *src, SS *dst, SS *aux_s, int P, int x0,
                                             int y0, int W, int H) {
    typedef Store<SS> St;
    float *aux = reinterpret_cast<float *>(aux_s);
    const int plane = P * P, w0 = stage == 0 ? 0 : 4;
    if (W <= 0 || H <= 0) return;
    const int A = flux_pitch(W), fp = A * (H + 2);   // packed as for EulerOp
    for_each_point<sizeof(SS) == 4, Tm>(W + 2, H + 2, [&](int xx, int yy) {
        const int off = (y0 + yy) * P + (x0 + xx);     // point (x0-1+xx, y0-1+yy)
        const int a = yy * A + xx;
        float u, v, pr, Ep;
        op.prims(St::ld(src[w0 * plane + off]), St::ld(src[(w0 + 1) * plane + off]),
                 St::ld(src[(w0 + 2) * plane + off]), St::ld(src[(w0 + 3) * plane + off]), u, v,
                 pr, Ep);
        aux[a] = u;
        aux[fp + a] = v;
        aux[2 * fp + a] = pr;
        aux[3 * fp + a] = Ep;
    });
    Tm::sync();
    for_each_point<sizeof(SS) == 4, Tm>(W, H, [&](int xx, int yy) {
        const int off = (y0 + yy + 1) * P + (x0 + xx + 1);
        const int a = (yy + 1) * A + xx + 1;
        const SS *M = src + (w0 + 1) * plane + off, *Q = src + (w0 + 2) * plane + off;
        const float mE = St::ld(M[1]), mW = St::ld(M[-1]), mS = St::ld(M[P]), mN = St::ld(M[-P]);
        const float qE = St::ld(Q[1]), qW = St::ld(Q[-1]), qS = St::ld(Q[P]), qN = St::ld(Q[-P]);
        float FE[4], FW[4], GS[4], GN[4];
        op.xflux(mE, qE, aux[a + 1], aux[2 * fp + a + 1], aux[3 * fp + a + 1], FE);
        op.xflux(mW, qW, aux[a - 1], aux[2 * fp + a - 1], aux[3 * fp + a - 1], FW);
        op.yflux(mS, qS, aux[fp + a + A], aux[2 * fp + a + A], aux[3 * fp + a + A], GS);
        op.yflux(mN, qN, aux[fp + a - A], aux[2 * fp + a - A], aux[3 * fp + a - A], GN);
        FE[0] = mE;
        FW[0] = mW;
        GS[0] = qS;
        GN[0] = qN;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const SS *Wc = src + (w0 + c) * plane + off;
            const float L = op.rate(St::ld(Wc[0]), St::ld(Wc[1]), St::ld(Wc[-1]), St::ld(Wc[P]),
                                    St::ld(Wc[-P]), __fsub_rn(FE[c], FW[c]),
                                    __fsub_rn(GS[c], GN[c]));
            // (in place, src == dst: the passed-through planes are already there)
            if (stage == 0) {
                dst[(4 + c) * plane + off] = op.midpoint(L, St::ld(src[c * plane + off]));
                if (src != dst) {
                    dst[c * plane + off] = src[c * plane + off];
                    dst[(8 + c) * plane + off] = src[(8 + c) * plane + off];
                }
            } else {
                const float u = St::ld(src[c * plane + off]), cc = St::ld(src[(8 + c) * plane + off]);
                op.accumulate(L, u, cc, dst[c * plane + off], dst[(8 + c) * plane + off]);
                if (src != dst) dst[(4 + c) * plane + off] = src[(4 + c) * plane + off];
            }
        }
    });
}

// Wave: the same pair-sum sharing as the heat update (pass 1 forms the
// east+south pair sums of the rectangle grown by one into the aux buffer,
// packed with row pitch W + 1), then
// u' = (2u - u_old) + C^2 d, u_old' = u. Pass 2 reads only the centre's two
// values and the pair sums, so it may write the level in place; `mid` runs
// between the passes.
template <class Tm = BlockTeam, class Mid>
__device__ __forceinline__ void compute_rect_mid(const WaveOp &op, int, u64, const double *src,
                                                 double *dst, double *aux, int P, int x0, int y0,
                                                 int W, int H, Mid &&mid) {
    const int plane = P * P;
    const int W1 = W + 1, cnt1 = W1 * (H + 1);
    const float rw1 = recip_small(W1), rw = recip_small(W);
    for (int e = Tm::rank(); e < cnt1; e += Tm::size()) {
        const int yy = div_small(e, rw1), xx = e - yy * W1;
        const int off = (y0 + yy) * P + (x0 + xx);      // point (x0-1+xx, y0-1+yy)
        aux[e] = __dadd_rn(src[off + 1], src[off + P]);
    }
    Tm::sync();
    mid();
    const int cnt = W * H;
    for (int e = Tm::rank(); e < cnt; e += Tm::size()) {
        const int yy = div_small(e, rw), xx = e - yy * W;
        const int off = (y0 + yy + 1) * P + (x0 + xx + 1);
        const int a = e + yy;                            // packed as for the heat update
        const double c = src[off], old = src[plane + off];
        const double d = __fma_rn(-4.0, c, __dadd_rn(aux[a + W1 + 1], aux[a]));
        dst[off] = __fma_rn(op.C2, d, __dsub_rn(__dmul_rn(2.0, c), old));
        dst[plane + off] = c;
    }
}

// One level of a rectangle: level k+1 on [x0, x0+W) x [y0, y0+H) from level k
// in `cur`, into `nxt` (the same buffer for in-place updates). `next` copies
// the next level's ring or strip into `nxt`: for INPLACE_AFTER_AUX updates
// after the level's first pass (it overwrites neighbour values that pass
// reads), otherwise before the computation (the caller's prefetch).
template <class Tm = BlockTeam, class Op, class Next>
__device__ __forceinline__ void level_step(const Op &op, int stage, u64 g,
                                           const typename Op::S *cur, typename Op::S *nxt,
                                           typename Op::S *aux, int P,
                                           int x0, int y0, int W, int H, Next &&next) {
    if constexpr (Op::INPLACE_AFTER_AUX) {
        compute_rect_mid<Tm>(op, stage, g, cur, nxt, aux, P, x0, y0, W, H, next);
    } else {
        next();
        compute_rect<Tm>(op, stage, g, cur, nxt, aux, P, x0, y0, W, H);
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

// Panel writes in element pairs, one store per pair (else one per element).
template <class S>
__host__ __device__ constexpr bool pair_stores() { return true; }

// One store of two consecutive panel elements: 16 bytes for 8-byte elements,
// 8 for 4-byte, 4 for 2-byte (dst aligned to the pair: every panel line starts
// at an even element and has an even length, and panels start on 64 bytes).
template <class S>
__device__ __forceinline__ void store_pair(S *dst, S a, S b) {
    if constexpr (sizeof(S) == 8) {
        unsigned long long x, y;
        memcpy(&x, &a, 8);
        memcpy(&y, &b, 8);
        asm volatile("st.global.v2.b64 [%0], {%1, %2};\n" ::"l"(dst), "l"(x), "l"(y) : "memory");
    } else if constexpr (sizeof(S) == 4) {
        unsigned x, y;
        memcpy(&x, &a, 4);
        memcpy(&y, &b, 4);
        asm volatile("st.global.v2.b32 [%0], {%1, %2};\n" ::"l"(dst), "r"(x), "r"(y) : "memory");
    } else {
        static_assert(sizeof(S) == 2, "2-, 4- or 8-byte elements");
        unsigned short x, y;
        memcpy(&x, &a, 2);
        memcpy(&y, &b, 2);
        const unsigned xy = (unsigned)x | ((unsigned)y << 16);   // a at the lower address
        asm volatile("st.global.b32 [%0], %1;\n" ::"l"(dst), "r"(xy) : "memory");
    }
}

// Write level k of the 4 up panels of the tile held in cur to slot `slot`.
// The block's threads take the level's 4 sides x 2 lines x L elements in
// order (element e: line e div L, position e mod L), so short lines at deep
// levels or small tiles do not leave most lanes idle; the elements go out in
// pairs, one store each (L = n - 2k is even): 16 bytes for 8-byte elements.
template <class S, int NV, class Tm = BlockTeam>
__device__ __forceinline__ void write_up_panels(const S *cur, int P, const Geom &G, int k,
                                                S *up, int slot) {
    const int n = G.n, L = n - 2 * k, plane = P * P;
    const int off = 2 * k * (n - k + 1);
    S *tile = up + (size_t)slot * 4 * NV * G.PS + off;
    if constexpr (pair_stores<S>()) {
        const int Lh = L >> 1;
        const float rh = recip_small(Lh);
        for (int e = Tm::rank(); e < 4 * L; e += Tm::size()) {
            const int q = div_small(e, rh);      // side * 2 + line
            const int p = 2 * (e - q * Lh), side = q >> 1, d = q & 1;
            int a, b;
            up_panel_xy(side, n, k, d, p, a, b);
            const S *src = cur + (b + 1) * P + (a + 1);
            const int step = side < 2 ? 1 : P;   // N, S lines run along x; W, E along y
            S *dst = tile + side * NV * G.PS + d * L + p;
#pragma unroll
            for (int v = 0; v < NV; ++v)
                store_pair(dst + v * G.PS, src[v * plane], src[v * plane + step]);
        }
        return;
    }
    const float rl = recip_small(L);
    for (int e = Tm::rank(); e < 8 * L; e += Tm::size()) {
        const int q = div_small(e, rl);          // side * 2 + line
        const int p = e - q * L, side = q >> 1, d = q & 1;
        int a, b;
        up_panel_xy(side, n, k, d, p, a, b);
        const S *src = cur + (b + 1) * P + (a + 1);
        S *dst = tile + side * NV * G.PS + d * L + p;
#pragma unroll
        for (int v = 0; v < NV; ++v) dst[v * G.PS] = src[v * plane];
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
    GlobalAcc<S> acc(in, plane, G.nx, G.ny, x, y);
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

// Reduced-precision heat, naive path: lane = column, each warp walks ROWS rows
// keeping north and centre in registers (4 loads per point).
template <class SS, int ROWS>
__global__ void __launch_bounds__(256) naive_heat_kahan_kernel(HeatKahanOp<SS> op, Geom G,
                                                               const SS *in, SS *out) {
    typedef Store<SS> St;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const int y0 = (blockIdx.y * 8 + warp) * ROWS;
    if (x >= G.nx || y0 >= G.ny) return;
    const int y1 = min(y0 + ROWS, G.ny);
    const size_t nx = G.nx, plane = (size_t)G.nx * G.ny;
    const int xw = x == 0 ? G.nx - 1 : x - 1, xe = x + 1 == G.nx ? 0 : x + 1;
    const int ym = y0 == 0 ? G.ny - 1 : y0 - 1;
    float un = St::ld(in[(size_t)ym * nx + x]), uc = St::ld(in[(size_t)y0 * nx + x]);
    for (int y = y0; y < y1; ++y) {
        const int ys = y + 1 == G.ny ? 0 : y + 1;
        const size_t row = (size_t)y * nx;
        const float us = St::ld(in[(size_t)ys * nx + x]);
        op.update(uc, St::ld(in[plane + row + x]), St::ld(in[row + xe]), us, St::ld(in[row + xw]),
                  un, out[row + x], out[plane + row + x]);
        un = uc;
        uc = us;
    }
}

// ------------------------------------------------------- UpwardPyramid (Alg. 1)
// Shared body: tile at level 0 of half cycle g0 is in buffer 0; builds levels
// 1..h-1 and writes the up panels of levels 0..h-1 to slot `slot`.
template <class Op, class Tm = BlockTeam>
__device__ __forceinline__ void up_body(const Op &op, const Geom &G, typename Op::S *buf0,
                                        typename Op::S *buf1, typename Op::S *aux, int P, u64 g0,
                                        typename Op::S *up, int slot, int first_parity) {
    typedef typename Op::S S;
    const int n = G.n, h = n / 2;
    for (int k = 0; k < h; ++k) {
        const int par = (first_parity + k) & 1;
        const S *cur = par ? buf1 : buf0;
        S *nxt = par ? buf0 : buf1;
        write_up_panels<S, Op::NV, Tm>(cur, P, G, k, up, slot);
        // panels read before the level is overwritten (INPLACE_AFTER_AUX updates
        // overwrite it only after the barrier between their two passes)
        if constexpr (Op::INPLACE) Tm::sync();
        if (k + 1 < h) {
            const u64 g = g0 + k;
            level_step<Tm>(op, (int)(g % Op::NST), g, cur, nxt, aux, P, k + 1, k + 1, n - 2 * k - 2,
                       n - 2 * k - 2, [] {});
        }
        Tm::sync();
    }
}

// K1: first upward pyramid of an advance, frame offset o, reading the state.
template <class Op, class Tm = BlockTeam, bool STG = false>
__device__ __forceinline__ void up_tile(const Op &op, const Geom &G, const typename Op::S *state,
                                        typename Op::S *up, int o, u64 g0, int I, int J) {
    typedef typename Op::S S;
    unsigned char *smem_raw = team_smem<Op, STG, Tm>(G.n);
    const int n = G.n, P = n + 2, plane = P * P;
    S *buf0 = reinterpret_cast<S *>(smem_raw);
    S *buf1 = one_buffer<Op>() ? buf0 : buf0 + Op::NV * plane;   // one buffer for in-place levels
    S *aux = buf1 + Op::NV * plane;
    const size_t gplane = (size_t)G.nx * G.ny;
    const int x0 = o + I * n, y0 = o + J * n;
    for (int e = Tm::rank(); e < n * n; e += Tm::size()) {
        const int b = e / n, a = e - b * n;
        int x = x0 + a; x -= x >= G.nx ? G.nx : 0;
        int y = y0 + b; y -= y >= G.ny ? G.ny : 0;
#pragma unroll
        for (int v = 0; v < Op::NV; ++v)
            buf0[v * plane + (b + 1) * P + (a + 1)] = state[v * gplane + (size_t)y * G.nx + x];
    }
    Tm::sync();
    up_body<Op, Tm>(op, G, buf0, buf1, aux, P, g0, up, J * G.T + I, 0);
}

template <class Op, int NC = 0>
__global__ void __launch_bounds__(SweptBounds<Op>::kThreads, SweptBounds<Op>::kMinBlocks)
up_kernel(Op op, Geom G, const typename Op::S *state, typename Op::S *up, int o, u64 g0) {
    up_tile(op, fixed_tile<NC>(G), state, up, o, g0, blockIdx.x, blockIdx.y);
}

// ------------------------------------------- Bridges (Algorithms 2 and 3)
// blockIdx.z == 0: longitudinal (y-) bridge between Up(I,J) and Up(I,J+1),
// frame (o, o+h); blockIdx.z == 1: latitudinal (x-) bridge between Up(I,J)
// and Up(I+1,J), frame (o+h, o). Both run levels 1..h-1 of half cycle g0.
// In "along/across" coordinates (u along the bridge, w across it) the two are
// the same; (x, y) = (u, w) for the y-bridge and (w, u) for the x-bridge.
template <class Op, bool STG, class Tm = BlockTeam>
__device__ __forceinline__ void bridge_tile(const Op &op, const Geom &G, const typename Op::S *up,
                                            typename Op::S *br, u64 g0, int *err, int I, int J,
                                            bool xb) {
    typedef typename Op::S S;
    constexpr int NV = Op::NV;
    unsigned char *smem_raw = team_smem<Op, STG, Tm>(G.n);
    const int n = G.n, h = n / 2, P = n + 2, plane = P * P;
    S *bufs[2];
    bufs[0] = reinterpret_cast<S *>(smem_raw);
    bufs[1] = one_buffer<Op>() ? bufs[0] : bufs[0] + NV * plane;   // one buffer for in-place levels
    S *aux = bufs[1] + NV * plane;
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
    const S *seg[2] = {up + ((size_t)slot * 4 + lo_side) * NV * G.PS,
                       up + ((size_t)hi_slot * 4 + hi_side) * NV * G.PS};

    const S *stg = nullptr;
    if constexpr (STG) {
        // the two input panels (every level) arrive in shared memory by TMA
        const SmemPlan pl = smem_plan<Op>(n, 2, true, true);
        S *st = reinterpret_cast<S *>(smem_raw + pl.stage_off);
        unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + pl.bar_off);
        if (Tm::rank() == 0) mbar_init(bar, 1);
        Tm::sync();
        if (Tm::rank() == 0) {
            const unsigned bytes = (unsigned)(G.PS * sizeof(S));
            mbar_expect_tx(bar, 2 * NV * bytes);
            for (int w = 0; w < 2; ++w)
                for (int v = 0; v < NV; ++v)
                    bulk_g2s(st + (w * NV + v) * G.PS, seg[w] + (size_t)v * G.PS, bytes, bar);
        }
        if (!block_wait_bulk<Tm>(bar, err)) return;
        if (Tm::rank() == 0) mbar_inval(bar);   // the block may stage again (persistent form)
        stg = st;
    }
    auto load_strips = [&](int k, S *dst) {
        const int L = n - 2 * k;
        const int off = 2 * k * (n - k + 1);
        const float rl = recip_small(L);
        for (int e = Tm::rank(); e < 4 * L; e += Tm::size()) {   // 2 strips x 2 lines x L
            const int q = div_small(e, rl);
            const int p = e - q * L, which = q >> 1, d = q & 1;
            const int ww = which ? h + k + d : h - 1 - k - d;
            const int uu = k + p;
            const int x = xb ? ww : uu, y = xb ? uu : ww;
            S *dd = dst + (y + 1) * P + (x + 1);
            if constexpr (STG) {
                const S *src = stg + which * NV * G.PS + off + d * L + p;
#pragma unroll
                for (int v = 0; v < NV; ++v) dd[v * plane] = src[v * G.PS];
            } else {
                const S *src = seg[which] + off + d * L + p;
#pragma unroll
                for (int v = 0; v < NV; ++v) async_copy(dd + v * plane, src + (size_t)v * G.PS);
            }
        }
        if constexpr (!STG) async_commit();
    };
    // strips copied level by level (staged panels; in-place levels, whose one
    // buffer cannot hold two levels' strips), or all at once before the first
    // level: strips of one parity never overlap, and no level's rectangle,
    // reads or panel reads touch a later level's strip, so the copies' latency
    // is paid once per tile instead of once per level
    constexpr bool per_level = STG || one_buffer<Op>();
    if constexpr (per_level) {
        load_strips(0, bufs[0]);
    } else {
        for (int k = 0; k < h; ++k) load_strips(k, bufs[k & 1]);
    }
    if constexpr (!STG) async_wait();
    Tm::sync();
    for (int k = 0; k < h; ++k) {
        S *cur = bufs[k & 1];
        S *nxt = bufs[(k + 1) & 1];
        // bridge panels of level k (2 sides x 2 lines x L, threads in order;
        // elements in pairs, one store each: L = 2k + 2 is even)
        if constexpr (pair_stores<S>()) {
            const int L = 2 * k + 2, Lh = k + 1;
            const int off = 2 * k * (k + 1);
            const float rh = recip_small(Lh);
            const int step = xb ? 1 : P;      // a line runs along the across axis
            for (int e = Tm::rank(); e < 2 * L; e += Tm::size()) {
                const int q = div_small(e, rh);
                const int p = 2 * (e - q * Lh), which = q >> 1, d = q & 1;
                const int uu = which ? n - 1 - k - d : k + d;
                const int ww = h - k + (which ? hi_w_shift : lo_w_shift) + p;
                const int x = xb ? ww : uu, y = xb ? uu : ww;
                S *dst = br + ((size_t)slot * 4 + (which ? out_hi : out_lo)) * NV * G.PS + off +
                         d * L + p;
                const S *src = cur + (y + 1) * P + (x + 1);
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    store_pair(dst + (size_t)v * G.PS, src[v * plane], src[v * plane + step]);
            }
        } else {
            const int L = 2 * k + 2;
            const int off = 2 * k * (k + 1);
            const float rl = recip_small(L);
            for (int e = Tm::rank(); e < 4 * L; e += Tm::size()) {
                const int q = div_small(e, rl);
                const int p = e - q * L, which = q >> 1, d = q & 1;
                const int uu = which ? n - 1 - k - d : k + d;
                const int ww = h - k + (which ? hi_w_shift : lo_w_shift) + p;
                const int x = xb ? ww : uu, y = xb ? uu : ww;
                S *dst = br + ((size_t)slot * 4 + (which ? out_hi : out_lo)) * NV * G.PS + off +
                         d * L + p;
                const S *src = cur + (y + 1) * P + (x + 1);
#pragma unroll
                for (int v = 0; v < NV; ++v) dst[(size_t)v * G.PS] = src[v * plane];
            }
        }
        // panels read before the strip copy below (INPLACE_AFTER_AUX updates
        // copy it only after the barrier between their two passes)
        if constexpr (Op::INPLACE) Tm::sync();
        if (k + 1 < h) {
            // the next strip lies outside the rectangle below; it overlaps the
            // rectangle's outermost neighbours: INPLACE updates keep the planes
            // read there unchanged between the levels, INPLACE_AFTER_AUX ones
            // copy the strip once those neighbours are read
            auto next = [&] {
                if constexpr (per_level) load_strips(k + 1, nxt);
            };
            const u64 g = g0 + k;
            const int u0 = k + 1, uw = n - 2 * k - 2, w0 = h - k - 1, ww = 2 * k + 2;
            if (xb)
                level_step<Tm>(op, (int)(g % Op::NST), g, cur, nxt, aux, P, w0, u0, ww, uw, next);
            else
                level_step<Tm>(op, (int)(g % Op::NST), g, cur, nxt, aux, P, u0, w0, uw, ww, next);
            if constexpr (per_level && !STG) async_wait();
        }
        Tm::sync();
    }
}

template <class Op, bool STG, int NC = 0>
__global__ void __launch_bounds__(SweptBounds<Op>::kThreads, SweptBounds<Op>::kMinBlocks)
bridge_kernel(Op op, Geom G, const typename Op::S *up, typename Op::S *br, u64 g0, int *err) {
    bridge_tile<Op, STG>(op, fixed_tile<NC>(G), up, br, g0, err, blockIdx.x, blockIdx.y,
                         blockIdx.z == 1);
}

// --------------------------------------------- DownwardPyramid (Algorithm 5)
// Down(I,J) in frame (o+h, o+h): levels 1..h of half cycle g0 from the bridge
// panels. Ends with the full tile at level h in buffer (h & 1).
template <class Op, bool STG, class Tm = BlockTeam>
__device__ __forceinline__ bool down_body(const Op &op, const Geom &G, unsigned char *smem_raw,
                                          typename Op::S *buf0, typename Op::S *buf1,
                                          typename Op::S *aux, int P, const typename Op::S *br,
                                          u64 g0, int *err, int I, int J) {
    typedef typename Op::S S;
    constexpr int NV = Op::NV;
    const int n = G.n, h = n / 2, plane = P * P;
    const int slot = J * G.T + I;
    const int east = J * G.T + (I + 1 == G.T ? 0 : I + 1);
    const int south = (J + 1 == G.Q ? 0 : J + 1) * G.T + I;
    // ring side -> (source slot, source panel side): west <- E of y-bridge(I,J),
    // east <- W of y-bridge(I+1,J), north <- S of x-bridge(I,J), south <- N of x-bridge(I,J+1)
    const S *seg[4] = {br + ((size_t)slot * 4 + 3) * NV * G.PS, br + ((size_t)east * 4 + 2) * NV * G.PS,
                       br + ((size_t)slot * 4 + 1) * NV * G.PS, br + ((size_t)south * 4 + 0) * NV * G.PS};
    const S *stg = nullptr;
    // staged panels: part 0 (rings 0..k1-1, or all of them) at block start,
    // part 1 (rings k1..h-1) once part 0's last ring is in the level buffer
    int k1 = 0, span = 0, base = 0;
    unsigned long long *bar = nullptr;
    S *st = nullptr;
    auto stage_part = [&](int part) {   // called by the team's rank 0
        const int lo = part ? 2 * k1 * (k1 + 1) : 0;
        const int hi = (part || !k1) ? G.PS : 2 * k1 * (k1 + 1);
        const unsigned bytes = (unsigned)((hi - lo) * sizeof(S));
        mbar_expect_tx(bar + part, 4 * NV * bytes);
        for (int side = 0; side < 4; ++side)
            for (int v = 0; v < NV; ++v)
                bulk_g2s(st + (side * NV + v) * span, seg[side] + (size_t)v * G.PS + lo, bytes,
                         bar + part);
    };
    if constexpr (STG) {
        const SmemPlan pl = smem_plan<Op>(n, 4, true);
        st = reinterpret_cast<S *>(smem_raw + pl.stage_off);
        bar = reinterpret_cast<unsigned long long *>(smem_raw + pl.bar_off);
        k1 = stage_split<S>(n);
        span = stage_span<S>(n);
        if (Tm::rank() == 0) {
            mbar_init(bar, 1);
            mbar_init(bar + 1, 1);
        }
        Tm::sync();
        if (Tm::rank() == 0) stage_part(0);
        if (!block_wait_bulk<Tm>(bar, err)) return false;
        if (Tm::rank() == 0) mbar_inval(bar);
        stg = st;
    }
    auto load_ring = [&](int k, S *dst) {
        const int L = 2 * k + 2;
        const int off = 2 * k * (k + 1);
        const float rl = recip_small(L);
        for (int e = Tm::rank(); e < 8 * L; e += Tm::size()) {   // 4 sides x 2 lines x L
            const int q = div_small(e, rl);
            const int p = e - q * L, side = q >> 1, d = q & 1;
            // (x, y) of element p: x = bx + p ax, y = by + p ay
            int bx, by, ax, ay;
            switch (side) {
                case 0: bx = h - 1 - k - d; by = h - k - 2; ax = 0; ay = 1; break;   // west
                case 1: bx = h + k + d; by = h - k; ax = 0; ay = 1; break;           // east
                case 2: bx = h - k; by = h - 1 - k - d; ax = 1; ay = 0; break;       // north
                default: bx = h - k - 2; by = h + k + d; ax = 1; ay = 0; break;      // south
            }
            S *dd = dst + (by + 1 + p * ay) * P + (bx + 1 + p * ax);
            if constexpr (STG) {
                const S *src = stg + side * NV * span + (off - base) + d * L + p;
#pragma unroll
                for (int v = 0; v < NV; ++v) dd[v * plane] = src[v * span];
            } else {
                const S *src = seg[side] + off + d * L + p;
#pragma unroll
                for (int v = 0; v < NV; ++v) async_copy(dd + v * plane, src + (size_t)v * G.PS);
            }
        }
        if constexpr (!STG) async_commit();
    };
    // rings copied level by level (staged panels; in-place levels), or all at
    // once before the first level: rings of one parity never overlap and lie
    // outside every earlier level's square and reads, so the copies' latency
    // is paid once per tile
    constexpr bool per_level = STG || one_buffer<Op>();
    bool failed = false;
    // staged in two parts: once ring r (the last of part 0) is copied, the
    // staging area is free for part 1; ring k1 waits for part 1
    auto after_ring = [&](int r) {
        if constexpr (STG) {
            if (k1 && r == k1 - 1) {
                // this team's reads of the staging area come before the bulk
                // copy that overwrites it (generic -> async proxy)
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                Tm::sync();
                if (Tm::rank() == 0) stage_part(1);
            }
        }
    };
    auto before_ring = [&](int r) {
        if constexpr (STG) {
            if (k1 && r == k1) {
                if (!block_wait_bulk<Tm>(bar + 1, err)) failed = true;
                if (Tm::rank() == 0) mbar_inval(bar + 1);
                base = 2 * k1 * (k1 + 1);
            }
        }
    };
    if constexpr (per_level) {
        load_ring(0, buf0);
        after_ring(0);
    } else {
        for (int k = 0; k < h; ++k) load_ring(k, (k & 1) ? buf1 : buf0);
    }
    if constexpr (!STG) async_wait();
    Tm::sync();
    for (int k = 0; k < h; ++k) {
        S *cur = (k & 1) ? buf1 : buf0;
        S *nxt = (k & 1) ? buf0 : buf1;
        // the next ring lies outside the square below; it overlaps the square's
        // outermost neighbours: INPLACE updates keep the planes read there
        // unchanged between the levels, INPLACE_AFTER_AUX ones copy the ring
        // once those neighbours are read
        auto next = [&] {
            if constexpr (per_level)
                if (k + 1 < h) {
                    before_ring(k + 1);
                    load_ring(k + 1, nxt);
                    after_ring(k + 1);
                }
        };
        const u64 g = g0 + k;
        level_step<Tm>(op, (int)(g % Op::NST), g, cur, nxt, aux, P, h - k - 1, h - k - 1, 2 * k + 2,
                   2 * k + 2, next);
        if constexpr (per_level && !STG) async_wait();
        Tm::sync();
        if (failed) return false;
    }
    return true;
}

// K3: octahedron = Down of half cycle g0 (frame o+h) fused with the Up of half
// cycle g0+h in the same tile and frame; writes the next up panels.
template <class Op, bool STG, class Tm = BlockTeam>
__device__ __forceinline__ void octahedron_tile(const Op &op, const Geom &G,
                                                const typename Op::S *br, typename Op::S *up,
                                                int o, u64 g0, int *err, int I, int J) {
    typedef typename Op::S S;
    unsigned char *smem_raw = team_smem<Op, STG, Tm>(G.n);
    const int n = G.n, h = n / 2, P = n + 2, plane = P * P;
    S *buf0 = reinterpret_cast<S *>(smem_raw);
    S *buf1 = one_buffer<Op>() ? buf0 : buf0 + Op::NV * plane;   // one buffer for in-place levels
    S *aux = buf1 + Op::NV * plane;
    if (!down_body<Op, STG, Tm>(op, G, smem_raw, buf0, buf1, aux, P, br, g0, err, I, J)) return;
    // Down(I,J) in frame o+h is Up(I,J) of frame h when o = 0, and Up(I+1,J+1)
    // of frame 0 when o = h.
    if (o != 0) {
        I = I + 1 == G.T ? 0 : I + 1;
        J = J + 1 == G.Q ? 0 : J + 1;
    }
    up_body<Op, Tm>(op, G, buf0, buf1, aux, P, g0 + h, up, J * G.T + I, h & 1);
}

template <class Op, bool STG, int NC = 0>
__global__ void __launch_bounds__(SweptBounds<Op>::kThreads, SweptBounds<Op>::kMinBlocks)
octahedron_kernel(Op op, Geom G, const typename Op::S *br, typename Op::S *up, int o, u64 g0,
                  int *err) {
    octahedron_tile<Op, STG>(op, fixed_tile<NC>(G), br, up, o, g0, err, blockIdx.x, blockIdx.y);
}

// K4: final Down of an advance; writes the tile at level h to the state.
template <class Op, bool STG, class Tm = BlockTeam>
__device__ __forceinline__ void down_tile(const Op &op, const Geom &G, const typename Op::S *br,
                                          typename Op::S *state, int o, u64 g0, int *err, int I,
                                          int J) {
    typedef typename Op::S S;
    unsigned char *smem_raw = team_smem<Op, STG, Tm>(G.n);
    const int n = G.n, h = n / 2, P = n + 2, plane = P * P;
    S *buf0 = reinterpret_cast<S *>(smem_raw);
    S *buf1 = one_buffer<Op>() ? buf0 : buf0 + Op::NV * plane;   // one buffer for in-place levels
    S *aux = buf1 + Op::NV * plane;
    if (!down_body<Op, STG, Tm>(op, G, smem_raw, buf0, buf1, aux, P, br, g0, err, I, J)) return;
    const S *fin = (h & 1) ? buf1 : buf0;
    const size_t gplane = (size_t)G.nx * G.ny;
    const int x0 = o + h + I * n, y0 = o + h + J * n;
    for (int e = Tm::rank(); e < n * n; e += Tm::size()) {
        const int b = e / n, a = e - b * n;
        int x = x0 + a; x -= x >= G.nx ? G.nx : 0;
        int y = y0 + b; y -= y >= G.ny ? G.ny : 0;
#pragma unroll
        for (int v = 0; v < Op::NV; ++v)
            state[v * gplane + (size_t)y * G.nx + x] = fin[v * plane + (b + 1) * P + (a + 1)];
    }
}

template <class Op, bool STG, int NC = 0>
__global__ void __launch_bounds__(SweptBounds<Op>::kThreads, SweptBounds<Op>::kMinBlocks)
down_kernel(Op op, Geom G, const typename Op::S *br, typename Op::S *state, int o, u64 g0,
            int *err) {
    down_tile<Op, STG>(op, fixed_tile<NC>(G), br, state, o, g0, err, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------- persistent form
// One launch runs a whole swept advance: resident blocks take work items from
// an atomic queue in phase order (phase 1: every tile's first Up; then per half
// cycle j the y- and x-bridge items of every tile, two items per tile, then an
// octahedron item per tile, or the final Down items). Each tile has a counter
// of its finished items, and an item of half cycle j on tile t starts once
// every tile of t's periodic 3 x 3 neighbourhood has finished all its items of
// the previous phase (count >= 1 + 3j for a bridge, 3 + 3j for an octahedron
// or Down). That neighbourhood holds every producer of the item's inputs and
// every reader of the panels it overwrites (the frame shift moves a tile's
// panels by at most one slot), so the kernel boundaries of the
// launch-per-phase schedule are replaced by those waits. Items are taken in
// index order and every dependency has a smaller index, so the lowest
// unfinished item can always run: no deadlock, whatever number of blocks is
// resident. Panels written by one block are read by another after an acquire
// of the writer's release (and, for the TMA bulk copies of the staged form, a
// generic-to-async proxy fence); the unstaged form's element copies are
// ordinary reads after that acquire. Waits are bounded: on timeout the error
// word is set and the block stops.
// A dependency is at most one work item away (tens of microseconds); the
// default bound (about a second of 64 ns naps and polls) only catches a block
// that never finishes.
constexpr long long kPersistSpinLimit = 1LL << 24;

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void add_release(int *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Where a work item's tile lives: its grid's geometry, the grid's offsets in
// the (pooled) state and panel buffers, the tile's (I, J), and the index of the
// grid's first tile among the launch's tiles (its phase counters start there).
struct TileAt {
    Geom G;
    long long soff, poff;
    int I, J, base;
    const double *c;        // the grid's own update constants (nullptr: the launch's)
};

// One grid: tile index t = J T + I.
struct OneGrid {
    Geom G;
    __device__ __forceinline__ TileAt operator()(int t) const {
        TileAt w;
        w.G = G;
        w.soff = w.poff = 0;
        w.J = t / G.T;
        w.I = t - w.J * G.T;
        w.base = 0;
        w.c = nullptr;
        return w;
    }
};

// Work items of the persistent form for NT tiles and H half cycles: NT first
// Ups, then per half cycle 2 NT bridge items (tile t, y- then x-bridge) and NT
// octahedron or final Down items.
__host__ __device__ inline long long persistent_items(long long NT, long long H) {
    return NT * (1 + 3 * H);
}

// The work loop of the persistent form over NT tiles (all of one tile side n)
// located by `at`. `first` is the first work item taken (0; a positive value
// skips items, which only the wait-timeout self-test does: the skipped items
// are never counted, so every wait runs out).
// `trace` (nullptr: none) receives, per work item, the SM clock cycles its
// block spent waiting for the item's neighbourhood (trace[2 item]) and running
// the item up to its release (trace[2 item + 1]).
// One work item of the persistent form (every thread of the team calls it
// with the same item): wait for the item's neighbourhood, run it, count it.
// Returns false when a wait gave up (the team must stop).
template <class Op, bool STG, int NC = 0, class Tm = BlockTeam, class Loc>
__device__ __forceinline__ bool persistent_item(const Op &op, const Loc &at, int NT, int n,
                                                typename Op::S *state, typename Op::S *upp,
                                                typename Op::S *br, int *stage, int H, u64 g0,
                                                int *err, int item, long long spin_limit,
                                                unsigned *trace) {
    __shared__ int s_fail_team[kMaxTeams];
    int &s_fail = s_fail_team[Tm::index()];
    long long t_start = 0, t_ready = 0;
    const int h = (NC > 0 ? NC : n) / 2;
    // decode: kind 0 first Up, 1 bridge (xb: x-bridge), 2 octahedron or Down
    int kind, t, j = 0, need = 0;
    bool xb = false;
    if (item < NT) {
        kind = 0;
        t = item;
    } else {
        const int r = item - NT;
        j = r / (3 * NT);
        const int q = r - j * 3 * NT;
        if (q < 2 * NT) {
            kind = 1;
            t = q >> 1;
            xb = (q & 1) != 0;
            need = 1 + 3 * j;
        } else {
            kind = 2;
            t = q - 2 * NT;
            need = 3 + 3 * j;
        }
    }
    const TileAt w = at(t);
    const Geom G = fixed_tile<NC>(w.G);
    const int I = w.I, J = w.J;
    const Op opi = w.c ? Op(w.c) : op;
    if (Tm::rank() == 0) s_fail = 0;
    if (trace && Tm::rank() == 0) t_start = clock64();
    if (kind != 0 && Tm::rank() < 32) {
        // lanes 0..8 wait for one tile each of the periodic 3 x 3 neighbourhood
        bool bad = false;
        if (Tm::rank() < 9) {
            const int dj = (int)Tm::rank() / 3 - 1, di = (int)Tm::rank() % 3 - 1;
            const int jj = J + dj < 0 ? G.Q - 1 : (J + dj == G.Q ? 0 : J + dj);
            const int ii = I + di < 0 ? G.T - 1 : (I + di == G.T ? 0 : I + di);
            const int *flag = stage + w.base + jj * G.T + ii;
            long long it = 0;
            while (ld_acquire(flag) < need) {
                // give up after the bound, or at once when another block
                // has already recorded a failure
                if (++it > spin_limit || ((it & 255) == 0 && ld_relaxed(err) != 0)) {
                    bad = true;
                    break;
                }
                __nanosleep(64);
            }
        }
        bad = __any_sync(0xffffffffu, bad);
        if (Tm::rank() == 0 && bad) {
            atomicExch(err, 2);
            s_fail = 1;
        }
    }
    Tm::sync();
    if (s_fail) return false;
    if (trace && Tm::rank() == 0) t_ready = clock64();
    // the acquired panels are read next by bulk copies (the async proxy)
    if (Tm::rank() == 0) asm volatile("fence.proxy.async.global;\n" ::: "memory");
    typename Op::S *st = state + w.soff, *u = upp + w.poff, *b = br + w.poff;
    const u64 gj = g0 + (u64)j * h;
    const int o = (j & 1) ? h : 0;
    if (kind == 0) {
        up_tile<Op, Tm, STG>(opi, G, st, u, 0, g0, I, J);
    } else if (kind == 1) {                     // one bridge of half cycle j
        bridge_tile<Op, STG, Tm>(opi, G, u, b, gj, err, I, J, xb);
    } else if (j + 1 < H) {
        octahedron_tile<Op, STG, Tm>(opi, G, b, u, o, gj, err, I, J);
    } else {
        down_tile<Op, STG, Tm>(opi, G, b, st, o, gj, err, I, J);
    }
    // make this item's panel (and state) stores visible, to the generic and
    // the async proxy, before the release of its count; order this item's
    // shared-memory accesses before the next item's bulk copies into it
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __threadfence();
    Tm::sync();
    if (Tm::rank() == 0) {
        if (trace) {
            trace[2 * (size_t)item] = (unsigned)(t_ready - t_start);
            trace[2 * (size_t)item + 1] = (unsigned)(clock64() - t_ready);
        }
        add_release(stage + t, 1);
    }
    return true;
}

template <class Op, bool STG, int NC = 0, class Loc>
__device__ __forceinline__ void persistent_loop(const Op &op, const Loc &at, int NT, int n,
                                                typename Op::S *state, typename Op::S *upp,
                                                typename Op::S *br, int *stage, int *queue, int H,
                                                u64 g0, int *err, int first, long long spin_limit,
                                                unsigned *trace = nullptr) {
    __shared__ int s_item;
    const int nitems = (int)persistent_items(NT, H);
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(queue, 1) + first;
            s_item = ld_relaxed(err) ? nitems : it;   // another block's failure ends this one
        }
        __syncthreads();
        const int item = s_item;
        if (item >= nitems) return;
        if (!persistent_item<Op, STG, NC>(op, at, NT, n, state, upp, br, stage, H, g0, err, item,
                                          spin_limit, trace))
            return;
    }
}

template <class Op, bool STG, int NC = 0>
__global__ void __launch_bounds__(kMaxPersistentThreads)
persistent_kernel(Op op, Geom G, typename Op::S *state, typename Op::S *upp, typename Op::S *br,
                  int *stage, int *queue, int H, u64 g0, int *err, int first,
                  long long spin_limit, unsigned *trace) {
    const Geom Gf = fixed_tile<NC>(G);
    persistent_loop<Op, STG, NC>(op, OneGrid{Gf}, Gf.T * Gf.Q, Gf.n, state, upp, br, stage, queue,
                                 H, g0, err, first, spin_limit, trace);
}

}  // namespace swept
