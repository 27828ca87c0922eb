// Point updates St_k (Section 2; the paper's timestep(i, p), Section 5).
//
// Each update is a functor with
//   S        storage element type of one state value
//   NV       values per point (the vector point state of Section 2, item 2)
//   NST      sub-steps (stages) per time step
//   AUX      extra shared-memory planes the update's level computation uses
//   STAGE    stage the block's input panels in shared memory by TMA
//   INPLACE  every stage writes only planes that it reads at the centre point
//            alone (never at a neighbour), so a level may be computed in place
//            in a single level buffer
//   INPLACE_AFTER_AUX  the level computation's first pass folds every
//            neighbour value it needs into the aux planes and its second pass
//            reads only the centre point and the aux planes, so the second
//            pass may write the level in place (one level buffer); the next
//            level's ring or strip may then be copied in only after the first
//            pass (the neighbour values change from one level to the next)
//   operator()(stage, g, a, out): a(dx, dy, v) reads value v of the neighbour at
//            offset (dx, dy) in {-1,0,1}^2 at the level below; out[0..NV) is the
//            new point state; g is the global sub-step index.
// The same functor runs in the naive kernel (neighbours from global memory) and
// in every swept component (neighbours from shared memory), so the two paths
// produce identical bits. All floating-point operations are written with
// explicit round-to-nearest intrinsics, so no contraction can change them.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

typedef unsigned long long u64;

namespace swept {

// Forward-Euler 5-point heat update, u' = u + r ((u_E + u_S) + (u_W + u_N) - 4u)
// with the last multiply-add fused. s - 4u is formed as fma(-4, u, s), which is
// the same rounding of the same exact value (4u is exact for |u| < 2^1021).
struct HeatOp {
    typedef double S;
    static constexpr int NV = 1, NST = 1, AUX = 1;
    static constexpr bool STAGE = false;
    static constexpr bool INPLACE = false;
    static constexpr bool INPLACE_AFTER_AUX = true;
    double r;
    __host__ __device__ explicit HeatOp(const double *c) : r(c[0]) {}
    template <class A>
    __device__ __forceinline__ void operator()(int, u64, const A &a, S *out) const {
        const double c = a(0, 0, 0);
        const double pe = __dadd_rn(a(1, 0, 0), a(0, 1, 0));    // east + south
        const double pw = __dadd_rn(a(-1, 0, 0), a(0, -1, 0));  // west + north
        const double d = __fma_rn(-4.0, c, __dadd_rn(pe, pw));
        out[0] = __fma_rn(r, d, c);
    }
};

// Storage <-> binary32 conversions of the reduced-precision forms.
template <class S>
struct Store;
template <>
struct Store<float> {
    __device__ static __forceinline__ float ld(float v) { return v; }
    __device__ static __forceinline__ float st(float v) { return v; }
};
template <>
struct Store<__nv_bfloat16> {
    __device__ static __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __forceinline__ __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};

// Heat in binary32 arithmetic with the time update accumulated by Kahan's
// compensated summation; point state (u, c) stored as SS (float or bfloat16):
//   delta = r ((u_E + u_S) + (u_W + u_N) - 4u)   (the difference fused)
//   y = delta - c;  t = u + y;  u' = store(t);  c' = store((u' - u) - y)
// Neighbours read the stored u. r is rounded to binary32 on the host.
template <class SS>
struct HeatKahanOp {
    typedef SS S;
    static constexpr int NV = 2, NST = 1, AUX = 0;
    // bfloat16 panels are staged by TMA (element copies of 2 bytes are slow);
    // binary32 ones are copied straight into the level buffers (more blocks fit)
    static constexpr bool STAGE = sizeof(SS) == 2;
    static constexpr bool INPLACE = false;
    static constexpr bool INPLACE_AFTER_AUX = false;
    float r;
    __host__ __device__ explicit HeatKahanOp(const double *c) : r((float)c[0]) {}
    // the update from the centre (u, c) and the four edge neighbours' u
    __device__ __forceinline__ void update(float uc, float cc, float ue, float us, float uw,
                                           float un, S &u_out, S &c_out) const {
        typedef Store<S> St;
        const float pe = __fadd_rn(ue, us);
        const float pw = __fadd_rn(uw, un);
        const float d = __fmaf_rn(-4.0f, uc, __fadd_rn(pe, pw));
        const float y = __fsub_rn(__fmul_rn(r, d), cc);
        u_out = St::st(__fadd_rn(uc, y));
        c_out = St::st(__fsub_rn(__fsub_rn(St::ld(u_out), uc), y));
    }
    template <class A>
    __device__ __forceinline__ void operator()(int, u64, const A &a, S *out) const {
        typedef Store<S> St;
        update(St::ld(a(0, 0, 0)), St::ld(a(0, 0, 1)), St::ld(a(1, 0, 0)), St::ld(a(0, 1, 0)),
               St::ld(a(-1, 0, 0)), St::ld(a(0, -1, 0)), out[0], out[1]);
    }
};

// The Euler system of EulerOp in binary32 arithmetic with reduced-precision
// storage SS (float or bfloat16) and the time accumulation of each step
// compensated as in HeatKahanOp. Point state: U (0-3), U* (4-7), C (8-11).
//   stage 0: U* = store(U + (dt/2) L(U))            (one fused multiply-add)
//   stage 1: y = dt L(U*) - C;  t = U + y;  U' = store(t);  C' = store((U' - U) - y)
// L is EulerOp's formula with the same fused operations, in binary32; the
// constants are EulerOp's (FP64, from the host) rounded once to binary32.
template <class SS>
struct EulerKahanOp {
    typedef SS S;
    // aux: the 4 binary32 primitive planes of a level (u, v, p, E + p), counted
    // in SS elements
    static constexpr int NV = 12, NST = 2, AUX = 4 * (int)(sizeof(float) / sizeof(SS));
    // bfloat16 panels are staged by TMA (element copies of 2 bytes are slow)
    static constexpr bool STAGE = sizeof(SS) == 2;
    // each stage writes only planes it reads at the centre alone, so a
    // level can be computed in place in one level buffer
    static constexpr bool INPLACE = true;
    static constexpr bool INPLACE_AFTER_AUX = false;
    float gm1, cx, cy, kax, kay, tau0, tau1;
    __host__ __device__ explicit EulerKahanOp(const double *c)
        : gm1((float)c[0]), cx((float)c[1]), cy((float)c[2]), kax((float)c[3]),
          kay((float)c[4]), tau0((float)c[5]), tau1((float)c[6]) {}

    // primitives u = m/rho, v = q/rho, p and E + p of one point
    __device__ __forceinline__ void prims(float r, float m, float q, float E, float &u, float &v,
                                          float &pr, float &Ep) const {
        const float iv = __fdiv_rn(1.0f, r);
        u = __fmul_rn(m, iv);
        v = __fmul_rn(q, iv);
        const float ke = __fmul_rn(0.5f, __fmaf_rn(m, u, __fmul_rn(q, v)));
        pr = __fmul_rn(gm1, __fsub_rn(E, ke));
        Ep = __fadd_rn(E, pr);
    }
    // F1-F3 and G1-G3 of a point from its primitives (F0 = m, G0 = q)
    __device__ __forceinline__ void xflux(float m, float q, float u, float pr, float Ep,
                                          float *F) const {
        F[1] = __fmaf_rn(m, u, pr);
        F[2] = __fmul_rn(q, u);
        F[3] = __fmul_rn(Ep, u);
    }
    __device__ __forceinline__ void yflux(float m, float q, float v, float pr, float Ep,
                                          float *G) const {
        G[1] = __fmul_rn(m, v);
        G[2] = __fmaf_rn(q, v, pr);
        G[3] = __fmul_rn(Ep, v);
    }
    __device__ __forceinline__ void fluxes(float r, float m, float q, float E, float *F,
                                           float *G) const {
        float u, v, pr, Ep;
        prims(r, m, q, E, u, v, pr, Ep);
        F[0] = m;
        xflux(m, q, u, pr, Ep, F);
        G[0] = q;
        yflux(m, q, v, pr, Ep, G);
    }
    // L of one conserved variable from the stencil values and flux differences
    __device__ __forceinline__ float rate(float wc, float wE, float wW, float wS, float wN,
                                          float dF, float dG) const {
        const float lx = __fmaf_rn(-2.0f, wc, __fadd_rn(wE, wW));
        const float ly = __fmaf_rn(-2.0f, wc, __fadd_rn(wS, wN));
        const float diss = __fmaf_rn(kax, lx, __fmul_rn(kay, ly));
        const float flux = __fmaf_rn(cx, dF, __fmul_rn(cy, dG));
        return __fsub_rn(diss, flux);
    }
    // stage 0: the midpoint value of variable c from its rate
    __device__ __forceinline__ S midpoint(float L, float u) const {
        return Store<S>::st(__fmaf_rn(tau0, L, u));
    }
    // stage 1: the compensated update of (u, c) from the rate
    __device__ __forceinline__ void accumulate(float L, float u, float cc, S &u_out,
                                               S &c_out) const {
        typedef Store<S> St;
        const float y = __fsub_rn(__fmul_rn(tau1, L), cc);
        u_out = St::st(__fadd_rn(u, y));
        c_out = St::st(__fsub_rn(__fsub_rn(St::ld(u_out), u), y));
    }
    template <class A>
    __device__ __forceinline__ void operator()(int stage, u64, const A &a, S *out) const {
        typedef Store<S> St;
        const int w0 = stage == 0 ? 0 : 4;
        float FW[4], GW[4], FE[4], GE[4], FN[4], GN[4], FS[4], GS[4];
        fluxes(St::ld(a(-1, 0, w0)), St::ld(a(-1, 0, w0 + 1)), St::ld(a(-1, 0, w0 + 2)),
               St::ld(a(-1, 0, w0 + 3)), FW, GW);
        fluxes(St::ld(a(1, 0, w0)), St::ld(a(1, 0, w0 + 1)), St::ld(a(1, 0, w0 + 2)),
               St::ld(a(1, 0, w0 + 3)), FE, GE);
        fluxes(St::ld(a(0, -1, w0)), St::ld(a(0, -1, w0 + 1)), St::ld(a(0, -1, w0 + 2)),
               St::ld(a(0, -1, w0 + 3)), FN, GN);
        fluxes(St::ld(a(0, 1, w0)), St::ld(a(0, 1, w0 + 1)), St::ld(a(0, 1, w0 + 2)),
               St::ld(a(0, 1, w0 + 3)), FS, GS);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float L = rate(St::ld(a(0, 0, w0 + c)), St::ld(a(1, 0, w0 + c)),
                                 St::ld(a(-1, 0, w0 + c)), St::ld(a(0, 1, w0 + c)),
                                 St::ld(a(0, -1, w0 + c)), __fsub_rn(FE[c], FW[c]),
                                 __fsub_rn(GS[c], GN[c]));
            if (stage == 0) {
                out[c] = a(0, 0, c);
                out[4 + c] = midpoint(L, St::ld(a(0, 0, c)));
                out[8 + c] = a(0, 0, 8 + c);
            } else {
                accumulate(L, St::ld(a(0, 0, c)), St::ld(a(0, 0, 8 + c)), out[c], out[8 + c]);
                out[4 + c] = a(0, 0, 4 + c);
            }
        }
    }
};

// 2D wave equation u_tt = c^2 laplace(u), leapfrog in time (Section 6's
// experiment); point state (u^n, u^{n-1}):
//   d = ((u_E + u_S) + (u_W + u_N)) - 4u,  u^{n+1} = (2u - u^{n-1}) + C^2 d (fused)
// C2 = (c dt / dx)^2 is formed on the host.
struct WaveOp {
    typedef double S;
    static constexpr int NV = 2, NST = 1, AUX = 1;   // aux: pair sums of a level
    static constexpr bool STAGE = false;
    static constexpr bool INPLACE = false;
    static constexpr bool INPLACE_AFTER_AUX = true;
    double C2;
    __host__ __device__ explicit WaveOp(const double *c) : C2(c[0]) {}
    template <class A>
    __device__ __forceinline__ void operator()(int, u64, const A &a, S *out) const {
        const double c = a(0, 0, 0);
        const double pe = __dadd_rn(a(1, 0, 0), a(0, 1, 0));
        const double pw = __dadd_rn(a(-1, 0, 0), a(0, -1, 0));
        const double d = __fma_rn(-4.0, c, __dadd_rn(pe, pw));
        out[0] = __fma_rn(C2, d, __dsub_rn(__dmul_rn(2.0, c), a(0, 0, 1)));
        out[1] = c;
    }
};

// Section 3.1 worked example: u' = u + 1.
struct IncrementOp {
    typedef double S;
    static constexpr int NV = 1, NST = 1, AUX = 0;
    static constexpr bool STAGE = false;
    static constexpr bool INPLACE = false;
    static constexpr bool INPLACE_AFTER_AUX = false;
    __host__ __device__ explicit IncrementOp(const double *) {}
    template <class A>
    __device__ __forceinline__ void operator()(int, u64, const A &a, S *out) const {
        out[0] = __dadd_rn(a(0, 0, 0), 1.0);
    }
};

// Test update: u' = u + 1 if all 9 neighbours hold the centre's level, else NaN.
struct LevelTagOp {
    typedef double S;
    static constexpr int NV = 1, NST = 1, AUX = 0;
    static constexpr bool STAGE = false;
    static constexpr bool INPLACE = false;
    static constexpr bool INPLACE_AFTER_AUX = false;
    __host__ __device__ explicit LevelTagOp(const double *) {}
    template <class A>
    __device__ __forceinline__ void operator()(int, u64, const A &a, S *out) const {
        const double c = a(0, 0, 0);
        bool same = true;
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di) same = same && (a(di, dj, 0) == c);
        out[0] = same ? __dadd_rn(c, 1.0) : __longlong_as_double(0x7ff8000000000000LL);
    }
};

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ u64 mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Test update on 64-bit words: h = mix(g + golden); h = mix(h + w) over the 9
// neighbours in row order (north row west..east, own row, south row).
struct HashOp {
    typedef u64 S;
    static constexpr int NV = 1, NST = 1, AUX = 0;
    static constexpr bool STAGE = false;
    static constexpr bool INPLACE = false;
    static constexpr bool INPLACE_AFTER_AUX = false;
    __host__ __device__ explicit HashOp(const double *) {}
    template <class A>
    __device__ __forceinline__ void operator()(int, u64 g, const A &a, S *out) const {
        u64 h = mix64(g + 0x9e3779b97f4a7c15ULL);
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di) h = mix64(h + a(di, dj, 0));
        out[0] = h;
    }
};

// Eq. (complex_step) as its two radius-1 sub-steps on 64-bit words (mod 2^64):
// eq. (substep1) pushes (u, u_W, u_E, u_N, u_S); eq. (substep2) forms
// u' = (west's 2nd + east's 3rd + north's 4th + south's 5th) - 4 (own 1st).
struct Wide2Op {
    typedef u64 S;
    static constexpr int NV = 5, NST = 2, AUX = 0;
    static constexpr bool STAGE = false;
    static constexpr bool INPLACE = false;
    static constexpr bool INPLACE_AFTER_AUX = false;
    __host__ __device__ explicit Wide2Op(const double *) {}
    template <class A>
    __device__ __forceinline__ void operator()(int stage, u64, const A &a, S *out) const {
        if (stage == 0) {
            out[0] = a(0, 0, 0);
            out[1] = a(-1, 0, 0);
            out[2] = a(1, 0, 0);
            out[3] = a(0, -1, 0);
            out[4] = a(0, 1, 0);
        } else {
            out[0] = a(-1, 0, 1) + a(1, 0, 2) + a(0, -1, 3) + a(0, 1, 4) - 4ULL * a(0, 0, 0);
            out[1] = out[2] = out[3] = out[4] = 0ULL;
        }
    }
};

// 2D compressible Euler, midpoint RK2, central flux + scalar dissipation.
// Point state: planes 0-3 U = (rho, m, q, E); planes 4-7 U*.
//   stage 0: (U, U*) <- (U, U + tau0 L(U))
//   stage 1: (U, U*) <- (U + tau1 L(U*), U*)
// L(W) = (kax ((W_E + W_W) - 2W) + kay ((W_S + W_N) - 2W)) - (cx (F_E - F_W) + cy (G_S - G_N))
// with F = (m, m u + p, q u, (E+p) u), G = (q, m v, q v + p, (E+p) v),
// u = m/rho, v = q/rho, p = (gamma-1)(E - 0.5 (m u + q v)). Products followed
// by a sum are fused exactly where the formula is written "a b + c".
// Host-precomputed constants c[] = {gamma-1, cx, cy, kax, kay, tau0, tau1}.
struct EulerOp {
    typedef double S;
    static constexpr int NV = 8, NST = 2, AUX = 4;   // aux: u, v, p, E + p of a level
    static constexpr bool STAGE = false;
    // each stage writes only planes it reads at the centre alone, so a
    // level can be computed in place in one level buffer
    static constexpr bool INPLACE = true;
    static constexpr bool INPLACE_AFTER_AUX = false;
    double gm1, cx, cy, kax, kay, tau0, tau1;
    __host__ __device__ explicit EulerOp(const double *c)
        : gm1(c[0]), cx(c[1]), cy(c[2]), kax(c[3]), kay(c[4]), tau0(c[5]), tau1(c[6]) {}

    __device__ __forceinline__ void prims(double r, double m, double q, double E, double &u,
                                          double &v, double &pr, double &Ep) const {
        const double iv = __ddiv_rn(1.0, r);
        u = __dmul_rn(m, iv);
        v = __dmul_rn(q, iv);
        const double ke = __dmul_rn(0.5, __fma_rn(m, u, __dmul_rn(q, v)));
        pr = __dmul_rn(gm1, __dsub_rn(E, ke));
        Ep = __dadd_rn(E, pr);
    }
    // F1-F3 and G1-G3 of a point from its primitives (F0 = m, G0 = q)
    __device__ __forceinline__ void xflux_p(double m, double q, double u, double pr, double Ep,
                                            double *F) const {
        F[1] = __fma_rn(m, u, pr);
        F[2] = __dmul_rn(q, u);
        F[3] = __dmul_rn(Ep, u);
    }
    __device__ __forceinline__ void yflux_p(double m, double q, double v, double pr, double Ep,
                                            double *G) const {
        G[1] = __dmul_rn(m, v);
        G[2] = __fma_rn(q, v, pr);
        G[3] = __dmul_rn(Ep, v);
    }
    __device__ __forceinline__ void xflux(double r, double m, double q, double E, double *F) const {
        double u, v, pr, Ep;
        prims(r, m, q, E, u, v, pr, Ep);
        F[0] = m;
        xflux_p(m, q, u, pr, Ep, F);
    }
    // the stage update of one point from its fluxes' differences (shared by the
    // per-point operator below and the swept level computation)
    __device__ __forceinline__ void combine(int stage, int c, double wc, double wE, double wW,
                                            double wS, double wN, double dF, double dG,
                                            double ubase, double &res) const {
        const double tau = stage == 0 ? tau0 : tau1;
        const double lx = __fma_rn(-2.0, wc, __dadd_rn(wE, wW));
        const double ly = __fma_rn(-2.0, wc, __dadd_rn(wS, wN));
        const double diss = __fma_rn(kax, lx, __dmul_rn(kay, ly));
        const double flux = __fma_rn(cx, dF, __dmul_rn(cy, dG));
        res = __fma_rn(tau, __dsub_rn(diss, flux), ubase);
    }
    __device__ __forceinline__ void yflux(double r, double m, double q, double E, double *G) const {
        double u, v, pr, Ep;
        prims(r, m, q, E, u, v, pr, Ep);
        G[0] = q;
        yflux_p(m, q, v, pr, Ep, G);
    }
    template <class A>
    __device__ __forceinline__ void operator()(int stage, u64, const A &a, S *out) const {
        const int w0 = stage == 0 ? 0 : 4;
        double FW[4], FE[4], GN[4], GS[4];
        xflux(a(-1, 0, w0), a(-1, 0, w0 + 1), a(-1, 0, w0 + 2), a(-1, 0, w0 + 3), FW);
        xflux(a(1, 0, w0), a(1, 0, w0 + 1), a(1, 0, w0 + 2), a(1, 0, w0 + 3), FE);
        yflux(a(0, -1, w0), a(0, -1, w0 + 1), a(0, -1, w0 + 2), a(0, -1, w0 + 3), GN);
        yflux(a(0, 1, w0), a(0, 1, w0 + 1), a(0, 1, w0 + 2), a(0, 1, w0 + 3), GS);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double res;
            combine(stage, c, a(0, 0, w0 + c), a(1, 0, w0 + c), a(-1, 0, w0 + c),
                    a(0, 1, w0 + c), a(0, -1, w0 + c), __dsub_rn(FE[c], FW[c]),
                    __dsub_rn(GS[c], GN[c]), a(0, 0, c), res);
            if (stage == 0) {
                out[c] = a(0, 0, c);
                out[4 + c] = res;
            } else {
                out[c] = res;
                out[4 + c] = a(0, 0, 4 + c);
            }
        }
    }
};

}  // namespace swept
