/*
 * Plain CPU oracle for explicit time advancing on a doubly periodic 2D grid.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this library. The
 * product path (the CUDA library under paper_1602_07558_gb300/) never links,
 * imports or calls it, and this file includes no header of that library.
 *
 * What it computes. The swept rule of space-time decomposition (Section 3,
 * Algorithms 1-5) reaches exactly the values of plain step-by-step explicit time
 * marching: every (point, level) is computed once, from its 9-point neighbourhood
 * at the level below (Section 4, first paragraph; abstract: "no redundant
 * computation"). So the oracle is that plain definition, written out:
 *
 *     for every sub-step:  v(i,j) = St(u on the 3x3 neighbourhood of (i,j))  for all (i,j)
 *                          u <- v
 *
 * with indices taken modulo nx, ny (doubly periodic grid, Section 2 item 1).
 * No blocking, no fusion, no reordering: one full sweep per sub-step, rows in
 * parallel with OpenMP (each output point is written once from the previous
 * sweep, so the result does not depend on the thread count).
 *
 * Conventions: row-major planes, x = i fastest, j = row; "north" = j-1, "south"
 * = j+1, "west" = i-1, "east" = i+1. Floating point is IEEE binary64, round to
 * nearest even; this file is compiled with -ffp-contract=off so that only the
 * fma() calls written below are fused.
 *
 * Point updates (the paper's St_k / timestep(i, p), Section 5):
 *   heat      forward-Euler 5-point heat update, one sub-step per step
 *   increment the paper's worked example u <- u + 1 (Section 3.1)
 *   hash      order-sensitive 64-bit mix of the 9 neighbour words and the
 *             sub-step index (a test update that detects any wrong dependency)
 *   leveltag  u <- u + 1 if all 9 neighbours hold the same level, else NaN
 *   wide2     the radius-2 scheme of eq. (complex_step), evaluated directly on
 *             64-bit integers modulo 2^64 (its 2-sub-step form, eqs. (substep1)-
 *             (substep2), is what the swept path runs)
 *   euler     2D compressible Euler, central flux plus scalar dissipation,
 *             midpoint (2-stage) Runge-Kutta, dt fixed from the initial state
 *   wave      the 2D wave equation u_tt = c^2 laplace(u), leapfrog in time with
 *             Courant number C (Section 6's experiment), point state (u^n, u^{n-1})
 *   heat_kahan the heat update in binary32 arithmetic with the time update
 *             accumulated by Kahan's compensated summation, state (u, c) stored
 *             in binary32 or in bfloat16 (reduced-precision storage forms)
 *   euler_kahan the Euler system in binary32 arithmetic, state (U, U*, C)
 *             stored in binary32 or bfloat16, compensated time accumulation
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int wrapi(long long i, int n) {
    long long r = i % n;
    return (int)(r < 0 ? r + n : r);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* OpenMP threads for the following calls (no result depends on it: every
 * output point is written once from the previous sweep). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ heat
 * u_t = laplace(u), forward Euler with diffusion number r on the 5-point stencil:
 *     s = (u_E + u_S) + (u_W + u_N)
 *     d = s - 4 u
 *     u' = u + r d     (one rounding: fma)
 * The 9-point neighbourhood of Section 2 contains the 5 points used here. The
 * paper fixes no evaluation order; this one pairs east with south and west with
 * north, each pair rounded once. */
int oracle_heat(int nx, int ny, double r, long long nsteps, double *u) {
    if (nx < 1 || ny < 1 || nsteps < 0 || !u) return -1;
    size_t npts = (size_t)nx * ny;
    double *v = (double *)malloc(npts * sizeof(double));
    if (!v) return -3;
    double *a = u, *b = v;
    for (long long s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            int jn = wrapi(j - 1, ny), js = wrapi(j + 1, ny);
            for (int i = 0; i < nx; ++i) {
                int iw = wrapi(i - 1, nx), ie = wrapi(i + 1, nx);
                double c = a[(size_t)j * nx + i];
                double sum = (a[(size_t)j * nx + ie] + a[(size_t)js * nx + i]) +
                             (a[(size_t)j * nx + iw] + a[(size_t)jn * nx + i]);
                double d = sum - 4.0 * c;
                b[(size_t)j * nx + i] = fma(r, d, c);
            }
        }
        double *t = a; a = b; b = t;
    }
    if (a != u) memcpy(u, a, npts * sizeof(double));
    free(v);
    return 0;
}

/* ------------------------------------------------------------------- increment
 * Section 3.1 worked example: u^{k+1} = u^k + 1. */
int oracle_increment(int nx, int ny, long long nsteps, double *u) {
    if (nx < 1 || ny < 1 || nsteps < 0 || !u) return -1;
    size_t npts = (size_t)nx * ny;
    for (long long s = 0; s < nsteps; ++s)
        for (size_t p = 0; p < npts; ++p) u[p] = u[p] + 1.0;
    return 0;
}

/* ------------------------------------------------------------------------ hash
 * SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014; as published
 * with Vigna's xorshift generators): z ^= z>>30, z *= 0xbf58476d1ce4e5b9,
 * z ^= z>>27, z *= 0x94d049bb133111eb, z ^= z>>31. */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t oracle_mix64(uint64_t z) { return mix64(z); }

/* One sub-step with global index g: h = mix(g + golden); then for the 9
 * neighbours in row order (north row west..east, own row, south row):
 * h = mix(h + w). The new word is h. */
int oracle_hash(int nx, int ny, long long substep0, long long nsub, uint64_t *u) {
    if (nx < 1 || ny < 1 || nsub < 0 || !u) return -1;
    size_t npts = (size_t)nx * ny;
    uint64_t *v = (uint64_t *)malloc(npts * sizeof(uint64_t));
    if (!v) return -3;
    uint64_t *a = u, *b = v;
    for (long long s = 0; s < nsub; ++s) {
        uint64_t g = (uint64_t)(substep0 + s);
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                uint64_t h = mix64(g + 0x9e3779b97f4a7c15ULL);
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di)
                        h = mix64(h + a[(size_t)wrapi(j + dj, ny) * nx + wrapi(i + di, nx)]);
                b[(size_t)j * nx + i] = h;
            }
        }
        uint64_t *t = a; a = b; b = t;
    }
    if (a != u) memcpy(u, a, npts * sizeof(uint64_t));
    free(v);
    return 0;
}

/* -------------------------------------------------------------------- leveltag
 * Each point holds the level it was computed at. A point at level k+1 may only
 * be computed from 9 neighbours that are all at level k (Section 4, first
 * paragraph): u' = u + 1 when all 9 equal the centre, NaN otherwise. */
int oracle_leveltag(int nx, int ny, long long nsub, double *u) {
    if (nx < 1 || ny < 1 || nsub < 0 || !u) return -1;
    size_t npts = (size_t)nx * ny;
    double *v = (double *)malloc(npts * sizeof(double));
    if (!v) return -3;
    double *a = u, *b = v;
    for (long long s = 0; s < nsub; ++s) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                double c = a[(size_t)j * nx + i];
                int same = 1;
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di)
                        if (!(a[(size_t)wrapi(j + dj, ny) * nx + wrapi(i + di, nx)] == c)) same = 0;
                b[(size_t)j * nx + i] = same ? c + 1.0 : NAN;
            }
        }
        double *t = a; a = b; b = t;
    }
    if (a != u) memcpy(u, a, npts * sizeof(double));
    free(v);
    return 0;
}

/* ----------------------------------------------------------------------- wide2
 * Eq. (complex_step), evaluated directly with its radius-2 neighbours:
 *     u^{n+1}_{i,j} = u_{i-2,j} + u_{i+2,j} + u_{i,j-2} + u_{i,j+2} - 4 u_{i,j}
 * in unsigned 64-bit arithmetic (modulo 2^64, so that long runs stay exact). */
int oracle_wide2(int nx, int ny, long long nsteps, uint64_t *u) {
    if (nx < 1 || ny < 1 || nsteps < 0 || !u) return -1;
    size_t npts = (size_t)nx * ny;
    uint64_t *v = (uint64_t *)malloc(npts * sizeof(uint64_t));
    if (!v) return -3;
    uint64_t *a = u, *b = v;
    for (long long s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                uint64_t c = a[(size_t)j * nx + i];
                uint64_t w2 = a[(size_t)j * nx + wrapi(i - 2, nx)];
                uint64_t e2 = a[(size_t)j * nx + wrapi(i + 2, nx)];
                uint64_t n2 = a[(size_t)wrapi(j - 2, ny) * nx + i];
                uint64_t s2 = a[(size_t)wrapi(j + 2, ny) * nx + i];
                b[(size_t)j * nx + i] = w2 + e2 + n2 + s2 - 4u * c;
            }
        }
        uint64_t *t = a; a = b; b = t;
    }
    if (a != u) memcpy(u, a, npts * sizeof(uint64_t));
    free(v);
    return 0;
}

/* ----------------------------------------------------------------------- euler
 * Conserved W = (rho, m = rho u, q = rho v, E), ideal gas:
 *     iv = 1/rho, u = m iv, v = q iv, ke = 0.5 (m u + q v), p = (gamma-1)(E - ke)
 *     F(W) = (m, m u + p, q u, (E + p) u)        x-flux
 *     G(W) = (q, m v, q v + p, (E + p) v)        y-flux
 * Semi-discrete operator at a point, with the 4 neighbours W_W, W_E, W_N, W_S:
 *     L_k = (kax ((W_E + W_W) - 2 W) + kay ((W_S + W_N) - 2 W))
 *           - (cx (F_E - F_W) + cy (G_S - G_N))
 * Rounding: every "a b + c" written above with a product first is one fused
 * multiply-add (fma(a, b, c)): m u + q v, m u + p, q v + p, kax lx + kay ly,
 * cx dF + cy dG, and base + tau L; all other operations round separately.
 *     cx = 0.5/dx, cy = 0.5/dy, kax = (kappa a)/dx, kay = (kappa a)/dy
 * (central flux difference plus scalar dissipation with a fixed global wave
 * speed a). Midpoint Runge-Kutta: U* = U + (0.5 dt) L(U); U <- U + dt L(U*).
 * Each sub-step is a radius-1 stencil operation with a vector point state
 * (Section 2, item 2). */
typedef struct { double cx, cy, kax, kay, gm1; } euler_consts;

static void euler_flux(const double *W, size_t p, size_t np, double gm1, double *F, double *G) {
    double r = W[p], m = W[np + p], q = W[2 * np + p], E = W[3 * np + p];
    double iv = 1.0 / r;
    double u = m * iv, v = q * iv;
    double ke = 0.5 * fma(m, u, q * v);
    double pr = gm1 * (E - ke);
    double Ep = E + pr;
    F[0] = m; F[1] = fma(m, u, pr); F[2] = q * u; F[3] = Ep * u;
    G[0] = q; G[1] = m * v; G[2] = fma(q, v, pr); G[3] = Ep * v;
}

/* out = base + tau * L(W) at every point. */
static void euler_stage(int nx, int ny, const euler_consts *k, double tau,
                        const double *W, const double *base, double *out) {
    size_t np = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        int jn = wrapi(j - 1, ny), js = wrapi(j + 1, ny);
        for (int i = 0; i < nx; ++i) {
            int iw = wrapi(i - 1, nx), ie = wrapi(i + 1, nx);
            size_t pc = (size_t)j * nx + i, pw = (size_t)j * nx + iw, pe = (size_t)j * nx + ie;
            size_t pn = (size_t)jn * nx + i, ps = (size_t)js * nx + i;
            double FW[4], GW[4], FE[4], GE[4], FN[4], GN[4], FS[4], GS[4];
            euler_flux(W, pw, np, k->gm1, FW, GW);
            euler_flux(W, pe, np, k->gm1, FE, GE);
            euler_flux(W, pn, np, k->gm1, FN, GN);
            euler_flux(W, ps, np, k->gm1, FS, GS);
            for (int c = 0; c < 4; ++c) {
                double wc = W[c * np + pc];
                double lx = (W[c * np + pe] + W[c * np + pw]) - 2.0 * wc;
                double ly = (W[c * np + ps] + W[c * np + pn]) - 2.0 * wc;
                double diss = fma(k->kax, lx, k->kay * ly);
                double flux = fma(k->cx, FE[c] - FW[c], k->cy * (GS[c] - GN[c]));
                double L = diss - flux;
                out[c * np + pc] = fma(tau, L, base[c * np + pc]);
            }
        }
    }
}

/* Maximum wave speed a = max over points of max(|u| + c, |v| + c),
 * c = sqrt(gamma p / rho). */
double oracle_euler_wavespeed(int nx, int ny, double gamma, const double *U) {
    size_t np = (size_t)nx * ny;
    double gm1 = gamma - 1.0, amax = 0.0;
    for (size_t p = 0; p < np; ++p) {
        double r = U[p], m = U[np + p], q = U[2 * np + p], E = U[3 * np + p];
        double iv = 1.0 / r;
        double u = m * iv, v = q * iv;
        double ke = 0.5 * fma(m, u, q * v);
        double pr = gm1 * (E - ke);
        double c = sqrt((gamma * pr) * iv);
        double su = fabs(u) + c, sv = fabs(v) + c;
        double s = su > sv ? su : sv;
        if (s > amax) amax = s;
    }
    return amax;
}

/* Fixed time step from the CFL number (dt = cfl min(dx,dy) / a), dx = lx/nx,
 * dy = ly/ny; writes a and dt. */
int oracle_euler_setup(int nx, int ny, double gamma, double cfl, double lx, double ly,
                       const double *U, double *a_out, double *dt_out) {
    if (nx < 1 || ny < 1 || !U) return -1;
    double dx = lx / nx, dy = ly / ny;
    double a = oracle_euler_wavespeed(nx, ny, gamma, U);
    double h = dx < dy ? dx : dy;
    *a_out = a;
    *dt_out = (cfl * h) / a;
    return 0;
}

/* nsteps of midpoint RK2 on U (4 planes), in place. */
int oracle_euler_rk2(int nx, int ny, double gamma, double dt, double lx, double ly,
                     double kappa, double a, long long nsteps, double *U) {
    if (nx < 1 || ny < 1 || nsteps < 0 || !U) return -1;
    size_t np = (size_t)nx * ny;
    double dx = lx / nx, dy = ly / ny;
    euler_consts k;
    k.cx = 0.5 / dx; k.cy = 0.5 / dy;
    k.kax = (kappa * a) / dx; k.kay = (kappa * a) / dy;
    k.gm1 = gamma - 1.0;
    double tau0 = 0.5 * dt, tau1 = dt;
    double *Us = (double *)malloc(4 * np * sizeof(double));
    double *Un = (double *)malloc(4 * np * sizeof(double));
    if (!Us || !Un) { free(Us); free(Un); return -3; }
    for (long long s = 0; s < nsteps; ++s) {
        euler_stage(nx, ny, &k, tau0, U, U, Us);   /* U* = U + dt/2 L(U)  */
        euler_stage(nx, ny, &k, tau1, Us, U, Un);  /* U' = U + dt L(U*)   */
        memcpy(U, Un, 4 * np * sizeof(double));
    }
    free(Us); free(Un);
    return 0;
}

/* ------------------------------------------------------------------ heat_kahan
 * Reduced-precision storage of the heat state with binary32 arithmetic. Each
 * point stores u and a compensation c (Kahan, "Further remarks on reducing
 * truncation errors", CACM 8(1), 1965): the increment of one step is
 *     delta = r * ((u_E + u_S) + (u_W + u_N) - 4u)        (last difference fused)
 * and it is added to u by compensated summation, the storage rounding playing
 * the role of the rounded sum:
 *     y = delta - c;  t = u + y;  u' = store(t);  c' = store((u' - u) - y)
 * store() is exact for binary32 and round-to-nearest-even to bfloat16 (the top
 * 16 bits of a binary32) for the bfloat16 form. Neighbours read the stored u. */

/* binary32 -> bfloat16, round to nearest, ties to even (NaN stays NaN). */
uint16_t oracle_f32_to_bf16(float f) {
    uint32_t x;
    memcpy(&x, &f, sizeof x);
    if ((x & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((x >> 16) | 0x0040u);
    uint32_t lsb = (x >> 16) & 1u;
    x += 0x7fffu + lsb;
    return (uint16_t)(x >> 16);
}

float oracle_bf16_to_f32(uint16_t h) {
    uint32_t x = (uint32_t)h << 16;
    float f;
    memcpy(&f, &x, sizeof f);
    return f;
}

static void kahan_point(float r, float uc, float cc, float e, float s, float w, float n,
                        float *t_out, float *y_out) {
    float pe = e + s;
    float pw = w + n;
    float d = fmaf(-4.0f, uc, pe + pw);
    float delta = r * d;
    float y = delta - cc;
    *t_out = uc + y;
    *y_out = y;
}

int oracle_heat_kahan_f32(int nx, int ny, double r64, long long nsteps, float *u, float *c) {
    if (nx < 1 || ny < 1 || nsteps < 0 || !u || !c) return -1;
    size_t npts = (size_t)nx * ny;
    float r = (float)r64;
    float *u2 = (float *)malloc(npts * sizeof(float));
    float *c2 = (float *)malloc(npts * sizeof(float));
    if (!u2 || !c2) { free(u2); free(c2); return -3; }
    float *ua = u, *ca = c, *ub = u2, *cb = c2;
    for (long long s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            int jn = wrapi(j - 1, ny), js = wrapi(j + 1, ny);
            for (int i = 0; i < nx; ++i) {
                int iw = wrapi(i - 1, nx), ie = wrapi(i + 1, nx);
                size_t p = (size_t)j * nx + i;
                float t, y;
                kahan_point(r, ua[p], ca[p], ua[(size_t)j * nx + ie], ua[(size_t)js * nx + i],
                            ua[(size_t)j * nx + iw], ua[(size_t)jn * nx + i], &t, &y);
                ub[p] = t;
                cb[p] = (t - ua[p]) - y;
            }
        }
        float *tu = ua; ua = ub; ub = tu;
        float *tc = ca; ca = cb; cb = tc;
    }
    if (ua != u) { memcpy(u, ua, npts * sizeof(float)); memcpy(c, ca, npts * sizeof(float)); }
    free(u2); free(c2);
    return 0;
}

int oracle_heat_kahan_bf16(int nx, int ny, double r64, long long nsteps, uint16_t *u, uint16_t *c) {
    if (nx < 1 || ny < 1 || nsteps < 0 || !u || !c) return -1;
    size_t npts = (size_t)nx * ny;
    float r = (float)r64;
    uint16_t *u2 = (uint16_t *)malloc(npts * sizeof(uint16_t));
    uint16_t *c2 = (uint16_t *)malloc(npts * sizeof(uint16_t));
    if (!u2 || !c2) { free(u2); free(c2); return -3; }
    uint16_t *ua = u, *ca = c, *ub = u2, *cb = c2;
    for (long long s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            int jn = wrapi(j - 1, ny), js = wrapi(j + 1, ny);
            for (int i = 0; i < nx; ++i) {
                int iw = wrapi(i - 1, nx), ie = wrapi(i + 1, nx);
                size_t p = (size_t)j * nx + i;
                float uc = oracle_bf16_to_f32(ua[p]);
                float t, y;
                kahan_point(r, uc, oracle_bf16_to_f32(ca[p]),
                            oracle_bf16_to_f32(ua[(size_t)j * nx + ie]),
                            oracle_bf16_to_f32(ua[(size_t)js * nx + i]),
                            oracle_bf16_to_f32(ua[(size_t)j * nx + iw]),
                            oracle_bf16_to_f32(ua[(size_t)jn * nx + i]), &t, &y);
                uint16_t un = oracle_f32_to_bf16(t);
                ub[p] = un;
                cb[p] = oracle_f32_to_bf16((oracle_bf16_to_f32(un) - uc) - y);
            }
        }
        uint16_t *tu = ua; ua = ub; ub = tu;
        uint16_t *tc = ca; ca = cb; cb = tc;
    }
    if (ua != u) { memcpy(u, ua, npts * sizeof(uint16_t)); memcpy(c, ca, npts * sizeof(uint16_t)); }
    free(u2); free(c2);
    return 0;
}

/* ----------------------------------------------------------------- euler_kahan
 * The Euler system above in binary32 arithmetic with reduced-precision storage,
 * each step's time accumulation compensated as in heat_kahan (the precision
 * forms of the scheme; the paper fixes no precision). Point state: 12 planes,
 * U (0-3), U* (4-7) and the compensation C (8-11), each value stored as a
 * binary32 or (bf16 != 0) as a value representable in bfloat16; store() rounds
 * a binary32 to the storage format (identity, or round to nearest even).
 * Constants: the FP64 constants of euler (cx, cy, kax, kay, gamma-1, dt/2, dt)
 * rounded once to binary32. L is the FP64 formula in binary32 arithmetic with
 * the same fused operations. One step:
 *   stage 0: U* = store(U + (dt/2) L(U))              (one fused multiply-add)
 *   stage 1: y = dt L(U*) - C;  t = U + y;  U' = store(t);  C' = store((U' - U) - y)
 * U and C pass through stage 0 unchanged, U* through stage 1; the stencil reads
 * the stored values. */
typedef struct { float cx, cy, kax, kay, gm1; } euler_consts_f;

static float store_f(float x, int bf16) {
    return bf16 ? oracle_bf16_to_f32(oracle_f32_to_bf16(x)) : x;
}

static void euler_flux_f(const float *W, size_t p, size_t np, float gm1, float *F, float *G) {
    float r = W[p], m = W[np + p], q = W[2 * np + p], E = W[3 * np + p];
    float iv = 1.0f / r;
    float u = m * iv, v = q * iv;
    float ke = 0.5f * fmaf(m, u, q * v);
    float pr = gm1 * (E - ke);
    float Ep = E + pr;
    F[0] = m; F[1] = fmaf(m, u, pr); F[2] = q * u; F[3] = Ep * u;
    G[0] = q; G[1] = m * v; G[2] = fmaf(q, v, pr); G[3] = Ep * v;
}

/* L(W) at point (i, j) of the 4-plane field W. */
static void euler_L_f(const float *W, int nx, int ny, int i, int j, const euler_consts_f *k,
                      float *L) {
    size_t np = (size_t)nx * ny;
    int jn = wrapi(j - 1, ny), js = wrapi(j + 1, ny);
    int iw = wrapi(i - 1, nx), ie = wrapi(i + 1, nx);
    size_t pc = (size_t)j * nx + i, pw = (size_t)j * nx + iw, pe = (size_t)j * nx + ie;
    size_t pn = (size_t)jn * nx + i, ps = (size_t)js * nx + i;
    float FW[4], GW[4], FE[4], GE[4], FN[4], GN[4], FS[4], GS[4];
    euler_flux_f(W, pw, np, k->gm1, FW, GW);
    euler_flux_f(W, pe, np, k->gm1, FE, GE);
    euler_flux_f(W, pn, np, k->gm1, FN, GN);
    euler_flux_f(W, ps, np, k->gm1, FS, GS);
    for (int c = 0; c < 4; ++c) {
        float wc = W[c * np + pc];
        float lx = (W[c * np + pe] + W[c * np + pw]) - 2.0f * wc;
        float ly = (W[c * np + ps] + W[c * np + pn]) - 2.0f * wc;
        float diss = fmaf(k->kax, lx, k->kay * ly);
        float flux = fmaf(k->cx, FE[c] - FW[c], k->cy * (GS[c] - GN[c]));
        L[c] = diss - flux;
    }
}

/* nsteps of the compensated binary32 midpoint RK2 on the 12-plane state S. */
int oracle_euler_kahan(int nx, int ny, int bf16, double gamma, double dt, double lx, double ly,
                       double kappa, double a, long long nsteps, float *S) {
    if (nx < 1 || ny < 1 || nsteps < 0 || !S) return -1;
    size_t np = (size_t)nx * ny;
    double dx = lx / nx, dy = ly / ny;
    euler_consts_f k;
    k.cx = (float)(0.5 / dx); k.cy = (float)(0.5 / dy);
    k.kax = (float)((kappa * a) / dx); k.kay = (float)((kappa * a) / dy);
    k.gm1 = (float)(gamma - 1.0);
    float tau0 = (float)(0.5 * dt), tau1 = (float)dt;
    float *T = (float *)malloc(12 * np * sizeof(float));
    if (!T) return -3;
    float *A = S, *B = T;
    for (long long s = 0; s < nsteps; ++s) {
        /* stage 0: U* = store(U + (dt/2) L(U)) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t pc = (size_t)j * nx + i;
                float L[4];
                euler_L_f(A, nx, ny, i, j, &k, L);
                for (int c = 0; c < 4; ++c) {
                    B[c * np + pc] = A[c * np + pc];
                    B[(4 + c) * np + pc] = store_f(fmaf(tau0, L[c], A[c * np + pc]), bf16);
                    B[(8 + c) * np + pc] = A[(8 + c) * np + pc];
                }
            }
        { float *t = A; A = B; B = t; }
        /* stage 1: compensated U += dt L(U*) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t pc = (size_t)j * nx + i;
                float L[4];
                euler_L_f(A + 4 * np, nx, ny, i, j, &k, L);
                for (int c = 0; c < 4; ++c) {
                    float u = A[c * np + pc], cc = A[(8 + c) * np + pc];
                    float y = tau1 * L[c] - cc;
                    float un = store_f(u + y, bf16);
                    B[c * np + pc] = un;
                    B[(4 + c) * np + pc] = A[(4 + c) * np + pc];
                    B[(8 + c) * np + pc] = store_f((un - u) - y, bf16);
                }
            }
        { float *t = A; A = B; B = t; }
    }
    if (A != S) memcpy(S, A, 12 * np * sizeof(float));
    free(A == S ? B : A);
    return 0;
}

/* ------------------------------------------------------------------------ wave
 * u_tt = c^2 laplace(u) with the leapfrog scheme (second order in time):
 *     d = ((u_E + u_S) + (u_W + u_N)) - 4u        (5-point Laplacian, same pairing as heat)
 *     u^{n+1} = (2u - u^{n-1}) + C^2 d            (one rounding: fma)
 * with C = c dt / dx the Courant number. The point state is (u^n, u^{n-1}), so
 * each step is a radius-1 stencil with a 2-value point (Section 2, item 2). */
int oracle_wave(int nx, int ny, double C2, long long nsteps, double *u, double *uold) {
    if (nx < 1 || ny < 1 || nsteps < 0 || !u || !uold) return -1;
    size_t npts = (size_t)nx * ny;
    double *un = (double *)malloc(npts * sizeof(double));
    double *uo = (double *)malloc(npts * sizeof(double));
    if (!un || !uo) { free(un); free(uo); return -3; }
    for (long long s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            int jn = wrapi(j - 1, ny), js = wrapi(j + 1, ny);
            for (int i = 0; i < nx; ++i) {
                int iw = wrapi(i - 1, nx), ie = wrapi(i + 1, nx);
                size_t p = (size_t)j * nx + i;
                double c = u[p];
                double sum = (u[(size_t)j * nx + ie] + u[(size_t)js * nx + i]) +
                             (u[(size_t)j * nx + iw] + u[(size_t)jn * nx + i]);
                double d = sum - 4.0 * c;
                un[p] = fma(C2, d, 2.0 * c - uold[p]);
                uo[p] = c;
            }
        }
        memcpy(u, un, npts * sizeof(double));
        memcpy(uold, uo, npts * sizeof(double));
    }
    free(un); free(uo);
    return 0;
}
