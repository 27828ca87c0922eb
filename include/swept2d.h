/*
 * swept2d.h -- C ABI of the GB300 swept-rule library (libswept2d.so).
 *
 * Explicit time advancing of a 2D PDE on a doubly periodic Cartesian grid
 * (Section 2, item 1) by the swept rule of space-time decomposition
 * (Sections 3-4): the grid is cut into n x n tiles; each half cycle builds an
 * upward pyramid per tile (Algorithm 1), the longitudinal and latitudinal
 * bridges between them (Algorithms 2 and 3) and a downward pyramid in the
 * frame shifted by (n/2, n/2) (Algorithm 5), glued as in Algorithm 4. On the
 * GPU a tile is one thread block, its local store is shared memory, and the
 * "network" is a panel buffer in device memory plus a kernel boundary. The
 * downward pyramid of one half cycle and the upward pyramid of the next act on
 * the same tile in the same frame, so they run fused in one kernel (the
 * "octahedron"): two launches per n/2 sub-steps, or one persistent launch per
 * advance (SWEPT2D_PERSISTENT). A plain one-kernel-per-sub-step path (mode
 * SWEPT2D_NAIVE) uses the same point-update code and gives bitwise identical
 * results. Many independent grids of uneven sizes share launches through the
 * swept2d_batch_* calls.
 *
 * Conventions.
 *  - State: nvars planes of ny x nx elements, row-major, x fastest. Plane v,
 *    row j, column i is element v*nx*ny + j*nx + i. "North" is j-1, "south"
 *    j+1, "west" i-1, "east" i+1; indices wrap modulo nx and ny.
 *  - One time step = nstages sub-steps; sub-step g (counted from the last
 *    set_state) applies the point update's stage g mod nstages
 *    (Section 2, item 2; the paper's timestep(i, p), Section 5).
 *  - All functions return SWEPT2D_OK (0) or a negative status and never abort.
 *    On failure, swept2d_last_error() gives a message for that handle.
 *  - Ownership: the caller owns every pointer it passes and may free it when
 *    the call returns. The library owns its device state and panel buffers
 *    (allocated in swept2d_create, freed in swept2d_destroy).
 *  - Streams: all device work of a handle runs on the CUDA stream given at
 *    create time (NULL = the legacy default stream). set_state with a host
 *    source and get_state synchronise that stream; advance does not.
 *  - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef SWEPT2D_H
#define SWEPT2D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swept2d swept2d_t;

/* Status codes. */
#define SWEPT2D_OK        0
#define SWEPT2D_EINVAL   (-1)   /* invalid argument (message says which) */
#define SWEPT2D_ECUDA    (-2)   /* a CUDA call or kernel launch failed */
#define SWEPT2D_ENOMEM   (-3)   /* device or host allocation failed */
#define SWEPT2D_ETIMEOUT (-4)   /* a kernel's bounded wait gave up (TMA panel copies or
                                   the persistent form's neighbourhood waits); the
                                   state is unspecified until the next set_state */
#define SWEPT2D_ESTATE   (-5)   /* call out of order (e.g. advance before set_state) */

/* Point updates (the paper's St_k; Section 2, Section 5).
 *  HEAT       nvars 1, nstages 1, dtype F64, params {r}:
 *             u' = u + r ((u_E + u_S) + (u_W + u_N) - 4u), the last
 *             multiply-add fused.
 *  EULER_RK2  nvars 8, nstages 2, dtype F64, params {gamma, cfl, kappa[, lx, ly]}:
 *             planes 0-3 = (rho, rho u, rho v, E), planes 4-7 = midpoint stage
 *             U*; central flux plus scalar dissipation kappa*a with a = max wave
 *             speed of the state given to set_state; dt = cfl*min(dx,dy)/a fixed
 *             at set_state; domain lx x ly (default 1 x 1). Stage 0 writes
 *             (U, U + dt/2 L(U)); stage 1 writes (U + dt L(U*), U*).
 *  INCREMENT  nvars 1, nstages 1, dtype F64: u' = u + 1 (Section 3.1 example).
 *  HASH       nvars 1, nstages 1, dtype U64: 64-bit mix of the sub-step index
 *             and the 9 neighbour words in row order (a test update).
 *  LEVELTAG   nvars 1, nstages 1, dtype F64: u' = u + 1 if all 9 neighbours
 *             equal u, else NaN (a test update: wrong-level inputs show up).
 *  WIDE2      nvars 5, nstages 2, dtype U64: eq. (complex_step) run as its
 *             two radius-1 sub-steps, eqs. (substep1)-(substep2), modulo 2^64;
 *             plane 0 holds u after each whole step.
 *  HEAT_KAHAN nvars 2, nstages 1, dtype F32 or BF16, params {r}: the heat
 *             update in binary32 arithmetic with the time update accumulated
 *             by Kahan's compensated summation; plane 0 = u, plane 1 = the
 *             compensation c (start it at 0): delta = r ((u_E + u_S) + (u_W +
 *             u_N) - 4u), y = delta - c, u' = store(u + y), c' = store((u' - u)
 *             - y), store() = rounding to the storage type (none for F32).
 *             r is rounded to binary32. u' - c' is the compensated value.
 *  WAVE       nvars 2, nstages 1, dtype F64, params {C}: the 2D wave equation
 *             u_tt = c^2 laplace(u) by leapfrog (Section 6), C = c dt/dx the
 *             Courant number; plane 0 = u^n, plane 1 = u^{n-1}:
 *             d = ((u_E + u_S) + (u_W + u_N)) - 4u, u' = (2u - u_old) + C^2 d
 *             (fused), and the new u_old is u. C^2 is formed as C*C.
 *  EULER_KAHAN nvars 12, nstages 2, dtype F32 or BF16, params as EULER_RK2:
 *             the same scheme in binary32 arithmetic with the time update
 *             compensated as in HEAT_KAHAN; planes 0-3 = U, 4-7 = U*, 8-11 =
 *             the compensation C of U (start it at 0). Stage 0 writes U* =
 *             store(U + dt/2 L(U)); stage 1: y = dt L(U*) - C, U' = store(U +
 *             y), C' = store((U' - U) - y). The constants (and a, dt) are formed
 *             in binary64 as for EULER_RK2 and rounded once to binary32.
 */
#define SWEPT2D_OP_HEAT       0
#define SWEPT2D_OP_EULER_RK2  1
#define SWEPT2D_OP_INCREMENT  2
#define SWEPT2D_OP_HASH       3
#define SWEPT2D_OP_LEVELTAG   4
#define SWEPT2D_OP_WIDE2      5
#define SWEPT2D_OP_HEAT_KAHAN 6
#define SWEPT2D_OP_WAVE       7
#define SWEPT2D_OP_EULER_KAHAN 8

/* Element types of the state. */
#define SWEPT2D_F64  0
#define SWEPT2D_F32  1
#define SWEPT2D_BF16 2   /* bfloat16: the upper 16 bits of a binary32 */
#define SWEPT2D_U64  3

/* Advance modes. */
#define SWEPT2D_SWEPT 0   /* swept rule: Up, then per half cycle Bridge + Octahedron, final Down */
#define SWEPT2D_NAIVE 1   /* one kernel launch per sub-step over the whole grid */
/* Flag OR-ed into the mode: run the advance's launch sequence as a CUDA graph.
 * The first advance with a given (nsteps, mode) and state buffer is captured
 * (stream capture on the handle's stream, which must not be the legacy default
 * stream) and cached (up to 8 per handle); later ones replay it with one graph
 * launch. Results are the same bits as without the flag. Changing the launch
 * shape (swept2d_set_tuning) drops the cached graphs. */
#define SWEPT2D_GRAPH 0x100
/* Flag OR-ed into SWEPT2D_SWEPT: run all half cycles of the advance as one
 * persistent launch (resident blocks take tile work items in phase order and
 * wait, with bounded spins, only for their 3 x 3 tile neighbourhood to finish
 * the previous phase), instead of two launches per half cycle. Uses the
 * handle's tuning (threads, staging); same bits. */
#define SWEPT2D_PERSISTENT 0x200
/* Batches only, OR-ed with SWEPT2D_SWEPT | SWEPT2D_PERSISTENT: one persistent
 * launch covers the half cycles of every tile class, instead of one persistent
 * launch per class. Its blocks (256 threads, shared memory for the largest
 * class) take the classes in order; the tile-16 and tile-32 classes run in
 * teams of warps (one small tile per team), larger ones one tile per block;
 * each class keeps its own tile side, half-cycle count, counters and item
 * counter. Staging follows swept2d_batch_set_tuning and is dropped if the
 * staged blocks do not fit; the thread count of that tuning is not used. Naive
 * tails (steps that do not fill a half cycle of a class) follow as before.
 * Same bits. EINVAL without SWEPT2D_PERSISTENT, for a single-grid handle, with
 * more than 16 classes, or if even unstaged blocks do not fit. */
#define SWEPT2D_ONE_LAUNCH 0x400

/*
 * Create a handle for an nx x ny grid.
 *   tile   side n of the square tiles for the swept mode: even, >= 4, dividing
 *          nx and ny, and small enough that a swept block's shared memory fits
 *          (the (n+2)^2 x nvars level buffer, two for the updates not computed
 *          in place, plus the level's scratch values: heat and wave one plane
 *          of pair sums, Euler four planes of primitives; SWEPT2D_Q_SMEM_BYTES
 *          gives the figure); 0 = naive mode only.
 *   params op parameters (see above); nparams their count.
 *   stream a cudaStream_t (NULL = legacy default stream).
 * Allocates the device state and, if tile > 0, two panel buffers of
 * 4 (n^2/2 + n) nvars elements per tile each. Errors: EINVAL (bad sizes, op
 * mismatch), ENOMEM, ECUDA. On error *out is NULL.
 */
int swept2d_create(swept2d_t **out, int nx, int ny, int nvars, int nstages, int tile,
                   int op, const double *params, int nparams, int dtype, void *stream);

/* Copy nvars*ny*nx elements from src (device memory if src_is_device, else host
 * memory) into the state, and reset the sub-step counter to 0. For EULER_RK2 it
 * also computes the wave speed a and the fixed dt (Section 7's CFL number read
 * as a fixed step from the initial state). Errors: EINVAL (NULL), ECUDA. */
int swept2d_set_state(swept2d_t *h, const void *src, int src_is_device);

/* Advance nsteps whole time steps (nsteps*nstages sub-steps) with mode
 * SWEPT2D_SWEPT or SWEPT2D_NAIVE. The swept mode runs
 * H = floor(nsteps*nstages / (n/2)) half cycles and the remaining sub-steps
 * with the naive kernel. Asynchronous on the handle's stream; the state is in
 * natural storage when the work completes. Errors: EINVAL (nsteps < 0, swept
 * mode on a naive-only handle), ESTATE (no set_state yet), ECUDA. */
int swept2d_advance(swept2d_t *h, long long nsteps, int mode);

/* Copy the state to dst (device memory if dst_is_device, else host memory),
 * after all work queued on the handle's stream; synchronises the stream.
 * Errors: EINVAL (NULL), ESTATE, ECUDA, ETIMEOUT (a kernel's bounded wait for
 * its panel copies gave up since the last set_state; the state is then
 * unspecified). */
int swept2d_get_state(swept2d_t *h, void *dst, int dst_is_device);

/*
 * Self-test of the persistent form's bounded waits (no counterpart in the
 * paper; Section 4's exchanges are the dependencies being waited for): runs the
 * persistent kernel for one half cycle with its first phase skipped, so the
 * phase counters those waits read are never released. Every block's wait gives
 * up after spin_limit polls (>= 1; each poll is a load plus a ~64 ns pause, so
 * a few thousand take milliseconds), records the timeout in the handle's error
 * word and returns. No work item runs, so the state is unchanged; the error
 * word is cleared again before the call returns.
 * Returns SWEPT2D_ETIMEOUT when the kernel reported the timed-out wait (the
 * expected outcome), SWEPT2D_ESTATE if it did not, EINVAL (no tile, bad
 * spin_limit, shared memory too large), ECUDA.
 */
int swept2d_selftest_wait_timeout(swept2d_t *h, long long spin_limit);

/* Free all device memory of the handle and the handle itself (NULL is a no-op).
 * Synchronises the handle's stream first. */
int swept2d_destroy(swept2d_t *h);

/* Last error message of the handle ("" if none). With h NULL: the message of
 * the last failed swept2d_create on the calling thread. */
const char *swept2d_last_error(const swept2d_t *h);

/* Read-only queries, written to *out as a double. */
#define SWEPT2D_Q_DT            0   /* EULER_RK2: fixed time step */
#define SWEPT2D_Q_WAVESPEED     1   /* EULER_RK2: max wave speed a of the initial state */
#define SWEPT2D_Q_SUBSTEPS      2   /* sub-steps advanced since set_state */
#define SWEPT2D_Q_LAUNCHES      3   /* kernels launched by this handle since create */
#define SWEPT2D_Q_STATE_BYTES   4   /* bytes of one state copy */
#define SWEPT2D_Q_PANEL_BYTES   5   /* bytes of one panel buffer (0 if naive-only) */
#define SWEPT2D_Q_SMEM_BYTES    6   /* dynamic shared memory per swept block */
#define SWEPT2D_Q_CELLS         7   /* points of the grid (of all grids, for a batch) */
#define SWEPT2D_Q_THREADS       8   /* swept threads per block (swept2d_set_tuning) */
#define SWEPT2D_Q_STAGE         9   /* 1 if the swept kernels stage panels by TMA */
int swept2d_query(const swept2d_t *h, int what, double *out);

/* Launch shape of the swept kernels of a handle (a tuning knob, not a change
 * of results: every setting gives the same bits). threads: 32, 64, 128, 256 or 512
 * per block (default 256; the persistent form also takes up to 512; the bridge
 * launches of the launch-per-phase form take at most 256). stage: 1 =
 * the bridge and downward-pyramid blocks bring their input panel set into
 * shared memory with TMA bulk copies (a bridge's at block start, a downward
 * pyramid's in two parts, the second once the first part's levels have taken
 * their rings); 0 = they copy every
 * level's strip or ring from device memory straight into its level buffer with
 * cp.async at block start (default: 1 for HEAT_KAHAN with BF16 storage, 0
 * otherwise, and 0 wherever the staged panels do not fit).
 * Errors: EINVAL (bad value, naive-only handle, does not fit). */
int swept2d_set_tuning(swept2d_t *h, int threads, int stage);

/* Kernel timing: when on, every launch of the handle is bracketed by CUDA
 * events on the handle's stream. swept2d_kernel_stats synchronises the stream
 * and returns, for one kernel kind, the number of timed launches and their
 * summed duration in milliseconds since timing was switched on. */
#define SWEPT2D_K_NAIVE       0
#define SWEPT2D_K_UP          1
#define SWEPT2D_K_BRIDGE      2
#define SWEPT2D_K_OCTAHEDRON  3
#define SWEPT2D_K_DOWN        4
#define SWEPT2D_K_REDUCE      5
#define SWEPT2D_K_COUNT       6
int swept2d_set_timing(swept2d_t *h, int on);

/* Per-item trace of the persistent form (a measurement aid; no counterpart in
 * the paper). With a device buffer of `items` pairs of unsigned 32-bit words
 * (the caller's; the library allocates nothing for it), every later persistent
 * advance of the handle records, for work item i in the kernel's order (tiles
 * T*Q first Ups, then per half cycle 2 T*Q bridge items and T*Q octahedron or
 * final Down items), buf[2i] = SM clock cycles the block waited for the item's
 * 3 x 3 neighbourhood and buf[2i+1] = cycles it spent on the item up to its
 * release. NULL and 0 turn it off. An advance with more items than `items`
 * fails with EINVAL. Captured graphs of the handle are dropped.
 * Errors: EINVAL (buffer without size or the reverse), ECUDA. */
int swept2d_set_trace(swept2d_t *h, void *device_buffer, long long items);
int swept2d_kernel_stats(swept2d_t *h, int kind, long long *launches, double *total_ms);

/* Measured rates of this GPU for the roofline, each timed with CUDA events on
 * `stream` (best of five launches after a warm-up), written to out[0..nout):
 *   out[0]  FP64 lane-operations per second: the maximum over fused
 *           multiply-add chains (4, 8 and 16 per thread) and add chains (8),
 *           each at 2, 4 and 8 blocks of 256 threads per SM (one FMA = one
 *           operation);
 *   out[1]  FP32 lane-operations per second (16 fused multiply-add chains per
 *           thread, 8 blocks of 256 threads per SM);
 *   out[2]  shared-memory wavefronts per second: warp loads of 32 consecutive
 *           4-byte words (one wavefront each, no bank conflict);
 *   out[3]  FP64 fused multiply-add warp instructions per second with all 32
 *           lanes of every warp active (8 chains, 8 blocks of 256 per SM);
 *   out[4]  the same with one active lane per warp (equal to out[3] where the
 *           FP64 pipe's time is per warp instruction, not per lane).
 * nout >= 1; entries beyond 5 are left alone. Allocates a small device buffer
 * for the kernels' results (freed before returning).
 * Errors: EINVAL (out NULL or nout < 1), ENOMEM, ECUDA. */
int swept2d_measure_peaks(void *stream, double *out, int nout);

/* out[0] of swept2d_measure_peaks alone: the FP64 lane-operation rate. */
int swept2d_measure_fp64_rate(void *stream, double *ops_per_s);

/*
 * Batched form: many independent periodic grids of uneven sizes, advanced
 * together by the same number of steps (the paper's method applied to each grid
 * separately; no grid exchanges data with another). Grids with the same tile
 * side form a class, and one launch per swept phase (or per naive sub-step)
 * covers every tile of every grid of the class, so a batch of small grids costs
 * the launches of one grid.
 *   count       number of grids; nx[i], ny[i] their sizes
 *   tile[i]     tile side of grid i (even, >= 4, dividing nx[i] and ny[i]), or 0
 *               for a grid that only takes naive steps
 *   op, params, dtype, stream   as for swept2d_create; supported: HEAT (F64),
 *               HEAT_KAHAN (F32, BF16), HASH (U64), EULER_RK2 (F64), EULER_KAHAN
 *               (F32, BF16); for the Euler updates each grid's wave speed a and
 *               time step dt come from its own state at set_state, its spacing
 *               is lx / nx[i], ly / ny[i]
 * State layout: the grids' states concatenated in grid order, each nvars planes
 * of ny[i] x nx[i]. Modes: SWEPT2D_SWEPT or SWEPT2D_NAIVE, optionally OR-ed with
 * SWEPT2D_GRAPH (not for HASH); SWEPT2D_SWEPT may also be OR-ed with
 * SWEPT2D_PERSISTENT (one persistent launch per tile class runs all of the
 * class's half cycles, waiting per grid on each tile's 3 x 3 neighbourhood),
 * and that with SWEPT2D_ONE_LAUNCH (one persistent launch for all classes).
 * Every call returns a status; messages through
 * swept2d_batch_last_error (NULL batch: the last failed create on this thread).
 */
typedef struct swept2d_batch swept2d_batch_t;
int swept2d_batch_create(swept2d_batch_t **out, int count, const int *nx, const int *ny,
                         const int *tile, int op, const double *params, int nparams, int dtype,
                         void *stream);
int swept2d_batch_set_state(swept2d_batch_t *b, const void *src, int src_is_device);
int swept2d_batch_advance(swept2d_batch_t *b, long long nsteps, int mode);
int swept2d_batch_get_state(swept2d_batch_t *b, void *dst, int dst_is_device);
/* Launch shape (as swept2d_set_tuning) of every class, or of the class of one
 * tile side (EINVAL if no grid uses it); never changes results. */
int swept2d_batch_set_tuning(swept2d_batch_t *b, int threads, int stage);
int swept2d_batch_set_class_tuning(swept2d_batch_t *b, int tile, int threads, int stage);
int swept2d_batch_destroy(swept2d_batch_t *b);
const char *swept2d_batch_last_error(const swept2d_batch_t *b);
int swept2d_batch_query(const swept2d_batch_t *b, int what, double *out);
/* Per-grid values: SWEPT2D_Q_DT and SWEPT2D_Q_WAVESPEED (Euler updates, fixed at
 * set_state; 0 otherwise) and SWEPT2D_Q_CELLS of grid `grid` (0-based).
 * Errors: EINVAL (bad handle, grid or query). */
int swept2d_batch_query_grid(const swept2d_batch_t *b, int grid, int what, double *out);

/*
 * Allocation-free swept advance of the heat equation (FP64). The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory where they advance a grid -- e.g. an application that owns all device
 * memory through its own fixed pool and forbids cudaMalloc outside it (or a
 * plugin running inside one), or a latency-critical loop that cannot afford the
 * implicit device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * It advances the nx x ny grid u_in (device memory, one FP64 plane, row-major)
 * by nsteps steps of HEAT with diffusion number r and tile n = `tile`, writing
 * u_out (device memory; must not overlap u_in; u_in is not modified). The result
 * is bit for bit that of a handle (op HEAT, same tile) advanced in mode
 * SWEPT2D_SWEPT, sub-step indices counted from 0. Work is queued on `stream`
 * (a cudaStream_t; NULL = legacy default stream) and the call returns without
 * synchronising.
 *
 * Memory. It calls no cudaMalloc, cudaFree or other allocating routine. Its only
 * scratch is a static device array of SWEPT2D_STATIC_SCRATCH_BYTES in this
 * library, which every GPU that loads the library holds until the process
 * exits. It needs 2 * 4 * (n*n/2 + n) * 8 bytes per tile (the two panel
 * buffers; n*n/2 + n rounded up to a multiple of 8) plus nx*ny*8 bytes when
 * nsteps is not a multiple of n/2, each part
 * rounded up to 256 bytes; larger grids are rejected with SWEPT2D_EINVAL and a
 * message. Nothing in the scratch needs to start at zero.
 *
 * Set-up. Every call looks up the device address of the scratch array on the
 * current device (cudaGetSymbolAddress; nothing is cached, so a device reset or
 * another context on the same device is harmless). The first call on a device
 * is also where the runtime loads this library's device code there; make that
 * first call before any stream capture begins.
 *
 * Concurrency. All calls on a device share the one scratch array, and it keeps
 * the contents of the last call: calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it and corrupt each other's results.
 * Order them on one stream or synchronise between them.
 *
 * Errors: SWEPT2D_EINVAL (bad sizes or pointers, grid too large for the
 * scratch), SWEPT2D_ECUDA; a message goes to err (errlen bytes, may be NULL).
 */
#define SWEPT2D_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
int swept2d_heat_advance_static(const double *u_in, double *u_out, int nx, int ny, int tile,
                                double r, long long nsteps, void *stream, char *err, int errlen);

#ifdef __cplusplus
}
#endif
#endif /* SWEPT2D_H */
