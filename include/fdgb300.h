/*
 * fdgb300.h -- C ABI of the GB300 (sm_103a) explicit finite-difference
 * Navier-Stokes library.
 *
 * The library advances the 3-D compressible Navier-Stokes equations with
 * constant viscosity (Jammy, Jacobs & Sandham, arXiv 1610.09146, Section 2,
 * Eqs. 1-7) on the periodic cube [0, 2*pi]^3 (Section 3), discretised with
 * fourth-order central differences, the skew-symmetric convective form
 * (Eq. skewscalar), viscous terms expanded to second derivatives, and a
 * three-stage low-storage Runge-Kutta scheme (Section 2, Fig. 1).  The
 * initial state is the Taylor-Green vortex used for validation (Section 3).
 *
 * Conventions for every function below:
 *  - Return value 0 (FD_OK) on success, a negative FD_E* code on failure;
 *    fd_last_error() then gives a one-line message.  No function aborts the
 *    process, and a failed call leaves the handle usable unless it says so.
 *  - Device buffers are owned by the library (allocated through the caller's
 *    fd_alloc callbacks when given, else cudaMalloc) and freed by fd_destroy.
 *    Host buffers are owned by the caller.
 *  - A handle is not thread-safe and is bound to one CUDA stream (the one
 *    given to fd_create, or the legacy default stream when NULL) and to the
 *    device current at fd_create.  Calls that return data synchronise that
 *    stream; fd_step only enqueues work.
 *  - State layout (host or device): double Q[5][nz][ny][nx], x fastest,
 *    var = (rho, rho*u, rho*v, rho*w, rho*E); grid point (i, j, k) sits at
 *    (i*2*pi/nx, j*2*pi/ny, k*2*pi/nz).
 */
#ifndef FDGB300_H
#define FDGB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define FD_OK 0
#define FD_EINVAL (-1)    /* bad argument (size, constant, enum, NULL pointer) */
#define FD_ENOMEM (-2)    /* device or host allocation failed                  */
#define FD_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed       */
#define FD_EUNSTABLE (-4) /* non-finite value found by fd_check_finite          */
#define FD_EBUSY (-5)     /* resource exhausted (batch slots, server capacity)  */

/* ---- algorithm families (Section 2, paragraphs BL, RA, SN, RS, SS) -------
 * FD_STORE_ALL       "BL": every derivative (and every product inside a
 *                    derivative, via a product work array) is written to a
 *                    grid-sized work array; the residual is then pointwise.
 * FD_STORE_SOME      "SS": the nine velocity gradients du_i/dx_j are stored
 *                    in work arrays; every other derivative is evaluated into
 *                    thread-local registers inside the fused residual kernel.
 * FD_RECOMPUTE_ALL   "RA": no derivative is stored; every derivative is
 *                    evaluated from its finite-difference formula where used.
 * FD_RECOMPUTE_SOME  "RS": the nine velocity gradients are stored; every other
 *                    derivative is written out inside each equation that uses
 *                    it, so a derivative two equations need is evaluated twice.
 * FD_STORE_NONE      "SN": no derivative is stored; each one is evaluated once
 *                    into a thread-local variable and the equations are
 *                    assembled from those.
 * SS and RA merge the derivatives that a residual adds along one direction
 * into one stencil (a GB300-specific arithmetic saving); BL, RS and SN
 * evaluate the derivative set of the paper as written, with identical
 * arithmetic per derivative.  In all five the primitive variables u_i, p, T
 * are evaluated and stored (Section 2, the paragraph after Fig. 1).  Every
 * family exists for the dtypes FD_F64, FD_F32_ACCDW and FD_DF64; FD_F64_DW is
 * store-some only; the batch and server take SS and RA. */
#define FD_STORE_ALL 0
#define FD_STORE_SOME 1
#define FD_RECOMPUTE_ALL 2
#define FD_RECOMPUTE_SOME 3
#define FD_STORE_NONE 4
/* FD_RECOMPUTE_ALL_INLINE  RA read literally, binary64 (FD_F64) only: not even
 *                    the primitive variables are stored; u_i, p and T are
 *                    recomputed from the five conserved values at every tap
 *                    that needs them (Section 2, paragraph RA; the paragraph
 *                    after Fig. 1 stores them in every algorithm, which the
 *                    other five families follow).  The least memory of all
 *                    (the state and the saved register only), the most
 *                    binary64 arithmetic; results equal FD_RECOMPUTE_ALL's bit
 *                    for bit (same formulas per value).  Not batched. */
#define FD_RECOMPUTE_ALL_INLINE 5

/* ---- arithmetic ----------------------------------------------------------
 * FD_F64        all arithmetic in IEEE binary64 (the paper's precision,
 *               Section 3).
 * FD_F32_ACCDW  stencils, fluxes and the residual in binary32 on
 *               perturbation variables (rho-1, p-p0, T-1, rhoE-rhoE0); the
 *               conserved state and the Runge-Kutta accumulation are kept in
 *               compensated binary32 (double-words of FD_DF64, about 48
 *               significant bits, shifted by (1, 0, 0, 0, rhoE0)), so a step
 *               issues no binary64 instruction; states cross the API as
 *               binary64 and the kinetic energy / enstrophy reductions run in
 *               binary64.  The paper has no counterpart; it is a precision
 *               mode of this library.
 * FD_DF64       results within a few units of 1e-12 of binary64 without
 *               binary64 instructions: the stencils, fluxes, residual, RK
 *               accumulation and the stored state use double-word
 *               ("double-float") arithmetic, pairs of binary32 numbers with
 *               about 48 significant bits (Knuth TwoSum, Dekker FastTwoSum,
 *               FMA-based products; the algorithms of Joldes, Muller & Popescu
 *               2017), on the shifted fields of FD_F32_ACCDW.  On GB300
 *               binary32 issues 64x faster than binary64.  States cross the
 *               API as binary64; the reductions run in binary64.  Bound
 *               against the binary64 oracle (relative L-inf per variable):
 *               1e-12 at 32^3 after 10 steps; 4e-12 on rho w after one step
 *               at 256^3 (measured 1.6e-12), where rho w (<= 2e-4) resolves
 *               the binary64 rounding of the pressure (its mean is ~70 times
 *               its variation), which the double-word pressure does not
 *               reproduce; FD_F64_DW keeps that pressure in binary64 and
 *               meets 1e-12 there.  No counterpart in the paper. */
#define FD_F64 0
#define FD_F32_ACCDW 1
#define FD_DF64 2
/* FD_F64_DW     binary64 results (the binary64 parity bound of FD_F64) from
 *               mixed arithmetic, store-some family only: the state, the saved
 *               register, the RK update, the velocities u_i, div u and the
 *               pressure p of Eq. 6 (whose mean is ~70 times its variation at
 *               Mach 0.1, so its binary64 rounding is what the smallest
 *               momentum component resolves) are binary64, and the pressure
 *               gradient differences the binary64 pressures exactly (their
 *               p - p0 is held exactly as a double-word at Mach 0.1, within
 *               2^-48 |p - p0| at higher Mach); every other term of the
 *               residual and the nine stored velocity gradients use the
 *               double-word arithmetic of FD_DF64 on shifted fields.  About 45
 *               binary64 instructions per point and stage instead of ~260.
 *               No counterpart in the paper. */
#define FD_F64_DW 3

/* Device allocator callbacks (for example PyTorch's caching allocator).
 * alloc returns a device pointer aligned to at least 256 bytes, or NULL;
 * free releases a pointer returned by alloc.  Both are called only from
 * fd_create / fd_destroy (and the batch / server create and destroy calls)
 * on the caller's thread.  `stream` is the handle's cudaStream_t. */
typedef struct fd_alloc {
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
    void* ctx;
} fd_alloc;

typedef struct fd_handle fd_handle;

/* Create a solver for an nx x ny x nz periodic grid and set the Taylor-Green
 * initial condition (Section 3): u = sin x cos y cos z, v = -cos x sin y cos z,
 * w = 0, p = 1/(gamma M^2) + (cos 2x + cos 2y)(cos 2z + 2)/16, rho = gamma M^2 p.
 *   nx, ny, nz  grid points per axis, each >= 5 (the 5-point stencil needs
 *               distinct neighbours) and nx*ny*nz <= 214748364 (598^3:
 *               ten fields of one grid are addressed with 32-bit offsets);
 *   Re, Mach, Pr, gamma  flow constants (Eqs. 4-7): Re, Mach, Pr > 0,
 *               gamma > 1; dt > 0 is the time step of every fd_step;
 *   algorithm   FD_STORE_ALL, FD_STORE_SOME, FD_RECOMPUTE_ALL,
 *               FD_RECOMPUTE_SOME or FD_STORE_NONE;
 *   dtype       FD_F64, FD_F32_ACCDW, FD_DF64, or FD_F64_DW (FD_STORE_SOME only);
 *   alloc       NULL for cudaMalloc/cudaFree, else allocator callbacks;
 *   cuda_stream cudaStream_t for all work of this handle (NULL = default).
 * On success *out receives the handle.  Errors: FD_EINVAL, FD_ENOMEM,
 * FD_ECUDA (then *out is NULL and fd_last_error(NULL) has the message). */
int fd_create(fd_handle** out, int nx, int ny, int nz, double Re, double Mach, double Pr,
              double gamma, double dt, int algorithm, int dtype, const fd_alloc* alloc,
              void* cuda_stream);

/* Enqueue n >= 0 full time steps (Fig. 1): save-state, then three stages of
 * primitives -> derivatives -> residual -> periodic boundaries -> update.
 * Asynchronous on the handle's stream.  Errors: FD_EINVAL (n < 0, NULL),
 * FD_ECUDA (launch failure). */
int fd_step(fd_handle* h, int n);

/* Copy the conserved state Q (5*nx*ny*nz doubles, layout above) to dst.
 * dst_is_device = 1: dst is device memory on the handle's device; 0: host
 * memory (pageable or pinned).  n_elems must equal 5*nx*ny*nz.  Synchronises
 * the handle's stream.  Errors: FD_EINVAL, FD_ECUDA. */
int fd_get_state(fd_handle* h, double* dst, size_t n_elems, int dst_is_device);

/* Replace the conserved state with src (same layout and rules as
 * fd_get_state); checkpoint / resume at a step boundary.  Synchronises. */
int fd_set_state(fd_handle* h, const double* src, size_t n_elems, int src_is_device);

/* Stream-ordered forms of fd_get_state / fd_set_state: the copy (and, in the
 * binary32 and df64 modes, the conversion to or from the double-word state) is
 * enqueued on the handle's stream after the work already there, and the call
 * returns without waiting.  The caller keeps the host buffer alive and
 * unchanged (set) or unread (get) until the stream has reached the copy, for
 * example by synchronising the stream or an event recorded after the call;
 * only page-locked host memory gives a copy that overlaps other work.  With
 * two handles on two streams, the copies of one solve overlap the steps of
 * the other.  A kernel error word is not checked here (the synchronising
 * calls check it).  Errors: FD_EINVAL, FD_ECUDA (enqueue failure). */
int fd_get_state_async(fd_handle* h, double* dst, size_t n_elems, int dst_is_device);
int fd_set_state_async(fd_handle* h, const double* src, size_t n_elems, int src_is_device);

/* Kinetic energy and enstrophy of the current state (Section 3, Fig. 3):
 *   ke  = (1/N) sum rho |u|^2 / 2,
 *   ens = (1/N) sum rho |omega|^2 / 2, omega = curl u with the 4th-order
 *         first-derivative stencil, N = nx*ny*nz,
 * accumulated in binary64 in a fixed order (bitwise reproducible run to run).
 * Synchronises.  Either output pointer may be NULL. */
int fd_diagnostics(fd_handle* h, double* ke, double* enstrophy);

/* Evaluate the residual R(Q) of the mass, momentum and energy equations
 * (Section 2, Eqs. 1-5 with Eq. skewscalar) of the current state without
 * advancing it, with the handle's algorithm and dtype, into R (5*nx*ny*nz
 * doubles, layout of Q) on the host (dst_is_device = 0) or device (1).
 * Synchronises.  Errors: FD_EINVAL, FD_ECUDA. */
int fd_residual(fd_handle* h, double* R, size_t n_elems, int dst_is_device);

/* Scan the state for NaN or infinity.  Returns FD_OK or FD_EUNSTABLE.
 * Synchronises. */
int fd_check_finite(fd_handle* h);

/* Bytes of device memory held by the handle (state, primitives, work arrays). */
size_t fd_device_bytes(const fd_handle* h);

/* ---- per-kernel timing ----------------------------------------------------
 * Kernel classes of one stage (Fig. 1), for fd_profile_read:
 *   FD_KERNEL_PRIMS     primitive variables u_i, p, T (Eqs. 6-7), all families
 *   FD_KERNEL_GRAD      SS: the nine stored velocity gradients (not in
 *                       FD_F64_DW, whose first fused kernel forms them)
 *   FD_KERNEL_FUSED     RA / SS: fused derivatives + residual + RK update;
 *                       BL: pointwise residual + RK update; FD_F64_DW
 *                       store-some: two kernels (the diagonal gradients,
 *                       div u and the convective terms, then the rest with
 *                       the update), timed as one pass
 *   FD_KERNEL_PRODUCTS  BL: product work arrays
 *   FD_KERNEL_DERIV1    BL: first-derivative work arrays
 *   FD_KERNEL_DERIV2    BL: second- and mixed-derivative work arrays */
#define FD_KERNEL_PRIMS 0
#define FD_KERNEL_GRAD 1
#define FD_KERNEL_FUSED 2
#define FD_KERNEL_PRODUCTS 3
#define FD_KERNEL_DERIV1 4
#define FD_KERNEL_DERIV2 5
#define FD_KERNEL_CLASSES 6

/* Turn per-kernel timing on (enable != 0) or off; either way the totals are
 * reset.  While on, every launch of fd_step / fd_residual is bracketed by a
 * pair of CUDA events recorded on the handle's stream (a few microseconds
 * per launch); events are created on the first enable and freed by
 * fd_destroy.  Errors: FD_EINVAL, FD_ECUDA. */
int fd_profile(fd_handle* h, int enable);

/* Total device time in milliseconds and number of timed passes of one
 * kernel class since the last fd_profile call (one launch per pass, except
 * the two-kernel FD_F64_DW fused pass).  Synchronises the stream.  Either
 * output may be NULL.  Errors: FD_EINVAL (class out of range), FD_ECUDA. */
int fd_profile_read(fd_handle* h, int kernel_class, double* total_ms, long long* launches);

/* ---- batched instances ----------------------------------------------------
 * The paper has no counterpart: a batch advances many independent
 * Taylor-Green instances (different grids, Re, Mach, ...) together.  Each
 * stage is one persistent launch per family present (SS adds its gradient
 * kernel): a fixed grid of blocks walks a work list of tiles (instance, first
 * point, point count).  The per-point arithmetic is the single-instance
 * arithmetic, so every instance evolves bitwise as it would alone with the
 * same family and dtype.  Steps are replayed from CUDA graphs captured on the
 * first fd_batch_step. */
typedef struct fd_instance_desc {
    int nx, ny, nz;                     /* grid, each axis >= 5, nx*ny*nz <= 214748364 */
    double Re, Mach, Pr, gamma, dt;     /* as for fd_create */
    int algorithm;                      /* FD_STORE_SOME or FD_RECOMPUTE_ALL */
    int tile_points;                    /* points per work item, >= 32; 0 = 1024 (binary32
                                           recompute-all uses fixed 32 x 8 x 64 tiles instead) */
} fd_instance_desc;

typedef struct fd_batch fd_batch;

/* Create `count` >= 1 instances described by desc[0..count-1], all in one
 * dtype (FD_F64, FD_F32_ACCDW, or FD_F64_DW with every instance store-some),
 * each set to its Taylor-Green initial state.
 * One device allocation holds every instance (through alloc, else
 * cudaMalloc).  Errors: FD_EINVAL (a bad descriptor; FD_STORE_ALL is not
 * batched), FD_ENOMEM, FD_ECUDA; the message is in fd_batch_last_error(NULL). */
int fd_batch_create(fd_batch** out, const fd_instance_desc* desc, int count, int dtype, const fd_alloc* alloc,
                    void* cuda_stream);

/* Enqueue n >= 0 RK3 steps of every instance (asynchronous). */
int fd_batch_step(fd_batch* b, int n);

/* State of instance i (same layout and rules as fd_get_state / fd_set_state). */
int fd_batch_get_state(fd_batch* b, int i, double* dst, size_t n_elems, int dst_is_device);
int fd_batch_set_state(fd_batch* b, int i, const double* src, size_t n_elems, int src_is_device);

/* Kinetic energy and enstrophy of every instance into ke[count], ens[count]
 * (host arrays; either may be NULL), as fd_diagnostics.  Synchronises. */
int fd_batch_diagnostics(fd_batch* b, double* ke, double* enstrophy);

/* Number of instances, device bytes held, and per-kernel timing (same kernel
 * classes and rules as fd_profile / fd_profile_read; the batched fused and
 * gradient kernels count as FD_KERNEL_FUSED / FD_KERNEL_GRAD; while timing is
 * on, steps launch kernels directly instead of replaying graphs). */
int fd_batch_count(const fd_batch* b);
size_t fd_batch_device_bytes(const fd_batch* b);
int fd_batch_profile(fd_batch* b, int enable);
int fd_batch_profile_read(fd_batch* b, int kernel_class, double* total_ms, long long* launches);

/* Free the batch (NULL is a no-op).  Synchronises its stream first. */
int fd_batch_destroy(fd_batch* b);

/* Message of the last failed call on b, or of the last failed batch call
 * without a batch (b == NULL) on this thread; "" when there was none. */
const char* fd_batch_last_error(const fd_batch* b);

/* ---- continuous-batching server -------------------------------------------
 * The paper has no counterpart.  A server owns one device arena of a fixed
 * size and runs every admitted Taylor-Green solve through the batched kernels
 * above: requests queue in submission order; each fd_server_tick admits the
 * queued requests whose device footprint fits the free arena space (first
 * fit, later requests may pass one that does not fit yet) up to max_active
 * solves, advances every active solve (all of them in the same launches,
 * grouped by dtype and family), and retires the solves that reached their
 * step count: their kinetic energy and enstrophy become results for
 * fd_server_poll, and their final state stays readable through
 * fd_server_get_state until the first tick after their result was polled,
 * which returns their memory to the arena.  One tick stays in flight: a
 * tick enqueues its work, then waits only for the previous tick's, so the
 * solves a tick finishes become results at the next tick (at once when the
 * tick leaves no solve active).  Ticks are
 * time-sliced: a solve advances by an odd number of RK3 steps per tick, one
 * for the solve with the dearest step of the active set and, for a cheaper
 * solve, as many as fit in that step's time (at most 31, never past its
 * request), so small solves do not move at the pace of the largest.  Results
 * are those of the same solve run alone (same per-point arithmetic and
 * reduction order). */
typedef struct fd_request {
    int nx, ny, nz;                  /* grid, as for fd_create */
    double Re, Mach, Pr, gamma, dt;  /* as for fd_create */
    int steps;                       /* RK3 steps to run, >= 1 */
    int dtype;                       /* FD_F64, FD_F32_ACCDW, or FD_F64_DW (store-some only) */
    int algorithm;                   /* FD_STORE_SOME or FD_RECOMPUTE_ALL */
    int tile_points;                 /* as in fd_instance_desc */
    long long tag;                   /* caller's identifier, returned with the result */
} fd_request;

typedef struct fd_result {
    long long tag;
    int status;              /* FD_OK, FD_EUNSTABLE (non-finite diagnostics) or FD_EBUSY (cancelled) */
    int steps_done;
    double ke, enstrophy;    /* of the final state (fd_diagnostics) */
} fd_result;

typedef struct fd_server_stats {
    int queued, active;
    long long submitted, completed, ticks;
    size_t arena_bytes, arena_used;
} fd_server_stats;

typedef struct fd_server fd_server;

/* A server with a device arena of arena_bytes (allocated once, through alloc
 * if given) and at most max_active concurrent solves.  Errors: FD_EINVAL,
 * FD_ENOMEM, FD_ECUDA (message in fd_server_last_error(NULL)). */
int fd_server_create(fd_server** out, size_t arena_bytes, int max_active, const fd_alloc* alloc, void* cuda_stream);

/* Queue a request (copied).  Errors: FD_EINVAL (bad request), FD_EBUSY (its
 * footprint exceeds the whole arena, so it could never be admitted). */
int fd_server_submit(fd_server* s, const fd_request* req);

/* Device bytes a request would occupy while active (0 for a bad request). */
size_t fd_server_footprint(const fd_request* req);

/* Cancel a queued or active request by tag: it is retired at the next tick
 * with status FD_EBUSY.  Errors: FD_EINVAL if no such request is pending. */
int fd_server_cancel(fd_server* s, long long tag);

/* Admit, advance every active solve by its steps for this tick (time-sliced,
 * see above), retire the solves the previous tick finished (and this tick's,
 * if it leaves no solve active).  Waits for the previous tick's work on the
 * server's stream (for its own too when it leaves no solve active); an error
 * of a kernel's bounded wait is reported by the tick that retires the work.
 * *active_out (may be NULL) receives the number of solves active during this
 * tick.  Errors: FD_ECUDA. */
int fd_server_tick(fd_server* s, int* active_out);

/* Move up to max finished results into out[]; *n_out receives the count.
 * The next fd_server_tick releases the polled solves' device memory (and
 * states). */
int fd_server_poll(fd_server* s, fd_result* out, int max, int* n_out);

/* Copy the final state of a finished solve (layout and rules of fd_get_state:
 * 5*nx*ny*nz doubles, host or device dst, binary64 also for FD_F32_ACCDW
 * requests); valid from the tick that finished it (before its result is
 * retired, too) until the first tick after its result was polled.  If several kept solves share the tag, the one that
 * finished first.  Synchronises the server's stream.  Errors: FD_EINVAL (no
 * such solve, wrong n_elems, NULL), FD_ECUDA. */
int fd_server_get_state(fd_server* s, long long tag, double* dst, size_t n_elems, int dst_is_device);

int fd_server_get_stats(const fd_server* s, fd_server_stats* out);

/* Free the server, dropping queued and active requests.  NULL is a no-op. */
int fd_server_destroy(fd_server* s);

const char* fd_server_last_error(const fd_server* s);

/* ---- residual without any allocation -------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they need a residual, for example
 * an external time integrator that owns its state and calls R(Q) while a
 * stream capture is in progress, inside a real-time loop with a fixed memory
 * budget, or in a process whose device memory is held by another framework's
 * pool.  fd_residual needs a handle and fd_create allocates; this call needs
 * neither and calls no allocating routine.
 *
 * Q (input) and R (output) are caller-owned device arrays of 5*nx*ny*nz
 * doubles in the state layout above, on the current device, not overlapping.
 * R receives the residual of Eqs. 1-5 (Section 2, Eq. skewscalar) evaluated
 * with the store-some family in binary64; it equals what fd_residual returns
 * for a FD_STORE_SOME / FD_F64 handle holding Q.  The work is enqueued on
 * cuda_stream (NULL = default stream) and the call returns without waiting.
 *
 * Scratch: a fixed device array inside the library holds the primitives,
 * the nine velocity gradients and three sums of them for at most
 * FD_NOALLOC_MAX_POINTS grid points (35.7 MB, kept by every GPU that loads
 * the library until the process exits).  All calls share it and it keeps the last call's contents, which
 * no call reads before overwriting; two calls whose work overlaps on the GPU
 * (different streams, or host threads racing on one device) race on it and
 * must be ordered by the caller.  The first call on each device (and the first
 * after that device's context was replaced, e.g. by cudaDeviceReset) looks up
 * the scratch address with cudaGetSymbolAddress; make that call before any
 * stream capture begins.
 *
 * Errors: FD_EINVAL for a NULL pointer, an axis below 5 points, more than
 * FD_NOALLOC_MAX_POINTS points, or Re, Mach, Pr <= 0 or gamma <= 1 (nothing is
 * launched); FD_ECUDA if the set-up lookup or a launch fails.  This function
 * does not set fd_last_error's message. */
#define FD_NOALLOC_MAX_POINTS 262144 /* 64^3 */
int fd_residual_noalloc(const double* Q, double* R, int nx, int ny, int nz, double Re, double Mach,
                        double Pr, double gamma, void* cuda_stream);

/* ---- failure-detection test hook ------------------------------------------
 * Every wait inside a kernel of this library is bounded.  This call makes one
 * run out on purpose, so that tests can check what a caller then sees, without
 * a fault or a hang: it creates a 32 x 8 x 8 binary32 recompute-all solver on
 * the current device (default stream), and launches one stage of the
 * TMA-staged kernel with the copy of one plane left out, so the wait for it
 * gives up after 0.5 s; the kernel records that in its error word, waits
 * (bounded) for its other copies and ends.  *err_word receives the word (1
 * when the wait ran out, as designed); the solver is then destroyed.  The
 * paper has no counterpart.  Errors: FD_EINVAL (err_word NULL, or TMA staging
 * turned off by FDGB300_NO_TMA=1), FD_ENOMEM, FD_ECUDA. */
int fd_selftest_wait_timeout(int* err_word);

/* ---- z-slab decomposition ---------------------------------------------------
 * The paper runs its solver over MPI ranks that each own a block of the grid
 * (Section 4.1, strong and weak scaling).  Here a rank owns the planes
 * z_first .. z_first + nz_local - 1 of a periodic grid of nz_global planes
 * (a z-slab) and keeps `ghost` copies of its neighbours' planes on either side,
 * so a handle of nz_local + 2 ghost planes advances one RK3 step exactly on its
 * own planes with no exchange inside the step: a stage's result at a plane
 * depends on planes within 2 of it in every family (the stored gradients and
 * derivative arrays are differenced along z only where they are in-plane
 * derivatives), so after three stages only the outer 3 x 2 planes of each
 * ghost band are stale.  Between steps the caller refreshes the ghost planes
 * from the neighbours (fd_get_planes_async / fd_set_planes_async on the
 * ranks' streams, and NCCL send / receive or a peer copy between them): rank r
 * sends its lowest `ghost` own planes down and its highest up.  The arithmetic
 * per point is that of the whole grid, so the slabs together give exactly the
 * whole-grid result.  The paper has no API for this (its decomposition is the
 * OPS runtime's); these calls are this library's form of it.
 *
 * fd_slab_ghost_planes: the least ghost depth for an algorithm (6 for every
 * family), or -1 for an unknown algorithm.
 *
 * fd_slab_create: as fd_create for a slab; the handle's own plane k (0 <= k <
 * nz_local + 2 ghost) is plane (z_first - ghost + k) mod nz_global of the
 * grid, and its z spacing is 2 pi / nz_global.  The state (fd_get_state /
 * fd_set_state) covers all of the handle's planes, own planes at ghost ..
 * ghost + nz_local - 1.  dtype FD_F64 or FD_F64_DW; ghost >=
 * fd_slab_ghost_planes(algorithm) and <= nz_global; 0 <= z_first < nz_global,
 * 1 <= nz_local <= nz_global.  Errors as fd_create.
 *
 * fd_get_planes_async / fd_set_planes_async: copy `count` planes starting at
 * the handle's plane z of the state to / from buf, laid out
 * double[5][count][ny][nx] (host or device memory, by *_is_device),
 * stream-ordered on the handle's stream like fd_get_state_async.  Any handle
 * with a binary64 state (FD_F64, FD_F64_DW).  Errors: FD_EINVAL (NULL,
 * planes outside the handle, other dtype), FD_ECUDA. */
int fd_slab_ghost_planes(int algorithm);
int fd_slab_create(fd_handle** out, int nx, int ny, int nz_global, int z_first, int nz_local, int ghost, double Re,
                   double Mach, double Pr, double gamma, double dt, int algorithm, int dtype, const fd_alloc* alloc,
                   void* cuda_stream);
int fd_get_planes_async(fd_handle* h, int z, int count, double* dst, int dst_is_device);
int fd_set_planes_async(fd_handle* h, int z, int count, const double* src, int src_is_device);

/* ---- measured binary64 rate -----------------------------------------------
 * The denominator of the binary64 kernels' roofline: runs a loop of
 * independent binary64 FMA chains over 8 blocks of 256 threads per SM of the
 * current device (one untimed launch, then three timed ones on a private
 * stream) and stores the rate in *flops_per_s (two flops per FMA).  scratch is
 * caller-owned device memory of at least SMs * 2048 doubles (16 KB per SM)
 * that the kernel overwrites.  The paper has no counterpart.  Synchronises the
 * private stream.  Errors: FD_EINVAL (NULL, scratch too small), FD_ECUDA. */
int fd_fp64_peak(double* flops_per_s, void* scratch, size_t scratch_bytes);

/* Free every device buffer of the handle and the handle itself.  NULL is a
 * no-op.  Synchronises the handle's stream first. */
int fd_destroy(fd_handle* h);

/* Message of the last failed call on h, or of the last failed call that had
 * no handle (fd_create, or h == NULL) on this thread.  Never NULL; "" when
 * there was none.  Valid until the next call on the same handle / thread. */
const char* fd_last_error(const fd_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* FDGB300_H */
