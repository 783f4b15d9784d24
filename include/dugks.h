/*
 * dugks.h -- C ABI of the GB300 (sm_103a) third-order DUGKS library.
 *
 * The library advances the isothermal BGK-Boltzmann equation
 *     df/dt = L(f) + Omega(f),  L = -xi . grad f,  Omega = -(f - feq)/tau
 * (arXiv:1709.05458, Sec. 2.1.1, eq. BE) on a uniform 2-D cell-centred
 * finite-volume mesh with a discrete velocity set, using the two-stage
 * third-order DUGKS time step of Sec. 2.1.3 (Steps (1)-(4), eq.
 * feqIntD3rdHat2_DS).  Every step of that path runs in the library's own
 * CUDA kernels on the stream given at init.
 *
 * Conventions shared by all calls
 *   - Status: every function returns an int, DUGKS_OK (0) on success or a
 *     negative DUGKS_E* code.  Nothing throws or exits across the ABI.
 *     dugks_last_error() returns a thread-local message for the last
 *     failing call on the calling thread (or a warning set by dugks_init).
 *   - Layout of per-(velocity, cell) arrays: structure of arrays
 *     f[k][j][i], velocity k = 0..nv-1 slowest, cell row j = 0..ny-1 (y),
 *     cell column i = 0..nx-1 (x) fastest; cell (i, j) is centred at
 *     ((i + 1/2) dx, (j + 1/2) dy).  Per-cell arrays are [j][i].
 *   - Memory: the context owns its device state.  Pointers passed in are
 *     borrowed for the duration of the call only.  With on_device = 0 they
 *     are host pointers (pageable or pinned); with on_device = 1 they are
 *     device pointers on the context's device, read or written on the
 *     context's stream (the caller keeps them alive until that stream
 *     reaches the call; device-side calls are asynchronous).
 *   - Threading: one context per stream; a context is not thread-safe.
 */
#ifndef DUGKS_H
#define DUGKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DUGKS_OK          0
#define DUGKS_EINVAL     (-1)  /* bad argument (sizes, tau, dt, boundary set, ...) */
#define DUGKS_ECUDA      (-2)  /* a CUDA runtime error; message in dugks_last_error */
#define DUGKS_ENOMEM     (-3)  /* device allocation failed */
#define DUGKS_EUNSTABLE  (-4)  /* non-finite or non-positive density detected */
#define DUGKS_ENOTIMPL   (-5)  /* option not provided by this build */

/* boundary kinds (Sec. 2.3) and side order of the bc[4] array */
enum { DUGKS_BC_PERIODIC = 0,   /* index wrap; opposite sides must both be periodic */
       DUGKS_BC_BOUNCEBACK = 1, /* eq. BB, wall velocity (uw_x, uw_y) */
       DUGKS_BC_DIFFUSE = 2 };  /* diffuse scattering, wall velocity (uw_x, uw_y) */
enum { DUGKS_WEST = 0, DUGKS_EAST = 1, DUGKS_SOUTH = 2, DUGKS_NORTH = 3 };

/* Storage and arithmetic form of the distribution.
 *   DUGKS_FP64   : FP64 storage and arithmetic throughout (any velocity set).
 *   DUGKS_G_FP32 : per-(cell, velocity) arrays hold the deviation
 *                  d = f - W_k rho0 (rho0 = 1) in FP32; interface stencils,
 *                  fluxes and the per-velocity equilibrium assembly run in
 *                  FP32; the moment sums (Sec. 2.2) are accumulated exactly
 *                  in 64-bit fixed point (2^-56 resolution) and rounded to
 *                  FP64; 1/rho and the equilibrium parameters u/RT,
 *                  |u|^2/(2RT) are FP64.  Deviations must stay below 8 in
 *                  magnitude (rho below ~18); larger ones turn the moment
 *                  into NaN, which dugks_check reports as DUGKS_EUNSTABLE.
 *   DUGKS_G_BF16 : as DUGKS_G_FP32 with the deviations stored in BF16.
 *   DUGKS_F64_DW : FP64 storage; every operation of the step in double-word
 *                  arithmetic (a value is an unevaluated sum of two FP32
 *                  numbers, 48-bit significand, unit roundoff 2^-48; sums
 *                  with a normwise error bound), which GB300 runs on its
 *                  FP32 pipes.  Fused D2Q9 kernels only: other velocity
 *                  sets, DUGKS_PATH_GENERIC, the T2 schemes, the adjoint
 *                  and the batched launch refuse it (DUGKS_ENOTIMPL; a batch
 *                  steps such a context with its own launches).
 * The description above is that of the fused D2Q9 kernels, taken when the
 * set is in the D2Q9 listing order of Sec. 2.2 (xi_k = c (k/3 - 1, k%3 - 1)).
 * Any other velocity set (Newton-Cotes grids) runs the deviation forms on
 * the generic kernels: the same FP32/BF16 storage and FP32 stencils, FP32
 * face values, moment sums of every cell and face accumulated as
 * compensated FP32 pairs (each product and sum error-free transformed, the
 * pair rounded once to FP64; no magnitude limit; a non-finite deviation
 * gives a non-finite moment).  States cross the ABI in FP64 for every
 * form. */
enum { DUGKS_FP64 = 0, DUGKS_G_FP32 = 1, DUGKS_G_BF16 = 2, DUGKS_F64_DW = 3 };

typedef struct dugks_ctx dugks_ctx;   /* opaque, owned by the library */

/* Uniform Cartesian mesh of nx * ny cells of size dx * dy (Sec. 2.1.2). */
typedef struct { int nx, ny; double dx, dy; } dugks_mesh;

/* Discrete velocity set (Sec. 2.2): nv velocities (xi_x[k], xi_y[k]) and the
 * weights W_k of the equilibrium feq_k = W_k rho [1 + xi.u/RT
 * + (xi.u)^2/(2 RT^2) - |u|^2/(2 RT)] (second-order expansion, Sec. 2.1.1).
 * For D2Q9 these are the Gauss-Hermite weights; for a Newton-Cotes grid
 * W_k is the quadrature weight times the Maxwellian factor.  Host arrays,
 * copied at dugks_init. */
typedef struct { int nv; const double* xi_x; const double* xi_y; const double* w; double RT; } dugks_velset;

/* One side of the domain: kind and wall velocity (ignored for periodic). */
typedef struct { int kind; double uw_x, uw_y; } dugks_bc;

/*
 * dugks_init -- validate the problem and allocate device state.
 *   mesh, vel   : problem definition (copied).
 *   tau, dt     : relaxation time and time step, both > 0.  dt/tau > 12
 *                 exceeds the stability bound of Sec. 2.1.1 (P^_n <= 1 at
 *                 a = 1/3): accepted, with a warning in dugks_last_error.
 *   bc[4]       : sides in the order WEST, EAST, SOUTH, NORTH.  A wall
 *                 direction needs at least 3 cells across (the stencil ghost
 *                 extrapolation uses three cells); bounce-back needs -xi_k in
 *                 the set for every velocity leaving that wall; diffuse walls
 *                 need at least one velocity leaving the wall.
 *   storage     : DUGKS_FP64, DUGKS_G_FP32, DUGKS_G_BF16 or DUGKS_F64_DW
 *                 (see above).
 *   cuda_stream : cudaStream_t (may be NULL = legacy default stream) on which
 *                 every later call of this context runs.
 *   out         : receives the new context.
 * The state is zero until dugks_set_state or dugks_set_equilibrium.
 * Errors: EINVAL, ENOTIMPL, ENOMEM, ECUDA.
 */
int dugks_init(const dugks_mesh* mesh, const dugks_velset* vel, double tau, double dt,
               const dugks_bc bc[4], int storage, void* cuda_stream, dugks_ctx** out);

/* Kernel paths of dugks_init_ex.  dugks_init takes DUGKS_PATH_AUTO: the
 * fused D2Q9 kernels for a set in the D2Q9 listing order of Sec. 2.2, the
 * optimised generic kernels for any other set.  DUGKS_PATH_GENERIC takes the
 * optimised generic kernels for every set (a D2Q9 set included);
 * DUGKS_PATH_REFERENCE the reference FP64 kernels that also run the T2
 * schemes, the adjoint's forward recomputation and dugks_step_static (FP64
 * storage only).  All paths compute the same step; the selector exists so
 * that one problem can be run on each of them and compared. */
enum { DUGKS_PATH_AUTO = 0, DUGKS_PATH_GENERIC = 1, DUGKS_PATH_REFERENCE = 2 };

/*
 * dugks_init_ex -- dugks_init with an explicit kernel path.
 *   path : DUGKS_PATH_AUTO, DUGKS_PATH_GENERIC or DUGKS_PATH_REFERENCE.
 * Errors: those of dugks_init; EINVAL for an unknown path; ENOTIMPL for
 * DUGKS_PATH_REFERENCE with a deviation storage form, and for
 * DUGKS_F64_DW on any path but DUGKS_PATH_AUTO with a D2Q9 set.
 */
int dugks_init_ex(const dugks_mesh* mesh, const dugks_velset* vel, double tau, double dt,
                  const dugks_bc bc[4], int storage, int path, void* cuda_stream,
                  dugks_ctx** out);

/*
 * dugks_set_equilibrium -- f^ = feq(rho, u) in every cell (the paper's
 * initialisation, Sec. 3: f = feq, hence f^ = f - dt/4 Omega = feq).
 *   rho, ux, uy : per-cell arrays [ny][nx], rho > 0.
 */
int dugks_set_equilibrium(dugks_ctx* ctx, const double* rho, const double* ux,
                          const double* uy, int on_device);

/* dugks_set_state -- copy f^ = f - dt/4 Omega (eq. feqIntD3rdHat2), array
 * [nv][ny][nx], into the context.  With on_device = 0 the call returns once
 * the host array has been copied (it may then be freed or reused); the
 * work that follows the copy (the conversion of the deviation forms, the
 * fused D2Q9 path's first pass, eq. f_bar_1_6) stays queued on the stream. */
int dugks_set_state(dugks_ctx* ctx, const double* fhat, int on_device);

/* dugks_get_state -- copy a distribution [nv][ny][nx] of the current state
 * out.  which = DUGKS_STATE_SCHEME: the scheme's own variable, the one
 * dugks_set_state takes (f^ = f - dt/4 Omega under T3S3, eq.
 * feqIntD3rdHat2; f~ = f - dt/2 Omega under a T2 scheme, eq.
 * feqIntD2nd_Explicit).  which = DUGKS_STATE_F: the distribution f itself,
 * f = (4 tau f^ + dt feq)/(4 tau + dt) (T3S3; (2 tau f~ + dt feq)/(2 tau + dt)
 * under T2), feq from the moments of the state (the collision conserves
 * them), computed on the device in FP64.  With on_device = 0 the call waits
 * for the context's stream.  Errors: EINVAL (NULL, unknown which), ECUDA. */
enum { DUGKS_STATE_SCHEME = 0, DUGKS_STATE_F = 1 };
int dugks_get_state(dugks_ctx* ctx, double* out, int which, int on_device);

/*
 * dugks_step -- advance n >= 0 T3S3 steps (Sec. 2.1.3, Steps (1)-(4)):
 *   (1) moments of f^, feq, f-bar^{+,dt/6} (eq. f_bar_1_6), interface values
 *       at t* = t_n + dt/6 by eqs. interfaceEvof/flux_DS with walls (Sec.
 *       2.3), f-bar -> f (eq. recover2f), micro-flux L* (eq. microflux);
 *   (2) f~(t') = f~+(t_n) + dt/3 L* (eqs. f_tilde_1_3, feqIntD2nd_Explicit),
 *       its moments and dt Omega(f') (eq. collisionterm);
 *   (3) f-bar^{+,5dt/12}(t') and L** at t** = t_n + 3dt/4;
 *   (4) f^^{n+1} = f^+ + 3/4 dt Omega' + dt/7 (3 L* + 4 L**).
 * Asynchronous on the context's stream; returns ECUDA if a launch failed.
 */
int dugks_step(dugks_ctx* ctx, int n);

/* dugks_moments -- rho = sum_k f_k, (ux, uy) = sum_k xi_k f_k / rho of the
 * current state (Sec. 2.2; the moments of f^ equal those of f because the
 * collision conserves them).  Each output is [ny][nx] FP64; any output
 * pointer may be NULL.  When ux = rho + nx*ny and uy = rho + 2*nx*ny (one
 * [3][ny][nx] buffer) the three arrays arrive in a single copy.  With
 * on_device = 0 the call waits for the context's stream. */
int dugks_moments(dugks_ctx* ctx, double* rho, double* ux, double* uy, int on_device);

/* dugks_check -- scan the state for non-finite values or rho <= 0 (waits
 * for the stream).  Returns DUGKS_OK or DUGKS_EUNSTABLE. */
int dugks_check(dugks_ctx* ctx);

/* dugks_synchronize -- wait for all work queued on the context's stream. */
int dugks_synchronize(dugks_ctx* ctx);

/*
 * Launch profiling.  dugks_profile(ctx, 1) brackets every kernel launch of
 * the context with CUDA events on its stream; dugks_profile_read waits for
 * the stream and returns, for kernel id 0..n-1, the number of launches and
 * the summed device time in ms since profiling was enabled.  Names of the
 * ids come from dugks_kernel_name.  Returns the number of kernel ids.
 */
int dugks_profile(dugks_ctx* ctx, int enable);
int dugks_profile_read(dugks_ctx* ctx, long long* launches, double* ms, int n);
const char* dugks_kernel_name(int id);

/*
 * dugks_autotune -- choose the tile height of the fused D2Q9 kernels for this
 * problem by timing `trials` steps for every height 4..16 (4..12 for
 * DUGKS_F64_DW, whose kernels keep two blocks per SM) on the context's
 * own stream and state (f^ is saved and restored; the state is unchanged on
 * return).  The chosen height is kept by the context and written to *ty_out.
 * Other velocity sets: DUGKS_ENOTIMPL.  Results of later steps are
 * identical for every tile height (same arithmetic per face and cell).
 */
int dugks_autotune(dugks_ctx* ctx, int trials, int* ty_out);

/*
 * dugks_set_tile_height -- fix the tile height (rows of cells per block) of
 * the fused D2Q9 kernels, e.g. one that dugks_autotune chose on an earlier
 * run of the same problem, without timing anything.  ty must lie in 4..16
 * (4..12 for DUGKS_F64_DW), else DUGKS_EINVAL and the height is unchanged;
 * other velocity sets: DUGKS_ENOTIMPL.  Results of later steps are identical
 * for every height.  A batch reads the height when it is created.
 * dugks_tile_height writes the current height to *ty_out.
 */
int dugks_set_tile_height(dugks_ctx* ctx, int ty);
int dugks_tile_height(dugks_ctx* ctx, int* ty_out);

/*
 * Batched stepping of many independent problems (contexts) in one CUDA
 * graph.  All FP64 D2Q9 contexts of the batch advance together through one
 * persistent launch per stage whose blocks take (instance, tile) work items
 * from an atomic counter, so uneven grid sizes and parameters share the
 * GPU; the other contexts (Newton-Cotes sets, deviation storage) run their
 * own launches inside the same graph, in up to eight concurrent branches
 * (largest first into the branch with the least cells x velocities).  The
 * contexts must share one non-default stream; their parameters and tile
 * heights are read at dugks_batch_create, and the fused instances run with
 * the largest of their tile heights (every block of the persistent launch
 * has that many rows of threads; results do not depend on the height).
 *   dugks_batch_create   -- ctxs[n] (borrowed; keep them alive while the
 *                           batch exists) -> *out.
 *   dugks_batch_step     -- advance every context nsteps steps: the graph for
 *                           this nsteps is captured on first use and replayed
 *                           afterwards (asynchronous on the stream).
 *   dugks_batch_autotune -- time `trials` steps of the persistent launch at
 *                           every tile height and keep the fastest (*ty_out,
 *                           0 without fused instances); the fused instances'
 *                           states are restored, results do not change, and
 *                           graphs captured before are dropped.  Synchronous.
 *   dugks_batch_destroy  -- free the batch (not the contexts).
 */
typedef struct dugks_batch dugks_batch;
int dugks_batch_create(dugks_ctx* const* ctxs, int n, dugks_batch** out);
int dugks_batch_step(dugks_batch* batch, int nsteps);
int dugks_batch_autotune(dugks_batch* batch, int trials, int* ty_out);
int dugks_batch_destroy(dugks_batch* batch);

/*
 * Adjoint (reverse-mode derivative) of the T3S3 step, FP64 storage only
 * (DUGKS_ENOTIMPL otherwise).  It is the exact transpose of the linearised
 * step of dugks_step (Sec. 2.1.3, Steps (1)-(4)): equilibrium Jacobians of
 * the cell and face moments, the transposed upwind reconstruction (eq.
 * flux_DS) and micro-flux (eq. microflux), the bounce-back (eq. BB) and
 * diffuse-scattering wall rules, and the derivatives of every coefficient
 * with respect to tau.  Parameter adjoints are ADDED to the caller's
 * accumulators: dJ_dtau[0], and dJ_duw[8] = (d/d uw_x, d/d uw_y) for the
 * sides WEST, EAST, SOUTH, NORTH.  Gradient arrays are host pointers.
 *
 * dugks_adjoint_step -- lam_out = (d f^^{n+1} / d f^^n)^T lam_in for the step
 *   taken from the context's current state f^^n (set it first); the
 *   forward intermediates are recomputed.  lam_in/lam_out [nv][ny][nx].
 */
int dugks_adjoint_step(dugks_ctx* ctx, const double* lam_in, double* lam_out, double* dJ_dtau,
                       double* dJ_duw, int on_device);

/*
 * dugks_adjoint_run -- run nsteps forward from fhat0, keeping a checkpoint
 * every `every` steps in device memory (ceil(nsteps/every) + every + 1
 * state-sized buffers, kept by the context), then sweep backwards from
 * lam_final = dJ/df^^N, recomputing each segment from its checkpoint.
 * lam0 receives dJ/df^^0; the parameter adjoints are added as above.  On
 * return the context's state is f^^N.
 */
int dugks_adjoint_run(dugks_ctx* ctx, const double* fhat0, int nsteps, int every,
                      const double* lam_final, double* lam0, double* dJ_dtau, double* dJ_duw,
                      int on_device);

/*
 * dugks_adjoint_equilibrium -- adjoint of dugks_set_equilibrium
 * (f^ = feq(rho, u), Sec. 2.1.1): from lam = dJ/df^ [nv][ny][nx] writes
 * dJ/drho, dJ/dux, dJ/duy [ny][nx] (any may be NULL).
 */
int dugks_adjoint_equilibrium(dugks_ctx* ctx, const double* rho, const double* ux,
                              const double* uy, const double* lam, double* drho, double* dux,
                              double* duy, int on_device);

/*
 * dugks_step_static -- advance nsteps T3S3 steps without allocating any device
 * memory.  It takes the same T3S3 step (Sec. 2.1.3) on the generic FP64
 * kernels and matches dugks_step to the FP64 parity tolerance (for D2Q9 sets
 * dugks_step runs the fused kernels, which agree to about 1e-12, not bit for
 * bit); there is no context, so a storage form or time scheme does not apply.
 * The paper has no counterpart: this
 * is a facility for callers that may not allocate device memory, such as a
 * plugin inside an application that owns all device memory through its own
 * pool, or a latency-critical loop that cannot accept the implicit device
 * synchronisation of cudaMalloc/cudaFree.
 *   mesh, vel, tau, dt, bc : as for dugks_init (host structures, read during
 *                  the call).
 *   fhat_in      : device pointer, f^ [nv][ny][nx] at t_n (not modified
 *                  unless it equals fhat_out).
 *   fhat_out     : device pointer, receives f^ after nsteps (may equal
 *                  fhat_in for an in-place update).
 *   nsteps       : >= 0.
 *   cuda_stream  : cudaStream_t for every copy and launch (NULL = legacy
 *                  default stream); the call is asynchronous on it.
 * All intermediates live in one fixed 32 MiB device array inside the
 * library (held on every GPU that loads the library until the process
 * exits).  A problem needing more than 32 MiB of intermediates (about
 * 5 * nv * nx * ny doubles, e.g. more than a 256^2 D2Q9 grid) is rejected
 * with DUGKS_EINVAL and a message giving the size.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make it before any stream capture.  Every call
 * uploads the velocity tables from call-local host memory, so a call made
 * while cuda_stream is capturing a CUDA graph is refused with DUGKS_EINVAL.
 * fhat_in and fhat_out must be the same array or not overlap at all
 * (DUGKS_EINVAL otherwise).  Calls share the array and it keeps the last
 * call's contents (nothing needs to start at zero); calls that overlap on the
 * GPU race on it and must be serialised.
 * Errors: EINVAL, ECUDA (message in dugks_last_error).
 */
int dugks_step_static(const dugks_mesh* mesh, const dugks_velset* vel, double tau, double dt,
                      const dugks_bc bc[4], const double* fhat_in, double* fhat_out,
                      int nsteps, void* cuda_stream);

/* Time schemes.  DUGKS_T3S3 (default) is the paper's two-stage third-order
 * step (Sec. 2.1.3).  DUGKS_T2S3 and DUGKS_T2S2 are the second-order
 * comparison methods of Sec. 3 (Remark I, eq. feqIntD2nd_Explicit):
 * f~^{n+1} = f~^{+,n} + dt L(t_n + dt/2) on f~ = f - dt/2 Omega, with the
 * face values at t_n + dt/2 from the quadratic upwind expansion of eq.
 * flux_DS (T2S3) or that expansion truncated after the gradient term (T2S2;
 * the paper does not print its reconstruction, this is the reading used). */
enum { DUGKS_T3S3 = 0, DUGKS_T2S3 = 1, DUGKS_T2S2 = 2 };

/* dugks_set_scheme -- select the time scheme of later dugks_step calls.
 *   scheme: DUGKS_T3S3, DUGKS_T2S3 or DUGKS_T2S2.
 * The state is not converted: under a T2 scheme the array that
 * dugks_set_state / dugks_get_state move (and that dugks_set_equilibrium
 * fills) is f~ = f - dt/2 Omega instead of f^ = f - dt/4 Omega; at
 * equilibrium both equal feq.  The T2 schemes run on the generic kernels
 * with DUGKS_FP64 storage (other storage: DUGKS_ENOTIMPL); the adjoint
 * entry points are those of T3S3 and return DUGKS_ENOTIMPL under a T2
 * scheme.  A context that belongs to a batch cannot change scheme.
 * Errors: EINVAL (unknown scheme, NULL, batched context), ENOTIMPL. */
int dugks_set_scheme(dugks_ctx* ctx, int scheme);

/*
 * dugks_alu_peak -- arithmetic-throughput microbenchmark.  The paper has no
 * counterpart: it measures the denominator of the ALU roofline that bounds
 * the FP64 form of the step.  One launch of SMs x blocks_per_sm blocks of
 * 256 threads; every thread runs 8 independent fused multiply-add chains
 * for iters x 16 rounds.  kind: 0 FP64 (DFMA), 1 FP32 (FFMA), 2 packed FP32
 * pairs (fma.rn.f32x2, two FMAs per instruction).
 *   out, out_len : device buffer of out_len >= SMs x blocks_per_sm x 256
 *                  doubles; receives the chains' final values.
 *   flops, ms    : host outputs: the launch's flops (an FMA counts 2) and
 *                  its device time from CUDA events on cuda_stream.
 * Waits for cuda_stream.  Errors: EINVAL (bad kind, iters < 1,
 * blocks_per_sm outside 1..32, short buffer), ECUDA.
 */
int dugks_alu_peak(int kind, int iters, int blocks_per_sm, double* out, long long out_len,
                   double* flops, float* ms, void* cuda_stream);

/* dugks_destroy -- free the context (NULL is accepted). */
int dugks_destroy(dugks_ctx* ctx);

/* dugks_last_error -- message of the last error or warning on this thread. */
const char* dugks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DUGKS_H */
