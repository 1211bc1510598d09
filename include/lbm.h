/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the well-balanced
 * phase-field lattice Boltzmann model of incompressible binary fluids
 * (Ju, Liu, Yan, Bao, Sun, Guo; arXiv:2311.10827).
 *
 * Naming.  As in the paper, f is the Cahn-Hilliard (CH) population
 * (Eq. BGK; velocity-free equilibrium Eq. H_i, convection source Eq. F_i)
 * and g the hydrodynamic population (Eq. BGK-NS; equilibrium Eq. G_i,
 * force Eq. GGi).  Some texts swap the letters; this library does not.
 *
 * One time step (Section 2.3) advances both populations:
 *   phi = sum_i f_i; mu = psi'(phi) - kappa lap(phi) (Eq. chemical_potencial);
 *   grad(phi), grad(mu) with the isotropic stencil (Eq. gradient), lap with
 *   Eq. Laplace; rho, nu linear in phi (Eq. vis); F = -phi grad(mu) + G;
 *   rho u = sum c_i g_i + F/2; p from the moment below Eq. GGi;
 *   S = u.grad(phi); f_i* = f_i - (f_i - f_i^eq)/tau_f + w_i b_i (1.5 S - 0.5 S_prev);
 *   g_i* = g_i - (g_i - g_i^eq)/tau_g + G_i; then periodic streaming.
 * The (1/2) dt^2 d_t F_i term of Eq. BGK is read as a backward difference in
 * time, which is why S of the previous step is part of the state.
 *
 * Conventions.
 *  - Every function returns LBM_OK (0) or a negative LBM_ERR_* code; no C++
 *    exception crosses this boundary.
 *  - An error that the device reports asynchronously (a non-finite value
 *    seen by the diagnostics, a CUDA fault) is recorded in the context and
 *    returned by the next call that can fail, then cleared ("sticky until
 *    read").  A CUDA error leaves the context unusable: destroy it.
 *  - Pointers passed in are never retained.  Host arrays are caller-owned
 *    and only read or written during the call.  Device arrays passed with
 *    on_device = 1 must be device memory of the context's GPU and must stay
 *    valid until the context's stream has passed the call.
 *  - Field layout: scalar fields are [nz][ny][nx] (x fastest), node index
 *    n = (z*ny + y)*nx + x, N = nx*ny*nz.  Vector fields are [D][N].
 *    Populations are [Q][N].  All boundaries are periodic (Section 3).
 *  - Lattice units: dx = dt = 1, cs^2 = 1/3.
 *  - The context owns all its device memory (allocated by lbm_create, freed
 *    by lbm_destroy).  Work is issued on the CUDA stream given to
 *    lbm_create (NULL = the legacy default stream).
 */
#ifndef WB_LBM_H
#define WB_LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define LBM_OK               0
#define LBM_ERR_INVALID_ARG (-1) /* bad pointer, size, parameter or call order */
#define LBM_ERR_OOM         (-2) /* device or host allocation failed */
#define LBM_ERR_CUDA        (-3) /* a CUDA runtime call failed (no GPU, fault) */
#define LBM_ERR_NONFINITE   (-4) /* the diagnostics saw NaN/Inf in the fields */
#define LBM_ERR_TIMEOUT     (-5) /* a bounded device wait gave up */
#define LBM_ERR_STATE       (-6) /* context not initialised (lbm_init_phi first) */

/* Grid: nz = 1 for D2Q9.  Every boundary is periodic. */
typedef struct {
    int nx, ny, nz;
} lbm_grid;

/* Lattices: D2Q9 for both populations (Eq. eq:ci, weights below Eq. H_iyang);
 * D3Q19 (not in the paper) with the same equilibria, sources and stencils. */
typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_lattice;

/* Precision of storage and arithmetic.  LBM_FP64: FP64 throughout (parity
 * form).  LBM_FP32: FP32 populations and arithmetic, the rest population of
 * f kept as a compensated pair of FP32 words (its per-step change near
 * equilibrium is below half an FP32 ulp of phi), and the f populations
 * stored minus a uniform equilibrium shift w_i alpha mu_ref (the rest one
 * plus (1 - w_0) alpha mu_ref): a uniform shift of mu in Eq. H_i changes no
 * moment the step uses, so it is exact, and with mu_ref near the equilibrium
 * chemical potential the small per-step changes of the moving populations
 * are not lost to FP32 rounding; lbm_diagnostics re-centres mu_ref to the
 * middle of the current mu range.  Diagnostics in FP64.
 * LBM_FP32_F16OFF / LBM_FP32_BF16OFF (D3Q19 only): FP32 arithmetic with every
 * population stored as a 16-bit (FP16 / BF16) offset from its equilibrium
 * (Eq. H_i for f, the g^eq of Eq. G_i for g), evaluated at FP32 macroscopic
 * fields (phi, mu, p, u) stored with the state; each population field has a
 * power-of-two scale, refreshed from the largest offset whenever diagnostics
 * run.  The rest population keeps phi's rounding residual in its offset (the
 * compensated pair of LBM_FP32).  Not a form of the paper: a storage format
 * that cuts the bytes moved per node update. */
typedef enum {
    LBM_FP64 = 0,
    LBM_FP32 = 1,
    LBM_FP32_F16OFF = 2,
    LBM_FP32_BF16OFF = 3
} lbm_precision;

/* The paper's statement of the problem (Section 2 and Section 3):
 *   W      interface thickness (Eq. beta)
 *   M      mobility M_phi (Eq. CH_equation, Eq. mobility)
 *   alpha  the adjustable CH equilibrium parameter (Eq. H_i)
 *   sigma  surface tension (Eq. suiface_tension); kappa and beta follow:
 *          kappa = 3 W sigma / (2 dphi^2), beta = 12 sigma / (W dphi^4)
 *   phi_l, phi_v   bulk order parameters (default 1 and 0)
 *   rho_l, rho_v   bulk densities; rho is linear in phi
 *   nu_l, nu_v     bulk kinematic viscosities; nu is linear in phi (Eq. vis),
 *                  tau_g = 1/2 + nu / cs^2 node by node
 *   body_force     G in F = F_s + G (text after Eq. GGi)
 *   tau_f  0: derive tau_f = 1/2 + M / (cs^2 alpha) (Eq. mobility);
 *          > 1/2: use it and derive alpha = M / (cs^2 (tau_f - 1/2))
 *   precision      an lbm_precision value
 *   diag_every     0: no automatic diagnostics; k > 0: lbm_step fuses the
 *                  diagnostics reduction into every k-th step and records a
 *                  non-finite value as LBM_ERR_NONFINITE */
typedef struct {
    double W, M, alpha, sigma;
    double phi_l, phi_v;
    double rho_l, rho_v, nu_l, nu_v;
    double body_force[3];
    double tau_f;
    int precision;
    int diag_every;
} lbm_params;

/* Diagnostics of the state at time `step` (all sums in FP64):
 *   sum_phi         sum over nodes of phi
 *   kinetic_energy  E = 1/2 sum rho |u|^2 (the paper's E, Section 3.1)
 *   u_max           max |u| (spurious velocity in the equilibrium tests)
 *   mu_min, mu_max  range of the chemical potential
 *   budget          sum of (1.5 S - 0.5 S_prev): the exact change of the
 *                   phi sum over the next step is -budget, because
 *                   sum_i f_i^eq = phi and sum_i F_i = -S (Eq. sumfeqandF)
 *   nonfinite       1 if any node had a NaN/Inf field value */
typedef struct {
    double sum_phi, kinetic_energy, u_max, mu_min, mu_max, budget;
    long long step;
    int nonfinite;
} lbm_diag;

typedef struct lbm_ctx lbm_ctx;

/* Fill *out with the paper's defaults (W 4, M 0.1, alpha 1, sigma 1e-3,
 * phi_l 1, phi_v 0, rho_l 10, rho_v 1, nu_l = nu_v = 0.1, no body force,
 * tau_f derived, FP32, no automatic diagnostics).  Errors: INVALID_ARG if
 * out is NULL. */
int lbm_params_default(lbm_params *out);

/* Validate the problem, derive kappa, beta and tau_f (Eqs. beta,
 * suiface_tension, mobility) and allocate the device state (double-buffered
 * f and g, S_prev, work buffers) on the current CUDA device.  `cuda_stream`
 * is a cudaStream_t (NULL = legacy default stream) on which all later work is
 * issued.  Errors: INVALID_ARG (NULL pointers, non-positive sizes, nz != 1
 * for D2Q9, W <= 0, sigma < 0, M <= 0 or alpha <= 0 when tau_f is derived,
 * tau_f <= 1/2, phi_l == phi_v, rho <= 0, nu <= 0, unknown precision, an
 * offset precision with D2Q9),
 * OOM, CUDA (no usable GPU).  Validation happens before any CUDA call, so a
 * host without a GPU reports INVALID_ARG for a bad problem. */
int lbm_create(const lbm_grid *grid, int lattice, const lbm_params *params,
               void *cuda_stream, lbm_ctx **out);

/* Byte sizes of the device state of a problem: out[0] one f buffer, out[1]
 * one g buffer, out[2] S_prev (the state is double-buffered: two f and two g
 * buffers).  For callers that supply the state memory themselves
 * (lbm_create_with_buffers).  Errors: INVALID_ARG (NULL out, or a problem
 * lbm_create rejects); no CUDA call is made. */
int lbm_state_bytes(const lbm_grid *grid, int lattice, const lbm_params *params, size_t out[3]);

/* As lbm_create, but the state lives in memory the caller owns -- for example
 * device tensors of a framework that manages its own pool, so that the
 * framework accounts for the populations, which are nearly all of the
 * footprint.  buffers = {f buffer 0, f buffer 1, g buffer 0, g buffer 1,
 * S_prev}, device pointers on the current device of at least the sizes
 * lbm_state_bytes reports (out[0] for the f buffers, out[1] for g, out[2]
 * for S_prev), each 256-byte aligned.  They are used in place, never freed
 * by the library, and must stay valid until lbm_destroy; lbm_save's payload
 * is their contents.  The small work buffers are still allocated here.
 * Errors: as lbm_create, and INVALID_ARG for a NULL or misaligned buffer. */
int lbm_create_with_buffers(const lbm_grid *grid, int lattice, const lbm_params *params,
                            void *cuda_stream, void *const buffers[5], lbm_ctx **out);

/* Set the initial condition from an order-parameter field phi[N] (FP64):
 * f = f^eq(phi, mu(phi)) (Eq. H_i), g = 0 (p = 0, u = 0), S_prev = 0, time 0.
 * on_device = 0: host array (uploaded through the context's own state
 * buffers, no allocation; the call returns once it is read);
 * on_device = 1: device array.  Errors: INVALID_ARG, CUDA. */
int lbm_init_phi(lbm_ctx *ctx, const double *phi, int on_device);

/* Advance n >= 0 time steps, asynchronously on the context's stream (one
 * fused stream-collide kernel per step; a CUDA graph for long runs).
 * Returns a recorded error, if any.  Errors: STATE, INVALID_ARG, CUDA,
 * NONFINITE (recorded by an earlier fused diagnostics step). */
int lbm_step(lbm_ctx *ctx, int n);

/* Macroscopic fields at the current time (FP64 outputs): phi[N], p[N]
 * (hydrodynamic pressure), u[D*N] ([D][N]), mu[N].  Any output may be NULL.
 * on_device = 0: host arrays (the call synchronises the stream); when every
 * given array is pinned host memory (cudaHostAlloc, cudaHostRegister), the
 * pass writes them directly through their device addresses, else it writes
 * a device staging buffer (allocated on the first such call) and copies;
 * on_device = 1: device arrays (asynchronous).  Errors: STATE, CUDA. */
int lbm_moments(lbm_ctx *ctx, double *phi, double *p, double *u, double *mu,
                int on_device);

/* Diagnostics of the current state (synchronises).  For LBM_FP32 it also
 * re-centres the equilibrium shift of the storage (applied by the next step;
 * not while an adjoint recorder is attached), and for the offset precisions
 * it refreshes the scales.  Errors: STATE, CUDA, INVALID_ARG.  A non-finite
 * field is reported through out->nonfinite (the call itself still returns
 * LBM_OK). */
int lbm_diagnostics(lbm_ctx *ctx, lbm_diag *out);

/* Diagnostics recorded by the most recent fused diagnostics step of
 * lbm_step (diag_every > 0), describing the state at out->step.  Synchronises.
 * Errors: STATE if none was recorded yet, CUDA. */
int lbm_last_diagnostics(lbm_ctx *ctx, lbm_diag *out);

/* Allocation-free diagnostics (the paper has no counterpart: this is a
 * deployment variant of lbm_diagnostics).  For callers that cannot call
 * cudaMalloc -- code confined to a host framework's memory pool or a
 * pre-sized arena, or running where the device allocator must not be
 * touched -- and so can neither create a context nor let the reduction
 * allocate its scratch.  It runs the same diagnostics pass and reduction as
 * lbm_diagnostics; the per-CTA partial records live in a fixed file-scope
 * device array of 4096 records (256 KiB) that every GPU which loads the
 * library holds until the process exits.  It calls no cudaMalloc, cudaFree
 * or allocating library routine.
 *   grid, lattice, params: the problem as for lbm_create (D2Q9 only).
 *   f, g: device arrays in the library's storage layout at
 *     params->precision (the layout of the population payload written by
 *     lbm_save: the paper's f_i(x,t) stored at node x - c_i): g is [Q][N];
 *     f is [Q][N] in FP64 and [Q+1][N] in FP32 (the last array holds the
 *     low word of the rest population; FP32 f may carry any uniform
 *     equilibrium shift, which the diagnostics do not see); S_prev: device array [N]
 *     (u.grad(phi) of the previous step).  Read only.
 *   out: device array of 8 doubles, written asynchronously:
 *     {sum phi, E, max |u|^2, mu_min, mu_max, budget, nonfinite (1 or 0), 0}.
 *   cuda_stream: stream of the two launches (NULL = legacy default stream).
 * The first call on a device looks up the array's device address on that
 * device (with it current); make that first call before any stream capture.
 * Every call shares the one array and it keeps the last call's contents
 * (each record is rewritten before it is read, so nothing needs clearing):
 * calls that overlap on the GPU, on any stream, race and give wrong results.
 * Errors: INVALID_ARG (NULL pointer, bad problem, or a grid whose pass needs
 * more than 4096 CTAs, about 134 million nodes), CUDA. */
int lbm_diagnostics_noalloc(const lbm_grid *grid, int lattice, const lbm_params *params,
                            const void *f, const void *g, const void *S_prev, double *out,
                            void *cuda_stream);

/* Exchange the full state in the paper's convention, FP64: f[Q*N], g[Q*N]
 * hold f_i(x,t), g_i(x,t) (after streaming, before collision) and
 * S_prev[N] holds u.grad(phi) of step t-1.  lbm_set_state also sets the
 * time to `step` and marks the context initialised.  on_device selects host
 * (synchronous) or device (asynchronous) arrays.  Errors: STATE (get before
 * init), INVALID_ARG, CUDA. */
int lbm_get_state(lbm_ctx *ctx, double *f, double *g, double *S_prev, int on_device);
int lbm_set_state(lbm_ctx *ctx, const double *f, const double *g,
                  const double *S_prev, long long step, int on_device);

/* Checkpoint to / restore from a host buffer in the library's own format
 * (header, which also records the FP32 equilibrium shift, then the raw
 * device state at the context's precision: f, g, S_prev in the storage
 * layout described at lbm_diagnostics_noalloc; for the offset precisions f
 * is the Q offset arrays (u16), then D + 4 FP32 arrays (the macros phi, mu,
 * p, u and the offset-free part of the next step's phi sum), then the two
 * FP32 scales, each part padded to 256 bytes, and g is the Q offset arrays;
 * a restore is bit-exact).  lbm_save with buf == NULL stores the required
 * size in *bytes.  lbm_load checks that grid, lattice and precision match.
 * Errors:
 * INVALID_ARG (size or header mismatch), STATE, CUDA. */
int lbm_save(lbm_ctx *ctx, void *buf, size_t *bytes);
int lbm_load(lbm_ctx *ctx, const void *buf, size_t bytes);

/* Wait for the context's stream; returns a recorded error, if any. */
int lbm_sync(lbm_ctx *ctx);

/* Current time step (number of steps taken since the initial condition). */
long long lbm_time(const lbm_ctx *ctx);

/* kappa, beta, tau_f and alpha actually used.  Errors: INVALID_ARG. */
int lbm_derived(const lbm_ctx *ctx, double out[4]);

/* Host-side fault injection for tests: write `value` into population f
 * (field 0) or g (field 1), direction i, node n of the current state.
 * Errors: STATE, INVALID_ARG, CUDA. */
int lbm_debug_poke(lbm_ctx *ctx, int field, int i, long long n, double value);

/* ---------------------------------------------------------------------------
 * Batched ensemble (not in the paper: a throughput form of the same step).
 * Many independent periodic D2Q9 grids, each with its own size and problem
 * parameters (all at one precision), advance together: every time step is a
 * single kernel launch over a flat table of tiles that covers all grids, long
 * runs replay a CUDA graph of such launches (or run as one cooperative launch
 * per call: lbm_batch_set_persistent), and the tile shape (strip width
 * 64 or 128 columns, rows per tile) is chosen by an autotuner that times
 * candidate shapes on the batch's own state.  Each grid is also an ordinary
 * context (lbm_batch_case) for initialisation, moments, diagnostics, state
 * exchange and checkpoints; those calls act on that grid only.
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* Create ncases contexts (grids[c], params[c]; lattice D2Q9; every
 * params[c].precision equal; params[c].diag_every is ignored by batch steps)
 * on the current device, issuing work on cuda_stream.  Errors: INVALID_ARG
 * (ncases < 1, NULL arrays, a grid or parameter set that lbm_create rejects,
 * mixed precisions), OOM, CUDA. */
int lbm_batch_create(int ncases, const lbm_grid *grids, const lbm_params *params,
                     void *cuda_stream, lbm_batch **out);

/* The context of grid c (owned by the batch; do not destroy it).  Stepping it
 * with lbm_step desynchronises it from the batch: lbm_batch_step then returns
 * LBM_ERR_STATE until every grid is re-initialised.  Errors: INVALID_ARG. */
int lbm_batch_case(lbm_batch *b, int c, lbm_ctx **ctx);

/* Advance every grid by n >= 0 steps (asynchronous).  All grids must be
 * initialised and at the same time step.  The first call runs the autotuner
 * unless lbm_batch_tune was called.  With diagnostics on
 * (lbm_batch_set_diag_every), the steps whose starting time is a multiple of
 * the cadence carry them.  Errors: STATE, INVALID_ARG, CUDA; TIMEOUT after a
 * multi-step launch gave up waiting (returned by every later call until
 * lbm_batch_set_shape or lbm_batch_tune rebuilds the tiles); NONFINITE (once)
 * when the last diagnostics saw NaN/Inf in a grid. */
int lbm_batch_step(lbm_batch *b, int n);

/* Fused diagnostics of every grid (a10): with k > 0, every batch step that
 * starts at a time t that is a multiple of k also computes the FP64
 * diagnostics of each grid's state at t (as lbm_step does with
 * params.diag_every) from the same pass: one partial record per tile, a
 * per-grid reduction on the device in a fixed order, and the records written
 * to pinned host memory with no host synchronisation.  FP32 grids then move
 * their equilibrium shift to the middle of the mu range, as lbm_diagnostics
 * does (taking effect with the next launch).  k = 0 turns them off (the
 * default).  The records are read with lbm_batch_last_diagnostics.  Errors:
 * INVALID_ARG (NULL, k < 0). */
int lbm_batch_set_diag_every(lbm_batch *b, int k);

/* The records of the most recent fused diagnostics step, one per grid
 * (out[ncases]; out[c].step = that step's time).  Waits for that step only.
 * Errors: INVALID_ARG, STATE (no diagnostics step has run), CUDA. */
int lbm_batch_last_diagnostics(lbm_batch *b, lbm_diag *out);

/* Wait for all work issued on the batch's stream; returns a pending error
 * (TIMEOUT, NONFINITE) as lbm_batch_step does.  Errors: INVALID_ARG, CUDA. */
int lbm_batch_sync(lbm_batch *b);

/* Time every candidate tile shape on the current state and keep the
 * fastest; report it in *width and *rows (either may be NULL).  With
 * per-step launches the candidates are single steps that write only to
 * scratch.  With multi-step launches on (lbm_batch_set_persistent) they are
 * multi-step launches of the grids' own state: the current population
 * buffers, S, the FP32 equilibrium shifts, the step count and parity are
 * copied to a temporary device buffer of the state's size first and put
 * back after, so the state is left unchanged either way.  Synchronises.
 * Errors: STATE (a grid not initialised), OOM (the temporary buffer), CUDA,
 * TIMEOUT (a multi-step candidate's wait gave up). */
int lbm_batch_tune(lbm_batch *b, int *width, int *rows);

/* Current tile shape and number of tiles (CTAs per step). */
int lbm_batch_shape(const lbm_batch *b, int *width, int *rows, int *ntiles);

/* Use tile shape (width 64 or 128, rows >= 2) without tuning; later
 * lbm_batch_step calls do not tune.  Errors: INVALID_ARG, OOM, CUDA. */
int lbm_batch_set_shape(lbm_batch *b, int width, int rows);

/* Multi-step launches.  With on = 1, an lbm_batch_step call of n >= 2 steps
 * runs as one cooperative launch (split where needed so that each launch
 * carries at most one diagnostics step).  The launch holds every resident
 * CTA slot of the GPU and works through a queue of (step, tile) pairs in
 * order: before a tile's next step, its CTA waits only until the tile and
 * the tiles its stencil reaches (3 nodes) have finished the previous step,
 * each of them publishing a per-tile step counter.  There is no grid-wide
 * barrier and no launch per step, any number of tiles fits (a batch of many
 * grids walks its tile list every step), and tiles of the next step start
 * while the last ones of a step still run.  The results are the same, bit
 * for bit, as those of per-step launches, except after a fused diagnostics
 * step that moves the FP32 equilibrium shift inside a launch (the launch
 * writes with the new shift from its next launch on, per-step launches from
 * the next step on; the two differ by rounding).  A launch holds at most
 * 1024 steps (longer calls are split).  A wait is bounded (about 2 s of
 * SM clock).  On a timeout the tile sets an error word, fills its region of
 * the rest population (both buffers) and of S with NaN (so that diagnostics
 * report non-finite fields) and stops; the launch then ends, lbm_batch_step
 * returns LBM_ERR_TIMEOUT from then on, and lbm_batch_persistent reports it.
 * FP32 batches whose grids all have rows of a multiple of 4 nodes run a
 * variant that stages each tile's pulls as 16-byte row-segment copies one
 * iteration ahead (read from L2 only).  Tunes first if the batch is untuned
 * (timing multi-step launches as lbm_batch_tune does, when every grid is
 * initialised; else timing single steps).  on = 0 returns to per-step
 * launches (CUDA-graph replay).  Single-step calls always launch once per
 * step.  Errors: INVALID_ARG (NULL, or on = 1 with a shape whose tiles have
 * more than 16 neighbour tiles), OOM, CUDA. */
int lbm_batch_set_persistent(lbm_batch *b, int on);

/* *on (optional): whether multi-step launches are in use.  *timed_out
 * (optional): whether a multi-step launch has timed out waiting for a
 * neighbour tile since the tiles were last built.  Reading timed_out
 * synchronises the device.
 * Errors: INVALID_ARG, CUDA. */
int lbm_batch_persistent(const lbm_batch *b, int *on, int *timed_out);

/* Fault injection for tests of the multi-step launch's bounded waits: make
 * tile `tile` of the current shape wait, before every step after the first,
 * on a counter that nothing sets.  The next multi-step launch then takes
 * about 2 s to end.  The stalled tile gives up after its limit and sets the
 * error word that lbm_batch_persistent reports.  The tiles waiting on it,
 * directly or through others, see the error word and stop.  The state is
 * left with NaN in the stalled tile's rest population and S.  The injection
 * lasts until the tiles are rebuilt (lbm_batch_set_shape, lbm_batch_tune).
 * Errors: INVALID_ARG (NULL, tile out of range, multi-step launches not in
 * use), CUDA. */
int lbm_batch_debug_stall(lbm_batch *b, int tile);

/* Release the batch and all its contexts (synchronises first).  NULL-safe. */
void lbm_batch_destroy(lbm_batch *b);

/* ---------------------------------------------------------------------------
 * Discrete adjoint (not in the paper: the gradient of the discrete map).
 * For a D2Q9 context, records a run from an initial field phi0 with a
 * checkpoint of the state every `checkpoint_every` steps (device memory),
 * then, given dL/dphi of the final state, returns dL/dphi0 and the gradients
 * with respect to the surface tension and the mobility.  Segments between
 * checkpoints are recomputed forward on the backward pass; the reverse step
 * runs at the context's precision (FP64 adjoint fields and arithmetic for an
 * FP64 context, FP32 for an FP32 one); parameter gradients accumulate in
 * FP64.
 * ------------------------------------------------------------------------- */
typedef struct lbm_adjoint lbm_adjoint;

/* Attach an adjoint recorder to ctx (D2Q9) for runs of at most max_steps
 * steps; allocates max_steps / checkpoint_every + 1 checkpoints and one
 * segment of checkpoint_every states, each with its moments (phi, mu, p, u:
 * 5 values per node).  Errors: INVALID_ARG (D3Q19 context,
 * checkpoint_every < 1, max_steps < 1), OOM, CUDA. */
int lbm_adjoint_create(lbm_ctx *ctx, int checkpoint_every, int max_steps, lbm_adjoint **out);

/* lbm_init_phi(phi0) then nsteps (<= max_steps) steps of the context, keeping
 * the checkpoints.  phi0 is FP64 [N], host (on_device = 0) or device.
 * Errors: INVALID_ARG, CUDA. */
int lbm_adjoint_forward(lbm_adjoint *a, const double *phi0, int on_device, int nsteps);

/* Given dL_dphi [N] (FP64, gradient of the loss with respect to the final
 * order parameter; host or device per on_device), compute dL/dphi0 into
 * dL_dphi0 [N] (same residence) and grads[4] (host) = {dL/dsigma, dL/dM,
 * dL/dkappa, dL/dbeta} (sigma acts through kappa and beta, M through tau_f
 * at fixed alpha).  The context is left at the final state.  Synchronises.
 * Errors: STATE (no recorded run), INVALID_ARG, CUDA. */
int lbm_adjoint_backward(lbm_adjoint *a, const double *dL_dphi, int on_device, double *dL_dphi0,
                         double grads[4]);

/* Release the recorder (not the context).  NULL-safe. */
void lbm_adjoint_destroy(lbm_adjoint *a);

/* Release the context and its device memory (synchronises first).
 * NULL-safe. */
void lbm_destroy(lbm_ctx *ctx);

/* Static description of an error code. */
const char *lbm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* WB_LBM_H */
