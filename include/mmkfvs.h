/*
 * mmkfvs -- C ABI of the GB300 (sm_103a) implementation of one time step of the 2D-2V
 * micro-macro kinetic flux-vector-splitting scheme for the Boltzmann-ES-BGK equation
 * (Rossmanith & Sar, arXiv 2509.21832, Section 5, with the diffuse walls of Section 6.3).
 *
 * State held on the device by a context:
 *   Q[6][ny][nx]         conserved moments (rho, rho u1, rho u2, E11, E12, E22), Eq. (5-40),
 *                        cell averages on the cell-centred grid of Section 5.2.
 *   G[ny][nx][nv2][nv1]  micro part g on the phase-space grid of Section 5.2 (v1 fastest),
 *                        FP64, or FP32 when params.precision == MM_PREC_G_FP32.
 *   H[4][ny][nx]         heat-flux tensor (H111, H112, H122, H222) of the last step, Eq. (5-99).
 * Host-side arrays passed to this API are always FP64, row-major, in exactly these layouts; the
 * library copies them and keeps no host pointer.  Device pointers passed to the *_device entry
 * points must be FP64 device memory of the same layouts, owned by the caller.
 *
 * Errors: every function returns an mm_status and never aborts.  Non-physical states met on the
 * device (rho <= 0, P11 <= 0, P22 <= 0, det(P/rho) <= 0, det(Tcal) <= 0, non-finite values) are
 * latched in a device word and reported as MM_ERR_NONPHYSICAL by the next mm_sync / mm_get_*.
 * mm_last_error() gives a text for the last failure of a context.
 *
 * Threading: one context per CUDA stream; calls on one context are not thread-safe.  All work
 * of a context is ordered on the stream given at creation (NULL = legacy default stream);
 * mm_step_host also runs its copies and sweeps on streams of its own, which wait for that stream
 * before they start and are joined to it before the call returns.
 */
#ifndef MMKFVS_H
#define MMKFVS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MM_OK = 0,
  MM_ERR_INVALID_ARG = 1,  /* argument rejected before any device work */
  MM_ERR_OOM = 2,          /* device allocation failed */
  MM_ERR_CUDA = 3,         /* a CUDA call failed; see mm_last_error */
  MM_ERR_NONPHYSICAL = 4,  /* a non-physical state was met on the device */
  MM_ERR_TIMEOUT = 5,      /* a bounded device wait ran out */
  MM_ERR_STATE = 6         /* call out of order (e.g. mm_step before mm_set_state) */
} mm_status;

/* Boundary kinds; side order in mm_params.bc: 0 left (x=x0), 1 right (x=x1), 2 bottom (y=y0),
 * 3 top (y=y1).  Periodic sides must come in pairs.
 *   PERIODIC  Eqs. (2d_periodic_micro_1..5), (2d_periodic_macro_1/2)
 *   EXTRAP    Eqs. (2d_extrap_micro_1..5), (2d_extrap_macro_1..4)
 *   SPECULAR  mirror ghost cells (the paper names reflecting walls without printing the specular
 *             form); needs a velocity mesh symmetric about 0 in the wall-normal component
 *   DIFFUSE   Section 6.3 (Eqs. lid_driven_bc_1..4, twodim_wall_densities_1/2) */
enum { MM_BC_PERIODIC = 0, MM_BC_EXTRAP = 1, MM_BC_SPECULAR = 2, MM_BC_DIFFUSE = 3 };

/* Collision frequency tau (Section 2.4 remark, Eq. tau-for-2d-es-bgk; Sections 4 and 6.2):
 *   RHO          tau = tau0 * rho
 *   HARDSPHERE2D tau = 3 pi C25 rho / (sqrt(2) (1 - nu)), C25 = 0.436 (equals the printed
 *                (3 C25 pi / (2 sqrt 2)) rho at nu = -1)
 *   PRESSURE     tau = tau0 * rho * T
 *   CONST        tau = tau0 */
enum { MM_TAU_RHO = 0, MM_TAU_HARDSPHERE2D = 1, MM_TAU_PRESSURE = 2, MM_TAU_CONST = 3 };

/* Time-step rule for mm_dt_for_cfl: the min form of Eq. (CFL-2D-part1) or the sum form
 * dt = CFL / (V1/dx + V2/dy) that reproduces the step counts printed in Section 6.2. */
enum { MM_CFL_MIN = 0, MM_CFL_SUM = 1 };

/* Storage of g: FP64, or FP32 with the Gaussian tensor inverse, 1/T, the projector scale, the
 * heat-flux totals and the macro update in FP64, and g's transport, velocity sums and
 * relaxation in FP32 (the paper uses FP64 throughout; FP32 g is this library's mixed-precision
 * extension). */
enum { MM_PREC_FP64 = 0, MM_PREC_G_FP32 = 1 };  /* MM_PREC_G_FP32 needs nv1 <= 32 */

typedef struct {
  int nx, ny;                        /* spatial cells, >= 1 each (ny = 1: 1D-2V, y periodic) */
  double x0, x1, y0, y1;             /* spatial box */
  int nv1, nv2;                      /* velocity cells, 1..1024 each */
  double v1min, v1max, v2min, v2max; /* velocity box */
} mm_grid;

typedef struct {
  double nu;            /* ES-BGK parameter, -1 <= nu < 1 (Eq. mod-press-esbgk), Pr = 1/(1-nu) */
  int tau_model;        /* MM_TAU_* */
  double tau0;          /* scale of the tau model */
  int bc[4];            /* MM_BC_* per side */
  double wall_T[4];     /* diffuse wall temperature per side (> 0 where DIFFUSE) */
  double wall_U[4];     /* diffuse wall tangential velocity per side (lid speed) */
  int wall_keep_es_term;/* 1: wall-adjacent Ghat keeps (G - M)/eps; 0: literal Section 6.3 form */
  int precision;        /* MM_PREC_* */
} mm_params;

typedef struct mm_ctx mm_ctx;

/* Create a context and allocate its device state (owned by the context).  cuda_stream is a
 * cudaStream_t (NULL for the legacy default stream).  Validates the grid and parameters
 * (MM_ERR_INVALID_ARG), e.g. unpaired periodic sides, nu outside [-1, 1), a velocity mesh that is
 * not symmetric where a specular wall needs it, or (FP32 g) a velocity mesh whose fused kernel
 * would need more shared memory than a CTA can have (three rows of G* per warp). */
mm_status mm_create(const mm_grid* grid, const mm_params* params, void* cuda_stream,
                    mm_ctx** out);

/* Device bytes mm_create allocates for this problem (state, scratch and flags; the scratch
 * pieces counted rounded up to 256 bytes).  0 for an invalid grid or parameters. */
size_t mm_device_bytes(const mm_grid* grid, const mm_params* params);

/* Bytes of caller scratch that mm_create_borrowed needs for this problem: every device buffer of
 * a context except Q and G (split-step copy of g, macro scratch, heat flux, per-cell
 * coefficients, row sums, Maxwellian factors, error word, diffuse-wall cell list), each rounded
 * up to 256 bytes.  0 for an invalid grid or parameters. */
size_t mm_scratch_bytes(const mm_grid* grid, const mm_params* params);

/* Create a context on caller-owned device memory (e.g. the storage of framework tensors), which
 * must outlive the context and which the context never frees:
 *   Q_dev       [6][ny][nx] doubles, 16-byte aligned: the macro state, updated in place;
 *   G_dev       [ny][nx][nv2][nv1] elements of the context's precision (double, or float for
 *               MM_PREC_G_FP32), 256-byte aligned: g, which holds the state whenever mm_step or
 *               a setter returns (FP32 g alternates between G_dev and a scratch copy inside
 *               mm_step, which copies it back to G_dev at the end of the call when needed);
 *   scratch_dev scratch_bytes >= mm_scratch_bytes(grid, params), 256-byte aligned.
 * Optional features enabled later (learned closure, manufactured-solution harness, mm_step_host
 * streams) allocate their own buffers, owned and freed by the context.  MM_ERR_INVALID_ARG for an
 * invalid grid or parameters, a NULL or misaligned pointer or too little scratch. */
mm_status mm_create_borrowed(const mm_grid* grid, const mm_params* params, void* cuda_stream,
                             double* Q_dev, void* G_dev, void* scratch_dev, size_t scratch_bytes,
                             mm_ctx** out);

/* Copy the state in from host memory: Q_host [6][ny][nx], G_host [ny][nx][nv2][nv1] (NULL
 * means g = 0).  Synchronous with respect to the host buffers (they may be reused on return). */
mm_status mm_set_state(mm_ctx* ctx, const double* Q_host, const double* G_host);

/* Same from caller-owned FP64 device memory; asynchronous on the context stream. */
mm_status mm_set_state_device(mm_ctx* ctx, const double* Q_dev, const double* G_dev);

/* Set the state from host primitive fields rho, u1, u2, T, each [ny][nx], with an isotropic
 * temperature tensor and g = 0, as the paper's examples start (Section 6): Q = (rho, rho u1,
 * rho u2, E11, E12, E22) with the energy tensor E = rho (u (x) u + T I) of Section 2 (ES-BGK
 * operator), formed on the device as E11 = rho (u1 u1 + T), E12 = rho (u1 u2),
 * E22 = rho (u2 u2 + T), each operation rounded once in that order.  Synchronous with respect to
 * the host buffers.  MM_ERR_INVALID_ARG for a NULL field, rho or T not positive and finite, or u
 * not finite (the state is then unchanged). */
mm_status mm_set_state_prim(mm_ctx* ctx, const double* rho, const double* u1, const double* u2,
                            const double* T);

/* The caller changed g (in place, in the buffer of a context from mm_create_borrowed) in the
 * cells [i0, i1) x [j0, j1) -- the halo cells of a block of a spatially decomposed problem after
 * an exchange with its neighbours (Section 5.5 distributes the grid this way): the library
 * re-forms what it keeps derived from g there (the row sums of g that FP64 contexts with one row
 * per pass keep for the x sweep); nothing else is needed before the next mm_step.  Asynchronous
 * on the context stream, which must be ordered after the caller's writes.  MM_ERR_INVALID_ARG for
 * a region outside the grid. */
mm_status mm_g_region_changed(mm_ctx* ctx, int i0, int i1, int j0, int j1);

/* Advance nsteps time steps of size dt at Knudsen number eps (Section 5: micro x sweep, micro y
 * sweep, backward-Euler relaxation, heat-flux moments, then the Strang-split macro update).
 * Asynchronous on the context stream.  dt > 0, eps > 0, nsteps >= 0. */
mm_status mm_step(mm_ctx* ctx, double dt, double eps, int nsteps);

/* Wait for the context stream and report device-side errors (MM_ERR_NONPHYSICAL). */
mm_status mm_sync(mm_ctx* ctx);

/* Copy Q (and H unless H_host is NULL) to host memory; synchronises the stream. */
mm_status mm_get_moments(mm_ctx* ctx, double* Q_host, double* H_host);

/* One time step from host state to host moments: the result of
 * mm_set_state(c, Q_host, G_host); mm_step(c, dt, eps, 1); mm_get_moments(c, Q_out, H_out), with
 * the host-to-device copy of G_host overlapped with the step (equal to rounding, relative 1e-13:
 * the x sweep sums its velocity moments per velocity here, from row sums of g in mm_step, so the
 * two differ in the order of additions; bitwise where the velocity mesh has no row sums, i.e.
 * nv1 <= 16 or nv1 > 32).  For plain FP64 contexts g is
 * copied in row chunks on a second stream and the micro sweeps of each chunk start as soon as
 * its rows (and those of its upper neighbour) are on the device; FP32-g, learned-closure and
 * manufactured-solution contexts run the three calls in sequence.  Q_host [6][ny][nx] and
 * G_host [ny][nx][nv2][nv1] are read (page-locked memory lets the copies run asynchronously);
 * Q_out [6][ny][nx] and, if not NULL, H_out [4][ny][nx] receive Q^{n+1} and the heat flux.
 * Synchronous; the context's state afterwards is that of the step.  Errors: MM_ERR_INVALID_ARG
 * for NULL Q_host, G_host, Q_out or dt, eps not > 0; MM_ERR_NONPHYSICAL as mm_sync. */
mm_status mm_step_host(mm_ctx* c, const double* Q_host, const double* G_host, double dt,
                       double eps, double* Q_out, double* H_out);

/* Copy Q (and H unless NULL) to caller-owned FP64 device memory; asynchronous. */
mm_status mm_get_moments_device(mm_ctx* ctx, double* Q_dev, double* H_dev);

/* Copy G to host memory as FP64 [ny][nx][nv2][nv1]; synchronises the stream. */
mm_status mm_get_g(mm_ctx* ctx, double* G_host);

/* Global time step of Eq. (CFL-2D-part1/2) (form MM_CFL_MIN) or of the sum form
 * (MM_CFL_SUM); with ny == 1 the 1D rule of Section 3.2 (dt = CFL dx / V1).  If t_final > 0,
 * N = ceil(t_final/dt) and dt <- t_final/N (N written to *nsteps_out if not NULL).  Returns a
 * negative value for invalid arguments. */
double mm_dt_for_cfl(const mm_grid* grid, double cfl, double t_final, int form, int* nsteps_out);

/* Text of the last error of ctx ("" if none); valid until the next call on ctx. */
const char* mm_last_error(const mm_ctx* ctx);

/* Per-kernel timing with CUDA events recorded around each launch on the context stream.
 * mm_get_timing writes the accumulated milliseconds and launch counts of each kernel kind
 * (arrays of mm_num_kernels() entries) since timing was enabled; synchronises the stream. */
mm_status mm_set_timing(mm_ctx* ctx, int enable);
mm_status mm_get_timing(mm_ctx* ctx, double* ms_out, long long* launches_out);
int mm_num_kernels(void);
const char* mm_kernel_name(int idx);

/* Release the context and its device memory (NULL is accepted). */
void mm_destroy(mm_ctx* ctx);

/* ---- batches of independent problems --------------------------------------------------------
 * Many independent problems of uneven size and Knudsen number stepped together (FP64; nv1 <=
 * 256), the batched form that the paper's MPI design has no counterpart of.  Every call of
 * mm_batch_step is ONE launch of a persistent kernel for all of its steps: its CTAs take work
 * items -- (step, problem, phase of the step of Section 5, tile of cells) -- from a queue in a
 * fixed order and wait, before each item, until the phases it depends on are complete for the
 * same problem.  Every wait is bounded (2 s); one that runs out ends the launch and is reported by
 * mm_batch_sync as MM_ERR_TIMEOUT, with the device left usable.  The launch is captured in a CUDA
 * graph (with the reset of its queue) and replayed.  The tile sizes (cells per item) come from
 * mm_batch_autotune (timed trial steps on the batch's own state, cached per process by the
 * multiset of problem shapes).  Problem q's arrays have the single-problem layouts of this
 * header. */
typedef struct mm_batch mm_batch;
/* grids[nprob], params[nprob]: as for mm_create, each validated the same way.  cuda_stream NULL:
 * the batch creates its own non-blocking stream (graph capture needs a non-default stream). */
mm_status mm_batch_create(int nprob, const mm_grid* grids, const mm_params* params,
                          void* cuda_stream, mm_batch** out);
/* State of problem q from host memory (G_host NULL: g = 0); clears the device error word;
 * synchronous. */
mm_status mm_batch_set_state(mm_batch* b, int q, const double* Q_host, const double* G_host);
/* nsteps steps of every problem, problem q with time step dt[q] and Knudsen number eps[q]
 * (host arrays of nprob values); asynchronous. */
mm_status mm_batch_step(mm_batch* b, const double* dt, const double* eps, int nsteps);
/* Choose the tile sizes of the work queue (cells per item of the phase-space phases: 1, 2, 4 or
 * 8; of the per-cell phases: 1 or 4 CTAs' worth) by timing two-step trial launches on the batch's
 * own state, which is saved before and restored after (the state is not changed; the batch
 * temporarily holds a second copy of its g).  The CTA size (whole warps covering the widest v1
 * mesh) and the persistent grid (every resident CTA) are written to the optional outputs.  Call
 * after the first mm_batch_step (so that dt, eps are set). */
mm_status mm_batch_autotune(mm_batch* b, int* threads_out, int* ctas_out);
/* The current tile sizes: cells per item of the phase-space phases and of the per-cell ones. */
mm_status mm_batch_tiles(const mm_batch* b, int* micro_cells, int* macro_cells);
/* 1 (default): replay a captured CUDA graph of the launch; 0: launch the kernel directly. */
mm_status mm_batch_set_graph(mm_batch* b, int enable);
/* Diagnostic of the bounded waits: with 0 <= q and 0 <= phase < 8 the following steps do not
 * count the completed items of that phase of problem q (phases: 0 (u, T), 1 per-cell
 * coefficients, 2 micro x, 3 micro y, 4 diffuse walls, 5 macro x half fluxes, 6 macro x
 * transport, 7 macro y), so that the items that depend on it wait in vain and give up after
 * wait_ms milliseconds (0 < wait_ms <= 60000); q < 0 or phase < 0 switches this off (waits back
 * to 2 s).  The state is meaningless after such a step; mm_batch_set_state restores it and
 * clears the error word. */
mm_status mm_batch_diag_hold(mm_batch* b, int q, int phase, double wait_ms);
/* Wait and report device errors: MM_ERR_TIMEOUT after a wait ran out, MM_ERR_NONPHYSICAL after
 * a non-physical state. */
mm_status mm_batch_sync(mm_batch* b);
mm_status mm_batch_get_moments(mm_batch* b, int q, double* Q_host, double* H_host);
mm_status mm_batch_get_g(mm_batch* b, int q, double* G_host);
const char* mm_batch_last_error(const mm_batch* b);
void mm_batch_destroy(mm_batch* b);

/* ---- learned heat-flux closure ---------------------------------------------------------------
 * The paper has no learned closure; this is the library's extension.  An MLP with MM_MLP_IN
 * inputs, two GELU hidden layers of MM_MLP_HIDDEN and MM_MLP_OUT outputs, BF16 weights, FP32
 * accumulation, maps local macro features of a cell to y = (H - H_CE) / (eps rho T^{3/2}), the
 * dimensionless part of the heat-flux tensor of Eq. (5-99) beyond its Chapman-Enskog value H_CE
 * (the moments of the transport part of Ghat, Eq. 5-97).  Parameters are one flat FP32 vector of
 * MM_MLP_NPARAM values [W1 (64x39, row-major by output), b1, W2 (64x64), b2, W3 (4x64), b3];
 * the normalisation vector holds [input mean (39), input 1/std (39), output mean (4), output
 * std (4)].  Feature and target arrays are FP32 device arrays, sample-major [n][39], [n][4]. */
#define MM_MLP_IN 39
#define MM_MLP_HIDDEN 64
#define MM_MLP_OUT 4
#define MM_MLP_NPARAM 6980
typedef struct mm_mlp mm_mlp;
mm_status mm_mlp_create(void* cuda_stream, mm_mlp** out);
/* Load FP32 parameters (rounded to BF16 for the kernels) and normalisation; resets Adam. */
mm_status mm_mlp_set_params(mm_mlp* m, const float* params_host, const float* norm_host);
/* FP32 master parameters and/or the BF16 parameters the kernels use (as FP32 values). */
mm_status mm_mlp_get_params(mm_mlp* m, float* params_host, float* params_bf16_as_f32_host);
/* Inference: Y[n][4] (de-standardised) from X[n][39]; asynchronous. */
mm_status mm_mlp_forward(mm_mlp* m, const float* X_dev, float* Y_dev, int n);
/* Gradient of the mean squared error of the standardised outputs with respect to the
 * parameters, and the loss; synchronous if outputs given.  Forward and backward run on the tensor
 * cores (mma m16n8k16) with BF16 operands -- the BF16 weights, the standardised inputs, the
 * activations and the back-propagated pre-activation gradients, each rounded to BF16 where it
 * enters a product -- and FP32 accumulation; the weight gradients are summed over chunks of 128
 * samples in a fixed order (deterministic).  Work buffer: about 680 bytes per sample. */
mm_status mm_mlp_grad(mm_mlp* m, const float* X_dev, const float* T_dev, int n, float* grad_host,
                      float* loss_host);
/* One Adam step (beta 0.9, 0.999) on a mini-batch; FP32 master weights, BF16 copies refreshed. */
mm_status mm_mlp_train_step(mm_mlp* m, const float* X_dev, const float* T_dev, int n, float lr,
                            float* loss_host);
const char* mm_mlp_last_error(const mm_mlp* m);
void mm_mlp_destroy(mm_mlp* m);

/* Hybrid stepping with the closure (FP64 contexts).  While a network is set, every mm_step
 * computes per cell the features of Q^n, the network's y and the indicator max_m |y_m|; a cell
 * that touches no non-periodic boundary and whose indicator is <= threshold takes the closure:
 * H = H_CE + eps rho T^{3/2} y and no micro update; every other cell takes the full micro update.
 * g is maintained where the micro sweeps read it: before the sweeps, every cell in the 3x3 block
 * of a micro cell whose g^n was not produced by the previous step's micro update is reset to
 * Ghat(Q^n) (the asymptotic-preserving limit of Eq. 5-98); elsewhere g of closure cells is left
 * as it was (mm_get_g returns it as is).  The context keeps the pointer: the network must
 * outlive its use.  m = NULL switches the closure off; the next step then first resets every
 * non-current g to Ghat.  Resets the statistics.  FP32-g contexts: MM_ERR_INVALID_ARG. */
mm_status mm_set_closure(mm_ctx* c, const mm_mlp* m, double threshold);
/* Fallback of the hybrid step at low closure fractions (defaults: min_fraction 0.25, period
 * 16).  With a closure set, every period-th step (counted from mm_set_closure or from this call)
 * is a hybrid step whose number of closure cells is read back (mm_step waits for the device once
 * there); when it is below min_fraction of the cells, the period - 1 steps that follow are plain
 * steps (the full micro sweeps, the first one resetting the g of the closure cells to Ghat(Q^n)),
 * else hybrid steps.  The choice depends only on the computed counts, so runs are reproducible.
 * min_fraction 0 keeps every step hybrid; period 1 evaluates every step without reading back.
 * MM_ERR_INVALID_ARG outside 0 <= min_fraction <= 1, period >= 1. */
mm_status mm_set_closure_fallback(mm_ctx* c, double min_fraction, int period);
/* Hybrid steps and plain fallback steps run since mm_set_closure. */
mm_status mm_closure_steps(mm_ctx* c, long long* hybrid_steps, long long* plain_steps);
/* Features X_dev [nc][39] (FP32) of the current state and aux_dev [5][ny][nx] (FP64: H_CE of
 * the four components, then the scale eps rho T^{3/2}); asynchronous. */
mm_status mm_closure_features(mm_ctx* c, double dt, double eps, float* X_dev, double* aux_dev);
/* Training data: the features of Q^n into X_dev [nc][39], then one plain (full micro) step, then
 * the targets y = (H - H_CE) / (eps rho T^{3/2}) into Y_dev [nc][4]; asynchronous. */
mm_status mm_closure_collect(mm_ctx* c, double dt, double eps, float* X_dev, float* Y_dev);
/* Closure flags of the last hybrid step, [ny][nx] bytes (1 = closure). */
mm_status mm_closure_flags(mm_ctx* c, unsigned char* flags_host);
/* Closure cells summed over the hybrid steps since mm_set_closure, and cells x those steps. */
mm_status mm_closure_stats(mm_ctx* c, long long* closure_cells, long long* cell_steps);

/* ---- manufactured-solution harness ----------------------------------------------------------
 * The 2D-2V manufactured solution of the paper's convergence study (Section 6.1, Method of
 * Manufactured Solutions Example; Table tab5-4): f = phi(v) F(t, x, y) with
 * phi = exp(-|v - (1,1)|^2) + 2 exp(-|v + (1,1)|^2), F = 2 - sin(2 pi (t-x)) cos(2 pi (t-y)),
 * on doubly periodic FP64 contexts (other contexts: MM_ERR_INVALID_ARG).
 * mm_mms_enable: while enabled, each mm_step adds the residual S = f_t + v.grad f
 * - (tau/eps)(Gcal[f] - f) at t^n to Ghat as (1/tau^n)(I - Pi_M)[S] and to the macro update as
 * dt int (1, v, v (x) v) S dv between the y transport and the last collision half step
 * (Eq. macro2d-split3b); t^n starts at t0 and advances by dt per step.  Not combinable with the
 * closure (MM_ERR_STATE).  Allocates one more phase-space buffer.
 * mm_mms_set_exact: the state becomes the exact solution at time t (Q at cell centres,
 * g = (f - M[f])/eps at the nodes).
 * mm_mms_error: relative L2 errors of Q and g against the exact solution at time t (the norms
 * of Section 6.1); synchronous. */
mm_status mm_mms_enable(mm_ctx* c, int enable, double t0);
mm_status mm_mms_set_exact(mm_ctx* c, double t, double eps);
mm_status mm_mms_error(mm_ctx* c, double t, double eps, double* macro_err, double* micro_err);

/* ---- 1D-1V micro-macro scheme for Boltzmann-BGK (Sections 3 and 4) --------------------------
 * Q [3][nx] = (rho, rho u, E) with E = rho T / 2 + rho u^2 / 2 (Eq. 5-11), G [nx][nv] (FP64,
 * host arrays), H [nx] = (eps/2) dv sum_k v_k^3 G_k (Eq. 5-26).  One step: Ghat (Eq. 5-19), the
 * upwind Z and its projection (Eqs. 5-20, 5-24, 5-21), the update of Eq. (5-25), the heat flux,
 * then the KFVS macro update of Eq. (5-27) with the fluxes of Eq. (flux1d_1/2).  Boundaries:
 * MM_BC_PERIODIC (both sides) or MM_BC_EXTRAP (Eqs. 1d_extrap_micro_1/2, 1d_extrap_macro_1/2).
 * tau: MM1D_TAU_HARDSPHERE = (16/5) sqrt(T / (2 pi)) (Eq. collision_parameter_1d) or
 * MM1D_TAU_CONST = tau0.  1 <= nv <= 65536, nx >= 2; other arguments: MM_ERR_INVALID_ARG. */
#define MM1D_TAU_HARDSPHERE 0
#define MM1D_TAU_CONST 1
typedef struct {
  int nx;
  double x0, x1;
  int nv;
  double vmin, vmax;
} mm1d_grid;
typedef struct {
  int bc[2];
  int tau_model;
  double tau0;
} mm1d_params;
typedef struct mm1d_ctx mm1d_ctx;
mm_status mm1d_create(const mm1d_grid* grid, const mm1d_params* params, void* cuda_stream,
                      mm1d_ctx** out);
/* G_host NULL: g = 0.  Synchronous. */
mm_status mm1d_set_state(mm1d_ctx* c, const double* Q_host, const double* G_host);
/* Asynchronous; non-physical states are reported by mm1d_get_state. */
mm_status mm1d_step(mm1d_ctx* c, double dt, double eps, int nsteps);
/* Any of the outputs may be NULL; synchronous; MM_ERR_NONPHYSICAL after a bad state. */
mm_status mm1d_get_state(mm1d_ctx* c, double* Q_host, double* G_host, double* H_host);
/* The 1D manufactured solution of Section 4.1 (periodic contexts): while enabled, each step adds
 * (1/tau)(I - Pi_M)[S] at t^n to Ghat and dt pi^{3/2} cos(2 pi (x - t^n)) (-8, 11, -7) to the
 * macro update; t^n starts at t0.  mm1d_mms_set_exact sets the exact state at time t. */
mm_status mm1d_mms_enable(mm1d_ctx* c, int enable, double t0);
mm_status mm1d_mms_set_exact(mm1d_ctx* c, double t, double eps);
const char* mm1d_last_error(const mm1d_ctx* c);
void mm1d_destroy(mm1d_ctx* c);

/* Diagnostic: evaluate the table-driven exponential used by the phase-space kernels (Tang's
 * method, see the micro kernels) and the CUDA library exp on n FP64 device values x_dev, into
 * caller-owned device arrays; synchronises cuda_stream.  Used to test the kernels' exp against
 * the library exp. */
mm_status mm_diag_exp(const double* x_dev, double* y_fast_dev, double* y_lib_dev, size_t n,
                      void* cuda_stream);

/* Diagnostic: evaluate the error function used by the KFVS half fluxes (Section 5.4: a
 * polynomial on |x| < 1.5, the library erf elsewhere) and the CUDA library erf on n FP64 device
 * values x_dev, into caller-owned device arrays; synchronises cuda_stream.  Used to test the
 * fluxes' erf against the library erf.  MM_ERR_INVALID_ARG for a NULL array. */
mm_status mm_diag_erf(const double* x_dev, double* y_fast_dev, double* y_lib_dev, size_t n,
                      void* cuda_stream);

/* Diagnostic: the FP64 pipe's throughput.  Launches `ctas` CTAs of 256 threads on cuda_stream;
 * each thread runs `iters` rounds of 8 independent FP64 fused multiply-adds d <- a d + b
 * (a = 1 - 2^-20, b = 2^-30, d starting at 1 + lane/256) and writes the sum of its 8 chains to
 * out_dev[thread] (caller-owned, ctas * 256 doubles).  The launch performs
 * ctas * 256 * iters * 16 FP64 flops and is not synchronised, so that the caller can time it with
 * events on cuda_stream.  MM_ERR_INVALID_ARG for ctas < 1, iters < 1 or out_dev NULL. */
mm_status mm_diag_fp64_fma(double* out_dev, int ctas, int iters, void* cuda_stream);

/* Diagnostic of the bounded device waits (the FP32-g kernels wait on an mbarrier for their bulk
 * copies, each wait giving up after a fixed number of attempts and setting an error bit that
 * mm_sync reports as MM_ERR_TIMEOUT).  One warp arms an mbarrier for a 16-byte copy; with
 * copy != 0 it issues that copy, else nothing completes the barrier and the wait gives up after
 * `spins` attempts (1 <= spins).  Returns MM_OK when the wait completed, MM_ERR_TIMEOUT when it
 * ran out (the device stays usable), MM_ERR_INVALID_ARG for spins < 1; synchronises cuda_stream. */
mm_status mm_diag_bounded_wait(int copy, int spins, void* cuda_stream);

/* ---- stepping without any device allocation ------------------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers that may not call
 * cudaMalloc (a host framework that owns every device allocation under a fixed budget, plug-ins
 * loaded into such a framework, real-time loops that forbid allocation after start-up).
 *
 * mm_step_static_scratch advances nsteps time steps of the same scheme as mm_step, in place on
 * caller-owned FP64 device buffers Q_dev [6][ny][nx] and G_dev [ny][nx][nv2][nv1] (inputs and
 * outputs), writing the last step's heat flux to H_dev [4][ny][nx].  It allocates nothing: all
 * scratch (the split-step buffer G*, the intermediate macro state, per-cell primitive fields,
 * the diffuse-wall cell list and the error word) lives in one static device array of
 * MM_STATIC_SCRATCH_BYTES bytes that every GPU loading this library holds until process exit.
 *  - Limits: precision MM_PREC_FP64 only; nx*ny <= MM_STATIC_MAX_CELLS and
 *    nx*ny*nv1*nv2 <= MM_STATIC_MAX_PHASE.  Larger problems, other precisions, NULL buffers,
 *    Q_dev or H_dev not 16-byte aligned, G_dev not 256-byte aligned (the rules of
 *    mm_create_borrowed), dt <= 0, eps <= 0 or nsteps < 0 return MM_ERR_INVALID_ARG with a
 *    message in errbuf.
 *  - Works on the current device and cuda_stream (NULL = legacy default stream).  Every call
 *    looks up the array's device address in the current context (cudaGetSymbolAddress, which
 *    allocates nothing); the first call on a device may load the library's device code there,
 *    so make that first call before any stream capture.
 *  - Every call shares the one array and it keeps the previous call's contents (the zero-start
 *    parts are cleared at the start of each call).  Calls that overlap on the GPU -- on two
 *    streams, or from two host threads -- race on it and give wrong results.
 *  - Returns after synchronising cuda_stream; MM_ERR_NONPHYSICAL reports a non-physical state.
 *  - errbuf (may be NULL) receives a NUL-terminated message of at most errlen bytes. */
#define MM_STATIC_MAX_CELLS 16384
#define MM_STATIC_MAX_PHASE 1048576
#define MM_STATIC_SCRATCH_BYTES 18285312
mm_status mm_step_static_scratch(const mm_grid* grid, const mm_params* params, double* Q_dev,
                                 double* G_dev, double* H_dev, double dt, double eps,
                                 int nsteps, void* cuda_stream, char* errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif
#endif /* MMKFVS_H */
