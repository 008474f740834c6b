/*
 * hweno.h -- C ABI of libhweno, the B300 (sm_103a) implementation of the
 * per-cell, per-stage spatial operator of the fifth-order finite-volume
 * derivative-based HWENO scheme with unified stencils (arxiv 2607.24325).
 *
 * Problem (Sec. 1, Eq. hyperbolic-conservation-laws): u_t + div F(u) = 0,
 * u(x, 0) = u0(x), in 1D (Sec. 2.1) or 2D (Sec. 2.2) on a uniform grid, with
 * F = advection, Burgers or the Euler equations of gas dynamics (Examples
 * 2, 4-9).  The library evolves the cell averages u-bar together with the
 * derivative moments v-bar (and w-bar in 2D), reconstructs from the unified
 * compact stencils without the target cell's own derivatives (Step 1-3),
 * applies global Lax-Friedrichs fluxes and the SSP-RK3 update with the
 * limited derivatives substituted at every stage (Step 4), characteristic-wise
 * for Euler (Remark 1).
 *
 * Conventions for every entry point:
 *  - Every call returns hweno_status; nothing throws or aborts across the ABI.
 *    On failure hweno_last_error() (thread-local) describes the cause.
 *  - Arrays are SoA planes, x fastest, no ghost cells: U[f][j][i] with
 *    f = d*nc + k, d = 0 cell averages, 1 x-derivative moments, 2
 *    y-derivative moments (2D); k the conserved component (nc = 1 for scalar
 *    equations, 3 for 1D Euler (rho, rho u, E), 4 for 2D Euler
 *    (rho, rho u, rho v, E)).  1D v-bar is the mean of u_x over the cell
 *    (Sec. 2.1); 2D v-bar = (1/dy) int u_x dOmega and w-bar = (1/dx) int u_y
 *    dOmega are the scaled moments of Sec. 2.2.
 *  - Element type is double for HWENO_FP64 solvers and float otherwise.
 *  - Pointers flagged on_device are device pointers on the current device;
 *    otherwise host pointers (pinned or pageable).  The caller owns every
 *    buffer it passes; the library owns its internal workspace (stage states,
 *    the stage-1 limited derivatives, the device control block).
 *  - Work runs on the solver's own CUDA stream (hweno_stream()).  A call that
 *    takes caller device buffers first waits for the caller's stream given
 *    at creation and, before returning, makes that stream wait for the
 *    library's work, so stream-ordered callers (e.g. PyTorch) need no extra
 *    synchronisation.  Calls that return host data synchronise.
 *  - Device-side faults and non-physical states (NaN, negative density or
 *    pressure) surface as HWENO_ERR_CUDA / HWENO_ERR_NONPHYSICAL at the next
 *    call that synchronises.
 */
#ifndef HWENO_H
#define HWENO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HWENO_OK = 0,
  HWENO_ERR_ARG = 1,          /* invalid argument (reported, nothing changed) */
  HWENO_ERR_CUDA = 2,         /* CUDA runtime error */
  HWENO_ERR_NONPHYSICAL = 3,  /* NaN / Inf / non-positive density or pressure */
  HWENO_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
  HWENO_ERR_OOM = 5,          /* device allocation failed */
  HWENO_ERR_STATE = 6         /* call out of order (e.g. no state set) */
} hweno_status;

enum { HWENO_EQ_ADVECTION = 0, HWENO_EQ_BURGERS = 1, HWENO_EQ_EULER = 2 };
enum { HWENO_BC_PERIODIC = 0, HWENO_BC_OUTFLOW = 1, HWENO_BC_REFLECT = 2, HWENO_BC_INFLOW = 3,
       HWENO_BC_SPLIT = 4, HWENO_BC_SHOCK = 5 };
enum { HWENO_FP64 = 0, HWENO_FP32 = 1, HWENO_FP32_IND64 = 2 };
enum { HWENO_DT_CFL = 0, HWENO_DT_CFL_DX53 = 1 };
enum { HWENO_BETA_MOMENT = 0, HWENO_BETA_TYPICAL = 1 };

/* Problem statement and scheme parameters.
 *  dim            1 or 2
 *  nx, ny         cells per direction (>= 3; ny ignored in 1D)
 *  xlo..yhi       domain [xlo, xhi] (x [ylo, yhi])
 *  equation       HWENO_EQ_*; adv_x, adv_y the advection velocity;
 *                 gamma_gas the ratio of specific heats (Euler)
 *  lin_w          linear weights gamma_0..gamma_2 (1D) / gamma_0..gamma_4
 *                 (2D), each > 0, summing to 1 (Eq. rewrite, rewrite-2D);
 *                 the paper's experiments use 1/400 per linear polynomial
 *  eps            epsilon of the nonlinear weights (paper: 1e-8)
 *  weight_pow     power of beta in the weight denominator: 1 (beta + eps,
 *                 which reproduces the paper's tables in 1D and 2D) or 2
 *                 (beta^2 + eps, as printed in Eq. nonlinear-weights-2D)
 *  charwise       Euler: 1 characteristic-wise (Remark 1), 0 component-wise
 *  linear_weights 1: omega = gamma everywhere (the linear reconstruction p0)
 *  cfl, dt_rule   dt = cfl h / alpha with h = dx (HWENO_DT_CFL) or dx^(5/3)
 *                 (HWENO_DT_CFL_DX53, for order studies); 2D uses
 *                 cfl / (alpha_x/hx + alpha_y/hy)
 *  bc[4]          x-low, x-high, y-low, y-high: HWENO_BC_*
 *  bc_state[4][4] conservative state imposed by HWENO_BC_INFLOW sides
 *                 (ghost derivative moments zero)
 *  HWENO_BC_SPLIT and HWENO_BC_SHOCK (2D only) decide per ghost cell by the
 *  coordinate s of its centre along the side (x on the y sides, y on the x
 *  sides) and the time t of the RK stage (t^n, t^n + dt, t^n + dt/2):
 *    SPLIT: s < bc_param[side][0] -> bc_state[side], else reflective --
 *           the wall of the double Mach reflection example (Sec. 3);
 *    SHOCK: s < bc_param[side][0] + bc_param[side][1] t -> bc_state[side],
 *           else bc_state2[side] -- a straight shock moving along the side
 *           (that example's top boundary).
 *  precision      HWENO_FP64, HWENO_FP32 (storage and stencil arithmetic), or
 *                 HWENO_FP32_IND64 (FP32 storage and stencil arithmetic; the
 *                 coefficients entering the smoothness indicators, the
 *                 indicators, tau and tau^2/(beta + eps) in FP64, the
 *                 normalisation of the nonlinear weights in FP32)
 *  smoothness     HWENO_BETA_MOMENT: the paper's indicator (Step 2 of Sec. 2.1
 *                 and 2.2, sum of squared scaled derivatives at the cell
 *                 centre); HWENO_BETA_TYPICAL: the Jiang-Shu integral
 *                 indicator it replaces, Eq. (smoothness-indicator-typical)
 *                 and its 2D form (cell means of the squared scaled
 *                 derivatives; identical for the linear polynomials)
 */
typedef struct {
  int dim;
  int nx, ny;
  double xlo, xhi, ylo, yhi;
  int equation;
  double adv_x, adv_y, gamma_gas;
  double lin_w[5];
  double eps;
  int weight_pow;
  int charwise;
  int linear_weights;
  double cfl;
  int dt_rule;
  int bc[4];
  double bc_state[4][4];
  int precision;
  int smoothness;
  double bc_state2[4][4];
  double bc_param[4][2];
} hweno_config;

typedef struct hweno_solver hweno_solver;
typedef struct hweno_batch hweno_batch;

/* Thread-local description of the last failure of this thread (never NULL). */
const char* hweno_last_error(void);
/* Library version string. */
const char* hweno_version(void);

/* Create a solver for one grid (Sec. 2.1 / 2.2).  cuda_stream is the
 * caller's cudaStream_t (NULL = legacy default stream) that data calls order
 * against.  Allocates the library workspace on the current device.
 * Errors: HWENO_ERR_ARG (bad config: dim not 1 or 2, fewer than 3 cells per
 * direction, more than 2^31 cells, an empty or non-finite domain, linear
 * weights not positive or not summing to 1, eps, cfl, gamma_gas (Euler) or
 * the advection speeds not finite and in range, unpaired periodic sides, an
 * unknown enum value), HWENO_ERR_OOM, HWENO_ERR_CUDA. */
hweno_status hweno_create(const hweno_config* cfg, void* cuda_stream, hweno_solver** out);
/* Free the solver and its workspace (NULL is a no-op). */
void hweno_destroy(hweno_solver* s);
/* The solver's own CUDA stream (cudaStream_t), on which kernels run. */
void* hweno_stream(hweno_solver* s);
/* Number of stored fields nf = nc * (dim + 1) and cells per field. */
hweno_status hweno_shape(const hweno_solver* s, int* nfields, size_t* ncells);

/* Initial data u0 (Sec. 1, Eq. hyperbolic-conservation-laws): u0 is called
 * with n points (x[k], y[k]) (y = 0 in 1D) and writes the nc conserved
 * components of u0 at each point to u[k*nc + c]; ctx is passed through.
 * Cell averages come from nq x nq (1D: nq) Gauss-Legendre points; the
 * derivative moments are exact face differences: 1D v-bar = (u0(x_{i+1/2})
 * - u0(x_{i-1/2})) / dx, 2D v-bar = Gauss mean over y of the x-face
 * difference (= (1/dy) int u_x), w-bar likewise.  Jumps must lie on faces or
 * be resolved by the caller.  Then acts as hweno_set_state.  Host code;
 * nq in [1, 16]. */
typedef void (*hweno_u0_fn)(int n, const double* x, const double* y, double* u, void* ctx);
hweno_status hweno_project(hweno_solver* s, hweno_u0_fn u0, void* ctx, int nq);

/* Copy a state in (U[nf][ny][nx]) and compute its wave speeds; resets t. */
hweno_status hweno_set_state(hweno_solver* s, const void* U, int on_device);
/* Copy the current state out (same layout); synchronises if !on_device. */
hweno_status hweno_get_state(hweno_solver* s, void* U, int on_device);

/* Simulation time of the current state and the steps taken by the last
 * advance (synchronises); set_time restores a checkpoint's time after
 * hweno_set_state (which resets it to 0).  The wave speeds are a function of
 * the state, so set_state + set_time resumes a run bit for bit. */
hweno_status hweno_get_time(hweno_solver* s, double* t, int* steps);
hweno_status hweno_set_time(hweno_solver* s, double t);

/* Max spectral radius over the cell averages of the current state
 * (alpha of the global Lax-Friedrichs flux, Sec. 2.1 and 2.2).  Synchronises. */
hweno_status hweno_alpha(hweno_solver* s, double* alpha_x, double* alpha_y);

/* One application of the spatial operator to the current state with the
 * given Lax-Friedrichs constants: L_out[nf][cells] = (L^u, L^v, L^w) of Eq.
 * semi-discrete-scheme / 2D-semi-discrete-scheme-uniform, dhat_out[nc*dim]
 * [cells] = the limited derivatives v-hat (and w-hat) of Step 3.  Both are
 * caller device buffers of the solver's element type.  Time-dependent
 * boundaries take the solver's current time. */
hweno_status hweno_apply_operator(hweno_solver* s, double alpha_x, double alpha_y,
                                  void* L_out, void* dhat_out);

/* One SSP-RK3 step (Step 4) with the given dt and Lax-Friedrichs constants,
 * from the solver's current time, which it advances by dt. */
hweno_status hweno_step(hweno_solver* s, double dt, double alpha_x, double alpha_y);

/* One RK stage (1, 2 or 3) of an SSP-RK3 step (Step 4 of Sec. 2.2) with the
 * given dt and Lax-Friedrichs constants, for single 2D solvers: the stages
 * of hweno_step one call at a time, so that a caller can replace rows of a
 * stage's output (hweno_rows) before the next stage reads them -- the halo
 * exchange of a grid split into slabs of rows.  Stage 1 reads the state and
 * writes the stage-1 buffer (and the limited derivatives of Step 3), stage 2
 * reads it and writes the stage-2 buffer, stage 3 reads that and writes the
 * state, moves the solver's time by dt and recomputes alpha.  The stages of
 * one step run in order with the same dt and alpha (else HWENO_ERR_STATE or
 * HWENO_ERR_ARG). */
hweno_status hweno_stage(hweno_solver* s, int stage, double dt, double alpha_x, double alpha_y);

/* Copy rows [row0, row0 + nrows) of every field plane of one of the solver's
 * buffers -- 0: the state, 1: the stage-1 output, 2: the stage-2 output --
 * to (to_solver = 0) or from (to_solver = 1) the caller's device buffer
 * `rows`, laid out [nf][nrows][nx] in the solver's element type.  Single 2D
 * solvers; ordered on the solver's stream after earlier calls. */
hweno_status hweno_rows(hweno_solver* s, int buffer, int row0, int nrows, void* rows, int to_solver);

/* Recompute alpha from the current state's cell averages (after hweno_rows
 * replaced some of them) and return it, as hweno_alpha.  Synchronises. */
hweno_status hweno_alpha_update(hweno_solver* s, double* alpha_x, double* alpha_y);

/* Advance to t_final with the device-resident CFL time step (alpha from the
 * averages at the start of each step, last step clipped to t_final), at most
 * max_steps steps.  Steps are replayed from a captured CUDA graph; the host
 * polls the device control block once per graph replay.  Returns the time
 * reached and the steps taken.  HWENO_ERR_NONPHYSICAL if a state became
 * non-physical (the state is left at the failing step). */
hweno_status hweno_advance(hweno_solver* s, double t_final, int max_steps, double* t_out,
                           int* steps_out);

/* Opt-in measurement of the stage kernels inside hweno_advance: while
 * enabled, advance launches every step directly (no graph) and brackets
 * each stage kernel launch with CUDA events on the solver's stream; the
 * totals accumulate until the next hweno_set_profiling call resets them.
 * hweno_profile returns the summed device time of the stage launches (ms),
 * their number, and the number of kernels advance launched (5 per step:
 * control begin, stages 1-3, control end). */
hweno_status hweno_set_profiling(hweno_solver* s, int enable);
hweno_status hweno_profile(hweno_solver* s, double* stage_ms, long long* stage_launches,
                           long long* kernel_launches);

/* Measured FMA throughput of the current GPU in flop/s (2 per FMA) for
 * HWENO_FP64 or HWENO_FP32: the ALU roofline of the stencil kernels.  Runs a
 * short probe kernel (milliseconds); synchronises the device. */
hweno_status hweno_peak_fma(int precision, double* flops_per_second);

/* Self-check of the integer-ALU conversions of the mixed-precision path
 * (HWENO_FP32_IND64 widens its FP32 inputs to FP64 and narrows the FP64
 * weights back without the FP64 pipe).  Not part of the paper's method: a
 * diagnostic that exposes those two routines.  For i < n (device pointers,
 * caller-owned): wide_out[i] = f_in[i] widened to FP64 (exact),
 * narrow_out[i] = d_in[i] rounded to FP32 (to nearest, ties to even), both
 * as IEEE 754 conversions must give.  Launches on the legacy default stream
 * and synchronises the device.  HWENO_ERR_ARG for n < 0 or a null pointer
 * with n > 0. */
hweno_status hweno_selftest_convert(const float* f_in, double* wide_out, const double* d_in, float* narrow_out,
                                    int n);

/* Self-check of the FP64 reciprocal the FP64 kernels use (two Newton-Raphson
 * steps from the hardware's approximate FP64 reciprocal, for 1/rho in the
 * fluxes and eigenvectors, 1/c, and the normalisation of the nonlinear
 * weights).  Not part of the paper's method: a diagnostic that exposes that
 * routine.  For i < n (device pointers, caller-owned): y_out[i] = the
 * library's 1 / x_in[i], to be within one unit in the last place of the
 * correctly rounded quotient wherever x_in[i] and its reciprocal are normal
 * numbers; zeros, infinities and NaN give the IEEE results, subnormal
 * arguments and results are flushed (+-inf, +-0).  Launches on the legacy
 * default stream and synchronises the device.  HWENO_ERR_ARG for n < 0 or a
 * null pointer with n > 0. */
hweno_status hweno_selftest_rcp64(const double* x_in, double* y_out, int n);

/* Autotuner: time the candidate launch shapes of the stage kernel on the
 * current state (reps operator applications each, CUDA events) and keep the
 * fastest for every later launch.  1D: warps per block {2, 4, 8} x resident
 * blocks per SM {4, 8, 16, 32}; 2D: persistent grid (tiles looped over one
 * CTA per SM slot) or one CTA per tile.  best_ms (may be NULL) receives the
 * winner's time per launch, shape_out[3] (may be NULL) the winner (warps,
 * blocks per SM, persistent).  Allocates and frees two temporary buffers. */
hweno_status hweno_autotune(hweno_solver* s, int reps, double* best_ms, int* shape_out);

/* ---- Batches of independent problems of uneven sizes, all 1D or all 2D
 * (one launch per stage for all instances: 1D a table of 30-cell warp tasks,
 * 2D a table of 30 x 30 tiles; per-instance alpha, dt, time and done flag;
 * whole steps replayed from a CUDA graph). ---- */
/* cfgs[n] share dim, equation, precision, characteristic/component-wise
 * reconstruction, linear weights, eps, weight power, indicator form, gamma
 * and the advection velocity; grid sizes, domains, boundaries, CFL numbers
 * and dt rules are per instance.  The learned indicator serves single
 * solvers only. */
hweno_status hweno_batch_create(int n, const hweno_config* cfgs, void* cuda_stream,
                                hweno_batch** out);
void hweno_batch_destroy(hweno_batch* b);
void* hweno_batch_stream(hweno_batch* b);
/* Total cells (sum of nx, or of nx * ny in 2D) and per-instance offsets
 * (n+1 entries, host). */
hweno_status hweno_batch_layout(const hweno_batch* b, size_t* total_cells, size_t* offsets);
/* U is [nf][total_cells]: instance k owns cells offsets[k] .. offsets[k+1]-1
 * of every field plane. */
hweno_status hweno_batch_set_state(hweno_batch* b, const void* U, int on_device);
hweno_status hweno_batch_get_state(hweno_batch* b, void* U, int on_device);
/* Advance every instance k to t_final[k] (host array); at most max_steps
 * steps per instance.  t_out, steps_out (host, may be NULL) receive per
 * instance results. */
hweno_status hweno_batch_advance(hweno_batch* b, const double* t_final, int max_steps,
                                 double* t_out, int* steps_out);
/* The autotuner of hweno_autotune for a batch (all instances at once). */
hweno_status hweno_batch_autotune(hweno_batch* b, int reps, double* best_ms, int* shape_out);
/* hweno_set_profiling / hweno_profile for a batch: the stage kernels'
 * device time over all instances (one launch per stage covers the batch). */
hweno_status hweno_batch_set_profiling(hweno_batch* b, int enable);
hweno_status hweno_batch_profile(hweno_batch* b, double* stage_ms, long long* stage_launches,
                                 long long* kernel_launches);
/* Apply the operator to every instance with per-instance Lax-Friedrichs
 * constants (host array): alpha[n] for 1D, alpha[n][2] = (alpha_x, alpha_y)
 * for 2D; L_out [nf][total], dhat_out [nc*dim][total] (device buffers; a 2D
 * instance occupies [offsets[k], offsets[k+1]) of every plane, row-major). */
hweno_status hweno_batch_apply_operator(hweno_batch* b, const double* alpha, void* L_out,
                                        void* dhat_out);

/* ---- Learned troubled-cell indicator (no counterpart in the paper; it
 * decides which cells may use the linear reconstruction p0, omega = gamma of
 * Eq. rewrite-2D, while the full nonlinear characteristic HWENO path stays
 * the fallback).  2D solvers only. ----
 * Features of a cell: the 5x5 patch (offsets -2..2, ghost cells by the
 * solver's boundary rules) of the density's u-bar, v-bar, w-bar, scaled by
 * s = 1/(range of the patch's u-bar + 1e-3 |centre u-bar| + 1e-30), the
 * centre value subtracted from the u-bar entries; 75 floats ordered
 * [field][dy][dx], dx fastest.  Network: 75 -> 32 (ReLU) -> 32 (ReLU) -> 1,
 * p = sigmoid(z); parameters as one float vector of 3521 entries: W1[32][75],
 * b1[32], W2[32][32], b2[32], w3[32], b3.  Label: the plain scheme's
 * largest |omega_m/gamma_m - 1| over every reconstructed field of both
 * passes (Step 3), compared with a threshold delta. */

/* feat_out: device float [cells][75] of the current state. */
hweno_status hweno_indicator_features(hweno_solver* s, float* feat_out);
/* dev_out: device float [cells], the label source above, of the current state. */
hweno_status hweno_indicator_labels(hweno_solver* s, float* dev_out);
/* Load trained parameters (host float[nparams], nparams = 3521) as FP16
 * tensor-core weights and switch the solver to the learned path: from then
 * on hweno_step / hweno_advance evaluate the network once per step on u^n,
 * mark cells with p > p_threshold troubled, dilate the mark by one cell, and
 * let every warp whose 32 cells are all unmarked reconstruct with p0. */
hweno_status hweno_indicator_load(hweno_solver* s, const float* params, int nparams, double p_threshold);
/* Back to the plain nonlinear path everywhere. */
hweno_status hweno_indicator_off(hweno_solver* s);
/* Run the network on the current state: smooth_out[cells] = 1 where the
 * linear path is allowed (after dilation), troubled_out[cells] = 1 where the
 * network itself marks the cell; device uint8 buffers, either may be NULL. */
hweno_status hweno_indicator_mask(hweno_solver* s, void* smooth_out, void* troubled_out);

/* Training on the GPU (FP32 master parameters, Adam with beta1 0.9,
 * beta2 0.999, eps 1e-8).  The loss is the class-weighted binary cross
 * entropy (positives weighted by pos_weight), mean over the minibatch.
 * feat/dev are device float arrays [N][75] and [N]; idx is a device int32
 * array [B] selecting the minibatch (the caller draws the permutation). */
typedef struct hweno_mlp hweno_mlp;
hweno_status hweno_mlp_create(int max_batch, void* cuda_stream, hweno_mlp** out);
void hweno_mlp_destroy(hweno_mlp* m);
/* Set the parameters (host float[3521]) and reset the Adam state. */
hweno_status hweno_mlp_set_params(hweno_mlp* m, const float* params);
hweno_status hweno_mlp_get_params(hweno_mlp* m, float* params);
/* Loss and gradient (host float[3521]) of one minibatch, no update. */
hweno_status hweno_mlp_gradient(hweno_mlp* m, const float* feat, const float* dev, const int* idx, int B,
                                double delta, double pos_weight, float* grad_out, double* loss_out);
/* One Adam step on one minibatch (asynchronous on the mlp's stream). */
hweno_status hweno_mlp_train_step(hweno_mlp* m, const float* feat, const float* dev, const int* idx, int B,
                                  double delta, double pos_weight, double lr);
/* Mean of the minibatch losses since the last call (synchronises). */
hweno_status hweno_mlp_mean_loss(hweno_mlp* m, double* loss);
/* FP32 probabilities prob[n] (device) of n samples feat[n][75] (device). */
hweno_status hweno_mlp_predict(hweno_mlp* m, const float* feat, long long n, float* prob);

/* The whole training of the indicator's network in one call (the loop of
 * hweno_mlp_train_step, on the GPU; the paper's own weights define the
 * labels: Sec. 2.2 Step 3).  feat [n][75] and dev [n] are device float
 * arrays (features and label sources of hweno_indicator_features /
 * hweno_indicator_labels; a cell is a positive when dev > delta).  Each
 * epoch visits the n samples in a seeded random order, minibatches of
 * `batch` (a trailing partial batch is skipped), one Adam step each; the
 * order of epoch e is the Fisher-Yates shuffle of 0..n-1 driven by SplitMix64
 * from the state seed + (e + 1) * 0xD1B54A32D192ED03 (index j = next() mod
 * (i + 1) for i = n-1 down to 1; hweno_train_permutation writes it).
 * pos_weight <= 0 takes min(50, max(1, negatives / positives)), counted on
 * the device.  init_params (host float[3521]) or, when NULL, seeded
 * He-normal hidden layers, N(0, 1/32) output weights and zero biases.
 * params_out (host float[3521]) receives the trained parameters, losses_out
 * (host double[epochs], may be NULL) each epoch's mean minibatch loss.
 * Allocates its work buffers and frees them before returning; runs on
 * cuda_stream and synchronises it. */
typedef struct {
  int epochs;                 /* passes over the data, >= 1 */
  int batch;                  /* minibatch size, 1 <= batch <= min(n, 2^24) */
  double lr;                  /* Adam step size, > 0 */
  double delta;               /* label threshold on max |omega_m / gamma_m - 1| */
  double pos_weight;          /* class weight of positives; <= 0: from the labels */
  unsigned long long seed;    /* permutations (and the default initialisation) */
} hweno_train_opts;
hweno_status hweno_indicator_train(const float* feat, const float* dev, long long n, const hweno_train_opts* opts,
                                   const float* init_params, float* params_out, double* losses_out,
                                   void* cuda_stream);
/* The visiting order of epoch `epoch` of hweno_indicator_train (host int[n]);
 * does nothing when perm is NULL or n < 1. */
void hweno_train_permutation(unsigned long long seed, int epoch, long long n, int* perm);

/* ---- Allocation-free step (the paper has no counterpart: this serves
 * callers that cannot allocate device memory when they need a step, e.g. a
 * host that has given the whole device memory budget to its own pool
 * allocator, or a latency-critical loop that must not pay cudaMalloc's
 * implicit device synchronisation). ----
 * One SSP-RK3 step (Sec. 2.1 Step 4) of the single 1D problem described by
 * cfg (dim must be 1), with the given dt and Lax-Friedrichs constant alpha:
 * U_out = step(U_in).  U_in and U_out are caller device buffers [2*nc][nx]
 * of the config's element type (they may be the same buffer); the work is
 * queued on cuda_stream (cudaStream_t, NULL = legacy default stream) and the
 * call returns without synchronising.
 * No memory is allocated: the two intermediate stage states, the stage-1
 * limited derivatives, the control block and the task table live in a
 * 16 MiB file-scope device array that every GPU which loads the library
 * holds until exit.  That caps nx at about 139,000 cells for FP64 Euler
 * (about 419,000 for FP64 scalar equations, twice these in FP32); larger nx
 * is rejected with HWENO_ERR_ARG and a message giving the limit.
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array, so calls whose work overlaps on
 * the GPU (different streams, or threads without ordering) race and corrupt
 * each other's results; order them on one stream.
 * Errors: HWENO_ERR_ARG (config, pointers, dt/alpha, size), HWENO_ERR_CUDA. */
hweno_status hweno_step_1d_noalloc(const hweno_config* cfg, const void* U_in, void* U_out, double dt,
                                   double alpha, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
