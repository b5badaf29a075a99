/*
 * grim.h -- C ABI of the B300 (sm_103a) implicit extended-GRMHD zone step.
 *
 * The library implements the hot path of the scheme of Chandra, Foucart &
 * Gammie (2017), "grim: a flexible, conservative scheme for relativistic
 * fluid theories": the two-stage semi-implicit time step of Section 2.3 for
 * the 10-field extended MHD system of Section 4, in which each zone's new
 * primitive variables are found by driving the discrete residual R(P) of
 * Eq. half_step_residual (and its full-step analogue, Eq. full_step) to zero
 * with Newton iterations on a finite-difference Jacobian (Section 3.1) and a
 * quadratic backtracking line search (Section 3.2).  Fluxes are local
 * Lax-Friedrichs or HLLE (Section 2.4.2) on generalized-minmod, WENO5 or PPM
 * states (Section 2.4.1) with flux-CT for the magnetic field (Section 4.2).
 *
 * Conventions shared by every entry point:
 *  - A state is a caller-owned DEVICE buffer of float64, structure of arrays
 *    [10][n3][n2][n1] (X1 fastest), fields in the order rho, u, u^1, u^2,
 *    u^3, B^1, B^2, B^3, q~, dP~, where q~ and dP~ are the rescaled heat flux
 *    and pressure anisotropy of Eqs. q and dP.  Units G = c = 1.
 *  - Every call is asynchronous on the stream given to grim_init and returns
 *    0 on success or a negative GRIM_E* code; grim_strerror names it.  No call
 *    traps, aborts or waits on the device.  Zones whose Newton solve does not
 *    converge keep their last iterate and are counted in grim_stats.
 *  - The library owns its scratch (stage constants, status bytes, counters),
 *    allocated once by grim_init and freed by grim_destroy (grim_step_static
 *    uses a static device array instead).
 *  - Grids: 2-D (n3 = 1) or 3-D, in Minkowski space or in the Kerr metric in
 *    modified Kerr-Schild coordinates (Section 2.1); 2-D Minkowski grids run
 *    specialised flat-space kernels, everything else the general-metric
 *    kernels.
 *  - Reconstruction: generalized minmod (MC), WENO5 or PPM (Section 2.4.1);
 *    Riemann solver: LLF or HLLE (Section 2.4.2).
 *  - Precision: float64 throughout, or the mixed solver (GRIM_MIXED): the
 *    finite-difference Jacobian and its LU in float32; the residual, the
 *    update, the line search and the convergence test in float64; the
 *    explicit face fluxes and the source terms at P^E in float-float
 *    (pairs of floats, about 48 bits), with U(P_n) and the flux divergence
 *    in float64.
 *  - Optionally, Newton starts from a small network's prediction
 *    (grim_mlp_*, grim_set_guess; inference and training GEMMs on the
 *    fifth-generation tensor cores), with the plain start P_n as fallback.
 */
#ifndef GRIM_H
#define GRIM_H

#ifdef __cplusplus
extern "C" {
#endif

#define GRIM_OK 0
#define GRIM_EINVAL (-1)   /* bad argument or unsupported configuration */
#define GRIM_ECUDA (-2)    /* a CUDA runtime call failed (message: grim_last_error) */
#define GRIM_ENOMEM (-3)   /* device allocation failed */
#define GRIM_ESIZE (-4)    /* a size is outside the limit of the entry point */

#define GRIM_BC_PERIODIC 0
#define GRIM_BC_OUTFLOW 1
#define GRIM_BC_REFLECT 2

#define GRIM_METRIC_MINKOWSKI 0
#define GRIM_METRIC_MKS_KERR 1 /* Kerr (M = 1, spin a) in modified Kerr-Schild coordinates (Section 2.1) */

#define GRIM_RECON_MC 0    /* generalized minmod, parameter theta (2 = MC, 1 = minmod) */
#define GRIM_RECON_WENO5 1 /* Jiang & Shu WENO5 */
#define GRIM_RECON_PPM 2   /* Colella & Woodward PPM face values with limited slopes (theta) */

#define GRIM_FLUX_LLF 0    /* local Lax-Friedrichs (Section 2.4.2) */
#define GRIM_FLUX_HLLE 1   /* HLLE with the bounds c_R = max(c, 0), c_L = max(-c, 0) (Section 2.4.2) */

#define GRIM_FP64 0        /* Jacobian, LU, residual all in float64 */
/* Jacobian and LU in float32; residual, update and test in float64; the
 * explicit stage's face states, fluxes and wave speeds (and, on 2-D
 * Minkowski grids, the MC reconstruction and the limited slopes) in
 * float-float, pairs of floats with about 48 significant bits, joined back
 * into float64 before they are stored; U(P_n), the flux divergence, flux-CT
 * and the stage constants stay float64.  A zone whose float32-Jacobian
 * iteration ends with a non-zero status (the float32 Jacobian of a cold zone
 * can lose the internal-energy column to rounding) is solved again with the
 * float64 Jacobian from P_n, or from P^E when the stage's output overwrites
 * P_n (grim_stats.rescued); with k_max = 0 there is no second solve. */
#define GRIM_MIXED 1

/* Grid (Section 2.1): uniform in X^i, dX^i = (x_end - x_start)/n_i. */
typedef struct {
  int dim, n1, n2, n3;
  double x_start[3], x_end[3];
  int bc[3][2]; /* GRIM_BC_* for the low and high side of each direction */
} grim_grid;

/* Metric.  GRIM_METRIC_MKS_KERR: X^1 = log r, theta = pi X^2 + ((1-h)/2)
 * sin(2 pi X^2), phi = X^3 (Section 2.1), over the Kerr-Schild form of the
 * Kerr metric with spin a; the relaxation time becomes tau_R r^{3/2}. */
typedef struct {
  int kind; /* GRIM_METRIC_* */
  double spin, h;
} grim_metric;

/* Physics (Section 4): gamma-law gas, closure chi = phi c_s^2 tau_R,
 * nu = psi c_s^2 tau_R, switches for conduction, viscosity and the
 * higher-order terms of Eqs. q_evol_eqn_rescaled and dP_evol_eqn_rescaled.
 * Each zone's Newton update solves the 7x7 block of rho, u, u^i, q~, dP~
 * (B is explicit, Section 8.2); with conduction and viscosity both off
 * (ideal MHD), a zone whose q~, dP~ and their residual rows are zero solves
 * the 5x5 block of rho, u, u^i: the same root at 5 instead of 7 Jacobian
 * columns. */
typedef struct {
  double gamma, tau_R, phi, psi;
  int conduction, viscosity, higher_order;
  int recon;    /* GRIM_RECON_* (grim_step_static: MC or WENO5) */
  double theta; /* generalized minmod parameter, also used for source slopes */
  int floors;   /* after every stage: a zone whose Newton iteration ended with a
                   non-zero status reverts to its start (P_n, flux-CT field);
                   then rho >= 1e-5 r^{-3/2}, u >= 1e-7 r^{-5/2} (r = 1 in
                   Minkowski space), -b^2 <= dP <= b^2/2.  General-metric
                   path only (3-D or Kerr grids). */
  int riemann;  /* GRIM_FLUX_LLF or GRIM_FLUX_HLLE (grim_step_static: LLF only) */
} grim_physics;

/* Nonlinear solver (Section 3).  Converged when max_a |r_a| <= tol with
 * r_a = dt_s R_a / (|U_a(P_n)| + |U_0(P_n)|).  eps_fd: the finite-difference
 * parameter epsilon of Section 3.1 (float64 Jacobian), eps_fd32 the same for
 * the float32 Jacobian of GRIM_MIXED.  k_max: Newton updates per stage;
 * ls_max: backtracks per line search.  fd32_central: 0 builds the float32
 * Jacobian with the one-sided differences of Section 3.1, 1 with centred
 * differences (r(P + h e_j) - r(P - h e_j))/(2h) on the same step h, which
 * float32 rounding favours (an inexact-Newton choice; the float64 Jacobian
 * always uses the paper's one-sided form). */
typedef struct {
  int precision; /* GRIM_FP64 or GRIM_MIXED */
  double tol, eps_fd, eps_fd32;
  int k_max, ls_max;
  int fd32_central;
} grim_solver;

/* Counters accumulated over calls since the last grim_reset_stats. */
typedef struct {
  unsigned long long zones;     /* zone solves (one per zone per stage) */
  unsigned long long failed;    /* zone solves that ended with a non-zero status */
  unsigned long long iters;     /* Newton updates */
  unsigned long long evals64;   /* float64 residual evaluations */
  unsigned long long evals32;   /* float32 residual evaluations */
  unsigned long long lu64;      /* float64 LU solves (7x7 block; 5x5 in ideal MHD) */
  unsigned long long lu32;      /* float32 LU solves (7x7 block; 5x5 in ideal MHD) */
  unsigned long long hist[32];  /* zone solves by number of Newton updates (31 = 31 or more) */
  double max_res;               /* largest final max_a |r_a| over zone solves */
  unsigned long long launches;  /* kernels launched by the library */
  unsigned long long fallbacks; /* zone solves whose learned start lost to P_n (grim_set_guess) */
  unsigned long long rescued;   /* GRIM_MIXED: zone solves whose float32-Jacobian iteration ended with a
                                   non-zero status and were solved again with the float64 Jacobian from
                                   P_n (their status is the float64 solve's) */
  unsigned long long mlp_stalls; /* learned-start launches that gave up waiting for their tensor-core
                                    work (a bounded wait); the zones not reached keep the plain start */
} grim_stats;

typedef struct grim_ctx grim_ctx;

/* Create a context: validates the configuration, allocates the library's
 * scratch for n1*n2*n3 zones on the current device, binds the CUDA stream
 * `stream` (a cudaStream_t; NULL = the legacy default stream).
 * dim 2 (n3 = 1) or 3.  Two-dimensional Minkowski grids run the specialised
 * flat-space kernels; 3-D grids and the Kerr metric run the general-metric
 * kernels, whose geometry tables (metric, inverse, sqrt(-g), lapse,
 * connection and tau_R at zone centres and faces; axisymmetric, so n1 x n2
 * only) are computed here once, on the stream.
 * Errors: GRIM_EINVAL (dim not 2 or 3, n3 != 1 in 2-D, sizes < 1, unsupported
 * metric or reconstruction), GRIM_ENOMEM, GRIM_ECUDA.  *out is NULL on
 * failure. */
int grim_init(const grim_grid* grid, const grim_metric* metric, const grim_physics* phys,
              const grim_solver* solver, void* stream, grim_ctx** out);

/* One time step (Section 2.3): the half step P_n -> P_{n+1/2} with P^E = P_n
 * and dt/2, then the full step P_n -> P_{n+1} with P^E = P_{n+1/2} and dt.
 * P_in, P_out: device states; P_out may equal P_in (the full stage then
 * reads a copy of P_in: one more state-sized device buffer, allocated by the
 * first such call, so make it before capturing the call into a graph).  The
 * initial guess of each stage is P_n with B set to the explicit flux-CT
 * update. */
int grim_step(grim_ctx* ctx, const double* P_in, double* P_out, double dt);

/* grim_step with HOST buffers: copies P_in_host to the device, steps, and
 * copies the result to P_out_host (pinned host memory gives asynchronous
 * copies); synchronises the stream before returning. */
int grim_step_host(grim_ctx* ctx, const double* P_in_host, double* P_out_host, double dt);

/* One stage: solve R(P) = 0 with explicit state P_E, start-of-step state P_n
 * and stage time step dts (dt/2 for the half step, dt for the full step).
 * guess: optional device state to start Newton from (NULL = P_n); its B
 * components are replaced by the explicit flux-CT update.  P_out may equal
 * P_n (the stage then reads a copy of P_n, as grim_step in place) but not
 * P_E (GRIM_EINVAL: neighbouring zones read P_E).  Writes P_out and,
 * if non-NULL, the per-zone Newton update count and status bits
 * (1 max-iterations, 2 line-search stall, 4 singular, 8 non-finite,
 * 16 inadmissible rho or u) to device byte arrays of n1*n2*n3 entries. */
int grim_stage(grim_ctx* ctx, const double* P_n, const double* P_E, double dts, const double* guess,
               double* P_out, unsigned char* iters, unsigned char* status);

/* Residual of a stage at P_k (Eq. half_step_residual): scaled r_a when
 * scaled != 0, else the raw R_a.  R_out: device state-shaped buffer. */
int grim_residual(grim_ctx* ctx, const double* P_n, const double* P_E, double dts, const double* P_k,
                  int scaled, double* R_out);

/* Kernel classes reported by grim_kernel_times. */
#define GRIM_K_EXPLICIT 0  /* fused tile kernel: reconstruction, fluxes, flux-CT, constants */
#define GRIM_K_NEWTON64 1  /* Newton, float64 Jacobian */
#define GRIM_K_NEWTON32 2  /* Newton, float32 Jacobian */
#define GRIM_K_RESIDUAL 3  /* single residual evaluation */
#define GRIM_K_FACES 4     /* face fluxes: reconstruction, LLF (one thread per face) */
#define GRIM_K_ZONECONST 5 /* flux-CT, divergence, slopes, stage constants */
#define GRIM_K_MLP 6       /* learned initial guess (MLP inference) */
#define GRIM_K_COUNT 8

/* Enable (1) or disable (0) per-kernel timing: CUDA events are recorded on
 * the context's stream around every kernel launch, and their durations are
 * accumulated per kernel class until read by grim_kernel_times. */
int grim_profile(grim_ctx* ctx, int enable);

/* Read and reset the accumulated per-kernel durations (milliseconds) and
 * launch counts, arrays of GRIM_K_COUNT entries indexed by GRIM_K_*.
 * Synchronises the stream. */
int grim_kernel_times(grim_ctx* ctx, double* ms, unsigned long long* launches);

/* Copy the accumulated counters to *out (synchronises the stream). */
int grim_get_stats(grim_ctx* ctx, grim_stats* out);
int grim_reset_stats(grim_ctx* ctx);

/* Message of the last failing call on this context (static storage). */
const char* grim_last_error(grim_ctx* ctx);
const char* grim_strerror(int code);

/* Free the context and its scratch (NULL is ignored). */
void grim_destroy(grim_ctx* ctx);

/* Largest grid (n1*n2*n3 zones) grim_step_static accepts. */
#define GRIM_STATIC_MAX_ZONES 65536

/* One time step, as grim_step, that allocates no device memory.  (The paper
 * has no counterpart; this is an interface for callers.)  It is meant for
 * callers that cannot call cudaMalloc: host applications that own all device
 * memory through their own pool, and loops that must not allocate after
 * start-up because cudaMalloc can synchronise the device.
 *  - Arguments: the configuration structs of grim_init, a cudaStream_t
 *    (NULL = legacy default stream) and the caller's device states P_in and
 *    P_out (layout as above; P_out may equal P_in).
 *  - Scratch: the stage constants, half-step state, status bytes and
 *    counters live in one static device array sized for
 *    GRIM_STATIC_MAX_ZONES zones (about 23 MB), which every GPU that loads
 *    the library holds until the process exits.  Larger grids return
 *    GRIM_ESIZE without launching anything.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.
 *  - All calls share the one array: calls that overlap on the GPU (other
 *    streams, other threads) race and must be serialised by the caller.
 *  - Accepts 2-D Minkowski grids (dim = 2, n3 = 1) with MC or WENO5
 *    reconstruction and the LLF flux; anything else returns GRIM_EINVAL.
 *  - Zones whose Newton solve does not converge keep their last iterate, as
 *    in grim_step; grim_step_static_stats reports how many.
 *  - Returns 0, GRIM_EINVAL (bad configuration or pointer), GRIM_ESIZE or
 *    GRIM_ECUDA; asynchronous on the stream like grim_step. */
int grim_step_static(const grim_grid* grid, const grim_metric* metric, const grim_physics* phys,
                     const grim_solver* solver, void* stream, const double* P_in, double* P_out, double dt);

/* Counters of the last grim_step_static call on the current device (its two
 * stages: zone solves, failures, Newton updates, residual evaluations, the
 * update histogram, the largest final max_a |r_a|), read from the shared
 * static array into *out.  Waits for `stream` (the stream of that call) to
 * finish; allocates nothing.  A call made since on another stream or
 * thread may have overwritten them (the array is shared).  Returns 0,
 * GRIM_EINVAL or GRIM_ECUDA. */
int grim_step_static_stats(void* stream, grim_stats* out);

/* Measure the float64 and float32 FMA throughput of the current device with
 * dependent FMA chains (no memory traffic): writes TFLOP/s (2 flops per
 * FMA) to *fp64_tflops and *fp32_tflops.  Allocates and frees a small
 * device buffer; synchronises the device. */
int grim_peak_flops(double* fp64_tflops, double* fp32_tflops);

/* ---- Launch shapes, compaction, graphs. */
/* Launch shape of a context.  newton_bs: threads per block of the Newton
 * kernels (32, 64 or 128).  newton_kcut: after this many Newton updates a
 * zone that has not converged leaves the in-order kernel for a queue that a
 * persistent kernel works through densely, so that a few slow zones do not
 * hold whole warps (>= k_max: no queue).  newton_rounds: 1 = the in-order
 * kernel makes one update per round and, between rounds, packs the block's
 * unconverged zones into its lowest threads (their state moves through
 * shared memory; the zone constants stay where they are), so that converged
 * zones stop costing their warps issue slots; 0 = each thread runs its zone
 * to convergence or newton_kcut updates in one pass.  Either way the
 * results are the same bits.  faces_bs, zone_bs: threads per block of the
 * face-flux and zone-constant kernels (64, 128 or 256). */
typedef struct {
  int newton_bs, newton_kcut, faces_bs, zone_bs, newton_rounds;
} grim_tuning;

int grim_get_tuning(grim_ctx* ctx, grim_tuning* out);
/* GRIM_EINVAL for a value outside the sets above (newton_kcut >= 1, newton_rounds 0 or 1). */
int grim_set_tuning(grim_ctx* ctx, const grim_tuning* tuning);

/* Choose the launch shape by timing grim_step from the device state P with
 * step dt (P is not modified): each field of grim_tuning in turn over its
 * allowed values, the others held, keeping the fastest, in two passes over
 * the fields (CUDA events, median of 5 steps after one warm-up step).  With cache_path non-NULL, a line of
 * that text file (one JSON object per line, keyed by device name, grid,
 * precision, reconstruction, closures and whether a learned guess is set)
 * is used instead when present, and the result is written there otherwise.
 * Sets the context's tuning, writes it to *out and the step time to
 * *step_ms (either may be NULL); resets the statistics.  Allocates and
 * frees one scratch state; synchronises the stream.  Errors: GRIM_EINVAL,
 * GRIM_ECUDA, GRIM_ENOMEM; an unreadable or unwritable cache file is
 * ignored. */
int grim_autotune(grim_ctx* ctx, const double* P, double dt, const char* cache_path, grim_tuning* out,
                  double* step_ms);

/* enable != 0: grim_step (and grim_step_host) replays a CUDA graph of the
 * step's launches, captured on the second call with the same (P_in, P_out,
 * dt, tuning, learned guess); up to four graphs are kept per context.  The
 * first call after enabling runs eagerly.  Ignored while profiling
 * (grim_profile). */
int grim_use_graphs(grim_ctx* ctx, int enable);

/* ---- Batched boxes.  nbox independent grids (any sizes; one metric,
 * physics and solver) stepped together: each box has its own context; a
 * batched step forks the caller's stream onto up to 16 side streams, gives
 * box i the side stream i mod 16, and joins them back, so that small boxes
 * run concurrently.  From the second call on (graphs enabled, the default)
 * the whole batched step is one CUDA graph launch, captured per distinct
 * (P_in[], P_out[], dt[]) (two graphs kept: ping-pong buffers).  Results
 * equal grim_step on each box. */
typedef struct grim_batch grim_batch;

/* Create nbox contexts (grids[0..nbox-1]); errors as grim_init. */
int grim_batch_init(int nbox, const grim_grid* grids, const grim_metric* metric, const grim_physics* phys,
                    const grim_solver* solver, void* stream, grim_batch** out);
void grim_batch_destroy(grim_batch* batch);
/* The context of box i (for grim_set_guess, grim_set_tuning, grim_stage...);
 * owned by the batch. */
int grim_batch_context(grim_batch* batch, int i, grim_ctx** out);
/* One step of every box: P_in[i], P_out[i] device states of box i (P_out[i]
 * may equal P_in[i]), dt[i] its step; host arrays of nbox entries. */
int grim_batch_step(grim_batch* batch, const double* const* P_in, double* const* P_out, const double* dt);
int grim_batch_use_graphs(grim_batch* batch, int enable);
/* Counters summed over the boxes (max_res: the largest); launches counts the
 * kernels of batched steps.  Synchronises the stream. */
int grim_batch_get_stats(grim_batch* batch, grim_stats* out);
int grim_batch_reset_stats(grim_batch* batch);
const char* grim_batch_last_error(grim_batch* batch);

/* ---- Learned initial guess.  The paper starts each Newton solve from P_n
 * (§3); these calls add a small MLP that predicts the stage change of the
 * primitives, with P_n kept as the fallback.  Network 30 -> 128 -> 128 ->
 * 128 -> head (SiLU), bfloat16 weights, float32 accumulation, on the tensor
 * cores.  Features per zone (float32 [32]): x_a = -r_a(P_n), the scaled
 * residual of the stage at its start (a = 0..9: for the conserved rows the
 * explicit increment U* - U(P_n) in the residual's row scaling, for q~ and
 * dP~ the explicit part of their relaxation equations), the ten g_{mu nu},
 * P_n in the units below (log rho, log u, u^i, q~/(|q~| + rho),
 * dP~/(|dP~| + rho)), two zeros.  The head's
 * 80 outputs hold a 7x10 matrix M(x) (row-major) and an offset c(x); the
 * standardised prediction of the seven predicted fields is y = M x_U + c,
 * x_U the ten standardised increment features, so that the network learns a
 * state-dependent inverse Jacobian.  Targets (float32 [16]): the stage's
 * change P_conv - P_n of rho, u, u^i, q~, dP~ at indices 0-4, 8, 9 in units
 * of P_n for rho and u, |X_n| + rho_n for q~ and dP~ and 1 for u^i (the
 * magnetic field is the explicit flux-CT update, not predicted), zeros
 * elsewhere; the start is P_n + y times that unit.  These are the units the
 * scaled residual measures each field in, which keeps a torus and its
 * tenuous atmosphere, many orders of magnitude apart, in one
 * standardisation.  X and Y arrays are device, zone-major ([M][32], [M][16]). */
typedef struct grim_mlp grim_mlp;

/* Create an MLP with Kaiming-uniform weights from `seed`, zero biases, and an
 * identity standardisation.  Allocates device memory; synchronises. */
int grim_mlp_create(unsigned long long seed, grim_mlp** out);
void grim_mlp_destroy(grim_mlp* mlp);
/* Number of float32 parameters: W1[128][32], b1, W2[128][128], b2,
 * W3[128][128], b3, W4[80][128], b4[80], in that order (row-major). */
int grim_mlp_param_count(void);
/* Copy parameters (host float32 [param_count]) and the standardisation
 * (host float32 [96]: x_mean[32], x_std[32], y_mean[16], y_std[16]); either
 * pointer may be NULL.  set resets the Adam state.  Synchronous. */
int grim_mlp_get_params(grim_mlp* mlp, float* params, float* norm);
int grim_mlp_set_params(grim_mlp* mlp, const float* params, const float* norm);
/* Fit the standardisation to M training rows (per-column mean and standard
 * deviation; a constant feature column keeps unit deviation, a constant
 * target column gets deviation 0 and is predicted as its mean).
 * Synchronous. */
int grim_mlp_fit_norm(grim_mlp* mlp, const float* X, const float* Y, long long M);
/* `steps` Adam steps (lr; betas 0.9, 0.999; eps 1e-8) on minibatches of
 * `batch` rows (a multiple of 64) of the M training rows, visited in a fixed
 * permutation that starts at `seed` mod M; loss = mean squared error of the
 * standardised targets over the seven predicted fields.  *mean_loss: the
 * mean of the minibatch losses.  Synchronous. */
int grim_mlp_train(grim_mlp* mlp, const float* X, const float* Y, long long M, int batch, int steps, double lr,
                   unsigned long long seed, double* mean_loss);
/* Gradient of the loss over all M rows (M a multiple of 64, one batch) with
 * respect to the parameters, to host float32 [param_count]; *loss its value. */
int grim_mlp_gradient(grim_mlp* mlp, const float* X, const float* Y, long long M, float* grad, double* loss);
/* The training contraction on its own: C[M][N] = A[M][K] B[N][K]^T with A
 * and B bfloat16 device matrices, row-major with K contiguous (row strides
 * lda, ldb elements), accumulated in float32 by the tensor cores (tcgen05,
 * operands copied by TMA) into the float32 device matrix C (row stride
 * ldc).  splits: the number of slices of K summed in a fixed order after the
 * tensor-core pass (1..16; 0 = 1).  Requirements: M, K >= 1; N >= 16 and a
 * multiple of 16; lda, ldb multiples of 8 and >= K; ldc a multiple of 4 and
 * >= N; A, B, C 16-byte aligned (else GRIM_EINVAL).  Synchronous: allocates
 * and frees a small device workspace (GRIM_ENOMEM); GRIM_ECUDA when a
 * launch failed or a CTA gave up waiting for its copies or MMAs (C is then
 * incomplete). */
int grim_gemm_nt_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                      int splits);
/* Features (and, when P_conv and Y are non-NULL, targets) of every zone of
 * the stage whose explicit kernels ran last on ctx (grim_stage,
 * grim_residual or the full step of grim_step), with start-of-step state P_n
 * and converged state P_conv. */
int grim_mlp_sample(grim_ctx* ctx, const double* P_n, const double* P_conv, float* X, float* Y);
/* Start every later Newton solve of ctx from the MLP's prediction (NULL:
 * from P_n).  The learned start is kept when its max |r_a| <= accept; else
 * the plain start P_n is evaluated too and the smaller |r|^2 wins (counted
 * in grim_stats.fallbacks).  The MLP must outlive its use by ctx.  The first
 * call with an MLP allocates a feature buffer (10 floats per zone), which the
 * zone-constant kernel fills each stage on 2-D Minkowski grids and a feature
 * kernel (the stage's residual at P_n) in a general metric, where the metric
 * features are the zone's g_{mu nu}.  GRIM_ENOMEM. */
int grim_set_guess(grim_ctx* ctx, grim_mlp* mlp, double accept);

/* Self-check of the float64 reciprocal the kernels use for finite-difference
 * divisors and LU pivots (a Newton-Raphson refinement of the hardware
 * approximation): over n seeded values spanning magnitudes 2^-300..2^300 of
 * both signs, writes the largest relative difference from IEEE division to
 * *max_rel_err.  Allocates and frees a small device buffer; synchronises the
 * device. */
int grim_math_selftest(int n, double* max_rel_err);

#ifdef __cplusplus
}
#endif
#endif /* GRIM_H */
