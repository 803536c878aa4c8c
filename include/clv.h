/*
 * clv.h -- C ABI of the GB300 (sm_103a) library for the space-time evolution
 * of (3+1)D second-order viscous hydrodynamics in Milne coordinates
 * (tau, x, y, eta_s), the CLVisc method of Pang, Petersen and Wang.
 *
 * What one step computes (the paper's Sec. 2 and Sec. 3):
 *   state: T~^{tau mu} (4), pi~^{mu nu} (10 symmetric components) and the
 *   primitives eps, u~^x, u~^y, u~^eta of the tilde variables of Sec. 2;
 *   one Heun / two-stage Runge-Kutta step of Sec. 3 with
 *     - Kurganov-Tadmor central fluxes with a minmod limiter, Eqs. (kt),
 *       (flux_out),
 *     - the Milne geometric sources S_T and the Israel-Stewart shear source
 *       S_pi with the Christoffel terms I^{mu nu} of Eq. (Ipi),
 *     - the velocity predictor u* = 2u^n - u^{n-1} (first step from one ideal
 *       step),
 *     - recovery of (eps, u) from T_ideal = T - pi by a per-cell root solve
 *       with an equation-of-state table,
 *     - the vacuum cutoff eps < eps_cut -> eps = 0 (Sec. 5).
 *
 * Conventions shared by every entry point:
 *   - Grid arrays are (nx, ny, neta) in C order, eta_s fastest; cell centres
 *     are x_i = (i - (nx-1)/2) dx, likewise for y and eta_s.
 *   - Units: fm, GeV/fm^3, GeV.
 *   - Host arrays are owned by the caller and only read or written during
 *     the call.  Device memory is owned by the handle (or by the caller when
 *     a workspace is passed to clv_create_ws).
 *   - Every call returns a status and never aborts the process.  A failing
 *     call leaves a message for clv_last_error.  Kernel-side errors (root
 *     solve cap, non-finite values) accumulate in a device word that the next
 *     synchronising call reports.
 *   - A handle is used by one host thread at a time.  All work is enqueued
 *     on the stream given at creation; calls that return host data
 *     synchronise that stream.
 */
#ifndef CLV_H
#define CLV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CLV_OK = 0,
  CLV_EINVAL = 1,      /* invalid argument or configuration */
  CLV_ENOMEM = 2,      /* device allocation failed / workspace too small */
  CLV_ECUDA = 3,       /* a CUDA runtime call failed */
  CLV_EROOT = 4,       /* a primitive root solve hit its iteration cap */
  CLV_ENONFINITE = 5,  /* a non-finite value appeared in the state */
  CLV_ETIMEOUT = 6     /* a bounded device wait gave up */
} clv_status;

enum { CLV_FP64 = 0, CLV_FP32 = 1 };
enum { CLV_EOS_CONFORMAL = 0, CLV_EOS_TABLE = 1 };

/* Run configuration.  Pointers are read during clv_create only. */
typedef struct {
  int nx, ny, neta;          /* cells per axis, each >= 1 */
  double dx, dy, deta;       /* spacings (fm, fm, 1) */
  double tau0, dtau;         /* initial proper time and step h (fm) */
  double eta_over_s;         /* shear viscosity over entropy; 0 = ideal (pi ignored) */
  int eos_kind;              /* CLV_EOS_CONFORMAL: P = eps/3, eps = 3 g pi^2 T^4/90 (hbar c)^3, g = 47.5
                                CLV_EOS_TABLE: P, T, c_s^2 tabulated at nodes uniform in ln eps */
  int eos_n;                 /* number of table nodes (>= 2) */
  double eos_lne0;           /* ln(eps) of node 0 */
  double eos_dlne;           /* node spacing in ln(eps) */
  const double* eos_P;       /* host, eos_n values; copied */
  const double* eos_T;       /* host, eos_n values (GeV); copied */
  const double* eos_cs2;     /* host, eos_n values; copied */
  int precision;             /* CLV_FP64 or CLV_FP32 (FP32 stencil, sources, pi~ and primitives; the
                                conserved T~^{tau mu} as float-float pairs, ~48 bits, accumulated
                                exactly and read by the root solve unrounded; float-float Newton
                                correction of every root, FP64 root polish near vacuum and at high
                                velocity; FP64 reductions) */
  int cartesian;             /* 1: Christoffel terms off and tau factors 1 (t, x, y, z) */
  int periodic;              /* 1: periodic boundaries; 0: zero-gradient (outflow) */
  double eps_cut;            /* vacuum cutoff, GeV/fm^3 (the paper uses 1e-7) */
  int kernel;                /* 0: tiled stage kernel (default); 1: direct per-cell stage kernel
                                (same arithmetic, simpler data flow; kept for cross-checks) */
  double taupi_coef;         /* b in tau_pi = b eta_v / (eps + P); 0 means 5 (the paper's choice) */
  double lambda1_hat;        /* lambda_1 = lambda1_hat / eps in Eq. (pimn) (conformal scaling);
                                0: no lambda_1 term (the default) */
  int halo_x;                /* 0: the whole grid (default); 2: an x-slab of a larger grid with two halo
                                planes on each x side, filled by the caller (clv_slab_*) */
  int charge;                /* 1: also transport a net charge (Eq. Ntilde, S_N = 0, no diffusion
                                current; the paper runs with n = 0): N~^tau = tau n u~^tau, set by
                                clv_set_initial_n; single events only (not a batch or an x-slab) */
  double zeta_over_s;        /* bulk viscosity over entropy (Eqs. Pi, Pitilde, tau_Pi = 5 zeta/(T s));
                                0: no bulk pressure (the paper's setting).  > 0 needs eta_over_s > 0
                                and a single event (not a batch or an x-slab).  Pi = 0 at tau0; it
                                relaxes by S_Pi = -(Pi + zeta theta)/tau_Pi - Pi theta/3 - Pi u^tau/tau
                                (theta = nabla_mu u^mu), is carried by the flux v^a u~^tau Pi and adds
                                to the pressure of T^{mu nu} (fluxes, S_T, the root solve) */
} clv_config;

/* Per-run statistics, filled by clv_step / clv_get_stats. */
typedef struct {
  double tau;                /* proper time after the last step */
  int64_t step;              /* completed steps */
  double eps_max;            /* max eps over the grid (GeV/fm^3) */
  double T_max;              /* temperature at eps_max (GeV); stopping rule input */
  double E_tot;              /* sum of T~^{tau tau} dx dy deta, FP64 accumulated */
  int64_t n_rescaled;        /* cells with |M| > E rescaled before the root solve */
  int64_t n_rootfail;        /* root solves that hit the iteration cap */
  int64_t n_polished;        /* FP32 path: cells refined by the FP64 Newton step */
  int64_t n_fp32_nonconverged; /* FP32 path: FP32 root solves that did not converge (then solved in FP64) */
  int64_t n_newton_iters;    /* Newton iterations of the root solves (working precision) */
  int64_t n_newton_cells;    /* root solves counted in n_newton_iters */
  int64_t n_polish_iters;    /* FP32 path: FP64 Newton iterations of the n_polished refinements */
  int64_t n_newton_warp_max; /* sum over warps of the largest Newton iteration count in the warp
                                (the divergence cost: a warp runs as long as its slowest lane) */
  int64_t n_newton_warps;    /* warps counted in n_newton_warp_max */
  uint32_t error_word;       /* bit 0 root cap, bit 1 non-finite, bit 2 wait timeout */
  uint32_t _pad;
} clv_stats;

typedef struct clv_handle clv_handle;

/* Device bytes a handle needs for this configuration (fields, stage buffers,
 * EOS table, reduction scratch).  Returns CLV_EINVAL for a bad config. */
clv_status clv_workspace_bytes(const clv_config* cfg, size_t* bytes);

/* Create a handle.  cuda_stream is a cudaStream_t (NULL = default stream).
 * The library allocates the device workspace itself. */
clv_status clv_create(const clv_config* cfg, void* cuda_stream, clv_handle** out);

/* Same, with a caller-owned device workspace of at least
 * clv_workspace_bytes bytes, 256-byte aligned, that must outlive the handle. */
clv_status clv_create_ws(const clv_config* cfg, void* cuda_stream, void* device_ws,
                         size_t ws_bytes, clv_handle** out);

/* Load the initial state at tau0 from primitives.  eps, ux, uy, ueta: host
 * arrays of nx*ny*neta doubles (u~^eta = tau u^eta); pi: host array of
 * 10*nx*ny*neta doubles (components tt tx ty te xx xy xe yy ye ee of pi~,
 * each a full grid) or NULL for pi = 0.  Cells with eps < eps_cut become
 * vacuum.  For eta_over_s > 0 this also runs the pi-free first step that
 * fixes u^{-1} (Sec. 3).  Resets tau and the step count. */
clv_status clv_set_initial(clv_handle* h, const double* eps, const double* ux, const double* uy,
                           const double* ueta, const double* pi);

/* Same as clv_set_initial with the five inputs already in device memory
 * (doubles, same layout); nothing is copied from the host. */
clv_status clv_set_initial_device(clv_handle* h, const double* d_eps, const double* d_ux,
                                  const double* d_uy, const double* d_ueta, const double* d_pi);

/* Initial state from T^{tau mu} with pi = 0 (mini-jet initial flow):
 * T holds 4 x N doubles, component-major in the cell order of
 * clv_set_initial: T^{tau tau}, T^{tau x}, T^{tau y} and the orthonormal
 * tau T^{tau eta} (GeV/fm^3) at tau0.  The primitives are the FP64 root of
 * the recovery problem of Sec. 3 with E = T^{tau tau}, M = T^{tau i}
 * (vacuum where the solved eps < eps_cut); the run then starts as from
 * clv_set_initial with those primitives.  CLV_ENONFINITE for non-finite
 * input, CLV_EROOT if a solve hit its cap.  Synchronises the stream.
 * _device: T is a device array. */
clv_status clv_set_initial_T(clv_handle* h, const double* T);
clv_status clv_set_initial_T_device(clv_handle* h, const double* d_T);

/* Net charge density n (fm^-3) at the current tau, for a handle created
 * with charge = 1, after clv_set_initial(_T): N~^tau = tau n u~^tau from the
 * current velocities (host array, or device array for _device, of
 * nx*ny*neta doubles).  From then on each step carries N~^tau with the flux
 * v^a N~^tau through the same limited reconstruction and local speed as the
 * other fields (one extra launch per stage).  clv_set_initial(_T) resets
 * the charge to zero (not transported).  CLV_EINVAL without charge = 1 or
 * before the initial state. */
clv_status clv_set_initial_n(clv_handle* h, const double* n);
clv_status clv_set_initial_n_device(clv_handle* h, const double* d_n);

/* Advance nsteps Heun steps.  If stats is not NULL the call synchronises and
 * fills it; otherwise it only enqueues work and returns.  Returns CLV_EROOT /
 * CLV_ENONFINITE when the device error word is set (checked only when stats
 * is requested). */
clv_status clv_step(clv_handle* h, int nsteps, clv_stats* stats);

/* Synchronise and report statistics of the current state. */
clv_status clv_get_stats(clv_handle* h, clv_stats* stats);

/* Field indices for clv_get_fields (bit i of the mask selects field i):
 *   0 eps, 1 u~^x, 2 u~^y, 3 u~^eta,
 *   4..7 T~^{tau mu} (mu = tau, x, y, eta),
 *   8..17 pi~ (tt tx ty te xx xy xe yy ye ee),
 *   18..20 u~^{x,y,eta} of the previous step,
 *   21 N~^tau and 22 n = N~^tau / (tau u~^tau) (charge = 1 only; CLV_EINVAL otherwise),
 *   23 the bulk pressure Pi (GeV/fm^3; zeta_over_s > 0 only; CLV_EINVAL otherwise).
 * host_out receives popcount(mask) grids of nx*ny*neta doubles, in
 * increasing field order.  Synchronises. */
clv_status clv_get_fields(clv_handle* h, uint32_t mask, double* host_out);

/* Same into device memory (doubles); enqueued, no synchronisation. */
clv_status clv_get_fields_device(clv_handle* h, uint32_t mask, double* device_out);

/* Proper time and step count of the current state (host-side bookkeeping). */
clv_status clv_get_time(const clv_handle* h, double* tau, int64_t* step);

/* Instrumentation.  While enabled, CUDA events are recorded on the handle's
 * stream around every kernel launch of clv_step (at most 8192 steps between
 * two reads).  clv_get_kernel_times synchronises and returns the accumulated
 * device milliseconds and launch counts per kernel, then resets them:
 * index 0 stage-1 stage kernel, 1 stage-1 recovery kernel, 2 stage-2 stage
 * kernel, 3 stage-2 recovery kernel (1 and 3 stay 0 with kernel = 1, whose
 * stage kernel includes the recovery).  With zeta_over_s > 0 the bulk kernel
 * of a stage is counted in that stage's stage-kernel slot; with charge = 1 the
 * charge kernel of stage 1 falls in slot 2, and that of stage 2, like the tau
 * advance, in none. */
clv_status clv_enable_kernel_timing(clv_handle* h, int enable);
clv_status clv_get_kernel_times(clv_handle* h, double ms[4], int64_t launches[4]);

/* Measurement (no counterpart in the paper): the fused multiply-add rate of
 * the current device in TFLOP/s (an FMA counts as 2 flops) for precision
 * CLV_FP64 or CLV_FP32, from independent FMA chains on 8 CTAs of 256
 * threads per SM, the best of three timed launches after a warm-up one.  It
 * is the peak of the ALU rooflines (the FP64 path, the Cooper-Frye sum).
 * Allocates and frees a small device buffer; runs on the legacy default
 * stream and synchronises.  CLV_EINVAL for another precision or a NULL
 * tflops, CLV_ECUDA on a CUDA error. */
clv_status clv_fma_rate(int precision, double* tflops);

/* ---------------- learned initial guess of the root solve ----------------
 * Not in the paper (which notes that the varying iteration counts of the
 * root finding make warps diverge): a 10 -> 64 -> 64 -> 4 SiLU network maps
 * features of a cell to (eps/E, v^x, v^y, v^eta); |v| seeds the Newton solve,
 * which then converges to the same tolerance as without it.  Features:
 * x0 = (ln E + 5)/5, x1..3 = M^{x,y,eta}/E, x4..9 = pi~^{xx,xy,x eta,yy,y eta,
 * eta eta}/E clamped to [-4, 4], with E, M the ideal part T~^{tau mu}/tau -
 * pi~^{tau mu} the root solve starts from.  Parameters: 5124 floats packed
 * W1 (64x10, row-major) | b1 (64) | W2 (64x64) | b2 (64) | W3 (4x64) | b3 (4).
 * Inference: BF16 weights on the tensor cores, FP32 accumulation. */
enum { CLV_GUESS_PREVIOUS = 0, CLV_GUESS_COLD = 1, CLV_GUESS_MLP = 2, CLV_GUESS_MLP_ALL = 3 };
#define CLV_MLP_NPARAM 5124

/* Initial guess of the root solve (Sec. 3 primitive recovery; the guess only
 * sets where Newton starts, the root is solved to the same tolerance):
 * CLV_GUESS_PREVIOUS (|v| of the cell's stage velocity; the default),
 * CLV_GUESS_COLD (v = M/(E + P(E))), CLV_GUESS_MLP (the network for cells
 * that were vacuum in the stage's input, whose stage velocity is the
 * vacuum's 0; the stage velocity elsewhere) or CLV_GUESS_MLP_ALL (the network
 * for every cell).  The two network modes need clv_set_mlp and the FP32 path;
 * other modes or precisions return CLV_EINVAL. */
clv_status clv_set_guess(clv_handle* h, int mode);

/* Load the network (host array of CLV_MLP_NPARAM floats; converted to BF16). */
clv_status clv_set_mlp(clv_handle* h, const float* params);

/* Training samples of the current state: features (d_X, 10 floats a row)
 * and targets (d_Y, 4 floats a row: eps/E, v^x, v^y, v^eta) of every
 * non-vacuum cell, compacted in cell order; *d_count (device int64) receives
 * the number of rows.  d_X and d_Y must hold N rows.  Device arrays;
 * enqueued on the handle's stream (which also uses the handle's host
 * staging buffer as scratch). */
clv_status clv_mlp_samples(clv_handle* h, float* d_X, float* d_Y, int64_t* d_count);

/* The tensor-core forward pass of the loaded network on n feature rows
 * (device, n x 10 floats) into d_Y (n x 4 floats).  Enqueued.  The arrays
 * may be null when n = 0. */
clv_status clv_mlp_forward(clv_handle* h, const float* d_X, int64_t n, float* d_Y);

/* Loss (mean over samples of the squared error summed over the 4 outputs)
 * and its gradient with respect to the packed parameters, over n device
 * samples, in FP32.  d_grad: CLV_MLP_NPARAM floats, d_loss: 1 float
 * (both overwritten).  d_work: CLV_MLP_PARTIAL_FLOATS floats of device
 * scratch (per-block partial sums, added in a fixed order, so the result is
 * bitwise reproducible).  Enqueued on cuda_stream. */
#define CLV_MLP_PARTIAL_FLOATS (256 * (CLV_MLP_NPARAM + 1))
clv_status clv_mlp_loss_grad(const float* d_params, const float* d_X, const float* d_Y, int64_t n,
                             void* cuda_stream, float* d_grad, float* d_loss, float* d_work);

/* iters Adam steps (lr, beta 0.9/0.999) on mini-batches of `batch` samples
 * drawn from the n device samples by a counter-based generator (seed != 0).
 * d_params is updated in place; d_work holds CLV_MLP_TRAIN_WORK_FLOATS floats:
 * the Adam moments (zero before the first call, kept between calls), the
 * gradient and the per-block partial sums of the deterministic gradient
 * reduction; step0 continues the Adam step count; d_loss[i] receives the
 * mini-batch loss of step i.  The same inputs give the same parameters bit
 * for bit.  Enqueued on cuda_stream. */
#define CLV_MLP_TRAIN_WORK_FLOATS (3 * CLV_MLP_NPARAM + CLV_MLP_PARTIAL_FLOATS)
clv_status clv_mlp_train(float* d_params, float* d_work, const float* d_X, const float* d_Y, int64_t n,
                         int iters, int batch, float lr, uint64_t seed, int step0, void* cuda_stream,
                         float* d_loss);

/* ---------------- batch of events ----------------
 * Many independent events of different grids (and eta/s) in one handle:
 * their fields are stored back to back, each stage is one persistent launch
 * whose CTAs take (event, tile-chunk) work items, most expensive first, and
 * the root solve is one launch over all cells.  The events must share tau0,
 * dtau, precision, the EOS, eps_cut, the coordinates and the boundaries
 * (kernel 0); they may differ in nx, ny, neta, dx, dy, deta and eta/s.
 * clv_step, the guess calls, clv_get_stats (E_tot = 0: per event below),
 * clv_get_state / clv_set_state and clv_get_fields (all events back to back)
 * take a batch handle; clv_set_initial(_T) and clv_set_tile do not
 * (CLV_EINVAL).  The batch starts (first-step predictor) at the first
 * clv_step, after every event's initial state was set.
 * Each event's tile follows a tiling policy shared by the batch: at most
 * max_threads threads per CTA (TJ as large as that allows, TK from neta, at
 * most 32 columns) and x chunks of about `chunk` planes; the default is 384
 * (128 in FP64) threads and 32 planes.  The persistent stage launch holds as
 * many CTAs per SM as the device's occupancy calculator allows for the
 * policy's largest tile.  clv_autotune on a started batch
 * times the current policy and up to max_candidates others (thread caps of
 * 1, 3/4 and 1/2 of the limit, chunks of 16-64 planes; reps stage-1 launches
 * each, which leave the state unchanged), keeps the fastest (the current
 * unless another is at least 2% faster) and reports it in clv_tile_info as
 * TJ = max_threads, TK = 0, CX = chunk.  The policy changes no result. */
clv_status clv_create_batch(const clv_config* cfgs, int nevents, void* cuda_stream, clv_handle** out);

/* Number of events and total cells of a batch (0 events for a single event). */
clv_status clv_batch_size(const clv_handle* h, int* nevents, int64_t* cells);

/* Initial state of one event, as clv_set_initial (host arrays of that
 * event's nx*ny*neta cells).  CLV_EINVAL once the batch has started. */
clv_status clv_batch_set_initial(clv_handle* h, int event, const double* eps, const double* ux,
                                 const double* uy, const double* ueta, const double* pi);

/* Fields of one event, as clv_get_fields (host). */
clv_status clv_batch_get_fields(clv_handle* h, int event, uint32_t which_mask, double* host_out);

/* eps_max, T_max and E_tot of one event (the counters are the batch's).
 * Synchronises the stream. */
clv_status clv_batch_event_stats(clv_handle* h, int event, clv_stats* out);

/* Explicit tiling policy of a batch (see above): max_threads in [32, 384]
 * (capped at 128 in FP64), chunk in [1, 4096] planes.  CLV_EINVAL if out of
 * range, not a batch, or if a tile would exceed the shared memory of a CTA.
 * Synchronises the stream. */
clv_status clv_batch_set_schedule(clv_handle* h, int max_threads, int chunk);

/* ---------------- x-slab of a larger grid (halo_x = 2) ----------------
 * One event split into slabs along x (one per GPU): each handle owns nx
 * consecutive x planes (nx >= 2) plus two halo planes on each x side, which
 * the caller fills before each stage: from the neighbouring slab
 * (clv_slab_pack on the neighbour, a transfer, clv_slab_unpack here) or, at
 * the ends of the global grid, by clv_slab_fill_edge (zero gradient).
 * set 1 = the inputs of stage 1 (T~, pi~, u~, P, c_s of the step), set 2 =
 * those of stage 2 (the stage-1 results).  side 0 = low x, 1 = high x.  A
 * packed side (the two boundary planes of every field of the set, in the
 * working precision; FP32: the low parts of T~ too) holds
 * clv_slab_halo_bytes bytes of device memory; pack(side 1) of the left
 * neighbour fills unpack(side 0) here and vice versa.  Stepping:
 *   after clv_set_initial, viscous runs:  for s in 1, 2: fill set s; clv_slab_predictor(s)
 *   every step:                           for s in 1, 2: fill set s; clv_stage(s)
 * clv_step refuses an x-slab.  All calls enqueue on the handle's stream. */
clv_status clv_slab_halo_bytes(const clv_handle* h, size_t* bytes);
clv_status clv_slab_pack(clv_handle* h, int set, int side, void* d_buf);
clv_status clv_slab_unpack(clv_handle* h, int set, int side, const void* d_buf);
clv_status clv_slab_fill_edge(clv_handle* h, int set, int side);
/* Stage 1 or 2 of the first-step predictor (Sec. 3) of a viscous x-slab. */
clv_status clv_slab_predictor(clv_handle* h, int stage);
/* Stage 1 or 2 of the current step; stage 2 completes it (and, with stats,
 * reduces them over the handle's cells and synchronises). */
clv_status clv_stage(clv_handle* h, int stage, clv_stats* stats);

/* ---------------- checkpoint ----------------
 * The complete evolution state: T~^{tau mu} (FP32: its float-float pairs),
 * pi~^{mu nu} and the primitives (eps, u~, P, c_s) of the current and the
 * previous step in the working precision, with tau, the step count and the
 * configuration it belongs to.
 * Restoring it into a handle of the same configuration continues the run
 * bit for bit.  Buffers are host memory of clv_state_bytes bytes, owned by
 * the caller; both calls synchronise the stream.  clv_set_state returns
 * CLV_EINVAL for a buffer of another configuration and resets the counters. */
clv_status clv_state_bytes(const clv_handle* h, size_t* bytes);
clv_status clv_get_state(clv_handle* h, void* buf, size_t bytes);
clv_status clv_set_state(clv_handle* h, const void* buf, size_t bytes);

/* Step graphs (on by default): clv_step replays pairs of plain steps from a
 * CUDA graph captured once per handle and buffer parity (tau lives on the
 * device, so the launches of a step are the same every step).  The step that
 * reduces statistics and timed steps (clv_enable_kernel_timing) are launched
 * directly.  Results are the same bit for bit either way. */
clv_status clv_set_graphs(clv_handle* h, int enable);

/* ---------------- tile shape of the stage kernel ----------------
 * The stage kernel works on (y, eta_s) tiles of TJ x TK cells, each CTA
 * marching along x over CX planes ((TJ + 1)(TK + 1) threads per CTA).  The
 * shape changes no result, only the speed. */
typedef struct {
  int TJ, TK, CX;            /* tile rows (y), columns (eta_s), planes per CTA (x) */
  int threads;               /* threads per CTA */
  int blocks;                /* CTAs per stage launch */
  int smem_bytes;            /* dynamic shared memory per CTA */
  double ms;                 /* clv_autotune: mean stage-1 time of the chosen shape (ms) */
} clv_tile_info;

clv_status clv_get_tile(clv_handle* h, clv_tile_info* out);

/* Explicit shape; CX = 0 picks the x chunking by the makespan rule (with as
 * many CTAs per SM as the occupancy calculator allows at this shape).
 * CLV_EINVAL if out of range or beyond the thread limit ((TJ + 1)(TK + 1) <=
 * 384 in FP32, 128 in FP64) or the 227 KiB shared-memory limit of a CTA. */
clv_status clv_set_tile(clv_handle* h, int TJ, int TK, int CX);

/* Autotuner: times the current shape and up to max_candidates modelled-best
 * shapes (reps stage-1 launches each, on the current state, which they leave
 * unchanged) on the handle's stream, keeps the fastest (the current shape
 * unless another is at least 2% faster) and reports it in *best (nullable).
 * Needs clv_set_initial; synchronises the stream. */
clv_status clv_autotune(clv_handle* h, int max_candidates, int reps, clv_tile_info* best);

/* Statistics without any allocation.  The paper has no counterpart: this is
 * a service for callers that cannot allocate device memory -- code running
 * under a fixed device-memory budget owned by another framework's pool, or in
 * a loop whose contract forbids allocations between its timing points.
 *
 * Computes, over caller-owned device arrays of n doubles (e.g. fields 0 and 4
 * exported by clv_get_fields_device), the same two statistics as
 * clv_get_stats: d_out[0] = cell_volume * sum of d_Ttt (E_tot) and
 * d_out[1] = max of d_eps (negative values count as 0).  d_out is a device
 * array of 2 doubles written on cuda_stream; the call only enqueues work and
 * does not synchronise.
 *
 * Scratch lives in a fixed array of the library (256 KiB + 8 bytes on every
 * device that loads it, held until the process exits); nothing is allocated
 * and no allocating library routine is called.  Limit: 1 <= n <= 8388608;
 * larger n returns CLV_EINVAL with a message in clv_last_error(NULL).
 * The first call on each device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  That address is cached per device for the life
 * of the process: do not call this entry point on a device after
 * cudaDeviceReset on it.  An error already pending in the CUDA runtime when
 * the call starts returns CLV_ECUDA without launching anything (and stays
 * pending).  Every call shares the scratch array: calls that overlap on the
 * GPU (other streams or host threads on the same device) race and must be
 * serialised by the caller. */
clv_status clv_field_stats_noalloc(const double* d_eps, const double* d_Ttt, int64_t n, double cell_volume,
                                   void* cuda_stream, double* d_out);

/* ---------------- freeze-out hypersurface ----------------
 * Surface elements dSigma_mu of the hypersurface eps = eps_f between two
 * time slices: the input of the Cooper-Frye integral, Eq. (cooper_frye) of
 * Sec. 4 (a constant T_f is a constant eps_f through the monotone equation
 * of state).  The paper runs its surface finder on the GPU (appendix on the
 * parallel reduction) and cites it without describing it.  Here the surface
 * is the level set of the piecewise-linear interpolant of eps over the
 * Freudenthal triangulation of every space-time hypercube:
 *   - hypercube (i, j, k) has its 16 corners at the cell centres i..i+1,
 *     j..j+1, k..k+1 of both slices: (nx-1)(ny-1)(neta-1) hypercubes;
 *   - it is cut into the 24 4-simplices of the orderings of the axes
 *     (tau, x, y, eta_s).  Inside a simplex the level set is a planar
 *     tetrahedron or triangular prism.  A corner is inside when eps >= eps_f;
 *   - dSigma_mu sums, over the pieces, -grad_mu eps / |grad eps| times the
 *     integral of tau over the piece (1 in Cartesian mode).  The geometry
 *     is taken in the coordinates (tau, x, y, eta_s) as R^4;
 *   - dSigma_mu is covariant, with dSigma_eta in fm^4.  It points to lower
 *     eps, so p^mu dSigma_mu > 0 for outgoing particles;
 *   - each crossed hypercube gives one element, placed at the
 *     3-volume-weighted mean of the piece centroids;
 *   - u~ and pi~ are interpolated at that point by the same interpolant, and
 *     u~^tau = sqrt(1 + u~_x^2 + u~_y^2 + u~_eta^2).
 * Element record: CLV_FO_NREC values of the slices' type, in this order:
 *   dSigma_tau, dSigma_x, dSigma_y, dSigma_eta, tau, x, y, eta_s,
 *   u~^tau, u~^x, u~^y, u~^eta, pi~ (tt tx ty te xx xy xe yy ye ee).
 * Elements come in increasing hypercube order ((i (ny-1) + j)(neta-1) + k);
 * the result does not depend on the launch. */
#define CLV_FO_NREC 22

typedef struct {
  int nx, ny, neta;          /* cells per axis of each slice, each >= 2; cell centres as in clv_config */
  int eta_pitch;             /* elements between consecutive eta rows (>= neta; 0 means neta) */
  double dx, dy, deta;       /* spacings (> 0) */
  int precision;             /* CLV_FP64: slice arrays and records are doubles; CLV_FP32: floats */
  int cartesian;             /* 1: no tau weight (coordinates t, x, y, z) */
} clv_fo_grid;

typedef struct {
  double tau;                /* proper time of the slice (> 0 unless cartesian) */
  const void* eps;           /* device array, nx*ny*eta_pitch values, eta_s fastest */
  const void* u[3];          /* u~^x, u~^y, u~^eta (device, same layout) */
  const void* pi[10];        /* pi~ tt..ee (device, same layout); all NULL means pi = 0 */
} clv_fo_slice;

/* Device scratch bytes that clv_fo_find needs for this grid. */
clv_status clv_fo_scratch_bytes(const clv_fo_grid* g, size_t* bytes);

/* Elements of eps = eps_f between the slices s0 and s1 (s1->tau > s0->tau).
 *   d_rec     device array of `capacity` records; records past capacity are not written;
 *   d_cube    nullable device int64 array of `capacity` hypercube indices;
 *   d_count   device int64; receives the number of elements, which may exceed capacity;
 *   d_scratch clv_fo_scratch_bytes bytes of device memory, 16-byte aligned.
 * Enqueued on cuda_stream (a cudaStream_t; NULL is the default stream); it
 * does not synchronise.  CLV_EINVAL for a bad argument: clv_last_error(NULL)
 * names it. */
clv_status clv_fo_find(const clv_fo_grid* g, const clv_fo_slice* s0, const clv_fo_slice* s1, double eps_f,
                       void* d_rec, int64_t* d_cube, int64_t capacity, int64_t* d_count, void* d_scratch,
                       void* cuda_stream);

/* The grid of a single-event handle (not a batch or an x-slab) and a slice
 * viewing its current state: eps, u~ and pi~ in the working precision at the
 * handle's tau.  The view is valid until the next step. */
clv_status clv_fo_grid_of(clv_handle* h, clv_fo_grid* out);
clv_status clv_fo_current(clv_handle* h, clv_fo_slice* out);

/* Device bytes of one slice copy.  clv_fo_snapshot copies the current slice
 * into d_buf (that many bytes, 256-byte aligned, caller-owned), enqueued on
 * the handle's stream; *out views the copy. */
clv_status clv_fo_slice_bytes(clv_handle* h, size_t* bytes);
clv_status clv_fo_snapshot(clv_handle* h, void* d_buf, clv_fo_slice* out);

/* ---------------- smooth Cooper-Frye spectra ----------------
 * The invariant momentum distribution of hadron species from freeze-out
 * surface elements, Sec. 4, Eqs. (cooper_frye) and (feq):
 *   dN/(dY pT dpT dphi) = g / (2 pi hbar c)^3  sum over elements of
 *                         p^mu dSigma_mu f_eq (1 + delta f),
 *   f_eq    = 1 / (exp[(p.u - mu)/T_f] + s),
 *   delta f = (1 - s f_eq) p_mu p_nu pi^{mu nu} / (2 T_f^2 (eps + P)),
 * with s = +1 (Fermi-Dirac), -1 (Bose-Einstein) or 0 (Boltzmann), in GeV^-2.
 *   - The elements are clv_fo_find records (CLV_FO_NREC values each).
 *   - Momentum at the element's eta_s: p^tau = mT cosh(Y - eta_s),
 *     tau p^eta = mT sinh(Y - eta_s), p^x = pT cos phi, p^y = pT sin phi.
 *   - p.u and p_mu p_nu pi^{mu nu} are taken in the tilde components of u~
 *     and pi~ (metric diag(1, -1, -1, -1)).
 *   - Elements with p^mu dSigma_mu < 0 are summed as they are.
 * The spectrum is evaluated at the points of a (Y, pT, phi) grid; the paper
 * uses 41 x 15 x 48 points, with pT and phi at Gauss quadrature nodes.
 * Several species share one pass over the elements (up to
 * CLV_CF_MAX_SPECIES per call). */
#define CLV_CF_MAX_SPECIES 32

typedef struct {
  double mass;               /* GeV, >= 0 */
  double g;                  /* degeneracy, > 0 */
  int stat;                  /* +1 Fermi-Dirac, -1 Bose-Einstein, 0 Boltzmann */
  double mu;                 /* chemical potential, GeV */
} clv_cf_species;

typedef struct {
  double Tf;                 /* freeze-out temperature, GeV (> 0) */
  double ePf;                /* eps + P at the freeze-out, GeV/fm^3 (> 0 when viscous) */
  int viscous;               /* 1: include delta f from the elements' pi~ */
  int precision;             /* CLV_FP64 or CLV_FP32: the type of the records; FP32 sums each
                                tile of 128 elements in FP32 and the tiles in FP64 */
} clv_cf_params;

/* Device scratch bytes of clv_cf_spectra for these sizes. */
clv_status clv_cf_scratch_bytes(const clv_cf_params* p, int64_t nel, int nsp, int nY, int npt, int nphi,
                                size_t* bytes);

/* Spectra of nsp species (host array) into d_out: nsp x nY x npt x nphi
 * doubles on the device, in the order [species][Y][pT][phi].
 *   d_rec          device records of the elements (type per p->precision);
 *   nel            number of records, or an upper bound when d_nel is given;
 *   d_nel          nullable device int64: the number of records (for example
 *                  the d_count of clv_fo_find), read on the device and
 *                  capped at nel, so nothing is synchronised;
 *   d_Y, d_pT, d_phi  device arrays (doubles) of the grid axes;
 *   d_scratch      clv_cf_scratch_bytes bytes of device memory, 256-byte aligned.
 * The sum over elements is deterministic (fixed order).  Enqueued on
 * cuda_stream; CLV_EINVAL for a bad argument (clv_last_error(NULL)). */
clv_status clv_cf_spectra(const clv_cf_params* p, const clv_cf_species* species, int nsp, const void* d_rec,
                          int64_t nel, const int64_t* d_nel, const double* d_Y, int nY, const double* d_pT, int npt,
                          const double* d_phi, int nphi, double* d_out, void* d_scratch, void* cuda_stream);

/* Release the handle and the memory it owns.  NULL is ignored. */
void clv_destroy(clv_handle* h);

/* Message of the last failing call on this handle ("" if none).  With
 * h == NULL: the last failure of a call without a handle (clv_create,
 * clv_create_ws, clv_workspace_bytes, clv_field_stats_noalloc, clv_fo_*, clv_cf_*). */
const char* clv_last_error(const clv_handle* h);

/* Library version string. */
const char* clv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CLV_H */
