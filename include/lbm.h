/*
 * lbm.h -- C ABI of liblbm.so, a GB300 (sm_103a) implementation of the
 * coupled central-moment lattice Boltzmann method of Schupbach & Premnath,
 * "A Robust Lattice Boltzmann Method for Interface-Bound Transport of a
 * Passive Scalar: Application to Surfactant-Laden Multiphase Flows"
 * (arXiv 2504.09024).
 *
 * One time step advances three D2Q9 lattices:
 *   f  conservative Allen-Cahn phase field phi          (App. C, Eq. LBE_CACE)
 *   h  interface-bound surfactant concentration c       (Sec. 3, Eq. LBE)
 *   g  pressure-based two-fluid flow P, u, forced by the
 *      capillary + Marangoni stress of Eq. (Fs) with the
 *      Langmuir isotherm sigma(c) of Eq. (EOS)          (App. D, Eq. centralmomentLBE2fluidflow)
 *
 * Conventions shared by every entry point
 *   - Grids are nx by ny cells; cell (i, j) has centre (i + 1/2, j + 1/2).
 *     Host and device field arrays are row-major [ny][nx] float64, x fastest.
 *     Population arrays are [9][ny][nx] float64 in the D2Q9 order of the
 *     paper's P matrix (App. A): 0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1)
 *     5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1).
 *   - x is periodic.  y is periodic (walls_y = 0) or bounded by half-way
 *     bounce-back walls at y = 0 and y = ny moving with -u_wall and +u_wall.
 *   - Units are lattice units (dx = dt = 1, cs^2 = 1/3).
 *   - The library owns all device memory of a context.  Pointers passed in
 *     are borrowed for the duration of the call only.
 *   - Every int-returning function returns LBM_OK (0) or a negative LBM_ERR_*
 *     code; no exception or abort crosses the ABI.  lbm_strerror() names it.
 *   - Work runs on the stream given to lbm_create (NULL: the library's own
 *     non-blocking stream).  lbm_step is asynchronous; functions that return
 *     data to the host synchronise that stream.  A CUDA error inside an
 *     asynchronous call is reported by the next call that synchronises.
 *   - A context is not thread-safe: calls on one context must be serialised.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 1

enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = -1,  /* bad pointer, size or parameter */
    LBM_ERR_RATE = -2,         /* a transport coefficient gives a relaxation rate outside (0, 2) */
    LBM_ERR_SIGMA_NEG = -3,    /* Langmuir sigma(c) < 0 for the declared concentration range */
    LBM_ERR_CUDA = -4,         /* CUDA runtime error (device, launch, copy) */
    LBM_ERR_NONFINITE = -5,    /* non-finite values found in fields or state */
    LBM_ERR_TIMEOUT = -6,      /* a bounded device wait expired */
    LBM_ERR_UNSUPPORTED = -7,  /* option not supported by this build or mode */
    LBM_ERR_IO = -8,           /* file open/read/write failure or bad file */
    LBM_ERR_NOMEM = -9         /* device or host allocation failed */
};

/* Storage type of the populations.  Collisions always compute in FP32. */
enum lbm_dtype {
    LBM_F32 = 1,    /* float32 populations; g stored as g - w_a P0 */
    LBM_F16S = 2,   /* float16, equilibrium-shifted and scaled */
    LBM_BF16S = 3   /* bfloat16, equilibrium-shifted and scaled */
};

enum lbm_mode {
    LBM_COUPLED = 0,  /* f + h + g, velocity from the flow lattice */
    LBM_FIXED_U = 1   /* f + h only, velocity prescribed by lbm_init_fields */
};

enum lbm_kernel {
    LBM_KERNEL_AUTO = 0,   /* library choice (the TMA-staged sweep) */
    LBM_KERNEL_SPLIT = 1,  /* three-kernel chain: moments, normals, collide */
    LBM_KERNEL_FUSED = 2,  /* one fused sweep kernel per step, per-thread loads */
    LBM_KERNEL_TMA = 3     /* one fused sweep kernel per step, rows staged by bulk-tensor copies */
};

typedef struct lbm_params {
    int32_t nx, ny;          /* grid size, each >= 4 */
    int32_t walls_y;         /* 0: periodic in y; 1: moving walls at y = 0 and y = ny */
    int32_t mode;            /* enum lbm_mode */
    int32_t dtype;           /* enum lbm_dtype */
    int32_t kernel;          /* enum lbm_kernel */
    int32_t sigma_literal;   /* 1: F_s exactly as Eq. (Fs); 0: scaled by 3W / (2 (phi_a - phi_b)^2)
                                so that its integral across the interface is sigma * kappa */
    int32_t reserved;        /* must be 0 */
    double u_wall;           /* wall speed U_o (x direction): bottom -u_wall, top +u_wall */
    double W;                /* interface width, Eq. (theta) */
    double phi_a, phi_b;     /* phase-field bounds, Eq. (CACE) */
    double M_phi;            /* CACE mobility; M_phi = cs^2 (1/w_kappa - 1/2), App. C */
    double D_s;              /* surface diffusivity; D_s = cs^2 (1/w_chi - 1/2), Eq. (diffcoeffscalarfield) */
    double nu_a, nu_b;       /* kinematic viscosities of the two phases (App. D) */
    double zeta;             /* bulk viscosity; zeta = cs^2 (1/w_zeta - 1/2) (App. D); 1/6 gives w_zeta = 1 */
    double rho_a, rho_b;     /* densities of the two phases (App. D) */
    double sigma_o;          /* clean-interface surface tension, Eq. (EOS) */
    double beta;             /* Gibbs elasticity, Eq. (EOS) */
    double c_max;            /* maximum concentration Gamma_inf, Eq. (EOS) */
    double fext_x, fext_y;   /* external body force F_ext */
} lbm_params;

typedef struct lbm_diag {
    int64_t step;            /* time steps taken since the last initialisation */
    double sum_phi, sum_c;   /* FP64 totals of phi and c over the grid */
    double D, L, B;          /* deformation D = (L - B)/(L + B) (Sec. 4.3, Fig. 8): L = 4 sqrt(l1),
                                B = 4 sqrt(l2) from the second moments of the drop
                                indicator w = clip((phi - phi_b) / (phi_a - phi_b), 0, 1) */
    double xc, yc;           /* w-weighted centroid (circular mean on periodic axes) */
    double umax;             /* max |u| */
    int64_t nonfinite;       /* cells with a non-finite phi, c or u */
    int64_t sigma_neg;       /* cells where 1 + beta ln(1 - c / c_max) < 0 (Eq. EOS); 0 when beta = 0 */
    int32_t status;          /* LBM_OK, or LBM_ERR_NONFINITE when nonfinite > 0 */
    int32_t reserved;
} lbm_diag;

typedef struct lbm_ctx lbm_ctx;

/* Fill *p with the defaults: W 4, phi_a 1, phi_b 0, M_phi 0.1, D_s 0.1,
 * nu 0.1, zeta 1/6, rho 1, c_max 1, periodic, coupled, FP32, AUTO kernel;
 * nx = ny = 0 (must be set).  Returns LBM_ERR_INVALID_ARG for p == NULL. */
int lbm_params_default(lbm_params *p);

/* Validate *p and create a context on the current CUDA device.
 * stream: a cudaStream_t to run on, or NULL.  Allocates two population
 * buffers (ping-pong) plus field scratch on the device.
 * Errors: INVALID_ARG (sizes < 4, NULL, bad enum), RATE (a coefficient <= 0),
 * UNSUPPORTED (dtype/mode/kernel combination), NOMEM, CUDA. */
int lbm_create(const lbm_params *p, void *stream, lbm_ctx **out);

/* Release all device and host memory of ctx (NULL is a no-op). */
void lbm_destroy(lbm_ctx *ctx);

/* Set the state to the discrete equilibria of the given macroscopic fields
 * (host float64 [ny][nx] arrays; P may be NULL for the uniform rest pressure
 * P = cs^2 (rho_a + rho_b) / 2, which is rho cs^2 at equal densities): for each
 * lattice P^-1 F^-1(u) applied to its equilibrium central moments, with
 * theta, theta_c and n from the given phi (Sec. 3, App. C, App. D).  In
 * LBM_FIXED_U mode (ux, uy) is also stored as the prescribed velocity.
 * Resets the step counter.  Synchronous.  Errors: INVALID_ARG, CUDA. */
int lbm_init_fields(lbm_ctx *ctx, const double *phi, const double *c, const double *ux,
                    const double *uy, const double *P);

/* Same with device float64 pointers (e.g. torch tensors on this device).
 * Asynchronous on the context stream; the inputs must stay valid until the
 * stream reaches this point. */
int lbm_init_fields_device(lbm_ctx *ctx, const double *phi, const double *c, const double *ux,
                           const double *uy, const double *P);

/* Advance nsteps >= 0 time steps: stream, moments, interface geometry,
 * forces, and the three central-moment collisions.  Asynchronous.  Steps are
 * replayed from captured CUDA graphs of 32, 16, 8, 4, 2 and 1 steps (largest
 * first); the first use of a graph captures it (host work, no device
 * allocation beyond the graph's own). */
int lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Macroscopic fields of the current state into host float64 [ny][nx]
 * arrays (any may be NULL): phi = sum f, c = sum h,
 * u = (sum e g + cs^2 F_t / 2) / (cs^2 rho), P = sum g + Gamma_00 / 2
 * (App. D update).  In LBM_FIXED_U mode u is the prescribed field and P is 0.
 * Synchronous. */
int lbm_get_fields(lbm_ctx *ctx, double *phi, double *c, double *ux, double *uy, double *P);

/* Same into device float64 arrays; asynchronous. */
int lbm_get_fields_device(lbm_ctx *ctx, double *phi, double *c, double *ux, double *uy,
                          double *P);

/* Current populations after streaming (the state the next collision reads),
 * unshifted, as host float64 [9][ny][nx] arrays (any may be NULL; g is
 * ignored in LBM_FIXED_U mode).  Synchronous. */
int lbm_get_populations(lbm_ctx *ctx, double *f, double *h, double *g);

/* Replace the state by the given post-streaming populations (host float64
 * [9][ny][nx]; NULL leaves that lattice unchanged).  Synchronous. */
int lbm_set_populations(lbm_ctx *ctx, const double *f, const double *h, const double *g);

/* FP64 reductions over the current state into *out (see lbm_diag).
 * Synchronous.  Returns LBM_OK even when out->status reports non-finite cells. */
int lbm_diagnostics(lbm_ctx *ctx, lbm_diag *out);

/* Wait for the context stream; report any pending CUDA error, or
 * LBM_ERR_TIMEOUT if a kernel's bounded wait for a staged row expired. */
int lbm_synchronize(lbm_ctx *ctx);

/* Number of 4-connected components of {phi > level} in the current state
 * (periodic in x, and in y without walls); a drop that has broken up has
 * more than one.  Synchronous; uses the context's staging buffer.
 * Errors: INVALID_ARG, NOMEM, CUDA. */
int lbm_count_components(lbm_ctx *ctx, double level, int32_t *count);

/* Steps taken since the last initialisation (-1 for a NULL context). */
int64_t lbm_get_step(const lbm_ctx *ctx);

/* Kernel variant the context runs (enum lbm_kernel, never AUTO) and the
 * number of kernel launches one step issues. */
int lbm_kernel_in_use(const lbm_ctx *ctx);
int lbm_launches_per_step(const lbm_ctx *ctx);

/* Launch shape of the sweep kernels: threads per block (tile_x; the block
 * owns tile_x - 4 columns; 128 for FUSED; 128 or 192 for TMA with 16-bit
 * storage; 64, 128 or 192 for TMA with FP32 storage) and rows per block
 * (seg_y >= 4).
 * 0 keeps the current value.
 * Errors: INVALID_ARG, UNSUPPORTED (split kernel, or tile_x not available). */
int lbm_set_launch_shape(lbm_ctx *ctx, int32_t tile_x, int32_t seg_y);
int lbm_get_launch_shape(const lbm_ctx *ctx, int32_t *tile_x, int32_t *seg_y);

/* Cells per thread of the TMA sweep: 1, or 2 horizontally adjacent cells
 * whose arithmetic runs on the packed two-lane FP32 instructions (tile_x 128
 * or 192).  Both forms compute the same expressions per cell; the flow
 * collision gives the same bits in both, the scalar lattices may differ in
 * the rounding of their packed sums.
 * Errors: INVALID_ARG (not 1 or 2), UNSUPPORTED (other kernels, or a block
 * width without the two-cell form). */
int lbm_set_cells_per_thread(lbm_ctx *ctx, int32_t cells);
int32_t lbm_get_cells_per_thread(const lbm_ctx *ctx);

/* How the TMA sweep writes collided cells: LBM_STORE_DIRECT (each thread
 * stores its cells; four staged raw rows in flight) or LBM_STORE_STAGED (each
 * warp group stages its row in shared memory and one bulk-tensor store writes
 * it; fewer raw rows in flight).  Same results either way.  Defaults: DIRECT
 * for FP32 storage, STAGED for 16-bit storage (the faster of each on the
 * 2048 x 1024 drop); the autotuner tries both.
 * Errors: INVALID_ARG, UNSUPPORTED. */
#define LBM_STORE_DIRECT 0
#define LBM_STORE_STAGED 1
int lbm_set_store_mode(lbm_ctx *ctx, int32_t mode);
int32_t lbm_get_store_mode(const lbm_ctx *ctx);

/* Checkpoint: parameters, step count and raw population buffers to a binary
 * file, and back (the file must come from a context with equal parameters).
 * A run continued from a checkpoint is bit-identical to an uninterrupted one.
 * Errors: IO, INVALID_ARG (parameter mismatch), CUDA. */
int lbm_save_state(lbm_ctx *ctx, const char *path);
int lbm_load_state(lbm_ctx *ctx, const char *path);

/* Test hook for the failure path of the bounded device waits (TMA kernel
 * only): the next step's kernel waits on a shared-memory barrier that no copy
 * completes, gives up after a short bound, sets the context's error flag and
 * returns.  The next synchronising call reports LBM_ERR_TIMEOUT; the context
 * stays usable but its state is undefined until re-initialised.
 * Errors: INVALID_ARG, UNSUPPORTED (other kernels). */
int lbm_debug_stall_next_step(lbm_ctx *ctx);

/* ------------------------------------------------------------------------
 * Launch-shape autotuner.  Times every candidate (block width tile_x, cells
 * per thread, store mode, rows per block seg_y) over `steps` steps of the
 * live state (after 2 warm-up steps, CUDA events on the context's stream),
 * restores the state, step count and buffer parity after each candidate,
 * and keeps the fastest shape.  Candidates (TMA kernel): (tile_x, cells per
 * thread) in {(128, 1), (192, 1), (64, 1), (128, 2), (192, 2)} with both
 * store modes for FP32 storage, and (128 or 192, 1 or 2) staged for 16-bit
 * storage; FUSED: tile_x 128.  seg_y in {8, 16, 32, 64, 128} plus the values
 * that fill one and two waves of resident blocks.  Needs one extra device buffer the size of a population
 * buffer while it runs.  Outputs (nullable): chosen shape and its time per
 * step in milliseconds.  Synchronous.
 * Errors: INVALID_ARG (steps < 1), UNSUPPORTED (split kernel), NOMEM, CUDA,
 * TIMEOUT. */
int lbm_autotune(lbm_ctx *ctx, int32_t steps, int32_t *tile_x, int32_t *seg_y,
                 double *ms_per_step);

/* ------------------------------------------------------------------------
 * Batches (ensembles of independent runs, e.g. drops in shear at different
 * grid sizes and parameters).  A batch owns one context per run and steps
 * them in one of two forms:
 *   LBM_BATCH_PERSISTENT  every time step is one launch of a persistent TMA
 *       sweep over the tiles of all runs, one launch per 64 runs; all runs
 *       share block width, cells per thread and rows per tile.  The runs'
 *       parameters live in a bank in constant memory of 256 runs per
 *       device; a batch that finds no room there has the chains form only;
 *   LBM_BATCH_CHAINS      every run is stepped by its own single-run
 *       launches with its own launch shape, the runs' launch chains spread
 *       over up to 16 side streams and running concurrently.
 * Step loops of either form are replayed from captured CUDA graphs of 32, 16,
 * 8, 4, 2 and 1 steps.  Runs are independent: each follows Sec. 3 and
 * App. C-D exactly as a single context does, and a batched step gives
 * results identical to stepping each run's context on its own with the same
 * launch shape.
 */
#define LBM_BATCH_CHAINS 0
#define LBM_BATCH_PERSISTENT 1
typedef struct lbm_batch lbm_batch;

/* params: array of nruns parameter sets (grid, physics, walls may differ;
 * mode must be the same for all; kernel must be AUTO or TMA).  stream:
 * cudaStream_t shared by the batch and its runs (NULL: a private stream).
 * Errors: INVALID_ARG, RATE, UNSUPPORTED (no TMA support, kernel choice),
 * NOMEM, CUDA. */
int lbm_batch_create(const lbm_params *params, int32_t nruns, void *stream, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);
int32_t lbm_batch_size(const lbm_batch *b);

/* Context of run `run` (owned by the batch; NULL if out of range).  Use it
 * with lbm_init_fields, lbm_get_fields, lbm_diagnostics, lbm_save_state and
 * the other single-run calls; stepping it alone is allowed (the next batched
 * step picks up its buffer parity). */
lbm_ctx *lbm_batch_run(lbm_batch *b, int32_t run);

/* Advance every run by nsteps (asynchronous on the batch stream). */
int lbm_batch_step(lbm_batch *b, int64_t nsteps);

/* Wait for the batch stream; reports a pending CUDA error or an expired
 * bounded wait (LBM_ERR_TIMEOUT) of a batched step. */
int lbm_batch_synchronize(lbm_batch *b);

/* Form of the batched step (LBM_BATCH_PERSISTENT, the default, or
 * LBM_BATCH_CHAINS).  Synchronous.  Errors: INVALID_ARG, UNSUPPORTED (the
 * persistent form for a batch without parameter-bank slots). */
int lbm_batch_set_form(lbm_batch *b, int32_t form);
int32_t lbm_batch_get_form(const lbm_batch *b);

/* Block width (64, 128 or 192; the block owns tile_x - 4 columns), rows per
 * tile (>= 4), cells per thread (1 or 2, see lbm_set_cells_per_thread) and
 * store mode (see lbm_set_store_mode) of the persistent form; 0 keeps the
 * current width and rows.  Setting them also sets
 * every run's own shape (chains form).  The getter also reports the
 * persistent grid size (blocks of all launches of a step) and the number of
 * tiles.  Errors: INVALID_ARG, UNSUPPORTED. */
int lbm_batch_set_launch_shape(lbm_batch *b, int32_t tile_x, int32_t seg_y);
int lbm_batch_set_cells_per_thread(lbm_batch *b, int32_t cells);
int lbm_batch_set_store_mode(lbm_batch *b, int32_t mode);
int lbm_batch_get_launch_shape(const lbm_batch *b, int32_t *tile_x, int32_t *seg_y,
                               int32_t *blocks, int32_t *tiles);

/* Autotuner of the batched step: the persistent form over (tile_x, cells
 * per thread, store mode) in {(64, 1, direct), (128, 1, direct), (192, 1,
 * direct), (64, 1, staged), (128, 1, staged), (128, 2, staged)} x seg_y in
 * {24, 32, 40, 48, 56, 64, 80}; the chains form with every run's shape from
 * lbm_autotune on one run of each grid size, and with the shapes (192, 38,
 * 1, direct), (128, 32, 1, direct) and (192, 38, 2, direct) for every run;
 * the fastest form and shapes are kept.  Every candidate is timed over `steps` rounded up to whole 32-step
 * graphs after one graph of warm-up, and the state, step counts and buffer
 * parities are restored after each (one snapshot buffer per run while it
 * runs).  Outputs (nullable): the persistent shape and the chosen form's time
 * per step in milliseconds.  Synchronous. */
int lbm_batch_autotune(lbm_batch *b, int32_t steps, int32_t *tile_x, int32_t *seg_y,
                       double *ms_per_step);

/* ------------------------------------------------------------------------
 * Surrogate network (the learned part that picks capillary numbers near
 * drop breakup; not in the paper).  A multilayer perceptron with 5 inputs,
 * four hidden layers of width 128 with SiLU, and 2 outputs (steady
 * deformation D and a breakup logit); BF16 weights, FP32 accumulation, FP32
 * master weights trained with Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Loss: mean((D - yD)^2) + mean(BCE(logit, yB)).
 *
 * Parameters form one FP32 vector of surr_param_count() values: for each
 * layer l = 0..4 (fan-in WIDTH[l], fan-out WIDTH[l+1], WIDTH = 5, 128, 128,
 * 128, 128, 2) the weights W[fout][fin] row-major, then the biases b[fout].
 * The forward and backward passes use the weights rounded to BF16 (nearest,
 * ties to even); biases stay FP32.
 *
 * Host arrays: X [n][5] float32 row-major; yD, yB, D_out, logit_out [n].
 * All calls are synchronous on the context's stream (NULL: legacy default).
 * Errors: INVALID_ARG, NOMEM, CUDA. */
typedef struct surr_ctx surr_ctx;
int32_t surr_param_count(void);
/* Create with He-initialised weights (N(0, 2/fan_in) from a SplitMix64 /
 * Box-Muller stream seeded by `seed`) and zero biases. */
int surr_create(uint64_t seed, void *stream, surr_ctx **out);
void surr_destroy(surr_ctx *ctx);
/* Replace / read the FP32 master parameters (set also resets Adam). */
int surr_set_params(surr_ctx *ctx, const float *params);
int surr_get_params(surr_ctx *ctx, float *params);
/* Outputs for n samples. */
int surr_predict(surr_ctx *ctx, const float *X, int32_t n, float *D_out, float *logit_out);
/* Gradient of the loss over n samples with respect to every parameter (same
 * layout as the parameters; NULL to skip) and the loss (NULL to skip);
 * parameters unchanged. */
int surr_grad(surr_ctx *ctx, const float *X, const float *yD, const float *yB, int32_t n,
              float *grads, double *loss);
/* `epochs` full-batch Adam steps on the n samples with learning rate lr;
 * loss_out (nullable): loss after the last step.  The step's launches are
 * captured once into a CUDA graph (kept for the next call with the same n
 * and lr) and the graph is replayed once per epoch. */
int surr_train(surr_ctx *ctx, const float *X, const float *yD, const float *yB, int32_t n,
               int32_t epochs, float lr, double *loss_out);

/* ------------------------------------------------------------------------
 * Field statistics without allocation.  The paper has no counterpart: this
 * entry point serves callers that cannot allocate device memory where they
 * need the statistics (a memory pool with a hard cap, a framework that
 * forbids allocations inside its step loop).  It computes, in FP64, the same
 * reductions as lbm_diagnostics over caller-owned device fields and allocates
 * nothing: its scratch is a file-scope device array of
 * LBM_NOALLOC_MAX_BLOCKS x 12 doubles (96 KiB) that every GPU loading this
 * library holds until the process exits.
 *
 * phi, c, ux, uy: device float64 [ny][nx] fields (inputs, not modified).
 * walls_y: 0 periodic y (circular-mean centroid), 1 walls (plain mean).
 * beta, c_max: Langmuir parameters for the sigma < 0 count (Eq. EOS).
 * phi_a, phi_b: the bulk phases (drop, matrix), as in lbm_params.
 * result: device array of LBM_FIELD_STATS_LEN doubles, written in full:
 *   [0] sum phi  [1] sum c  [2] xc  [3] yc  [4] non-finite cells
 *   [5] cells with sigma < 0  [6] max |u|  [7] Ixx  [8] Iyy  [9] Ixy
 *   [10] L  [11] B  [12] D   (centroid, moments, L, B, D as in lbm_diag, of
 *   the drop indicator clip((phi - phi_b) / (phi_a - phi_b), 0, 1))
 * stream: cudaStream_t to run on (NULL: the legacy default stream).
 * Asynchronous on `stream`.  The first call in a CUDA context looks up the
 * device address of the scratch array (cudaGetSymbolAddress) and keeps it
 * for that context (by context ID, so a reset or new context looks it up
 * again); make that first call before any stream capture.  Every call
 * overwrites the scratch before reading it, so nothing needs clearing, but
 * calls that overlap on the GPU share the array and race.
 * Errors: INVALID_ARG (NULL pointer, nx or ny < 1, nx * ny >
 * LBM_NOALLOC_MAX_CELLS, bad walls_y or c_max, phi_a == phi_b or not
 * finite), CUDA. */
#define LBM_FIELD_STATS_LEN 13
#define LBM_NOALLOC_MAX_BLOCKS 1024
#define LBM_NOALLOC_MAX_CELLS 1073741824
int lbm_field_stats_noalloc(const double *phi, const double *c, const double *ux,
                            const double *uy, int32_t nx, int32_t ny, int32_t walls_y,
                            double beta, double c_max, double phi_a, double phi_b,
                            double *result, void *stream);

/* Static description of an error code. */
const char *lbm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
