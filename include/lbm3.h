/*
 * lbm3.h -- C ABI of the three-dimensional (D3Q27) scalar lattices in
 * liblbm.so: the conservative Allen-Cahn phase field phi (App. C) and the
 * interface-bound surfactant c (Sec. 3) of Schupbach & Premnath (arXiv
 * 2504.09024), advected by a prescribed velocity.  The paper states both
 * schemes on D2Q9 and names the 3-D extension as future work (Sec. 5); this
 * library carries them to 27 velocities:
 *   - moment basis |e_x^m e_y^n e_z^p>, m, n, p in {0, 1, 2} (the 3-D
 *     counterpart of Eq. Pi), central moments by the binomial frame change of
 *     Eq. (cmscalar) on each axis;
 *   - equilibria: Maxwellian central moments of the scalar (mu(0) = 1,
 *     mu(1) = 0, mu(2) = cs^2 on each axis), first-order moments replaced by
 *     M_phi theta n (f) and D_s theta_c n (h), Eqs. (theta) and (ISS);
 *   - first-order moments relax with w (M = cs^2 (1/w - 1/2)), all others
 *     with rate 1;
 *   - n = grad phi / |grad phi| by the isotropic D3Q27 stencil
 *     d_i A = (1/cs^2) sum_a w_a e_ai A(x + e_a), weights 8/27, 2/27, 1/54, 1/216.
 * Because every moment but the first-order ones is relaxed to its
 * equilibrium, a collision needs only the zeroth and first raw moments of the
 * incoming populations, and the outgoing populations factor into products of
 * one-dimensional factors per axis (the tensor structure of P and F(u)).
 *
 * Conventions (in addition to those of lbm.h, whose status codes apply):
 *   - Grids are nx by ny by nz cells, periodic on every axis; cell (i, j, k)
 *     has centre (i + 1/2, j + 1/2, k + 1/2).  Field arrays are [nz][ny][nx]
 *     float64, x fastest.
 *   - Population arrays are [27][nz][ny][nx] float64.  Population a has
 *     velocity (E[a % 3], E[(a / 3) % 3], E[a / 9]) with E = {0, +1, -1};
 *     lbm3_velocities() returns the list.
 *   - Populations are stored on the device as int32 fixed point in units of
 *     2^-28 (range +-8), plane by plane ([nz][27][ny][nx] words per lattice),
 *     two buffers of 2 x 27 x nx ny nz words (ping-pong);
 *     the collision arithmetic is FP32.  The pull sums are exact integer sums
 *     and each collision gives its rest population the integer remainder of
 *     the cell's zeroth moment, so sum phi and sum c are conserved exactly.
 *     A cell whose phi or c leaves (-4, 4) marks its populations invalid;
 *     outputs show them as NaN and lbm3_sums counts them.
 *   - Work runs on the stream given to lbm3_create (NULL: the library's own
 *     non-blocking stream).  lbm3_step is asynchronous; calls that return data
 *     to the host synchronise that stream.
 */
#ifndef LBM3_H
#define LBM3_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* nx * ny * nz may not exceed this (populations of 2^31 cells would need
 * 464 GB; 2^30 cells need 232 GB of the GPU's memory), and 27 * nx * ny must
 * stay below 2^31 (offsets inside a plane's 27 populations are 32-bit). */
#define LBM3_MAX_CELLS 1073741824LL

typedef struct lbm3_params {
    int32_t nx, ny, nz;        /* >= 1 each, product <= LBM3_MAX_CELLS */
    int32_t velocity_field;    /* 0: uniform velocity u[3]; 1: a per-cell field given to lbm3_init_fields */
    double W;                  /* interface width, > 0 */
    double phi_a, phi_b;       /* phase values, phi_a != phi_b */
    double M_phi, D_s;         /* mobility and surface diffusivity, > 0 (relaxation rate in (0, 2)) */
    double u[3];               /* uniform velocity when velocity_field = 0 */
} lbm3_params;

typedef struct lbm3_ctx lbm3_ctx;

/* Defaults: W 4, phi_a 1, phi_b 0, M_phi 0.1, D_s 0.1, uniform u = 0;
 * nx = ny = nz = 0 (must be set).  INVALID_ARG for p == NULL. */
int lbm3_params_default(lbm3_params *p);

/* Validate *p and create a context on the current CUDA device.
 * stream: a cudaStream_t or NULL.  Allocates the two population buffers, the
 * velocity field (velocity_field = 1) and reduction scratch.
 * Errors: INVALID_ARG (NULL, a size < 1, too many cells, 27 nx ny >= 2^31, phi_a == phi_b,
 * |phi_a| or |phi_b| > 2, a uniform |u_i| >= 1/2, W <= 0, a non-finite
 * value), RATE (M_phi or D_s <= 0), NOMEM, CUDA. */
int lbm3_create(const lbm3_params *p, void *stream, lbm3_ctx **out);

/* Release all memory of ctx (NULL is a no-op). */
void lbm3_destroy(lbm3_ctx *ctx);

/* Set the state to the discrete equilibria of the given fields (host float64
 * [nz][ny][nx]); the first-order moments carry the flux terms of the given
 * phi and c.  ux, uy, uz: the prescribed velocity field, required when
 * velocity_field = 1 and ignored (may be NULL) otherwise.  Resets the step
 * counter.  Synchronous.  Errors: INVALID_ARG, CUDA. */
int lbm3_init_fields(lbm3_ctx *ctx, const double *phi, const double *c, const double *ux,
                     const double *uy, const double *uz);

/* Same with device float64 pointers; asynchronous on the context stream. */
int lbm3_init_fields_device(lbm3_ctx *ctx, const double *phi, const double *c,
                            const double *ux, const double *uy, const double *uz);

/* Advance nsteps >= 0 time steps, one kernel launch per step: streaming
 * (pull), phi and c, the normal and theta, theta_c, and both collisions.
 * Asynchronous. */
int lbm3_step(lbm3_ctx *ctx, int64_t nsteps);

/* phi = sum f and c = sum h of the current state (post-streaming
 * populations) into host float64 [nz][ny][nx] arrays (either may be NULL;
 * NaN where a population is invalid).  Synchronous. */
int lbm3_get_fields(lbm3_ctx *ctx, double *phi, double *c);

/* Same into device float64 arrays; asynchronous. */
int lbm3_get_fields_device(lbm3_ctx *ctx, double *phi, double *c);

/* Current post-streaming populations as host float64 [27][nz][ny][nx]
 * arrays in the order of lbm3_velocities() (either may be NULL).
 * Synchronous. */
int lbm3_get_populations(lbm3_ctx *ctx, double *f, double *h);

/* Same into device float64 [27][nz][ny][nx] arrays; asynchronous. */
int lbm3_get_populations_device(lbm3_ctx *ctx, double *f, double *h);

/* Totals of the current state: out[0] = sum phi, out[1] = sum c (exact sums
 * of the fixed-point populations, as float64), out[2] = number of invalid
 * populations.  Synchronous, deterministic. */
int lbm3_sums(lbm3_ctx *ctx, double out[3]);

/* The 27 velocities, out[3 * a + axis]. */
int lbm3_velocities(int32_t out[81]);

/* Wait for the context stream and report any pending CUDA error. */
int lbm3_synchronize(lbm3_ctx *ctx);

int64_t lbm3_get_step(const lbm3_ctx *ctx);

/* Launch shape of the step kernel: rows = tile height in cells including the
 * one-cell halo on each side (one warp per row, 32 columns of which 30 are
 * updated), one of 6, 10, 18; seg_z = planes a block marches through, >= 1.
 * 0 keeps the current value.  INVALID_ARG otherwise. */
int lbm3_set_launch_shape(lbm3_ctx *ctx, int32_t rows, int32_t seg_z);
int lbm3_get_launch_shape(const lbm3_ctx *ctx, int32_t *rows, int32_t *seg_z);

/* Time `steps` steps (CUDA events, after one warm-up step) for each
 * candidate shape (rows in {6, 10, 18} x seg_z in {4, 8, 16, 32, 64, nz}),
 * keep the fastest and report it (outputs may be NULL).  Advances the state
 * by the steps it timed; call it before lbm3_init_fields.  Synchronous. */
int lbm3_autotune(lbm3_ctx *ctx, int32_t steps, int32_t *rows, int32_t *seg_z, double *ms_per_step);

#ifdef __cplusplus
}
#endif
#endif /* LBM3_H */
