/*
 * FP64 CPU oracle of the three-dimensional (D3Q27) form of the two scalar
 * lattices of Schupbach & Premnath (arXiv 2504.09024), driven by a prescribed
 * velocity field:
 *   f: conservative Allen-Cahn phase field phi       (App. C, D2Q9 in the paper)
 *   h: interface-bound surfactant scalar c           (Sec. 3, D2Q9 in the paper)
 * The paper names the 3-D version as future work (Sec. 5); the readings that
 * carry each D2Q9 step over to 27 velocities are listed in lbm_oracle3.c.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this library; the product path never does.  It shares
 * no source with the CUDA library.
 *
 * Arrays are [nz][ny][nx] (x fastest), float64, periodic in x, y and z.
 * Population arrays are [27][nz][ny][nx] in the velocity order that
 * orc3_velocities() returns: rest, the 6 faces, the 12 edges, the 8 corners.
 */
#ifndef LBM_ORACLE3_H
#define LBM_ORACLE3_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz, pad_;
    double W, phi_a, phi_b;
    double M_phi, D_s;
    /* The flow lattice (mode = 1): the pressure-based two-fluid flow of App. D
     * on D3Q27, forced by the capillary and Marangoni stress of Eq. (Fs). */
    int mode;           /* 0: prescribed velocity, f + h only; 1: coupled f + h + g */
    int walls_y;        /* 1: half-way bounce-back walls at y = 0 (-u_wall) and y = ny (+u_wall), x-directed */
    int sigma_literal;  /* 1: surface-tension force as printed; 0: scaled by 3W / (2 (phi_a - phi_b)^2) */
    int pad2_;
    double u_wall, nu_a, nu_b, zeta, rho_a, rho_b;
    double sigma_o, beta, c_max;
    double fext[3];
} orc3_params;

typedef struct orc3_sim orc3_sim;

orc3_sim *orc3_create(const orc3_params *p);
void orc3_destroy(orc3_sim *s);
/* Discrete equilibria of the given fields (first-order moments carrying the
 * flux terms of the given phi and c); u is the prescribed velocity. */
int orc3_init(orc3_sim *s, const double *phi, const double *c, const double *ux,
              const double *uy, const double *uz);
/* The same with the flow lattice's initial pressure P (mode 1; NULL: the
 * uniform rest pressure cs^2 (rho_a + rho_b) / 2). */
int orc3_init_pressure(orc3_sim *s, const double *phi, const double *c, const double *ux,
                       const double *uy, const double *uz, const double *P);
void orc3_step(orc3_sim *s, int nsteps);
long long orc3_get_step(const orc3_sim *s);
/* phi = sum f and c = sum h of the current populations (either may be NULL). */
void orc3_fields(orc3_sim *s, double *phi, double *c);
/* Unit normal of the current phi (components may be NULL). */
void orc3_normals(orc3_sim *s, double *nx_, double *ny_, double *nz_);
void orc3_get_pops(const orc3_sim *s, double *f, double *h);
/* Flow lattice (mode 1): velocity and pressure of the current state, as the
 * macroscopic update of App. D defines them (any output may be NULL), and
 * the populations g. */
void orc3_flow_fields(orc3_sim *s, double *ux, double *uy, double *uz, double *P);
void orc3_get_flow_pops(const orc3_sim *s, double *g);
/* Curvature kappa = div n of the current phi (the stencil of the gradient). */
void orc3_curvature(orc3_sim *s, double *kappa);
/* Replace the post-streaming populations (NULL leaves that lattice unchanged). */
void orc3_set_pops(orc3_sim *s, const double *f, const double *h);
/* The 27 velocities, e[3 * a + axis]. */
void orc3_velocities(int out[81]);
/* Building blocks, exposed for the pins: the 27 x 27 matrices, row-major. */
void orc3_matrix_P(double out[729]);
void orc3_matrix_Pinv(double out[729]);
void orc3_matrix_F(double ux, double uy, double uz, double out[729]);
void orc3_matrix_Finv(double ux, double uy, double uz, double out[729]);
/* Isotropic gradient of an arbitrary [nz][ny][nx] field (periodic). */
void orc3_gradient(const orc3_sim *s, const double *a, double *gx, double *gy, double *gz);

#ifdef __cplusplus
}
#endif
#endif
