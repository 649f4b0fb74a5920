/*
 * FP64 CPU oracle for the three coupled central-moment D2Q9 lattice
 * Boltzmann schemes of Schupbach & Premnath (arXiv 2504.09024):
 *   f: conservative Allen-Cahn phase field phi        (App. C)
 *   h: interface-bound surfactant scalar c            (Sec. 3)
 *   g: pressure-based two-fluid flow P, u             (App. D)
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this library; the product path never does.  It shares
 * no source with the CUDA library.
 *
 * Arrays are row-major [ny][nx] (x fastest), float64.  Population arrays are
 * [9][ny][nx] in the D2Q9 order of the paper's P matrix (App. A):
 *   0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;
    int walls_y;        /* 0: periodic in y; 1: half-way bounce-back walls at y = 0 and y = ny */
    int mode;           /* 0: coupled f + h + g; 1: prescribed velocity, f + h only */
    int sigma_literal;  /* 1: surface-tension force as printed; 0: scaled by 3W / (2 (phi_a - phi_b)^2) */
    int pad_;
    double u_wall;      /* top wall moves with +u_wall, bottom wall with -u_wall (x direction) */
    double W, phi_a, phi_b;
    double M_phi, D_s, nu_a, nu_b, zeta;
    double rho_a, rho_b;
    double sigma_o, beta, c_max;
    double fext_x, fext_y;
} orc_params;

typedef struct orc_sim orc_sim;

typedef struct {
    long long step;
    double sum_phi, sum_c, D, L, B, xc, yc, umax;
    long long nonfinite, sigma_neg;
} orc_diag;

orc_sim *orc_create(const orc_params *p);
void orc_destroy(orc_sim *s);
/* Equilibrium populations from macroscopic fields (P may be NULL: P = rho cs^2). */
int orc_init(orc_sim *s, const double *phi, const double *c, const double *ux,
             const double *uy, const double *P);
void orc_step(orc_sim *s, int nsteps);
long long orc_get_step(const orc_sim *s);
/* Macroscopic fields of the current state: phi, c, u and P as the paper's
 * macroscopic update defines them (any output may be NULL). */
void orc_fields(orc_sim *s, double *phi, double *c, double *ux, double *uy, double *P);
/* Extra per-cell quantities of the current state (any may be NULL):
 * unit normal, |grad phi|, curvature div n, surface-tension force F_s. */
void orc_geometry(orc_sim *s, double *nx_, double *ny_, double *gmag, double *kappa,
                  double *Fsx, double *Fsy);
void orc_get_pops(const orc_sim *s, double *f, double *h, double *g);
void orc_set_pops(orc_sim *s, const double *f, const double *h, const double *g);
/* Prescribed velocity (mode 1). */
void orc_set_velocity(orc_sim *s, const double *ux, const double *uy);
/* Replace the f populations by the equilibrium of a given phi (other lattices untouched). */
void orc_reset_f(orc_sim *s, const double *phi);
void orc_diagnostics(orc_sim *s, orc_diag *out);

/* Building blocks, exposed for the pins. */
void orc_matrix_P(double out[81]);
void orc_matrix_Pinv(double out[81]);
void orc_matrix_F(double ux, double uy, double out[81]);
void orc_matrix_Finv(double ux, double uy, double out[81]);
/* Isotropic gradient of an arbitrary [ny][nx] field with this sim's boundaries. */
void orc_gradient(const orc_sim *s, const double *a, double *gx, double *gy);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
