/*
 * FP64 CPU oracle for the coupled central-moment lattice Boltzmann method of
 * Schupbach & Premnath, "A Robust Lattice Boltzmann Method for Interface-Bound
 * Transport of a Passive Scalar" (arXiv 2504.09024).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * bench's CPU-baseline leg, never by the product path.  No code is shared with
 * the CUDA library.
 *
 * It is deliberately plain and slow: every collision is computed with the
 * literal 9x9 matrices P, F(u), F^-1(u), P^-1 (and B, B^-1 for the flow
 * lattice), in the order the paper's algorithm lists give, one cell at a time.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *  - velocity set: the one of the P matrix (App. A); the printed e_x list ends
 *    in 0, which contradicts P (its last entry must be 1).
 *  - F and F^-1 are generated from the binomial definition, Eq. (cmscalar);
 *    the printed matrices (App. B) miss a factor 2 in two entries of the last row.
 *  - gradients: isotropic stencil d_i A = (1/cs2) sum_a w_a e_ai A(x + e_a),
 *    periodic in x; with walls the field is mirrored about the wall plane.
 *  - unit normal n = grad phi / |grad phi|, n = 0 where |grad phi| <= 1e-12.
 *  - curvature kappa = div n with the same stencil; grad sigma by the same
 *    stencil applied to the field sigma(c(x)).
 *  - F_s carries the factor N = 3W / (2 (phi_a - phi_b)^2) unless
 *    sigma_literal is set, so that its integral across the tanh profile is
 *    sigma kappa (effective tension sigma_o, as Ca presumes).
 *  - pressure force F_p = -grad(P* - rho cs2) with P* = sum g (the zeroth
 *    moment before the half-source correction), then P = P* + Gamma_00 / 2.
 *  - first-order flow equilibria -psi u (the sign that makes the raw first
 *    moment of g^eq equal rho cs2 u, as the velocity definition requires).
 *  - all three collisions at step n use fields of the step-n populations.
 *  - walls: half-way bounce-back, node rows at y = j + 1/2, walls at y = 0 and
 *    y = ny moving with -u_wall and +u_wall; the flow lattice gets the moving-
 *    wall term 2 w_a rho (e_a . u_w), rho of the wall-adjacent node.
 *  - initial populations are the discrete equilibria of the given fields.
 */
#include "lbm_oracle.h"

#define _USE_MATH_DEFINES
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

/* D2Q9 velocities in the order of the P matrix rows e_x, e_y (App. A). */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* Lattice weights of D2Q9 (used by the gradient stencil and the wall term). */
static const double WQ[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* Moment orders (m, n) of the basis |p_k> = |e_x^m e_y^n>, Eq. (Pi):
 * 00, 10, 01, 20, 02, 11, 21, 12, 22. */
static const int MOM_M[Q] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
static const int MOM_N[Q] = {0, 0, 1, 0, 2, 1, 1, 2, 2};

static const double CS2 = 1.0 / 3.0;
static const double EPS_N = 1e-12;

/* P^-1 exactly as printed in App. A (Eq. Pinv). */
static const double PINV[Q][Q] = {
    {1, 0, 0, -1, -1, 0, 0, 0, 1},
    {0, 0.5, 0, 0.5, 0, 0, 0, -0.5, -0.5},
    {0, 0, 0.5, 0, 0.5, 0, -0.5, 0, -0.5},
    {0, -0.5, 0, 0.5, 0, 0, 0, 0.5, -0.5},
    {0, 0, -0.5, 0, 0.5, 0, 0.5, 0, -0.5},
    {0, 0, 0, 0, 0, 0.25, 0.25, 0.25, 0.25},
    {0, 0, 0, 0, 0, -0.25, 0.25, -0.25, 0.25},
    {0, 0, 0, 0, 0, 0.25, -0.25, -0.25, 0.25},
    {0, 0, 0, 0, 0, -0.25, -0.25, 0.25, 0.25},
};

struct orc_sim {
    orc_params p;
    int N;
    long long step;
    double *f, *h, *g;          /* [9][N] post-streaming (pre-collision) populations */
    double *ft, *ht, *gt;       /* [9][N] post-collision populations */
    /* per-cell fields of the current step */
    double *phi, *c, *Pstar, *jx, *jy;
    double *rho, *sig, *psistar;
    double *ux, *uy, *P, *psi, *nu;
    double *nxv, *nyv, *gmag, *kappa;
    double *Fsx, *Fsy, *Ftx, *Fty, *Fpx, *Fpy;
    double *theta, *thetac;
    double *ufx, *ufy;          /* prescribed velocity (mode 1) */
    double P_matrix[Q][Q];
    double Bm[Q][Q], Binv[Q][Q];
};

/* ------------------------------------------------------------------------ */
/* Matrices                                                                  */
/* ------------------------------------------------------------------------ */

/* P_{k,a} = e_ax^m_k e_ay^n_k, the rows being the basis vectors of Eq. (Pi). */
static void build_P(double P[Q][Q]) {
    for (int k = 0; k < Q; ++k)
        for (int a = 0; a < Q; ++a) {
            double v = 1.0;
            for (int t = 0; t < MOM_M[k]; ++t) v *= EX[a];
            for (int t = 0; t < MOM_N[k]; ++t) v *= EY[a];
            P[k][a] = v;
        }
}

static double binom(int n, int k) {
    double r = 1.0;
    for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
    return r;
}

static double ipow(double x, int n) {
    double r = 1.0;
    for (int t = 0; t < n; ++t) r *= x;
    return r;
}

/* Frame change from raw to central moments by the binomial expansion of
 * (e_x - u_x)^m (e_y - u_y)^n, Eq. (cmscalar):
 *   kappa_mn = sum_{j<=m, k<=n} C(m,j) C(n,k) (-u_x)^(m-j) (-u_y)^(n-k) kappa'_jk.
 * With s = -1 this is F(u); with s = +1 it is the inverse map
 * e^m = ((e - u) + u)^m, i.e. F^-1(u). */
static void build_frame(double ux, double uy, double s, double F[Q][Q]) {
    for (int r = 0; r < Q; ++r) {
        for (int col = 0; col < Q; ++col) {
            int m = MOM_M[r], n = MOM_N[r], j = MOM_M[col], k = MOM_N[col];
            if (j > m || k > n) {
                F[r][col] = 0.0;
                continue;
            }
            F[r][col] = binom(m, j) * binom(n, k) * ipow(s * ux, m - j) * ipow(s * uy, n - k);
        }
    }
}

static void matvec(const double A[Q][Q], const double *x, double *y) {
    for (int r = 0; r < Q; ++r) {
        double acc = 0.0;
        for (int col = 0; col < Q; ++col) acc += A[r][col] * x[col];
        y[r] = acc;
    }
}

/* B combines the diagonal second-order moments: hat_2s = m20 + m02,
 * hat_2d = m20 - m02 (Eq. combinedforms); B^-1 recovers them. */
static void build_B(double B[Q][Q], double Bi[Q][Q]) {
    memset(B, 0, sizeof(double) * Q * Q);
    memset(Bi, 0, sizeof(double) * Q * Q);
    for (int k = 0; k < Q; ++k) {
        B[k][k] = 1.0;
        Bi[k][k] = 1.0;
    }
    B[3][3] = 1.0;  B[3][4] = 1.0;
    B[4][3] = 1.0;  B[4][4] = -1.0;
    Bi[3][3] = 0.5; Bi[3][4] = 0.5;
    Bi[4][3] = 0.5; Bi[4][4] = -0.5;
}

void orc_matrix_P(double out[81]) {
    double P[Q][Q];
    build_P(P);
    memcpy(out, P, sizeof(P));
}
void orc_matrix_Pinv(double out[81]) { memcpy(out, PINV, sizeof(PINV)); }
void orc_matrix_F(double ux, double uy, double out[81]) {
    double F[Q][Q];
    build_frame(ux, uy, -1.0, F);
    memcpy(out, F, sizeof(F));
}
void orc_matrix_Finv(double ux, double uy, double out[81]) {
    double F[Q][Q];
    build_frame(ux, uy, +1.0, F);
    memcpy(out, F, sizeof(F));
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Allocation                                                                */
/* ------------------------------------------------------------------------ */

static double *alloc_d(size_t n) { return (double *)calloc(n, sizeof(double)); }

orc_sim *orc_create(const orc_params *p) {
    if (p->nx < 1 || p->ny < 1) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->N = p->nx * p->ny;
    size_t N = (size_t)s->N;
    s->f = alloc_d(Q * N); s->h = alloc_d(Q * N); s->g = alloc_d(Q * N);
    s->ft = alloc_d(Q * N); s->ht = alloc_d(Q * N); s->gt = alloc_d(Q * N);
    double **fields[] = {&s->phi, &s->c, &s->Pstar, &s->jx, &s->jy, &s->rho, &s->sig,
                         &s->psistar, &s->ux, &s->uy, &s->P, &s->psi, &s->nu, &s->nxv,
                         &s->nyv, &s->gmag, &s->kappa, &s->Fsx, &s->Fsy, &s->Ftx, &s->Fty,
                         &s->Fpx, &s->Fpy, &s->theta, &s->thetac, &s->ufx, &s->ufy};
    for (size_t k = 0; k < sizeof(fields) / sizeof(fields[0]); ++k) *fields[k] = alloc_d(N);
    build_P(s->P_matrix);
    build_B(s->Bm, s->Binv);
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    double *ptrs[] = {s->f, s->h, s->g, s->ft, s->ht, s->gt, s->phi, s->c, s->Pstar, s->jx,
                      s->jy, s->rho, s->sig, s->psistar, s->ux, s->uy, s->P, s->psi, s->nu,
                      s->nxv, s->nyv, s->gmag, s->kappa, s->Fsx, s->Fsy, s->Ftx, s->Fty,
                      s->Fpx, s->Fpy, s->theta, s->thetac, s->ufx, s->ufy};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(s);
}

long long orc_get_step(const orc_sim *s) { return s->step; }

/* ------------------------------------------------------------------------ */
/* Extended-field access and stencils                                        */
/* ------------------------------------------------------------------------ */

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* Row index of the extended field: periodic, or mirrored about the wall
 * planes y = 0 and y = ny (row -1-k is row k, row ny+k is row ny-1-k). */
static int ext_row(const orc_sim *s, int j) {
    int ny = s->p.ny;
    if (!s->p.walls_y) return wrap(j, ny);
    while (j < 0 || j >= ny) {
        if (j < 0) j = -1 - j;
        if (j >= ny) j = 2 * ny - 1 - j;
    }
    return j;
}

static double at(const orc_sim *s, const double *a, int i, int j) {
    return a[(size_t)ext_row(s, j) * s->p.nx + wrap(i, s->p.nx)];
}

/* Isotropic central-difference gradient, d_i A = (1/cs2) sum_a w_a e_ai A(x + e_a). */
static void grad_at(const orc_sim *s, const double *a, int i, int j, double *gx, double *gy) {
    double sx = 0.0, sy = 0.0;
    for (int q = 0; q < Q; ++q) {
        double v = at(s, a, i + EX[q], j + EY[q]);
        sx += WQ[q] * EX[q] * v;
        sy += WQ[q] * EY[q] * v;
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
}

void orc_gradient(const orc_sim *s, const double *a, double *gx, double *gy) {
    int nx = s->p.nx, ny = s->p.ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) grad_at(s, a, i, j, &gx[(size_t)j * nx + i], &gy[(size_t)j * nx + i]);
}

/* Unit normal n = grad phi / |grad phi| at any (possibly ghost) position. */
static void normal_at(const orc_sim *s, int i, int j, double *nx_, double *ny_, double *mag) {
    double gx, gy;
    grad_at(s, s->phi, i, j, &gx, &gy);
    double m = sqrt(gx * gx + gy * gy);
    *mag = m;
    if (m > EPS_N) {
        *nx_ = gx / m;
        *ny_ = gy / m;
    } else {
        *nx_ = 0.0;
        *ny_ = 0.0;
    }
}

/* kappa = div n, same isotropic stencil applied to the normal field. */
static double div_normal_at(const orc_sim *s, int i, int j) {
    double acc = 0.0;
    for (int q = 0; q < Q; ++q) {
        double ax, ay, m;
        normal_at(s, i + EX[q], j + EY[q], &ax, &ay, &m);
        acc += WQ[q] * (EX[q] * ax + EY[q] * ay);
    }
    return acc / CS2;
}

/* ------------------------------------------------------------------------ */
/* Macroscopic fields (the "update" bullets of the three algorithm lists)    */
/* ------------------------------------------------------------------------ */

static double lin_interp(const orc_params *p, double phi, double va, double vb) {
    return vb + (phi - p->phi_b) / (p->phi_a - p->phi_b) * (va - vb);
}

/* Langmuir equation of state, Eq. (EOS).  With beta = 0 (a clean interface)
 * the tension is sigma_o whatever c is: the logarithm is not formed, so a
 * passive surfactant that reaches c_max leaves the tension defined. */
static double sigma_of_c(const orc_params *p, double c) {
    if (p->beta == 0.0) return p->sigma_o;
    return p->sigma_o * (1.0 + p->beta * log(1.0 - c / p->c_max));
}

static void compute_moments(orc_sim *s) {
    int N = s->N;
    int coupled = (s->p.mode == 0);
#pragma omp parallel for schedule(static)
    for (int x = 0; x < N; ++x) {
        double sf = 0, sh = 0, sg = 0, gx = 0, gy = 0;
        for (int q = 0; q < Q; ++q) {
            sf += s->f[(size_t)q * N + x];
            sh += s->h[(size_t)q * N + x];
            if (coupled) {
                double v = s->g[(size_t)q * N + x];
                sg += v;
                gx += EX[q] * v;
                gy += EY[q] * v;
            }
        }
        s->phi[x] = sf;   /* phi = sum f  (App. C) */
        s->c[x] = sh;     /* c = sum h    (Sec. 3) */
        s->Pstar[x] = sg; /* sum g        (App. D) */
        s->jx[x] = gx;
        s->jy[x] = gy;
        s->rho[x] = lin_interp(&s->p, sf, s->p.rho_a, s->p.rho_b);
        s->nu[x] = lin_interp(&s->p, sf, s->p.nu_a, s->p.nu_b);
        s->sig[x] = sigma_of_c(&s->p, sh);
        s->psistar[x] = sg - s->rho[x] * CS2;
    }
}

static void compute_macroscopic(orc_sim *s) {
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    int coupled = (p->mode == 0);
    double phim = 0.5 * (p->phi_a + p->phi_b);
    double dphi = p->phi_a - p->phi_b;
    double Nsig = p->sigma_literal ? 1.0 : 1.5 * p->W / (dphi * dphi);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            double phi = s->phi[x], c = s->c[x];
            double nxx, nyy, mag;
            normal_at(s, i, j, &nxx, &nyy, &mag);
            s->nxv[x] = nxx;
            s->nyv[x] = nyy;
            s->gmag[x] = mag;
            /* theta (Eq. theta) and theta_c (Eq. ISS) */
            s->theta[x] = (4.0 / p->W) * (p->phi_a - phi) * (phi - p->phi_b) / dphi;
            s->thetac[x] = (8.0 * c / p->W) * (phim - phi) / dphi;
            if (!coupled) {
                s->ux[x] = s->ufx[x];
                s->uy[x] = s->ufy[x];
                s->P[x] = 0.0;
                s->psi[x] = 0.0;
                continue;
            }
            double kap = div_normal_at(s, i, j);
            s->kappa[x] = kap;
            /* surface-tension force, Eq. (Fs): capillary + Marangoni */
            double sgx, sgy;
            grad_at(s, s->sig, i, j, &sgx, &sgy);
            double ndots = nxx * sgx + nyy * sgy;
            double msx = sgx - nxx * ndots, msy = sgy - nyy * ndots; /* (I - nn) grad sigma */
            double g2 = mag * mag;
            double sg = s->sig[x];
            double Fsx = Nsig * (-sg * g2 * kap * nxx + g2 * msx);
            double Fsy = Nsig * (-sg * g2 * kap * nyy + g2 * msy);
            s->Fsx[x] = Fsx;
            s->Fsy[x] = Fsy;
            double Ftx = Fsx + p->fext_x, Fty = Fsy + p->fext_y;
            s->Ftx[x] = Ftx;
            s->Fty[x] = Fty;
            double rho = s->rho[x];
            /* c_s^2 rho u = sum e g + (1/2) c_s^2 F_t  (App. D) */
            double ux = (s->jx[x] + 0.5 * CS2 * Ftx) / (CS2 * rho);
            double uy = (s->jy[x] + 0.5 * CS2 * Fty) / (CS2 * rho);
            s->ux[x] = ux;
            s->uy[x] = uy;
            /* F_p = -grad psi, psi = P - rho cs2 taken with P* = sum g */
            double pgx, pgy;
            grad_at(s, s->psistar, i, j, &pgx, &pgy);
            double Fpx = -pgx, Fpy = -pgy;
            s->Fpx[x] = Fpx;
            s->Fpy[x] = Fpy;
            double G00 = Fpx * ux + Fpy * uy;
            double P = s->Pstar[x] + 0.5 * G00; /* P = sum g + sigma_00 / 2 */
            s->P[x] = P;
            s->psi[x] = P - rho * CS2;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Collisions (literal matrix form)                                          */
/* ------------------------------------------------------------------------ */

/* Equilibrium central moments of the advection-diffusion lattices f and h:
 * (s, Kflux_x, Kflux_y, cs2 s, cs2 s, 0, 0, 0, cs2^2 s). */
static void eq_scalar(double s0, double qx, double qy, double *eq) {
    eq[0] = s0;
    eq[1] = qx;
    eq[2] = qy;
    eq[3] = CS2 * s0;
    eq[4] = CS2 * s0;
    eq[5] = 0.0;
    eq[6] = 0.0;
    eq[7] = 0.0;
    eq[8] = CS2 * CS2 * s0;
}

/* Equilibrium central moments of the flow lattice, with -psi u in first order. */
static void eq_flow(double P, double psi, double rho, double ux, double uy, double *eq) {
    eq[0] = P;
    eq[1] = -psi * ux;
    eq[2] = -psi * uy;
    eq[3] = CS2 * P + psi * ux * ux;
    eq[4] = CS2 * P + psi * uy * uy;
    eq[5] = psi * ux * uy;
    eq[6] = -psi * (ux * ux + CS2) * uy;
    eq[7] = -psi * (uy * uy + CS2) * ux;
    eq[8] = CS2 * CS2 * CS2 * rho + psi * (ux * ux + CS2) * (uy * uy + CS2);
}

/* Central moments of the source terms (App. D). */
static void source_flow(double ux, double uy, double Ftx, double Fty, double Fpx, double Fpy,
                        double *sg) {
    double G = Fpx * ux + Fpy * uy;
    sg[0] = G;
    sg[1] = CS2 * Ftx - ux * G;
    sg[2] = CS2 * Fty - uy * G;
    sg[3] = 2.0 * CS2 * Fpx * ux + (ux * ux + CS2) * G;
    sg[4] = 2.0 * CS2 * Fpy * uy + (uy * uy + CS2) * G;
    sg[5] = CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;
    sg[6] = 0.0;
    sg[7] = 0.0;
    sg[8] = 0.0;
}

/* One advection-diffusion collision: raw moments P a, central moments F(u) .,
 * relax with diag(1, w, w, 1, ..., 1) towards eq, back with F^-1 then P^-1. */
static void collide_scalar(const double Pm[Q][Q], const double F[Q][Q], const double Fi[Q][Q],
                           double w1, const double *eq, const double *in, double *out) {
    double raw[Q], cm[Q], cmt[Q], rawt[Q];
    matvec(Pm, in, raw);
    matvec(F, raw, cm);
    for (int k = 0; k < Q; ++k) {
        double lam = (k == 1 || k == 2) ? w1 : 1.0;
        cmt[k] = cm[k] + lam * (eq[k] - cm[k]);
    }
    matvec(Fi, cmt, rawt);
    matvec(PINV, rawt, out);
}

static double rate_from_coeff(double coeff) { return 1.0 / (coeff / CS2 + 0.5); }

static void collide_all(orc_sim *s) {
    const orc_params *p = &s->p;
    int N = s->N;
    int coupled = (p->mode == 0);
    double w_kappa = rate_from_coeff(p->M_phi); /* M_phi = cs2 (1/w - 1/2) */
    double w_chi = rate_from_coeff(p->D_s);     /* D_s = cs2 (1/w - 1/2) */
    double w_zeta = rate_from_coeff(p->zeta);
#pragma omp parallel for schedule(static)
    for (int x = 0; x < N; ++x) {
        double F[Q][Q], Fi[Q][Q];
        double ux = s->ux[x], uy = s->uy[x];
        build_frame(ux, uy, -1.0, F);
        build_frame(ux, uy, +1.0, Fi);
        double in[Q], out[Q], eq[Q];

        /* f: CACE, kappa^eq = (phi, M theta n, cs2 phi, cs2 phi, 0, 0, 0, cs4 phi) */
        for (int q = 0; q < Q; ++q) in[q] = s->f[(size_t)q * N + x];
        double phi = s->phi[x];
        eq_scalar(phi, p->M_phi * s->theta[x] * s->nxv[x], p->M_phi * s->theta[x] * s->nyv[x], eq);
        collide_scalar(s->P_matrix, F, Fi, w_kappa, eq, in, out);
        for (int q = 0; q < Q; ++q) s->ft[(size_t)q * N + x] = out[q];

        /* h: interface-bound scalar, chi^eq = (c, D_s theta_c n, cs2 c, cs2 c, 0, 0, 0, cs4 c) */
        for (int q = 0; q < Q; ++q) in[q] = s->h[(size_t)q * N + x];
        eq_scalar(s->c[x], p->D_s * s->thetac[x] * s->nxv[x], p->D_s * s->thetac[x] * s->nyv[x], eq);
        collide_scalar(s->P_matrix, F, Fi, w_chi, eq, in, out);
        for (int q = 0; q < Q; ++q) s->ht[(size_t)q * N + x] = out[q];

        if (!coupled) continue;

        /* g: flow, Eq. (centralmomentLBE2fluidflow) */
        double raw[Q], cm[Q], src[Q], hat[Q], hateq[Q], hatsrc[Q], hatt[Q], cmt[Q], rawt[Q];
        for (int q = 0; q < Q; ++q) in[q] = s->g[(size_t)q * N + x];
        matvec(s->P_matrix, in, raw);
        matvec(F, raw, cm);
        eq_flow(s->P[x], s->psi[x], s->rho[x], ux, uy, eq);
        source_flow(ux, uy, s->Ftx[x], s->Fty[x], s->Fpx[x], s->Fpy[x], src);
        matvec(s->Bm, cm, hat);
        matvec(s->Bm, eq, hateq);
        matvec(s->Bm, src, hatsrc);
        double w_nu = rate_from_coeff(s->nu[x]);
        double lam[Q] = {1, 1, 1, w_zeta, w_nu, w_nu, 1, 1, 1};
        for (int k = 0; k < Q; ++k)
            hatt[k] = hat[k] + lam[k] * (hateq[k] - hat[k]) + (1.0 - 0.5 * lam[k]) * hatsrc[k];
        matvec(s->Binv, hatt, cmt);
        matvec(Fi, cmt, rawt);
        matvec(PINV, rawt, out);
        for (int q = 0; q < Q; ++q) s->gt[(size_t)q * N + x] = out[q];
    }
}

/* ------------------------------------------------------------------------ */
/* Streaming with boundary conditions                                        */
/* ------------------------------------------------------------------------ */

/* Pull: a(x, t+1) = a~(x - e_a, t).  Periodic in x (and y without walls).
 * With walls, a population whose source lies beyond a wall is the reflected
 * post-collision population of the same node (half-way bounce-back); the flow
 * lattice adds 2 w_a rho (e_a . u_w). */
static void stream_all(orc_sim *s) {
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny, N = s->N;
    int coupled = (p->mode == 0);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            for (int q = 0; q < Q; ++q) {
                int si = wrap(i - EX[q], nx);
                int sj = j - EY[q];
                size_t dst = (size_t)q * N + x;
                if (!p->walls_y || (sj >= 0 && sj < ny)) {
                    size_t src = (size_t)q * N + (size_t)wrap(sj, ny) * nx + si;
                    s->f[dst] = s->ft[src];
                    s->h[dst] = s->ht[src];
                    if (coupled) s->g[dst] = s->gt[src];
                } else {
                    size_t src = (size_t)OPP[q] * N + x;
                    double uw = (sj < 0) ? -p->u_wall : p->u_wall;
                    s->f[dst] = s->ft[src];
                    s->h[dst] = s->ht[src];
                    if (coupled) s->g[dst] = s->gt[src] + 2.0 * WQ[q] * s->rho[x] * (EX[q] * uw);
                }
            }
        }
    }
}

void orc_step(orc_sim *s, int nsteps) {
    for (int t = 0; t < nsteps; ++t) {
        compute_moments(s);     /* zeroth / first moments of the current populations */
        compute_macroscopic(s); /* normal, theta, theta_c, forces, u, P */
        collide_all(s);         /* f, h, g central-moment collisions */
        stream_all(s);          /* streaming with bounce-back walls */
        s->step += 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Initialisation: discrete equilibria of the given fields                   */
/* ------------------------------------------------------------------------ */

static void equilibrium_pops(orc_sim *s, int which_f, int which_h, int which_g) {
    const orc_params *p = &s->p;
    int N = s->N;
#pragma omp parallel for schedule(static)
    for (int x = 0; x < N; ++x) {
        double Fi[Q][Q], eq[Q], raw[Q], out[Q];
        build_frame(s->ux[x], s->uy[x], +1.0, Fi);
        if (which_f) {
            eq_scalar(s->phi[x], p->M_phi * s->theta[x] * s->nxv[x],
                      p->M_phi * s->theta[x] * s->nyv[x], eq);
            matvec(Fi, eq, raw);
            matvec(PINV, raw, out);
            for (int q = 0; q < Q; ++q) s->f[(size_t)q * N + x] = out[q];
        }
        if (which_h) {
            eq_scalar(s->c[x], p->D_s * s->thetac[x] * s->nxv[x],
                      p->D_s * s->thetac[x] * s->nyv[x], eq);
            matvec(Fi, eq, raw);
            matvec(PINV, raw, out);
            for (int q = 0; q < Q; ++q) s->h[(size_t)q * N + x] = out[q];
        }
        if (which_g && p->mode == 0) {
            eq_flow(s->P[x], s->psi[x], s->rho[x], s->ux[x], s->uy[x], eq);
            matvec(Fi, eq, raw);
            matvec(PINV, raw, out);
            for (int q = 0; q < Q; ++q) s->g[(size_t)q * N + x] = out[q];
        }
    }
}

static void init_geometry_from_fields(orc_sim *s) {
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    double phim = 0.5 * (p->phi_a + p->phi_b);
    double dphi = p->phi_a - p->phi_b;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            double nxx, nyy, mag;
            normal_at(s, i, j, &nxx, &nyy, &mag);
            s->nxv[x] = nxx;
            s->nyv[x] = nyy;
            s->gmag[x] = mag;
            double phi = s->phi[x];
            s->theta[x] = (4.0 / p->W) * (p->phi_a - phi) * (phi - p->phi_b) / dphi;
            s->thetac[x] = (8.0 * s->c[x] / p->W) * (phim - phi) / dphi;
            s->rho[x] = lin_interp(p, phi, p->rho_a, p->rho_b);
        }
}

int orc_init(orc_sim *s, const double *phi, const double *c, const double *ux, const double *uy,
             const double *P) {
    int N = s->N;
    for (int x = 0; x < N; ++x) {
        s->phi[x] = phi[x];
        s->c[x] = c[x];
        s->ux[x] = ux[x];
        s->uy[x] = uy[x];
        s->ufx[x] = ux[x];
        s->ufy[x] = uy[x];
    }
    init_geometry_from_fields(s);
    /* Default pressure: uniform, cs2 times the mean of the phase densities (the
     * fluid at rest; psi = P - rho cs2 then carries the density contrast).  With
     * equal densities this is rho cs2 everywhere. */
    const double P_rest = CS2 * 0.5 * (s->p.rho_a + s->p.rho_b);
    for (int x = 0; x < N; ++x) {
        s->P[x] = P ? P[x] : P_rest;
        s->psi[x] = s->P[x] - s->rho[x] * CS2;
    }
    equilibrium_pops(s, 1, 1, 1);
    s->step = 0;
    return 0;
}

void orc_reset_f(orc_sim *s, const double *phi) {
    int N = s->N;
    /* keep the current velocity: macroscopic fields of the current state first */
    compute_moments(s);
    compute_macroscopic(s);
    for (int x = 0; x < N; ++x) s->phi[x] = phi[x];
    init_geometry_from_fields(s);
    equilibrium_pops(s, 1, 0, 0);
}

void orc_set_velocity(orc_sim *s, const double *ux, const double *uy) {
    for (int x = 0; x < s->N; ++x) {
        s->ufx[x] = ux[x];
        s->ufy[x] = uy[x];
    }
}

/* ------------------------------------------------------------------------ */
/* Outputs                                                                   */
/* ------------------------------------------------------------------------ */

void orc_fields(orc_sim *s, double *phi, double *c, double *ux, double *uy, double *P) {
    compute_moments(s);
    compute_macroscopic(s);
    size_t bytes = sizeof(double) * (size_t)s->N;
    if (phi) memcpy(phi, s->phi, bytes);
    if (c) memcpy(c, s->c, bytes);
    if (ux) memcpy(ux, s->ux, bytes);
    if (uy) memcpy(uy, s->uy, bytes);
    if (P) memcpy(P, s->P, bytes);
}

void orc_geometry(orc_sim *s, double *nx_, double *ny_, double *gmag, double *kappa,
                  double *Fsx, double *Fsy) {
    compute_moments(s);
    compute_macroscopic(s);
    int coupled = (s->p.mode == 0);
    if (!coupled) {
        /* curvature is only needed by the flow lattice; compute it here on demand */
        int nx = s->p.nx, ny = s->p.ny;
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) s->kappa[(size_t)j * nx + i] = div_normal_at(s, i, j);
    }
    size_t bytes = sizeof(double) * (size_t)s->N;
    if (nx_) memcpy(nx_, s->nxv, bytes);
    if (ny_) memcpy(ny_, s->nyv, bytes);
    if (gmag) memcpy(gmag, s->gmag, bytes);
    if (kappa) memcpy(kappa, s->kappa, bytes);
    if (Fsx) memcpy(Fsx, s->Fsx, bytes);
    if (Fsy) memcpy(Fsy, s->Fsy, bytes);
}

void orc_get_pops(const orc_sim *s, double *f, double *h, double *g) {
    size_t bytes = sizeof(double) * Q * (size_t)s->N;
    if (f) memcpy(f, s->f, bytes);
    if (h) memcpy(h, s->h, bytes);
    if (g) memcpy(g, s->g, bytes);
}

void orc_set_pops(orc_sim *s, const double *f, const double *h, const double *g) {
    size_t bytes = sizeof(double) * Q * (size_t)s->N;
    if (f) memcpy(s->f, f, bytes);
    if (h) memcpy(s->h, h, bytes);
    if (g) memcpy(s->g, g, bytes);
}

/* Periodic-aware centroid along one axis: circular mean of the phi-weighted
 * positions when the axis is periodic, plain mean otherwise. */
/* Phase indicator of the drop: (phi - phi_b) / (phi_a - phi_b) clipped to
 * [0, 1].  The drop's axes L and B (Sec. 4.3, D = (L - B) / (L + B)) belong to
 * the drop region; the clip keeps the small overshoot and undershoot of phi
 * away from the interface out of the shape moments, where their distance
 * from the drop would weigh them heavily. */
static double drop_indicator(const orc_params *p, double phi) {
    double w = (phi - p->phi_b) / (p->phi_a - p->phi_b);
    return w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
}

static double axis_centroid(const orc_sim *s, int axis, int periodic) {
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny, n = axis == 0 ? nx : ny;
    double s0 = 0, a = 0, b = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            double phi = s->phi[x];
            if (!isfinite(phi)) continue;
            double w = drop_indicator(p, phi);
            double pos = (axis == 0 ? i : j) + 0.5;
            if (periodic) {
                double ang = 2.0 * M_PI * pos / n;
                a += w * cos(ang);
                b += w * sin(ang);
            } else {
                a += w * pos;
            }
            s0 += w;
        }
    if (s0 == 0) return 0.5 * n;
    if (!periodic) return a / s0;
    double ang = atan2(b, a);
    if (ang < 0) ang += 2.0 * M_PI;
    return ang * n / (2.0 * M_PI);
}

static double min_image(double d, int n, int periodic) {
    if (!periodic) return d;
    while (d >= 0.5 * n) d -= n;
    while (d < -0.5 * n) d += n;
    return d;
}

/* Sums of phi and c, the centroid and second moments of the drop indicator
 * (the drop shape: L = 4 sqrt(l1), B = 4 sqrt(l2), D = (L - B) / (L + B)), max |u|,
 * and counts of non-finite cells and of cells with negative sigma(c).
 * Periodic axes use the circular-mean centroid and minimum-image distances. */
void orc_diagnostics(orc_sim *s, orc_diag *out) {
    compute_moments(s);
    compute_macroscopic(s);
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    int py = !p->walls_y;
    double s0 = 0, sc = 0, umax = 0;
    long long nonfin = 0, neg = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            double phi = s->phi[x], c = s->c[x];
            if (!isfinite(phi) || !isfinite(c) || !isfinite(s->ux[x]) || !isfinite(s->uy[x])) {
                nonfin++;
                continue;
            }
            s0 += phi;
            sc += c;
            double um = sqrt(s->ux[x] * s->ux[x] + s->uy[x] * s->uy[x]);
            if (um > umax) umax = um;
            double arg = 1.0 - c / p->c_max;
            if (p->beta != 0.0 && (arg <= 0.0 || 1.0 + p->beta * log(arg) < 0.0)) neg++;
        }
    double xc = axis_centroid(s, 0, 1), yc = axis_centroid(s, 1, py);
    double Ixx = 0, Iyy = 0, Ixy = 0, sw = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            double phi = s->phi[x];
            if (!isfinite(phi) || !isfinite(s->c[x]) || !isfinite(s->ux[x]) || !isfinite(s->uy[x]))
                continue;
            double w = drop_indicator(p, phi);
            double dx = min_image(i + 0.5 - xc, nx, 1), dy = min_image(j + 0.5 - yc, ny, py);
            Ixx += w * dx * dx;
            Iyy += w * dy * dy;
            Ixy += w * dx * dy;
            sw += w;
        }
    if (sw != 0) {
        Ixx /= sw;
        Iyy /= sw;
        Ixy /= sw;
    }
    double tr = Ixx + Iyy, det = Ixx * Iyy - Ixy * Ixy;
    double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
    double l1 = 0.5 * tr + disc, l2 = fmax(0.5 * tr - disc, 0.0);
    double L = 4.0 * sqrt(l1), B = 4.0 * sqrt(l2);
    out->step = s->step;
    out->sum_phi = s0;
    out->sum_c = sc;
    out->L = L;
    out->B = B;
    out->D = (L + B) > 0 ? (L - B) / (L + B) : 0.0;
    out->xc = xc;
    out->yc = yc;
    out->umax = umax;
    out->nonfinite = nonfin;
    out->sigma_neg = neg;
}
