/*
 * FP64 CPU oracle of the D3Q27 form of the two scalar central-moment lattices
 * of Schupbach & Premnath (arXiv 2504.09024) under a prescribed velocity.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * bench's CPU-baseline leg, never by the product path.  No code is shared with
 * the CUDA library.
 *
 * Plain and slow on purpose: every collision multiplies the literal 27 x 27
 * matrices P, F(u), F^-1(u) and P^-1, one cell at a time, in the order of the
 * paper's algorithm lists (Sec. 3 for h, App. C for f): zeroth moments, normal
 * and theta, raw moments, central moments, relaxation, back to raw moments,
 * back to populations, then streaming.
 *
 * The paper states the scheme on D2Q9 and calls the 3-D extension
 * straightforward (Sec. 5).  Readings that carry each D2Q9 step to D3Q27:
 *  - velocities e in {-1, 0, 1}^3, weights the products of the 1-D weights
 *    (2/3, 1/6, 1/6): 8/27 (rest), 2/27 (faces), 1/54 (edges), 1/216 (corners).
 *  - moment basis |e_x^m e_y^n e_z^p>, m, n, p in {0, 1, 2}: the 27-moment
 *    tensor-product counterpart of Eq. (Pi), which is the 9-moment tensor
 *    product in 2-D.  P^-1 is obtained by Gauss-Jordan elimination.
 *  - F(u) and F^-1(u) from the binomial expansion of (e_i - u_i)^m_i on each
 *    axis, the 3-D form of Eq. (cmscalar).
 *  - equilibrium central moments: the continuous Maxwellian central moments
 *    of density s, s * mu(m) mu(n) mu(p) with mu(0) = 1, mu(1) = 0,
 *    mu(2) = cs2 (matching principle of Sec. 3), with the three first-order
 *    ones replaced by the extended flux K theta n_i (K = M_phi for f with theta
 *    of Eq. theta; K = D_s for h with theta_c of Eq. ISS).
 *  - relaxation: the first-order moments with w, K = cs2 (1/w - 1/2); all other
 *    moments with rate 1, as in the D2Q9 schemes.
 *  - gradient: d_i A = (1/cs2) sum_a w_a e_ai A(x + e_a), periodic in x, y, z;
 *    n = grad phi / |grad phi|, n = 0 where |grad phi| <= 1e-12.
 *  - initial populations: the discrete equilibria of the given fields.
 *
 * The flow lattice (mode 1) carries App. D to D3Q27 by the same product rule:
 *  - equilibrium central moments rho cs2 mu(m) mu(n) mu(p) + psi W(m, u_x)
 *    W(n, u_y) W(p, u_z), W = (1, -u, cs2 + u^2) the central moments of the
 *    1-D weights about u; on D2Q9 this is exactly the printed equilibrium;
 *  - source central moments: Gamma = F_p.u at zeroth order, cs2 F_t,i - u_i
 *    Gamma at first, 2 cs2 F_p,i u_i + (u_i^2 + cs2) Gamma on the diagonal
 *    and cs2 (F_p,i u_j + F_p,j u_i) + u_i u_j Gamma off it at second order,
 *    zero above (as printed on D2Q9);
 *  - second-order moments combined into the trace m200 + m020 + m002,
 *    relaxed with the rate of zeta (zeta = cs2 (1/w - 1/2), as on D2Q9), and
 *    the deviatoric m200 - m020, m200 - m002, m110, m101, m011 with the rate
 *    of nu; every other moment with rate 1 (the D2Q9 pattern of Eq.
 *    combinedforms);
 *  - curvature kappa = div n with the same stencil, F_s = N (-sigma
 *    |grad phi|^2 kappa n + |grad phi|^2 (I - nn) grad sigma), N as on D2Q9;
 *    u = (sum e g + cs2 F_t / 2) / (cs2 rho), F_p = -grad(P* - rho cs2),
 *    P = P* + Gamma / 2;
 *  - walls: half-way bounce-back at y = 0 and y = ny moving with -u_wall and
 *    +u_wall along x (g adds 2 w_a rho e_a.u_w); fields are mirrored about
 *    the wall planes for the stencils; x and z periodic.
 */
#include "lbm_oracle3.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q3 27

/* The 27 velocities: rest, faces, edges, corners. */
static const int E3[Q3][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
    {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1},
};

static const double CS2 = 1.0 / 3.0;
static const double EPS_N = 1e-12;

/* Weight of velocity a by its number of non-zero components. */
static double weight(int a) {
    int k = abs(E3[a][0]) + abs(E3[a][1]) + abs(E3[a][2]);
    static const double W_BY_K[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    return W_BY_K[k];
}

/* Moment k has orders (m, n, p) = (k % 3, (k / 3) % 3, k / 9). */
static int mom(int k, int axis) {
    if (axis == 0) return k % 3;
    if (axis == 1) return (k / 3) % 3;
    return k / 9;
}

static int is_first_order(int k) { return mom(k, 0) + mom(k, 1) + mom(k, 2) == 1; }

struct orc3_sim {
    orc3_params p;
    int N;
    long long step;
    double *f, *h;        /* [27][N] post-streaming populations */
    double *ft, *ht;      /* [27][N] post-collision populations */
    double *phi, *c;
    double *ux, *uy, *uz; /* velocity: prescribed (mode 0) or of the flow lattice (mode 1) */
    double *nv[3];        /* unit normal */
    double *theta, *thetac;
    double Pm[Q3][Q3], Pinv[Q3][Q3];
    /* flow lattice (mode 1) */
    double *g, *gt;                       /* [27][N] */
    double *Pstar, *jv[3], *rho, *nu, *sig, *psistar, *P, *psi, *gmag;
    double *Ft[3], *Fp[3];
    double Bm[Q3][Q3], Binv[Q3][Q3];
};

/* ------------------------------------------------------------------------ */
/* Matrices                                                                  */
/* ------------------------------------------------------------------------ */

static double ipow(double x, int n) {
    double r = 1.0;
    for (int t = 0; t < n; ++t) r *= x;
    return r;
}

static double binom(int n, int k) {
    double r = 1.0;
    for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
    return r;
}

/* P_{k,a} = e_ax^m e_ay^n e_az^p. */
static void build_P(double P[Q3][Q3]) {
    for (int k = 0; k < Q3; ++k)
        for (int a = 0; a < Q3; ++a)
            P[k][a] = ipow(E3[a][0], mom(k, 0)) * ipow(E3[a][1], mom(k, 1)) * ipow(E3[a][2], mom(k, 2));
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success. */
static int invert(const double A[Q3][Q3], double out[Q3][Q3]) {
    double M[Q3][2 * Q3];
    for (int r = 0; r < Q3; ++r)
        for (int col = 0; col < 2 * Q3; ++col)
            M[r][col] = col < Q3 ? A[r][col] : (col - Q3 == r ? 1.0 : 0.0);
    for (int col = 0; col < Q3; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q3; ++r)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (fabs(M[piv][col]) < 1e-12) return -1;
        if (piv != col)
            for (int t = 0; t < 2 * Q3; ++t) {
                double tmp = M[col][t];
                M[col][t] = M[piv][t];
                M[piv][t] = tmp;
            }
        double d = M[col][col];
        for (int t = 0; t < 2 * Q3; ++t) M[col][t] /= d;
        for (int r = 0; r < Q3; ++r) {
            if (r == col || M[r][col] == 0.0) continue;
            double m = M[r][col];
            for (int t = 0; t < 2 * Q3; ++t) M[r][t] -= m * M[col][t];
        }
    }
    for (int r = 0; r < Q3; ++r)
        for (int col = 0; col < Q3; ++col) out[r][col] = M[r][col + Q3];
    return 0;
}

/* Frame change of the moment (m, n, p) by the binomial expansion on each axis:
 *   kappa_mnp = sum C(m,j) C(n,k) C(p,l) (s u_x)^(m-j) (s u_y)^(n-k) (s u_z)^(p-l) kappa'_jkl.
 * s = -1 gives F(u) (raw to central), s = +1 gives F^-1(u). */
static void build_frame(double ux, double uy, double uz, double s, double F[Q3][Q3]) {
    const double u[3] = {s * ux, s * uy, s * uz};
    for (int r = 0; r < Q3; ++r)
        for (int col = 0; col < Q3; ++col) {
            double v = 1.0;
            for (int ax = 0; ax < 3; ++ax) {
                int m = mom(r, ax), j = mom(col, ax);
                if (j > m) {
                    v = 0.0;
                    break;
                }
                v *= binom(m, j) * ipow(u[ax], m - j);
            }
            F[r][col] = v;
        }
}

static void matvec(const double A[Q3][Q3], const double *x, double *y) {
    for (int r = 0; r < Q3; ++r) {
        double acc = 0.0;
        for (int col = 0; col < Q3; ++col) acc += A[r][col] * x[col];
        y[r] = acc;
    }
}

/* B combines the diagonal second-order moments: the trace m200 + m020 + m002
 * (row of m200) and the deviatoric m200 - m020 (row of m020) and
 * m200 - m002 (row of m002); identity elsewhere.  B^-1 by elimination. */
static void build_B(double B[Q3][Q3]) {
    memset(B, 0, sizeof(double) * Q3 * Q3);
    for (int k = 0; k < Q3; ++k) B[k][k] = 1.0;
    const int a = 2, b = 6, c = 18; /* m200, m020, m002 */
    B[a][a] = 1.0;  B[a][b] = 1.0;  B[a][c] = 1.0;
    B[b][a] = 1.0;  B[b][b] = -1.0; B[b][c] = 0.0;
    B[c][a] = 1.0;  B[c][b] = 0.0;  B[c][c] = -1.0;
}

static void copy_out(const double A[Q3][Q3], double out[729]) {
    for (int r = 0; r < Q3; ++r)
        for (int col = 0; col < Q3; ++col) out[r * Q3 + col] = A[r][col];
}

void orc3_velocities(int out[81]) {
    for (int a = 0; a < Q3; ++a)
        for (int ax = 0; ax < 3; ++ax) out[3 * a + ax] = E3[a][ax];
}

void orc3_matrix_P(double out[729]) {
    double P[Q3][Q3];
    build_P(P);
    copy_out(P, out);
}

void orc3_matrix_Pinv(double out[729]) {
    double P[Q3][Q3], Pi[Q3][Q3];
    build_P(P);
    invert(P, Pi);
    copy_out(Pi, out);
}

void orc3_matrix_F(double ux, double uy, double uz, double out[729]) {
    double F[Q3][Q3];
    build_frame(ux, uy, uz, -1.0, F);
    copy_out(F, out);
}

void orc3_matrix_Finv(double ux, double uy, double uz, double out[729]) {
    double F[Q3][Q3];
    build_frame(ux, uy, uz, +1.0, F);
    copy_out(F, out);
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */

static double *alloc_d(size_t n) { return (double *)calloc(n, sizeof(double)); }

orc3_sim *orc3_create(const orc3_params *p) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || !(p->W > 0.0) || p->phi_a == p->phi_b) return NULL;
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    s->p = *p;
    s->N = p->nx * p->ny * p->nz;
    size_t N = (size_t)s->N;
    s->f = alloc_d(Q3 * N);
    s->h = alloc_d(Q3 * N);
    s->ft = alloc_d(Q3 * N);
    s->ht = alloc_d(Q3 * N);
    s->phi = alloc_d(N);
    s->c = alloc_d(N);
    s->ux = alloc_d(N);
    s->uy = alloc_d(N);
    s->uz = alloc_d(N);
    for (int ax = 0; ax < 3; ++ax) s->nv[ax] = alloc_d(N);
    s->theta = alloc_d(N);
    s->thetac = alloc_d(N);
    s->g = alloc_d(Q3 * N);
    s->gt = alloc_d(Q3 * N);
    s->Pstar = alloc_d(N);
    s->rho = alloc_d(N);
    s->nu = alloc_d(N);
    s->sig = alloc_d(N);
    s->psistar = alloc_d(N);
    s->P = alloc_d(N);
    s->psi = alloc_d(N);
    s->gmag = alloc_d(N);
    for (int ax = 0; ax < 3; ++ax) {
        s->jv[ax] = alloc_d(N);
        s->Ft[ax] = alloc_d(N);
        s->Fp[ax] = alloc_d(N);
    }
    build_P(s->Pm);
    build_B(s->Bm);
    if (invert(s->Pm, s->Pinv) != 0 || invert(s->Bm, s->Binv) != 0) {
        orc3_destroy(s);
        return NULL;
    }
    return s;
}

void orc3_destroy(orc3_sim *s) {
    if (!s) return;
    free(s->f);
    free(s->h);
    free(s->ft);
    free(s->ht);
    free(s->phi);
    free(s->c);
    free(s->ux);
    free(s->uy);
    free(s->uz);
    for (int ax = 0; ax < 3; ++ax) free(s->nv[ax]);
    free(s->theta);
    free(s->thetac);
    free(s->g);
    free(s->gt);
    free(s->Pstar);
    free(s->rho);
    free(s->nu);
    free(s->sig);
    free(s->psistar);
    free(s->P);
    free(s->psi);
    free(s->gmag);
    for (int ax = 0; ax < 3; ++ax) {
        free(s->jv[ax]);
        free(s->Ft[ax]);
        free(s->Fp[ax]);
    }
    free(s);
}

long long orc3_get_step(const orc3_sim *s) { return s->step; }

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

static size_t idx(const orc3_sim *s, int i, int j, int k) {
    return ((size_t)wrap(k, s->p.nz) * s->p.ny + wrap(j, s->p.ny)) * s->p.nx + wrap(i, s->p.nx);
}

/* Row of the extended field: periodic, or mirrored about the wall planes
 * y = 0 and y = ny (row -1-k is row k, row ny+k is row ny-1-k). */
static int ext_row(const orc3_sim *s, int j) {
    int ny = s->p.ny;
    if (!s->p.walls_y) return wrap(j, ny);
    while (j < 0 || j >= ny) {
        if (j < 0) j = -1 - j;
        if (j >= ny) j = 2 * ny - 1 - j;
    }
    return j;
}

static size_t sidx(const orc3_sim *s, int i, int j, int k) {
    return ((size_t)wrap(k, s->p.nz) * s->p.ny + ext_row(s, j)) * s->p.nx + wrap(i, s->p.nx);
}

/* Isotropic gradient, d_i A = (1/cs2) sum_a w_a e_ai A(x + e_a). */
static void grad_at(const orc3_sim *s, const double *a, int i, int j, int k, double g[3]) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < Q3; ++q) {
        double v = a[sidx(s, i + E3[q][0], j + E3[q][1], k + E3[q][2])];
        for (int ax = 0; ax < 3; ++ax) acc[ax] += weight(q) * E3[q][ax] * v;
    }
    for (int ax = 0; ax < 3; ++ax) g[ax] = acc[ax] / CS2;
}

void orc3_gradient(const orc3_sim *s, const double *a, double *gx, double *gy, double *gz) {
    const orc3_params *p = &s->p;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) {
                double g[3];
                grad_at(s, a, i, j, k, g);
                size_t x = idx(s, i, j, k);
                gx[x] = g[0];
                gy[x] = g[1];
                gz[x] = g[2];
            }
}

static double lin_interp(const orc3_params *p, double phi, double va, double vb) {
    return vb + (phi - p->phi_b) / (p->phi_a - p->phi_b) * (va - vb);
}

/* Langmuir equation of state, Eq. (EOS); sigma_o whatever c at beta = 0. */
static double sigma_of_c(const orc3_params *p, double c) {
    if (p->beta == 0.0) return p->sigma_o;
    return p->sigma_o * (1.0 + p->beta * log(1.0 - c / p->c_max));
}

/* phi = sum f (App. C), c = sum h (Sec. 3); with the flow lattice also
 * P* = sum g, j = sum e g, rho, nu, sigma(c) and psi* = P* - rho cs2 (App. D). */
static void compute_moments(orc3_sim *s) {
    const orc3_params *p = &s->p;
    size_t N = (size_t)s->N;
    const int coupled = p->mode == 1;
#pragma omp parallel for schedule(static)
    for (size_t x = 0; x < N; ++x) {
        double sf = 0.0, sh = 0.0, sg = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < Q3; ++q) {
            sf += s->f[q * N + x];
            sh += s->h[q * N + x];
            if (coupled) {
                double v = s->g[q * N + x];
                sg += v;
                for (int ax = 0; ax < 3; ++ax) j[ax] += E3[q][ax] * v;
            }
        }
        s->phi[x] = sf;
        s->c[x] = sh;
        if (!coupled) continue;
        s->Pstar[x] = sg;
        for (int ax = 0; ax < 3; ++ax) s->jv[ax][x] = j[ax];
        s->rho[x] = lin_interp(p, sf, p->rho_a, p->rho_b);
        s->nu[x] = lin_interp(p, sf, p->nu_a, p->nu_b);
        s->sig[x] = sigma_of_c(p, sh);
        s->psistar[x] = sg - s->rho[x] * CS2;
    }
}

/* Unit normal n = grad phi / |grad phi| at any (possibly ghost) position. */
static void normal_at(const orc3_sim *s, int i, int j, int k, double n[3], double *mag) {
    double g[3];
    grad_at(s, s->phi, i, j, k, g);
    double m = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    *mag = m;
    for (int ax = 0; ax < 3; ++ax) n[ax] = m > EPS_N ? g[ax] / m : 0.0;
}

/* kappa = div n, the same stencil applied to the normal field. */
static double div_normal_at(const orc3_sim *s, int i, int j, int k) {
    double acc = 0.0;
    for (int q = 0; q < Q3; ++q) {
        double n[3], m;
        normal_at(s, i + E3[q][0], j + E3[q][1], k + E3[q][2], n, &m);
        acc += weight(q) * (E3[q][0] * n[0] + E3[q][1] * n[1] + E3[q][2] * n[2]);
    }
    return acc / CS2;
}

/* Normal, theta (Eq. theta) and theta_c (Eq. ISS) of the current phi and c;
 * with the flow lattice (and with_flow) also the forces, u and P of App. D. */
static void compute_geometry(orc3_sim *s, int with_flow) {
    const orc3_params *p = &s->p;
    const double phim = 0.5 * (p->phi_a + p->phi_b);
    const double dphi = p->phi_a - p->phi_b;
    const int coupled = p->mode == 1 && with_flow;
    const double Nsig = p->sigma_literal ? 1.0 : 1.5 * p->W / (dphi * dphi);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) {
                size_t x = idx(s, i, j, k);
                double n[3], m;
                normal_at(s, i, j, k, n, &m);
                for (int ax = 0; ax < 3; ++ax) s->nv[ax][x] = n[ax];
                s->gmag[x] = m;
                double phi = s->phi[x];
                s->theta[x] = (4.0 / p->W) * (p->phi_a - phi) * (phi - p->phi_b) / dphi;
                s->thetac[x] = (8.0 * s->c[x] / p->W) * (phim - phi) / dphi;
                if (!coupled) continue;
                /* surface-tension force, Eq. (Fs): capillary + Marangoni */
                double kap = div_normal_at(s, i, j, k);
                double gs[3];
                grad_at(s, s->sig, i, j, k, gs);
                double nds = n[0] * gs[0] + n[1] * gs[1] + n[2] * gs[2];
                double g2 = m * m, sg = s->sig[x], rho = s->rho[x];
                double u[3];
                for (int ax = 0; ax < 3; ++ax) {
                    double Fs = Nsig * (-sg * g2 * kap * n[ax] + g2 * (gs[ax] - n[ax] * nds));
                    s->Ft[ax][x] = Fs + p->fext[ax];
                    /* cs2 rho u = sum e g + cs2 F_t / 2 (App. D) */
                    u[ax] = (s->jv[ax][x] + 0.5 * CS2 * s->Ft[ax][x]) / (CS2 * rho);
                }
                s->ux[x] = u[0];
                s->uy[x] = u[1];
                s->uz[x] = u[2];
                /* F_p = -grad psi*, P = P* + Gamma / 2, Gamma = F_p . u */
                double gp[3];
                grad_at(s, s->psistar, i, j, k, gp);
                double G = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    s->Fp[ax][x] = -gp[ax];
                    G += -gp[ax] * u[ax];
                }
                s->P[x] = s->Pstar[x] + 0.5 * G;
                s->psi[x] = s->P[x] - rho * CS2;
            }
}

/* Equilibrium central moments: s mu(m) mu(n) mu(p), first order = flux q. */
static void eq_scalar(double s0, const double q[3], double *eq) {
    static const double MU[3] = {1.0, 0.0, 1.0 / 3.0};
    for (int k = 0; k < Q3; ++k) eq[k] = s0 * MU[mom(k, 0)] * MU[mom(k, 1)] * MU[mom(k, 2)];
    eq[1] = q[0]; /* (1,0,0) */
    eq[3] = q[1]; /* (0,1,0) */
    eq[9] = q[2]; /* (0,0,1) */
}

static double rate_from_coeff(double coeff) { return 1.0 / (coeff / CS2 + 0.5); }

/* Flow equilibrium central moments: rho cs2 mu mu mu + psi W W W. */
static void eq_flow(double P, double psi, double rho, const double u[3], double *eq) {
    static const double MU_F[3] = {1.0, 0.0, CS2};
    for (int k = 0; k < Q3; ++k) {
        double w = 1.0, mu = 1.0;
        for (int ax = 0; ax < 3; ++ax) {
            int m = mom(k, ax);
            mu *= MU_F[m];
            w *= m == 0 ? 1.0 : m == 1 ? -u[ax] : CS2 + u[ax] * u[ax];
        }
        eq[k] = rho * CS2 * mu + psi * w;
    }
    (void)P;
}

/* Central moments of the source terms (App. D carried to three axes). */
static void source_flow(const double u[3], const double Ft[3], const double Fp[3], double *sg) {
    double G = Fp[0] * u[0] + Fp[1] * u[1] + Fp[2] * u[2];
    for (int k = 0; k < Q3; ++k) sg[k] = 0.0;
    sg[0] = G;
    const int first[3] = {1, 3, 9}, diag[3] = {2, 6, 18};
    for (int a = 0; a < 3; ++a) {
        sg[first[a]] = CS2 * Ft[a] - u[a] * G;
        sg[diag[a]] = 2.0 * CS2 * Fp[a] * u[a] + (u[a] * u[a] + CS2) * G;
    }
    /* off-diagonal second order: 110, 101, 011 */
    const int off[3][3] = {{4, 0, 1}, {10, 0, 2}, {12, 1, 2}};
    for (int t = 0; t < 3; ++t) {
        int k = off[t][0], a = off[t][1], b = off[t][2];
        sg[k] = CS2 * (Fp[a] * u[b] + Fp[b] * u[a]) + u[a] * u[b] * G;
    }
}

/* One scalar collision: raw moments P a, central moments F(u) ., relaxation
 * (w for the first-order moments, 1 for the rest), then F^-1(u) and P^-1. */
static void collide_scalar(const orc3_sim *s, const double F[Q3][Q3], const double Fi[Q3][Q3],
                           double w1, const double *eq, const double *in, double *out) {
    double raw[Q3], cm[Q3], cmt[Q3], rawt[Q3];
    matvec(s->Pm, in, raw);
    matvec(F, raw, cm);
    for (int k = 0; k < Q3; ++k) {
        double lam = is_first_order(k) ? w1 : 1.0;
        cmt[k] = cm[k] + lam * (eq[k] - cm[k]);
    }
    matvec(Fi, cmt, rawt);
    matvec(s->Pinv, rawt, out);
}

static void collide_all(orc3_sim *s) {
    const orc3_params *p = &s->p;
    size_t N = (size_t)s->N;
    const double w_kappa = rate_from_coeff(p->M_phi);
    const double w_chi = rate_from_coeff(p->D_s);
    const double w_zeta = rate_from_coeff(p->zeta);
#pragma omp parallel for schedule(static)
    for (size_t x = 0; x < N; ++x) {
        double F[Q3][Q3], Fi[Q3][Q3], in[Q3], out[Q3], eq[Q3], q[3];
        build_frame(s->ux[x], s->uy[x], s->uz[x], -1.0, F);
        build_frame(s->ux[x], s->uy[x], s->uz[x], +1.0, Fi);
        const double n[3] = {s->nv[0][x], s->nv[1][x], s->nv[2][x]};

        /* f: CACE, first-order equilibria M_phi theta n */
        for (int a = 0; a < Q3; ++a) in[a] = s->f[a * N + x];
        for (int ax = 0; ax < 3; ++ax) q[ax] = p->M_phi * s->theta[x] * n[ax];
        eq_scalar(s->phi[x], q, eq);
        collide_scalar(s, F, Fi, w_kappa, eq, in, out);
        for (int a = 0; a < Q3; ++a) s->ft[a * N + x] = out[a];

        /* h: interface-bound scalar, first-order equilibria D_s theta_c n */
        for (int a = 0; a < Q3; ++a) in[a] = s->h[a * N + x];
        for (int ax = 0; ax < 3; ++ax) q[ax] = p->D_s * s->thetac[x] * n[ax];
        eq_scalar(s->c[x], q, eq);
        collide_scalar(s, F, Fi, w_chi, eq, in, out);
        for (int a = 0; a < Q3; ++a) s->ht[a * N + x] = out[a];

        if (p->mode != 1) continue;
        /* g: flow, raw -> central -> combined moments, relax with sources */
        double raw[Q3], cm[Q3], src[Q3], hat[Q3], hateq[Q3], hatsrc[Q3], hatt[Q3], cmt[Q3], rawt[Q3];
        const double u[3] = {s->ux[x], s->uy[x], s->uz[x]};
        const double Ft[3] = {s->Ft[0][x], s->Ft[1][x], s->Ft[2][x]};
        const double Fp[3] = {s->Fp[0][x], s->Fp[1][x], s->Fp[2][x]};
        for (int a = 0; a < Q3; ++a) in[a] = s->g[a * N + x];
        matvec(s->Pm, in, raw);
        matvec(F, raw, cm);
        eq_flow(s->P[x], s->psi[x], s->rho[x], u, eq);
        source_flow(u, Ft, Fp, src);
        matvec(s->Bm, cm, hat);
        matvec(s->Bm, eq, hateq);
        matvec(s->Bm, src, hatsrc);
        const double w_nu = rate_from_coeff(s->nu[x]);
        for (int k = 0; k < Q3; ++k) {
            double lam = 1.0;
            if (k == 2) lam = w_zeta;                                      /* trace */
            if (k == 6 || k == 18 || k == 4 || k == 10 || k == 12) lam = w_nu; /* deviatoric, shear */
            hatt[k] = hat[k] + lam * (hateq[k] - hat[k]) + (1.0 - 0.5 * lam) * hatsrc[k];
        }
        matvec(s->Binv, hatt, cmt);
        matvec(Fi, cmt, rawt);
        matvec(s->Pinv, rawt, out);
        for (int a = 0; a < Q3; ++a) s->gt[a * N + x] = out[a];
    }
}

static int opposite(int a) {
    for (int b = 0; b < Q3; ++b)
        if (E3[b][0] == -E3[a][0] && E3[b][1] == -E3[a][1] && E3[b][2] == -E3[a][2]) return b;
    return a;
}

/* Pull streaming, a(x, t+1) = a~(x - e_a, t), periodic on every axis; with
 * walls, a population whose source lies beyond a wall is the reflected
 * post-collision population of the same node (half-way bounce-back), and g
 * adds 2 w_a rho (e_a . u_w). */
static void stream_all(orc3_sim *s) {
    const orc3_params *p = &s->p;
    size_t N = (size_t)s->N;
    const int coupled = p->mode == 1;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) {
                size_t x = idx(s, i, j, k);
                for (int a = 0; a < Q3; ++a) {
                    int sj = j - E3[a][1];
                    if (p->walls_y && (sj < 0 || sj >= p->ny)) {
                        size_t src = (size_t)opposite(a) * N + x;
                        double uw = sj < 0 ? -p->u_wall : p->u_wall;
                        s->f[a * N + x] = s->ft[src];
                        s->h[a * N + x] = s->ht[src];
                        if (coupled) s->g[a * N + x] = s->gt[src] + 2.0 * weight(a) * s->rho[x] * (E3[a][0] * uw);
                        continue;
                    }
                    size_t src = idx(s, i - E3[a][0], j - E3[a][1], k - E3[a][2]);
                    s->f[a * N + x] = s->ft[a * N + src];
                    s->h[a * N + x] = s->ht[a * N + src];
                    if (coupled) s->g[a * N + x] = s->gt[a * N + src];
                }
            }
}

void orc3_step(orc3_sim *s, int nsteps) {
    for (int t = 0; t < nsteps; ++t) {
        compute_moments(s);  /* phi, c */
        compute_geometry(s, 1); /* n, theta, theta_c; forces, u, P */
        collide_all(s);
        stream_all(s);
        s->step += 1;
    }
}

static int init_state(orc3_sim *s, const double *phi, const double *c, const double *ux,
                      const double *uy, const double *uz, const double *P);

int orc3_init(orc3_sim *s, const double *phi, const double *c, const double *ux,
              const double *uy, const double *uz) {
    return init_state(s, phi, c, ux, uy, uz, NULL);
}

int orc3_init_pressure(orc3_sim *s, const double *phi, const double *c, const double *ux,
                       const double *uy, const double *uz, const double *P) {
    return init_state(s, phi, c, ux, uy, uz, P);
}

static int init_state(orc3_sim *s, const double *phi, const double *c, const double *ux,
                      const double *uy, const double *uz, const double *P) {
    const orc3_params *p = &s->p;
    size_t N = (size_t)s->N;
    for (size_t x = 0; x < N; ++x) {
        s->phi[x] = phi[x];
        s->c[x] = c[x];
        s->ux[x] = ux[x];
        s->uy[x] = uy[x];
        s->uz[x] = uz[x];
    }
    compute_geometry(s, 0);
#pragma omp parallel for schedule(static)
    for (size_t x = 0; x < N; ++x) {
        double Fi[Q3][Q3], eq[Q3], raw[Q3], out[Q3], q[3];
        build_frame(s->ux[x], s->uy[x], s->uz[x], +1.0, Fi);
        for (int ax = 0; ax < 3; ++ax) q[ax] = p->M_phi * s->theta[x] * s->nv[ax][x];
        eq_scalar(s->phi[x], q, eq);
        matvec(Fi, eq, raw);
        matvec(s->Pinv, raw, out);
        for (int a = 0; a < Q3; ++a) s->f[a * N + x] = out[a];
        for (int ax = 0; ax < 3; ++ax) q[ax] = p->D_s * s->thetac[x] * s->nv[ax][x];
        eq_scalar(s->c[x], q, eq);
        matvec(Fi, eq, raw);
        matvec(s->Pinv, raw, out);
        for (int a = 0; a < Q3; ++a) s->h[a * N + x] = out[a];
        if (p->mode != 1) continue;
        /* g: the given pressure, else the fluid at rest P = cs2 (rho_a + rho_b) / 2;
         * psi = P - rho cs2 */
        const double rho = lin_interp(p, s->phi[x], p->rho_a, p->rho_b);
        const double P0 = P ? P[x] : CS2 * 0.5 * (p->rho_a + p->rho_b);
        const double u[3] = {s->ux[x], s->uy[x], s->uz[x]};
        eq_flow(P0, P0 - rho * CS2, rho, u, eq);
        matvec(Fi, eq, raw);
        matvec(s->Pinv, raw, out);
        for (int a = 0; a < Q3; ++a) s->g[a * N + x] = out[a];
    }
    s->step = 0;
    return 0;
}

void orc3_fields(orc3_sim *s, double *phi, double *c) {
    compute_moments(s);
    size_t bytes = sizeof(double) * (size_t)s->N;
    if (phi) memcpy(phi, s->phi, bytes);
    if (c) memcpy(c, s->c, bytes);
}

void orc3_normals(orc3_sim *s, double *nx_, double *ny_, double *nz_) {
    compute_moments(s);
    compute_geometry(s, 1);
    size_t bytes = sizeof(double) * (size_t)s->N;
    if (nx_) memcpy(nx_, s->nv[0], bytes);
    if (ny_) memcpy(ny_, s->nv[1], bytes);
    if (nz_) memcpy(nz_, s->nv[2], bytes);
}

void orc3_get_pops(const orc3_sim *s, double *f, double *h) {
    size_t bytes = sizeof(double) * Q3 * (size_t)s->N;
    if (f) memcpy(f, s->f, bytes);
    if (h) memcpy(h, s->h, bytes);
}

void orc3_set_pops(orc3_sim *s, const double *f, const double *h) {
    size_t bytes = sizeof(double) * Q3 * (size_t)s->N;
    if (f) memcpy(s->f, f, bytes);
    if (h) memcpy(s->h, h, bytes);
}

void orc3_flow_fields(orc3_sim *s, double *ux, double *uy, double *uz, double *P) {
    compute_moments(s);
    compute_geometry(s, 1);
    size_t bytes = sizeof(double) * (size_t)s->N;
    if (ux) memcpy(ux, s->ux, bytes);
    if (uy) memcpy(uy, s->uy, bytes);
    if (uz) memcpy(uz, s->uz, bytes);
    if (P) memcpy(P, s->P, bytes);
}

void orc3_get_flow_pops(const orc3_sim *s, double *g) {
    if (g) memcpy(g, s->g, sizeof(double) * Q3 * (size_t)s->N);
}

void orc3_curvature(orc3_sim *s, double *kappa) {
    const orc3_params *p = &s->p;
    compute_moments(s);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) kappa[idx(s, i, j, k)] = div_normal_at(s, i, j, k);
}
