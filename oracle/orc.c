/*
 * FP64 CPU oracle of the MRT lattice Boltzmann model of Liu, He, Li and Tao
 * (arXiv:1308.2071).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke
 * check and the benchmark's CPU baseline, never by the CUDA library.
 *
 * Plain per-node loops; every formula carries the equation it restates.
 * Full populations (no shifted storage), collision then a separate pull
 * streaming pass then the wall rule, exactly as Section 3 describes.
 * Build with -O2 -ffp-contract=off so that no fused multiply-add changes the
 * rounding of the written expressions.
 */
#include "orc.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---- lattices ---------------------------------------------------------- */

/* D2Q9 velocities of Eq. 8 with c = 1: rest, E, N, W, S, NE, NW, SW, SE. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* D2Q9 weights, stated after Eq. 13. */
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* c_s^2 = c^2 / 3, stated after Eq. 13. */
static const double CS2 = 1.0 / 3.0;

/* Transformation matrix of Eq. 11, row k = moment k of Eq. 10. */
static const double MMAT[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
};

/* D2Q5 velocities of Eq. 26: rest, E, N, W, S. */
static const int EX5[5] = {0, 1, 0, -1, 0};
static const int EY5[5] = {0, 0, 1, 0, -1};

/* Transformation matrix of Eq. 28. */
static const double NMAT[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {-4, 1, 1, 1, 1},
    {0, 1, -1, 1, -1},
};

void orc_velocities(int ex9[9], int ey9[9], int ex5[5], int ey5[5]) {
    for (int i = 0; i < 9; ++i) {
        ex9[i] = EX[i];
        ey9[i] = EY[i];
    }
    for (int i = 0; i < 5; ++i) {
        ex5[i] = EX5[i];
        ey5[i] = EY5[i];
    }
}

/* The rows of M (and of N) are mutually orthogonal (the paper calls the
 * matrices orthogonal, Section 3.1 and 3.2), so the inverse is the transpose
 * with each column divided by the squared norm of the matching row. */
void orc_matrix_M(double M[81]) {
    for (int k = 0; k < 9; ++k)
        for (int i = 0; i < 9; ++i) M[k * 9 + i] = MMAT[k][i];
}

void orc_matrix_Minv(double Minv[81]) {
    for (int k = 0; k < 9; ++k) {
        double norm2 = 0.0;
        for (int i = 0; i < 9; ++i) norm2 += MMAT[k][i] * MMAT[k][i];
        for (int i = 0; i < 9; ++i) Minv[i * 9 + k] = MMAT[k][i] / norm2;
    }
}

void orc_matrix_N(double N[25]) {
    for (int k = 0; k < 5; ++k)
        for (int i = 0; i < 5; ++i) N[k * 5 + i] = NMAT[k][i];
}

void orc_matrix_Ninv(double Ninv[25]) {
    for (int k = 0; k < 5; ++k) {
        double norm2 = 0.0;
        for (int i = 0; i < 5; ++i) norm2 += NMAT[k][i] * NMAT[k][i];
        for (int i = 0; i < 5; ++i) Ninv[i * 5 + k] = NMAT[k][i] / norm2;
    }
}

/* ---- single-node formulas ---------------------------------------------- */

/* Eq. 14. */
static double s_fun(int i, const double u[2], double phi) {
    double eu = EX[i] * u[0] + EY[i] * u[1];
    double uu = u[0] * u[0] + u[1] * u[1];
    return W9[i] * (eu / CS2 + (eu * eu) / (2.0 * phi * CS2 * CS2) - uu / (2.0 * phi * CS2));
}

/* Eq. 13, with P = phi * p. */
void orc_feq(double rho0, double P, const double u[2], double phi, double feq[9]) {
    feq[0] = rho0 - (1.0 - W9[0]) * P / CS2 + rho0 * s_fun(0, u, phi);
    for (int i = 1; i < 9; ++i) feq[i] = W9[i] * P / CS2 + rho0 * s_fun(i, u, phi);
}

/* Eq. 15-16, with P = phi * p. */
void orc_meq(double rho0, double P, const double u[2], double phi, double meq[9]) {
    double uu = u[0] * u[0] + u[1] * u[1];
    meq[0] = rho0;
    meq[1] = -4.0 * rho0 + 6.0 * P + 3.0 * rho0 * uu / phi;
    meq[2] = 4.0 * rho0 - 9.0 * P - 3.0 * rho0 * uu / phi;
    meq[3] = rho0 * u[0];
    meq[4] = -rho0 * u[0];
    meq[5] = rho0 * u[1];
    meq[6] = -rho0 * u[1];
    meq[7] = rho0 * (u[0] * u[0] - u[1] * u[1]) / phi;
    meq[8] = rho0 * u[0] * u[1] / phi;
}

/* Eq. 19. */
void orc_force_moments(double rho0, const double u[2], const double F[2], double phi, double S[9]) {
    double uF = u[0] * F[0] + u[1] * F[1];
    S[0] = 0.0;
    S[1] = 6.0 * rho0 * uF / phi;
    S[2] = -6.0 * rho0 * uF / phi;
    S[3] = rho0 * F[0];
    S[4] = -rho0 * F[0];
    S[5] = rho0 * F[1];
    S[6] = -rho0 * F[1];
    S[7] = 2.0 * rho0 * (u[0] * F[0] - u[1] * F[1]) / phi;
    S[8] = rho0 * (u[0] * F[1] + u[1] * F[0]) / phi;
}

/* Weights and sound speed of the D2Q5 model, stated after Eq. 37 (first). */
static double w5(int i, double varpi) { return i == 0 ? (1.0 - varpi) / 5.0 : (4.0 + varpi) / 20.0; }
static double csT2(double varpi) { return (4.0 + varpi) / 10.0; }

/* Eq. 37 (first occurrence). */
void orc_geq(double T, const double u[2], double sigma, double varpi, double geq[5]) {
    for (int i = 0; i < 5; ++i) {
        double eu = EX5[i] * u[0] + EY5[i] * u[1];
        geq[i] = w5(i, varpi) * T * (1.0 + eu / (sigma * csT2(varpi)));
    }
}

/* Eq. 29. */
void orc_neq(double T, const double u[2], double sigma, double varpi, double neq[5]) {
    neq[0] = T;
    neq[1] = u[0] * T / sigma;
    neq[2] = u[1] * T / sigma;
    neq[3] = varpi * T;
    neq[4] = 0.0;
}

/* Eq. 21-22 with delta_t = 1; l0 and l1 as defined after Eq. 22. */
void orc_velocity(double rho0, const double f[9], double phi, double nu, double K, double Fphi,
                  const double G[2], double u[2]) {
    double v[2] = {0.0, 0.0};
    for (int i = 0; i < 9; ++i) {
        v[0] += EX[i] * f[i];
        v[1] += EY[i] * f[i];
    }
    v[0] = v[0] / rho0 + 0.5 * phi * G[0];
    v[1] = v[1] / rho0 + 0.5 * phi * G[1];
    double l0 = 0.5 * (1.0 + phi * 0.5 * nu / K);
    double l1 = phi * 0.5 * Fphi / sqrt(K);
    double vmag = sqrt(v[0] * v[0] + v[1] * v[1]);
    double den = l0 + sqrt(l0 * l0 + l1 * vmag);
    u[0] = v[0] / den;
    u[1] = v[1] / den;
}

/* Eq. 23. */
double orc_pressure(double rho0, const double f[9], const double u[2], double phi) {
    double sum = 0.0;
    for (int i = 1; i < 9; ++i) sum += f[i];
    return CS2 / (phi * (1.0 - W9[0])) * (sum + rho0 * s_fun(0, u, phi));
}

/* Eq. 5 with d_p^2 given. */
void orc_ergun(double phi, double dp2, double* K, double* Fphi) {
    *Fphi = 1.75 / sqrt(150.0 * phi * phi * phi);
    *K = phi * phi * phi * dp2 / (150.0 * (1.0 - phi) * (1.0 - phi));
}

/* Eq. 4. */
static void total_force(const double u[2], double phi, double nu, double K, double Fphi,
                        const double G[2], double F[2]) {
    double umag = sqrt(u[0] * u[0] + u[1] * u[1]);
    for (int a = 0; a < 2; ++a)
        F[a] = -phi * nu / K * u[a] - phi * Fphi / sqrt(K) * umag * u[a] + phi * G[a];
}

/* Eq. 17 then f+ = M^-1 m+ (Eq. 18), and Eq. 34 then g+ = N^-1 n+ (Eq. 35). */
static double MINV[81], NINV[25];
static pthread_once_t inv_once = PTHREAD_ONCE_INIT;
static void make_inverses(void) {
    orc_matrix_Minv(MINV);
    orc_matrix_Ninv(NINV);
}

void orc_collide(const orc_lattice* lat, double phi, const double f[9], const double g[5],
                 const double u[2], double P, double T, const double F[2], double fplus[9],
                 double gplus[5]) {
    pthread_once(&inv_once, make_inverses);
    const double* Minv = MINV;
    const double* Ninv = NINV;

    double m[9], meq[9], S[9], mplus[9];
    for (int k = 0; k < 9; ++k) {
        m[k] = 0.0;
        for (int i = 0; i < 9; ++i) m[k] += MMAT[k][i] * f[i];
    }
    orc_meq(lat->rho0, P, u, phi, meq);
    orc_force_moments(lat->rho0, u, F, phi, S);
    for (int k = 0; k < 9; ++k)
        mplus[k] = m[k] - lat->s[k] * (m[k] - meq[k]) + (1.0 - lat->s[k] / 2.0) * S[k];
    for (int i = 0; i < 9; ++i) {
        fplus[i] = 0.0;
        for (int k = 0; k < 9; ++k) fplus[i] += Minv[i * 9 + k] * mplus[k];
    }

    double n[5], neq[5], psi[5], nplus[5];
    for (int k = 0; k < 5; ++k) {
        n[k] = 0.0;
        for (int i = 0; i < 5; ++i) n[k] += NMAT[k][i] * g[i];
    }
    orc_neq(T, u, lat->sigma, lat->varpi, neq);
    /* Eq. 30 */
    psi[0] = lat->Q / lat->sigma;
    psi[1] = 0.0;
    psi[2] = 0.0;
    psi[3] = lat->varpi * lat->Q / lat->sigma;
    psi[4] = 0.0;
    for (int k = 0; k < 5; ++k)
        nplus[k] = n[k] - lat->zeta[k] * (n[k] - neq[k]) + (1.0 - lat->zeta[k] / 2.0) * psi[k];
    for (int i = 0; i < 5; ++i) {
        gplus[i] = 0.0;
        for (int k = 0; k < 5; ++k) gplus[i] += Ninv[i * 5 + k] * nplus[k];
    }
}

/* ---- parameters ---------------------------------------------------------- */

void orc_derive(const orc_physical* ph, orc_lattice* lat) {
    memset(lat, 0, sizeof(*lat));
    lat->nx = ph->nx;
    lat->ny = ph->ny;
    lat->rho0 = 1.0;
    double L = (double)(ph->nx - 1); /* walls on the perimeter nodes */
    double cs = sqrt(CS2);
    double cT2 = (4.0 + ph->varpi) / 10.0;
    int cooled = ph->thermal_bc == 1;
    /* Eq. 37 (second occurrence); Section 4.2 writes it with Ra_I */
    double Rs = cooled ? ph->RaI : ph->Ra;
    double tau_nu = 0.5 + ph->Ma * ph->J * L / cs * sqrt(ph->Pr / Rs);
    double tau_T = 0.5 + CS2 * (tau_nu - 0.5) / (ph->sigma * cT2 * ph->Pr);
    /* Section 4 rate choices */
    double s[9] = {1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2, 1.0 / tau_nu, 1.0 / tau_nu};
    double z[5] = {1.0, 1.0 / tau_T, 1.0 / tau_T, 1.5, 1.5};
    memcpy(lat->s, s, sizeof(s));
    memcpy(lat->zeta, z, sizeof(z));
    /* Eq. 24, and nu = nu_e / J from the definition of J */
    lat->nu = CS2 * (tau_nu - 0.5) / ph->J;
    lat->phi_bar = ph->phi;
    lat->K_bar = ph->Da * L * L; /* Da = K / L^2 */
    lat->forchheimer = 1;
    /* U = sqrt(g beta dT L) = Ma c_s */
    double U = ph->Ma * cs;
    double dT = ph->Th - ph->Tc;
    lat->gbeta = U * U / (dT * L);
    lat->sigma = ph->sigma;
    lat->varpi = ph->varpi;
    lat->Th = ph->Th;
    lat->Tc = ph->Tc;
    lat->T0 = cooled ? ph->Tc : 0.5 * (ph->Th + ph->Tc);
    lat->L = L;
    lat->dT = dT;
    lat->adiabatic_order = 1;
    lat->thermal_bc = ph->thermal_bc;
    /* A9: alpha_e = sigma (4 + varpi)/10 (tau_T - 1/2) */
    double alpha = ph->sigma * cT2 * (tau_T - 0.5);
    if (cooled) lat->Q = dT * alpha / (L * L);
    else if (ph->RaI > 0.0) lat->Q = ph->RaI / ph->Ra * alpha * dT / (L * L);
}

/* ---- state ----------------------------------------------------------------- */

struct orc_state {
    orc_lattice lat;
    int nx, ny;
    long t;
    double *f, *g;       /* post-stream, post-wall-rule populations */
    double *fp, *gp;     /* post-collision populations */
    double *phi, *K, *Fphi;
    double *Pb, *Tb;     /* imposed P = phi p and T on wall nodes */
    unsigned char* wall; /* 1 on wall nodes */
    signed char *nxd, *nyd; /* inward normal of wall nodes */
};

#define IDX(st, x, y) ((size_t)(y) * (size_t)(st)->nx + (size_t)(x))

static size_t plane(const orc_state* st) { return (size_t)st->nx * (size_t)st->ny; }

static void load_node(const orc_state* st, const double* f, const double* g, size_t k,
                      double fn[9], double gn[5]) {
    size_t n = plane(st);
    for (int i = 0; i < 9; ++i) fn[i] = f[i * n + k];
    for (int i = 0; i < 5; ++i) gn[i] = g[i * n + k];
}

/* Macroscopic values of a non-wall node from its populations (Section 3 order). */
static void node_macros(const orc_state* st, const double fn[9], const double gn[5], size_t k,
                        double u[2], double* P, double* T, double F[2]) {
    const orc_lattice* lat = &st->lat;
    double phi = st->phi[k];
    double sumg = 0.0;
    for (int i = 0; i < 5; ++i) sumg += gn[i];
    *T = sumg + 0.5 * lat->Q / lat->sigma; /* Eq. 36 */
    double G[2] = {lat->Gx, lat->Gy + lat->gbeta * (*T - lat->T0)};
    orc_velocity(lat->rho0, fn, phi, lat->nu, st->K[k], st->Fphi[k], G, u);
    *P = phi * orc_pressure(lat->rho0, fn, u, phi);
    total_force(u, phi, lat->nu, st->K[k], st->Fphi[k], G, F);
}

/* Imposed wall values (u = 0, P_b, T_b) and the force there (Eq. 4 at u = 0). */
static void wall_macros(const orc_state* st, size_t k, double u[2], double* P, double* T,
                        double F[2]) {
    const orc_lattice* lat = &st->lat;
    u[0] = 0.0;
    u[1] = 0.0;
    *P = st->Pb[k];
    *T = st->Tb[k];
    double G[2] = {lat->Gx, lat->Gy + lat->gbeta * (*T - lat->T0)};
    F[0] = st->phi[k] * G[0];
    F[1] = st->phi[k] * G[1];
}

/* Non-equilibrium extrapolation on every wall node (Section 4, ref. [43]).
 * With write_pops = 0 only the imposed values are recomputed. */
static void wall_rule(orc_state* st, int write_pops) {
    const orc_lattice* lat = &st->lat;
    size_t n = plane(st);
    for (int y = 0; y < st->ny; ++y) {
        for (int x = 0; x < st->nx; ++x) {
            size_t kb = IDX(st, x, y);
            if (!st->wall[kb]) continue;
            int dx = st->nxd[kb], dy = st->nyd[kb];
            size_t kf = IDX(st, x + dx, y + dy);
            double ff[9], gf[5], uf[2], Pf, Tf, Ff[2];
            load_node(st, st->f, st->g, kf, ff, gf);
            node_macros(st, ff, gf, kf, uf, &Pf, &Tf, Ff);
            double pf = Pf / st->phi[kf];
            double feqf[9], geqf[5];
            orc_feq(lat->rho0, Pf, uf, st->phi[kf], feqf);
            orc_geq(Tf, uf, lat->sigma, lat->varpi, geqf);

            double Tb;
            int dirichlet = (lat->thermal_bc == 1) || (dx != 0);
            if (dirichlet) {
                if (lat->thermal_bc == 1) Tb = lat->Tc;
                else Tb = (x == 0) ? lat->Th : lat->Tc;
            } else if (lat->adiabatic_order == 2) {
                size_t kff = IDX(st, x + 2 * dx, y + 2 * dy);
                double fff[9], gff[5], uff[2], Pff, Tff, Fff[2];
                load_node(st, st->f, st->g, kff, fff, gff);
                node_macros(st, fff, gff, kff, uff, &Pff, &Tff, Fff);
                Tb = (4.0 * Tf - Tff) / 3.0;
            } else {
                Tb = Tf;
            }
            double Pb = st->phi[kb] * pf; /* p_b = p_f */
            st->Pb[kb] = Pb;
            st->Tb[kb] = Tb;
            if (!write_pops) continue;
            double zero[2] = {0.0, 0.0};
            double feqb[9], geqb[5];
            orc_feq(lat->rho0, Pb, zero, st->phi[kb], feqb);
            orc_geq(Tb, zero, lat->sigma, lat->varpi, geqb);
            for (int i = 0; i < 9; ++i) st->f[i * n + kb] = feqb[i] + (ff[i] - feqf[i]);
            for (int i = 0; i < 5; ++i) st->g[i * n + kb] = geqb[i] + (gf[i] - geqf[i]);
        }
    }
}

orc_state* orc_create(const orc_lattice* lat, const double* phi_field) {
    if (lat->nx < 5 || lat->ny < 5) return NULL;
    orc_state* st = (orc_state*)calloc(1, sizeof(orc_state));
    st->lat = *lat;
    st->nx = lat->nx;
    st->ny = lat->ny;
    size_t n = plane(st);
    st->f = (double*)malloc(9 * n * sizeof(double));
    st->g = (double*)malloc(5 * n * sizeof(double));
    st->fp = (double*)malloc(9 * n * sizeof(double));
    st->gp = (double*)malloc(5 * n * sizeof(double));
    st->phi = (double*)malloc(n * sizeof(double));
    st->K = (double*)malloc(n * sizeof(double));
    st->Fphi = (double*)malloc(n * sizeof(double));
    st->Pb = (double*)calloc(n, sizeof(double));
    st->Tb = (double*)calloc(n, sizeof(double));
    st->wall = (unsigned char*)calloc(n, 1);
    st->nxd = (signed char*)calloc(n, 1);
    st->nyd = (signed char*)calloc(n, 1);

    /* Ergun anchor: d_p^2 chosen so that K(phi_bar) = K_bar (Eq. 5). */
    double pb = lat->phi_bar;
    double dp2 = (pb < 1.0) ? 150.0 * lat->K_bar * (1.0 - pb) * (1.0 - pb) / (pb * pb * pb) : 0.0;
    for (size_t k = 0; k < n; ++k) {
        if (phi_field) {
            st->phi[k] = phi_field[k];
            orc_ergun(phi_field[k], dp2, &st->K[k], &st->Fphi[k]);
        } else {
            st->phi[k] = pb;
            st->K[k] = lat->K_bar;
            st->Fphi[k] = 1.75 / sqrt(150.0 * pb * pb * pb); /* Eq. 5 */
        }
        if (!lat->forchheimer) st->Fphi[k] = 0.0;
    }
    for (int y = 0; y < st->ny; ++y)
        for (int x = 0; x < st->nx; ++x) {
            size_t k = IDX(st, x, y);
            int dx = 0, dy = 0;
            if (!lat->periodic_x) dx = (x == 0) ? 1 : (x == st->nx - 1) ? -1 : 0;
            if (!lat->periodic_y) dy = (y == 0) ? 1 : (y == st->ny - 1) ? -1 : 0;
            st->wall[k] = (dx != 0 || dy != 0);
            st->nxd[k] = (signed char)dx;
            st->nyd[k] = (signed char)dy;
        }
    /* Initial state: rest populations at p = rho0 c_s^2 / phi, T = T0. */
    for (size_t k = 0; k < n; ++k) {
        for (int i = 0; i < 9; ++i) st->f[i * n + k] = W9[i] * lat->rho0;
        for (int i = 0; i < 5; ++i) st->g[i * n + k] = w5(i, lat->varpi) * lat->T0;
    }
    wall_rule(st, 1);
    st->t = 0;
    return st;
}

void orc_destroy(orc_state* st) {
    if (!st) return;
    free(st->f);
    free(st->g);
    free(st->fp);
    free(st->gp);
    free(st->phi);
    free(st->K);
    free(st->Fphi);
    free(st->Pb);
    free(st->Tb);
    free(st->wall);
    free(st->nxd);
    free(st->nyd);
    free(st);
}

long orc_time(const orc_state* st) { return st->t; }

/* Collision of rows [y0, y1). */
static void collide_rows(orc_state* st, int y0, int y1) {
    size_t n = plane(st);
    for (int y = y0; y < y1; ++y)
        for (int x = 0; x < st->nx; ++x) {
            size_t k = IDX(st, x, y);
            double fn[9], gn[5], u[2], P, T, F[2], fplus[9], gplus[5];
            load_node(st, st->f, st->g, k, fn, gn);
            if (st->wall[k]) wall_macros(st, k, u, &P, &T, F);
            else node_macros(st, fn, gn, k, u, &P, &T, F);
            orc_collide(&st->lat, st->phi[k], fn, gn, u, P, T, F, fplus, gplus);
            for (int i = 0; i < 9; ++i) st->fp[i * n + k] = fplus[i];
            for (int i = 0; i < 5; ++i) st->gp[i * n + k] = gplus[i];
        }
}

/* Pull streaming of rows [y0, y1) (Eq. 18 and Eq. 35).  A population whose
 * source lies outside a non-periodic edge only occurs on wall nodes, which
 * the wall rule overwrites; it is set to NaN so that any use shows. */
static void stream_rows(orc_state* st, int y0, int y1) {
    size_t n = plane(st);
    for (int y = y0; y < y1; ++y)
        for (int x = 0; x < st->nx; ++x) {
            size_t k = IDX(st, x, y);
            for (int i = 0; i < 9; ++i) {
                int xs = x - EX[i], ys = y - EY[i];
                if (st->lat.periodic_x) xs = (xs + st->nx) % st->nx;
                if (st->lat.periodic_y) ys = (ys + st->ny) % st->ny;
                if (xs < 0 || xs >= st->nx || ys < 0 || ys >= st->ny) st->f[i * n + k] = NAN;
                else st->f[i * n + k] = st->fp[i * n + IDX(st, xs, ys)];
            }
            for (int i = 0; i < 5; ++i) {
                int xs = x - EX5[i], ys = y - EY5[i];
                if (st->lat.periodic_x) xs = (xs + st->nx) % st->nx;
                if (st->lat.periodic_y) ys = (ys + st->ny) % st->ny;
                if (xs < 0 || xs >= st->nx || ys < 0 || ys >= st->ny) st->g[i * n + k] = NAN;
                else st->g[i * n + k] = st->gp[i * n + IDX(st, xs, ys)];
            }
        }
}

typedef struct {
    orc_state* st;
    long nsteps;
    int tid, nthreads;
    pthread_barrier_t* bar;
} worker_arg;

static void* worker(void* p) {
    worker_arg* a = (worker_arg*)p;
    orc_state* st = a->st;
    int y0 = (int)((long)st->ny * a->tid / a->nthreads);
    int y1 = (int)((long)st->ny * (a->tid + 1) / a->nthreads);
    for (long s = 0; s < a->nsteps; ++s) {
        collide_rows(st, y0, y1);
        pthread_barrier_wait(a->bar);
        stream_rows(st, y0, y1);
        pthread_barrier_wait(a->bar);
        if (a->tid == 0) wall_rule(st, 1);
        pthread_barrier_wait(a->bar);
    }
    return NULL;
}

void orc_step(orc_state* st, long nsteps, int nthreads) {
    if (nsteps <= 0) return;
    if (nthreads > st->ny) nthreads = st->ny;
    if (nthreads <= 1) {
        for (long s = 0; s < nsteps; ++s) {
            collide_rows(st, 0, st->ny);
            stream_rows(st, 0, st->ny);
            wall_rule(st, 1);
        }
    } else {
        pthread_barrier_t bar;
        pthread_barrier_init(&bar, NULL, (unsigned)nthreads);
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
        worker_arg* args = (worker_arg*)malloc(sizeof(worker_arg) * (size_t)nthreads);
        for (int t = 0; t < nthreads; ++t) {
            args[t].st = st;
            args[t].nsteps = nsteps;
            args[t].tid = t;
            args[t].nthreads = nthreads;
            args[t].bar = &bar;
            pthread_create(&th[t], NULL, worker, &args[t]);
        }
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
        pthread_barrier_destroy(&bar);
        free(th);
        free(args);
    }
    st->t += nsteps;
}

void orc_get_state(const orc_state* st, double* f, double* g) {
    size_t n = plane(st);
    memcpy(f, st->f, 9 * n * sizeof(double));
    memcpy(g, st->g, 5 * n * sizeof(double));
}

void orc_set_state(orc_state* st, const double* f, const double* g) {
    size_t n = plane(st);
    memcpy(st->f, f, 9 * n * sizeof(double));
    memcpy(st->g, g, 5 * n * sizeof(double));
    wall_rule(st, 0);
}

void orc_macros(const orc_state* st, double* ux, double* uy, double* p, double* T) {
    for (int y = 0; y < st->ny; ++y)
        for (int x = 0; x < st->nx; ++x) {
            size_t k = IDX(st, x, y);
            double fn[9], gn[5], u[2], P, Tk, F[2];
            load_node(st, st->f, st->g, k, fn, gn);
            if (st->wall[k]) wall_macros(st, k, u, &P, &Tk, F);
            else node_macros(st, fn, gn, k, u, &P, &Tk, F);
            if (ux) ux[k] = u[0];
            if (uy) uy[k] = u[1];
            if (p) p[k] = P / st->phi[k];
            if (T) T[k] = Tk;
        }
}

/* Eq. 38: Nu(y) = -L dT/dx / dT at the wall, with a one-sided fourth-order
 * five-point derivative, averaged over y by the trapezoidal rule. */
void orc_nusselt(const orc_state* st, double* nu_left, double* nu_right) {
    size_t n = plane(st);
    double* T = (double*)malloc(n * sizeof(double));
    orc_macros(st, NULL, NULL, NULL, T);
    const orc_lattice* lat = &st->lat;
    int nx = st->nx, ny = st->ny;
    double sl = 0.0, sr = 0.0;
    for (int y = 0; y < ny; ++y) {
        const double* r = T + (size_t)y * (size_t)nx;
        double dl = (-25.0 * r[0] + 48.0 * r[1] - 36.0 * r[2] + 16.0 * r[3] - 3.0 * r[4]) / 12.0;
        double dr = (25.0 * r[nx - 1] - 48.0 * r[nx - 2] + 36.0 * r[nx - 3] - 16.0 * r[nx - 4] +
                     3.0 * r[nx - 5]) / 12.0;
        double nl = -lat->L * dl / lat->dT;
        double nr = -lat->L * dr / lat->dT;
        double wgt = (y == 0 || y == ny - 1) ? 0.5 : 1.0;
        sl += wgt * nl;
        sr += wgt * nr;
    }
    *nu_left = sl / (double)(ny - 1);
    *nu_right = sr / (double)(ny - 1);
    free(T);
}
