/*
 * FP64 CPU oracle of the REV-scale MRT lattice Boltzmann model for convection
 * heat transfer in porous media (Liu, He, Li, Tao, arXiv:1308.2071).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library and never calls it.
 *
 * What it computes, per time step, in the paper's order (Section 3):
 *   1. macroscopic fields at every node: T (Eq. 36), G (Section 2, after
 *      Eq. 4), temporal velocity v (Eq. 22), u (Eq. 21), p (Eq. 23), F (Eq. 4);
 *   2. flow collision in moment space: m = M f (Eq. 9-11), m_eq (Eq. 15-16),
 *      S (Eq. 19), m+ (Eq. 17), f+ = M^-1 m+ (Eq. 18);
 *   3. thermal collision: n = N g (Eq. 27-28), n_eq (Eq. 29), Psi (Eq. 30),
 *      n+ (Eq. 34), g+ = N^-1 n+ (Eq. 35);
 *   4. streaming of f+ and g+ (Eq. 18, 35), pull form, in a separate pass;
 *   5. the non-equilibrium extrapolation wall rule (Section 4, ref. [43]).
 * Wall nodes collide with their imposed macroscopic values (u = 0, the
 * extrapolated pressure and the wall temperature).
 *
 * Readings where the paper is silent (all stated in the design notes):
 *   - walls lie on the perimeter nodes, so L = nx - 1;
 *   - non-equilibrium extrapolation: inner neighbour x_f = x_b + n (corners use
 *     the diagonal neighbour), p_b = p_f, u_b = 0, T_b = wall value on
 *     isothermal walls, T_b = T_f on adiabatic walls (optional second-order
 *     variant (4 T_f - T_ff) / 3); corners belong to the isothermal walls;
 *   - initial state f_i = w_i rho0, g_i = w~_i T0, then the wall rule once;
 *   - Nu uses a one-sided fourth-order five-point derivative and the
 *     trapezoidal mean over the wall nodes.
 *
 * Storage: full populations (not deviations), f[i][y][x], g[j][y][x],
 * row-major with x fastest.  All arithmetic is IEEE FP64, compiled with
 * -ffp-contract=off.
 */
#ifndef ORC_H
#define ORC_H

#ifdef __cplusplus
extern "C" {
#endif

/* Physical inputs of a cavity run (Section 2 and Section 4). */
typedef struct {
    int nx, ny;            /* nodes including the wall nodes                      */
    double Ra, Da, Pr, J;  /* Rayleigh, Darcy, Prandtl, viscosity ratio (P. 61)   */
    double phi;            /* mean porosity                                       */
    double Ma;             /* Mach number U / c_s (Section 4)                     */
    double sigma, varpi;   /* thermal capacity ratio, D2Q5 constant (Eq. 29)      */
    double Th, Tc;         /* wall temperatures (Section 4.2: Th - Tc is the scale dT) */
    double RaI;            /* internal Rayleigh number, 0 = no heat source        */
    int thermal_bc;        /* 0: side-heated cavity (Section 4.1, 4.3); 1: every wall at Tc (4.2) */
} orc_physical;

/* Lattice-level parameters of one run.  Produced by orc_derive() from the
 * physical inputs, or filled directly by a test. */
typedef struct {
    int nx, ny;
    double rho0;           /* mean density (1 in the paper)                       */
    double T0;             /* reference temperature of the buoyancy term          */
    double s[9];           /* flow relaxation rates, Eq. 20                        */
    double zeta[5];        /* thermal relaxation rates, Eq. 31                     */
    double nu;             /* fluid viscosity in the Darcy term, nu = nu_e / J     */
    double phi_bar;        /* uniform porosity (or the anchor of a porosity field) */
    double K_bar;          /* permeability at phi_bar                              */
    int forchheimer;       /* 1: F_phi from Ergun (Eq. 5); 0: F_phi = 0            */
    double gbeta;          /* g * beta of the Boussinesq force                     */
    double Gx, Gy;         /* constant body force added to G (test hook)           */
    double sigma, varpi;
    double Q;              /* internal heat source Q''' (lattice units)            */
    double Th, Tc;
    double L, dT;          /* length and temperature scale of the Nusselt number   */
    int periodic_x, periodic_y;
    int thermal_bc;        /* 0: x-walls Th (left) / Tc (right), y-walls adiabatic
                              1: every wall at Tc                                   */
    int adiabatic_order;   /* 1: T_b = T_f; 2: T_b = (4 T_f - T_ff) / 3            */
} orc_lattice;

typedef struct orc_state orc_state;

/* Eq. 37 (second occurrence, Section 4) and the constants of Section 4:
 * rho0 = 1, delta_t = 1, s = (1, 1.1, 1.1, 1, 1.2, 1, 1.2, 1/tau_nu, 1/tau_nu),
 * zeta = (1, 1/tau_T, 1/tau_T, 1.5, 1.5), K = Da L^2, gbeta from U = Ma c_s.
 * Internal heating: with thermal_bc = 1 (Section 4.2) tau_nu uses Ra_I in
 * place of Ra, T0 = Tc and dT = Q''' L^2 / alpha_e; with thermal_bc = 0 and
 * RaI > 0 (Section 4.3) Q''' follows from Ra_I / Ra = Q''' L^2 / (alpha_e dT)
 * (definitions of Section 2), alpha_e from A9. */
void orc_derive(const orc_physical* ph, orc_lattice* lat);

/* Creates a run.  phi_field (ny*nx, optional) gives a per-cell porosity; K and
 * F_phi then follow Ergun's relation (Eq. 5) with d_p fixed so that
 * K(phi_bar) = K_bar.  Returns NULL on invalid input. */
orc_state* orc_create(const orc_lattice* lat, const double* phi_field);
void orc_destroy(orc_state* st);

/* Advances nsteps time steps using nthreads row-parallel threads. */
void orc_step(orc_state* st, long nsteps, int nthreads);
long orc_time(const orc_state* st);

/* Post-stream, post-wall-rule populations at the current time (the state
 * that the next collision reads). */
void orc_get_state(const orc_state* st, double* f, double* g);
/* Replaces that state; the imposed wall values are recomputed from the inner
 * neighbours of the given populations. */
void orc_set_state(orc_state* st, const double* f, const double* g);

/* Macroscopic fields of the current state (walls report their imposed values). */
void orc_macros(const orc_state* st, double* ux, double* uy, double* p, double* T);
/* Mean Nusselt numbers of the left and right walls (Eq. 38). */
void orc_nusselt(const orc_state* st, double* nu_left, double* nu_right);

/* ---- single-node building blocks, exposed for the unit tests ---------- */
/* Velocity sets of Eq. 8 (D2Q9) and Eq. 26 (D2Q5). */
void orc_velocities(int ex9[9], int ey9[9], int ex5[5], int ey5[5]);
void orc_matrix_M(double M[81]);
void orc_matrix_Minv(double Minv[81]);
void orc_matrix_N(double N[25]);
void orc_matrix_Ninv(double Ninv[25]);
/* Eq. 13-14: incompressible porous equilibrium, P = phi * p. */
void orc_feq(double rho0, double P, const double u[2], double phi, double feq[9]);
/* Eq. 16. */
void orc_meq(double rho0, double P, const double u[2], double phi, double meq[9]);
/* Eq. 19. */
void orc_force_moments(double rho0, const double u[2], const double F[2], double phi, double S[9]);
/* Eq. 37 (first occurrence): D2Q5 equilibrium. */
void orc_geq(double T, const double u[2], double sigma, double varpi, double geq[5]);
/* Eq. 29. */
void orc_neq(double T, const double u[2], double sigma, double varpi, double neq[5]);
/* Eq. 21-22: returns u for populations f with porosity phi, buoyancy G. */
void orc_velocity(double rho0, const double f[9], double phi, double nu, double K,
                  double Fphi, const double G[2], double u[2]);
/* Eq. 23: returns p. */
double orc_pressure(double rho0, const double f[9], const double u[2], double phi);
/* Eq. 5. */
void orc_ergun(double phi, double dp2, double* K, double* Fphi);
/* One full node collision (Eq. 17 and Eq. 34) with the macroscopic values
 * given; writes f+ and g+. */
void orc_collide(const orc_lattice* lat, double phi, const double f[9], const double g[5],
                 const double u[2], double P, double T, const double F[2],
                 double fplus[9], double gplus[5]);

#ifdef __cplusplus
}
#endif
#endif
