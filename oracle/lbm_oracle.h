/*
 * FP64 CPU oracle of the MRT-Smagorinsky lattice Boltzmann step with Guo
 * forcing (Khan, Succi & Falcucci, "Validating the Boltzmann approach to the
 * large-eddy simulations of forced homogeneous incompressible turbulence").
 *
 * TEST INFRASTRUCTURE ONLY.  This header and lbm_oracle.c are the parity
 * oracle for the CUDA path: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may build, load or call them.
 * They share no code, header, table or constant with the CUDA library.
 *
 * Layout of every field exchanged through this header (fp64, host memory):
 *   populations  f'[a][z][y][x]   a = 0..18 is the paper's index 1..19
 *                                 (App. B, D3Q19 table; rest particle last),
 *                                 f' = f - w_a  (weight-shifted, rho0 = 1)
 *   vectors      v[d][z][y][x]    d = 0,1,2 = x,y,z components
 *   scalars      s[z][y][x]
 * x is the fastest index.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_FORCE_NONE = 0,       /* F = 0 */
  ORC_FORCE_PAPER_SIN = 1,  /* Eq. (forcing_pattern): Fx(y), Fy(z), Fz(x) */
  ORC_FORCE_CONST = 2,      /* uniform body force */
  ORC_FORCE_KOLMOGOROV = 3  /* Fx = F0 sin(2 pi y / ny) only */
};

typedef struct orc_lbm orc_lbm;

/* ---- the method's building blocks (App. A and B) ----------------------- */

/* D3Q19 velocities and weights in the paper's order (App. B table). */
void orc_lattice(int c[19][3], double w[19]);
/* Moment matrix M as printed in App. B, Eq. (moment-matrix), row-major. */
void orc_moment_matrix(double M[19 * 19]);
/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix.
 * Returns 0 on success, -1 if singular. */
int orc_invert(const double* A, double* Ainv, int n);
/* Relaxation rates of Eq. (relaxation-matrix) with shear rate s_nu. */
void orc_relaxation_rates(double s_nu, double lam[19]);
/* Equilibrium moments of Eq. (meq_fm), left column; rho = 1 + drho. */
void orc_meq(double drho, const double u[3], double meq[19]);
/* Force moments of Eq. (meq_fm), right column, as printed. */
void orc_force_moments_printed(const double u[3], const double F[3], double Fm[19]);
/* Guo source Phi_a of Eq. (guo_force) in population space. */
void orc_guo_source(const double u[3], const double F[3], double Phi[19]);
/* Polynomial equilibrium of Eq. (feq) (full populations, not shifted). */
void orc_feq_poly(double rho, const double u[3], double feq[19]);
/* Strain rate components of Eq. (yu_strain) from non-equilibrium moments:
 * S = {Sxx, Syy, Szz, Sxy, Sxz, Syz}; rho0 = dt = 1. */
void orc_strain(const double mneq[19], double s1, double s9, double S[6]);
/* Frobenius-type norm of Eq. (strain_norm). */
double orc_strain_norm(const double S[6]);
/* Effective relaxation time tau_e of Eqs. (nu_eff_mrt)-(les_viscosity),
 * Delta = dx = 1. */
double orc_tau_e(double nu0, double C, double S_norm);

/* Self-consistent strain norm: Eq. (yu_strain) with s9 = s_nu(|S|) =
 * 1/(1/2 + 3 (nu0 + C |S|)) (Eq. les_viscosity) instead of the bare rate,
 * solved for |S| by bisection to round-off.  Returns |S|. */
double orc_strain_norm_selfconsistent(const double mneq[19], double s1, double nu0, double C);

/* Strain evaluation of the collision: 0 = explicit, s9 = bare s_nu0 (default
 * reading); 1 = self-consistent (orc_strain_norm_selfconsistent). */
void orc_set_strain_mode(orc_lbm* L, int mode);

/* One collision (Eq. mrt_les_guo, moment space) of a single cell, outside any
 * lattice: fp = the 19 pre-collision f', F = the force at the cell; returns the
 * post-collision f'* and, when theta is not NULL, tau_e - 1/2.  fixed_rate = 1
 * relaxes with the bare rate (no strain). */
void orc_collide_one(const double fp[19], const double F[3], double nu0, double C,
                     int fixed_rate, double fstar[19], double* theta);

/* ---- lattice state -------------------------------------------------------- */

/* nu0 > 0: bare viscosity; C >= 0: Smagorinsky constant (linear, Eq. eddy_visc);
 * F0: forcing amplitude for the sinusoidal modes; body: constant force.
 * Returns NULL on invalid arguments or allocation failure. */
orc_lbm* orc_create(int nx, int ny, int nz, double nu0, double C,
                    int force_mode, double F0, const double body[3]);
void orc_destroy(orc_lbm* L);
/* Force on cell (x, y, z). */
void orc_force_at(const orc_lbm* L, int x, int y, int z, double F[3]);
/* f' = M^-1 m^eq(drho, u) at every cell; drho may be NULL (zero). */
int orc_init_equilibrium(orc_lbm* L, const double* drho, const double* u);
int orc_set_populations(orc_lbm* L, const double* fprime);
int orc_get_populations(const orc_lbm* L, double* fprime);
/* Advance nsteps time steps (collide, then push-stream; two lattices).
 * nthreads <= 0 uses the OpenMP default. */
int orc_step(orc_lbm* L, int64_t nsteps, int nthreads);
/* Per-cell quantities of the current state, as the next collision sees them:
 * drho, u (Guo-corrected), |S|, theta = tau_e - 1/2.  Any pointer may be NULL. */
int orc_fields(const orc_lbm* L, double* drho, double* u, double* snorm,
               double* theta, int nthreads);
/* Set to 1 to skip the strain computation and relax with the bare rate
 * s_nu0 (the constant-viscosity MRT model). */
void orc_set_fixed_rate(orc_lbm* L, int fixed);
int64_t orc_time(const orc_lbm* L);

#ifdef __cplusplus
}
#endif
#endif
