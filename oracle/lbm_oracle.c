/*
 * FP64 CPU oracle of the MRT-Smagorinsky lattice Boltzmann step with Guo
 * forcing.  TEST INFRASTRUCTURE ONLY (see lbm_oracle.h): the parity oracle of
 * the CUDA path, written from the paper's equations, step by step and
 * without any blocking, fusion or factorisation:
 *
 *   macroscopics      Eqs. (macroscopic_eq), (guo_velocity)          App. A
 *   moments m = M f   Eq. (moment-matrix), dense 19x19 product        App. B
 *   m^eq              Eq. (meq_fm), left column                        App. B
 *   force moments     M Phi with Phi from Eq. (guo_force)              App. A
 *   strain, |S|       Eqs. (yu_strain), (strain_norm)                  App. B.1, Sec. 2.3
 *   tau_e             Eqs. (nu_eff_mrt), (eddy_visc), (les_viscosity)  Sec. 2.3
 *   collision         Eq. (mrt_les_guo) in moment space, Lambda of
 *                     Eq. (relaxation-matrix)                          Sec. 2.3, App. B
 *   back-transform    generic Gauss-Jordan inverse of M
 *   streaming         push, periodic, two lattices                     Sec. 3.1
 *   forcing           Eqs. (forcing_pattern), (forcing_amplitude)      Sec. 2.2
 *
 * Readings where the paper is silent:
 *  - populations are stored weight-shifted, f' = f - w, rho0 = 1, so that the
 *    printed m^eq (whose first entry is drho = rho - rho0) is consistent with
 *    M f' (M w = (1, -11, 3, 0, ..., 0));
 *  - the collision relaxes towards the printed m^eq (not M f^eq of Eq. feq);
 *  - the strain formula uses s1 = 1.19 and s9 = the bare shear rate s_nu0;
 *  - the forcing index (i, j, k) is the 0-based (x, y, z) cell index.
 *
 * Parity pins of every function: tests/test_oracle_*.py.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* App. B, D3Q19 table: index 1..19 -> 0..18. */
static const int C19[19][3] = {
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0}, {0, 0, 1},
    {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {1, 0, 1},
    {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {0, 0, 0}};

/* App. B, Eq. (moment-matrix), typed row by row as printed. */
static const int M19[19][19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, -30},
    {-4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 12},
    {1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0},
    {-4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0},
    {0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 0},
    {0, 0, -4, 4, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0},
    {0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0},
    {2, 2, -1, -1, -1, -1, 1, 1, 1, 1, -2, -2, -2, -2, 1, 1, 1, 1, 0},
    {-4, -4, 2, 2, 2, 2, 1, 1, 1, 1, -2, -2, -2, -2, 1, 1, 1, 1, 0},
    {0, 0, 1, 1, -1, -1, 1, 1, 1, 1, 0, 0, 0, 0, -1, -1, -1, -1, 0},
    {0, 0, -2, -2, 2, 2, 1, 1, 1, 1, 0, 0, 0, 0, -1, -1, -1, -1, 0},
    {0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0},
    {0, 0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, -1, 1, -1, 1, 0},
    {0, 0, 0, 0, 0, 0, -1, 1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 1, 1, -1, 1, -1, -1, 1, 0}};

void orc_lattice(int c[19][3], double w[19]) {
  for (int a = 0; a < 19; ++a) {
    int n2 = 0;
    for (int d = 0; d < 3; ++d) {
      c[a][d] = C19[a][d];
      n2 += C19[a][d] * C19[a][d];
    }
    /* App. B table: 1/18 for the six axis links, 1/36 for the twelve
     * diagonals, 1/3 for the rest particle. */
    w[a] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
}

void orc_moment_matrix(double M[19 * 19]) {
  for (int k = 0; k < 19; ++k)
    for (int a = 0; a < 19; ++a) M[k * 19 + a] = (double)M19[k][a];
}

int orc_invert(const double* A, double* Ainv, int n) {
  double* W = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(2 * n));
  if (!W) return -1;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) W[i * 2 * n + j] = A[i * n + j];
    for (int j = 0; j < n; ++j) W[i * 2 * n + n + j] = (i == j) ? 1.0 : 0.0;
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(W[r * 2 * n + col]) > fabs(W[piv * 2 * n + col])) piv = r;
    if (W[piv * 2 * n + col] == 0.0) {
      free(W);
      return -1;
    }
    if (piv != col)
      for (int j = 0; j < 2 * n; ++j) {
        double t = W[col * 2 * n + j];
        W[col * 2 * n + j] = W[piv * 2 * n + j];
        W[piv * 2 * n + j] = t;
      }
    double p = W[col * 2 * n + col];
    for (int j = 0; j < 2 * n; ++j) W[col * 2 * n + j] /= p;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double fct = W[r * 2 * n + col];
      if (fct == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) W[r * 2 * n + j] -= fct * W[col * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = W[i * 2 * n + n + j];
  free(W);
  return 0;
}

void orc_relaxation_rates(double s_nu, double lam[19]) {
  /* Eq. (relaxation-matrix). */
  const double fixed[19] = {1.0, 1.19, 1.4, 1.0, 1.2, 1.0, 1.2, 1.0, 1.2, 0.0,
                            1.4, 0.0,  1.4, 0.0, 0.0, 0.0, 1.98, 1.98, 1.98};
  for (int k = 0; k < 19; ++k) lam[k] = fixed[k];
  lam[9] = lam[11] = lam[13] = lam[14] = lam[15] = s_nu;
}

void orc_meq(double drho, const double u[3], double meq[19]) {
  /* Eq. (meq_fm), left column, rho = rho0 + drho with rho0 = 1. */
  const double rho = 1.0 + drho;
  const double ux = u[0], uy = u[1], uz = u[2];
  const double uu = ux * ux + uy * uy + uz * uz;
  meq[0] = drho;
  meq[1] = -11.0 * drho + 19.0 * rho * uu;
  meq[2] = -475.0 / 63.0 * rho * uu;
  meq[3] = rho * ux;
  meq[4] = -2.0 * rho * ux / 3.0;
  meq[5] = rho * uy;
  meq[6] = -2.0 * rho * uy / 3.0;
  meq[7] = rho * uz;
  meq[8] = -2.0 * rho * uz / 3.0;
  meq[9] = rho * (2.0 * ux * ux - uy * uy - uz * uz);
  meq[10] = 0.0;
  meq[11] = rho * (uy * uy - uz * uz);
  meq[12] = 0.0;
  meq[13] = rho * ux * uy;
  meq[14] = rho * uy * uz;
  meq[15] = rho * ux * uz;
  meq[16] = 0.0;
  meq[17] = 0.0;
  meq[18] = 0.0;
}

void orc_force_moments_printed(const double u[3], const double F[3], double Fm[19]) {
  /* Eq. (meq_fm), right column, as printed. */
  const double ux = u[0], uy = u[1], uz = u[2];
  const double Fx = F[0], Fy = F[1], Fz = F[2];
  const double uF = ux * Fx + uy * Fy + uz * Fz;
  Fm[0] = 0.0;
  Fm[1] = 38.0 * uF;
  Fm[2] = -11.0 * uF;
  Fm[3] = Fx;
  Fm[4] = -2.0 * Fx / 3.0;
  Fm[5] = Fy;
  Fm[6] = -2.0 * Fy / 3.0;
  Fm[7] = Fz;
  Fm[8] = -2.0 * Fz / 3.0;
  Fm[9] = 2.0 * (2.0 * ux * Fx - uy * Fy - uz * Fz);
  Fm[10] = -(2.0 * ux * Fx - uy * Fy - uz * Fz);
  Fm[11] = 2.0 * (uy * Fy - uz * Fz);
  Fm[12] = -(uy * Fy - uz * Fz);
  Fm[13] = ux * Fy + uy * Fx;
  Fm[14] = uy * Fz + uz * Fy;
  Fm[15] = ux * Fz + uz * Fx;
  Fm[16] = 0.0;
  Fm[17] = 0.0;
  Fm[18] = 0.0;
}

void orc_guo_source(const double u[3], const double F[3], double Phi[19]) {
  /* Eq. (guo_force): Phi_a = w_a [ (c_a - u)/cs^2 + (c_a.u) c_a / cs^4 ] . F,
   * cs^2 = 1/3. */
  int c[19][3];
  double w[19];
  orc_lattice(c, w);
  const double cs2 = 1.0 / 3.0;
  for (int a = 0; a < 19; ++a) {
    double cu = c[a][0] * u[0] + c[a][1] * u[1] + c[a][2] * u[2];
    double s = 0.0;
    for (int d = 0; d < 3; ++d)
      s += ((c[a][d] - u[d]) / cs2 + cu * c[a][d] / (cs2 * cs2)) * F[d];
    Phi[a] = w[a] * s;
  }
}

void orc_feq_poly(double rho, const double u[3], double feq[19]) {
  /* Eq. (feq). */
  int c[19][3];
  double w[19];
  orc_lattice(c, w);
  const double cs2 = 1.0 / 3.0;
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int a = 0; a < 19; ++a) {
    double cu = c[a][0] * u[0] + c[a][1] * u[1] + c[a][2] * u[2];
    feq[a] = w[a] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
  }
}

void orc_strain(const double mneq[19], double s1, double s9, double S[6]) {
  /* Eq. (yu_strain) with rho0 = dt = 1. */
  const double m1 = mneq[1], m9 = mneq[9], m11 = mneq[11];
  const double m13 = mneq[13], m14 = mneq[14], m15 = mneq[15];
  S[0] = -(s1 * m1 + 19.0 * s9 * m9) / 38.0;                      /* Sxx */
  S[1] = -(2.0 * s1 * m1 - 19.0 * s9 * (m9 - 3.0 * m11)) / 76.0;  /* Syy */
  S[2] = -(2.0 * s1 * m1 - 19.0 * s9 * (m9 + 3.0 * m11)) / 76.0;  /* Szz */
  S[3] = -1.5 * s9 * m13;                                         /* Sxy */
  S[4] = -1.5 * s9 * m15;                                         /* Sxz */
  S[5] = -1.5 * s9 * m14;                                         /* Syz */
}

double orc_strain_norm(const double S[6]) {
  /* Eq. (strain_norm). */
  return sqrt(2.0 * (S[0] * S[0] + S[1] * S[1] + S[2] * S[2] +
                     2.0 * S[3] * S[3] + 2.0 * S[4] * S[4] + 2.0 * S[5] * S[5]));
}

double orc_tau_e(double nu0, double C, double S_norm) {
  /* nu_t = C Delta^2 |S| with Delta = 1; 1/s_nu = 1/2 + 3 (nu0 + nu_t). */
  const double nu_t = C * S_norm;
  return 0.5 + 3.0 * (nu0 + nu_t);
}

double orc_strain_norm_selfconsistent(const double mneq[19], double s1, double nu0, double C) {
  /* g(x) = |S| evaluated with s9 = 1/(1/2 + 3 (nu0 + C x)); the fixed point
   * x = g(x) is the root of h(x) = g(x) - x.  g decreases in x, so h is
   * strictly decreasing: h(0) >= 0 and h(g(0)) <= 0 bracket the root. */
  double lo = 0.0, hi;
  {
    double S[6];
    orc_strain(mneq, s1, 1.0 / (0.5 + 3.0 * nu0), S);
    hi = orc_strain_norm(S);
  }
  if (!(C > 0.0) || hi == 0.0) return hi;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    double S[6];
    orc_strain(mneq, s1, 1.0 / (0.5 + 3.0 * (nu0 + C * mid)), S);
    if (orc_strain_norm(S) - mid > 0.0) lo = mid;
    else hi = mid;
    if (hi - lo <= 1e-17 * hi) break;
  }
  return 0.5 * (lo + hi);
}

/* ---- lattice state ------------------------------------------------------ */

struct orc_lbm {
  int nx, ny, nz;
  double nu0, C, s_nu0, F0;
  double body[3];
  int force_mode;
  int fixed_rate;
  int strain_mode;
  int64_t t;
  int c[19][3];
  double w[19];
  double M[19 * 19];
  double Minv[19 * 19];
  double* f; /* current populations, AoS: f[cell * 19 + a] */
  double* g; /* streaming target */
};

static size_t cell_index(const orc_lbm* L, int x, int y, int z) {
  return ((size_t)z * (size_t)L->ny + (size_t)y) * (size_t)L->nx + (size_t)x;
}

static int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

orc_lbm* orc_create(int nx, int ny, int nz, double nu0, double C, int force_mode,
                    double F0, const double body[3]) {
  if (nx < 1 || ny < 1 || nz < 1 || !(nu0 > 0.0) || !(C >= 0.0)) return NULL;
  if (force_mode < ORC_FORCE_NONE || force_mode > ORC_FORCE_KOLMOGOROV) return NULL;
  orc_lbm* L = (orc_lbm*)calloc(1, sizeof(orc_lbm));
  if (!L) return NULL;
  L->nx = nx;
  L->ny = ny;
  L->nz = nz;
  L->nu0 = nu0;
  L->C = C;
  /* Eq. (bare_viscosity): nu0 = cs^2 (1/s_nu - 1/2), cs^2 = 1/3. */
  L->s_nu0 = 1.0 / (0.5 + 3.0 * nu0);
  L->F0 = F0;
  L->force_mode = force_mode;
  for (int d = 0; d < 3; ++d) L->body[d] = body ? body[d] : 0.0;
  orc_lattice(L->c, L->w);
  orc_moment_matrix(L->M);
  if (orc_invert(L->M, L->Minv, 19) != 0) {
    free(L);
    return NULL;
  }
  size_t n = (size_t)nx * (size_t)ny * (size_t)nz * 19u;
  L->f = (double*)calloc(n, sizeof(double));
  L->g = (double*)calloc(n, sizeof(double));
  if (!L->f || !L->g) {
    orc_destroy(L);
    return NULL;
  }
  return L;
}

void orc_destroy(orc_lbm* L) {
  if (!L) return;
  free(L->f);
  free(L->g);
  free(L);
}

void orc_set_fixed_rate(orc_lbm* L, int fixed) { L->fixed_rate = fixed; }

void orc_set_strain_mode(orc_lbm* L, int mode) { L->strain_mode = mode; }

int64_t orc_time(const orc_lbm* L) { return L->t; }

void orc_force_at(const orc_lbm* L, int x, int y, int z, double F[3]) {
  const double two_pi = 6.283185307179586476925286766559;
  F[0] = F[1] = F[2] = 0.0;
  switch (L->force_mode) {
    case ORC_FORCE_PAPER_SIN: /* Eq. (forcing_pattern), (i, j, k) = (x, y, z). */
      F[0] = L->F0 * sin(two_pi * y / L->ny);
      F[1] = L->F0 * sin(two_pi * z / L->nz);
      F[2] = L->F0 * sin(two_pi * x / L->nx);
      break;
    case ORC_FORCE_CONST:
      F[0] = L->body[0];
      F[1] = L->body[1];
      F[2] = L->body[2];
      break;
    case ORC_FORCE_KOLMOGOROV:
      F[0] = L->F0 * sin(two_pi * y / L->ny);
      break;
    default:
      break;
  }
}

int orc_init_equilibrium(orc_lbm* L, const double* drho, const double* u) {
  const size_t ncell = (size_t)L->nx * L->ny * L->nz;
  for (size_t i = 0; i < ncell; ++i) {
    double uu[3] = {u[i], u[ncell + i], u[2 * ncell + i]};
    double dr = drho ? drho[i] : 0.0;
    double meq[19];
    orc_meq(dr, uu, meq);
    for (int a = 0; a < 19; ++a) {
      double s = 0.0;
      for (int k = 0; k < 19; ++k) s += L->Minv[a * 19 + k] * meq[k];
      L->f[i * 19 + a] = s;
    }
  }
  L->t = 0;
  return 0;
}

int orc_set_populations(orc_lbm* L, const double* fprime) {
  const size_t ncell = (size_t)L->nx * L->ny * L->nz;
  for (size_t i = 0; i < ncell; ++i)
    for (int a = 0; a < 19; ++a) L->f[i * 19 + a] = fprime[(size_t)a * ncell + i];
  return 0;
}

int orc_get_populations(const orc_lbm* L, double* fprime) {
  const size_t ncell = (size_t)L->nx * L->ny * L->nz;
  for (size_t i = 0; i < ncell; ++i)
    for (int a = 0; a < 19; ++a) fprime[(size_t)a * ncell + i] = L->f[i * 19 + a];
  return 0;
}

/* One cell: macroscopics, moments, closure and the post-collision
 * populations fstar.  Optional outputs: drho, u, |S|, theta. */
static void collide_cell(const orc_lbm* L, const double* fp, const double F[3],
                         double fstar[19], double* o_drho, double o_u[3],
                         double* o_snorm, double* o_theta) {
  /* Eqs. (macroscopic_eq), (guo_velocity): rho = sum f, rho u = sum f c + F/2;
   * with f' = f - w: sum w = 1 and sum w c = 0. */
  double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < 19; ++a) {
    drho += fp[a];
    for (int d = 0; d < 3; ++d) j[d] += fp[a] * L->c[a][d];
  }
  const double rho = 1.0 + drho;
  double u[3];
  for (int d = 0; d < 3; ++d) u[d] = (j[d] + 0.5 * F[d]) / rho;

  double m[19];
  for (int k = 0; k < 19; ++k) {
    double s = 0.0;
    for (int a = 0; a < 19; ++a) s += L->M[k * 19 + a] * fp[a];
    m[k] = s;
  }
  double meq[19], Phi[19], Fm[19], mneq[19];
  orc_meq(drho, u, meq);
  orc_guo_source(u, F, Phi);
  for (int k = 0; k < 19; ++k) {
    double s = 0.0;
    for (int a = 0; a < 19; ++a) s += L->M[k * 19 + a] * Phi[a];
    Fm[k] = s;
  }
  for (int k = 0; k < 19; ++k) mneq[k] = m[k] - meq[k];

  double snorm = 0.0, tau_e;
  if (L->fixed_rate) {
    tau_e = 1.0 / L->s_nu0;
  } else if (L->strain_mode == 1) {
    snorm = orc_strain_norm_selfconsistent(mneq, 1.19, L->nu0, L->C);
    tau_e = orc_tau_e(L->nu0, L->C, snorm);
  } else {
    double S[6];
    orc_strain(mneq, 1.19, L->s_nu0, S);
    snorm = orc_strain_norm(S);
    tau_e = orc_tau_e(L->nu0, L->C, snorm);
  }
  const double s_nu = 1.0 / tau_e;
  double lam[19];
  orc_relaxation_rates(s_nu, lam);

  /* Eq. (mrt_les_guo): m* = m - Lambda (m - m^eq) + (I - Lambda/2) M Phi. */
  double mstar[19];
  for (int k = 0; k < 19; ++k) mstar[k] = m[k] - lam[k] * mneq[k] + (1.0 - 0.5 * lam[k]) * Fm[k];
  for (int a = 0; a < 19; ++a) {
    double s = 0.0;
    for (int k = 0; k < 19; ++k) s += L->Minv[a * 19 + k] * mstar[k];
    fstar[a] = s;
  }
  if (o_drho) *o_drho = drho;
  if (o_u) for (int d = 0; d < 3; ++d) o_u[d] = u[d];
  if (o_snorm) *o_snorm = snorm;
  if (o_theta) *o_theta = tau_e - 0.5;
}

void orc_collide_one(const double fp[19], const double F[3], double nu0, double C,
                     int fixed_rate, double fstar[19], double* theta) {
  orc_lbm L;
  memset(&L, 0, sizeof L);
  L.nu0 = nu0;
  L.C = C;
  L.s_nu0 = 1.0 / (0.5 + 3.0 * nu0);
  L.fixed_rate = fixed_rate;
  orc_lattice(L.c, L.w);
  orc_moment_matrix(L.M);
  orc_invert(L.M, L.Minv, 19);
  collide_cell(&L, fp, F, fstar, NULL, NULL, NULL, theta);
}

int orc_step(orc_lbm* L, int64_t nsteps, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
      for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
          double F[3], fstar[19];
          orc_force_at(L, x, y, z, F);
          collide_cell(L, &L->f[cell_index(L, x, y, z) * 19], F, fstar, NULL, NULL, NULL, NULL);
          /* Push streaming: f_a(x + c_a, t + 1) = f*_a(x, t), periodic. */
          for (int a = 0; a < 19; ++a) {
            int xd = wrap(x + L->c[a][0], nx);
            int yd = wrap(y + L->c[a][1], ny);
            int zd = wrap(z + L->c[a][2], nz);
            L->g[cell_index(L, xd, yd, zd) * 19 + a] = fstar[a];
          }
        }
      }
    }
    double* t = L->f;
    L->f = L->g;
    L->g = t;
    L->t += 1;
  }
  return 0;
}

int orc_fields(const orc_lbm* L, double* drho, double* u, double* snorm, double* theta,
               int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  const size_t ncell = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z) {
    for (int y = 0; y < ny; ++y) {
      for (int x = 0; x < nx; ++x) {
        size_t i = cell_index(L, x, y, z);
        double F[3], fstar[19], dr, uu[3], sn, th;
        orc_force_at(L, x, y, z, F);
        collide_cell(L, &L->f[i * 19], F, fstar, &dr, uu, &sn, &th);
        if (drho) drho[i] = dr;
        if (u)
          for (int d = 0; d < 3; ++d) u[(size_t)d * ncell + i] = uu[d];
        if (snorm) snorm[i] = sn;
        if (theta) theta[i] = th;
      }
    }
  }
  return 0;
}
