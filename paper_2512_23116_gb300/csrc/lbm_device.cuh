// Device building blocks of the D3Q19 Guo-MRT-Smagorinsky step: velocity
// set, storage conversions, and the per-cell collision in FP32 registers.
//
// The collision follows Eq. (mrt_les_guo) (Sec. 2.3) with the moment basis,
// relaxation rates and equilibrium / force moments of App. B, the strain of
// Eq. (yu_strain) and the closure of Eqs. (eddy_visc), (les_viscosity),
// (strain_norm).  The 19x19 transforms are not multiplied out: the basis is
// orthogonal with integer rows, so
//   forward  m = M f'   uses the sums s_p and differences d_p of the nine
//                        opposite pairs (even rows see only s_p, odd rows d_p);
//   inverse  f* = M^T diag(1/|M_k|^2) m*  splits into an even part E_p and an
//                        odd part O_p per pair, f*_{+c} = E_p + O_p,
//                        f*_{-c} = E_p - O_p.
// About 250 FP32 operations per cell, all in registers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#include "lbm_check.cuh"
#include "lbm_internal.h"

namespace lbm {

// D3Q19 velocities in the paper's order (App. B table, index 1..19 -> 0..18);
// a and a^1 are opposite for a < 18, 18 is the rest particle.
__host__ __device__ constexpr int cx(int a) {
  constexpr int t[19] = {1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0};
  return t[a];
}
__host__ __device__ constexpr int cy(int a) {
  constexpr int t[19] = {0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 0};
  return t[a];
}
__host__ __device__ constexpr int cz(int a) {
  constexpr int t[19] = {0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0};
  return t[a];
}
__host__ __device__ constexpr int opp(int a) { return a == 18 ? 18 : (a ^ 1); }

// Position of population slot a inside a cell row of the row-interleaved
// layout (and inside a shared-memory tile of the TMA kernel): the slots are
// grouped by their own (cy, cz), so that each group is what one neighbouring
// cell row supplies to an odd-step tile.  Groups, in position order: (0,0)
// {0,1,18}, (-1,-1) {11}, (-1,0) {3,7,8}, (-1,1) {13}, (0,-1) {5,15,16},
// (0,1) {4,14,17}, (1,-1) {12}, (1,0) {2,6,9}, (1,1) {10}.
__host__ __device__ constexpr int gpos(int a) {
  constexpr int t[19] = {0, 1, 15, 4, 11, 8, 16, 5, 6, 17, 18, 3, 14, 7, 12, 9, 10, 13, 2};
  return t[a];
}
__host__ __device__ constexpr double weight(int a) {
  return a == 18 ? 1.0 / 3.0 : (a < 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Storage <-> FP32 conversions.
template <typename T> struct Storage;
template <> struct Storage<float> {
  static __device__ __forceinline__ float load(const float* p) { return *p; }
  static __device__ __forceinline__ float cvt(float v) { return v; }
  static __device__ __forceinline__ float pack(float v) { return v; }
};
template <> struct Storage<__half> {
  static __device__ __forceinline__ float load(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ float cvt(__half v) { return __half2float(v); }
  static __device__ __forceinline__ __half pack(float v) { return __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
  static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 pack(float v) { return __float2bfloat16_rn(v); }
};

// Per-cell quantities of the collision, used by the fused statistics.
struct CellDiag {
  float drho, ux, uy, uz, snorm, theta;
};

// Squared norms |M_k|^2 of the rows of M (orthogonal basis, App. B).
#define LBM_N0 19.f
#define LBM_N1 2394.f
#define LBM_N2 252.f
#define LBM_N3 10.f
#define LBM_N4 40.f
#define LBM_N9 36.f
#define LBM_N10 72.f
#define LBM_N11 12.f
#define LBM_N12 24.f
#define LBM_N13 4.f
#define LBM_N16 8.f

// Fixed relaxation rates of Eq. (relaxation-matrix): s1 (energy), s2 (energy
// square), s4 (heat flux), s10 = s12, s16 = s17 = s18; conserved moments have
// rate 1 and the five shear moments the local s_nu.
#define LBM_S1 1.19f
#define LBM_S2 1.4f
#define LBM_S4 1.2f
#define LBM_S10 1.4f
#define LBM_S16 1.98f

// Strain norm |S| from TT = T_ab T_ab (traceless part of the strain without the
// s9 factor) and Qt = 3 a1^2 (the energy-mode part), for one cell.
//   strain_mode 0: s9 = bare s_nu0, |S|^2 = 2 (s_nu0^2 TT + Qt);
//   strain_mode 1: s9 = s_nu(|S|) = 1/(b + 3 C |S|), b = 1/2 + 3 nu0, i.e. x = |S|
//     solves h(x) = x^2 - 2 TT s_nu(x)^2 - 2 Qt = 0.  Without Qt this is the
//     quadratic 3 C x^2 + b x = sqrt(2 TT), solved in its cancellation-free
//     form; two Newton steps then add the Qt part.
// |S| = SS2 rsqrt(SS2); below 1e-30 (|S| < 1e-15, so nu_t < 1e-15 for any
// C <= 1) the strain is taken as zero: the reciprocal square root of a
// subnormal is infinite, and 0 x inf would poison theta.
__device__ __forceinline__ float strain_norm(float TT, float Qt, float nu0, float s_nu0, float C,
                                             int strain_mode) {
  if (strain_mode != 1) {
    const float SS2 = 2.f * (s_nu0 * s_nu0 * TT + Qt);
    return SS2 > 1e-30f ? SS2 * rsqrtf(SS2) : 0.f;
  }
  const float b = 0.5f + 3.f * nu0;
  const float p2 = 2.f * TT;
  const float p = p2 > 1e-30f ? p2 * rsqrtf(p2) : 0.f;
  const float q = b * b + 12.f * C * p;  // >= b^2 >= 1/4
  const float xs = __fdividef(2.f * p, b + q * rsqrtf(q));
  const float x2 = xs * xs + 2.f * Qt;
  float x = x2 > 1e-30f ? x2 * rsqrtf(x2) : 0.f;
  // Newton on h(x) with h and h' both multiplied by w^3, w = b + 3 C x = 1/s_nu
  // (> 0): one division per step
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float w = fmaf(3.f * C, x, b);
    const float w3 = w * w * w;
    const float num = fmaf(x, x, -2.f * Qt) * w3 - p2 * w;
    const float den = fmaf(2.f * x, w3, 6.f * C * p2);
    if (den > 1e-30f) x -= __fdividef(num, den);
  }
  return x;
}

// In place: f (19 weight-shifted pre-collision populations) -> f* (post-collision),
// force F at the cell.  nu0, s_nu0: bare viscosity and shear rate; C: Smagorinsky
// constant (Delta = dx = 1).
__device__ __forceinline__ void mrt_collide(float (&f)[19], const float Fx, const float Fy,
                                            const float Fz, const float nu0, const float s_nu0,
                                            const float C, CellDiag& dg, const int strain_mode = 0) {
  // ---- m = M f' via pair sums and differences -------------------------------
  float s[9], d[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    s[p] = f[2 * p] + f[2 * p + 1];
    d[p] = f[2 * p] - f[2 * p + 1];
  }
  const float f18 = f[18];
  const float A = s[0] + s[1] + s[2];           // axis links
  const float Dxy = s[3] + s[4], Dyz = s[5] + s[6], Dxz = s[7] + s[8];
  const float D = Dxy + Dyz + Dxz;              // diagonal links
  const float m0 = A + D + f18;                 // drho
  const float m1 = fmaf(-11.f, A, fmaf(8.f, D, -30.f * f18));
  const float m2 = fmaf(-4.f, A, fmaf(12.f, f18, D));
  // momentum and the third-order moments m16..m18 share the pair combinations
  const float p34 = d[3] + d[4], q34 = d[3] - d[4];
  const float p56 = d[5] + d[6], q56 = d[5] - d[6];
  const float p78 = d[7] + d[8], q78 = d[7] - d[8];
  const float jx = d[0] + p34 + p78;
  const float jy = d[1] + q34 + p56;
  const float jz = d[2] + q56 + q78;
  const float m4 = fmaf(-5.f, d[0], jx);
  const float m6 = fmaf(-5.f, d[1], jy);
  const float m8 = fmaf(-5.f, d[2], jz);
  const float Pxx = fmaf(-1.f, A, 3.f * s[0]);  // 2 s0 - s1 - s2
  const float Qxx = fmaf(-3.f, Dyz, D);         // Dxy - 2 Dyz + Dxz
  const float m9 = Pxx + Qxx;
  const float m10 = fmaf(-2.f, Pxx, Qxx);
  const float Pww = s[1] - s[2];
  const float Qww = Dxy - Dxz;
  const float m11 = Pww + Qww;
  const float m12 = fmaf(-2.f, Pww, Qww);
  const float m13 = s[3] - s[4];
  const float m14 = s[5] - s[6];
  const float m15 = s[7] - s[8];
  const float m16 = p34 - p78;
  const float m17 = p56 - q34;
  const float m18 = q78 - q56;

  // ---- macroscopic fields, Eqs. (macroscopic_eq), (guo_velocity) ------------
  const float rho = 1.f + m0;
  // rho ~ 1: the MUFU reciprocal is within 2 ulp
  const float irho = __fdividef(1.f, rho);
  const float gx = fmaf(0.5f, Fx, jx), gy = fmaf(0.5f, Fy, jy), gz = fmaf(0.5f, Fz, jz);  // rho u
  const float ux = gx * irho, uy = gy * irho, uz = gz * irho;
  const float uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
  const float uu = uxx + uyy + uzz;

  // ---- equilibrium moments (Eq. meq_fm) and non-equilibrium parts ----------
  const float ruu = rho * uu;
  const float eq1 = fmaf(19.f, ruu, -11.f * m0);
  const float eq2 = (-475.f / 63.f) * ruu;
  const float n1 = m1 - eq1;
  const float n9 = fmaf(rho, fmaf(-3.f, uxx, uu), m9);  // m9 - rho (2 uxx - uyy - uzz)
  const float n11 = fmaf(rho, uzz - uyy, m11);          // m11 - rho (uyy - uzz)
  const float n13 = m13 - gx * uy;
  const float n14 = m14 - gy * uz;
  const float n15 = m15 - gx * uz;

  // ---- strain (Eq. yu_strain, s1 = 1.19) and closure -------------------------
  // S_ab = s9 T_ab + Q_ab with Q = -(s1 m1/38) on the diagonal; T is traceless,
  // so |S|^2 = 2 (s9^2 TT + 3 a1^2) (Eq. strain_norm) with TT = T_ab T_ab.
  const float a1 = (LBM_S1 / 38.f) * n1;
  const float Txx = -0.5f * n9;
  const float Tyy = 0.25f * fmaf(-3.f, n11, n9);
  const float Tzz = 0.25f * fmaf(3.f, n11, n9);
  const float Toff = fmaf(n13, n13, fmaf(n14, n14, n15 * n15));
  const float TT = fmaf(4.5f, Toff, fmaf(Txx, Txx, fmaf(Tyy, Tyy, Tzz * Tzz)));
  const float Qt = 3.f * (a1 * a1);
  const float snorm = strain_norm(TT, Qt, nu0, s_nu0, C, strain_mode);
  const float theta = fmaf(3.f * C, snorm, 3.f * nu0);  // tau_e - 1/2, Eq. (les_viscosity)
  // -s_nu = -1/(1/2 + theta); h = 1 - s_nu/2
  const float nsnu = __fdividef(-1.f, 0.5f + theta);
  const float h = fmaf(0.5f, nsnu, 1.f);
  const float h2 = h + h;

  // ---- force moments F_m (Eq. meq_fm) --------------------------------------
  const float uFx = ux * Fx, uFy = uy * Fy, uFz = uz * Fz;
  const float uF = uFx + uFy + uFz;
  const float tF = fmaf(-1.f, uF, 3.f * uFx);  // 2 uFx - uFy - uFz
  const float wF = uFy - uFz;

  // ---- m* = m - Lambda (m - m^eq) + (I - Lambda/2) F_m, scaled by 1/|M_k|^2
  const float mu0 = (1.f / LBM_N0) * m0;
  const float mu1 = fmaf(-LBM_S1 / LBM_N1, n1, fmaf((1.f - 0.5f * LBM_S1) * 38.f / LBM_N1, uF, (1.f / LBM_N1) * m1));
  const float mu2 = fmaf(LBM_S2 / LBM_N2, eq2,
                     fmaf((1.f - 0.5f * LBM_S2) * (-11.f) / LBM_N2, uF, ((1.f - LBM_S2) / LBM_N2) * m2));
  const float mu3 = (1.f / LBM_N3) * (jx + Fx);
  const float mu5 = (1.f / LBM_N3) * (jy + Fy);
  const float mu7 = (1.f / LBM_N3) * (jz + Fz);
  // heat-flux moments: m^eq = -2/3 rho u, F_m = -2/3 F
  constexpr float c4m = (1.f - LBM_S4) / LBM_N4, c4g = -LBM_S4 * (2.f / 3.f) / LBM_N4,
                  c4f = -(1.f - 0.5f * LBM_S4) * (2.f / 3.f) / LBM_N4;
  const float mu4 = fmaf(c4m, m4, fmaf(c4g, gx, c4f * Fx));
  const float mu6 = fmaf(c4m, m6, fmaf(c4g, gy, c4f * Fy));
  const float mu8 = fmaf(c4m, m8, fmaf(c4g, gz, c4f * Fz));
  const float mu9 = (1.f / LBM_N9) * fmaf(h2, tF, fmaf(nsnu, n9, m9));
  const float mu10 = fmaf((1.f - LBM_S10) / LBM_N10, m10, (-(1.f - 0.5f * LBM_S10) / LBM_N10) * tF);
  const float mu11 = (1.f / LBM_N11) * fmaf(h2, wF, fmaf(nsnu, n11, m11));
  const float mu12 = fmaf((1.f - LBM_S10) / LBM_N12, m12, (-(1.f - 0.5f * LBM_S10) / LBM_N12) * wF);
  const float mu13 = (1.f / LBM_N13) * fmaf(h, fmaf(uy, Fx, ux * Fy), fmaf(nsnu, n13, m13));
  const float mu14 = (1.f / LBM_N13) * fmaf(h, fmaf(uz, Fy, uy * Fz), fmaf(nsnu, n14, m14));
  const float mu15 = (1.f / LBM_N13) * fmaf(h, fmaf(uz, Fx, ux * Fz), fmaf(nsnu, n15, m15));
  const float mu16 = ((1.f - LBM_S16) / LBM_N16) * m16;
  const float mu17 = ((1.f - LBM_S16) / LBM_N16) * m17;
  const float mu18 = ((1.f - LBM_S16) / LBM_N16) * m18;

  // ---- f* = M^T mu: even part per pair, odd part per pair ------------------
  const float ca = fmaf(-11.f, mu1, fmaf(-4.f, mu2, mu0));  // axis columns: rows 0, 1, 2
  const float cd = fmaf(8.f, mu1, mu0 + mu2);               // diagonal columns
  const float e9 = mu9 + mu10, e11 = mu11 + mu12;
  const float P = fmaf(-2.f, mu10, mu9), Q = fmaf(-2.f, mu12, mu11);
  const float caP = ca - P;
  const float E0 = fmaf(2.f, P, ca);
  const float E1 = caP + Q;
  const float E2 = caP - Q;
  const float cde = cd + e9;
  const float Exy = cde + e11;
  const float Eyz = fmaf(-2.f, e9, cd);
  const float Exz = cde - e11;
  const float X = mu3 + mu4, Y = mu5 + mu6, Z = mu7 + mu8;
  const float O0 = fmaf(-4.f, mu4, mu3);
  const float O1 = fmaf(-4.f, mu6, mu5);
  const float O2 = fmaf(-4.f, mu8, mu7);
  const float O3 = (X + Y) + (mu16 - mu17);
  const float O4 = (X - Y) + (mu16 + mu17);
  const float O5 = (Y + Z) + (mu17 - mu18);
  const float O6 = (Y - Z) + (mu17 + mu18);
  const float O7 = (X + Z) + (mu18 - mu16);
  const float O8 = (X - Z) - (mu16 + mu18);
  const float Exyp = Exy + mu13, Exym = Exy - mu13;
  const float Eyzp = Eyz + mu14, Eyzm = Eyz - mu14;
  const float Exzp = Exz + mu15, Exzm = Exz - mu15;
  f[0] = E0 + O0;     f[1] = E0 - O0;
  f[2] = E1 + O1;     f[3] = E1 - O1;
  f[4] = E2 + O2;     f[5] = E2 - O2;
  f[6] = Exyp + O3;   f[7] = Exyp - O3;
  f[8] = Exym + O4;   f[9] = Exym - O4;
  f[10] = Eyzp + O5;  f[11] = Eyzp - O5;
  f[12] = Eyzm + O6;  f[13] = Eyzm - O6;
  f[14] = Exzp + O7;  f[15] = Exzp - O7;
  f[16] = Exzm + O8;  f[17] = Exzm - O8;
  f[18] = fmaf(-30.f, mu1, fmaf(12.f, mu2, mu0));

  dg.drho = m0;
  dg.ux = ux;
  dg.uy = uy;
  dg.uz = uz;
  dg.snorm = snorm;
  dg.theta = theta;
}

// Local equilibrium f' = M^-1 m^eq(drho, u) (App. B), for initialisation:
// m^eq has entries in rows 0-9, 11, 13-15 only.  FP32 arithmetic (the result
// is rounded to the storage precision anyway; FP64 is slow on this part).
__device__ __forceinline__ void equilibrium(float drho, float ux, float uy, float uz, float (&f)[19]) {
  const float rho = 1.f + drho;
  const float uxx = ux * ux, uyy = uy * uy, uzz = uz * uz, uu = uxx + uyy + uzz;
  const float mu0 = drho * (1.f / 19.f);
  const float mu1 = (-11.f * drho + 19.f * rho * uu) * (1.f / 2394.f);
  const float mu2 = (-475.f / 63.f / 252.f) * rho * uu;
  const float mu3 = rho * ux * 0.1f, mu5 = rho * uy * 0.1f, mu7 = rho * uz * 0.1f;
  const float mu4 = (-2.f / 3.f / 40.f) * rho * ux;
  const float mu6 = (-2.f / 3.f / 40.f) * rho * uy;
  const float mu8 = (-2.f / 3.f / 40.f) * rho * uz;
  const float mu9 = rho * (2.f * uxx - uyy - uzz) * (1.f / 36.f);
  const float mu11 = rho * (uyy - uzz) * (1.f / 12.f);
  const float mu13 = rho * ux * uy * 0.25f, mu14 = rho * uy * uz * 0.25f, mu15 = rho * ux * uz * 0.25f;
  const float ca = mu0 - 11.f * mu1 - 4.f * mu2;
  const float cd = mu0 + 8.f * mu1 + mu2;
  const float E0 = ca + 2.f * mu9;
  const float E1 = ca - mu9 + mu11;
  const float E2 = ca - mu9 - mu11;
  const float Exy = cd + mu9 + mu11, Eyz = cd - 2.f * mu9, Exz = cd + mu9 - mu11;
  const float X = mu3 + mu4, Y = mu5 + mu6, Z = mu7 + mu8;
  const float O0 = mu3 - 4.f * mu4, O1 = mu5 - 4.f * mu6, O2 = mu7 - 4.f * mu8;
  const float O3 = X + Y, O4 = X - Y, O5 = Y + Z, O6 = Y - Z, O7 = X + Z, O8 = X - Z;
  f[0] = E0 + O0;          f[1] = E0 - O0;
  f[2] = E1 + O1;          f[3] = E1 - O1;
  f[4] = E2 + O2;          f[5] = E2 - O2;
  f[6] = Exy + mu13 + O3;  f[7] = Exy + mu13 - O3;
  f[8] = Exy - mu13 + O4;  f[9] = Exy - mu13 - O4;
  f[10] = Eyz + mu14 + O5; f[11] = Eyz + mu14 - O5;
  f[12] = Eyz - mu14 + O6; f[13] = Eyz - mu14 - O6;
  f[14] = Exz + mu15 + O7; f[15] = Exz + mu15 - O7;
  f[16] = Exz - mu15 + O8; f[17] = Exz - mu15 - O8;
  f[18] = mu0 - 30.f * mu1 + 12.f * mu2;
}

__device__ __forceinline__ int wrap_dec(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int wrap_inc(int i, int n) { return i == n - 1 ? 0 : i + 1; }

// Position of cell (x, y, z) in a dense [nz][ny][nxp] array (one population).
__device__ __forceinline__ int64_t cell_off(int x, int y, int z, int ny, int nxp) {
  return ((int64_t)z * ny + y) * nxp + x;
}

// Position of population slot a of cell (x, y, z) in an instance's array.
__device__ __forceinline__ int64_t pop_off(const InstDesc& d, int a, int x, int y, int z) {
  return (d.slot_grouped ? gpos(a) : a) * d.slot_stride + z * d.plane_stride + y * d.row_stride + x;
}

// Index of the instance owning global tile t (tiles are sorted by instance),
// searching forward from `hint` (a block visits its tiles in increasing order).
__device__ __forceinline__ int find_instance(const InstDesc* __restrict__ insts, int ninst,
                                             int64_t t, int hint = 0) {
  int i = hint < 0 ? 0 : hint;
  if (i > 0 && t < insts[i].tile_begin) i = 0;
  while (i + 1 < ninst && t >= insts[i].tile_end) ++i;
  return i;
}

}  // namespace lbm
