/*
 * clbm_oracle.c -- FP64 CPU oracle of the D3Q19 cascaded central-moment LBM
 * for power-law fluids (Adam, Hajabdollahi & Premnath, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY (see clbm_oracle.h).  Plain loops in the order the
 * paper states the method; no blocking, fusion or reordering.  Built with
 * -ffp-contract=off so that no multiply-add is fused behind the reader's back.
 *
 * Readings of passages where the paper is silent or garbled (each is named at
 * the line that depends on it):
 *   [c1] matrix K, entry (alpha=15, j=14): built from the definition of K_14,
 *        which gives +1 where the printed matrix shows -1.
 *   [c2] post-collision f~_15: follows from K (coefficient +1 on g^_6) where
 *        the printed list shows -g^_6.
 *   [c3] brackets of g^_15, g^_16, g^_17 (Eqs. collisionkernelg15..17).
 *   [c4] 4th-order factorised attractor k~ii k~jj / rho.
 *   [c5] omega_nu solved implicitly at the node (S_ij depends on omega_nu).
 *   [c6] kinematic viscosity clamped to [nu_min, nu_max].
 *   [c7] body force: symmetric (Strang) split, half source before and after
 *        the collision, u* = (j + F/2)/rho.
 *   [c8] moving lid: halfway bounce-back plus 6 w_a rho0 (e_a . U), lid taking
 *        precedence over other walls on edges and corners.
 *   [c10] rest initial state f = w rho0.
 *   [c11] residual R = ||u - u_prev|| / (delta ||u||).
 */
#include "clbm_oracle.h"

#include <math.h>
#include <stddef.h>
#include <string.h>

/* D3Q19 velocity set in the paper's order (Eq. velocityd3qq19 and the
 * component vectors |e_x>, |e_y>, |e_z> listed after the raw basis). */
static const int E[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, 1, 0},  {1, -1, 0},
    {-1, -1, 0}, {1, 0, 1}, {-1, 0, 1}, {1, 0, -1},  {-1, 0, -1},
    {0, 1, 1},  {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};

/* Lattice weights.  The paper does not print them; these are the D3Q19
 * weights fixed by c_s^2 = 1/3 (Sec. 3, Maxwellian) and the fourth-order
 * moment c_s^4 rho of the Maxwellian central moments. */
static double W(int a) {
  int s = E[a][0] * E[a][0] + E[a][1] * E[a][1] + E[a][2] * E[a][2];
  if (s == 0) return 1.0 / 3.0;
  if (s == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

static int opposite(int a) {
  for (int b = 0; b < 19; ++b)
    if (E[b][0] == -E[a][0] && E[b][1] == -E[a][1] && E[b][2] == -E[a][2])
      return b;
  return -1;
}

/* Orthogonal basis |K_j> evaluated at velocity (x, y, z) (Sec. 3, the
 * Gram-Schmidt basis written as polynomials of e).  [c1]: entry (15, 14)
 * comes out as +1 here. */
static double kbasis(int j, double x, double y, double z) {
  double x2 = x * x, y2 = y * y, z2 = z * z, e2 = x2 + y2 + z2;
  switch (j) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * y;
    case 5: return x * z;
    case 6: return y * z;
    case 7: return x2 - y2;
    case 8: return e2 - 3.0 * z2;
    case 9: return 19.0 * e2 - 30.0;
    case 10: return 5.0 * x * e2 - 9.0 * x;
    case 11: return 5.0 * y * e2 - 9.0 * y;
    case 12: return 5.0 * z * e2 - 9.0 * z;
    case 13: return x * y2 - x * z2;
    case 14: return z2 * y - y * x2;
    case 15: return x2 * z - y2 * z;
    case 16: return 21.0 * (x2 * y2 + x2 * z2 + y2 * z2) - 16.0 * e2 + 12.0;
    case 17: return 3.0 * (x2 * y2 + x2 * z2 - 2.0 * y2 * z2) -
                    2.0 * (2.0 * x2 - y2 - z2);
    case 18: return 3.0 * (x2 * y2 - x2 * z2) - 2.0 * (y2 - z2);
  }
  return 0.0;
}

/* K[alpha][j] and the opposite directions, evaluated once from the
 * definitions above when the library is loaded. */
static double KMAT[19][19];
static int OPP[19];
__attribute__((constructor)) static void build_tables(void) {
  for (int a = 0; a < 19; ++a) {
    OPP[a] = opposite(a);
    for (int j = 0; j < 19; ++j)
      KMAT[a][j] = kbasis(j, E[a][0], E[a][1], E[a][2]);
  }
}

void orc_velocities(int e_out[19][3]) { memcpy(e_out, E, sizeof(E)); }

void orc_weights(double w_out[19]) {
  for (int a = 0; a < 19; ++a) w_out[a] = W(a);
}

void orc_kmatrix(double K_out[19][19]) {
  for (int a = 0; a < 19; ++a)
    for (int j = 0; j < 19; ++j)
      K_out[a][j] = kbasis(j, E[a][0], E[a][1], E[a][2]);
}

void orc_default_params(orc_params* p) {
  memset(p, 0, sizeof(*p));
  p->nx = p->ny = p->nz = 1;
  p->K = 0.1;
  p->n = 1.0;
  p->rho0 = 1.0;
  p->nu_min = 5e-4;
  p->nu_max = 10.0;
  for (int j = 0; j < 19; ++j) p->omega[j] = 1.0;
  p->attractor_over_rho = 1;
}

/* ------------------------------------------------------------------------ */
/* Shear rate and local relaxation rate (Sec. 3.2).                          */

/* |gamma_dot| from the strain-rate tensor of Eq. strainratetensor at a trial
 * omega_nu, through Eq. shearrateexpression.  m[4..9] are the
 * non-equilibrium moments m^(1)_4..9; omega_zeta = omega_9. */
static double shear_rate(double omega, double omega_zeta, double rho,
                         const double m[10]) {
  double Sxy = -3.0 / (2.0 * rho) * omega * m[4];
  double Sxz = -3.0 / (2.0 * rho) * omega * m[5];
  double Syz = -3.0 / (2.0 * rho) * omega * m[6];
  double Sxx = -1.0 / (2.0 * rho) * (omega * (m[7] + m[8]) + omega_zeta * m[9]);
  double Syy =
      -1.0 / (2.0 * rho) * (omega * (-2.0 * m[7] + m[8]) + omega_zeta * m[9]);
  double Szz =
      -1.0 / (2.0 * rho) * (omega * (m[7] - 2.0 * m[8]) + omega_zeta * m[9]);
  double s = Sxx * Sxx + Syy * Syy + Szz * Szz +
             2.0 * (Sxy * Sxy + Syz * Syz + Sxz * Sxz);
  return sqrt(2.0 * s);
}

/* Kinematic viscosity of the power-law fluid, nu = mu/rho with
 * mu = K |gamma_dot|^(n-1) (Eq. 6), clamped to [nu_min, nu_max] [c6].
 * At zero shear rate: n < 1 -> nu_max, n > 1 -> nu_min, n = 1 -> K/rho. */
static double viscosity(const orc_params* p, double rho, double gd) {
  double nu;
  if (p->n == 1.0) {
    nu = p->K / rho;
  } else if (gd == 0.0) {
    nu = (p->n < 1.0) ? p->nu_max : p->nu_min;
  } else {
    nu = p->K / rho * pow(gd, p->n - 1.0);
  }
  if (nu < p->nu_min) nu = p->nu_min;
  if (nu > p->nu_max) nu = p->nu_max;
  return nu;
}

/* h(omega) = 1/omega - 1/2 - nu(gamma_dot(omega)) / c_s^2, the residual of
 * Eq. localvarationsrelaxationtimes with mu/rho = nu and c_s^2 = 1/3. */
static double h_of(const orc_params* p, double rho, const double m[10],
                   double omega) {
  double gd = shear_rate(omega, p->omega[9], rho, m);
  return 1.0 / omega - 0.5 - 3.0 * viscosity(p, rho, gd);
}

double orc_omega_solve(const orc_params* p, double rho, const double m[10],
                       double* gamma_dot) {
  double omega;
  if (p->n == 1.0) {
    /* Newtonian: omega = [K/(rho c_s^2) + 1/2]^-1 with the clamp. */
    double nu = viscosity(p, rho, 0.0);
    omega = 1.0 / (3.0 * nu + 0.5);
  } else {
    /* [c5] Implicit solve.  h is decreasing through its unique root, and
     * the clamp puts the root inside [omega(nu_max), omega(nu_min)]. */
    double lo = 1.0 / (3.0 * p->nu_max + 0.5);
    double hi = 1.0 / (3.0 * p->nu_min + 0.5);
    double hlo = h_of(p, rho, m, lo);
    double hhi = h_of(p, rho, m, hi);
    if (hhi >= 0.0) {
      omega = hi;
    } else if (hlo <= 0.0) {
      omega = lo;
    } else {
      /* Plain bisection down to adjacent doubles. */
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (h_of(p, rho, m, mid) > 0.0)
          lo = mid;
        else
          hi = mid;
      }
      omega = 0.5 * (lo + hi);
    }
  }
  if (gamma_dot) *gamma_dot = shear_rate(omega, p->omega[9], rho, m);
  return omega;
}

/* ------------------------------------------------------------------------ */
/* Collision (Sec. 3.1 - 3.3).                                               */

void orc_collide(const orc_params* p, const double f[19], double ft[19],
                 orc_node_info* info) {
  /* Hydrodynamic fields, Eqs. hydrodynamicfields1/2. */
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int a = 0; a < 19; ++a) {
    rho += f[a];
    jx += f[a] * E[a][0];
    jy += f[a] * E[a][1];
    jz += f[a] * E[a][2];
  }
  const double Fx = p->F[0], Fy = p->F[1], Fz = p->F[2];
  /* [c7] half-force velocity and the source S_a whose moments are 0, F and
   * uF + Fu. */
  double ux = (jx + 0.5 * Fx) / rho;
  double uy = (jy + 0.5 * Fy) / rho;
  double uz = (jz + 0.5 * Fz) / rho;
  double S[19], fs[19];
  for (int a = 0; a < 19; ++a) {
    double eF = E[a][0] * Fx + E[a][1] * Fy + E[a][2] * Fz;
    double eu = E[a][0] * ux + E[a][1] * uy + E[a][2] * uz;
    double uF = ux * Fx + uy * Fy + uz * Fz;
    S[a] = W(a) * (3.0 * eF + 9.0 * eu * eF - 3.0 * uF);
    fs[a] = f[a] + 0.5 * S[a];
  }

  /* Raw moments k'_{x^m y^n z^p} = <e_x^m e_y^n e_z^p | f>
   * (Eq. rawmomentdistributionfunction1), of the half-forced populations. */
  double kxx = 0, kyy = 0, kzz = 0, kxy = 0, kxz = 0, kyz = 0;
  double kxyy = 0, kxzz = 0, kxxy = 0, kyzz = 0, kxxz = 0, kyyz = 0;
  double kxxyy = 0, kxxzz = 0, kyyzz = 0;
  for (int a = 0; a < 19; ++a) {
    double x = E[a][0], y = E[a][1], z = E[a][2], v = fs[a];
    kxx += x * x * v;
    kyy += y * y * v;
    kzz += z * z * v;
    kxy += x * y * v;
    kxz += x * z * v;
    kyz += y * z * v;
    kxyy += x * y * y * v;
    kxzz += x * z * z * v;
    kxxy += x * x * y * v;
    kyzz += y * z * z * v;
    kxxz += x * x * z * v;
    kyyz += y * y * z * v;
    kxxyy += x * x * y * y * v;
    kxxzz += x * x * z * z * v;
    kyyzz += y * y * z * z * v;
  }

  const double ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;

  /* Non-equilibrium second moments m^(1)_4..9 (Sec. 3.2). */
  double m[10] = {0};
  m[4] = kxy - rho * ux * uy;
  m[5] = kxz - rho * ux * uz;
  m[6] = kyz - rho * uy * uz;
  m[7] = (kxx - kyy) - rho * (ux2 - uy2);
  m[8] = (kxx - kzz) - rho * (ux2 - uz2);
  m[9] = (kxx + kyy + kzz) - (rho * (ux2 + uy2 + uz2) + rho);

  /* Local relaxation rate of the second-order moments. */
  double gd = 0.0;
  double wnu = orc_omega_solve(p, rho, m, &gd);
  double w[19];
  for (int j = 0; j < 19; ++j) w[j] = p->omega[j];
  w[4] = w[5] = w[6] = w[7] = w[8] = wnu;

  /* Change of moments under collision, Eqs. collisionkernelg4..g18.
   * g^_0..g^_3 = 0 (collision invariants). */
  double g[19] = {0};
  g[4] = w[4] / 4.0 * (-kxy + rho * ux * uy);
  g[5] = w[5] / 4.0 * (-kxz + rho * ux * uz);
  g[6] = w[6] / 4.0 * (-kyz + rho * uy * uz);
  g[7] = w[7] / 12.0 * (-(kxx - kyy) + rho * (ux2 - uy2));
  g[8] = w[8] / 36.0 *
         (-(kxx + kyy - 2.0 * kzz) + rho * (ux2 + uy2 - 2.0 * uz2));
  g[9] = w[9] / 126.0 *
         (-(kxx + kyy + kzz) + rho * (ux2 + uy2 + uz2) + rho);

  g[10] = w[10] / 8.0 *
              (-(kxyy + kxzz) + 2.0 * (uy * kxy + uz * kxz) +
               ux * (kyy + kzz) - 2.0 * rho * ux * (uy2 + uz2)) +
          (uy * g[4] + uz * g[5]) +
          0.75 * ux * (-(g[7] + g[8]) + 14.0 * g[9]);
  g[11] = w[11] / 8.0 *
              (-(kyzz + kxxy) + 2.0 * (ux * kxy + uz * kyz) +
               uy * (kxx + kzz) - 2.0 * rho * uy * (ux2 + uz2)) +
          (ux * g[4] + uz * g[6]) + 0.75 * uy * (g[7] - g[8] + 14.0 * g[9]);
  g[12] = w[12] / 8.0 *
              (-(kxxz + kyyz) + 2.0 * (ux * kxz + uy * kyz) +
               uz * (kxx + kyy) - 2.0 * rho * uz * (ux2 + uy2)) +
          (ux * g[5] + uy * g[6]) + 1.5 * uz * (g[8] + 7.0 * g[9]);
  g[13] = w[13] / 8.0 *
              (-(kxyy - kxzz) + 2.0 * (uy * kxy - uz * kxz) +
               ux * (kyy - kzz) - 2.0 * rho * ux * (uy2 - uz2)) +
          (uy * g[4] - uz * g[5]) + 0.75 * ux * (-g[7] + 3.0 * g[8]);
  g[14] = w[14] / 8.0 *
              (-(kyzz - kxxy) + 2.0 * (uz * kyz - ux * kxy) +
               uy * (kzz - kxx) - 2.0 * rho * uy * (uz2 - ux2)) +
          (-ux * g[4] + uz * g[6]) + 0.75 * uy * (-g[7] - 3.0 * g[8]);
  /* [c3] the omega_15/8 bracket closes after -2 rho u_z (u_x^2 - u_y^2). */
  g[15] = w[15] / 8.0 *
              (-(kxxz - kyyz) + 2.0 * (ux * kxz - uy * kyz) +
               uz * (kxx - kyy) - 2.0 * rho * uz * (ux2 - uy2)) +
          (ux * g[5] - uy * g[6]) + 1.5 * uz * g[7];

  /* Post-collision central second moments, from the moments of K g^ (the
   * <K g^ | e_i^2> rows of Eq. momentscascadedcollisionterm) added to the
   * pre-collision central moments k_ii = k'_ii - rho u_i^2. */
  double Kxx = (kxx - rho * ux2) + 6.0 * g[7] + 6.0 * g[8] + 42.0 * g[9];
  double Kyy = (kyy - rho * uy2) - 6.0 * g[7] + 6.0 * g[8] + 42.0 * g[9];
  double Kzz = (kzz - rho * uz2) - 12.0 * g[8] + 42.0 * g[9];
  /* [c4] factorised 4th-order attractors k~ii k~jj / rho. */
  double sc = p->attractor_over_rho ? 1.0 / rho : 1.0;
  double Axy = Kxx * Kyy * sc, Axz = Kxx * Kzz * sc, Ayz = Kyy * Kzz * sc;

  /* [c3] g^_16: the stray parenthesis after (k'_yy + k'_zz) is dropped. */
  g[16] = w[16] / 12.0 *
              (-(kxxyy + kxxzz + kyyzz) + 2.0 * ux * (kxyy + kxzz) +
               2.0 * uy * (kxxy + kyzz) + 2.0 * uz * (kxxz + kyyz) -
               ux2 * (kyy + kzz) - uy2 * (kzz + kxx) - uz2 * (kxx + kyy) -
               4.0 * (ux * uy * kxy + ux * uz * kxz + uy * uz * kyz) +
               3.0 * rho * (ux2 * uy2 + ux2 * uz2 + uy2 * uz2) +
               (Axy + Axz + Ayz)) -
          4.0 / 3.0 * ux * uy * g[4] - 4.0 / 3.0 * ux * uz * g[5] -
          4.0 / 3.0 * uy * uz * g[6] + 0.5 * (ux2 - uy2) * g[7] +
          0.5 * (ux2 + uy2 - 2.0 * uz2) * g[8] +
          (-7.0 * (ux2 + uy2 + uz2) - 8.0) * g[9] + 4.0 / 3.0 * ux * g[10] +
          4.0 / 3.0 * uy * g[11] + 4.0 / 3.0 * uz * g[12];
  /* [c3] g^_17: the third-order group is
   * 2[(u_x k'_xyy + u_x k'_xzz + u_y k'_xxy + u_z k'_xxz)
   *   - 2(u_y k'_yzz + u_z k'_yyz)]. */
  g[17] = w[17] / 24.0 *
              (-(kxxyy + kxxzz - 2.0 * kyyzz) +
               2.0 * ((ux * kxyy + ux * kxzz + uy * kxxy + uz * kxxz) -
                      2.0 * (uy * kyzz + uz * kyyz)) -
               ux2 * (kyy + kzz) - uy2 * (kxx - 2.0 * kzz) -
               uz2 * (kxx - 2.0 * kyy) -
               4.0 * (ux * uy * kxy + ux * uz * kxz - 2.0 * uy * uz * kyz) +
               (Axy + Axz - 2.0 * Ayz) +
               3.0 * rho * (ux2 * uy2 + ux2 * uz2 - 2.0 * uy2 * uz2)) -
          2.0 / 3.0 * ux * uy * g[4] - 2.0 / 3.0 * ux * uz * g[5] +
          4.0 / 3.0 * uy * uz * g[6] +
          0.25 * (ux2 - uy2 - 3.0 * uz2 - 2.0) * g[7] +
          0.25 * (ux2 - 5.0 * uy2 + uz2 - 2.0) * g[8] +
          1.75 * (-2.0 * ux2 + uy2 + uz2) * g[9] + 2.0 / 3.0 * ux * g[10] -
          1.0 / 3.0 * uy * g[11] - 1.0 / 3.0 * uz * g[12] - uy * g[14] +
          uz * g[15];
  g[18] = w[18] / 8.0 *
              (-(kxxyy - kxxzz) +
               2.0 * (ux * kxyy - ux * kxzz + uy * kxxy - uz * kxxz) -
               ux2 * (kyy - kzz) - uy2 * kxx + uz2 * kxx -
               4.0 * (ux * uy * kxy - ux * uz * kxz) + (Axy - Axz) +
               3.0 * rho * (ux2 * uy2 - ux2 * uz2)) -
          2.0 * ux * uy * g[4] + 2.0 * ux * uz * g[5] +
          0.75 * (ux2 - uy2 + uz2 + 2.0 / 3.0) * g[7] +
          0.75 * (-3.0 * ux2 - uy2 + uz2 - 2.0) * g[8] +
          5.25 * (-uy2 + uz2) * g[9] + uy * g[11] - uz * g[12] +
          2.0 * ux * g[13] - uy * g[14] - uz * g[15];

  /* Post-collision populations f~ = f + K g^ (Eqs. cascadecollision1,
   * cascadedcollision1), with the second half of the source [c7].  [c2]: the
   * f~_15 row follows from K. */
  for (int a = 0; a < 19; ++a) {
    double Kg = 0.0;
    for (int j = 0; j < 19; ++j)
      Kg += KMAT[a][j] * g[j];
    ft[a] = fs[a] + Kg + 0.5 * S[a];
  }

  if (info) {
    info->rho = rho;
    info->u[0] = ux;
    info->u[1] = uy;
    info->u[2] = uz;
    info->gamma_dot = gd;
    info->omega_nu = wnu;
    for (int j = 0; j < 19; ++j) info->g[j] = g[j];
  }
}

/* ------------------------------------------------------------------------ */
/* Streaming with boundaries and the time loop.                             */

static size_t idx(const orc_params* p, int q, int x, int y, int z) {
  return (((size_t)q * p->nz + z) * p->ny + y) * p->nx + x;
}

/* Pull of direction a into node (x, y, z): f_a(x) = f~_a(x - e_a)
 * (Eq. cascadedstreaming1).  A source outside the box is resolved by the face
 * it lies beyond: periodic faces wrap; otherwise halfway bounce-back
 * f_a(x) = f~_abar(x) (Sec. 4.1), and if one of the crossed faces is a lid,
 * plus the momentum correction 6 w_a rho0 (e_a . U) [c8]. */
static double pull_one(const orc_params* p, const double* A, int a, int x,
                       int y, int z) {
  int pos[3] = {x, y, z};
  int dim[3] = {p->nx, p->ny, p->nz};
  int src[3];
  int bounced = 0, lid = 0;
  for (int d = 0; d < 3; ++d) {
    int s = pos[d] - E[a][d];
    if (s < 0 || s >= dim[d]) {
      int face = 2 * d + (s < 0 ? 0 : 1);
      if (p->face[face] == ORC_PERIODIC) {
        s = (s + dim[d]) % dim[d];
      } else {
        bounced = 1;
        if (p->face[face] == ORC_LID) lid = 1;
      }
    }
    src[d] = s;
  }
  if (!bounced) return A[idx(p, a, src[0], src[1], src[2])];
  double v = A[idx(p, OPP[a], x, y, z)];
  if (lid) {
    double eU = E[a][0] * p->U[0] + E[a][1] * p->U[1] + E[a][2] * p->U[2];
    v += 6.0 * W(a) * p->rho0 * eU;
  }
  return v;
}

void orc_rest_state(const orc_params* p, double* f) {
  size_t N = (size_t)p->nx * p->ny * p->nz;
  for (int a = 0; a < 19; ++a)
    for (size_t i = 0; i < N; ++i) f[(size_t)a * N + i] = W(a) * p->rho0;
}

void orc_pull(const orc_params* p, const double* A, double* out) {
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x)
        for (int a = 0; a < 19; ++a)
          out[idx(p, a, x, y, z)] = pull_one(p, A, a, x, y, z);
}

static void step_once(const orc_params* p, const double* A, double* B) {
#pragma omp parallel for schedule(static) if (p->nz >= 4)
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        double f[19], ft[19];
        for (int a = 0; a < 19; ++a) f[a] = pull_one(p, A, a, x, y, z);
        orc_collide(p, f, ft, NULL);
        for (int a = 0; a < 19; ++a) B[idx(p, a, x, y, z)] = ft[a];
      }
}

int orc_run(const orc_params* p, double* A, double* B, int64_t nsteps) {
  size_t total = (size_t)19 * p->nx * p->ny * p->nz;
  for (int64_t s = 0; s < nsteps; ++s) {
    step_once(p, A, B);
    /* plain copy back so that A holds the state between calls */
    memcpy(A, B, total * sizeof(double));
  }
  return 0;
}

void orc_fields(const orc_params* p, const double* A, double* rho, double* u,
                double* gamma_dot) {
  size_t N = (size_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static) if (p->nz >= 4)
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        double f[19], ft[19];
        orc_node_info info;
        for (int a = 0; a < 19; ++a) f[a] = pull_one(p, A, a, x, y, z);
        orc_collide(p, f, ft, &info);
        size_t i = ((size_t)z * p->ny + y) * p->nx + x;
        if (rho) rho[i] = info.rho;
        if (u) {
          u[i] = info.u[0];
          u[N + i] = info.u[1];
          u[2 * N + i] = info.u[2];
        }
        if (gamma_dot) gamma_dot[i] = info.gamma_dot;
      }
}

double orc_residual(const double* u, const double* u_prev, int64_t N,
                    int64_t delta) {
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < 3 * N; ++i) {
    double d = u[i] - u_prev[i];
    num += d * d;
    den += u[i] * u[i];
  }
  if (den == 0.0) return num == 0.0 ? 0.0 : INFINITY;
  return sqrt(num) / ((double)delta * sqrt(den));
}

double orc_mass(const orc_params* p, const double* A) {
  size_t total = (size_t)19 * p->nx * p->ny * p->nz;
  double s = 0.0;
  for (size_t i = 0; i < total; ++i) s += A[i];
  return s;
}
