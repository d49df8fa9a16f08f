// collide.cuh -- cascaded central-moment collision of one node (Sec. 3),
// written in deviation form d_a = f_a - w_a rho0.
//
// Working with deviations keeps the large rest-state constant out of every
// sum: the raw moments of w rho0 are rho0 * (1, 0, 1/3, 0, 1/9) by order, so
// each raw moment k' of f is that constant plus the same moment D of d, and
// the constants cancel analytically in m^(1), in g^_4..g^_9 and in the
// fourth-order attractor terms of g^_16..g^_18 (expanded around rho/3 below).
// The FP32 and FP16-storage forms therefore lose no precision to a rest value
// of order 1, and the FP64 form computes the same expressions.
#pragma once

#include "d3q19.cuh"
#include "v2.cuh"

namespace clbm {

// Scalar type of the per-lattice constants for a math type R (a pair of FP32
// nodes uses FP32 constants).
template <typename R> struct ScalarOf { using type = R; };
template <> struct ScalarOf<V2> { using type = float; };

// Per-lattice constants of the collision, in the math precision R.
template <typename R>
struct CollideConst {
  R rho0;
  R F[3];        // body force
  R K3;          // 3 K (K = mu_p, consistency coefficient, Eq. 5)
  R logK3;       // log(3 K)
  R n;           // power-law index
  R ehalf;       // (n - 1) / 2
  R ylo, yhi;    // log(3 nu_min), log(3 nu_max): clamp of y = log(1/w - 1/2)
  R nu_min, nu_max;
  int newtonian; // n == 1: omega_nu has a closed form
  int has_force;
  // The rates omega_9..18 enter only as factors of their own relaxation
  // brackets (Eqs. collisionkernelg4..g18; the lower-order g^ terms carry no
  // rate), and omega_9 scales the isotropic part of the strain rate.  They
  // are folded into the brackets' constants: c9 = -omega_9/126,
  // c10..c15 = omega_j/8, c16 = omega_16/12, c17 = omega_17/24,
  // c18 = omega_18/8, cB = 6 omega_9^2 (unit rates give the constants of the
  // printed forms exactly).
  R c9, c10, c11, c12, c13, c14, c15, c16, c17, c18, cB;
};

// Outputs of one collision besides the populations.
template <typename R>
struct NodeOut {
  R rho, ux, uy, uz, gamma_dot;
};

template <typename R> __device__ __forceinline__ R rlog(R x);
template <> __device__ __forceinline__ float rlog<float>(float x) { return __logf(x); }
template <> __device__ __forceinline__ double rlog<double>(double x) { return log(x); }
template <typename R> __device__ __forceinline__ R rexp(R x);
template <> __device__ __forceinline__ float rexp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double rexp<double>(double x) { return exp(x); }
template <typename R> __device__ __forceinline__ R rdiv(R a, R b);
template <> __device__ __forceinline__ float rdiv<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double rdiv<double>(double a, double b) { return a / b; }

// Reciprocal: fast approximate (MUFU based, ~1 ulp) in FP32, IEEE in FP64.
template <typename R> __device__ __forceinline__ R rrcp(R x);
template <> __device__ __forceinline__ float rrcp<float>(float x) { return __fdividef(1.0f, x); }
template <> __device__ __forceinline__ double rrcp<double>(double x) { return 1.0 / x; }

template <> __device__ __forceinline__ V2 rlog<V2>(V2 x) { return V2(__logf(x.v.x), __logf(x.v.y)); }
template <> __device__ __forceinline__ V2 rexp<V2>(V2 x) { return V2(__expf(x.v.x), __expf(x.v.y)); }
template <> __device__ __forceinline__ V2 rdiv<V2>(V2 a, V2 b) {
  return V2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y));
}
template <> __device__ __forceinline__ V2 rrcp<V2>(V2 x) {
  return V2(__fdividef(1.0f, x.v.x), __fdividef(1.0f, x.v.y));
}

template <typename R> __device__ __forceinline__ R tiny();
template <> __device__ __forceinline__ float tiny<float>() { return 1e-36f; }
template <> __device__ __forceinline__ double tiny<double>() { return 1e-300; }
template <> __device__ __forceinline__ V2 tiny<V2>() { return V2(1e-36f); }

// Newton iterations on y = log(1/omega - 1/2) for
//   G(y) = y - log(3K/rho) - (n-1)/2 log(omega(y)^2 A + B) = 0,
// i.e. 1/omega - 1/2 = 3 nu with nu = (K/rho) gamma_dot^(n-1) (Eq. 6,
// Eq. localvarationsrelaxationtimes) and gamma_dot^2 = omega^2 A + B: the
// omega part of the strain rate of Eq. strainratetensor is traceless, so its
// invariant (Eq. shearrateexpression) is quadratic in omega.
// dG/dy = 1 + (n-1) r tau omega with r = omega^2 A / gamma_dot^2 and
// tau omega in (0, 1), so G is increasing with slope between min(n, 1) and
// max(n, 1) and has one root; projecting each iterate onto [ylo, yhi] makes
// the iteration land on the clamp when the root lies beyond it.
template <typename R>
__device__ __forceinline__ R newton_y(R y, R c, R ehalf, R nm1, R A, R B,
                                      R ylo, R yhi, int iters) {
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
    R tau = rexp<R>(y);
    R w = rrcp<R>(tau + R(0.5));
    R wwA = w * w * A;
    R g2 = fmax(wwA + B, tiny<R>());
    R G = y - c - ehalf * rlog<R>(g2);
    R dG = R(1) + nm1 * rdiv<R>(wwA, g2) * (tau * w);
    y = fmin(fmax(y - rdiv<R>(G, dG), ylo), yhi);
  }
  return y;
}

// omega_nu from A and B (see above); writes |gamma_dot| at that omega.
// FP32 (one node or a pair): four Newton iterations from the guess
// omega = 2/3 reach the FP32 rounding level.
template <typename R>
__device__ __forceinline__ R omega_nu(const CollideConst<float>& C, R rho, R rinv, R A, R B,
                                      R* gd) {
  R w;
  if (C.newtonian) {
    R nu = fmin(fmax(R(C.K3 * (1.0f / 3.0f)) * rinv, R(C.nu_min)), R(C.nu_max));
    w = rrcp<R>(R(3.0f) * nu + R(0.5f));
  } else {
    const R c = R(C.logK3) - rlog<R>(rho);
    R y0 = c + R(C.ehalf) * rlog<R>(fmax(A * R(4.0f / 9.0f) + B, tiny<R>()));
    y0 = fmin(fmax(y0, R(C.ylo)), R(C.yhi));
    const R y = newton_y<R>(y0, c, R(C.ehalf), R(C.n - 1.0f), A, B, R(C.ylo), R(C.yhi), 4);
    w = rrcp<R>(rexp<R>(y) + R(0.5f));
  }
  *gd = sqrt(fmax(w * w * A + B, R(0.0f)));
  return w;
}

// FP64: the same four iterations in FP32, then two in FP64, which take the
// FP32 estimate to the FP64 rounding level (quadratic convergence).
__device__ __forceinline__ double omega_nu(const CollideConst<double>& C, double rho,
                                           double rinv, double A, double B, double* gd) {
  double w;
  if (C.newtonian) {
    double nu = fmin(fmax(C.K3 * (1.0 / 3.0) * rinv, C.nu_min), C.nu_max);
    w = 1.0 / (3.0 * nu + 0.5);
  } else {
    float cf = float(C.logK3) - __logf(float(rho));
    float Af = float(A), Bf = float(B);
    float y0 = cf + float(C.ehalf) * __logf(fmaxf(Af * (4.0f / 9.0f) + Bf, 1e-36f));
    y0 = fminf(fmaxf(y0, float(C.ylo)), float(C.yhi));
    float yf = newton_y<float>(y0, cf, float(C.ehalf), float(C.n) - 1.0f, Af, Bf,
                               float(C.ylo), float(C.yhi), 4);
    const double c = C.logK3 - log(rho);
    double y = newton_y<double>(double(yf), c, C.ehalf, C.n - 1.0, A, B, C.ylo, C.yhi, 2);
    w = 1.0 / (exp(y) + 0.5);
  }
  *gd = sqrt(fmax(w * w * A + B, 0.0));
  return w;
}

// Coefficient of g^_j (j >= 4) in f~_q as the grouped back-transform in
// collide() forms it; grouping_is_K() checks it against every entry of K.
constexpr int grouped_coef(int q, int j) {
  const int x = cx(q), y = cy(q), z = cz(q);
  const int axes = (x != 0) + (y != 0) + (z != 0);
  if (axes == 0) return j == 9 ? -30 : j == 16 ? 12 : 0;
  if (axes == 1) {  // Ca = -11 g9 - 4 g16, then the axis's own terms
    int c = j == 9 ? -11 : j == 16 ? -4 : 0;
    if (x) c += (j == 7 || j == 8) ? 1 : j == 17 ? -4 : j == 10 ? -4 * x : 0;
    if (y) c += j == 7 ? -1 : j == 8 ? 1 : j == 17 ? 2 : j == 18 ? -2 : j == 11 ? -4 * y : 0;
    if (z) c += j == 8 ? -2 : (j == 17 || j == 18) ? 2 : j == 12 ? -4 * z : 0;
    return c;
  }
  int c = j == 9 ? 8 : j == 16 ? 1 : 0;  // C9 = 8 g9 + g16
  if (z == 0)  // xy: 2 g8 + g17 + g18 + xy g4; odd x (g10 + g13) + y (g11 - g14)
    c += j == 8 ? 2 : (j == 17 || j == 18) ? 1 : j == 4 ? x * y : (j == 10 || j == 13) ? x
         : j == 11 ? y : j == 14 ? -y : 0;
  else if (y == 0)  // xz: g7 - g8 + g17 - g18 + xz g5; odd x (g10 - g13) + z (g12 + g15)
    c += j == 7 ? 1 : j == 8 ? -1 : j == 17 ? 1 : j == 18 ? -1 : j == 5 ? x * z : j == 10 ? x
         : j == 13 ? -x : (j == 12 || j == 15) ? z : 0;
  else  // yz: -g7 - g8 - 2 g17 + yz g6; odd y (g11 + g14) + z (g12 - g15)
    c += (j == 7 || j == 8) ? -1 : j == 17 ? -2 : j == 6 ? y * z : (j == 11 || j == 14) ? y
         : j == 12 ? z : j == 15 ? -z : 0;
  return c;
}
constexpr bool grouping_is_K() {
  for (int q = 0; q < Q; ++q)
    for (int j = 4; j < Q; ++j)
      if (grouped_coef(q, j) != kb(j, cx(q), cy(q), cz(q))) return false;
  return true;
}
static_assert(grouping_is_K(), "the grouped back-transform must reproduce K");

// Collide one node.  d[19] holds the pre-collision deviations on entry and
// the post-collision deviations f~ - w rho0 on return.
template <typename R, bool FORCE>
__device__ __forceinline__ void collide(const CollideConst<typename ScalarOf<R>::type>& C,
                                        R (&d)[Q], NodeOut<R>& out) {
  using T = typename ScalarOf<R>::type;
  // ---- mass and momentum (Eqs. hydrodynamicfields1/2) -------------------
  // Everything below the populations is formed from the nine +/- pairs: the
  // axis pairs (sum sA, difference tA) and, in each coordinate plane, the
  // two diagonal pairs P (e_i e_j = +1) and M (e_i e_j = -1), whose sums and
  // differences give that plane's moments directly, e.g. in the xy plane
  //   D_xxyy = sP + sM, D_xy = sP - sM, D_xyy = tP + tM, D_xxy = tP - tM.
  static_assert(opp(1) == 2 && opp(3) == 4 && opp(5) == 6 && opp(7) == 10 && opp(9) == 8 &&
                    opp(11) == 14 && opp(13) == 12 && opp(15) == 18 && opp(17) == 16,
                "pair layout");
  static_assert(cx(1) == 1 && cy(3) == 1 && cz(5) == 1 && cx(7) == 1 && cy(7) == 1 &&
                    cx(9) == 1 && cy(9) == -1 && cx(11) == 1 && cz(11) == 1 && cx(13) == 1 &&
                    cz(13) == -1 && cy(15) == 1 && cz(15) == 1 && cy(17) == 1 && cz(17) == -1,
                "pair members");
  R sAx, sAy, sAz, tAx, tAy, tAz;
  R Dxy, Dxz, Dyz, Dxyy, Dxzz, Dxxy, Dyzz, Dxxz, Dyyz, Dxxyy, Dxxzz, Dyyzz;
  auto pair_moments = [&]() {
    sAx = d[1] + d[2];
    tAx = d[1] - d[2];
    sAy = d[3] + d[4];
    tAy = d[3] - d[4];
    sAz = d[5] + d[6];
    tAz = d[5] - d[6];
    {
      const R sP = d[7] + d[10], tP = d[7] - d[10], sM = d[9] + d[8], tM = d[9] - d[8];
      Dxxyy = sP + sM;
      Dxy = sP - sM;
      Dxyy = tP + tM;
      Dxxy = tP - tM;
    }
    {
      const R sP = d[11] + d[14], tP = d[11] - d[14], sM = d[13] + d[12], tM = d[13] - d[12];
      Dxxzz = sP + sM;
      Dxz = sP - sM;
      Dxzz = tP + tM;
      Dxxz = tP - tM;
    }
    {
      const R sP = d[15] + d[18], tP = d[15] - d[18], sM = d[17] + d[16], tM = d[17] - d[16];
      Dyyzz = sP + sM;
      Dyz = sP - sM;
      Dyzz = tP + tM;
      Dyyz = tP - tM;
    }
  };
  pair_moments();
  const R drho = d[0] + (sAx + sAy + sAz) + (Dxxyy + Dxxzz + Dyyzz);
  const R jx = tAx + (Dxyy + Dxzz), jy = tAy + (Dxxy + Dyzz), jz = tAz + (Dxxz + Dyyz);
  const R rho = R(C.rho0) + drho;
  const R rinv = rrcp<R>(rho);
  R ux, uy, uz;
  if (FORCE) {
    // Symmetric split of the body force: the velocity is (j + F/2)/rho and
    // half of the source S_a = w_a [3 e.F + 9 (e.u)(e.F) - 3 u.F] is added
    // before the collision (its moments are 0, F and uF + Fu).
    ux = (jx + R(T(0.5) * C.F[0])) * rinv;
    uy = (jy + R(T(0.5) * C.F[1])) * rinv;
    uz = (jz + R(T(0.5) * C.F[2])) * rinv;
  } else {
    ux = jx * rinv;
    uy = jy * rinv;
    uz = jz * rinv;
  }
  R Sa[FORCE ? Q : 1];
  if (FORCE) {
    const R uF = ux * R(C.F[0]) + uy * R(C.F[1]) + uz * R(C.F[2]);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const T eF = T(cx(q)) * C.F[0] + T(cy(q)) * C.F[1] + T(cz(q)) * C.F[2];
      R eu = R(cx(q)) * ux + R(cy(q)) * uy + R(cz(q)) * uz;
      Sa[q] = R(wt<T>(q)) * (R(T(3) * eF) + R(T(9) * eF) * eu - R(3) * uF);
      d[q] += R(0.5) * Sa[q];
    }
    pair_moments();
  }

  // ---- raw moments of the deviations (Eq. rawmomentdistributionfunction1)
  // k'_ii = rho0/3 + Dii, k'_ij = Dij, third order k' = D, k'_iijj = rho0/9 + D.
  const R Dxx = sAx + (Dxxyy + Dxxzz), Dyy = sAy + (Dxxyy + Dyyzz), Dzz = sAz + (Dxxzz + Dyyzz);

  const R ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  const R r3 = R(C.rho0 * T(1.0 / 3.0));
  const R kxx = r3 + Dxx, kyy = r3 + Dyy, kzz = r3 + Dzz;

  // ---- non-equilibrium second moments m^(1)_4..9 (Sec. 3.2) -------------
  const R m4 = Dxy - rho * ux * uy;
  const R m5 = Dxz - rho * ux * uz;
  const R m6 = Dyz - rho * uy * uz;
  const R m7 = (Dxx - Dyy) - rho * (ux2 - uy2);
  const R m8 = (Dxx - Dzz) - rho * (ux2 - uz2);
  const R m9 = (Dxx + Dyy + Dzz) - drho - rho * (ux2 + uy2 + uz2);

  // gamma_dot^2 = omega^2 A + B from Eq. strainratetensor (bulk rate
  // omega_9): with q = 1/(2 rho), the traceless part gives
  // A = 12 q^2 [m7^2 - m7 m8 + m8^2 + 3 (m4^2 + m5^2 + m6^2)] and the
  // isotropic part B = 6 omega_9^2 q^2 m9^2.
  const R q2 = R(0.25) * rinv * rinv;
  const R A = R(12) * q2 * (m7 * m7 - m7 * m8 + m8 * m8 + R(3) * (m4 * m4 + m5 * m5 + m6 * m6));
  const R B = R(C.cB) * q2 * m9 * m9;   // 6 omega_9^2 q^2 m9^2
  R gd;
  const R w = omega_nu(C, rho, rinv, A, B, &gd);

  // ---- change of moments, Eqs. collisionkernelg4..g18 --------------------
  // omega_4..8 = w (Sec. 3.1); omega_9..18 from the constants above (1 in Sec. 3.1).
  const R g4 = R(-0.25) * w * m4;
  const R g5 = R(-0.25) * w * m5;
  const R g6 = R(-0.25) * w * m6;
  const R g7 = R(-1.0 / 12.0) * w * m7;
  const R g8 = R(-1.0 / 36.0) * w * (R(2) * m8 - m7);
  const R g9 = R(C.c9) * m9;

  // g^_10..15 in +/- pairs: with the row sums
  //   Xy = ux k'yy - k'xyy + 2 uy k'xy - 2 rho ux uy^2 (and Xz, Yx, Yz, Zx, Zy
  //   alike), the bracket of g^_10 is Xy + Xz and that of g^_13 is Xy - Xz
  //   (k'yy - k'zz = Dyy - Dzz), and so on for 11/14 and 12/15.
  const R tux = R(2) * ux, tuy = R(2) * uy, tuz = R(2) * uz;
  const R rho2 = R(2) * rho;
  const R rx2 = rho2 * ux, ry2 = rho2 * uy, rz2 = rho2 * uz;
  const R Xy = ux * kyy - Dxyy + tuy * Dxy - rx2 * uy2;
  const R Xz = ux * kzz - Dxzz + tuz * Dxz - rx2 * uz2;
  const R Yx = uy * kxx - Dxxy + tux * Dxy - ry2 * ux2;
  const R Yz = uy * kzz - Dyzz + tuz * Dyz - ry2 * uz2;
  const R Zx = uz * kxx - Dxxz + tux * Dxz - rz2 * ux2;
  const R Zy = uz * kyy - Dyyz + tuy * Dyz - rz2 * uy2;
  const R a4y = uy * g4, a5z = uz * g5, a4x = ux * g4, a6z = uz * g6, a5x = ux * g5, a6y = uy * g6;
  const R hx = R(0.75) * ux, hy = R(0.75) * uy, hz = R(1.5) * uz;
  const R w9 = R(14) * g9;
  const R g10 = R(C.c10) * (Xy + Xz) + (a4y + a5z) + hx * (w9 - (g7 + g8));
  const R g13 = R(C.c13) * (Xy - Xz) + (a4y - a5z) + hx * (R(3) * g8 - g7);
  const R g11 = R(C.c11) * (Yx + Yz) + (a4x + a6z) + hy * (w9 + (g7 - g8));
  const R g14 = R(C.c14) * (Yz - Yx) + (a6z - a4x) - hy * (g7 + R(3) * g8);
  const R g12 = R(C.c12) * (Zx + Zy) + (a5x + a6y) + hz * (g8 + R(7) * g9);
  const R g15 = R(C.c15) * (Zx - Zy) + (a5x - a6y) + hz * g7;

  // Post-collision diagonal central moments k~ii = rho/3 + a_i (the <K g^|e_i^2>
  // rows of Eq. momentscascadedcollisionterm added to k'_ii - rho u_i^2), and
  // the factorised attractors k~ii k~jj / rho expanded around rho/3, so that
  // the rho0/9 of the raw fourth moments cancels analytically.
  const R third = R(1.0 / 3.0);
  const R ax = Dxx - third * drho - rho * ux2 + R(6) * g7 + R(6) * g8 + R(42) * g9;
  const R ay = Dyy - third * drho - rho * uy2 - R(6) * g7 + R(6) * g8 + R(42) * g9;
  const R az = Dzz - third * drho - rho * uz2 - R(12) * g8 + R(42) * g9;

  // The brackets b16..b18 of g^_16..18 are sums over the axis pairs (xy, xz,
  // yz) of one pair term each, e.g.
  //   Wxy = ax ay / rho - k'xxyy + 2 ux k'xyy + 2 uy k'xxy - ux^2 k'yy
  //         - uy^2 k'xx - 4 ux uy k'xy + 3 rho ux^2 uy^2,
  // with b16 = rho/3 - rho0/3 + 2/3 (ax + ay + az) + Wxy + Wxz + Wyz,
  // b17 = (2 ax - ay - az)/3 + Wxy + Wxz - 2 Wyz and b18 = (ay - az)/3 + Wxy - Wxz.
  const R uxy = ux * uy, uxz = ux * uz, uyz = uy * uz;
  const R rho3 = R(3) * rho;
  const R axr = ax * rinv, ayr = ay * rinv;
  const R Wxy = axr * ay - Dxxyy + tux * Dxyy + tuy * Dxxy - ux2 * kyy - uy2 * kxx -
                R(4) * uxy * Dxy + rho3 * (ux2 * uy2);
  const R Wxz = axr * az - Dxxzz + tux * Dxzz + tuz * Dxxz - ux2 * kzz - uz2 * kxx -
                R(4) * uxz * Dxz + rho3 * (ux2 * uz2);
  const R Wyz = ayr * az - Dyyzz + tuy * Dyzz + tuz * Dyyz - uy2 * kzz - uz2 * kyy -
                R(4) * uyz * Dyz + rho3 * (uy2 * uz2);
  const R b16 = third * drho + R(2.0 / 3.0) * (ax + ay + az) + (Wxy + Wxz + Wyz);
  const R b17 = third * (R(2) * ax - ay - az) + (Wxy + Wxz) - R(2) * Wyz;
  const R b18 = third * (ay - az) + (Wxy - Wxz);
  // shared products: ux uy g4, ux uz g5, uy uz g6 and ux g10, uy g11, uz g12
  const R p4 = ux * a4y, p5 = ux * a5z, p6 = uy * a6z;
  const R v10 = ux * g10, v11 = uy * g11, v12 = uz * g12;
  const R g16 = R(C.c16) * b16 - R(4.0 / 3.0) * (p4 + p5 + p6) +
                R(0.5) * (ux2 - uy2) * g7 + R(0.5) * (ux2 + uy2 - R(2) * uz2) * g8 +
                (R(-7) * (ux2 + uy2 + uz2) - R(8)) * g9 + R(4.0 / 3.0) * (v10 + v11 + v12);
  const R g17 = R(C.c17) * b17 - R(2.0 / 3.0) * (p4 + p5) + R(4.0 / 3.0) * p6 +
                R(0.25) * (ux2 - uy2 - R(3) * uz2 - R(2)) * g7 +
                R(0.25) * (ux2 - R(5) * uy2 + uz2 - R(2)) * g8 +
                R(1.75) * (R(-2) * ux2 + uy2 + uz2) * g9 + R(2.0 / 3.0) * v10 -
                third * (v11 + v12) - uy * g14 + uz * g15;
  const R g18 = R(C.c18) * b18 - R(2) * (p4 - p5) +
                R(0.75) * (ux2 - uy2 + uz2 + R(2.0 / 3.0)) * g7 +
                R(0.75) * (R(-3) * ux2 - uy2 + uz2 - R(2)) * g8 + R(5.25) * (uz2 - uy2) * g9 +
                (v11 - v12) + R(2) * ux * g13 - uy * g14 - uz * g15;

  // ---- back-transform f~ = f + K g^ (+ second half of the source) --------
  // Columns of K grouped by velocity class (Sec. 2, the basis vectors): the
  // rest node; the three axis pairs, which share -11 g9 - 4 g16; and the
  // three coordinate planes of diagonal velocities, which share 8 g9 + g16.
  // In a plane the four velocities differ only in the sign of the plane's
  // product moment g4/g5/g6 (even part) and of two odd sums, e.g. in the xy
  // plane Px = g10 + g13 (odd in x) and Py = g11 - g14 (odd in y).
  static_assert(cx(7) == 1 && cy(7) == 1 && cx(8) == -1 && cy(8) == 1 && cx(9) == 1 &&
                    cy(9) == -1 && cx(10) == -1 && cy(10) == -1,
                "xy-plane velocity order");
  static_assert(cx(11) == 1 && cz(11) == 1 && cx(12) == -1 && cz(12) == 1 && cx(13) == 1 &&
                    cz(13) == -1 && cx(14) == -1 && cz(14) == -1,
                "xz-plane velocity order");
  static_assert(cy(15) == 1 && cz(15) == 1 && cy(16) == -1 && cz(16) == 1 && cy(17) == 1 &&
                    cz(17) == -1 && cy(18) == -1 && cz(18) == -1,
                "yz-plane velocity order");
  static_assert(cx(1) == 1 && cx(2) == -1 && cy(3) == 1 && cy(4) == -1 && cz(5) == 1 &&
                    cz(6) == -1,
                "axis velocity order");
  static_assert(kb(9, 0, 0, 0) == -30 && kb(16, 0, 0, 0) == 12 && kb(9, 1, 0, 0) == -11 &&
                    kb(16, 1, 0, 0) == -4 && kb(9, 1, 1, 0) == 8 && kb(16, 1, 1, 0) == 1,
                "K entries of the grouping");
  d[0] += R(-30) * g9 + R(12) * g16;
  const R Ca = R(-11) * g9 - R(4) * g16;
  {
    const R Ex = Ca + (g7 + g8) - R(4) * g17;
    d[1] = (d[1] + Ex) - R(4) * g10;
    d[2] = (d[2] + Ex) + R(4) * g10;
    const R Ey = Ca + (g8 - g7) + R(2) * (g17 - g18);
    d[3] = (d[3] + Ey) - R(4) * g11;
    d[4] = (d[4] + Ey) + R(4) * g11;
    const R Ez = Ca - R(2) * g8 + R(2) * (g17 + g18);
    d[5] = (d[5] + Ez) - R(4) * g12;
    d[6] = (d[6] + Ez) + R(4) * g12;
  }
  const R C9 = R(8) * g9 + g16;
  {
    const R E = C9 + R(2) * g8 + (g17 + g18);
    const R Ep = E + g4, Em = E - g4;
    const R Px = g10 + g13, Py = g11 - g14;
    const R S = Px + Py, D = Py - Px;
    d[7] += Ep + S;
    d[10] += Ep - S;
    d[8] += Em + D;
    d[9] += Em - D;
  }
  {
    const R E = C9 + (g7 - g8) + (g17 - g18);
    const R Ep = E + g5, Em = E - g5;
    const R Qx = g10 - g13, Qz = g12 + g15;
    const R S = Qx + Qz, D = Qz - Qx;
    d[11] += Ep + S;
    d[14] += Ep - S;
    d[12] += Em + D;
    d[13] += Em - D;
  }
  {
    const R E = C9 - (g7 + g8) - R(2) * g17;
    const R Ep = E + g6, Em = E - g6;
    const R Ry = g11 + g14, Rz = g12 - g15;
    const R S = Ry + Rz, D = Rz - Ry;
    d[15] += Ep + S;
    d[18] += Ep - S;
    d[16] += Em + D;
    d[17] += Em - D;
  }
  if (FORCE) {
#pragma unroll
    for (int q = 0; q < Q; ++q) d[q] += R(0.5) * Sa[q];
  }
  out.rho = rho;
  out.ux = ux;
  out.uy = uy;
  out.uz = uz;
  out.gamma_dot = gd;
}

}  // namespace clbm
