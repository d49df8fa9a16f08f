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
  R rhoS;        // lam rho0 and lam F: rest density and force of deviations
  R FS[3];       //   carried scaled by lam (FP16 storage: lam = 1024; else 1)
  R K3;          // 3 K (K = mu_p, consistency coefficient, Eq. 5)
  R logK3;       // log(3 K)
  R log2K3;      // log2(3 K)
  R n;           // power-law index
  R rn;          // 1 / n
  R ehalf;       // (n - 1) / 2
  R ylo, yhi;    // log(3 nu_min), log(3 nu_max): clamp of y = log(1/w - 1/2)
  R ylo2, yhi2;  // the same clamp in base 2
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

// Base-2 logarithm and power of two on the special-function unit (PTX
// lg2.approx / ex2.approx, about 22 correct bits): the FP32 solve for
// omega_nu works in base 2, so no conversion factor is spent on either.
__device__ __forceinline__ float lg2f(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2f(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <typename R> __device__ __forceinline__ R rlg2(R x);
template <> __device__ __forceinline__ float rlg2<float>(float x) { return lg2f(x); }
template <typename R> __device__ __forceinline__ R rex2(R x);
template <> __device__ __forceinline__ float rex2<float>(float x) { return ex2f(x); }
template <typename R> __device__ __forceinline__ R rdiv(R a, R b);
template <> __device__ __forceinline__ float rdiv<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double rdiv<double>(double a, double b) { return a / b; }

// Reciprocal: fast approximate (MUFU based, ~1 ulp) in FP32, IEEE in FP64.
template <typename R> __device__ __forceinline__ R rrcp(R x);
template <> __device__ __forceinline__ float rrcp<float>(float x) { return __fdividef(1.0f, x); }
template <> __device__ __forceinline__ double rrcp<double>(double x) { return 1.0 / x; }

template <> __device__ __forceinline__ V2 rlg2<V2>(V2 x) { return V2(lg2f(x.v.x), lg2f(x.v.y)); }
template <> __device__ __forceinline__ V2 rex2<V2>(V2 x) { return V2(ex2f(x.v.x), ex2f(x.v.y)); }
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

// Starting point of the solve below.  Without the bulk part B, the unknown
// z = 1/omega - 1/2 = 3 nu solves z (z + 1/2)^(n-1) = P with
// log2 P = log2(3K/rho) + (n-1)/2 log2 A, whose two asymptotes are
// z = P^(1/n) (z >> 1/2) and z = 2^(n-1) P (z << 1/2); they meet at z = 1/2,
// where log2 P = -n.  The guess takes the asymptote of its side (with A + B
// for A), which three Newton steps then take to the FP32 rounding level
// over the workloads' range of n, K and shear rate.
__device__ __forceinline__ float regime_guess(float lp, float n, float rn) {
  return lp > -n ? lp * rn : lp + (n - 1.0f);
}
__device__ __forceinline__ V2 regime_guess(V2 lp, float n, float rn) {
  return V2(regime_guess(lp.v.x, n, rn), regime_guess(lp.v.y, n, rn));
}

// Newton iterations on y = log2(1/omega - 1/2) for
//   G(y) = y - log2(3K/rho) - (n-1)/2 log2(omega(y)^2 A + B) = 0,
// i.e. 1/omega - 1/2 = 3 nu with nu = (K/rho) gamma_dot^(n-1) (Eq. 6,
// Eq. localvarationsrelaxationtimes) and gamma_dot^2 = omega^2 A + B: the
// omega part of the strain rate of Eq. strainratetensor is traceless, so its
// invariant (Eq. shearrateexpression) is quadratic in omega.
// dG/dy = 1 + (n-1) r tau omega with r = omega^2 A / gamma_dot^2 and
// tau omega in (0, 1) (the base of the logarithm cancels), so G is
// increasing with slope between min(n, 1) and max(n, 1) and has one root;
// projecting each iterate onto [ylo, yhi] makes the iteration land on the
// clamp when the root lies beyond it.
template <typename R>
__device__ __forceinline__ R newton_y2(R y, R c, R ehalf, R nm1, R A, R B, R ylo, R yhi,
                                       int iters) {
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
    R tau = rex2<R>(y);
    R w = rrcp<R>(tau + R(0.5));
    R wwA = w * w * A;
    R g2 = fmax(wwA + B, tiny<R>());
    R G = (y - c) - ehalf * rlg2<R>(g2);
    R dG = R(1) + nm1 * rdiv<R>(wwA, g2) * (tau * w);
    y = fmin(fmax(y - rdiv<R>(G, dG), ylo), yhi);
  }
  return y;
}

// omega_nu from A and B (see above); writes |gamma_dot| at that omega.
// FP32 (one node or a pair): the regime guess and three Newton steps reach
// the FP32 rounding level.
template <typename R>
__device__ __forceinline__ R omega_nu(const CollideConst<float>& C, R rho, R rinv, R A, R B,
                                      R* gd) {
  R w;
  if (C.newtonian) {
    R nu = fmin(fmax(R(C.K3 * (1.0f / 3.0f)) * rinv, R(C.nu_min)), R(C.nu_max));
    w = rrcp<R>(R(3.0f) * nu + R(0.5f));
  } else {
    const R c = R(C.log2K3) - rlg2<R>(rho);
    const R lp = c + R(C.ehalf) * rlg2<R>(fmax(A + B, tiny<R>()));
    R y0 = regime_guess(lp, C.n, C.rn);
    y0 = fmin(fmax(y0, R(C.ylo2)), R(C.yhi2));
    const R y = newton_y2<R>(y0, c, R(C.ehalf), R(C.n - 1.0f), A, B, R(C.ylo2), R(C.yhi2), 3);
    w = rrcp<R>(rex2<R>(y) + R(0.5f));
  }
  *gd = sqrt(fmax(w * w * A + B, R(0.0f)));
  return w;
}

// FP64: the FP32 solve, then one Halley step in FP64 on the natural-log
// y = log(1/omega - 1/2).  Halley's step converges cubically, so from the
// FP32 estimate (relative error ~1e-5) it lands at the FP64 rounding level.
// With s = tau omega and r as above,
//   G'  = 1 + (n-1) r s,
//   G'' = (n-1) [s omega r / 2 - 2 r (1 - r) s^2]
// (from d(tau omega)/dy = tau omega^2 / 2 and dr/dy = -2 r (1 - r) s), and
// the step is dy = -2 G G' / (2 G'^2 - G G'').  tau = exp(y) is then carried
// to the new y by exp(dy) = 1 + dy + dy^2/2 + dy^3/6 (|dy| ~ 1e-5, so the
// omitted terms lie below 1e-20), or set to 3 nu exactly on a clamp.
__device__ __forceinline__ double omega_nu(const CollideConst<double>& C, double rho,
                                           double rinv, double A, double B, double* gd) {
  double w;
  if (C.newtonian) {
    double nu = fmin(fmax(C.K3 * (1.0 / 3.0) * rinv, C.nu_min), C.nu_max);
    w = 1.0 / (3.0 * nu + 0.5);
  } else {
    const float rf = float(rho), Af = float(A), Bf = float(B);
    const float cf = float(C.log2K3) - lg2f(rf);
    const float lp = cf + float(C.ehalf) * lg2f(fmaxf(Af + Bf, 1e-36f));
    float yf = regime_guess(lp, float(C.n), float(C.rn));
    yf = fminf(fmaxf(yf, float(C.ylo2)), float(C.yhi2));
    yf = newton_y2<float>(yf, cf, float(C.ehalf), float(C.n) - 1.0f, Af, Bf, float(C.ylo2),
                          float(C.yhi2), 3);
    const double y0 = fmin(fmax(double(yf) * 0.69314718055994530942, C.ylo), C.yhi);
    const double tau = exp(y0);
    const double w0 = 1.0 / (tau + 0.5);
    const double wwA = w0 * w0 * A;
    const double g2 = fmax(wwA + B, 1e-300);
    const double nm1 = C.n - 1.0;
    const double G = (y0 - (C.logK3 - log(rho))) - C.ehalf * log(g2);
    const double r = wwA / g2;
    const double sw = tau * w0;
    const double G1 = 1.0 + nm1 * r * sw;
    const double G2 = nm1 * (sw * (0.5 * w0) * r - 2.0 * r * (1.0 - r) * sw * sw);
    const double dy = -2.0 * G * G1 / (2.0 * G1 * G1 - G * G2);
    const double y1 = y0 + dy;
    double tau1;
    if (y1 <= C.ylo) tau1 = 3.0 * C.nu_min;
    else if (y1 >= C.yhi) tau1 = 3.0 * C.nu_max;
    else tau1 = tau + tau * (dy * (1.0 + dy * (0.5 + dy * (1.0 / 6.0))));
    w = 1.0 / (tau1 + 0.5);
  }
  *gd = sqrt(fmax(w * w * A + B, 0.0));
  return w;
}

// ---- pair space -------------------------------------------------------------
// The collision works on the nine +/- velocity pairs instead of the 19
// populations.  An axis pair (e, -e) is held as its sum s and difference t;
// in each coordinate plane the two diagonal pairs P (e_i e_j = +1) and
// M (e_i e_j = -1) are held as four moments of the plane, e.g. in the xy
// plane, with sP = d7 + d10, tP = d7 - d10, sM = d9 + d8, tM = d9 - d8,
//   Dxxyy = sP + sM, Dxy = sP - sM, Dxyy = tP + tM, Dxxy = tP - tM.
// These 19 values are the rest population, the axis sums and differences and
// the plane moments: the raw moments of Eq. rawmomentdistributionfunction1
// are sums of them, and the populations are recovered from them exactly.
// The post-collision populations are rebuilt from the pair values and g^
// at the end, so the 19 pre-collision populations need not stay live
// through the collision.
template <typename R>
struct Pairs {
  R d0;
  R sAx, tAx, sAy, tAy, sAz, tAz;
  R Dxxyy, Dxy, Dxyy, Dxxy;  // xy plane: velocities 7, 10 (P) and 9, 8 (M)
  R Dxxzz, Dxz, Dxzz, Dxxz;  // xz plane: 11, 14 (P) and 13, 12 (M)
  R Dyyzz, Dyz, Dyzz, Dyyz;  // yz plane: 15, 18 (P) and 17, 16 (M)
};

// Pair values of 19 populations in the paper's order (Eq. velocityd3qq19).
template <typename R>
__host__ __device__ constexpr Pairs<R> to_pairs(const R (&d)[Q]) {
  Pairs<R> p{};
  p.d0 = d[0];
  p.sAx = d[1] + d[2];
  p.tAx = d[1] - d[2];
  p.sAy = d[3] + d[4];
  p.tAy = d[3] - d[4];
  p.sAz = d[5] + d[6];
  p.tAz = d[5] - d[6];
  {
    const R sP = d[7] + d[10], tP = d[7] - d[10], sM = d[9] + d[8], tM = d[9] - d[8];
    p.Dxxyy = sP + sM;
    p.Dxy = sP - sM;
    p.Dxyy = tP + tM;
    p.Dxxy = tP - tM;
  }
  {
    const R sP = d[11] + d[14], tP = d[11] - d[14], sM = d[13] + d[12], tM = d[13] - d[12];
    p.Dxxzz = sP + sM;
    p.Dxz = sP - sM;
    p.Dxzz = tP + tM;
    p.Dxxz = tP - tM;
  }
  {
    const R sP = d[15] + d[18], tP = d[15] - d[18], sM = d[17] + d[16], tM = d[17] - d[16];
    p.Dyyzz = sP + sM;
    p.Dyz = sP - sM;
    p.Dyzz = tP + tM;
    p.Dyyz = tP - tM;
  }
  return p;
}

// Four populations of a coordinate plane from its four moments plus the
// plane's part of K g^ (Eq. cascadedcollision1): E (shared by the plane),
// Ex (the product moment g4/g5/g6) and the two odd sums Oa, Ob.  With
// q1 = Dii jj/4 + E, q2 = Dij/4 + Ex, q3 = Dijj/4 + Oa, q4 = Diij/4 + Ob the
// populations are P+ = q1+q2+q3+q4, P- = q1+q2-q3-q4, M+ = q1-q2+q3-q4,
// M- = q1-q2-q3+q4 (P+, P-: the pair with e_i e_j = +1, positive and
// negative e_i; M+, M-: the other pair, positive and negative e_i).
template <typename R>
__host__ __device__ constexpr void plane_out(R Diijj, R Dij, R Dijj, R Diij, R E, R Ex, R Oa,
                                             R Ob, R& Pp, R& Pm, R& Mp, R& Mm) {
  const R q1 = R(0.25) * Diijj + E, q2 = R(0.25) * Dij + Ex;
  const R q3 = R(0.25) * Dijj + Oa, q4 = R(0.25) * Diij + Ob;
  const R a = q1 + q2, b = q1 - q2, c = q3 + q4, e = q3 - q4;
  Pp = a + c;
  Pm = a - c;
  Mp = b + e;
  Mm = b - e;
}

// Populations f~ = f + K g^ from the pair values of f and g^_4..g^_18
// (entries 0..3 of g unused): the columns of K grouped by velocity class
// (Sec. 2, the basis vectors).  The rest node; the three axis pairs, which
// share -11 g9 - 4 g16; and the three coordinate planes of diagonal
// velocities, which share 8 g9 + g16.  In a plane the four velocities differ
// only in the sign of the plane's product moment g4/g5/g6 and of two odd
// sums, e.g. in the xy plane g10 + g13 (odd in x) and g11 - g14 (odd in y).
template <typename R>
__host__ __device__ constexpr void from_pairs(const Pairs<R>& p, const R (&g)[Q], R (&d)[Q]) {
  d[0] = p.d0 + (R(-30) * g[9] + R(12) * g[16]);
  const R Ca = R(-11) * g[9] - R(4) * g[16];
  {
    const R hs = R(0.5) * p.sAx + (Ca + (g[7] + g[8]) - R(4) * g[17]);
    const R ht = R(0.5) * p.tAx - R(4) * g[10];
    d[1] = hs + ht;
    d[2] = hs - ht;
  }
  {
    const R hs = R(0.5) * p.sAy + (Ca + (g[8] - g[7]) + R(2) * (g[17] - g[18]));
    const R ht = R(0.5) * p.tAy - R(4) * g[11];
    d[3] = hs + ht;
    d[4] = hs - ht;
  }
  {
    const R hs = R(0.5) * p.sAz + (Ca - R(2) * g[8] + R(2) * (g[17] + g[18]));
    const R ht = R(0.5) * p.tAz - R(4) * g[12];
    d[5] = hs + ht;
    d[6] = hs - ht;
  }
  const R C9 = R(8) * g[9] + g[16];
  plane_out(p.Dxxyy, p.Dxy, p.Dxyy, p.Dxxy, C9 + R(2) * g[8] + (g[17] + g[18]), g[4],
            g[10] + g[13], g[11] - g[14], d[7], d[10], d[9], d[8]);
  plane_out(p.Dxxzz, p.Dxz, p.Dxzz, p.Dxxz, C9 + (g[7] - g[8]) + (g[17] - g[18]), g[5],
            g[10] - g[13], g[12] + g[15], d[11], d[14], d[13], d[12]);
  plane_out(p.Dyyzz, p.Dyz, p.Dyzz, p.Dyyz, C9 - (g[7] + g[8]) - R(2) * g[17], g[6],
            g[11] + g[14], g[12] - g[15], d[15], d[18], d[17], d[16]);
}

// Compile-time checks of the pair space against the basis definitions:
// the populations come back unchanged from their pair values, and a unit
// g^_j adds column j of K to them.
constexpr bool pairs_roundtrip() {
  for (int q = 0; q < Q; ++q) {
    double d[Q] = {}, out[Q] = {}, g[Q] = {};
    d[q] = 1.0;
    from_pairs(to_pairs(d), g, out);
    for (int k = 0; k < Q; ++k)
      if (out[k] != (k == q ? 1.0 : 0.0)) return false;
  }
  return true;
}
constexpr bool pairs_add_K() {
  for (int j = 4; j < Q; ++j) {
    double d[Q] = {}, out[Q] = {}, g[Q] = {};
    g[j] = 1.0;
    from_pairs(to_pairs(d), g, out);
    for (int q = 0; q < Q; ++q)
      if (out[q] != double(kb(j, cx(q), cy(q), cz(q)))) return false;
  }
  return true;
}
static_assert(pairs_roundtrip(), "pair values must give back the populations");
static_assert(pairs_add_K(), "the pair-space back-transform must add the columns of K");

// Half the pair values of the source S_a = w_a [3 e.F + 9 (e.u)(e.F) - 3 u.F]
// of the symmetric force split (reading of the deferred forcing: its moments
// are 0, F and uF + Fu).  Summed over each pair and plane with the D3Q19
// weights (1/3, 1/18, 1/36) they are, with a_i = u_i F_i and t = u.F / 3:
//   rest -u.F; axis i: s = a_i - t, d = F_i / 3;
//   plane ij: Diijj = a_i + a_j - t, Dij = u_i F_j + u_j F_i,
//             Dijj = F_i / 3, Diij = F_j / 3.
template <typename R, typename T>
__device__ __forceinline__ void add_half_source(Pairs<R>& p, R ux, R uy, R uz,
                                                const T (&F)[3]) {
  const R ax = ux * R(F[0]), ay = uy * R(F[1]), az = uz * R(F[2]);
  const R uF = ax + ay + az;
  const R ht = R(1.0 / 6.0) * uF;  // t / 2
  const R f6x = R(T(F[0]) * T(1.0 / 6.0)), f6y = R(T(F[1]) * T(1.0 / 6.0)),
          f6z = R(T(F[2]) * T(1.0 / 6.0));
  p.d0 -= R(0.5) * uF;
  p.sAx += R(0.5) * ax - ht;
  p.sAy += R(0.5) * ay - ht;
  p.sAz += R(0.5) * az - ht;
  p.tAx += f6x;
  p.tAy += f6y;
  p.tAz += f6z;
  p.Dxxyy += R(0.5) * (ax + ay) - ht;
  p.Dxxzz += R(0.5) * (ax + az) - ht;
  p.Dyyzz += R(0.5) * (ay + az) - ht;
  p.Dxy += R(0.5) * (ux * R(F[1]) + uy * R(F[0]));
  p.Dxz += R(0.5) * (ux * R(F[2]) + uz * R(F[0]));
  p.Dyz += R(0.5) * (uy * R(F[2]) + uz * R(F[1]));
  p.Dxyy += f6x;
  p.Dxzz += f6x;
  p.Dxxy += f6y;
  p.Dyzz += f6y;
  p.Dxxz += f6z;
  p.Dyyz += f6z;
}

// Post-collision populations f~ = f + K g^ (+ S, the whole body-force source
// of the symmetric split: half before and half after the collision), added
// to the pre-collision deviations as one correction per population, so that
// each population is rounded once at its own scale.  The correction is
// grouped by velocity class as in from_pairs.  With FP32 populations this
// matters: rebuilding them from pair values rounds sums of populations each
// step, and near a steady state those roundings repeat and accumulate.
// For a +/- pair (e, -e) the source is S_+- = w [9 (e.u)(e.F) - 3 u.F] +- 3 w e.F.
template <typename R, bool FORCE, typename T>
__host__ __device__ constexpr void add_K_g(R (&d)[Q], const R (&g)[Q], R ux, R uy, R uz,
                                           const T (&F)[3]) {
  R se = R(0), so = R(0), uF = R(0);
  if (FORCE) uF = ux * R(F[0]) + uy * R(F[1]) + uz * R(F[2]);
  d[0] += (R(-30) * g[9] + R(12) * g[16]) - (FORCE ? uF : R(0));
  const R Ca = R(-11) * g[9] - R(4) * g[16];
  const R u6 = R(1.0 / 6.0) * uF;  // 3 w u.F for the axis weight 1/18
  {
    const R E = Ca + (g[7] + g[8]) - R(4) * g[17];
    const R O = R(4) * g[10];
    if (FORCE) { se = R(0.5) * ux * R(F[0]) - u6; so = R(T(F[0]) * T(1.0 / 6.0)); }
    d[1] += (E - O) + (se + so);
    d[2] += (E + O) + (se - so);
  }
  {
    const R E = Ca + (g[8] - g[7]) + R(2) * (g[17] - g[18]);
    const R O = R(4) * g[11];
    if (FORCE) { se = R(0.5) * uy * R(F[1]) - u6; so = R(T(F[1]) * T(1.0 / 6.0)); }
    d[3] += (E - O) + (se + so);
    d[4] += (E + O) + (se - so);
  }
  {
    const R E = Ca - R(2) * g[8] + R(2) * (g[17] + g[18]);
    const R O = R(4) * g[12];
    if (FORCE) { se = R(0.5) * uz * R(F[2]) - u6; so = R(T(F[2]) * T(1.0 / 6.0)); }
    d[5] += (E - O) + (se + so);
    d[6] += (E + O) + (se - so);
  }
  const R C9 = R(8) * g[9] + g[16];
  const R u12 = R(1.0 / 12.0) * uF;  // 3 w u.F for the diagonal weight 1/36
  // One plane: pair P = (Pp, Pm) with e_i e_j = +1 and M = (Mp, Mm) with
  // e_i e_j = -1 (first member positive along the plane's first axis); its
  // part of K g^ is E +- Ex (product moment) plus the odd sums (Oa, Ob), and
  // ea/eb, ua/ub are e.F and e.u of the P and M pairs' positive members.
  auto plane = [&](R& Pp, R& Pm, R& Mp, R& Mm, R E, R Ex, R Oa, R Ob, R fP, R fM, R vP,
                   R vM) {
    const R Ep = E + Ex, Em = E - Ex;
    const R Sg = Oa + Ob, Dg = Ob - Oa;
    R sP = R(0), oP = R(0), sM = R(0), oM = R(0);
    if (FORCE) {
      sP = R(0.25) * vP * fP - u12;
      oP = R(1.0 / 12.0) * fP;
      sM = R(0.25) * vM * fM - u12;
      oM = R(1.0 / 12.0) * fM;
    }
    Pp += (Ep + Sg) + (sP + oP);
    Pm += (Ep - Sg) + (sP - oP);
    Mp += (Em - Dg) + (sM + oM);
    Mm += (Em + Dg) + (sM - oM);
  };
  const R Fx = FORCE ? R(F[0]) : R(0), Fy = FORCE ? R(F[1]) : R(0), Fz = FORCE ? R(F[2]) : R(0);
  plane(d[7], d[10], d[9], d[8], C9 + R(2) * g[8] + (g[17] + g[18]), g[4], g[10] + g[13],
        g[11] - g[14], Fx + Fy, Fx - Fy, ux + uy, ux - uy);
  plane(d[11], d[14], d[13], d[12], C9 + (g[7] - g[8]) + (g[17] - g[18]), g[5], g[10] - g[13],
        g[12] + g[15], Fx + Fz, Fx - Fz, ux + uz, ux - uz);
  plane(d[15], d[18], d[17], d[16], C9 - (g[7] + g[8]) - R(2) * g[17], g[6], g[11] + g[14],
        g[12] - g[15], Fy + Fz, Fy - Fz, uy + uz, uy - uz);
}

// Compile-time checks of the additive back-transform: a unit g^_j adds
// column j of K, and the body-force correction equals the source
// w_a [3 e.F + 9 (e.u)(e.F) - 3 u.F] of every direction.
constexpr bool add_K_g_is_K() {
  for (int j = 4; j < Q; ++j) {
    double d[Q] = {}, g[Q] = {};
    const double F[3] = {0.0, 0.0, 0.0};
    g[j] = 1.0;
    add_K_g<double, false>(d, g, 0.0, 0.0, 0.0, F);
    for (int q = 0; q < Q; ++q)
      if (d[q] != double(kb(j, cx(q), cy(q), cz(q)))) return false;
  }
  return true;
}
constexpr bool add_K_g_source() {
  const double F[3] = {0.375, -0.625, 0.8125};
  const double u[3] = {0.25, 0.5, -0.125};
  double d[Q] = {}, g[Q] = {};
  add_K_g<double, true>(d, g, u[0], u[1], u[2], F);
  for (int q = 0; q < Q; ++q) {
    const double eF = cx(q) * F[0] + cy(q) * F[1] + cz(q) * F[2];
    const double eu = cx(q) * u[0] + cy(q) * u[1] + cz(q) * u[2];
    const double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const double S = wt<double>(q) * (3.0 * eF + 9.0 * eu * eF - 3.0 * uF);
    const double diff = d[q] - S;
    if (diff > 1e-15 || diff < -1e-15) return false;
  }
  return true;
}
static_assert(add_K_g_is_K(), "the additive back-transform must add the columns of K");
static_assert(add_K_g_source(), "the additive back-transform must add the body-force source");

// gamma_dot^2 = omega^2 A + B from Eq. strainratetensor (bulk rate omega_9)
// and Eq. shearrateexpression, for the non-equilibrium moments m^(1)_4..9
// (Sec. 3.2): with q = 1/(2 rho), the traceless part gives
// A = 12 q^2 [m7^2 - m7 m8 + m8^2 + 3 (m4^2 + m5^2 + m6^2)] and the
// isotropic part B = 6 omega_9^2 q^2 m9^2.
template <typename R, typename T>
__device__ __forceinline__ void strain_AB(const CollideConst<T>& C, R rinv, R m4, R m5, R m6,
                                          R m7, R m8, R m9, R& A, R& B) {
  const R q2 = R(0.25) * rinv * rinv;
  A = R(12) * q2 * (m7 * m7 - m7 * m8 + m8 * m8 + R(3) * (m4 * m4 + m5 * m5 + m6 * m6));
  B = R(C.cB) * q2 * m9 * m9;  // 6 omega_9^2 q^2 m9^2
}

// Collide one node.  d[19] holds the pre-collision deviations on entry and
// the post-collision deviations f~ - w rho0 on return.
// PAIR_OUT selects how the populations are written back: rebuilt from the
// pair values (fewer registers: the 19 inputs are dead after the pair values
// are formed), which is exact when the inputs are FP16 values decoded to FP32
// (sums of a few of them need no rounding), or as one correction added to
// each input population (add_K_g), which keeps FP32 populations to a single
// rounding per step.
//
// LOG2LAM: the deviations are carried scaled by lam = 2^LOG2LAM (the FP16
// storage scale), and C holds lam rho0, lam F, lam 3K and log(lam 3K).  All
// moments and g^ then scale with lam, rho becomes lam rho and 1/rho
// 1/(lam rho): every term is either linear in the deviations or a product
// whose factors of lam cancel (the attractors a_i a_j / rho, the strain rate
// of m^(1)/rho, the omega solve of 3K/rho), so the scaled populations come
// out exactly as lam times the unscaled ones up to rounding, and only rho
// is unscaled for the output.
template <typename R, bool FORCE, bool PAIR_OUT = false, int LOG2LAM = 0>
__device__ __forceinline__ void collide(const CollideConst<typename ScalarOf<R>::type>& C,
                                        R (&d)[Q], NodeOut<R>& out) {
  using T = typename ScalarOf<R>::type;
  // ---- mass and momentum (Eqs. hydrodynamicfields1/2) -------------------
  static_assert(cx(1) == 1 && cy(3) == 1 && cz(5) == 1 && cx(7) == 1 && cy(7) == 1 &&
                    cx(9) == 1 && cy(9) == -1 && cx(11) == 1 && cz(11) == 1 && cx(13) == 1 &&
                    cz(13) == -1 && cy(15) == 1 && cz(15) == 1 && cy(17) == 1 && cz(17) == -1,
                "pair members");
  Pairs<R> p = to_pairs(d);
  const R drho = p.d0 + (p.sAx + p.sAy + p.sAz) + (p.Dxxyy + p.Dxxzz + p.Dyyzz);
  const R jx = p.tAx + (p.Dxyy + p.Dxzz), jy = p.tAy + (p.Dxxy + p.Dyzz),
          jz = p.tAz + (p.Dxxz + p.Dyyz);
  const R rho = R(C.rhoS) + drho;
  const R rinv = rrcp<R>(rho);
  R ux, uy, uz;
  if (FORCE) {
    // Symmetric split of the body force: the velocity is (j + F/2)/rho and
    // half of the source is added before the collision, half after.
    ux = (jx + R(T(0.5) * C.FS[0])) * rinv;
    uy = (jy + R(T(0.5) * C.FS[1])) * rinv;
    uz = (jz + R(T(0.5) * C.FS[2])) * rinv;
    add_half_source(p, ux, uy, uz, C.FS);
  } else {
    ux = jx * rinv;
    uy = jy * rinv;
    uz = jz * rinv;
  }

  // ---- raw moments of the deviations (Eq. rawmomentdistributionfunction1)
  // k'_ii = rho0/3 + Dii, k'_ij = Dij, third order k' = D, k'_iijj = rho0/9 + D.
  const R Dxy = p.Dxy, Dxz = p.Dxz, Dyz = p.Dyz;
  const R Dxyy = p.Dxyy, Dxzz = p.Dxzz, Dxxy = p.Dxxy, Dyzz = p.Dyzz, Dxxz = p.Dxxz,
          Dyyz = p.Dyyz;
  const R Dxxyy = p.Dxxyy, Dxxzz = p.Dxxzz, Dyyzz = p.Dyyzz;
  const R Dxx = p.sAx + (Dxxyy + Dxxzz), Dyy = p.sAy + (Dxxyy + Dyyzz),
          Dzz = p.sAz + (Dxxzz + Dyyzz);

  const R ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  const R r3 = R(C.rhoS * T(1.0 / 3.0));
  const R kxx = r3 + Dxx, kyy = r3 + Dyy, kzz = r3 + Dzz;

  // ---- non-equilibrium second moments m^(1)_4..9 (Sec. 3.2) -------------
  const R m4 = Dxy - rho * ux * uy;
  const R m5 = Dxz - rho * ux * uz;
  const R m6 = Dyz - rho * uy * uz;
  const R m7 = (Dxx - Dyy) - rho * (ux2 - uy2);
  const R m8 = (Dxx - Dzz) - rho * (ux2 - uz2);
  const R m9 = (Dxx + Dyy + Dzz) - drho - rho * (ux2 + uy2 + uz2);

  R A, B;
  strain_AB(C, rinv, m4, m5, m6, m7, m8, m9, A, B);
  R gd;
  const R w = omega_nu(C, rho, rinv, A, B, &gd);

  // ---- change of moments, Eqs. collisionkernelg4..g18 --------------------
  // omega_4..8 = w (Sec. 3.1); omega_9..18 from the constants above (1 in Sec. 3.1).
  R g[Q];
  g[4] = R(-0.25) * w * m4;
  g[5] = R(-0.25) * w * m5;
  g[6] = R(-0.25) * w * m6;
  g[7] = R(-1.0 / 12.0) * w * m7;
  g[8] = R(-1.0 / 36.0) * w * (R(2) * m8 - m7);
  g[9] = R(C.c9) * m9;
  const R g4 = g[4], g5 = g[5], g6 = g[6], g7 = g[7], g8 = g[8], g9 = g[9];

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
  g[10] = R(C.c10) * (Xy + Xz) + (a4y + a5z) + hx * (w9 - (g7 + g8));
  g[13] = R(C.c13) * (Xy - Xz) + (a4y - a5z) + hx * (R(3) * g8 - g7);
  g[11] = R(C.c11) * (Yx + Yz) + (a4x + a6z) + hy * (w9 + (g7 - g8));
  g[14] = R(C.c14) * (Yz - Yx) + (a6z - a4x) - hy * (g7 + R(3) * g8);
  g[12] = R(C.c12) * (Zx + Zy) + (a5x + a6y) + hz * (g8 + R(7) * g9);
  g[15] = R(C.c15) * (Zx - Zy) + (a5x - a6y) + hz * g7;
  const R g10 = g[10], g11 = g[11], g12 = g[12], g13 = g[13], g14 = g[14], g15 = g[15];

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
  g[16] = R(C.c16) * b16 - R(4.0 / 3.0) * (p4 + p5 + p6) +
          R(0.5) * (ux2 - uy2) * g7 + R(0.5) * (ux2 + uy2 - R(2) * uz2) * g8 +
          (R(-7) * (ux2 + uy2 + uz2) - R(8)) * g9 + R(4.0 / 3.0) * (v10 + v11 + v12);
  g[17] = R(C.c17) * b17 - R(2.0 / 3.0) * (p4 + p5) + R(4.0 / 3.0) * p6 +
          R(0.25) * (ux2 - uy2 - R(3) * uz2 - R(2)) * g7 +
          R(0.25) * (ux2 - R(5) * uy2 + uz2 - R(2)) * g8 +
          R(1.75) * (R(-2) * ux2 + uy2 + uz2) * g9 + R(2.0 / 3.0) * v10 -
          third * (v11 + v12) - uy * g14 + uz * g15;
  g[18] = R(C.c18) * b18 - R(2) * (p4 - p5) +
          R(0.75) * (ux2 - uy2 + uz2 + R(2.0 / 3.0)) * g7 +
          R(0.75) * (R(-3) * ux2 - uy2 + uz2 - R(2)) * g8 + R(5.25) * (uz2 - uy2) * g9 +
          (v11 - v12) + R(2) * ux * g13 - uy * g14 - uz * g15;

  // ---- back-transform f~ = f + K g^ (+ second half of the source) --------
  if constexpr (PAIR_OUT) {
    if (FORCE) add_half_source(p, ux, uy, uz, C.FS);
    from_pairs(p, g, d);
  } else {
    add_K_g<R, FORCE>(d, g, ux, uy, uz, C.FS);
  }
  if constexpr (LOG2LAM != 0) out.rho = rho * R(T(1.0 / double(1 << LOG2LAM)));
  else out.rho = rho;
  out.ux = ux;
  out.uy = uy;
  out.uz = uz;
  out.gamma_dot = gd;
}

}  // namespace clbm
