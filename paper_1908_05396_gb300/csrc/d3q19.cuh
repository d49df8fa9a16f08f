// d3q19.cuh -- D3Q19 lattice constants of the cascaded LBM (Sec. 3).
//
// Every table is a constexpr function so that, inside fully unrolled loops,
// nvcc folds the integer coefficients into adds and fused multiply-adds.
#pragma once

namespace clbm {

constexpr int Q = 19;

// Velocity e_alpha, Eq. velocityd3qq19, in the order of the component vectors
// |e_x>, |e_y>, |e_z> printed in Sec. 3.
__host__ __device__ constexpr int cx(int q) {
  return q == 1 || q == 7 || q == 9 || q == 11 || q == 13   ? 1
         : q == 2 || q == 8 || q == 10 || q == 12 || q == 14 ? -1
                                                              : 0;
}
__host__ __device__ constexpr int cy(int q) {
  return q == 3 || q == 7 || q == 8 || q == 15 || q == 17   ? 1
         : q == 4 || q == 9 || q == 10 || q == 16 || q == 18 ? -1
                                                              : 0;
}
__host__ __device__ constexpr int cz(int q) {
  return q == 5 || q == 11 || q == 12 || q == 15 || q == 16  ? 1
         : q == 6 || q == 13 || q == 14 || q == 17 || q == 18 ? -1
                                                               : 0;
}

// Opposite direction: e_opp(q) = -e_q.
__host__ __device__ constexpr int opp(int q) {
  return q == 0 ? 0 : (q <= 6 ? ((q & 1) ? q + 1 : q - 1) : (q == 7 ? 10 : q == 10 ? 7 : q == 8 ? 9 : q == 9 ? 8 : q == 11 ? 14 : q == 14 ? 11 : q == 12 ? 13 : q == 13 ? 12 : q == 15 ? 18 : q == 18 ? 15 : q == 16 ? 17 : 16));
}

// Lattice weights (c_s^2 = 1/3): rest 1/3, axis 1/18, diagonal 1/36.
template <typename R>
__host__ __device__ constexpr R wt(int q) {
  return q == 0 ? R(1) / R(3) : (q <= 6 ? R(1) / R(18) : R(1) / R(36));
}

// Orthogonal basis vector K_j evaluated at velocity (x, y, z): the
// Gram-Schmidt basis of Sec. 3 written as polynomials of e.
__host__ __device__ constexpr int kb(int j, int x, int y, int z) {
  return j == 0    ? 1
         : j == 1  ? x
         : j == 2  ? y
         : j == 3  ? z
         : j == 4  ? x * y
         : j == 5  ? x * z
         : j == 6  ? y * z
         : j == 7  ? x * x - y * y
         : j == 8  ? x * x + y * y - 2 * z * z
         : j == 9  ? 19 * (x * x + y * y + z * z) - 30
         : j == 10 ? 5 * x * (x * x + y * y + z * z) - 9 * x
         : j == 11 ? 5 * y * (x * x + y * y + z * z) - 9 * y
         : j == 12 ? 5 * z * (x * x + y * y + z * z) - 9 * z
         : j == 13 ? x * y * y - x * z * z
         : j == 14 ? y * z * z - y * x * x
         : j == 15 ? z * x * x - z * y * y
         : j == 16 ? 21 * (x * x * y * y + x * x * z * z + y * y * z * z) -
                         16 * (x * x + y * y + z * z) + 12
         : j == 17 ? 3 * (x * x * y * y + x * x * z * z - 2 * y * y * z * z) -
                         2 * (2 * x * x - y * y - z * z)
                   : 3 * (x * x * y * y - x * x * z * z) - 2 * (y * y - z * z);
}

// The nine +/- velocity pairs: pos(p) and opp(pos(p)).  Even moments and the
// even basis vectors see d_a + d_abar, odd ones d_a - d_abar.
__host__ __device__ constexpr int pair_pos(int p) {
  return p == 0 ? 1 : p == 1 ? 3 : p == 2 ? 5 : p == 3 ? 7 : p == 4 ? 9 : p == 5 ? 11 : p == 6 ? 13 : p == 7 ? 15 : 16;
}
constexpr int NPAIR = 9;

// Basis vectors with an odd number of velocity factors.
__host__ __device__ constexpr bool kb_odd(int j) {
  return (j >= 1 && j <= 3) || (j >= 10 && j <= 15);
}

}  // namespace clbm
