// kernels.cuh -- fused pull-stream + cascaded-collision step and its helpers.
//
// Storage: structure of arrays pop[q][z][y][x] with a padded row pitch, two
// buffers (A-B).  A thread owns one node: it pulls the 19 post-collision
// populations of its upwind neighbours from buffer A (Eq. cascadedstreaming1),
// resolving walls, the lid and periodic faces from its own index, collides
// (Sec. 3) and writes the 19 results to its own slot of buffer B.  Every
// read and write of a warp covers consecutive x, so the accesses coalesce;
// the +/-x directions are offset by one element, which costs one extra
// sector per warp in L1/L2 but no extra DRAM traffic.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "collide.cuh"
#include "launch.h"

namespace clbm {

// ---- storage codecs: stored value <-> deviation f - w rho0 -----------------
template <typename S, typename R> struct Codec;
template <typename R> struct Codec<double, R> {
  static __device__ __forceinline__ R dec(double v, R) { return R(v); }
  static __device__ __forceinline__ double enc(R v, R) { return double(v); }
};
template <typename R> struct Codec<float, R> {
  static __device__ __forceinline__ R dec(float v, R) { return R(v); }
  static __device__ __forceinline__ float enc(R v, R) { return float(v); }
};
template <typename R> struct Codec<__half, R> {
  // (f - w rho0) * 1024 in FP16, round to nearest even.  The power-of-two
  // scale is exact and lifts deviations down to ~6e-8 out of the FP16
  // subnormal range while keeping |f - w rho0| < 64 representable.  The
  // kernels work on the scaled deviations directly (log2_scale): the scale
  // is folded into the collision's constants, so decoding and encoding are
  // plain conversions.
  static __device__ __forceinline__ R dec(__half v, R) { return R(__half2float(v)); }
  static __device__ __forceinline__ __half enc(R v, R) { return __float2half_rn(float(v)); }
};

// log2 of the factor by which storage type S holds the deviations f - w rho0
// (and by which the kernels carry them): 10 for FP16, 0 otherwise.
template <typename S>
__host__ __device__ constexpr int log2_scale() {
  return std::is_same<S, __half>::value ? 10 : 0;
}

// Whether the collision rebuilds the populations of storage type S from its
// pair values (see collide): for FP16 storage, whose decoded values sum
// without rounding, and for FP64, whose rounding stays far below every
// tolerance; FP32 storage takes one added correction per population.
template <typename S>
__host__ __device__ constexpr bool pair_out() {
  return std::is_same<S, __half>::value || std::is_same<S, double>::value;
}

// Collision constants for deviations carried scaled by lam (a power of two;
// see collide): the rest density and the force of the scaled moments, and
// 3K, log(3K) so that nu and the omega solve come out unscaled.
template <typename R>
__host__ __device__ __forceinline__ CollideConst<R> make_const(const PhysParams& P,
                                                             double lam = 1.0) {
  CollideConst<R> C;
  C.rho0 = R(P.rho0);
  C.rhoS = R(lam * P.rho0);
  C.FS[0] = R(lam * P.F[0]);
  C.FS[1] = R(lam * P.F[1]);
  C.FS[2] = R(lam * P.F[2]);
  C.F[0] = R(P.F[0]);
  C.F[1] = R(P.F[1]);
  C.F[2] = R(P.F[2]);
  C.K3 = R(3.0 * P.K * lam);
  C.logK3 = R(P.logK3 + log(lam));
  C.log2K3 = R(P.logK3 * 1.4426950408889634074 + log2(lam));
  C.n = R(P.n);
  C.rn = R(1.0 / P.n);
  C.ehalf = R(0.5 * (P.n - 1.0));
  C.ylo = R(P.ylo);
  C.yhi = R(P.yhi);
  C.ylo2 = R(P.ylo * 1.4426950408889634074);
  C.yhi2 = R(P.yhi * 1.4426950408889634074);
  C.nu_min = R(P.nu_min);
  C.nu_max = R(P.nu_max);
  C.newtonian = P.newtonian;
  C.has_force = P.has_force;
  const double* w = P.omega_high;  // omega_9 .. omega_18
  C.c9 = R(-w[0] / 126.0);
  C.c10 = R(0.125 * w[1]);
  C.c11 = R(0.125 * w[2]);
  C.c12 = R(0.125 * w[3]);
  C.c13 = R(0.125 * w[4]);
  C.c14 = R(0.125 * w[5]);
  C.c15 = R(0.125 * w[6]);
  C.c16 = R(w[7] / 12.0);
  C.c17 = R(w[8] / 24.0);
  C.c18 = R(0.125 * w[9]);
  C.cB = R(6.0 * w[0] * w[0]);
  return C;
}

// Pull the 19 pre-collision deviations of node (x, y, z).
template <typename S, typename R>
__device__ __forceinline__ void pull(const S* __restrict__ src, const Geom& g,
                                     int x, int y, int z, int64_t i, R lam,
                                     R (&d)[Q]) {
  const bool interior = x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1 &&
                        z > 0 && z < g.nz - 1;
  if (interior) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int64_t off = int64_t(cz(q)) * g.plane + int64_t(cy(q)) * g.pitch + cx(q);
      d[q] = Codec<S, R>::dec(src[q * g.qstride + i - off], lam);
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int s[3] = {x - cx(q), y - cy(q), z - cz(q)};
    const int n3[3] = {g.nx, g.ny, g.nz};
    bool bounce = false, lid = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (s[a] < 0 || s[a] >= n3[a]) {
        const int kind = (g.facebits >> (2 * (2 * a + (s[a] < 0 ? 0 : 1)))) & 3;
        if (kind == BC_PERIODIC) {
          s[a] += (s[a] < 0) ? n3[a] : -n3[a];
        } else {
          bounce = true;
          lid = lid || kind == BC_LID;
        }
      }
    }
    if (bounce) {
      // Halfway bounce-back f_q(x) = f~_opp(q)(x); a lid adds
      // 6 w_q rho0 (e_q . U), which is the same for deviations.
      R v = Codec<S, R>::dec(src[opp(q) * g.qstride + i], lam);
      if (lid)
        v += lam * R(6) * wt<R>(q) * R(g.rho0) *
             (R(cx(q)) * R(g.U[0]) + R(cy(q)) * R(g.U[1]) + R(cz(q)) * R(g.U[2]));
      d[q] = v;
    } else {
      const int64_t j = int64_t(s[2]) * g.plane + int64_t(s[1]) * g.pitch + s[0];
      d[q] = Codec<S, R>::dec(src[q * g.qstride + j], lam);
    }
  }
}

// Block-wide FP64 sum of v, added atomically to *acc by one thread.
__device__ __forceinline__ void block_sum_add(double v, double* acc, double* smem) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  const int nwarp = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < nwarp) ? smem[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(acc, v);
  }
  __syncthreads();
}

// ---- the fused step ---------------------------------------------------------
// Direction tables for the general pull, where the direction is a run-time value.
static __constant__ signed char c_ex[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static __constant__ signed char c_ey[Q] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
static __constant__ signed char c_ez[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
static __constant__ signed char c_opp[Q] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15};

// Everything one step launch needs, precomputed on the host in the math
// precision R (no double arithmetic is left in the FP32 kernels).
template <typename S, typename R>
struct StepArgs {
  const S* srcq[Q];  // srcq[q][i]: stored f~_q of the upwind neighbour of node i
  S* dstq[Q];        // dstq[q][i]: slot of direction q of node i
  const S* src;      // source buffer base (bounce-back and general path)
  int64_t qstride;
  int nx, ny, nz, pitch, plane;
  unsigned facebits;
  int zrev;          // 1: planes in descending z (every other step, see launch_step_t)
  R lidc[Q];         // 6 w_q rho0 (e_q . U_lid): lid momentum correction
  CollideConst<R> C;
  CheckBufs cb;
};

// Pull of all 19 directions into node (x, y, z) with index i, for a node on
// any face.  A direction whose upwind node lies inside the lattice is loaded
// as in the interior (its address is formed only then); the others follow the
// face rules -- the periodic wrap along a periodic axis, or else (any crossed
// wall or lid face) halfway bounce-back from the node's own opposite
// population, plus the lid term when a crossed face is the lid.  With the directions unrolled, a warp on a face issues one load per
// direction instead of a call with table lookups.
template <typename S, typename R>
__device__ __forceinline__ void pull_face(const S* __restrict__ src, int64_t qstride, int nx,
                                          int ny, int nz, int pitch, int plane, unsigned fb,
                                          int x, int y, int z, int i, const R* lidc, R (&d)[Q]) {
  const bool fx0 = x == 0, fx1 = x == nx - 1, fy0 = y == 0, fy1 = y == ny - 1;
  const bool fz0 = z == 0, fz1 = z == nz - 1;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const S* sq = src + int64_t(q) * qstride;
    const bool ox = (cx(q) == 1 && fx0) || (cx(q) == -1 && fx1);
    const bool oy = (cy(q) == 1 && fy0) || (cy(q) == -1 && fy1);
    const bool oz = (cz(q) == 1 && fz0) || (cz(q) == -1 && fz1);
    const int up = i - (cz(q) * plane + cy(q) * pitch + cx(q));
    if (!(ox || oy || oz)) {
      d[q] = Codec<S, R>::dec(sq[up], R(1));
      continue;
    }
    // kind of each crossed face (faces -x, +x, -y, +y, -z, +z, two bits each)
    const int kx = ox ? int((fb >> (cx(q) == 1 ? 0 : 2)) & 3u) : int(BC_PERIODIC);
    const int ky = oy ? int((fb >> (cy(q) == 1 ? 4 : 6)) & 3u) : int(BC_PERIODIC);
    const int kz = oz ? int((fb >> (cz(q) == 1 ? 8 : 10)) & 3u) : int(BC_PERIODIC);
    if (kx != BC_PERIODIC || ky != BC_PERIODIC || kz != BC_PERIODIC) {
      const bool lid = kx == BC_LID || ky == BC_LID || kz == BC_LID;
      const R v = Codec<S, R>::dec(src[int64_t(opp(q)) * qstride + i], R(1));
      d[q] = lid ? v + lidc[q] : v;
    } else {
      int j = up;
      if (ox) j += cx(q) == 1 ? nx : -nx;
      if (oy) j += cy(q) == 1 ? ny * pitch : -ny * pitch;
      if (oz) j += cz(q) == 1 ? nz * plane : -nz * plane;
      d[q] = Codec<S, R>::dec(sq[j], R(1));
    }
  }
}

// For a node off the y and z faces whose d[] holds the plain upwind values:
// replace the directions that cross an x face (bounce-back with the lid term,
// or the periodic wrap).  Only lanes at x = 0 or x = nx - 1 do any work.
template <typename S, typename R>
__device__ __forceinline__ void xface_fix(const StepArgs<S, R>& a, int x, int i, R (&d)[Q]) {
  if (x == 0 || x == a.nx - 1) {
    const int kl = a.facebits & 3, kr = (a.facebits >> 2) & 3;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
      if (cx(q) == 1 && x == 0) {
        d[q] = kl == BC_PERIODIC
                   ? Codec<S, R>::dec(a.srcq[q][i + a.nx], R(1))
                   : Codec<S, R>::dec(a.src[opp(q) * a.qstride + i], R(1)) +
                         (kl == BC_LID ? a.lidc[q] : R(0));
      }
      if (cx(q) == -1 && x == a.nx - 1) {
        d[q] = kr == BC_PERIODIC
                   ? Codec<S, R>::dec(a.srcq[q][i - a.nx], R(1))
                   : Codec<S, R>::dec(a.src[opp(q) * a.qstride + i], R(1)) +
                         (kr == BC_LID ? a.lidc[q] : R(0));
      }
    }
  }
}

// Programmatic dependent launch between consecutive steps.  A step launched
// with the programmatic stream-serialisation attribute may be scheduled
// while the previous step's last blocks still run: each of its threads waits
// here until the previous grid has completed and its writes are visible,
// before any global access, and then allows the next step to be scheduled.
// The next grid is only scheduled once every block of this one has passed
// this point (or exited), so its waiting blocks never take SM slots that a
// block of this grid still needs.  Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Launch a kernel whose threads start with pdl_enter(), with the programmatic
// stream-serialisation attribute (compiled out with -DCLBM_NO_PDL) and
// `smem` bytes of dynamic shared memory.
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t st, const Args&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
#ifdef CLBM_NO_PDL
  cfg.numAttrs = 0;
#else
  cfg.numAttrs = 1;
#endif
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                              const Args&... args) {
  return pdl_launch_smem(kernel, grid, block, 0, st, args...);
}

// One time step.  Warps off the y and z faces load all 19 upwind values
// unconditionally and then, in the one or two lanes on an x face, replace the
// five directions that come from outside the box; warps on a y or z face go
// through pull_face.  CHECK = true also writes u into uprev (after reading
// the previous check's value there) and reduces sum|u - uprev|^2, sum|u|^2,
// sum(rho - rho0) and a divergence flag in FP64.
// CAP = true caps registers so that four 256-thread (or eight 128-thread)
// blocks fit on an SM: more warps to hide DRAM latency, at the risk of
// spills; the autotuner decides.
template <typename S, typename R, bool FORCE, bool CHECK, bool CAP>
__global__ void __launch_bounds__(256, CAP ? 4 : 1) step_kernel(const StepArgs<S, R> a) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = a.zrev ? a.nz - 1 - int(blockIdx.z) : int(blockIdx.z);
  const bool active = x < a.nx && y < a.ny;
  if (!CHECK && !active) return;
  double du2 = 0.0, uu = 0.0, dr = 0.0;
  int bad = 0;
  if (active) {
    const int i = z * a.plane + y * a.pitch + x;
    R d[Q];
    if (y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1) {
#pragma unroll
      for (int q = 0; q < Q; ++q) d[q] = Codec<S, R>::dec(a.srcq[q][i], R(1));
      xface_fix(a, x, i, d);
    } else {
      pull_face<S, R>(a.src, a.qstride, a.nx, a.ny, a.nz, a.pitch, a.plane, a.facebits, x, y, z,
                      i, a.lidc, d);
    }
    NodeOut<R> o;
    collide<R, FORCE, pair_out<S>(), log2_scale<S>()>(a.C, d, o);
#pragma unroll
    for (int q = 0; q < Q; ++q) a.dstq[q][i] = Codec<S, R>::enc(d[q], R(1));
    if (CHECK) {
      R* up = reinterpret_cast<R*>(a.cb.uprev);
      const int64_t nst = int64_t(a.plane) * a.nz;
      const R px = up[i], py = up[nst + i], pz = up[2 * nst + i];
      up[i] = o.ux;
      up[nst + i] = o.uy;
      up[2 * nst + i] = o.uz;
      const double ex = double(o.ux) - double(px), ey = double(o.uy) - double(py),
                   ez = double(o.uz) - double(pz);
      du2 = ex * ex + ey * ey + ez * ez;
      uu = double(o.ux) * double(o.ux) + double(o.uy) * double(o.uy) +
           double(o.uz) * double(o.uz);
      dr = double(o.rho) - double(a.C.rho0);
      const double chk = double(o.rho) + double(o.ux) + double(o.uy) + double(o.uz);
      bad = !(chk == chk) || !(fabs(chk) < 1e30) || !(double(o.rho) > 0.5 && double(o.rho) < 2.0);
    }
  }
  if (CHECK) {
    __shared__ double smem[32];
    block_sum_add(du2, &a.cb.acc[0], smem);
    block_sum_add(uu, &a.cb.acc[1], smem);
    block_sum_add(dr, &a.cb.acc[2], smem);
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(a.cb.flag, 1);
  }
}

// Two nodes per thread, rows y and y + 1 at the same (x, z), collided as a
// pair with packed FP32 arithmetic (R = V2).  Loads and stores stay 32-bit
// per row, so every warp access still covers 32 consecutive x.  Both nodes
// share x, so the x-face replacement is the same for the pair; a pair that
// touches a y or z face pulls node by node through pull_face.
template <typename S, bool FORCE, bool CHECK, bool CAP>
__global__ void __launch_bounds__(128, CAP ? 4 : 1) step2_kernel(const StepArgs<S, float> a) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = 2 * (blockIdx.y * blockDim.y + threadIdx.y);
  const int z = blockIdx.z;
  const bool activeA = x < a.nx && y < a.ny;
  const bool activeB = activeA && y + 1 < a.ny;
  if (!CHECK && !activeA) return;
  double du2 = 0.0, uu = 0.0, dr = 0.0;
  int bad = 0;
  if (activeA) {
    const int iA = z * a.plane + y * a.pitch + x;
    const int iB = activeB ? iA + a.pitch : iA;
    V2 d[Q];
    if (y > 0 && y + 1 < a.ny - 1 && z > 0 && z < a.nz - 1) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
        d[q] = V2(Codec<S, float>::dec(a.srcq[q][iA], 1.0f),
                  Codec<S, float>::dec(a.srcq[q][iB], 1.0f));
      if (x == 0 || x == a.nx - 1) {
        const int kl = a.facebits & 3, kr = (a.facebits >> 2) & 3;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
          if (cx(q) == 1 && x == 0) {
            d[q] = kl == BC_PERIODIC
                       ? V2(Codec<S, float>::dec(a.srcq[q][iA + a.nx], 1.0f),
                            Codec<S, float>::dec(a.srcq[q][iB + a.nx], 1.0f))
                       : V2(Codec<S, float>::dec(a.src[opp(q) * a.qstride + iA], 1.0f),
                            Codec<S, float>::dec(a.src[opp(q) * a.qstride + iB], 1.0f)) +
                             V2(kl == BC_LID ? a.lidc[q] : 0.0f);
          }
          if (cx(q) == -1 && x == a.nx - 1) {
            d[q] = kr == BC_PERIODIC
                       ? V2(Codec<S, float>::dec(a.srcq[q][iA - a.nx], 1.0f),
                            Codec<S, float>::dec(a.srcq[q][iB - a.nx], 1.0f))
                       : V2(Codec<S, float>::dec(a.src[opp(q) * a.qstride + iA], 1.0f),
                            Codec<S, float>::dec(a.src[opp(q) * a.qstride + iB], 1.0f)) +
                             V2(kr == BC_LID ? a.lidc[q] : 0.0f);
          }
        }
      }
    } else {
      const int yB = activeB ? y + 1 : y;
      float dA[Q], dB[Q];
      pull_face<S, float>(a.src, a.qstride, a.nx, a.ny, a.nz, a.pitch, a.plane, a.facebits, x, y,
                          z, iA, a.lidc, dA);
      pull_face<S, float>(a.src, a.qstride, a.nx, a.ny, a.nz, a.pitch, a.plane, a.facebits, x, yB,
                          z, iB, a.lidc, dB);
#pragma unroll
      for (int q = 0; q < Q; ++q) d[q] = V2(dA[q], dB[q]);
    }
    NodeOut<V2> o;
    collide<V2, FORCE, pair_out<S>(), log2_scale<S>()>(a.C, d, o);
#pragma unroll
    for (int q = 0; q < Q; ++q) a.dstq[q][iA] = Codec<S, float>::enc(lane0(d[q]), 1.0f);
    if (activeB) {
#pragma unroll
      for (int q = 0; q < Q; ++q) a.dstq[q][iB] = Codec<S, float>::enc(lane1(d[q]), 1.0f);
    }
    if (CHECK) {
      float* up = reinterpret_cast<float*>(a.cb.uprev);
      const int64_t nst = int64_t(a.plane) * a.nz;
      const float ux[2] = {lane0(o.ux), lane1(o.ux)}, uy[2] = {lane0(o.uy), lane1(o.uy)},
                  uz[2] = {lane0(o.uz), lane1(o.uz)}, rh[2] = {lane0(o.rho), lane1(o.rho)};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (k == 1 && !activeB) break;
        const int i = k == 0 ? iA : iB;
        const float px = up[i], py = up[nst + i], pz = up[2 * nst + i];
        up[i] = ux[k];
        up[nst + i] = uy[k];
        up[2 * nst + i] = uz[k];
        const double ex = double(ux[k]) - double(px), ey = double(uy[k]) - double(py),
                     ez = double(uz[k]) - double(pz);
        du2 += ex * ex + ey * ey + ez * ez;
        uu += double(ux[k]) * double(ux[k]) + double(uy[k]) * double(uy[k]) +
              double(uz[k]) * double(uz[k]);
        dr += double(rh[k]) - double(a.C.rho0);
        const double chk = double(rh[k]) + double(ux[k]) + double(uy[k]) + double(uz[k]);
        bad |= !(chk == chk) || !(fabs(chk) < 1e30) ||
               !(double(rh[k]) > 0.5 && double(rh[k]) < 2.0);
      }
    }
  }
  if (CHECK) {
    __shared__ double smem[32];
    block_sum_add(du2, &a.cb.acc[0], smem);
    block_sum_add(uu, &a.cb.acc[1], smem);
    block_sum_add(dr, &a.cb.acc[2], smem);
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(a.cb.flag, 1);
  }
}

// Macroscopic fields of the current state (pull + moments + omega solve).
template <typename S, typename R, bool FORCE>
__global__ void __launch_bounds__(256) fields_kernel(const S* __restrict__ src, Geom g,
                                                     PhysParams P, double* rho,
                                                     double* u, double* gd) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const double lam = double(1 << log2_scale<S>());
  const CollideConst<R> C = make_const<R>(P, lam);
  const int64_t i = int64_t(z) * g.plane + int64_t(y) * g.pitch + x;
  R d[Q];
  pull<S, R>(src, g, x, y, z, i, R(lam), d);
  NodeOut<R> o;
  collide<R, FORCE, pair_out<S>(), log2_scale<S>()>(C, d, o);
  const int64_t N = int64_t(g.nx) * g.ny * g.nz;
  const int64_t k = (int64_t(z) * g.ny + y) * g.nx + x;
  if (rho) rho[k] = double(o.rho);
  if (u) {
    u[k] = double(o.ux);
    u[N + k] = double(o.uy);
    u[2 * N + k] = double(o.uz);
  }
  if (gd) gd[k] = double(o.gamma_dot);
}

// Collide M independent nodes given as plain FP64 populations [q][node].
template <typename S, typename R, bool FORCE>
__global__ void collide_nodes_kernel(PhysParams P, const double* __restrict__ fin,
                                     double* __restrict__ fout, double* rho,
                                     double* u, double* gd, int64_t M) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const double lam = double(1 << log2_scale<S>());
  const CollideConst<R> C = make_const<R>(P, lam);
  R d[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const R dev = R((fin[q * M + k] - wt<double>(q) * P.rho0) * lam);
    d[q] = Codec<S, R>::dec(Codec<S, R>::enc(dev, R(lam)), R(lam));
  }
  NodeOut<R> o;
  collide<R, FORCE, pair_out<S>(), log2_scale<S>()>(C, d, o);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const R st = Codec<S, R>::dec(Codec<S, R>::enc(d[q], R(lam)), R(lam));
    fout[q * M + k] = double(st) / lam + wt<double>(q) * P.rho0;
  }
  if (rho) rho[k] = double(o.rho);
  if (u) {
    u[k] = double(o.ux);
    u[M + k] = double(o.uy);
    u[2 * M + k] = double(o.uz);
  }
  if (gd) gd[k] = double(o.gamma_dot);
}

// The local relaxation rate omega_nu and |gamma_dot| of M nodes from their
// density and non-equilibrium moments m^(1)_4..9 ([6][node], FP64), solved
// in the math precision R exactly as the collision does.
template <typename R>
__global__ void omega_nodes_kernel(PhysParams P, const double* __restrict__ rho_in,
                                   const double* __restrict__ m, double* omega, double* gd,
                                   int64_t M) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const CollideConst<R> C = make_const<R>(P);
  const R rho = R(rho_in[k]);
  const R rinv = rrcp<R>(rho);
  R A, B;
  strain_AB(C, rinv, R(m[k]), R(m[M + k]), R(m[2 * M + k]), R(m[3 * M + k]), R(m[4 * M + k]),
            R(m[5 * M + k]), A, B);
  R g;
  const R w = omega_nu(C, rho, rinv, A, B, &g);
  omega[k] = double(w);
  if (gd) gd[k] = double(g);
}

// Stored populations <-> plain FP64 f in the unpadded layout [q][z][y][x].
template <typename S>
__global__ void export_kernel(const S* __restrict__ src, Geom g, double rho0,
                              double inv_scale, double* __restrict__ out) {
  const int64_t N = int64_t(g.nx) * g.ny * g.nz;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= N * Q) return;
  const int q = int(t / N);
  const int64_t k = t - int64_t(q) * N;
  const int x = int(k % g.nx), y = int((k / g.nx) % g.ny), z = int(k / (int64_t(g.nx) * g.ny));
  const int64_t i = int64_t(z) * g.plane + int64_t(y) * g.pitch + x;
  const double w = wt<double>(q);
  out[t] = double(Codec<S, double>::dec(src[q * g.qstride + i], inv_scale)) * inv_scale + w * rho0;
}

template <typename S>
__global__ void import_kernel(const double* __restrict__ in, Geom g, double rho0,
                              double inv_scale, S* __restrict__ dst) {
  const int64_t N = int64_t(g.nx) * g.ny * g.nz;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= N * Q) return;
  const int q = int(t / N);
  const int64_t k = t - int64_t(q) * N;
  const int x = int(k % g.nx), y = int((k / g.nx) % g.ny), z = int(k / (int64_t(g.nx) * g.ny));
  const int64_t i = int64_t(z) * g.plane + int64_t(y) * g.pitch + x;
  const double w = wt<double>(q);
  dst[q * g.qstride + i] = Codec<S, double>::enc((in[t] - w * rho0) / inv_scale, inv_scale);
}

}  // namespace clbm

#include "tma_step.cuh"
#include "inplace.cuh"

namespace clbm {

// ---- host-side launchers, instantiated once per storage type --------------
template <typename S, typename R>
cudaError_t launch_step_t(const void* src, void* dst, const Geom& g, const PhysParams& P,
                          const CheckBufs& cb, bool check, dim3 block, int npt,
                          cudaStream_t st) {
  StepArgs<S, R> a;
  const S* s = static_cast<const S*>(src);
  S* d = static_cast<S*>(dst);
  for (int q = 0; q < Q; ++q) {
    const int64_t off = int64_t(cz(q)) * g.plane + int64_t(cy(q)) * g.pitch + cx(q);
    // address arithmetic through integers: the shifted base may precede the
    // buffer, only base + i of a node in the box is dereferenced
    a.srcq[q] = reinterpret_cast<const S*>(reinterpret_cast<uintptr_t>(s) +
                                            (int64_t(q) * g.qstride - off) * int64_t(sizeof(S)));
    a.dstq[q] = d + int64_t(q) * g.qstride;
    a.lidc[q] = R(6.0 * wt<double>(q) * g.rho0 * double(1 << log2_scale<S>()) *
                  (cx(q) * g.U[0] + cy(q) * g.U[1] + cz(q) * g.U[2]));
  }
  a.src = s;
  a.qstride = g.qstride;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.pitch = g.pitch;
  a.plane = int(g.plane);
  a.facebits = g.facebits;
  // Blocks run roughly in launch order, z planes last, so a step ends with
  // its highest planes still in L2.  Sweeping z downward on every other step
  // (the steps that write the lower-addressed of the two buffers) makes the
  // next step read those planes first, from L2.
  a.zrev = reinterpret_cast<uintptr_t>(dst) < reinterpret_cast<uintptr_t>(src) ? 1 : 0;
  a.C = make_const<R>(P, double(1 << log2_scale<S>()));
  a.cb = cb;
  // npt: 1 or 2 nodes per thread; +4 selects the register-capped variant;
  // TMA_NPT + 32 v the TMA-staged kernel of shape v (check steps take the
  // plain kernel with the same block).
  if constexpr (std::is_same<R, float>::value && !std::is_same<S, double>::value) {
    if ((npt & TMA_NPT) && !check)
      return launch_step_tma<S>(a, src, g, P.has_force != 0, npt >> 5, cb.flag + 1, st);
  }
  const bool cap = (npt & 4) != 0;
  npt &= 3;
#define CLBM_STEP_LAUNCH(KERNEL, GRID, ...)                                                 \
  do {                                                                                     \
    if (P.has_force) {                                                                     \
      if (check) {                                                                         \
        if (cap) e_ = pdl_launch(KERNEL<__VA_ARGS__, true, true, true>, GRID, block, st, a);         \
        else e_ = pdl_launch(KERNEL<__VA_ARGS__, true, true, false>, GRID, block, st, a);            \
      } else {                                                                             \
        if (cap) e_ = pdl_launch(KERNEL<__VA_ARGS__, true, false, true>, GRID, block, st, a);        \
        else e_ = pdl_launch(KERNEL<__VA_ARGS__, true, false, false>, GRID, block, st, a);           \
      }                                                                                    \
    } else {                                                                               \
      if (check) {                                                                         \
        if (cap) e_ = pdl_launch(KERNEL<__VA_ARGS__, false, true, true>, GRID, block, st, a);        \
        else e_ = pdl_launch(KERNEL<__VA_ARGS__, false, true, false>, GRID, block, st, a);           \
      } else {                                                                             \
        if (cap) e_ = pdl_launch(KERNEL<__VA_ARGS__, false, false, true>, GRID, block, st, a);       \
        else e_ = pdl_launch(KERNEL<__VA_ARGS__, false, false, false>, GRID, block, st, a);          \
      }                                                                                    \
    }                                                                                      \
  } while (0)
  if constexpr (std::is_same<R, float>::value) {
    if (npt == 2) {
      dim3 grid2((g.nx + block.x - 1) / block.x, (g.ny + 2 * block.y - 1) / (2 * block.y), g.nz);
      cudaError_t e_ = cudaSuccess;
      CLBM_STEP_LAUNCH(step2_kernel, grid2, S);
      return e_ != cudaSuccess ? e_ : cudaGetLastError();
    }
  }
  dim3 grid((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, g.nz);
  cudaError_t e_ = cudaSuccess;
  CLBM_STEP_LAUNCH(step_kernel, grid, S, R);
#undef CLBM_STEP_LAUNCH
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_fields_t(const void* src, const Geom& g, const PhysParams& P, double* rho,
                            double* u, double* gd, cudaStream_t st) {
  dim3 block(32, 4);
  dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
  const S* s = static_cast<const S*>(src);
  if (P.has_force) fields_kernel<S, R, true><<<grid, block, 0, st>>>(s, g, P, rho, u, gd);
  else fields_kernel<S, R, false><<<grid, block, 0, st>>>(s, g, P, rho, u, gd);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_collide_nodes_t(const PhysParams& P, const double* fin, double* fout,
                                   double* rho, double* u, double* gd, int64_t M,
                                   cudaStream_t st) {
  const int b = 128;
  const unsigned grid = unsigned((M + b - 1) / b);
  if (P.has_force) collide_nodes_kernel<S, R, true><<<grid, b, 0, st>>>(P, fin, fout, rho, u, gd, M);
  else collide_nodes_kernel<S, R, false><<<grid, b, 0, st>>>(P, fin, fout, rho, u, gd, M);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_omega_nodes_t(const PhysParams& P, const double* rho, const double* m,
                                 double* omega, double* gd, int64_t M, cudaStream_t st) {
  const int b = 128;
  omega_nodes_kernel<R><<<unsigned((M + b - 1) / b), b, 0, st>>>(P, rho, m, omega, gd, M);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_export_t(const void* src, const Geom& g, double rho0, double inv_scale,
                            double* out, cudaStream_t st) {
  const int64_t total = int64_t(g.nx) * g.ny * g.nz * Q;
  const int b = 256;
  export_kernel<S><<<unsigned((total + b - 1) / b), b, 0, st>>>(static_cast<const S*>(src), g,
                                                                 rho0, inv_scale, out);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_import_t(const double* in, const Geom& g, double rho0, double inv_scale,
                            void* dst, cudaStream_t st) {
  const int64_t total = int64_t(g.nx) * g.ny * g.nz * Q;
  const int b = 256;
  import_kernel<S><<<unsigned((total + b - 1) / b), b, 0, st>>>(in, g, rho0, inv_scale,
                                                                 static_cast<S*>(dst));
  return cudaGetLastError();
}

}  // namespace clbm

// Defines the launchers of launch.h for one storage type S with math type R.
#define CLBM_DEFINE_LAUNCHERS(SUFFIX, S, R)                                                   \
  namespace clbm {                                                                            \
  cudaError_t launch_step_##SUFFIX(const void* src, void* dst, const Geom& g,                 \
                                   const PhysParams& P, const CheckBufs& cb, bool check,      \
                                   dim3 block, int npt, cudaStream_t st) {                    \
    return launch_step_t<S, R>(src, dst, g, P, cb, check, block, npt, st);                    \
  }                                                                                           \
  cudaError_t launch_fields_##SUFFIX(const void* src, const Geom& g, const PhysParams& P,     \
                                     double* rho, double* u, double* gd, cudaStream_t st) {   \
    return launch_fields_t<S, R>(src, g, P, rho, u, gd, st);                                  \
  }                                                                                           \
  cudaError_t launch_collide_nodes_##SUFFIX(const PhysParams& P, const double* fin,           \
                                            double* fout, double* rho, double* u, double* gd, \
                                            int64_t M, cudaStream_t st) {                     \
    return launch_collide_nodes_t<S, R>(P, fin, fout, rho, u, gd, M, st);                     \
  }                                                                                           \
  cudaError_t launch_export_##SUFFIX(const void* src, const Geom& g, double rho0,             \
                                     double inv_scale, double* out, cudaStream_t st) {        \
    return launch_export_t<S>(src, g, rho0, inv_scale, out, st);                              \
  }                                                                                           \
  cudaError_t launch_omega_nodes_##SUFFIX(const PhysParams& P, const double* rho,             \
                                          const double* m, double* omega, double* gd,         \
                                          int64_t M, cudaStream_t st) {                       \
    return launch_omega_nodes_t<R>(P, rho, m, omega, gd, M, st);                              \
  }                                                                                           \
  cudaError_t launch_import_##SUFFIX(const double* in, const Geom& g, double rho0,            \
                                     double inv_scale, void* dst, cudaStream_t st) {          \
    return launch_import_t<S>(in, g, rho0, inv_scale, dst, st);                               \
  }                                                                                           \
  }
