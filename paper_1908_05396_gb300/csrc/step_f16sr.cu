// step_f16sr.cu -- the F16S form (FP16 of 1024 (f - w rho0), the shifted
// storage of the populations) stepped with stochastically rounded stores.
//
// Round-to-nearest FP16 drops every per-step change below half an ulp of the
// stored value, and near a steady state those are all of them: the stored
// state freezes short of the steady state at the same nodes every step.
// Stochastic rounding keeps such changes on average (see sround.cuh).  The
// stored layout, decoding and collision are those of the F16S step kernel;
// only the store differs, so state import and export, fields and every
// other entry point treat the lattice as F16S.
#include "kernels.cuh"
#include "sround.cuh"
#include "launch_f16sr.h"

namespace clbm {
namespace {

template <bool FORCE, bool CHECK, bool CAP>
__global__ void __launch_bounds__(256, CAP ? 4 : 1) step_sr_kernel(const StepArgs<__half, float> a,
                                                                   unsigned step) {
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
    float d[Q];
    if (y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1) {
#pragma unroll
      for (int q = 0; q < Q; ++q) d[q] = Codec<__half, float>::dec(a.srcq[q][i], 1.0f);
      xface_fix(a, x, i, d);
    } else {
      pull_face<__half, float>(a.src, a.qstride, a.nx, a.ny, a.nz, a.pitch, a.plane, a.facebits,
                               x, y, z, i, a.lidc, d);
    }
    NodeOut<float> o;
    collide<float, FORCE, pair_out<__half>(), log2_scale<__half>()>(a.C, d, o);
    // the deviations are carried scaled by 1024, as they are stored
    uint32_t state = sr_seed(uint32_t(i), step);
#pragma unroll
    for (int q = 0; q < Q; q += 2) {
      __half hi, lo;
      enc16_sr2(d[q], q + 1 < Q ? d[q + 1 < Q ? q + 1 : q] : 0.0f, state, hi, lo);
      a.dstq[q][i] = hi;
      if (q + 1 < Q) a.dstq[q + 1 < Q ? q + 1 : q][i] = lo;
    }
    if (CHECK) {
      float* up = reinterpret_cast<float*>(a.cb.uprev);
      const int64_t nst = int64_t(a.plane) * a.nz;
      const float px = up[i], py = up[nst + i], pz = up[2 * nst + i];
      up[i] = o.ux;
      up[nst + i] = o.uy;
      up[2 * nst + i] = o.uz;
      const double ex = double(o.ux) - double(px), ey = double(o.uy) - double(py),
                   ez = double(o.uz) - double(pz);
      du2 = ex * ex + ey * ey + ez * ez;
      uu = double(o.ux) * double(o.ux) + double(o.uy) * double(o.uy) + double(o.uz) * double(o.uz);
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

}  // namespace

// The arguments are those launch_step_t gives the F16S step kernel (upwind
// base pointers, scaled lid terms and collision constants, the alternating
// z sweep); npt 1 (plus 4: register-capped) is the only shape.
cudaError_t launch_step_f16sr(const void* src, void* dst, const Geom& g, const PhysParams& P,
                              const CheckBufs& cb, bool check, dim3 block, int npt, int64_t step,
                              cudaStream_t st) {
  StepArgs<__half, float> a;
  const __half* s = static_cast<const __half*>(src);
  __half* d = static_cast<__half*>(dst);
  const double lam = double(1 << log2_scale<__half>());
  for (int q = 0; q < Q; ++q) {
    const int64_t off = int64_t(cz(q)) * g.plane + int64_t(cy(q)) * g.pitch + cx(q);
    // the shifted base may precede the buffer; only base + i of a node in
    // the box is dereferenced
    a.srcq[q] = reinterpret_cast<const __half*>(reinterpret_cast<uintptr_t>(s) +
                                                 (int64_t(q) * g.qstride - off) * 2);
    a.dstq[q] = d + int64_t(q) * g.qstride;
    a.lidc[q] = float(6.0 * wt<double>(q) * g.rho0 * lam *
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
  a.zrev = reinterpret_cast<uintptr_t>(dst) < reinterpret_cast<uintptr_t>(src) ? 1 : 0;
  a.C = make_const<float>(P, lam);
  a.cb = cb;
  const unsigned sstep = unsigned(uint64_t(step));
  const bool cap = (npt & 4) != 0;
  dim3 grid((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, g.nz);
  cudaError_t e_ = cudaSuccess;
#define CLBM_SR_LAUNCH(F, C_)                                                                  \
  do {                                                                                        \
    if (cap) e_ = pdl_launch(step_sr_kernel<F, C_, true>, grid, block, st, a, sstep);         \
    else e_ = pdl_launch(step_sr_kernel<F, C_, false>, grid, block, st, a, sstep);            \
  } while (0)
  if (P.has_force) {
    if (check) CLBM_SR_LAUNCH(true, true);
    else CLBM_SR_LAUNCH(true, false);
  } else {
    if (check) CLBM_SR_LAUNCH(false, true);
    else CLBM_SR_LAUNCH(false, false);
  }
#undef CLBM_SR_LAUNCH
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

}  // namespace clbm
