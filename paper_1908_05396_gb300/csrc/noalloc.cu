// noalloc.cu -- one check step between caller-owned buffers, allocating nothing.
//
// Some callers cannot allocate device memory when they step: a solver embedded
// in a host application that owns a fixed device-memory pool handed out at
// start-up, code running where cudaMalloc is forbidden (inside a memory-budget
// manager, or a framework that has already reserved all of the device), or
// callers that must never stall on the allocator's implicit synchronisation.
// clbm_step_noalloc() serves them: it runs the same fused step as a check step
// of clbm_step() on buffers the caller passes in, and keeps the per-block
// partial sums of its FP64 reductions in a fixed file-scope device array
// instead of memory obtained from cudaMalloc.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/clbm.h"
#include "kernels.cuh"
#include "validate.h"

namespace clbm {
namespace {

// Partial sums of one call: 4 doubles per thread block of the step.  Every
// GPU that loads the library holds this array (2 MiB) until the process ends.
constexpr int NOALLOC_MAX_BLOCKS = 65536;
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS * 4];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_partials_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device with that device current.
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return cudaSuccess;
}

// The fused step of step_kernel<..., CHECK = true>, with each block writing
// its partial sums (sum|u - uprev|^2, sum|u|^2, sum(rho - rho0), divergence)
// to its own slot of the scratch array instead of adding them atomically.
template <typename S, typename R, bool FORCE>
__global__ void __launch_bounds__(256) step_partials_kernel(const S* __restrict__ src,
                                                            S* __restrict__ dst, Geom g,
                                                            PhysParams P, R* uprev,
                                                            double* partials) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool active = x < g.nx && y < g.ny;
  const double lam = double(1 << log2_scale<S>());
  const CollideConst<R> C = make_const<R>(P, lam);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (active) {
    const int64_t i = int64_t(z) * g.plane + int64_t(y) * g.pitch + x;
    R d[Q];
    pull<S, R>(src, g, x, y, z, i, R(lam), d);
    NodeOut<R> o;
    collide<R, FORCE, pair_out<S>(), log2_scale<S>()>(C, d, o);
#pragma unroll
    for (int q = 0; q < Q; ++q) dst[q * g.qstride + i] = Codec<S, R>::enc(d[q], R(lam));
    const int64_t nst = g.plane * g.nz;
    const R px = uprev[i], py = uprev[nst + i], pz = uprev[2 * nst + i];
    uprev[i] = o.ux;
    uprev[nst + i] = o.uy;
    uprev[2 * nst + i] = o.uz;
    const double ex = double(o.ux) - double(px), ey = double(o.uy) - double(py),
                 ez = double(o.uz) - double(pz);
    v[0] = ex * ex + ey * ey + ez * ez;
    v[1] = double(o.ux) * double(o.ux) + double(o.uy) * double(o.uy) +
           double(o.uz) * double(o.uz);
    v[2] = double(o.rho) - double(P.rho0);
    const double chk = double(o.rho) + double(o.ux) + double(o.uy) + double(o.uz);
    v[3] = (!(chk == chk) || !(fabs(chk) < 1e30) ||
            !(double(o.rho) > 0.5 && double(o.rho) < 2.0)) ? 1.0 : 0.0;
  }
  // Fixed-order block reduction (warp shuffles, then warp 0), so that the
  // result does not depend on scheduling.
  __shared__ double sm[4][32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sm[k][warp] = a;
  }
  __syncthreads();
  if (warp == 0) {
    const int64_t b = (int64_t(blockIdx.z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double a = lane < nwarp ? sm[k][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) partials[b * 4 + k] = a;
    }
  }
}

// Second pass: one block sums the nblocks partials in a fixed order and
// writes the four results (the divergence entry as 0 or 1).
__global__ void __launch_bounds__(256) finish_kernel(const double* __restrict__ partials,
                                                     int nblocks, double* stats) {
  __shared__ double sm[4][256];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] += partials[int64_t(b) * 4 + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (int(threadIdx.x) < s)
#pragma unroll
      for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[0] = sm[0][0];
    stats[1] = sm[1][0];
    stats[2] = sm[2][0];
    stats[3] = sm[3][0] > 0.0 ? 1.0 : 0.0;
  }
}

template <typename S, typename R>
cudaError_t launch_noalloc(const void* src, void* dst, const Geom& g, const PhysParams& P,
                           void* uprev, double* partials, double* stats, dim3 grid, dim3 block,
                           cudaStream_t st) {
  const S* s = static_cast<const S*>(src);
  S* d = static_cast<S*>(dst);
  R* up = static_cast<R*>(uprev);
  if (P.has_force)
    step_partials_kernel<S, R, true><<<grid, block, 0, st>>>(s, d, g, P, up, partials);
  else
    step_partials_kernel<S, R, false><<<grid, block, 0, st>>>(s, d, g, P, up, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finish_kernel<<<1, 256, 0, st>>>(partials, int(grid.x * grid.y * grid.z), stats);
  return cudaGetLastError();
}

int noalloc_fail(int code, const char* msg) {
  set_unbound_error(msg);
  return code;
}

}  // namespace
}  // namespace clbm

using namespace clbm;

extern "C" int clbm_step_noalloc(const clbm_domain* d, double K, double n, const double U_lid[3],
                                 const double body_force[3], clbm_dtype dtype, const void* src,
                                 void* dst, void* u_prev, double* stats) {
  if (!d || !src || !dst || !u_prev || !stats)
    return noalloc_fail(CLBM_ERR_ARG, "null domain or buffer");
  if (src == dst) return noalloc_fail(CLBM_ERR_ARG, "src and dst must be different buffers");
  if (dtype == CLBM_F16R)
    return noalloc_fail(CLBM_ERR_UNSUPPORTED, "the F16R form is not available here");
  if (dtype != CLBM_F64 && dtype != CLBM_F32 && dtype != CLBM_F16S)
    return noalloc_fail(CLBM_ERR_ARG, "unknown dtype");
  std::string why;
  double U[3];
  if (!check_domain(d, U_lid, U, why)) return noalloc_fail(CLBM_ERR_ARG, why.c_str());
  double rho0, nu_min, nu_max;
  domain_defaults(d, &rho0, &nu_min, &nu_max);
  if (!check_phys(K, n, nu_min, nu_max, why)) return noalloc_fail(CLBM_ERR_ARG, why.c_str());
  if (!check_force(body_force, why)) return noalloc_fail(CLBM_ERR_ARG, why.c_str());

  // Dense layout: pop[q][z][y][x] with no padding, u_prev[3][z][y][x].
  Geom g{};
  g.nx = d->nx;
  g.ny = d->ny;
  g.nz = d->nz;
  g.pitch = d->nx;
  g.plane = int64_t(d->nx) * d->ny;
  g.qstride = g.plane * d->nz;
  g.facebits = 0;
  for (int f = 0; f < 6; ++f) g.facebits |= unsigned(d->face[f]) << (2 * f);
  for (int a = 0; a < 3; ++a) g.U[a] = U[a];
  g.rho0 = rho0;
  PhysParams P{};
  fill_params(P, K, n, body_force, rho0, nu_min, nu_max, dtype);
  const dim3 block(32, 4, 1);
  const dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
  const int64_t nblocks = int64_t(grid.x) * grid.y * grid.z;
  if (nblocks > NOALLOC_MAX_BLOCKS) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "lattice needs %lld thread blocks of 32x4 nodes; the fixed scratch of "
             "clbm_step_noalloc holds partial sums for at most %d (about 8.4 million nodes)",
             (long long)nblocks, NOALLOC_MAX_BLOCKS);
    return noalloc_fail(CLBM_ERR_ARG, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  double* partials = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(d->stream);
  if (e == cudaSuccess) e = scratch_address(dev, &partials);
  if (e != cudaSuccess) {
    // The first call on a device looks the scratch address up, which a
    // stream capture in progress does not allow.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      std::string m = std::string(cudaGetErrorString(e)) +
                      ": the first clbm_step_noalloc call on a device must come before any "
                      "stream capture";
      return noalloc_fail(CLBM_ERR_CUDA, m.c_str());
    }
    return noalloc_fail(CLBM_ERR_CUDA, cudaGetErrorString(e));
  }
  switch (dtype) {
    case CLBM_F64:
      e = launch_noalloc<double, double>(src, dst, g, P, u_prev, partials, stats, grid, block, st);
      break;
    case CLBM_F32:
      e = launch_noalloc<float, float>(src, dst, g, P, u_prev, partials, stats, grid, block, st);
      break;
    default:
      e = launch_noalloc<__half, float>(src, dst, g, P, u_prev, partials, stats, grid, block, st);
      break;
  }
  if (e != cudaSuccess) return noalloc_fail(CLBM_ERR_CUDA, cudaGetErrorString(e));
  return CLBM_OK;
}
