// batch.cuh -- one persistent launch that steps many lattices of uneven size.
//
// Every lattice is cut into tiles of (block_x x block_y) nodes times a chunk
// of zc planes.  A device table maps each tile to its lattice, and each
// lattice has a descriptor (buffers, geometry, collision constants) in device
// memory.  A persistent grid of blocks strides over the tiles; a block
// computes the per-direction offsets of its lattice once per tile and reuses
// them for every plane of the chunk.  Parameters live in device memory, so a
// CUDA graph captured once stays valid when lattices join or leave: only the
// tables change.
#pragma once

#include "kernels.cuh"

namespace clbm {

template <typename R>
struct LatDesc {
  const void* buf[2];  // buf[p]: source buffer at parity p (the other is the destination)
  void* uprev;         // velocities of the previous check (math type)
  int64_t qstride;
  int nx, ny, nz, pitch, plane;
  unsigned facebits;
  int tiles_x, tiles_y, tile_begin;
  int slot;            // row of this lattice in the batch's reduction array
  R lidc[Q];
  CollideConst<R> C;
};

// One node of the batched step: same pull, boundaries and collision as
// step_kernel, with addresses from base + per-direction offset.
template <typename S, typename R, bool FORCE>
__device__ __forceinline__ void batch_node(const LatDesc<R>& L, const S* __restrict__ src,
                                           S* __restrict__ dst, const int (&off)[Q],
                                           int x, int y, int z, NodeOut<R>& o) {
  const int i = z * L.plane + y * L.pitch + x;
  R d[Q];
  if (y > 0 && y < L.ny - 1 && z > 0 && z < L.nz - 1) {
#pragma unroll
    for (int q = 0; q < Q; ++q) d[q] = Codec<S, R>::dec(src[off[q] + i], R(1));
    if (x == 0 || x == L.nx - 1) {
      const int kl = L.facebits & 3, kr = (L.facebits >> 2) & 3;
#pragma unroll
      for (int q = 1; q < Q; ++q) {
        if (cx(q) == 1 && x == 0) {
          d[q] = kl == BC_PERIODIC
                     ? Codec<S, R>::dec(src[off[q] + i + L.nx], R(1))
                     : Codec<S, R>::dec(src[opp(q) * L.qstride + i], R(1)) +
                           (kl == BC_LID ? L.lidc[q] : R(0));
        }
        if (cx(q) == -1 && x == L.nx - 1) {
          d[q] = kr == BC_PERIODIC
                     ? Codec<S, R>::dec(src[off[q] + i - L.nx], R(1))
                     : Codec<S, R>::dec(src[opp(q) * L.qstride + i], R(1)) +
                           (kr == BC_LID ? L.lidc[q] : R(0));
        }
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < Q; ++q)
      d[q] = pull_general<S, R>(src, L.qstride, L.nx, L.ny, L.nz, L.pitch, L.plane, L.facebits,
                                q, x, y, z, i, L.lidc[q]);
  }
  collide<R, FORCE>(L.C, d, o);
#pragma unroll
  for (int q = 0; q < Q; ++q) dst[q * L.qstride + i] = Codec<S, R>::enc(d[q], R(1));
}

template <typename S, typename R, bool CHECK>
__global__ void __launch_bounds__(256) batch_step_kernel(const LatDesc<R>* __restrict__ lats,
                                                         const int* __restrict__ owner,
                                                         BatchHeader* hdr, int parity,
                                                         double* acc) {
  const int ntiles = hdr->ntiles;
  const int nlat = hdr->nlat;
  const int zc = hdr->zc;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int li = owner[t];
    // Self-check of the tables before any access through them.
    bool ok = li >= 0 && li < nlat && zc >= 1;
    const LatDesc<R>& L = lats[ok ? li : 0];
    if (ok) {
      const int ntl = L.tiles_x * L.tiles_y * ((L.nz + zc - 1) / zc);
      ok = L.buf[0] != nullptr && L.buf[1] != nullptr && L.nx >= 1 && L.ny >= 1 && L.nz >= 1 &&
           L.tiles_x >= 1 && L.tiles_y >= 1 && t >= L.tile_begin && t < L.tile_begin + ntl &&
           L.tiles_x * int(blockDim.x) >= L.nx && L.tiles_y * int(blockDim.y) >= L.ny &&
           L.pitch >= L.nx && L.plane == L.pitch * L.ny && L.qstride >= int64_t(L.plane) * L.nz;
    }
    if (!ok) {  // block-uniform: skip the tile, report it
      if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(&hdr->err, 1);
      continue;
    }
    const int local = t - L.tile_begin;
    const int tx = local % L.tiles_x;
    const int rest = local / L.tiles_x;
    const int ty = rest % L.tiles_y;
    const int z0 = (rest / L.tiles_y) * zc;
    const int x = tx * blockDim.x + threadIdx.x;
    const int y = ty * blockDim.y + threadIdx.y;
    const S* src = static_cast<const S*>(L.buf[parity]);
    S* dst = static_cast<S*>(const_cast<void*>(L.buf[parity ^ 1]));
    // element offset of the upwind source of direction q (19 * qstride < 2^31
    // is required of batched lattices)
    int off[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q)
      off[q] = q * int(L.qstride) - (cz(q) * L.plane + cy(q) * L.pitch + cx(q));
    const bool active = x < L.nx && y < L.ny;
    const int z1 = min(z0 + zc, L.nz);
    double du2 = 0.0, uu = 0.0, dr = 0.0;
    int bad = 0;
    if (active) {
      for (int z = z0; z < z1; ++z) {
        NodeOut<R> o;
        if (L.C.has_force)
          batch_node<S, R, true>(L, src, dst, off, x, y, z, o);
        else
          batch_node<S, R, false>(L, src, dst, off, x, y, z, o);
        if (CHECK) {
          R* up = static_cast<R*>(L.uprev);
          const int64_t nst = int64_t(L.plane) * L.nz;
          const int64_t i = int64_t(z) * L.plane + int64_t(y) * L.pitch + x;
          const R px = up[i], py = up[nst + i], pz = up[2 * nst + i];
          up[i] = o.ux;
          up[nst + i] = o.uy;
          up[2 * nst + i] = o.uz;
          const double ex = double(o.ux) - double(px), ey = double(o.uy) - double(py),
                       ez = double(o.uz) - double(pz);
          du2 += ex * ex + ey * ey + ez * ez;
          uu += double(o.ux) * double(o.ux) + double(o.uy) * double(o.uy) +
                double(o.uz) * double(o.uz);
          dr += double(o.rho) - double(L.C.rho0);
          const double chk = double(o.rho) + double(o.ux) + double(o.uy) + double(o.uz);
          bad |= !(chk == chk) || !(fabs(chk) < 1e30) ||
                 !(double(o.rho) > 0.5 && double(o.rho) < 2.0);
        }
      }
    }
    if (CHECK) {
      __shared__ double smem[32];
      double* a = acc + 4 * L.slot;
      block_sum_add(du2, &a[0], smem);
      block_sum_add(uu, &a[1], smem);
      block_sum_add(dr, &a[2], smem);
      if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0)
        atomicOr(reinterpret_cast<int*>(&a[3]), 1);
    }
  }
}

template <typename S, typename R>
cudaError_t launch_batch_t(const void* lats, const int* owner, const void* hdr, int parity,
                           bool check, double* acc, dim3 block, int grid, cudaStream_t st) {
  const LatDesc<R>* L = static_cast<const LatDesc<R>*>(lats);
  BatchHeader* H = static_cast<BatchHeader*>(const_cast<void*>(hdr));
  if (check) batch_step_kernel<S, R, true><<<grid, block, 0, st>>>(L, owner, H, parity, acc);
  else batch_step_kernel<S, R, false><<<grid, block, 0, st>>>(L, owner, H, parity, acc);
  return cudaGetLastError();
}

// Host-side fill of one descriptor (constants converted once, in double).
template <typename R>
void fill_desc_t(void* out, const Geom& g, const PhysParams& P, const void* cur, const void* other,
                 void* uprev, int tiles_x, int tiles_y, int tile_begin, int slot) {
  LatDesc<R> L{};
  L.buf[0] = cur;
  L.buf[1] = other;
  L.uprev = uprev;
  L.qstride = g.qstride;
  L.nx = g.nx;
  L.ny = g.ny;
  L.nz = g.nz;
  L.pitch = g.pitch;
  L.plane = int(g.plane);
  L.facebits = g.facebits;
  L.tiles_x = tiles_x;
  L.tiles_y = tiles_y;
  L.tile_begin = tile_begin;
  L.slot = slot;
  for (int q = 0; q < Q; ++q)
    L.lidc[q] = R(6.0 * wt<double>(q) * g.rho0 *
                  (cx(q) * g.U[0] + cy(q) * g.U[1] + cz(q) * g.U[2]));
  L.C = make_const<R>(P);
  *static_cast<LatDesc<R>*>(out) = L;
}

}  // namespace clbm

#define CLBM_DEFINE_BATCH(SUFFIX, S, R)                                                        \
  namespace clbm {                                                                             \
  cudaError_t launch_batch_##SUFFIX(const void* lats, const int* owner, const void* hdr,       \
                                    int parity, bool check, double* acc, dim3 block, int grid, \
                                    cudaStream_t st) {                                         \
    return launch_batch_t<S, R>(lats, owner, hdr, parity, check, acc, block, grid, st);        \
  }                                                                                            \
  size_t desc_size_##SUFFIX() { return sizeof(LatDesc<R>); }                                    \
  void fill_desc_##SUFFIX(void* out, const Geom& g, const PhysParams& P, const void* cur,        \
                          const void* other, void* uprev, int tx, int ty, int tb, int slot) {  \
    fill_desc_t<R>(out, g, P, cur, other, uprev, tx, ty, tb, slot);                            \
  }                                                                                            \
  }
