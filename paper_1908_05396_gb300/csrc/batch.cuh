// batch.cuh -- one persistent launch that steps many lattices of uneven size.
//
// Every lattice is cut into tiles of (block_x x block_y) nodes of one plane.
// A device table maps each tile to its lattice, and each lattice has a
// descriptor (buffers, geometry, collision constants) in a __constant__ table
// of the translation unit.  A persistent grid of blocks strides over the
// tiles.  Lattices with a body force come last in the tile table and are
// stepped by a second launch compiled with the force path, so neither kernel
// carries the registers of both paths.  Parameters live in device memory, so
// a CUDA graph captured once stays valid when lattices join or leave: only
// the tables change.
#pragma once

#include "kernels.cuh"
#include "sround.cuh"

namespace clbm {

template <typename R>
struct LatDesc {
  const void* buf[2];  // buf[p]: source buffer at parity p (the other is the destination)
  const void* ref[2];  // F16R form: the reference moments kept with buf[p] (else null)
  void* uprev;         // velocities of the previous check (math type)
  int64_t qstride;
  int nx, ny, nz, pitch, plane;
  unsigned facebits;
  int tiles_x, tiles_y;
  int tw_log2;         // tile width (nodes along x) = 1 << tw_log2, height = threads / width
  int slot;            // row of this lattice in the batch's reduction array
  unsigned step_offset;  // lattice steps minus batch steps (seeds stochastic rounding)
  int sround;            // F16S: stores rounded stochastically
  R lidc[Q];
  CollideConst<R> C;
};

// One node of the batched step: same pull, boundaries and collision as
// step_kernel.  Source offsets are formed from compile-time direction
// constants right before each load, so no per-direction table is held in
// registers.
template <typename S, typename R, bool FORCE>
__device__ __forceinline__ void batch_node(const LatDesc<R>& L, const S* __restrict__ src,
                                           S* __restrict__ dst, int x, int y, int z,
                                           unsigned step, NodeOut<R>& o) {
  const int qs = int(L.qstride), plane = L.plane, pitch = L.pitch;
  const int i = z * plane + y * pitch + x;
  R d[Q];
  if (y > 0 && y < L.ny - 1 && z > 0 && z < L.nz - 1) {
#pragma unroll
    for (int q = 0; q < Q; ++q)
      d[q] = Codec<S, R>::dec(src[q * qs + i - (cz(q) * plane + cy(q) * pitch + cx(q))], R(1));
    if (x == 0 || x == L.nx - 1) {
      const int kl = L.facebits & 3, kr = (L.facebits >> 2) & 3;
#pragma unroll
      for (int q = 1; q < Q; ++q) {
        const int j = q * qs + i - (cz(q) * plane + cy(q) * pitch + cx(q));
        if (cx(q) == 1 && x == 0) {
          d[q] = kl == BC_PERIODIC
                     ? Codec<S, R>::dec(src[j + L.nx], R(1))
                     : Codec<S, R>::dec(src[opp(q) * qs + i], R(1)) +
                           (kl == BC_LID ? L.lidc[q] : R(0));
        }
        if (cx(q) == -1 && x == L.nx - 1) {
          d[q] = kr == BC_PERIODIC
                     ? Codec<S, R>::dec(src[j - L.nx], R(1))
                     : Codec<S, R>::dec(src[opp(q) * qs + i], R(1)) +
                           (kr == BC_LID ? L.lidc[q] : R(0));
        }
      }
    }
  } else {
    pull_face<S, R>(src, L.qstride, L.nx, L.ny, L.nz, pitch, plane, L.facebits, x, y, z, i,
                    L.lidc, d);
  }
  collide<R, FORCE, pair_out<S>(), log2_scale<S>()>(L.C, d, o);
  if constexpr (std::is_same<S, __half>::value) {
    if (L.sround) {  // as step_f16sr.cu: two directions per stochastic conversion
      uint32_t state = sr_seed(uint32_t(i), step);
#pragma unroll
      for (int q = 0; q < Q; q += 2) {
        __half hi, lo;
        enc16_sr2(d[q], q + 1 < Q ? d[q + 1 < Q ? q + 1 : q] : 0.0f, state, hi, lo);
        dst[q * qs + i] = hi;
        if (q + 1 < Q) dst[(q + 1 < Q ? q + 1 : q) * qs + i] = lo;
      }
      return;
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) dst[q * qs + i] = Codec<S, R>::enc(d[q], R(1));
}

// One node of the batched step in the F16R form (defined with the other F16R
// kernels, the only translation unit that instantiates the batch with REF).
template <bool FORCE>
__device__ void batch_node_ref(const LatDesc<float>& L, int parity, int x, int y, int z,
                               unsigned step, NodeOut<float>& o);

// tile word: x tile (8 bits) | y tile (12 bits) | z chunk (12 bits)
__host__ __device__ __forceinline__ unsigned tile_word(int tx, int ty, int tz) {
  return unsigned(tx) | (unsigned(ty) << 8) | (unsigned(tz) << 20);
}

// The tile loop of the batched step.  get(li) returns lattice li's
// descriptor from the translation unit's __constant__ table, so ptxas can
// reload its fields where it needs them instead of holding them in registers.
template <typename S, typename R, bool CHECK, bool FORCE, bool REF, typename Get>
__device__ __forceinline__ void batch_tiles(Get get, const int* __restrict__ owner,
                                            const unsigned* __restrict__ coord,
                                            BatchHeader* hdr, int parity, double* acc, int zc) {
  // tiles [0, ntiles0) belong to lattices without force, [ntiles0, ntiles) with
  // F16R and F16S (whose lattices may round stochastically): this chain's
  // step count, advanced at the end of each of its launches by the launch's
  // last CTA
  constexpr bool STEPS = REF || std::is_same<S, __half>::value;
  const unsigned bstep =
      STEPS ? *reinterpret_cast<volatile const unsigned*>(&hdr->step[FORCE ? 1 : 0]) : 0u;
  const int t0 = FORCE ? hdr->ntiles0 : 0;
  const int t1 = FORCE ? hdr->ntiles : hdr->ntiles0;
  const int nlat = hdr->nlat;
  // The next tile's table entries are loaded while this tile collides, so a
  // tile starts with one dependent round trip (descriptor) instead of two.
  int t = t0 + int(blockIdx.x);
  int li_next = t < t1 ? owner[t] : 0;
  unsigned w_next = t < t1 ? coord[t] : 0u;
  for (; t < t1; t += gridDim.x) {
    const int li = li_next;
    const unsigned w = w_next;
    if (t + int(gridDim.x) < t1) {
      li_next = owner[t + gridDim.x];
      w_next = coord[t + gridDim.x];
    }
    const int tx = int(w & 0xffu), ty = int((w >> 8) & 0xfffu), tz = int(w >> 20);
    // Self-check of the tables before any access through them.
    bool ok = li >= 0 && li < nlat;
    const LatDesc<R>& L = get(ok ? li : 0);
    if (ok)
      ok = L.buf[0] != nullptr && L.buf[1] != nullptr && tx < L.tiles_x && ty < L.tiles_y &&
           L.tw_log2 >= 0 && L.tw_log2 <= 10 && (1 << L.tw_log2) <= int(blockDim.x * blockDim.y) &&
           (int(blockDim.x * blockDim.y) & ((1 << L.tw_log2) - 1)) == 0 &&
           zc >= 1 && tz * zc < L.nz && L.pitch >= L.nx && L.plane == L.pitch * L.ny &&
           L.qstride >= int64_t(L.plane) * L.nz && 19 * L.qstride < (int64_t(1) << 31) &&
           (L.C.has_force != 0) == FORCE && (!REF || (L.ref[0] != nullptr && L.ref[1] != nullptr));
    if (!ok) {  // block-uniform: skip the tile, report it
      if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(&hdr->err, 1);
      continue;
    }
    // the block's threads in row order over a tile of 2^tw_log2 x (threads
    // >> tw_log2) nodes (the tile width is chosen per lattice)
    const int lin = int(threadIdx.y * blockDim.x + threadIdx.x);
    const int x = (tx << L.tw_log2) + (lin & ((1 << L.tw_log2) - 1));
    const int y = ty * (int(blockDim.x * blockDim.y) >> L.tw_log2) + (lin >> L.tw_log2);
    const S* src = static_cast<const S*>(L.buf[parity]);
    S* dst = static_cast<S*>(const_cast<void*>(L.buf[parity ^ 1]));
    const bool active = x < L.nx && y < L.ny;
    double du2 = 0.0, uu = 0.0, dr = 0.0;
    int bad = 0;
    // the tile's zc planes: the per-tile work (table entries, descriptor,
    // checks, the check-step reductions) is shared by zc nodes per thread
    const int z1 = min(tz * zc + zc, L.nz);
#pragma unroll 1
    for (int z = tz * zc; z < z1; ++z) {
      if (active) {
        NodeOut<R> o;
        if constexpr (REF) batch_node_ref<FORCE>(L, parity, x, y, z, bstep + L.step_offset, o);
        else batch_node<S, R, FORCE>(L, src, dst, x, y, z, bstep + L.step_offset, o);
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
  if constexpr (STEPS) {
    // every CTA of this launch has read its chain's step count: the last one
    // to finish advances it
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      __threadfence();
      if (atomicAdd(&hdr->done[FORCE ? 1 : 0], 1) == int(gridDim.x) - 1) {
        atomicExch(&hdr->done[FORCE ? 1 : 0], 0);
        atomicAdd(&hdr->step[FORCE ? 1 : 0], 1u);
      }
    }
  }
}

// Bytes of __constant__ memory given to the descriptor table of one storage
// form; batches reserve disjoint ranges of it.
constexpr int BATCH_CONST_BYTES = 60 * 1024;

// Host-side fill of one descriptor (constants converted once, in double).
template <typename R>
void fill_desc_t(void* out, double lam, const Geom& g, const PhysParams& P, const void* cur,
                 const void* other,
                 const void* ref_cur, const void* ref_other, void* uprev, int tiles_x,
                 int tiles_y, int tw_log2, int slot, unsigned step_offset) {
  LatDesc<R> L{};
  L.buf[0] = cur;
  L.buf[1] = other;
  L.ref[0] = ref_cur;
  L.ref[1] = ref_other;
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
  L.tw_log2 = tw_log2;
  L.slot = slot;
  L.step_offset = step_offset;
  L.sround = 0;
  for (int q = 0; q < Q; ++q)
    L.lidc[q] = R(6.0 * wt<double>(q) * g.rho0 * lam *
                  (cx(q) * g.U[0] + cy(q) * g.U[1] + cz(q) * g.U[2]));
  L.C = make_const<R>(P, lam);
  *static_cast<LatDesc<R>*>(out) = L;
}

}  // namespace clbm

#define CLBM_DEFINE_BATCH(SUFFIX, S, R, REF)                                                   \
  namespace clbm {                                                                             \
  __constant__ LatDesc<R> c_lat_##SUFFIX[BATCH_CONST_BYTES / sizeof(LatDesc<R>)];              \
  template <bool CHECK, bool CAP, bool FORCE>                                                  \
  __global__ void __launch_bounds__(256, CAP ? 4 : 1)                                          \
      batch_kernel_##SUFFIX(int base, const int* __restrict__ owner,                           \
                            const unsigned* __restrict__ coord, BatchHeader* hdr, int parity,  \
                            double* acc, int zc) {                                             \
    batch_tiles<S, R, CHECK, FORCE, REF>(                                                      \
        [base](int li) -> const LatDesc<R>& { return c_lat_##SUFFIX[base + li]; }, owner,      \
        coord, hdr, parity, acc, zc);                                                          \
  }                                                                                            \
  cudaError_t launch_batch_##SUFFIX(int base, const int* owner, const unsigned* coord,         \
                                    const void* hdr, int parity, bool check, double* acc,      \
                                    int zc, dim3 block, int grid, cudaStream_t st,             \
                                    cudaStream_t stf) {                                         \
    BatchHeader* H = static_cast<BatchHeader*>(const_cast<void*>(hdr));                        \
    const bool cap = grid < 0;                                                                 \
    if (cap) grid = -grid;                                                                     \
    /* tiles without force on st, tiles with force on stf (an empty range exits at once) */   \
    if (check) {                                                                               \
      if (cap) {                                                                               \
        batch_kernel_##SUFFIX<true, true, false><<<grid, block, 0, st>>>(base, owner, coord, H, parity, acc, zc); \
        batch_kernel_##SUFFIX<true, true, true><<<grid, block, 0, stf>>>(base, owner, coord, H, parity, acc, zc); \
      } else {                                                                                 \
        batch_kernel_##SUFFIX<true, false, false><<<grid, block, 0, st>>>(base, owner, coord, H, parity, acc, zc); \
        batch_kernel_##SUFFIX<true, false, true><<<grid, block, 0, stf>>>(base, owner, coord, H, parity, acc, zc); \
      }                                                                                        \
    } else {                                                                                   \
      if (cap) {                                                                               \
        batch_kernel_##SUFFIX<false, true, false><<<grid, block, 0, st>>>(base, owner, coord, H, parity, acc, zc); \
        batch_kernel_##SUFFIX<false, true, true><<<grid, block, 0, stf>>>(base, owner, coord, H, parity, acc, zc); \
      } else {                                                                                 \
        batch_kernel_##SUFFIX<false, false, false><<<grid, block, 0, st>>>(base, owner, coord, H, parity, acc, zc); \
        batch_kernel_##SUFFIX<false, false, true><<<grid, block, 0, stf>>>(base, owner, coord, H, parity, acc, zc); \
      }                                                                                        \
    }                                                                                          \
    return cudaGetLastError();                                                                 \
  }                                                                                            \
  size_t desc_size_##SUFFIX() { return sizeof(LatDesc<R>); }                                    \
  int desc_capacity_##SUFFIX() { return int(BATCH_CONST_BYTES / sizeof(LatDesc<R>)); }         \
  void fill_desc_##SUFFIX(void* out, const Geom& g, const PhysParams& P, const void* cur,        \
                          const void* other, const void* ref_cur, const void* ref_other,       \
                          void* uprev, int tx, int ty, int twl, int slot, unsigned so) {       \
    /* FP16 storage (F16S, F16R) carries its deviations scaled by 1024 */                    \
    fill_desc_t<R>(out, double(1 << log2_scale<S>()), g, P, cur, other, ref_cur,             \
                   ref_other, uprev, tx, ty, twl, slot, so);                                   \
  }                                                                                            \
  void desc_set_sround_##SUFFIX(void* out, int on) {                                           \
    static_cast<LatDesc<R>*>(out)->sround = on;                                                \
  }                                                                                            \
  cudaError_t upload_desc_##SUFFIX(const void* host, int base, int n) {                        \
    return cudaMemcpyToSymbol(c_lat_##SUFFIX, host, size_t(n) * sizeof(LatDesc<R>),            \
                              size_t(base) * sizeof(LatDesc<R>), cudaMemcpyHostToDevice);      \
  }                                                                                            \
  }
