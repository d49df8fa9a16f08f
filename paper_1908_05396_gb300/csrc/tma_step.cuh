// tma_step.cuh -- the fused step with the upwind populations staged in shared
// memory by the tensor memory accelerator (TMA), for FP32 and FP16 storage.
//
// The lattice is cut into plane tiles of BX x BY nodes (one node per thread),
// numbered in (column, z) order.  CTA b of a persistent grid of G CTAs takes
// tiles b, b + G, b + 2G, ..., which spreads the (slightly slower) face tiles
// evenly over the CTAs.
// For a tile at plane z, direction q needs the box of array q shifted by
// -e_q: one tiled TMA load of BY rows, BX wide (e_qx = 0) or BX + PAD wide
// (e_qx != 0; the box then starts PAD elements early when e_qx = +1, since a
// TMA box must start on a 16-byte boundary in x).  Boxes that leave the
// lattice are zero-filled by the TMA unit; a node on a face replaces the
// directions whose upwind node is outside (face_fix).
//
// NST stages of 19 boxes form a ring.  A stage's loads complete on its "full"
// mbarrier; every warp arrives on its "empty" mbarrier once it has read the
// stage, and the last warp to do so refills it at once with the tile NST
// uses ahead.  Warps never wait for one another, the loads of NST - 1 tiles
// overlap each tile's collisions, and no thread holds registers for loads in
// flight.  The collision and the stores are
// those of step_kernel.
//
// Every mbarrier wait is bounded (about one second).  A CTA whose wait gives
// up sets the error word, waits (again bounded) for the loads it issued, and
// returns.  Later launches see the word and return at once, and the host
// reports the error at the next check.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

// Included by kernels.cuh after the step kernels (StepArgs, pull_face,
// xface_fix, collide, pdl_enter) and before the host launchers.

namespace clbm {

// Shared-memory layout of one stage: 19 boxes, each in a 128-byte aligned slot.
template <typename S, int BX, int BY>
struct TmaTile {
  static constexpr int PAD = 16 / int(sizeof(S));  // elements in 16 bytes
  static constexpr int WB = BX + PAD;              // width of an x-shifted box
  __host__ __device__ static constexpr int width(int q) { return cx(q) ? WB : BX; }
  __host__ __device__ static constexpr int box_bytes(int q) { return BY * width(q) * int(sizeof(S)); }
  __host__ __device__ static constexpr int slot_bytes(int q) { return (box_bytes(q) + 127) / 128 * 128; }
  __host__ __device__ static constexpr int off(int q) {
    int o = 0;
    for (int k = 0; k < q; ++k) o += slot_bytes(k);
    return o;
  }
  __host__ __device__ static constexpr int stage_bytes() { return off(Q); }
  __host__ __device__ static constexpr int tx_bytes() {
    int b = 0;
    for (int k = 0; k < Q; ++k) b += box_bytes(k);
    return b;
  }
  // x origin of the box relative to the tile's x0, and the element of the
  // box row that holds the upwind value of the thread at tx (tx - e_qx
  // relative to the origin)
  __host__ __device__ static constexpr int xorg(int q) { return cx(q) == 1 ? -PAD : 0; }
  __host__ __device__ static constexpr int shift(int q) { return cx(q) == 1 ? PAD - 1 : (cx(q) == -1 ? 1 : 0); }
  static_assert(BX % PAD == 0, "tile x extent must keep every box origin 16-byte aligned");
};

// Work of one launch: tiles ntx x nty per plane, items = ntx * nty * nz
// (< 2^31, checked by the launcher).
struct TmaSched {
  int ntx, nty;
  int items;
  int* err;  // set to 1 by a CTA whose pipeline wait gave up
};

constexpr unsigned long long TMA_WAIT_NS = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity to complete; false after ~limit ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit) return false;
  }
}
// One tiled 4-D box (x, y, z, q) from global memory into shared memory,
// completing `bytes` on the mbarrier.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// For a node of the TMA kernel whose d[] holds the upwind value wherever the
// upwind node exists (and anything where it does not): replace the
// directions whose upwind node lies outside the lattice, by the rules of
// pull_face -- the periodic wrap, or else bounce-back from the node's own
// opposite population, plus the lid term when a crossed face is the lid.
// Interior nodes return at the first test.
template <typename S>
__device__ __forceinline__ void face_fix(const StepArgs<S, float>& a, int x, int y, int z, int i,
                                         float (&d)[Q]) {
  const bool fx0 = x == 0, fx1 = x == a.nx - 1, fy0 = y == 0, fy1 = y == a.ny - 1;
  const bool fz0 = z == 0, fz1 = z == a.nz - 1;
  if (!(fx0 || fx1 || fy0 || fy1 || fz0 || fz1)) return;
  const unsigned fb = a.facebits;
#pragma unroll
  for (int q = 1; q < Q; ++q) {
    const bool ox = (cx(q) == 1 && fx0) || (cx(q) == -1 && fx1);
    const bool oy = (cy(q) == 1 && fy0) || (cy(q) == -1 && fy1);
    const bool oz = (cz(q) == 1 && fz0) || (cz(q) == -1 && fz1);
    if (!(ox || oy || oz)) continue;
    // kind of each crossed face (faces -x, +x, -y, +y, -z, +z, two bits each)
    const int kx = ox ? int((fb >> (cx(q) == 1 ? 0 : 2)) & 3u) : int(BC_PERIODIC);
    const int ky = oy ? int((fb >> (cy(q) == 1 ? 4 : 6)) & 3u) : int(BC_PERIODIC);
    const int kz = oz ? int((fb >> (cz(q) == 1 ? 8 : 10)) & 3u) : int(BC_PERIODIC);
    if (kx != BC_PERIODIC || ky != BC_PERIODIC || kz != BC_PERIODIC) {
      const bool lid = kx == BC_LID || ky == BC_LID || kz == BC_LID;
      d[q] = Codec<S, float>::dec(a.src[opp(q) * a.qstride + i], 1.0f) + (lid ? a.lidc[q] : 0.0f);
    } else {
      int j = i;
      if (ox) j += cx(q) == 1 ? a.nx : -a.nx;
      if (oy) j += cy(q) == 1 ? a.ny * a.pitch : -a.ny * a.pitch;
      if (oz) j += cz(q) == 1 ? a.nz * a.plane : -a.nz * a.plane;
      d[q] = Codec<S, float>::dec(a.srcq[q][j], 1.0f);
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// NP = 1: one node per thread (BX x BY threads).  NP = 2: BX x BY/2 threads,
// each owning rows 2 ty and 2 ty + 1 of the tile at the same x, collided as a
// pair with packed FP32 arithmetic (V2), as in step2_kernel.
template <typename S, int BX, int BY, int NP, int NST, int MINB, bool FORCE>
__global__ void __launch_bounds__(BX * BY / NP, MINB)
    step_tma_kernel(const __grid_constant__ CUtensorMap mapA,
                    const __grid_constant__ CUtensorMap mapB, const StepArgs<S, float> a,
                    const TmaSched ts) {
  using T = TmaTile<S, BX, BY>;
  static_assert(NP == 1 || (NP == 2 && BY % 2 == 0), "two nodes per thread need an even BY");
  constexpr int NW = BX * BY / NP / 32;
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ __align__(8) uint64_t full[NST];   // stage loaded (TMA bytes landed)
  __shared__ __align__(8) uint64_t empty[NST];  // stage read by every warp
  __shared__ int4 meta[NST];   // per stage: item, x0, y0, z (item >= items: no more work)
  __shared__ int nread[NST];   // warps done with the stage's current use
  __shared__ int used[NST];    // the use (k) last put into the stage
  pdl_enter();
  // an earlier launch gave up: do nothing until the host has seen it
  if (*reinterpret_cast<volatile const int*>(ts.err)) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BX + tx;
  const int lane = tid & 31;
  const int G = int(gridDim.x);
  // stage 0 at the first 128-byte boundary of the dynamic shared memory
  // (the launch adds 128 bytes for this)
  const uint32_t sbase = (smem_u32(tsm) + 127u) & ~127u;
  const unsigned char* sgen = tsm + (sbase - smem_u32(tsm));
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), NW);
      nread[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // Use k of this CTA is item blockIdx.x + k G (stage k % NST).  issue(): the
  // 19 boxes of use k into its stage, or an empty phase past the last item.
  auto issue = [&](int k) {
    const int s = k % NST;
    const int t = int(blockIdx.x) + k * G;
    const uint32_t bar = smem_u32(&full[s]);
    used[s] = k;
    if (t < ts.items) {
      const int z = t % a.nz;
      const int col = t / a.nz;
      const int x0 = (col % ts.ntx) * BX, y0 = (col / ts.ntx) * BY;
      meta[s] = make_int4(t, x0, y0, z);
      const uint32_t base = sbase + uint32_t(s) * T::stage_bytes();
      mbar_expect_tx(bar, T::tx_bytes());
#pragma unroll
      for (int q = 0; q < Q; ++q)
        tma_load_4d(base + T::off(q), cx(q) ? &mapB : &mapA, x0 + T::xorg(q), y0 - cy(q),
                    z - cz(q), q, bar);
    } else {
      meta[s] = make_int4(t, 0, 0, 0);
      mbar_arrive(bar);
    }
  };
  if (tid == 0)
    for (int k = 0; k < NST; ++k) issue(k);

  bool ok = true;
  for (int k = 0;; ++k) {
    const int s = k % NST;
    const uint32_t par = uint32_t(k / NST) & 1u;
    // warp-uniform outcome of the wait
    if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&full[s]), par, TMA_WAIT_NS))) {
      ok = false;
      break;
    }
    const int4 m = meta[s];  // after the wait (its asm clobbers memory)
    const bool work = m.x < ts.items;  // the same for every thread
    const int x = m.y + tx, y = m.z + NP * ty, z = m.w;
    const bool active = work && x < a.nx && y < a.ny;
    const bool activeB = NP == 2 && active && y + 1 < a.ny;
    const unsigned char* st = sgen + s * T::stage_bytes();
    float d[Q], dB[NP == 2 ? Q : 1];
    if (active) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
        d[q] = Codec<S, float>::dec(
            reinterpret_cast<const S*>(st + T::off(q))[NP * ty * T::width(q) + tx + T::shift(q)],
            1.0f);
      if constexpr (NP == 2) {
        // row 2 ty + 1 is inside the box (zero-filled past the lattice)
#pragma unroll
        for (int q = 0; q < Q; ++q)
          dB[q] = Codec<S, float>::dec(reinterpret_cast<const S*>(
                                           st + T::off(q))[(2 * ty + 1) * T::width(q) + tx +
                                                           T::shift(q)],
                                       1.0f);
      }
    }
    __syncwarp();
    if (lane == 0 && work) {
      // Release the stage; the last warp to do so refills it at once with
      // use k + NST (its empty phase is then complete: the wait acquires
      // every warp's reads before the TMA overwrites them).
      mbar_arrive(smem_u32(&empty[s]));
      if (atomicAdd(&nread[s], 1) == NW - 1) {
        nread[s] = 0;
        if (mbar_wait(smem_u32(&empty[s]), par, TMA_WAIT_NS)) issue(k + NST);
        else ok = false;
      }
    }
    if (!work) break;
    if (active) {
      const int i = z * a.plane + y * a.pitch + x;
      face_fix(a, x, y, z, i, d);
      if constexpr (NP == 1) {
        NodeOut<float> o;
        collide<float, FORCE, pair_out<S>(), log2_scale<S>()>(a.C, d, o);
#pragma unroll
        for (int q = 0; q < Q; ++q) a.dstq[q][i] = Codec<S, float>::enc(d[q], 1.0f);
      } else {
        const int iB = i + a.pitch;
        if (activeB) face_fix(a, x, y + 1, z, iB, dB);
        V2 p[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) p[q] = V2(d[q], dB[q]);
        NodeOut<V2> o;
        collide<V2, FORCE, pair_out<S>(), log2_scale<S>()>(a.C, p, o);
#pragma unroll
        for (int q = 0; q < Q; ++q) a.dstq[q][i] = Codec<S, float>::enc(lane0(p[q]), 1.0f);
        if (activeB) {
#pragma unroll
          for (int q = 0; q < Q; ++q) a.dstq[q][iB] = Codec<S, float>::enc(lane1(p[q]), 1.0f);
        }
      }
    }
    if (!__all_sync(0xffffffffu, ok)) break;  // the refill of this warp failed
  }
  // A wait gave up somewhere: record it and let thread 0 wait (bounded) for
  // the last use put into each stage before the shared memory goes.
  if (__syncthreads_or(!ok) && tid == 0) {
    atomicExch(ts.err, 1);
    for (int s = 0; s < NST; ++s)
      mbar_wait(smem_u32(&full[s]), uint32_t(used[s] / NST) & 1u, TMA_WAIT_NS);
  }
}

// ---- host side ---------------------------------------------------------------
inline PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <typename S> constexpr CUtensorMapDataType tma_dtype();
template <> constexpr CUtensorMapDataType tma_dtype<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> constexpr CUtensorMapDataType tma_dtype<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

// The 4-D view (x < nx, y < ny, z < nz, q < 19) of a population buffer with a
// box of `boxw` x BY x 1 x 1 elements.
template <typename S>
cudaError_t tma_map(CUtensorMap* m, const void* buf, const Geom& g, int boxw, int by) {
  auto fn = tma_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {cuuint64_t(g.nx), cuuint64_t(g.ny), cuuint64_t(g.nz), cuuint64_t(Q)};
  const cuuint64_t strides[3] = {cuuint64_t(g.pitch) * sizeof(S), cuuint64_t(g.plane) * sizeof(S),
                                 cuuint64_t(g.qstride) * sizeof(S)};
  const cuuint32_t box[4] = {cuuint32_t(boxw), cuuint32_t(by), 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(m, tma_dtype<S>(), 4, const_cast<void*>(buf), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Launch one TMA-staged step: tiles BX x BY, NP nodes per thread, NST
// stages, MINB CTAs per SM (the register budget).
template <typename S, int BX, int BY, int NP, int NST, int MINB>
cudaError_t launch_tma_shape(const StepArgs<S, float>& a, const void* src, const Geom& g,
                             bool force, int* err, cudaStream_t st) {
  using T = TmaTile<S, BX, BY>;
  CUtensorMap mA, mB;
  cudaError_t e = tma_map<S>(&mA, src, g, BX, BY);
  if (e == cudaSuccess) e = tma_map<S>(&mB, src, g, T::WB, BY);
  if (e != cudaSuccess) return e;
  const size_t smem = size_t(NST) * T::stage_bytes() + 128;
  auto kernel = force ? step_tma_kernel<S, BX, BY, NP, NST, MINB, true>
                      : step_tma_kernel<S, BX, BY, NP, NST, MINB, false>;
  // per kernel and device: the shared-memory opt-in and the resident CTAs
  static int nres[2][64] = {};
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int& nr = nres[force ? 1 : 0][dev];
  if (nr == 0) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               int(cudaSharedmemCarveoutMaxShared));
    int per_sm = 0, nsm = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BX * BY / NP, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    nr = per_sm * nsm;
  }
  TmaSched ts;
  ts.ntx = (g.nx + BX - 1) / BX;
  ts.nty = (g.ny + BY - 1) / BY;
  const long long items = (long long)ts.ntx * ts.nty * g.nz;
  if (items >= (1ll << 31)) return cudaErrorInvalidValue;
  ts.items = int(items);
  ts.err = err;
  const int grid = ts.items < nr ? ts.items : nr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(BX, BY / NP);
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
  e = cudaLaunchKernelEx(&cfg, kernel, mA, mB, a, ts);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The TMA shapes, selected by npt = TMA_NPT + 32 v; their blocks are
// tma_bx(v) x tma_by(v) (launch.h).
template <typename S>
cudaError_t launch_step_tma(const StepArgs<S, float>& a, const void* src, const Geom& g,
                            bool force, int v, int* err, cudaStream_t st) {
  switch (v) {
    case 0: return launch_tma_shape<S, 64, 4, 1, 2, 3>(a, src, g, force, err, st);
    case 1: return launch_tma_shape<S, 128, 2, 1, 2, 3>(a, src, g, force, err, st);
    case 2: return launch_tma_shape<S, 32, 8, 1, 2, 3>(a, src, g, force, err, st);
    case 3: return launch_tma_shape<S, 64, 4, 1, 3, 3>(a, src, g, force, err, st);
    case 4: return launch_tma_shape<S, 32, 4, 1, 2, 6>(a, src, g, force, err, st);
    case 5: return launch_tma_shape<S, 64, 2, 1, 2, 6>(a, src, g, force, err, st);
    case 6: return launch_tma_shape<S, 64, 4, 2, 2, 3>(a, src, g, force, err, st);
    case 7: return launch_tma_shape<S, 32, 8, 2, 2, 3>(a, src, g, force, err, st);
    case 8: return launch_tma_shape<S, 64, 4, 2, 2, 4>(a, src, g, force, err, st);
    case 9: return launch_tma_shape<S, 128, 2, 2, 2, 3>(a, src, g, force, err, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace clbm
