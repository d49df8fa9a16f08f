// inplace.cuh -- the fused step with ONE population buffer (in-place
// streaming), for the FP64, FP32 and F16S forms.
//
// Two kinds of step alternate, and the buffer A[q][node] holds one of two
// layouts between steps:
//   layout 0 ("swapped"): A[opp(q)][x] = f~_q(x), the post-collision value of
//       node x in direction q kept in its opposite slot;
//   layout 1 ("streamed"): A[q][x] = f~_q(x - e_q), the value node x pulls in
//       direction q (or, where x - e_q is beyond a wall or the lid, the
//       bounced value f~_opp(q)(x)).
// A neighbour step (layout 0 -> 1) reads f_q(x) from A[opp(q)][x - e_q],
// collides and writes f~_q(x) to A[q][x + e_q]; a local step (layout 1 -> 0)
// reads A[q][x], collides and writes f~_q(x) to A[opp(q)][x].  In both, the
// 19 slots a node reads are exactly the 19 it writes, so one thread per node
// updates the buffer in place with no race.  Walls and the lid follow the
// pull rules of the two-buffer step (pull_face): a value whose source or
// destination crosses a non-periodic face stays at the node in the opposite
// slot (halfway bounce-back), the lid term 6 w_q rho0 (e_q . U) is added when
// it is read (so stored values are the exact post-collision ones), and
// periodic faces wrap.  Every step computes exactly what the two-buffer step
// computes, with the same bytes per update and half the memory.
#pragma once

namespace clbm {

// Where the node at (x, y, z) crosses a face going one step along -e_q
// (up = true, the upwind side) or +e_q (the downstream side): for each axis
// whether it crosses, the kind of the crossed face, and the index shift that
// wraps a periodic crossing.
struct Crossing {
  bool any, bounce, lid;
  int wrap;  // index offset of the periodic wrap (when !bounce)
};

template <int q, bool UP>
__device__ __forceinline__ Crossing crossing(int x, int y, int z, int nx, int ny, int nz,
                                             int pitch, int plane, unsigned fb) {
  constexpr int s = UP ? -1 : 1;                  // step along s * e_q
  constexpr int ex = s * cx(q), ey = s * cy(q), ez = s * cz(q);
  const bool ox = (ex == -1 && x == 0) || (ex == 1 && x == nx - 1);
  const bool oy = (ey == -1 && y == 0) || (ey == 1 && y == ny - 1);
  const bool oz = (ez == -1 && z == 0) || (ez == 1 && z == nz - 1);
  // faces -x, +x, -y, +y, -z, +z: two bits each
  const int kx = ox ? int((fb >> (ex == -1 ? 0 : 2)) & 3u) : int(BC_PERIODIC);
  const int ky = oy ? int((fb >> (ey == -1 ? 4 : 6)) & 3u) : int(BC_PERIODIC);
  const int kz = oz ? int((fb >> (ez == -1 ? 8 : 10)) & 3u) : int(BC_PERIODIC);
  Crossing c;
  c.any = ox || oy || oz;
  c.bounce = kx != BC_PERIODIC || ky != BC_PERIODIC || kz != BC_PERIODIC;
  c.lid = kx == BC_LID || ky == BC_LID || kz == BC_LID;
  c.wrap = (ox ? -ex * nx : 0) + (oy ? -ey * ny * pitch : 0) + (oz ? -ez * nz * plane : 0);
  return c;
}

// Pre-collision values of node i in layout L (any node, faces included).
template <typename S, typename R, int L, int q>
__device__ __forceinline__ R aa_read_one(const S* A, int64_t qs, int x, int y, int z, int i,
                                         int nx, int ny, int nz, int pitch, int plane,
                                         unsigned fb, R lid) {
  const Crossing c = crossing<q, true>(x, y, z, nx, ny, nz, pitch, plane, fb);
  if (L == 1) {  // streamed layout: own slot; bounced values get the lid term
    const R v = Codec<S, R>::dec(A[q * qs + i], R(1));
    return (c.any && c.bounce && c.lid) ? v + lid : v;
  }
  // swapped layout: the upwind node's opposite slot, or the own slot q
  // (bounce: f~_opp(q)(x) sits in slot opp(opp(q)) = q)
  if (c.any && c.bounce) {
    const R v = Codec<S, R>::dec(A[q * qs + i], R(1));
    return c.lid ? v + lid : v;
  }
  const int up = i - (cz(q) * plane + cy(q) * pitch + cx(q)) + (c.any ? c.wrap : 0);
  return Codec<S, R>::dec(A[opp(q) * qs + up], R(1));
}

template <typename S, typename R, int L, int q = 0>
__device__ __forceinline__ void aa_read(const S* A, int64_t qs, int x, int y, int z, int i,
                                        int nx, int ny, int nz, int pitch, int plane,
                                        unsigned fb, const R* lidc, R (&d)[Q]) {
  d[q] = aa_read_one<S, R, L, q>(A, qs, x, y, z, i, nx, ny, nz, pitch, plane, fb, lidc[q]);
  if constexpr (q + 1 < Q) aa_read<S, R, L, q + 1>(A, qs, x, y, z, i, nx, ny, nz, pitch, plane, fb, lidc, d);
}

// Post-collision values of node i written for the next layout: after a
// neighbour step (layout 1) to the downstream node's slot q, or back into
// the own opposite slot where the downstream side crosses a wall or the lid.
template <typename S, typename R, int q = 0>
__device__ __forceinline__ void aa_write_streamed(S* A, int64_t qs, int x, int y, int z, int i,
                                                  int nx, int ny, int nz, int pitch, int plane,
                                                  unsigned fb, const R (&d)[Q]) {
  const Crossing c = crossing<q, false>(x, y, z, nx, ny, nz, pitch, plane, fb);
  if (c.any && c.bounce) {
    A[opp(q) * qs + i] = Codec<S, R>::enc(d[q], R(1));
  } else {
    const int dn = i + (cz(q) * plane + cy(q) * pitch + cx(q)) + (c.any ? c.wrap : 0);
    A[q * qs + dn] = Codec<S, R>::enc(d[q], R(1));
  }
  if constexpr (q + 1 < Q) aa_write_streamed<S, R, q + 1>(A, qs, x, y, z, i, nx, ny, nz, pitch, plane, fb, d);
}

// Lid terms of the bounced values in the streamed layout (local step).
template <typename S, typename R, int q = 1>
__device__ __forceinline__ void aa_lid_fix(int x, int y, int z, int nx, int ny, int nz, int pitch,
                                           int plane, unsigned fb, const R* lidc, R (&d)[Q]) {
  const Crossing c = crossing<q, true>(x, y, z, nx, ny, nz, pitch, plane, fb);
  if (c.any && c.bounce && c.lid) d[q] += lidc[q];
  if constexpr (q + 1 < Q) aa_lid_fix<S, R, q + 1>(x, y, z, nx, ny, nz, pitch, plane, fb, lidc, d);
}

// One in-place step.  LIN is the layout the step reads: 0 -> neighbour step
// (srcq[q] = A + opp(q) qs - off(q), dstq[q] = A + q qs + off(q)), 1 -> local
// step (srcq[q] = A + q qs, dstq[q] = A + opp(q) qs); a.src is the buffer A.
// Nodes off the y and z faces take the direct path (the x-face lanes fix
// their crossing directions); nodes on a y or z face resolve every direction.
template <typename S, typename R, int LIN, bool FORCE, bool CHECK, bool CAP>
__global__ void __launch_bounds__(256, CAP ? 4 : 1) step_aa_kernel(const StepArgs<S, R> a) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = a.zrev ? a.nz - 1 - int(blockIdx.z) : int(blockIdx.z);  // as step_kernel
  const bool active = x < a.nx && y < a.ny;
  if (!CHECK && !active) return;
  double du2 = 0.0, uu = 0.0, dr = 0.0;
  int bad = 0;
  if (active) {
    const int i = z * a.plane + y * a.pitch + x;
    S* A = const_cast<S*>(a.src);
    const bool inyz = y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1;
    const bool xface = x == 0 || x == a.nx - 1;
    const int kl = a.facebits & 3, kr = (a.facebits >> 2) & 3;
    R d[Q];
    if (LIN == 1) {
#pragma unroll
      for (int q = 0; q < Q; ++q) d[q] = Codec<S, R>::dec(a.srcq[q][i], R(1));
      if (!inyz || xface)
        aa_lid_fix<S, R>(x, y, z, a.nx, a.ny, a.nz, a.pitch, a.plane, a.facebits, a.lidc, d);
    } else if (inyz) {
#pragma unroll
      for (int q = 0; q < Q; ++q) d[q] = Codec<S, R>::dec(a.srcq[q][i], R(1));
      if (xface) {
#pragma unroll
        for (int q = 1; q < Q; ++q) {
          const bool left = cx(q) == 1 && x == 0, right = cx(q) == -1 && x == a.nx - 1;
          if (left || right) {
            const int k = left ? kl : kr;
            if (k == BC_PERIODIC)
              d[q] = Codec<S, R>::dec(a.srcq[q][left ? i + a.nx : i - a.nx], R(1));
            else
              d[q] = Codec<S, R>::dec(A[q * a.qstride + i], R(1)) +
                     (k == BC_LID ? a.lidc[q] : R(0));
          }
        }
      }
    } else {
      aa_read<S, R, 0>(A, a.qstride, x, y, z, i, a.nx, a.ny, a.nz, a.pitch, a.plane, a.facebits,
                       a.lidc, d);
    }
    NodeOut<R> o;
    collide<R, FORCE, pair_out<S>(), log2_scale<S>()>(a.C, d, o);
    if (LIN == 1) {
#pragma unroll
      for (int q = 0; q < Q; ++q) a.dstq[q][i] = Codec<S, R>::enc(d[q], R(1));
    } else if (inyz) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        // downstream across an x face: wrap, or keep at the node (bounce)
        const bool right = cx(q) == 1 && x == a.nx - 1, left = cx(q) == -1 && x == 0;
        const S v = Codec<S, R>::enc(d[q], R(1));
        if (right || left) {
          const int k = right ? kr : kl;
          if (k == BC_PERIODIC) a.dstq[q][right ? i - a.nx : i + a.nx] = v;
          else A[opp(q) * a.qstride + i] = v;
        } else {
          a.dstq[q][i] = v;
        }
      }
    } else {
      aa_write_streamed<S, R>(A, a.qstride, x, y, z, i, a.nx, a.ny, a.nz, a.pitch, a.plane,
                              a.facebits, d);
    }
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

// rho, u and |gamma_dot| of the next collision, from either layout.
template <typename S, typename R, int L, bool FORCE>
__global__ void __launch_bounds__(256) fields_aa_kernel(const S* __restrict__ A, Geom g,
                                                        PhysParams P, double* rho, double* u,
                                                        double* gd) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const CollideConst<R> C = make_const<R>(P, double(1 << log2_scale<S>()));
  R lidc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q)
    lidc[q] = R(6.0 * wt<double>(q) * g.rho0 * double(1 << log2_scale<S>()) *
                (cx(q) * g.U[0] + cy(q) * g.U[1] + cz(q) * g.U[2]));
  const int i = z * int(g.plane) + y * g.pitch + x;
  R d[Q];
  aa_read<S, R, L>(A, g.qstride, x, y, z, i, g.nx, g.ny, g.nz, g.pitch, int(g.plane), g.facebits,
                   lidc, d);
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

// The post-collision populations f~_q(x) (the state the two-buffer form
// stores), from either layout: layout 0 holds them in the opposite slots;
// layout 1 holds them at the downstream node, or at the node itself in the
// opposite slot where the downstream side is a wall or the lid.
template <typename S>
__global__ void export_aa_kernel(const S* __restrict__ A, Geom g, double rho0, double inv_scale,
                                 int layout, double* __restrict__ out) {
  const int64_t N = int64_t(g.nx) * g.ny * g.nz;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= N * Q) return;
  const int q = int(t / N);
  const int64_t k = t - int64_t(q) * N;
  const int x = int(k % g.nx), y = int((k / g.nx) % g.ny), z = int(k / (int64_t(g.nx) * g.ny));
  const int64_t i = int64_t(z) * g.plane + int64_t(y) * g.pitch + x;
  int64_t j = int64_t(c_opp[q]) * g.qstride + i;  // layout 0, or a bounced value
  if (layout == 1) {
    const int ex = c_ex[q], ey = c_ey[q], ez = c_ez[q];
    const bool ox = (ex == -1 && x == 0) || (ex == 1 && x == g.nx - 1);
    const bool oy = (ey == -1 && y == 0) || (ey == 1 && y == g.ny - 1);
    const bool oz = (ez == -1 && z == 0) || (ez == 1 && z == g.nz - 1);
    const int kx = ox ? int((g.facebits >> (ex == -1 ? 0 : 2)) & 3u) : int(BC_PERIODIC);
    const int ky = oy ? int((g.facebits >> (ey == -1 ? 4 : 6)) & 3u) : int(BC_PERIODIC);
    const int kz = oz ? int((g.facebits >> (ez == -1 ? 8 : 10)) & 3u) : int(BC_PERIODIC);
    if (kx == BC_PERIODIC && ky == BC_PERIODIC && kz == BC_PERIODIC) {
      const int xd = ox ? x + ex - ex * g.nx : x + ex, yd = oy ? y + ey - ey * g.ny : y + ey,
                zd = oz ? z + ez - ez * g.nz : z + ez;
      j = int64_t(q) * g.qstride + int64_t(zd) * g.plane + int64_t(yd) * g.pitch + xd;
    }
  }
  out[t] = double(Codec<S, double>::dec(A[j], inv_scale)) * inv_scale + wt<double>(q) * rho0;
}

// Import a state f~ into layout 0.
template <typename S>
__global__ void import_aa_kernel(const double* __restrict__ in, Geom g, double rho0,
                                 double inv_scale, S* __restrict__ A) {
  const int64_t N = int64_t(g.nx) * g.ny * g.nz;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= N * Q) return;
  const int q = int(t / N);
  const int64_t k = t - int64_t(q) * N;
  const int x = int(k % g.nx), y = int((k / g.nx) % g.ny), z = int(k / (int64_t(g.nx) * g.ny));
  const int64_t i = int64_t(z) * g.plane + int64_t(y) * g.pitch + x;
  A[int64_t(c_opp[q]) * g.qstride + i] =
      Codec<S, double>::enc((in[t] - wt<double>(q) * rho0) / inv_scale, inv_scale);
}

// ---- host-side launchers ------------------------------------------------------
template <typename S, typename R>
cudaError_t launch_step_aa_t(void* buf, const Geom& g, const PhysParams& P, const CheckBufs& cb,
                             bool check, dim3 block, int npt, int layout, cudaStream_t st) {
  StepArgs<S, R> a;
  S* A = static_cast<S*>(buf);
  const uintptr_t base = reinterpret_cast<uintptr_t>(A);
  a.zrev = 0;  // an alternating sweep (either parity) measured 2 % slower here
  for (int q = 0; q < Q; ++q) {
    const int64_t off = int64_t(cz(q)) * g.plane + int64_t(cy(q)) * g.pitch + cx(q);
    // address arithmetic through integers: a shifted base may lie outside the
    // buffer; only base + i of a node whose partner node exists is used
    const int64_t sq = layout == 0 ? int64_t(opp(q)) * g.qstride - off : int64_t(q) * g.qstride;
    const int64_t dq = layout == 0 ? int64_t(q) * g.qstride + off : int64_t(opp(q)) * g.qstride;
    a.srcq[q] = reinterpret_cast<const S*>(base + sq * int64_t(sizeof(S)));
    a.dstq[q] = reinterpret_cast<S*>(base + dq * int64_t(sizeof(S)));
    a.lidc[q] = R(6.0 * wt<double>(q) * g.rho0 * double(1 << log2_scale<S>()) *
                  (cx(q) * g.U[0] + cy(q) * g.U[1] + cz(q) * g.U[2]));
  }
  a.src = A;
  a.qstride = g.qstride;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.pitch = g.pitch;
  a.plane = int(g.plane);
  a.facebits = g.facebits;
  a.C = make_const<R>(P, double(1 << log2_scale<S>()));
  a.cb = cb;
  const bool cap = (npt & 4) != 0;
  const dim3 grid((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, g.nz);
  cudaError_t e = cudaSuccess;
#define CLBM_AA_LAUNCH(L, F, C_)                                                                \
  e = cap ? pdl_launch(step_aa_kernel<S, R, L, F, C_, true>, grid, block, st, a)                \
          : pdl_launch(step_aa_kernel<S, R, L, F, C_, false>, grid, block, st, a)
  if (layout == 0) {
    if (P.has_force) { if (check) CLBM_AA_LAUNCH(0, true, true); else CLBM_AA_LAUNCH(0, true, false); }
    else { if (check) CLBM_AA_LAUNCH(0, false, true); else CLBM_AA_LAUNCH(0, false, false); }
  } else {
    if (P.has_force) { if (check) CLBM_AA_LAUNCH(1, true, true); else CLBM_AA_LAUNCH(1, true, false); }
    else { if (check) CLBM_AA_LAUNCH(1, false, true); else CLBM_AA_LAUNCH(1, false, false); }
  }
#undef CLBM_AA_LAUNCH
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_fields_aa_t(const void* buf, const Geom& g, const PhysParams& P, int layout,
                               double* rho, double* u, double* gd, cudaStream_t st) {
  const dim3 block(32, 4);
  const dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
  const S* A = static_cast<const S*>(buf);
  if (layout == 0) {
    if (P.has_force) fields_aa_kernel<S, R, 0, true><<<grid, block, 0, st>>>(A, g, P, rho, u, gd);
    else fields_aa_kernel<S, R, 0, false><<<grid, block, 0, st>>>(A, g, P, rho, u, gd);
  } else {
    if (P.has_force) fields_aa_kernel<S, R, 1, true><<<grid, block, 0, st>>>(A, g, P, rho, u, gd);
    else fields_aa_kernel<S, R, 1, false><<<grid, block, 0, st>>>(A, g, P, rho, u, gd);
  }
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_export_aa_t(const void* buf, const Geom& g, double rho0, double inv_scale,
                               int layout, double* out, cudaStream_t st) {
  const int64_t total = int64_t(g.nx) * g.ny * g.nz * Q;
  const int b = 256;
  export_aa_kernel<S><<<unsigned((total + b - 1) / b), b, 0, st>>>(
      static_cast<const S*>(buf), g, rho0, inv_scale, layout, out);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_import_aa_t(const double* in, const Geom& g, double rho0, double inv_scale,
                               void* buf, cudaStream_t st) {
  const int64_t total = int64_t(g.nx) * g.ny * g.nz * Q;
  const int b = 256;
  import_aa_kernel<S><<<unsigned((total + b - 1) / b), b, 0, st>>>(in, g, rho0, inv_scale,
                                                                   static_cast<S*>(buf));
  return cudaGetLastError();
}

}  // namespace clbm

// Defines the in-place launchers of launch.h for storage type S, math type R.
#define CLBM_DEFINE_AA(SUFFIX, S, R)                                                           \
  namespace clbm {                                                                             \
  cudaError_t launch_step_aa_##SUFFIX(void* buf, const Geom& g, const PhysParams& P,           \
                                      const CheckBufs& cb, bool check, dim3 block, int npt,    \
                                      int layout, cudaStream_t st) {                           \
    return launch_step_aa_t<S, R>(buf, g, P, cb, check, block, npt, layout, st);               \
  }                                                                                            \
  cudaError_t launch_fields_aa_##SUFFIX(const void* buf, const Geom& g, const PhysParams& P,   \
                                        int layout, double* rho, double* u, double* gd,        \
                                        cudaStream_t st) {                                     \
    return launch_fields_aa_t<S, R>(buf, g, P, layout, rho, u, gd, st);                        \
  }                                                                                            \
  cudaError_t launch_export_aa_##SUFFIX(const void* buf, const Geom& g, double rho0,           \
                                        double inv_scale, int layout, double* out,             \
                                        cudaStream_t st) {                                     \
    return launch_export_aa_t<S>(buf, g, rho0, inv_scale, layout, out, st);                    \
  }                                                                                            \
  cudaError_t launch_import_aa_##SUFFIX(const double* in, const Geom& g, double rho0,          \
                                        double inv_scale, void* buf, cudaStream_t st) {        \
    return launch_import_aa_t<S>(in, g, rho0, inv_scale, buf, st);                             \
  }                                                                                            \
  }
