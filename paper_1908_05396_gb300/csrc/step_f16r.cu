// step_f16r.cu -- kernels of the F16R storage form: FP16 populations stored
// relative to the writing node's first-order equilibrium.
//
// The deviations are carried scaled by lam = 1024 (as in the F16S form, with
// the factor folded into the collision's constants).  Each node keeps a
// reference (lam (rho - rho0), lam 3 rho u) of its last collision as four
// FP16 values next to its populations, and stores
//     s_q = fp16( lam ( f~_q - w_q rho0 ) - r_q ),
//     r_q = w_q [ dr + e_q . v ],  (dr, v) the reference,
// which removes the rest value and the first-order (velocity) part of the
// equilibrium, the largest parts of f~, before FP16 rounding (stochastic in
// the step kernels, see enc16_sr2).  A reader decodes with the reference of
// the node that wrote the value: the upwind neighbour for a streamed value,
// itself for a bounced one.  Both sides use the reference exactly as stored,
// so decoding undoes the encoding up to the FP16 rounding of the small
// remainder (and one FP32 rounding).  A reference is read by 19 readers, one
// 64-bit load each: in FP16 the 19 loads of a node need half the registers in
// flight (and half the L1/L2 traffic) of FP32 references.
// The reference arrays are double-buffered with the populations.
#include "batch.cuh"
#include "sround.cuh"

namespace clbm {
namespace {

// The back-transform of the collision: unforced, the populations are rebuilt
// from the pair values (the inputs die early, which frees registers; the FP16
// rounding noise of the stores lies far above the FP32 roundings of the
// rebuild); with a body force, one correction per population, which keeps a
// weak force's increments to one rounding (rebuilt from the pairs, a forced
// channel's velocity drifted by 1e-3 against FP64).
constexpr int LOG2LAM = 10;  // log2 of the scale of the carried deviations
constexpr float LAM = float(1 << LOG2LAM);
static_assert(double(1 << LOG2LAM) == F16_SCALE, "one FP16 storage scale");

struct Ref4 {
  float dr, vx, vy, vz;  // lam (rho - rho0) and v = lam 3 rho u, as stored (FP16)
};

__device__ __forceinline__ Ref4 ref_load(const uint2* p) {
  const uint2 v = *p;
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
  return {a.x, a.y, b.x, b.y};
}

// The reference of a node with density rho = rho0 + drho and velocity u,
// rounded to FP16 for storage; r receives the rounded values.
__device__ __forceinline__ uint2 ref_make(float drho, float rho, float ux, float uy, float uz,
                                          Ref4& r) {
  const float r3 = (3.0f * LAM) * rho;
  const __half2 a = __floats2half2_rn(LAM * drho, r3 * ux), b = __floats2half2_rn(r3 * uy, r3 * uz);
  const float2 fa = __half22float2(a), fb = __half22float2(b);
  r = {fa.x, fa.y, fb.x, fb.y};
  uint2 v;
  v.x = *reinterpret_cast<const unsigned*>(&a);
  v.y = *reinterpret_cast<const unsigned*>(&b);
  return v;
}

// First-order equilibrium deviation of direction q about the reference,
// lam w_q [drho + 3 rho (e_q . u)]: the stored v = lam 3 rho u saves the
// product per direction.
__device__ __forceinline__ float ref_term(int q, const Ref4& r) {
  const float ev = float(cx(q)) * r.vx + float(cy(q)) * r.vy + float(cz(q)) * r.vz;
  return wt<float>(q) * (r.dr + ev);
}

__device__ __forceinline__ float dec16(__half v) { return __half2float(v); }
__device__ __forceinline__ __half enc16(float v) { return __float2half_rn(v); }

// Store the 19 post-collision remainders of node i with stochastic rounding,
// two directions per conversion.
template <typename Dst>
__device__ __forceinline__ void store_sr(Dst&& dst_q, const float (&d)[Q], const Ref4& rr,
                                         uint32_t state) {
#pragma unroll
  for (int q = 0; q < Q; q += 2) {
    const float a = d[q] - ref_term(q, rr);
    const float b = q + 1 < Q ? d[q + 1] - ref_term(q + 1 < Q ? q + 1 : q, rr) : 0.0f;
    __half hi, lo;
    enc16_sr2(a, b, state, hi, lo);
    dst_q(q) = hi;
    if (q + 1 < Q) dst_q(q + 1) = lo;
  }
}

struct RefArgs {
  const uint2* refq[Q];  // refq[q][i]: reference of the upwind neighbour of node i
  const uint2* ref_src;  // references of the source step
  uint2* ref_dst;        // references written by this step
  unsigned step;         // the lattice's steps done before this one
};

// Pull of all 19 directions into node (x, y, z) with index i, for a node on
// any face, by the face rules of pull_face; each value is decoded with the
// reference of the node that wrote it: the upwind (or wrapped) node for a
// streamed value, the node itself for a bounced one.
__device__ __forceinline__ void pull_face_ref(const __half* __restrict__ src,
                                              const uint2* __restrict__ ref, int64_t qstride,
                                              int nx, int ny, int nz, int pitch, int plane,
                                              unsigned fb, int x, int y, int z, int i,
                                              const float* lidc, float (&d)[Q]) {
  const bool fx0 = x == 0, fx1 = x == nx - 1, fy0 = y == 0, fy1 = y == ny - 1;
  const bool fz0 = z == 0, fz1 = z == nz - 1;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const __half* sq = src + int64_t(q) * qstride;
    const bool ox = (cx(q) == 1 && fx0) || (cx(q) == -1 && fx1);
    const bool oy = (cy(q) == 1 && fy0) || (cy(q) == -1 && fy1);
    const bool oz = (cz(q) == 1 && fz0) || (cz(q) == -1 && fz1);
    const int up = i - (cz(q) * plane + cy(q) * pitch + cx(q));
    if (!(ox || oy || oz)) {
      d[q] = dec16(sq[up]) + ref_term(q, ref_load(ref + up));
      continue;
    }
    const int kx = ox ? int((fb >> (cx(q) == 1 ? 0 : 2)) & 3u) : int(BC_PERIODIC);
    const int ky = oy ? int((fb >> (cy(q) == 1 ? 4 : 6)) & 3u) : int(BC_PERIODIC);
    const int kz = oz ? int((fb >> (cz(q) == 1 ? 8 : 10)) & 3u) : int(BC_PERIODIC);
    if (kx != BC_PERIODIC || ky != BC_PERIODIC || kz != BC_PERIODIC) {
      const bool lid = kx == BC_LID || ky == BC_LID || kz == BC_LID;
      const float v = dec16(src[int64_t(opp(q)) * qstride + i]) +
                      ref_term(opp(q), ref_load(ref + i));
      d[q] = lid ? v + lidc[q] : v;
    } else {
      int j = up;
      if (ox) j += cx(q) == 1 ? nx : -nx;
      if (oy) j += cy(q) == 1 ? ny * pitch : -ny * pitch;
      if (oz) j += cz(q) == 1 ? nz * plane : -nz * plane;
      d[q] = dec16(sq[j]) + ref_term(q, ref_load(ref + j));
    }
  }
}

template <bool FORCE, bool CHECK, bool CAP>
__global__ void __launch_bounds__(256, CAP ? 4 : 1) step_ref_kernel(const StepArgs<__half, float> a,
                                                                    const RefArgs r) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = a.zrev ? a.nz - 1 - int(blockIdx.z) : int(blockIdx.z);  // as step_kernel
  const bool active = x < a.nx && y < a.ny;
  if (!CHECK && !active) return;
  const float rho0 = a.C.rho0;
  double du2 = 0.0, uu = 0.0, dr = 0.0;
  int bad = 0;
  if (active) {
    const int i = z * a.plane + y * a.pitch + x;
    float d[Q];
    if (y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1) {
      // One population and one reference load per direction: a lane on an x
      // face takes, for the five directions that come from outside, the
      // periodic wrap or the halfway bounce-back from its own opposite
      // population, decoded with its own reference (the term of opp(q) is
      // w_q (dr - e_q.v)), plus the lid term -- a select of the addresses,
      // so that every lane issues the same loads.
      const bool fl = x == 0, fr = x == a.nx - 1;
      const int kl = a.facebits & 3, kr = (a.facebits >> 2) & 3;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const __half* pq = a.srcq[q] + i;
        const uint2* rq = r.refq[q] + i;
        float sgn = 1.0f, extra = 0.0f;
        if ((cx(q) == 1 && fl) || (cx(q) == -1 && fr)) {
          const int k = cx(q) == 1 ? kl : kr;
          if (k == BC_PERIODIC) {
            pq += cx(q) == 1 ? a.nx : -a.nx;
            rq += cx(q) == 1 ? a.nx : -a.nx;
          } else {
            pq = a.src + int64_t(opp(q)) * a.qstride + i;
            rq = r.ref_src + i;
            sgn = -1.0f;
            extra = k == BC_LID ? a.lidc[q] : 0.0f;
          }
        }
        const Ref4 t = ref_load(rq);
        const float ev = float(cx(q)) * t.vx + float(cy(q)) * t.vy + float(cz(q)) * t.vz;
        d[q] = dec16(*pq) + wt<float>(q) * (t.dr + sgn * ev) + extra;
      }
    } else {
      pull_face_ref(a.src, r.ref_src, a.qstride, a.nx, a.ny, a.nz, a.pitch, a.plane, a.facebits,
                    x, y, z, i, a.lidc, d);
    }
    NodeOut<float> o;
    collide<float, FORCE, !FORCE, LOG2LAM>(a.C, d, o);
    Ref4 rr;
    r.ref_dst[i] = ref_make(o.rho - rho0, o.rho, o.ux, o.uy, o.uz, rr);
    store_sr([&](int q) -> __half& { return a.dstq[q][i]; }, d, rr, sr_seed(uint32_t(i), r.step));
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
      dr = double(o.rho) - double(rho0);
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

template <bool FORCE>
__global__ void __launch_bounds__(256) fields_ref_kernel(const __half* __restrict__ src,
                                                         const uint2* __restrict__ ref, Geom g,
                                                         CollideConst<float> C,
                                                         const float* __restrict__ lidc,
                                                         double* rho, double* u, double* gd) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int i = z * int(g.plane) + y * g.pitch + x;
  float d[Q];
  pull_face_ref(src, ref, g.qstride, g.nx, g.ny, g.nz, g.pitch, int(g.plane), g.facebits, x, y,
                z, i, lidc, d);
  NodeOut<float> o;
  collide<float, FORCE, !FORCE, LOG2LAM>(C, d, o);
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

__global__ void export_ref_kernel(const __half* __restrict__ src, const uint2* __restrict__ ref,
                                  Geom g, float rho0, double* __restrict__ out) {
  const int64_t N = int64_t(g.nx) * g.ny * g.nz;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= N * Q) return;
  const int q = int(t / N);
  const int64_t k = t - int64_t(q) * N;
  const int x = int(k % g.nx), y = int((k / g.nx) % g.ny), z = int(k / (int64_t(g.nx) * g.ny));
  const int64_t i = int64_t(z) * g.plane + int64_t(y) * g.pitch + x;
  const float dev = dec16(src[q * g.qstride + i]) + ref_term(q, ref_load(ref + i));
  out[t] = double(dev) * (1.0 / double(LAM)) + wt<double>(q) * double(rho0);
}

// One thread per node: the reference is the node's own moments of the
// imported populations.
__global__ void import_ref_kernel(const double* __restrict__ in, Geom g, float rho0,
                                  __half* __restrict__ dst, uint2* __restrict__ ref) {
  const int64_t N = int64_t(g.nx) * g.ny * g.nz;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int x = int(k % g.nx), y = int((k / g.nx) % g.ny), z = int(k / (int64_t(g.nx) * g.ny));
  const int64_t i = int64_t(z) * g.plane + int64_t(y) * g.pitch + x;
  double f[Q], rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    f[q] = in[q * N + k];
    rho += f[q];
    jx += cx(q) * f[q];
    jy += cy(q) * f[q];
    jz += cz(q) * f[q];
  }
  Ref4 rr;
  ref[i] = ref_make(float(rho - rho0), float(rho), float(jx / rho), float(jy / rho),
                    float(jz / rho), rr);
#pragma unroll
  for (int q = 0; q < Q; ++q)
    dst[q * g.qstride + i] =
        enc16(float((f[q] - wt<double>(q) * rho0) * double(LAM)) - ref_term(q, rr));
}

// M independent nodes: store (with its own reference), load, collide, store
// again with the new reference, load.
template <bool FORCE>
__global__ void collide_nodes_ref_kernel(CollideConst<float> C, const double* __restrict__ fin,
                                         double* __restrict__ fout, double* rho, double* u,
                                         double* gd, int64_t M) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const float rho0 = C.rho0;
  double r0 = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const double v = fin[q * M + k];
    r0 += v;
    jx += cx(q) * v;
    jy += cy(q) * v;
    jz += cz(q) * v;
  }
  Ref4 rr;
  ref_make(float(r0 - rho0), float(r0), float(jx / r0), float(jy / r0), float(jz / r0), rr);
  float d[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float t = ref_term(q, rr);
    d[q] = dec16(enc16(float((fin[q * M + k] - wt<double>(q) * rho0) * double(LAM)) - t)) + t;
  }
  NodeOut<float> o;
  collide<float, FORCE, !FORCE, LOG2LAM>(C, d, o);
  ref_make(o.rho - rho0, o.rho, o.ux, o.uy, o.uz, rr);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float t = ref_term(q, rr);
    fout[q * M + k] = double(dec16(enc16(d[q] - t)) + t) * (1.0 / double(LAM)) +
                      wt<double>(q) * double(rho0);
  }
  if (rho) rho[k] = double(o.rho);
  if (u) {
    u[k] = double(o.ux);
    u[M + k] = double(o.uy);
    u[2 * M + k] = double(o.uz);
  }
  if (gd) gd[k] = double(o.gamma_dot);
}

// Lid terms of the bounce-back, in the scaled deviations.
void lid_table(const Geom& g, float* out) {
  for (int q = 0; q < Q; ++q)
    out[q] = float(6.0 * double(LAM) * wt<double>(q) * g.rho0 *
                   (cx(q) * g.U[0] + cy(q) * g.U[1] + cz(q) * g.U[2]));
}

}  // namespace

// One node of the batched step in the F16R form: the same pull, references
// and collision as step_ref_kernel.
template <bool FORCE>
__device__ void batch_node_ref(const LatDesc<float>& L, int parity, int x, int y, int z,
                               unsigned step, NodeOut<float>& o) {
  const __half* src = static_cast<const __half*>(L.buf[parity]);
  __half* dst = static_cast<__half*>(const_cast<void*>(L.buf[parity ^ 1]));
  const uint2* rs = static_cast<const uint2*>(L.ref[parity]);
  uint2* rd = static_cast<uint2*>(const_cast<void*>(L.ref[parity ^ 1]));
  const float rho0 = L.C.rho0;
  const int qs = int(L.qstride), plane = L.plane, pitch = L.pitch;
  const int i = z * plane + y * pitch + x;
  float d[Q];
  if (y > 0 && y < L.ny - 1 && z > 0 && z < L.nz - 1) {
    // as in step_ref_kernel: one load of each kind per direction, x faces
    // by a select
    const bool fl = x == 0, fr = x == L.nx - 1;
    const int kl = L.facebits & 3, kr = (L.facebits >> 2) & 3;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int up = i - (cz(q) * plane + cy(q) * pitch + cx(q));
      int j = q * qs + up, jr = up;
      float sgn = 1.0f, extra = 0.0f;
      if ((cx(q) == 1 && fl) || (cx(q) == -1 && fr)) {
        const int k = cx(q) == 1 ? kl : kr;
        if (k == BC_PERIODIC) {
          j += cx(q) == 1 ? L.nx : -L.nx;
          jr += cx(q) == 1 ? L.nx : -L.nx;
        } else {
          j = opp(q) * qs + i;
          jr = i;
          sgn = -1.0f;
          extra = k == BC_LID ? L.lidc[q] : 0.0f;
        }
      }
      const Ref4 t = ref_load(rs + jr);
      const float ev = float(cx(q)) * t.vx + float(cy(q)) * t.vy + float(cz(q)) * t.vz;
      d[q] = dec16(src[j]) + wt<float>(q) * (t.dr + sgn * ev) + extra;
    }
  } else {
    pull_face_ref(src, rs, L.qstride, L.nx, L.ny, L.nz, pitch, plane, L.facebits, x, y, z, i,
                  L.lidc, d);
  }
  collide<float, FORCE, !FORCE, LOG2LAM>(L.C, d, o);
  Ref4 rr;
  rd[i] = ref_make(o.rho - rho0, o.rho, o.ux, o.uy, o.uz, rr);
  store_sr([&](int q) -> __half& { return dst[q * qs + i]; }, d, rr, sr_seed(uint32_t(i), step));
}

cudaError_t launch_step_f16r(const void* src, void* dst, const void* ref_src, void* ref_dst,
                             const Geom& g, const PhysParams& P, const CheckBufs& cb, bool check,
                             dim3 block, int npt, int64_t step, cudaStream_t st) {
  StepArgs<__half, float> a;
  RefArgs r;
  r.step = unsigned(uint64_t(step));
  const __half* s = static_cast<const __half*>(src);
  __half* d = static_cast<__half*>(dst);
  const uint2* rs = static_cast<const uint2*>(ref_src);
  for (int q = 0; q < Q; ++q) {
    const int64_t off = int64_t(cz(q)) * g.plane + int64_t(cy(q)) * g.pitch + cx(q);
    a.srcq[q] = reinterpret_cast<const __half*>(reinterpret_cast<uintptr_t>(s) +
                                                 (int64_t(q) * g.qstride - off) * 2);
    a.dstq[q] = d + int64_t(q) * g.qstride;
    r.refq[q] = reinterpret_cast<const uint2*>(reinterpret_cast<uintptr_t>(rs) -
                                                 off * int64_t(sizeof(uint2)));
  }
  lid_table(g, a.lidc);
  r.ref_src = rs;
  r.ref_dst = static_cast<uint2*>(ref_dst);
  a.zrev = reinterpret_cast<uintptr_t>(dst) < reinterpret_cast<uintptr_t>(src) ? 1 : 0;
  a.src = s;
  a.qstride = g.qstride;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.pitch = g.pitch;
  a.plane = int(g.plane);
  a.facebits = g.facebits;
  a.C = make_const<float>(P, double(LAM));
  a.cb = cb;
  const bool cap = (npt & 4) != 0;
  dim3 grid((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, g.nz);
  cudaError_t e_ = cudaSuccess;
#define CLBM_REF_LAUNCH(F, C_)                                                                  \
  do {                                                                                         \
    if (cap) e_ = pdl_launch(step_ref_kernel<F, C_, true>, grid, block, st, a, r);            \
    else e_ = pdl_launch(step_ref_kernel<F, C_, false>, grid, block, st, a, r);               \
  } while (0)
  if (P.has_force) {
    if (check) CLBM_REF_LAUNCH(true, true);
    else CLBM_REF_LAUNCH(true, false);
  } else {
    if (check) CLBM_REF_LAUNCH(false, true);
    else CLBM_REF_LAUNCH(false, false);
  }
#undef CLBM_REF_LAUNCH
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

cudaError_t launch_fields_f16r(const void* src, const void* ref, const Geom& g,
                               const PhysParams& P, double* rho, double* u, double* gd,
                               cudaStream_t st) {
  float lid[Q];
  lid_table(g, lid);
  float* dlid = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dlid), sizeof(lid), st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(dlid, lid, sizeof(lid), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    dim3 block(32, 4);
    dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
    const CollideConst<float> C = make_const<float>(P, double(LAM));
    const __half* s = static_cast<const __half*>(src);
    const uint2* r = static_cast<const uint2*>(ref);
    if (P.has_force) fields_ref_kernel<true><<<grid, block, 0, st>>>(s, r, g, C, dlid, rho, u, gd);
    else fields_ref_kernel<false><<<grid, block, 0, st>>>(s, r, g, C, dlid, rho, u, gd);
    e = cudaGetLastError();
  }
  cudaFreeAsync(dlid, st);
  return e;
}

cudaError_t launch_export_f16r(const void* src, const void* ref, const Geom& g, double rho0,
                               double* out, cudaStream_t st) {
  const int64_t total = int64_t(g.nx) * g.ny * g.nz * Q;
  const int b = 256;
  export_ref_kernel<<<unsigned((total + b - 1) / b), b, 0, st>>>(
      static_cast<const __half*>(src), static_cast<const uint2*>(ref), g, float(rho0), out);
  return cudaGetLastError();
}

cudaError_t launch_import_f16r(const double* in, const Geom& g, double rho0, void* dst, void* ref,
                               cudaStream_t st) {
  const int64_t N = int64_t(g.nx) * g.ny * g.nz;
  const int b = 128;
  import_ref_kernel<<<unsigned((N + b - 1) / b), b, 0, st>>>(in, g, float(rho0),
                                                              static_cast<__half*>(dst),
                                                              static_cast<uint2*>(ref));
  return cudaGetLastError();
}

cudaError_t launch_collide_nodes_f16r(const PhysParams& P, const double* fin, double* fout,
                                      double* rho, double* u, double* gd, int64_t M,
                                      cudaStream_t st) {
  const int b = 128;
  const unsigned grid = unsigned((M + b - 1) / b);
  const CollideConst<float> C = make_const<float>(P, double(LAM));
  if (P.has_force) collide_nodes_ref_kernel<true><<<grid, b, 0, st>>>(C, fin, fout, rho, u, gd, M);
  else collide_nodes_ref_kernel<false><<<grid, b, 0, st>>>(C, fin, fout, rho, u, gd, M);
  return cudaGetLastError();
}

}  // namespace clbm

CLBM_DEFINE_BATCH(f16r, __half, float, true)
