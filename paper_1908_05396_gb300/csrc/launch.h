// launch.h -- internal interface between the host library and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace clbm {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_LID = 2 };
constexpr int NQ = 19;  // D3Q19 directions
enum { DT_F64 = 0, DT_F32 = 1, DT_F16S = 2, DT_F16R = 3 };

// Power-of-two scale of the FP16 shifted storage: stored = (f - w rho0) * 1024.
constexpr double F16_SCALE = 1024.0;

// Lattice geometry and the stored layout pop[q][z][y][x] with row pitch.
struct Geom {
  int nx, ny, nz;
  int pitch;        // elements per stored row, >= nx
  int64_t plane;    // pitch * ny
  int64_t qstride;  // elements per direction array, >= plane * nz
  unsigned facebits; // 2 bits per face (BC_*), faces -x, +x, -y, +y, -z, +z
  double U[3];      // lid velocity
  double rho0;
};

// Width (nodes along x) of the tiles of a lattice nx nodes wide, for blocks
// of `threads` threads whose x extent is `bx`: bx, or the narrowest of 32,
// 16, 8 below it whose padded row is at least 1/8 shorter than the wider
// one's.  Narrow lattices (the 8-wide channels, 16..48-wide cavities) then
// leave fewer lanes idle.  A row keeps at least 32 bytes (one DRAM sector) of
// elements of `elem` bytes, and the width divides the block.
inline int tile_width(int nx, int elem, int bx, int threads) {
  int w = bx;
  for (int c = 32; c >= 8; c /= 2) {
    if (c >= w) continue;
    if (c * elem < 32 || threads % c) break;
    const int pw = (nx + w - 1) / w * w, pc = (nx + c - 1) / c * c;
    if (8 * pc <= 7 * pw) w = c;
  }
  return w;
}

// Physical parameters of the collision (host precision; kernels convert).
struct PhysParams {
  double rho0;
  double F[3];
  double K, logK3, n;
  double ylo, yhi;  // log(3 nu_min), log(3 nu_max)
  double nu_min, nu_max;
  double inv_scale; // storage decode scale (1 except FP16)
  int newtonian;
  int has_force;
  // relaxation rates omega_9 .. omega_18 (bulk, third and fourth order;
  // Sec. 3.1 sets them to 1, Sec. 5 notes they may be tuned)
  double omega_high[10] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
};

// Work buffers of a check step.
struct CheckBufs {
  void* uprev;      // 3 x (plane * nz) velocities of the previous check, math type
  double* acc;      // [0] sum|u-uprev|^2, [1] sum|u|^2, [2] sum(rho - rho0)
  int* flag;        // [0] divergence flag, [1] set when a TMA pipeline wait gave up
};

// TMA-staged FP32 / FP16 step (tma_step.cuh): npt = TMA_NPT + 32 v selects
// shape v, whose block must be tma_bx(v) x tma_by(v).
constexpr int TMA_NPT = 16;
constexpr int TMA_NVAR = 10;
// block of shape v: tiles 64x4, 128x2, 32x8, 64x4, 32x4, 64x2 with one node
// per thread (v < 6), then 64x4, 32x8, 64x4, 128x2 with two (rows 2ty, 2ty+1)
__host__ __device__ constexpr int tma_bx(int v) {
  return (v == 1 || v == 9) ? 128 : (v == 2 || v == 4 || v == 7) ? 32 : 64;
}
__host__ __device__ constexpr int tma_by(int v) {
  return v == 9 ? 1 : (v == 1 || v == 5 || v == 6 || v == 8) ? 2 : v == 2 ? 8 : 4;
}

// Launchers, one instantiation per storage type (one translation unit each).
#define CLBM_DECLARE_LAUNCHERS(SUFFIX)                                                        \
  cudaError_t launch_step_##SUFFIX(const void* src, void* dst, const Geom& g,                 \
                                   const PhysParams& P, const CheckBufs& cb, bool check,      \
                                   dim3 block, int npt, cudaStream_t st);                     \
  cudaError_t launch_fields_##SUFFIX(const void* src, const Geom& g, const PhysParams& P,     \
                                     double* rho, double* u, double* gd, cudaStream_t st);    \
  cudaError_t launch_collide_nodes_##SUFFIX(const PhysParams& P, const double* fin,           \
                                            double* fout, double* rho, double* u, double* gd, \
                                            int64_t M, cudaStream_t st);                      \
  cudaError_t launch_export_##SUFFIX(const void* src, const Geom& g, double rho0,             \
                                     double inv_scale, double* out, cudaStream_t st);         \
  cudaError_t launch_omega_nodes_##SUFFIX(const PhysParams& P, const double* rho,             \
                                          const double* m, double* omega, double* gd,         \
                                          int64_t M, cudaStream_t st);                        \
  cudaError_t launch_import_##SUFFIX(const double* in, const Geom& g, double rho0,            \
                                     double inv_scale, void* dst, cudaStream_t st);

// Record the text that clbm_last_error(NULL) returns on this thread.
void set_unbound_error(const char* msg);

// Batched step (batch.cuh): descriptors are opaque bytes to the host code.
// The unforced and the forced lattices form two independent chains of
// launches (on two streams), so each chain counts its own steps.
struct BatchHeader {
  int nlat;
  int ntiles;   // all tiles
  int ntiles0;  // tiles of lattices without force (they come first)
  int err;      // set by the kernel if a tile's descriptor fails its checks
  unsigned step[2];  // steps done by the unforced [0] / forced [1] chain (F16R: each
                     // lattice's step is its chain's count plus an offset)
  int done[2];       // F16R: CTAs of that chain's current launch that finished
};
#define CLBM_DECLARE_BATCH(SUFFIX)                                                              \
  cudaError_t launch_batch_##SUFFIX(int base, const int* owner, const unsigned* coord,         \
                                    const void* hdr, int parity, bool check, double* acc,       \
                                    int zc, dim3 block, int grid, cudaStream_t st,              \
                                    cudaStream_t st_forced);                                    \
  size_t desc_size_##SUFFIX();                                                                  \
  int desc_capacity_##SUFFIX();                                                                 \
  cudaError_t upload_desc_##SUFFIX(const void* host, int base, int n);                          \
  void fill_desc_##SUFFIX(void* out, const Geom& g, const PhysParams& P, const void* cur,       \
                          const void* other, const void* ref_cur, const void* ref_other,      \
                          void* uprev, int tx, int ty, int tw_log2, int slot,               \
                          unsigned step_offset);
CLBM_DECLARE_BATCH(f64)
CLBM_DECLARE_BATCH(f32)
CLBM_DECLARE_BATCH(f16)
CLBM_DECLARE_BATCH(f16r)

// F16R form (step_f16r.cu): FP16 populations relative to each node's stored
// first-order equilibrium reference, stored with stochastic rounding; `step`
// is the lattice's count of steps done before this one (it seeds the rounding).
cudaError_t launch_step_f16r(const void* src, void* dst, const void* ref_src, void* ref_dst,
                             const Geom& g, const PhysParams& P, const CheckBufs& cb, bool check,
                             dim3 block, int npt, int64_t step, cudaStream_t st);
cudaError_t launch_fields_f16r(const void* src, const void* ref, const Geom& g,
                               const PhysParams& P, double* rho, double* u, double* gd,
                               cudaStream_t st);
cudaError_t launch_export_f16r(const void* src, const void* ref, const Geom& g, double rho0,
                               double* out, cudaStream_t st);
cudaError_t launch_import_f16r(const double* in, const Geom& g, double rho0, void* dst, void* ref,
                               cudaStream_t st);
cudaError_t launch_collide_nodes_f16r(const PhysParams& P, const double* fin, double* fout,
                                      double* rho, double* u, double* gd, int64_t M,
                                      cudaStream_t st);

CLBM_DECLARE_LAUNCHERS(f64)
CLBM_DECLARE_LAUNCHERS(f32)
CLBM_DECLARE_LAUNCHERS(f16)

// In-place (one buffer) step, fields and state transfer (inplace.cuh);
// `layout` is the layout the buffer holds (0 swapped, 1 streamed).
#define CLBM_DECLARE_AA(SUFFIX)                                                                 \
  cudaError_t launch_step_aa_##SUFFIX(void* buf, const Geom& g, const PhysParams& P,            \
                                      const CheckBufs& cb, bool check, dim3 block, int npt,     \
                                      int layout, cudaStream_t st);                             \
  cudaError_t launch_fields_aa_##SUFFIX(const void* buf, const Geom& g, const PhysParams& P,    \
                                        int layout, double* rho, double* u, double* gd,         \
                                        cudaStream_t st);                                       \
  cudaError_t launch_export_aa_##SUFFIX(const void* buf, const Geom& g, double rho0,            \
                                        double inv_scale, int layout, double* out,              \
                                        cudaStream_t st);                                       \
  cudaError_t launch_import_aa_##SUFFIX(const double* in, const Geom& g, double rho0,           \
                                        double inv_scale, void* buf, cudaStream_t st);
CLBM_DECLARE_AA(f64)
CLBM_DECLARE_AA(f32)
CLBM_DECLARE_AA(f16)

}  // namespace clbm
