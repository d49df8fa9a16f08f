// clbm_lib.cu -- host side of the C ABI declared in include/clbm.h.
//
// A handle owns two population buffers (A-B), the check-step work buffers and
// a stream.  clbm_step() queues kernels and returns; check steps copy their
// FP64 reduction results into pinned host memory behind an event, so the host
// learns about divergence without stalling the stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/clbm.h"
#include "ctx.h"
#include "launch.h"
#include "validate.h"
#include "launch_f16sr.h"

using namespace clbm;


namespace {

thread_local std::string g_create_err;

int fail(clbm_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_fail(clbm_ctx* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? CLBM_ERR_OOM : CLBM_ERR_CUDA, m);
}

// The allocator registered with clbm_set_allocator (none: cudaMalloc); a
// handle copies it at creation.
std::mutex g_alloc_mu;
clbm_alloc_fn g_alloc_fn = nullptr;
clbm_free_fn g_free_fn = nullptr;
void* g_alloc_user = nullptr;

// A long-lived device buffer of h, from its allocator or cudaMalloc.
int dev_alloc(clbm_ctx* h, void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (!h->alloc_fn) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      *p = nullptr;
      return fail(h, CLBM_ERR_OOM, std::string(what) + " allocation failed");
    }
    return CLBM_OK;
  }
  void* q = h->alloc_fn(bytes, h->device, h->stream, h->alloc_user);
  if (!q) return fail(h, CLBM_ERR_OOM, std::string(what) + ": the external allocator failed");
  if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
    h->free_fn(q, bytes, h->device, h->stream, h->alloc_user);
    return fail(h, CLBM_ERR_ARG,
                std::string(what) + ": the external allocator returned a pointer not aligned "
                                    "to 256 bytes");
  }
  *p = q;
  return CLBM_OK;
}

void dev_free(clbm_ctx* h, void* p, size_t bytes) {
  if (!p) return;
  if (h->free_fn) h->free_fn(p, bytes, h->device, h->stream, h->alloc_user);
  else cudaFree(p);
}

#define CK(h, expr)                                   \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr); \
  } while (0)

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

cudaError_t dispatch_step(clbm_ctx* h, bool check) {
  CheckBufs cb{h->uprev, h->acc, h->flag};
  if (h->in_place) {
    const int npt = h->npt & 4 ? 5 : 1;
    switch (h->dtype) {
      case CLBM_F64: return launch_step_aa_f64(h->buf[0], h->g, h->P, cb, check, h->block, npt, h->layout, h->stream);
      case CLBM_F32: return launch_step_aa_f32(h->buf[0], h->g, h->P, cb, check, h->block, npt, h->layout, h->stream);
      default: return launch_step_aa_f16(h->buf[0], h->g, h->P, cb, check, h->block, npt, h->layout, h->stream);
    }
  }
  const void* src = h->buf[h->cur];
  void* dst = h->buf[1 - h->cur];
  switch (h->dtype) {
    case CLBM_F64: return launch_step_f64(src, dst, h->g, h->P, cb, check, h->block, h->npt & 4 ? 5 : 1, h->stream);
    case CLBM_F32: return launch_step_f32(src, dst, h->g, h->P, cb, check, h->block, h->npt, h->stream);
    case CLBM_F16R:
      return launch_step_f16r(src, dst, h->ref[h->cur], h->ref[1 - h->cur], h->g, h->P, cb, check,
                              h->block, h->npt, h->steps, h->stream);
    default:
      if (h->sround)
        return launch_step_f16sr(src, dst, h->g, h->P, cb, check, h->block, h->npt, h->steps,
                                 h->stream);
      return launch_step_f16(src, dst, h->g, h->P, cb, check, h->block, h->npt, h->stream);
  }
}

// After a step: the other buffer holds the state, or (in place) the buffer
// holds the other layout.
void advance_state(clbm_ctx* h) {
  if (h->in_place) h->layout ^= 1;
  else h->cur = 1 - h->cur;
}

int set_device(clbm_ctx* h) {
  CK(h, cudaSetDevice(h->device));
  // A batched lattice is written on the batch's stream: let it finish first.
  if (h->batch) {
    int r = clbm_batch_sync(h->batch);
    if (r != CLBM_OK) return fail(h, r, "batch: " + std::string(clbm_last_error(nullptr)));
  }
  return CLBM_OK;
}

bool bad(const clbm_ctx* h) { return h == nullptr || h->buf[0] == nullptr; }

}  // namespace

namespace clbm {
void set_unbound_error(const char* msg) { g_create_err = msg; }
}  // namespace clbm

extern "C" {

int clbm_create(const clbm_domain* d, double K, double n, const double U_lid[3],
                const double body_force[3], clbm_dtype dtype, clbm_handle* out) {
  if (!d || !out) return fail(nullptr, CLBM_ERR_ARG, "null domain or output pointer");
  *out = nullptr;
  if (dtype != CLBM_F64 && dtype != CLBM_F32 && dtype != CLBM_F16S && dtype != CLBM_F16R)
    return fail(nullptr, CLBM_ERR_ARG, "unknown dtype");
  if (d->in_place && dtype == CLBM_F16R)
    return fail(nullptr, CLBM_ERR_UNSUPPORTED, "in-place streaming takes FP64, FP32 or F16S storage");
  std::string why;
  double U[3];
  if (!check_domain(d, U_lid, U, why)) return fail(nullptr, CLBM_ERR_ARG, why);
  // The kernels index one direction's array (padded rows, 128-byte pitch)
  // with 32-bit integers, neighbours included: keep it well below 2^31.
  {
    const int64_t elem = dtype == CLBM_F64 ? 8 : dtype == CLBM_F32 ? 4 : 2;
    const int64_t pitch = (int64_t(d->nx) + 128 / elem - 1) / (128 / elem) * (128 / elem);
    const int64_t padded = pitch * d->ny * d->nz;
    if (padded > (int64_t(1) << 31) - (int64_t(1) << 24))
      return fail(nullptr, CLBM_ERR_ARG,
                  "lattice too large: at most 2^31 - 2^24 padded nodes (32-bit indexing)");
  }
  double rho0, nu_min, nu_max;
  domain_defaults(d, &rho0, &nu_min, &nu_max);
  if (!check_phys(K, n, nu_min, nu_max, why)) return fail(nullptr, CLBM_ERR_ARG, why);
  if (!check_force(body_force, why)) return fail(nullptr, CLBM_ERR_ARG, why);

  clbm_ctx* h = new (std::nothrow) clbm_ctx();
  if (!h) return fail(nullptr, CLBM_ERR_OOM, "host allocation failed");
  h->dom = *d;
  h->dom.rho0 = rho0;
  h->dom.nu_min = nu_min;
  h->dom.nu_max = nu_max;
  if (h->dom.check_interval <= 0) h->dom.check_interval = 100;
  h->dtype = dtype;
  h->elem = dtype == CLBM_F64 ? 8 : dtype == CLBM_F32 ? 4 : 2;  // F16S, F16R: 2
  h->rsize = dtype == CLBM_F64 ? 8 : 4;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(nullptr, e, "cudaGetDevice");
  }

  Geom& g = h->g;
  g.nx = d->nx;
  g.ny = d->ny;
  g.nz = d->nz;
  g.pitch = int(round_up(d->nx, int64_t(128 / h->elem)));  // 128-byte rows
  g.plane = int64_t(g.pitch) * g.ny;
  g.qstride = round_up(g.plane * g.nz, 256);
  g.facebits = 0;
  for (int f = 0; f < 6; ++f) g.facebits |= unsigned(d->face[f]) << (2 * f);
  for (int a = 0; a < 3; ++a) g.U[a] = U[a];
  g.rho0 = rho0;
  fill_params(h->P, K, n, body_force, rho0, nu_min, nu_max, dtype);
  h->block.x = d->nx <= 32 ? unsigned(tile_width(d->nx, int(h->elem), 32, 128))
                           : d->nx <= 64 ? 64 : 128;
  h->block.y = 128 / h->block.x;
  h->block.z = 1;
  h->npt = 1;  // the autotuner may switch to two nodes per thread

  auto cleanup = [&](int code, const std::string& m) {
    g_create_err = m + (h->err.empty() ? "" : (": " + h->err));
    clbm_destroy(h);
    return code;
  };
  if (d->stream) {
    h->stream = static_cast<cudaStream_t>(d->stream);
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(CLBM_ERR_CUDA, cudaGetErrorString(e));
    h->own_stream = true;
  }
  const size_t pop_bytes = size_t(NQ) * size_t(g.qstride) * h->elem;
  h->in_place = d->in_place != 0;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    h->alloc_fn = g_alloc_fn;
    h->free_fn = g_free_fn;
    h->alloc_user = g_alloc_user;
  }
  h->pop_bytes = pop_bytes;
  h->uprev_bytes = 3 * size_t(g.plane) * g.nz * h->rsize;
  int rc = CLBM_OK;
  for (int b = 0; b < (h->in_place ? 1 : 2) && rc == CLBM_OK; ++b)
    rc = dev_alloc(h, &h->buf[b], pop_bytes, "population buffer");
  if (rc != CLBM_OK) return cleanup(rc, "clbm_create");
  if (dtype == CLBM_F16R) {
    h->ref_bytes = f16r_ref_bytes(g.plane * g.nz);
    for (int b = 0; b < 2 && rc == CLBM_OK; ++b) {
      rc = dev_alloc(h, &h->ref[b], h->ref_bytes, "reference buffer");
      if (rc == CLBM_OK && cudaMemsetAsync(h->ref[b], 0, h->ref_bytes, h->stream) != cudaSuccess)
        rc = fail(h, CLBM_ERR_CUDA, "reference buffer clear failed");
    }
    if (rc != CLBM_OK) return cleanup(rc, "clbm_create");
  }
  rc = dev_alloc(h, &h->uprev, h->uprev_bytes, "velocity buffer");
  if (rc != CLBM_OK) return cleanup(rc, "clbm_create");
  // acc: 3 FP64 sums, then the divergence flag and the TMA error word
  rc = dev_alloc(h, reinterpret_cast<void**>(&h->acc), 4 * sizeof(double), "reduction buffer");
  if (rc != CLBM_OK) return cleanup(rc, "clbm_create");
  h->flag = reinterpret_cast<int*>(h->acc + 3);
  e = cudaMallocHost(&h->host, 4 * sizeof(double));
  if (e != cudaSuccess) return cleanup(CLBM_ERR_OOM, "pinned buffer allocation failed");
  std::memset(h->host, 0, 4 * sizeof(double));
  e = cudaEventCreateWithFlags(&h->check_done, cudaEventDisableTiming);
  if (e != cudaSuccess) return cleanup(CLBM_ERR_CUDA, cudaGetErrorString(e));
  // Rest state: stored deviation f - w rho0 = 0 (all-zero bits in every form).
  for (int b = 0; b < (h->in_place ? 1 : 2); ++b) {
    e = cudaMemsetAsync(h->buf[b], 0, pop_bytes, h->stream);
    if (e != cudaSuccess) return cleanup(CLBM_ERR_CUDA, cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(h->uprev, 0, 3 * size_t(g.plane) * g.nz * h->rsize, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->acc, 0, 4 * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cleanup(CLBM_ERR_CUDA, cudaGetErrorString(e));
  *out = h;
  return CLBM_OK;
}

int clbm_step(clbm_handle h, int64_t nsteps) {
  if (bad(h)) return fail(h, CLBM_ERR_ARG, "invalid handle");
  if (nsteps < 0) return fail(h, CLBM_ERR_ARG, "nsteps must be >= 0");
  if (h->batch) return fail(h, CLBM_ERR_ARG, "lattice is in a batch: step the batch");
  if (int r = set_device(h)) return r;
  const int64_t every = h->dom.check_interval;
  for (int64_t s = 0; s < nsteps; ++s) {
    const bool check = ((h->steps + 1) % every) == 0;
    if (check) CK(h, cudaMemsetAsync(h->acc, 0, 3 * sizeof(double), h->stream));
    CK(h, dispatch_step(h, check));
    advance_state(h);
    h->steps += 1;
    if (check) {
      h->checks += 1;
      CK(h, cudaMemcpyAsync(h->host, h->acc, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
      CK(h, cudaEventRecord(h->check_done, h->stream));
    }
  }
  if (!h->diverged && h->checks > 0 && cudaEventQuery(h->check_done) == cudaSuccess) {
    int f[2] = {0, 0};
    std::memcpy(f, &h->host[3], sizeof(f));
    h->diverged = f[0] != 0;
    h->pipeline_err = h->pipeline_err || f[1] != 0;
  }
  if (h->pipeline_err)
    return fail(h, CLBM_ERR_CUDA, "a TMA pipeline wait in the step kernel gave up");
  if (h->diverged)
    return fail(h, CLBM_ERR_DIVERGED, "divergence: non-finite value or density out of [0.5, 2]");
  return CLBM_OK;
}

static int fields_impl(clbm_handle h, double* rho, double* u, double* gd) {
  const void* src = h->buf[h->cur];
  cudaError_t e;
  if (h->in_place) {
    switch (h->dtype) {
      case CLBM_F64: e = launch_fields_aa_f64(src, h->g, h->P, h->layout, rho, u, gd, h->stream); break;
      case CLBM_F32: e = launch_fields_aa_f32(src, h->g, h->P, h->layout, rho, u, gd, h->stream); break;
      default: e = launch_fields_aa_f16(src, h->g, h->P, h->layout, rho, u, gd, h->stream); break;
    }
    CK(h, e);
    return CLBM_OK;
  }
  switch (h->dtype) {
    case CLBM_F64: e = launch_fields_f64(src, h->g, h->P, rho, u, gd, h->stream); break;
    case CLBM_F32: e = launch_fields_f32(src, h->g, h->P, rho, u, gd, h->stream); break;
    case CLBM_F16R:
      e = launch_fields_f16r(src, h->ref[h->cur], h->g, h->P, rho, u, gd, h->stream);
      break;
    default: e = launch_fields_f16(src, h->g, h->P, rho, u, gd, h->stream); break;
  }
  CK(h, e);
  return CLBM_OK;
}

int clbm_fields_device(clbm_handle h, double* rho, double* u, double* gamma_dot) {
  if (bad(h)) return fail(h, CLBM_ERR_ARG, "invalid handle");
  if (int r = set_device(h)) return r;
  if (int r = fields_impl(h, rho, u, gamma_dot)) return r;
  CK(h, cudaStreamSynchronize(h->stream));
  return CLBM_OK;
}

int clbm_fields(clbm_handle h, double* rho, double* u, double* gamma_dot) {
  if (bad(h)) return fail(h, CLBM_ERR_ARG, "invalid handle");
  if (int r = set_device(h)) return r;
  const size_t N = size_t(h->g.nx) * h->g.ny * h->g.nz;
  double* dev = nullptr;
  CK(h, cudaMallocAsync(reinterpret_cast<void**>(&dev), 5 * N * sizeof(double), h->stream));
  int r = fields_impl(h, rho ? dev : nullptr, u ? dev + N : nullptr, gamma_dot ? dev + 4 * N : nullptr);
  cudaError_t e = cudaSuccess;
  if (r == CLBM_OK) {
    if (rho) e = cudaMemcpyAsync(rho, dev, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (u && e == cudaSuccess)
      e = cudaMemcpyAsync(u, dev + N, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (gamma_dot && e == cudaSuccess)
      e = cudaMemcpyAsync(gamma_dot, dev + 4 * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream);
  }
  cudaFreeAsync(dev, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (r != CLBM_OK) return r;
  CK(h, e);
  return CLBM_OK;
}

int clbm_residual(clbm_handle h, double* out) {
  if (bad(h) || !out) return fail(h, CLBM_ERR_ARG, "invalid handle or output");
  if (int r = set_device(h)) return r;
  CK(h, cudaStreamSynchronize(h->stream));
  if (h->checks < 2) {
    *out = INFINITY;
  } else if (!(h->host[1] > 0.0)) {
    *out = h->host[0] == 0.0 ? 0.0 : INFINITY;   // fluid at rest
  } else {
    *out = std::sqrt(h->host[0]) / (double(h->dom.check_interval) * std::sqrt(h->host[1]));
  }
  int f[2] = {0, 0};
  std::memcpy(f, &h->host[3], sizeof(f));
  h->diverged = h->diverged || f[0] != 0;
  h->pipeline_err = h->pipeline_err || f[1] != 0;
  if (h->pipeline_err)
    return fail(h, CLBM_ERR_CUDA, "a TMA pipeline wait in the step kernel gave up");
  if (h->diverged)
    return fail(h, CLBM_ERR_DIVERGED, "divergence: non-finite value or density out of [0.5, 2]");
  return CLBM_OK;
}

int clbm_mass(clbm_handle h, double* out) {
  if (bad(h) || !out) return fail(h, CLBM_ERR_ARG, "invalid handle or output");
  if (int r = set_device(h)) return r;
  CK(h, cudaStreamSynchronize(h->stream));
  if (h->checks < 1) return fail(h, CLBM_ERR_ARG, "no check step has run yet");
  const double N = double(h->g.nx) * h->g.ny * h->g.nz;
  *out = N * h->g.rho0 + h->host[2];
  return CLBM_OK;
}

static int state_io(clbm_handle h, double* out, const double* in) {
  if (bad(h) || (!out && !in)) return fail(h, CLBM_ERR_ARG, "invalid handle or buffer");
  if (int r = set_device(h)) return r;
  const size_t n = size_t(h->g.nx) * h->g.ny * h->g.nz * NQ;
  double* dev = nullptr;
  CK(h, cudaMallocAsync(reinterpret_cast<void**>(&dev), n * sizeof(double), h->stream));
  cudaError_t e = cudaSuccess;
  const double isc = h->P.inv_scale;
  if (in) {
    e = cudaMemcpyAsync(dev, in, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && h->in_place) {
      // the state goes into the swapped layout
      switch (h->dtype) {
        case CLBM_F64: e = launch_import_aa_f64(dev, h->g, h->g.rho0, isc, h->buf[0], h->stream); break;
        case CLBM_F32: e = launch_import_aa_f32(dev, h->g, h->g.rho0, isc, h->buf[0], h->stream); break;
        default: e = launch_import_aa_f16(dev, h->g, h->g.rho0, isc, h->buf[0], h->stream); break;
      }
      h->layout = 0;
    } else if (e == cudaSuccess) {
      switch (h->dtype) {
        case CLBM_F64: e = launch_import_f64(dev, h->g, h->g.rho0, isc, h->buf[h->cur], h->stream); break;
        case CLBM_F32: e = launch_import_f32(dev, h->g, h->g.rho0, isc, h->buf[h->cur], h->stream); break;
        case CLBM_F16R:
          e = launch_import_f16r(dev, h->g, h->g.rho0, h->buf[h->cur], h->ref[h->cur], h->stream);
          break;
        default: e = launch_import_f16(dev, h->g, h->g.rho0, isc, h->buf[h->cur], h->stream); break;
      }
    }
  } else if (h->in_place) {
    switch (h->dtype) {
      case CLBM_F64: e = launch_export_aa_f64(h->buf[0], h->g, h->g.rho0, isc, h->layout, dev, h->stream); break;
      case CLBM_F32: e = launch_export_aa_f32(h->buf[0], h->g, h->g.rho0, isc, h->layout, dev, h->stream); break;
      default: e = launch_export_aa_f16(h->buf[0], h->g, h->g.rho0, isc, h->layout, dev, h->stream); break;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, dev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  } else {
    switch (h->dtype) {
      case CLBM_F64: e = launch_export_f64(h->buf[h->cur], h->g, h->g.rho0, isc, dev, h->stream); break;
      case CLBM_F32: e = launch_export_f32(h->buf[h->cur], h->g, h->g.rho0, isc, dev, h->stream); break;
      case CLBM_F16R:
        e = launch_export_f16r(h->buf[h->cur], h->ref[h->cur], h->g, h->g.rho0, dev, h->stream);
        break;
      default: e = launch_export_f16(h->buf[h->cur], h->g, h->g.rho0, isc, dev, h->stream); break;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, dev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  }
  cudaFreeAsync(dev, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  CK(h, e);
  return CLBM_OK;
}

int clbm_get_state(clbm_handle h, double* f_host) { return state_io(h, f_host, nullptr); }
int clbm_set_state(clbm_handle h, const double* f_host) {
  if (!f_host) return fail(h, CLBM_ERR_ARG, "null state");
  return state_io(h, nullptr, f_host);
}

int clbm_steps_done(clbm_handle h, int64_t* out) {
  if (bad(h) || !out) return fail(h, CLBM_ERR_ARG, "invalid handle or output");
  *out = h->steps;
  return CLBM_OK;
}

int clbm_sync(clbm_handle h) {
  if (bad(h)) return fail(h, CLBM_ERR_ARG, "invalid handle");
  if (int r = set_device(h)) return r;
  CK(h, cudaStreamSynchronize(h->stream));
  return CLBM_OK;
}

namespace {
// Autotuner cache: (dtype, nx, ny, nz, force, newtonian) -> (bx, by, npt).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::tuple<int, int, int, double>> g_tune;
}  // namespace

int clbm_autotune(clbm_handle h, int steps, int* block_x, int* block_y, int* npt,
                  double* us_per_step) {
  if (bad(h)) return fail(h, CLBM_ERR_ARG, "invalid handle");
  if (int r = set_device(h)) return r;
  if (steps <= 0) steps = 10;
  const auto key = std::make_tuple(int(h->dtype) + (h->in_place ? 16 : 0) + (h->sround ? 32 : 0), h->g.nx, h->g.ny,
                                   h->g.nz, h->P.has_force, h->P.newtonian);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      h->block = dim3(std::get<0>(it->second), std::get<1>(it->second), 1);
      h->npt = std::get<2>(it->second);
      if (block_x) *block_x = h->block.x;
      if (block_y) *block_y = h->block.y;
      if (npt) *npt = h->npt;
      if (us_per_step) *us_per_step = std::get<3>(it->second);
      return CLBM_OK;
    }
  }
  // Candidates: block shapes up to 256 threads (128 for two nodes per thread,
  // whose kernel is compiled for 128), x extent at most the padded row.
  struct Cand { int bx, by, npt; };
  std::vector<Cand> cands;
  const int shapes[][2] = {{32, 1}, {32, 2}, {32, 4}, {32, 8}, {64, 1}, {64, 2}, {64, 4},
                           {128, 1}, {128, 2}, {256, 1}};
  for (int capped = 0; capped <= 1; ++capped)
    for (int np = 1; np <= ((h->dtype == CLBM_F64 || h->dtype == CLBM_F16R || h->in_place || h->sround) ? 1 : 2); ++np)
      for (auto& sh : shapes) {
        if (sh[0] * sh[1] > (np == 2 ? 128 : 256)) continue;
        if (sh[0] > 32 && sh[0] > h->g.pitch) continue;
        cands.push_back({sh[0], sh[1], np + 4 * capped});
      }
  // a lattice narrower than a warp: blocks as wide as its tile width
  const int tw = tile_width(h->g.nx, int(h->elem), 32, 64);
  if (tw < 32)
    for (int capped = 0; capped <= 1; ++capped)
      for (int t : {64, 128, 256}) cands.push_back({tw, t / tw, 1 + 4 * capped});
  // FP32 and FP16 storage: the TMA-staged kernel in each of its shapes
  if ((h->dtype == CLBM_F32 || h->dtype == CLBM_F16S) && !h->in_place && !h->sround)
    for (int v = 0; v < TMA_NVAR; ++v) cands.push_back({tma_bx(v), tma_by(v), TMA_NPT + 32 * v});
  // Save the state: tuning runs real steps.
  const size_t pop_bytes = size_t(NQ) * size_t(h->g.qstride) * h->elem;
  const size_t ref_bytes = h->ref[0] ? f16r_ref_bytes(h->g.plane * h->g.nz) : 0;
  void* saved = nullptr;
  CK(h, cudaMallocAsync(&saved, pop_bytes + ref_bytes, h->stream));
  CK(h, cudaMemcpyAsync(saved, h->buf[h->cur], pop_bytes, cudaMemcpyDeviceToDevice, h->stream));
  if (ref_bytes)
    CK(h, cudaMemcpyAsync(static_cast<char*>(saved) + pop_bytes, h->ref[h->cur], ref_bytes,
                          cudaMemcpyDeviceToDevice, h->stream));
  const int cur0 = h->cur, layout0 = h->layout;
  cudaEvent_t e0, e1;
  CK(h, cudaEventCreate(&e0));
  CK(h, cudaEventCreate(&e1));
  const dim3 block0 = h->block;
  const int npt0 = h->npt;
  double best = 1e300;
  Cand bestc{int(block0.x), int(block0.y), npt0};
  cudaError_t err = cudaSuccess;
  for (const Cand& c : cands) {
    h->block = dim3(c.bx, c.by, 1);
    h->npt = c.npt;
    for (int s = 0; s < 2 && err == cudaSuccess; ++s) {
      err = dispatch_step(h, false);
      advance_state(h);
    }
    if (err == cudaSuccess) err = cudaEventRecord(e0, h->stream);
    for (int s = 0; s < steps && err == cudaSuccess; ++s) {
      err = dispatch_step(h, false);
      advance_state(h);
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err != cudaSuccess) break;
    const double us = 1e3 * double(ms) / steps;
    if (us < best) {
      best = us;
      bestc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // Restore the state into the buffer that held it (and its layout).
  h->cur = cur0;
  h->layout = layout0;
  cudaError_t e2 = cudaMemcpyAsync(h->buf[h->cur], saved, pop_bytes, cudaMemcpyDeviceToDevice,
                                   h->stream);
  if (e2 == cudaSuccess && ref_bytes)
    e2 = cudaMemcpyAsync(h->ref[h->cur], static_cast<char*>(saved) + pop_bytes, ref_bytes,
                         cudaMemcpyDeviceToDevice, h->stream);
  cudaFreeAsync(saved, h->stream);
  if (err == cudaSuccess) err = e2;
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  if (err != cudaSuccess) {
    h->block = block0;
    h->npt = npt0;
    return cuda_fail(h, err, "clbm_autotune");
  }
  h->block = dim3(bestc.bx, bestc.by, 1);
  h->npt = bestc.npt;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = std::make_tuple(bestc.bx, bestc.by, bestc.npt, best);
  }
  if (block_x) *block_x = bestc.bx;
  if (block_y) *block_y = bestc.by;
  if (npt) *npt = bestc.npt;
  if (us_per_step) *us_per_step = best;
  return CLBM_OK;
}

int clbm_set_rounding(clbm_handle h, clbm_rounding mode) {
  if (bad(h)) return fail(h, CLBM_ERR_ARG, "invalid handle");
  if (mode != CLBM_ROUND_NEAREST && mode != CLBM_ROUND_STOCHASTIC)
    return fail(h, CLBM_ERR_ARG, "unknown rounding mode");
  if (h->batch) return fail(h, CLBM_ERR_ARG, "lattice is in a batch: detach it first");
  const bool sr = mode == CLBM_ROUND_STOCHASTIC;
  if (h->dtype == CLBM_F16R) {
    if (!sr) return fail(h, CLBM_ERR_UNSUPPORTED, "the F16R form always rounds stochastically");
    return CLBM_OK;
  }
  if (h->dtype != CLBM_F16S) {
    if (sr) return fail(h, CLBM_ERR_UNSUPPORTED, "stochastic rounding is an F16S option");
    return CLBM_OK;
  }
  if (sr && h->in_place)
    return fail(h, CLBM_ERR_UNSUPPORTED, "stochastic rounding takes two-buffer lattices");
  h->sround = sr;
  // the stochastic kernel has one shape family: one node per thread
  if (sr && ((h->npt & TMA_NPT) || (h->npt & 3) == 2)) h->npt = 1;
  return CLBM_OK;
}

int clbm_set_rates(clbm_handle h, const double omega[10]) {
  if (bad(h) || !omega) return fail(h, CLBM_ERR_ARG, "invalid handle or rates");
  if (h->batch) return fail(h, CLBM_ERR_ARG, "lattice is in a batch: detach it first");
  for (int k = 0; k < 10; ++k)
    if (!(omega[k] > 0.0 && omega[k] < 2.0))
      return fail(h, CLBM_ERR_ARG, "every relaxation rate must lie in (0, 2)");
  for (int k = 0; k < 10; ++k) h->P.omega_high[k] = omega[k];
  return CLBM_OK;
}

int clbm_set_launch(clbm_handle h, int block_x, int block_y, int npt) {
  if (bad(h)) return fail(h, CLBM_ERR_ARG, "invalid handle");
  if (h->in_place && ((npt & TMA_NPT) || (npt & 3) == 2))
    return fail(h, CLBM_ERR_UNSUPPORTED, "in-place lattices take one node per thread (npt 1 or 5)");
  if (npt & TMA_NPT) {
    const int v = npt >> 5;
    if ((npt & 31) != TMA_NPT || v >= TMA_NVAR)
      return fail(h, CLBM_ERR_ARG, "npt: TMA_NPT + 32 v with v < TMA_NVAR for the TMA kernel");
    if (h->dtype != CLBM_F32 && h->dtype != CLBM_F16S)
      return fail(h, CLBM_ERR_UNSUPPORTED, "the TMA-staged kernel takes FP32 or F16S storage");
    if (h->sround)
      return fail(h, CLBM_ERR_UNSUPPORTED, "stochastic rounding runs one node per thread (npt 1 or 5)");
    if (block_x != tma_bx(v) || block_y != tma_by(v))
      return fail(h, CLBM_ERR_ARG, "block does not match the TMA shape");
    h->block = dim3(block_x, block_y, 1);
    h->npt = npt;
    return CLBM_OK;
  }
  const int np = npt & 3;
  if ((np != 1 && np != 2) || (npt & ~7))
    return fail(h, CLBM_ERR_ARG, "npt must be 1 or 2, plus 4 for the register-capped kernel");
  if (block_x < 1 || block_y < 1 || block_x * block_y > (np == 2 ? 128 : 256) ||
      block_x * block_y % 32 != 0)
    return fail(h, CLBM_ERR_ARG, "block must have a multiple of 32 threads, at most 256 "
                                 "(128 with two nodes per thread)");
  if (np == 2 && (h->dtype == CLBM_F64 || h->dtype == CLBM_F16R))
    return fail(h, CLBM_ERR_UNSUPPORTED, "two nodes per thread needs FP32 math");
  if (np == 2 && h->sround)
    return fail(h, CLBM_ERR_UNSUPPORTED, "stochastic rounding runs one node per thread (npt 1 or 5)");
  h->block = dim3(block_x, block_y, 1);
  h->npt = npt;
  return CLBM_OK;
}

int clbm_destroy(clbm_handle h) {
  if (!h) return CLBM_OK;
  if (h->batch) clbm_batch_detach(h->batch, h);
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int b = 0; b < 2; ++b) {
    dev_free(h, h->buf[b], h->pop_bytes);
    dev_free(h, h->ref[b], h->ref_bytes);
  }
  dev_free(h, h->uprev, h->uprev_bytes);
  dev_free(h, h->acc, 4 * sizeof(double));
  if (h->host) cudaFreeHost(h->host);
  if (h->check_done) cudaEventDestroy(h->check_done);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return CLBM_OK;
}

int clbm_set_allocator(clbm_alloc_fn alloc_fn, clbm_free_fn free_fn, void* user) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr))
    return fail(nullptr, CLBM_ERR_ARG, "give both allocator functions, or neither");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc_fn = alloc_fn;
  g_free_fn = free_fn;
  g_alloc_user = alloc_fn ? user : nullptr;
  return CLBM_OK;
}

const char* clbm_last_error(clbm_handle h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

int clbm_collide_nodes(clbm_dtype dtype, double K, double n, const double body_force[3],
                       double rho0, double nu_min, double nu_max, const double* f_in,
                       double* f_out, double* rho, double* u, double* gamma_dot, int64_t M) {
  if (!f_in || !f_out || M <= 0) return fail(nullptr, CLBM_ERR_ARG, "bad node arrays");
  if (dtype != CLBM_F64 && dtype != CLBM_F32 && dtype != CLBM_F16S && dtype != CLBM_F16R)
    return fail(nullptr, CLBM_ERR_ARG, "unknown dtype");
  rho0 = rho0 > 0 ? rho0 : 1.0;
  nu_min = nu_min > 0 ? nu_min : 5e-4;
  nu_max = nu_max > 0 ? nu_max : 10.0;
  std::string why;
  if (!check_phys(K, n, nu_min, nu_max, why)) return fail(nullptr, CLBM_ERR_ARG, why);
  PhysParams P{};
  fill_params(P, K, n, body_force, rho0, nu_min, nu_max, dtype);
  double* dev = nullptr;
  const size_t bytes = size_t(M) * (19 + 19 + 1 + 3 + 1) * sizeof(double);
  cudaError_t e = cudaMalloc(&dev, bytes);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMalloc");
  double* din = dev;
  double* dout = dev + 19 * M;
  double* drho = dout + 19 * M;
  double* du = drho + M;
  double* dgd = du + 3 * M;
  e = cudaMemcpy(din, f_in, 19 * M * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    switch (dtype) {
      case CLBM_F64: e = launch_collide_nodes_f64(P, din, dout, drho, du, dgd, M, 0); break;
      case CLBM_F32: e = launch_collide_nodes_f32(P, din, dout, drho, du, dgd, M, 0); break;
      case CLBM_F16R: e = launch_collide_nodes_f16r(P, din, dout, drho, du, dgd, M, 0); break;
      default: e = launch_collide_nodes_f16(P, din, dout, drho, du, dgd, M, 0); break;
    }
  }
  if (e == cudaSuccess) e = cudaMemcpy(f_out, dout, 19 * M * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && rho) e = cudaMemcpy(rho, drho, M * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && u) e = cudaMemcpy(u, du, 3 * M * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && gamma_dot)
    e = cudaMemcpy(gamma_dot, dgd, M * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "clbm_collide_nodes");
  return CLBM_OK;
}

int clbm_omega_nodes(clbm_dtype dtype, double K, double n, double nu_min, double nu_max,
                     const double* rho, const double* m, double* omega, double* gamma_dot,
                     int64_t M) {
  if (!rho || !m || !omega || M <= 0) return fail(nullptr, CLBM_ERR_ARG, "bad node arrays");
  if (dtype != CLBM_F64 && dtype != CLBM_F32 && dtype != CLBM_F16S && dtype != CLBM_F16R)
    return fail(nullptr, CLBM_ERR_ARG, "unknown dtype");
  nu_min = nu_min > 0 ? nu_min : 5e-4;
  nu_max = nu_max > 0 ? nu_max : 10.0;
  std::string why;
  if (!check_phys(K, n, nu_min, nu_max, why)) return fail(nullptr, CLBM_ERR_ARG, why);
  PhysParams P{};
  fill_params(P, K, n, nullptr, 1.0, nu_min, nu_max, dtype);
  double* dev = nullptr;
  const size_t bytes = size_t(M) * (1 + 6 + 1 + 1) * sizeof(double);
  cudaError_t e = cudaMalloc(&dev, bytes);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMalloc");
  double* drho = dev;
  double* dm = drho + M;
  double* dw = dm + 6 * M;
  double* dgd = dw + M;
  e = cudaMemcpy(drho, rho, M * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dm, m, 6 * M * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    // every FP32-math form solves in FP32 with the same code
    e = dtype == CLBM_F64 ? launch_omega_nodes_f64(P, drho, dm, dw, dgd, M, 0)
                          : launch_omega_nodes_f32(P, drho, dm, dw, dgd, M, 0);
  }
  if (e == cudaSuccess) e = cudaMemcpy(omega, dw, M * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && gamma_dot)
    e = cudaMemcpy(gamma_dot, dgd, M * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "clbm_omega_nodes");
  return CLBM_OK;
}

}  // extern "C"
