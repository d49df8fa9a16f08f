// clbm_batch.cu -- host side of the batched multi-lattice step (include/clbm.h).
//
// A batch holds up to `capacity` lattices (clbm_handle) of one storage form
// and steps them together: per time step, one launch of the persistent batch
// kernel over the lattices without body force and one over those with it, on
// two streams (the two launches touch disjoint lattices).  Whole check
// intervals run as one CUDA graph captured on first use: (check_interval - 1)
// plain steps of alternating parity, then a check step whose per-lattice FP64
// sums are copied to pinned host memory.  The kernel reads its tile table and lattice descriptors from device
// memory, so the graph stays valid when lattices join or leave; only a change
// of launch shape or of the table's capacity recaptures it.
//
// A second mode launches every lattice's own step kernel (kernels.cuh) once
// per step instead, the lattices spread over a few streams that fork from the
// batch's stream at the start of a check interval and join it at the end.
// Each lattice then runs with its parameters as kernel arguments and no tile
// table, and the streams fill each other's tails.  Its graph holds the
// lattices' buffer addresses, so a change of membership recaptures it.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/clbm.h"
#include "ctx.h"
#include "launch.h"
#include "launch_f16sr.h"

using namespace clbm;

struct clbm_batch_ctx {
  int device = 0;
  clbm_dtype dtype = CLBM_F32;
  int capacity = 0;
  int check_interval = 100;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<clbm_ctx*> slots;
  std::vector<int64_t> slot_checks;   // checks run since the lattice joined
  std::vector<int64_t> slot_joined;   // batch step at which it joined
  size_t desc_bytes = 0;
  int desc_base = -1;                 // first entry of this batch in the constant table
  void* d_desc = nullptr;             // small device allocation marking a live batch
  int* d_owner = nullptr;             // tile -> lattice index
  unsigned* d_coord = nullptr;        // tile -> packed tile coordinates
  int owner_cap = 0;
  BatchHeader* d_hdr = nullptr;
  double* d_acc = nullptr;            // capacity x 4
  double* h_acc = nullptr;            // pinned copy
  void* h_stage = nullptr;            // pinned staging of descriptors
  std::vector<int> h_owner;
  std::vector<unsigned> h_coord;
  int parity = 0;                     // steps since the tables were written, mod 2
  int64_t steps = 0;
  bool dirty = true;
  dim3 block{32, 4, 1};
  int zc = 1;                         // planes per tile (autotuned)
  // Until tuned (FP32-math forms): the register-capped kernel, eight CTAs
  // per SM, which is within a few per cent of the tuned launch from 4 to 64
  // small lattices and 1.8x faster than four uncapped CTAs once they fill the
  // GPU.  FP64 keeps four uncapped CTAs (its registers are twice as wide).
  int blocks_per_sm = 8;
  bool cap = true;                    // register-capped kernel variant
  int sms = 1;
  int mode = 0;                       // 0: persistent kernel; 1: one launch per lattice
  dim3 pl_block{32, 2, 1};            // mode 1: block of every lattice's step kernel
  int pl_npt = 5;                     // mode 1: 1, or 5 for the register-capped kernel
  int pl_streams = 4;                 // mode 1: streams the lattices are spread over
  std::vector<cudaStream_t> aux;      // mode 1: the streams besides `stream`
  std::vector<cudaEvent_t> ev;        // mode 1: fork event, then one join event per aux stream
  std::vector<int> stream_of;         // mode 1: slot -> stream (0 is `stream`)
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t check_done = nullptr;
  std::string err;
};

namespace {

int bfail(clbm_batch_ctx* b, int code, const std::string& m) {
  if (b) b->err = m;
  clbm::set_unbound_error(m.c_str());
  return code;
}

#define BCK(b, expr)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? CLBM_ERR_OOM : CLBM_ERR_CUDA,        \
                   std::string(#expr) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

size_t desc_size(clbm_dtype t) {
  return t == CLBM_F64   ? desc_size_f64()
         : t == CLBM_F32 ? desc_size_f32()
         : t == CLBM_F16R ? desc_size_f16r()
                          : desc_size_f16();
}

// Ranges of the per-form __constant__ descriptor tables held by live batches.
std::mutex g_table_mu;
std::vector<std::pair<int, int>> g_table_used[4];  // (base, count) per dtype

int table_capacity(clbm_dtype t) {
  return t == CLBM_F64    ? desc_capacity_f64()
         : t == CLBM_F32  ? desc_capacity_f32()
         : t == CLBM_F16R ? desc_capacity_f16r()
                          : desc_capacity_f16();
}

int table_reserve(clbm_dtype t, int n) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  auto& used = g_table_used[int(t)];
  std::sort(used.begin(), used.end());
  int base = 0;
  for (auto& r : used) {
    if (base + n <= r.first) break;
    base = std::max(base, r.first + r.second);
  }
  if (base + n > table_capacity(t)) return -1;
  used.emplace_back(base, n);
  return base;
}

void table_release(clbm_dtype t, int base) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  auto& used = g_table_used[int(t)];
  for (size_t i = 0; i < used.size(); ++i)
    if (used[i].first == base) {
      used.erase(used.begin() + long(i));
      return;
    }
}

cudaError_t upload_desc(clbm_dtype t, const void* host, int base, int n) {
  return t == CLBM_F64    ? upload_desc_f64(host, base, n)
         : t == CLBM_F32  ? upload_desc_f32(host, base, n)
         : t == CLBM_F16R ? upload_desc_f16r(host, base, n)
                          : upload_desc_f16(host, base, n);
}

void fill_desc(clbm_dtype t, void* out, const clbm_ctx* h, int tx, int ty, int twl, int slot,
               unsigned so) {
  const void* cur = h->buf[h->cur];
  const void* other = h->buf[1 - h->cur];
  // F16R: the reference moments travel with their population buffers
  const void* rcur = h->ref[h->cur];
  const void* rother = h->ref[1 - h->cur];
  if (t == CLBM_F64)
    fill_desc_f64(out, h->g, h->P, cur, other, rcur, rother, h->uprev, tx, ty, twl, slot, so);
  else if (t == CLBM_F32)
    fill_desc_f32(out, h->g, h->P, cur, other, rcur, rother, h->uprev, tx, ty, twl, slot, so);
  else if (t == CLBM_F16R)
    fill_desc_f16r(out, h->g, h->P, cur, other, rcur, rother, h->uprev, tx, ty, twl, slot, so);
  else {
    fill_desc_f16(out, h->g, h->P, cur, other, rcur, rother, h->uprev, tx, ty, twl, slot, so);
    desc_set_sround_f16(out, h->sround ? 1 : 0);
  }
}

// Whether an attached lattice rounds its stores stochastically: its seeds
// come from the batch's device-side step count, which only the persistent
// kernel advances (a replayed graph of per-lattice launches would repeat them).
bool any_sround(const clbm_batch_ctx* b) {
  for (int s = 0; s < b->capacity; ++s)
    if (b->slots[s] && b->slots[s]->sround) return true;
  return false;
}

// One step of the persistent kernel: the unforced lattices' launch on
// `stream`, the forced lattices' on the first extra stream.  The two touch
// disjoint lattices, so between fork_streams(b, 2) and join_streams(b, 2) they
// run concurrently, each chain in step order.
cudaError_t launch(clbm_batch_ctx* b, bool check) {
  const int grid = b->blocks_per_sm * b->sms * (b->cap ? -1 : 1);
  const cudaStream_t sf = b->aux[0];
  switch (b->dtype) {
    case CLBM_F64:
      return launch_batch_f64(b->desc_base, b->d_owner, b->d_coord, b->d_hdr, b->parity, check,
                              b->d_acc, b->zc, b->block, grid, b->stream, sf);
    case CLBM_F32:
      return launch_batch_f32(b->desc_base, b->d_owner, b->d_coord, b->d_hdr, b->parity, check,
                              b->d_acc, b->zc, b->block, grid, b->stream, sf);
    case CLBM_F16R:
      return launch_batch_f16r(b->desc_base, b->d_owner, b->d_coord, b->d_hdr, b->parity, check,
                               b->d_acc, b->zc, b->block, grid, b->stream, sf);
    default:
      return launch_batch_f16(b->desc_base, b->d_owner, b->d_coord, b->d_hdr, b->parity, check,
                              b->d_acc, b->zc, b->block, grid, b->stream, sf);
  }
}

void drop_graph(clbm_batch_ctx* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

// ---- mode 1: one launch per lattice --------------------------------------

cudaStream_t pl_stream(const clbm_batch_ctx* b, int k) {
  return k == 0 ? b->stream : b->aux[size_t(k - 1)];
}

// Create the extra streams and the fork/join events that `streams` needs.
cudaError_t ensure_streams(clbm_batch_ctx* b, int streams) {
  while (int(b->aux.size()) < streams - 1) {
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    b->aux.push_back(st);
  }
  while (int(b->ev.size()) < streams) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    b->ev.push_back(ev);
  }
  return cudaSuccess;
}

// Spread the lattices over the streams: largest first, each onto the stream
// with the fewest nodes so far.
void assign_streams(clbm_batch_ctx* b) {
  std::vector<int> order;
  for (int s = 0; s < b->capacity; ++s)
    if (b->slots[s]) order.push_back(s);
  auto nodes = [b](int s) {
    const clbm_ctx* h = b->slots[size_t(s)];
    return double(h->g.nx) * h->g.ny * h->g.nz;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return nodes(a) > nodes(c); });
  std::vector<double> load(size_t(b->pl_streams), 0.0);
  b->stream_of.assign(size_t(b->capacity), 0);
  for (int s : order) {
    const size_t k = size_t(std::min_element(load.begin(), load.end()) - load.begin());
    b->stream_of[size_t(s)] = int(k);
    load[k] += nodes(s);
  }
}

// The first n - 1 extra streams wait for everything queued on `stream` so far.
cudaError_t fork_streams(clbm_batch_ctx* b, int n) {
  cudaError_t e = cudaEventRecord(b->ev[0], b->stream);
  for (int k = 1; k < n && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(b->aux[size_t(k - 1)], b->ev[0], 0);
  return e;
}

// `stream` waits for everything queued on the first n - 1 extra streams so far.
cudaError_t join_streams(clbm_batch_ctx* b, int n) {
  cudaError_t e = cudaSuccess;
  for (int k = 1; k < n && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->ev[size_t(k)], b->aux[size_t(k - 1)]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev[size_t(k)], 0);
  }
  return e;
}

// One step of every lattice, each on its stream.  `flip` = 1 when the state
// sits in the other buffer than h->cur says (inside a captured interval).
// The check sums of slot s go to the batch's row s, as in mode 0.
cudaError_t launch_lattices(clbm_batch_ctx* b, bool check, int flip) {
  for (int s = 0; s < b->capacity; ++s) {
    clbm_ctx* h = b->slots[size_t(s)];
    if (!h) continue;
    double* acc = b->d_acc + 4 * size_t(s);
    CheckBufs cb{h->uprev, acc, reinterpret_cast<int*>(acc + 3)};
    const cudaStream_t st = pl_stream(b, b->stream_of[size_t(s)]);
    // the lattice's own block: the tile width of the persistent kernel's rule
    const int threads = int(b->pl_block.x * b->pl_block.y);
    const int tw = tile_width(h->g.nx, int(h->elem), int(b->pl_block.x), threads);
    const dim3 blk(unsigned(tw), unsigned(threads / tw), 1);
    cudaError_t e;
    if (h->in_place) {  // one buffer, the layout alternating with the steps
      const int lay = h->layout ^ flip;
      switch (b->dtype) {
        case CLBM_F64:
          e = launch_step_aa_f64(h->buf[0], h->g, h->P, cb, check, blk, b->pl_npt, lay, st);
          break;
        case CLBM_F32:
          e = launch_step_aa_f32(h->buf[0], h->g, h->P, cb, check, blk, b->pl_npt, lay, st);
          break;
        default:
          e = launch_step_aa_f16(h->buf[0], h->g, h->P, cb, check, blk, b->pl_npt, lay, st);
          break;
      }
      if (e != cudaSuccess) return e;
      continue;
    }
    const int c = h->cur ^ flip;
    const void* src = h->buf[c];
    void* dst = h->buf[1 - c];
    switch (b->dtype) {
      case CLBM_F64:
        e = launch_step_f64(src, dst, h->g, h->P, cb, check, blk, b->pl_npt, st);
        break;
      case CLBM_F32:
        e = launch_step_f32(src, dst, h->g, h->P, cb, check, blk, b->pl_npt, st);
        break;
      default:
        e = launch_step_f16(src, dst, h->g, h->P, cb, check, blk, b->pl_npt, st);
        break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Rebuild and upload the tables from the attached lattices' current state.
int upload(clbm_batch_ctx* b) {
  BCK(b, cudaStreamSynchronize(b->stream));  // staging buffers and tables are free
  int ntiles = 0, nlat = 0, ntiles0 = 0;
  b->h_owner.clear();
  b->h_coord.clear();
  char* stage = static_cast<char*>(b->h_stage);
  // lattices without body force first, then those with: two launches
  for (int pass = 0; pass < 2; ++pass) {
    for (int s = 0; s < b->capacity; ++s) {
      clbm_ctx* h = b->slots[s];
      // in-place lattices (mode 1 only) have no place in the tile tables
      if (!h || h->in_place || (h->P.has_force != 0) != (pass == 1)) continue;
      const int threads = int(b->block.x * b->block.y);
      const int tw = tile_width(h->g.nx, int(h->elem), int(b->block.x), threads);
      int twl = 0;
      while ((1 << twl) < tw) ++twl;
      const int th = threads / tw;
      const int tx = (h->g.nx + tw - 1) / tw;
      const int ty = (h->g.ny + th - 1) / th;
      const int tz = (h->g.nz + b->zc - 1) / b->zc;   // chunks of zc planes
      if (tx > 255 || ty > 4095 || tz > 4095)
        return bfail(b, CLBM_ERR_UNSUPPORTED, "lattice has too many tiles for the batch table");
      // the lattice's step count minus the batch's: the kernels add the
      // batch's device-side count to recover the lattice's own
      const unsigned so = unsigned(uint64_t(h->steps) - uint64_t(b->steps));
      fill_desc(b->dtype, stage + size_t(nlat) * b->desc_bytes, h, tx, ty, twl, s, so);
      for (int kz = 0; kz < tz; ++kz)
        for (int ky = 0; ky < ty; ++ky)
          for (int kx = 0; kx < tx; ++kx) {
            b->h_owner.push_back(nlat);
            b->h_coord.push_back(unsigned(kx) | (unsigned(ky) << 8) | (unsigned(kz) << 20));
          }
      ntiles += tx * ty * tz;
      ++nlat;
    }
    if (pass == 0) ntiles0 = ntiles;
  }
  if (ntiles > b->owner_cap) {
    if (b->d_owner) BCK(b, cudaFree(b->d_owner));
    if (b->d_coord) BCK(b, cudaFree(b->d_coord));
    b->d_owner = nullptr;
    b->d_coord = nullptr;
    const int cap = std::max(ntiles, 2 * b->owner_cap);
    BCK(b, cudaMalloc(reinterpret_cast<void**>(&b->d_owner), size_t(cap) * sizeof(int)));
    BCK(b, cudaMalloc(reinterpret_cast<void**>(&b->d_coord), size_t(cap) * sizeof(unsigned)));
    b->owner_cap = cap;
    drop_graph(b);  // the graph holds the old table address
  }
  const unsigned st0 = unsigned(uint64_t(b->steps));
  BatchHeader hdr{nlat, ntiles, ntiles0, 0, {st0, st0}, {0, 0}};
  if (nlat) BCK(b, upload_desc(b->dtype, stage, b->desc_base, nlat));
  if (ntiles) {
    BCK(b, cudaMemcpy(b->d_owner, b->h_owner.data(), size_t(ntiles) * sizeof(int),
                      cudaMemcpyHostToDevice));
    BCK(b, cudaMemcpy(b->d_coord, b->h_coord.data(), size_t(ntiles) * sizeof(unsigned),
                      cudaMemcpyHostToDevice));
  }
  BCK(b, cudaMemcpy(b->d_hdr, &hdr, sizeof(hdr), cudaMemcpyHostToDevice));
  if (b->mode == 1) {
    assign_streams(b);
    drop_graph(b);  // the graph holds the lattices' buffer addresses
  }
  b->parity = 0;
  b->dirty = false;
  return CLBM_OK;
}

// Advance the host-side bookkeeping of the attached handles by n steps.
void advance(clbm_batch_ctx* b, int64_t n) {
  for (clbm_ctx* h : b->slots)
    if (h) {
      h->steps += n;
      if (n & 1) {
        if (h->in_place) h->layout ^= 1;
        else h->cur = 1 - h->cur;
      }
    }
  b->steps += n;
}

int one_step(clbm_batch_ctx* b) {
  const bool check = ((b->steps + 1) % b->check_interval) == 0;
  if (check) BCK(b, cudaMemsetAsync(b->d_acc, 0, size_t(b->capacity) * 4 * sizeof(double), b->stream));
  if (b->mode == 1) {
    BCK(b, fork_streams(b, b->pl_streams));
    BCK(b, launch_lattices(b, check, 0));
    BCK(b, join_streams(b, b->pl_streams));
  } else {
    BCK(b, fork_streams(b, 2));
    BCK(b, launch(b, check));
    BCK(b, join_streams(b, 2));
  }
  b->parity ^= 1;
  if (check) {
    BCK(b, cudaMemcpyAsync(b->h_acc, b->d_acc, size_t(b->capacity) * 4 * sizeof(double),
                           cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaEventRecord(b->check_done, b->stream));
    for (int s = 0; s < b->capacity; ++s)
      if (b->slots[s]) b->slot_checks[s] += 1;
  }
  advance(b, 1);
  return CLBM_OK;
}

// Capture one check interval as a graph (parity 0 at its start).
int capture(clbm_batch_ctx* b) {
  drop_graph(b);
  cudaGraph_t g = nullptr;
  BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  if (b->mode == 1) {
    // Only the last step's check writes the sums: clear them up front, so
    // that the streams stay forked for the whole interval.
    e = cudaMemsetAsync(b->d_acc, 0, size_t(b->capacity) * 4 * sizeof(double), b->stream);
    if (e == cudaSuccess) e = fork_streams(b, b->pl_streams);
    for (int k = 0; k < b->check_interval && e == cudaSuccess; ++k)
      e = launch_lattices(b, k == b->check_interval - 1, k & 1);
    if (e == cudaSuccess) e = join_streams(b, b->pl_streams);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_acc, b->d_acc, size_t(b->capacity) * 4 * sizeof(double),
                          cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->check_done, b->stream);
  }
  if (b->mode == 0) {
    // as in mode 1: the sums are cleared up front, so that the two chains stay
    // forked for the whole interval
    e = cudaMemsetAsync(b->d_acc, 0, size_t(b->capacity) * 4 * sizeof(double), b->stream);
    if (e == cudaSuccess) e = fork_streams(b, 2);
    const int keep = b->parity;
    for (int k = 0; k < b->check_interval && e == cudaSuccess; ++k) {
      b->parity = k & 1;
      e = launch(b, k == b->check_interval - 1);
    }
    b->parity = keep;
    if (e == cudaSuccess) e = join_streams(b, 2);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_acc, b->d_acc, size_t(b->capacity) * 4 * sizeof(double),
                          cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->check_done, b->stream);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, CLBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  return CLBM_OK;
}

bool valid(const clbm_batch_ctx* b) { return b && b->d_desc; }

// Results of the last completed check of an occupied slot (the stream has
// been synchronised): residual as clbm_residual (+Inf before two checks in
// this batch), mass, divergence flag, steps.
void slot_stats(const clbm_batch_ctx* b, int slot, double* residual, double* mass,
                int* diverged, int64_t* steps) {
  const double* a = b->h_acc + 4 * slot;
  const clbm_ctx* h = b->slots[size_t(slot)];
  if (residual) {
    if (b->slot_checks[size_t(slot)] < 2) *residual = INFINITY;
    else if (!(a[1] > 0.0)) *residual = a[0] == 0.0 ? 0.0 : INFINITY;
    else *residual = std::sqrt(a[0]) / (double(b->check_interval) * std::sqrt(a[1]));
  }
  if (mass) *mass = double(h->g.nx) * h->g.ny * h->g.nz * h->g.rho0 + a[2];
  int f = 0;
  std::memcpy(&f, &a[3], sizeof(int));
  if (b->slot_checks[size_t(slot)] < 1) f = 0;
  if (diverged) *diverged = f;
  if (steps) *steps = h->steps;
}

// The kernel skips any tile whose descriptor fails its checks and sets the
// header's error word; report that instead of silently wrong results.
int check_tables(clbm_batch_ctx* b) {
  BatchHeader hdr{};
  BCK(b, cudaMemcpy(&hdr, b->d_hdr, sizeof(hdr), cudaMemcpyDeviceToHost));
  if (hdr.err) return bfail(b, CLBM_ERR_CUDA, "batch kernel found an inconsistent tile table");
  return CLBM_OK;
}

}  // namespace

extern "C" {

int clbm_batch_create(clbm_dtype dtype, int capacity, int check_interval, void* stream,
                      clbm_batch* out) {
  if (!out) return bfail(nullptr, CLBM_ERR_ARG, "null output");
  *out = nullptr;
  if (dtype != CLBM_F64 && dtype != CLBM_F32 && dtype != CLBM_F16S && dtype != CLBM_F16R)
    return bfail(nullptr, CLBM_ERR_ARG, "unknown dtype");
  if (capacity < 1 || capacity > (1 << 16)) return bfail(nullptr, CLBM_ERR_ARG, "capacity must be in [1, 65536]");
  if (check_interval <= 0) check_interval = 100;
  if (check_interval % 2) return bfail(nullptr, CLBM_ERR_ARG, "check_interval must be even");
  clbm_batch_ctx* b = new (std::nothrow) clbm_batch_ctx();
  if (!b) return bfail(nullptr, CLBM_ERR_OOM, "host allocation failed");
  b->dtype = dtype;
  if (dtype == CLBM_F64) {
    b->blocks_per_sm = 4;
    b->cap = false;
  }
  b->capacity = capacity;
  b->check_interval = check_interval;
  b->slots.assign(size_t(capacity), nullptr);
  b->slot_checks.assign(size_t(capacity), 0);
  b->slot_joined.assign(size_t(capacity), 0);
  b->desc_bytes = desc_size(dtype);  // the kernel indexes the table with this stride
  b->desc_base = table_reserve(dtype, capacity);
  if (b->desc_base < 0) {
    delete b;
    return bfail(nullptr, CLBM_ERR_UNSUPPORTED,
                 "the descriptor table of this storage form is full (" +
                     std::to_string(table_capacity(dtype)) + " lattices over all live batches)");
  }
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) {
    if (stream) {
      b->stream = static_cast<cudaStream_t>(stream);
    } else {
      e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      b->own_stream = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_desc, 256);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_hdr), sizeof(BatchHeader));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_acc), size_t(capacity) * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b->h_acc), size_t(capacity) * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_stage, size_t(capacity) * b->desc_bytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->check_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = ensure_streams(b, 2);  // the forced lattices' chain
  if (e == cudaSuccess) std::memset(b->h_acc, 0, size_t(capacity) * 4 * sizeof(double));
  if (e != cudaSuccess) {
    std::string m = std::string("clbm_batch_create: ") + cudaGetErrorString(e);
    clbm_batch_destroy(b);
    return bfail(nullptr, e == cudaErrorMemoryAllocation ? CLBM_ERR_OOM : CLBM_ERR_CUDA, m);
  }
  *out = b;
  return CLBM_OK;
}

int clbm_batch_add(clbm_batch b, clbm_handle h, int* slot) {
  if (!valid(b) || !h || !h->buf[0]) return bfail(b, CLBM_ERR_ARG, "invalid batch or handle");
  if (h->dtype != b->dtype) return bfail(b, CLBM_ERR_ARG, "lattice dtype differs from the batch's");
  if (h->in_place && b->mode != 1)
    return bfail(b, CLBM_ERR_UNSUPPORTED,
                 "in-place lattices join a batch only in its one-launch-per-lattice mode "
                 "(clbm_batch_set_lattice_launch): the persistent kernel's tiles need two buffers");
  if (h->device != b->device) return bfail(b, CLBM_ERR_ARG, "lattice lives on another device");
  if (h->sround && b->mode == 1)
    return bfail(b, CLBM_ERR_UNSUPPORTED,
                 "lattices with stochastic rounding take the persistent kernel, not the "
                 "one-launch-per-lattice mode");
  if (h->batch) return bfail(b, CLBM_ERR_ARG, "lattice is already in a batch");
  if (int64_t(NQ) * h->g.qstride >= (int64_t(1) << 31))
    return bfail(b, CLBM_ERR_UNSUPPORTED, "lattice too large to batch (19 x padded nodes >= 2^31)");
  int s = 0;
  while (s < b->capacity && b->slots[s]) ++s;
  if (s == b->capacity) return bfail(b, CLBM_ERR_ARG, "batch is full");
  BCK(b, cudaSetDevice(b->device));
  BCK(b, cudaStreamSynchronize(h->stream));  // the lattice's own queued work is done
  b->slots[s] = h;
  b->slot_checks[s] = 0;
  b->slot_joined[s] = b->steps;
  h->batch = b;
  b->dirty = true;
  if (slot) *slot = s;
  return CLBM_OK;
}

int clbm_batch_remove(clbm_batch b, int slot) {
  if (!valid(b) || slot < 0 || slot >= b->capacity || !b->slots[slot])
    return bfail(b, CLBM_ERR_ARG, "invalid batch or slot");
  BCK(b, cudaSetDevice(b->device));
  BCK(b, cudaStreamSynchronize(b->stream));  // its last batched steps are done
  b->slots[slot]->batch = nullptr;
  b->slots[slot] = nullptr;
  b->dirty = true;
  return CLBM_OK;
}

int clbm_batch_step(clbm_batch b, int64_t nsteps) {
  if (!valid(b) || nsteps < 0) return bfail(b, CLBM_ERR_ARG, "invalid batch or step count");
  BCK(b, cudaSetDevice(b->device));
  int64_t left = nsteps;
  while (left > 0) {
    if (b->dirty) {
      if (int r = upload(b)) return r;
    }
    const int64_t ci = b->check_interval;
    if (b->steps % ci == 0 && b->parity == 0 && left >= ci) {
      if (!b->graph) {
        if (int r = capture(b)) return r;
      }
      BCK(b, cudaGraphLaunch(b->graph, b->stream));
      for (int s = 0; s < b->capacity; ++s)
        if (b->slots[s]) b->slot_checks[s] += 1;
      advance(b, ci);
      left -= ci;
      continue;
    }
    if (int r = one_step(b)) return r;
    left -= 1;
  }
  return CLBM_OK;
}

int clbm_batch_stats(clbm_batch b, int slot, double* residual, double* mass, int* diverged,
                     int64_t* steps) {
  if (!valid(b) || slot < 0 || slot >= b->capacity || !b->slots[slot])
    return bfail(b, CLBM_ERR_ARG, "invalid batch or slot");
  BCK(b, cudaSetDevice(b->device));
  BCK(b, cudaStreamSynchronize(b->stream));
  if (int r = check_tables(b)) return r;
  slot_stats(b, slot, residual, mass, diverged, steps);
  return CLBM_OK;
}

int clbm_batch_stats_all(clbm_batch b, double* residual, double* mass, int* diverged,
                         int64_t* steps) {
  if (!valid(b)) return bfail(b, CLBM_ERR_ARG, "invalid batch");
  BCK(b, cudaSetDevice(b->device));
  BCK(b, cudaStreamSynchronize(b->stream));
  if (int r = check_tables(b)) return r;
  for (int s = 0; s < b->capacity; ++s) {
    if (b->slots[size_t(s)]) {
      slot_stats(b, s, residual ? residual + s : nullptr, mass ? mass + s : nullptr,
                 diverged ? diverged + s : nullptr, steps ? steps + s : nullptr);
    } else {
      if (residual) residual[s] = NAN;
      if (mass) mass[s] = NAN;
      if (diverged) diverged[s] = 0;
      if (steps) steps[s] = -1;
    }
  }
  return CLBM_OK;
}

int clbm_batch_set_launch(clbm_batch b, int block_x, int block_y, int zc, int blocks_per_sm) {
  if (!valid(b)) return bfail(b, CLBM_ERR_ARG, "invalid batch");
  const bool cap = blocks_per_sm < 0;
  if (cap) blocks_per_sm = -blocks_per_sm;
  if (block_x < 1 || block_y < 1 || block_x * block_y > 256 || (block_x * block_y) % 32 ||
      zc < 1 || blocks_per_sm < 1 || blocks_per_sm > 32)
    return bfail(b, CLBM_ERR_ARG, "bad launch shape");
  for (clbm_ctx* h : b->slots)
    if (h && h->in_place)
      return bfail(b, CLBM_ERR_UNSUPPORTED,
                   "the batch holds in-place lattices: the persistent kernel needs two buffers");
  BCK(b, cudaSetDevice(b->device));
  BCK(b, cudaStreamSynchronize(b->stream));
  b->block = dim3(block_x, block_y, 1);
  b->zc = zc;
  b->blocks_per_sm = blocks_per_sm;
  b->cap = cap;
  b->mode = 0;
  b->dirty = true;
  drop_graph(b);
  return CLBM_OK;
}

int clbm_batch_set_lattice_launch(clbm_batch b, int block_x, int block_y, int npt, int streams) {
  if (!valid(b)) return bfail(b, CLBM_ERR_ARG, "invalid batch");
  if (b->dtype == CLBM_F16R)
    return bfail(b, CLBM_ERR_UNSUPPORTED,
                 "F16R batches take the persistent kernel (its rounding is seeded by the step)");
  if (any_sround(b))
    return bfail(b, CLBM_ERR_UNSUPPORTED,
                 "a lattice rounds stochastically: the batch takes the persistent kernel");
  if (block_x < 1 || block_y < 1 || block_x * block_y > 256 || (block_x * block_y) % 32 ||
      (npt != 1 && npt != 5) || streams < 1 || streams > 16)
    return bfail(b, CLBM_ERR_ARG, "bad launch shape");
  BCK(b, cudaSetDevice(b->device));
  BCK(b, cudaStreamSynchronize(b->stream));
  BCK(b, ensure_streams(b, streams));
  b->pl_block = dim3(block_x, block_y, 1);
  b->pl_npt = npt;
  b->pl_streams = streams;
  b->mode = 1;
  b->dirty = true;
  drop_graph(b);
  return CLBM_OK;
}

int clbm_batch_autotune(clbm_batch b, int steps, int* block_x, int* block_y, int* zc,
                        int* blocks_per_sm, double* us_per_step) {
  if (!valid(b)) return bfail(b, CLBM_ERR_ARG, "invalid batch");
  BCK(b, cudaSetDevice(b->device));
  if (steps <= 0) steps = 6;
  // Save every lattice's current state: tuning runs real steps.
  BCK(b, cudaStreamSynchronize(b->stream));
  std::vector<void*> saved(size_t(b->capacity), nullptr);
  std::vector<int> cur0(size_t(b->capacity), 0), lay0(size_t(b->capacity), 0);
  std::vector<int64_t> steps0(size_t(b->capacity), 0);
  bool any_in_place = false;
  cudaError_t err = cudaSuccess;
  for (int s = 0; s < b->capacity && err == cudaSuccess; ++s) {
    clbm_ctx* h = b->slots[s];
    if (!h) continue;
    const size_t bytes = size_t(NQ) * size_t(h->g.qstride) * h->elem;
    const size_t rbytes = h->ref[0] ? f16r_ref_bytes(h->g.plane * h->g.nz) : 0;
    err = cudaMallocAsync(&saved[s], bytes + rbytes, b->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(saved[s], h->buf[h->cur], bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (err == cudaSuccess && rbytes)
      err = cudaMemcpyAsync(static_cast<char*>(saved[s]) + bytes, h->ref[h->cur], rbytes,
                            cudaMemcpyDeviceToDevice, b->stream);
    cur0[s] = h->cur;
    lay0[s] = h->layout;
    steps0[s] = h->steps;
    any_in_place = any_in_place || h->in_place;
  }
  const int64_t bsteps0 = b->steps;
  const dim3 block0 = b->block;
  const int zc0 = b->zc, bps0 = b->blocks_per_sm;
  const int shapes[][2] = {{32, 2}, {32, 4}, {32, 8}, {64, 2}, {64, 4}, {128, 1}, {128, 2}};
  const int zcs[] = {1, 2, 4};
  const int bpss[] = {4, 6, 8};
  const bool cap0 = b->cap;
  double best = 1e300;
  int bx = block0.x, by = block0.y, bz = zc0, bb = bps0;
  bool bc = cap0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  // the persistent kernel only when every lattice has two buffers
  for (int capped = 0; capped <= 1 && !any_in_place; ++capped)
  for (auto& sh : shapes)
    for (int z : zcs)
      for (int bp : bpss) {
        if (err != cudaSuccess) break;
        if (sh[0] * sh[1] * bp > 2048) continue;   // at most 2048 threads per SM
        b->mode = 0;
        b->cap = capped != 0;
        b->block = dim3(sh[0], sh[1], 1);
        b->zc = z;
        b->blocks_per_sm = bp;
        b->dirty = true;
        if (upload(b) != CLBM_OK) { err = cudaErrorUnknown; break; }
        err = fork_streams(b, 2);
        for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
          err = launch(b, false);
          b->parity ^= 1;
        }
        if (err == cudaSuccess) err = join_streams(b, 2);
        if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
        if (err == cudaSuccess) err = fork_streams(b, 2);
        for (int k = 0; k < steps && err == cudaSuccess; ++k) {
          err = launch(b, false);
          b->parity ^= 1;
        }
        if (err == cudaSuccess) err = join_streams(b, 2);
        if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && 1e3 * ms / steps < best) {
          best = 1e3 * ms / steps;
          bx = sh[0];
          by = sh[1];
          bz = z;
          bb = bp;
          bc = capped != 0;
        }
      }
  // One launch per lattice (not for F16R, nor with a stochastically rounding
  // lattice): block x kernel variant x streams.
  int bmode = 0, pbx = 32, pby = 2, pnpt = 5, pst = 4;
  if (b->dtype != CLBM_F16R && !any_sround(b)) {
    const int pshapes[][2] = {{32, 2}, {32, 4}, {64, 2}};
    const int pnpts[] = {5, 1};
    const int pstreams[] = {2, 4, 8};
    if (err == cudaSuccess) err = ensure_streams(b, 8);
    for (auto& sh : pshapes)
      for (int np : pnpts)
        for (int ns : pstreams) {
          if (err != cudaSuccess) break;
          b->mode = 1;
          b->pl_block = dim3(sh[0], sh[1], 1);
          b->pl_npt = np;
          b->pl_streams = ns;
          b->dirty = true;
          if (upload(b) != CLBM_OK) { err = cudaErrorUnknown; break; }
          err = fork_streams(b, b->pl_streams);
          for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
            err = launch_lattices(b, false, b->parity);
            b->parity ^= 1;
          }
          if (err == cudaSuccess) err = join_streams(b, b->pl_streams);
          if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
          if (err == cudaSuccess) err = fork_streams(b, b->pl_streams);
          for (int k = 0; k < steps && err == cudaSuccess; ++k) {
            err = launch_lattices(b, false, b->parity);
            b->parity ^= 1;
          }
          if (err == cudaSuccess) err = join_streams(b, b->pl_streams);
          if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
          if (err == cudaSuccess) err = cudaEventSynchronize(e1);
          float ms = 0.0f;
          if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
          if (err == cudaSuccess && 1e3 * ms / steps < best) {
            best = 1e3 * ms / steps;
            bmode = 1;
            pbx = sh[0];
            pby = sh[1];
            pnpt = np;
            pst = ns;
          }
        }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // Restore states, counters and the chosen shape.
  for (int s = 0; s < b->capacity; ++s) {
    clbm_ctx* h = b->slots[s];
    if (!h || !saved[s]) continue;
    h->cur = cur0[s];
    h->layout = lay0[s];
    h->steps = steps0[s];
    const size_t bytes = size_t(NQ) * size_t(h->g.qstride) * h->elem;
    const size_t rbytes = h->ref[0] ? f16r_ref_bytes(h->g.plane * h->g.nz) : 0;
    cudaError_t e2 = cudaMemcpyAsync(h->buf[h->cur], saved[s], bytes, cudaMemcpyDeviceToDevice,
                                     b->stream);
    if (e2 == cudaSuccess && rbytes)
      e2 = cudaMemcpyAsync(h->ref[h->cur], static_cast<char*>(saved[s]) + bytes, rbytes,
                           cudaMemcpyDeviceToDevice, b->stream);
    if (err == cudaSuccess) err = e2;
    cudaFreeAsync(saved[s], b->stream);
  }
  b->steps = bsteps0;
  b->block = dim3(bx, by, 1);
  b->zc = bz;
  b->blocks_per_sm = bb;
  b->cap = bc;
  b->mode = bmode;
  b->pl_block = dim3(pbx, pby, 1);
  b->pl_npt = pnpt;
  b->pl_streams = pst;
  b->dirty = true;
  drop_graph(b);
  cudaError_t e3 = cudaStreamSynchronize(b->stream);
  if (err == cudaSuccess) err = e3;
  if (err != cudaSuccess)
    return bfail(b, CLBM_ERR_CUDA, std::string("clbm_batch_autotune: ") + cudaGetErrorString(err));
  if (bmode == 1) {
    // zc = 0: one launch per lattice; |blocks_per_sm| = streams, negative
    // for the register-capped kernel
    if (block_x) *block_x = pbx;
    if (block_y) *block_y = pby;
    if (zc) *zc = 0;
    if (blocks_per_sm) *blocks_per_sm = pnpt == 5 ? -pst : pst;
  } else {
    if (block_x) *block_x = bx;
    if (block_y) *block_y = by;
    if (zc) *zc = bz;
    if (blocks_per_sm) *blocks_per_sm = bc ? -bb : bb;  // negative: register-capped variant
  }
  if (us_per_step) *us_per_step = best;
  return CLBM_OK;
}

int clbm_batch_sync(clbm_batch b) {
  if (!valid(b)) return bfail(b, CLBM_ERR_ARG, "invalid batch");
  BCK(b, cudaSetDevice(b->device));
  BCK(b, cudaStreamSynchronize(b->stream));
  return check_tables(b);
}

int clbm_batch_destroy(clbm_batch b) {
  if (!b) return CLBM_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (clbm_ctx* h : b->slots)
    if (h) h->batch = nullptr;
  drop_graph(b);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->desc_base >= 0) table_release(b->dtype, b->desc_base);
  if (b->d_owner) cudaFree(b->d_owner);
  if (b->d_coord) cudaFree(b->d_coord);
  if (b->d_hdr) cudaFree(b->d_hdr);
  if (b->d_acc) cudaFree(b->d_acc);
  if (b->h_acc) cudaFreeHost(b->h_acc);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->check_done) cudaEventDestroy(b->check_done);
  for (cudaEvent_t ev : b->ev) cudaEventDestroy(ev);
  for (cudaStream_t st : b->aux) cudaStreamDestroy(st);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return CLBM_OK;
}

const char* clbm_batch_last_error(clbm_batch b) { return b ? b->err.c_str() : ""; }

int clbm_batch_detach(clbm_batch b, clbm_handle h) {
  if (!valid(b) || !h) return bfail(b, CLBM_ERR_ARG, "invalid batch or handle");
  for (int s = 0; s < b->capacity; ++s)
    if (b->slots[s] == h) return clbm_batch_remove(b, s);
  return bfail(b, CLBM_ERR_ARG, "lattice is not in this batch");
}

}  // extern "C"
