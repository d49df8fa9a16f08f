// ctx.h -- the handle behind clbm_handle, shared by the host translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/clbm.h"
#include "launch.h"

namespace clbm {
// Bytes of the F16R form's reference arrays (four FP16 values per stored node, and
// slack for the stencil's reach past the last node), per buffer.
inline size_t f16r_ref_bytes(int64_t stored_nodes) { return size_t(stored_nodes + 64) * 8; }
}  // namespace clbm

struct clbm_ctx {
  int device = 0;
  clbm_domain dom{};
  clbm_dtype dtype = CLBM_F64;
  clbm::Geom g{};
  clbm::PhysParams P{};
  size_t elem = 8;       // bytes per stored population
  size_t rsize = 8;      // bytes per math-precision value
  void* buf[2] = {nullptr, nullptr};
  void* ref[2] = {nullptr, nullptr};  // F16R: per-node reference moments, with buf
  int cur = 0;           // buffer holding the current state (0 when in place)
  bool in_place = false; // one buffer, streamed in place (inplace.cuh)
  bool sround = false;   // F16S: stores rounded stochastically (step_f16sr.cu)
  int layout = 0;        // in place: the layout the buffer holds (0 swapped, 1 streamed)
  void* uprev = nullptr;
  double* acc = nullptr; // device: 3 doubles, then the int flag and the TMA error word
  int* flag = nullptr;
  double* host = nullptr; // pinned: acc[3], flag as double
  cudaEvent_t check_done = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t steps = 0;
  int64_t checks = 0;    // check steps queued so far
  bool diverged = false; // sticky once a completed check saw divergence
  bool pipeline_err = false; // sticky once a check saw a TMA wait give up
  dim3 block{32, 4, 1};
  int npt = 1;           // nodes per thread (1 or 2), + 4 for the register-capped kernel,
                         // or TMA_NPT + 32 v for the TMA-staged kernel of shape v
  struct clbm_batch_ctx* batch = nullptr;  // batch stepping this lattice, if any
  clbm_alloc_fn alloc_fn = nullptr;  // registered allocator at creation (NULL: cudaMalloc)
  clbm_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  size_t pop_bytes = 0, ref_bytes = 0, uprev_bytes = 0;  // sizes handed to free_fn
  std::string err;
};

namespace clbm {
// Queue one step of a handle (clbm_lib.cu).
cudaError_t handle_dispatch_step(clbm_ctx* h, bool check);
}  // namespace clbm
