// launch_f16sr.h -- host entry of the F16S step with stochastically rounded
// stores (step_f16sr.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"

namespace clbm {

// One step of an F16S lattice from src into dst with stochastic rounding
// seeded by (node, step); npt 1 or 5 (register-capped).
cudaError_t launch_step_f16sr(const void* src, void* dst, const Geom& g, const PhysParams& P,
                              const CheckBufs& cb, bool check, dim3 block, int npt, int64_t step,
                              cudaStream_t st);

// Mark a filled F16S batch descriptor (fill_desc_f16) as rounding its
// stores stochastically (batch.cuh, LatDesc::sround).
void desc_set_sround_f16(void* out, int on);

}  // namespace clbm
