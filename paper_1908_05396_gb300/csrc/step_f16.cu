// step_f16.cu -- kernels of the f16 storage form (__half storage, float collision).
#include "batch.cuh"
#include "kernels.cuh"

CLBM_DEFINE_LAUNCHERS(f16, __half, float)
CLBM_DEFINE_AA(f16, __half, float)
CLBM_DEFINE_BATCH(f16, __half, float, false)
