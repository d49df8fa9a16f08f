// step_f32.cu -- kernels of the f32 storage form (float storage, float collision).
#include "batch.cuh"
#include "kernels.cuh"

CLBM_DEFINE_LAUNCHERS(f32, float, float)
CLBM_DEFINE_AA(f32, float, float)
CLBM_DEFINE_BATCH(f32, float, float, false)
