// step_f64.cu -- kernels of the f64 storage form (double storage, double collision).
#include "batch.cuh"
#include "kernels.cuh"

CLBM_DEFINE_LAUNCHERS(f64, double, double)
CLBM_DEFINE_AA(f64, double, double)
CLBM_DEFINE_BATCH(f64, double, double, false)
