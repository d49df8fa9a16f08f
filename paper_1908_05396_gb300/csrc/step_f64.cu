// step_f64.cu -- kernels of the f64 storage form (double storage, double collision).
#include "kernels.cuh"

CLBM_DEFINE_LAUNCHERS(f64, double, double)
