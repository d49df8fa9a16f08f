// probe.cu -- fused multiply-add throughput of the current GPU in FP64 and
// FP32: the arithmetic ceiling of a step form whose collision is bound by
// its arithmetic pipe rather than by HBM (the FP64 form on GB300).
//
// Every thread runs eight independent FMA chains a <- a * b + c (b just
// below 1, so the chains settle at c / (1 - b) with no overflow and no
// subnormals) in a loop the compiler cannot remove: the result of one
// thread in the whole grid is written to a file-scope device word.
#include <cuda_runtime.h>

#include "../../include/clbm.h"

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;

static __device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T b, T c, int iters) {
  T a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = a[0];
#pragma unroll
  for (int k = 1; k < CHAINS; ++k) s += a[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) g_probe_sink = double(s);
}

template <typename T>
int probe(int iters, double* flops_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CLBM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CLBM_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CLBM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CLBM_ERR_CUDA;
  }
  const T b = T(0.999999), c = T(1e-7);
  fma_chains_kernel<T><<<blocks, threads>>>(b, c, iters / 8);  // warm-up, clocks up
  cudaEventRecord(e0, 0);
  fma_chains_kernel<T><<<blocks, threads>>>(b, c, iters);
  cudaEventRecord(e1, 0);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.0f)) return CLBM_ERR_CUDA;
  const double flops = 2.0 * CHAINS * UNROLL * double(iters) * double(blocks) * threads;
  *flops_per_s = flops / (double(ms) * 1e-3);
  return CLBM_OK;
}

}  // namespace

extern "C" int clbm_probe_fma_rate(clbm_dtype dtype, double* flops_per_s) {
  if (!flops_per_s) return CLBM_ERR_ARG;
  // iteration counts sized for roughly 0.1 s on a GB300 (about 1.2 TFLOP/s
  // FP64, 80 TFLOP/s FP32)
  if (dtype == CLBM_F64) return probe<double>(1536, flops_per_s);
  if (dtype == CLBM_F32) return probe<float>(98304, flops_per_s);
  return CLBM_ERR_ARG;
}
