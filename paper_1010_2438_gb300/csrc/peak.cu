// The FP64 pipe's peak rate on the current GPU, measured: the denominator of
// the simulation kernels' roofline.  The method itself needs no such kernel;
// it is part of the library so that a benchmark measures the peak on the same
// device and clocks as the kernels it rates.
//
// Every thread runs eight independent chains x <- x * m + a as separate,
// unfused round-to-nearest multiplies and adds (the instructions the
// simulation kernels issue), long enough that launch overhead vanishes, over
// a grid of 32 warps per SM.  Rate = lane-operations / CUDA-event time.
#include <cuda_runtime.h>

#include "cwcgpu.h"

namespace cwcgpu {

__device__ double g_fp64_peak_sink;

__global__ void __launch_bounds__(256) fp64_stream_kernel(int iters, double m, double a) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = __dadd_rn(__dmul_rn(x[k], m), a);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s = __dadd_rn(s, x[k]);
  if (s == 12345.678) g_fp64_peak_sink = s;   // keeps the chains live; never true for these inputs
}

}  // namespace cwcgpu

extern "C" cwc_status cwc_fp64_peak(void* stream, double* lane_ops_per_s) {
  using namespace cwcgpu;
  if (lane_ops_per_s == nullptr) return CWC_ERR_INVALID_ARG;
  *lane_ops_per_s = 0.0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CWC_ERR_CUDA;
  const int threads = 256, blocks = sms * 4, iters = 4096;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CWC_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CWC_ERR_CUDA;
  }
  // m just below 1 and a small keep x finite and normal for any iteration count
  fp64_stream_kernel<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-6);   // warm-up
  float best = -1.0f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    fp64_stream_kernel<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-6);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return CWC_ERR_CUDA;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.0f || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || best <= 0.0f) return CWC_ERR_CUDA;
  const double ops = (double)blocks * threads * (double)iters * 8.0 * 2.0;
  *lane_ops_per_s = ops / (best * 1e-3);
  return CWC_OK;
}
