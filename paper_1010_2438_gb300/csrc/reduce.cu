// Reductions over replicas (Sec. 5.2: on-line reduction of many instances
// into mean trajectories; sensitivities of those means).
#include <cuda_runtime.h>

#include "cwc_internal.h"

namespace cwcgpu {

// means[i] = (double)sums[i] / R, one IEEE division per element.
__global__ void means_kernel(const unsigned long long* __restrict__ sums, double* __restrict__ means, long long n,
                             double R) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    means[i] = __ddiv_rn(__ll2double_rn((long long)sums[i]), R);
}

// grad[p][j] = (sum over r of partials[p][r][j]) / R with a fixed order:
// thread t of 256 adds r = t, t+256, ... left to right, then a pairwise tree
// over the 256 partial sums (halving).  Identical from run to run.
__global__ void __launch_bounds__(256) reduce_partials_kernel(const double* __restrict__ partials,
                                                              double* __restrict__ grad, int R, int M) {
  __shared__ double s[256];
  const int p = blockIdx.x, j = blockIdx.y, t = threadIdx.x;
  const double* base = partials + (size_t)p * R * M + j;
  double acc = 0.0;
  for (int r = t; r < R; r += 256) acc = __dadd_rn(acc, base[(size_t)r * M]);
  s[t] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) s[t] = __dadd_rn(s[t], s[t + w]);
    __syncthreads();
  }
  if (t == 0) grad[(size_t)p * M + j] = __ddiv_rn(s[0], (double)R);
}

cudaError_t launch_means(const unsigned long long* sums, double* means, long long n, int R, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  means_kernel<<<(unsigned)blocks, 256, 0, st>>>(sums, means, n, (double)R);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, double* grad, int P, int R, int M, cudaStream_t st) {
  dim3 grid((unsigned)P, (unsigned)M);
  reduce_partials_kernel<<<grid, 256, 0, st>>>(partials, grad, R, M);
  return cudaGetLastError();
}

}  // namespace cwcgpu
