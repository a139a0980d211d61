// Reductions over replicas (Sec. 5.2: on-line reduction of many instances
// into mean trajectories; sensitivities of those means).
#include <cuda_runtime.h>

#include "cwc_internal.h"
#include "ssa_device.cuh"

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

// Variance and 90 % confidence half-width per (p, g, o) from the exact sums:
// num = R * sumsq - sum^2 (exact, unsigned 128-bit), variance =
// RN(num) / (R * (R - 1)), ci90 = z * sqrt(variance / R), each operation
// rounded to nearest.  RN(num) is assembled with integer operations.
__device__ double u128_to_double_rn(unsigned __int128 x) {
  if (x == 0) return 0.0;
  const unsigned long long hi = (unsigned long long)(x >> 64), lo = (unsigned long long)x;
  int lead = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  unsigned long long m;
  if (lead <= 52) {
    m = lo << (52 - lead);
  } else {
    const int sh = lead - 52;
    m = (unsigned long long)(x >> sh);
    const unsigned __int128 rem = x & ((((unsigned __int128)1) << sh) - 1);
    const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) m += 1ull;
    if (m == (1ull << 53)) {
      m >>= 1;
      lead += 1;
    }
  }
  return __longlong_as_double((long long)(((unsigned long long)(1023 + lead) << 52) | (m & 0x000FFFFFFFFFFFFFull)));
}

__global__ void stats_kernel(const unsigned long long* __restrict__ sums, const unsigned long long* __restrict__ sumsq,
                             double* __restrict__ variance, double* __restrict__ ci90, long long n, long long R) {
  const double Z90 = 1.6448536269514722;   // the double nearest the 0.95 quantile of N(0, 1)
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned __int128 s = sums[i];
    const unsigned __int128 q = ((unsigned __int128)sumsq[2 * i + 1] << 64) | sumsq[2 * i];
    const unsigned __int128 num = (unsigned __int128)R * q - s * s;
    const double var = R > 1 ? __ddiv_rn(u128_to_double_rn(num), __dmul_rn((double)R, (double)(R - 1))) : 0.0;
    if (variance) variance[i] = var;
    if (ci90) ci90[i] = __dmul_rn(Z90, __dsqrt_rn(__ddiv_rn(var, (double)R)));
  }
}

cudaError_t launch_stats(const unsigned long long* sums, const unsigned long long* sumsq, double* variance,
                         double* ci90, long long n, int R, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  stats_kernel<<<(unsigned)blocks, 256, 0, st>>>(sums, sumsq, variance, ci90, n, (long long)R);
  return cudaGetLastError();
}

cudaError_t launch_means(const unsigned long long* sums, double* means, long long n, int R, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  means_kernel<<<(unsigned)blocks, 256, 0, st>>>(sums, means, n, (double)R);
  return cudaGetLastError();
}

// inv[i] = 1 / k[i] (IEEE division), once per call of the score replay, so
// that a trajectory's grid points multiply by 1/k_j instead of dividing by k_j.
__global__ void reciprocal_kernel(const double* __restrict__ k, double* __restrict__ inv, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    inv[i] = __ddiv_rn(1.0, k[i]);
}

cudaError_t launch_reciprocal(const double* k, double* inv, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  reciprocal_kernel<<<(unsigned)blocks, 256, 0, st>>>(k, inv, n);
  return cudaGetLastError();
}

// The simulation's fixed logarithm over an array (for checking it against
// the oracle bit for bit).  Inputs outside [2^-53, 1), the range of the
// uniforms, give NaN.
__global__ void log_spec_kernel(const double* __restrict__ u, double* __restrict__ out, long long n,
                                const __grid_constant__ LogConstants lc) {
  __shared__ unsigned long long s_rj[64], s_tj[64];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    s_rj[i] = lc.rj[i];
    s_tj[i] = lc.tj[i];
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = u[i];
    const long long b = dbits(v);
    const bool ok = b >= 0x3CA0000000000000ll && b < 0x3FF0000000000000ll;   // 2^-53 <= v < 1
    out[i] = ok ? log_spec_q(v, lc, s_rj, s_tj) : __longlong_as_double(0x7FF8000000000000ll);
  }
}

cudaError_t launch_log_spec(const double* u, double* out, long long n, const LogConstants& lc, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  log_spec_kernel<<<(unsigned)blocks, 256, 0, st>>>(u, out, n, lc);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, double* grad, int P, int R, int M, cudaStream_t st) {
  dim3 grid((unsigned)P, (unsigned)M);
  reduce_partials_kernel<<<grid, 256, 0, st>>>(partials, grad, R, M);
  return cudaGetLastError();
}

}  // namespace cwcgpu
