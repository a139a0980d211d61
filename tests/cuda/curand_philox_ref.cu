// Test helper: raw Philox4_32_10 words from cuRAND (a library routine) for
// given (event n, purpose, replica r, point p) counters, to pin the oracle's
// Philox4x32-10.  curand_init(seed, subsequence = r | p << 32,
// offset = 4 * (n + purpose * 2^32)) positions the generator on counter
// (n, purpose, r, p); curand4 returns that counter's four words.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_ref_kernel(const unsigned* ctr, unsigned long long seed, unsigned* out, int count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  unsigned long long n = ctr[4 * i + 0], purpose = ctr[4 * i + 1], r = ctr[4 * i + 2], p = ctr[4 * i + 3];
  curandStatePhilox4_32_10_t st;
  curand_init(seed, r | (p << 32), 4ull * (n + (purpose << 32)), &st);
  uint4 w = curand4(&st);
  out[4 * i + 0] = w.x;
  out[4 * i + 1] = w.y;
  out[4 * i + 2] = w.z;
  out[4 * i + 3] = w.w;
}

extern "C" int curand_ref(const unsigned* h_ctr, unsigned long long seed, unsigned* h_out, int count) {
  unsigned *d_ctr = nullptr, *d_out = nullptr;
  size_t bytes = sizeof(unsigned) * 4 * (size_t)count;
  if (cudaMalloc(&d_ctr, bytes) != cudaSuccess) return 1;
  if (cudaMalloc(&d_out, bytes) != cudaSuccess) return 2;
  cudaMemcpy(d_ctr, h_ctr, bytes, cudaMemcpyHostToDevice);
  curand_ref_kernel<<<(count + 127) / 128, 128>>>(d_ctr, seed, d_out, count);
  cudaError_t e = cudaMemcpy(h_out, d_out, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d_ctr);
  cudaFree(d_out);
  return e == cudaSuccess ? 0 : 3;
}
