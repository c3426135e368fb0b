// Test-only: Philox4x32-10 outputs from cuRAND's device generator
// (curandStatePhilox4_32_10_t), an implementation independent of this
// project's, for bit-for-bit comparison with the oracle's generator.
//
// For counter (c0, c1, c2, c3) and key (k0, k1): curand_init(seed = k0 | k1 << 32,
// subsequence = c2 | c3 << 32, offset = 4 (c0 | c1 << 32)) sets cuRAND's
// 128-bit counter to exactly (c0, c1, c2, c3) (subsequences advance the high
// 64 bits, offsets the low 64 bits in units of four outputs), and curand4
// returns the four output words of that counter.  c1 < 2^30 keeps the offset
// within 64 bits.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_philox_curand(const uint4* ctr, const uint2* key, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = ctr[i];
  const uint2 k = key[i];
  curandStatePhilox4_32_10_t st;
  curand_init((unsigned long long)k.x | ((unsigned long long)k.y << 32),
              (unsigned long long)c.z | ((unsigned long long)c.w << 32),
              4ull * ((unsigned long long)c.x | ((unsigned long long)c.y << 32)), &st);
  out[i] = curand4(&st);
}

// ctr: n x 4 words, key: n x 2 words, out: n x 4 words (host arrays).
// Returns 0 on success, else the CUDA error code.
extern "C" int philox_curand(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
  uint4 *dc = nullptr, *dout = nullptr;
  uint2* dk = nullptr;
  cudaError_t e = cudaMalloc(&dc, sizeof(uint4) * n);
  if (!e) e = cudaMalloc(&dk, sizeof(uint2) * n);
  if (!e) e = cudaMalloc(&dout, sizeof(uint4) * n);
  if (!e) e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
  if (!e) {
    k_philox_curand<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
    e = cudaGetLastError();
  }
  if (!e) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return (int)e;
}
