// Test-only check of the library's tcgen05 primitives (csrc/tc.cuh): one CTA
// of 128 threads computes C (128 x N, FP32) = A (128 x K, BF16) * B (N x K,
// BF16)^T with A and B staged in shared memory in the no-swizzle K-major
// core-matrix layout, the MMAs issued by one thread into a tensor-memory
// accumulator, completion through an mbarrier (bounded wait), the result
// read back with tcgen05.ld.  `swap` exchanges the two byte-offset fields
// of the descriptors (the check of which field is which); every address
// either reading can form stays inside the operand tiles.
#include <cstdint>
#include <cuda_bf16.h>

#include "../../paper_2105_00448_gb300/csrc/tc.cuh"

using namespace hca;

constexpr int kM = 128, kMaxN = 64, kMaxK = 64;

__global__ void __launch_bounds__(128) k_tc_gemm(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B,
                                                 float* __restrict__ C, int N, int K, int swap, int* status) {
  __shared__ __align__(128) uint16_t sA[kM * kMaxK];
  __shared__ __align__(128) uint16_t sB[kMaxN * kMaxK];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_holder;
  const int t = threadIdx.x, w = t >> 5;
  // core matrices adjacent along K consecutive (128 B apart), 8-row groups K/8 core matrices apart
  const uint32_t kstride = 128, rstrideA = (uint32_t)(K / 8) * 128, rstrideB = rstrideA;
  for (int i = t; i < kM * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    sA[tc::core_offset(r, k, kstride, rstrideA) / 2] = A[i];
  }
  for (int i = t; i < N * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    sB[tc::core_offset(r, k, kstride, rstrideB) / 2] = B[i];
  }
  if (t == 0) tc::mbar_init(&mbar, 1);
  if (w == 0) tc::alloc(&tmem_holder, 64);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_holder;
  if (t == 0) {
    const uint32_t idesc = tc::idesc_bf16(kM, N);
    for (int kk = 0; kk < K / 16; ++kk) {
      // this instruction's 16 columns: two core matrices along K
      const uint32_t aoff = (uint32_t)kk * 2 * kstride, boff = aoff;
      const uint32_t lboA = swap ? rstrideA : kstride, sboA = swap ? kstride : rstrideA;
      const uint32_t lboB = swap ? rstrideB : kstride, sboB = swap ? kstride : rstrideB;
      const uint64_t ad = tc::smem_desc(tc::smem_u32(sA) + aoff, lboA, sboA);
      const uint64_t bd = tc::smem_desc(tc::smem_u32(sB) + boff, lboB, sboB);
      tc::mma_bf16(tmem, ad, bd, idesc, kk > 0);
    }
    tc::commit(&mbar);
  }
  const bool ok = tc::mbar_wait(&mbar, 0, 1 << 22);
  if (!ok && (t & 31) == 0) atomicExch(status, 1);
  tc::fence_after();
  if (ok) {
    const int row = 32 * w + (t & 31);
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) C[row * N + c0 + j] = v[j];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (w == 0) tc::dealloc(tmem, 64);
}

extern "C" int tc_gemm(const uint16_t* A, const uint16_t* B, float* C, int N, int K, int swap) {
  if (N < 16 || N > kMaxN || N % 16 || K < 16 || K > kMaxK || K % 16) return -1;
  uint16_t *dA, *dB;
  float* dC;
  int* dS;
  int st = 0;
  if (cudaMalloc(&dA, kM * K * 2) || cudaMalloc(&dB, N * K * 2) || cudaMalloc(&dC, kM * N * 4) ||
      cudaMalloc(&dS, 4))
    return -2;
  cudaMemcpy(dA, A, kM * K * 2, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, B, N * K * 2, cudaMemcpyHostToDevice);
  cudaMemset(dC, 0, kM * N * 4);
  cudaMemset(dS, 0, 4);
  k_tc_gemm<<<1, 128>>>(dA, dB, dC, N, K, swap, dS);
  const cudaError_t e = cudaDeviceSynchronize();
  cudaMemcpy(C, dC, kM * N * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&st, dS, 4, cudaMemcpyDeviceToHost);
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  cudaFree(dS);
  if (e != cudaSuccess) return -3;
  return st ? -4 : 0;
}
