// fno_gemm.cuh -- strided, batched matrix product on BF16 tensor cores with FP32
// accumulation, used by every dense contraction of the learned surrogate (the truncated
// DFT products, the pointwise channel maps and their weight gradients).
//
//   C[b](m, n) = alpha * sum_k A[b](m, k) B[b](k, n) + beta * C[b](m, n)
//
// Every operand is addressed through explicit strides, so transposes and batched views
// cost nothing.  K may be two-level, k = k1 * K0 + k0, which lets a weight gradient sum
// over (batch, cell) in one product.  Split-K (gridDim.z = batch * splits) adds partial
// products into an FP32 C with atomics.  Operands may be FP32 or BF16 in memory; tiles
// are converted to BF16 in shared memory and multiplied by the tcgen05 tensor cores
// (bf16 x bf16 -> f32, accumulator in tensor memory).  CTA tile 128 x 64 x 32.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace sslbm {

struct GemmArgs {
  int M, N, K, K0;  // K0 = inner extent of a two-level K (K0 == K for one level)
  int batch, splits;
  const void* A;
  int a_bf16;
  int64_t sAb, sAm, sAk0, sAk1;
  const void* B;
  int b_bf16;
  int64_t sBb, sBk0, sBk1, sBn;
  void* C;
  int c_bf16;
  int64_t sCb, sCm, sCn;
  float alpha, beta;
  int atomic;  // add into FP32 C with atomics (split-K); beta is ignored
  long long wait_limit;  // polls per tensor-core wait (0: the default bound, 2^24)
  int stall;             // test hook: issue no MMA and no completion signal, so the waits run out
  unsigned int* fault;   // device word set to 1 when a wait runs out (may be NULL)
};

cudaError_t gemm_bf16(const GemmArgs& g, cudaStream_t s);

}  // namespace sslbm
