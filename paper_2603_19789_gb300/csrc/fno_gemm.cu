// fno_gemm.cu -- the strided batched BF16 tensor-core product of fno_gemm.cuh.
#include <cuda_bf16.h>

#include "fno_gemm.cuh"

namespace sslbm {

namespace {

constexpr int TM = 64, TN = 64, TK = 32, PAD = 40;  // smem rows padded to 40 bf16 (80 B)

__device__ __forceinline__ float load_elem(const void* p, int bf16, int64_t off) {
  return bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(p)[off])
              : static_cast<const float*>(p)[off];
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 sA[TM][PAD];  // [m][k]
  __shared__ __align__(16) __nv_bfloat16 sB[TN][PAD];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int bz = blockIdx.z / g.splits, sz = blockIdx.z % g.splits;
  const int kchunk = ((g.K + g.splits - 1) / g.splits + TK - 1) / TK * TK;
  const int kbeg = sz * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const bool a_kfast = g.sAk0 == 1, b_kfast = g.sBk0 == 1;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  for (int k0 = kbeg; k0 < kend; k0 += TK) {
    // A tile: 64 x 32 elements, 16 per thread; consecutive threads walk the unit-stride
    // dimension so global reads are coalesced.
#pragma unroll 4
    for (int e = 0; e < (TM * TK) / 128; ++e) {
      const int idx = tid + e * 128;
      const int i = a_kfast ? idx / TK : idx % TM;
      const int j = a_kfast ? idx % TK : idx / TM;
      const int m = m0 + i, k = k0 + j;
      float v = 0.f;
      if (m < g.M && k < kend) {
        const int k1 = (g.K0 == g.K) ? 0 : k / g.K0, kk = (g.K0 == g.K) ? k : k - k1 * g.K0;
        v = load_elem(g.A, g.a_bf16, bz * g.sAb + (int64_t)m * g.sAm + (int64_t)kk * g.sAk0 +
                                         (int64_t)k1 * g.sAk1);
      }
      sA[i][j] = __float2bfloat16_rn(v);
    }
#pragma unroll 4
    for (int e = 0; e < (TN * TK) / 128; ++e) {
      const int idx = tid + e * 128;
      const int i = b_kfast ? idx / TK : idx % TN;  // i: n within the tile
      const int j = b_kfast ? idx % TK : idx / TN;  // j: k within the tile
      const int n = n0 + i, k = k0 + j;
      float v = 0.f;
      if (n < g.N && k < kend) {
        const int k1 = (g.K0 == g.K) ? 0 : k / g.K0, kk = (g.K0 == g.K) ? k : k - k1 * g.K0;
        v = load_elem(g.B, g.b_bf16, bz * g.sBb + (int64_t)kk * g.sBk0 + (int64_t)k1 * g.sBk1 +
                                         (int64_t)n * g.sBn);
      }
      sB[i][j] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; kk += 16) {
      const int gr = lane >> 2, tg = lane & 3;
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gr;
        a[i][0] = *reinterpret_cast<const uint32_t*>(&sA[r][kk + 2 * tg]);
        a[i][1] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][kk + 2 * tg]);
        a[i][2] = *reinterpret_cast<const uint32_t*>(&sA[r][kk + 2 * tg + 8]);
        a[i][3] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][kk + 2 * tg + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + gr;
        b[j][0] = *reinterpret_cast<const uint32_t*>(&sB[c][kk + 2 * tg]);
        b[j][1] = *reinterpret_cast<const uint32_t*>(&sB[c][kk + 2 * tg + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }

  // epilogue: fragment (row gr / gr+8, cols 2tg, 2tg+1) of each m16n8 tile
  const int gr = lane >> 2, tg = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + i * 16 + gr + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * tg + (r & 1);
        if (m >= g.M || n >= g.N) continue;
        const int64_t off = bz * g.sCb + (int64_t)m * g.sCm + (int64_t)n * g.sCn;
        const float v = g.alpha * acc[i][j][r];
        if (g.atomic) {
          atomicAdd(static_cast<float*>(g.C) + off, v);
        } else if (g.c_bf16) {
          __nv_bfloat16* c = static_cast<__nv_bfloat16*>(g.C) + off;
          const float old = g.beta != 0.f ? __bfloat162float(*c) : 0.f;
          *c = __float2bfloat16_rn(v + g.beta * old);
        } else {
          float* c = static_cast<float*>(g.C) + off;
          *c = g.beta != 0.f ? v + g.beta * *c : v;
        }
      }
}

}  // namespace

cudaError_t gemm_bf16(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0 || g.splits <= 0 || g.K0 <= 0 ||
      g.K % g.K0 != 0)
    return cudaErrorInvalidValue;
  if (g.atomic && g.c_bf16) return cudaErrorInvalidValue;
  if ((int64_t)g.batch * g.splits > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, g.batch * g.splits);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace sslbm
