// fno_gemm.cu -- the strided batched product of fno_gemm.cuh on the fifth-generation tensor
// cores (tcgen05.mma, BF16 x BF16 -> FP32, accumulator in tensor memory).
//
// CTA tile 128 (M) x 64 (N) x 32 (K), four warps.  Per K-tile, all threads gather the A and
// B elements through the operand strides (FP32 or BF16 in memory), round them to BF16 and
// store them in shared memory in the tensor core's K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes (8 BF16), 128 bytes apart along K and 512 bytes apart from
// one 8-row group to the next.  One thread then issues the two K = 16 MMAs of the tile
// (shared-memory descriptors for A and B, instruction descriptor for M = 128, N = 64) and
// commits them to the mbarrier of the tile's stage.  Two stages alternate, so the gather of
// the next tile overlaps the MMAs of the current one; a stage is overwritten only after its
// previous MMAs have completed, and the last commit (which covers every earlier MMA) is
// awaited before the accumulator is read.
// The FP32 accumulator occupies 64 columns of tensor memory, row i in lane i; each warp
// reads back its 32 rows (tcgen05.ld 32x32b) for the epilogue, alpha * acc + beta * C or an
// atomic add.
//
// Waits are bounded: if an MMA has not completed after kWaitLimit polls (or the caller's
// bound), the kernel raises the caller's fault word, writes NaN into its tile (so the result
// cannot pass for a valid one) and drains: the issuing thread commits once more to a
// separate mbarrier, which tracks every MMA it issued, and the CTA waits for that (bounded
// as well) before it frees its tensor memory.  Only if the drain wait also runs out does
// the CTA return without freeing, since MMAs may then still write that memory; the fault
// word stays set.  The test hook (GemmArgs::stall) issues neither the MMAs nor their
// commits, so every wait for a tile runs out with no tensor-core work in flight and the
// drain completes at once.  The 29 KB of shared memory per CTA keeps at most 7 CTAs on an
// SM, whose 7 x 64 columns fit in the 512 columns of tensor memory, so the allocation
// never has to wait for another CTA.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "fno_gemm.cuh"

namespace sslbm {

namespace {

constexpr int TM = 128, TN = 64, TK = 32;
constexpr int kTmemCols = 64;
constexpr uint32_t kLbo = 128, kSbo = 512;  // bytes: next core matrix along K / next 8-row group
constexpr int kABytes = TM * TK * 2, kBBytes = TN * TK * 2, kStageBytes = kABytes + kBBytes;
constexpr int kSmemBytes = 29 * 1024;  // caps residency at 7 CTAs per SM (tensor memory budget)
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ float load_elem(const void* p, int bf16, int64_t off) {
  return bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(p)[off])
              : static_cast<const float*>(p)[off];
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a K-major operand tile in the no-swizzle core-matrix layout
__device__ __forceinline__ uint32_t tile_offset(int row, int k) {
  return (uint32_t)(k >> 3) * kLbo + (uint32_t)(row >> 3) * kSbo + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// Elements k .. k+7 (those below kend) of one row or column of an operand, rounded to BF16 and
// packed in k order (the lower k in the lower half of each 32-bit word); zeros outside.
__device__ __forceinline__ uint4 gather8(const void* p, int bf16, bool in_range, int64_t base, int64_t sk0,
                                         int64_t sk1, int k, int kend, int K, int K0) {
  // eight consecutive in-range elements at a 16-byte boundary: vector loads, same values
  if (in_range && sk0 == 1 && K0 == K && k + 8 <= kend) {
    if (bf16) {
      const __nv_bfloat16* q = static_cast<const __nv_bfloat16*>(p) + base + k;
      if ((reinterpret_cast<uintptr_t>(q) & 15) == 0) return *reinterpret_cast<const uint4*>(q);
    } else {
      const float* q = static_cast<const float*>(p) + base + k;
      if ((reinterpret_cast<uintptr_t>(q) & 15) == 0) {
        const float4 lo = reinterpret_cast<const float4*>(q)[0], hi = reinterpret_cast<const float4*>(q)[1];
        const __nv_bfloat162 t0 = __floats2bfloat162_rn(lo.x, lo.y), t1 = __floats2bfloat162_rn(lo.z, lo.w);
        const __nv_bfloat162 t2 = __floats2bfloat162_rn(hi.x, hi.y), t3 = __floats2bfloat162_rn(hi.z, hi.w);
        return make_uint4(*reinterpret_cast<const uint32_t*>(&t0), *reinterpret_cast<const uint32_t*>(&t1),
                          *reinterpret_cast<const uint32_t*>(&t2), *reinterpret_cast<const uint32_t*>(&t3));
      }
    }
  }
  float v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int kq = k + q;
    v[q] = 0.f;
    if (in_range && kq < kend) {
      const int k1 = (K0 == K) ? 0 : kq / K0, kk = (K0 == K) ? kq : kq - k1 * K0;
      v[q] = load_elem(p, bf16, base + (int64_t)kk * sk0 + (int64_t)k1 * sk1);
    }
  }
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    w[q] = *reinterpret_cast<const uint32_t*>(&t);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets,
// fixed version bits 46..48 = 0b001, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLbo >> 4) << 16) | ((uint64_t)(kSbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

// C(off) = alpha v + beta C(off), or an atomic add of alpha v (split-K)
__device__ __forceinline__ void store_c(const GemmArgs& g, int64_t off, float acc) {
  const float v = g.alpha * acc;
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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(128) gemm_tc_kernel(const GemmArgs g) {
  static_assert(2 * kStageBytes + 32 <= kSmemBytes, "two stages, the barriers and the tensor-memory slot fit");
  static_assert(4 * 32 * 33 * 4 <= 2 * kStageBytes, "the epilogue's staging fits in the stage buffers");
  __shared__ __align__(1024) unsigned char smem[kSmemBytes];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kStageBytes);  // one per stage, then the drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * kStageBytes + 24);
  __shared__ int s_fault, s_stuck;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int bz = blockIdx.z / g.splits, sz = blockIdx.z % g.splits;
  const int kchunk = ((g.K + g.splits - 1) / g.splits + TK - 1) / TK * TK;
  const int kbeg = sz * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const bool a_kfast = g.sAk0 == 1, b_kfast = g.sBk0 == 1;
  const uint32_t bar_addr[2] = {smem_u32(bar), smem_u32(bar + 1)};
  const uint32_t drain_addr = smem_u32(bar + 2);
  const long long limit = g.wait_limit > 0 ? g.wait_limit : kWaitLimit;

  if (tid == 0) {
    s_fault = 0;
    s_stuck = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_addr[0]) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_addr[1]) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(drain_addr) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  bool any = false;
  int t = 0;  // K-tile number; tile t uses stage t & 1 and is that stage's (t >> 1)-th commit
  for (int k0 = kbeg; k0 < kend; k0 += TK, ++t) {
    const int st = t & 1;
    unsigned char* sA = smem + st * kStageBytes;
    unsigned char* sB = sA + kABytes;
    if (t >= 2) {  // the stage's previous MMAs (tile t - 2) must have read it
      if (!mbar_wait(bar_addr[st], (uint32_t)((t - 2) >> 1) & 1u, limit)) s_fault = 1;
      __syncthreads();
      if (s_fault) break;
    }
    // gather the tiles, one 16-byte core-matrix row (8 consecutive k) per unit; consecutive
    // threads walk the operand's unit-stride dimension, so global reads stay coalesced
    for (int u = tid; u < TM * (TK / 8); u += 128) {
      const int i = a_kfast ? u / (TK / 8) : u % TM;
      const int kg = a_kfast ? u % (TK / 8) : u / TM;
      *reinterpret_cast<uint4*>(sA + tile_offset(i, 8 * kg)) =
          gather8(g.A, g.a_bf16, m0 + i < g.M, bz * g.sAb + (int64_t)(m0 + i) * g.sAm, g.sAk0, g.sAk1, k0 + 8 * kg,
                  kend, g.K, g.K0);
    }
    for (int u = tid; u < TN * (TK / 8); u += 128) {
      const int i = b_kfast ? u / (TK / 8) : u % TN;  // n within the tile
      const int kg = b_kfast ? u % (TK / 8) : u / TN;
      *reinterpret_cast<uint4*>(sB + tile_offset(i, 8 * kg)) =
          gather8(g.B, g.b_bf16, n0 + i < g.N, bz * g.sBb + (int64_t)(n0 + i) * g.sBn, g.sBk0, g.sBk1, k0 + 8 * kg,
                  kend, g.K, g.K0);
    }
    // make the generic-proxy stores visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && !g.stall) {  // the test hook issues nothing, so no wait can succeed
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int s = 0; s < TK / 16; ++s) {
        const uint64_t ad = smem_desc(smem_u32(sA) + s * 2 * kLbo);
        const uint64_t bd = smem_desc(smem_u32(sB) + s * 2 * kLbo);
        const uint32_t acc = (any || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       bar_addr[st])
                   : "memory");
    }
    any = true;
  }
  if (any && !s_fault) {  // the last commit covers every MMA issued before it
    const int last = t - 1;
    if (!mbar_wait(bar_addr[last & 1], (uint32_t)(last >> 1) & 1u, limit)) s_fault = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  const bool fault = s_fault != 0;
  if (fault) {
    // drain: a commit tracks every earlier MMA of the thread that issues it, so once this
    // one arrives no MMA of the CTA can still read shared memory or write tensor memory
    if (tid == 0) {
      if (g.fault) atomicExch(g.fault, 1u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       drain_addr)
                   : "memory");
      if (!mbar_wait(drain_addr, 0u, limit)) s_stuck = 1;
    }
    __syncthreads();
  }
  // epilogue: thread (warp, lane) holds row 32 warp + lane, columns 32 h .. 32 h + 31 of each
  // half; when C is row-major the warp passes its 32 x 32 block through shared memory (the
  // stage buffers are idle now) so that lanes write consecutive columns
  const bool rowmajor = g.sCn == 1;
  float* stage = reinterpret_cast<float*>(smem) + warp * (32 * 33);
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    uint32_t r[32];
    if (any && !fault) {
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * h);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    } else {
      const float fill = fault ? __int_as_float(0x7fc00000) : 0.f;  // NaN marks a timed-out tile
#pragma unroll
      for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(fill);
    }
    if (rowmajor) {
#pragma unroll
      for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);
      __syncwarp();
      const int n = n0 + 32 * h + lane;
      for (int i = 0; i < 32; ++i) {
        const int mi = m0 + 32 * warp + i;
        if (mi < g.M && n < g.N) store_c(g, bz * g.sCb + (int64_t)mi * g.sCm + n, stage[i * 33 + lane]);
      }
      __syncwarp();
    } else {
      const int m = m0 + 32 * warp + lane;
      if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + 32 * h + j;
          if (n < g.N) store_c(g, bz * g.sCb + (int64_t)m * g.sCm + (int64_t)n * g.sCn, __uint_as_float(r[j]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  // after a drain that also ran out, MMAs may still write this tensor memory: it is not
  // handed back (the fault word is set and the results are NaN)
  if (warp == 0 && !s_stuck) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

cudaError_t gemm_bf16(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0 || g.splits <= 0 || g.K0 <= 0 || g.K % g.K0 != 0)
    return cudaErrorInvalidValue;
  if (g.atomic && g.c_bf16) return cudaErrorInvalidValue;
  if ((int64_t)g.batch * g.splits > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, g.batch * g.splits);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  gemm_tc_kernel<<<grid, 128, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace sslbm
