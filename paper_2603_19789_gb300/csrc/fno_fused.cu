// fno_fused.cu -- fused forward kernels of the learned surrogate (see fno_fused.cuh).
#include <cuda_bf16.h>

#include <atomic>

#include "fno_fused.cuh"

namespace sslbm {
namespace fno_fused {
namespace {

typedef __nv_bfloat162 bf162;

constexpr int kRowThreads = 256;  // 8 warps; warp w owns grid columns [w n/8, (w+1) n/8)
constexpr int kCin = 8;           // input channels

__device__ __forceinline__ unsigned saddr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_groups() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ldmatrix: four (or two) 8x8 b16 tiles; lane l supplies the address of row l % 8 of tile l / 8
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(saddr(p)));
}

__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The A fragment of a 16 x 16 tile of a row-major [m][k] array with row stride ld (elements)
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const bf16* base, int ld, int m0, int k0, int lane) {
  ldsm_x4(a, base + (m0 + (lane & 15)) * ld + k0 + (lane >> 4) * 8);
}
// B fragments (k16 x n8) of n tiles n0 and n0 + 8 from a [k][n] array (n contiguous)
__device__ __forceinline__ void load_b_kn2(uint32_t (&b)[4], const bf16* base, int ld, int k0, int n0, int lane) {
  ldsm_x4_t(b, base + (k0 + (lane & 15)) * ld + n0 + (lane >> 4) * 8);
}
__device__ __forceinline__ void load_b_kn1(uint32_t (&b)[2], const bf16* base, int ld, int k0, int n0, int lane) {
  ldsm_x2_t(b, base + (k0 + (lane & 15)) * ld + n0);
}
// B fragments from an [n][k] array (k contiguous)
__device__ __forceinline__ void load_b_nk2(uint32_t (&b)[4], const bf16* base, int ld, int k0, int n0, int lane) {
  ldsm_x4(b, base + (n0 + (lane & 7) + (lane >> 4) * 8) * ld + k0 + ((lane >> 3) & 1) * 8);
}
__device__ __forceinline__ void load_b_nk1(uint32_t (&b)[2], const bf16* base, int ld, int k0, int n0, int lane) {
  ldsm_x2(b, base + (n0 + (lane & 7)) * ld + k0 + ((lane >> 3) & 1) * 8);
}

// the same GELU as the unfused path: the tanh form, 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
// with the hardware tanh (tanh.approx.f32)
__device__ __forceinline__ float gelu(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.7978845608028654f * fmaf(0.044715f * z, z * z, z)));
  const float h = 0.5f * z;
  return fmaf(h, t, h);
}

__device__ __forceinline__ void st_bf2(bf16* p, float a, float b) {
  *reinterpret_cast<bf162*>(p) = __floats2bfloat162_rn(a, b);
}

// ---- row kernel -------------------------------------------------------------------------

template <int W, int KF, int H, int NT, int MODE>
struct RowSmem {
  static constexpr int n = 64 * NT, SH = n + 8, SF = KF + 8, SB = W + 8, SQ = H + 8;
  static constexpr bool lift = MODE == ROW_LIFT, last = MODE == ROW_LAST;
  static constexpr size_t oF = 0;                                             // bf16 [n][SF]
  static constexpr size_t oBl = oF + (size_t)n * SF * 2;                       // bf16 [W][SB]
  static constexpr size_t oOut = oBl + (lift ? 0 : (size_t)W * SB * 2);        // bf16 [W][SH]
  // one input row: x (8 planes, FP32) or {h_{l-1} [W][SH], G1 [W][SF]} (BF16)
  static constexpr size_t stage = lift ? (size_t)kCin * n * 4 : (size_t)W * SH * 2 + (size_t)W * SF * 2;
  // f32 [2][W][KF] partial sums of the next layer's transform along x: in the current input
  // stage (dead after the first product) when they fit, else a region of their own
  static constexpr size_t red_bytes = (size_t)2 * W * KF * 4;
  static constexpr bool red_in_stage = MODE == ROW_MID && red_bytes <= stage;
  static constexpr size_t oRed = oOut + (size_t)W * SH * 2;
  static constexpr size_t oQ1 = oRed + (last || red_in_stage ? 0 : red_bytes);  // bf16 [H][SB]
  static constexpr size_t oQ2 = oQ1 + (last ? (size_t)H * SB * 2 : 0);         // bf16 [16][SQ]
  static constexpr size_t oA0 = oQ2 + (last ? (size_t)16 * SQ * 2 : 0);        // f32 [W][12]
  static constexpr size_t oStage = oA0 + (lift ? (size_t)W * 12 * 4 : 0);
  // input rows in flight: two ahead, except the last layer (two CTAs per SM need the room)
  static constexpr int NST = last ? 2 : 3;
  static constexpr size_t bytes = oStage + NST * stage;
  static_assert(!last || (H / 2 <= W && H % 32 == 0), "half of the projection fits in a stage");
};

template <int W, int KF, int H, int NT, int MODE>
__global__ void __launch_bounds__(kRowThreads, 2) row_kernel(const RowArgs a) {
  using S = RowSmem<W, KF, H, NT, MODE>;
  constexpr int n = S::n, SH = S::SH, SF = S::SF, SB = S::SB, SQ = S::SQ;
  constexpr int CW = 8 * NT;  // columns per warp
  constexpr int MT = W / 16;  // 16-row tiles of the channel dimension
  static_assert(W % 16 == 0 && KF % 16 == 0 && H % 16 == 0, "tile multiples");
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* sF = reinterpret_cast<bf16*>(smem + S::oF);
  bf16* sBl = reinterpret_cast<bf16*>(smem + S::oBl);
  bf16* sOut = reinterpret_cast<bf16*>(smem + S::oOut);
  bf16* sQ1 = reinterpret_cast<bf16*>(smem + S::oQ1);
  bf16* sQ2 = reinterpret_cast<bf16*>(smem + S::oQ2);
  float* sA0 = reinterpret_cast<float*>(smem + S::oA0);
  unsigned char* stage0 = smem + S::oStage;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gr = lane >> 2, tg = lane & 3;
  const int rows = a.B * n;

  // constants, published by the first barrier of the row loop
  for (int i = tid; i < n * (KF / 8); i += kRowThreads) {
    const int r = i / (KF / 8), c = i - r * (KF / 8);
    *reinterpret_cast<uint4*>(sF + r * SF + 8 * c) = *reinterpret_cast<const uint4*>(a.F + (size_t)r * KF + 8 * c);
  }
  if (MODE == ROW_LIFT) {
    // sA0[o][0..7] = A0[o][:], sA0[o][8] = a0[o]
    for (int i = tid; i < W * 9; i += kRowThreads) {
      const int o = i / 9, c = i - o * 9;
      sA0[o * 12 + c] = c < kCin ? a.A0[o * kCin + c] : a.a0[o];
    }
  } else {
    for (int i = tid; i < W * W; i += kRowThreads) sBl[(i / W) * SB + i % W] = a.Bl[i];
  }
  if (MODE == ROW_LAST) {
    for (int i = tid; i < H * W; i += kRowThreads) sQ1[(i / W) * SB + i % W] = a.Q1[i];
    for (int i = tid; i < 16 * H; i += kRowThreads) {
      const int r = i / H, c = i - r * H;
      sQ2[r * SQ + c] = r < 5 ? a.Q2[r * H + c] : __float2bfloat16_rn(0.f);
    }
  }
  float bias[MT][2];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    bias[mt][0] = MODE == ROW_LIFT ? 0.f : a.bl[mt * 16 + gr];
    bias[mt][1] = MODE == ROW_LIFT ? 0.f : a.bl[mt * 16 + gr + 8];
  }

  auto issue = [&](int row, int s) {
    if (row < rows) {
      const int b = row / n, y = row - b * n;
      unsigned char* st = stage0 + s * S::stage;
      if (MODE == ROW_LIFT) {
        float* dx = reinterpret_cast<float*>(st);
        for (int i = tid; i < kCin * (n / 4); i += kRowThreads) {
          const int c = i / (n / 4), j = i - c * (n / 4);
          cp16(dx + c * n + 4 * j, a.x + (((size_t)b * kCin + c) * n + y) * n + 4 * j);
        }
      } else {
        bf16* dh = reinterpret_cast<bf16*>(st);
        bf16* dg = dh + W * SH;
        for (int i = tid; i < W * (n / 8); i += kRowThreads) {
          const int c = i / (n / 8), j = i - c * (n / 8);
          cp16(dh + c * SH + 8 * j, a.hin + (((size_t)b * W + c) * n + y) * n + 8 * j);
        }
        for (int i = tid; i < W * (KF / 8); i += kRowThreads) {
          const int c = i / (KF / 8), j = i - c * (KF / 8);
          cp16(dg + c * SF + 8 * j, a.g1 + (((size_t)b * n + y) * W + c) * KF + 8 * j);
        }
      }
    }
    commit();  // possibly empty: every thread keeps the same group count
  };

  constexpr int NST = S::NST;
#pragma unroll
  for (int k = 0; k < NST - 1; ++k) issue(blockIdx.x + k * gridDim.x, k);
  int s = 0;
  for (int row = blockIdx.x; row < rows; row += gridDim.x, s = s + 1 == NST ? 0 : s + 1) {
    issue(row + (NST - 1) * gridDim.x, s == 0 ? NST - 1 : s - 1);
    wait_groups<NST - 1>();
    __syncthreads();
    const int b = row / n, y = row - b * n;
    const int x0 = warp * CW;
    unsigned char* st = stage0 + s * S::stage;
    // scratch that reuses the current input stage once the first product has read it
    float* sRed = S::red_in_stage ? reinterpret_cast<float*>(st) : reinterpret_cast<float*>(smem + S::oRed);
    bf16* sP = reinterpret_cast<bf16*>(st);  // [H/2][SH] (last layer)

    if (MODE == ROW_LIFT) {
      // h0 = A0 x + a0 in FP32, one grid column per thread
      const float* xs = reinterpret_cast<const float*>(st);
      for (int xx = tid; xx < n; xx += kRowThreads) {
        float xin[kCin];
#pragma unroll
        for (int c = 0; c < kCin; ++c) xin[c] = xs[c * n + xx];
        for (int o = 0; o < W; ++o) {
          float acc = sA0[o * 12 + kCin];
#pragma unroll
          for (int c = 0; c < kCin; ++c) acc = fmaf(sA0[o * 12 + c], xin[c], acc);
          sOut[o * SH + xx] = __float2bfloat16_rn(acc);
        }
      }
    } else {
      // z[o, x] = sum_i B[o, i] h[i, x] + sum_k G1[o, k] Fxi[k, x] + b[o]  (K = W + 4m)
      const bf16* sh = reinterpret_cast<const bf16*>(st);
      const bf16* sg = sh + W * SH;
      float acc[MT][NT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0.f;
#pragma unroll
      for (int k0 = 0; k0 < W; k0 += 16) {
        uint32_t af[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) load_a(af[mt], sBl, SB, mt * 16, k0, lane);
#pragma unroll
        for (int nt = 0; nt < NT; nt += 2) {
          if (nt + 1 < NT) {
            uint32_t bf[4];
            load_b_kn2(bf, sh, SH, k0, x0 + nt * 8, lane);
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
              mma(acc[mt][nt], af[mt], bf[0], bf[1]);
              mma(acc[mt][nt + 1], af[mt], bf[2], bf[3]);
            }
          } else {
            uint32_t bf[2];
            load_b_kn1(bf, sh, SH, k0, x0 + nt * 8, lane);
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) mma(acc[mt][nt], af[mt], bf[0], bf[1]);
          }
        }
      }
#pragma unroll
      for (int k0 = 0; k0 < KF; k0 += 16) {
        uint32_t af[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) load_a(af[mt], sg, SF, mt * 16, k0, lane);
#pragma unroll
        for (int nt = 0; nt < NT; nt += 2) {
          if (nt + 1 < NT) {
            uint32_t bf[4];
            load_b_nk2(bf, sF, SF, k0, x0 + nt * 8, lane);  // Fxi[k][x] = Fx[x][k]
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
              mma(acc[mt][nt], af[mt], bf[0], bf[1]);
              mma(acc[mt][nt + 1], af[mt], bf[2], bf[3]);
            }
          } else {
            uint32_t bf[2];
            load_b_nk1(bf, sF, SF, k0, x0 + nt * 8, lane);
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) mma(acc[mt][nt], af[mt], bf[0], bf[1]);
          }
        }
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int o = mt * 16 + gr + 8 * h2, xx = x0 + nt * 8 + 2 * tg;
            float z0 = acc[mt][nt][2 * h2] + bias[mt][h2], z1 = acc[mt][nt][2 * h2 + 1] + bias[mt][h2];
            if (MODE == ROW_MID) {
              if (a.store) st_bf2(a.zout + (((size_t)b * W + o) * n + y) * n + xx, z0, z1);
              z0 = gelu(z0);
              z1 = gelu(z1);
            }
            st_bf2(sOut + o * SH + xx, z0, z1);
          }
    }
    __syncthreads();

    if (MODE != ROW_LAST || a.store) {
      for (int i = tid; i < W * (n / 8); i += kRowThreads) {
        const int c = i / (n / 8), j = i - c * (n / 8);
        *reinterpret_cast<uint4*>(a.hout + (((size_t)b * W + c) * n + y) * n + 8 * j) =
            *reinterpret_cast<const uint4*>(sOut + c * SH + 8 * j);
      }
    }

    if (MODE != ROW_LAST) {
      // next layer's transform along x: H1[o, k] = sum_x h[o, x] Fx[x, k]; warp = (tile group,
      // half of x); the two halves meet in shared memory
      constexpr int T2 = MT * (KF / 8), TPG = T2 / 4;
      static_assert(T2 % 4 == 0, "tile groups");
      const int g = warp & 3, kh = warp >> 2;
      float acc2[TPG][4];
#pragma unroll
      for (int u = 0; u < TPG; ++u)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc2[u][r] = 0.f;
      for (int k0 = kh * (n / 2); k0 < (kh + 1) * (n / 2); k0 += 16) {
#pragma unroll
        for (int u = 0; u < TPG; ++u) {
          const int t = g * TPG + u, mt = t / (KF / 8), nt = t - mt * (KF / 8);
          uint32_t af[4], bf[2];
          load_a(af, sOut, SH, mt * 16, k0, lane);
          load_b_kn1(bf, sF, SF, k0, nt * 8, lane);
          mma(acc2[u], af, bf[0], bf[1]);
        }
      }
#pragma unroll
      for (int u = 0; u < TPG; ++u) {
        const int t = g * TPG + u, mt = t / (KF / 8), nt = t - mt * (KF / 8);
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int o = mt * 16 + gr + 8 * h2, c = nt * 8 + 2 * tg;
          sRed[(kh * W + o) * KF + c] = acc2[u][2 * h2];
          sRed[(kh * W + o) * KF + c + 1] = acc2[u][2 * h2 + 1];
        }
      }
      __syncthreads();
      bf16* dst = a.H1out + ((size_t)b * n + y) * W * KF;
      for (int i = tid; i < W * KF / 2; i += kRowThreads)
        st_bf2(dst + 2 * i, sRed[2 * i] + sRed[W * KF + 2 * i], sRed[2 * i + 1] + sRed[W * KF + 2 * i + 1]);
    } else {
      // projection on the warp's own columns: p = gelu(Q1 h_L + q1), delta = Q2 p + q2, in two
      // halves of the H rows of p (each half staged in the warp's columns of sP)
      constexpr int MH = H / 32;  // 16-row tiles per half
      float acc4[NT][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc4[nt][r] = 0.f;
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        const int h0 = half * (H / 2);
        float acc3[MH][NT][4];
#pragma unroll
        for (int mh = 0; mh < MH; ++mh)
#pragma unroll
          for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc3[mh][nt][r] = 0.f;
#pragma unroll
        for (int k0 = 0; k0 < W; k0 += 16) {
          uint32_t af[MH][4];
#pragma unroll
          for (int mh = 0; mh < MH; ++mh) load_a(af[mh], sQ1, SB, h0 + mh * 16, k0, lane);
#pragma unroll
          for (int nt = 0; nt < NT; nt += 2) {
            if (nt + 1 < NT) {
              uint32_t bf[4];
              load_b_kn2(bf, sOut, SH, k0, x0 + nt * 8, lane);
#pragma unroll
              for (int mh = 0; mh < MH; ++mh) {
                mma(acc3[mh][nt], af[mh], bf[0], bf[1]);
                mma(acc3[mh][nt + 1], af[mh], bf[2], bf[3]);
              }
            } else {
              uint32_t bf[2];
              load_b_kn1(bf, sOut, SH, k0, x0 + nt * 8, lane);
#pragma unroll
              for (int mh = 0; mh < MH; ++mh) mma(acc3[mh][nt], af[mh], bf[0], bf[1]);
            }
          }
        }
        __syncwarp();  // the previous half's reads of this warp's sP columns are done
#pragma unroll
        for (int mh = 0; mh < MH; ++mh)
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int hl = mh * 16 + gr + 8 * h2, hh = h0 + hl;
            const float qv = a.q1[hh];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
              const int xx = x0 + nt * 8 + 2 * tg;
              const float z0 = acc3[mh][nt][2 * h2] + qv, z1 = acc3[mh][nt][2 * h2 + 1] + qv;
              const size_t off = (((size_t)b * H + hh) * n + y) * n + xx;
              if (a.store) st_bf2(a.zp + off, z0, z1);
              const bf162 pv = __floats2bfloat162_rn(gelu(z0), gelu(z1));
              *reinterpret_cast<bf162*>(sP + hl * SH + xx) = pv;
              if (a.store) *reinterpret_cast<bf162*>(a.p + off) = pv;
            }
          }
        __syncwarp();
#pragma unroll
        for (int k0 = 0; k0 < H / 2; k0 += 16) {
          uint32_t af[4];
          load_a(af, sQ2, SQ, 0, h0 + k0, lane);
#pragma unroll
          for (int nt = 0; nt < NT; nt += 2) {
            if (nt + 1 < NT) {
              uint32_t bf[4];
              load_b_kn2(bf, sP, SH, k0, x0 + nt * 8, lane);
              mma(acc4[nt], af, bf[0], bf[1]);
              mma(acc4[nt + 1], af, bf[2], bf[3]);
            } else {
              uint32_t bf[2];
              load_b_kn1(bf, sP, SH, k0, x0 + nt * 8, lane);
              mma(acc4[nt], af, bf[0], bf[1]);
            }
          }
        }
      }
      if (gr < 5) {
        // v_c = sigma_c max(x_c + delta_c, 0), sigma_E = sigma_I = 10^(4e - 4) from the scale
        // channel: the nonnegative raw prediction (the conservation step rescales it); the
        // clamp keeps a NaN a NaN, so a non-finite prediction stays visible to the checks
        const int c = gr;
        const float qc = a.q2[c];
        const float sig = (c == 1 || c == 2) ? exp10f(4.f * a.x[((size_t)b * kCin + 7) * n * n] - 4.f) : 1.f;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int xx = x0 + nt * 8 + 2 * tg;
          const float2 xv = *reinterpret_cast<const float2*>(a.x + (((size_t)b * kCin + c) * n + y) * n + xx);
          float2 out;
          out.x = xv.x + (acc4[nt][0] + qc);
          out.y = xv.y + (acc4[nt][1] + qc);
          out.x = out.x < 0.f ? 0.f : out.x;
          out.y = out.y < 0.f ? 0.f : out.y;
          if (c == 1 || c == 2) {
            out.x *= sig;
            out.y *= sig;
          }
          *reinterpret_cast<float2*>(a.y + (((size_t)b * 5 + c) * n + y) * n + xx) = out;
        }
      }
    }
    __syncthreads();
  }
  wait_groups<0>();
}

// ---- transform along y and combine ---------------------------------------------------------

// CTA = (sample b, CG channels): T[c] = Fy (2m x n) H1[b, :, c, :] (n x 4m), combined into
// hat[b, c, j, q] = (T[2q, 2j] - T[2q+1, 2j+1], T[2q, 2j+1] + T[2q+1, 2j])
template <int KF, int CG>
__global__ void __launch_bounds__(128) dft_y_kernel(const bf16* __restrict__ H1, const bf16* __restrict__ Fy,
                                                    float* __restrict__ hat, int W, int n) {
  constexpr int M2 = KF / 2, m = KF / 4, NC = CG * KF, SC = NC + 8, modes = 2 * m * m;
  constexpr int NTT = NC / 8, TPW = NTT / 4;
  static_assert(NTT % 4 == 0 && M2 <= 32, "tiling");
  extern __shared__ __align__(16) unsigned char smem[];
  const int SY = n + 8;
  bf16* sFy = reinterpret_cast<bf16*>(smem);          // [32][SY], rows >= 2m zero
  bf16* sT = sFy + 32 * SY;                            // [n][SC]
  float* sO = reinterpret_cast<float*>(sT + (size_t)n * SC);  // [2m][NC]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gr = lane >> 2, tg = lane & 3;
  const int b = blockIdx.y, c0 = blockIdx.x * CG;
  for (int i = tid; i < 32 * (n / 8); i += 128) {
    const int r = i / (n / 8), j = i - r * (n / 8);
    if (r < M2)
      cp16(sFy + r * SY + 8 * j, Fy + (size_t)r * n + 8 * j);
    else
      *reinterpret_cast<uint4*>(sFy + r * SY + 8 * j) = make_uint4(0, 0, 0, 0);
  }
  for (int i = tid; i < n * (NC / 8); i += 128) {
    const int yy = i / (NC / 8), j = i - yy * (NC / 8);
    cp16(sT + yy * SC + 8 * j, H1 + (((size_t)b * n + yy) * W + c0) * KF + 8 * j);
  }
  commit();
  wait_groups<0>();
  __syncthreads();
  float acc[2][TPW][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int u = 0; u < TPW; ++u)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[mt][u][r] = 0.f;
  for (int k0 = 0; k0 < n; k0 += 16) {
    uint32_t af[2][4];
    load_a(af[0], sFy, SY, 0, k0, lane);
    load_a(af[1], sFy, SY, 16, k0, lane);
#pragma unroll
    for (int u = 0; u < TPW; ++u) {
      uint32_t bf[2];
      load_b_kn1(bf, sT, SC, k0, (warp * TPW + u) * 8, lane);
      mma(acc[0][u], af[0], bf[0], bf[1]);
      mma(acc[1][u], af[1], bf[0], bf[1]);
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int u = 0; u < TPW; ++u)
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int r = mt * 16 + gr + 8 * h2, col = (warp * TPW + u) * 8 + 2 * tg;
        if (r < M2) {
          sO[r * NC + col] = acc[mt][u][2 * h2];
          sO[r * NC + col + 1] = acc[mt][u][2 * h2 + 1];
        }
      }
  __syncthreads();
  for (int i = tid; i < CG * modes; i += 128) {
    const int cc = i / modes, k = i - cc * modes, j = k / m, q = k - j * m;
    const float* T = sO + cc * KF;
    const float re = T[(2 * q) * NC + 2 * j] - T[(2 * q + 1) * NC + 2 * j + 1];
    const float im = T[(2 * q) * NC + 2 * j + 1] + T[(2 * q + 1) * NC + 2 * j];
    float* h = hat + (((size_t)b * W + c0 + cc) * modes + k) * 2;
    h[0] = re;
    h[1] = im;
  }
}

// ---- spectral mix ------------------------------------------------------------------------

// CTA = MC modes: hatg[b, o, k] = sum_i hat[b, i, k] R[i, o, k] (complex), all b and o.  Each
// mode's weights R[:, :, k] are read once and applied to the whole batch.
template <int MC, int BC>
__global__ void __launch_bounds__(256) mix_kernel(const float2* __restrict__ hat, const float2* __restrict__ R,
                                                  float2* __restrict__ hatg, int B, int W, int modes) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* sR = reinterpret_cast<float2*>(smem);  // [W][W][MC]
  float2* sHt = sR + (size_t)W * W * MC;         // [BC][W][MC]
  const int tid = threadIdx.x;
  const int k0 = blockIdx.x * MC;
  const int mc = min(MC, modes - k0);
  const float2 zero = make_float2(0.f, 0.f);
  for (int i = tid; i < W * W * MC; i += 256) {
    const int io = i / MC, kk = i - io * MC;
    sR[i] = kk < mc ? R[(size_t)io * modes + k0 + kk] : zero;
  }
  for (int b0 = 0; b0 < B; b0 += BC) {
    const int nb = min(BC, B - b0);
    __syncthreads();
    for (int i = tid; i < nb * W * MC; i += 256) {
      const int bi = i / MC, kk = i - bi * MC;
      sHt[i] = kk < mc ? hat[((size_t)b0 * W + bi) * modes + k0 + kk] : zero;
    }
    __syncthreads();
    for (int t = tid; t < nb * W; t += 256) {
      const int bl = t / W, o = t - bl * W;
      float re[MC], im[MC];
#pragma unroll
      for (int kk = 0; kk < MC; ++kk) re[kk] = im[kk] = 0.f;
      for (int i = 0; i < W; ++i) {
#pragma unroll
        for (int kk = 0; kk < MC; ++kk) {
          const float2 h = sHt[(bl * W + i) * MC + kk], r = sR[(i * W + o) * MC + kk];
          re[kk] = fmaf(h.x, r.x, fmaf(-h.y, r.y, re[kk]));
          im[kk] = fmaf(h.x, r.y, fmaf(h.y, r.x, im[kk]));
        }
      }
#pragma unroll
      for (int kk = 0; kk < MC; ++kk)
        if (kk < mc) hatg[((size_t)(b0 + bl) * W + o) * modes + k0 + kk] = make_float2(re[kk], im[kk]);
    }
  }
}

// ---- inverse transform along y -------------------------------------------------------------

// CTA = (sample b, OG output channels): U[o] = expand(hatg[b, o]) (2m x 4m, the c_ky weights
// of the real inverse), then G1[b, y, o, :] = bf16(scale * Fyi[y, :] U[o])
template <int KF, int OG>
__global__ void __launch_bounds__(256) idft_y_kernel(const float2* __restrict__ hatg, const bf16* __restrict__ Fyi,
                                                     bf16* __restrict__ G1, int W, int n, float scale) {
  constexpr int M2 = KF / 2, m = KF / 4, modes = 2 * m * m, NC = OG * KF, SU = NC + 8, SY = 40;
  constexpr int NTT = NC / 8;
  static_assert(NTT % 2 == 0 && M2 <= 32, "tiling");
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* sFyi = reinterpret_cast<bf16*>(smem);  // [n][SY], columns >= 2m zero
  bf16* sU = sFyi + (size_t)n * SY;             // [32][SU], rows >= 2m zero
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gr = lane >> 2, tg = lane & 3;
  const int b = blockIdx.y, o0 = blockIdx.x * OG;
  const bf16 zero = __float2bfloat16_rn(0.f);
  for (int i = tid; i < n * 32; i += 256) {
    const int yy = i >> 5, r = i & 31;
    sFyi[yy * SY + r] = r < M2 ? Fyi[(size_t)yy * M2 + r] : zero;
  }
  for (int i = tid; i < (32 - M2) * NC; i += 256) sU[(M2 + i / NC) * SU + i % NC] = zero;
  for (int i = tid; i < OG * modes; i += 256) {
    const int oo = i / modes, k = i - oo * modes;
    const float2 g = hatg[((size_t)b * W + o0 + oo) * modes + k];
    const int j = k / m, q = k - j * m;
    const float cw = q == 0 ? 1.f : 2.f;
    bf16* U = sU + oo * KF;
    U[(2 * q) * SU + 2 * j] = __float2bfloat16_rn(cw * g.x);
    U[(2 * q + 1) * SU + 2 * j] = __float2bfloat16_rn(-cw * g.y);
    U[(2 * q) * SU + 2 * j + 1] = __float2bfloat16_rn(cw * g.y);
    U[(2 * q + 1) * SU + 2 * j + 1] = __float2bfloat16_rn(cw * g.x);
  }
  __syncthreads();
  for (int mt = warp; mt < n / 16; mt += 8) {
    float acc[NTT][4];
#pragma unroll
    for (int t = 0; t < NTT; ++t)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[t][r] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < 32; k0 += 16) {
      uint32_t af[4];
      load_a(af, sFyi, SY, mt * 16, k0, lane);
#pragma unroll
      for (int t = 0; t < NTT; t += 2) {
        uint32_t bf[4];
        load_b_kn2(bf, sU, SU, k0, t * 8, lane);
        mma(acc[t], af, bf[0], bf[1]);
        mma(acc[t + 1], af, bf[2], bf[3]);
      }
    }
#pragma unroll
    for (int t = 0; t < NTT; ++t)
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int yy = mt * 16 + gr + 8 * h2, col = t * 8 + 2 * tg;
        st_bf2(G1 + (((size_t)b * n + yy) * W + o0) * KF + col, acc[t][2 * h2] * scale, acc[t][2 * h2 + 1] * scale);
      }
  }
}

// ---- per-cell channel products (the backward pass's contractions over channels) ---------------

constexpr int kCellChunk = 128;  // grid cells per work item

// S chunk [K][128] (FP32 or BF16 in memory) -> BF16 shared tile [64][136], zero outside
__device__ __forceinline__ void load_cell_tile(bf16* dst, const void* src, int src_bf16, int K, int64_t P,
                                               int64_t p0, int tid, int nthreads) {
  const bf16 zero = __float2bfloat16_rn(0.f);
  if ((P & 3) == 0) {
    for (int i = tid; i < 64 * (kCellChunk / 4); i += nthreads) {
      const int k = i / (kCellChunk / 4), j = 4 * (i - k * (kCellChunk / 4));
      bf16* d = dst + k * (kCellChunk + 8) + j;
      const int64_t p = p0 + j;
      if (k < K && p < P) {
        if (src_bf16) {
          const uint2 v = *reinterpret_cast<const uint2*>(static_cast<const bf16*>(src) + (size_t)k * P + p);
          *reinterpret_cast<uint2*>(d) = v;
        } else {
          const float4 v = *reinterpret_cast<const float4*>(static_cast<const float*>(src) + (size_t)k * P + p);
          *reinterpret_cast<bf162*>(d) = __floats2bfloat162_rn(v.x, v.y);
          *reinterpret_cast<bf162*>(d + 2) = __floats2bfloat162_rn(v.z, v.w);
        }
      } else {
        d[0] = d[1] = d[2] = d[3] = zero;
      }
    }
  } else {
    for (int i = tid; i < 64 * kCellChunk; i += nthreads) {
      const int k = i / kCellChunk, j = i - k * kCellChunk;
      const int64_t p = p0 + j;
      float v = 0.f;
      if (k < K && p < P)
        v = src_bf16 ? __bfloat162float(static_cast<const bf16*>(src)[(size_t)k * P + p])
                     : static_cast<const float*>(src)[(size_t)k * P + p];
      dst[k * (kCellChunk + 8) + j] = __float2bfloat16_rn(v);
    }
  }
}

// C[b](rows x P) = alpha Wm (rows x K) S[b] (K x P) + beta C[b];  rows, K <= 64.  CTA work item:
// (b, 128 cells); warp w owns cells [16w, 16w + 16) of the item, all rows.
__global__ void __launch_bounds__(256) cell_map_kernel(int B, int rows, int K, int64_t P, const bf16* __restrict__ Wm,
                                                       int64_t sWr, int64_t sWk, const void* __restrict__ S,
                                                       int s_bf16, void* __restrict__ C, int c_bf16, float alpha,
                                                       float beta) {
  constexpr int SW = 72, SS = kCellChunk + 8;
  __shared__ __align__(16) bf16 sW[64 * SW];
  __shared__ __align__(16) bf16 sS[64 * SS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gr = lane >> 2, tg = lane & 3;
  for (int i = tid; i < 64 * 64; i += 256) {
    const int r = i >> 6, k = i & 63;
    sW[r * SW + k] = (r < rows && k < K) ? Wm[r * sWr + k * sWk] : __float2bfloat16_rn(0.f);
  }
  const int MT = (rows + 15) / 16, KS = (K + 15) / 16;
  const int64_t chunks = (P + kCellChunk - 1) / kCellChunk, items = (int64_t)B * chunks;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int b = (int)(it / chunks);
    const int64_t p0 = (it - (int64_t)b * chunks) * kCellChunk;
    __syncthreads();
    load_cell_tile(sS, s_bf16 ? (const void*)(static_cast<const bf16*>(S) + (size_t)b * K * P)
                              : (const void*)(static_cast<const float*>(S) + (size_t)b * K * P),
                   s_bf16, K, P, p0, tid, 256);
    __syncthreads();
    float acc[4][2][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0.f;
    for (int ks = 0; ks < KS; ++ks) {
      uint32_t bf[4];
      load_b_kn2(bf, sS, SS, ks * 16, warp * 16, lane);
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        if (mt < MT) {
          uint32_t af[4];
          load_a(af, sW, SW, mt * 16, ks * 16, lane);
          mma(acc[mt][0], af, bf[0], bf[1]);
          mma(acc[mt][1], af, bf[2], bf[3]);
        }
      }
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      if (mt >= MT) continue;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int r = mt * 16 + gr + 8 * h2;
          const int64_t p = p0 + warp * 16 + nt * 8 + 2 * tg;
          if (r >= rows) continue;
          const size_t off = ((size_t)b * rows + r) * P + p;
          for (int e = 0; e < 2; ++e) {
            if (p + e >= P) continue;
            const float v = alpha * acc[mt][nt][2 * h2 + e];
            if (c_bf16) {
              bf16* c = static_cast<bf16*>(C) + off + e;
              *c = __float2bfloat16_rn(beta != 0.f ? v + beta * __bfloat162float(*c) : v);
            } else {
              float* c = static_cast<float*>(C) + off + e;
              *c = beta != 0.f ? v + beta * *c : v;
            }
          }
        }
    }
  }
}

// dW (rows x cols) += sum_b sum_p D[b](rows x P) A[b](cols x P)^T;  rows, cols <= 64.  Each CTA
// accumulates its work items in registers and adds them to dW once.
__global__ void __launch_bounds__(256) cell_wgrad_kernel(int B, int rows, int cols, int64_t P,
                                                         const float* __restrict__ D, const void* __restrict__ A,
                                                         int a_bf16, float* __restrict__ dW) {
  constexpr int SS = kCellChunk + 8;
  __shared__ __align__(16) bf16 sD[64 * SS];
  __shared__ __align__(16) bf16 sA[64 * SS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gr = lane >> 2, tg = lane & 3;
  const int MT = (rows + 15) / 16, NT = (cols + 7) / 8, T = MT * NT;
  const int64_t chunks = (P + kCellChunk - 1) / kCellChunk, items = (int64_t)B * chunks;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[u][r] = 0.f;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int b = (int)(it / chunks);
    const int64_t p0 = (it - (int64_t)b * chunks) * kCellChunk;
    __syncthreads();
    load_cell_tile(sD, D + (size_t)b * rows * P, 0, rows, P, p0, tid, 256);
    load_cell_tile(sA, a_bf16 ? (const void*)(static_cast<const bf16*>(A) + (size_t)b * cols * P)
                              : (const void*)(static_cast<const float*>(A) + (size_t)b * cols * P),
                   a_bf16, cols, P, p0, tid, 256);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = warp + 8 * u;
      if (t >= T) continue;
      const int mt = t / NT, nt = t - mt * NT;
#pragma unroll
      for (int k0 = 0; k0 < kCellChunk; k0 += 16) {
        uint32_t af[4], bf[2];
        load_a(af, sD, SS, mt * 16, k0, lane);
        load_b_nk1(bf, sA, SS, k0, nt * 8, lane);
        mma(acc[u], af, bf[0], bf[1]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int t = warp + 8 * u;
    if (t >= T) continue;
    const int mt = t / NT, nt = t - mt * NT;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int r = mt * 16 + gr + 8 * h2, c = nt * 8 + 2 * tg;
      if (r < rows && c < cols) atomicAdd(dW + r * cols + c, acc[u][2 * h2]);
      if (r < rows && c + 1 < cols) atomicAdd(dW + r * cols + c + 1, acc[u][2 * h2 + 1]);
    }
  }
}

// ---- launchers -------------------------------------------------------------------------------

constexpr int kMaxDev = 64;

// Per-device caches are atomics: concurrent callers on several host threads may fill the same
// entry, with equal values.
int sm_count() {
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (!v && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
    cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

template <int W, int KF, int H, int NT, int MODE>
cudaError_t launch_row_t(const RowArgs& a, cudaStream_t s) {
  using S = RowSmem<W, KF, H, NT, MODE>;
  static std::atomic<int> per_sm[kMaxDev];  // set after the kernel's shared-memory attribute
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  auto kern = row_kernel<W, KF, H, NT, MODE>;
  int per = per_sm[dev].load(std::memory_order_acquire);
  if (!per) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kRowThreads, S::bytes)) != cudaSuccess)
      return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    per_sm[dev].store(per, std::memory_order_release);
  }
  const int rows = a.B * S::n;
  const int grid = rows < per * sm_count() ? rows : per * sm_count();
  kern<<<grid, kRowThreads, S::bytes, s>>>(a);
  return cudaGetLastError();
}

template <int W, int KF, int H, int MODE>
cudaError_t row_by_n(const RowArgs& a, cudaStream_t s) {
  switch (a.n) {
    case 64: return launch_row_t<W, KF, H, 1, MODE>(a, s);
    case 128: return launch_row_t<W, KF, H, 2, MODE>(a, s);
    case 256: return launch_row_t<W, KF, H, 4, MODE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int W, int KF, int H>
cudaError_t row_by_mode(int mode, const RowArgs& a, cudaStream_t s) {
  switch (mode) {
    case ROW_LIFT: return row_by_n<W, KF, H, ROW_LIFT>(a, s);
    case ROW_MID: return row_by_n<W, KF, H, ROW_MID>(a, s);
    case ROW_LAST: return row_by_n<W, KF, H, ROW_LAST>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int KF, int CG>
cudaError_t launch_dft_y_t(int W, int B, int n, const bf16* H1, const bf16* Fy, float* hat, cudaStream_t s) {
  constexpr int NC = CG * KF;
  const size_t bytes = (size_t)32 * (n + 8) * 2 + (size_t)n * (NC + 8) * 2 + (size_t)(KF / 2) * NC * 4;
  cudaError_t e = cudaFuncSetAttribute(dft_y_kernel<KF, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  dft_y_kernel<KF, CG><<<dim3(W / CG, B), 128, bytes, s>>>(H1, Fy, hat, W, n);
  return cudaGetLastError();
}

template <int KF, int OG>
cudaError_t launch_mix_t(int W, int B, int n, const float* hat, const float* R, const bf16* Fyi, bf16* G1,
                         float* hatg, float scale, cudaStream_t s) {
  constexpr int MC = 2, BC = 64, m = KF / 4, modes = 2 * m * m;
  const size_t mbytes = ((size_t)W * W * MC + (size_t)BC * W * MC) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(mix_kernel<MC, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mbytes);
  if (e != cudaSuccess) return e;
  mix_kernel<MC, BC><<<(modes + MC - 1) / MC, 256, mbytes, s>>>(reinterpret_cast<const float2*>(hat),
                                                              reinterpret_cast<const float2*>(R),
                                                              reinterpret_cast<float2*>(hatg), B, W, modes);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t bytes = (size_t)n * 40 * 2 + (size_t)32 * (OG * KF + 8) * 2;
  e = cudaFuncSetAttribute(idft_y_kernel<KF, OG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  idft_y_kernel<KF, OG><<<dim3(W / OG, B), 256, bytes, s>>>(reinterpret_cast<const float2*>(hatg), Fyi, G1, W, n,
                                                           scale);
  return cudaGetLastError();
}

}  // namespace

cudaError_t cell_map(int B, int rows, int K, int64_t P, const bf16* Wm, int64_t sWr, int64_t sWk, const void* S,
                     int s_bf16, void* C, int c_bf16, float alpha, float beta, cudaStream_t s) {
  if (B < 1 || rows < 1 || rows > 64 || K < 1 || K > 64 || P < 1) return cudaErrorInvalidValue;
  const int64_t items = (int64_t)B * ((P + kCellChunk - 1) / kCellChunk);
  const int grid = (int)(items < 8 * sm_count() ? items : 8 * sm_count());
  cell_map_kernel<<<grid, 256, 0, s>>>(B, rows, K, P, Wm, sWr, sWk, S, s_bf16, C, c_bf16, alpha, beta);
  return cudaGetLastError();
}

cudaError_t cell_wgrad(int B, int rows, int cols, int64_t P, const float* D, const void* A, int a_bf16, float* dW,
                       cudaStream_t s) {
  if (B < 1 || rows < 1 || rows > 64 || cols < 1 || cols > 64 || P < 1) return cudaErrorInvalidValue;
  const int64_t items = (int64_t)B * ((P + kCellChunk - 1) / kCellChunk);
  const int grid = (int)(items < 4 * sm_count() ? items : 4 * sm_count());
  cell_wgrad_kernel<<<grid, 256, 0, s>>>(B, rows, cols, P, D, A, a_bf16, dW);
  return cudaGetLastError();
}

bool supported(int W, int m, int H, int n) {
  const bool shape = (W == 32 && m == 12 && H == 64) || (W == 16 && m == 8 && H == 32);
  return shape && (n == 64 || n == 128 || n == 256);
}

static bool spectral_supported(int W, int m, int n) {
  return ((W == 32 && m == 12) || (W == 16 && m == 8)) && (n == 64 || n == 128 || n == 256);
}

cudaError_t launch_row(int mode, int W, int m, int H, const RowArgs& a, cudaStream_t s) {
  if (!supported(W, m, H, a.n) || a.B < 1) return cudaErrorInvalidValue;
  if (W == 32) return row_by_mode<32, 48, 64>(mode, a, s);
  return row_by_mode<16, 32, 32>(mode, a, s);
}

cudaError_t launch_dft_y(int W, int m, int B, int n, const bf16* H1, const bf16* Fy, float* hat, cudaStream_t s) {
  if (!spectral_supported(W, m, n) || B < 1) return cudaErrorInvalidValue;
  if (m == 12) return launch_dft_y_t<48, 2>(W, B, n, H1, Fy, hat, s);
  return launch_dft_y_t<32, 2>(W, B, n, H1, Fy, hat, s);
}

cudaError_t launch_mix_idft_y(int W, int m, int B, int n, const float* hat, const float* R, const bf16* Fyi,
                              bf16* G1, float* hatg, float scale, cudaStream_t s) {
  if (!spectral_supported(W, m, n) || B < 1) return cudaErrorInvalidValue;
  if (m == 12) return launch_mix_t<48, 2>(W, B, n, hat, R, Fyi, G1, hatg, scale, s);
  return launch_mix_t<32, 2>(W, B, n, hat, R, Fyi, G1, hatg, scale, s);
}

}  // namespace fno_fused
}  // namespace sslbm
