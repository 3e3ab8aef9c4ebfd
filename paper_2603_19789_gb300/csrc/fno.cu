// fno.cu -- the learned surrogate: a Fourier-neural-operator-style network that advances
// the five SEIRD fields of a periodic n x n grid by 20 SSLBM steps, with hand-written
// forward and backward passes, MSE loss and Adam, behind the C ABI of include/sslbm.h.
// The paper has no learned component; the network is defined by this project:
//
//   s  = max(max E, max I, 1e-12) per scenario (the infection scale), e = (log10 s + 4)/4,
//   s' = 10^(4e - 4);  x = [S, E/s', I/s', R, D, (R0 - 2.6)/1.4, log10(d) + 2, e]   (8 channels)
//   h0 = A0 x + a0
//   z_l = K_l(h_{l-1}) + B_l h_{l-1} + b_l, h_l = gelu(z_l) for l < L, h_L = z_L
//   p  = gelu(Q1 h_L + q1),  delta = Q2 p + q2,  v_c = sigma_c (x_c + delta_c)
//   with sigma = (1, s', s', 1, 1): E and I enter and leave in units of the infection scale;
//   y = v - u kappa with u_c = sigma_c x_c the input state and kappa = (sum v - sum u) / sum u
//   per sample, so the prediction conserves the total population.
//
// K_l is the spectral convolution on the 2m x m retained Fourier modes, evaluated as real
// DFT products: H1 = h Fx (along x), T = Fy H1 (along y), combine to complex, mix with the
// complex weights R_l, expand, G1 = Fyi U, K(h) = G1 Fxi / n^2.  The DFT products and the
// channel maps run on BF16 tensor cores with FP32 accumulation (fno_gemm.cu); activations
// are stored in BF16, parameters, gradients and optimizer moments in FP32, the spectral
// mixing in FP32 SIMT (it is small).  Parameters are one flat FP32 vector in the order
// A0, a0, {R_l, B_l, b_l}_{l=1..L}, Q1, q1, Q2, q2.
#include <cuda_bf16.h>
#include <float.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "fno_fused.cuh"
#include "fno_gemm.cuh"
#include "handles_access.cuh"
#include "sslbm_internal.cuh"

namespace sslbm {
int record_error(int status, const char* msg);
}

using sslbm::GemmArgs;
typedef __nv_bfloat16 bf16;

namespace {

int err(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return sslbm::record_error(status, buf);
}

int cuda_err(cudaError_t e, const char* what) {
  return err(SSLBM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(call, what)                            \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_err(e_, what); \
  } while (0)

// GELU in its tanh form, g(z) = 0.5 z (1 + tanh(u)), u = sqrt(2/pi) (z + 0.044715 z^3), with the
// hardware tanh (tanh.approx.f32); g'(z) = 0.5 (1 + t) + 0.5 z (1 - t^2) du/dz
__device__ __forceinline__ float tanh_hw(float x) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x));
  return t;
}
__device__ __forceinline__ float gelu_f(float z) {
  const float t = tanh_hw(0.7978845608028654f * fmaf(0.044715f * z, z * z, z));
  const float h = 0.5f * z;
  return fmaf(h, t, h);
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float t = tanh_hw(0.7978845608028654f * fmaf(0.044715f * z, z * z, z));
  const float du = 0.7978845608028654f * fmaf(3.f * 0.044715f * z, z, 1.f);
  return fmaf(0.5f * z * du, fmaf(-t, t, 1.f), 0.5f * (1.f + t));
}

constexpr int kThreads = 256;
constexpr int kCin = 8;                 // input channels
constexpr float kScaleFloor = 1e-12f;   // infection scale of a scenario without E and I

// sigma of E and I from the scale channel e of the input: s' = 10^(4e - 4)
__device__ __forceinline__ float scale_from_e(float e) { return exp10f(4.f * e - 4.f); }
// blocks per sample of the per-sample kernels (grid.y = sample)
unsigned rows_grid(int64_t P) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(32, (P + kThreads - 1) / kThreads)); }
unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads > 1048576 ? 1048576 : (n + kThreads - 1) / kThreads); }

// ---- elementwise / small kernels ---------------------------------------------------------

// h0[b, o, p] = sum_c A0[o, c] x[b, c, p] + a0[o]
__global__ void lift_kernel(const float* __restrict__ x, const float* __restrict__ A0,
                            const float* __restrict__ a0, bf16* __restrict__ h, int B, int W,
                            int64_t P) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * P;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / P, p = t - b * P;
    float xin[kCin];
#pragma unroll
    for (int c = 0; c < kCin; ++c) xin[c] = x[(b * kCin + c) * P + p];
    for (int o = 0; o < W; ++o) {
      float acc = a0[o];
#pragma unroll
      for (int c = 0; c < kCin; ++c) acc = fmaf(A0[o * kCin + c], xin[c], acc);
      h[(b * W + o) * P + p] = __float2bfloat16_rn(acc);
    }
  }
}

// z = acc + bias[ch]; optionally store z (bf16) and h = gelu(z) (or h = z) (bf16)
__global__ void bias_act_kernel(const float* __restrict__ acc, const float* __restrict__ bias,
                                bf16* __restrict__ zout, bf16* __restrict__ hout, int C, int64_t P,
                                int64_t total, int act) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)((t / P) % C);
    const float z = acc[t] + bias[ch];
    if (zout) zout[t] = __float2bfloat16_rn(z);
    hout[t] = __float2bfloat16_rn(act ? gelu_f(z) : z);
  }
}

// d *= gelu'(z)
__global__ void gelu_bwd_kernel(float* __restrict__ d, const bf16* __restrict__ z, int64_t total) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x)
    d[t] *= gelu_grad_f(__bfloat162float(z[t]));
}

// out[ch] += sum over (b, p) of src[b, ch, p]   (bias gradients)
__global__ void channel_sum_kernel(const float* __restrict__ src, float* __restrict__ out, int B,
                                   int C, int64_t P) {
  const int ch = blockIdx.y;
  float acc = 0.f;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * P;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / P, p = t - b * P;
    acc += src[(b * C + ch) * P + p];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ float sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (threadIdx.x == 0) atomicAdd(out + ch, acc);
  }
}

// v[b, c, p] = sigma_c max(x[b, c, p] + (y[b, c, p] + q2[c]), 0) with y holding Q2 p on entry:
// the nonnegative raw prediction.  The clamp keeps a NaN a NaN (fmaxf would turn it into 0,
// and the rescale would then hide a non-finite prediction from the rollout's checks).
__global__ void output_kernel(float* __restrict__ y, const float* __restrict__ q2,
                              const float* __restrict__ x, int B, int64_t P) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * 5 * P;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / (5 * P), r = t - b * 5 * P;
    const int c = (int)(r / P);
    const float a = x[b * kCin * P + r] + (y[t] + q2[c]);
    const float v = a < 0.f ? 0.f : a;
    y[t] = (c == 1 || c == 2) ? scale_from_e(x[(b * kCin + 7) * P]) * v : v;
  }
}

// Block-wide sums of FP64 values (blockDim.x a multiple of 32, <= 1024); thread 0 adds them
// to out[] (shared memory scratch of 64 doubles)
__device__ __forceinline__ void block_add2(double a, double b, double* out, double* sh) {
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[w] = a;
    sh[32 + w] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    b = threadIdx.x < nw ? sh[32 + threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, off);
      b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if (threadIdx.x == 0) {
      atomicAdd(out, a);
      atomicAdd(out + 1, b);
    }
  }
}

__device__ __forceinline__ void block_add1(double a, double* out, double* sh) {
  for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[w] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    a = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (threadIdx.x == 0) atomicAdd(out, a);
  }
}

// this block's share (strided over gridDim.x) of the sum of a plane of P values: FP32
// partials per thread, float4 loads when aligned
__device__ __forceinline__ float plane_sum(const float* __restrict__ a, int64_t P) {
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((P & 3) == 0 && (reinterpret_cast<uintptr_t>(a) & 15) == 0) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    for (int64_t i = i0; i < P / 4; i += stride) {
      const float4 v = a4[i];
      acc += (v.x + v.y) + (v.z + v.w);
    }
  } else {
    for (int64_t i = i0; i < P; i += stride) acc += a[i];
  }
  return acc;
}

// per sample b = blockIdx.y: sums[2b] += sum_{c,p} dy[b, c, p] y[b, c, p], sums[2b+1] += sum y[b, c, p]
// (y the cached prediction): the backward pass's lambda = sum(dy y) / sum y
__global__ void seed_sums_kernel(const float* __restrict__ dy, const float* __restrict__ y,
                                 double* __restrict__ sums, int64_t P5) {
  __shared__ double sh[64];
  const int64_t b = blockIdx.y;
  float sa = 0.f, sy = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P5; i += (int64_t)gridDim.x * blockDim.x) {
    const float yv = y[b * P5 + i];
    sa = fmaf(dy[b * P5 + i], yv, sa);
    sy += yv;
  }
  block_add2((double)sa, (double)sy, sums + 2 * b, sh);
}

// The forward pass's sums in one sweep (b = blockIdx.y): sums[2b] += sum of the prediction v
// over its five planes, sums[2b+1] += sum of u (u_c = sigma_c x_c, the input state).  All ten
// planes are read in one loop body, four values per plane at a time, so that many loads are
// in flight per thread.
__global__ void pred_sums_kernel(const float* __restrict__ v, const float* __restrict__ x, double* __restrict__ sums,
                                 int64_t P) {
  __shared__ double sh[64];
  const int64_t b = blockIdx.y;
  const float sg = scale_from_e(x[(b * kCin + 7) * P]);
  const float* vb = v + b * 5 * P;
  const float* xb = x + b * kCin * P;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float sv = 0.f, su_plain = 0.f, su_scaled = 0.f;  // u of E and I carries the scale sigma
  if ((P & 3) == 0 && (reinterpret_cast<uintptr_t>(vb) & 15) == 0 && (reinterpret_cast<uintptr_t>(xb) & 15) == 0) {
    for (int64_t i = i0; i < P / 4; i += stride) {
      float4 a[5], u[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        a[c] = reinterpret_cast<const float4*>(vb + c * P)[i];
        u[c] = reinterpret_cast<const float4*>(xb + c * P)[i];
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        sv += (a[c].x + a[c].y) + (a[c].z + a[c].w);
        const float q = (u[c].x + u[c].y) + (u[c].z + u[c].w);
        if (c == 1 || c == 2) su_scaled += q;
        else su_plain += q;
      }
    }
  } else {
    for (int64_t i = i0; i < P; i += stride)
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        sv += vb[c * P + i];
        if (c == 1 || c == 2) su_scaled += xb[c * P + i];
        else su_plain += xb[c * P + i];
      }
  }
  block_add2((double)sv, (double)su_plain + (double)sg * (double)su_scaled, sums + 2 * b, sh);
}

// y = v r, r = sum u / sum v (0 if sum v = 0): the prediction holds the input's population and
// stays nonnegative (b = blockIdx.y).  ratio[b] = r for the backward pass, and with ycache
// != NULL a copy of y, whose signs and sums the backward pass needs.
__global__ void conserve_kernel(float* __restrict__ y, const double* __restrict__ sums, float* __restrict__ ratio,
                                float* __restrict__ ycache, int64_t P) {
  __shared__ float rat;
  const int64_t b = blockIdx.y;
  if (threadIdx.x == 0) {
    const double sv = sums[2 * b], su = sums[2 * b + 1];
    rat = sv > 0.0 ? (float)(su / sv) : 0.f;
    if (blockIdx.x == 0) ratio[b] = rat;
  }
  __syncthreads();
  const float r = rat;
  float* yb = y + b * 5 * P;
  float* cb = ycache ? ycache + b * 5 * P : nullptr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (((5 * P) & 3) == 0 && (reinterpret_cast<uintptr_t>(yb) & 15) == 0 &&
      (cb == nullptr || (reinterpret_cast<uintptr_t>(cb) & 15) == 0)) {
    for (int64_t i = i0; i < 5 * P / 4; i += stride) {
      float4 v = reinterpret_cast<float4*>(yb)[i];
      v.x *= r, v.y *= r, v.z *= r, v.w *= r;
      reinterpret_cast<float4*>(yb)[i] = v;
      if (cb) reinterpret_cast<float4*>(cb)[i] = v;
    }
  } else {
    for (int64_t i = i0; i < 5 * P; i += stride) {
      const float v = yb[i] * r;
      yb[i] = v;
      if (cb) cb[i] = v;
    }
  }
}

// dd = sigma r [y > 0] (dy - lambda), lambda = sum(dy y) / sum y: the derivative with respect to
// delta = Q2 p + q2 through y = r v, r = sum u / sum v, v_c = sigma_c max(x_c + delta_c, 0)
// (dL/dv = r (dy - sum(dy v) / sum v), and sum(dy v) / sum v = sum(dy y) / sum y)  (b = blockIdx.y)
__global__ void scale_dy_kernel(const float* __restrict__ dy, const float* __restrict__ x,
                                const float* __restrict__ y, const double* __restrict__ sums,
                                const float* __restrict__ ratio, float* __restrict__ dd, int64_t P) {
  __shared__ float lm;
  const int64_t b = blockIdx.y;
  if (threadIdx.x == 0) {
    const double sy = sums[2 * b + 1];
    lm = sy > 0.0 ? (float)(sums[2 * b] / sy) : 0.f;
  }
  __syncthreads();
  const float lam = lm, r = ratio[b], sg = scale_from_e(x[(b * kCin + 7) * P]);
  for (int c = 0; c < 5; ++c) {
    const float f = ((c == 1 || c == 2) ? sg : 1.f) * r;
    const float* g = dy + (b * 5 + c) * P;
    const float* yc = y + (b * 5 + c) * P;
    float* d = dd + (b * 5 + c) * P;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
      d[i] = yc[i] > 0.f ? f * (g[i] - lam) : 0.f;
  }
}

// T[(b,i), 2m, 4m] -> hat[(b,i), 2m(kx), m(ky), 2]
__global__ void combine_kernel(const float* __restrict__ T, float* __restrict__ hat, int BW, int m) {
  const int64_t total = (int64_t)BW * 2 * m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % m), j = (int)((t / m) % (2 * m));
    const int64_t bi = t / (2 * m * m);
    const float* Tb = T + bi * (2 * m) * (4 * m);
    const float re = Tb[(2 * q) * 4 * m + 2 * j] - Tb[(2 * q + 1) * 4 * m + 2 * j + 1];
    const float im = Tb[(2 * q) * 4 * m + 2 * j + 1] + Tb[(2 * q + 1) * 4 * m + 2 * j];
    hat[t * 2] = re;
    hat[t * 2 + 1] = im;
  }
}

// hat_g[b, o, j, q] = sum_i hat[b, i, j, q] R[i, o, j, q] (complex), written expanded into
// U[(b,o), 2m, 4m] with the c_ky weights (c_0 = 1, c_ky = 2)
__global__ void mix_expand_kernel(const float* __restrict__ hat, const float* __restrict__ R,
                                  float* __restrict__ U, int B, int W, int m) {
  const int modes = 2 * m * m;
  const int64_t total = (int64_t)B * W * modes;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % modes);
    const int o = (int)((t / modes) % W);
    const int64_t b = t / ((int64_t)modes * W);
    float re = 0.f, im = 0.f;
    for (int i = 0; i < W; ++i) {
      const float hr = hat[((b * W + i) * modes + k) * 2], hi = hat[((b * W + i) * modes + k) * 2 + 1];
      const float rr = R[(((int64_t)i * W + o) * modes + k) * 2], ri = R[(((int64_t)i * W + o) * modes + k) * 2 + 1];
      re = fmaf(hr, rr, fmaf(-hi, ri, re));
      im = fmaf(hr, ri, fmaf(hi, rr, im));
    }
    const int q = k % m, j = k / m;
    const float c = q == 0 ? 1.f : 2.f;
    float* Ub = U + (b * W + o) * (2 * m) * (4 * m);
    Ub[(2 * q) * 4 * m + 2 * j] = c * re;
    Ub[(2 * q + 1) * 4 * m + 2 * j] = -c * im;
    Ub[(2 * q) * 4 * m + 2 * j + 1] = c * im;
    Ub[(2 * q + 1) * 4 * m + 2 * j + 1] = c * re;
  }
}

// adjoint of expand: dU[(b,o), 2m, 4m] -> dG[b, o, j, q, 2]
__global__ void expand_adj_kernel(const float* __restrict__ dU, float* __restrict__ dG, int BW, int m) {
  const int modes = 2 * m * m;
  const int64_t total = (int64_t)BW * modes;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % modes);
    const int64_t bo = t / modes;
    const int q = k % m, j = k / m;
    const float c = q == 0 ? 1.f : 2.f;
    const float* D = dU + bo * (2 * m) * (4 * m);
    const float dre = D[(2 * q) * 4 * m + 2 * j] + D[(2 * q + 1) * 4 * m + 2 * j + 1];
    const float dim = -D[(2 * q + 1) * 4 * m + 2 * j] + D[(2 * q) * 4 * m + 2 * j + 1];
    dG[t * 2] = c * dre;
    dG[t * 2 + 1] = c * dim;
  }
}

// dR[i, o, k] += sum_b conj(hat[b, i, k]) dG[b, o, k]
__global__ void dR_kernel(const float* __restrict__ hat, const float* __restrict__ dG,
                          float* __restrict__ dR, int B, int W, int m) {
  const int modes = 2 * m * m;
  const int64_t total = (int64_t)W * W * modes;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % modes);
    const int o = (int)((t / modes) % W);
    const int i = (int)(t / ((int64_t)modes * W));
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; ++b) {
      const float hr = hat[(((int64_t)b * W + i) * modes + k) * 2], hi = hat[(((int64_t)b * W + i) * modes + k) * 2 + 1];
      const float gr = dG[(((int64_t)b * W + o) * modes + k) * 2], gi = dG[(((int64_t)b * W + o) * modes + k) * 2 + 1];
      re = fmaf(hr, gr, fmaf(hi, gi, re));
      im = fmaf(hr, gi, fmaf(-hi, gr, im));
    }
    dR[t * 2] += re;
    dR[t * 2 + 1] += im;
  }
}

// dhat[b, i, k] = sum_o dG[b, o, k] conj(R[i, o, k]), written as dT (adjoint of combine)
__global__ void dhat_combine_adj_kernel(const float* __restrict__ dG, const float* __restrict__ R,
                                        float* __restrict__ dT, int B, int W, int m) {
  const int modes = 2 * m * m;
  const int64_t total = (int64_t)B * W * modes;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % modes);
    const int i = (int)((t / modes) % W);
    const int64_t b = t / ((int64_t)modes * W);
    float re = 0.f, im = 0.f;
    for (int o = 0; o < W; ++o) {
      const float gr = dG[((b * W + o) * modes + k) * 2], gi = dG[((b * W + o) * modes + k) * 2 + 1];
      const float rr = R[(((int64_t)i * W + o) * modes + k) * 2], ri = R[(((int64_t)i * W + o) * modes + k) * 2 + 1];
      re = fmaf(gr, rr, fmaf(gi, ri, re));
      im = fmaf(gi, rr, fmaf(-gr, ri, im));
    }
    const int q = k % m, j = k / m;
    float* D = dT + (b * W + i) * (2 * m) * (4 * m);
    D[(2 * q) * 4 * m + 2 * j] = re;
    D[(2 * q + 1) * 4 * m + 2 * j + 1] = -re;
    D[(2 * q) * 4 * m + 2 * j + 1] = im;
    D[(2 * q + 1) * 4 * m + 2 * j] = im;
  }
}

// per sample: sums[3b] += sum (y - t), sums[3b+1] += sum t, sums[3b+2] += sum max(-y, 0)
__global__ void loss_sums_kernel(const float* __restrict__ y, const float* __restrict__ tgt,
                                 double* __restrict__ sums, int64_t P5) {
  const int64_t b = blockIdx.y;
  double se = 0.0, st = 0.0, sn = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P5;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float tv = tgt[b * P5 + t], yv = y[b * P5 + t];
    se += (double)(yv - tv);
    st += tv;
    sn += yv < 0.f ? -(double)yv : 0.0;
  }
  for (int off = 16; off > 0; off >>= 1) {
    se += __shfl_down_sync(0xffffffffu, se, off);
    st += __shfl_down_sync(0xffffffffu, st, off);
    sn += __shfl_down_sync(0xffffffffu, sn, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums + 3 * b, se);
    atomicAdd(sums + 3 * b + 1, st);
    atomicAdd(sums + 3 * b + 2, sn);
  }
}

// The training loss (N = B * 5 * P):
//   mse_w = (1/N) sum ((y - t) / sigma_c)^2,  r_b = sum(y_b - t_b) / sum t_b,
//   n_b = sum max(-y_b, 0) / sum t_b,  L = mse_w + lm mean_b r_b^2 + ln mean_b n_b^2;
// dy = dL/dy; loss receives mse_w.  sums may be NULL when lm = ln = 0.
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ tgt,
                            const float* __restrict__ x, float* __restrict__ dy, double* __restrict__ loss,
                            int64_t N, int64_t P, const double* __restrict__ sums, float lm, float ln, int B) {
  double acc = 0.0;
  const float inv = 1.f / (float)N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / (5 * P);
    const int c = (int)((t - b * 5 * P) / P);
    const float d = y[t] - tgt[t];
    const float rs = (c == 1 || c == 2) ? 1.f / scale_from_e(x[(b * kCin + 7) * P]) : 1.f;
    const float dn = d * rs;
    float g = 2.f * dn * rs * inv;
    if (sums) {
      const double st = sums[3 * b + 1];
      if (st != 0.0) {
        g += (float)(2.0 * lm / B * (sums[3 * b] / st) / st);
        if (y[t] < 0.f) g -= (float)(2.0 * ln / B * (sums[3 * b + 2] / st) / st);
      }
    }
    dy[t] = g;
    acc += (double)dn * dn;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (double)N);
}

// Adam (decoupled weight decay), then refresh the BF16 copy used as GEMM operand
// Adam; skipped altogether when a tensor-core product of this step timed out (*fault != 0),
// so NaN gradients never reach the parameters or the moments
__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ mo,
                            float* __restrict__ ve, bf16* __restrict__ th16, int64_t P, float lr,
                            float b1, float b2, float eps, float wd, float c1, float c2,
                            const unsigned int* __restrict__ fault) {
  if (*fault) return;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float gr = g[t];
    const float m_ = b1 * mo[t] + (1.f - b1) * gr;
    const float v_ = b2 * ve[t] + (1.f - b2) * gr * gr;
    mo[t] = m_;
    ve[t] = v_;
    const float upd = (m_ / c1) / (sqrtf(v_ / c2) + eps);
    const float nt = th[t] - lr * (upd + wd * th[t]);
    th[t] = nt;
    th16[t] = __float2bfloat16_rn(nt);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ a, bf16* __restrict__ b, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    b[t] = __float2bfloat16_rn(a[t]);
}

// real DFT factors (see fno.py's dft_mats): Fx [n][4m], Fy [2m][n], Fyi [n][2m], Fxi [4m][n]
__global__ void dft_init_kernel(bf16* Fx, bf16* Fy, bf16* Fyi, bf16* Fxi, int n, int m) {
  const int64_t total = (int64_t)n * 4 * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(t / (4 * m)), c = (int)(t % (4 * m));
    const int j = c >> 1;
    const int kx = j < m ? j : n - 2 * m + j;
    double s, co;
    sincospi(2.0 * (double)((int64_t)kx * x % n) / n, &s, &co);
    Fx[(int64_t)x * 4 * m + c] = __float2bfloat16_rn((float)((c & 1) ? -s : co));
    Fxi[(int64_t)c * n + x] = __float2bfloat16_rn((float)((c & 1) ? -s : co));
    if (c < 2 * m) {
      const int q = c >> 1;
      double s2, c2;
      sincospi(2.0 * (double)((int64_t)q * x % n) / n, &s2, &c2);
      Fy[(int64_t)c * n + x] = __float2bfloat16_rn((float)((c & 1) ? -s2 : c2));
      Fyi[(int64_t)x * 2 * m + c] = __float2bfloat16_rn((float)((c & 1) ? s2 : c2));
    }
  }
}

// whether n floats at p can be read as float4 (P a multiple of 4 keeps every plane aligned)
__device__ __forceinline__ bool vec4_ok(const void* p, int64_t n) {
  return (n & 3) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// smax[b] = max over the grid of (E, I, 0) as float bits (non-negative floats order as ints)
__global__ void infection_scale_kernel(const float* __restrict__ u, int* __restrict__ smax, int64_t P) {
  const int64_t b = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float* ub = u + (b * 5 + 1) * P;
  float mx = 0.f;
  if (vec4_ok(ub, 2 * P)) {
    for (int64_t t = i0; t < 2 * P / 4; t += stride) {
      const float4 v = reinterpret_cast<const float4*>(ub)[t];
      mx = fmaxf(mx, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
    }
  } else {
    for (int64_t t = i0; t < 2 * P; t += stride) mx = fmaxf(mx, ub[t]);
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) atomicMax(smax + b, __float_as_int(mx));
}

// x[b] = [S, E/s', I/s', R, D, (R0 - 2.6)/1.4, log10(d) + 2, e]   (b = blockIdx.y)
__global__ void make_input_kernel(const float* __restrict__ u, const float* __restrict__ r0,
                                  const float* __restrict__ logd, const int* __restrict__ smax,
                                  float* __restrict__ x, int64_t P) {
  const int64_t b = blockIdx.y;
  const float e = (log10f(fmaxf(__int_as_float(smax[b]), kScaleFloor)) + 4.f) * 0.25f;
  const float sp = scale_from_e(e);
  const float c5 = (r0[b] - 2.6f) / 1.4f, c6 = logd[b] + 2.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool v4 = vec4_ok(x + b * kCin * P, P) && vec4_ok(u + b * 5 * P, P);
  for (int c = 0; c < kCin; ++c) {
    float* xb = x + (b * kCin + c) * P;
    const float* ub = u + (b * 5 + (c < 5 ? c : 0)) * P;
    const float cv = c == 5 ? c5 : (c == 6 ? c6 : e);
    if (v4) {
      for (int64_t i = i0; i < P / 4; i += stride) {
        float4 o;
        if (c >= 5) {
          o = make_float4(cv, cv, cv, cv);
        } else {
          o = reinterpret_cast<const float4*>(ub)[i];
          if (c == 1 || c == 2) o.x = o.x / sp, o.y = o.y / sp, o.z = o.z / sp, o.w = o.w / sp;
        }
        reinterpret_cast<float4*>(xb)[i] = o;
      }
    } else {
      for (int64_t i = i0; i < P; i += stride) xb[i] = c < 5 ? ((c == 1 || c == 2) ? ub[i] / sp : ub[i]) : cv;
    }
  }
}

// per scenario: totals of the raw prediction and of the input state, and the mass clipped
// below zero -> res[3b..3b+2] = {sum y, sum u, sum max(-y, 0)} in double (b = blockIdx.y)
__global__ void residual_kernel(const float* __restrict__ y, const float* __restrict__ u,
                                double* __restrict__ res, int64_t P5) {
  __shared__ double sh[64];
  const int64_t b = blockIdx.y;
  float sy = 0.f, su = 0.f, sn = 0.f;
  // one value per thread and iteration: the residual |sum y - sum u| is a difference of
  // nearly equal totals, so the partial sums stay short
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P5; t += (int64_t)gridDim.x * blockDim.x) {
    const float yv = y[b * P5 + t];
    sy += yv;
    su += u[b * P5 + t];
    sn += yv < 0.f ? -yv : 0.f;
  }
  block_add2(sy, su, res + 3 * b, sh);
  __syncthreads();
  block_add1(sn, res + 3 * b + 2, sh);
}

// per scenario, as float bits: scales[2b] = max(E + I), scales[2b+1] = max(R + D) over the grid
__global__ void support_scales_kernel(const float* __restrict__ u, int* __restrict__ scales, int64_t P) {
  const int64_t b = blockIdx.y;
  float ei = 0.f, rd = 0.f;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
    const float* ub = u + b * 5 * P + t;
    ei = fmaxf(ei, ub[P] + ub[2 * P]);
    rd = fmaxf(rd, ub[3 * P] + ub[4 * P]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    ei = fmaxf(ei, __shfl_down_sync(0xffffffffu, ei, off));
    rd = fmaxf(rd, __shfl_down_sync(0xffffffffu, rd, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(scales + 2 * b, __float_as_int(ei));
    atomicMax(scales + 2 * b + 1, __float_as_int(rd));
  }
}

// ind = 1 where the input holds infected (E + I) or removed (R + D) population above a
// fraction thr of the scenario's maximum, else 0
__global__ void support_kernel(const float* __restrict__ u, const int* __restrict__ scales,
                               unsigned char* __restrict__ ind, int B, int64_t P, float thr) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * P;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / P, p = t - b * P;
    const float* ub = u + b * 5 * P + p;
    const float sei = __int_as_float(scales[2 * b]), srd = __int_as_float(scales[2 * b + 1]);
    ind[t] = (ub[P] + ub[2 * P] > thr * sei && sei > 0.f) || (ub[3 * P] + ub[4 * P] > thr * srd && srd > 0.f);
  }
}

// out = max of in over the periodic window [-r, r] along x (dir 0) or y (dir 1)
__global__ void dilate_kernel(const unsigned char* __restrict__ in, unsigned char* __restrict__ out, int B, int n,
                              int r, int dir) {
  const int64_t P = (int64_t)n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * P;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / P;
    const int p = (int)(t - b * P), y = p / n, x = p - y * n;
    const unsigned char* ib = in + b * P;
    unsigned char v = 0;
    for (int d = -r; d <= r && !v; ++d) {
      const int q = ((dir ? y : x) + d) % n;
      const int qq = q < 0 ? q + n : q;
      v = dir ? ib[(int64_t)qq * n + x] : ib[(int64_t)y * n + qq];
    }
    out[t] = v;
  }
}

// projection: E, I, R, D set to zero outside the mask (when given), every value clamped at
// zero; sums[b] += the projected total (the rescaling's denominator)
__global__ void mask_clamp_kernel(float* __restrict__ y, const unsigned char* __restrict__ mask,
                                  double* __restrict__ sums, int64_t P) {
  __shared__ double sh[64];
  const int64_t b = blockIdx.y;
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool v4 = vec4_ok(y + b * 5 * P, P) && (!mask || (reinterpret_cast<uintptr_t>(mask + b * P) & 3) == 0);
  for (int c = 0; c < 5; ++c) {
    float* yb = y + (b * 5 + c) * P;
    const unsigned char* mb = mask && c > 0 ? mask + b * P : nullptr;
    if (v4) {
      for (int64_t p = i0; p < P / 4; p += stride) {
        float4 v = reinterpret_cast<float4*>(yb)[p];
        if (mb) {
          const uchar4 m = reinterpret_cast<const uchar4*>(mb)[p];
          if (!m.x) v.x = 0.f;
          if (!m.y) v.y = 0.f;
          if (!m.z) v.z = 0.f;
          if (!m.w) v.w = 0.f;
        }
        v.x = v.x > 0.f ? v.x : 0.f, v.y = v.y > 0.f ? v.y : 0.f, v.z = v.z > 0.f ? v.z : 0.f, v.w = v.w > 0.f ? v.w : 0.f;
        reinterpret_cast<float4*>(yb)[p] = v;
        acc += (v.x + v.y) + (v.z + v.w);
      }
    } else {
      for (int64_t p = i0; p < P; p += stride) {
        float v = yb[p];
        if (mb && !mb[p]) v = 0.f;
        v = v > 0.f ? v : 0.f;
        yb[p] = v;
        acc += v;
      }
    }
  }
  block_add1(acc, sums + b, sh);
}

// y *= sum u / sum y (res[3b+1] = sum u)
__global__ void rescale_kernel(float* __restrict__ y, const double* __restrict__ res, const double* __restrict__ sums,
                               int64_t P5) {
  __shared__ float scl;
  const int64_t b = blockIdx.y;
  if (threadIdx.x == 0) scl = sums[b] > 0.0 ? (float)(res[3 * b + 1] / sums[b]) : 1.f;
  __syncthreads();
  const float scale = scl;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float* yb = y + b * P5;
  if (vec4_ok(yb, P5)) {
    for (int64_t t = i0; t < P5 / 4; t += stride) {
      float4 v = reinterpret_cast<float4*>(yb)[t];
      v.x *= scale, v.y *= scale, v.z *= scale, v.w *= scale;
      reinterpret_cast<float4*>(yb)[t] = v;
    }
  } else {
    for (int64_t t = i0; t < P5; t += stride) yb[t] *= scale;
  }
}

// ---- parameter layout ------------------------------------------------------------------

struct Layout {
  int n, W, m, L, H, maxB;
  int64_t P;  // cells per plane
  int64_t nparams;
  int64_t off_A0, off_a0, off_R[16], off_B[16], off_b[16], off_Q1, off_q1, off_Q2, off_q2;
};

int make_param_layout(const sslbm_fno_config* c, Layout* L) {
  if (!c) return err(SSLBM_ERR_BAD_ARG, "config is NULL");
  if (c->n < 8 || c->width < 1 || c->modes < 1 || c->layers < 1 || c->layers > 16 || c->hidden < 1 ||
      c->max_batch < 1 || 2 * c->modes > c->n || c->n > 4096 || c->width > 64 || c->hidden > 64)
    return err(SSLBM_ERR_BAD_ARG, "invalid surrogate configuration (n=%d width=%d modes=%d layers=%d "
               "hidden=%d max_batch=%d; need 2*modes <= n, width and hidden <= 64)", c->n, c->width, c->modes, c->layers,
               c->hidden, c->max_batch);
  L->n = c->n; L->W = c->width; L->m = c->modes; L->L = c->layers; L->H = c->hidden; L->maxB = c->max_batch;
  L->P = (int64_t)c->n * c->n;
  int64_t o = 0;
  const int W = L->W, m = L->m;
  L->off_A0 = o; o += (int64_t)W * kCin;
  L->off_a0 = o; o += W;
  for (int l = 0; l < L->L; ++l) {
    L->off_R[l] = o; o += (int64_t)W * W * 2 * m * m * 2;
    L->off_B[l] = o; o += (int64_t)W * W;
    L->off_b[l] = o; o += W;
  }
  L->off_Q1 = o; o += (int64_t)L->H * W;
  L->off_q1 = o; o += L->H;
  L->off_Q2 = o; o += (int64_t)5 * L->H;
  L->off_q2 = o; o += 5;
  L->nparams = o;
  return SSLBM_OK;
}

struct Buffers {
  size_t total;
  size_t theta, theta16, grad, mom, vel, dft, hcat, zcat, zp, p, f32a, f32b, f32p, h1, tt, hat, dg, dd, smax, csum,
      mask, mscale, loss, res, fault, ratio, ycache;
};

size_t rup(size_t v) { return (v + 255) / 256 * 256; }

void make_buffers(const Layout& L, Buffers* b) {
  const size_t P = (size_t)L.P, B = (size_t)L.maxB, W = (size_t)L.W, m = (size_t)L.m, n = (size_t)L.n;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += rup(bytes); return r; };
  b->theta = take(L.nparams * 4);
  b->theta16 = take(L.nparams * 2);
  b->grad = take(L.nparams * 4);
  b->mom = take(L.nparams * 4);
  b->vel = take(L.nparams * 4);
  b->dft = take((4 * m * n * 2 + 2 * m * n * 2) * 2);
  b->hcat = take((size_t)(L.L + 1) * B * W * P * 2);       // h_0 .. h_L (bf16)
  b->zcat = take((size_t)(L.L > 1 ? L.L - 1 : 1) * B * W * P * 2);  // z_1 .. z_{L-1} (bf16)
  b->zp = take(B * L.H * P * 2);
  b->p = take(B * L.H * P * 2);
  b->f32a = take(B * W * P * 4);
  b->f32b = take(B * W * P * 4);
  b->f32p = take(B * L.H * P * 4);
  b->h1 = take(B * W * n * 4 * m * 4);
  b->tt = take(B * W * 2 * m * 4 * m * 4);
  b->hat = take((size_t)L.L * B * W * 2 * m * m * 2 * 4);
  b->dg = take(B * W * 2 * m * m * 2 * 4);
  b->dd = take(B * 5 * P * 4);
  b->smax = take(B * 4);
  b->csum = take(B * 2 * 8);
  b->mask = take(B * P * 2);
  b->mscale = take(B * 2 * 4);
  b->loss = take(8);
  b->res = take(B * 3 * 8);
  b->fault = take(4);  // set by a tensor-core product whose wait ran out
  b->ratio = take(B * 4);  // per sample: sum u / sum v of the last forward pass
  b->ycache = take(B * 5 * P * 4);  // the last stored forward pass's prediction
  b->total = o;
}

}  // namespace

struct sslbm_fno {
  Layout L;
  Buffers bu;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
  long long gemm_wait_limit = 0;  // tensor-core waits: polls (0 = default) and the stall hook
  int gemm_stall = 0;
  int64_t adam_t = 0;
  float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f, wd = 0.f;
  float mass_weight = 0.f, neg_weight = 0.f;
  int cached_batch = 0;  // batch whose intermediates the backward pass can use (0: none)
  template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
  float* theta() const { return at<float>(bu.theta); }
  bf16* theta16() const { return at<bf16>(bu.theta16); }
  float* grad() const { return at<float>(bu.grad); }
  bf16* Fx() const { return at<bf16>(bu.dft); }
  bf16* Fxi() const { return Fx() + (size_t)L.n * 4 * L.m; }
  bf16* Fy() const { return Fxi() + (size_t)L.n * 4 * L.m; }
  bf16* Fyi() const { return Fy() + (size_t)L.n * 2 * L.m; }
  bf16* h(int l, int B) const { return at<bf16>(bu.hcat) + (size_t)l * B * L.W * L.P; }
  bf16* z(int l, int B) const { return at<bf16>(bu.zcat) + (size_t)(l - 1) * B * L.W * L.P; }
  float* hat(int l, int B) const { return at<float>(bu.hat) + (size_t)(l - 1) * B * L.W * 2 * L.m * L.m * 2; }
};

namespace {

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

GemmArgs gemm0() {
  GemmArgs g{};
  g.K0 = 0;
  g.batch = 1;
  g.splits = 1;
  g.alpha = 1.f;
  g.beta = 0.f;
  return g;
}

int run(const sslbm_fno* f, const GemmArgs& g0, const char* what) {
  GemmArgs g = g0;
  if (g.K0 == 0) g.K0 = g.K;
  g.wait_limit = f->gemm_wait_limit;
  g.stall = f->gemm_stall;
  g.fault = f->at<unsigned int>(f->bu.fault);
  cudaError_t e = sslbm::gemm_bf16(g, f->stream);
  if (e != cudaSuccess) return cuda_err(e, what);
  return SSLBM_OK;
}

// C[b] (rows x P) = Wt (rows x cin) * src[b] (cin x P) (+ beta C): the per-cell channel map
int channel_map(const sslbm_fno* f, const bf16* Wt, int rows, int cin, const void* src, int src_bf16,
                void* C, int c_bf16, float beta, int B, const char* what) {
  CK(sslbm::fno_fused::cell_map(B, rows, cin, f->L.P, Wt, cin, 1, src, src_bf16, C, c_bf16, 1.f, beta, f->stream),
     what);
  return SSLBM_OK;
}

// C[b] (rows x P) = Wt^T (rows x cin, Wt stored cin x rows) * src[b] (cin x P) (+ beta C)
int channel_map_t(const sslbm_fno* f, const bf16* Wt, int rows, int cin, const float* src, float* C,
                  float beta, int B, const char* what) {
  CK(sslbm::fno_fused::cell_map(B, rows, cin, f->L.P, Wt, 1, rows, src, 0, C, 0, 1.f, beta, f->stream), what);
  return SSLBM_OK;
}

// dW (rows x cols) += sum_b sum_p d[b](rows x P) * act[b](cols x P)^T
int weight_grad(const sslbm_fno* f, const float* d, int rows, const void* act, int act_bf16, int cols,
                float* dW, int B, const char* what) {
  CK(sslbm::fno_fused::cell_wgrad(B, rows, cols, f->L.P, d, act, act_bf16, dW, f->stream), what);
  return SSLBM_OK;
}

int channel_sum(const sslbm_fno* f, const float* src, float* out, int B, int C) {
  dim3 grid(std::min<int64_t>(256, (B * f->L.P + kThreads - 1) / kThreads), C);
  channel_sum_kernel<<<grid, kThreads, 0, f->stream>>>(src, out, B, C, f->L.P);
  CK(cudaGetLastError(), "channel_sum");
  return SSLBM_OK;
}

// the spectral convolution of layer l (1-based): out (FP32 [B, W, P]) = K_l(h_{l-1})
int spectral_fwd(sslbm_fno* f, int l, int B, const bf16* hin, float* out) {
  const Layout& L = f->L;
  const int n = L.n, m = L.m, W = L.W, BW = B * W;
  float* H1 = f->at<float>(f->bu.h1);
  float* T = f->at<float>(f->bu.tt);
  const float* R = f->theta() + L.off_R[l - 1];
  int st;
  {  // H1[(b,c,y), 4m] = h[(b,c,y), x] Fx[x, 4m]
    GemmArgs g = gemm0();
    g.M = BW * n; g.N = 4 * m; g.K = n;
    g.A = hin; g.a_bf16 = 1; g.sAm = n; g.sAk0 = 1;
    g.B = f->Fx(); g.b_bf16 = 1; g.sBk0 = 4 * m; g.sBn = 1;
    g.C = H1; g.sCm = 4 * m; g.sCn = 1;
    if ((st = run(f, g, "dft x"))) return st;
  }
  {  // T[(b,c)] (2m x 4m) = Fy (2m x n) H1[(b,c)] (n x 4m)
    GemmArgs g = gemm0();
    g.M = 2 * m; g.N = 4 * m; g.K = n; g.batch = BW;
    g.A = f->Fy(); g.a_bf16 = 1; g.sAb = 0; g.sAm = n; g.sAk0 = 1;
    g.B = H1; g.sBb = (int64_t)n * 4 * m; g.sBk0 = 4 * m; g.sBn = 1;
    g.C = T; g.sCb = 2 * m * 4 * m; g.sCm = 4 * m; g.sCn = 1;
    if ((st = run(f, g, "dft y"))) return st;
  }
  float* hat = f->hat(l, B);
  combine_kernel<<<blocks_for((int64_t)BW * 2 * m * m), kThreads, 0, f->stream>>>(T, hat, BW, m);
  CK(cudaGetLastError(), "combine");
  mix_expand_kernel<<<blocks_for((int64_t)BW * 2 * m * m), kThreads, 0, f->stream>>>(hat, R, T, B, W, m);
  CK(cudaGetLastError(), "mix");
  {  // G1[(b,o)] (n x 4m) = Fyi (n x 2m) U[(b,o)] (2m x 4m)   (G1 reuses H1)
    GemmArgs g = gemm0();
    g.M = n; g.N = 4 * m; g.K = 2 * m; g.batch = BW;
    g.A = f->Fyi(); g.a_bf16 = 1; g.sAb = 0; g.sAm = 2 * m; g.sAk0 = 1;
    g.B = T; g.sBb = 2 * m * 4 * m; g.sBk0 = 4 * m; g.sBn = 1;
    g.C = H1; g.sCb = (int64_t)n * 4 * m; g.sCm = 4 * m; g.sCn = 1;
    if ((st = run(f, g, "idft y"))) return st;
  }
  {  // out[(b,o,y), x] = G1[(b,o,y), 4m] Fxi[4m, x] / n^2
    GemmArgs g = gemm0();
    g.M = BW * n; g.N = n; g.K = 4 * m;
    g.A = H1; g.sAm = 4 * m; g.sAk0 = 1;
    g.B = f->Fxi(); g.b_bf16 = 1; g.sBk0 = n; g.sBn = 1;
    g.C = out; g.sCm = n; g.sCn = 1;
    g.alpha = 1.f / ((float)n * (float)n);
    if ((st = run(f, g, "idft x"))) return st;
  }
  return SSLBM_OK;
}

// adjoint of spectral_fwd: dh (FP32 [B, W, P], overwritten) and dR (accumulated)
int spectral_bwd(sslbm_fno* f, int l, int B, const float* dz, float* dh) {
  const Layout& L = f->L;
  const int n = L.n, m = L.m, W = L.W, BW = B * W;
  float* H1 = f->at<float>(f->bu.h1);
  float* T = f->at<float>(f->bu.tt);
  float* dG = f->at<float>(f->bu.dg);
  const float* R = f->theta() + L.off_R[l - 1];
  float* dR = f->grad() + L.off_R[l - 1];
  int st;
  {  // dG1[(b,o,y), 4m] = dz[(b,o,y), x] Fxi^T[x, 4m] / n^2
    GemmArgs g = gemm0();
    g.M = BW * n; g.N = 4 * m; g.K = n;
    g.A = dz; g.sAm = n; g.sAk0 = 1;
    g.B = f->Fxi(); g.b_bf16 = 1; g.sBk0 = 1; g.sBn = n;
    g.C = H1; g.sCm = 4 * m; g.sCn = 1;
    g.alpha = 1.f / ((float)n * (float)n);
    if ((st = run(f, g, "idft x adjoint"))) return st;
  }
  {  // dU[(b,o)] (2m x 4m) = Fyi^T (2m x n) dG1[(b,o)] (n x 4m)
    GemmArgs g = gemm0();
    g.M = 2 * m; g.N = 4 * m; g.K = n; g.batch = BW;
    g.A = f->Fyi(); g.a_bf16 = 1; g.sAb = 0; g.sAm = 1; g.sAk0 = 2 * m;
    g.B = H1; g.sBb = (int64_t)n * 4 * m; g.sBk0 = 4 * m; g.sBn = 1;
    g.C = T; g.sCb = 2 * m * 4 * m; g.sCm = 4 * m; g.sCn = 1;
    if ((st = run(f, g, "idft y adjoint"))) return st;
  }
  expand_adj_kernel<<<blocks_for((int64_t)BW * 2 * m * m), kThreads, 0, f->stream>>>(T, dG, BW, m);
  CK(cudaGetLastError(), "expand adjoint");
  dR_kernel<<<blocks_for((int64_t)W * W * 2 * m * m), kThreads, 0, f->stream>>>(f->hat(l, B), dG, dR, B, W, m);
  CK(cudaGetLastError(), "dR");
  dhat_combine_adj_kernel<<<blocks_for((int64_t)BW * 2 * m * m), kThreads, 0, f->stream>>>(dG, R, T, B, W, m);
  CK(cudaGetLastError(), "dhat");
  {  // dH1[(b,c)] (n x 4m) = Fy^T (n x 2m) dT[(b,c)] (2m x 4m)
    GemmArgs g = gemm0();
    g.M = n; g.N = 4 * m; g.K = 2 * m; g.batch = BW;
    g.A = f->Fy(); g.a_bf16 = 1; g.sAb = 0; g.sAm = 1; g.sAk0 = n;
    g.B = T; g.sBb = 2 * m * 4 * m; g.sBk0 = 4 * m; g.sBn = 1;
    g.C = H1; g.sCb = (int64_t)n * 4 * m; g.sCm = 4 * m; g.sCn = 1;
    if ((st = run(f, g, "dft y adjoint"))) return st;
  }
  {  // dh[(b,c,y), x] = dH1[(b,c,y), 4m] Fx^T[4m, x]
    GemmArgs g = gemm0();
    g.M = BW * n; g.N = n; g.K = 4 * m;
    g.A = H1; g.sAm = 4 * m; g.sAk0 = 1;
    g.B = f->Fx(); g.b_bf16 = 1; g.sBk0 = 1; g.sBn = 4 * m;
    g.C = dh; g.sCm = n; g.sCn = 1;
    if ((st = run(f, g, "dft x adjoint"))) return st;
  }
  return SSLBM_OK;
}

// the generic forward pass: one strided tensor-core product per contraction (any shape)
int forward_generic(sslbm_fno* f, int B, const float* x, float* y) {
  const Layout& L = f->L;
  const int W = L.W;
  const int64_t P = L.P;
  float* acc = f->at<float>(f->bu.f32a);
  int st;
  lift_kernel<<<blocks_for(B * P), kThreads, 0, f->stream>>>(x, f->theta() + L.off_A0, f->theta() + L.off_a0,
                                                            f->h(0, B), B, W, P);
  CK(cudaGetLastError(), "lift");
  for (int l = 1; l <= L.L; ++l) {
    if ((st = spectral_fwd(f, l, B, f->h(l - 1, B), acc))) return st;
    if ((st = channel_map(f, f->theta16() + L.off_B[l - 1], W, W, f->h(l - 1, B), 1, acc, 0, 1.f, B,
                          "pointwise"))) return st;
    bias_act_kernel<<<blocks_for(B * W * P), kThreads, 0, f->stream>>>(
        acc, f->theta() + L.off_b[l - 1], l < L.L ? f->z(l, B) : nullptr, f->h(l, B), W, P,
        (int64_t)B * W * P, l < L.L ? 1 : 0);
    CK(cudaGetLastError(), "bias/gelu");
  }
  float* accp = f->at<float>(f->bu.f32p);
  if ((st = channel_map(f, f->theta16() + L.off_Q1, L.H, W, f->h(L.L, B), 1, accp, 0, 0.f, B, "projection 1")))
    return st;
  bias_act_kernel<<<blocks_for(B * L.H * P), kThreads, 0, f->stream>>>(
      accp, f->theta() + L.off_q1, f->at<bf16>(f->bu.zp), f->at<bf16>(f->bu.p), L.H, P, (int64_t)B * L.H * P, 1);
  CK(cudaGetLastError(), "projection gelu");
  if ((st = channel_map(f, f->theta16() + L.off_Q2, 5, L.H, f->at<bf16>(f->bu.p), 1, y, 0, 0.f, B,
                        "projection 2"))) return st;
  output_kernel<<<blocks_for(B * 5 * P), kThreads, 0, f->stream>>>(y, f->theta() + L.off_q2, x, B, P);
  CK(cudaGetLastError(), "output");
  return SSLBM_OK;
}

// the fused forward pass (fno_fused.cu): 1 + 4L launches; store = write what backward reads
int forward_fused(sslbm_fno* f, int B, const float* x, float* y, int store) {
  namespace F = sslbm::fno_fused;
  const Layout& L = f->L;
  const int W = L.W, m = L.m, n = L.n, KF = 4 * L.m;
  if (reinterpret_cast<uintptr_t>(x) % 16 || reinterpret_cast<uintptr_t>(y) % 16)
    return err(SSLBM_ERR_BAD_ARG, "x and y must be 16-byte aligned");
  bf16* H1 = f->at<bf16>(f->bu.h1);
  bf16* G1 = H1 + (size_t)B * n * W * KF;
  F::RowArgs a{};
  a.B = B;
  a.n = n;
  a.x = x;
  a.F = f->Fx();
  a.store = store;
  a.A0 = f->theta() + L.off_A0;
  a.a0 = f->theta() + L.off_a0;
  a.hout = f->h(0, B);
  a.H1out = H1;
  CK(F::launch_row(F::ROW_LIFT, W, m, L.H, a, f->stream), "fused lift");
  for (int l = 1; l <= L.L; ++l) {
    float* hat = f->hat(l, B);
    CK(F::launch_dft_y(W, m, B, n, H1, f->Fy(), hat, f->stream), "fused transform along y");
    CK(F::launch_mix_idft_y(W, m, B, n, hat, f->theta() + L.off_R[l - 1], f->Fyi(), G1, f->at<float>(f->bu.dg),
                            1.f / ((float)n * (float)n), f->stream),
       "fused spectral mix");
    F::RowArgs r{};
    r.B = B;
    r.n = n;
    r.x = x;
    r.F = f->Fx();
    r.store = store;
    r.hin = f->h(l - 1, B);
    r.g1 = G1;
    r.Bl = f->theta16() + L.off_B[l - 1];
    r.bl = f->theta() + L.off_b[l - 1];
    r.hout = f->h(l, B);
    if (l < L.L) {
      r.zout = f->z(l, B);
      r.H1out = H1;
      CK(F::launch_row(F::ROW_MID, W, m, L.H, r, f->stream), "fused layer");
    } else {
      r.Q1 = f->theta16() + L.off_Q1;
      r.q1 = f->theta() + L.off_q1;
      r.Q2 = f->theta16() + L.off_Q2;
      r.q2 = f->theta() + L.off_q2;
      r.zp = f->at<bf16>(f->bu.zp);
      r.p = f->at<bf16>(f->bu.p);
      r.y = y;
      CK(F::launch_row(F::ROW_LAST, W, m, L.H, r, f->stream), "fused last layer");
    }
  }
  return SSLBM_OK;
}

// the per-sample conservation step of the output: y = v sum u / sum v; store = keep a copy of
// y for the backward pass
int conserve(sslbm_fno* f, int B, const float* x, float* y, int store) {
  double* sums = f->at<double>(f->bu.csum);
  CK(cudaMemsetAsync(sums, 0, (size_t)B * 2 * 8, f->stream), "zero population sums");
  const int64_t P = f->L.P;
  pred_sums_kernel<<<dim3(rows_grid(P), B), kThreads, 0, f->stream>>>(y, x, sums, P);
  CK(cudaGetLastError(), "population sums");
  conserve_kernel<<<dim3(rows_grid(P), B), kThreads, 0, f->stream>>>(
      y, sums, f->at<float>(f->bu.ratio), store ? f->at<float>(f->bu.ycache) : nullptr, P);
  CK(cudaGetLastError(), "conservation");
  return SSLBM_OK;
}

int forward_impl(sslbm_fno* f, int B, const float* x, float* y, int store) {
  int st;
  if (sslbm::fno_fused::supported(f->L.W, f->L.m, f->L.H, f->L.n))
    st = forward_fused(f, B, x, y, store);
  else
    st = forward_generic(f, B, x, y);  // always stores
  const bool keeps = store || !sslbm::fno_fused::supported(f->L.W, f->L.m, f->L.H, f->L.n);
  if (st == SSLBM_OK) st = conserve(f, B, x, y, keeps ? 1 : 0);
  f->cached_batch = st == SSLBM_OK && keeps ? B : 0;
  return st;
}

int backward_impl(sslbm_fno* f, int B, const float* x, const float* dy_out) {
  const Layout& L = f->L;
  const int W = L.W;
  const int64_t P = L.P;
  float* g = f->grad();
  int st;
  CK(cudaMemsetAsync(g, 0, L.nparams * sizeof(float), f->stream), "zero gradients");
  // seed: the derivative with respect to delta = Q2 p + q2, through the clamp and the rescale
  float* dy = f->at<float>(f->bu.dd);
  double* sums = f->at<double>(f->bu.csum);
  const float* ycache = f->at<float>(f->bu.ycache);
  CK(cudaMemsetAsync(sums, 0, (size_t)B * 2 * 8, f->stream), "zero population sums");
  dim3 sgrid((unsigned)std::min<int64_t>(64, (5 * P + kThreads - 1) / kThreads), B);
  seed_sums_kernel<<<sgrid, kThreads, 0, f->stream>>>(dy_out, ycache, sums, 5 * P);
  CK(cudaGetLastError(), "seed sums");
  scale_dy_kernel<<<dim3(rows_grid(P), B), kThreads, 0, f->stream>>>(dy_out, x, ycache, sums,
                                                                    f->at<float>(f->bu.ratio), dy, P);
  CK(cudaGetLastError(), "output scale");
  if ((st = channel_sum(f, dy, g + L.off_q2, B, 5))) return st;
  if ((st = weight_grad(f, dy, 5, f->at<bf16>(f->bu.p), 1, L.H, g + L.off_Q2, B, "dQ2"))) return st;
  float* dp = f->at<float>(f->bu.f32p);
  if ((st = channel_map_t(f, f->theta16() + L.off_Q2, L.H, 5, dy, dp, 0.f, B, "dp"))) return st;
  gelu_bwd_kernel<<<blocks_for(B * L.H * P), kThreads, 0, f->stream>>>(dp, f->at<bf16>(f->bu.zp), (int64_t)B * L.H * P);
  CK(cudaGetLastError(), "gelu' projection");
  if ((st = channel_sum(f, dp, g + L.off_q1, B, L.H))) return st;
  if ((st = weight_grad(f, dp, L.H, f->h(L.L, B), 1, W, g + L.off_Q1, B, "dQ1"))) return st;
  float* dz = f->at<float>(f->bu.f32a);
  float* dh = f->at<float>(f->bu.f32b);
  if ((st = channel_map_t(f, f->theta16() + L.off_Q1, W, L.H, dp, dz, 0.f, B, "dh_L"))) return st;
  for (int l = L.L; l >= 1; --l) {
    if ((st = channel_sum(f, dz, g + L.off_b[l - 1], B, W))) return st;
    if ((st = weight_grad(f, dz, W, f->h(l - 1, B), 1, W, g + L.off_B[l - 1], B, "dB"))) return st;
    if ((st = spectral_bwd(f, l, B, dz, dh))) return st;
    if ((st = channel_map_t(f, f->theta16() + L.off_B[l - 1], W, W, dz, dh, 1.f, B, "dh pointwise"))) return st;
    if (l > 1) {
      gelu_bwd_kernel<<<blocks_for(B * W * P), kThreads, 0, f->stream>>>(dh, f->z(l - 1, B), (int64_t)B * W * P);
      CK(cudaGetLastError(), "gelu'");
    }
    float* t = dz;
    dz = dh;
    dh = t;
  }
  // lift: dA0 = sum dh0 x^T, da0 = sum dh0
  if ((st = channel_sum(f, dz, g + L.off_a0, B, W))) return st;
  if ((st = weight_grad(f, dz, W, x, 0, kCin, g + L.off_A0, B, "dA0"))) return st;
  return SSLBM_OK;
}

int check_batch(const sslbm_fno* f, int B) {
  if (!f) return err(SSLBM_ERR_BAD_ARG, "surrogate is NULL");
  if (B < 1 || B > f->L.maxB) return err(SSLBM_ERR_BAD_ARG, "batch %d not in [1, %d]", B, f->L.maxB);
  return SSLBM_OK;
}

}  // namespace

extern "C" {

int sslbm_fno_workspace_bytes(const sslbm_fno_config* c, size_t* bytes) {
  if (!bytes) return err(SSLBM_ERR_BAD_ARG, "bytes is NULL");
  Layout L;
  int st = make_param_layout(c, &L);
  if (st) return st;
  Buffers b;
  make_buffers(L, &b);
  *bytes = b.total;
  return SSLBM_OK;
}

int sslbm_fno_create(const sslbm_fno_config* c, void* dev_ws, size_t ws_bytes, void* stream,
                     sslbm_fno** out) {
  if (!out) return err(SSLBM_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  Layout L;
  int st = make_param_layout(c, &L);
  if (st) return st;
  Buffers bu;
  make_buffers(L, &bu);
  if (!dev_ws || reinterpret_cast<uintptr_t>(dev_ws) % 256)
    return err(SSLBM_ERR_WORKSPACE, "workspace missing or not 256-byte aligned");
  if (ws_bytes < bu.total) return err(SSLBM_ERR_WORKSPACE, "workspace of %zu bytes < %zu", ws_bytes, bu.total);
  cudaPointerAttributes attr;
  CK(cudaPointerGetAttributes(&attr, dev_ws), "cudaPointerGetAttributes");
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return err(SSLBM_ERR_WORKSPACE, "workspace is not device memory");
  sslbm_fno* f = new (std::nothrow) sslbm_fno();
  if (!f) return err(SSLBM_ERR_BAD_ARG, "out of host memory");
  f->L = L;
  f->bu = bu;
  f->ws = static_cast<char*>(dev_ws);
  f->stream = static_cast<cudaStream_t>(stream);
  f->device = attr.device;
  DevGuard dg(f->device);
  cudaError_t e = cudaMemsetAsync(f->ws, 0, bu.total, f->stream);
  if (e == cudaSuccess) {
    dft_init_kernel<<<blocks_for((int64_t)L.n * 4 * L.m), kThreads, 0, f->stream>>>(f->Fx(), f->Fy(), f->Fyi(),
                                                                                   f->Fxi(), L.n, L.m);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    delete f;
    return cuda_err(e, "surrogate init");
  }
  *out = f;
  return SSLBM_OK;
}

void sslbm_fno_destroy(sslbm_fno* f) { delete f; }

int64_t sslbm_fno_num_params(const sslbm_fno* f) { return f ? f->L.nparams : -1; }

int sslbm_fno_set_params(sslbm_fno* f, const float* theta, int on_device) {
  if (!f || !theta) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  DevGuard dg(f->device);
  CK(cudaMemcpyAsync(f->theta(), theta, f->L.nparams * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     f->stream), "set params");
  to_bf16_kernel<<<blocks_for(f->L.nparams), kThreads, 0, f->stream>>>(f->theta(), f->theta16(), f->L.nparams);
  CK(cudaGetLastError(), "params to bf16");
  CK(cudaMemsetAsync(f->at<float>(f->bu.mom), 0, f->L.nparams * 4, f->stream), "reset moments");
  CK(cudaMemsetAsync(f->at<float>(f->bu.vel), 0, f->L.nparams * 4, f->stream), "reset moments");
  f->adam_t = 0;
  if (!on_device) CK(cudaStreamSynchronize(f->stream), "sync");
  return SSLBM_OK;
}

int sslbm_fno_get_params(sslbm_fno* f, float* theta, int on_device) {
  if (!f || !theta) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  DevGuard dg(f->device);
  CK(cudaMemcpyAsync(theta, f->theta(), f->L.nparams * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     f->stream), "get params");
  if (!on_device) CK(cudaStreamSynchronize(f->stream), "sync");
  return SSLBM_OK;
}

int sslbm_fno_get_grads(sslbm_fno* f, float* grad, int on_device) {
  if (!f || !grad) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  DevGuard dg(f->device);
  CK(cudaMemcpyAsync(grad, f->grad(), f->L.nparams * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     f->stream), "get grads");
  if (!on_device) CK(cudaStreamSynchronize(f->stream), "sync");
  return SSLBM_OK;
}

int sslbm_fno_make_input(sslbm_fno* f, int batch, const float* u, const float* r0, const float* logd, float* x) {
  int st = check_batch(f, batch);
  if (st) return st;
  if (!u || !r0 || !logd || !x) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  DevGuard dg(f->device);
  int* smax = f->at<int>(f->bu.smax);
  CK(cudaMemsetAsync(smax, 0, (size_t)batch * 4, f->stream), "zero scale");
  dim3 grid((unsigned)std::min<int64_t>(64, (2 * f->L.P + kThreads - 1) / kThreads), batch);
  infection_scale_kernel<<<grid, kThreads, 0, f->stream>>>(u, smax, f->L.P);
  CK(cudaGetLastError(), "infection scale");
  make_input_kernel<<<dim3(rows_grid(f->L.P), batch), kThreads, 0, f->stream>>>(u, r0, logd, smax, x, f->L.P);
  CK(cudaGetLastError(), "make input");
  return SSLBM_OK;
}

int sslbm_fno_forward(sslbm_fno* f, int batch, const float* x, float* y) {
  int st = check_batch(f, batch);
  if (st) return st;
  if (!x || !y) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  DevGuard dg(f->device);
  return forward_impl(f, batch, x, y, 1);
}

int sslbm_fno_infer(sslbm_fno* f, int batch, const float* x, float* y) {
  int st = check_batch(f, batch);
  if (st) return st;
  if (!x || !y) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  DevGuard dg(f->device);
  return forward_impl(f, batch, x, y, 0);
}

int sslbm_fno_fused(const sslbm_fno* f) {
  if (!f) return err(SSLBM_ERR_BAD_ARG, "surrogate is NULL");
  return sslbm::fno_fused::supported(f->L.W, f->L.m, f->L.H, f->L.n) ? 1 : 0;
}

int sslbm_fno_backward(sslbm_fno* f, int batch, const float* x, const float* dy) {
  int st = check_batch(f, batch);
  if (st) return st;
  if (!x || !dy) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  if (f->cached_batch != batch)
    return err(SSLBM_ERR_STATE, "backward needs a preceding sslbm_fno_forward on the same batch");
  DevGuard dg(f->device);
  return backward_impl(f, batch, x, dy);
}

int sslbm_fno_set_adam(sslbm_fno* f, float beta1, float beta2, float eps, float weight_decay) {
  if (!f) return err(SSLBM_ERR_BAD_ARG, "surrogate is NULL");
  f->b1 = beta1; f->b2 = beta2; f->eps = eps; f->wd = weight_decay;
  return SSLBM_OK;
}

int sslbm_fno_set_wait_limit(sslbm_fno* f, long long polls, int stall) {
  if (!f) return err(SSLBM_ERR_BAD_ARG, "handle is NULL");
  if (polls < 0) return err(SSLBM_ERR_BAD_ARG, "polls %lld < 0", polls);
  f->gemm_wait_limit = polls;
  f->gemm_stall = stall != 0;
  return SSLBM_OK;
}

int sslbm_fno_set_loss_weights(sslbm_fno* f, float mass_weight, float neg_weight) {
  if (!f) return err(SSLBM_ERR_BAD_ARG, "surrogate is NULL");
  if (!(mass_weight >= 0.f) || !std::isfinite(mass_weight) || !(neg_weight >= 0.f) || !std::isfinite(neg_weight))
    return err(SSLBM_ERR_BAD_ARG, "loss weights must be finite and >= 0");
  f->mass_weight = mass_weight;
  f->neg_weight = neg_weight;
  return SSLBM_OK;
}

int sslbm_fno_train_step(sslbm_fno* f, int batch, const float* x, const float* target, float* y_scratch,
                         float* dy_scratch, float lr, double* loss) {
  int st = check_batch(f, batch);
  if (st) return st;
  if (!x || !target || !y_scratch || !dy_scratch) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  DevGuard dg(f->device);
  if ((st = forward_impl(f, batch, x, y_scratch, 1))) return st;
  double* dl = f->at<double>(f->bu.loss);
  CK(cudaMemsetAsync(dl, 0, 8, f->stream), "zero loss");
  const int64_t P5 = 5 * f->L.P, N = (int64_t)batch * P5;
  double* sums = nullptr;
  if (f->mass_weight != 0.f || f->neg_weight != 0.f) {
    sums = f->at<double>(f->bu.res);
    CK(cudaMemsetAsync(sums, 0, (size_t)batch * 3 * 8, f->stream), "zero loss sums");
    dim3 grid((unsigned)std::min<int64_t>(64, (P5 + kThreads - 1) / kThreads), batch);
    loss_sums_kernel<<<grid, kThreads, 0, f->stream>>>(y_scratch, target, sums, P5);
    CK(cudaGetLastError(), "loss sums");
  }
  loss_kernel<<<blocks_for(N), kThreads, 0, f->stream>>>(y_scratch, target, x, dy_scratch, dl, N, f->L.P, sums,
                                                         f->mass_weight, f->neg_weight, batch);
  CK(cudaGetLastError(), "loss");
  if ((st = backward_impl(f, batch, x, dy_scratch))) return st;
  const int64_t t_next = f->adam_t + 1;
  const float c1 = 1.f - powf(f->b1, (float)t_next), c2 = 1.f - powf(f->b2, (float)t_next);
  unsigned int* fault_word = f->at<unsigned int>(f->bu.fault);
  adam_kernel<<<blocks_for(f->L.nparams), kThreads, 0, f->stream>>>(
      f->theta(), f->grad(), f->at<float>(f->bu.mom), f->at<float>(f->bu.vel), f->theta16(), f->L.nparams, lr,
      f->b1, f->b2, f->eps, f->wd, c1, c2, fault_word);
  CK(cudaGetLastError(), "adam");
  // every call reports its own products' status: read the fault word, and clear it if set
  unsigned int fault = 0;
  CK(cudaMemcpyAsync(&fault, fault_word, sizeof(fault), cudaMemcpyDeviceToHost, f->stream), "product status");
  if (loss) CK(cudaMemcpyAsync(loss, dl, 8, cudaMemcpyDeviceToHost, f->stream), "loss");
  CK(cudaStreamSynchronize(f->stream), "sync");
  if (fault) {
    CK(cudaMemsetAsync(fault_word, 0, sizeof(unsigned int), f->stream), "clear product status");
    return err(SSLBM_ERR_TIMEOUT,
               "a tensor-core product timed out waiting for its MMAs (results are NaN; the update was skipped)");
  }
  f->adam_t = t_next;
  return SSLBM_OK;
}

int sslbm_fno_check_project(sslbm_fno* f, int batch, float* y, const float* u, int reach, double* residuals) {
  int st = check_batch(f, batch);
  if (st) return st;
  if (!y || !u || !residuals) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  if (reach < 0) return err(SSLBM_ERR_BAD_ARG, "reach %d < 0", reach);
  DevGuard dg(f->device);
  double* res = f->at<double>(f->bu.res);
  double* sums = f->at<double>(f->bu.csum);
  CK(cudaMemsetAsync(res, 0, (size_t)batch * 3 * 8, f->stream), "zero residuals");
  CK(cudaMemsetAsync(sums, 0, (size_t)batch * 8, f->stream), "zero sums");
  const int64_t P = f->L.P, P5 = 5 * P;
  dim3 grid((unsigned)std::min<int64_t>(64, (P5 + kThreads - 1) / kThreads), batch);
  residual_kernel<<<grid, kThreads, 0, f->stream>>>(y, u, res, P5);
  CK(cudaGetLastError(), "residual");
  unsigned char* mask = nullptr;
  if (reach > 0) {
    const int r = std::min(reach, f->L.n / 2);
    unsigned char* ind = f->at<unsigned char>(f->bu.mask);
    mask = ind + (size_t)batch * P;
    int* scales = f->at<int>(f->bu.mscale);
    CK(cudaMemsetAsync(scales, 0, (size_t)batch * 2 * 4, f->stream), "zero scales");
    dim3 g1((unsigned)std::min<int64_t>(64, (P + kThreads - 1) / kThreads), batch);
    support_scales_kernel<<<g1, kThreads, 0, f->stream>>>(u, scales, P);
    support_kernel<<<blocks_for((int64_t)batch * P), kThreads, 0, f->stream>>>(u, scales, ind, batch, P, 1e-6f);
    dilate_kernel<<<blocks_for((int64_t)batch * P), kThreads, 0, f->stream>>>(ind, mask, batch, f->L.n, r, 0);
    dilate_kernel<<<blocks_for((int64_t)batch * P), kThreads, 0, f->stream>>>(mask, ind, batch, f->L.n, r, 1);
    mask = ind;
    CK(cudaGetLastError(), "support mask");
  }
  mask_clamp_kernel<<<grid, kThreads, 0, f->stream>>>(y, mask, sums, P);
  CK(cudaGetLastError(), "clamp");
  rescale_kernel<<<grid, kThreads, 0, f->stream>>>(y, res, sums, P5);
  CK(cudaGetLastError(), "rescale");
  std::vector<double> r((size_t)batch * 3);
  CK(cudaMemcpyAsync(r.data(), res, r.size() * 8, cudaMemcpyDeviceToHost, f->stream), "residual copy");
  CK(cudaStreamSynchronize(f->stream), "sync");
  for (int b = 0; b < batch; ++b) {
    const double su = r[3 * b + 1];
    residuals[2 * b] = su != 0 ? std::fabs(r[3 * b] - su) / std::fabs(su) : std::fabs(r[3 * b]);
    residuals[2 * b + 1] = su != 0 ? r[3 * b + 2] / std::fabs(su) : r[3 * b + 2];
    // a prediction with a NaN or Inf anywhere fails both checks, whatever the clamp made of it
    if (!std::isfinite(r[3 * b]) || !std::isfinite(r[3 * b + 2])) {
      residuals[2 * b] = HUGE_VAL;
      residuals[2 * b + 1] = HUGE_VAL;
    }
  }
  return SSLBM_OK;
}

}  // extern "C"

namespace sslbm {

int fno_shape(const sslbm_fno* f, int* n, int* max_batch, int* device, cudaStream_t* stream) {
  if (!f) return SSLBM_ERR_BAD_ARG;
  if (n) *n = f->L.n;
  if (max_batch) *max_batch = f->L.maxB;
  if (device) *device = f->device;
  if (stream) *stream = f->stream;
  return SSLBM_OK;
}

}  // namespace sslbm
