// fd4.cu -- the fourth-order finite-difference reference of Sec. III on the GPU (and, for the
// cost comparison of Sec. IV, its second-order counterpart, sslbm_fd4_set_order): classical
// RK4 in time and the fourth-order centred Laplacian in space,
//   L4 u = sum over axes of (-u[-2] + 16 u[-1] - 30 u[0] + 16 u[+1] - u[+2]) / (12 dx^2),
//   d/dt C = Psi^C + d^C L4 C (C = S, E, I, R),  d/dt D = phi gamma I   (Eqs. EqSEIRD_S..D),
// with the reactions of Eq. (sources) evaluated at every stage.  Ghost cells: periodic wrap,
// or (no-flux) the even reflection about the boundary face, u[-1] = u[0], u[-2] = u[1].
//
// One step is four stage launches.  Stage s reads the previous stage's state with the
// stencil and writes the next stage's state and the running sum of the slopes:
//   s = 1: acc = k1,         t = u + (dt/2) k1
//   s = 2: acc = acc + 2 k2, t = u + (dt/2) k2
//   s = 3: acc = acc + 2 k3, t = u + dt k3
//   s = 4: u = u + (dt/6) (acc + k4)
// Every operation is rounded on its own (no contraction) in the order of the formulas
// above, so the FP64 path reproduces a plain evaluation of them operation by operation.
// Each stage has two kernels: one cell per thread on 32 x 8 tiles (any width, any
// precision), and for FP32 grids of width a multiple of 4 with at least 1.5 waves of tiles,
// four cells per thread on 128 x 8 tiles; both evaluate the same expressions.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>

#include "sslbm.h"

namespace sslbm {
int record_error(int status, const char* msg);
}

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

#define CK(call, what)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_err(e_, what);   \
  } while (0)

__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float dvd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double dvd(double a, double b) { return __ddiv_rn(a, b); }

template <typename T>
struct Fd4Coeffs {
  T beta, alpha, gamma, rg, dg;  // rg = (1 - phi) gamma, dg = phi gamma
  T d[4];                        // diffusivities of S, E, I, R
  T inv, inv2;                   // 1 / (12 dx^2), 1 / dx^2
  T half_dt, dt, dt6;            // dt/2, dt, dt/6
};

// index of a (possibly ghost) cell along an axis of n cells
__device__ __forceinline__ int64_t ghost2(int64_t i, int64_t n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == SSLBM_BC_PERIODIC) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
  }
  if (i < 0) i = -1 - i;
  if (i >= n) i = 2 * n - 1 - i;
  if (i < 0) i = 0;  // grids narrower than the stencil
  if (i >= n) i = n - 1;
  return i;
}

constexpr int kTX = 32, kTY = 8, kH = 2;  // tile of cells per CTA and the stencil's halo

// One RK4 stage on a kTX x kTY tile of cells: the four mobile planes of the stage input are
// staged in shared memory with a halo of two cells (ghost cells resolved once, at load),
// then every cell evaluates its right-hand side from the tile.
template <typename T, int STAGE, int ORDER>
__global__ void __launch_bounds__(kTX * kTY) fd4_stage_kernel(int64_t nx, int64_t ny, int bc, const Fd4Coeffs<T> k,
                                                              const T* __restrict__ src, const T* u, T* acc,
                                                              T* dst) {
  constexpr int SX = kTX + 2 * kH, SY = kTY + 2 * kH;
  __shared__ T tile[4][SY][SX];
  const int64_t M = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
  const int64_t bx0 = (int64_t)blockIdx.x * kTX;
  for (int64_t by0 = (int64_t)blockIdx.y * kTY; by0 < ny; by0 += (int64_t)gridDim.y * kTY) {
    __syncthreads();  // the previous tile's readers are done
    for (int i = tid; i < SX * SY; i += kTX * kTY) {
      const int sy = i / SX, sx = i - sy * SX;
      const int64_t gx = ghost2(bx0 + sx - kH, nx, bc), gy = ghost2(by0 + sy - kH, ny, bc);
      const int64_t off = gy * nx + gx;
#pragma unroll
      for (int c = 0; c < 4; ++c) tile[c][sy][sx] = src[c * M + off];
    }
    __syncthreads();
    const int64_t x = bx0 + tx, y = by0 + ty;
    if (x >= nx || y >= ny) continue;
    const int64_t c0 = y * nx + x;
    const int cx = tx + kH, cy = ty + kH;
    const T S = tile[0][cy][cx], E = tile[1][cy][cx], I = tile[2][cy][cx], R = tile[3][cy][cx];
    // reactions, Eq. (sources)
    const T Nc = add(add(add(S, E), I), R);
    const T F = Nc != T(0) ? dvd(mul(mul(k.beta, S), I), Nc) : T(0);
    const T aE = mul(k.alpha, E);
    T rhs[5];
    rhs[0] = -F;
    rhs[1] = sub(F, aE);
    rhs[2] = sub(aE, mul(k.gamma, I));
    rhs[3] = mul(k.rg, I);
    rhs[4] = mul(k.dg, I);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T u0 = tile[c][cy][cx];
      T lx, ly;
      if (ORDER == 4) {
        lx = sub(add(sub(add(-tile[c][cy][cx - 2], mul(T(16), tile[c][cy][cx - 1])), mul(T(30), u0)),
                     mul(T(16), tile[c][cy][cx + 1])),
                 tile[c][cy][cx + 2]);
        ly = sub(add(sub(add(-tile[c][cy - 2][cx], mul(T(16), tile[c][cy - 1][cx])), mul(T(30), u0)),
                     mul(T(16), tile[c][cy + 1][cx])),
                 tile[c][cy + 2][cx]);
      } else {  // second order: u[-1] - 2 u[0] + u[+1]
        lx = add(sub(tile[c][cy][cx - 1], mul(T(2), u0)), tile[c][cy][cx + 1]);
        ly = add(sub(tile[c][cy - 1][cx], mul(T(2), u0)), tile[c][cy + 1][cx]);
      }
      rhs[c] = add(rhs[c], mul(mul(k.d[c], add(lx, ly)), ORDER == 4 ? k.inv : k.inv2));
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int64_t i = c * M + c0;
      const T r = rhs[c];
      if (STAGE == 1) {
        acc[i] = r;
        dst[i] = add(u[i], mul(k.half_dt, r));
      } else if (STAGE == 2) {
        acc[i] = add(acc[i], mul(T(2), r));
        dst[i] = add(u[i], mul(k.half_dt, r));
      } else if (STAGE == 3) {
        acc[i] = add(acc[i], mul(T(2), r));
        dst[i] = add(u[i], mul(k.dt, r));
      } else {
        dst[i] = add(u[i], mul(k.dt6, add(acc[i], r)));
      }
    }
  }
}

// The FP32 stage for grids whose width is a multiple of 4: a 128 x 8 tile, each thread
// four consecutive cells of one row.  Rows are staged with 16-byte loads (row starts and
// planes are then 16-byte aligned), the two halo columns on each side separately through
// ghost2, and u, acc, dst move as float4.  Only the slopes of the four cells stay live
// across planes (64 registers, four CTAs per SM).  Per cell the expressions and their
// order are those of fd4_stage_kernel, so both give the same bits.
constexpr int kVX = 128, kVY = 8, kVPad = 4;  // tile columns and rows; shared rows start 4 columns left
constexpr int kVS = kVX + 2 * kVPad;            // floats per shared row

template <int STAGE, int ORDER>
__global__ void __launch_bounds__(32 * kVY, 4) fd4_stage_f32v_kernel(int64_t nx, int64_t ny, int bc,
                                                                  const Fd4Coeffs<float> k,
                                                                  const float* __restrict__ src, const float* u,
                                                                  float* acc, float* dst) {
  constexpr int RY = kVY + 2 * kH;  // staged rows
  static_assert(4 * 4 * RY <= 32 * kVY, "one thread per halo cell of the staged rows");
  __shared__ __align__(16) float tile[4][RY][kVS];
  const int64_t M = nx * ny;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int64_t bx0 = (int64_t)blockIdx.x * kVX;
  const int64_t x = bx0 + 4 * lane;
  for (int64_t by0 = (int64_t)blockIdx.y * kVY; by0 < ny; by0 += (int64_t)gridDim.y * kVY) {
    __syncthreads();  // the previous tile's readers are done
    for (int j = wy; j < 4 * RY; j += kVY) {  // staged row j % RY of plane j / RY, one warp per row
      const int r = j % RY, c = j / RY;
      const float* row = src + c * M + ghost2(by0 + r - kH, ny, bc) * nx;
      float4 v;
      if (x + 3 < nx) {
        v = *reinterpret_cast<const float4*>(row + x);
      } else {  // past the last column: ghost images
        v.x = row[ghost2(x, nx, bc)];
        v.y = row[ghost2(x + 1, nx, bc)];
        v.z = row[ghost2(x + 2, nx, bc)];
        v.w = row[ghost2(x + 3, nx, bc)];
      }
      *reinterpret_cast<float4*>(&tile[c][r][kVPad + 4 * lane]) = v;
    }
    if (threadIdx.x < 4 * 4 * RY) {  // halo columns -2, -1, kVX, kVX+1 of every staged row
      const int h = threadIdx.x & 3, rc = threadIdx.x >> 2;
      const int r = rc % RY, c = rc / RY;
      const int col = h < 2 ? h - kH : kVX + h - 2;
      tile[c][r][kVPad + col] = src[c * M + ghost2(by0 + r - kH, ny, bc) * nx + ghost2(bx0 + col, nx, bc)];
    }
    __syncthreads();
    const int64_t y = by0 + wy;
    if (x >= nx || y >= ny) continue;
    const int cy = wy + kH;
    float rhs[5][4];
    {  // reactions at this thread's four cells, Eq. (sources)
      const float4 S4 = *reinterpret_cast<const float4*>(&tile[0][cy][kVPad + 4 * lane]);
      const float4 E4 = *reinterpret_cast<const float4*>(&tile[1][cy][kVPad + 4 * lane]);
      const float4 I4 = *reinterpret_cast<const float4*>(&tile[2][cy][kVPad + 4 * lane]);
      const float4 R4 = *reinterpret_cast<const float4*>(&tile[3][cy][kVPad + 4 * lane]);
      const float Sv[4] = {S4.x, S4.y, S4.z, S4.w}, Ev[4] = {E4.x, E4.y, E4.z, E4.w};
      const float Iv[4] = {I4.x, I4.y, I4.z, I4.w}, Rv[4] = {R4.x, R4.y, R4.z, R4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float S = Sv[e], E = Ev[e], I = Iv[e], R = Rv[e];
        const float Nc = add(add(add(S, E), I), R);
        const float F = Nc != 0.f ? dvd(mul(mul(k.beta, S), I), Nc) : 0.f;
        const float aE = mul(k.alpha, E);
        rhs[0][e] = -F;
        rhs[1][e] = sub(F, aE);
        rhs[2][e] = sub(aE, mul(k.gamma, I));
        rhs[3][e] = mul(k.rg, I);
        rhs[4][e] = mul(k.dg, I);
      }
    }
    // the Laplacian, one plane at a time: h[2 + e] is cell e of this thread in the centre row,
    // h[0..1] and h[6..7] the two cells on each side; col[dy + 2][e] the rows above and below
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float* row = &tile[c][cy][0];
      const float2 hl = *reinterpret_cast<const float2*>(row + 4 * lane + 2);
      const float4 hc = *reinterpret_cast<const float4*>(row + kVPad + 4 * lane);
      const float2 hr = *reinterpret_cast<const float2*>(row + 2 * kVPad + 4 * lane);
      const float h[8] = {hl.x, hl.y, hc.x, hc.y, hc.z, hc.w, hr.x, hr.y};
      float col[2 * kH + 1][4];
#pragma unroll
      for (int dy = -kH; dy <= kH; ++dy) {
        if (dy != 0 && (ORDER == 4 || dy == -1 || dy == 1)) {
          const float4 t = *reinterpret_cast<const float4*>(&tile[c][cy + dy][kVPad + 4 * lane]);
          col[dy + kH][0] = t.x, col[dy + kH][1] = t.y, col[dy + kH][2] = t.z, col[dy + kH][3] = t.w;
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float u0 = h[2 + e];
        float lx, ly;
        if (ORDER == 4) {
          lx = sub(add(sub(add(-h[e], mul(16.f, h[1 + e])), mul(30.f, u0)), mul(16.f, h[3 + e])), h[4 + e]);
          ly = sub(add(sub(add(-col[0][e], mul(16.f, col[1][e])), mul(30.f, u0)), mul(16.f, col[3][e])),
                   col[4][e]);
        } else {
          lx = add(sub(h[1 + e], mul(2.f, u0)), h[3 + e]);
          ly = add(sub(col[1][e], mul(2.f, u0)), col[3][e]);
        }
        rhs[c][e] = add(rhs[c][e], mul(mul(k.d[c], add(lx, ly)), ORDER == 4 ? k.inv : k.inv2));
      }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int64_t i = c * M + y * nx + x;
      const float4 uu = *reinterpret_cast<const float4*>(u + i);
      const float uv[4] = {uu.x, uu.y, uu.z, uu.w};
      float o[4], a[4];
      if (STAGE == 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          a[e] = rhs[c][e];
          o[e] = add(uv[e], mul(k.half_dt, rhs[c][e]));
        }
      } else {
        const float4 aa = *reinterpret_cast<const float4*>(acc + i);
        const float av[4] = {aa.x, aa.y, aa.z, aa.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (STAGE == 4) {
            o[e] = add(uv[e], mul(k.dt6, add(av[e], rhs[c][e])));
          } else {
            a[e] = add(av[e], mul(2.f, rhs[c][e]));
            o[e] = add(uv[e], mul(STAGE == 2 ? k.half_dt : k.dt, rhs[c][e]));
          }
        }
      }
      if (STAGE != 4) *reinterpret_cast<float4*>(acc + i) = make_float4(a[0], a[1], a[2], a[3]);
      *reinterpret_cast<float4*>(dst + i) = make_float4(o[0], o[1], o[2], o[3]);
    }
  }
}

template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ a, B* __restrict__ b, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = (B)a[t];
}

size_t rup(size_t v) { return (v + 255) / 256 * 256; }

int check_grid(const sslbm_grid* g) {
  if (!g) return err(SSLBM_ERR_BAD_ARG, "grid is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nx > (1 << 20) || g->ny > (1 << 20))
    return err(SSLBM_ERR_BAD_ARG, "grid %lld x %lld out of range", (long long)g->nx, (long long)g->ny);
  if (!(g->dx > 0) || !(g->dt > 0) || !std::isfinite(g->dx) || !std::isfinite(g->dt))
    return err(SSLBM_ERR_BAD_ARG, "dx and dt must be finite and > 0");
  if (g->bc != SSLBM_BC_PERIODIC && g->bc != SSLBM_BC_NOFLUX) return err(SSLBM_ERR_BAD_ARG, "bc %d", g->bc);
  if (g->precision != SSLBM_FP64 && g->precision != SSLBM_FP32)
    return err(SSLBM_ERR_UNSUPPORTED, "the FD4 reference runs in FP64 or FP32");
  return SSLBM_OK;
}

size_t state_bytes(const sslbm_grid* g) {
  return rup((size_t)5 * g->nx * g->ny * (g->precision == SSLBM_FP64 ? 8 : 4));
}

unsigned blocks1(int64_t n) { return (unsigned)std::min<int64_t>(65536, (n + 255) / 256); }

}  // namespace

struct sslbm_fd4 {
  sslbm_grid g;
  cudaStream_t stream = nullptr;
  int device = 0;
  char* ws = nullptr;
  size_t sb = 0;  // bytes of one 5-plane state
  Fd4Coeffs<double> k64;
  Fd4Coeffs<float> k32;
  int64_t steps = 0;
  int order = 4;  // order of the Laplacian: 4 (the reference) or 2
  int sms = 1;    // multiprocessors of the device
  void* buf(int i) const { return ws + (size_t)i * sb; }  // 0 u, 1 t1, 2 t2, 3 acc
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

template <int ORDER>
cudaError_t run_step_f32v(const sslbm_fd4* f, const Fd4Coeffs<float>& k) {
  const int64_t nx = f->g.nx, ny = f->g.ny;
  dim3 grid((unsigned)((nx + kVX - 1) / kVX), (unsigned)std::min<int64_t>(65535, (ny + kVY - 1) / kVY));
  float* u = static_cast<float*>(f->buf(0));
  float* t1 = static_cast<float*>(f->buf(1));
  float* t2 = static_cast<float*>(f->buf(2));
  float* acc = static_cast<float*>(f->buf(3));
  const int bc = f->g.bc;
  fd4_stage_f32v_kernel<1, ORDER><<<grid, 32 * kVY, 0, f->stream>>>(nx, ny, bc, k, u, u, acc, t1);
  fd4_stage_f32v_kernel<2, ORDER><<<grid, 32 * kVY, 0, f->stream>>>(nx, ny, bc, k, t1, u, acc, t2);
  fd4_stage_f32v_kernel<3, ORDER><<<grid, 32 * kVY, 0, f->stream>>>(nx, ny, bc, k, t2, u, acc, t1);
  fd4_stage_f32v_kernel<4, ORDER><<<grid, 32 * kVY, 0, f->stream>>>(nx, ny, bc, k, t1, u, acc, u);
  return cudaGetLastError();
}

template <typename T, int ORDER>
cudaError_t run_step(const sslbm_fd4* f, const Fd4Coeffs<T>& k) {
  const int64_t nx = f->g.nx, ny = f->g.ny;
  dim3 block(kTX, kTY);
  dim3 grid((unsigned)((nx + kTX - 1) / kTX), (unsigned)std::min<int64_t>(65535, (ny + kTY - 1) / kTY));
  T* u = static_cast<T*>(f->buf(0));
  T* t1 = static_cast<T*>(f->buf(1));
  T* t2 = static_cast<T*>(f->buf(2));
  T* acc = static_cast<T*>(f->buf(3));
  const int bc = f->g.bc;
  fd4_stage_kernel<T, 1, ORDER><<<grid, block, 0, f->stream>>>(nx, ny, bc, k, u, u, acc, t1);
  fd4_stage_kernel<T, 2, ORDER><<<grid, block, 0, f->stream>>>(nx, ny, bc, k, t1, u, acc, t2);
  fd4_stage_kernel<T, 3, ORDER><<<grid, block, 0, f->stream>>>(nx, ny, bc, k, t2, u, acc, t1);
  fd4_stage_kernel<T, 4, ORDER><<<grid, block, 0, f->stream>>>(nx, ny, bc, k, t1, u, acc, u);
  return cudaGetLastError();
}

// The four-cells-per-thread FP32 stage needs a width that is a multiple of 4, and at
// least 1.5 waves of its tiles (four resident per SM): on smaller grids the one-cell tiles
// keep more of the GPU busy.
bool use_f32v(const sslbm_fd4* f) {
  const int64_t tiles = ((f->g.nx + kVX - 1) / kVX) * ((f->g.ny + kVY - 1) / kVY);
  return f->g.nx % 4 == 0 && tiles >= 6 * (int64_t)f->sms;
}

template <typename T>
Fd4Coeffs<T> make_coeffs(const sslbm_grid* g, const sslbm_params* p) {
  Fd4Coeffs<T> k;
  k.beta = (T)p->beta;
  k.alpha = (T)p->alpha;
  k.gamma = (T)p->gamma;
  k.rg = (T)((1.0 - p->phi) * p->gamma);
  k.dg = (T)(p->phi * p->gamma);
  for (int c = 0; c < 4; ++c) k.d[c] = (T)p->d[c];
  k.inv = (T)(1.0 / (12.0 * g->dx * g->dx));
  k.inv2 = (T)(1.0 / (g->dx * g->dx));
  k.half_dt = (T)(0.5 * g->dt);
  k.dt = (T)g->dt;
  k.dt6 = (T)(g->dt / 6.0);
  return k;
}

}  // namespace

extern "C" {

int sslbm_fd4_workspace_bytes(const sslbm_grid* g, size_t* bytes) {
  if (!bytes) return err(SSLBM_ERR_BAD_ARG, "bytes is NULL");
  int st = check_grid(g);
  if (st) return st;
  *bytes = 4 * state_bytes(g);
  return SSLBM_OK;
}

int sslbm_fd4_create(const sslbm_grid* g, const sslbm_params* p, void* dev_ws, size_t ws_bytes, void* stream,
                     sslbm_fd4** out) {
  if (!out) return err(SSLBM_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  int st = check_grid(g);
  if (st) return st;
  if (!p) return err(SSLBM_ERR_BAD_ARG, "params is NULL");
  if (p->use_tau) return err(SSLBM_ERR_BAD_ARG, "the FD4 reference takes diffusivities d, not tau");
  const double rates[4] = {p->beta, p->alpha, p->gamma, p->phi};
  for (double r : rates)
    if (!std::isfinite(r) || r < 0) return err(SSLBM_ERR_BAD_ARG, "rates must be finite and >= 0");
  if (p->phi > 1) return err(SSLBM_ERR_BAD_ARG, "phi %g > 1", p->phi);
  for (int c = 0; c < 4; ++c)
    if (!std::isfinite(p->d[c]) || p->d[c] < 0) return err(SSLBM_ERR_BAD_ARG, "d[%d] must be finite and >= 0", c);
  if (p->d[4] != 0) return err(SSLBM_ERR_BAD_ARG, "d[D] must be 0 (D does not move)");
  // RK4 is stable on the negative real axis up to |z| = 2.78; the fourth-order Laplacian's
  // most negative eigenvalue is -(64/12) per axis / dx^2, so d dt / dx^2 <= 0.26 in 2D
  for (int c = 0; c < 4; ++c)
    if (p->d[c] * g->dt / (g->dx * g->dx) > 0.26)
      return err(SSLBM_ERR_UNSTABLE, "d[%d] dt / dx^2 = %g > 0.26 (RK4 with the fourth-order Laplacian)", c,
                 p->d[c] * g->dt / (g->dx * g->dx));
  const size_t need = 4 * state_bytes(g);
  if (!dev_ws || reinterpret_cast<uintptr_t>(dev_ws) % 256)
    return err(SSLBM_ERR_WORKSPACE, "workspace missing or not 256-byte aligned");
  if (ws_bytes < need) return err(SSLBM_ERR_WORKSPACE, "workspace of %zu bytes < %zu", ws_bytes, need);
  cudaPointerAttributes attr;
  CK(cudaPointerGetAttributes(&attr, dev_ws), "cudaPointerGetAttributes");
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return err(SSLBM_ERR_WORKSPACE, "workspace is not device memory");
  sslbm_fd4* f = new (std::nothrow) sslbm_fd4();
  if (!f) return err(SSLBM_ERR_BAD_ARG, "out of host memory");
  f->g = *g;
  f->ws = static_cast<char*>(dev_ws);
  f->sb = state_bytes(g);
  f->stream = static_cast<cudaStream_t>(stream);
  f->device = attr.device;
  f->k64 = make_coeffs<double>(g, p);
  f->k32 = make_coeffs<float>(g, p);
  DevGuard dg(f->device);
  if (cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, f->device) != cudaSuccess || f->sms < 1)
    f->sms = 1;
  cudaError_t e = cudaMemsetAsync(f->ws, 0, need, f->stream);
  if (e != cudaSuccess) {
    delete f;
    return cuda_err(e, "zero workspace");
  }
  *out = f;
  return SSLBM_OK;
}

void sslbm_fd4_destroy(sslbm_fd4* f) { delete f; }

int sslbm_fd4_write(sslbm_fd4* f, const void* src, int src_dtype, int src_on_device) {
  if (!f || !src) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  if (src_dtype != SSLBM_DT_F64 && src_dtype != SSLBM_DT_F32) return err(SSLBM_ERR_BAD_ARG, "dtype %d", src_dtype);
  DevGuard dg(f->device);
  const int64_t n = 5 * f->g.nx * f->g.ny;
  const size_t esz = src_dtype == SSLBM_DT_F64 ? 8 : 4;
  const void* s = src;
  if (!src_on_device) {  // stage through the second stage buffer (two buffers when FP32 holds FP64)
    CK(cudaMemcpyAsync(f->buf(1), src, (size_t)n * esz, cudaMemcpyHostToDevice, f->stream), "host -> device");
    s = f->buf(1);
  }
  const bool f64 = f->g.precision == SSLBM_FP64;
  if (src_dtype == SSLBM_DT_F64 && f64)
    CK(cudaMemcpyAsync(f->buf(0), s, (size_t)n * 8, cudaMemcpyDeviceToDevice, f->stream), "copy");
  else if (src_dtype == SSLBM_DT_F32 && !f64)
    CK(cudaMemcpyAsync(f->buf(0), s, (size_t)n * 4, cudaMemcpyDeviceToDevice, f->stream), "copy");
  else if (src_dtype == SSLBM_DT_F64)
    convert_kernel<double, float><<<blocks1(n), 256, 0, f->stream>>>(static_cast<const double*>(s),
                                                                     static_cast<float*>(f->buf(0)), n);
  else
    convert_kernel<float, double><<<blocks1(n), 256, 0, f->stream>>>(static_cast<const float*>(s),
                                                                     static_cast<double*>(f->buf(0)), n);
  CK(cudaGetLastError(), "convert");
  if (!src_on_device) CK(cudaStreamSynchronize(f->stream), "sync");
  f->steps = 0;
  return SSLBM_OK;
}

int sslbm_fd4_read(sslbm_fd4* f, void* dst, int dst_dtype, int dst_on_device) {
  if (!f || !dst) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  if (dst_dtype != SSLBM_DT_F64 && dst_dtype != SSLBM_DT_F32) return err(SSLBM_ERR_BAD_ARG, "dtype %d", dst_dtype);
  DevGuard dg(f->device);
  const int64_t n = 5 * f->g.nx * f->g.ny;
  const size_t esz = dst_dtype == SSLBM_DT_F64 ? 8 : 4;
  void* d = dst_on_device ? dst : f->buf(1);
  const bool f64 = f->g.precision == SSLBM_FP64;
  if ((dst_dtype == SSLBM_DT_F64) == f64)
    CK(cudaMemcpyAsync(d, f->buf(0), (size_t)n * esz, cudaMemcpyDeviceToDevice, f->stream), "copy");
  else if (f64)
    convert_kernel<double, float><<<blocks1(n), 256, 0, f->stream>>>(static_cast<const double*>(f->buf(0)),
                                                                     static_cast<float*>(d), n);
  else
    convert_kernel<float, double><<<blocks1(n), 256, 0, f->stream>>>(static_cast<const float*>(f->buf(0)),
                                                                     static_cast<double*>(d), n);
  CK(cudaGetLastError(), "convert");
  if (!dst_on_device) CK(cudaMemcpyAsync(dst, d, (size_t)n * esz, cudaMemcpyDeviceToHost, f->stream), "device -> host");
  CK(cudaStreamSynchronize(f->stream), "sync");
  return SSLBM_OK;
}

int sslbm_fd4_step(sslbm_fd4* f, int64_t n) {
  if (!f) return err(SSLBM_ERR_BAD_ARG, "NULL handle");
  if (n < 0) return err(SSLBM_ERR_BAD_ARG, "n < 0");
  DevGuard dg(f->device);
  for (int64_t i = 0; i < n; ++i) {
    cudaError_t e;
    if (f->g.precision == SSLBM_FP64)
      e = f->order == 4 ? run_step<double, 4>(f, f->k64) : run_step<double, 2>(f, f->k64);
    else if (use_f32v(f))
      e = f->order == 4 ? run_step_f32v<4>(f, f->k32) : run_step_f32v<2>(f, f->k32);
    else
      e = f->order == 4 ? run_step<float, 4>(f, f->k32) : run_step<float, 2>(f, f->k32);
    if (e != cudaSuccess) return cuda_err(e, "FD4 stage launch");
    ++f->steps;
  }
  return SSLBM_OK;
}

int64_t sslbm_fd4_steps_done(const sslbm_fd4* f) { return f ? f->steps : -1; }

int sslbm_fd4_set_order(sslbm_fd4* f, int order) {
  if (!f) return err(SSLBM_ERR_BAD_ARG, "NULL handle");
  if (order != 2 && order != 4) return err(SSLBM_ERR_BAD_ARG, "order %d is not 2 or 4", order);
  f->order = order;  // the create-time stability check (d dt / dx^2 <= 0.26) covers both orders
  return SSLBM_OK;
}

}  // extern "C"
