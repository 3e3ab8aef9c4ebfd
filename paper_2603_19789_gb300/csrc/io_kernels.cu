// io_kernels.cu -- conversion between the caller's contiguous ny x nx planes and the
// solver's pitched storage, and the diagnostics reduction of Sec. II.C 'Mass conservation'
// (per-compartment totals in double precision, peak infected density).
#include <float.h>
#include <stdint.h>

#include "bounds.cuh"
#include "sslbm_internal.cuh"

SSLBM_OOB_ACCESSOR(io)

namespace sslbm {

namespace {

dim3 row_grid(const GridView& g, int threads) {
  int64_t gy = g.ny < 65535 ? g.ny : 65535;
  return dim3((unsigned)((g.nx + threads - 1) / threads), (unsigned)gy);
}

// plane <- src (contiguous).  dev_S: store s_ref - value.  comp (Kahan): the rounding residue
// of the stored value, so that value - compensation reproduces the input.
template <typename T, typename U>
__global__ void plane_write_kernel(const GridView g, const U* __restrict__ src,
                                   T* __restrict__ plane, T* __restrict__ comp, int dev_S,
                                   double s_ref) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  for (int64_t y = blockIdx.y; y < g.ny; y += gridDim.y) {
    double v = (double)src[y * g.nx + x];
    if (dev_S) v = s_ref - v;
    const T hi = (T)v;
    plane[y * g.pitch + x] = hi;
    if (comp) comp[y * g.pitch + x] = (T)((double)hi - v);
  }
}

// dst (contiguous) <- plane, evaluated in double: value - compensation, s_ref - sigma.
template <typename T, typename U>
__global__ void plane_read_kernel(const GridView g, const T* __restrict__ plane,
                                  const T* __restrict__ comp, int dev_S, double s_ref,
                                  U* __restrict__ dst) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  for (int64_t y = blockIdx.y; y < g.ny; y += gridDim.y) {
    double v = (double)plane[y * g.pitch + x];
    if (comp) v -= (double)comp[y * g.pitch + x];
    if (dev_S) v = s_ref - v;
    dst[y * g.nx + x] = (U)v;
  }
}

// Block-wide reduction of kDiagSlots values (sums of slots 0..4, max of slot 5) in a fixed
// order, result valid in thread 0.
__device__ void block_reduce6(double (&v)[kDiagSlots]) {
  __shared__ double sh[32][kDiagSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] += __shfl_down_sync(0xffffffffu, v[j], off);
    v[5] = fmax(v[5], __shfl_down_sync(0xffffffffu, v[5], off));
  }
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < kDiagSlots; ++j) sh[warp][j] = v[j];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] = lane < nw ? sh[lane][j] : 0.0;
    v[5] = lane < nw ? sh[lane][5] : -DBL_MAX;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int j = 0; j < 5; ++j) v[j] += __shfl_down_sync(0xffffffffu, v[j], off);
      v[5] = fmax(v[5], __shfl_down_sync(0xffffffffu, v[5], off));
    }
  }
}

// Per-block partial totals of the five compartments and the maximum of I.
// LAYOUT 0: SSLBM planes (value minus Kahan compensation when comp != nullptr);
// LAYOUT 1: BGK populations, rho^C = sum_i f_i^C, and D in plane 20.
template <typename T, int LAYOUT>
__global__ void __launch_bounds__(256) diag_partial_kernel(const GridView g,
                                                           const T* __restrict__ st,
                                                           const T* __restrict__ comp,
                                                           double* __restrict__ partials, int n_comp) {
  double v[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, -DBL_MAX};
  for (int64_t y = blockIdx.x; y < g.ny; y += gridDim.x) {
    for (int64_t x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const int64_t idx = y * g.pitch + x;
      double r[5];
      if (LAYOUT == 0) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          r[c] = (double)st[c * g.plane + idx];
          if (comp && c < n_comp) r[c] -= (double)comp[c * g.plane + idx];
        }
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T a = st[(c * 5) * g.plane + idx];
#pragma unroll
          for (int i = 1; i < 5; ++i) a = add_rn(a, st[(c * 5 + i) * g.plane + idx]);
          r[c] = (double)a;
        }
        r[4] = (double)st[20 * g.plane + idx];
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) v[c] += r[c];
      v[5] = fmax(v[5], r[2]);
    }
  }
  block_reduce6(v);
  if (threadIdx.x == 0 && SSLBM_IN(blockIdx.x, 1, kDiagBlocks, 31)) {
#pragma unroll
    for (int j = 0; j < kDiagSlots; ++j) partials[blockIdx.x * kDiagSlots + j] = v[j];
  }
}

// Knuth's TwoSum: hi + lo <- hi + x with the rounding error of the addition carried into lo,
// so that FP32 arithmetic keeps the running sum to about twice FP32's precision.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// The FP32 partials of diag_partial_kernel without per-cell FP64 arithmetic (few FP64 units
// on this GPU): each thread reads 4 cells per plane at a time (16-byte loads; the pitch and
// the plane stride are multiples of 4) and keeps its share of the rows as a TwoSum pair per
// compartment, renormalised (Fast2Sum) after every 4 cells and added to the FP64 partial every
// kFlushRows rows and at the end.  After a renormalisation the pair's low part is at most half
// an ulp of its high part, so the pair's own rounding stays near FP32's unit roundoff squared
// per group of 4 cells.  (Adding the pair to FP64 after every row, the earlier form, took
// 265 us per 8192^2 call against 255 us now: GB300 has few FP64 units.)
// NCOMP: the first NCOMP compartments carry a compensation plane (0; 1 for the split S; 5 for
// Kahan), subtracted from the values.  The peak of I is taken in FP32 (the same value as in
// FP64), or in FP64 as value minus compensation when I has one.
template <int LAYOUT, int NCOMP>
__global__ void __launch_bounds__(256) diag_partial_f32x4_kernel(const GridView g, const float* __restrict__ st,
                                                                 const float* __restrict__ comp,
                                                                 double* __restrict__ partials) {
  constexpr int kFlushRows = 16;
  double v[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, -DBL_MAX};
  float hi[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, lo[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float pk = -FLT_MAX;
  int rows = 0;
  auto flush = [&]() {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      v[c] += (double)hi[c] + (double)lo[c];
      hi[c] = lo[c] = 0.f;
    }
  };
  for (int64_t y = blockIdx.x; y < g.ny; y += gridDim.x) {
    for (int64_t x = 4 * (int64_t)threadIdx.x; x < g.nx; x += 4 * (int64_t)blockDim.x) {
      if (!SSLBM_IN(x, 4, g.pitch, 30)) continue;
      const int64_t idx = y * g.pitch + x;
      const int nv = g.nx - x < 4 ? (int)(g.nx - x) : 4;
      float r[5][4];
      if (LAYOUT == 0) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const float4 a = *reinterpret_cast<const float4*>(st + c * g.plane + idx);
          r[c][0] = a.x, r[c][1] = a.y, r[c][2] = a.z, r[c][3] = a.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float4 a = *reinterpret_cast<const float4*>(st + (c * 5) * g.plane + idx);
#pragma unroll
          for (int i = 1; i < 5; ++i) {
            const float4 b = *reinterpret_cast<const float4*>(st + (c * 5 + i) * g.plane + idx);
            a.x = __fadd_rn(a.x, b.x), a.y = __fadd_rn(a.y, b.y), a.z = __fadd_rn(a.z, b.z), a.w = __fadd_rn(a.w, b.w);
          }
          r[c][0] = a.x, r[c][1] = a.y, r[c][2] = a.z, r[c][3] = a.w;
        }
        const float4 d = *reinterpret_cast<const float4*>(st + 20 * g.plane + idx);
        r[4][0] = d.x, r[4][1] = d.y, r[4][2] = d.z, r[4][3] = d.w;
      }
      float q[5][4];
      if (NCOMP > 0) {
#pragma unroll
        for (int c = 0; c < NCOMP; ++c) {
          const float4 b = *reinterpret_cast<const float4*>(comp + c * g.plane + idx);
          q[c][0] = b.x, q[c][1] = b.y, q[c][2] = b.z, q[c][3] = b.w;
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= nv) break;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          two_sum_add(hi[c], lo[c], r[c][j]);
          if (c < NCOMP) two_sum_add(hi[c], lo[c], -q[c][j]);
        }
        if (NCOMP > 2)
          v[5] = fmax(v[5], (double)r[2][j] - (double)q[2][j]);
        else
          pk = fmaxf(pk, r[2][j]);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) {  // Fast2Sum: |lo| <= ulp(hi) / 2 again
        const float t = __fadd_rn(hi[c], lo[c]);
        lo[c] = __fsub_rn(lo[c], __fsub_rn(t, hi[c]));
        hi[c] = t;
      }
    }
    if (++rows == kFlushRows) {
      flush();
      rows = 0;
    }
  }
  flush();
  if (NCOMP <= 2) v[5] = fmax(v[5], (double)pk);
  block_reduce6(v);
  if (threadIdx.x == 0 && SSLBM_IN(blockIdx.x, 1, kDiagBlocks, 31)) {
#pragma unroll
    for (int j = 0; j < kDiagSlots; ++j) partials[blockIdx.x * kDiagSlots + j] = v[j];
  }
}

// Sum of the per-block partials in a fixed order (deterministic).
__global__ void __launch_bounds__(256) diag_final_kernel(const double* __restrict__ partials,
                                                         int nblocks, double* __restrict__ result) {
  double v[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, -DBL_MAX};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] += partials[b * kDiagSlots + j];
    v[5] = fmax(v[5], partials[b * kDiagSlots + 5]);
  }
  block_reduce6(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < kDiagSlots; ++j) result[j] = v[j];
  }
}

}  // namespace

cudaError_t launch_plane_write(int precision, const GridView& g, const void* src, int src_dtype,
                               void* plane, void* comp_plane, int dev_S, double s_ref,
                               cudaStream_t s) {
  const dim3 grid = row_grid(g, 128);
  if (precision == SSLBM_FP64) {
    if (src_dtype == SSLBM_DT_F64)
      plane_write_kernel<double, double><<<grid, 128, 0, s>>>(g, (const double*)src, (double*)plane,
                                                              (double*)comp_plane, dev_S, s_ref);
    else
      plane_write_kernel<double, float><<<grid, 128, 0, s>>>(g, (const float*)src, (double*)plane,
                                                             (double*)comp_plane, dev_S, s_ref);
  } else {
    if (src_dtype == SSLBM_DT_F64)
      plane_write_kernel<float, double><<<grid, 128, 0, s>>>(g, (const double*)src, (float*)plane,
                                                             (float*)comp_plane, dev_S, s_ref);
    else
      plane_write_kernel<float, float><<<grid, 128, 0, s>>>(g, (const float*)src, (float*)plane,
                                                            (float*)comp_plane, dev_S, s_ref);
  }
  return cudaGetLastError();
}

cudaError_t launch_plane_read(int precision, const GridView& g, const void* plane,
                              const void* comp_plane, int dev_S, double s_ref, void* dst,
                              int dst_dtype, cudaStream_t s) {
  const dim3 grid = row_grid(g, 128);
  if (precision == SSLBM_FP64) {
    if (dst_dtype == SSLBM_DT_F64)
      plane_read_kernel<double, double><<<grid, 128, 0, s>>>(g, (const double*)plane,
                                                             (const double*)comp_plane, dev_S,
                                                             s_ref, (double*)dst);
    else
      plane_read_kernel<double, float><<<grid, 128, 0, s>>>(g, (const double*)plane,
                                                            (const double*)comp_plane, dev_S,
                                                            s_ref, (float*)dst);
  } else {
    if (dst_dtype == SSLBM_DT_F64)
      plane_read_kernel<float, double><<<grid, 128, 0, s>>>(g, (const float*)plane,
                                                            (const float*)comp_plane, dev_S, s_ref,
                                                            (double*)dst);
    else
      plane_read_kernel<float, float><<<grid, 128, 0, s>>>(g, (const float*)plane,
                                                           (const float*)comp_plane, dev_S, s_ref,
                                                           (float*)dst);
  }
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(int precision, int layout, const GridView& g, const void* planes,
                               const void* comp_planes, double* partials, double* result,
                               cudaStream_t s, int n_comp) {
  if (!comp_planes) n_comp = 0;
  if (n_comp != 0 && n_comp != 1 && n_comp != 5) return cudaErrorInvalidValue;
  int64_t blocks = g.ny < kDiagBlocks ? g.ny : kDiagBlocks;
  if (blocks < 1) blocks = 1;
  if (precision == SSLBM_FP64) {
    if (layout == 0)
      diag_partial_kernel<double, 0><<<(unsigned)blocks, 256, 0, s>>>(
          g, (const double*)planes, (const double*)comp_planes, partials, n_comp);
    else
      diag_partial_kernel<double, 1><<<(unsigned)blocks, 256, 0, s>>>(g, (const double*)planes,
                                                                      nullptr, partials, 0);
  } else if (g.pitch % 4 == 0 && g.plane % 4 == 0 && reinterpret_cast<uintptr_t>(planes) % 16 == 0 &&
             reinterpret_cast<uintptr_t>(comp_planes) % 16 == 0) {
    const float* st = (const float*)planes;
    const float* cp = (const float*)comp_planes;
    if (layout == 1)
      diag_partial_f32x4_kernel<1, 0><<<(unsigned)blocks, 256, 0, s>>>(g, st, nullptr, partials);
    else if (n_comp == 5)
      diag_partial_f32x4_kernel<0, 5><<<(unsigned)blocks, 256, 0, s>>>(g, st, cp, partials);
    else if (n_comp == 1)
      diag_partial_f32x4_kernel<0, 1><<<(unsigned)blocks, 256, 0, s>>>(g, st, cp, partials);
    else
      diag_partial_f32x4_kernel<0, 0><<<(unsigned)blocks, 256, 0, s>>>(g, st, nullptr, partials);
  } else {
    if (layout == 0)
      diag_partial_kernel<float, 0><<<(unsigned)blocks, 256, 0, s>>>(
          g, (const float*)planes, (const float*)comp_planes, partials, n_comp);
    else
      diag_partial_kernel<float, 1><<<(unsigned)blocks, 256, 0, s>>>(g, (const float*)planes,
                                                                     nullptr, partials, 0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, 256, 0, s>>>(partials, (int)blocks, result);
  return cudaGetLastError();
}

cudaError_t launch_diag_final(const double* partials, int nblocks, double* result, cudaStream_t s) {
  if (nblocks < 1 || nblocks > kDiagBlocks) return cudaErrorInvalidValue;
  diag_final_kernel<<<1, 256, 0, s>>>(partials, nblocks, result);
  return cudaGetLastError();
}

namespace {
// One index check with no memory access behind it (site 999).
__global__ void oob_probe_kernel(long long v, long long limit) { (void)SSLBM_IN(v, 1, limit, 999); }
}  // namespace

cudaError_t launch_oob_probe(long long v, long long limit, cudaStream_t s) {
  oob_probe_kernel<<<1, 1, 0, s>>>(v, limit);
  return cudaGetLastError();
}

}  // namespace sslbm
