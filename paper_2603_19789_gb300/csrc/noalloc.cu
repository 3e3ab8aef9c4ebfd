// noalloc.cu -- population totals and peak infected of caller-provided fields, computed
// without allocating any device memory: the reduction's scratch is a file-scope
// __device__ array that lives in the library image.
//
// Who needs this: code that holds device buffers handed to it but cannot allocate --
// for instance a monitoring hook running inside another framework's time loop, where
// that framework's memory pool already owns the free device memory (a cudaMalloc there
// could fail, fragment the pool, or force a device-wide synchronisation), or a plain C
// caller that has no allocator wired to this device.  Such a caller cannot provide the
// workspace that sslbm_create() needs for sslbm_diagnostics().
//
// Scratch: one row of 6 doubles per lattice row (5 totals and a maximum) plus one
// result row, for at most kNoAllocMaxRows lattice rows: (16384 + 1) * 6 * 8 bytes
// = 768 KiB on every device that loads the library, held until the process exits.
// The array belongs to this file's device code: CUDA reserves it when it loads that code
// on a device, which under the default lazy module loading is the first call here (the
// symbol lookup below), and with CUDA_MODULE_LOADING=EAGER context creation.  A caller
// that cannot afford even that reservation later makes its first call at set-up.
// Every call writes each slot it later reads (no accumulation across calls), so nothing
// has to be cleared between calls; the array keeps the last call's partial sums.
// All calls on one device share the array: calls that overlap on the GPU (unordered
// streams, several host threads) race on it.
#include <float.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "sslbm_internal.cuh"

namespace sslbm {
int record_error(int status, const char* msg);
}

namespace {

constexpr int64_t kNoAllocMaxRows = 16384;
constexpr int kSlots = 6;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxRows + 1) * kSlots];

std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

__device__ void block_sum6(double (&v)[kSlots]) {
  __shared__ double sh[32][kSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] += __shfl_down_sync(0xffffffffu, v[j], off);
    v[5] = fmax(v[5], __shfl_down_sync(0xffffffffu, v[5], off));
  }
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < kSlots; ++j) sh[warp][j] = v[j];
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
  __syncthreads();  // sh is reused by the next row
}

// Row y's totals of the five planes (fields laid out [5][ny][nx]) and its maximum of I.
template <typename T>
__global__ void __launch_bounds__(256) noalloc_rows_kernel(const T* __restrict__ f, int64_t nx,
                                                           int64_t ny, double* __restrict__ scratch) {
  for (int64_t y = blockIdx.x; y < ny; y += gridDim.x) {
    double v[kSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, -DBL_MAX};
    for (int64_t x = threadIdx.x; x < nx; x += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const double r = (double)f[((int64_t)c * ny + y) * nx + x];
        v[c] += r;
        if (c == 2) v[5] = fmax(v[5], r);
      }
    }
    block_sum6(v);
    if (threadIdx.x == 0)
#pragma unroll
      for (int j = 0; j < kSlots; ++j) scratch[y * kSlots + j] = v[j];
  }
}

// Fixed-order total of the row partials into the result row.
__global__ void __launch_bounds__(256) noalloc_final_kernel(int64_t ny, double* __restrict__ scratch) {
  double v[kSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, -DBL_MAX};
  for (int64_t y = threadIdx.x; y < ny; y += blockDim.x) {
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] += scratch[y * kSlots + j];
    v[5] = fmax(v[5], scratch[y * kSlots + 5]);
  }
  block_sum6(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < kSlots; ++j) scratch[kNoAllocMaxRows * kSlots + j] = v[j];
}

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

}  // namespace

extern "C" int sslbm_diagnostics_noalloc(const void* fields, int dtype, int64_t nx, int64_t ny,
                                         double* totals, double* peak_I, void* stream) {
  if (!fields) return err(SSLBM_ERR_BAD_ARG, "fields is NULL");
  if (dtype != SSLBM_DT_F64 && dtype != SSLBM_DT_F32)
    return err(SSLBM_ERR_BAD_ARG, "dtype=%d is neither SSLBM_DT_F64 nor SSLBM_DT_F32", dtype);
  if (nx < 1 || nx > (int64_t(1) << 30) || ny < 1)
    return err(SSLBM_ERR_BAD_ARG, "nx=%lld ny=%lld must be >= 1 (nx <= 2^30)", (long long)nx,
               (long long)ny);
  if (ny > kNoAllocMaxRows)
    return err(SSLBM_ERR_BAD_ARG,
               "ny=%lld exceeds the %lld rows the built-in scratch of sslbm_diagnostics_noalloc "
               "holds; use sslbm_diagnostics with a workspace instead",
               (long long)ny, (long long)kNoAllocMaxRows);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return err(SSLBM_ERR_UNSUPPORTED, "device %d", dev);
  double* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(scratch)");
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned blocks = (unsigned)(ny < 1024 ? ny : 1024);
  if (dtype == SSLBM_DT_F64)
    noalloc_rows_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(fields), nx, ny, scratch);
  else
    noalloc_rows_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(fields), nx, ny, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "row reduction launch");
  noalloc_final_kernel<<<1, 256, 0, s>>>(ny, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "final reduction launch");
  double r[kSlots];
  e = cudaMemcpyAsync(r, scratch + kNoAllocMaxRows * kSlots, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync(result)");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "cudaStreamSynchronize");
  if (totals)
    for (int c = 0; c < 5; ++c) totals[c] = r[c];
  if (peak_I) *peak_I = r[5];
  for (int c = 0; c < 5; ++c)
    if (!(r[c] == r[c]) || r[c] == 1.0 / 0.0 || r[c] == -1.0 / 0.0)
      return err(SSLBM_ERR_NONFINITE, "total of compartment %d is %g", c, r[c]);
  return SSLBM_OK;
}
