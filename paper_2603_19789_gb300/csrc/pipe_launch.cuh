// pipe_launch.cuh -- the kernel and the host launchers of the temporal-blocked pipeline tile
// (sslbm_pipe.cuh), instantiated per mode by the translation units that launch it:
// sslbm_kernels.cu for the D2Q5 storages, pipe_d2q9.cu, pipe_d2q9_aligned.cu, pipe_vard.cu and
// pipe_kahan.cu for the D2Q9 and varying-diffusion lattices and the Kahan storage, pipe_diag.cu
// for the D2Q5 pipelines with the fused diagnostics (separate units, so that the build compiles
// them in parallel).
#pragma once
#include <atomic>

#include "bounds.cuh"
#include "sslbm_internal.cuh"
#include "sslbm_pipe.cuh"

namespace sslbm {
namespace {

// Dynamic shared memory of the pipeline tile: the row rings, and on the varying-diffusion
// lattice the static ring of the scale rows after them, or with the fused diagnostics their
// rows and reduction slots.
template <int MODE, int K, bool DIAG = false>
constexpr size_t pipe_smem_bytes() {
  return sizeof(PipeSmem<K, mode_planes<MODE>()>) + (MODE == MODE_VARD ? sizeof(float) * kRingK * 2 * 128 : 0) +
         (DIAG ? sizeof(DiagSmem<mode_planes<MODE>()>) : 0);
}

// kx, ky: the scale planes of the varying-diffusion lattice (MODE_VARD), else unused.
// DIAG: also the diagnostics partial of the CTA's output cells into diag[6 blockIdx.x ...].
template <int MODE, int K, bool DIAG = false>
__global__ void __launch_bounds__(32 * K, MODE == MODE_KAHAN ? 1 : 16 / K) pipe_kernel(const GridView g, const Coeffs<float> k,
                                                             const float* __restrict__ in,
                                                             float* __restrict__ out,
                                                             const int seg_rows, const int nstrips,
                                                             const float* __restrict__ kx,
                                                             const float* __restrict__ ky,
                                                             double* __restrict__ diag) {
  constexpr int NF = mode_planes<MODE>();
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  PipeSmem<K, NF>& sm = *reinterpret_cast<PipeSmem<K, NF>*>(pipe_smem);
  float* rk = reinterpret_cast<float*>(pipe_smem + sizeof(PipeSmem<K, NF>));
  const int strip = (int)(blockIdx.x % (unsigned)nstrips);
  const int64_t y0 = (int64_t)(blockIdx.x / (unsigned)nstrips) * seg_rows;
  const int64_t y1 = (y0 + seg_rows < g.ny) ? y0 + seg_rows : g.ny;
  if constexpr (DIAG) {
    DiagSmem<NF>* dsm = reinterpret_cast<DiagSmem<NF>*>(pipe_smem + sizeof(PipeSmem<K, NF>));
    pipe_tile<MODE, K, false, true, true>(sm, g, k, in, out, strip, y0, y1, nullptr, nullptr, nullptr, dsm, diag,
                                          (int)blockIdx.x);
  } else if ((MODE == MODE_D2Q9_NOFLUX || MODE == MODE_D2Q9_NOFLUX4) && strip != 0 && strip != nstrips - 1) {
    pipe_tile<MODE, K, false, false>(sm, g, k, in, out, strip, y0, y1);  // no wall column in this strip
  } else {
    pipe_tile<MODE, K>(sm, g, k, in, out, strip, y0, y1, kx, ky, rk);
  }
}

// The fused kernel's shared-memory attributes, set once per device (a bit per device in an
// atomic mask: host threads may launch concurrently; setting them twice is harmless).
template <int MODE, int K, bool DIAG = false>
void prefer_shared() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  cudaFuncSetAttribute(pipe_kernel<MODE, K, DIAG>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(pipe_kernel<MODE, K, DIAG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pipe_smem_bytes<MODE, K, DIAG>());
  done.fetch_or(bit, std::memory_order_release);
}

// Columns written per strip at depth K (128 computed, K of halo on each side rounded up to lanes).
constexpr int64_t pipe_strip_cols(int K) { return 128 - 8 * ((K + 3) / 4); }

// DIAG: diag receives one 6-double partial per CTA (at most kDiagBlocks CTAs).
template <int MODE, int K, bool DIAG = false>
cudaError_t launch_blocked_t(const GridView& g, const void* coeffs, const void* in, void* out,
                             int seg_rows, cudaStream_t s, const void* kx = nullptr, const void* ky = nullptr,
                             double* diag = nullptr) {
  constexpr int64_t WV = pipe_strip_cols(K);
  prefer_shared<MODE, K, DIAG>();
  if (seg_rows <= 0) return cudaErrorInvalidValue;
  const int64_t nstrips = (g.nx + WV - 1) / WV;
  const int64_t nseg = (g.ny + seg_rows - 1) / seg_rows;
  const int64_t blocks = nstrips * nseg;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (DIAG && (blocks > kDiagBlocks || diag == nullptr)) return cudaErrorInvalidConfiguration;
  pipe_kernel<MODE, K, DIAG><<<(unsigned)blocks, 32 * K, pipe_smem_bytes<MODE, K, DIAG>(), s>>>(
      g, *static_cast<const Coeffs<float>*>(coeffs), static_cast<const float*>(in),
      static_cast<float*>(out), seg_rows, (int)nstrips, static_cast<const float*>(kx),
      static_cast<const float*>(ky), diag);
  return cudaGetLastError();
}

template <int MODE, int K>
int default_seg_rows_t(const GridView& g) {
  constexpr int64_t WV = pipe_strip_cols(K);
  prefer_shared<MODE, K>();
  const int64_t nstrips = (g.nx + WV - 1) / WV;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pipe_kernel<MODE, K>, 32 * K, pipe_smem_bytes<MODE, K>());
  // one wave: as many CTAs as fit on the device at once, split into row segments.  D2Q9
  // no-flux: two waves, since the first and last strips (wall code) take longer than the rest
  const int64_t resident = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  int64_t nseg = (MODE == MODE_D2Q9_NOFLUX || MODE == MODE_D2Q9_NOFLUX4 ? 2 : 1) * resident / nstrips;
  if (nseg < 1) nseg = 1;
  int64_t rows = (g.ny + nseg - 1) / nseg;
  if (rows < 4 * K) rows = 4 * K;
  if (rows > (1 << 30)) rows = 1 << 30;
  return (int)rows;
}

template <int MODE, bool DIAG = false>
cudaError_t launch_blocked_mode(const GridView& g, const void* coeffs, const void* in, void* out,
                                int depth, int seg_rows, cudaStream_t s, const void* kx = nullptr,
                                const void* ky = nullptr, double* diag = nullptr) {
  switch (depth) {
    case 2: return launch_blocked_t<MODE, 2, DIAG>(g, coeffs, in, out, seg_rows, s, kx, ky, diag);
    case 3: return launch_blocked_t<MODE, 3, DIAG>(g, coeffs, in, out, seg_rows, s, kx, ky, diag);
    case 4: return launch_blocked_t<MODE, 4, DIAG>(g, coeffs, in, out, seg_rows, s, kx, ky, diag);
    case 5: return launch_blocked_t<MODE, 5, DIAG>(g, coeffs, in, out, seg_rows, s, kx, ky, diag);
    case 6: return launch_blocked_t<MODE, 6, DIAG>(g, coeffs, in, out, seg_rows, s, kx, ky, diag);
    case 7: return launch_blocked_t<MODE, 7, DIAG>(g, coeffs, in, out, seg_rows, s, kx, ky, diag);
    case 8: return launch_blocked_t<MODE, 8, DIAG>(g, coeffs, in, out, seg_rows, s, kx, ky, diag);
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE>
int default_seg_rows_mode(const GridView& g, int depth) {
  switch (depth) {
    case 2: return default_seg_rows_t<MODE, 2>(g);
    case 3: return default_seg_rows_t<MODE, 3>(g);
    case 4: return default_seg_rows_t<MODE, 4>(g);
    case 5: return default_seg_rows_t<MODE, 5>(g);
    case 6: return default_seg_rows_t<MODE, 6>(g);
    case 7: return default_seg_rows_t<MODE, 7>(g);
    case 8: return default_seg_rows_t<MODE, 8>(g);
    default: return 0;
  }
}

}  // namespace
}  // namespace sslbm
