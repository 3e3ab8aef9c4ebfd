// sslbm_kernels.cu -- SSLBM time-step kernels (Sec. II.C, Eq. sslbm_final_clean with the
// sources of Eq. sources and the deceased update of Eq. rhoD).
//
// Two kernels advance the same update:
//   step1_kernel    one step per launch (FP64, FP32, FP32 deviation-S, FP32 split-S).
//   kahan_stream_kernel  one step per launch of the Kahan storage (ten planes): warps stream
//                   down column strips through a cp.async ring of rows in shared memory.  Each thread updates V consecutive cells of a row with
//                   16-byte vector loads (float4 / double2) of the centre, upper and lower
//                   rows and two scalar edge loads; neighbouring rows come from L1/L2.
//   pipe_kernel     K steps per launch (temporal blocking, K = 2..8) for FP32, FP32
//                   deviation-S and FP32 split-S (a sixth plane), as a pipeline of K warps per CTA: warp s computes level s+1
//                   of the time-step wavefront.  A CTA owns a 128-column strip (4 columns
//                   per lane, 16-byte accesses) with a K-column halo on each side and
//                   streams down a segment of rows, two rows per step of the pipeline.
//                   Warp 0 brings level-0 rows in with cp.async into a shared-memory ring
//                   three row pairs ahead; every level's output pair goes through a
//                   double-buffered shared-memory slot (dynamic shared memory) to the next
//                   warp, one CTA barrier per pair; the last warp writes level K to global
//                   memory.  Each warp keeps only its own level's rows in four register
//                   buffers (about 110 registers per thread), so two or more CTAs share an
//                   SM.  x neighbours come from warp shuffles.  Rows and columns
//                   outside the domain are loaded as ghost images (periodic wrap or the
//                   even mirror extension), which the uniform stencil keeps consistent, so
//                   no boundary logic is needed inside the pipeline.  DRAM traffic is one
//                   read and one write of the five planes per K steps.
// Both use the same per-cell expressions (sslbm_internal.cuh), so a blocked launch gives
// the same bits as K one-step launches.
#include <atomic>

#include "bounds.cuh"
#include "sslbm_internal.cuh"
#include "sslbm_pipe.cuh"

SSLBM_OOB_ACCESSOR(kernels)

namespace sslbm {

namespace {

template <typename T, int V>
struct Vec;
template <>
struct Vec<float, 4> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  static __device__ __forceinline__ void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec<double, 2> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
  static __device__ __forceinline__ void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

template <typename T, int V, int MODE>
__global__ void __launch_bounds__(256, 1) step1_kernel(const GridView g, const Coeffs<T> k,
                                                    const T* __restrict__ in, T* __restrict__ out) {
  const int64_t nvec = (g.nx + V - 1) / V;
  const int64_t vx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vx >= nvec) return;
  const int64_t x0 = vx * V;
  const int nvalid = (int)((g.nx - x0) < V ? (g.nx - x0) : V);
  const int64_t xl = link_index(x0 - 1, g.nx, g.bc);
  const int64_t xr = link_index(x0 + nvalid, g.nx, g.bc);
  for (int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; y < g.ny;
       y += (int64_t)gridDim.y * blockDim.y) {
    const int64_t yu = link_index(y - 1, g.ny, g.bc), yd = link_index(y + 1, g.ny, g.bc);
    if (!(SSLBM_IN(yu, 1, g.ny, 10) && SSLBM_IN(yd, 1, g.ny, 11) && SSLBM_IN(x0, V, g.pitch, 12) &&
          SSLBM_IN(xl, 1, g.nx, 13) && SSLBM_IN(xr, 1, g.nx, 14)))
      continue;
    const int64_t rc = y * g.pitch;
    const int64_t ru = yu * g.pitch;
    const int64_t rd = yd * g.pitch;
    T c[4][V], lap[4][V];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T* P = in + f * g.plane;
      T u[V], d[V];
      Vec<T, V>::load(P + rc + x0, c[f]);
      Vec<T, V>::load(P + ru + x0, u);
      Vec<T, V>::load(P + rd + x0, d);
      const T L = P[rc + xl];
      const T R = P[rc + xr];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const T l = (j == 0) ? L : c[f][j > 0 ? j - 1 : 0];
        T r = R;
        if (j + 1 < V) {
          if (j + 1 < nvalid) r = c[f][j + 1 < V ? j + 1 : j];
        }
        if (MODE == MODE_SPLIT && f == 0)
          lap[f][j] = lap5_diff(c[f][j], l, r, u[j], d[j]);
        else
          lap[f][j] = lap5(c[f][j], l, r, u[j], d[j]);
      }
      if (MODE == MODE_SPLIT && f == 0) {
        // the represented value is value - compensation: subtract the compensation's laplacian
        const T* Q = in + (5 + f) * g.plane;
        T qc[V], qu[V], qd[V];
        Vec<T, V>::load(Q + rc + x0, qc);
        Vec<T, V>::load(Q + ru + x0, qu);
        Vec<T, V>::load(Q + rd + x0, qd);
        const T QL = Q[rc + xl];
        const T QR = Q[rc + xr];
#pragma unroll
        for (int j = 0; j < V; ++j) {
          const T l = (j == 0) ? QL : qc[j > 0 ? j - 1 : 0];
          T r = QR;
          if (j + 1 < V) {
            if (j + 1 < nvalid) r = qc[j + 1 < V ? j + 1 : j];
          }
          lap[f][j] = sub_rn(lap[f][j], lap5_diff(qc[j], l, r, qu[j], qd[j]));
        }
      }
    }
    T D[V];
    Vec<T, V>::load(in + 4 * g.plane + rc + x0, D);
    T n[5][V];
    if constexpr (MODE == MODE_SPLIT) {
      T cmp[V], ncmp[V];
      Vec<T, V>::load(in + 5 * g.plane + rc + x0, cmp);
#pragma unroll
      for (int j = 0; j < V; ++j)
        seird_cell_split(k, c[0][j], cmp[j], c[1][j], c[2][j], c[3][j], D[j], lap[0][j], lap[1][j], lap[2][j],
                         lap[3][j], n[0][j], ncmp[j], n[1][j], n[2][j], n[3][j], n[4][j]);
      if (nvalid == V) {
        Vec<T, V>::store(out + 5 * g.plane + rc + x0, ncmp);
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j)
          if (j < nvalid) out[5 * g.plane + rc + x0 + j] = ncmp[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if constexpr (MODE == MODE_DEV) {
          seird_cell_dev(k, c[0][j], c[1][j], c[2][j], c[3][j], D[j], lap[0][j], lap[1][j],
                         lap[2][j], lap[3][j], n[0][j], n[1][j], n[2][j], n[3][j], n[4][j]);
        } else {
          seird_cell(k, c[0][j], c[1][j], c[2][j], c[3][j], D[j], lap[0][j], lap[1][j], lap[2][j],
                     lap[3][j], n[0][j], n[1][j], n[2][j], n[3][j], n[4][j]);
        }
      }
    }
    if (nvalid == V) {
#pragma unroll
      for (int f = 0; f < 5; ++f) Vec<T, V>::store(out + f * g.plane + rc + x0, n[f]);
    } else {
#pragma unroll
      for (int f = 0; f < 5; ++f)
#pragma unroll
        for (int j = 0; j < V; ++j)
          if (j < nvalid) out[f * g.plane + rc + x0 + j] = n[f][j];
    }
  }
}

// ---- streaming one-step kernel of the Kahan storage -------------------------------------
// Each warp owns a strip of kKsCols columns and a segment of kKsSeg rows and walks down it.
// The rows of the ten planes (values and compensations, one halo column on each side,
// periodic wrap or mirror at the domain's edges) arrive by cp.async in a ring of kKsRing
// rows in shared memory, kKsRing - 3 rows ahead of the rows being read; every plane is read
// from global memory once per step.  Lane l updates columns xs + l and xs + 32 + l with the
// compensated update: lap5_diff of values minus that of compensations, seird_increments,
// kahan_add (the per-cell expressions of the earlier two-cells-per-thread Kahan kernel, so
// results are unchanged; it ran at 38.6 GLUPS on the 8192^2 grid, 46% of HBM).  Ring row
// layout per plane: index i holds column xs - 4 + i; the 64 interior columns start at
// index 4 (16-byte aligned for the vector copies), the halos sit at 3 and 68.
// Ring depth and warps per CTA measured at 8192^2: 8 rows (five in flight) and 2 warps
// (four CTAs, eight warps per SM) 77.3 GLUPS; 8 and 4 warps 76.5; 7 and 3 warps 68.3;
// 6 and 4 warps 61.3; 10 and 2 warps (three CTAs per SM) 66.6.
constexpr int kKsCols = 64, kKsStride = 72, kKsRing = 8, kKsSeg = 128, kKsWarps = 2;
constexpr int kKsWarpFloats = kKsRing * 10 * kKsStride;

__device__ __forceinline__ int64_t ks_col(int64_t x, const GridView& g) {
  if (x >= 0 && x < g.nx) return x;
  if (x == -1 || x == g.nx) return link_index(x, g.nx, g.bc);
  return x < 0 ? 0 : g.nx - 1;  // never a neighbour of a written cell
}

__global__ void __launch_bounds__(32 * kKsWarps, 4) kahan_stream_kernel(const GridView g, const Coeffs<float> k,
                                                                       const float* __restrict__ in,
                                                                       float* __restrict__ out, const int nstrips,
                                                                       const int nitems) {
  extern __shared__ __align__(16) float ks_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int item = blockIdx.x * kKsWarps + warp;
  if (item >= nitems) return;
  float* ring = ks_smem + (size_t)warp * kKsWarpFloats;
  const int strip = item % nstrips;
  const int64_t xs = (int64_t)strip * kKsCols;
  const int64_t y0 = (int64_t)(item / nstrips) * kKsSeg;
  const int64_t y1 = y0 + kKsSeg < g.ny ? y0 + kKsSeg : g.ny;
  const bool vec = xs + kKsCols <= g.nx;
  const int64_t xl = ks_col(xs - 1, g), xr = ks_col(xs + kKsCols, g);
  const int64_t q0 = y0 - 1;  // first logical row in the ring
  auto issue = [&](int64_t q) {  // rows q0 .. y1 (one beyond the segment on each side)
    const int64_t yq = link_index(q, g.ny, g.bc);
    if (q <= y1 && SSLBM_IN(yq, 1, g.ny, 15)) {
      const int64_t row = yq * g.pitch;
      float* dst = ring + (int)((q - q0) % kKsRing) * (10 * kKsStride);
      if (vec) {
        for (int u = lane; u < 10 * 16; u += 32) {
          const int f = u >> 4, part = u & 15;
          if (SSLBM_IN(xs + 4 * part, 4, g.nx, 16))
            cp_async16(dst + f * kKsStride + 4 + 4 * part, in + f * g.plane + row + xs + 4 * part);
        }
        if (lane < 20) {
          const int f = lane % 10;
          const int64_t xh = lane < 10 ? xl : xr;
          if (SSLBM_IN(xh, 1, g.nx, 17)) cp_async4(dst + f * kKsStride + (lane < 10 ? 3 : 68), in + f * g.plane + row + xh);
        }
      } else {
        for (int u = lane; u < 10 * 66; u += 32) {
          const int f = u / 66, i = 3 + u % 66;
          const int64_t xc = ks_col(xs - 4 + i, g);
          if (SSLBM_IN(xc, 1, g.nx, 18)) cp_async4(dst + f * kKsStride + i, in + f * g.plane + row + xc);
        }
      }
    }
    cp_async_commit();  // one group per row, empty beyond the segment
  };
  // rows y - 1, y, y + 1 are in use, kKsRing - 3 further rows are in flight
  for (int64_t q = q0; q < q0 + kKsRing - 1; ++q) issue(q);
  for (int64_t y = y0; y < y1; ++y) {
    __syncwarp();  // every lane is done with the slot that row y + kKsRing - 2 takes over
    issue(y + kKsRing - 2);
    cp_async_wait<kKsRing - 3>();  // rows up to y + 1 are in
    __syncwarp();
    const float* U = ring + (int)((y - 1 - q0) % kKsRing) * (10 * kKsStride);
    const float* C = ring + (int)((y - q0) % kKsRing) * (10 * kKsStride);
    const float* N = ring + (int)((y + 1 - q0) % kKsRing) * (10 * kKsStride);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t x = xs + lane + 32 * h;
      if (x >= g.nx || !SSLBM_IN(y, 1, g.ny, 19)) continue;
      const int i = 4 + lane + 32 * h;
      float c[5], cmp[5], lap[4];
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        const float* P = C + f * kKsStride;
        const float* Q = C + (5 + f) * kKsStride;
        c[f] = P[i];
        cmp[f] = Q[i];
        if (f < 4) {
          lap[f] = lap5_diff(P[i], P[i - 1], P[i + 1], U[f * kKsStride + i], N[f * kKsStride + i]);
          lap[f] = sub_rn(lap[f], lap5_diff(Q[i], Q[i - 1], Q[i + 1], U[(5 + f) * kKsStride + i],
                                            N[(5 + f) * kKsStride + i]));
        }
      }
      float inc[5];
      seird_increments(k, c[0], c[1], c[2], c[3], lap[0], lap[1], lap[2], lap[3], inc);
      float* o = out + y * g.pitch + x;
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        float v = c[f], q = cmp[f];
        kahan_add(v, q, inc[f]);
        o[f * g.plane] = v;
        o[(5 + f) * g.plane] = q;
      }
    }
  }
  cp_async_wait<0>();
}

template <int MODE, int K>
__global__ void __launch_bounds__(32 * K, 16 / K) pipe_kernel(const GridView g, const Coeffs<float> k,
                                                             const float* __restrict__ in,
                                                             float* __restrict__ out,
                                                             const int seg_rows, const int nstrips) {
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  PipeSmem<K, mode_planes<MODE>()>& sm = *reinterpret_cast<PipeSmem<K, mode_planes<MODE>()>*>(pipe_smem);
  const int strip = (int)(blockIdx.x % (unsigned)nstrips);
  const int64_t y0 = (int64_t)(blockIdx.x / (unsigned)nstrips) * seg_rows;
  const int64_t y1 = (y0 + seg_rows < g.ny) ? y0 + seg_rows : g.ny;
  pipe_tile<MODE, K>(sm, g, k, in, out, strip, y0, y1);
}

template <typename T, int V, int MODE>
cudaError_t launch_step1_t(const GridView& g, const void* coeffs, const void* in, void* out,
                           cudaStream_t s) {
  const int64_t nvec = (g.nx + V - 1) / V;
  dim3 block(32, 8);
  int64_t gy = (g.ny + 7) / 8;
  if (gy > 65535) gy = 65535;
  dim3 grid((unsigned)((nvec + 31) / 32), (unsigned)gy);
  step1_kernel<T, V, MODE><<<grid, block, 0, s>>>(g, *static_cast<const Coeffs<T>*>(coeffs),
                                                  static_cast<const T*>(in), static_cast<T*>(out));
  return cudaGetLastError();
}

// The fused kernel's shared-memory attributes, set once per device (a bit per device in an
// atomic mask: host threads may launch concurrently; setting them twice is harmless).
template <int MODE, int K>
void prefer_shared() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  cudaFuncSetAttribute(pipe_kernel<MODE, K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(pipe_kernel<MODE, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(PipeSmem<K, mode_planes<MODE>()>));
  done.fetch_or(bit, std::memory_order_release);
}

template <int MODE, int K>
cudaError_t launch_blocked_t(const GridView& g, const void* coeffs, const void* in, void* out,
                             int seg_rows, cudaStream_t s) {
  constexpr int HL = (K + 3) / 4;
  constexpr int WV = 128 - 8 * HL;
  prefer_shared<MODE, K>();
  if (seg_rows <= 0) return cudaErrorInvalidValue;
  const int64_t nstrips = (g.nx + WV - 1) / WV;
  const int64_t nseg = (g.ny + seg_rows - 1) / seg_rows;
  const int64_t blocks = nstrips * nseg;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  pipe_kernel<MODE, K><<<(unsigned)blocks, 32 * K, sizeof(PipeSmem<K, mode_planes<MODE>()>), s>>>(
      g, *static_cast<const Coeffs<float>*>(coeffs), static_cast<const float*>(in),
      static_cast<float*>(out), seg_rows, (int)nstrips);
  return cudaGetLastError();
}

cudaError_t launch_kahan_stream(const GridView& g, const void* coeffs, const void* in, void* out,
                                cudaStream_t s) {
  constexpr size_t smem = sizeof(float) * kKsWarpFloats * kKsWarps;
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && !(done.load(std::memory_order_acquire) & (1ull << (dev & 63)))) {
    cudaFuncSetAttribute(kahan_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done.fetch_or(1ull << (dev & 63), std::memory_order_release);
  }
  const int64_t nstrips = (g.nx + kKsCols - 1) / kKsCols;
  const int64_t items = nstrips * ((g.ny + kKsSeg - 1) / kKsSeg);
  if (items > 0x7fffffffLL - kKsWarps) return cudaErrorInvalidConfiguration;
  kahan_stream_kernel<<<(unsigned)((items + kKsWarps - 1) / kKsWarps), 32 * kKsWarps, smem, s>>>(
      g, *static_cast<const Coeffs<float>*>(coeffs), static_cast<const float*>(in), static_cast<float*>(out),
      (int)nstrips, (int)items);
  return cudaGetLastError();
}

template <int MODE, int K>
int default_seg_rows_t(const GridView& g) {
  constexpr int HL = (K + 3) / 4;
  constexpr int WV = 128 - 8 * HL;
  prefer_shared<MODE, K>();
  const int64_t nstrips = (g.nx + WV - 1) / WV;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pipe_kernel<MODE, K>, 32 * K,
                                                sizeof(PipeSmem<K, mode_planes<MODE>()>));
  // one wave: as many CTAs as fit on the device at once, split into row segments
  const int64_t resident = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  int64_t nseg = resident / nstrips;
  if (nseg < 1) nseg = 1;
  int64_t rows = (g.ny + nseg - 1) / nseg;
  if (rows < 4 * K) rows = 4 * K;
  if (rows > (1 << 30)) rows = 1 << 30;
  return (int)rows;
}

template <int MODE>
cudaError_t launch_blocked_mode(const GridView& g, const void* coeffs, const void* in, void* out,
                                int depth, int seg_rows, cudaStream_t s) {
  switch (depth) {
    case 2: return launch_blocked_t<MODE, 2>(g, coeffs, in, out, seg_rows, s);
    case 3: return launch_blocked_t<MODE, 3>(g, coeffs, in, out, seg_rows, s);
    case 4: return launch_blocked_t<MODE, 4>(g, coeffs, in, out, seg_rows, s);
    case 5: return launch_blocked_t<MODE, 5>(g, coeffs, in, out, seg_rows, s);
    case 6: return launch_blocked_t<MODE, 6>(g, coeffs, in, out, seg_rows, s);
    case 7: return launch_blocked_t<MODE, 7>(g, coeffs, in, out, seg_rows, s);
    case 8: return launch_blocked_t<MODE, 8>(g, coeffs, in, out, seg_rows, s);
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

int blocked_default_seg_rows(int precision, const GridView& g, int depth) {
  if (precision == SSLBM_FP32) return default_seg_rows_mode<MODE_PLAIN>(g, depth);
  if (precision == SSLBM_FP32_DEV) return default_seg_rows_mode<MODE_DEV>(g, depth);
  if (precision == SSLBM_FP32_SPLIT) return default_seg_rows_mode<MODE_SPLIT>(g, depth);
  return 0;
}

bool blocked_supported(int precision, const GridView&) {
  return precision == SSLBM_FP32 || precision == SSLBM_FP32_DEV || precision == SSLBM_FP32_SPLIT;
}

cudaError_t launch_sslbm_step1(int precision, const GridView& g, const void* coeffs, const void* in,
                               void* out, cudaStream_t s) {
  switch (precision) {
    case SSLBM_FP64: return launch_step1_t<double, 2, MODE_PLAIN>(g, coeffs, in, out, s);
    case SSLBM_FP32: return launch_step1_t<float, 4, MODE_PLAIN>(g, coeffs, in, out, s);
    case SSLBM_FP32_DEV: return launch_step1_t<float, 4, MODE_DEV>(g, coeffs, in, out, s);
    case SSLBM_FP32_SPLIT: return launch_step1_t<float, 4, MODE_SPLIT>(g, coeffs, in, out, s);
    case SSLBM_FP32_KAHAN: return launch_kahan_stream(g, coeffs, in, out, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sslbm_blocked(int precision, const GridView& g, const void* coeffs,
                                 const void* in, void* out, int depth, int seg_rows,
                                 cudaStream_t s) {
  if (precision == SSLBM_FP32)
    return launch_blocked_mode<MODE_PLAIN>(g, coeffs, in, out, depth, seg_rows, s);
  if (precision == SSLBM_FP32_DEV)
    return launch_blocked_mode<MODE_DEV>(g, coeffs, in, out, depth, seg_rows, s);
  if (precision == SSLBM_FP32_SPLIT)
    return launch_blocked_mode<MODE_SPLIT>(g, coeffs, in, out, depth, seg_rows, s);
  return cudaErrorInvalidValue;
}

}  // namespace sslbm
