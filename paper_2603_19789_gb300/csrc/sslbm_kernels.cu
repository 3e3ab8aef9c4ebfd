// sslbm_kernels.cu -- SSLBM time-step kernels (Sec. II.C, Eq. sslbm_final_clean with the
// sources of Eq. sources and the deceased update of Eq. rhoD).
//
//   step1_kernel    one FP64 step per launch: each thread updates two consecutive cells of a
//                   row with 16-byte vector loads (double2) of the centre, upper and lower rows
//                   and two scalar edge loads; neighbouring rows come from L1/L2.  The FP32
//                   storages advance one step per launch in the streaming kernel (stream.cu).
//   pipe_kernel     (pipe_launch.cuh) K steps per launch (temporal blocking, K = 2..8) for
//                   FP32, FP32 deviation-S and FP32 split-S (a sixth plane); pipe_d2q9*.cu and
//                   pipe_vard.cu instantiate it for FP32 on the D2Q9 lattice (periodic, or no-flux with the
//                   bounce-back substituted into the row update) and on the varying-diffusion
//                   lattice (the scale rows in a static shared-memory ring), as a pipeline of
//                   K warps per
//                   CTA: warp s computes level s+1 of the time-step wavefront.  A CTA owns a
//                   128-column strip (4 columns per lane, 16-byte accesses) with a K-column halo
//                   on each side and streams down a segment of rows, two rows per step of the
//                   pipeline.  Warp 0 brings level-0 rows in with cp.async into a shared-memory
//                   ring three row pairs ahead; every level's output pair goes through a
//                   double-buffered shared-memory slot (dynamic shared memory) to the next
//                   warp, one CTA barrier per pair; the last warp writes level K to global
//                   memory.  Each warp keeps only its own level's rows in four register
//                   buffers (about 110 registers per thread), so two or more CTAs share an SM.
//                   x neighbours come from warp shuffles.  Rows and columns outside the domain
//                   are loaded as ghost images (periodic wrap or the even mirror extension),
//                   which the uniform stencil keeps consistent, so no boundary logic is needed
//                   inside the pipeline.  DRAM traffic is one read and one write of the five
//                   planes per K steps.
// The pipeline and the streaming kernel evaluate the same packed per-cell expressions
// (sslbm_internal.cuh), so a blocked launch gives the same bits as K one-step launches.
#include <atomic>

#include "bounds.cuh"
#include "sslbm_internal.cuh"
#include "pipe_launch.cuh"

SSLBM_OOB_ACCESSOR(kernels)

namespace sslbm {

namespace {

// One FP64 step: each thread updates two consecutive cells of a row.
__global__ void __launch_bounds__(256, 1) step1_kernel(const GridView g, const Coeffs<double> k,
                                                    const double* __restrict__ in, double* __restrict__ out) {
  constexpr int V = 2;
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
    double c[4][V], lap[4][V];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const double* P = in + f * g.plane;
      const double2 cv = *reinterpret_cast<const double2*>(P + rc + x0);
      const double2 uv = *reinterpret_cast<const double2*>(P + ru + x0);
      const double2 dv = *reinterpret_cast<const double2*>(P + rd + x0);
      c[f][0] = cv.x, c[f][1] = cv.y;
      const double u[V] = {uv.x, uv.y}, d[V] = {dv.x, dv.y};
      const double L = P[rc + xl];
      const double R = P[rc + xr];
      // the right neighbour of the first cell is the second cell unless the row ends there
      lap[f][0] = lap5(c[f][0], L, nvalid > 1 ? c[f][1] : R, u[0], d[0]);
      lap[f][1] = lap5(c[f][1], c[f][0], R, u[1], d[1]);
    }
    const double2 Dv = *reinterpret_cast<const double2*>(in + 4 * g.plane + rc + x0);
    const double D[V] = {Dv.x, Dv.y};
    double n[5][V];
#pragma unroll
    for (int j = 0; j < V; ++j)
      seird_cell(k, c[0][j], c[1][j], c[2][j], c[3][j], D[j], lap[0][j], lap[1][j], lap[2][j], lap[3][j], n[0][j],
                 n[1][j], n[2][j], n[3][j], n[4][j]);
    if (nvalid == V) {
#pragma unroll
      for (int f = 0; f < 5; ++f)
        *reinterpret_cast<double2*>(out + f * g.plane + rc + x0) = make_double2(n[f][0], n[f][1]);
    } else {
#pragma unroll
      for (int f = 0; f < 5; ++f) out[f * g.plane + rc + x0] = n[f][0];
    }
  }
}

cudaError_t launch_step1_fp64(const GridView& g, const void* coeffs, const void* in, void* out, cudaStream_t s) {
  const int64_t nvec = (g.nx + 1) / 2;
  dim3 block(32, 8);
  int64_t gy = (g.ny + 7) / 8;
  if (gy > 65535) gy = 65535;
  dim3 grid((unsigned)((nvec + 31) / 32), (unsigned)gy);
  step1_kernel<<<grid, block, 0, s>>>(g, *static_cast<const Coeffs<double>*>(coeffs),
                                      static_cast<const double*>(in), static_cast<double*>(out));
  return cudaGetLastError();
}

}  // namespace

int blocked_default_seg_rows(int precision, const GridView& g, int depth) {
  if (precision == SSLBM_FP32) return default_seg_rows_mode<MODE_PLAIN>(g, depth);
  if (precision == SSLBM_FP32_DEV) return default_seg_rows_mode<MODE_DEV>(g, depth);
  if (precision == SSLBM_FP32_SPLIT) return default_seg_rows_mode<MODE_SPLIT>(g, depth);
  if (precision == SSLBM_FP32_KAHAN) return blocked_kahan_default_seg_rows(g, depth);
  return 0;
}

bool blocked_supported(int precision, const GridView&) {
  return precision == SSLBM_FP32 || precision == SSLBM_FP32_DEV || precision == SSLBM_FP32_SPLIT ||
         precision == SSLBM_FP32_KAHAN;
}

cudaError_t launch_sslbm_step1(int precision, const GridView& g, const void* coeffs, const void* in,
                               void* out, cudaStream_t s) {
  switch (precision) {
    case SSLBM_FP64: return launch_step1_fp64(g, coeffs, in, out, s);
    case SSLBM_FP32:
    case SSLBM_FP32_DEV:
    case SSLBM_FP32_SPLIT:
    case SSLBM_FP32_KAHAN: return launch_stream_d2q5(precision, g, coeffs, in, out, s);
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
  if (precision == SSLBM_FP32_KAHAN) return launch_kahan_blocked(g, coeffs, in, out, depth, seg_rows, s);
  return cudaErrorInvalidValue;
}

}  // namespace sslbm
