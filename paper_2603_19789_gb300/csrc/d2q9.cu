// d2q9.cu -- the SSLBM step on the D2Q9 lattice (Sec. II.C, isotropy discussion).
//
// Eq. (sslbm_final_clean) with rho_f = rho_b summed over the nine D2Q9 velocities (weights
// 4/9, 1/9 on the axes, 1/36 on the diagonals) reduces, like the D2Q5 form, to
//   rho_new = rho_c + (2 tau - 1)(rho_f - rho_c) + Psi dt
//           = rho_c + d_lattice (4 sum_axes rho + sum_diagonals rho - 20 rho_c) / 6 + Psi dt,
// the isotropic 9-point Laplacian, with d_lattice = (tau - 1/2)/3 as on D2Q5.  Boundaries:
// periodic wrap; no-flux as halfway bounce-back, where a link leaving the domain sees the
// cell's own value (on the axes this is the cell-centred mirror; on the diagonals it keeps
// the population exactly conserved).
//
// FP64: a CTA stages a 32 x 8 tile of S, E, I, R with a one-cell halo in shared memory
// (periodic: the wrapped neighbours; no-flux: the clamped ones, corrected per link at the
// walls), one cell per thread.  FP32 runs the same per-cell operations in the streaming
// one-step kernel (stream.cu).
#include <cuda_runtime.h>

#include "variants.cuh"

namespace sslbm {
namespace {

constexpr int kGX = 32, kGY = 8;  // the one-cell-per-thread tile kernel (FP64)

template <typename T>
__global__ void __launch_bounds__(kGX * kGY) d2q9_step_kernel(const GridView g, const Coeffs<T> k,
                                                              const T* __restrict__ in, T* __restrict__ out) {
  constexpr int SX = kGX + 2, SY = kGY + 2;
  __shared__ T tile[4][SY][SX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kGX + tx;
  const int64_t bx0 = (int64_t)blockIdx.x * kGX;
  const T sixth = T(1) / T(6);
  for (int64_t by0 = (int64_t)blockIdx.y * kGY; by0 < g.ny; by0 += (int64_t)gridDim.y * kGY) {
    __syncthreads();
    for (int i = tid; i < SX * SY; i += kGX * kGY) {
      const int sy = i / SX, sx = i - sy * SX;
      const int64_t gx = link_index(bx0 + sx - 1, g.nx, g.bc), gy = link_index(by0 + sy - 1, g.ny, g.bc);
      // tiles narrower than the halo (nx or ny = 1 with the wrap) still index inside the grid
      const int64_t cx = gx < 0 ? 0 : (gx >= g.nx ? g.nx - 1 : gx), cy = gy < 0 ? 0 : (gy >= g.ny ? g.ny - 1 : gy);
      const int64_t off = cy * g.pitch + cx;
#pragma unroll
      for (int c = 0; c < 4; ++c) tile[c][sy][sx] = in[c * g.plane + off];
    }
    __syncthreads();
    const int64_t x = bx0 + tx, y = by0 + ty;
    if (x >= g.nx || y >= g.ny) continue;
    const int cx = tx + 1, cy = ty + 1;
    // links that leave the domain under no-flux see the cell's own value
    const bool wl = g.bc != 0 && x == 0, wr = g.bc != 0 && x == g.nx - 1;
    const bool wd = g.bc != 0 && y == 0, wu = g.bc != 0 && y == g.ny - 1;
    T lap[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T ctr = tile[c][cy][cx];
      const T l = wl ? ctr : tile[c][cy][cx - 1], r = wr ? ctr : tile[c][cy][cx + 1];
      const T d = wd ? ctr : tile[c][cy - 1][cx], u = wu ? ctr : tile[c][cy + 1][cx];
      const T ne = (wr || wu) ? ctr : tile[c][cy + 1][cx + 1], nw = (wl || wu) ? ctr : tile[c][cy + 1][cx - 1];
      const T se = (wr || wd) ? ctr : tile[c][cy - 1][cx + 1], sw = (wl || wd) ? ctr : tile[c][cy - 1][cx - 1];
      const T axes = add_rn(add_rn(l, r), add_rn(u, d));
      const T diag = add_rn(add_rn(ne, nw), add_rn(se, sw));
      // (4 axes + diagonals - 20 c) / 6
      lap[c] = mul_rn(fma_rn(T(-20), ctr, fma_rn(T(4), axes, diag)), sixth);
    }
    const int64_t o = y * g.pitch + x;
    T n[5];
    seird_cell(k, tile[0][cy][cx], tile[1][cy][cx], tile[2][cy][cx], tile[3][cy][cx], in[4 * g.plane + o], lap[0],
               lap[1], lap[2], lap[3], n[0], n[1], n[2], n[3], n[4]);
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c * g.plane + o] = n[c];
  }
}

template <typename T>
cudaError_t launch_t(const GridView& g, const void* coeffs, const void* in, void* out, cudaStream_t s) {
  dim3 block(kGX, kGY);
  dim3 grid((unsigned)((g.nx + kGX - 1) / kGX), (unsigned)std::min<int64_t>(65535, (g.ny + kGY - 1) / kGY));
  d2q9_step_kernel<T><<<grid, block, 0, s>>>(g, *static_cast<const Coeffs<T>*>(coeffs), static_cast<const T*>(in),
                                             static_cast<T*>(out));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sslbm9_step1(int precision, const GridView& g, const void* coeffs, const void* in, void* out,
                                cudaStream_t s) {
  switch (precision) {
    case SSLBM_FP64: return launch_t<double>(g, coeffs, in, out, s);
    case SSLBM_FP32: return launch_stream_d2q9(g, coeffs, in, out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sslbm
