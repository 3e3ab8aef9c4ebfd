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
// A CTA stages a 32 x 8 tile of S, E, I, R with a one-cell halo in shared memory (periodic:
// the wrapped neighbours; no-flux: the clamped ones, corrected per link at the walls).
#include <cuda_runtime.h>

#include "variants.cuh"

namespace sslbm {
namespace {

constexpr int kTX = 32, kTY = 8;  // threads per CTA (x, y); each thread computes 4 cells of a row
constexpr int kTW = 4 * kTX;        // tile width in cells
constexpr int kSW = kTW + 8;        // shared row: 4 padding columns each side, the halo at 3 and kTW + 4

// The D2Q9 step for FP32: a CTA stages S, E, I, R of a 128 x 8 tile with a one-cell halo in
// shared memory -- interior rows as aligned float4 vectors, halo rows through link_index,
// the halo columns (and, for a tile narrower than 128 cells, the column after the last cell)
// through link_index -- and each thread evaluates 4 consecutive cells of one row.
__global__ void __launch_bounds__(kTX * kTY) d2q9_step_f32_kernel(const GridView g, const Coeffs<float> k,
                                                                  const float* __restrict__ in,
                                                                  float* __restrict__ out) {
  __shared__ __align__(16) float tile[4][kTY + 2][kSW];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
  const int64_t bx0 = (int64_t)blockIdx.x * kTW;
  const int64_t nvalid_x = g.nx - bx0 < kTW ? g.nx - bx0 : kTW;  // cells of this tile along x
  const float sixth = 1.f / 6.f;
  for (int64_t by0 = (int64_t)blockIdx.y * kTY; by0 < g.ny; by0 += (int64_t)gridDim.y * kTY) {
    __syncthreads();  // the previous tile's readers are done
    // interior columns: (kTY + 2) rows x kTX float4 groups per plane
    for (int i = tid; i < (kTY + 2) * kTX; i += kTX * kTY) {
      const int r = i / kTX, q = i - r * kTX;
      const int64_t x = bx0 + 4 * q;
      if (x >= g.pitch) continue;  // a group wholly past the padded row is never read
      const int64_t gy = link_index(by0 - 1 + r, g.ny, g.bc);
      const int64_t gyc = gy < 0 ? 0 : (gy >= g.ny ? g.ny - 1 : gy);  // rows narrower than the halo
#pragma unroll
      for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4*>(&tile[c][r][4 + 4 * q]) =
            *reinterpret_cast<const float4*>(in + c * g.plane + gyc * g.pitch + x);
    }
    __syncthreads();  // the vector loads may cover the column after the last cell: overwrite after them
    // the left halo column, and the column right after the tile's last cell
    for (int i = tid; i < 2 * (kTY + 2); i += kTX * kTY) {
      const int r = i >> 1, side = i & 1;
      const int64_t gy = link_index(by0 - 1 + r, g.ny, g.bc);
      const int64_t gyc = gy < 0 ? 0 : (gy >= g.ny ? g.ny - 1 : gy);
      const int64_t gx = link_index(side ? bx0 + nvalid_x : bx0 - 1, g.nx, g.bc);
      const int64_t gxc = gx < 0 ? 0 : (gx >= g.nx ? g.nx - 1 : gx);
      const int col = side ? 4 + (int)nvalid_x : 3;
#pragma unroll
      for (int c = 0; c < 4; ++c) tile[c][r][col] = in[c * g.plane + gyc * g.pitch + gxc];
    }
    __syncthreads();
    const int64_t y = by0 + ty;
    const int64_t x0 = bx0 + 4 * tx;
    if (y >= g.ny || x0 >= g.nx) continue;
    const bool wd = g.bc != 0 && y == 0, wu = g.bc != 0 && y == g.ny - 1;
    float lap[4][4], ctr[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[3][6];  // rows y-1, y, y+1; columns x0-1 .. x0+4
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float* row = &tile[c][ty + r][4 + 4 * tx];
        const float4 m = *reinterpret_cast<const float4*>(row);
        v[r][0] = row[-1], v[r][1] = m.x, v[r][2] = m.y, v[r][3] = m.z, v[r][4] = m.w, v[r][5] = row[4];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t x = x0 + j;
        // links that leave the domain under no-flux see the cell's own value
        const bool wl = g.bc != 0 && x == 0, wr = g.bc != 0 && x == g.nx - 1;
        const float cc = v[1][j + 1];
        const float l = wl ? cc : v[1][j], r = wr ? cc : v[1][j + 2];
        const float d = wd ? cc : v[0][j + 1], u = wu ? cc : v[2][j + 1];
        const float ne = (wr || wu) ? cc : v[2][j + 2], nw = (wl || wu) ? cc : v[2][j];
        const float se = (wr || wd) ? cc : v[0][j + 2], sw = (wl || wd) ? cc : v[0][j];
        const float axes = add_rn(add_rn(l, r), add_rn(u, d));
        const float diag = add_rn(add_rn(ne, nw), add_rn(se, sw));
        // (4 axes + diagonals - 20 c) / 6
        lap[c][j] = mul_rn(fma_rn(-20.f, cc, fma_rn(4.f, axes, diag)), sixth);
        ctr[c][j] = cc;
      }
    }
    const int64_t o = y * g.pitch + x0;
    const float4 D4 = *reinterpret_cast<const float4*>(in + 4 * g.plane + o);
    const float Dv[4] = {D4.x, D4.y, D4.z, D4.w};
    float n[5][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      seird_cell(k, ctr[0][j], ctr[1][j], ctr[2][j], ctr[3][j], Dv[j], lap[0][j], lap[1][j], lap[2][j], lap[3][j],
                 n[0][j], n[1][j], n[2][j], n[3][j], n[4][j]);
    if (x0 + 3 < g.nx) {
#pragma unroll
      for (int c = 0; c < 5; ++c)
        *reinterpret_cast<float4*>(out + c * g.plane + o) = make_float4(n[c][0], n[c][1], n[c][2], n[c][3]);
    } else {
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (x0 + j < g.nx) out[c * g.plane + o + j] = n[c][j];
    }
  }
}

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
    case SSLBM_FP32: {
      dim3 block(kTX, kTY);
      dim3 grid((unsigned)((g.nx + kTW - 1) / kTW), (unsigned)std::min<int64_t>(65535, (g.ny + kTY - 1) / kTY));
      d2q9_step_f32_kernel<<<grid, block, 0, s>>>(g, *static_cast<const Coeffs<float>*>(coeffs),
                                                  static_cast<const float*>(in), static_cast<float*>(out));
      return cudaGetLastError();
    }
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sslbm
