// vard.cu -- the SSLBM with spatially varying, axis-anisotropic diffusion, which Sec. IV lists
// as future work.  The paper gives no discretisation; this is the D2Q5 update in its link
// (flux) form,
//   rho_new = rho_c + sum_i D_i (rho(x + c_i) - rho_c) + Psi dt,
//   D_i = d_lattice^C (k_a(x) + k_a(x + c_i)) / 2,   a = x on the x links, y on the y links,
// with two per-cell scale planes kx, ky stored like the state planes.  Both cells of a link
// use the same coefficient, so the population is conserved exactly (Sec. II.C); uniform
// planes of 1 give Eq. (sslbm_final_clean).  Neighbours: the periodic wrap, or the cell
// itself, whose difference is zero (no flux through a wall).
//
// FP64: one step per launch, V = 2 cells of a row per thread: vector loads of the cell's row
// and of the rows above and below, two scalar loads for the columns left and right of the
// group.  FP32 runs the same per-cell operations in the streaming one-step kernel
// (stream.cu).  The four link coefficients of a cell are formed once and
// serve all four mobile compartments; each flux term is rounded on its own and the sum pairs
// the two x links and the two y links, ((+x) + (-x)) + ((+y) + (-y)), an order that a mirror
// image leaves unchanged (so the no-flux boundary is exactly a ghost image, which the
// temporal-blocked kernel relies on).
#include <cuda_runtime.h>
#include <float.h>

#include "variants.cuh"

namespace sslbm {
namespace {

template <typename T, int V>
struct VRow;
template <>
struct VRow<double, 2> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x, v[1] = t.y;
  }
  static __device__ __forceinline__ void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

template <typename T, int V>
__global__ void __launch_bounds__(256) vard_step_kernel(const GridView g, const Coeffs<T> k, const T* __restrict__ kx,
                                                        const T* __restrict__ ky, const T* __restrict__ in,
                                                        T* __restrict__ out) {
  const int64_t nvec = (g.nx + V - 1) / V;
  const int64_t vx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vx >= nvec) return;
  const int64_t x0 = vx * V;
  const int nvalid = (int)((g.nx - x0) < V ? (g.nx - x0) : V);
  const int64_t xl = link_index(x0 - 1, g.nx, g.bc), xr = link_index(x0 + nvalid, g.nx, g.bc);
  const T half = T(0.5);
  for (int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; y < g.ny; y += (int64_t)gridDim.y * blockDim.y) {
    const int64_t rc = y * g.pitch, rm = link_index(y - 1, g.ny, g.bc) * g.pitch,
                  rp = link_index(y + 1, g.ny, g.bc) * g.pitch;
    // link coefficients (without d_lattice) of the V cells: +x, +y, -x, -y
    T lxp[V], lyp[V], lxm[V], lym[V];
    {
      T a[V], b[V], bm[V], bp[V];
      VRow<T, V>::load(kx + rc + x0, a);
      VRow<T, V>::load(ky + rc + x0, b);
      VRow<T, V>::load(ky + rm + x0, bm);
      VRow<T, V>::load(ky + rp + x0, bp);
      const T aL = kx[rc + xl], aR = kx[rc + xr];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const T left = j == 0 ? aL : a[j > 0 ? j - 1 : 0];
        const T right = j + 1 < nvalid ? a[j + 1 < V ? j + 1 : j] : aR;
        lxp[j] = mul_rn(half, add_rn(a[j], right));
        lyp[j] = mul_rn(half, add_rn(b[j], bp[j]));
        lxm[j] = mul_rn(half, add_rn(a[j], left));
        lym[j] = mul_rn(half, add_rn(b[j], bm[j]));
      }
    }
    T ctr[4][V], flux[4][V];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T* P = in + c * g.plane;
      T m[V], p[V];
      VRow<T, V>::load(P + rc + x0, ctr[c]);
      VRow<T, V>::load(P + rm + x0, m);
      VRow<T, V>::load(P + rp + x0, p);
      const T L = P[rc + xl], R = P[rc + xr];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const T cc = ctr[c][j];
        const T left = j == 0 ? L : ctr[c][j > 0 ? j - 1 : 0];
        const T right = j + 1 < nvalid ? ctr[c][j + 1 < V ? j + 1 : j] : R;
        const T t1 = mul_rn(lxp[j], sub_rn(right, cc));
        const T t2 = mul_rn(lyp[j], sub_rn(p[j], cc));
        const T t3 = mul_rn(lxm[j], sub_rn(left, cc));
        const T t4 = mul_rn(lym[j], sub_rn(m[j], cc));
        flux[c][j] = add_rn(add_rn(t1, t3), add_rn(t2, t4));
      }
    }
    T D[V];
    VRow<T, V>::load(in + 4 * g.plane + rc + x0, D);
    T n[5][V];
#pragma unroll
    for (int j = 0; j < V; ++j)
      seird_cell(k, ctr[0][j], ctr[1][j], ctr[2][j], ctr[3][j], D[j], flux[0][j], flux[1][j], flux[2][j], flux[3][j],
                 n[0][j], n[1][j], n[2][j], n[3][j], n[4][j]);
    if (nvalid == V) {
#pragma unroll
      for (int c = 0; c < 5; ++c) VRow<T, V>::store(out + c * g.plane + rc + x0, n[c]);
    } else {
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int j = 0; j < V; ++j)
          if (j < nvalid) out[c * g.plane + rc + x0 + j] = n[c][j];
    }
  }
}

// Block-wide max of a and sum of b, in thread 0.
__device__ void block_max_sum(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, off));
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  if (lane == 0) sa[warp] = a, sb[warp] = b;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      a = fmax(a, __shfl_down_sync(0xffffffffu, a, off));
      b += __shfl_down_sync(0xffffffffu, b, off);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) vard_check_kernel(const GridView g, const T* __restrict__ kx,
                                                         const T* __restrict__ ky, double* __restrict__ partials) {
  double smax = 0.0, bad = 0.0;
  const bool wall = g.bc != 0;
  for (int64_t y = blockIdx.x; y < g.ny; y += gridDim.x) {
    for (int64_t x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const double a = (double)kx[y * g.pitch + x], b = (double)ky[y * g.pitch + x];
      if (!(a >= 0.0) || !(b >= 0.0) || a > DBL_MAX || b > DBL_MAX) {
        bad += 1.0;
        continue;
      }
      double s = 0.0;
      if (!(wall && x + 1 >= g.nx)) s += 0.5 * (a + (double)kx[y * g.pitch + link_index(x + 1, g.nx, g.bc)]);
      if (!(wall && y + 1 >= g.ny)) s += 0.5 * (b + (double)ky[link_index(y + 1, g.ny, g.bc) * g.pitch + x]);
      if (!(wall && x == 0)) s += 0.5 * (a + (double)kx[y * g.pitch + link_index(x - 1, g.nx, g.bc)]);
      if (!(wall && y == 0)) s += 0.5 * (b + (double)ky[link_index(y - 1, g.ny, g.bc) * g.pitch + x]);
      smax = fmax(smax, s);
    }
  }
  block_max_sum(smax, bad);
  if (threadIdx.x == 0) partials[2 * blockIdx.x] = smax, partials[2 * blockIdx.x + 1] = bad;
}

__global__ void __launch_bounds__(256) vard_check_final_kernel(const double* __restrict__ partials, int nblocks,
                                                               double* __restrict__ result) {
  double smax = 0.0, bad = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    smax = fmax(smax, partials[2 * i]);
    bad += partials[2 * i + 1];
  }
  block_max_sum(smax, bad);
  if (threadIdx.x == 0) result[0] = smax, result[1] = bad;
}

template <typename T, int V>
cudaError_t launch_t(const GridView& g, const void* coeffs, const void* kx, const void* ky, const void* in, void* out,
                     cudaStream_t s) {
  const int64_t nvec = (g.nx + V - 1) / V;
  dim3 block(32, 8);
  dim3 grid((unsigned)((nvec + 31) / 32), (unsigned)std::min<int64_t>(65535, (g.ny + 7) / 8));
  vard_step_kernel<T, V><<<grid, block, 0, s>>>(g, *static_cast<const Coeffs<T>*>(coeffs), static_cast<const T*>(kx),
                                                static_cast<const T*>(ky), static_cast<const T*>(in),
                                                static_cast<T*>(out));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sslbm_vard_step(int precision, const GridView& g, const void* coeffs, const void* kx,
                                   const void* ky, const void* in, void* out, cudaStream_t s) {
  switch (precision) {
    case SSLBM_FP64: return launch_t<double, 2>(g, coeffs, kx, ky, in, out, s);
    case SSLBM_FP32: return launch_stream_vard(g, coeffs, kx, ky, in, out, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_vard_check(int precision, const GridView& g, const void* kx, const void* ky, double* partials,
                              double* result, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<int64_t>(g.ny, kDiagBlocks);
  if (precision == SSLBM_FP64)
    vard_check_kernel<double><<<blocks, 256, 0, s>>>(g, static_cast<const double*>(kx), static_cast<const double*>(ky),
                                                     partials);
  else if (precision == SSLBM_FP32)
    vard_check_kernel<float><<<blocks, 256, 0, s>>>(g, static_cast<const float*>(kx), static_cast<const float*>(ky),
                                                    partials);
  else
    return cudaErrorInvalidValue;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vard_check_final_kernel<<<1, 256, 0, s>>>(partials, (int)blocks, result);
  return cudaGetLastError();
}

}  // namespace sslbm
