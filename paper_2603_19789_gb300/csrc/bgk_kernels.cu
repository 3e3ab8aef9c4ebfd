// bgk_kernels.cu -- the BGK lattice Boltzmann comparison scheme (Sec. II.B, Eq. pdf) on the
// D2Q5 lattice: one population set f_i^C (i = 0..4) per mobile compartment C in {S,E,I,R},
// plus the deceased density D, which does not diffuse and is advanced by Eq. (rhoD).
//
// Storage: 21 planes per state buffer -- plane c*5 + i holds f_i of compartment c, plane 20
// holds D -- in the pitched layout of sslbm_internal.cuh.  The buffer always holds the
// pre-collision populations at an integer time, so a state read back is directly
// comparable to the scheme as written in the paper.
//
// One kernel performs a full step: each thread loads the 20 populations and D of its
// cell, forms rho^C = sum_i f_i^C and the sources of Eq. (sources), relaxes every
// population towards w_i rho^C with rate 1/tau^C, adds w_i Psi^C dt, and pushes the result
// along its link c_i into the other buffer (coalesced: neighbouring threads write
// neighbouring addresses).  A population that would leave through a no-flux wall is
// written back into the opposite direction at the same cell (halfway bounce-back);
// with periodic boundaries it wraps.
#include "bounds.cuh"
#include "sslbm_internal.cuh"

SSLBM_OOB_ACCESSOR(bgk)

namespace sslbm {

namespace {

__constant__ int kCx[5] = {0, 1, 0, -1, 0};
__constant__ int kCy[5] = {0, 0, 1, 0, -1};
__constant__ int kOpp[5] = {0, 3, 4, 1, 2};

template <typename T>
__device__ __forceinline__ T weight(int i) {
  return i == 0 ? T(1) / T(3) : T(1) / T(6);
}

template <typename T>
__global__ void __launch_bounds__(256) bgk_step_kernel(const GridView g, const Coeffs<T> k,
                                                       const T* __restrict__ fin,
                                                       T* __restrict__ fout) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  for (int64_t y = blockIdx.y; y < g.ny; y += gridDim.y) {
    const int64_t idx = y * g.pitch + x;
    T f[4][5];
    T rho[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int i = 0; i < 5; ++i) f[c][i] = fin[(c * 5 + i) * g.plane + idx];
      rho[c] = add_rn(add_rn(add_rn(add_rn(f[c][0], f[c][1]), f[c][2]), f[c][3]), f[c][4]);
    }
    const T Dv = fin[20 * g.plane + idx];
    const T F = force_dt(k, rho[0], rho[1], rho[2], rho[3]);
    T psi[4];
    psi[0] = -F;
    psi[1] = fma_rn(-k.adt, rho[1], F);
    psi[2] = fma_rn(k.adt, rho[1], -mul_rn(k.gdt, rho[2]));
    psi[3] = mul_rn(k.rdt, rho[2]);
    fout[20 * g.plane + idx] = fma_rn(k.ddt, rho[2], Dv);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const T w = weight<T>(i);
      int64_t tx = x + kCx[i], ty = y + kCy[i];
      bool inside = tx >= 0 && tx < g.nx && ty >= 0 && ty < g.ny;
      int dir = i;
      int64_t tidx;
      if (inside) {
        tidx = ty * g.pitch + tx;
      } else if (g.bc == 0) {
        tx = tx < 0 ? tx + g.nx : (tx >= g.nx ? tx - g.nx : tx);
        ty = ty < 0 ? ty + g.ny : (ty >= g.ny ? ty - g.ny : ty);
        tidx = ty * g.pitch + tx;
      } else {
        tidx = idx;
        dir = kOpp[i];
        tx = x;
        ty = y;
      }
      if (!(SSLBM_IN(tx, 1, g.nx, 20) && SSLBM_IN(ty, 1, g.ny, 21))) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        // f + (w rho - f)/tau + w Psi dt
        const T relax = mul_rn(fma_rn(w, rho[c], -f[c][i]), k.itau[c]);
        const T post = fma_rn(w, psi[c], add_rn(f[c][i], relax));
        fout[(c * 5 + dir) * g.plane + tidx] = post;
      }
    }
  }
}

// Equilibrium initialisation f_i = w_i rho of one compartment (c < 4), or a copy of D (c = 4),
// from a contiguous ny x nx source of type U.
template <typename T, typename U>
__global__ void bgk_init_kernel(const GridView g, int c, const U* __restrict__ rho,
                                T* __restrict__ f) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  for (int64_t y = blockIdx.y; y < g.ny; y += gridDim.y) {
    const T r = (T)rho[y * g.nx + x];
    const int64_t idx = y * g.pitch + x;
    if (c == 4) {
      f[20 * g.plane + idx] = r;
    } else {
#pragma unroll
      for (int i = 0; i < 5; ++i) f[(c * 5 + i) * g.plane + idx] = weight<T>(i) * r;
    }
  }
}

// rho^C = sum_i f_i^C (or D) into a contiguous ny x nx destination of type U.
template <typename T, typename U>
__global__ void bgk_density_kernel(const GridView g, int c, const T* __restrict__ f,
                                   U* __restrict__ rho) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  for (int64_t y = blockIdx.y; y < g.ny; y += gridDim.y) {
    const int64_t idx = y * g.pitch + x;
    T r;
    if (c == 4) {
      r = f[20 * g.plane + idx];
    } else {
      r = f[(c * 5) * g.plane + idx];
#pragma unroll
      for (int i = 1; i < 5; ++i) r = add_rn(r, f[(c * 5 + i) * g.plane + idx]);
    }
    rho[y * g.nx + x] = (U)r;
  }
}

dim3 row_grid(const GridView& g, int threads) {
  int64_t gy = g.ny < 65535 ? g.ny : 65535;
  return dim3((unsigned)((g.nx + threads - 1) / threads), (unsigned)gy);
}

}  // namespace

cudaError_t launch_bgk_step(int precision, const GridView& g, const void* coeffs, const void* f_in,
                            void* f_out, cudaStream_t s) {
  if (precision == SSLBM_FP64) {
    bgk_step_kernel<double><<<row_grid(g, 128), 128, 0, s>>>(
        g, *static_cast<const Coeffs<double>*>(coeffs), static_cast<const double*>(f_in),
        static_cast<double*>(f_out));
  } else if (precision == SSLBM_FP32) {
    bgk_step_kernel<float><<<row_grid(g, 128), 128, 0, s>>>(
        g, *static_cast<const Coeffs<float>*>(coeffs), static_cast<const float*>(f_in),
        static_cast<float*>(f_out));
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_bgk_init(int precision, const GridView& g, int comp, const void* rho,
                            int rho_dtype, void* f, cudaStream_t s) {
  const dim3 grid = row_grid(g, 128);
  if (precision == SSLBM_FP64 && rho_dtype == SSLBM_DT_F64)
    bgk_init_kernel<double, double><<<grid, 128, 0, s>>>(g, comp, (const double*)rho, (double*)f);
  else if (precision == SSLBM_FP64 && rho_dtype == SSLBM_DT_F32)
    bgk_init_kernel<double, float><<<grid, 128, 0, s>>>(g, comp, (const float*)rho, (double*)f);
  else if (precision == SSLBM_FP32 && rho_dtype == SSLBM_DT_F64)
    bgk_init_kernel<float, double><<<grid, 128, 0, s>>>(g, comp, (const double*)rho, (float*)f);
  else if (precision == SSLBM_FP32 && rho_dtype == SSLBM_DT_F32)
    bgk_init_kernel<float, float><<<grid, 128, 0, s>>>(g, comp, (const float*)rho, (float*)f);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_bgk_density(int precision, const GridView& g, int comp, const void* f, void* rho,
                               int rho_dtype, cudaStream_t s) {
  const dim3 grid = row_grid(g, 128);
  if (precision == SSLBM_FP64 && rho_dtype == SSLBM_DT_F64)
    bgk_density_kernel<double, double><<<grid, 128, 0, s>>>(g, comp, (const double*)f, (double*)rho);
  else if (precision == SSLBM_FP64 && rho_dtype == SSLBM_DT_F32)
    bgk_density_kernel<double, float><<<grid, 128, 0, s>>>(g, comp, (const double*)f, (float*)rho);
  else if (precision == SSLBM_FP32 && rho_dtype == SSLBM_DT_F64)
    bgk_density_kernel<float, double><<<grid, 128, 0, s>>>(g, comp, (const float*)f, (double*)rho);
  else if (precision == SSLBM_FP32 && rho_dtype == SSLBM_DT_F32)
    bgk_density_kernel<float, float><<<grid, 128, 0, s>>>(g, comp, (const float*)f, (float*)rho);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace sslbm
