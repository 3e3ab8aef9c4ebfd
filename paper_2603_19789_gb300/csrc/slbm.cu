// slbm.cu -- the two-pass simplified LBM (SLBM) of Sec. II.C, Eqs. (SLBM1, SLBM2), on D2Q5:
//   predictor  rho*(x) = sum_i w_i rho(x - c_i, t)              = rho + lap5(rho) / 6
//   corrector  rho(x, t+dt) = rho*(x) + (tau - 1)(sum_i w_i rho*(x + c_i) - rho(x, t)) + Psi dt
//                          = rho* + (tau - 1)(rho* + lap5(rho*) / 6 - rho) + Psi dt
// for C in {S, E, I, R}; D takes the explicit update of Eq. (rhoD).  Two kernels per step:
// the predictor writes rho* of the four mobile compartments to a scratch of four planes, the
// corrector reads it with the stencil.  This is the double pass the single-step SSLBM
// removes; it is kept for the comparison.  Boundaries as for the SSLBM (periodic wrap or
// the cell-centred mirror, one link).
#include <cuda_runtime.h>

#include "variants.cuh"

namespace sslbm {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) slbm_predict_kernel(const GridView g, const T* __restrict__ in,
                                                           T* __restrict__ pred) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int64_t xl = link_index(x - 1, g.nx, g.bc), xr = link_index(x + 1, g.nx, g.bc);
  const T sixth = T(1) / T(6);
  for (int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; y < g.ny; y += (int64_t)gridDim.y * blockDim.y) {
    const int64_t r = y * g.pitch, ru = link_index(y - 1, g.ny, g.bc) * g.pitch,
                  rd = link_index(y + 1, g.ny, g.bc) * g.pitch;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T* p = in + c * g.plane;
      const T v = p[r + x];
      pred[c * g.plane + r + x] = fma_rn(lap5(v, p[r + xl], p[r + xr], p[ru + x], p[rd + x]), sixth, v);
    }
  }
}

template <typename T>
struct Tm1 {
  T v[4];  // tau - 1 per mobile compartment
};

template <typename T>
__global__ void __launch_bounds__(256) slbm_correct_kernel(const GridView g, const Coeffs<T> k, const Tm1<T> tm1,
                                                           const T* __restrict__ in, const T* __restrict__ pred,
                                                           T* __restrict__ out) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int64_t xl = link_index(x - 1, g.nx, g.bc), xr = link_index(x + 1, g.nx, g.bc);
  const T sixth = T(1) / T(6);
  for (int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; y < g.ny; y += (int64_t)gridDim.y * blockDim.y) {
    const int64_t r = y * g.pitch, ru = link_index(y - 1, g.ny, g.bc) * g.pitch,
                  rd = link_index(y + 1, g.ny, g.bc) * g.pitch;
    const int64_t o = r + x;
    const T S = in[o], E = in[g.plane + o], I = in[2 * g.plane + o], R = in[3 * g.plane + o];
    const T F = force_dt(k, S, E, I, R);
    T src[4];
    src[0] = -F;
    src[1] = fma_rn(-k.adt, E, F);
    src[2] = fma_rn(k.adt, E, -mul_rn(k.gdt, I));
    src[3] = mul_rn(k.rdt, I);
    const T rho[4] = {S, E, I, R};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T* q = pred + c * g.plane;
      const T ps = q[o];
      const T s = fma_rn(lap5(ps, q[r + xl], q[r + xr], q[ru + x], q[rd + x]), sixth, ps);
      out[c * g.plane + o] = add_rn(fma_rn(tm1.v[c], sub_rn(s, rho[c]), ps), src[c]);
    }
    out[4 * g.plane + o] = fma_rn(k.ddt, I, in[4 * g.plane + o]);
  }
}

template <typename T>
cudaError_t launch_t(const GridView& g, const void* coeffs, const double tm1d[4], const void* in, void* pred,
                     void* out, cudaStream_t s) {
  Tm1<T> tm1;
  for (int c = 0; c < 4; ++c) tm1.v[c] = (T)tm1d[c];
  dim3 block(32, 8);
  dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)std::min<int64_t>(65535, (g.ny + 7) / 8));
  slbm_predict_kernel<T><<<grid, block, 0, s>>>(g, static_cast<const T*>(in), static_cast<T*>(pred));
  slbm_correct_kernel<T><<<grid, block, 0, s>>>(g, *static_cast<const Coeffs<T>*>(coeffs), tm1, static_cast<const T*>(in),
                                                static_cast<const T*>(pred), static_cast<T*>(out));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_slbm_step(int precision, const GridView& g, const void* coeffs, const double tm1[4],
                             const void* in, void* pred, void* out, cudaStream_t s) {
  switch (precision) {
    case SSLBM_FP64: return launch_t<double>(g, coeffs, tm1, in, pred, out, s);
    case SSLBM_FP32: return launch_t<float>(g, coeffs, tm1, in, pred, out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sslbm
