// slbm.cu -- the two-pass simplified LBM (SLBM) of Sec. II.C, Eqs. (SLBM1, SLBM2), on D2Q5:
//   predictor  rho*(x) = sum_i w_i rho(x - c_i, t)              = rho + lap5(rho) / 6
//   corrector  rho(x, t+dt) = rho*(x) + (tau - 1)(sum_i w_i rho*(x + c_i) - rho(x, t)) + Psi dt
//                          = rho* + (tau - 1)(rho* + lap5(rho*) / 6 - rho) + Psi dt
// for C in {S, E, I, R}; D takes the explicit update of Eq. (rhoD).  Two kernels per step:
// the predictor writes rho* of the four mobile compartments to a scratch of four planes, the
// corrector reads it with the stencil.  Each thread handles V cells of a row (4 in FP32, 2 in
// FP64) with vector loads of its row and of the rows above and below.  This is the double pass the single-step SSLBM
// removes; it is kept for the comparison.  Boundaries as for the SSLBM (periodic wrap or
// the cell-centred mirror, one link).
#include <cuda_runtime.h>

#include "variants.cuh"

namespace sslbm {
namespace {

// V consecutive cells of a row as one aligned vector access (the pitch is a multiple of 32).
template <typename T, int V>
struct SRow;
template <>
struct SRow<float, 4> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  }
  static __device__ __forceinline__ void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct SRow<double, 2> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x, v[1] = t.y;
  }
  static __device__ __forceinline__ void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// Position of a thread's V cells: x0, the cells that lie in the grid, their left and right
// link neighbours (wrap or clamp).
struct Cols {
  int64_t x0, xl, xr;
  int nvalid;
};
template <int V>
__device__ __forceinline__ bool cols_of(const GridView& g, Cols& c) {
  const int64_t vx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nvec = (g.nx + V - 1) / V;
  if (vx >= nvec) return false;
  c.x0 = vx * V;
  c.nvalid = (int)((g.nx - c.x0) < V ? (g.nx - c.x0) : V);
  c.xl = link_index(c.x0 - 1, g.nx, g.bc);
  c.xr = link_index(c.x0 + c.nvalid, g.nx, g.bc);
  return true;
}

// s[j] = p + lap5(p) / 6 at the V cells of row r (rows ru above, rd below), with the centre
// values in ctr[j]: the neighbour sum of Eqs. (SLBM1) and (SLBM2) on D2Q5.
template <typename T, int V>
__device__ __forceinline__ void nsum(const T* P, const Cols& c, int64_t r, int64_t ru, int64_t rd, T (&ctr)[V],
                                     T (&out)[V]) {
  const T sixth = T(1) / T(6);
  T u[V], d[V];
  SRow<T, V>::load(P + r + c.x0, ctr);
  SRow<T, V>::load(P + ru + c.x0, u);
  SRow<T, V>::load(P + rd + c.x0, d);
  const T L = P[r + c.xl], R = P[r + c.xr];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const T l = j == 0 ? L : ctr[j > 0 ? j - 1 : 0];
    const T rr = j + 1 < c.nvalid ? ctr[j + 1 < V ? j + 1 : j] : R;
    out[j] = fma_rn(lap5(ctr[j], l, rr, u[j], d[j]), sixth, ctr[j]);
  }
}

template <typename T, int V>
__device__ __forceinline__ void store_row(T* p, const Cols& c, const T (&v)[V]) {
  if (c.nvalid == V) {
    SRow<T, V>::store(p, v);
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j)
      if (j < c.nvalid) p[j] = v[j];
  }
}

template <typename T, int V>
__global__ void __launch_bounds__(256) slbm_predict_kernel(const GridView g, const T* __restrict__ in,
                                                           T* __restrict__ pred) {
  Cols c;
  if (!cols_of<V>(g, c)) return;
  for (int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; y < g.ny; y += (int64_t)gridDim.y * blockDim.y) {
    const int64_t r = y * g.pitch, ru = link_index(y - 1, g.ny, g.bc) * g.pitch,
                  rd = link_index(y + 1, g.ny, g.bc) * g.pitch;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      T ctr[V], s[V];
      nsum<T, V>(in + f * g.plane, c, r, ru, rd, ctr, s);
      store_row<T, V>(pred + f * g.plane + r + c.x0, c, s);
    }
  }
}

template <typename T>
struct Tm1 {
  T v[4];  // tau - 1 per mobile compartment
};

template <typename T, int V>
__global__ void __launch_bounds__(256) slbm_correct_kernel(const GridView g, const Coeffs<T> k, const Tm1<T> tm1,
                                                           const T* __restrict__ in, const T* __restrict__ pred,
                                                           T* __restrict__ out) {
  Cols c;
  if (!cols_of<V>(g, c)) return;
  for (int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; y < g.ny; y += (int64_t)gridDim.y * blockDim.y) {
    const int64_t r = y * g.pitch, ru = link_index(y - 1, g.ny, g.bc) * g.pitch,
                  rd = link_index(y + 1, g.ny, g.bc) * g.pitch;
    const int64_t o = r + c.x0;
    T rho[5][V];
#pragma unroll
    for (int f = 0; f < 5; ++f) SRow<T, V>::load(in + f * g.plane + o, rho[f]);
    T n[5][V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const T S = rho[0][j], E = rho[1][j], I = rho[2][j], R = rho[3][j];
      const T F = force_dt(k, S, E, I, R);
      n[0][j] = -F;
      n[1][j] = fma_rn(-k.adt, E, F);
      n[2][j] = fma_rn(k.adt, E, -mul_rn(k.gdt, I));
      n[3][j] = mul_rn(k.rdt, I);
      n[4][j] = fma_rn(k.ddt, I, rho[4][j]);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      T ps[V], s[V];
      nsum<T, V>(pred + f * g.plane, c, r, ru, rd, ps, s);
#pragma unroll
      for (int j = 0; j < V; ++j) n[f][j] = add_rn(fma_rn(tm1.v[f], sub_rn(s[j], rho[f][j]), ps[j]), n[f][j]);
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) store_row<T, V>(out + f * g.plane + o, c, n[f]);
  }
}

template <typename T, int V>
cudaError_t launch_t(const GridView& g, const void* coeffs, const double tm1d[4], const void* in, void* pred,
                     void* out, cudaStream_t s) {
  Tm1<T> tm1;
  for (int c = 0; c < 4; ++c) tm1.v[c] = (T)tm1d[c];
  const int64_t nvec = (g.nx + V - 1) / V;
  dim3 block(32, 8);
  dim3 grid((unsigned)((nvec + 31) / 32), (unsigned)std::min<int64_t>(65535, (g.ny + 7) / 8));
  slbm_predict_kernel<T, V><<<grid, block, 0, s>>>(g, static_cast<const T*>(in), static_cast<T*>(pred));
  slbm_correct_kernel<T, V><<<grid, block, 0, s>>>(g, *static_cast<const Coeffs<T>*>(coeffs), tm1,
                                                   static_cast<const T*>(in), static_cast<const T*>(pred),
                                                   static_cast<T*>(out));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_slbm_step(int precision, const GridView& g, const void* coeffs, const double tm1[4],
                             const void* in, void* pred, void* out, cudaStream_t s) {
  switch (precision) {
    case SSLBM_FP64: return launch_t<double, 2>(g, coeffs, tm1, in, pred, out, s);
    case SSLBM_FP32: return launch_t<float, 4>(g, coeffs, tm1, in, pred, out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sslbm
