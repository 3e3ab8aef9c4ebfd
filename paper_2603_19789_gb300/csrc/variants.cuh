// variants.cuh -- launchers of the update variants beside the D2Q5 SSLBM: the D2Q9 lattice
// (d2q9.cu), the two-pass SLBM predictor-corrector (slbm.cu) and spatially varying,
// anisotropic diffusion (vard.cu).
#pragma once
#include "sslbm_internal.cuh"

namespace sslbm {

// one SSLBM step on the D2Q9 lattice (FP64 or FP32)
cudaError_t launch_sslbm9_step1(int precision, const GridView& g, const void* coeffs, const void* in, void* out,
                                cudaStream_t s);
// the FP32 D2Q9 step and the FP32 varying-diffusion step through the streaming one-step
// kernel (stream.cu)
cudaError_t launch_stream_d2q9(const GridView& g, const void* coeffs, const void* in, void* out, cudaStream_t s);
// The FP64-accurate double-word storage (SSLBM_FP64_DW), one step: coeffs is a Coeffs<double>.
cudaError_t launch_stream_dw(const GridView& g, const void* coeffs, const void* in, void* out, cudaStream_t s);
cudaError_t launch_stream_vard(const GridView& g, const void* coeffs, const void* kx, const void* ky, const void* in,
                               void* out, cudaStream_t s);

// one step of the two-pass SLBM (FP64 or FP32): predictor into pred (4 planes of the state's
// layout), then the corrector into out; tm1[c] = tau_c - 1
cudaError_t launch_slbm_step(int precision, const GridView& g, const void* coeffs, const double tm1[4],
                             const void* in, void* pred, void* out, cudaStream_t s);

// one SSLBM step with per-cell diffusivity scale planes kx, ky (FP64 or FP32, grid layout)
cudaError_t launch_sslbm_vard_step(int precision, const GridView& g, const void* coeffs, const void* kx,
                                   const void* ky, const void* in, void* out, cudaStream_t s);

// validation of the scale planes: result[0] = max over cells of the sum of the link means
// (k(x) + k(x + c_i)) / 2 over the links that carry flux, result[1] = number of values that
// are negative or not finite; partials: gridDim (<= kDiagBlocks) x 2 doubles
cudaError_t launch_vard_check(int precision, const GridView& g, const void* kx, const void* ky, double* partials,
                              double* result, cudaStream_t s);

}  // namespace sslbm
