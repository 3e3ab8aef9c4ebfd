// variants.cuh -- launchers of the update variants beside the D2Q5 SSLBM: the D2Q9 lattice
// (d2q9.cu) and the two-pass SLBM predictor-corrector (slbm.cu).
#pragma once
#include "sslbm_internal.cuh"

namespace sslbm {

// one SSLBM step on the D2Q9 lattice (FP64 or FP32)
cudaError_t launch_sslbm9_step1(int precision, const GridView& g, const void* coeffs, const void* in, void* out,
                                cudaStream_t s);

// one step of the two-pass SLBM (FP64 or FP32): predictor into pred (4 planes of the state's
// layout), then the corrector into out; tm1[c] = tau_c - 1
cudaError_t launch_slbm_step(int precision, const GridView& g, const void* coeffs, const double tm1[4],
                             const void* in, void* pred, void* out, cudaStream_t s);

}  // namespace sslbm
