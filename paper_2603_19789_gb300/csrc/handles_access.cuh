// handles_access.cuh -- read-only views of the surrogate and ensemble handles for the other
// translation units of the library (the rollout drives both through the public calls and
// needs their grids and the surrogate's stream).  C++ linkage: not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sslbm.h"

namespace sslbm {

// Number of scenarios of an ensemble (-1 for NULL) and the grid of scenario idx
// (SSLBM_ERR_BAD_ARG for NULL or an index out of range).
int ensemble_count(const sslbm_ensemble* e);
int ensemble_grid(const sslbm_ensemble* e, int idx, int64_t* nx, int64_t* ny);

// The surrogate's grid side, largest batch, device and stream (SSLBM_ERR_BAD_ARG for NULL).
int fno_shape(const sslbm_fno* f, int* n, int* max_batch, int* device, cudaStream_t* stream);

}  // namespace sslbm
