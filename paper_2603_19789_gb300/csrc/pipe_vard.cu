// pipe_vard.cu -- the temporal-blocked pipeline on the varying-diffusion lattice, FP32 (the
// launchers of pipe_launch.cuh instantiated for MODE_VARD: the scale rows in a static
// shared-memory ring after the row rings).
#include "pipe_launch.cuh"

SSLBM_OOB_ACCESSOR(vard)

namespace sslbm {

int blocked_vard_default_seg_rows(const GridView& g, int depth) { return default_seg_rows_mode<MODE_VARD>(g, depth); }

cudaError_t launch_sslbm_vard_blocked(const GridView& g, const void* coeffs, const void* kx, const void* ky,
                                      const void* in, void* out, int depth, int seg_rows, cudaStream_t s) {
  return launch_blocked_mode<MODE_VARD>(g, coeffs, in, out, depth, seg_rows, s, kx, ky);
}

}  // namespace sslbm
