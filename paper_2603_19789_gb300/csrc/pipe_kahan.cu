// pipe_kahan.cu -- the temporal-blocked pipeline for the Kahan storage (ten planes per
// row: values and compensations), the launchers of pipe_launch.cuh instantiated for
// MODE_KAHAN: one CTA of K warps per SM, up to 255 registers a thread for the ten-plane rows.
#include "pipe_launch.cuh"

SSLBM_OOB_ACCESSOR(kahan)

namespace sslbm {

int blocked_kahan_default_seg_rows(const GridView& g, int depth) {
  return default_seg_rows_mode<MODE_KAHAN>(g, depth);
}

cudaError_t launch_kahan_blocked(const GridView& g, const void* coeffs, const void* in, void* out, int depth,
                                 int seg_rows, cudaStream_t s) {
  return launch_blocked_mode<MODE_KAHAN>(g, coeffs, in, out, depth, seg_rows, s);
}

}  // namespace sslbm
