// pipe_d2q9_aligned.cu -- the temporal-blocked D2Q9 pipeline under no-flux for widths that
// are a multiple of 4 (MODE_D2Q9_NOFLUX4: x = nx - 1 is the last of a lane's four columns, so
// the right wall needs fewer substitutions).
#include "pipe_launch.cuh"

SSLBM_OOB_ACCESSOR(d2q9a)

namespace sslbm {

int blocked9_aligned_default_seg_rows(const GridView& g, int depth) {
  return default_seg_rows_mode<MODE_D2Q9_NOFLUX4>(g, depth);
}

cudaError_t launch_sslbm9_aligned_blocked(const GridView& g, const void* coeffs, const void* in, void* out,
                                          int depth, int seg_rows, cudaStream_t s) {
  return launch_blocked_mode<MODE_D2Q9_NOFLUX4>(g, coeffs, in, out, depth, seg_rows, s);
}

}  // namespace sslbm
