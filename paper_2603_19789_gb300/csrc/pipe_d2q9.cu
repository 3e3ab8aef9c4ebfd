// pipe_d2q9.cu -- the temporal-blocked pipeline on the D2Q9 lattice, FP32: periodic, and
// no-flux for any width (the launchers of pipe_launch.cuh instantiated for MODE_D2Q9 and
// MODE_D2Q9_NOFLUX; widths that are a multiple of 4 go to pipe_d2q9_aligned.cu).  The
// instantiations are spread over three units so that the build compiles them in parallel.
#include "pipe_launch.cuh"

SSLBM_OOB_ACCESSOR(d2q9)

namespace sslbm {

int blocked9_default_seg_rows(const GridView& g, int depth) {
  if (g.bc == 0) return default_seg_rows_mode<MODE_D2Q9>(g, depth);
  if ((g.nx & 3) == 0) return blocked9_aligned_default_seg_rows(g, depth);
  return default_seg_rows_mode<MODE_D2Q9_NOFLUX>(g, depth);
}

cudaError_t launch_sslbm9_blocked(const GridView& g, const void* coeffs, const void* in, void* out, int depth,
                                  int seg_rows, cudaStream_t s) {
  if (g.bc == 0) return launch_blocked_mode<MODE_D2Q9>(g, coeffs, in, out, depth, seg_rows, s);
  if ((g.nx & 3) == 0) return launch_sslbm9_aligned_blocked(g, coeffs, in, out, depth, seg_rows, s);
  return launch_blocked_mode<MODE_D2Q9_NOFLUX>(g, coeffs, in, out, depth, seg_rows, s);
}

}  // namespace sslbm
