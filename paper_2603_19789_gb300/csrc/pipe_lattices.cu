// pipe_lattices.cu -- the temporal-blocked pipeline on the D2Q9 lattice (periodic and
// no-flux) and on the varying-diffusion lattice, FP32 (the launchers of pipe_launch.cuh
// instantiated for MODE_D2Q9, MODE_D2Q9_NOFLUX and MODE_VARD).
#include "pipe_launch.cuh"

SSLBM_OOB_ACCESSOR(lattices)

namespace sslbm {

int blocked9_default_seg_rows(const GridView& g, int depth) {
  return g.bc != 0 ? default_seg_rows_mode<MODE_D2Q9_NOFLUX>(g, depth) : default_seg_rows_mode<MODE_D2Q9>(g, depth);
}

cudaError_t launch_sslbm9_blocked(const GridView& g, const void* coeffs, const void* in, void* out, int depth,
                                  int seg_rows, cudaStream_t s) {
  if (g.bc != 0) return launch_blocked_mode<MODE_D2Q9_NOFLUX>(g, coeffs, in, out, depth, seg_rows, s);
  return launch_blocked_mode<MODE_D2Q9>(g, coeffs, in, out, depth, seg_rows, s);
}

int blocked_vard_default_seg_rows(const GridView& g, int depth) { return default_seg_rows_mode<MODE_VARD>(g, depth); }

cudaError_t launch_sslbm_vard_blocked(const GridView& g, const void* coeffs, const void* kx, const void* ky,
                                      const void* in, void* out, int depth, int seg_rows, cudaStream_t s) {
  return launch_blocked_mode<MODE_VARD>(g, coeffs, in, out, depth, seg_rows, s, kx, ky);
}

}  // namespace sslbm
