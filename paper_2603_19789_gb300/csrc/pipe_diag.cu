// pipe_diag.cu -- the D2Q5 pipelines of the FP32 and deviation-S storages with the fused
// diagnostics (the population totals and the peak of I of the pass's output, Sec. II.C 'Mass
// conservation'), instantiated apart from the plain pipelines so that the build compiles them
// in parallel.  The state they write is the plain pipelines' (the diagnostics only read it).
#include "pipe_launch.cuh"

SSLBM_OOB_ACCESSOR(diag)

namespace sslbm {

int64_t blocked_ctas(const GridView& g, int depth, int seg_rows) {
  if (depth < 2 || depth > 8 || seg_rows <= 0) return -1;
  const int64_t wv = pipe_strip_cols(depth);
  return ((g.nx + wv - 1) / wv) * ((g.ny + seg_rows - 1) / seg_rows);
}

bool blocked_diag_supported(int precision, const GridView& g, int depth, int seg_rows) {
  const int64_t ctas = blocked_ctas(g, depth, seg_rows);
  return (precision == SSLBM_FP32 || precision == SSLBM_FP32_DEV) && ctas > 0 && ctas <= kDiagBlocks;
}

cudaError_t launch_sslbm_blocked_diag(int precision, const GridView& g, const void* coeffs, const void* in,
                                      void* out, int depth, int seg_rows, double* partials, cudaStream_t s) {
  if (!blocked_diag_supported(precision, g, depth, seg_rows) || !partials) return cudaErrorInvalidValue;
  if (precision == SSLBM_FP32)
    return launch_blocked_mode<MODE_PLAIN, true>(g, coeffs, in, out, depth, seg_rows, s, nullptr, nullptr, partials);
  return launch_blocked_mode<MODE_DEV, true>(g, coeffs, in, out, depth, seg_rows, s, nullptr, nullptr, partials);
}

}  // namespace sslbm
