// bounds.cuh -- index checks of the debug build (compiled with -DSSLBM_BOUNDS_CHECK into
// libsslbm_check.so).  The hot-path kernels test each row and column index of their global
// loads and stores against the grid before the access; an index outside is not used (the
// access is skipped) and is recorded -- count, first value, its limit and a site number -- in a
// record of the translation unit, which the host collects with sslbm_debug_bounds().  In
// release builds SSLBM_IN is the constant true and the checks compile away.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace sslbm {

struct OobRecord {
  unsigned long long count;
  long long value, limit;  // the first offending index and the exclusive upper limit it missed
  int site, pad;
};

// Collect and clear the record of one translation unit (checked builds; zeros otherwise).
int oob_take_kernels(OobRecord* out);
int oob_take_ensemble(OobRecord* out);
int oob_take_bgk(OobRecord* out);
int oob_take_io(OobRecord* out);
int oob_take_stream(OobRecord* out);
int oob_take_d2q9(OobRecord* out);
int oob_take_d2q9a(OobRecord* out);
int oob_take_vard(OobRecord* out);
int oob_take_kahan(OobRecord* out);
int oob_take_diag(OobRecord* out);
// Evaluate one check of index v against limit on the device, with no access behind it.
cudaError_t launch_oob_probe(long long v, long long limit, cudaStream_t s);

}  // namespace sslbm

#ifdef SSLBM_BOUNDS_CHECK
static __device__ sslbm::OobRecord g_oob_record;

// true when [v, v + n) lies in [0, limit); otherwise counts the miss, keeps the first one, false
__device__ __forceinline__ bool sslbm_in_range(long long v, long long n, long long limit, int site) {
  if (v >= 0 && v + n <= limit) return true;
  if (atomicAdd(&g_oob_record.count, 1ull) == 0ull) {
    g_oob_record.value = v;
    g_oob_record.limit = limit;
    g_oob_record.site = site;
  }
  return false;
}
#define SSLBM_IN(v, n, limit, site) sslbm_in_range((long long)(v), (long long)(n), (long long)(limit), (site))

// Defines oob_take_<name>: copy the record to the host and clear it.
#define SSLBM_OOB_ACCESSOR(name)                                                            \
  namespace sslbm {                                                                         \
  int oob_take_##name(OobRecord* out) {                                                     \
    if (cudaMemcpyFromSymbol(out, g_oob_record, sizeof(OobRecord)) != cudaSuccess) return -1; \
    const OobRecord zero{};                                                                 \
    return cudaMemcpyToSymbol(g_oob_record, &zero, sizeof(OobRecord)) == cudaSuccess ? 0 : -1; \
  }                                                                                         \
  }
#else
#define SSLBM_IN(v, n, limit, site) true
#define SSLBM_OOB_ACCESSOR(name)                         \
  namespace sslbm {                                      \
  int oob_take_##name(OobRecord* out) {                  \
    *out = OobRecord{};                                  \
    return 0;                                            \
  }                                                      \
  }
#endif
