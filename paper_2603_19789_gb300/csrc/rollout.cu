// rollout.cu -- the learned surrogate's rollout with residual checks and SSLBM fallback
// (sslbm_surrogate_rollout in sslbm.h).  Not part of the paper's method: the surrogate is
// this library's addition.
//
// One surrogate step of a batch: x = make_input(u), y = network(x), then the checks of y
// against u -- the conservation residual |sum y - sum u| / sum u and the negative mass
// sum max(-y, 0) / sum u, infinite for a non-finite prediction -- and, for every scenario
// that fails either check, the SSLBM itself: the scenario's state u goes into its slot of
// the fallback ensemble, the ensemble kernel advances it by the network's horizon, and the
// result replaces y.  Accepted predictions are projected (with reach > 0) as
// sslbm_fno_check_project describes.  The step's residuals are needed on the host for the
// decision, so each step synchronises the surrogate's stream once; the ensemble's calls
// synchronise its own stream before they return, so the two streams never overlap on u or y.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "handles_access.cuh"

namespace sslbm {
int record_error(int status, const char* msg);
}

namespace {

int err(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return sslbm::record_error(status, buf);
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" int sslbm_surrogate_rollout(sslbm_fno* f, sslbm_ensemble* fallback, int batch, int steps, int k_steps,
                                       float* u, const float* r0, const float* log10d, float* x_scratch,
                                       float* y_scratch, double mass_threshold, double neg_threshold, int reach,
                                       double* residuals, unsigned char* fell_back, sslbm_rollout_stats* stats) {
  if (!f || !fallback || !u || !r0 || !log10d || !x_scratch || !y_scratch)
    return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  int n = 0, max_batch = 0, device = 0;
  cudaStream_t stream = nullptr;
  sslbm::fno_shape(f, &n, &max_batch, &device, &stream);
  if (batch < 1 || batch > max_batch) return err(SSLBM_ERR_BAD_ARG, "batch %d not in [1, %d]", batch, max_batch);
  if (steps < 0) return err(SSLBM_ERR_BAD_ARG, "steps %d < 0", steps);
  if (k_steps < 1) return err(SSLBM_ERR_BAD_ARG, "k_steps %d < 1", k_steps);
  if (reach < 0) return err(SSLBM_ERR_BAD_ARG, "reach %d < 0", reach);
  if (!(mass_threshold == mass_threshold) || !(neg_threshold == neg_threshold))
    return err(SSLBM_ERR_BAD_ARG, "thresholds must not be NaN");
  if (sslbm::ensemble_count(fallback) < batch)
    return err(SSLBM_ERR_BAD_ARG, "the fallback ensemble holds %d scenarios, the rollout %d",
               sslbm::ensemble_count(fallback), batch);
  for (int b = 0; b < batch; ++b) {
    int64_t nx = 0, ny = 0;
    sslbm::ensemble_grid(fallback, b, &nx, &ny);
    if (nx != n || ny != n)
      return err(SSLBM_ERR_BAD_ARG, "fallback scenario %d is %lld x %lld, the surrogate's grid %d x %d", b,
                 (long long)nx, (long long)ny, n, n);
  }
  DevGuard dg(device);
  sslbm_rollout_stats st{};
  st.max_mass_residual = 0.0;
  st.max_neg_residual = 0.0;
  const size_t per = (size_t)5 * n * n;  // floats per state
  std::vector<double> res((size_t)2 * batch);
  std::vector<int> bad;
  float* cur = u;
  float* nxt = y_scratch;
  int s;
  for (int step = 0; step < steps; ++step) {
    if ((s = sslbm_fno_make_input(f, batch, cur, r0, log10d, x_scratch))) return s;
    if ((s = sslbm_fno_infer(f, batch, x_scratch, nxt))) return s;
    if ((s = sslbm_fno_check_project(f, batch, nxt, cur, reach, res.data()))) return s;  // synchronises
    bad.clear();
    for (int b = 0; b < batch; ++b) {
      const double rm = res[2 * b], rn = res[2 * b + 1];
      // written so that a NaN residual fails (a non-finite prediction reports +inf anyway)
      const bool mass_ok = rm <= mass_threshold, neg_ok = rn <= neg_threshold;
      if (!mass_ok) ++st.failed_conservation;
      if (!neg_ok) ++st.failed_nonnegativity;
      if (std::isfinite(rm) && rm > st.max_mass_residual) st.max_mass_residual = rm;
      if (std::isfinite(rn) && rn > st.max_neg_residual) st.max_neg_residual = rn;
      if (!(mass_ok && neg_ok)) bad.push_back(b);
      if (residuals) {
        residuals[((size_t)step * batch + b) * 2] = rm;
        residuals[((size_t)step * batch + b) * 2 + 1] = rn;
      }
      if (fell_back) fell_back[(size_t)step * batch + b] = (mass_ok && neg_ok) ? 0 : 1;
    }
    st.surrogate_steps += batch - (int64_t)bad.size();
    st.fallbacks += (int64_t)bad.size();
    if (!bad.empty()) {
      for (int b : bad)
        if ((s = sslbm_ensemble_write(fallback, b, cur + (size_t)b * per, SSLBM_DT_F32, 1))) return s;
      if ((s = sslbm_ensemble_run(fallback, k_steps))) return s;
      for (int b : bad)
        if ((s = sslbm_ensemble_read(fallback, b, nxt + (size_t)b * per, SSLBM_DT_F32, 1))) return s;
    }
    float* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != u) {
    cudaError_t e = cudaMemcpyAsync(u, cur, (size_t)batch * per * sizeof(float), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
      return err(SSLBM_ERR_CUDA, "final state copy: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
  }
  if (stats) *stats = st;
  return SSLBM_OK;
}
