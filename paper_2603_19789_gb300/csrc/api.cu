// api.cu -- the C ABI of libsslbm.so (declared and documented in include/sslbm.h).
//
// Host side only: parameter validation (Eq. diffusivity for d -> tau, the von Neumann
// bound 1/2 <= tau <= 5/4, the optional nonnegativity condition), carving of the
// caller's workspace, stream-ordered dispatch of the kernels and status reporting, the
// checkpoint format (header plus the stored planes) and the collection of the debug
// build's index-check records.  No device memory is allocated here; the caller provides it.
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "bounds.cuh"
#include "sslbm_internal.cuh"
#include "variants.cuh"

using sslbm::Coeffs;
using sslbm::GridView;

namespace {

thread_local char g_err[512] = "";

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SSLBM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
  int64_t pitch = 0, plane = 0;
  size_t esize = 0, plane_bytes = 0;
  int s_planes = 0;  // SSLBM planes per state buffer (5; 6 with the split S; 10 with Kahan)
  size_t off_diag = 0, off_s[2] = {0, 0}, off_b[2] = {0, 0}, off_pred = 0, off_kappa = 0, total = 0;
};

constexpr int kBgkPlanes = 21;
constexpr int64_t kMaxSide = int64_t(1) << 30;

int check_grid(const sslbm_grid* g) {
  if (!g) return fail(SSLBM_ERR_BAD_ARG, "grid is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nx > kMaxSide || g->ny > kMaxSide)
    return fail(SSLBM_ERR_BAD_ARG, "nx=%lld ny=%lld: each must be in [1, 2^30]", (long long)g->nx,
                (long long)g->ny);
  if (!(g->dx > 0) || !(g->dt > 0) || !std::isfinite(g->dx) || !std::isfinite(g->dt))
    return fail(SSLBM_ERR_BAD_ARG, "dx and dt must be finite and > 0");
  if (g->bc != SSLBM_BC_PERIODIC && g->bc != SSLBM_BC_NOFLUX)
    return fail(SSLBM_ERR_BAD_ARG, "bc=%d is not a boundary code", g->bc);
  if (g->precision < SSLBM_FP64 || g->precision > SSLBM_FP64_DW)
    return fail(SSLBM_ERR_BAD_ARG, "precision=%d is not a precision code", g->precision);
  if (g->schemes < 1 || g->schemes > 3)
    return fail(SSLBM_ERR_BAD_ARG, "schemes=%d must be a nonzero mask of 1 (SSLBM) and 2 (BGK)",
                g->schemes);
  if (g->lattice != SSLBM_LATTICE_D2Q5 && g->lattice != SSLBM_LATTICE_D2Q9 && g->lattice != SSLBM_LATTICE_D2Q5_SLBM &&
      g->lattice != SSLBM_LATTICE_D2Q5_VARD)
    return fail(SSLBM_ERR_BAD_ARG, "lattice=%d is not a lattice code", g->lattice);
  if (g->lattice != SSLBM_LATTICE_D2Q5 &&
      (g->schemes != SSLBM_WANT_SSLBM || (g->precision != SSLBM_FP64 && g->precision != SSLBM_FP32)))
    return fail(SSLBM_ERR_UNSUPPORTED,
                "the D2Q9, two-pass and varying-diffusivity updates are provided for the SSLBM scheme in FP64 and FP32");
  if ((g->schemes & SSLBM_WANT_BGK) && g->precision != SSLBM_FP64 && g->precision != SSLBM_FP32)
    return fail(SSLBM_ERR_UNSUPPORTED, "BGK state is provided in FP64 and FP32 only");
  return SSLBM_OK;
}

int make_layout(const sslbm_grid* g, Layout* L) {
  int st = check_grid(g);
  if (st) return st;
  L->esize = g->precision == SSLBM_FP64 ? 8 : 4;
  L->pitch = (g->nx + 31) / 32 * 32;
  L->plane = (L->pitch * g->ny + 63) / 64 * 64;
  const double bytes_est = (double)L->plane * (double)L->esize * (10.0 + 2 * kBgkPlanes) * 2.0;
  if (bytes_est > 9.0e18) return fail(SSLBM_ERR_BAD_ARG, "grid too large");
  L->plane_bytes = round_up((size_t)L->plane * L->esize, kAlign);
  // the double-word storage keeps the Kahan storage's ten planes (hi, and -lo as compensation)
  L->s_planes = (g->precision == SSLBM_FP32_KAHAN || g->precision == SSLBM_FP64_DW) ? 10
                : g->precision == SSLBM_FP32_SPLIT                                  ? 6
                                                                                    : 5;
  size_t off = 0;
  L->off_diag = off;
  off += round_up((sslbm::kDiagBlocks * sslbm::kDiagSlots + 8) * sizeof(double), kAlign);
  if (g->schemes & SSLBM_WANT_SSLBM)
    for (int b = 0; b < 2; ++b) {
      L->off_s[b] = off;
      off += (size_t)L->s_planes * L->plane_bytes;
    }
  if (g->schemes & SSLBM_WANT_BGK)
    for (int b = 0; b < 2; ++b) {
      L->off_b[b] = off;
      off += (size_t)kBgkPlanes * L->plane_bytes;
    }
  if (g->lattice == SSLBM_LATTICE_D2Q5_SLBM) {  // the predictor's four planes
    L->off_pred = off;
    off += (size_t)4 * L->plane_bytes;
  }
  if (g->lattice == SSLBM_LATTICE_D2Q5_VARD) {  // the diffusivity scale planes kx, ky
    L->off_kappa = off;
    off += (size_t)2 * L->plane_bytes;
  }
  L->total = off;
  return SSLBM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

namespace sslbm {
// Record a failure for sslbm_last_error() from another translation unit.
int record_error(int status, const char* msg) { return fail(status, "%s", msg); }
}  // namespace sslbm

struct sslbm_handle {
  sslbm_grid g;
  sslbm_params p;
  Layout L;
  GridView gv;
  int device = 0;
  double tau[4];
  Coeffs<double> cd;
  Coeffs<float> cf;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  char* s_buf[2] = {nullptr, nullptr};
  char* b_buf[2] = {nullptr, nullptr};
  char* pred = nullptr;  // two-pass SLBM predictor planes
  char* kappa = nullptr;  // varying diffusivity: scale planes kx, ky
  bool kappa_ok = false;  // the scale planes hold validated fields
  int s_cur = 0, b_cur = 0;
  int64_t s_steps = 0, b_steps = 0;
  int depth = 1, seg_rows = 0;
  int seg_cache[SSLBM_MAX_DEPTH + 1] = {0};
  bool fuse_diag = false;   // sslbm_set_fused_diagnostics
  bool diag_ready = false;  // diag_result() holds the diagnostics of the current SSLBM state

  // Coeffs<double> for FP64 and for the double-word storage (which splits them into pairs)
  const void* coeffs() const {
    return (g.precision == SSLBM_FP64 || g.precision == SSLBM_FP64_DW) ? static_cast<const void*>(&cd)
                                                                       : static_cast<const void*>(&cf);
  }
  char* s_plane(int buf, int c) const { return s_buf[buf] + (size_t)c * L.plane_bytes; }
  double* diag_partials() const { return reinterpret_cast<double*>(ws + L.off_diag); }
  double* diag_result() const {
    return diag_partials() + sslbm::kDiagBlocks * sslbm::kDiagSlots;
  }
};

extern "C" {

const char* sslbm_strerror(int status) {
  switch (status) {
    case SSLBM_OK: return "SSLBM_OK";
    case SSLBM_ERR_BAD_ARG: return "SSLBM_ERR_BAD_ARG";
    case SSLBM_ERR_UNSTABLE: return "SSLBM_ERR_UNSTABLE";
    case SSLBM_ERR_CUDA: return "SSLBM_ERR_CUDA";
    case SSLBM_ERR_TIMEOUT: return "SSLBM_ERR_TIMEOUT";
    case SSLBM_ERR_NONFINITE: return "SSLBM_ERR_NONFINITE";
    case SSLBM_ERR_WORKSPACE: return "SSLBM_ERR_WORKSPACE";
    case SSLBM_ERR_UNSUPPORTED: return "SSLBM_ERR_UNSUPPORTED";
    case SSLBM_ERR_STATE: return "SSLBM_ERR_STATE";
    default: return "SSLBM_ERR_UNKNOWN";
  }
}

const char* sslbm_last_error(void) { return g_err; }

int sslbm_version(void) { return 100; }

int sslbm_workspace_bytes(const sslbm_grid* g, size_t* bytes) {
  if (!bytes) return fail(SSLBM_ERR_BAD_ARG, "bytes is NULL");
  Layout L;
  int st = make_layout(g, &L);
  if (st) return st;
  *bytes = L.total;
  return SSLBM_OK;
}

// The storages of ten planes: values and compensations (Kahan), or high parts and minus the
// low parts (double word); both are read as value - compensation.
static bool ten_planes(const sslbm_handle* h) {
  return h->g.precision == SSLBM_FP32_KAHAN || h->g.precision == SSLBM_FP64_DW;
}

// The D2Q5 FP32 storages and the FP32 D2Q9 and varying-diffusion lattices have the
// temporal-blocked kernel.
static bool can_block(const sslbm_handle* h) {
  if (h->g.lattice == SSLBM_LATTICE_D2Q5) return sslbm::blocked_supported(h->g.precision, h->gv);
  return (h->g.lattice == SSLBM_LATTICE_D2Q9 || h->g.lattice == SSLBM_LATTICE_D2Q5_VARD) &&
         h->g.precision == SSLBM_FP32;
}

// One pass of k steps (k = 1: the one-step kernel) from the current buffer into the spare one,
// on the D2Q5 or D2Q9 lattice.
static cudaError_t launch_pass(sslbm_handle* h, int k, int seg) {
  const bool q9 = h->g.lattice == SSLBM_LATTICE_D2Q9;
  void* out = h->s_buf[1 - h->s_cur];
  if (h->g.lattice == SSLBM_LATTICE_D2Q5_VARD) {  // scale planes kx, ky in the kappa area
    const char* kx = h->kappa;
    const char* ky = h->kappa + h->L.plane_bytes;
    if (k == 1)
      return sslbm::launch_sslbm_vard_step(h->g.precision, h->gv, h->coeffs(), kx, ky, h->s_buf[h->s_cur], out,
                                           h->stream);
    return sslbm::launch_sslbm_vard_blocked(h->gv, &h->cf, kx, ky, h->s_buf[h->s_cur], out, k, seg, h->stream);
  }
  if (k == 1 && h->g.precision == SSLBM_FP64_DW)  // the double word: its own streaming cell
    return sslbm::launch_stream_dw(h->gv, h->coeffs(), h->s_buf[h->s_cur], out, h->stream);
  if (k == 1)
    return q9 ? sslbm::launch_sslbm9_step1(h->g.precision, h->gv, h->coeffs(), h->s_buf[h->s_cur], out, h->stream)
              : sslbm::launch_sslbm_step1(h->g.precision, h->gv, h->coeffs(), h->s_buf[h->s_cur], out, h->stream);
  return q9 ? sslbm::launch_sslbm9_blocked(h->gv, &h->cf, h->s_buf[h->s_cur], out, k, seg, h->stream)
            : sslbm::launch_sslbm_blocked(h->g.precision, h->gv, &h->cf, h->s_buf[h->s_cur], out, k, seg, h->stream);
}

static int default_seg(const sslbm_handle* h, int k) {
  if (h->g.lattice == SSLBM_LATTICE_D2Q5_VARD) return sslbm::blocked_vard_default_seg_rows(h->gv, k);
  return h->g.lattice == SSLBM_LATTICE_D2Q9 ? sslbm::blocked9_default_seg_rows(h->gv, k)
                                            : sslbm::blocked_default_seg_rows(h->g.precision, h->gv, k);
}

int sslbm_create(const sslbm_grid* g, const sslbm_params* p, void* dev_ws, size_t ws_bytes,
                 void* stream, sslbm_handle** out) {
  if (!out) return fail(SSLBM_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  Layout L;
  int st = make_layout(g, &L);
  if (st) return st;
  if (!p) return fail(SSLBM_ERR_BAD_ARG, "params is NULL");
  const double rates[4] = {p->beta, p->alpha, p->gamma, p->phi};
  for (double r : rates)
    if (!std::isfinite(r) || r < 0) return fail(SSLBM_ERR_BAD_ARG, "rates must be finite and >= 0");
  if (p->phi > 1) return fail(SSLBM_ERR_BAD_ARG, "phi=%g must be in [0, 1]", p->phi);
  if (!std::isfinite(p->s_ref)) return fail(SSLBM_ERR_BAD_ARG, "s_ref must be finite");
  double tau[4];
  for (int c = 0; c < 4; ++c) {
    if (p->use_tau) {
      tau[c] = p->tau[c];
    } else {
      if (!std::isfinite(p->d[c]) || p->d[c] < 0)
        return fail(SSLBM_ERR_BAD_ARG, "d[%d]=%g must be finite and >= 0", c, p->d[c]);
      tau[c] = 3.0 * p->d[c] * g->dt / (g->dx * g->dx) + 0.5;  // Eq. (diffusivity)
    }
    if (!std::isfinite(tau[c]))
      return fail(SSLBM_ERR_BAD_ARG, "tau[%d] is not finite", c);
    // |G| <= 1 for all modes needs (2 tau - 1) * max(1 - Lambda) <= 2, with max(1 - Lambda)
    // = 4/3 on D2Q5 (tau <= 5/4) and 8/9 on D2Q9 (tau <= 13/8)
    // (two-pass SLBM: G = Lambda + (tau - 1)(Lambda^2 - 1), |G| <= 1 on Lambda in [-1/3, 1]
    // for tau <= 7/4)
    // (varying diffusivity: the scale fields decide, checked by sslbm_set_diffusivity_scale)
    const double tau_max = g->lattice == SSLBM_LATTICE_D2Q9 ? 1.625
                           : g->lattice == SSLBM_LATTICE_D2Q5_SLBM ? 1.75
                           : g->lattice == SSLBM_LATTICE_D2Q5_VARD ? HUGE_VAL : 1.25;
    if (tau[c] < 0.5 || tau[c] > tau_max)
      return fail(SSLBM_ERR_UNSTABLE, "tau[%d]=%.17g outside the stable range [1/2, %g]", c, tau[c], tau_max);
  }
  if (!p->use_tau && p->d[4] != 0.0)
    return fail(SSLBM_ERR_BAD_ARG, "d[D]=%g: the deceased do not diffuse (must be 0)", p->d[4]);
  double dl[4];
  for (int c = 0; c < 4; ++c) dl[c] = (tau[c] - 0.5) / 3.0;
  if (p->strict && g->lattice != SSLBM_LATTICE_D2Q5_VARD) {
    const double out_rate[4] = {p->beta, p->alpha, p->gamma, 0.0};
    // the centre's weight in the update must stay >= 0: 1 - 4 d (D2Q5) or 1 - 20 d / 6 (D2Q9)
    const double cw = g->lattice == SSLBM_LATTICE_D2Q9 ? 20.0 / 6.0 : 4.0;
    for (int c = 0; c < 4; ++c)
      if (cw * dl[c] + out_rate[c] * g->dt > 1.0)
        return fail(SSLBM_ERR_UNSTABLE,
                    "compartment %d: %g d_lattice + outflow*dt = %g > 1 (nonnegativity)", c, cw,
                    cw * dl[c] + out_rate[c] * g->dt);
  }
  if (!dev_ws) return fail(SSLBM_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(dev_ws) % kAlign)
    return fail(SSLBM_ERR_WORKSPACE, "workspace must be %zu-byte aligned", kAlign);
  if (ws_bytes < L.total)
    return fail(SSLBM_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes, L.total);
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, dev_ws);
  if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes(workspace)");
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(SSLBM_ERR_WORKSPACE, "workspace is not device memory");

  sslbm_handle* h = new (std::nothrow) sslbm_handle();
  if (!h) return fail(SSLBM_ERR_BAD_ARG, "out of host memory");
  h->g = *g;
  h->p = *p;
  h->L = L;
  h->device = attr.device;
  h->gv = GridView{g->nx, g->ny, L.pitch, L.plane, g->bc};
  for (int c = 0; c < 4; ++c) {
    h->tau[c] = tau[c];
    h->cd.dl[c] = dl[c];
    h->cd.itau[c] = 1.0 / tau[c];
    h->cf.dl[c] = (float)dl[c];
    h->cf.itau[c] = (float)(1.0 / tau[c]);
  }
  const double dt = g->dt;
  h->cd.bdt = p->beta * dt;
  h->cd.adt = p->alpha * dt;
  h->cd.gdt = p->gamma * dt;
  h->cd.rdt = (1.0 - p->phi) * p->gamma * dt;
  h->cd.ddt = p->phi * p->gamma * dt;
  h->cd.s_ref = p->s_ref;
  h->cf.bdt = (float)h->cd.bdt;
  h->cf.adt = (float)h->cd.adt;
  h->cf.gdt = (float)h->cd.gdt;
  h->cf.rdt = (float)h->cd.rdt;
  h->cf.ddt = (float)h->cd.ddt;
  h->cf.s_ref = (float)p->s_ref;
  h->stream = static_cast<cudaStream_t>(stream);
  h->ws = static_cast<char*>(dev_ws);
  if (g->schemes & SSLBM_WANT_SSLBM)
    for (int b = 0; b < 2; ++b) h->s_buf[b] = h->ws + L.off_s[b];
  if (g->schemes & SSLBM_WANT_BGK)
    for (int b = 0; b < 2; ++b) h->b_buf[b] = h->ws + L.off_b[b];
  if (g->lattice == SSLBM_LATTICE_D2Q5_SLBM) h->pred = h->ws + L.off_pred;
  if (g->lattice == SSLBM_LATTICE_D2Q5_VARD) h->kappa = h->ws + L.off_kappa;
  h->depth = can_block(h) ? 4 : 1;
  DeviceGuard dg(h->device);
  // zero state buffers (and their row padding) so every scheme starts from a defined state
  e = cudaMemsetAsync(h->ws, 0, L.total, h->stream);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaMemsetAsync(workspace)");
  }
  *out = h;
  return SSLBM_OK;
}

int sslbm_set_stream(sslbm_handle* h, void* stream) {
  if (!h) return fail(SSLBM_ERR_BAD_ARG, "handle is NULL");
  h->stream = static_cast<cudaStream_t>(stream);
  return SSLBM_OK;
}

void sslbm_destroy(sslbm_handle* h) { delete h; }

static int check_scheme(const sslbm_handle* h, int scheme) {
  if (!h) return fail(SSLBM_ERR_BAD_ARG, "handle is NULL");
  if (scheme == SSLBM_SCHEME_SSLBM && (h->g.schemes & SSLBM_WANT_SSLBM)) return SSLBM_OK;
  if (scheme == SSLBM_SCHEME_BGK && (h->g.schemes & SSLBM_WANT_BGK)) return SSLBM_OK;
  return fail(SSLBM_ERR_BAD_ARG, "scheme %d not held by this handle", scheme);
}

int sslbm_write(sslbm_handle* h, int scheme, int comp, const void* src, int src_dtype,
                int src_on_device) {
  int st = check_scheme(h, scheme);
  if (st) return st;
  if (!src) return fail(SSLBM_ERR_BAD_ARG, "src is NULL");
  if (comp != SSLBM_ALL && (comp < 0 || comp >= SSLBM_NCOMP))
    return fail(SSLBM_ERR_BAD_ARG, "comp=%d", comp);
  if (src_dtype != SSLBM_DT_F64 && src_dtype != SSLBM_DT_F32)
    return fail(SSLBM_ERR_BAD_ARG, "src_dtype=%d", src_dtype);
  DeviceGuard dg(h->device);
  const size_t usize = src_dtype == SSLBM_DT_F64 ? 8 : 4;
  const size_t plane_user = (size_t)h->g.nx * (size_t)h->g.ny * usize;
  const int c0 = comp == SSLBM_ALL ? 0 : comp, c1 = comp == SSLBM_ALL ? 5 : comp + 1;
  const bool bgk = scheme == SSLBM_SCHEME_BGK;
  if (!bgk) h->diag_ready = false;
  char* staging = bgk ? h->b_buf[1 - h->b_cur] : h->s_buf[1 - h->s_cur];
  const int own_dtype = h->g.precision == SSLBM_FP64 ? SSLBM_DT_F64 : SSLBM_DT_F32;
  for (int c = c0; c < c1; ++c) {
    const char* s = static_cast<const char*>(src) + (size_t)(c - c0) * plane_user;
    // values stored as given (same type, no deviation or compensation plane): one strided copy
    // into the pitched plane, without staging or a conversion pass
    if (!bgk && src_dtype == own_dtype && !ten_planes(h) &&
        !((h->g.precision == SSLBM_FP32_DEV || h->g.precision == SSLBM_FP32_SPLIT) && c == SSLBM_S)) {
      cudaError_t e = cudaMemcpy2DAsync(h->s_plane(h->s_cur, c), (size_t)h->L.pitch * usize, s,
                                        (size_t)h->g.nx * usize, (size_t)h->g.nx * usize, (size_t)h->g.ny,
                                        src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync(write)");
      continue;
    }
    if (!src_on_device) {
      cudaError_t e = cudaMemcpyAsync(staging, s, plane_user, cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(H2D)");
      s = staging;
    }
    cudaError_t e;
    if (bgk) {
      e = sslbm::launch_bgk_init(h->g.precision, h->gv, c, s, src_dtype, h->b_buf[h->b_cur],
                                 h->stream);
    } else {
      const bool kahan = ten_planes(h);
      const bool split = h->g.precision == SSLBM_FP32_SPLIT && c == SSLBM_S;
      const int dev_S = (h->g.precision == SSLBM_FP32_DEV && c == SSLBM_S) ? 1 : 0;
      e = sslbm::launch_plane_write(h->g.precision, h->gv, s, src_dtype, h->s_plane(h->s_cur, c),
                                    (kahan || split) ? h->s_plane(h->s_cur, 5 + c) : nullptr, dev_S,
                                    h->p.s_ref, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "write kernel");
  }
  if (!src_on_device) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(write)");
  }
  if (comp == SSLBM_ALL) {
    if (bgk) h->b_steps = 0;
    else h->s_steps = 0;
  }
  return SSLBM_OK;
}

int sslbm_set_diffusivity_scale(sslbm_handle* h, const void* kx, const void* ky, int src_dtype,
                                int src_on_device) {
  int st = check_scheme(h, SSLBM_SCHEME_SSLBM);
  if (st) return st;
  if (h->g.lattice != SSLBM_LATTICE_D2Q5_VARD)
    return fail(SSLBM_ERR_UNSUPPORTED, "diffusivity scale fields need the lattice SSLBM_LATTICE_D2Q5_VARD");
  if (!kx) return fail(SSLBM_ERR_BAD_ARG, "kx is NULL");
  if (!ky) ky = kx;
  if (src_dtype != SSLBM_DT_F64 && src_dtype != SSLBM_DT_F32)
    return fail(SSLBM_ERR_BAD_ARG, "src_dtype=%d", src_dtype);
  DeviceGuard dg(h->device);
  h->kappa_ok = false;
  const size_t usize = src_dtype == SSLBM_DT_F64 ? 8 : 4;
  const size_t plane_user = (size_t)h->g.nx * (size_t)h->g.ny * usize;
  char* staging = h->s_buf[1 - h->s_cur];  // the step's output buffer, free between steps
  const void* srcs[2] = {kx, ky};
  for (int f = 0; f < 2; ++f) {
    const void* s = srcs[f];
    if (!src_on_device) {
      cudaError_t e = cudaMemcpyAsync(staging, s, plane_user, cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(H2D)");
      s = staging;
    }
    cudaError_t e = sslbm::launch_plane_write(h->g.precision, h->gv, s, src_dtype,
                                              h->kappa + (size_t)f * h->L.plane_bytes, nullptr, 0, 0.0, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "scale field write kernel");
  }
  cudaError_t e = sslbm::launch_vard_check(h->g.precision, h->gv, h->kappa, h->kappa + h->L.plane_bytes,
                                           h->diag_partials(), h->diag_result(), h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "scale field check launch");
  double r[2];
  e = cudaMemcpyAsync(r, h->diag_result(), sizeof(r), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(scale field check)");
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(scale field check)");
  if (r[1] > 0)
    return fail(SSLBM_ERR_BAD_ARG, "%.0f scale values are negative or not finite", r[1]);
  const double out_rate[4] = {h->p.beta, h->p.alpha, h->p.gamma, 0.0};
  for (int c = 0; c < 4; ++c) {
    const double w = h->cd.dl[c] * r[0] + (h->p.strict ? out_rate[c] * h->g.dt : 0.0);
    if (w > 1.0 + 1e-12)
      return fail(SSLBM_ERR_UNSTABLE,
                  "compartment %d: d_lattice %.17g x max link sum %.17g%s = %.17g > 1 (centre weight < 0)", c,
                  h->cd.dl[c], r[0], h->p.strict ? " + outflow*dt" : "", w);
  }
  h->kappa_ok = true;
  return SSLBM_OK;
}

int sslbm_read(sslbm_handle* h, int scheme, int comp, void* dst, int dst_dtype, int dst_on_device) {
  int st = check_scheme(h, scheme);
  if (st) return st;
  if (!dst) return fail(SSLBM_ERR_BAD_ARG, "dst is NULL");
  if (comp != SSLBM_ALL && (comp < 0 || comp >= SSLBM_NCOMP))
    return fail(SSLBM_ERR_BAD_ARG, "comp=%d", comp);
  if (dst_dtype != SSLBM_DT_F64 && dst_dtype != SSLBM_DT_F32)
    return fail(SSLBM_ERR_BAD_ARG, "dst_dtype=%d", dst_dtype);
  DeviceGuard dg(h->device);
  const size_t usize = dst_dtype == SSLBM_DT_F64 ? 8 : 4;
  const size_t plane_user = (size_t)h->g.nx * (size_t)h->g.ny * usize;
  const int c0 = comp == SSLBM_ALL ? 0 : comp, c1 = comp == SSLBM_ALL ? 5 : comp + 1;
  const bool bgk = scheme == SSLBM_SCHEME_BGK;
  char* staging = bgk ? h->b_buf[1 - h->b_cur] : h->s_buf[1 - h->s_cur];
  const int own_dtype = h->g.precision == SSLBM_FP64 ? SSLBM_DT_F64 : SSLBM_DT_F32;
  for (int c = c0; c < c1; ++c) {
    char* d = static_cast<char*>(dst) + (size_t)(c - c0) * plane_user;
    // values stored as they are returned: one strided copy out of the pitched plane
    if (!bgk && dst_dtype == own_dtype && !ten_planes(h) &&
        !((h->g.precision == SSLBM_FP32_DEV || h->g.precision == SSLBM_FP32_SPLIT) && c == SSLBM_S)) {
      cudaError_t e = cudaMemcpy2DAsync(d, (size_t)h->g.nx * usize, h->s_plane(h->s_cur, c),
                                        (size_t)h->L.pitch * usize, (size_t)h->g.nx * usize, (size_t)h->g.ny,
                                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                        h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync(read)");
      continue;
    }
    char* target = dst_on_device ? d : staging;
    cudaError_t e;
    if (bgk) {
      e = sslbm::launch_bgk_density(h->g.precision, h->gv, c, h->b_buf[h->b_cur], target,
                                    dst_dtype, h->stream);
    } else {
      const bool kahan = ten_planes(h);
      const bool split = h->g.precision == SSLBM_FP32_SPLIT && c == SSLBM_S;
      const int dev_S = (h->g.precision == SSLBM_FP32_DEV && c == SSLBM_S) ? 1 : 0;
      e = sslbm::launch_plane_read(h->g.precision, h->gv, h->s_plane(h->s_cur, c),
                                   (kahan || split) ? h->s_plane(h->s_cur, 5 + c) : nullptr, dev_S,
                                   h->p.s_ref, target, dst_dtype, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "read kernel");
    if (!dst_on_device) {
      e = cudaMemcpyAsync(d, staging, plane_user, cudaMemcpyDeviceToHost, h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(D2H)");
    }
  }
  if (!dst_on_device) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(read)");
  }
  return SSLBM_OK;
}

int sslbm_step(sslbm_handle* h, int64_t n) {
  int st = check_scheme(h, SSLBM_SCHEME_SSLBM);
  if (st) return st;
  if (n < 0) return fail(SSLBM_ERR_BAD_ARG, "n=%lld < 0", (long long)n);
  DeviceGuard dg(h->device);
  if (h->g.lattice == SSLBM_LATTICE_D2Q5_SLBM) {
    double tm1[4];
    for (int c = 0; c < 4; ++c) tm1[c] = h->tau[c] - 1.0;
    for (; n > 0; --n) {
      cudaError_t e = sslbm::launch_slbm_step(h->g.precision, h->gv, h->coeffs(), tm1, h->s_buf[h->s_cur], h->pred,
                                              h->s_buf[1 - h->s_cur], h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "SLBM step launch");
      h->s_cur = 1 - h->s_cur;
      h->s_steps += 1;
    }
    return SSLBM_OK;
  }
  if (h->g.lattice == SSLBM_LATTICE_D2Q5_VARD && !h->kappa_ok)
    return fail(SSLBM_ERR_BAD_ARG, "the diffusivity scale fields are not set (sslbm_set_diffusivity_scale)");
  const bool blocked = can_block(h);
  if (n > 0) h->diag_ready = false;
  while (n > 0) {
    int k = 1;
    cudaError_t e;
    if (blocked && h->depth > 1 && n > 1) {
      // depth >= 2: the temporal-blocked kernel; a single step uses the one-step kernel,
      // which produces the same bits.  The n steps take ceil(n / depth) passes whose depths
      // differ by at most one (100 steps at depth 7: 10 of 7 and 5 of 6), rather than full
      // passes and a shallow remainder, which runs at a lower rate per step.
      const int64_t passes = (n + h->depth - 1) / h->depth;
      k = (int)((n + passes - 1) / passes);
      int seg = h->seg_rows;
      if (seg <= 0) {
        if (!h->seg_cache[k]) h->seg_cache[k] = default_seg(h, k);
        seg = h->seg_cache[k];
      }
      // the last pass of the call takes the diagnostics of its output when they are fused
      if (h->fuse_diag && n == k && h->g.lattice == SSLBM_LATTICE_D2Q5 &&
          sslbm::blocked_diag_supported(h->g.precision, h->gv, k, seg)) {
        e = sslbm::launch_sslbm_blocked_diag(h->g.precision, h->gv, &h->cf, h->s_buf[h->s_cur],
                                             h->s_buf[1 - h->s_cur], k, seg, h->diag_partials(), h->stream);
        if (e == cudaSuccess)
          e = sslbm::launch_diag_final(h->diag_partials(), (int)sslbm::blocked_ctas(h->gv, k, seg),
                                       h->diag_result(), h->stream);
        if (e == cudaSuccess) h->diag_ready = true;
      } else {
        e = launch_pass(h, k, seg);
      }
    } else {
      e = launch_pass(h, 1, 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "SSLBM step launch");
    h->s_cur = 1 - h->s_cur;
    h->s_steps += k;
    n -= k;
  }
  return SSLBM_OK;
}

int bgk_step(sslbm_handle* h, int64_t n) {
  int st = check_scheme(h, SSLBM_SCHEME_BGK);
  if (st) return st;
  if (n < 0) return fail(SSLBM_ERR_BAD_ARG, "n=%lld < 0", (long long)n);
  DeviceGuard dg(h->device);
  for (int64_t i = 0; i < n; ++i) {
    cudaError_t e = sslbm::launch_bgk_step(h->g.precision, h->gv, h->coeffs(), h->b_buf[h->b_cur],
                                           h->b_buf[1 - h->b_cur], h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "BGK step launch");
    h->b_cur = 1 - h->b_cur;
    h->b_steps += 1;
  }
  return SSLBM_OK;
}

int64_t sslbm_steps_done(const sslbm_handle* h, int scheme) {
  if (!h) return -1;
  return scheme == SSLBM_SCHEME_BGK ? h->b_steps : h->s_steps;
}

}  // extern "C"

namespace {
constexpr uint32_t kCkptMagic = 0x434C5353u;  // the bytes "SSLC"
constexpr uint32_t kCkptVersion = 2;
constexpr size_t kCkptData = 128;  // the planes start here
// s_ref is the reference the FP32_DEV storage holds S against (sigma = s_ref - S): a stored
// deviation plane means a different S under another reference, so a load compares it.
struct CkptHeader {
  uint32_t magic, version;
  int64_t nx, ny;
  int32_t precision, lattice, bc, schemes;
  int64_t s_steps, b_steps;
  int32_t s_planes, b_planes, esize, reserved;
  double s_ref;
};
static_assert(sizeof(CkptHeader) <= kCkptData, "checkpoint header");

CkptHeader ckpt_header(const sslbm_handle* h) {
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  hd.magic = kCkptMagic;
  hd.version = kCkptVersion;
  hd.nx = h->g.nx;
  hd.ny = h->g.ny;
  hd.precision = h->g.precision;
  hd.lattice = h->g.lattice;
  hd.bc = h->g.bc;
  hd.schemes = h->g.schemes;
  hd.s_steps = h->s_steps;
  hd.b_steps = h->b_steps;
  hd.s_planes = (h->g.schemes & SSLBM_WANT_SSLBM) ? h->L.s_planes : 0;
  hd.b_planes = (h->g.schemes & SSLBM_WANT_BGK) ? kBgkPlanes : 0;
  hd.esize = (int32_t)h->L.esize;
  hd.s_ref = h->p.s_ref;
  return hd;
}

size_t ckpt_bytes(const CkptHeader& hd) {
  return kCkptData + (size_t)(hd.s_planes + hd.b_planes) * (size_t)hd.nx * (size_t)hd.ny * (size_t)hd.esize;
}

// The i-th stored plane: SSLBM planes first, then BGK.
char* ckpt_plane(const sslbm_handle* h, const CkptHeader& hd, int i) {
  if (i < hd.s_planes) return h->s_plane(h->s_cur, i);
  return h->b_buf[h->b_cur] + (size_t)(i - hd.s_planes) * h->L.plane_bytes;
}
}  // namespace

extern "C" {

int sslbm_debug_bounds(long long* count, long long* value, long long* limit, int* site) {
#ifndef SSLBM_BOUNDS_CHECK
  (void)count, (void)value, (void)limit, (void)site;
  return fail(SSLBM_ERR_UNSUPPORTED, "this library was built without SSLBM_BOUNDS_CHECK");
#else
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize(bounds records)");
  int (*const take[])(sslbm::OobRecord*) = {sslbm::oob_take_kernels, sslbm::oob_take_ensemble, sslbm::oob_take_bgk,
                                            sslbm::oob_take_io, sslbm::oob_take_stream,
                                            sslbm::oob_take_d2q9, sslbm::oob_take_d2q9a, sslbm::oob_take_vard,
                                            sslbm::oob_take_kahan, sslbm::oob_take_diag};
  const int tu_site[] = {0, 100, 200, 300, 400, 500, 600, 700, 800, 900};  // offset by translation unit
  unsigned long long total = 0;
  sslbm::OobRecord first{};
  int first_site = -1;
  for (int i = 0; i < 10; ++i) {
    sslbm::OobRecord r{};
    if (take[i](&r) != 0) return fail(SSLBM_ERR_CUDA, "reading the bounds record of unit %d", i);
    if (r.count && first_site < 0) {
      first = r;
      first_site = tu_site[i] + r.site;
    }
    total += r.count;
  }
  if (count) *count = (long long)total;
  if (value) *value = first.value;
  if (limit) *limit = first.limit;
  if (site) *site = first_site;
  return SSLBM_OK;
#endif
}

int sslbm_debug_bounds_probe(long long value, long long limit) {
#ifndef SSLBM_BOUNDS_CHECK
  (void)value, (void)limit;
  return fail(SSLBM_ERR_UNSUPPORTED, "this library was built without SSLBM_BOUNDS_CHECK");
#else
  cudaError_t e = sslbm::launch_oob_probe(value, limit, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "bounds probe");
  return SSLBM_OK;
#endif
}

int sslbm_checkpoint_bytes(const sslbm_handle* h, size_t* bytes) {
  if (!h || !bytes) return fail(SSLBM_ERR_BAD_ARG, "handle or bytes is NULL");
  *bytes = ckpt_bytes(ckpt_header(h));
  return SSLBM_OK;
}

int sslbm_checkpoint_save(sslbm_handle* h, void* dst, size_t bytes, int dst_on_device) {
  if (!h || !dst) return fail(SSLBM_ERR_BAD_ARG, "handle or dst is NULL");
  const CkptHeader hd = ckpt_header(h);
  const size_t need = ckpt_bytes(hd);
  if (bytes < need) return fail(SSLBM_ERR_BAD_ARG, "checkpoint buffer of %zu bytes < %zu", bytes, need);
  DeviceGuard dg(h->device);
  unsigned char head[kCkptData];
  std::memset(head, 0, sizeof(head));
  std::memcpy(head, &hd, sizeof(hd));
  if (dst_on_device) {
    cudaError_t e = cudaMemcpyAsync(dst, head, kCkptData, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(checkpoint header)");
  } else {
    std::memcpy(dst, head, kCkptData);
  }
  const size_t row = (size_t)hd.nx * hd.esize, plane_user = row * (size_t)hd.ny;
  char* d = static_cast<char*>(dst) + kCkptData;
  for (int i = 0; i < hd.s_planes + hd.b_planes; ++i, d += plane_user) {
    cudaError_t e = cudaMemcpy2DAsync(d, row, ckpt_plane(h, hd, i), (size_t)h->L.pitch * h->L.esize, row,
                                      (size_t)hd.ny, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                      h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync(checkpoint save)");
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(checkpoint save)");
  return SSLBM_OK;
}

int sslbm_checkpoint_load(sslbm_handle* h, const void* src, size_t bytes, int src_on_device) {
  if (!h || !src) return fail(SSLBM_ERR_BAD_ARG, "handle or src is NULL");
  if (bytes < kCkptData) return fail(SSLBM_ERR_BAD_ARG, "checkpoint of %zu bytes has no header", bytes);
  DeviceGuard dg(h->device);
  CkptHeader got;
  if (src_on_device) {
    cudaError_t e = cudaMemcpyAsync(&got, src, sizeof(got), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint header");
  } else {
    std::memcpy(&got, src, sizeof(got));
  }
  if (got.magic != kCkptMagic || got.version != kCkptVersion)
    return fail(SSLBM_ERR_BAD_ARG, "not a checkpoint of this format (magic %08x, version %u)", got.magic,
                got.version);
  const CkptHeader own = ckpt_header(h);
  if (got.nx != own.nx || got.ny != own.ny || got.precision != own.precision || got.lattice != own.lattice ||
      got.bc != own.bc || got.schemes != own.schemes || got.s_planes != own.s_planes ||
      got.b_planes != own.b_planes || got.esize != own.esize)
    return fail(SSLBM_ERR_BAD_ARG,
                "checkpoint of a %lld x %lld grid (precision %d, lattice %d, bc %d, schemes %d) does not match "
                "this %lld x %lld solver (precision %d, lattice %d, bc %d, schemes %d)",
                (long long)got.nx, (long long)got.ny, got.precision, got.lattice, got.bc, got.schemes,
                (long long)own.nx, (long long)own.ny, own.precision, own.lattice, own.bc, own.schemes);
  if (own.precision == SSLBM_FP32_DEV && (own.s_planes > 0) && got.s_ref != own.s_ref)
    return fail(SSLBM_ERR_BAD_ARG,
                "checkpoint stores S as a deviation from s_ref = %.17g, this solver's s_ref is %.17g", got.s_ref,
                own.s_ref);
  if (got.s_steps < 0 || got.b_steps < 0) return fail(SSLBM_ERR_BAD_ARG, "negative step counters");
  const size_t need = ckpt_bytes(own);
  if (bytes < need) return fail(SSLBM_ERR_BAD_ARG, "checkpoint of %zu bytes < %zu", bytes, need);
  const size_t row = (size_t)own.nx * own.esize, plane_user = row * (size_t)own.ny;
  const char* sp = static_cast<const char*>(src) + kCkptData;
  h->diag_ready = false;
  for (int i = 0; i < own.s_planes + own.b_planes; ++i, sp += plane_user) {
    cudaError_t e = cudaMemcpy2DAsync(ckpt_plane(h, own, i), (size_t)h->L.pitch * h->L.esize, sp, row, row,
                                      (size_t)own.ny, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                      h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync(checkpoint load)");
  }
  if (!src_on_device) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(checkpoint load)");
  }
  h->s_steps = got.s_steps;
  h->b_steps = got.b_steps;
  return SSLBM_OK;
}

int sslbm_diagnostics(sslbm_handle* h, int scheme, double* totals, double* peak_I) {
  int st = check_scheme(h, scheme);
  if (st) return st;
  DeviceGuard dg(h->device);
  const bool bgk = scheme == SSLBM_SCHEME_BGK;
  cudaError_t e = cudaSuccess;
  if (bgk || !h->diag_ready) {  // else the last step's fused pass left them in diag_result()
    const void* planes = bgk ? (const void*)h->b_buf[h->b_cur] : (const void*)h->s_buf[h->s_cur];
    const bool comp = !bgk && (ten_planes(h) || h->g.precision == SSLBM_FP32_SPLIT);
    const void* comps = comp ? h->s_plane(h->s_cur, 5) : nullptr;
    h->diag_ready = false;  // the reduction below overwrites the result
    e = sslbm::launch_diagnostics(h->g.precision, bgk ? 1 : 0, h->gv, planes, comps, h->diag_partials(),
                                  h->diag_result(), h->stream, h->g.precision == SSLBM_FP32_SPLIT ? 1 : 5);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics launch");
  }
  double r[sslbm::kDiagSlots];
  e = cudaMemcpyAsync(r, h->diag_result(), sizeof(r), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(diagnostics)");
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(diagnostics)");
  if (!bgk && h->g.precision == SSLBM_FP32_DEV)
    r[0] = h->p.s_ref * (double)h->g.nx * (double)h->g.ny - r[0];
  if (totals)
    for (int c = 0; c < 5; ++c) totals[c] = r[c];
  if (peak_I) *peak_I = r[5];
  for (int c = 0; c < 5; ++c)
    if (!std::isfinite(r[c])) return fail(SSLBM_ERR_NONFINITE, "total of compartment %d is %g", c, r[c]);
  return SSLBM_OK;
}

int sslbm_set_fused_diagnostics(sslbm_handle* h, int on) {
  if (!h) return fail(SSLBM_ERR_BAD_ARG, "handle is NULL");
  if (on != 0 && on != 1) return fail(SSLBM_ERR_BAD_ARG, "on=%d (0 or 1)", on);
  h->fuse_diag = on == 1;
  return SSLBM_OK;
}

int sslbm_get_fused_diagnostics(const sslbm_handle* h, int* on, int* ready) {
  if (!h) return fail(SSLBM_ERR_BAD_ARG, "handle is NULL");
  if (on) *on = h->fuse_diag ? 1 : 0;
  if (ready) *ready = h->diag_ready ? 1 : 0;
  return SSLBM_OK;
}

int sslbm_set_blocking(sslbm_handle* h, int k, int seg_rows) {
  if (!h) return fail(SSLBM_ERR_BAD_ARG, "handle is NULL");
  if (k < 0 || k > SSLBM_MAX_DEPTH) return fail(SSLBM_ERR_BAD_ARG, "k=%d", k);
  if (seg_rows < 0) return fail(SSLBM_ERR_BAD_ARG, "seg_rows=%d", seg_rows);
  const bool blocked = can_block(h);
  if (!blocked && k > 1)
    return fail(SSLBM_ERR_UNSUPPORTED,
                "temporal blocking is provided for the FP32 storages on D2Q5 and for FP32 on D2Q9 "
                "and the varying-diffusion lattice");
  h->depth = k == 0 ? (blocked ? 4 : 1) : k;
  if (seg_rows > 0 && seg_rows < 4 * h->depth) seg_rows = 4 * h->depth;
  h->seg_rows = seg_rows;
  return SSLBM_OK;
}

namespace {
struct TuneKey {
  int device, precision, lattice, bc;
  int64_t nx, ny;
  bool operator<(const TuneKey& o) const {
    return std::tie(device, precision, lattice, bc, nx, ny) <
           std::tie(o.device, o.precision, o.lattice, o.bc, o.nx, o.ny);
  }
};
struct TuneResult {
  int depth, seg_rows;
  double ms_per_step;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneResult> g_tune_cache;

}  // namespace

int sslbm_autotune(sslbm_handle* h, double budget_ms, int* depth_out, int* seg_out,
                   double* ms_per_step_out) {
  int st = check_scheme(h, SSLBM_SCHEME_SSLBM);
  if (st) return st;
  if (!(budget_ms >= 0)) return fail(SSLBM_ERR_BAD_ARG, "budget_ms must be >= 0");
  if (budget_ms == 0) budget_ms = 300.0;
  if (h->g.lattice != SSLBM_LATTICE_D2Q5 && h->g.lattice != SSLBM_LATTICE_D2Q9 &&
      h->g.lattice != SSLBM_LATTICE_D2Q5_VARD)
    return fail(SSLBM_ERR_UNSUPPORTED, "the autotuner tunes the D2Q5, D2Q9 and varying-diffusion kernels");
  if (h->g.lattice == SSLBM_LATTICE_D2Q5_VARD && !h->kappa_ok)
    return fail(SSLBM_ERR_BAD_ARG, "the diffusivity scale fields are not set (sslbm_set_diffusivity_scale)");
  DeviceGuard dg(h->device);
  const TuneKey key{h->device, h->g.precision, h->g.lattice, h->g.bc, h->g.nx, h->g.ny};
  TuneResult best{1, 0, 0.0};
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
      cached = true;
    }
  }
  if (!cached) {
    std::vector<std::pair<int, int>> cand;
    cand.push_back({1, 0});
    if (can_block(h)) {
      for (int d = 2; d <= SSLBM_MAX_DEPTH; ++d) {
        const int base = default_seg(h, d);
        int segs[3] = {base, base / 2, base * 2};
        for (int sg : segs) {
          if (sg < 4 * d) sg = 4 * d;
          bool dup = false;
          for (auto& c : cand) dup |= (c.first == d && c.second == sg);
          if (!dup) cand.push_back({d, sg});
        }
      }
    }
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      return cuda_fail(e, "cudaEventCreate");
    }
    const double per_cand = budget_ms / (double)cand.size();
    best.ms_per_step = 1e300;
    for (auto& c : cand) {
      // one untimed launch (also sizes the repetition count), then the timed repetitions
      e = cudaEventRecord(e0, h->stream);
      if (e == cudaSuccess) e = launch_pass(h, c.first, c.second);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms1 = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms1, e0, e1);
      int reps = ms1 > 0 ? (int)(per_cand / (double)ms1) : 3;
      if (reps < 2) reps = 2;
      if (reps > 50) reps = 50;
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_pass(h, c.first, c.second);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e, "autotune timing");
      }
      const double per_step = (double)ms / (double)(reps * c.first);
      if (per_step < best.ms_per_step) best = TuneResult{c.first, c.second, per_step};
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
  }
  h->depth = best.depth;
  h->seg_rows = best.depth > 1 ? best.seg_rows : 0;
  if (depth_out) *depth_out = best.depth;
  if (seg_out) *seg_out = h->seg_rows;
  if (ms_per_step_out) *ms_per_step_out = best.ms_per_step;
  return SSLBM_OK;
}

int sslbm_get_blocking(const sslbm_handle* h, int* k, int* seg_rows) {
  if (!h) return fail(SSLBM_ERR_BAD_ARG, "handle is NULL");
  if (k) *k = h->depth;
  if (seg_rows) *seg_rows = h->seg_rows;
  return SSLBM_OK;
}

}  // extern "C"
