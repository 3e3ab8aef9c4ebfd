// ensemble.cu -- many SEIRD scenarios (each its own periodic grid size, contact rate and
// diffusivities) advanced together by one persistent launch, captured in a CUDA graph.
//
// Work decomposition: a step-block is K fused SSLBM steps (the pipeline tile of
// sslbm_pipe.cuh); a work item is (step-block b, scenario s, tile t), where the tiles of a
// scenario are its 128-column strips times row segments.  Items are numbered block-major
// and handed out in increasing order by one global atomic counter, so every CTA runs
// items until none are left.  Item (b, s, t) reads scenario s's state written by block
// b-1 and overwrites the buffer block b-1 read, so it waits until all tiles of (b-1, s)
// have finished: each finished tile increments done[s] (after a device-scope fence), and
// the waiter polls done[s] >= b * tiles(s).  Because an item only waits for items with
// smaller numbers, which running CTAs have already claimed and which wait on nothing
// later, the launch always makes progress.  Every wait is bounded by a spin limit: when
// it runs out the CTA raises an error flag, and all CTAs stop taking work as soon as they
// see the flag; the host then reports SSLBM_ERR_TIMEOUT.
//
// State layout: two buffers; in each, scenario s owns the planes of its storage -- five, or
// six with the compensation of S of the split storage (pitched as in sslbm_internal.cuh) --
// starting at element offset off[s].  Loads use L2-only cp.async.cg
// (periodic grids, nx a multiple of 4), because other CTAs of the same launch write them.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "bounds.cuh"
#include "sslbm_internal.cuh"
#include "sslbm_pipe.cuh"
#include "handles_access.cuh"

SSLBM_OOB_ACCESSOR(ensemble)

namespace sslbm {
int record_error(int status, const char* msg);
}

using sslbm::Coeffs;
using sslbm::GridView;

namespace {

struct EnsScenario {
  GridView g;
  Coeffs<float> k;
  int64_t off;  // element offset of the scenario's planes in each buffer
  int nstrips, seg_rows, tiles, tile_base;
};

struct EnsControl {
  unsigned long long next_item;
  int error;
  int pad;
};

int err(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return sslbm::record_error(status, buf);
}

int cuda_err(cudaError_t e, const char* what) {
  return err(SSLBM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int MODE, int K>
__global__ void __launch_bounds__(32 * K, 16 / K)
    ensemble_kernel(const EnsScenario* __restrict__ tab, const int n, const int total_tiles,
                    const int nblocks, float* __restrict__ buf0, float* __restrict__ buf1,
                    EnsControl* ctl, unsigned* done, const long long spin_limit,
                    const long long stall_item) {
  extern __shared__ __align__(16) unsigned char ens_smem[];
  using Smem = sslbm::PipeSmem<K, sslbm::mode_planes<MODE>()>;
  Smem& sm = *reinterpret_cast<Smem*>(ens_smem);
  __shared__ long long item_sh;
  __shared__ int go_sh;
  const long long total = (long long)nblocks * total_tiles;
  for (;;) {
    if (threadIdx.x == 0) item_sh = (long long)atomicAdd(&ctl->next_item, 1ULL);
    __syncthreads();
    const long long item = item_sh;
    if (item >= total) break;
    const int b = (int)(item / total_tiles);
    const int u = (int)(item - (long long)b * total_tiles);
    int lo = 0, hi = n - 1;  // scenario owning tile u: last tile_base <= u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab[mid].tile_base <= u) lo = mid;
      else hi = mid - 1;
    }
    const int sidx = lo;
    const GridView g = tab[sidx].g;
    const Coeffs<float> k = tab[sidx].k;
    const int64_t off = tab[sidx].off;
    const int nstrips = tab[sidx].nstrips, seg_rows = tab[sidx].seg_rows, tiles = tab[sidx].tiles;
    const int t = u - tab[sidx].tile_base;
    if (threadIdx.x == 0) {
      int ok = *(volatile int*)&ctl->error == 0;
      if (ok && b > 0) {
        const unsigned target = (unsigned)b * (unsigned)tiles;
        long long it = 0;
        while (ld_acquire(&done[sidx]) < target) {
          if (*(volatile int*)&ctl->error) { ok = 0; break; }
          if (++it > spin_limit) {
            atomicExch(&ctl->error, 1);
            ok = 0;
            break;
          }
          __nanosleep(128);
        }
      }
      go_sh = ok;
    }
    __syncthreads();
    if (!go_sh) break;
    const float* in = ((b & 1) ? buf1 : buf0) + off;
    float* out = ((b & 1) ? buf0 : buf1) + off;
    const int strip = t % nstrips;
    const int64_t y0 = (int64_t)(t / nstrips) * seg_rows;
    const int64_t y1 = (y0 + seg_rows < g.ny) ? y0 + seg_rows : g.ny;
    sslbm::pipe_tile<MODE, K, true>(sm, g, k, in, out, strip, y0, y1);
    __threadfence();  // this thread's tile writes are visible device-wide ...
    __syncthreads();  // ... for every thread of the CTA, before the completion count
    if (threadIdx.x == 0 && item != stall_item) atomicAdd(&done[sidx], 1u);
  }
}

typedef void (*EnsKernel)(const EnsScenario*, int, int, int, float*, float*, EnsControl*, unsigned*,
                          long long, long long);

template <int MODE>
EnsKernel pick_kernel(int depth) {
  switch (depth) {
    case 2: return ensemble_kernel<MODE, 2>;
    case 3: return ensemble_kernel<MODE, 3>;
    case 4: return ensemble_kernel<MODE, 4>;
    case 5: return ensemble_kernel<MODE, 5>;
    case 6: return ensemble_kernel<MODE, 6>;
    case 8: return ensemble_kernel<MODE, 8>;
    default: return nullptr;
  }
}

template <int NF>
size_t pipe_smem_bytes_nf(int depth) {
  switch (depth) {
    case 2: return sizeof(sslbm::PipeSmem<2, NF>);
    case 3: return sizeof(sslbm::PipeSmem<3, NF>);
    case 4: return sizeof(sslbm::PipeSmem<4, NF>);
    case 5: return sizeof(sslbm::PipeSmem<5, NF>);
    case 6: return sizeof(sslbm::PipeSmem<6, NF>);
    case 7: return sizeof(sslbm::PipeSmem<7, NF>);
    case 8: return sizeof(sslbm::PipeSmem<8, NF>);
    default: return 0;
  }
}

// dynamic shared memory of the pipeline tile at this depth (six planes under the split storage)
size_t pipe_smem_bytes(int depth, int precision) {
  return precision == SSLBM_FP32_SPLIT ? pipe_smem_bytes_nf<6>(depth) : pipe_smem_bytes_nf<5>(depth);
}

constexpr size_t kAlign = 256;
size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct EnsLayout {
  size_t off_ctl, off_done, off_tab, off_partials, off_results, off_buf[2], total;
  std::vector<int64_t> pitch, plane, elem_off;
  int64_t buf_elems;
};

// planes a scenario stores: five, and the compensation of S under the split storage
int ens_planes(int precision) { return precision == SSLBM_FP32_SPLIT ? 6 : 5; }

int make_layout(int n, const sslbm_scenario* sc, int precision, EnsLayout* L) {
  L->pitch.resize(n);
  L->plane.resize(n);
  L->elem_off.resize(n);
  int64_t e = 0;
  for (int i = 0; i < n; ++i) {
    L->pitch[i] = (sc[i].nx + 31) / 32 * 32;
    L->plane[i] = (L->pitch[i] * sc[i].ny + 63) / 64 * 64;
    L->elem_off[i] = e;
    e += ens_planes(precision) * L->plane[i];
  }
  L->buf_elems = e;
  size_t off = 0;
  L->off_ctl = off;
  off += round_up(sizeof(EnsControl), kAlign);
  L->off_done = off;
  off += round_up((size_t)n * sizeof(unsigned), kAlign);
  L->off_tab = off;
  off += round_up((size_t)n * sizeof(EnsScenario), kAlign);
  L->off_partials = off;
  off += round_up((size_t)sslbm::kDiagBlocks * sslbm::kDiagSlots * sizeof(double), kAlign);
  L->off_results = off;
  off += round_up((size_t)n * sslbm::kDiagSlots * sizeof(double), kAlign);
  for (int b = 0; b < 2; ++b) {
    L->off_buf[b] = off;
    off += round_up((size_t)e * sizeof(float), kAlign);
  }
  L->total = off;
  return SSLBM_OK;
}

int check_scenarios(int n, const sslbm_scenario* sc, int bc, int precision) {
  if (n < 1 || !sc) return err(SSLBM_ERR_BAD_ARG, "need n >= 1 scenarios");
  if (bc != SSLBM_BC_PERIODIC)
    return err(SSLBM_ERR_UNSUPPORTED, "the ensemble launch takes periodic grids");
  if (precision != SSLBM_FP32 && precision != SSLBM_FP32_DEV && precision != SSLBM_FP32_SPLIT)
    return err(SSLBM_ERR_UNSUPPORTED, "the ensemble launch runs FP32, FP32_DEV or FP32_SPLIT");
  for (int i = 0; i < n; ++i) {
    const sslbm_scenario& s = sc[i];
    if (s.nx < 4 || s.ny < 1 || s.nx % 4 || s.nx > (1 << 24) || s.ny > (1 << 24))
      return err(SSLBM_ERR_BAD_ARG, "scenario %d: nx=%lld must be a multiple of 4 in [4, 2^24], "
                 "ny in [1, 2^24]", i, (long long)s.nx);
    const double r[4] = {s.beta, s.alpha, s.gamma, s.phi};
    for (double v : r)
      if (!std::isfinite(v) || v < 0) return err(SSLBM_ERR_BAD_ARG, "scenario %d: bad rate", i);
    if (s.phi > 1) return err(SSLBM_ERR_BAD_ARG, "scenario %d: phi > 1", i);
    if (!(s.dx > 0) || !(s.dt > 0)) return err(SSLBM_ERR_BAD_ARG, "scenario %d: dx, dt > 0", i);
    if (s.d[4] != 0) return err(SSLBM_ERR_BAD_ARG, "scenario %d: d[D] must be 0", i);
    for (int c = 0; c < 4; ++c) {
      if (!std::isfinite(s.d[c]) || s.d[c] < 0) return err(SSLBM_ERR_BAD_ARG, "scenario %d: bad d", i);
      const double tau = 3.0 * s.d[c] * s.dt / (s.dx * s.dx) + 0.5;  // Eq. (diffusivity)
      if (tau > 1.25)
        return err(SSLBM_ERR_UNSTABLE, "scenario %d: tau[%d]=%g > 5/4", i, c, tau);
    }
  }
  return SSLBM_OK;
}

}  // namespace

struct sslbm_ensemble {
  int n = 0, precision = SSLBM_FP32, device = 0;
  std::vector<sslbm_scenario> sc;
  std::vector<EnsScenario> tab;
  EnsLayout L;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int cur = 0;  // which buffer holds the current state
  int depth = 4, seg_rows = 64, total_tiles = 0;
  long long spin_limit = 1LL << 24;
  long long stall_item = -1;
  int64_t steps = 0;
  // cached graph of one run (n_blocks step-blocks from buffer `cur`)
  cudaGraphExec_t exec = nullptr;
  int exec_blocks = -1, exec_cur = -1, exec_depth = -1;

  float* buf(int b) const { return reinterpret_cast<float*>(ws + L.off_buf[b]); }
  EnsControl* ctl() const { return reinterpret_cast<EnsControl*>(ws + L.off_ctl); }
  unsigned* done() const { return reinterpret_cast<unsigned*>(ws + L.off_done); }
  EnsScenario* dtab() const { return reinterpret_cast<EnsScenario*>(ws + L.off_tab); }
  GridView gv(int i) const {
    return GridView{sc[i].nx, sc[i].ny, L.pitch[i], L.plane[i], SSLBM_BC_PERIODIC};
  }
  float* plane(int b, int i, int c) const { return buf(b) + L.elem_off[i] + (int64_t)c * L.plane[i]; }
};

namespace {

int upload_table(sslbm_ensemble* e) {
  e->tab.resize(e->n);
  int base = 0;
  for (int i = 0; i < e->n; ++i) {
    const sslbm_scenario& s = e->sc[i];
    EnsScenario& t = e->tab[i];
    t.g = e->gv(i);
    for (int c = 0; c < 4; ++c) {
      const double tau = 3.0 * s.d[c] * s.dt / (s.dx * s.dx) + 0.5;
      t.k.dl[c] = (float)((tau - 0.5) / 3.0);
      t.k.itau[c] = (float)(1.0 / tau);
    }
    t.k.bdt = (float)(s.beta * s.dt);
    t.k.adt = (float)(s.alpha * s.dt);
    t.k.gdt = (float)(s.gamma * s.dt);
    t.k.rdt = (float)((1.0 - s.phi) * s.gamma * s.dt);
    t.k.ddt = (float)(s.phi * s.gamma * s.dt);
    t.k.s_ref = (float)s.s_ref;
    t.off = e->L.elem_off[i];
    const int hl = (e->depth + 3) / 4, wv = 128 - 8 * hl;
    t.nstrips = (int)((s.nx + wv - 1) / wv);
    t.seg_rows = (int)std::min<int64_t>(e->seg_rows, s.ny);
    const int nsegs = (int)((s.ny + t.seg_rows - 1) / t.seg_rows);
    t.tiles = t.nstrips * nsegs;
    t.tile_base = base;
    base += t.tiles;
  }
  e->total_tiles = base;
  cudaError_t ce = cudaMemcpyAsync(e->dtab(), e->tab.data(), sizeof(EnsScenario) * e->n,
                                   cudaMemcpyHostToDevice, e->stream);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaMemcpyAsync(table)");
  ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaStreamSynchronize(table)");
  if (e->exec) {
    cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
    e->exec_blocks = -1;
  }
  return SSLBM_OK;
}

int resident_ctas(EnsKernel kern, int depth, int precision, int* out) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (ce == cudaSuccess)
    ce = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
  if (ce == cudaSuccess)
    ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)pipe_smem_bytes(depth, precision));
  if (ce == cudaSuccess)
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * depth, pipe_smem_bytes(depth, precision));
  if (ce != cudaSuccess) return cuda_err(ce, "occupancy query");
  *out = sms * (per > 0 ? per : 1);
  return SSLBM_OK;
}

// Enqueue nblocks step-blocks of depth e->depth (counters reset first), captured once in a
// CUDA graph and replayed.
int launch_blocks(sslbm_ensemble* e, int nblocks) {
  if (nblocks <= 0) return SSLBM_OK;
  EnsKernel kern = e->precision == SSLBM_FP32_DEV     ? pick_kernel<sslbm::MODE_DEV>(e->depth)
                    : e->precision == SSLBM_FP32_SPLIT ? pick_kernel<sslbm::MODE_SPLIT>(e->depth)
                                                       : pick_kernel<sslbm::MODE_PLAIN>(e->depth);
  if (!kern) return err(SSLBM_ERR_BAD_ARG, "depth %d has no ensemble kernel", e->depth);
  if (!(e->exec && e->exec_blocks == nblocks && e->exec_cur == e->cur && e->exec_depth == e->depth)) {
    if (e->exec) {
      cudaGraphExecDestroy(e->exec);
      e->exec = nullptr;
    }
    int grid = 0;
    int st = resident_ctas(kern, e->depth, e->precision, &grid);
    if (st) return st;
    cudaStream_t cap;
    cudaError_t ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return cuda_err(ce, "cudaStreamCreate");
    cudaGraph_t graph = nullptr;
    ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess)
      ce = cudaMemsetAsync(e->ws + e->L.off_ctl, 0, e->L.off_tab - e->L.off_ctl, cap);
    if (ce == cudaSuccess) {
      float* b0 = e->buf(e->cur);
      float* b1 = e->buf(1 - e->cur);
      kern<<<grid, 32 * e->depth, pipe_smem_bytes(e->depth, e->precision), cap>>>(e->dtab(), e->n, e->total_tiles, nblocks, b0, b1, e->ctl(),
                                            e->done(), e->spin_limit, e->stall_item);
      ce = cudaGetLastError();
    }
    cudaError_t ce2 = cudaStreamEndCapture(cap, &graph);
    if (ce == cudaSuccess) ce = ce2;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (ce != cudaSuccess) return cuda_err(ce, "ensemble graph capture");
    e->exec_blocks = nblocks;
    e->exec_cur = e->cur;
    e->exec_depth = e->depth;
  }
  cudaError_t ce = cudaGraphLaunch(e->exec, e->stream);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaGraphLaunch");
  if (nblocks & 1) e->cur = 1 - e->cur;
  return SSLBM_OK;
}

int check_error_flag(sslbm_ensemble* e) {
  EnsControl c;
  cudaError_t ce = cudaMemcpyAsync(&c, e->ctl(), sizeof(c), cudaMemcpyDeviceToHost, e->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return cuda_err(ce, "ensemble status");
  if (c.error) return err(SSLBM_ERR_TIMEOUT, "a dependency wait of the ensemble launch ran out");
  return SSLBM_OK;
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

extern "C" {

int sslbm_ensemble_workspace_bytes(int n, const sslbm_scenario* sc, int precision, size_t* bytes) {
  if (!bytes) return err(SSLBM_ERR_BAD_ARG, "bytes is NULL");
  int st = check_scenarios(n, sc, SSLBM_BC_PERIODIC, precision);
  if (st) return st;
  EnsLayout L;
  make_layout(n, sc, precision, &L);
  *bytes = L.total;
  return SSLBM_OK;
}

int sslbm_ensemble_create(int n, const sslbm_scenario* sc, int precision, void* dev_ws,
                          size_t ws_bytes, void* stream, sslbm_ensemble** out) {
  if (!out) return err(SSLBM_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  int st = check_scenarios(n, sc, SSLBM_BC_PERIODIC, precision);
  if (st) return st;
  EnsLayout L;
  make_layout(n, sc, precision, &L);
  if (!dev_ws || reinterpret_cast<uintptr_t>(dev_ws) % kAlign)
    return err(SSLBM_ERR_WORKSPACE, "workspace missing or not 256-byte aligned");
  if (ws_bytes < L.total)
    return err(SSLBM_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes, L.total);
  cudaPointerAttributes attr;
  cudaError_t ce = cudaPointerGetAttributes(&attr, dev_ws);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaPointerGetAttributes");
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return err(SSLBM_ERR_WORKSPACE, "workspace is not device memory");
  sslbm_ensemble* e = new (std::nothrow) sslbm_ensemble();
  if (!e) return err(SSLBM_ERR_BAD_ARG, "out of host memory");
  e->n = n;
  e->precision = precision;
  e->device = attr.device;
  e->sc.assign(sc, sc + n);
  e->L = L;
  e->ws = static_cast<char*>(dev_ws);
  e->stream = static_cast<cudaStream_t>(stream);
  DevGuard dg(e->device);
  ce = cudaMemsetAsync(e->ws, 0, L.total, e->stream);
  if (ce != cudaSuccess) {
    delete e;
    return cuda_err(ce, "cudaMemsetAsync(workspace)");
  }
  st = upload_table(e);
  if (st) {
    delete e;
    return st;
  }
  *out = e;
  return SSLBM_OK;
}

void sslbm_ensemble_destroy(sslbm_ensemble* e) {
  if (!e) return;
  if (e->exec) cudaGraphExecDestroy(e->exec);
  delete e;
}

int sslbm_ensemble_set_tiling(sslbm_ensemble* e, int depth, int seg_rows) {
  if (!e) return err(SSLBM_ERR_BAD_ARG, "ensemble is NULL");
  if (depth < 2 || depth > 8 || depth == 7) return err(SSLBM_ERR_BAD_ARG, "depth %d not in {2..6, 8}", depth);
  if (seg_rows < 4 * depth) return err(SSLBM_ERR_BAD_ARG, "seg_rows %d < 4 * depth", seg_rows);
  DevGuard dg(e->device);
  e->depth = depth;
  e->seg_rows = seg_rows;
  return upload_table(e);
}

int sslbm_ensemble_get_tiling(const sslbm_ensemble* e, int* depth, int* seg_rows) {
  if (!e) return err(SSLBM_ERR_BAD_ARG, "ensemble is NULL");
  if (depth) *depth = e->depth;
  if (seg_rows) *seg_rows = e->seg_rows;
  return SSLBM_OK;
}

int sslbm_ensemble_set_wait_limit(sslbm_ensemble* e, long long spin_limit, long long stall_item) {
  if (!e) return err(SSLBM_ERR_BAD_ARG, "ensemble is NULL");
  if (spin_limit < 0) return err(SSLBM_ERR_BAD_ARG, "spin_limit < 0");
  e->spin_limit = spin_limit;
  e->stall_item = stall_item;
  if (e->exec) {
    cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
    e->exec_blocks = -1;
  }
  return SSLBM_OK;
}

int sslbm_ensemble_write(sslbm_ensemble* e, int idx, const void* src, int src_dtype, int on_device) {
  if (!e || !src) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  if (idx < 0 || idx >= e->n) return err(SSLBM_ERR_BAD_ARG, "scenario %d out of range", idx);
  if (src_dtype != SSLBM_DT_F64 && src_dtype != SSLBM_DT_F32)
    return err(SSLBM_ERR_BAD_ARG, "dtype %d", src_dtype);
  DevGuard dg(e->device);
  const GridView g = e->gv(idx);
  const size_t bytes = (size_t)g.nx * g.ny * (src_dtype == SSLBM_DT_F64 ? 8 : 4);
  char* staging = reinterpret_cast<char*>(e->plane(1 - e->cur, idx, 0));
  for (int c = 0; c < 5; ++c) {
    const char* s = static_cast<const char*>(src) + c * bytes;
    cudaError_t ce;
    if (!on_device) {
      ce = cudaMemcpyAsync(staging, s, bytes, cudaMemcpyHostToDevice, e->stream);
      if (ce != cudaSuccess) return cuda_err(ce, "cudaMemcpyAsync(H2D)");
      s = staging;
    }
    const int dev_S = (e->precision == SSLBM_FP32_DEV && c == 0) ? 1 : 0;
    void* comp = (e->precision == SSLBM_FP32_SPLIT && c == 0) ? e->plane(e->cur, idx, 5) : nullptr;
    ce = sslbm::launch_plane_write(SSLBM_FP32, g, s, src_dtype, e->plane(e->cur, idx, c), comp, dev_S,
                                   e->sc[idx].s_ref, e->stream);
    if (ce != cudaSuccess) return cuda_err(ce, "plane write");
  }
  if (!on_device) {
    cudaError_t ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) return cuda_err(ce, "cudaStreamSynchronize");
  }
  return SSLBM_OK;
}

int sslbm_ensemble_read(sslbm_ensemble* e, int idx, void* dst, int dst_dtype, int on_device) {
  if (!e || !dst) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  if (idx < 0 || idx >= e->n) return err(SSLBM_ERR_BAD_ARG, "scenario %d out of range", idx);
  if (dst_dtype != SSLBM_DT_F64 && dst_dtype != SSLBM_DT_F32)
    return err(SSLBM_ERR_BAD_ARG, "dtype %d", dst_dtype);
  DevGuard dg(e->device);
  const GridView g = e->gv(idx);
  const size_t bytes = (size_t)g.nx * g.ny * (dst_dtype == SSLBM_DT_F64 ? 8 : 4);
  char* staging = reinterpret_cast<char*>(e->plane(1 - e->cur, idx, 0));
  for (int c = 0; c < 5; ++c) {
    char* d = static_cast<char*>(dst) + c * bytes;
    const int dev_S = (e->precision == SSLBM_FP32_DEV && c == 0) ? 1 : 0;
    const void* comp = (e->precision == SSLBM_FP32_SPLIT && c == 0) ? e->plane(e->cur, idx, 5) : nullptr;
    cudaError_t ce = sslbm::launch_plane_read(SSLBM_FP32, g, e->plane(e->cur, idx, c), comp, dev_S,
                                              e->sc[idx].s_ref, on_device ? d : staging, dst_dtype,
                                              e->stream);
    if (ce != cudaSuccess) return cuda_err(ce, "plane read");
    if (!on_device) {
      ce = cudaMemcpyAsync(d, staging, bytes, cudaMemcpyDeviceToHost, e->stream);
      if (ce != cudaSuccess) return cuda_err(ce, "cudaMemcpyAsync(D2H)");
    }
  }
  cudaError_t ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaStreamSynchronize");
  return SSLBM_OK;
}

int sslbm_ensemble_run(sslbm_ensemble* e, int64_t nsteps) {
  if (!e) return err(SSLBM_ERR_BAD_ARG, "ensemble is NULL");
  if (nsteps < 0) return err(SSLBM_ERR_BAD_ARG, "nsteps < 0");
  if (nsteps == 0) return SSLBM_OK;
  DevGuard dg(e->device);
  const int64_t full = nsteps / e->depth;
  const int rem = (int)(nsteps % e->depth);
  if (full > 0x7fffffff) return err(SSLBM_ERR_BAD_ARG, "too many steps for one run");
  int st = launch_blocks(e, (int)full);
  if (st) return st;
  if (rem) {
    // remaining steps: one-step launches per scenario (same bits as fused steps)
    for (int r = 0; r < rem; ++r) {
      for (int i = 0; i < e->n; ++i) {
        cudaError_t ce = sslbm::launch_sslbm_step1(e->precision, e->gv(i), &e->tab[i].k,
                                                   e->buf(e->cur) + e->L.elem_off[i],
                                                   e->buf(1 - e->cur) + e->L.elem_off[i], e->stream);
        if (ce != cudaSuccess) return cuda_err(ce, "remainder step");
      }
      e->cur = 1 - e->cur;
    }
  }
  e->steps += nsteps;
  return full > 0 ? check_error_flag(e) : SSLBM_OK;
}

int sslbm_ensemble_diagnostics(sslbm_ensemble* e, double* totals, double* peak_I) {
  if (!e) return err(SSLBM_ERR_BAD_ARG, "ensemble is NULL");
  DevGuard dg(e->device);
  double* partials = reinterpret_cast<double*>(e->ws + e->L.off_partials);
  double* results = reinterpret_cast<double*>(e->ws + e->L.off_results);
  for (int i = 0; i < e->n; ++i) {
    const bool split = e->precision == SSLBM_FP32_SPLIT;  // S = value - compensation (plane 5)
    cudaError_t ce = sslbm::launch_diagnostics(SSLBM_FP32, 0, e->gv(i), e->plane(e->cur, i, 0),
                                               split ? e->plane(e->cur, i, 5) : nullptr, partials,
                                               results + (size_t)i * sslbm::kDiagSlots, e->stream, 1);
    if (ce != cudaSuccess) return cuda_err(ce, "diagnostics");
  }
  std::vector<double> r((size_t)e->n * sslbm::kDiagSlots);
  cudaError_t ce = cudaMemcpyAsync(r.data(), results, r.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                   e->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return cuda_err(ce, "diagnostics copy");
  int status = SSLBM_OK;
  for (int i = 0; i < e->n; ++i) {
    double* ri = &r[(size_t)i * sslbm::kDiagSlots];
    if (e->precision == SSLBM_FP32_DEV) ri[0] = e->sc[i].s_ref * (double)e->sc[i].nx * (double)e->sc[i].ny - ri[0];
    for (int c = 0; c < 5; ++c) {
      if (totals) totals[(size_t)i * 5 + c] = ri[c];
      if (!std::isfinite(ri[c])) status = SSLBM_ERR_NONFINITE;
    }
    if (peak_I) peak_I[i] = ri[5];
  }
  if (status) return err(status, "non-finite total in the ensemble");
  return SSLBM_OK;
}

int sslbm_ensemble_autotune(sslbm_ensemble* e, int trial_blocks, int* depth_out, int* seg_out,
                            double* ms_per_step_out) {
  if (!e) return err(SSLBM_ERR_BAD_ARG, "ensemble is NULL");
  if (trial_blocks <= 0) trial_blocks = 3;
  DevGuard dg(e->device);
  const int depths[5] = {2, 3, 4, 6, 8};
  const int segs[4] = {32, 64, 128, 256};
  int best_d = e->depth, best_s = e->seg_rows;
  double best = 1e300;
  cudaEvent_t a, b;
  cudaError_t ce = cudaEventCreate(&a);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaEventCreate");
  ce = cudaEventCreate(&b);
  if (ce != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_err(ce, "cudaEventCreate");
  }
  int st = SSLBM_OK;
  for (int d : depths) {
    for (int sg : segs) {
      if (sg < 4 * d) continue;
      e->depth = d;
      e->seg_rows = sg;
      st = upload_table(e);
      if (!st) st = launch_blocks(e, trial_blocks);  // capture + warm-up
      if (!st) {
        ce = cudaEventRecord(a, e->stream);
        if (ce == cudaSuccess) st = launch_blocks(e, trial_blocks);
        if (!st && ce == cudaSuccess) ce = cudaEventRecord(b, e->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(b);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, b);
        if (ce != cudaSuccess) st = cuda_err(ce, "ensemble autotune timing");
        if (!st) st = check_error_flag(e);
        const double per_step = (double)ms / (double)(trial_blocks * d);
        if (!st && per_step < best) {
          best = per_step;
          best_d = d;
          best_s = sg;
        }
      }
      if (st) break;
    }
    if (st) break;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st) return st;
  e->depth = best_d;
  e->seg_rows = best_s;
  st = upload_table(e);
  if (st) return st;
  // the trials advanced the states: start again from zero
  ce = cudaMemsetAsync(e->ws + e->L.off_buf[0], 0, e->L.total - e->L.off_buf[0], e->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return cuda_err(ce, "ensemble reset");
  e->cur = 0;
  e->steps = 0;
  if (depth_out) *depth_out = best_d;
  if (seg_out) *seg_out = best_s;
  if (ms_per_step_out) *ms_per_step_out = best;
  return SSLBM_OK;
}

int64_t sslbm_ensemble_steps_done(const sslbm_ensemble* e) { return e ? e->steps : -1; }

}  // extern "C"

namespace {
constexpr uint32_t kEnsCkptMagic = 0x454C5353u;  // the bytes "SSLE"
constexpr uint32_t kEnsCkptVersion = 2;
struct EnsCkptHeader {
  uint32_t magic, version;
  int32_t n, precision;
  int64_t steps;
  int64_t reserved[5];
};
static_assert(sizeof(EnsCkptHeader) == 64, "ensemble checkpoint header");

// header, then (nx, ny, s_ref) of every scenario (two int64 and a double: s_ref is the
// reference of the FP32_DEV storage, sigma = s_ref - S), then the planes from this offset
constexpr size_t kEnsCkptEntry = 24;
size_t ens_ckpt_data_offset(int n) {
  return (sizeof(EnsCkptHeader) + (size_t)n * kEnsCkptEntry + 127) / 128 * 128;
}

size_t ens_ckpt_bytes(const sslbm_ensemble* e) {
  size_t b = ens_ckpt_data_offset(e->n);
  for (int i = 0; i < e->n; ++i) b += (size_t)ens_planes(e->precision) * e->sc[i].nx * e->sc[i].ny * sizeof(float);
  return b;
}
}  // namespace

extern "C" {

int sslbm_ensemble_checkpoint_bytes(const sslbm_ensemble* e, size_t* bytes) {
  if (!e || !bytes) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  *bytes = ens_ckpt_bytes(e);
  return SSLBM_OK;
}

int sslbm_ensemble_checkpoint_save(sslbm_ensemble* e, void* dst, size_t bytes, int dst_on_device) {
  if (!e || !dst) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  const size_t need = ens_ckpt_bytes(e);
  if (bytes < need) return err(SSLBM_ERR_BAD_ARG, "checkpoint buffer of %zu bytes < %zu", bytes, need);
  DevGuard dg(e->device);
  const size_t data = ens_ckpt_data_offset(e->n);
  std::vector<unsigned char> head(data, 0);
  EnsCkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  hd.magic = kEnsCkptMagic;
  hd.version = kEnsCkptVersion;
  hd.n = e->n;
  hd.precision = e->precision;
  hd.steps = e->steps;
  std::memcpy(head.data(), &hd, sizeof(hd));
  for (int i = 0; i < e->n; ++i) {
    const int64_t dims[2] = {e->sc[i].nx, e->sc[i].ny};
    const double sref = e->sc[i].s_ref;
    unsigned char* ent = head.data() + sizeof(hd) + (size_t)i * kEnsCkptEntry;
    std::memcpy(ent, dims, 16);
    std::memcpy(ent + 16, &sref, 8);
  }
  cudaError_t ce;
  if (dst_on_device) {
    ce = cudaMemcpyAsync(dst, head.data(), data, cudaMemcpyHostToDevice, e->stream);
    if (ce != cudaSuccess) return cuda_err(ce, "cudaMemcpyAsync(checkpoint header)");
  } else {
    std::memcpy(dst, head.data(), data);
  }
  char* d = static_cast<char*>(dst) + data;
  for (int i = 0; i < e->n; ++i) {
    const GridView g = e->gv(i);
    const size_t row = (size_t)g.nx * sizeof(float);
    for (int c = 0; c < ens_planes(e->precision); ++c, d += row * (size_t)g.ny) {
      ce = cudaMemcpy2DAsync(d, row, e->plane(e->cur, i, c), (size_t)g.pitch * sizeof(float), row, (size_t)g.ny,
                             dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, e->stream);
      if (ce != cudaSuccess) return cuda_err(ce, "cudaMemcpy2DAsync(checkpoint save)");
    }
  }
  ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaStreamSynchronize(checkpoint save)");
  return SSLBM_OK;
}

int sslbm_ensemble_checkpoint_load(sslbm_ensemble* e, const void* src, size_t bytes, int src_on_device) {
  if (!e || !src) return err(SSLBM_ERR_BAD_ARG, "NULL argument");
  const size_t data = ens_ckpt_data_offset(e->n);
  if (bytes < sizeof(EnsCkptHeader)) return err(SSLBM_ERR_BAD_ARG, "checkpoint of %zu bytes has no header", bytes);
  DevGuard dg(e->device);
  EnsCkptHeader hd;
  cudaError_t ce;
  if (src_on_device) {
    ce = cudaMemcpyAsync(&hd, src, sizeof(hd), cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) return cuda_err(ce, "checkpoint header");
  } else {
    std::memcpy(&hd, src, sizeof(hd));
  }
  if (hd.magic != kEnsCkptMagic || hd.version != kEnsCkptVersion)
    return err(SSLBM_ERR_BAD_ARG, "not an ensemble checkpoint of this format (magic %08x, version %u)", hd.magic,
               hd.version);
  if (hd.n != e->n || hd.precision != e->precision)
    return err(SSLBM_ERR_BAD_ARG, "checkpoint of %d scenarios (precision %d) for an ensemble of %d (precision %d)", hd.n,
               hd.precision, e->n, e->precision);
  if (hd.steps < 0) return err(SSLBM_ERR_BAD_ARG, "negative step counter");
  const size_t need = ens_ckpt_bytes(e);
  if (bytes < need) return err(SSLBM_ERR_BAD_ARG, "checkpoint of %zu bytes < %zu", bytes, need);
  std::vector<unsigned char> tab((size_t)e->n * kEnsCkptEntry);
  const char* tsrc = static_cast<const char*>(src) + sizeof(hd);
  if (src_on_device) {
    ce = cudaMemcpyAsync(tab.data(), tsrc, tab.size(), cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) return cuda_err(ce, "checkpoint scenario table");
  } else {
    std::memcpy(tab.data(), tsrc, tab.size());
  }
  for (int i = 0; i < e->n; ++i) {
    int64_t dims[2];
    double sref;
    std::memcpy(dims, tab.data() + (size_t)i * kEnsCkptEntry, 16);
    std::memcpy(&sref, tab.data() + (size_t)i * kEnsCkptEntry + 16, 8);
    if (dims[0] != e->sc[i].nx || dims[1] != e->sc[i].ny)
      return err(SSLBM_ERR_BAD_ARG, "scenario %d: checkpoint grid %lld x %lld, ensemble grid %lld x %lld", i,
                 (long long)dims[0], (long long)dims[1], (long long)e->sc[i].nx, (long long)e->sc[i].ny);
    if (e->precision == SSLBM_FP32_DEV && sref != e->sc[i].s_ref)
      return err(SSLBM_ERR_BAD_ARG,
                 "scenario %d: checkpoint stores S as a deviation from s_ref = %.17g, the ensemble's is %.17g", i,
                 sref, e->sc[i].s_ref);
  }
  const char* s = static_cast<const char*>(src) + data;
  for (int i = 0; i < e->n; ++i) {
    const GridView g = e->gv(i);
    const size_t row = (size_t)g.nx * sizeof(float);
    for (int c = 0; c < ens_planes(e->precision); ++c, s += row * (size_t)g.ny) {
      ce = cudaMemcpy2DAsync(e->plane(e->cur, i, c), (size_t)g.pitch * sizeof(float), s, row, row, (size_t)g.ny,
                             src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, e->stream);
      if (ce != cudaSuccess) return cuda_err(ce, "cudaMemcpy2DAsync(checkpoint load)");
    }
  }
  if (!src_on_device) {
    ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) return cuda_err(ce, "cudaStreamSynchronize(checkpoint load)");
  }
  e->steps = hd.steps;
  return SSLBM_OK;
}

}  // extern "C"

namespace sslbm {

int ensemble_count(const sslbm_ensemble* e) { return e ? e->n : -1; }

int ensemble_grid(const sslbm_ensemble* e, int idx, int64_t* nx, int64_t* ny) {
  if (!e || idx < 0 || idx >= e->n || !nx || !ny) return SSLBM_ERR_BAD_ARG;
  *nx = e->sc[idx].nx;
  *ny = e->sc[idx].ny;
  return SSLBM_OK;
}

}  // namespace sslbm
