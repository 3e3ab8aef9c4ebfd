// sslbm_internal.cuh -- internal definitions shared by the libsslbm translation units.
//
// Field layout in device memory: each plane (one compartment, or one BGK population
// of one compartment) holds ny rows of `pitch` elements, x fastest; pitch is nx
// rounded up to 32 elements so every row starts on a 128-byte boundary (FP32) and
// vector loads never straddle rows.  Cells with x >= nx are padding, kept at zero
// and never read as neighbours.  Planes are `plane` elements apart (pitch*ny rounded
// up to 64 elements, i.e. 256-byte aligned for both precisions).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sslbm.h"

namespace sslbm {

// MODE_D2Q9 / MODE_D2Q9_NOFLUX: the plain FP32 storage on the D2Q9 lattice (the nine-point
// laplacian), periodic or with bounce-back walls, for the temporal-blocked pipeline.
// MODE_VARD: the plain FP32 storage with spatially varying diffusion (the flux form).
enum Mode {
  MODE_PLAIN = 0,
  MODE_DEV = 1,
  MODE_KAHAN = 2,
  MODE_SPLIT = 3,
  MODE_D2Q9 = 4,
  MODE_D2Q9_NOFLUX = 5,
  MODE_VARD = 6,
  MODE_D2Q9_NOFLUX4 = 7  // no-flux with nx a multiple of 4: x = nx - 1 ends a lane's four columns
};

// Stored planes per state of a mode: the five compartments, plus the compensation of S
// (MODE_SPLIT) or of all five (MODE_KAHAN), which follow them.
template <int MODE>
constexpr int mode_planes() {
  return MODE == MODE_KAHAN ? 10 : MODE == MODE_SPLIT ? 6 : 5;
}

struct GridView {
  int64_t nx, ny, pitch, plane;
  int bc;  // 0 periodic, 1 no-flux
};

// Per-step constants of the SSLBM / BGK updates in lattice form.
//   dl[c]  lattice diffusivity d dt/dx^2 = (tau - 1/2)/3 (Eq. diffusivity)
//   bdt    beta dt,  adt alpha dt,  gdt gamma dt,
//   rdt    (1 - phi) gamma dt (inflow of R),  ddt phi gamma dt (inflow of D)
//   s_ref  reference value of S for the deviation storage
//   itau   1/tau (BGK collision)
template <typename T>
struct Coeffs {
  T dl[4];
  T itau[4];
  T bdt, adt, gdt, rdt, ddt;
  T s_ref;
};

// Map a row/column index that left [0, n) by at most one link (periodic wrap or the
// cell-centred mirror, whose ghost equals the boundary cell).
__device__ __forceinline__ int64_t link_index(int64_t i, int64_t n, int bc) {
  if (i < 0) return bc == 0 ? i + n : 0;
  if (i >= n) return bc == 0 ? i - n : n - 1;
  return i;
}

// Map any index onto [0, n) for ghost layers of arbitrary width: periodic wrap, or the
// even extension about the faces (period 2n), which is what repeated cell-centred
// mirroring produces.  Evolving such a ghost layer with the same stencil keeps it the
// mirror image of the interior, so interior results equal those of per-step mirroring.
__device__ __forceinline__ int64_t ghost_index(int64_t i, int64_t n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 0) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
  }
  int64_t p = 2 * n;
  int64_t r = i % p;
  if (r < 0) r += p;
  return r < n ? r : p - 1 - r;
}

// Explicitly rounded operations: the per-cell arithmetic is spelled out with fma and
// _rn intrinsics so the compiler has no freedom to contract or reorder it, and every
// kernel that uses these helpers produces the same bits for the same cell.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
// Force of infection times dt, beta S I / N_c dt (Eq. sources).  The quotient is taken
// against max(N_c, smallest normal): for nonnegative states N_c = 0 forces S = I = 0, so
// the force is 0 there -- the reading used for the case the paper leaves open -- without
// a branch.  FP32 multiplies by the hardware reciprocal (rcp.approx, <= 1 ulp).  FP64, whose
// arithmetic rate bounds every FP64 kernel here, refines a float reciprocal seed by two
// Newton-Raphson steps (relative error ~1e-7, then ~1e-14, then below the double rounding)
// and corrects the quotient with its exact FMA remainder (Markstein, IBM J. Res. Dev. 34,
// 1990): within one ulp of the IEEE quotient, and equal to it except near ties.  Divisors
// outside the float seed's range take the IEEE division.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float force_quot(float num, float Nc) {
  return __fmul_rn(num, rcp_approx(fmaxf(Nc, 1.17549435e-38f)));
}
__device__ __forceinline__ double force_quot(double num, double Nc) {
  const double d = fmax(Nc, 2.2250738585072014e-308);
  if (!(d > 1e-30 && d < 1e30)) return __ddiv_rn(num, d);
  double r = (double)rcp_approx(__double2float_rn(d));
  r = __fma_rn(r, __fma_rn(-d, r, 1.0), r);
  r = __fma_rn(r, __fma_rn(-d, r, 1.0), r);
  const double q = __dmul_rn(num, r);
  return __fma_rn(r, __fma_rn(-d, q, num), q);
}

template <typename T>
__device__ __forceinline__ T force_dt(const Coeffs<T>& k, T S, T E, T I, T R) {
  const T Nc = add_rn(add_rn(S, E), add_rn(I, R));
  const T num = mul_rn(mul_rn(k.bdt, S), I);
  return force_quot(num, Nc);
}

// Neighbour sum minus four times the centre.  On D2Q5 rho_f = rho_b = rho_c/3 + (sum of
// the four neighbours)/6, so Eq. (sslbm_final_clean) equals
//   rho_c + (2 tau - 1)/6 * (l + r + u + d - 4 rho_c) + Psi dt = rho_c + d_lattice * lap.
template <typename T>
__device__ __forceinline__ T lap5(T c, T l, T r, T u, T d) {
  return fma_rn(T(-4), c, add_rn(add_rn(l, r), add_rn(u, d)));
}

// The same neighbour sum formed from differences to the centre: for a nearly constant
// field (S ~ 1) each difference is exact (Sterbenz), so the laplacian keeps full relative
// accuracy where (l + r) + (u + d) - 4c would lose ~1e-7 absolute.  Used by the
// compensated (Kahan) variant, whose memory-bound kernel has ALU to spare.
__device__ __forceinline__ float lap5_diff(float c, float l, float r, float u, float d) {
  return __fadd_rn(__fadd_rn(__fsub_rn(l, c), __fsub_rn(r, c)),
                   __fadd_rn(__fsub_rn(u, c), __fsub_rn(d, c)));
}

// Increments of S, E, I, R, D of one cell over one step (Eq. sslbm_final_clean in
// reduced form with Eq. sources; Eq. rhoD): d_lattice * lap + Psi dt.
template <typename T>
__device__ __forceinline__ void seird_cell(const Coeffs<T>& k, T S, T E, T I, T R, T D, T lS, T lE,
                                           T lI, T lR, T& nS, T& nE, T& nI, T& nR, T& nD) {
  const T F = force_dt(k, S, E, I, R);
  nS = sub_rn(fma_rn(k.dl[0], lS, S), F);
  nE = add_rn(fma_rn(k.dl[1], lE, E), fma_rn(-k.adt, E, F));
  nI = add_rn(fma_rn(k.dl[2], lI, I), fma_rn(k.adt, E, -mul_rn(k.gdt, I)));
  nR = fma_rn(k.rdt, I, fma_rn(k.dl[3], lR, R));
  nD = fma_rn(k.ddt, I, D);
}

// Deviation storage: plane 0 holds sigma = s_ref - S.  The laplacian of sigma is minus
// that of S (the constant s_ref is annihilated exactly), so
// sigma' = sigma + d lap(sigma) + F dt.
template <typename T>
__device__ __forceinline__ void seird_cell_dev(const Coeffs<T>& k, T sig, T E, T I, T R, T D,
                                               T lsig, T lE, T lI, T lR, T& nsig, T& nE, T& nI,
                                               T& nR, T& nD) {
  const T S = sub_rn(k.s_ref, sig);
  const T F = force_dt(k, S, E, I, R);
  nsig = add_rn(fma_rn(k.dl[0], lsig, sig), F);
  nE = add_rn(fma_rn(k.dl[1], lE, E), fma_rn(-k.adt, E, F));
  nI = add_rn(fma_rn(k.dl[2], lI, I), fma_rn(k.adt, E, -mul_rn(k.gdt, I)));
  nR = fma_rn(k.rdt, I, fma_rn(k.dl[3], lR, R));
  nD = fma_rn(k.ddt, I, D);
}

// Compensated (Kahan) accumulation of an increment: value v, running compensation c
// (the part of earlier increments lost to rounding, with the sign Kahan's algorithm
// gives it: the represented value is v - c).
__device__ __forceinline__ void kahan_add(float& v, float& c, float inc) {
  const float y = __fsub_rn(inc, c);
  const float t = __fadd_rn(v, y);
  c = __fsub_rn(__fsub_rn(t, v), y);
  v = t;
}

// Split storage of S (MODE_SPLIT): S = v - c with v the FP32 value plane and c its FP32
// compensation plane, a hi/lo pair carrying about twice FP32's precision.  The laplacian of
// S is lap5_diff(v) - lap5_diff(c); the force uses v; the increment is added to (v, c) with
// kahan_add; E, I, R and D take the plain update of seird_cell.
__device__ __forceinline__ void seird_cell_split(const Coeffs<float>& k, float v, float c, float E, float I,
                                                 float R, float D, float lS, float lE, float lI, float lR,
                                                 float& nv, float& nc, float& nE, float& nI, float& nR,
                                                 float& nD) {
  const float F = force_dt(k, v, E, I, R);
  nv = v;
  nc = c;
  kahan_add(nv, nc, fma_rn(k.dl[0], lS, -F));
  nE = add_rn(fma_rn(k.dl[1], lE, E), fma_rn(-k.adt, E, F));
  nI = add_rn(fma_rn(k.dl[2], lI, I), fma_rn(k.adt, E, -mul_rn(k.gdt, I)));
  nR = fma_rn(k.rdt, I, fma_rn(k.dl[3], lR, R));
  nD = fma_rn(k.ddt, I, D);
}

// Increments of S, E, I, R, D for the Kahan variant (same expressions as seird_cell).
__device__ __forceinline__ void seird_increments(const Coeffs<float>& k, float S, float E, float I,
                                                 float R, float lS, float lE, float lI, float lR,
                                                 float inc[5]) {
  const float F = force_dt(k, S, E, I, R);
  inc[0] = fma_rn(k.dl[0], lS, -F);
  inc[1] = add_rn(mul_rn(k.dl[1], lE), fma_rn(-k.adt, E, F));
  inc[2] = add_rn(mul_rn(k.dl[2], lI), fma_rn(k.adt, E, -mul_rn(k.gdt, I)));
  inc[3] = fma_rn(k.rdt, I, mul_rn(k.dl[3], lR));
  inc[4] = mul_rn(k.ddt, I);
}

// ---- packed FP32 (two cells per instruction) ---------------------------------------
// __fadd2_rn / __fmul2_rn / __ffma2_rn round each component exactly like the scalar
// __fadd_rn / __fmul_rn / __fmaf_rn, and a - b is a + (-b) exactly, so the packed cell
// update below gives the same bits as seird_cell / seird_cell_dev on each component.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// lap5 on two cells: lr = l + r (formed by the caller), u, d the rows above and below.
__device__ __forceinline__ float2 lap5x2(float2 c, float2 lr, float2 u, float2 d) {
  return fma2(splat2(-4.f), c, add2(lr, add2(u, d)));
}

__device__ __forceinline__ float2 force_dt2(const Coeffs<float>& k, float2 S, float2 E, float2 I,
                                            float2 R) {
  const float2 Nc = add2(add2(S, E), add2(I, R));
  const float2 num = mul2(mul2(splat2(k.bdt), S), I);
  const float2 r = make_float2(rcp_approx(fmaxf(Nc.x, 1.17549435e-38f)),
                               rcp_approx(fmaxf(Nc.y, 1.17549435e-38f)));
  return mul2(num, r);
}

// lap5_diff on two cells: l, r the left and right neighbours (formed by the caller), u, d the
// rows above and below; the same operations, in the same order, as lap5_diff.
__device__ __forceinline__ float2 lap5diff_x2(float2 c, float2 l, float2 r, float2 u, float2 d) {
  const float2 nc = neg2(c);
  return add2(add2(add2(l, nc), add2(r, nc)), add2(add2(u, nc), add2(d, nc)));
}

// kahan_add on two cells.
__device__ __forceinline__ void kahan_add2(float2& v, float2& c, float2 inc) {
  const float2 y = add2(inc, neg2(c));
  const float2 t = add2(v, y);
  c = add2(add2(t, neg2(v)), neg2(y));
  v = t;
}

// seird_cell_split on two cells (x0 = v, xc = c of S; l0 the laplacian of S).
__device__ __forceinline__ void seird_cell2_split(const Coeffs<float>& k, float2 x0, float2 xc, float2 E, float2 I,
                                                  float2 R, float2 D, float2 l0, float2 lE, float2 lI, float2 lR,
                                                  float2& n0, float2& nc, float2& nE, float2& nI, float2& nR,
                                                  float2& nD) {
  const float2 F = force_dt2(k, x0, E, I, R);
  n0 = x0;
  nc = xc;
  kahan_add2(n0, nc, fma2(splat2(k.dl[0]), l0, neg2(F)));
  nE = add2(fma2(splat2(k.dl[1]), lE, E), fma2(splat2(-k.adt), E, F));
  nI = add2(fma2(splat2(k.dl[2]), lI, I), fma2(splat2(k.adt), E, neg2(mul2(splat2(k.gdt), I))));
  nR = fma2(splat2(k.rdt), I, fma2(splat2(k.dl[3]), lR, R));
  nD = fma2(splat2(k.ddt), I, D);
}

// MODE 0: plain storage (x0 = S); MODE 1: deviation storage (x0 = sigma = s_ref - S).
template <int DEV>
__device__ __forceinline__ void seird_cell2(const Coeffs<float>& k, float2 x0, float2 E, float2 I,
                                            float2 R, float2 D, float2 l0, float2 lE, float2 lI,
                                            float2 lR, float2& n0, float2& nE, float2& nI,
                                            float2& nR, float2& nD) {
  const float2 S = DEV ? add2(splat2(k.s_ref), neg2(x0)) : x0;
  const float2 F = force_dt2(k, S, E, I, R);
  n0 = DEV ? add2(fma2(splat2(k.dl[0]), l0, x0), F) : add2(fma2(splat2(k.dl[0]), l0, x0), neg2(F));
  nE = add2(fma2(splat2(k.dl[1]), lE, E), fma2(splat2(-k.adt), E, F));
  nI = add2(fma2(splat2(k.dl[2]), lI, I), fma2(splat2(k.adt), E, neg2(mul2(splat2(k.gdt), I))));
  nR = fma2(splat2(k.rdt), I, fma2(splat2(k.dl[3]), lR, R));
  nD = fma2(splat2(k.ddt), I, D);
}

// ---- launchers (defined in the kernel translation units) --------------------------
// SSLBM: one step per launch (every precision) and K fused steps per launch (FP32, FP32
// deviation-S, FP32 split-S and FP32 Kahan).  seg_rows > 0 is the blocked kernel's row-segment
// length.
cudaError_t launch_sslbm_step1(int precision, const GridView& g, const void* coeffs, const void* in,
                               void* out, cudaStream_t s);
// The streaming one-step kernel (stream.cu) of the FP32 storages: FP32, FP32 deviation-S,
// FP32 split-S and the Kahan storage.
cudaError_t launch_stream_d2q5(int precision, const GridView& g, const void* coeffs, const void* in, void* out,
                               cudaStream_t s);
cudaError_t launch_sslbm_blocked(int precision, const GridView& g, const void* coeffs,
                                 const void* in, void* out, int depth, int seg_rows,
                                 cudaStream_t s);
bool blocked_supported(int precision, const GridView& g);
// The Kahan storage's blocked kernel (pipe_kahan.cu) and its default segment.
cudaError_t launch_kahan_blocked(const GridView& g, const void* coeffs, const void* in, void* out, int depth,
                                 int seg_rows, cudaStream_t s);
int blocked_kahan_default_seg_rows(const GridView& g, int depth);
// The D2Q9 lattice (plain FP32 storage): K fused steps per launch, and its default segment.
cudaError_t launch_sslbm9_blocked(const GridView& g, const void* coeffs, const void* in, void* out, int depth,
                                  int seg_rows, cudaStream_t s);
int blocked9_default_seg_rows(const GridView& g, int depth);
// ... under no-flux with nx a multiple of 4 (pipe_d2q9_aligned.cu)
cudaError_t launch_sslbm9_aligned_blocked(const GridView& g, const void* coeffs, const void* in, void* out,
                                          int depth, int seg_rows, cudaStream_t s);
int blocked9_aligned_default_seg_rows(const GridView& g, int depth);
// The varying-diffusion lattice (plain FP32 storage, scale planes kx, ky): K fused steps per
// launch, and its default segment.
cudaError_t launch_sslbm_vard_blocked(const GridView& g, const void* coeffs, const void* kx, const void* ky,
                                      const void* in, void* out, int depth, int seg_rows, cudaStream_t s);
int blocked_vard_default_seg_rows(const GridView& g, int depth);
// Segment length that makes one blocked launch a single wave of resident warps.
int blocked_default_seg_rows(int precision, const GridView& g, int depth);
// The same pass with the fused diagnostics (FP32 and FP32_DEV storages, at most kDiagBlocks
// CTAs): partials receives one 6-double partial per CTA (the five totals of the stored planes,
// then the largest I), which launch_diag_final reduces.  blocked_ctas: the CTAs of such a pass
// (-1 for an invalid depth or segment length).
int64_t blocked_ctas(const GridView& g, int depth, int seg_rows);
bool blocked_diag_supported(int precision, const GridView& g, int depth, int seg_rows);
cudaError_t launch_sslbm_blocked_diag(int precision, const GridView& g, const void* coeffs, const void* in,
                                      void* out, int depth, int seg_rows, double* partials, cudaStream_t s);
// BGK: one collide-and-stream step; equilibrium initialisation and density of one
// compartment from / to a contiguous ny x nx plane of type rho_dtype.
cudaError_t launch_bgk_step(int precision, const GridView& g, const void* coeffs, const void* f_in,
                            void* f_out, cudaStream_t s);
cudaError_t launch_bgk_init(int precision, const GridView& g, int comp, const void* rho,
                            int rho_dtype, void* f, cudaStream_t s);
cudaError_t launch_bgk_density(int precision, const GridView& g, int comp, const void* f, void* rho,
                               int rho_dtype, cudaStream_t s);
// plane <-> contiguous user layout (dev_S: deviation storage of S; comp_plane: compensation
// of the Kahan or split storage, the FP32 rounding residue of the value on write (so that
// value - compensation reproduces the input) and subtracted on read)
cudaError_t launch_plane_write(int precision, const GridView& g, const void* src, int src_dtype,
                               void* plane, void* comp_plane, int dev_S, double s_ref,
                               cudaStream_t s);
cudaError_t launch_plane_read(int precision, const GridView& g, const void* plane,
                              const void* comp_plane, int dev_S, double s_ref, void* dst,
                              int dst_dtype, cudaStream_t s);
// diagnostics: per-block partial sums of the 5 compartments and max of I into `partials`
// (kDiagBlocks x kDiagSlots doubles), then their fixed-order total into result[6].
// layout 0: SSLBM planes; layout 1: BGK populations.
constexpr int kDiagBlocks = 1024;
constexpr int kDiagSlots = 6;
// comp_planes: the compensation planes of the first n_comp compartments (5 for the Kahan
// storage, 1 for the split storage of S), subtracted from the values; NULL for none.
cudaError_t launch_diagnostics(int precision, int layout, const GridView& g, const void* planes,
                               const void* comp_planes, double* partials, double* result,
                               cudaStream_t s, int n_comp = 5);
// The fixed-order FP64 total of nblocks 6-double partials into result[6] (one CTA).
cudaError_t launch_diag_final(const double* partials, int nblocks, double* result, cudaStream_t s);

}  // namespace sslbm
