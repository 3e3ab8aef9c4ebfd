// sslbm_pipe.cuh -- one tile of the temporal-blocked SSLBM pipeline (FP32 variants),
// shared by the single-grid launch (sslbm_kernels.cu) and the persistent ensemble launch
// (ensemble.cu).
//
// A tile is a 128-column strip (4 columns per lane, 16-byte accesses; K columns of halo
// on each side are recomputed) times a segment of rows [y0, y1), advanced K steps.  The
// CTA's K warps form a pipeline over the time levels: warp s computes level s+1 of the
// wavefront, two rows per iteration.  Warp 0 brings level-0 rows in with cp.async into a
// shared-memory ring three row pairs ahead; each level's output pair goes through a
// double-buffered shared-memory slot to the next warp, one CTA barrier per pair; the last
// warp writes level K to global memory.  Each warp keeps its own level's rows in four
// register buffers (the two previous rows and the arriving pair) whose roles rotate, so no
// row is copied.  x neighbours come from warp shuffles.  Rows and columns outside the domain
// are loaded as ghost images (periodic wrap or the even mirror extension), which the
// uniform stencil keeps consistent, so no boundary logic is needed inside the pipeline.
// The arithmetic is the packed form of seird_cell / seird_cell_dev / seird_cell_split,
// bit-identical to the one-step kernel; the split storage of S carries its compensation as a
// sixth plane through the pipeline.  On the D2Q9 lattice (cell_row9) the row update is the
// nine-point one of the one-step D2Q9 kernel; its no-flux walls (bounce-back) are not a ghost
// image, so they are substituted into the row update instead.
#pragma once
#include <cfloat>

#include "bounds.cuh"
#include "sslbm_internal.cuh"

namespace sslbm {

constexpr int kRing0 = 8;  // level-0 rows per tile in the ring: four pairs, three in flight

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// Asynchronous global -> shared copies (cp.async): 16 bytes bypassing L1, or 4 bytes.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// r0: level-0 rows (warp 0's lanes read back exactly what they copied);
// rl[s-1]: the pair of level-s rows from warp s-1 to warp s, double-buffered by iteration
// parity.  Over 48 KB from K = 5 on: the kernels take it as dynamic shared memory.
// NF = the planes a state of the mode stores (5, or 6 with the compensation of S).
template <int K, int NF = 5>
struct alignas(16) PipeSmem {
  float r0[kRing0][NF][128];
  float rl[K - 1][2][2][NF][128];
};

// Fused diagnostics (DIAG): the last warp also stores its output pair here, double-buffered
// by iteration parity like the level handoff; at the next iteration every warp adds its share
// (plane-rows j = row * NF + plane, j = (w - 2) mod K + i K for warp w) to running TwoSum
// pairs, and at the end of the tile the lanes' sums go to FP64, one partial per CTA.
constexpr int kDiagMaxWarps = 8;
template <int NF>
struct alignas(16) DiagSmem {
  float rows[2][2][NF][128];
  double part[kDiagMaxWarps][2 * NF];  // per warp and slot: the sum over the warp's lanes
  float peak;                          // the CTA's largest I (last warp)
};
template <int K, int NF>
constexpr int diag_slots() {
  return (2 * NF + K - 1) / K;
}

// a - b for two pairs in one instruction: b * (-1) is exact, so the fused multiply-add rounds
// a - b once, like the subtraction.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, splat2(-1.f), a); }
// hi + lo <- hi + x, the rounding error of the addition carried into lo (Knuth's TwoSum),
// for two independent pairs at once.
__device__ __forceinline__ void two_sum2(float2& hi, float2& lo, float2 x) {
  const float2 s = add2(hi, x);
  const float2 bp = sub2(s, hi);
  const float2 e = add2(sub2(hi, sub2(s, bp)), sub2(x, bp));
  hi = s;
  lo = add2(lo, e);
}
// Renormalise (Fast2Sum, |hi| >= |lo|): afterwards |lo| is at most half an ulp of hi, which
// keeps the rounding errors of later additions to lo at FP32's unit roundoff squared.
__device__ __forceinline__ void fast_two_sum2(float2& hi, float2& lo) {
  const float2 s = add2(hi, lo);
  lo = sub2(lo, sub2(s, hi));
  hi = s;
}

// Level s+1 of row C (two float2 column pairs per field) from level-s rows P, C, N: x
// neighbours by shuffles, the packed lap5 and the packed cell update.  MODE_SPLIT: field 5
// is the compensation of S, and the laplacian of S is lap5_diff(v) - lap5_diff(c).
template <int MODE, int NF = mode_planes<MODE>()>
__device__ __forceinline__ void cell_row(const Coeffs<float>& k, const float2 (&P)[NF][2], const float2 (&C)[NF][2],
                                         const float2 (&N)[NF][2], float2 (&M)[NF][2]) {
  constexpr unsigned kFull = 0xffffffffu;
  float2 lp[4][2];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float L = __shfl_up_sync(kFull, C[f][1].y, 1);
    const float R = __shfl_down_sync(kFull, C[f][0].x, 1);
    if (MODE == MODE_SPLIT && f == 0) {
      // the difference form on the value and on the compensation (field Q = NF - 1), columns 0..3
      constexpr int Q = NF - 1;
      const float LC = __shfl_up_sync(kFull, C[Q][1].y, 1);
      const float RC = __shfl_down_sync(kFull, C[Q][0].x, 1);
      const float2 v0 = lap5diff_x2(C[0][0], make_float2(L, C[0][0].x), make_float2(C[0][0].y, C[0][1].x),
                                    P[0][0], N[0][0]);
      const float2 v1 = lap5diff_x2(C[0][1], make_float2(C[0][0].y, C[0][1].x), make_float2(C[0][1].y, R),
                                    P[0][1], N[0][1]);
      const float2 c0 = lap5diff_x2(C[Q][0], make_float2(LC, C[Q][0].x), make_float2(C[Q][0].y, C[Q][1].x),
                                    P[Q][0], N[Q][0]);
      const float2 c1 = lap5diff_x2(C[Q][1], make_float2(C[Q][0].y, C[Q][1].x), make_float2(C[Q][1].y, RC),
                                    P[Q][1], N[Q][1]);
      lp[0][0] = add2(v0, neg2(c0));
      lp[0][1] = add2(v1, neg2(c1));
      continue;
    }
    // left + right neighbour of columns 0..3, then the packed rest of lap5
    const float2 lr0 = make_float2(__fadd_rn(L, C[f][0].y), __fadd_rn(C[f][0].x, C[f][1].x));
    const float2 lr1 = make_float2(__fadd_rn(C[f][0].y, C[f][1].y), __fadd_rn(C[f][1].x, R));
    lp[f][0] = lap5x2(C[f][0], lr0, P[f][0], N[f][0]);
    lp[f][1] = lap5x2(C[f][1], lr1, P[f][1], N[f][1]);
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if constexpr (MODE == MODE_SPLIT)
      seird_cell2_split(k, C[0][h], C[NF - 1][h], C[1][h], C[2][h], C[3][h], C[4][h], lp[0][h], lp[1][h], lp[2][h],
                        lp[3][h], M[0][h], M[NF - 1][h], M[1][h], M[2][h], M[3][h], M[4][h]);
    else
      seird_cell2<MODE == MODE_DEV>(k, C[0][h], C[1][h], C[2][h], C[3][h], C[4][h], lp[0][h], lp[1][h], lp[2][h],
                                    lp[3][h], M[0][h], M[1][h], M[2][h], M[3][h], M[4][h]);
  }
}

// Level s+1 of row C on the D2Q9 lattice (plain FP32 storage) from level-s rows P, C, N: the
// nine-point laplacian (4 ((l + r) + (u + d)) + ((ne + nw) + (se + sw)) - 20 c) / 6 of S, E,
// I, R, each pair sum formed as row[x-1] + row[x+1] (equal bits: the sums commute), then the
// packed cell update -- the operations of the one-step D2Q9 kernel.  One column pair at a
// time (h = 0: columns 0, 1 with the left neighbours shuffled in; h = 1: columns 2, 3 with the
// right ones), which keeps the live registers within the pipeline's budget.
//
// ALIGNED: nx is a multiple of 4, so x = nx - 1 is column 3 of its lane (jr = 3 or none).
// WALLS (no-flux): a link that leaves the domain sees the cell's own value (halfway
// bounce-back).  At x = 0 (column 0 of the lane with xs = 0) the shuffled-in left neighbours
// of the three rows are replaced by the centre; at x = nx - 1 (column jr of its lane) the right
// neighbours, in-lane or shuffled in, likewise.  ROWWALL (row 0 or ny - 1, warp-uniform): the
// row beyond the wall enters as the centre, its pair sum as centre + centre.  Cells outside the
// domain are never read by an in-domain cell, so their values do not matter.
template <bool ROWWALL, bool WALLS, bool ALIGNED = false>
__device__ __forceinline__ void cell_row9(const Coeffs<float>& k, const GridView& g, const float2 (&P)[5][2],
                                          const float2 (&C)[5][2], const float2 (&N)[5][2], float2 (&M)[5][2],
                                          const int64_t xs, const int64_t row) {
  constexpr unsigned kFull = 0xffffffffu;
  const bool wl = WALLS && xs == 0;                            // column 0 is x = 0
  const int jr = WALLS ? (int)(g.nx - 1 - xs) : -1;           // column of x = nx - 1, if in [0, 3]
  const bool wd = ROWWALL && row == 0, wu = ROWWALL && row == g.ny - 1;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float2 lp[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      // the neighbour beyond the pair: from the lane on the left (h = 0) or on the right (h = 1)
      float XP = h == 0 ? __shfl_up_sync(kFull, P[f][1].y, 1) : __shfl_down_sync(kFull, P[f][0].x, 1);
      float XC = h == 0 ? __shfl_up_sync(kFull, C[f][1].y, 1) : __shfl_down_sync(kFull, C[f][0].x, 1);
      float XN = h == 0 ? __shfl_up_sync(kFull, N[f][1].y, 1) : __shfl_down_sync(kFull, N[f][0].x, 1);
      // right neighbours of the pair's columns inside the lane (h = 0: columns 1, 2; h = 1:
      // column 3), the centre where that column is x = nx - 1
      float RP, RC, RN;
      if (h == 0) {
        if (WALLS && wl) XP = XC = XN = C[f][0].x;
        const bool w0 = WALLS && !ALIGNED && jr == 0;
        RP = w0 ? C[f][0].x : P[f][0].y;
        RC = w0 ? C[f][0].x : C[f][0].y;
        RN = w0 ? C[f][0].x : N[f][0].y;
      } else {
        if (WALLS && jr == 3) XP = XC = XN = C[f][1].y;
        const bool w2 = WALLS && !ALIGNED && jr == 2;
        RP = w2 ? C[f][1].x : P[f][1].y;
        RC = w2 ? C[f][1].x : C[f][1].y;
        RN = w2 ? C[f][1].x : N[f][1].y;
      }
      float2 hP, hC, hN;
      if (h == 0) {
        const bool w1 = WALLS && !ALIGNED && jr == 1;
        hP = make_float2(__fadd_rn(XP, RP), __fadd_rn(P[f][0].x, w1 ? C[f][0].y : P[f][1].x));
        hC = make_float2(__fadd_rn(XC, RC), __fadd_rn(C[f][0].x, w1 ? C[f][0].y : C[f][1].x));
        hN = make_float2(__fadd_rn(XN, RN), __fadd_rn(N[f][0].x, w1 ? C[f][0].y : N[f][1].x));
      } else {
        hP = make_float2(__fadd_rn(P[f][0].y, RP), __fadd_rn(P[f][1].x, XP));
        hC = make_float2(__fadd_rn(C[f][0].y, RC), __fadd_rn(C[f][1].x, XC));
        hN = make_float2(__fadd_rn(N[f][0].y, RN), __fadd_rn(N[f][1].x, XN));
      }
      float2 Pv = P[f][h], Nv = N[f][h];
      if (ROWWALL) {
        if (wd) Pv = C[f][h], hP = add2(C[f][h], C[f][h]);
        if (wu) Nv = C[f][h], hN = add2(C[f][h], C[f][h]);
      }
      lp[f] = mul2(fma2(splat2(-20.f), C[f][h], fma2(splat2(4.f), add2(hC, add2(Nv, Pv)), add2(hN, hP))),
                   splat2(1.f / 6.f));
    }
    seird_cell2<0>(k, C[0][h], C[1][h], C[2][h], C[3][h], C[4][h], lp[0], lp[1], lp[2], lp[3], M[0][h], M[1][h],
                   M[2][h], M[3][h], M[4][h]);
  }
}

// Static rows of the varying-diffusion lattice: the scale planes kx, ky of the rows in the
// pipeline's window, kRingK rows of 128 columns each in shared memory (row q in slot
// (q - qa) mod kRingK).  A level-s warp reads rows up to 3(K - 1) + 2 behind the level-0
// rows, which are copied three row pairs ahead, so kRingK >= 3K + 8.
constexpr int kRingK = 32;

// Level s+1 of row C on the varying-diffusion lattice (plain FP32 storage) from level-s rows
// P, C, N: the link coefficients (k_a(x) + k_a(x + c_i)) / 2 from the scale rows (kx of the
// row, x neighbours by shuffles; ky of the rows y-1, y, y+1), the flux terms of S, E, I, R,
// each rounded on its own, summed as ((+x) + (-x)) + ((+y) + (-y)) in scalar adds, then the
// packed cell update -- the operations of the one-step kernel.  The sum is unchanged by a
// mirror image, so the no-flux ghost images evolve as the cells they mirror, as on D2Q5.
// kxr, kyp, kyc, kyn: this lane's four columns of kx (row y) and ky (rows y-1, y, y+1).
__device__ __forceinline__ void cell_rowv(const Coeffs<float>& k, const float2 (&P)[5][2], const float2 (&C)[5][2],
                                          const float2 (&N)[5][2], float2 (&M)[5][2], const float* kxr,
                                          const float* kyp, const float* kyc, const float* kyn) {
  constexpr unsigned kFull = 0xffffffffu;
  const float4 ax = *reinterpret_cast<const float4*>(kxr);
  const float axL = __shfl_up_sync(kFull, ax.w, 1), axR = __shfl_down_sync(kFull, ax.x, 1);
  const float4 bc = *reinterpret_cast<const float4*>(kyc);
  const float4 bp = *reinterpret_cast<const float4*>(kyp);
  const float4 bn = *reinterpret_cast<const float4*>(kyn);
  const float2 half = splat2(0.5f);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 a = h == 0 ? make_float2(ax.x, ax.y) : make_float2(ax.z, ax.w);
    const float2 aR = h == 0 ? make_float2(ax.y, ax.z) : make_float2(ax.w, axR);
    const float2 aL = h == 0 ? make_float2(axL, ax.x) : make_float2(ax.y, ax.z);
    const float2 b = h == 0 ? make_float2(bc.x, bc.y) : make_float2(bc.z, bc.w);
    const float2 bN = h == 0 ? make_float2(bn.x, bn.y) : make_float2(bn.z, bn.w);
    const float2 bP = h == 0 ? make_float2(bp.x, bp.y) : make_float2(bp.z, bp.w);
    const float2 lxp = mul2(half, add2(a, aR)), lyp = mul2(half, add2(b, bN));
    const float2 lxm = mul2(half, add2(a, aL)), lym = mul2(half, add2(b, bP));
    float2 flux[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      // the neighbour beyond the pair: from the lane on the left (h = 0) or on the right (h = 1)
      const float X = h == 0 ? __shfl_up_sync(kFull, C[f][1].y, 1) : __shfl_down_sync(kFull, C[f][0].x, 1);
      const float2 cc = C[f][h], ncc = neg2(cc);
      const float2 right = h == 0 ? make_float2(C[f][0].y, C[f][1].x) : make_float2(C[f][1].y, X);
      const float2 left = h == 0 ? make_float2(X, C[f][0].x) : make_float2(C[f][0].y, C[f][1].x);
      const float2 t1 = mul2(lxp, add2(right, ncc));
      const float2 t2 = mul2(lyp, add2(N[f][h], ncc));
      const float2 t3 = mul2(lxm, add2(left, ncc));
      const float2 t4 = mul2(lym, add2(P[f][h], ncc));
      flux[f] = make_float2(__fadd_rn(__fadd_rn(t1.x, t3.x), __fadd_rn(t2.x, t4.x)),
                            __fadd_rn(__fadd_rn(t1.y, t3.y), __fadd_rn(t2.y, t4.y)));
    }
    seird_cell2<0>(k, C[0][h], C[1][h], C[2][h], C[3][h], C[4][h], flux[0], flux[1], flux[2], flux[3], M[0][h],
                   M[1][h], M[2][h], M[3][h], M[4][h]);
  }
}

// Level s+1 of row C in the Kahan storage (ten planes: the values of S, E, I, R, D, then
// their compensations) from level-s rows P, C, N: per compartment the laplacian
// lap5_diff(value) - lap5_diff(compensation), the increments of seird_increments (the force
// from the values), each added to its (value, compensation) pair with kahan_add -- the
// operations of the one-step Kahan kernel, packed.  The adds whose operand is a packed
// product, and the product that enters kahan_add directly, stay scalar: packed, the compiler
// may fuse the product into the add (measured: the compensation of D then differed in its
// last bits from the one-step kernel's).
__device__ __forceinline__ void cell_row_kahan(const Coeffs<float>& k, const float2 (&P)[10][2],
                                               const float2 (&C)[10][2], const float2 (&N)[10][2],
                                               float2 (&M)[10][2]) {
  constexpr unsigned kFull = 0xffffffffu;
  float2 lp[4][2];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    float2 d[2][2];  // [value, compensation][column pair]
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int p = q == 0 ? f : 5 + f;
      const float L = __shfl_up_sync(kFull, C[p][1].y, 1);
      const float R = __shfl_down_sync(kFull, C[p][0].x, 1);
      d[q][0] = lap5diff_x2(C[p][0], make_float2(L, C[p][0].x), make_float2(C[p][0].y, C[p][1].x), P[p][0], N[p][0]);
      d[q][1] = lap5diff_x2(C[p][1], make_float2(C[p][0].y, C[p][1].x), make_float2(C[p][1].y, R), P[p][1], N[p][1]);
    }
    lp[f][0] = add2(d[0][0], neg2(d[1][0]));
    lp[f][1] = add2(d[0][1], neg2(d[1][1]));
  }
  auto sadd = [](float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); };
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 S = C[0][h], E = C[1][h], I = C[2][h];
    const float2 F = force_dt2(k, S, E, I, C[3][h]);
    float2 inc[5];
    inc[0] = fma2(splat2(k.dl[0]), lp[0][h], neg2(F));
    inc[1] = sadd(mul2(splat2(k.dl[1]), lp[1][h]), fma2(splat2(-k.adt), E, F));
    inc[2] = sadd(mul2(splat2(k.dl[2]), lp[2][h]), fma2(splat2(k.adt), E, neg2(mul2(splat2(k.gdt), I))));
    inc[3] = fma2(splat2(k.rdt), I, mul2(splat2(k.dl[3]), lp[3][h]));
    // scalar products: a packed product feeding kahan_add's first add could be fused into it
    inc[4] = make_float2(__fmul_rn(k.ddt, I.x), __fmul_rn(k.ddt, I.y));
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      float2 v = C[f][h], c = C[5 + f][h];
      kahan_add2(v, c, inc[f]);
      M[f][h] = v;
      M[5 + f][h] = c;
    }
  }
}

// Hand level-(s+1) row M to the next warp (slot row `which` of parity par) or, for the last
// warp, write it to row r of the output.
// DIAG: the last warp also stores the row into slot row `which` of dsl (the parity's
// diagnostics rows; zeros for cells outside the tile's output) and takes the largest I of
// the cells it writes into *pk.
template <int K, int NF, bool DIAG = false>
__device__ __forceinline__ void emit_row(PipeSmem<K, NF>& sm, const GridView& g, const float2 (&M)[NF][2],
                                         float* __restrict__ out, const int s, const int lane, const int par,
                                         const int which, const bool writer, const int64_t xs, const int64_t r,
                                         const int64_t y0, const int64_t y1, float* dsl = nullptr,
                                         float* pk = nullptr) {
  if (s < K - 1) {
    float* dst = &sm.rl[s < K - 1 ? s : 0][par][which][0][4 * lane];
#pragma unroll
    for (int f = 0; f < NF; ++f)
      *reinterpret_cast<float4*>(dst + 128 * f) = make_float4(M[f][0].x, M[f][0].y, M[f][1].x, M[f][1].y);
    return;
  }
  if constexpr (DIAG) {
    const bool rv = writer && r >= y0 && r < y1;
    // columns xs + j that lie in the grid (a writer's first column always does)
    const bool c1 = xs + 1 < g.nx, c2 = xs + 2 < g.nx, c3 = xs + 3 < g.nx;
    float* d = dsl + which * (NF * 128) + 4 * lane;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rv) v = make_float4(M[f][0].x, c1 ? M[f][0].y : 0.f, c2 ? M[f][1].x : 0.f, c3 ? M[f][1].y : 0.f);
      *reinterpret_cast<float4*>(d + 128 * f) = v;
    }
    if (rv) {
      float m = M[2][0].x;
      if (c1) m = fmaxf(m, M[2][0].y);
      if (c2) m = fmaxf(m, M[2][1].x);
      if (c3) m = fmaxf(m, M[2][1].y);
      *pk = fmaxf(*pk, m);
    }
  }
  if (writer && r >= y0 && r < y1 && SSLBM_IN(r, 1, g.ny, 5)) {
    float* o = out + r * g.pitch + xs;
    if (xs + 3 < g.nx) {
      if (SSLBM_IN(xs, 4, g.nx, 6)) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
          *reinterpret_cast<float4*>(o + f * g.plane) = make_float4(M[f][0].x, M[f][0].y, M[f][1].x, M[f][1].y);
      }
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float v[4] = {M[f][0].x, M[f][0].y, M[f][1].x, M[f][1].y};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (xs + jj < g.nx && SSLBM_IN(xs + jj, 1, g.nx, 7)) o[f * g.plane + jj] = v[jj];
      }
    }
  }
}

// One iteration of warp s: read the pair of level-s rows b, b+1 (N0, N1) from src (row b+1
// 128 NF floats further), compute level-(s+1) rows b-1 (from A = b-2, B = b-1, N0) and b (from
// B, N0, N1), hand them on or write them as rows r, r+1.  Ends with the CTA barrier.
// DIAG: dsl, pk as in emit_row (dsl: the diagnostics rows of parity par).
template <int MODE, int K, bool COLW = true, bool DIAG = false, int NF = mode_planes<MODE>()>
__device__ __forceinline__ void pipe_pair(PipeSmem<K, NF>& sm, const GridView& g, const Coeffs<float>& k,
                                          const float* src, const float2 (&A)[NF][2], const float2 (&B)[NF][2],
                                          float2 (&N0)[NF][2], float2 (&N1)[NF][2], float* __restrict__ out,
                                          const int s, const int lane, const int par, const bool writer,
                                          const int64_t xs, const int64_t r, const int64_t y0, const int64_t y1,
                                          const float* rk = nullptr, const int sk = 0, float* dsl = nullptr,
                                          float* pk = nullptr) {
  auto load_row = [&](const float* p, float2 (&R)[NF][2]) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float4 t = *reinterpret_cast<const float4*>(p + 128 * f);
      R[f][0] = make_float2(t.x, t.y);
      R[f][1] = make_float2(t.z, t.w);
    }
  };
  float2 M[NF][2];
  if constexpr (MODE == MODE_D2Q9 || MODE == MODE_D2Q9_NOFLUX || MODE == MODE_D2Q9_NOFLUX4) {
    // the second row of the pair is read after the first is done: fewer live registers for
    // the nine-point stencil's wider neighbourhood
    constexpr bool W = MODE == MODE_D2Q9_NOFLUX || MODE == MODE_D2Q9_NOFLUX4;
    constexpr bool AL = MODE == MODE_D2Q9_NOFLUX4;
    const int64_t row = r + 3 * (K - 1 - s);  // the first row this warp computes (r: the last warp's)
    load_row(src, N0);
    if (W && (row == 0 || row == g.ny - 1))
      cell_row9<true, W>(k, g, A, B, N0, M, xs, row);
    else
      cell_row9<false, W && COLW, AL>(k, g, A, B, N0, M, xs, row);
    emit_row<K, NF, DIAG>(sm, g, M, out, s, lane, par, 0, writer, xs, r, y0, y1, dsl, pk);
    load_row(src + 128 * NF, N1);
    if (W && (row + 1 == 0 || row + 1 == g.ny - 1))
      cell_row9<true, W>(k, g, B, N0, N1, M, xs, row + 1);
    else
      cell_row9<false, W && COLW, AL>(k, g, B, N0, N1, M, xs, row + 1);
  } else if constexpr (MODE == MODE_KAHAN) {
    // ten planes: the second row of the pair is read after the first is done
    load_row(src, N0);
    cell_row_kahan(k, A, B, N0, M);
    emit_row<K, NF, DIAG>(sm, g, M, out, s, lane, par, 0, writer, xs, r, y0, y1, dsl, pk);
    load_row(src + 128 * NF, N1);
    cell_row_kahan(k, B, N0, N1, M);
  } else if constexpr (MODE == MODE_VARD) {
    // sk: the static-ring slot of the first row this warp computes (row b - 1)
    auto krow = [&](int d, int plane) {  // this lane's columns of scale plane `plane`, row b - 1 + d
      return rk + ((sk + d + kRingK) & (kRingK - 1)) * 256 + plane * 128 + 4 * lane;
    };
    load_row(src, N0);
    cell_rowv(k, A, B, N0, M, krow(0, 0), krow(-1, 1), krow(0, 1), krow(1, 1));
    emit_row<K, NF, DIAG>(sm, g, M, out, s, lane, par, 0, writer, xs, r, y0, y1, dsl, pk);
    load_row(src + 128 * NF, N1);
    cell_rowv(k, B, N0, N1, M, krow(1, 0), krow(0, 1), krow(1, 1), krow(2, 1));
  } else {
    load_row(src, N0);
    load_row(src + 128 * NF, N1);
    cell_row<MODE>(k, A, B, N0, M);
    emit_row<K, NF, DIAG>(sm, g, M, out, s, lane, par, 0, writer, xs, r, y0, y1, dsl, pk);
    cell_row<MODE>(k, B, N0, N1, M);
  }
  emit_row<K, NF, DIAG>(sm, g, M, out, s, lane, par, 1, writer, xs, r + 1, y0, y1, dsl, pk);
  __syncthreads();
}

// WRAP16: periodic grid with nx a multiple of 4 -- every lane's four columns, ghosts
// included, are one contiguous 16-byte group at the wrapped position, so all loads are
// L2-only cp.async.cg (required when other CTAs of the same launch wrote the input, since
// L1 is not coherent).
// COLW = false: the strip holds neither x = 0 nor x = nx - 1 (D2Q9 no-flux: no column wall
// code in its rows).
// DIAG (five planes): also the totals of the five output planes over the tile's output cells
// and their largest I, written as FP64 partial `diag_slot` of diag (6 doubles: the totals,
// then the peak), with dsm as the diagnostics' shared memory.
template <int MODE, int K, bool WRAP16 = false, bool COLW = true, bool DIAG = false, int NF = mode_planes<MODE>()>
__device__ __forceinline__ void pipe_tile(PipeSmem<K, NF>& sm, const GridView& g, const Coeffs<float>& k,
                                          const float* __restrict__ in, float* __restrict__ out,
                                          const int strip, const int64_t y0, const int64_t y1,
                                          const float* __restrict__ kx = nullptr,
                                          const float* __restrict__ ky = nullptr, float* rk = nullptr,
                                          DiagSmem<NF>* dsm = nullptr, double* __restrict__ diag = nullptr,
                                          const int diag_slot = 0) {
  static_assert(!DIAG || (NF == 5 && K <= kDiagMaxWarps), "fused diagnostics: five planes, up to 8 warps");
  constexpr int HL = (K + 3) / 4;   // halo lanes on each side of the strip
  constexpr int WV = 128 - 8 * HL;  // columns written per strip
  const int lane = threadIdx.x & 31;
  const int s = threadIdx.x >> 5;  // this warp computes level s + 1
  const int64_t xs = (int64_t)strip * WV - 4 * HL + 4 * lane;
  const bool vec_ok = xs >= 0 && xs + 3 < g.nx;
  const bool writer = lane >= HL && lane < 32 - HL && xs < g.nx;
  // A column more than K cells outside the domain cannot influence a written cell within
  // K steps, so lanes made only of such columns (the tail of the last strip) load nothing.
  const bool loads = xs < g.nx + K && xs + 3 >= -K;
  const int64_t xw = WRAP16 ? ((xs % g.nx) + g.nx) % g.nx : xs;
  int xm[4];  // ghost images of this lane's columns, for lanes on a domain edge
#pragma unroll
  for (int j = 0; j < 4; ++j) xm[j] = (int)ghost_index(xs + j, g.nx, g.bc);
  // Rows go through the pipeline in pairs.  At iteration t warp s reads the level-s rows
  // b, b+1 with b = qa + 2t - 3s (warp 0 from the ring, the others from the previous warp's
  // output of iteration t-1) and computes level-(s+1) rows b-1 and b.  Level-0 rows span
  // [y0-K, y1+K); the last warp finishes row y1-1 once b >= y1-1 for s = K-1.
  const int64_t qa = y0 - K, load_end = y1 + K;
  const int nt = (int)(((y1 - y0) + 4 * K - 4 + 1) / 2) + 1;
  const int64_t rbase = qa - 3 * (K - 1) - 1;  // the first row the last warp emits (iteration 0)

  for (int i = threadIdx.x; i < kRing0 * NF * 128; i += 32 * K) (&sm.r0[0][0][0])[i] = 0.f;
  for (int i = threadIdx.x; i < (K - 1) * 2 * 2 * NF * 128; i += 32 * K) (&sm.rl[0][0][0][0][0])[i] = 0.f;
  if (MODE == MODE_VARD)
    for (int i = threadIdx.x; i < kRingK * 2 * 128; i += 32 * K) rk[i] = 0.f;
  if constexpr (DIAG)
    for (int i = threadIdx.x; i < 2 * 2 * NF * 128; i += 32 * K) (&dsm->rows[0][0][0][0])[i] = 0.f;
  __syncthreads();

  auto issue = [&](int64_t q) {  // warp 0: copy level-0 row q into its ring slot
    if (!loads || q >= load_end) return;
    const int slot = (int)((q - qa) % kRing0);
    const int64_t yq = ghost_index(q, g.ny, g.bc);
    if (!SSLBM_IN(yq, 1, g.ny, 1)) return;
    const int64_t row = yq * g.pitch;
    // the state planes, and on the varying-diffusion lattice the two scale planes (static ring)
#pragma unroll
    for (int f = 0; f < (MODE == MODE_VARD ? NF + 2 : NF); ++f) {
      const float* src = (f < NF ? in + f * g.plane : f == NF ? kx : ky) + row;
      float* dst = f < NF ? &sm.r0[slot][f][4 * lane]
                          : rk + ((int)(q - qa) & (kRingK - 1)) * 256 + (f - NF) * 128 + 4 * lane;
      if (WRAP16) {
        if (SSLBM_IN(xw, 4, g.nx, 2)) cp_async16(dst, src + xw);
      } else if (vec_ok) {
        if (SSLBM_IN(xs, 4, g.nx, 3)) cp_async16(dst, src + xs);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (SSLBM_IN(xm[j], 1, g.nx, 4)) cp_async4(dst + j, src + xm[j]);
      }
    }
  };
  constexpr int kPairsAhead = kRing0 / 2 - 1;
  if (s == 0) {
#pragma unroll
    for (int p = 0; p < kPairsAhead; ++p) {
      issue(qa + 2 * p);
      issue(qa + 2 * p + 1);
      cp_async_commit();
    }
  }

  // Four row buffers: A, B hold rows b-2, b-1; the pair b, b+1 arrives in the other two, and
  // the roles swap every iteration (unrolled two ways, so no row is copied between registers).
  float2 RA[NF][2], RB[NF][2], RC[NF][2], RD[NF][2];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int h = 0; h < 2; ++h) RA[f][h] = RB[f][h] = make_float2(0.f, 0.f);
  // source of the pair of iteration t: warp 0's ring slots, or the previous warp's slot
  auto fetch = [&](int t) -> const float* {
    if (s == 0) {
      issue(qa + 2 * (t + kPairsAhead));
      issue(qa + 2 * (t + kPairsAhead) + 1);
      cp_async_commit();
      cp_async_wait<kPairsAhead>();
      return &sm.r0[(2 * t) & (kRing0 - 1)][0][4 * lane];
    }
    return &sm.rl[s - 1][(t + 1) & 1][0][0][4 * lane];
  };
  // the static-ring slot of the first row warp s computes at iteration t (row qa + 2t - 3s - 1)
  auto kslot = [&](int t) { return (2 * t - 3 * s - 1) & (kRingK - 1); };

  // Fused diagnostics: this lane's TwoSum pairs, one per plane-row slot of the warp, and (last
  // warp) the largest I it wrote.  Before iteration t every warp adds its plane-rows of the
  // last warp's output of iteration t - 1 (parity (t + 1) & 1; zeros at t = 0).
  constexpr int NS = DIAG ? diag_slots<K, NF>() : 1;
  const int j0 = (s + 2 * K - 2) % K;  // this warp's first plane-row
  float2 dh[NS], dl[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) dh[i] = dl[i] = make_float2(0.f, 0.f);
  float pk = -FLT_MAX;
  auto dsl = [&](int par) -> float* { return DIAG ? &dsm->rows[par][0][0][0] : nullptr; };
  auto diag_take = [&](int par) {
    if constexpr (DIAG) {
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        const int j = j0 + i * K;
        if (j < 2 * NF) {
          const float4 v = *reinterpret_cast<const float4*>(&dsm->rows[par][0][0][0] + j * 128 + 4 * lane);
          two_sum2(dh[i], dl[i], make_float2(v.x, v.y));
          two_sum2(dh[i], dl[i], make_float2(v.z, v.w));
          fast_two_sum2(dh[i], dl[i]);
        }
      }
    }
  };

  int t = 0;
  for (; t + 2 <= nt; t += 2) {
    diag_take((t + 1) & 1);
    pipe_pair<MODE, K, COLW, DIAG>(sm, g, k, fetch(t), RA, RB, RC, RD, out, s, lane, t & 1, writer, xs, rbase + 2 * t,
                                   y0, y1, rk, kslot(t), dsl(t & 1), &pk);
    diag_take(t & 1);
    pipe_pair<MODE, K, COLW, DIAG>(sm, g, k, fetch(t + 1), RC, RD, RA, RB, out, s, lane, (t + 1) & 1, writer, xs,
                                   rbase + 2 * t + 2, y0, y1, rk, kslot(t + 1), dsl((t + 1) & 1), &pk);
  }
  if (t < nt) {
    diag_take((t + 1) & 1);
    pipe_pair<MODE, K, COLW, DIAG>(sm, g, k, fetch(t), RA, RB, RC, RD, out, s, lane, t & 1, writer, xs, rbase + 2 * t,
                                   y0, y1, rk, kslot(t), dsl(t & 1), &pk);
  }
  if (s == 0) cp_async_wait<0>();
  if constexpr (DIAG) {
    diag_take((nt - 1) & 1);  // the last iteration's output (the last pipe_pair ended with a barrier)
    constexpr unsigned kFull = 0xffffffffu;
    double acc[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      acc[i] = ((double)dh[i].x + (double)dl[i].x) + ((double)dh[i].y + (double)dl[i].y);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(kFull, acc[i], o);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pk = fmaxf(pk, __shfl_xor_sync(kFull, pk, o));
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NS; ++i) dsm->part[s][i] = acc[i];
      if (s == K - 1) dsm->peak = pk;
    }
    __syncthreads();
    if (threadIdx.x == 0 && SSLBM_IN(diag_slot, 1, kDiagBlocks, 8)) {
      double tot[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int w = 0; w < K; ++w)  // fixed order: the partial does not depend on timing
        for (int i = 0; i < NS; ++i) {
          const int j = (w + 2 * K - 2) % K + i * K;
          if (j < 2 * NF) tot[j % NF] += dsm->part[w][i];
        }
#pragma unroll
      for (int c = 0; c < 5; ++c) diag[diag_slot * kDiagSlots + c] = tot[c];
      diag[diag_slot * kDiagSlots + 5] = (double)dsm->peak;
    }
  }
}

}  // namespace sslbm
