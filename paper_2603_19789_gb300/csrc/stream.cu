// stream.cu -- the streaming one-step kernel of the FP32 updates that advance one step per
// launch: the Kahan storage of the D2Q5 SSLBM (Sec. II.C, Eq. sslbm_final_clean, with the
// sources of Eq. sources and Eq. rhoD), the one-step D2Q5 update of the plain, deviation and
// split storages, the D2Q9 lattice (Sec. II.C, isotropy) and the spatially varying diffusion
// (the flux form of vard.cu).
//
// A warp owns a strip of kStCols columns and a segment of kStSeg rows and walks down it.  The
// rows of the planes its update reads arrive by cp.async in a ring of Cell::kRing rows in
// shared memory, kRing - 3 rows ahead of the rows being read, so every plane is read from
// global memory once per step (the two rows beyond a segment's ends a second time) and no
// CTA barrier is needed: each warp fills and reads only its own ring.  Lane l updates
// columns xs + l and xs + 32 + l, reading its neighbours from the ring rows y - 1, y, y + 1.
//
// Ring row layout, per plane: index i holds column xs - 4 + i, so the 64 interior columns
// start at index 4 (16-byte aligned for the vector copies) and the halo columns sit at 3 and
// 68.  Ring column x in [-1, nx] holds the value at link_index(x): the periodic wrap, or
// the cell-centred mirror of no-flux, as the one-step kernels read it; rows likewise.  The
// first Cell::kHaloPlanes ring planes carry the halo columns (the planes whose x neighbours
// enter the update); the others only their interior columns.
//
// Each cell update performs the same operations, in the same order, as the kernel it
// replaces, so results are bit-identical to those kernels (and to K one-step launches of the
// blocked pipeline for the D2Q5 storages).
#include <cuda_runtime.h>

#include <atomic>

#include "bounds.cuh"
#include "dword.cuh"
#include "sslbm_internal.cuh"
#include "sslbm_pipe.cuh"
#include "variants.cuh"

SSLBM_OOB_ACCESSOR(stream)

namespace sslbm {
namespace {

constexpr int kStCols = 64;     // columns per strip: two per lane
constexpr int kStStride = 72;   // floats per plane row in the ring
constexpr int kStSeg = 128;     // rows per segment

// Column index of ring column x: link_index for the halo columns -1 and nx; columns
// further out (the unused tail of a strip past the grid) read a clamped in-range cell.
__device__ __forceinline__ int64_t st_col(int64_t x, const GridView& g) {
  if (x >= 0 && x < g.nx) return x;
  if (x == -1 || x == g.nx) return link_index(x, g.nx, g.bc);
  return x < 0 ? 0 : g.nx - 1;  // never a neighbour of a written cell
}

// Ring rows of one update: U = row y - 1, C = row y, N = row y + 1; plane f of a row starts
// at f * kStStride; i is the ring index of the cell's column.
struct Rows {
  const float* U;
  const float* C;
  const float* N;
};

// A cell update is update(g, rows, i, x, y, state, first): state is the cell's own carry from
// row y - 1 of the same column (first: y is the segment's first row, the carry is unset).
// A packed cell (kPacked) updates both of the lane's columns, x and x + 32 (ring indices i
// and i + 32), in one call with two-lane FP32 arithmetic (add2, fma2, ...: each component
// rounded as the scalar operation), the second column only where x + 32 < nx.
struct NoState {};

// The values of ring indices i and i + 32 of a plane row: the lane's two columns.
__device__ __forceinline__ float2 ld2(const float* p, int i) { return make_float2(p[i], p[i + 32]); }

template <class Cell>
__global__ void __launch_bounds__(32 * Cell::kWarps, Cell::kMinBlocks)
    stream_kernel(const GridView g, const Cell cell, const int nstrips, const int nitems) {
  constexpr int NP = Cell::kPlanes, NH = Cell::kHaloPlanes, RING = Cell::kRing;
  constexpr int ROWF = NP * kStStride;
  static_assert(NH <= 16 && NH <= NP && RING >= 4, "ring shape");
  extern __shared__ __align__(16) float st_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int item = blockIdx.x * Cell::kWarps + warp;
  if (item >= nitems) return;
  float* ring = st_smem + (size_t)warp * (RING * ROWF);
  const int strip = item % nstrips;
  const int64_t xs = (int64_t)strip * kStCols;
  const int64_t y0 = (int64_t)(item / nstrips) * kStSeg;
  const int64_t y1 = y0 + kStSeg < g.ny ? y0 + kStSeg : g.ny;
  const bool vec = xs + kStCols <= g.nx;
  const int64_t xl = st_col(xs - 1, g), xr = st_col(xs + kStCols, g);
  const int64_t q0 = y0 - 1;  // first logical row in the ring
  auto issue = [&](int64_t q) {  // rows q0 .. y1 (one beyond the segment on each side)
    const int64_t yq = link_index(q, g.ny, g.bc);
    if (q <= y1 && SSLBM_IN(yq, 1, g.ny, 1)) {
      const int64_t row = yq * g.pitch;
      float* dst = ring + (int)((unsigned)(q - q0) % RING) * ROWF;
      if (vec) {
        for (int u = lane; u < NP * 16; u += 32) {
          const int f = u >> 4, part = u & 15;
          if (SSLBM_IN(xs + 4 * part, 4, g.nx, 2))
            cp_async16(dst + f * kStStride + 4 + 4 * part, cell.src(f, g) + row + xs + 4 * part);
        }
        if (lane < 2 * NH) {
          const bool left = lane < NH;
          const int f = left ? lane : lane - NH;
          const int64_t xh = left ? xl : xr;
          if (SSLBM_IN(xh, 1, g.nx, 3))
            cp_async4(dst + f * kStStride + (left ? 3 : 4 + kStCols), cell.src(f, g) + row + xh);
        }
      } else {
        for (int u = lane; u < NP * (kStCols + 2); u += 32) {
          const int f = u / (kStCols + 2), i = 3 + u % (kStCols + 2);
          const int64_t xc = st_col(xs - 4 + i, g);
          if (SSLBM_IN(xc, 1, g.nx, 4)) cp_async4(dst + f * kStStride + i, cell.src(f, g) + row + xc);
        }
      }
    }
    cp_async_commit();  // one group per row, empty beyond the segment
  };
  typename Cell::State st[2];  // what a cell carries from row to row, per column of the lane
  // rows y - 1, y, y + 1 are in use, RING - 3 further rows are in flight
  for (int64_t q = q0; q < q0 + RING - 1; ++q) issue(q);
  for (int64_t y = y0; y < y1; ++y) {
    __syncwarp();  // every lane is done with the slot that row y + RING - 2 takes over
    issue(y + RING - 2);
    cp_async_wait<RING - 3>();  // rows up to y + 1 are in
    __syncwarp();
    const unsigned rel = (unsigned)(y - q0);
    const Rows r{ring + (int)((rel - 1) % RING) * ROWF, ring + (int)(rel % RING) * ROWF,
                 ring + (int)((rel + 1) % RING) * ROWF};
    if (!SSLBM_IN(y, 1, g.ny, 5)) continue;
    if constexpr (Cell::kPacked) {
      const int64_t x = xs + lane;
      if (x < g.nx && SSLBM_IN(x, 1, g.nx, 6)) cell.update(g, r, 4 + lane, x, y, st[0], y == y0);
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t x = xs + lane + 32 * h;
        if (x < g.nx && SSLBM_IN(x, 1, g.nx, 6)) cell.update(g, r, 4 + lane + 32 * h, x, y, st[h], y == y0);
      }
    }
  }
  cp_async_wait<0>();
}

// ---- cell updates ----------------------------------------------------------------------

// The Kahan storage: ten planes (values of S, E, I, R, D, then their compensations).  The
// laplacian is lap5_diff of the values minus that of the compensations, the increments those
// of seird_increments, each added to its (value, compensation) pair with kahan_add.
// Ring depth and warps per CTA measured at 8192^2: 8 rows and 2 warps (four CTAs, eight
// warps per SM) 77.3 GLUPS; 8 and 4 warps 76.5; 7 and 3 warps 68.3; 6 and 4 warps 61.3; 10
// and 2 warps (three CTAs per SM) 66.6.
struct KahanCell {
  static constexpr int kPlanes = 10, kHaloPlanes = 9, kRing = 8, kWarps = 2, kMinBlocks = 4;
  static constexpr bool kPacked = false;
  const float* in;
  float* out;
  Coeffs<float> k;
  __device__ __forceinline__ const float* src(int f, const GridView& g) const { return in + f * g.plane; }
  using State = NoState;
  __device__ __forceinline__ void update(const GridView& g, const Rows& r, int i, int64_t x, int64_t y, State&,
                                         bool) const {
    float c[5], cmp[5], lap[4];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const float* P = r.C + f * kStStride;
      const float* Q = r.C + (5 + f) * kStStride;
      c[f] = P[i];
      cmp[f] = Q[i];
      if (f < 4) {
        lap[f] = lap5_diff(P[i], P[i - 1], P[i + 1], r.U[f * kStStride + i], r.N[f * kStStride + i]);
        lap[f] = sub_rn(lap[f], lap5_diff(Q[i], Q[i - 1], Q[i + 1], r.U[(5 + f) * kStStride + i],
                                          r.N[(5 + f) * kStStride + i]));
      }
    }
    float inc[5];
    seird_increments(k, c[0], c[1], c[2], c[3], lap[0], lap[1], lap[2], lap[3], inc);
    float* o = out + y * g.pitch + x;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      float v = c[f], q = cmp[f];
      kahan_add(v, q, inc[f]);
      o[f * g.plane] = v;
      o[(5 + f) * g.plane] = q;
    }
  }
};

// Stores of a packed update: plane f of the lane's two columns.
__device__ __forceinline__ void st2(float* o, int64_t plane_off, float2 v, bool second) {
  o[plane_off] = v.x;
  if (second) o[plane_off + 32] = v.y;
}

// The FP64-accurate double-word storage (SSLBM_FP64_DW): the Kahan storage's ten planes, read
// as values hi and lo = -(compensation plane), and the update of seird_cell (the FP64
// kernel's operations, in its order) in double-word arithmetic (dword.cuh), except the
// laplacian, taken as ((l - c) + (r - c)) + ((u - c) + (d - c)): for a smooth field every
// difference is small and carries the double-word precision of the values, where the sum of
// the neighbours minus 4c would lose their high part's magnitude.  Ring planes: the high
// parts of S, E, I, R, their compensations (the planes with x neighbours), then D's two.
// The additions are the 11-flop form (add_abs), whose absolute error bound is what a
// max-norm against the fields' peak needs: 37.5 GLUPS at 8192^2 against 27.8 with the
// 20-flop accurate sum, with the same errors against the oracle (1.6e-13 after 2000 steps of
// the paper's case).  Ring rows and warps, 8192^2: 4 rows, 4 warps, 4 CTAs (16 warps per SM)
// 40.7 GLUPS; 4 rows, 2 warps, 8 CTAs 40.7; 5 rows, 4 warps, 3 CTAs 37.5; 6 rows, 2 warps,
// 6 CTAs 37.7.  The laplacian with one normalisation (dw::lap5_diff) instead of seven
// add_abs: 43.8, the same errors (the native FP64 kernel: 11.9).
struct DwCell {
  static constexpr int kPlanes = 10, kHaloPlanes = 8, kRing = 4, kWarps = 4, kMinBlocks = 4;
  static constexpr bool kPacked = true;
  const float* in;
  float* out;
  DwCoeffs k;
  __device__ __forceinline__ const float* src(int f, const GridView& g) const {
    return in + (f < 4 ? f : f < 8 ? f + 1 : f == 8 ? 4 : 9) * g.plane;
  }
  using State = NoState;
  __device__ __forceinline__ void update(const GridView& g, const Rows& r, int i, int64_t x, int64_t y, State&,
                                         bool) const {
    using dw::W;
    // the pair of ring plane f (high part) and f + off (compensation) at ring index j of row p
    auto val = [&](const float* p, int f, int off, int j) {
      return W{ld2(p + f * kStStride, j), neg2(ld2(p + (f + off) * kStStride, j))};
    };
    W c[5], lap[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      c[f] = val(r.C, f, 4, i);
      lap[f] = dw::lap5_diff(c[f], val(r.C, f, 4, i - 1), val(r.C, f, 4, i + 1), val(r.U, f, 4, i),
                             val(r.N, f, 4, i));
    }
    c[4] = val(r.C, 8, 1, i);
    const W &S = c[0], &E = c[1], &I = c[2], &R = c[3], &D = c[4];
    // force of infection times dt, beta S I / N_c dt, against max(N_c, smallest normal)
    W Nc = dw::add_abs(dw::add_abs(S, E), dw::add_abs(I, R));
    if (!(Nc.h.x >= 1.17549435e-38f)) Nc.h.x = 1.17549435e-38f, Nc.l.x = 0.f;
    if (!(Nc.h.y >= 1.17549435e-38f)) Nc.h.y = 1.17549435e-38f, Nc.l.y = 0.f;
    const W F = dw::div(dw::mul(dw::mul(dw::splat(k.bdt), S), I), Nc);
    const W adt = dw::splat(k.adt);
    W n[5];
    n[0] = dw::sub_abs(dw::add_abs(dw::mul(dw::splat(k.dl[0]), lap[0]), S), F);
    n[1] = dw::add_abs(dw::add_abs(dw::mul(dw::splat(k.dl[1]), lap[1]), E), dw::add_abs(dw::mul(dw::neg(adt), E), F));
    n[2] = dw::add_abs(dw::add_abs(dw::mul(dw::splat(k.dl[2]), lap[2]), I),
                   dw::sub_abs(dw::mul(adt, E), dw::mul(dw::splat(k.gdt), I)));
    n[3] = dw::add_abs(dw::mul(dw::splat(k.rdt), I), dw::add_abs(dw::mul(dw::splat(k.dl[3]), lap[3]), R));
    n[4] = dw::add_abs(dw::mul(dw::splat(k.ddt), I), D);
    float* o = out + y * g.pitch + x;
    const bool second = x + 32 < g.nx;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      st2(o, f * g.plane, n[f].h, second);
      st2(o, (5 + f) * g.plane, neg2(n[f].l), second);
    }
  }
};

// The D2Q5 one-step update of the plain (MODE_PLAIN), deviation (MODE_DEV) and split
// (MODE_SPLIT) storages, as step1_kernel computes it: lap5 of S, E, I, R (lap5_diff of the
// value minus that of the compensation for the split S), then seird_cell / seird_cell_dev /
// seird_cell_split, in their packed forms.  Ring planes: S, E, I, R, [the compensation of
// S], D -- the planes with x neighbours first.
template <int MODE>
struct D2q5Cell {
  static constexpr int kPlanes = mode_planes<MODE>(), kHaloPlanes = kPlanes - 1;
  static constexpr int kRing = 8, kWarps = 4, kMinBlocks = 4;
  static constexpr bool kPacked = true;
  static constexpr int kD = kPlanes - 1;  // ring plane of D
  const float* in;
  float* out;
  Coeffs<float> k;
  __device__ __forceinline__ const float* src(int f, const GridView& g) const {
    if (MODE == MODE_SPLIT) return in + (f == 4 ? 5 : f == 5 ? 4 : f) * g.plane;
    return in + f * g.plane;
  }
  using State = NoState;
  __device__ __forceinline__ void update(const GridView& g, const Rows& r, int i, int64_t x, int64_t y, State&,
                                         bool) const {
    float2 c[4], lap[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float* P = r.C + f * kStStride;
      c[f] = ld2(P, i);
      const float2 l = ld2(P, i - 1), rt = ld2(P, i + 1);
      const float2 u = ld2(r.U + f * kStStride, i), d = ld2(r.N + f * kStStride, i);
      if (MODE == MODE_SPLIT && f == 0) {
        const float* Q = r.C + 4 * kStStride;
        const float2 lq = lap5diff_x2(ld2(Q, i), ld2(Q, i - 1), ld2(Q, i + 1), ld2(r.U + 4 * kStStride, i),
                                      ld2(r.N + 4 * kStStride, i));
        lap[f] = add2(lap5diff_x2(c[f], l, rt, u, d), neg2(lq));
      } else {
        lap[f] = lap5x2(c[f], add2(l, rt), u, d);
      }
    }
    const float2 D = ld2(r.C + kD * kStStride, i);
    float2 n[6];
    if constexpr (MODE == MODE_SPLIT)
      seird_cell2_split(k, c[0], ld2(r.C + 4 * kStStride, i), c[1], c[2], c[3], D, lap[0], lap[1], lap[2], lap[3],
                        n[0], n[5], n[1], n[2], n[3], n[4]);
    else
      seird_cell2<MODE == MODE_DEV>(k, c[0], c[1], c[2], c[3], D, lap[0], lap[1], lap[2], lap[3], n[0], n[1], n[2],
                                    n[3], n[4]);
    float* o = out + y * g.pitch + x;
    const bool second = x + 32 < g.nx;
#pragma unroll
    for (int f = 0; f < kPlanes; ++f) st2(o, f * g.plane, n[f], second);
  }
};

// The D2Q9 lattice: the isotropic nine-point laplacian (4 sum_axes + sum_diagonals - 20 c)/6
// of S, E, I, R and seird_cell, with the sums in the order ((l + r) + (u + d)) and
// ((ne + nw) + (se + sw)).  Each row's pair sum h = row[x - 1] + row[x + 1] enters three
// laplacians -- as l + r of its own row, ne + nw of the row below, se + sw of the row above --
// so a column carries h and the centre value of rows y - 1 and y from row to row and reads
// only row y + 1 from the ring.  Under no-flux a link that leaves the domain sees the cell's
// own value (halfway bounce-back); the cells on the domain's edge take the links one by one
// from the ring with that substitution.
struct D2q9Cell {
  static constexpr int kPlanes = 5, kHaloPlanes = 4, kRing = 8, kWarps = 4, kMinBlocks = 4;
  static constexpr bool kPacked = true;
  const float* in;
  float* out;
  Coeffs<float> k;
  __device__ __forceinline__ const float* src(int f, const GridView& g) const { return in + f * g.plane; }
  struct State {
    float2 hU[4], hC[4], cU[4], cC[4];  // pair sums and centres of rows y - 1 and y
  };
  // the laplacians of a cell on the no-flux boundary, every link from the ring
  __device__ __forceinline__ void wall_lap(const GridView& g, const Rows& r, int i, int64_t x, int64_t y,
                                           float (&lap)[4]) const {
    const bool wl = x == 0, wr = x == g.nx - 1, wd = y == 0, wu = y == g.ny - 1;
    const float sixth = 1.f / 6.f;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float* Pd = r.U + f * kStStride;
      const float* Pc = r.C + f * kStStride;
      const float* Pu = r.N + f * kStStride;
      const float cc = Pc[i];
      const float l = wl ? cc : Pc[i - 1], rt = wr ? cc : Pc[i + 1];
      const float d = wd ? cc : Pd[i], u = wu ? cc : Pu[i];
      const float ne = (wr || wu) ? cc : Pu[i + 1], nw = (wl || wu) ? cc : Pu[i - 1];
      const float se = (wr || wd) ? cc : Pd[i + 1], sw = (wl || wd) ? cc : Pd[i - 1];
      const float axes = add_rn(add_rn(l, rt), add_rn(u, d));
      const float diag = add_rn(add_rn(ne, nw), add_rn(se, sw));
      lap[f] = mul_rn(fma_rn(-20.f, cc, fma_rn(4.f, axes, diag)), sixth);
    }
  }
  __device__ __forceinline__ void update(const GridView& g, const Rows& r, int i, int64_t x, int64_t y, State& s,
                                         bool first) const {
    if (first) {
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float* Pd = r.U + f * kStStride;
        const float* Pc = r.C + f * kStStride;
        s.hU[f] = add2(ld2(Pd, i - 1), ld2(Pd, i + 1));
        s.cU[f] = ld2(Pd, i);
        s.hC[f] = add2(ld2(Pc, i - 1), ld2(Pc, i + 1));
        s.cC[f] = ld2(Pc, i);
      }
    }
    float2 c[4], lap[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float* Pu = r.N + f * kStStride;
      const float2 nc = ld2(Pu, i);
      const float2 hN = add2(ld2(Pu, i - 1), ld2(Pu, i + 1));
      const float2 axes = add2(s.hC[f], add2(nc, s.cU[f]));
      const float2 diag = add2(hN, s.hU[f]);
      lap[f] = mul2(fma2(splat2(-20.f), s.cC[f], fma2(splat2(4.f), axes, diag)), splat2(1.f / 6.f));
      c[f] = s.cC[f];
      s.hU[f] = s.hC[f];
      s.cU[f] = s.cC[f];
      s.hC[f] = hN;
      s.cC[f] = nc;
    }
    const bool second = x + 32 < g.nx;
    if (g.bc != 0) {
      const bool edge_row = y == 0 || y == g.ny - 1;
      float wl[4];
      if (edge_row || x == 0 || x == g.nx - 1) {
        wall_lap(g, r, i, x, y, wl);
#pragma unroll
        for (int f = 0; f < 4; ++f) lap[f].x = wl[f];
      }
      if (second && (edge_row || x + 32 == g.nx - 1)) {
        wall_lap(g, r, i + 32, x + 32, y, wl);
#pragma unroll
        for (int f = 0; f < 4; ++f) lap[f].y = wl[f];
      }
    }
    float2 n[5];
    seird_cell2<0>(k, c[0], c[1], c[2], c[3], ld2(r.C + 4 * kStStride, i), lap[0], lap[1], lap[2], lap[3], n[0], n[1],
                   n[2], n[3], n[4]);
    float* o = out + y * g.pitch + x;
#pragma unroll
    for (int f = 0; f < 5; ++f) st2(o, f * g.plane, n[f], second);
  }
};

// Spatially varying, axis-anisotropic diffusion in flux form: the link coefficients
// (k_a(x) + k_a(x + c_i)) / 2 of the links +x, +y, -x, -y, each flux term rounded on its own
// and summed as ((+x) + (-x)) + ((+y) + (-y)) (the order of vard.cu), then seird_cell.  Ring
// planes: S, E, I, R, kx (x neighbours), ky, D.
struct VardCell {
  static constexpr int kPlanes = 7, kHaloPlanes = 5, kRing = 8, kWarps = 4, kMinBlocks = 3;
  static constexpr bool kPacked = true;
  const float* in;
  const float* kx;
  const float* ky;
  float* out;
  Coeffs<float> k;
  __device__ __forceinline__ const float* src(int f, const GridView& g) const {
    return f < 4 ? in + f * g.plane : f == 4 ? kx : f == 5 ? ky : in + 4 * g.plane;
  }
  using State = NoState;
  __device__ __forceinline__ void update(const GridView& g, const Rows& r, int i, int64_t x, int64_t y, State&,
                                         bool) const {
    const float2 half = splat2(0.5f);
    const float* A = r.C + 4 * kStStride;
    const float2 a = ld2(A, i), b = ld2(r.C + 5 * kStStride, i);
    const float2 lxp = mul2(half, add2(a, ld2(A, i + 1)));
    const float2 lyp = mul2(half, add2(b, ld2(r.N + 5 * kStStride, i)));
    const float2 lxm = mul2(half, add2(a, ld2(A, i - 1)));
    const float2 lym = mul2(half, add2(b, ld2(r.U + 5 * kStStride, i)));
    float2 c[4], flux[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float* P = r.C + f * kStStride;
      const float2 cc = ld2(P, i), ncc = neg2(cc);
      const float2 t1 = mul2(lxp, add2(ld2(P, i + 1), ncc));
      const float2 t2 = mul2(lyp, add2(ld2(r.N + f * kStStride, i), ncc));
      const float2 t3 = mul2(lxm, add2(ld2(P, i - 1), ncc));
      const float2 t4 = mul2(lym, add2(ld2(r.U + f * kStStride, i), ncc));
      // ((+x) + (-x)) + ((+y) + (-y)), in scalar adds: summed with packed adds (the intrinsic
      // or inline PTX) the results differed in the last bit from the scalar kernel's on 0.1-1%
      // of cells, although the packed add, multiply and FMA each match their scalar forms bit
      // for bit on 4M random operand pairs (subnormals included); with scalar adds of the
      // packed products every bit agrees
      flux[f] = make_float2(add_rn(add_rn(t1.x, t3.x), add_rn(t2.x, t4.x)),
                            add_rn(add_rn(t1.y, t3.y), add_rn(t2.y, t4.y)));
      c[f] = cc;
    }
    float2 n[5];
    seird_cell2<0>(k, c[0], c[1], c[2], c[3], ld2(r.C + 6 * kStStride, i), flux[0], flux[1], flux[2], flux[3], n[0],
                   n[1], n[2], n[3], n[4]);
    float* o = out + y * g.pitch + x;
    const bool second = x + 32 < g.nx;
#pragma unroll
    for (int f = 0; f < 5; ++f) st2(o, f * g.plane, n[f], second);
  }
};

// One launch: a warp per (strip, 128-row segment).  Cutting the rows so that the items fill
// the resident warps exactly once (segments of ~900 rows at 8192^2, no tail wave) measured
// slower at 8192^2 for every cell -- 65.2 against 76.3 GLUPS for the Kahan storage, 114.9
// against 141.6 for D2Q9 -- so the grid keeps short segments and several waves.
template <class Cell>
cudaError_t launch_stream(const GridView& g, const Cell& cell, cudaStream_t s) {
  constexpr size_t smem = sizeof(float) * Cell::kRing * Cell::kPlanes * kStStride * Cell::kWarps;
  // the dynamic shared-memory limit, set once per device (a bit per device in an atomic mask:
  // host threads may launch concurrently; setting it twice is harmless)
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && !(done.load(std::memory_order_acquire) & (1ull << (dev & 63)))) {
    cudaFuncSetAttribute(stream_kernel<Cell>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done.fetch_or(1ull << (dev & 63), std::memory_order_release);
  }
  const int64_t nstrips = (g.nx + kStCols - 1) / kStCols;
  const int64_t items = nstrips * ((g.ny + kStSeg - 1) / kStSeg);
  if (items > 0x7fffffffLL - Cell::kWarps) return cudaErrorInvalidConfiguration;
  if (items == 0) return cudaSuccess;
  stream_kernel<Cell><<<(unsigned)((items + Cell::kWarps - 1) / Cell::kWarps), 32 * Cell::kWarps, smem, s>>>(
      g, cell, (int)nstrips, (int)items);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stream_d2q5(int precision, const GridView& g, const void* coeffs, const void* in, void* out,
                               cudaStream_t s) {
  const Coeffs<float>& k = *static_cast<const Coeffs<float>*>(coeffs);
  const float* src = static_cast<const float*>(in);
  float* dst = static_cast<float*>(out);
  switch (precision) {
    case SSLBM_FP32: return launch_stream(g, D2q5Cell<MODE_PLAIN>{src, dst, k}, s);
    case SSLBM_FP32_DEV: return launch_stream(g, D2q5Cell<MODE_DEV>{src, dst, k}, s);
    case SSLBM_FP32_SPLIT: return launch_stream(g, D2q5Cell<MODE_SPLIT>{src, dst, k}, s);
    case SSLBM_FP32_KAHAN: return launch_stream(g, KahanCell{src, dst, k}, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stream_dw(const GridView& g, const void* coeffs, const void* in, void* out, cudaStream_t s) {
  const Coeffs<double>& c = *static_cast<const Coeffs<double>*>(coeffs);
  auto pair = [](double v) {  // hi = v rounded to float, lo = the rest rounded to float
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  };
  DwCoeffs k;
  for (int f = 0; f < 4; ++f) k.dl[f] = pair(c.dl[f]);
  k.bdt = pair(c.bdt), k.adt = pair(c.adt), k.gdt = pair(c.gdt), k.rdt = pair(c.rdt), k.ddt = pair(c.ddt);
  return launch_stream(g, DwCell{static_cast<const float*>(in), static_cast<float*>(out), k}, s);
}

cudaError_t launch_stream_d2q9(const GridView& g, const void* coeffs, const void* in, void* out, cudaStream_t s) {
  return launch_stream(g, D2q9Cell{static_cast<const float*>(in), static_cast<float*>(out),
                                   *static_cast<const Coeffs<float>*>(coeffs)},
                       s);
}

cudaError_t launch_stream_vard(const GridView& g, const void* coeffs, const void* kx, const void* ky, const void* in,
                               void* out, cudaStream_t s) {
  return launch_stream(g, VardCell{static_cast<const float*>(in), static_cast<const float*>(kx),
                                   static_cast<const float*>(ky), static_cast<float*>(out),
                                   *static_cast<const Coeffs<float>*>(coeffs)},
                       s);
}

}  // namespace sslbm
