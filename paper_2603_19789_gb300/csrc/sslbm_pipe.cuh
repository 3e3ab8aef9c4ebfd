// sslbm_pipe.cuh -- one tile of the temporal-blocked SSLBM pipeline (FP32 variants),
// shared by the single-grid launch (sslbm_kernels.cu) and the persistent ensemble launch
// (ensemble.cu).
//
// A tile is a 128-column strip (4 columns per lane, 16-byte accesses; K columns of halo
// on each side are recomputed) times a segment of rows [y0, y1), advanced K steps.  The
// CTA's K warps form a pipeline over the time levels: warp s computes level s+1 of the
// wavefront.  Warp 0 brings level-0 rows in with cp.async into a shared-memory ring
// several rows ahead; each level's output row goes through a double-buffered
// shared-memory slot to the next warp, one CTA barrier per row; the last warp writes
// level K to global memory.  Each warp keeps only its own level's two previous rows in
// registers.  x neighbours come from warp shuffles.  Rows and columns outside the domain
// are loaded as ghost images (periodic wrap or the even mirror extension), which the
// uniform stencil keeps consistent, so no boundary logic is needed inside the pipeline.
// The arithmetic is the packed form of seird_cell / seird_cell_dev, bit-identical to the
// one-step kernel.
#pragma once
#include "sslbm_internal.cuh"

namespace sslbm {

constexpr int kRing0 = 4;  // level-0 rows in flight per tile

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
// rl[s-1]: level-s rows from warp s-1 to warp s, double-buffered by iteration parity.
template <int K>
struct PipeSmem {
  float r0[kRing0][5][128];
  float rl[K - 1][2][5][128];
};

// One iteration of warp s: read its level's next row N from src, compute level s+1 of row C
// from P, C, N (x neighbours by shuffles), and pass it to warp s+1 through the slot of parity
// par, or (last warp) write it to row r of the output.  Ends with the CTA barrier.
template <int MODE, int K>
__device__ __forceinline__ void pipe_row(PipeSmem<K>& sm, const GridView& g, const Coeffs<float>& k,
                                         const float* src, const float2 (&P)[5][2], const float2 (&C)[5][2],
                                         float2 (&N)[5][2], float* __restrict__ out, const int s, const int lane,
                                         const int par, const bool writer, const int64_t xs, const int64_t r,
                                         const int64_t y0, const int64_t y1) {
  constexpr unsigned kFull = 0xffffffffu;
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    const float4 t = *reinterpret_cast<const float4*>(src + 128 * f);
    N[f][0] = make_float2(t.x, t.y);
    N[f][1] = make_float2(t.z, t.w);
  }
  float2 lp[4][2];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float L = __shfl_up_sync(kFull, C[f][1].y, 1);
    const float R = __shfl_down_sync(kFull, C[f][0].x, 1);
    // left + right neighbour of columns 0..3, then the packed rest of lap5
    const float2 lr0 = make_float2(__fadd_rn(L, C[f][0].y), __fadd_rn(C[f][0].x, C[f][1].x));
    const float2 lr1 = make_float2(__fadd_rn(C[f][0].y, C[f][1].y), __fadd_rn(C[f][1].x, R));
    lp[f][0] = lap5x2(C[f][0], lr0, P[f][0], N[f][0]);
    lp[f][1] = lap5x2(C[f][1], lr1, P[f][1], N[f][1]);
  }
  float2 M[5][2];
#pragma unroll
  for (int h = 0; h < 2; ++h)
    seird_cell2<MODE == MODE_DEV>(k, C[0][h], C[1][h], C[2][h], C[3][h], C[4][h], lp[0][h], lp[1][h], lp[2][h],
                                  lp[3][h], M[0][h], M[1][h], M[2][h], M[3][h], M[4][h]);
  if (s < K - 1) {
    float* dst = &sm.rl[s < K - 1 ? s : 0][par][0][4 * lane];
#pragma unroll
    for (int f = 0; f < 5; ++f)
      *reinterpret_cast<float4*>(dst + 128 * f) = make_float4(M[f][0].x, M[f][0].y, M[f][1].x, M[f][1].y);
  } else if (writer && r >= y0 && r < y1) {
    float* o = out + r * g.pitch + xs;
    if (xs + 3 < g.nx) {
#pragma unroll
      for (int f = 0; f < 5; ++f)
        *reinterpret_cast<float4*>(o + f * g.plane) = make_float4(M[f][0].x, M[f][0].y, M[f][1].x, M[f][1].y);
    } else {
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        const float v[4] = {M[f][0].x, M[f][0].y, M[f][1].x, M[f][1].y};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (xs + jj < g.nx) o[f * g.plane + jj] = v[jj];
      }
    }
  }
  __syncthreads();
}

// WRAP16: periodic grid with nx a multiple of 4 -- every lane's four columns, ghosts
// included, are one contiguous 16-byte group at the wrapped position, so all loads are
// L2-only cp.async.cg (required when other CTAs of the same launch wrote the input, since
// L1 is not coherent).
template <int MODE, int K, bool WRAP16 = false>
__device__ __forceinline__ void pipe_tile(PipeSmem<K>& sm, const GridView& g, const Coeffs<float>& k,
                                          const float* __restrict__ in, float* __restrict__ out,
                                          const int strip, const int64_t y0, const int64_t y1) {
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
  // Warp s computes, at iteration q, level s+1 of row q - 2s - 1 from level-s rows
  // q-2s-2 (P), q-2s-1 (C) and q-2s (N).  Level-0 rows span [y0-K, y1+K); the last warp
  // finishes row y1-1 at iteration y1 + 2K - 2.
  const int64_t qa = y0 - K, qb = y1 + 2 * K - 1, load_end = y1 + K;

  for (int i = threadIdx.x; i < kRing0 * 5 * 128; i += 32 * K) (&sm.r0[0][0][0])[i] = 0.f;
  for (int i = threadIdx.x; i < (K - 1) * 2 * 5 * 128; i += 32 * K) (&sm.rl[0][0][0][0])[i] = 0.f;
  __syncthreads();

  auto issue = [&](int64_t q) {  // warp 0: copy level-0 row q into its ring slot
    if (!loads) return;
    const int slot = (int)((q - qa) % kRing0);
    const int64_t row = ghost_index(q, g.ny, g.bc) * g.pitch;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const float* src = in + f * g.plane + row;
      float* dst = &sm.r0[slot][f][4 * lane];
      if (WRAP16) {
        cp_async16(dst, src + xw);
      } else if (vec_ok) {
        cp_async16(dst, src + xs);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) cp_async4(dst + j, src + xm[j]);
      }
    }
  };
  if (s == 0) {
#pragma unroll
    for (int p = 0; p < kRing0 - 1; ++p) {
      if (qa + p < load_end) issue(qa + p);
      cp_async_commit();
    }
  }

  // Three row buffers rotate through the roles P (row q-2s-2), C (q-2s-1) and N (q-2s) of
  // this warp's level, unrolled three ways so that no row is copied between registers.
  float2 RA[5][2], RB[5][2], RC[5][2];
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int h = 0; h < 2; ++h) RA[f][h] = RB[f][h] = make_float2(0.f, 0.f);

  const int nq = (int)(qb - qa), nload = (int)(load_end - qa), par0 = (int)((qa - 1) & 1);
  const int64_t r0 = qa - 2 * K + 1;  // the level-K row the last warp finishes at iteration 0
  // Row source of iteration j (q = qa + j): warp 0's ring slot, or the previous warp's slot.
  auto fetch = [&](int j) -> const float* {
    if (s == 0) {
      if (j + kRing0 - 1 < nload) issue(qa + j + kRing0 - 1);
      cp_async_commit();
      cp_async_wait<kRing0 - 1>();
      return &sm.r0[j & (kRing0 - 1)][0][4 * lane];
    }
    return &sm.rl[s - 1][(j + par0) & 1][0][4 * lane];
  };
  int j = 0;
  for (; j + 3 <= nq; j += 3) {
    pipe_row<MODE, K>(sm, g, k, fetch(j), RA, RB, RC, out, s, lane, (j + par0 + 1) & 1, writer, xs, r0 + j, y0, y1);
    pipe_row<MODE, K>(sm, g, k, fetch(j + 1), RB, RC, RA, out, s, lane, (j + par0) & 1, writer, xs, r0 + j + 1, y0,
                      y1);
    pipe_row<MODE, K>(sm, g, k, fetch(j + 2), RC, RA, RB, out, s, lane, (j + par0 + 1) & 1, writer, xs, r0 + j + 2,
                      y0, y1);
  }
  if (j < nq)
    pipe_row<MODE, K>(sm, g, k, fetch(j), RA, RB, RC, out, s, lane, (j + par0 + 1) & 1, writer, xs, r0 + j, y0, y1);
  if (j + 1 < nq)
    pipe_row<MODE, K>(sm, g, k, fetch(j + 1), RB, RC, RA, out, s, lane, (j + par0) & 1, writer, xs, r0 + j + 1, y0,
                      y1);
  if (s == 0) cp_async_wait<0>();
}

}  // namespace sslbm
