// fno_fused.cuh -- the surrogate's forward pass as three fused kernels per layer.
//
// Per grid row (b, y) the network is local except for the spectral convolution's
// transform along y.  So the forward pass runs as (1 + 4L launches)
//
//   row kernel, lift:   h0 = A0 x + a0;                        H1 = h0 Fx
//   per layer l:
//     y kernel:         T = Fy H1 (per channel), combined into the complex modes hat_l
//     mix kernel:       hatg = mix(hat_l, R_l)   (per mode, the whole batch)
//     inverse y kernel: U = expand(hatg), G1 = Fyi U / n^2   (per output channel)
//     row kernel, mid:  z = B_l h + G1 Fxi + b_l, h_l = gelu(z);  H1 = h_l Fx
//     row kernel, last: z = B_L h + G1 Fxi + b_L = h_L;
//                       y_c = sigma_c (x_c + (Q2 gelu(Q1 h_L + q1) + q2)_c)
//
// The row kernel keeps one row of every activation in shared memory: the channel map and
// the inverse transform along x are one product with K = W + 4m ([B_l | G1] times
// [h ; Fxi]), the next layer's transform along x reads the new row straight from shared
// memory, and the last layer's projection MLP never leaves the chip.  Products run on BF16
// tensor cores (mma.sync m16n8k16, FP32 accumulation) with the same BF16 rounding points
// as the unfused path: activations, H1, G1 and U in BF16, everything else FP32.
// H1 and G1 are stored row-major per grid row: [b][y][channel][4m].
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sslbm {
namespace fno_fused {

typedef __nv_bfloat16 bf16;

enum RowMode { ROW_LIFT = 0, ROW_MID = 1, ROW_LAST = 2 };

struct RowArgs {
  int B, n;
  const float* x;     // [B][8][n][n] network input
  const bf16* hin;    // [B][W][n][n] h_{l-1} (mid/last)
  const bf16* g1;     // [B][n][W][4m] G1 / n^2 (mid/last)
  const bf16* F;      // [n][4m] Fx (its transpose is Fxi)
  const float* A0;    // [W][8], a0 [W] (lift)
  const float* a0;
  const bf16* Bl;     // [W][W] (mid/last)
  const float* bl;    // [W]
  const bf16* Q1;     // [H][W] (last)
  const float* q1;    // [H]
  const bf16* Q2;     // [5][H] (last)
  const float* q2;    // [5]
  bf16* hout;         // [B][W][n][n] h_l (lift/mid always, last when storing)
  bf16* zout;         // [B][W][n][n] z_l (mid, when storing)
  bf16* H1out;        // [B][n][W][4m] (lift/mid)
  bf16* zp;           // [B][H][n][n] (last, when storing)
  bf16* p;            // [B][H][n][n] (last, when storing)
  float* y;           // [B][5][n][n] (last)
  int store;          // write the intermediates the backward pass reads
};

// true when (W, m, H, n) has a fused instantiation
bool supported(int W, int m, int H, int n);

cudaError_t launch_row(int mode, int W, int m, int H, const RowArgs& a, cudaStream_t s);
// hat[b][c][2m*m][2] (FP32) from H1
cudaError_t launch_dft_y(int W, int m, int B, int n, const bf16* H1, const bf16* Fy, float* hat,
                         cudaStream_t s);
// G1[b][y][o][4m] = bf16(Fyi expand(mix(hat, R)) * scale); hatg [B][W][2m*m][2] FP32 scratch
cudaError_t launch_mix_idft_y(int W, int m, int B, int n, const float* hat, const float* R,
                              const bf16* Fyi, bf16* G1, float* hatg, float scale, cudaStream_t s);

// Per-cell channel products on tensor cores (any shape with rows, K, cols <= 64):
//   cell_map:   C[b](rows x P) = alpha Wm (rows x K) S[b] (K x P) + beta C[b], Wm(r, k) = Wm[r sWr + k sWk]
//   cell_wgrad: dW (rows x cols, FP32) += sum_b D[b](rows x P) A[b](cols x P)^T
// S, A: FP32 or BF16; C: FP32 or BF16; operands are rounded to BF16, accumulation is FP32.
cudaError_t cell_map(int B, int rows, int K, int64_t P, const bf16* Wm, int64_t sWr, int64_t sWk, const void* S,
                     int s_bf16, void* C, int c_bf16, float alpha, float beta, cudaStream_t s);
cudaError_t cell_wgrad(int B, int rows, int cols, int64_t P, const float* D, const void* A, int a_bf16, float* dW,
                       cudaStream_t s);

}  // namespace fno_fused
}  // namespace sslbm
