// Kernels of the learned warm start (nn.cu), used by the network runtime (nn_api.cu).
// Tensors are channels-last BF16 [N][D][H][W][C]; weights FP32 masters [27][Cin][Cout] with
// BF16 copies W [27][Cin][Cout] (data gradient) and W^T [27][Cout][Cin] (forward).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace hrt {
namespace nn {

using bf16 = __nv_bfloat16;

// 'same' 3x3x3 convolution: out = act(bias + conv(in, B)); Cin % 16 == 0, Cout % 32 == 0.
// Forward: B = W^T; data gradient: in = dY, B = W, flip = true, no bias, no ReLU.
// conv3d runs on the tcgen05 tensor cores (nn_tc.cu); conv3d_mma is the same convolution with
// warp-level mma.sync, kept as the measured baseline.
// Bp (may be null): B packed by pack_tma_weights, which the TMA-fed kernel needs; without it
// conv3d runs the per-phase kernel.
cudaError_t conv3d(const bf16* in, const bf16* B, const bf16* Bp, const float* bias, bf16* out, int N, int D, int H,
                   int W, int Cin, int Cout, bool flip, bool relu, cudaStream_t s);
cudaError_t conv3d_phased(const bf16* in, const bf16* B, const float* bias, bf16* out, int N, int D, int H, int W, int Cin,
                   int Cout, bool flip, bool relu, cudaStream_t s);
cudaError_t conv3d_mma(const bf16* in, const bf16* B, const float* bias, bf16* out, int N, int D, int H, int W,
                       int Cin, int Cout, bool flip, bool relu, cudaStream_t s);
// after a synchronisation of s: *failed = 1 if a tcgen05 convolution block gave up a wait
cudaError_t tc_status(int* failed, cudaStream_t s);
// dw [27][Cin][Cout] += sum over voxels (FP32 atomics; zero dw first).  conv3d_wgrad runs on the
// tcgen05 tensor cores (nn_tc.cu): the brick form (halo loaded once for 9 taps by TMA) for
// Cin % 32 == 0 and Cout % 8 == 0, else the stacked-tap form for Cin % 16 == 0 (<= 128, or a
// multiple of 64) and Cout % 32 == 0, other shapes on mma.sync (conv3d_wgrad_mma).
cudaError_t conv3d_wgrad(const bf16* in, const bf16* dy, float* dw, int N, int D, int H, int W, int Cin, int Cout,
                         cudaStream_t s);
cudaError_t conv3d_wgrad_mma(const bf16* in, const bf16* dy, float* dw, int N, int D, int H, int W, int Cin, int Cout,
                             cudaStream_t s);
cudaError_t bias_grad(const bf16* dy, float* db, long long V, int C, cudaStream_t s);
cudaError_t relu_mask(bf16* g, const bf16* h, long long n, cudaStream_t s);
cudaError_t pool2(const bf16* x, bf16* y, int N, int D, int H, int W, int C, cudaStream_t s);
cudaError_t pool2_back(const bf16* dy, bf16* dx, int N, int D, int H, int W, int C, bool accumulate, cudaStream_t s);
// y [N][D][H][W][C1 + C2] = concat(upsample2(low [N][D/2][H/2][W/2][C1]), skip [N][D][H][W][C2])
cudaError_t concat_up(const bf16* low, const bf16* skip, bf16* y, int N, int D, int H, int W, int C1, int C2,
                      cudaStream_t s);
// gradient of concat_up: dlow (overwritten), dskip (accumulated)
cudaError_t concat_up_back(const bf16* g, bf16* dlow, bf16* dskip, int N, int D, int H, int W, int C1, int C2,
                           cudaStream_t s);
cudaError_t head_forward(const bf16* h, const float* w, const float* b, float* y, long long NV, int C, cudaStream_t s);
cudaError_t mse_loss(const float* y, const float* t, float* dy, double* loss, long long NV, cudaStream_t s);
cudaError_t head_backward(const bf16* h, const float* w, const float* dy, bf16* dh, float* dw, float* db, long long NV,
                          int C, cudaStream_t s);
cudaError_t adam(float* p, const float* g, float* m, float* v, long long n, float lr, int step, cudaStream_t s);
cudaError_t weights_bf16(const float* w, bf16* wb, bf16* wt, int cin_real, int Cin, int Cout, cudaStream_t s);
// Weights for the TMA-fed convolution: B [27][Cout][Cin] rearranged as [Cin/8][Cout/BN][27][BN][8]
// (BN = tma_tile_n(Cout) output channels per tile), so that what one pipeline stage needs of an
// 8-channel slice -- all 27 taps of one output-channel tile -- is one contiguous block, moved by
// one bulk copy.  Cin % 8 == 0, Cout % 32 == 0.
constexpr int tma_tile_n(int Cout) { return Cout % 64 == 0 ? 64 : 32; }
cudaError_t pack_tma_weights(const bf16* B, bf16* Bp, int Cin, int Cout, cudaStream_t s);
cudaError_t init_uniform(float* p, long long n, float bound, unsigned long long seed, cudaStream_t s);
cudaError_t pack_input(const float* x, bf16* y, long long NV, int cin, int Cpad, cudaStream_t s);
cudaError_t bf16_to_f32(const bf16* x, float* y, long long n, cudaStream_t s);
cudaError_t f32_to_bf16(const float* x, bf16* y, long long n, cudaStream_t s);

}  // namespace nn
}  // namespace hrt
