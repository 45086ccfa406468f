// FP16 inference of the rank-predictor MLP, shared by the prediction kernel
// and the row kernel.  Layout of the FP16 model (kMlpParams halves):
// W1 (64 x kMlpFeatures, row-major), b1 (64), W2 (64 x 64), b2 (64),
// w3 (64), b3 (1).
#pragma once
#include <cuda_fp16.h>

namespace ce {

constexpr int kMlpHidden = 64;
constexpr int kMlpFeatures = 11;
constexpr int kMlpParams = kMlpHidden * kMlpFeatures + kMlpHidden + kMlpHidden * kMlpHidden +
                           kMlpHidden + kMlpHidden + 1;

__device__ __forceinline__ float mlp_sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }

// One warp: x (kMlpFeatures floats) and hbuf (64 floats) in shared memory.
// Weights and activations are FP16, products accumulate in FP32.  Returns the
// sigmoid output (a predicted r / n) on every lane.
__device__ __forceinline__ float mlp_infer_warp(const __half* model, const float* x, float* hbuf) {
  constexpr int H = kMlpHidden, NF = kMlpFeatures;
  constexpr int OW1 = 0, OB1 = OW1 + H * NF, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
                OB3 = OW3 + H;
  const int lane = threadIdx.x & 31;
  float h1[2];
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float z = __half2float(model[OB1 + j]);
    for (int f = 0; f < NF; ++f)
      z += __half2float(model[OW1 + j * NF + f]) * __half2float(__float2half_rn(x[f]));
    h1[u] = __half2float(__float2half_rn(fmaxf(z, 0.f)));
  }
  __syncwarp();
  hbuf[lane] = h1[0];
  hbuf[lane + 32] = h1[1];
  __syncwarp();
  float z3 = 0.f;
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float z = __half2float(model[OB2 + j]);
    for (int k = 0; k < H; ++k) z += __half2float(model[OW2 + j * H + k]) * hbuf[k];
    z3 += __half2float(model[OW3 + j]) * __half2float(__float2half_rn(fmaxf(z, 0.f)));
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) z3 += __shfl_xor_sync(0xffffffffu, z3, o);
  return mlp_sigmoid(z3 + __half2float(model[OB3]));
}

}  // namespace ce
