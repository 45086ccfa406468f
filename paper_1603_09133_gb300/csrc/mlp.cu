// Rank predictor: a 3-layer MLP (NFEAT -> 64 -> 64 -> 1, ReLU, sigmoid) that
// maps cheap per-block features to r_i / n_i, so the compression step can use
// a randomized range finder of width r_hat + p instead of a full SVD.
//
// Training runs in FP32 on the GPU: the full-batch gradient of the mean
// squared error is computed per CTA over 128 samples (forward, backward and
// the weight-gradient sums in shared memory, fixed summation order) and the
// per-CTA partial gradients are reduced in a fixed order by the Adam update
// kernel, so a training run is deterministic.  Inference runs with FP16
// weights and FP16 activations (FP32 accumulation).
//
// Parameter layout (flat): W1 (64 x NFEAT, row-major), b1 (64), W2 (64 x 64),
// b2 (64), w3 (64), b3 (1).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "kernels.h"
#include "mlp_infer.cuh"
#include "rng.cuh"

namespace ce {

namespace {

constexpr int H = kMlpHidden;
constexpr int NF = kMlpFeatures;
constexpr int OW1 = 0, OB1 = OW1 + H * NF, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + H;
constexpr int S = 128;       // samples per CTA in the gradient kernel
constexpr int GT = 256;      // threads of the gradient kernel
constexpr int HP = H + 1;    // padded row of the per-sample activations


__global__ void mlp_init_kernel(float* theta, unsigned long long seed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  float sc = 0.f;
  if (p < OB1)
    sc = sqrtf(2.0f / NF);
  else if (p >= OW2 && p < OB2)
    sc = sqrtf(2.0f / H);
  else if (p >= OW3 && p < OB3)
    sc = sqrtf(2.0f / H);
  float v = 0.f;
  if (sc > 0.f) {  // Box-Muller from two 53-bit uniforms
    const unsigned long long a = splitmix64(seed * 0x100000001ull + 2ull * p);
    const unsigned long long b = splitmix64(seed * 0x100000001ull + 2ull * p + 1);
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    v = static_cast<float>(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2)) * sc;
  }
  theta[p] = v;
}

// Partial gradient of 0.5 * mean (y - t)^2 over the samples of this CTA.
__global__ void __launch_bounds__(GT) mlp_grad_kernel(const float* X, const float* t, int ns,
                                                      const float* theta, float* partial) {
  extern __shared__ float sm[];
  float* th = sm;                 // kMlpParams
  float* xs = th + kMlpParams;    // S x NF
  float* z1 = xs + S * NF;        // S x HP  (then d1)
  float* z2 = z1 + S * HP;        // S x HP  (then d2)
  float* d3 = z2 + S * HP;        // S
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * S;
  const int cnt = min(S, ns - s0);
  const float inv = 1.0f / ns;
  for (int p = tid; p < kMlpParams; p += GT) th[p] = theta[p];
  for (int e = tid; e < S * NF; e += GT) xs[e] = (e / NF < cnt) ? X[(size_t)s0 * NF + e] : 0.f;
  __syncthreads();
  // forward, one sample per thread
  for (int s = tid; s < cnt; s += GT) {
    const float* x = xs + s * NF;
    for (int j = 0; j < H; ++j) {
      float z = th[OB1 + j];
      for (int f = 0; f < NF; ++f) z += th[OW1 + j * NF + f] * x[f];
      z1[s * HP + j] = z;
    }
    for (int j = 0; j < H; ++j) {
      float z = th[OB2 + j];
      for (int k = 0; k < H; ++k) z += th[OW2 + j * H + k] * fmaxf(z1[s * HP + k], 0.f);
      z2[s * HP + j] = z;
    }
    float z3 = th[OB3];
    for (int k = 0; k < H; ++k) z3 += th[OW3 + k] * fmaxf(z2[s * HP + k], 0.f);
    const float y = mlp_sigmoid(z3);
    d3[s] = (y - t[s0 + s]) * y * (1.f - y) * inv;
  }
  __syncthreads();
  // gradients of the output layer (sums over the samples in order)
  float* g = partial + (size_t)blockIdx.x * kMlpParams;
  for (int k = tid; k <= H; k += GT) {
    float acc = 0.f;
    for (int s = 0; s < cnt; ++s) acc += d3[s] * (k < H ? fmaxf(z2[s * HP + k], 0.f) : 1.f);
    g[k < H ? OW3 + k : OB3] = acc;
  }
  __syncthreads();
  // d2 = d3 w3 * [z2 > 0]  (in place of z2)
  for (int e = tid; e < cnt * H; e += GT) {
    const int s = e / H, j = e - s * H;
    z2[s * HP + j] = (z2[s * HP + j] > 0.f) ? d3[s] * th[OW3 + j] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < H * H + H; e += GT) {   // W2 and b2
    float acc = 0.f;
    if (e < H * H) {
      const int j = e / H, k = e - j * H;
      for (int s = 0; s < cnt; ++s) acc += z2[s * HP + j] * fmaxf(z1[s * HP + k], 0.f);
      g[OW2 + e] = acc;
    } else {
      const int j = e - H * H;
      for (int s = 0; s < cnt; ++s) acc += z2[s * HP + j];
      g[OB2 + j] = acc;
    }
  }
  __syncthreads();
  // d1 = (W2^T d2) * [z1 > 0]  (in place of z1; one thread per (s, k))
  for (int e = tid; e < cnt * H; e += GT) {
    const int s = e / H, k = e - s * H;
    float acc = 0.f;
    for (int j = 0; j < H; ++j) acc += z2[s * HP + j] * th[OW2 + j * H + k];
    z1[s * HP + k] = (z1[s * HP + k] > 0.f) ? acc : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < H * NF + H; e += GT) {  // W1 and b1
    float acc = 0.f;
    if (e < H * NF) {
      const int j = e / NF, f = e - j * NF;
      for (int s = 0; s < cnt; ++s) acc += z1[s * HP + j] * xs[s * NF + f];
      g[OW1 + e] = acc;
    } else {
      const int j = e - H * NF;
      for (int s = 0; s < cnt; ++s) acc += z1[s * HP + j];
      g[OB1 + j] = acc;
    }
  }
}

// g = sum of the partial gradients (fixed order); optionally one Adam step.
__global__ void mlp_reduce_adam_kernel(const float* partial, int nblk, float* grad, float* theta,
                                       float* m, float* v, float lr, int step) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += partial[(size_t)b * kMlpParams + p];
  if (grad) grad[p] = g;
  if (theta) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.f - powf(b1, (float)step));
    const float vh = vv / (1.f - powf(b2, (float)step));
    theta[p] -= lr * mh / (sqrtf(vh) + eps);
  }
}

__global__ void mlp_pack_kernel(const float* theta, __half* model) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) model[p] = __float2half_rn(theta[p]);
}

__global__ void mlp_predict_kernel(const float* X, int ns, const __half* model, float* out) {
  __shared__ float xs[8][NF];
  __shared__ float hb[8][H];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * 8 + warp;
  if (s >= ns) return;
  for (int f = lane; f < NF; f += 32) xs[warp][f] = X[(size_t)s * NF + f];
  __syncwarp();
  const float y = mlp_infer_warp(model, xs[warp], hb[warp]);
  if (lane == 0) out[s] = y;
}

size_t grad_smem() { return sizeof(float) * (kMlpParams + S * NF + 2 * S * HP + S); }

cudaError_t grad_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)grad_smem());
  if (e == cudaSuccess) done = true;
  return e;
}

}  // namespace

cudaError_t mlp_init(float* theta, unsigned long long seed, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  mlp_init_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta, seed);
  return cudaGetLastError();
}

cudaError_t mlp_grad(const float* X, const float* t, int ns, const float* theta, float* partial,
                     float* grad, cudaStream_t s) {
  cudaError_t e = grad_smem_attr();
  if (e != cudaSuccess) return e;
  const int nblk = (ns + S - 1) / S;
  g_launches.fetch_add(2, std::memory_order_relaxed);
  mlp_grad_kernel<<<nblk, GT, grad_smem(), s>>>(X, t, ns, theta, partial);
  mlp_reduce_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(partial, nblk, grad, nullptr, nullptr,
                                                                   nullptr, 0.f, 0);
  return cudaGetLastError();
}

cudaError_t mlp_adam_step(const float* X, const float* t, int ns, float* theta, float* partial,
                          float* m, float* v, float lr, int step, cudaStream_t s) {
  cudaError_t e = grad_smem_attr();
  if (e != cudaSuccess) return e;
  const int nblk = (ns + S - 1) / S;
  g_launches.fetch_add(2, std::memory_order_relaxed);
  mlp_grad_kernel<<<nblk, GT, grad_smem(), s>>>(X, t, ns, theta, partial);
  mlp_reduce_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(partial, nblk, nullptr, theta, m, v, lr,
                                                                   step);
  return cudaGetLastError();
}

int mlp_partial_blocks(int ns) { return (ns + S - 1) / S; }

cudaError_t mlp_pack(const float* theta, void* model, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  mlp_pack_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta, static_cast<__half*>(model));
  return cudaGetLastError();
}

cudaError_t mlp_predict(const float* X, int ns, const void* model, float* out, cudaStream_t s) {
  if (ns <= 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  mlp_predict_kernel<<<(ns + 7) / 8, 256, 0, s>>>(X, ns, static_cast<const __half*>(model), out);
  return cudaGetLastError();
}

}  // namespace ce
