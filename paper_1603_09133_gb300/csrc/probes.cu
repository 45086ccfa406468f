// Arithmetic peak probes: short kernels that keep one execution unit busy,
// timed with CUDA events on the caller's stream.  Their rates are the
// denominators of the roofline fractions of the kernels bound by that unit
// (the row kernel's FP32 FMA work, its 3xTF32 tensor-core products, the FP64
// form's arithmetic).  Not part of the paper.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;   // independent FMA chains per thread (hide the pipe latency)
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == T(-1.25)) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

__device__ __forceinline__ void probe_mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t probe_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// split3 = false: plain TF32 m16n8k8 products (4 independent accumulators per
// warp); true: the 3xTF32 product of the row kernel (operands split into
// hi + lo, three MMAs per product), counted as one product's flops.
template <bool kSplit3>
__global__ void __launch_bounds__(kProbeThreads) mma_probe(float* out, int iters) {
  const int lane = threadIdx.x & 31;
  float av[4], bv[2];
#pragma unroll
  for (int u = 0; u < 4; ++u) av[u] = 1.0f + 1e-3f * (lane + u);
  bv[0] = 0.5f + 1e-3f * lane;
  bv[1] = 0.25f + 1e-3f * lane;
  float c[4][4] = {};
  for (int it = 0; it < iters; ++it) {
    if (kSplit3) {
      uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ah[u] = probe_tf32(av[u]);
        al[u] = probe_tf32(av[u] - __uint_as_float(ah[u]));
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        bh[u] = probe_tf32(bv[u]);
        bl[u] = probe_tf32(bv[u] - __uint_as_float(bh[u]));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        probe_mma_tf32(c[q], al, bh);
        probe_mma_tf32(c[q], ah, bl);
        probe_mma_tf32(c[q], ah, bh);
      }
      av[0] += 1e-7f;   // a new product each iteration (the splits are recomputed)
    } else {
      uint32_t a[4], b[2];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = __float_as_uint(av[u]);
      b[0] = __float_as_uint(bv[0]);
      b[1] = __float_as_uint(bv[1]);
#pragma unroll
      for (int q = 0; q < 4; ++q) probe_mma_tf32(c[q], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int u = 0; u < 4; ++u) s += c[q][u];
  if (s == -1.25f) out[blockIdx.x] = s;
}

}  // namespace

namespace ce {

cudaError_t measure_peak(int kind, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = sms * 8;   // 8 CTAs of 256 threads per SM: 64 warps, full occupancy
  void* out = nullptr;
  e = cudaMallocAsync(&out, grid * sizeof(double), s);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  // flops per launch for `iters` iterations
  auto run = [&](int iters, double& flops) -> cudaError_t {
    const double threads = double(grid) * kProbeThreads;
    switch (kind) {
      case 0:
        fma_probe<float><<<grid, kProbeThreads, 0, s>>>(static_cast<float*>(out), iters, 0.999999f, 1e-7f);
        flops = threads * iters * kUnroll * kChains * 2.0;
        break;
      case 1:
        fma_probe<double><<<grid, kProbeThreads, 0, s>>>(static_cast<double*>(out), iters, 0.999999, 1e-7);
        flops = threads * iters * kUnroll * kChains * 2.0;
        break;
      case 2:
        mma_probe<false><<<grid, kProbeThreads, 0, s>>>(static_cast<float*>(out), iters);
        flops = threads / 32 * iters * 4 * (2.0 * 16 * 8 * 8);
        break;
      default:
        mma_probe<true><<<grid, kProbeThreads, 0, s>>>(static_cast<float*>(out), iters);
        flops = threads / 32 * iters * 4 * (2.0 * 16 * 8 * 8);
        break;
    }
    return cudaGetLastError();
  };
  // iteration counts for launches of a few milliseconds at the expected rates
  const int iters = kind == 0 ? 2048 : kind == 1 ? 64 : kind == 2 ? 4096 : 2048;
  double flops = 0.0;
  e = run(iters, flops);  // warm-up
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    e = run(iters, flops);
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  g_launches.fetch_add(4, std::memory_order_relaxed);
  *tflops = best;
  return e;
}

}  // namespace ce
