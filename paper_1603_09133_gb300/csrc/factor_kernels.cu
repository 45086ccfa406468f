// CUDA kernels of the CE factorization around the row kernel (sm_103a):
// scatter of the CSR values into the level-1 block pairs, the reassembly
// copies that join J blocks into super-blocks (Section 2.4), and the blocked
// FP64 Cholesky of the dense remainder A_K (Algorithm 1, last step).
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"

namespace ce {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int LD = kNMax + 1;   // shared-memory leading dimension
constexpr int kChunk = kNMax;   // rows of F_i^T per Householder pass
constexpr int kMaxSweeps = 40;  // Jacobi sweep cap (bounded loop)
constexpr int kMaxTargets = 32;

template <typename T>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double v = 2.220446049250313e-16;
};
template <>
struct Eps<float> {
  static constexpr float v = 1.1920928955078125e-07f;
};

template <typename T>
struct Tiny;  // smallest normal number
template <>
struct Tiny<double> {
  static constexpr double v = 2.2250738585072014e-308;
};
template <>
struct Tiny<float> {
  static constexpr float v = 1.1754943508222875e-38f;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int width_of(const LevelDev& L, int k, int ci) {
  return (L.colour[k] < ci) ? L.rank[k] : L.n[k];
}

__device__ void set_status(int* status, int code, int level, int block, int reason = 0,
                           int pivot = -1, double value = 0.0) {
  if (atomicCAS(status, 0, code) == 0) {
    status[1] = level;
    status[2] = block;
    status[3] = reason;
    status[4] = pivot;
    *reinterpret_cast<double*>(status + 6) = value;
  }
}

template <typename T>
__global__ void scatter_csr_kernel(const int64_t* scatter, const double* val, int64_t nnz, T* pool) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = scatter[e];
    if (d >= 0) pool[d] = static_cast<T>(val[e]);
  }
}

template <typename Ts, typename Td>
__global__ void copy_tasks_kernel(const CopyTask* tasks, const Ts* src, Td* dst) {
  const CopyTask t = tasks[blockIdx.x];
  const int total = t.rows * t.cols;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int a = e / t.cols, b = e - a * t.cols;
    Td v = static_cast<Td>(src[t.src_off + (int64_t)a * t.src_ld + b]);
    if (!t.transpose)
      dst[t.dst_off + (int64_t)(t.r0 + a) * t.dst_ld + t.c0 + b] = v;
    else
      dst[t.dst_off + (int64_t)(t.r0 + b) * t.dst_ld + t.c0 + a] = v;
  }
}

// ---------------- coarse dense Cholesky (FP64, lower, row-major) -----------
// One dense matrix per independent system: system y = blockIdx.y has size
// desc[y] and starts at element desc[nsys + y] of the coarse storage.
// Right-looking, panels of NB = 32 columns: POTRF of the diagonal tile (one
// CTA), TRSM of the rows below (one CTA per 32 rows), SYRK of the trailing
// lower triangle (one CTA per 32 x 32 tile).  FP64 runs at about 2 fused
// multiply-adds per clock per SM on this GPU, so the panel is kept narrow
// (short serial chains) and the trailing update is cut into many small tiles
// to spread it over all SMs.
constexpr int NB = 32;
constexpr int NBL = NB + 1;

__device__ __forceinline__ bool coarse_sys(double*& A, int& n, const int64_t* desc, int nsys, int k0) {
  const int y = blockIdx.y;
  n = static_cast<int>(desc[y]);
  A += desc[nsys + y];
  return k0 < n;
}

// 1 / sqrt(x) for x > 0 in FP64: a single-precision estimate refined by two
// Newton-Raphson steps y <- y (3 - x y^2) / 2 (each doubles the correct bits,
// 24 -> 48 -> beyond 53); inputs outside the float range take the library
// function.
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(x > 1e-30 && x < 1e30)) return rsqrt(x);
  double y = static_cast<double>(rsqrtf(static_cast<float>(x)));
  const double hx = 0.5 * x;
  y = y * (1.5 - hx * y * y);
  y = y * (1.5 - hx * y * y);
  return y;
}

// Cholesky of the diagonal tile, then its inverse (for the TRSM below):
// tile inverse of system y at Tinv[y * NB * NB] (row-major, lower)
__global__ void __launch_bounds__(256) potrf_tile_kernel(double* A, const int64_t* desc, int nsys, int k0,
                                                         int level, int* status, double* Tinv) {
  if (*status) return;
  int n;
  if (!coarse_sys(A, n, desc, nsys, k0)) return;
  __shared__ double t[NB * NBL];
  __shared__ double x[NB * NBL];
  const int nb = min(NB, n - k0);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    t[a * NBL + b] = A[(int64_t)(k0 + a) * n + k0 + b];
  }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    const double piv = t[k * NBL + k];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) set_status(status, CE_ERR_NOT_SPD, level, -1 - (int)blockIdx.y, 1, k0 + k, piv);
      return;
    }
    const double inv = rsqrt_nr(piv);
    // column k below the pivot (each thread scales the entries it reads next)
    const int rem = nb - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int a = k + 1 + e / rem, b = k + 1 + e % rem;
      if (b <= a) t[a * NBL + b] -= (t[a * NBL + k] * inv) * (t[b * NBL + k] * inv);
    }
    __syncthreads();
    for (int a = k + 1 + threadIdx.x; a < nb; a += blockDim.x) t[a * NBL + k] *= inv;
    if (threadIdx.x == 0) t[k * NBL + k] = piv * inv;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    A[(int64_t)(k0 + a) * n + k0 + b] = (b <= a) ? t[a * NBL + b] : 0.0;
  }
  // inverse of the lower tile: column j by forward substitution (thread j),
  // with the reciprocals of the diagonal formed once, in parallel
  __shared__ double rd[NB];
  if (threadIdx.x < nb) rd[threadIdx.x] = 1.0 / t[threadIdx.x * NBL + threadIdx.x];
  __syncthreads();
  const int j = threadIdx.x;
  if (j < nb) {
    for (int a = 0; a < j; ++a) x[a * NBL + j] = 0.0;
    for (int a = j; a < nb; ++a) {
      double s0 = (a == j) ? 1.0 : 0.0, s1 = 0.0;
      int k = j;
      for (; k + 1 < a; k += 2) {
        s0 -= t[a * NBL + k] * x[k * NBL + j];
        s1 -= t[a * NBL + k + 1] * x[(k + 1) * NBL + j];
      }
      if (k < a) s0 -= t[a * NBL + k] * x[k * NBL + j];
      x[a * NBL + j] = (s0 + s1) * rd[a];
    }
  }
  __syncthreads();
  double* Ti = Tinv + (size_t)blockIdx.y * NB * NB;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    Ti[a * NB + b] = x[a * NBL + b];
  }
}

// L_ik = A_ik L_kk^{-T} for the 32-row tiles below the diagonal tile k0, as a
// product with the tile inverse: L_ik[a][b] = sum_{c <= b} A_ik[a][c] Tinv[b][c]
__global__ void __launch_bounds__(256) trsm_tile_kernel(double* A, const int64_t* desc, int nsys, int k0,
                                                        const int* status, const double* Tinv) {
  if (*status) return;
  int n;
  if (!coarse_sys(A, n, desc, nsys, k0)) return;
  __shared__ double Ti[NB * NBL];
  __shared__ double X[NB * NBL];
  const int nb = min(NB, n - k0);
  const int i0 = k0 + nb + blockIdx.x * NB;
  if (i0 >= n) return;
  const int rows = min(NB, n - i0);
  const double* T = Tinv + (size_t)blockIdx.y * NB * NB;
  for (int e = threadIdx.x; e < nb * nb; e += 256) {
    int a = e / nb, b = e - a * nb;
    Ti[a * NBL + b] = T[a * NB + b];
  }
  for (int e = threadIdx.x; e < rows * nb; e += 256) {
    int a = e / nb, b = e - a * nb;
    X[a * NBL + b] = A[(int64_t)(i0 + a) * n + k0 + b];
  }
  __syncthreads();
  double out[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = threadIdx.x + u * 256, a = e / NB, b = e % NB;
    double s0 = 0.0, s1 = 0.0;
    if (a < rows && b < nb) {
      int c = 0;
      for (; c + 1 <= b; c += 2) {
        s0 += X[a * NBL + c] * Ti[b * NBL + c];
        s1 += X[a * NBL + c + 1] * Ti[b * NBL + c + 1];
      }
      if (c <= b) s0 += X[a * NBL + c] * Ti[b * NBL + c];
    }
    out[u] = s0 + s1;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = threadIdx.x + u * 256, a = e / NB, b = e % NB;
    if (a < rows && b < nb) A[(int64_t)(i0 + a) * n + k0 + b] = out[u];
  }
}

// A_ij -= L_ik L_jk^T for the trailing 32 x 32 tiles j <= i (2 x 2 outputs
// per thread)
__global__ void __launch_bounds__(256) syrk_tile_kernel(double* A, const int64_t* desc, int nsys, int k0,
                                                        const int* status) {
  if (*status) return;
  int n;
  if (!coarse_sys(A, n, desc, nsys, k0)) return;
  __shared__ double Li[NB * NBL];
  __shared__ double Lj[NB * NBL];
  const int nb = min(NB, n - k0);
  const int t0 = k0 + nb;
  // blockIdx.x enumerates the lower-triangular tile pairs (ti >= tj)
  int ti = 0, idx = blockIdx.x;
  while (idx > ti) {
    idx -= ti + 1;
    ++ti;
  }
  const int tj = idx;
  const int i0 = t0 + ti * NB, j0 = t0 + tj * NB;
  if (i0 >= n) return;
  const int ri = min(NB, n - i0), rj = min(NB, n - j0);
  for (int e = threadIdx.x; e < NB * nb; e += 256) {
    int a = e / nb, b = e - a * nb;
    Li[a * NBL + b] = a < ri ? A[(int64_t)(i0 + a) * n + k0 + b] : 0.0;
    Lj[a * NBL + b] = a < rj ? A[(int64_t)(j0 + a) * n + k0 + b] : 0.0;
  }
  __syncthreads();
  const int a0 = (threadIdx.x / 16) * 2, b0 = (threadIdx.x % 16) * 2;
  double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
  for (int c = 0; c < nb; ++c) {
    const double x0 = Li[a0 * NBL + c], x1 = Li[(a0 + 1) * NBL + c];
    const double y0 = Lj[b0 * NBL + c], y1 = Lj[(b0 + 1) * NBL + c];
    c00 += x0 * y0;
    c01 += x0 * y1;
    c10 += x1 * y0;
    c11 += x1 * y1;
  }
  double* C = A + (int64_t)i0 * n + j0;
  if (a0 < ri && b0 < rj) C[(int64_t)a0 * n + b0] -= c00;
  if (a0 < ri && b0 + 1 < rj) C[(int64_t)a0 * n + b0 + 1] -= c01;
  if (a0 + 1 < ri && b0 < rj) C[(int64_t)(a0 + 1) * n + b0] -= c10;
  if (a0 + 1 < ri && b0 + 1 < rj) C[(int64_t)(a0 + 1) * n + b0 + 1] -= c11;
}

}  // namespace

cudaError_t launch_scatter_csr(int esize, const int64_t* scatter, const double* val, int64_t nnz,
                               void* pool, cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<int64_t>((nnz + 255) / 256, (int64_t)device_sms() * 16));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (esize == 8)
    scatter_csr_kernel<double><<<grid, 256, 0, s>>>(scatter, val, nnz, (double*)pool);
  else
    scatter_csr_kernel<float><<<grid, 256, 0, s>>>(scatter, val, nnz, (float*)pool);
  return cudaGetLastError();
}

cudaError_t launch_copy_tasks(int esize_src, int esize_dst, const CopyTask* tasks, int ntasks,
                              const void* src, void* dst, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (esize_src == 8 && esize_dst == 8)
    copy_tasks_kernel<double, double><<<ntasks, 128, 0, s>>>(tasks, (const double*)src, (double*)dst);
  else if (esize_src == 4 && esize_dst == 4)
    copy_tasks_kernel<float, float><<<ntasks, 128, 0, s>>>(tasks, (const float*)src, (float*)dst);
  else if (esize_src == 4 && esize_dst == 8)
    copy_tasks_kernel<float, double><<<ntasks, 128, 0, s>>>(tasks, (const float*)src, (double*)dst);
  else
    copy_tasks_kernel<double, float><<<ntasks, 128, 0, s>>>(tasks, (const double*)src, (float*)dst);
  return cudaGetLastError();
}

cudaError_t coarse_cholesky(double* A, const int64_t* desc, int nsys, int nmax, int level, int* status,
                            double* tinv, cudaStream_t s) {
  // the grids cover the largest system; smaller ones return early
  for (int k0 = 0; k0 < nmax; k0 += NB) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    potrf_tile_kernel<<<dim3(1, nsys), 256, 0, s>>>(A, desc, nsys, k0, level, status, tinv);
    const int nb = std::min(NB, nmax - k0);
    const int below = nmax - k0 - nb;
    if (below > 0) {
      const int tiles = (below + NB - 1) / NB;
      g_launches.fetch_add(2, std::memory_order_relaxed);
      trsm_tile_kernel<<<dim3(tiles, nsys), 256, 0, s>>>(A, desc, nsys, k0, status, tinv);
      syrk_tile_kernel<<<dim3(tiles * (tiles + 1) / 2, nsys), 256, 0, s>>>(A, desc, nsys, k0, status);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t coarse_tile_scratch(int nsys) { return (size_t)nsys * NB * NB * sizeof(double); }

}  // namespace ce
