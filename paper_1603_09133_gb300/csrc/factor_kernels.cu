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
constexpr int NB = 64;
constexpr int NBL = NB + 1;

__device__ __forceinline__ bool coarse_sys(double*& A, int& n, const int64_t* desc, int nsys, int k0) {
  const int y = blockIdx.y;
  n = static_cast<int>(desc[y]);
  A += desc[nsys + y];
  return k0 < n;
}

__global__ void potrf_tile_kernel(double* A, const int64_t* desc, int nsys, int k0, int level, int* status) {
  if (*status) return;
  int n;
  if (!coarse_sys(A, n, desc, nsys, k0)) return;
  __shared__ double t[NB * NBL];
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
    const double d = sqrt(piv);
    __syncthreads();
    for (int a = k + threadIdx.x; a < nb; a += blockDim.x) {
      if (a == k)
        t[k * NBL + k] = d;
      else
        t[a * NBL + k] /= d;
    }
    __syncthreads();
    const int rem = nb - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int a = k + 1 + e / rem, b = k + 1 + e % rem;
      if (b <= a) t[a * NBL + b] -= t[a * NBL + k] * t[b * NBL + k];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    A[(int64_t)(k0 + a) * n + k0 + b] = (b <= a) ? t[a * NBL + b] : 0.0;
  }
}

// L_ik = A_ik L_kk^{-T} for the row tiles below the diagonal tile k0
__global__ void trsm_tile_kernel(double* A, const int64_t* desc, int nsys, int k0, const int* status) {
  if (*status) return;
  int n;
  if (!coarse_sys(A, n, desc, nsys, k0)) return;
  extern __shared__ double tile_smem[];
  double* Lk = tile_smem;
  double* X = tile_smem + NB * NBL;
  const int nb = min(NB, n - k0);
  const int i0 = k0 + nb + blockIdx.x * NB;
  if (i0 >= n) return;
  const int rows = min(NB, n - i0);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    Lk[a * NBL + b] = A[(int64_t)(k0 + a) * n + k0 + b];
  }
  for (int e = threadIdx.x; e < rows * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    X[a * NBL + b] = A[(int64_t)(i0 + a) * n + k0 + b];
  }
  __syncthreads();
  // row a of X solves  x L^T = a  ->  x_b = (a_b - sum_{c<b} x_c L_bc) / L_bb
  for (int a = threadIdx.x; a < rows; a += blockDim.x) {
    for (int b = 0; b < nb; ++b) {
      double s = X[a * NBL + b];
      for (int c = 0; c < b; ++c) s -= X[a * NBL + c] * Lk[b * NBL + c];
      X[a * NBL + b] = s / Lk[b * NBL + b];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    A[(int64_t)(i0 + a) * n + k0 + b] = X[a * NBL + b];
  }
}

// A_ij -= L_ik L_jk^T for the trailing tiles j <= i
__global__ void syrk_tile_kernel(double* A, const int64_t* desc, int nsys, int k0, const int* status) {
  if (*status) return;
  int n;
  if (!coarse_sys(A, n, desc, nsys, k0)) return;
  extern __shared__ double tile_smem[];
  double* Li = tile_smem;
  double* Lj = tile_smem + NB * NBL;
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
  for (int e = threadIdx.x; e < ri * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    Li[a * NBL + b] = A[(int64_t)(i0 + a) * n + k0 + b];
  }
  for (int e = threadIdx.x; e < rj * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    Lj[a * NBL + b] = A[(int64_t)(j0 + a) * n + k0 + b];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ri * rj; e += blockDim.x) {
    int a = e / rj, b = e - a * rj;
    double s = 0.0;
    for (int c = 0; c < nb; ++c) s += Li[a * NBL + c] * Lj[b * NBL + c];
    A[(int64_t)(i0 + a) * n + j0 + b] -= s;
  }
}

}  // namespace

cudaError_t launch_scatter_csr(int esize, const int64_t* scatter, const double* val, int64_t nnz,
                               void* pool, cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<int64_t>((nnz + 255) / 256, 152 * 16));
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
                            cudaStream_t s) {
  const int tile_bytes = 2 * NB * NBL * static_cast<int>(sizeof(double));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(trsm_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tile_bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(syrk_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // the grids cover the largest system; smaller ones return early
  for (int k0 = 0; k0 < nmax; k0 += NB) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    potrf_tile_kernel<<<dim3(1, nsys), 256, 0, s>>>(A, desc, nsys, k0, level, status);
    const int nb = std::min(NB, nmax - k0);
    const int below = nmax - k0 - nb;
    if (below > 0) {
      const int tiles = (below + NB - 1) / NB;
      g_launches.fetch_add(1, std::memory_order_relaxed);
      trsm_tile_kernel<<<dim3(tiles, nsys), 64, tile_bytes, s>>>(A, desc, nsys, k0, status);
      g_launches.fetch_add(1, std::memory_order_relaxed);
      syrk_tile_kernel<<<dim3(tiles * (tiles + 1) / 2, nsys), 256, tile_bytes, s>>>(A, desc, nsys, k0, status);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ce
