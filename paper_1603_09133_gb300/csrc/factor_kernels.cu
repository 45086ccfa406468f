// CUDA kernels of the CE factorization around the row kernel (sm_103a):
// scatter of the CSR values into the level-1 block pairs, the reassembly
// copies that join J blocks into super-blocks (Section 2.4), and the blocked
// FP64 Cholesky of the dense remainder A_K (Algorithm 1, last step).
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <algorithm>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace ce {

namespace {

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

// Cholesky of the nb x nb tile t (shared memory, lower, ld NBL) by one warp
// without CTA barriers: lane a holds row a; step k scales column k below the
// pivot and updates the trailing lower triangle.  false (and the failing
// pivot) when a pivot is not positive.
__device__ bool warp_potrf(double* t, int nb, int lane, int& bad_k, double& bad_v) {
  for (int k = 0; k < nb; ++k) {
    const double piv = t[k * NBL + k];
    if (!(piv > 0.0)) {
      bad_k = k;
      bad_v = piv;
      return false;
    }
    const double inv = rsqrt_nr(piv);
    double lak = 0.0;
    if (lane > k && lane < nb) lak = t[lane * NBL + k] * inv;
    __syncwarp();
    if (lane > k && lane < nb) t[lane * NBL + k] = lak;
    if (lane == k) t[k * NBL + k] = piv * inv;
    __syncwarp();
    if (lane > k && lane < nb)
      for (int b = k + 1; b <= lane; ++b) t[lane * NBL + b] -= lak * t[b * NBL + k];
    __syncwarp();
  }
  return true;
}

// Work items of a panel step for system y (n_y rows, panel at k0): the
// diagonal tile and the row tiles below it (phase A); the copy of the
// factored diagonal tile and the trailing lower tile pairs (phase B).
__device__ __forceinline__ int panel_tiles(int n, int k0) {
  if (k0 >= n) return -1;
  const int nb = min(NB, n - k0);
  return (n - k0 - nb + NB - 1) / NB;
}

constexpr int kCC = 256;

// Dense FP64 Cholesky of every system's coarse matrix in one cooperative
// launch: per 32-column panel, phase A factors the diagonal tile (each work
// item redundantly, by one warp) and solves its own 32-row tile below it
// (L_ik = A_ik L_kk^{-T}, forward substitution per row); the factored tile is
// staged in Tfac[y] because other items still read the original; a grid
// barrier; phase B copies the staged tile and updates the trailing lower
// tiles A_ij -= L_ik L_jk^T; a grid barrier.  A recorded failure turns the
// remaining work off (every CTA still meets every barrier).
__global__ void __launch_bounds__(kCC) coarse_chol_coop_kernel(double* A, const int64_t* desc, int nsys, int nmax,
                                                               int level, int* status, double* Tfac) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double t[NB * NBL], X[NB * NBL], rd[NB];
  __shared__ int s_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k0 = 0; k0 < nmax; k0 += NB) {
    // ---- phase A ----
    int total = 0;
    for (int y = 0; y < nsys; ++y) {
      const int T = panel_tiles(static_cast<int>(desc[y]), k0);
      if (T >= 0) total += 1 + T;
    }
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
      if (tid == 0) s_stop = *(volatile int*)status;   // one reading per CTA: the exit is uniform
      __syncthreads();
      if (s_stop) break;
      int y = 0, r = it;
      for (;; ++y) {
        const int T = panel_tiles(static_cast<int>(desc[y]), k0);
        if (T < 0) continue;
        if (r < 1 + T) break;
        r -= 1 + T;
      }
      const int n = static_cast<int>(desc[y]);
      double* Ay = A + desc[nsys + y];
      const int nb = min(NB, n - k0);
      for (int e = tid; e < nb * nb; e += kCC) {
        const int a = e / nb, c = e - a * nb;
        t[a * NBL + c] = Ay[(int64_t)(k0 + a) * n + k0 + c];
      }
      __syncthreads();
      __shared__ int s_ok;
      if (warp == 0) {
        int bk = 0;
        double bv = 0.0;
        const bool ok = warp_potrf(t, nb, lane, bk, bv);
        if (lane == 0) {
          s_ok = ok;
          if (!ok && r == 0) set_status(status, CE_ERR_NOT_SPD, level, -1 - y, 1, k0 + bk, bv);
        }
        if (ok && lane < nb) rd[lane] = 1.0 / t[lane * NBL + lane];
      }
      __syncthreads();
      if (!s_ok) continue;
      if (r == 0) {
        double* Tf = Tfac + (size_t)y * NB * NB;
        for (int e = tid; e < NB * NB; e += kCC) {
          const int a = e / NB, c = e - a * NB;
          Tf[e] = (a < nb && c <= a) ? t[a * NBL + c] : 0.0;
        }
      } else {
        const int i0 = k0 + nb + (r - 1) * NB, rows = min(NB, n - i0);
        for (int e = tid; e < rows * nb; e += kCC) {
          const int a = e / nb, c = e - a * nb;
          X[a * NBL + c] = Ay[(int64_t)(i0 + a) * n + k0 + c];
        }
        __syncthreads();
        if (tid < rows) {
          for (int c = 0; c < nb; ++c) {
            double s0 = X[tid * NBL + c];
            for (int q = 0; q < c; ++q) s0 -= X[tid * NBL + q] * t[c * NBL + q];
            X[tid * NBL + c] = s0 * rd[c];
          }
        }
        __syncthreads();
        for (int e = tid; e < rows * nb; e += kCC) {
          const int a = e / nb, c = e - a * nb;
          Ay[(int64_t)(i0 + a) * n + k0 + c] = X[a * NBL + c];
        }
      }
      __syncthreads();
    }
    grid.sync();
    // ---- phase B ----
    total = 0;
    for (int y = 0; y < nsys; ++y) {
      const int T = panel_tiles(static_cast<int>(desc[y]), k0);
      if (T >= 0) total += 1 + T * (T + 1) / 2;
    }
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
      if (tid == 0) s_stop = *(volatile int*)status;
      __syncthreads();
      if (s_stop) break;
      int y = 0, r = it;
      for (;; ++y) {
        const int T = panel_tiles(static_cast<int>(desc[y]), k0);
        if (T < 0) continue;
        if (r < 1 + T * (T + 1) / 2) break;
        r -= 1 + T * (T + 1) / 2;
      }
      const int n = static_cast<int>(desc[y]);
      double* Ay = A + desc[nsys + y];
      const int nb = min(NB, n - k0);
      if (r == 0) {
        const double* Tf = Tfac + (size_t)y * NB * NB;
        for (int e = tid; e < nb * nb; e += kCC) {
          const int a = e / nb, c = e - a * nb;
          Ay[(int64_t)(k0 + a) * n + k0 + c] = Tf[a * NB + c];
        }
        __syncthreads();
        continue;
      }
      int ti = 0, idx = r - 1;
      while (idx > ti) {
        idx -= ti + 1;
        ++ti;
      }
      const int tj = idx;
      const int t0 = k0 + nb, i0 = t0 + ti * NB, j0 = t0 + tj * NB;
      const int ri = min(NB, n - i0), rj = min(NB, n - j0);
      for (int e = tid; e < NB * nb; e += kCC) {
        const int a = e / nb, c = e - a * nb;
        t[a * NBL + c] = a < ri ? Ay[(int64_t)(i0 + a) * n + k0 + c] : 0.0;
        X[a * NBL + c] = a < rj ? Ay[(int64_t)(j0 + a) * n + k0 + c] : 0.0;
      }
      __syncthreads();
      const int a0 = (tid / 16) * 2, b0 = (tid % 16) * 2;
      double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
      for (int c = 0; c < nb; ++c) {
        const double x0 = t[a0 * NBL + c], x1 = t[(a0 + 1) * NBL + c];
        const double y0 = X[b0 * NBL + c], y1 = X[(b0 + 1) * NBL + c];
        c00 += x0 * y0;
        c01 += x0 * y1;
        c10 += x1 * y0;
        c11 += x1 * y1;
      }
      double* C = Ay + (int64_t)i0 * n + j0;
      if (a0 < ri && b0 < rj) C[(int64_t)a0 * n + b0] -= c00;
      if (a0 < ri && b0 + 1 < rj) C[(int64_t)a0 * n + b0 + 1] -= c01;
      if (a0 + 1 < ri && b0 < rj) C[(int64_t)(a0 + 1) * n + b0] -= c10;
      if (a0 + 1 < ri && b0 + 1 < rj) C[(int64_t)(a0 + 1) * n + b0 + 1] -= c11;
      __syncthreads();
    }
    grid.sync();
  }
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
  if (nmax <= 0) return cudaSuccess;
  // one resident wave of cooperative CTAs (every CTA meets every grid barrier)
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_chol_coop_kernel, kCC, 0);
    if (e != cudaSuccess) return e;
    cap = std::max(1, std::min(per_sm, 2)) * sms;
  }
  // enough CTAs for the largest panel step's work, at most one wave
  const int T = (nmax + NB - 1) / NB;
  const int64_t work = (int64_t)nsys * (1 + (int64_t)T * (T + 1) / 2);
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(cap, work)));
  void* args[] = {&A, const_cast<int64_t**>(&desc), &nsys, &nmax, &level, &status, &tinv};
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaLaunchCooperativeKernel((const void*)coarse_chol_coop_kernel, dim3(grid), dim3(kCC), args, 0, s);
}

size_t coarse_tile_scratch(int nsys) { return (size_t)nsys * NB * NB * sizeof(double); }

}  // namespace ce
