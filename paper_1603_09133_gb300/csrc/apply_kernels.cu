// CUDA kernels of the CE solve x = Q^T L^{-T} L^{-1} Q b (solve proposition,
// Section 2.5) and of the FP64 conjugate-gradient loop around it.
//
// The level vector of level l holds block i at [vec_off[i], vec_off[i]+n_i).
// Forward step of block i (same order as the factorization, one launch per
// colour): y_i <- U_i^T y_i; z = L_hat^{-1} y_i[r:]; y_i[:r] -= W_b^T z;
// y_p[:w_p] -= W_p^T z for every close p; z is stored in y_i[r:].  The basis
// parts then move to the next level's vector (super-blocks of J children).
// The backward step is the transpose, in reverse order.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"

namespace ce {

namespace {

constexpr int kApplyThreads = 128;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int width_of_a(const LevelDev& L, int k, int ci) {
  return (L.colour[k] < ci) ? L.rank[k] : L.n[k];
}

template <typename T>
__global__ void __launch_bounds__(kApplyThreads) apply_fwd_kernel(LevelDev L, int first, double* vec) {
  __shared__ double ys[kNMax], yt[kNMax], z[kNMax];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = L.order[first + blockIdx.x];
  const int n = L.n[i];
  if (n == 0) return;
  const int r = L.rank[i], m = n - r, ci = L.colour[i];
  double* v = vec + L.vec_off[i];
  const T* U = reinterpret_cast<const T*>(L.U) + L.u_off[i];
  const T* Lh = reinterpret_cast<const T*>(L.L) + L.l_off[i];
  const T* W = reinterpret_cast<const T*>(L.W) + L.w_off[i];
  for (int a = tid; a < n; a += kApplyThreads) ys[a] = v[a];
  __syncthreads();
  for (int a = tid; a < n; a += kApplyThreads) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += static_cast<double>(U[k * n + a]) * ys[k];
    yt[a] = s;
  }
  __syncthreads();
  if (warp == 0) {
    for (int a = 0; a < m; ++a) {
      double s = 0.0;
      for (int k = lane; k < a; k += 32) s += static_cast<double>(Lh[a * m + k]) * z[k];
      s = warp_sum_d(s);
      if (lane == 0) z[a] = (yt[r + a] - s) / static_cast<double>(Lh[a * m + a]);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int b = tid; b < r; b += kApplyThreads) {
    double s = yt[b];
    for (int k = 0; k < m; ++k) s -= static_cast<double>(W[k * r + b]) * z[k];
    v[b] = s;
  }
  for (int a = tid; a < m; a += kApplyThreads) v[r + a] = z[a];
  if (m == 0) return;
  int colst = n;
  for (int t = L.close_ptr[i]; t < L.close_ptr[i + 1]; ++t) {
    const int p = L.close_blk[t];
    const int w = width_of_a(L, p, ci);
    const T* Wp = W + (int64_t)n * colst;
    double* vp = vec + L.vec_off[p];
    for (int c = tid; c < w; c += kApplyThreads) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += static_cast<double>(Wp[k * w + c]) * z[k];
      vp[c] -= s;
    }
    colst += L.n[p];
  }
}

template <typename T>
__global__ void __launch_bounds__(kApplyThreads) apply_bwd_kernel(LevelDev L, int first, double* vec) {
  __shared__ double xf[kNMax], rhs[kNMax];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = L.order[first + blockIdx.x];
  const int n = L.n[i];
  if (n == 0) return;
  const int r = L.rank[i], m = n - r, ci = L.colour[i];
  double* v = vec + L.vec_off[i];
  const T* U = reinterpret_cast<const T*>(L.U) + L.u_off[i];
  const T* Lh = reinterpret_cast<const T*>(L.L) + L.l_off[i];
  const T* W = reinterpret_cast<const T*>(L.W) + L.w_off[i];
  for (int a = tid; a < n; a += kApplyThreads) xf[a] = v[a];   // [x_b; z]
  __syncthreads();
  constexpr int nw = kApplyThreads / 32;
  for (int a = warp; a < m; a += nw) {
    double s = 0.0;
    for (int b = lane; b < r; b += 32) s += static_cast<double>(W[a * r + b]) * xf[b];
    int colst = n;
    for (int t = L.close_ptr[i]; t < L.close_ptr[i + 1]; ++t) {
      const int p = L.close_blk[t];
      const int w = width_of_a(L, p, ci);
      const T* Wp = W + (int64_t)n * colst;
      const double* vp = vec + L.vec_off[p];
      for (int c = lane; c < w; c += 32) s += static_cast<double>(Wp[a * w + c]) * vp[c];
      colst += L.n[p];
    }
    s = warp_sum_d(s);
    if (lane == 0) rhs[a] = xf[r + a] - s;
  }
  __syncthreads();
  if (warp == 0) {
    for (int a = m - 1; a >= 0; --a) {
      double s = 0.0;
      for (int k = a + 1 + lane; k < m; k += 32) s += static_cast<double>(Lh[k * m + a]) * xf[r + k];
      s = warp_sum_d(s);
      if (lane == 0) xf[r + a] = (rhs[a] - s) / static_cast<double>(Lh[a * m + a]);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int a = tid; a < n; a += kApplyThreads) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += static_cast<double>(U[a * n + k]) * xf[k];
    v[a] = s;
  }
}

// basis parts between a level vector and the next (forward: gather)
__global__ void level_move_kernel(LevelDev L, double* cur, double* next, int forward) {
  const int i = blockIdx.x;
  const int r = L.rank[i];
  const int64_t src = L.vec_off[i], dst = L.gdst[i];
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    if (forward)
      next[dst + a] = cur[src + a];
    else
      cur[src + a] = next[dst + a];
  }
}

__global__ void perm_kernel(const int32_t* perm, int64_t n, const double* in, double* out,
                            int gather) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (gather)
      out[k] = in[perm[k]];
    else
      out[perm[k]] = in[k];
  }
}

// dense lower-triangular solves with the coarse factor, one CTA
constexpr int kCS = 1024;
constexpr int kPan = 64;

__global__ void __launch_bounds__(kCS) coarse_solve_kernel(const double* Lc, int n, double* yg) {
  extern __shared__ double y[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = kCS / 32;
  for (int a = tid; a < n; a += kCS) y[a] = yg[a];
  __syncthreads();
  // forward: L y = b
  for (int s0 = 0; s0 < n; s0 += kPan) {
    const int pe = min(n, s0 + kPan);
    if (warp == 0) {
      for (int a = s0; a < pe; ++a) {
        double s = 0.0;
        for (int k = s0 + lane; k < a; k += 32) s += Lc[(int64_t)a * n + k] * y[k];
        s = warp_sum_d(s);
        if (lane == 0) y[a] = (y[a] - s) / Lc[(int64_t)a * n + a];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int a = pe + warp; a < n; a += nw) {
      double s = 0.0;
      for (int k = s0 + lane; k < pe; k += 32) s += Lc[(int64_t)a * n + k] * y[k];
      s = warp_sum_d(s);
      if (lane == 0) y[a] -= s;
    }
    __syncthreads();
  }
  // backward: L^T x = y
  for (int pe = n; pe > 0; pe -= kPan) {
    const int s0 = max(0, pe - kPan);
    if (warp == 0) {
      for (int a = pe - 1; a >= s0; --a) {
        double s = 0.0;
        for (int k = a + 1 + lane; k < pe; k += 32) s += Lc[(int64_t)k * n + a] * y[k];
        s = warp_sum_d(s);
        if (lane == 0) y[a] = (y[a] - s) / Lc[(int64_t)a * n + a];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int c = tid; c < s0; c += kCS) {
      double s = 0.0;
      for (int a = s0; a < pe; ++a) s += Lc[(int64_t)a * n + c] * y[a];
      y[c] -= s;
    }
    __syncthreads();
  }
  for (int a = tid; a < n; a += kCS) yg[a] = y[a];
}

// ---------------- PCG building blocks -----------------------------------
constexpr int kRed = 256;

__device__ double block_sum(double v) {
  __shared__ double red[kRed / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_d(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = (lane < kRed / 32) ? red[lane] : 0.0;
    s = warp_sum_d(s);
  }
  __syncthreads();
  return s;
}

// y = A x and partial sums of x . y
__global__ void __launch_bounds__(kRed) spmv_dot_kernel(int64_t n, const int64_t* rowptr,
                                                        const int32_t* col, const double* val,
                                                        const double* x, double* y, double* partial) {
  double acc = 0.0;
  for (int64_t row = blockIdx.x * (int64_t)kRed + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * kRed) {
    double s = 0.0;
    for (int64_t e = rowptr[row]; e < rowptr[row + 1]; ++e) s += val[e] * x[col[e]];
    y[row] = s;
    acc += x[row] * s;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRed) dot_kernel(int64_t n, const double* a, const double* b,
                                                   double* partial) {
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)kRed + threadIdx.x; k < n; k += (int64_t)gridDim.x * kRed)
    acc += a[k] * b[k];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRed) reduce_kernel(const double* partial, int nparts, double* out) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < nparts; k += kRed) acc += partial[k];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

// scal: [0] rz, [1] pAp, [2] alpha, [3] rr, [4] rz_new, [5] beta
__global__ void __launch_bounds__(kRed) update_xr_kernel(int64_t n, double* x, double* r,
                                                         const double* p, const double* Ap,
                                                         const double* scal, double* partial) {
  const double alpha = scal[2];
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)kRed + threadIdx.x; k < n; k += (int64_t)gridDim.x * kRed) {
    x[k] += alpha * p[k];
    const double rk = r[k] - alpha * Ap[k];
    r[k] = rk;
    acc += rk * rk;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void update_p_kernel(int64_t n, double* p, const double* z, const double* scal, int first) {
  const double beta = first ? 0.0 : scal[5];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    p[k] = z[k] + beta * p[k];
}

__global__ void pcg_scalars_kernel(double* scal, int stage) {
  if (stage == 0) {
    scal[2] = scal[0] / scal[1];  // alpha = rz / pAp
  } else {
    scal[5] = scal[4] / scal[0];  // beta = rz_new / rz
    scal[0] = scal[4];
  }
}

template <typename T>
cudaError_t apply_launch(const LevelDev& L, int first, int count, double* vec, cudaStream_t s,
                         bool fwd) {
  if (count <= 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (fwd)
    apply_fwd_kernel<T><<<count, kApplyThreads, 0, s>>>(L, first, vec);
  else
    apply_bwd_kernel<T><<<count, kApplyThreads, 0, s>>>(L, first, vec);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply_fwd(int esize, const LevelDev& L, int first, int count, double* vec,
                             cudaStream_t s) {
  return esize == 8 ? apply_launch<double>(L, first, count, vec, s, true)
                    : apply_launch<float>(L, first, count, vec, s, true);
}

cudaError_t launch_apply_bwd(int esize, const LevelDev& L, int first, int count, double* vec,
                             cudaStream_t s) {
  return esize == 8 ? apply_launch<double>(L, first, count, vec, s, false)
                    : apply_launch<float>(L, first, count, vec, s, false);
}

cudaError_t launch_level_move(const LevelDev& L, double* cur, double* next, int forward,
                              cudaStream_t s) {
  if (L.M <= 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  level_move_kernel<<<L.M, 64, 0, s>>>(L, cur, next, forward);
  return cudaGetLastError();
}

cudaError_t launch_perm(const int32_t* perm, int64_t n, const double* in, double* out, int gather,
                        cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 152 * 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  perm_kernel<<<grid, 256, 0, s>>>(perm, n, in, out, gather);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const double* Lc, int n, double* y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * static_cast<size_t>(n);
  static int attr_set = 0;
  if (smem > 48 * 1024 && smem > static_cast<size_t>(attr_set)) {
    cudaError_t e = cudaFuncSetAttribute(coarse_solve_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = static_cast<int>(smem);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  coarse_solve_kernel<<<1, kCS, smem, s>>>(Lc, n, y);
  return cudaGetLastError();
}

cudaError_t launch_spmv_dot(int64_t n, const int64_t* rowptr, const int32_t* col,
                            const double* val, const double* x, double* y, double* partial,
                            int nparts, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  spmv_dot_kernel<<<nparts, kRed, 0, s>>>(n, rowptr, col, val, x, y, partial);
  return cudaGetLastError();
}

cudaError_t launch_dot(int64_t n, const double* a, const double* b, double* partial, int nparts,
                       cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  dot_kernel<<<nparts, kRed, 0, s>>>(n, a, b, partial);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partial, int nparts, double* out, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  reduce_kernel<<<1, kRed, 0, s>>>(partial, nparts, out);
  return cudaGetLastError();
}

cudaError_t launch_update_xr(int64_t n, double* x, double* r, const double* p, const double* Ap,
                             const double* scal, double* partial, int nparts, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  update_xr_kernel<<<nparts, kRed, 0, s>>>(n, x, r, p, Ap, scal, partial);
  return cudaGetLastError();
}

cudaError_t launch_update_p(int64_t n, double* p, const double* z, const double* scal, int first,
                            cudaStream_t s) {
  const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 152 * 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  update_p_kernel<<<grid, 256, 0, s>>>(n, p, z, scal, first);
  return cudaGetLastError();
}

cudaError_t launch_pcg_scalars(double* scal, int stage, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  pcg_scalars_kernel<<<1, 1, 0, s>>>(scal, stage);
  return cudaGetLastError();
}

}  // namespace ce
