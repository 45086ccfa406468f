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

#include <cooperative_groups.h>

#include <algorithm>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace ce {

namespace {

constexpr int kApplyThreads = 128;
constexpr int kMaxTgt = 32;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int width_of_a(const LevelDev& L, int k, int ci) {
  return (L.colour[k] < ci) ? L.rank[k] : L.n[k];
}

// Targets of block i's W (basis of i first, then close blocks): width,
// start of their W columns, offset of their values in the level vector and
// the prefix of widths over the flattened column index.
struct Targets {
  int nt;
  int w[kMaxTgt], pre[kMaxTgt + 1];
  int64_t woff[kMaxTgt], voff[kMaxTgt];
};

__device__ void targets_of(const LevelDev& L, int i, int n, int r, Targets& T) {
  const int ci = L.colour[i];
  const int c0 = L.close_ptr[i], c1 = L.close_ptr[i + 1];
  T.nt = min(1 + (c1 - c0), kMaxTgt);
  T.w[0] = r;
  T.woff[0] = 0;
  T.voff[0] = L.vec_off[i];
  T.pre[0] = 0;
  int colst = n;
  for (int t = 1; t < T.nt; ++t) {
    const int p = L.close_blk[c0 + t - 1];
    T.w[t] = width_of_a(L, p, ci);
    T.woff[t] = (int64_t)n * colst;
    T.voff[t] = L.vec_off[p];
    colst += L.n[p];
  }
  for (int t = 0; t < T.nt; ++t) T.pre[t + 1] = T.pre[t] + T.w[t];
}

// Every factor element is read exactly once per apply, so U_i, L_hat_i^{-1}
// and W_i are streamed from global memory (no staging) and the arithmetic is
// done in the factor's own precision T: the FP32 form applies its
// preconditioner in FP32 (the level vectors stay FP64 in memory, so PCG sees
// an FP64 operator whose error is the FP32 rounding of M^{-1}, far below the
// compression tolerance); the FP64 form stays FP64 throughout.

// 4 independent partial sums of x[k] * M[k * stride] for k in [k0, k1)
template <typename T>
__device__ __forceinline__ T dot_strided(const T* __restrict__ M, int stride, const T* x, int k0, int k1) {
  T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int k = k0;
  for (; k + 3 < k1; k += 4) {
    s0 += M[(int64_t)k * stride] * x[k];
    s1 += M[(int64_t)(k + 1) * stride] * x[k + 1];
    s2 += M[(int64_t)(k + 2) * stride] * x[k + 2];
    s3 += M[(int64_t)(k + 3) * stride] * x[k + 3];
  }
  for (; k < k1; ++k) s0 += M[(int64_t)k * stride] * x[k];
  return (s0 + s1) + (s2 + s3);
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Forward step of block i: y_i <- U_i^T y_i; z = L_hat^{-1} y_i[r:];
// y_t[:w_t] -= W_t^T z for every target t (basis of i first); y_i[r:] = z.
template <typename T>
__global__ void __launch_bounds__(kApplyThreads) apply_fwd_kernel(LevelDev L, int first, double* vec) {
  __shared__ T ys[kNMax], yt[kNMax], z[kNMax];
  __shared__ T part[kApplyThreads];
  __shared__ Targets tg;
  const int tid = threadIdx.x;
  const int i = L.order[first + blockIdx.x];
  const int n = L.n[i];
  if (n == 0) return;
  const int r = L.rank[i], m = n - r;
  double* v = vec + L.vec_off[i];
  const T* U = reinterpret_cast<const T*>(L.U) + L.u_off[i];
  const T* Li = reinterpret_cast<const T*>(L.L) + L.l_off[i];
  const T* W = reinterpret_cast<const T*>(L.W) + L.w_off[i];
  for (int a = tid; a < n; a += kApplyThreads) ys[a] = static_cast<T>(v[a]);
  if (tid == 0) targets_of(L, i, n, r, tg);
  __syncthreads();
  // yt = U^T ys: thread (a, g) sums rows k = g (mod G) of column a
  {
    const int G = kApplyThreads / n, a = tid % n, g = tid / n;
    if (g < G) {
      T s = 0;
      for (int k = g; k < n; k += G) s += U[k * n + a] * ys[k];
      part[g * n + a] = s;
    }
    __syncthreads();
    if (tid < n) {
      T s = 0;
      for (int h = 0; h < G; ++h) s += part[h * n + tid];
      yt[tid] = s;
    }
    __syncthreads();
  }
  // z = L_hat^{-1} yt[r:] (lower, row-major: one warp per row)
  {
    const int lane = tid & 31, warp = tid >> 5;
    for (int a = warp; a < m; a += kApplyThreads / 32) {
      T s = 0;
      for (int k = lane; k <= a; k += 32) s += Li[a * m + k] * yt[r + k];
      s = warp_sum_t(s);
      if (lane == 0) z[a] = s;
    }
    __syncthreads();
  }
  for (int a = tid; a < m; a += kApplyThreads) v[r + a] = static_cast<double>(z[a]);
  const int tot = tg.pre[tg.nt];
  for (int f = tid; f < tot; f += kApplyThreads) {
    int t = 0;
    while (f >= tg.pre[t + 1]) ++t;
    const int c = f - tg.pre[t], w = tg.w[t];
    const T s = dot_strided(W + tg.woff[t] + c, w, z, 0, m);
    if (t == 0)
      v[c] = static_cast<double>(yt[c] - s);
    else
      vec[tg.voff[t] + c] -= static_cast<double>(s);
  }
}

// Backward step of block i (transpose, reverse order): rhs = z - W x_t over
// all targets; x_n = L_hat^{-T} rhs; y_i <- U_i [x_b; x_n].
template <typename T>
__global__ void __launch_bounds__(kApplyThreads) apply_bwd_kernel(LevelDev L, int first, double* vec) {
  __shared__ T xf[kNMax], rhs[kNMax];
  __shared__ T xt[kMaxTgt * kNMax];
  __shared__ Targets tg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = L.order[first + blockIdx.x];
  const int n = L.n[i];
  if (n == 0) return;
  const int r = L.rank[i], m = n - r;
  double* v = vec + L.vec_off[i];
  const T* U = reinterpret_cast<const T*>(L.U) + L.u_off[i];
  const T* Li = reinterpret_cast<const T*>(L.L) + L.l_off[i];
  const T* W = reinterpret_cast<const T*>(L.W) + L.w_off[i];
  for (int a = tid; a < n; a += kApplyThreads) xf[a] = static_cast<T>(v[a]);   // [x_b; z]
  if (tid == 0) targets_of(L, i, n, r, tg);
  __syncthreads();
  const int tot = tg.pre[tg.nt];
  for (int f = tid; f < tot; f += kApplyThreads) {
    int t = 0;
    while (f >= tg.pre[t + 1]) ++t;
    const int c = f - tg.pre[t];
    xt[f] = (t == 0) ? xf[c] : static_cast<T>(vec[tg.voff[t] + c]);
  }
  __syncthreads();
  // rhs = z - W x_t: one warp per row of W (contiguous within each target)
  for (int a = warp; a < m; a += kApplyThreads / 32) {
    T s = 0;
    for (int t = 0; t < tg.nt; ++t) {
      const int w = tg.w[t];
      const T* Wt = W + tg.woff[t] + (int64_t)a * w;
      const T* x = xt + tg.pre[t];
      for (int c = lane; c < w; c += 32) s += Wt[c] * x[c];
    }
    s = warp_sum_t(s);
    if (lane == 0) rhs[a] = xf[r + a] - s;
  }
  __syncthreads();
  // x_n = L_hat^{-T} rhs: column a of L_hat^{-1}, contiguous across threads
  for (int a = tid; a < m; a += kApplyThreads) xf[r + a] = dot_strided(Li + a, m, rhs, a, m);
  __syncthreads();
  // y_i = U_i xf: one warp per row
  for (int a = warp; a < n; a += kApplyThreads / 32) {
    T s = 0;
    for (int k = lane; k < n; k += 32) s += U[a * n + k] * xf[k];
    s = warp_sum_t(s);
    if (lane == 0) v[a] = static_cast<double>(s);
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

// Dense triangular solves with the coarse factor L_K (FP64), one grid of
// CTAs cooperating through grid-wide barriers.  L_K is cut into panels of
// kPan rows; Dinv holds the inverses of its diagonal kPan x kPan blocks, so
// a panel is solved by CTA 0 as a small GEMV, and the remaining rows are
// updated by all CTAs.
constexpr int kPan = 64;
constexpr int kCS = 256;

__global__ void __launch_bounds__(kCS) coarse_solve_kernel(const double* Lc, const double* Dinv, int n,
                                                           double* y) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double yp[kPan], yq[kPan];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gw = blockIdx.x * (kCS / 32) + warp, nwarps = gridDim.x * (kCS / 32);
  const int npan = (n + kPan - 1) / kPan;
  // forward: L y = b
  for (int p = 0; p < npan; ++p) {
    const int s0 = p * kPan, pe = min(n, s0 + kPan), h = pe - s0;
    if (blockIdx.x == 0) {
      for (int a = tid; a < h; a += kCS) yp[a] = y[s0 + a];
      __syncthreads();
      const double* D = Dinv + (size_t)p * kPan * kPan;
      for (int a = tid; a < h; a += kCS) {
        double s = 0.0;
        for (int k = 0; k <= a; ++k) s += D[a * kPan + k] * yp[k];
        yq[a] = s;
      }
      __syncthreads();
      for (int a = tid; a < h; a += kCS) y[s0 + a] = yq[a];
    }
    grid.sync();
    for (int a = pe + gw; a < n; a += nwarps) {
      double s = 0.0;
      for (int k = s0 + lane; k < pe; k += 32) s += Lc[(int64_t)a * n + k] * y[k];
      s = warp_sum_d(s);
      if (lane == 0) y[a] -= s;
    }
    grid.sync();
  }
  // backward: L^T x = y
  const int gt = blockIdx.x * kCS + tid, nthr = gridDim.x * kCS;
  for (int p = npan - 1; p >= 0; --p) {
    const int s0 = p * kPan, pe = min(n, s0 + kPan), h = pe - s0;
    if (blockIdx.x == 0) {
      for (int a = tid; a < h; a += kCS) yp[a] = y[s0 + a];
      __syncthreads();
      const double* D = Dinv + (size_t)p * kPan * kPan;
      for (int a = tid; a < h; a += kCS) {
        double s = 0.0;
        for (int k = a; k < h; ++k) s += D[k * kPan + a] * yp[k];
        yq[a] = s;
      }
      __syncthreads();
      for (int a = tid; a < h; a += kCS) y[s0 + a] = yq[a];
    }
    grid.sync();
    for (int c = gt; c < s0; c += nthr) {
      double s = 0.0;
      for (int a = s0; a < pe; ++a) s += Lc[(int64_t)a * n + c] * y[a];
      y[c] -= s;
    }
    grid.sync();
  }
}

// Independent systems, one CTA each: the same panel solves with
// __syncthreads in place of the grid barrier.  System y has its coarse size
// at desc[y], its factor at desc[nsys + y], its slice of the coarse vector at
// desc[2 nsys + y] and its diagonal inverses at desc[3 nsys + y].
__global__ void __launch_bounds__(kCS) coarse_solve_sys_kernel(const double* Lc, const double* Dinv,
                                                               const int64_t* desc, int nsys, double* y) {
  __shared__ double yp[kPan];
  const int sy = blockIdx.x;
  const int n = static_cast<int>(desc[sy]);
  Lc += desc[nsys + sy];
  y += desc[2 * nsys + sy];
  Dinv += desc[3 * nsys + sy];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int npan = (n + kPan - 1) / kPan;
  for (int p = 0; p < npan; ++p) {
    const int s0 = p * kPan, pe = min(n, s0 + kPan), h = pe - s0;
    for (int a = tid; a < h; a += kCS) yp[a] = y[s0 + a];
    __syncthreads();
    const double* D = Dinv + (size_t)p * kPan * kPan;
    for (int a = tid; a < h; a += kCS) {
      double s = 0.0;
      for (int k = 0; k <= a; ++k) s += D[a * kPan + k] * yp[k];
      y[s0 + a] = s;
    }
    __syncthreads();
    for (int a = pe + warp; a < n; a += kCS / 32) {
      double s = 0.0;
      for (int k = s0 + lane; k < pe; k += 32) s += Lc[(int64_t)a * n + k] * y[k];
      s = warp_sum_d(s);
      if (lane == 0) y[a] -= s;
    }
    __syncthreads();
  }
  for (int p = npan - 1; p >= 0; --p) {
    const int s0 = p * kPan, pe = min(n, s0 + kPan), h = pe - s0;
    for (int a = tid; a < h; a += kCS) yp[a] = y[s0 + a];
    __syncthreads();
    const double* D = Dinv + (size_t)p * kPan * kPan;
    for (int a = tid; a < h; a += kCS) {
      double s = 0.0;
      for (int k = a; k < h; ++k) s += D[k * kPan + a] * yp[k];
      y[s0 + a] = s;
    }
    __syncthreads();
    for (int c = tid; c < s0; c += kCS) {
      double s = 0.0;
      for (int a = s0; a < pe; ++a) s += Lc[(int64_t)a * n + c] * y[a];
      y[c] -= s;
    }
    __syncthreads();
  }
}

// Inverses of the diagonal kPan x kPan blocks of L_K (one CTA per block and
// system, one column of the inverse per thread).
__global__ void __launch_bounds__(kPan) coarse_dinv_kernel(const double* Lc, const int64_t* desc, int nsys,
                                                           double* Dinv) {
  __shared__ double Lb[kPan * (kPan + 1)];
  const int n = static_cast<int>(desc[blockIdx.y]);
  Lc += desc[nsys + blockIdx.y];
  Dinv += desc[3 * nsys + blockIdx.y];
  const int p = blockIdx.x, s0 = p * kPan;
  if (s0 >= n) return;
  const int h = min(n, s0 + kPan) - s0;
  for (int e = threadIdx.x; e < h * h; e += kPan) {
    int a = e / h, b = e - a * h;
    Lb[a * (kPan + 1) + b] = Lc[(int64_t)(s0 + a) * n + s0 + b];
  }
  __syncthreads();
  double* D = Dinv + (size_t)p * kPan * kPan;
  const int j = threadIdx.x;
  for (int a = 0; a < kPan; ++a) D[a * kPan + j] = 0.0;
  if (j < h) {
    for (int a = j; a < h; ++a) {
      double x = (a == j) ? 1.0 : 0.0;
      for (int k = j; k < a; ++k) x -= Lb[a * (kPan + 1) + k] * D[k * kPan + j];
      D[a * kPan + j] = x / Lb[a * (kPan + 1) + a];
    }
  }
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
cudaError_t apply_launch(const LevelDev& L, int first, int count, double* vec, cudaStream_t s, bool fwd) {
  if (count <= 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (fwd)
    apply_fwd_kernel<T><<<count, kApplyThreads, 0, s>>>(L, first, vec);
  else
    apply_bwd_kernel<T><<<count, kApplyThreads, 0, s>>>(L, first, vec);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply_fwd(int esize, const LevelDev& L, int first, int count, int nmax, double* vec,
                             cudaStream_t s) {
  return esize == 8 ? apply_launch<double>(L, first, count, vec, s, true)
                    : apply_launch<float>(L, first, count, vec, s, true);
}

cudaError_t launch_apply_bwd(int esize, const LevelDev& L, int first, int count, int nmax, double* vec,
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

cudaError_t launch_coarse_dinv(const double* Lc, const int64_t* desc, int nsys, int nmax, double* Dinv,
                               cudaStream_t s) {
  if (nmax <= 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  coarse_dinv_kernel<<<dim3((nmax + kPan - 1) / kPan, nsys), kPan, 0, s>>>(Lc, desc, nsys, Dinv);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve_sys(const double* Lc, const double* Dinv, const int64_t* desc, int nsys,
                                    double* y, cudaStream_t s) {
  if (nsys <= 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  coarse_solve_sys_kernel<<<nsys, kCS, 0, s>>>(Lc, Dinv, desc, nsys, y);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const double* Lc, const double* Dinv, int n, double* y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_solve_kernel, kCS, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    grid = sms;
  }
  void* args[] = {(void*)&Lc, (void*)&Dinv, (void*)&n, (void*)&y};
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaLaunchCooperativeKernel((const void*)coarse_solve_kernel, dim3(grid), dim3(kCS), args, 0, s);
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
