// CUDA kernels of the CE solve x = Q^T L^{-T} L^{-1} Q b (solve proposition,
// Section 2.5) and of the FP64 conjugate-gradient loop around it.
//
// The level vector of level l holds block i at [vec_off[i], vec_off[i]+n_i).
// Forward step of block i (in the factorization's colour order, one persistent
// launch per level): y_i <- U_i^T y_i; z = L_hat^{-1} y_i[r:];
// y_i[:r] -= W_b^T z; y_p[:w_p] -= W_p^T z for every close p; z is stored in
// y_i[r:].  The basis parts then move to the next level's vector
// (super-blocks of consecutive children).  The backward step is the
// transpose, in reverse order.
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <algorithm>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace ce {

namespace {

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

// Filled by the 32 lanes of one warp, lane t for target t (the loads of all
// targets in flight at once; prefix sums by warp scans).
__device__ void targets_of(const LevelDev& L, int i, int n, int r, Targets& T, int lane) {
  const int ci = L.colour[i];
  const int c0 = L.close_ptr[i], c1 = L.close_ptr[i + 1];
  const int nt = min(1 + (c1 - c0), kMaxTgt);
  int w = 0, np = 0;
  int64_t vo = 0;
  if (lane == 0) {
    w = r;
    np = n;
    vo = L.vec_off[i];
  } else if (lane < nt) {
    const int p = L.close_blk[c0 + lane - 1];
    w = width_of_a(L, p, ci);
    np = L.n[p];
    vo = L.vec_off[p];
  }
  int sw = w, sn = np;  // inclusive scans of the widths and of the block sizes
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int a = __shfl_up_sync(0xffffffffu, sw, o), b = __shfl_up_sync(0xffffffffu, sn, o);
    if (lane >= o) {
      sw += a;
      sn += b;
    }
  }
  if (lane < nt) {
    T.w[lane] = w;
    T.woff[lane] = (int64_t)n * (sn - np);  // W columns of target t start after n + sizes before it
    T.voff[lane] = vo;
    T.pre[lane] = sw - w;
  }
  if (lane == nt - 1) T.pre[nt] = sw;
  if (lane == 0) T.nt = nt;
}

// Every factor element is read exactly once per apply, so U_i, L_hat_i^{-1}
// and W_i are streamed from global memory (no staging) and the arithmetic is
// done in the factor's own precision T: the FP32 form applies its
// preconditioner in FP32 (the level vectors stay FP64 in memory, so PCG sees
// an FP64 operator whose error is the FP32 rounding of M^{-1}, far below the
// compression tolerance); the FP64 form stays FP64 throughout.

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A strided vector of the factor: element k is p[k * s].
template <typename T>
struct Strided {
  const T* p;
  int64_t s;
};

// sum_{k in [k0, k1)} M.p[k M.s] x[k] with 8 independent partial sums, so a
// thread keeps 8 loads of the factor in flight
template <typename T>
__device__ __forceinline__ T dot8(Strided<T> M, const T* x, int k0, int k1) {
  T s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int k = k0;
  for (; k + 7 < k1; k += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) s[u] += M.p[(k + u) * M.s] * x[k + u];
  }
  for (; k < k1; ++k) s[0] += M.p[k * M.s] * x[k];
  return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// CTA GEMV: out(a, sum_{k in [lo(a), hi(a))} row(a)[k] x[k]) for a < A.
// With A <= NT / 2 the k range of each output is split over G = NT / A
// threads (partial sums in part[G * A], added in slice order); otherwise one
// thread per output.  Ends with a barrier.
template <typename T, int NT, class Row, class Lo, class Hi, class Out>
__device__ __forceinline__ void cta_gemv(int A, Row row, const T* x, Lo lo, Hi hi, Out out, T* part) {
  const int tid = threadIdx.x;
  if (A > NT / 2) {
    for (int a = tid; a < A; a += NT) out(a, dot8<T>(row(a), x, lo(a), hi(a)));
  } else if (A > 0) {
    const int G = NT / A, a = tid % A, g = tid / A;
    if (g < G) {
      const int l0 = lo(a), len = hi(a) - l0;
      part[g * A + a] = dot8<T>(row(a), x, l0 + len * g / G, l0 + len * (g + 1) / G);
    }
    __syncthreads();
    for (int b = tid; b < A; b += NT) {
      T acc = 0;
      for (int h = 0; h < G; ++h) acc += part[h * A + b];
      out(b, acc);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ int target_of(const Targets& tg, int f) {
  int t = 0;
  while (f >= tg.pre[t + 1]) ++t;
  return t;
}

// Forward step of block i: y_i <- U_i^T y_i; z = L_hat^{-1} y_i[r:];
// y_t[:w_t] -= W_t^T z for every target t (basis of i first); y_i[r:] = z.
template <typename T, int NT>
__device__ __forceinline__ void fwd_block(const LevelDev& L, const int i, double* vec) {
  __shared__ T ys[kNMax], yt[kNMax], z[kNMax];
  __shared__ T part[NT];
  __shared__ Targets tg;
  const int tid = threadIdx.x;
  const int n = L.n[i];
  if (n == 0) return;
  const int r = L.rank[i], m = n - r;
  double* v = vec + L.vec_off[i];
  const T* U = reinterpret_cast<const T*>(L.U) + L.u_off[i];
  const T* Li = reinterpret_cast<const T*>(L.L) + L.l_off[i];
  const T* W = reinterpret_cast<const T*>(L.W) + L.w_off[i];
  for (int a = tid; a < n; a += NT) ys[a] = static_cast<T>(v[a]);
  if (tid < 32) targets_of(L, i, n, r, tg, tid);
  __syncthreads();
  auto zero = [](int) { return 0; };
  // yt = U^T ys: column a of U
  cta_gemv<T, NT>(
      n, [&](int a) { return Strided<T>{U + a, n}; }, ys, zero, [&](int) { return n; },
      [&](int a, T s) { yt[a] = s; }, part);
  // z = L_hat^{-1} yt[r:]: row a of the lower factor, k <= a
  cta_gemv<T, NT>(
      m, [&](int a) { return Strided<T>{Li + a * m, 1}; }, yt + r, zero, [](int a) { return a + 1; },
      [&](int a, T s) {
        z[a] = s;
        v[r + a] = static_cast<double>(s);
      },
      part);
  // every target column c of W_t: y_t[c] -= (W_t^T z)[c]; the basis of i gets yt - W_b^T z
  cta_gemv<T, NT>(
      tg.pre[tg.nt],
      [&](int f) {
        const int t = target_of(tg, f);
        return Strided<T>{W + tg.woff[t] + (f - tg.pre[t]), tg.w[t]};
      },
      z, zero, [&](int) { return m; },
      [&](int f, T s) {
        const int t = target_of(tg, f), c = f - tg.pre[t];
        if (t == 0)
          v[c] = static_cast<double>(yt[c] - s);
        else if (L.accumulate)   // rows of a distance-1 colour may share target t
          atomicAdd(&vec[tg.voff[t] + c], -static_cast<double>(s));
        else
          vec[tg.voff[t] + c] -= static_cast<double>(s);
      },
      part);
}

// Backward step of block i (transpose, reverse order): rhs = z - W x_t over
// all targets; x_n = L_hat^{-T} rhs; y_i <- U_i [x_b; x_n].
template <typename T, int NT>
__device__ __forceinline__ void bwd_block(const LevelDev& L, const int i, double* vec) {
  __shared__ T xf[kNMax], rhs[kNMax];
  __shared__ T xt[kMaxTgt * kNMax];
  __shared__ T pt[kNMax * kMaxTgt];  // (W_t x_t)[a] per row a and target t
  __shared__ T part[NT];
  __shared__ Targets tg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = L.n[i];
  if (n == 0) return;
  const int r = L.rank[i], m = n - r;
  double* v = vec + L.vec_off[i];
  const T* U = reinterpret_cast<const T*>(L.U) + L.u_off[i];
  const T* Li = reinterpret_cast<const T*>(L.L) + L.l_off[i];
  const T* W = reinterpret_cast<const T*>(L.W) + L.w_off[i];
  for (int a = tid; a < n; a += NT) xf[a] = static_cast<T>(v[a]);   // [x_b; z]
  if (warp == 0) targets_of(L, i, n, r, tg, lane);
  __syncthreads();
  const int nt = tg.nt, tot = tg.pre[nt];
  for (int f = tid; f < tot; f += NT) {
    const int t = target_of(tg, f), c = f - tg.pre[t];
    xt[f] = (t == 0) ? xf[c] : static_cast<T>(vec[tg.voff[t] + c]);
  }
  __syncthreads();
  auto zero = [](int) { return 0; };
  // (W_t x_t)[a] for every (row a, target t): row a of W_t against xt[pre[t]:pre[t+1]]
  cta_gemv<T, NT>(
      m * nt,
      [&](int e) {
        const int a = e / nt, t = e - a * nt;
        return Strided<T>{W + tg.woff[t] + (int64_t)a * tg.w[t] - tg.pre[t], 1};
      },
      xt, [&](int e) { return tg.pre[e % nt]; }, [&](int e) { return tg.pre[e % nt + 1]; },
      [&](int e, T s) { pt[e] = s; }, part);
  for (int a = tid; a < m; a += NT) {
    T acc = 0;
    for (int t = 0; t < nt; ++t) acc += pt[a * nt + t];
    rhs[a] = xf[r + a] - acc;
  }
  __syncthreads();
  // x_n = L_hat^{-T} rhs: column a of the lower factor, k >= a
  cta_gemv<T, NT>(
      m, [&](int a) { return Strided<T>{Li + a, m}; }, rhs, [](int a) { return a; }, [&](int) { return m; },
      [&](int a, T s) { xf[r + a] = s; }, part);
  // y_i = U_i xf: row a of U
  cta_gemv<T, NT>(
      n, [&](int a) { return Strided<T>{U + (int64_t)a * n, 1}; }, xf, zero, [&](int) { return n; },
      [&](int a, T s) { v[a] = static_cast<double>(s); }, part);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kWaitPolls = 1 << 24;  // a dependency wait gives up after wait_ns or this many polls

// Warp-wide wait until flag[idx[d]] == want for every d in [d0, d1): each
// lane polls its own flags, the warp votes.  Ends early (false) on a
// recorded error or after wait_ns / kWaitPolls, recording reason 6.
__device__ bool wait_flags(const int* flag, const int* idx, int d0, int d1, int want, int* status, int row,
                           int lane, unsigned long long wait_ns) {
  const unsigned long long t0 = globaltimer_ns();
  int polls = 0;
  for (int base = d0; base < d1; base += 32) {
    const int d = base + lane;
    const int* f = d < d1 ? flag + idx[d] : nullptr;
    for (;;) {
      const bool ok = f == nullptr || ld_acquire(f) == want;
      if (__all_sync(0xffffffffu, ok)) break;
      int bad = 0;
      if (lane == 0) {
        if (ld_acquire(status) != 0)
          bad = 1;
        else if (++polls > kWaitPolls || globaltimer_ns() - t0 > wait_ns)
          bad = 2;
        if (bad == 2 && atomicCAS(status, 0, CE_ERR_CUDA) == 0) {
          status[2] = row;
          status[3] = 6;
        }
      }
      if (__shfl_sync(0xffffffffu, bad, 0)) return false;
      __nanosleep(64);
    }
  }
  return true;
}

// One persistent launch per level and direction.  Rows are taken from a
// counter in the level's elimination order (forward) or its reverse
// (backward); a row waits until every row of an earlier step within distance
// 2 (lower colour forward, higher colour backward) carries this apply's epoch
// in its flag, so every vector entry sees its updates in the colour order of
// the per-colour schedule.  Rows only wait for rows taken earlier, held by
// running CTAs; waits are bounded anyway and end on a recorded error.  The
// epoch and counters live in device memory (advanced by apply_prep_kernel),
// so the launches can be replayed from a CUDA graph.
template <typename T, int NT, bool kFwd>
__global__ void __launch_bounds__(NT) apply_level_kernel(LevelDev L, double* vec, int* status) {
  __shared__ int s_q;
  const int tid = threadIdx.x;
  const int count = L.M;
  const int ep = *L.epoch;
  int* qctr = L.aq + (kFwd ? 0 : 1);
  int* flag = kFwd ? L.fdone : L.bdone;
  const int* dp = kFwd ? L.dep_ptr : L.rdep_ptr;
  const int* di = kFwd ? L.dep_idx : L.rdep_idx;
  const int lane = tid & 31;
  for (;;) {
    if (tid < 32) {
      int q = 0;
      if (lane == 0) {
        q = atomicAdd(qctr, 1);
        if (q >= count || ld_acquire(status) != 0) q = -1;
      }
      q = __shfl_sync(0xffffffffu, q, 0);
      if (q >= 0) {
        const int i = L.order[kFwd ? q : count - 1 - q];
        if (!wait_flags(flag, di, dp[i], dp[i + 1], ep, status, i, lane, L.wait_ns)) q = -1;
      }
      if (lane == 0) s_q = q;
    }
    __syncthreads();
    const int q = s_q;
    if (q < 0) return;
    __threadfence();
    const int i = L.order[kFwd ? q : count - 1 - q];
    if (kFwd)
      fwd_block<T, NT>(L, i, vec);
    else
      bwd_block<T, NT>(L, i, vec);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(flag + i, ep);
    }
  }
}

// start of an apply: next epoch, queue counters of every level back to 0
__global__ void apply_prep_kernel(int* q, int nq, int* epoch) {
  for (int t = threadIdx.x; t < nq; t += blockDim.x) q[t] = 0;
  if (threadIdx.x == 0) *epoch += 1;
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
// CTAs cooperating through grid-wide barriers, one barrier per panel of kPan
// rows.  Dinv holds the inverses of the diagonal kPan x kPan blocks; every
// CTA solves the current panel itself (a small GEMV from shared memory) and
// then updates its share of the rows still to come with that solution.  CTA
// 0 stores a panel's solution one step later, when no CTA reads the panel's
// right-hand side any more.
constexpr int kPan = 64;
constexpr int kCS = 256;

__global__ void __launch_bounds__(kCS) coarse_solve_kernel(const double* Lc, const double* Dinv, int n,
                                                           double* y) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double yp[kPan], yq[kPan];
  __shared__ double Ds[kPan * (kPan + 1)];  // one diagonal inverse, loaded coalesced
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gw = blockIdx.x * (kCS / 32) + warp, nwarps = gridDim.x * (kCS / 32);
  const int gt = blockIdx.x * kCS + tid, nthr = gridDim.x * kCS;
  const int npan = (n + kPan - 1) / kPan;
  const bool lead = blockIdx.x == 0;
  int prev0 = -1, prevh = 0;  // panel whose solution CTA 0 still has to store
  // forward: L y = b
  for (int p = 0; p < npan; ++p) {
    const int s0 = p * kPan, pe = min(n, s0 + kPan), h = pe - s0;
    if (lead && prev0 >= 0)
      for (int a = tid; a < prevh; a += kCS) y[prev0 + a] = yq[a];
    __syncthreads();
    for (int a = tid; a < h; a += kCS) yp[a] = y[s0 + a];
    const double* D = Dinv + (size_t)p * kPan * kPan;
    for (int e = tid; e < kPan * kPan; e += kCS) Ds[(e / kPan) * (kPan + 1) + e % kPan] = D[e];
    __syncthreads();
    for (int a = tid; a < h; a += kCS) {
      double s = 0.0;
      for (int k = 0; k <= a; ++k) s += Ds[a * (kPan + 1) + k] * yp[k];
      yq[a] = s;
    }
    __syncthreads();
    for (int a = pe + gw; a < n; a += nwarps) {
      double s = 0.0;
      for (int k = lane; k < h; k += 32) s += Lc[(int64_t)a * n + s0 + k] * yq[k];
      s = warp_sum_d(s);
      if (lane == 0) y[a] -= s;
    }
    prev0 = s0;
    prevh = h;
    grid.sync();
  }
  // backward: L^T x = y (the last panel's right-hand side is the yq just solved)
  prev0 = -1;
  for (int p = npan - 1; p >= 0; --p) {
    const int s0 = p * kPan, pe = min(n, s0 + kPan), h = pe - s0;
    if (p == npan - 1) {
      for (int a = tid; a < h; a += kCS) yp[a] = yq[a];
    } else {
      if (lead && prev0 >= 0)
        for (int a = tid; a < prevh; a += kCS) y[prev0 + a] = yq[a];
      __syncthreads();
      for (int a = tid; a < h; a += kCS) yp[a] = y[s0 + a];
    }
    const double* D = Dinv + (size_t)p * kPan * kPan;
    for (int e = tid; e < kPan * kPan; e += kCS) Ds[(e / kPan) * (kPan + 1) + e % kPan] = D[e];
    __syncthreads();
    for (int a = tid; a < h; a += kCS) {
      double s = 0.0;
      for (int k = a; k < h; ++k) s += Ds[k * (kPan + 1) + a] * yp[k];
      yq[a] = s;
    }
    __syncthreads();
    for (int c = gt; c < s0; c += nthr) {
      double s = 0.0;
      for (int a = 0; a < h; ++a) s += Lc[(int64_t)(s0 + a) * n + c] * yq[a];
      y[c] -= s;
    }
    prev0 = s0;
    prevh = h;
    grid.sync();
  }
  if (lead)
    for (int a = tid; a < prevh; a += kCS) y[prev0 + a] = yq[a];
}

// Independent systems, one CTA each: the same panel solves with
// __syncthreads in place of the grid barrier.  System y has its coarse size
// at desc[y], its factor at desc[nsys + y], its slice of the coarse vector at
// desc[2 nsys + y] and its diagonal inverses at desc[3 nsys + y].
__global__ void __launch_bounds__(kCS) coarse_solve_sys_kernel(const double* Lc, const double* Dinv,
                                                               const int64_t* desc, int nsys, double* y) {
  __shared__ double yp[kPan];
  __shared__ double Ds[kPan * (kPan + 1)];
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
    const double* D = Dinv + (size_t)p * kPan * kPan;
    for (int e = tid; e < kPan * kPan; e += kCS) Ds[(e / kPan) * (kPan + 1) + e % kPan] = D[e];
    __syncthreads();
    for (int a = tid; a < h; a += kCS) {
      double s = 0.0;
      for (int k = 0; k <= a; ++k) s += Ds[a * (kPan + 1) + k] * yp[k];
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
    const double* D = Dinv + (size_t)p * kPan * kPan;
    for (int e = tid; e < kPan * kPan; e += kCS) Ds[(e / kPan) * (kPan + 1) + e % kPan] = D[e];
    __syncthreads();
    for (int a = tid; a < h; a += kCS) {
      double s = 0.0;
      for (int k = a; k < h; ++k) s += Ds[k * (kPan + 1) + a] * yp[k];
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
// system, one column of the inverse per thread, built in shared memory by
// forward substitution and written out row by row).
__global__ void __launch_bounds__(kPan) coarse_dinv_kernel(const double* Lc, const int64_t* desc, int nsys,
                                                           double* Dinv) {
  extern __shared__ double dinv_smem[];     // 2 kPan (kPan + 1) doubles
  double* Lb = dinv_smem;
  double* X = dinv_smem + kPan * (kPan + 1);
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
  const int j = threadIdx.x;
  for (int a = 0; a < kPan; ++a) X[a * (kPan + 1) + j] = 0.0;
  if (j < h) {
    for (int a = j; a < h; ++a) {
      double x0 = (a == j) ? 1.0 : 0.0, x1 = 0.0;
      int k = j;
      for (; k + 1 < a; k += 2) {
        x0 -= Lb[a * (kPan + 1) + k] * X[k * (kPan + 1) + j];
        x1 -= Lb[a * (kPan + 1) + k + 1] * X[(k + 1) * (kPan + 1) + j];
      }
      if (k < a) x0 -= Lb[a * (kPan + 1) + k] * X[k * (kPan + 1) + j];
      X[a * (kPan + 1) + j] = (x0 + x1) / Lb[a * (kPan + 1) + a];
    }
  }
  __syncthreads();
  double* D = Dinv + (size_t)p * kPan * kPan;
  for (int a = 0; a < kPan; ++a) D[a * kPan + j] = X[a * (kPan + 1) + j];
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

// p = z on the first pass (p is not read: its memory may hold anything,
// NaN patterns included), p = z + beta p afterwards
__global__ void update_p_kernel(int64_t n, double* p, const double* z, const double* scal, int first) {
  const double beta = first ? 0.0 : scal[5];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    p[k] = first ? z[k] : z[k] + beta * p[k];
}

__global__ void pcg_scalars_kernel(double* scal, int stage) {
  if (stage == 0) {
    scal[2] = scal[0] / scal[1];  // alpha = rz / pAp
  } else {
    scal[5] = scal[4] / scal[0];  // beta = rz_new / rz
    scal[0] = scal[4];
  }
}

template <typename T, int NT, bool kFwd>
cudaError_t apply_launch_nt(const LevelDev& L, double* vec, int* status, cudaStream_t s) {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_level_kernel<T, NT, kFwd>, NT, 0);
    if (e != cudaSuccess) return e;
    cap = std::max(per_sm, 1) * sms;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  apply_level_kernel<T, NT, kFwd><<<std::min(L.M, cap), NT, 0, s>>>(L, vec, status);
  return cudaGetLastError();
}

// CTA width by level size: many small rows want many CTAs in flight, a
// coarse level (few rows on its critical path) wants wide CTAs
template <typename T, bool kFwd>
cudaError_t apply_launch(const LevelDev& L, double* vec, int* status, cudaStream_t s) {
  if (L.M <= 0) return cudaSuccess;
  if (L.M >= 4096) return apply_launch_nt<T, 128, kFwd>(L, vec, status, s);
  if (L.M >= 1024) return apply_launch_nt<T, 256, kFwd>(L, vec, status, s);
  return apply_launch_nt<T, 512, kFwd>(L, vec, status, s);
}

}  // namespace

cudaError_t launch_apply_prep(int* q, int nq, int* epoch, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  apply_prep_kernel<<<1, 64, 0, s>>>(q, nq, epoch);
  return cudaGetLastError();
}

cudaError_t launch_apply_fwd(int esize, const LevelDev& L, double* vec, int* status, cudaStream_t s) {
  return esize == 8 ? apply_launch<double, true>(L, vec, status, s) : apply_launch<float, true>(L, vec, status, s);
}

cudaError_t launch_apply_bwd(int esize, const LevelDev& L, double* vec, int* status, cudaStream_t s) {
  return esize == 8 ? apply_launch<double, false>(L, vec, status, s)
                    : apply_launch<float, false>(L, vec, status, s);
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
  const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, (int64_t)device_sms() * 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  perm_kernel<<<grid, 256, 0, s>>>(perm, n, in, out, gather);
  return cudaGetLastError();
}

cudaError_t launch_coarse_dinv(const double* Lc, const int64_t* desc, int nsys, int nmax, double* Dinv,
                               cudaStream_t s) {
  if (nmax <= 0) return cudaSuccess;
  constexpr int smem = 2 * kPan * (kPan + 1) * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(coarse_dinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  coarse_dinv_kernel<<<dim3((nmax + kPan - 1) / kPan, nsys), kPan, smem, s>>>(Lc, desc, nsys, Dinv);
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
  const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, (int64_t)device_sms() * 8));
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
