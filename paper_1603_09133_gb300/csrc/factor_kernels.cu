// CUDA kernels of the CE factorization (sm_103a).
//
// ce_row_kernel: one CTA per block row i of one colour (Algorithm 2, one
// iteration of its loop, for many independent rows at once):
//   A. compression (Section 2.2, eq. rreav): R factor of F_i^T by Householder
//      reflections, streamed in chunks of rows of F_i^T through shared memory
//      (F_i F_i^T = R^T R, so F_i and R^T share left singular vectors);
//   B. one-sided (Hestenes) Jacobi on the columns of R, warp per column pair,
//      round-robin pair schedule: R V = U' S  =>  U_i = V, sigma = S, sorted
//      descending; r_i = #{sigma_k > tau_i}, tau_i never below the rounding
//      floor u ||D_i||_F of the block row;
//   C. transform and elimination (eq. q, eq. sm_L): D <- U^T D U, close rows
//      <- U^T C, far rows <- U_b^T F (the E_i rows are dropped), Cholesky of
//      the non-basis block S_ii = L_hat L_hat^T, W = L_hat^{-1} S_i and the
//      Schur update A(p, q) -= W_p^T W_q over the targets {basis of i} U
//      close(i).
// Blocks of one colour have disjoint closed neighbourhoods (distance-2
// colouring), so the CTAs of one launch touch disjoint block pairs.
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

// Householder QR update of the stacked matrix [R; C] (R: n x n upper
// triangular, C: c x n): after the call R is the triangular factor of the
// stack and C is annihilated (its contents are left undefined).
// Reflector of column j in the unit-leading form H = I - tau v v^T,
// v = [1; s C(:, j)], beta = -sign(x0) ||x||, tau = (beta - x0) / beta,
// s = 1 / (x0 - beta): tau lies in [1, 2] and ||x|| is formed from the
// column scaled by its largest entry, so fill at the level of rounding noise
// (whose squares underflow) gives no inf or NaN.
template <typename T>
__device__ void householder_stack(T* R, T* C, int n, int c, T* s_scale, T* s_tau) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      T amax = 0;
      for (int q = lane; q < c; q += 32) amax = fmax(amax, fabs(C[q * LD + j]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      // a column whose largest entry is subnormal is rounding noise far
      // below any truncation threshold: it is treated as zero
      if (!(amax >= Tiny<T>::v)) amax = T(0);
      T s = 0;
      if (amax > T(0)) {
        for (int q = lane; q < c; q += 32) {
          T x = C[q * LD + j] / amax;
          s += x * x;
        }
      }
      s = warp_sum(s);
      if (lane == 0) {
        if (amax == T(0)) {
          *s_tau = T(0);
          *s_scale = T(0);
        } else {
          const T x0 = R[j * LD + j];
          const T a = fmax(amax, fabs(x0));
          const T x0a = x0 / a, ca = amax / a;
          const T nrm = a * sqrt(x0a * x0a + s * ca * ca);
          const T beta = (x0 >= T(0)) ? -nrm : nrm;
          *s_tau = (beta - x0) / beta;
          *s_scale = T(1) / (x0 - beta);
          R[j * LD + j] = beta;
        }
      }
    }
    __syncthreads();
    const T tau = *s_tau, sc = *s_scale;
    if (tau != T(0)) {
      for (int l = j + 1 + warp; l < n; l += kWarps) {
        T d = 0;
        for (int q = lane; q < c; q += 32) d += C[q * LD + j] * C[q * LD + l];
        d = warp_sum(d);
        d = (R[j * LD + l] + sc * d) * tau;
        if (lane == 0) R[j * LD + l] -= d;
        const T ds = d * sc;
        for (int q = lane; q < c; q += 32) C[q * LD + l] -= ds * C[q * LD + j];
      }
    }
    __syncthreads();
  }
}

// load an n x w tile of the block pair (i, k) seen from row i into sm
// (row-major, LD); the pair is stored once as (min, max)
template <typename T>
__device__ void load_row_tile(T* sm, const T* X, int i, int k, int n, int nk, int w) {
  if (i < k) {  // stored n x nk
    for (int e = threadIdx.x; e < n * w; e += kThreads) {
      int a = e / w, b = e - a * w;
      sm[a * LD + b] = X[(int64_t)a * nk + b];
    }
  } else {      // stored nk x n, tile = X[0:w, :]^T
    for (int e = threadIdx.x; e < n * w; e += kThreads) {
      int b = e / n, a = e - b * n;
      sm[a * LD + b] = X[(int64_t)b * n + a];
    }
  }
}

// store rows 0..rows-1 of an n x w row tile back into the pair (i, k)
template <typename T>
__device__ void store_row_tile(const T* sm, T* X, int i, int k, int n, int nk, int rows, int w) {
  if (i < k) {
    for (int e = threadIdx.x; e < rows * w; e += kThreads) {
      int a = e / w, b = e - a * w;
      X[(int64_t)a * nk + b] = sm[a * LD + b];
    }
  } else {
    for (int e = threadIdx.x; e < rows * w; e += kThreads) {
      int b = e / rows, a = e - b * rows;
      X[(int64_t)b * n + a] = sm[a * LD + b];
    }
  }
}

// in-place forward substitution: rows r0..r0+m-1 of columns 0..w-1 of Y
// become L^{-1} Y, L = lower triangle of Lm[r0.., r0..] (both in LD layout)
template <typename T>
__device__ void trsm_lower(const T* Lm, int r0, int m, T* Y, int w) {
  for (int b = threadIdx.x; b < w; b += kThreads) {
    for (int a = 0; a < m; ++a) {
      T x = Y[(r0 + a) * LD + b];
      for (int k = 0; k < a; ++k) x -= Lm[(r0 + a) * LD + r0 + k] * Y[(r0 + k) * LD + b];
      Y[(r0 + a) * LD + b] = x / Lm[(r0 + a) * LD + r0 + a];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    ce_row_kernel(LevelDev L, int first, int level, double tol, int tol_mode, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + kNMax * LD;
  T* bufC = bufB + kNMax * LD;
  T* bufD = bufC + kNMax * LD;
  T* sig = bufD + kNMax * LD;       // kNMax
  T* sig_tmp = sig + kNMax;         // kNMax
  __shared__ T s_scale, s_tau;
  __shared__ int s_flag;
  __shared__ int s_pos[kNMax];
  __shared__ int s_colst[kMaxTargets];
  __shared__ int s_tgt[kMaxTargets];
  __shared__ int s_w[kMaxTargets];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = L.order[first + blockIdx.x];
  const int n = L.n[i];
  const int ci = L.colour[i];
  T* pool = reinterpret_cast<T*>(L.pool);
  if (n == 0) {
    if (tid == 0) {
      L.rank[i] = 0;
      L.tau[i] = 0.0;
    }
    return;
  }

  // Frobenius norm of D_i: the rounding floor u ||D_i||_F of the threshold
  __shared__ double s_red[kWarps];
  {
    const T* Dg0 = pool + L.diag_off[i];
    double ss = 0.0;
    for (int e = tid; e < n * n; e += kThreads) {
      double v = static_cast<double>(Dg0[e]);
      ss += v * v;
    }
    ss = warp_sum(ss);
    if (lane == 0) s_red[warp] = ss;
  }

  // ---------------- A. R factor of F_i^T --------------------------------
  T* R = bufA;
  T* C = bufB;
  for (int e = tid; e < n * LD; e += kThreads) R[e] = T(0);
  __syncthreads();
  int crow = 0, total_rows = 0;
  for (int f = L.far_ptr[i]; f < L.far_ptr[i + 1]; ++f) {
    const int k = L.far_blk[f];
    const int w = width_of(L, k, ci);
    const int nk = L.n[k];
    const T* X = pool + L.far_off[f];
    int q0 = 0;
    while (q0 < w) {
      const int take = min(w - q0, kChunk - crow);
      if (i < k) {  // F = X[:, q0:q0+take]: F^T row q = column q of X
        for (int e = tid; e < take * n; e += kThreads) {
          int a = e / take, q = e - a * take;
          C[(crow + q) * LD + a] = X[(int64_t)a * nk + q0 + q];
        }
      } else {      // F^T rows are rows of X
        for (int e = tid; e < take * n; e += kThreads) {
          int q = e / n, a = e - q * n;
          C[(crow + q) * LD + a] = X[(int64_t)(q0 + q) * n + a];
        }
      }
      crow += take;
      q0 += take;
      total_rows += take;
      if (crow == kChunk) {
        __syncthreads();
        householder_stack(R, C, n, crow, &s_scale, &s_tau);
        crow = 0;
      }
    }
  }
  if (crow > 0) {
    __syncthreads();
    householder_stack(R, C, n, crow, &s_scale, &s_tau);
  }

  // ---------------- B. one-sided Jacobi on R ----------------------------
  T* X = bufA;   // R, rotated in place
  T* V = bufC;
  T* U = bufD;
  int r = 0;
  double tau = 0.0;
  if (total_rows > 0) {
    for (int e = tid; e < n * LD; e += kThreads) {
      int a = e / LD, b = e - a * LD;
      V[e] = (a == b) ? T(1) : T(0);
    }
    __syncthreads();
    const int nb = n + (n & 1);
    const T tolJ = T(n) * Eps<T>::v;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
      if (tid == 0) s_flag = 0;
      __syncthreads();
      for (int rnd = 0; rnd < nb - 1; ++rnd) {
        for (int t = warp; t < nb / 2; t += kWarps) {
          int p, q;
          if (t == 0) {
            p = nb - 1;
            q = rnd;
          } else {
            p = (rnd + t) % (nb - 1);
            q = (rnd - t + nb - 1) % (nb - 1);
          }
          if (p >= n || q >= n) continue;
          T a = 0, b = 0, g = 0;
          for (int row = lane; row < n; row += 32) {
            T xp = X[row * LD + p], xq = X[row * LD + q];
            a += xp * xp;
            b += xq * xq;
            g += xp * xq;
          }
          a = warp_sum(a);
          b = warp_sum(b);
          g = warp_sum(g);
          if (g != T(0) && fabs(g) > tolJ * sqrt(a) * sqrt(b)) {
            T zeta = (b - a) / (T(2) * g);
            T az = fabs(zeta);
            T den = (az > T(1)) ? az * (T(1) + sqrt(T(1) + T(1) / (az * az)))
                                : az + sqrt(T(1) + az * az);
            T tt = ((zeta >= T(0)) ? T(1) : T(-1)) / den;
            T cs = T(1) / sqrt(T(1) + tt * tt), sn = cs * tt;
            for (int row = lane; row < n; row += 32) {
              T xp = X[row * LD + p], xq = X[row * LD + q];
              X[row * LD + p] = cs * xp - sn * xq;
              X[row * LD + q] = sn * xp + cs * xq;
              T vp = V[row * LD + p], vq = V[row * LD + q];
              V[row * LD + p] = cs * vp - sn * vq;
              V[row * LD + q] = sn * vp + cs * vq;
            }
            if (lane == 0) s_flag = 1;
          }
        }
        __syncthreads();
      }
      const int rotated = s_flag;
      __syncthreads();
      if (!rotated) break;
    }
    // singular values = column norms, sorted descending (stable)
    for (int j = tid; j < n; j += kThreads) {
      T s = 0;
      for (int row = 0; row < n; ++row) s += X[row * LD + j] * X[row * LD + j];
      sig_tmp[j] = sqrt(s);
    }
    __syncthreads();
    for (int j = tid; j < n; j += kThreads) {
      T sj = sig_tmp[j];
      int pos = 0;
      for (int k = 0; k < n; ++k) pos += (sig_tmp[k] > sj) || (sig_tmp[k] == sj && k < j);
      s_pos[j] = pos;
      sig[pos] = sj;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += kThreads) {
      int a = e / n, j = e - a * n;
      U[a * LD + s_pos[j]] = V[a * LD + j];
    }
    const double smax = static_cast<double>(sig[0]);
    if (!isfinite(smax)) {
      if (tid == 0) set_status(status, CE_ERR_NOT_SPD, level, i, 2);
      return;
    }
    if (tol == 0.0)
      tau = n * static_cast<double>(Eps<T>::v) * smax;
    else
      tau = (tol_mode == CE_TOL_ABS) ? tol : tol * smax;
    double dn2 = 0.0;
    for (int w = 0; w < kWarps; ++w) dn2 += s_red[w];
    tau = fmax(tau, static_cast<double>(Eps<T>::v) * sqrt(dn2));
    for (int k = 0; k < n; ++k) r += (static_cast<double>(sig[k]) > tau) ? 1 : 0;
  } else {
    for (int e = tid; e < n * LD; e += kThreads) {
      int a = e / LD, b = e - a * LD;
      U[e] = (a == b) ? T(1) : T(0);
    }
    for (int k = tid; k < n; k += kThreads) sig[k] = T(0);
  }
  __syncthreads();
  const int m = n - r;
  if (tid == 0) {
    L.rank[i] = r;
    L.tau[i] = tau;
  }
  for (int k = tid; k < n; k += kThreads) L.sigma[L.vec_off[i] + k] = static_cast<double>(sig[k]);
  T* Ug = reinterpret_cast<T*>(L.U) + L.u_off[i];
  for (int e = tid; e < n * n; e += kThreads) {
    int a = e / n, b = e - a * n;
    Ug[e] = U[a * LD + b];
  }

  // ---------------- C. transform + elimination --------------------------
  T* Dg = pool + L.diag_off[i];
  for (int e = tid; e < n * n; e += kThreads) {
    int a = e / n, b = e - a * n;
    bufB[a * LD + b] = Dg[e];
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += kThreads) {   // bufC = D U
    int a = e / n, b = e - a * n;
    T s = 0;
    for (int k = 0; k < n; ++k) s += bufB[a * LD + k] * U[k * LD + b];
    bufC[a * LD + b] = s;
  }
  __syncthreads();
  T* Tm = bufA;                                     // Tm = U^T D U
  for (int e = tid; e < n * n; e += kThreads) {
    int a = e / n, b = e - a * n;
    T s = 0;
    for (int k = 0; k < n; ++k) s += U[k * LD + a] * bufC[k * LD + b];
    Tm[a * LD + b] = s;
  }
  __syncthreads();
  // Cholesky of the non-basis block Tm[r:, r:] (right-looking)
  for (int k = 0; k < m; ++k) {
    const T piv = Tm[(r + k) * LD + r + k];
    if (!(piv > T(0))) {
      if (tid == 0) set_status(status, CE_ERR_NOT_SPD, level, i, 1, k, static_cast<double>(piv));
      return;
    }
    const T d = sqrt(piv);
    __syncthreads();
    for (int a = k + tid; a < m; a += kThreads) {
      if (a == k)
        Tm[(r + k) * LD + r + k] = d;
      else
        Tm[(r + a) * LD + r + k] /= d;
    }
    __syncthreads();
    const int rem = m - k - 1;
    for (int e = tid; e < rem * rem; e += kThreads) {
      int a = k + 1 + e / rem, b = k + 1 + e % rem;
      if (b <= a) Tm[(r + a) * LD + r + b] -= Tm[(r + a) * LD + r + k] * Tm[(r + b) * LD + r + k];
    }
    __syncthreads();
  }
  T* Lg = reinterpret_cast<T*>(L.L) + L.l_off[i];
  for (int e = tid; e < m * m; e += kThreads) {
    int a = e / m, b = e - a * m;
    Lg[e] = (b <= a) ? Tm[(r + a) * LD + r + b] : T(0);
  }
  // W_b = L_hat^{-1} Tm[r:, :r] (in place)
  trsm_lower(Tm, r, m, Tm, r);
  __syncthreads();
  T* Wbase = reinterpret_cast<T*>(L.W) + L.w_off[i];
  for (int e = tid; e < m * r; e += kThreads) {
    int a = e / r, b = e - a * r;
    Wbase[e] = Tm[(r + a) * LD + b];
  }
  // basis diagonal block: Tm[:r, :r] - W_b^T W_b
  for (int e = tid; e < r * r; e += kThreads) {
    int a = e / r, b = e - a * r;
    T s = Tm[a * LD + b];
    for (int k = 0; k < m; ++k) s -= Tm[(r + k) * LD + a] * Tm[(r + k) * LD + b];
    Dg[(int64_t)a * n + b] = s;
  }
  // target bookkeeping
  const int c0 = L.close_ptr[i], c1 = L.close_ptr[i + 1];
  const int nt = 1 + (c1 - c0);
  if (tid == 0) {
    s_tgt[0] = i;
    s_w[0] = r;
    s_colst[0] = 0;
    int cs = n;
    for (int t = 1; t < nt && t < kMaxTargets; ++t) {
      int p = L.close_blk[c0 + t - 1];
      s_tgt[t] = p;
      s_w[t] = width_of(L, p, ci);
      s_colst[t] = cs;
      cs += L.n[p];
    }
  }
  __syncthreads();
  if (nt > kMaxTargets) {
    if (tid == 0) set_status(status, CE_ERR_LIMIT, level, i);
    return;
  }
  // close rows: Y = U^T X_ip; W_p = L_hat^{-1} Y[r:]; basis rows Y[:r] - W_b^T W_p
  for (int t = 1; t < nt; ++t) {
    const int p = s_tgt[t], w = s_w[t], np = L.n[p];
    T* Xg = pool + L.close_off[c0 + t - 1];
    load_row_tile(bufB, Xg, i, p, n, np, w);
    __syncthreads();
    for (int e = tid; e < n * w; e += kThreads) {
      int a = e / w, b = e - a * w;
      T s = 0;
      for (int k = 0; k < n; ++k) s += U[k * LD + a] * bufB[k * LD + b];
      bufC[a * LD + b] = s;
    }
    __syncthreads();
    trsm_lower(Tm, r, m, bufC, w);
    __syncthreads();
    T* Wp = Wbase + (int64_t)n * s_colst[t];
    for (int e = tid; e < m * w; e += kThreads) {
      int a = e / w, b = e - a * w;
      Wp[e] = bufC[(r + a) * LD + b];
    }
    for (int e = tid; e < r * w; e += kThreads) {
      int a = e / w, b = e - a * w;
      T s = bufC[a * LD + b];
      for (int k = 0; k < m; ++k) s -= Tm[(r + k) * LD + a] * bufC[(r + k) * LD + b];
      bufB[a * LD + b] = s;
    }
    __syncthreads();
    store_row_tile(bufB, Xg, i, p, n, np, r, w);
    __syncthreads();
  }
  // far rows: keep U_b^T F (the rows r.. are E_i and are dropped)
  for (int f = L.far_ptr[i]; f < L.far_ptr[i + 1]; ++f) {
    const int k = L.far_blk[f];
    const int w = width_of(L, k, ci);
    const int nk = L.n[k];
    T* Xg = pool + L.far_off[f];
    load_row_tile(bufB, Xg, i, k, n, nk, w);
    __syncthreads();
    for (int e = tid; e < r * w; e += kThreads) {
      int a = e / w, b = e - a * w;
      T s = 0;
      for (int kk = 0; kk < n; ++kk) s += U[kk * LD + a] * bufB[kk * LD + b];
      bufC[a * LD + b] = s;
    }
    __syncthreads();
    store_row_tile(bufC, Xg, i, k, n, nk, r, w);
    __syncthreads();
  }
  // Schur update between close targets: A(p, q) -= W_p^T W_q
  if (m > 0) {
    int idx = L.schur_ptr[i] + nt;   // skip the row of the basis of i
    for (int a = 1; a < nt; ++a) {
      for (int b = a; b < nt; ++b, ++idx) {
        const int wa = s_w[a], wb = s_w[b];
        const T* Wa = Wbase + (int64_t)n * s_colst[a];
        const T* Wb = Wbase + (int64_t)n * s_colst[b];
        T* Xg = pool + L.schur_off[idx];
        const int ld = L.n[s_tgt[b]];
        for (int e = tid; e < wa * wb; e += kThreads) {
          int x = e / wb, y = e - x * wb;
          T s = 0;
          for (int k = 0; k < m; ++k) s += Wa[k * wa + x] * Wb[k * wb + y];
          Xg[(int64_t)x * ld + y] -= s;
        }
      }
    }
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
constexpr int NB = 64;
constexpr int NBL = NB + 1;

__global__ void potrf_tile_kernel(double* A, int n, int k0, int level, int* status) {
  if (*status) return;
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
      if (threadIdx.x == 0) set_status(status, CE_ERR_NOT_SPD, level, -1, 1, k0 + k, piv);
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
__global__ void trsm_tile_kernel(double* A, int n, int k0, const int* status) {
  if (*status) return;
  extern __shared__ double tile_smem[];
  double* Lk = tile_smem;
  double* X = tile_smem + NB * NBL;
  const int nb = min(NB, n - k0);
  const int i0 = k0 + nb + blockIdx.x * NB;
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
__global__ void syrk_tile_kernel(double* A, int n, int k0, const int* status) {
  if (*status) return;
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

size_t row_kernel_smem(int esize) {
  return static_cast<size_t>(esize) * (4 * kNMax * LD + 2 * kNMax);
}

cudaError_t launch_row_kernel(int esize, const LevelDev& L, int first, int count, int level,
                              double tol, int tol_mode, int* status, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = row_kernel_smem(esize);
  if (esize == 8) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(ce_row_kernel<double>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ce_row_kernel<double><<<count, kThreads, smem, s>>>(L, first, level, tol, tol_mode, status);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(ce_row_kernel<float>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ce_row_kernel<float><<<count, kThreads, smem, s>>>(L, first, level, tol, tol_mode, status);
  }
  return cudaGetLastError();
}

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

cudaError_t coarse_cholesky(double* A, int n, int level, int* status, cudaStream_t s) {
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
  for (int k0 = 0; k0 < n; k0 += NB) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    potrf_tile_kernel<<<1, 256, 0, s>>>(A, n, k0, level, status);
    const int nb = std::min(NB, n - k0);
    const int below = n - k0 - nb;
    if (below > 0) {
      const int tiles = (below + NB - 1) / NB;
      g_launches.fetch_add(1, std::memory_order_relaxed);
      trsm_tile_kernel<<<tiles, 64, tile_bytes, s>>>(A, n, k0, status);
      g_launches.fetch_add(1, std::memory_order_relaxed);
      syrk_tile_kernel<<<tiles * (tiles + 1) / 2, 256, tile_bytes, s>>>(A, n, k0, status);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ce
