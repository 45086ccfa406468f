// Large block rows: Algorithm 2 for levels whose blocks outgrow the row
// kernel's shared memory (more than 64 rows, more than 32 close or 128 far
// blocks), as in 3D, where super-blocks of J = 8 boxes of boxes hold hundreds
// of rows (Section 2.4) and the per-row products become true GEMM shapes.
//
// One colour at a time (its rows are independent: distance-2 colouring), the
// steps of every row of the colour run as batched kernels with the row's
// matrices in global memory:
//   1. gather F_i^T (mF x n) from the far pairs            (copy tasks)
//   2. R = R factor of F_i^T: parts on several CTAs, merge tree (tsqr_*_kernel)
//   3. one-sided Jacobi on R: U_i, sigma, r_i, tau_i        (jacobi_kernel)
//   4. X = D U, T = U^T D U                                (grouped GEMM)
//   5. T_nn = L_hat L_hat^T, L_hat^{-1}                    (cholinv_kernel)
//   6. W_b = L_hat^{-1} T[r:, :r], Y_p = U^T C_ip, U_b^T F (grouped GEMM)
//   7. D_i <- T[:r, :r] - W_b^T W_b, W_p = L_hat^{-1} Y_p[r:]
//   8. kept close rows Y_p[:r] - W_b^T W_p, Schur A(p, q) -= W_p^T W_q
// The factor keeps the row kernel's layout (U_i, L_hat_i^{-1}, W_i), so the
// reassembly and the level vectors are shared; the apply of such a level runs
// one launch per colour (apply_big_kernel).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "rng.cuh"

namespace ce {

namespace {

namespace cg = cooperative_groups;

template <typename T>
struct EpsB;
template <>
struct EpsB<double> {
  static constexpr double v = 2.220446049250313e-16;
};
template <>
struct EpsB<float> {
  static constexpr float v = 1.1920928955078125e-07f;
};
template <typename T>
struct TinyB;
template <>
struct TinyB<double> {
  static constexpr double v = 2.2250738585072014e-308;
};
template <>
struct TinyB<float> {
  static constexpr float v = 1.1754943508222875e-38f;
};

constexpr int kBigMaxSweeps = 40;
constexpr double kBigTieRel = 1e-3;

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T wmax(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ void big_status(int* status, int code, int level, int block, int reason, int pivot = -1,
                           double value = 0.0) {
  if (atomicCAS(status, 0, code) == 0) {
    status[1] = level;
    status[2] = block;
    status[3] = reason;
    status[4] = pivot;
    *reinterpret_cast<double*>(status + 6) = value;
  }
}

// ---------------------------------------------------------------------------
// Grouped GEMM on the CUDA cores: 64 x 64 output tiles, 16-deep K slices in
// shared memory, 4 x 4 outputs per thread.  Task t covers tiles
// [tile0, tile0 + ceil(M/64) ceil(N/64)).
// ---------------------------------------------------------------------------
constexpr int kGT = 64, kGK = 16, kGThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kGThreads) gemm_tasks_kernel(const GemmTask* tasks, int ntasks) {
  __shared__ T As[kGK][kGT + 1], Bs[kGK][kGT + 1];
  __shared__ int s_task;
  const int tid = threadIdx.x;
  if (tid == 0) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_task = lo;
  }
  __syncthreads();
  const GemmTask& tk = tasks[s_task];
  const int M = tk.M, N = tk.N, K = tk.K;
  const int tl = blockIdx.x - tk.tile0, tn = (N + kGT - 1) / kGT;
  const int m0 = (tl / tn) * kGT, n0 = (tl % tn) * kGT;
  const T* A = static_cast<const T*>(tk.A);
  const T* B = static_cast<const T*>(tk.B);
  const int tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < K; k0 += kGK) {
#pragma unroll
    for (int u = 0; u < (kGT * kGK) / kGThreads; ++u) {
      const int e = tid + u * kGThreads;
      int m, k;
      if (tk.ta) {  // A stored K x M: m contiguous
        m = e % kGT;
        k = e / kGT;
      } else {
        k = e % kGK;
        m = e / kGK;
      }
      const int gm = m0 + m, gk = k0 + k;
      T v = T(0);
      if (gm < M && gk < K) v = tk.ta ? A[(int64_t)gk * tk.lda + gm] : A[(int64_t)gm * tk.lda + gk];
      As[k][m] = v;
      int n2, k2;
      if (tk.tb) {  // B stored N x K: k contiguous
        k2 = e % kGK;
        n2 = e / kGK;
      } else {
        n2 = e % kGT;
        k2 = e / kGT;
      }
      const int gn = n0 + n2, gk2 = k0 + k2;
      T w = T(0);
      if (gn < N && gk2 < K) w = tk.tb ? B[(int64_t)gn * tk.ldb + gk2] : B[(int64_t)gk2 * tk.ldb + gn];
      Bs[k2][n2] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  const T alpha = static_cast<T>(tk.alpha), beta = static_cast<T>(tk.beta);
  const T* Cin = static_cast<const T*>(tk.Cin);
  T* C = static_cast<T*>(tk.C);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      T v = alpha * acc[i][j];
      T* dst = tk.tc ? &C[(int64_t)n * tk.ldc + m] : &C[(int64_t)m * tk.ldc + n];
      if (tk.atomic) {
        atomicAdd(dst, v);
        continue;
      }
      if (beta != T(0)) v += beta * (tk.tcin ? Cin[(int64_t)n * tk.ldcin + m] : Cin[(int64_t)m * tk.ldcin + n]);
      *dst = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Per-row descriptors of a colour's rows (device copy).
// ---------------------------------------------------------------------------
struct BigRowDev {
  int i;          // block index in the level
  int n, mF;      // block size and far rows of F_i^T
  int parts;      // CTAs of the TSQR of F_i^T (a power of 2)
  int64_t g_off;  // F_i^T, mF x n row-major (work space)
  int64_t x_off;  // parts x n x n: the TSQR's R_p (R_0 = R, the result)
  int64_t v_off;  // n x n: V (column-major)
  int64_t t_off;  // n x n: T = U^T D U (row-major)
  int64_t w2_off; // n x n: D U (row-major), then the Cholesky work matrix
  int mode;       // Jacobi output: 0 U_i, sigma, r_i, tau_i of block i (exact SVD);
                  // 1 the sketch's k x k factor: V sorted at u_out, sigma at s_out,
                  // r and tau in the row's SketchRes
  int64_t u_out, s_out;
};

// result of the randomized range finder of one row
struct SketchRes {
  double tau;      // threshold from the sketch's sigma_1
  double probe;    // largest ||(I - Q Q^T) F w|| of the two probe columns
  int rank;        // #{sigma > tau} of the sketch
  int accepted;    // rank < k and probe <= tau / 2
};

// ---------------------------------------------------------------------------
// R factor of F_i^T (mF x n) by stacked Householder steps: chunks of CH rows
// of F_i^T are pushed into the triangular R (n x n, global memory) panel by
// panel; one warp factorizes each 32-column panel of [R; C], the CTA applies
// the panel's compact WY form (I - V T V^T) to the trailing columns.
// ---------------------------------------------------------------------------
constexpr int kPW = 32;
constexpr int kBigThreads = 512;
constexpr int kTsqrThreads = 256;   // the trailing update keeps 64 values per thread in registers
constexpr int kJacThreads = 1024;   // Jacobi: 64 column pairs of a round at a time

template <typename T>
__device__ __forceinline__ bool hh_reflector(T x0, T c, T& beta, T& tau, T& sc) {
  const T amax = wmax(fabs(c));
  if (!(amax >= TinyB<T>::v)) return false;
  const T ia = T(1) / amax;
  const T xl = c * ia;
  const T s = wsum(xl * xl);
  const T a = fmax(amax, fabs(x0));
  const T x0a = x0 / a, ca = amax / a;
  const T nrm = a * sqrt(x0a * x0a + s * ca * ca);
  beta = (x0 >= T(0)) ? -nrm : nrm;
  tau = (beta - x0) / beta;
  sc = T(1) / (x0 - beta);
  return true;
}

// Push the CH rows held in shared memory (C, CH x n) into the upper
// triangular R (n x n, global), panels from column p_start (the columns
// before it are zero in these rows).
template <typename T, int CH>
__device__ void stack_chunk(T* R, int n, T* C, int p_start, T (&Rp)[kPW][kPW + 1], T (&Vc)[CH][kPW + 1],
                            T (&Tm)[kPW][kPW + 1], T (&tauv)[kPW]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int p0 = p_start; p0 < n; p0 += kPW) {
    const int pw = min(kPW, n - p0);
    if (warp == 0) {
      for (int e = lane; e < kPW * kPW; e += 32) {
        const int j = e / kPW, l = e % kPW;
        Rp[j][l] = (j < pw && l < pw) ? R[(int64_t)(p0 + j) * n + p0 + l] : T(0);
      }
      for (int e = lane; e < CH * kPW; e += 32) Vc[e / kPW][e % kPW] = T(0);
      __syncwarp();
      for (int j = 0; j < pw; ++j) {
        const T c = (lane < CH) ? C[lane * n + p0 + j] : T(0);
        T beta, tau, sc;
        const bool ok = hh_reflector(Rp[j][j], c, beta, tau, sc);
        if (lane < CH) Vc[lane][j] = ok ? c * sc : T(0);
        if (lane == 0) tauv[j] = ok ? tau : T(0);
        __syncwarp();
        if (ok) {
          if (lane == 0) Rp[j][j] = beta;
          const int l = j + 1 + lane;
          if (l < pw) {
            T d = Rp[j][l];
            for (int q = 0; q < CH; ++q) d += Vc[q][j] * C[q * n + p0 + l];
            d *= tau;
            Rp[j][l] -= d;
            for (int q = 0; q < CH; ++q) C[q * n + p0 + l] -= d * Vc[q][j];
          }
        }
        __syncwarp();
      }
      for (int e = lane; e < pw * pw; e += 32) {
        const int j = e / pw, l = e % pw;
        if (l >= j) R[(int64_t)(p0 + j) * n + p0 + l] = Rp[j][l];
      }
      // compact WY: T upper triangular, T[:j, j] = -tau_j T[:j, :j] (V[:, :j]^T v_j);
      // the R parts of the reflectors are distinct unit vectors, so
      // v_i^T v_j = vc_i . vc_j
      for (int j = 0; j < pw; ++j) {
        T g = T(0);
        if (lane < j)
          for (int q = 0; q < CH; ++q) g += Vc[q][lane] * Vc[q][j];
        Tm[lane][j] = g;   // temporarily v_lane . v_j
      }
      __syncwarp();
      for (int j = 0; j < pw; ++j) {
        // column j: Tm[i][j] = -tau_j sum_{k=i}^{j-1} T[i][k] g[k][j], i < j
        T acc = T(0);
        if (lane < j)
          for (int k = lane; k < j; ++k) acc += (k == lane ? tauv[k] : Tm[lane][k]) * Tm[k][j];
        __syncwarp();
        if (lane < j) Tm[lane][j] = -tauv[j] * acc;
        __syncwarp();
      }
      if (lane < pw) Tm[lane][lane] = tauv[lane];
    }
    __syncthreads();
    // trailing columns: X <- X - V T^T (V^T X), X = [R rows p0.. ; C]
    for (int l = p0 + pw + tid; l < n; l += kTsqrThreads) {
      T w[kPW];
#pragma unroll
      for (int j = 0; j < kPW; ++j) {
        T sacc = (j < pw) ? R[(int64_t)(p0 + j) * n + l] : T(0);
        for (int q = 0; q < CH; ++q) sacc += Vc[q][j] * C[q * n + l];
        w[j] = sacc;
      }
      T w2[kPW];
#pragma unroll
      for (int j = 0; j < kPW; ++j) {
        T sacc = T(0);
#pragma unroll
        for (int i2 = 0; i2 <= j; ++i2) sacc += Tm[i2][j] * w[i2];
        w2[j] = (j < pw) ? sacc : T(0);
      }
#pragma unroll
      for (int j = 0; j < kPW; ++j)
        if (j < pw) R[(int64_t)(p0 + j) * n + l] -= w2[j];
      for (int q = 0; q < CH; ++q) {
        T sacc = T(0);
#pragma unroll
        for (int j = 0; j < kPW; ++j) sacc += Vc[q][j] * w2[j];
        C[q * n + l] -= sacc;
      }
    }
    __syncthreads();
  }
}

// Part p of the TSQR of F_i^T: rows [p mF / P, (p + 1) mF / P) of F_i^T
// stacked into R_p (n x n at x_off + p n^2), one CTA per (part, row).
template <typename T, int CH>
__global__ void __launch_bounds__(kTsqrThreads) tsqr_part_kernel(const BigRowDev* rows, T* ws) {
  const BigRowDev rw = rows[blockIdx.y];
  const int n = rw.n, mF = rw.mF, P = rw.parts, p = blockIdx.x;
  if (mF <= 0 || n <= 0 || p >= P) return;
  extern __shared__ __align__(16) unsigned char big_smem[];
  T* C = reinterpret_cast<T*>(big_smem);          // CH x n
  __shared__ T Rp[kPW][kPW + 1], Vc[CH][kPW + 1], Tm[kPW][kPW + 1], tauv[kPW];
  const int tid = threadIdx.x;
  T* R = ws + rw.x_off + (int64_t)p * n * n;
  const T* G = ws + rw.g_off;
  const int r0 = (int)((int64_t)mF * p / P), r1 = (int)((int64_t)mF * (p + 1) / P);
  for (int64_t e = tid; e < (int64_t)n * n; e += kTsqrThreads) R[e] = T(0);
  __syncthreads();
  for (int g0 = r0; g0 < r1; g0 += CH) {
    const int nr = min(CH, r1 - g0);
    for (int e = tid; e < CH * n; e += kTsqrThreads) {
      const int q = e / n, a = e - q * n;
      C[e] = (q < nr) ? G[(int64_t)(g0 + q) * n + a] : T(0);
    }
    __syncthreads();
    stack_chunk<T, CH>(R, n, C, 0, Rp, Vc, Tm, tauv);
  }
}

// One level of the TSQR merge tree: R_a <- R factor of [R_a; R_b] with
// a = 2 h j, b = a + h (parts of one row); the rows of the triangular R_b are
// pushed in chunks, each from the panel of its first row.
template <typename T, int CH>
__global__ void __launch_bounds__(kTsqrThreads) tsqr_merge_kernel(const BigRowDev* rows, T* ws, int h) {
  const BigRowDev rw = rows[blockIdx.y];
  const int n = rw.n, mF = rw.mF, P = rw.parts;
  const int a = 2 * h * blockIdx.x, b = a + h;
  if (mF <= 0 || n <= 0 || b >= P) return;
  extern __shared__ __align__(16) unsigned char big_smem[];
  T* C = reinterpret_cast<T*>(big_smem);
  __shared__ T Rp[kPW][kPW + 1], Vc[CH][kPW + 1], Tm[kPW][kPW + 1], tauv[kPW];
  const int tid = threadIdx.x;
  T* Ra = ws + rw.x_off + (int64_t)a * n * n;
  const T* Rb = ws + rw.x_off + (int64_t)b * n * n;
  for (int c0 = 0; c0 < n; c0 += CH) {
    const int nr = min(CH, n - c0);
    for (int e = tid; e < CH * n; e += kTsqrThreads) {
      const int q = e / n, col = e - q * n;
      C[e] = (q < nr && col >= c0 + q) ? Rb[(int64_t)(c0 + q) * n + col] : T(0);
    }
    __syncthreads();
    stack_chunk<T, CH>(Ra, n, C, (c0 / kPW) * kPW, Rp, Vc, Tm, tauv);
  }
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the columns of X = R3^T, starting from the
// pivoted-QR preconditioner's X and V = Q3 (qrcp_precond_kernel): X V' = U' S,
// U_i = Q3 V' (accumulated in V) and sigma = S sorted descending; the
// truncation rule of the compression step (CE(eps), CE(r)) with the rounding
// floor u ||D_i||_F.  Columns are stored contiguously, half a warp per column
// pair of a round-robin round.  Rows without far columns get U_i = I, r_i = 0.
// ---------------------------------------------------------------------------
struct BigLevelArgs {
  int level;
  double tol;
  int tol_mode;
  int* status;
  int* stats;     // kStatsWords counters (Jacobi cap at [32 + level])
  int engine;     // FP32 GEMMs: 0 tensor cores (3 split-BF16 products), 1 CUDA cores,
                  // 2 tensor cores with one BF16 product for the Schur updates
  int* tc_err;    // set by a tensor-core pipeline wait that expired
  double* phase_ms; // host, 8 phase times accumulated (see ce_info.big_ms)
  int sketch;       // 1: randomized range finder first (learned form, FP32)
  unsigned long long seed;  // key of the sketch's Gaussians
};

// ---------------------------------------------------------------------------
// Preconditioning of the large-row Jacobi by a QR factorization with column
// pivoting (Drmac and Veselic, "New fast and accurate Jacobi SVD algorithm",
// SIAM J. Matrix Anal. Appl. 29, 2008): with R from the TSQR of F_i^T and
// R^T P = Q3 R3, the left singular vectors of F_i are Q3 times those of R3,
// and one-sided Jacobi on the columns of X = R3^T (accumulating into V = Q3)
// yields them directly, in a few sweeps because the pivoted factor is graded.
// One CTA per row; R^T is R's row-major buffer read as column-major, factored
// in place; X and V are written to the Jacobi's workspace.  Column norms are
// recomputed after every step (no downdating); a pivot ties to the lowest
// index.
// ---------------------------------------------------------------------------
constexpr int kQrThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kQrThreads) qrcp_precond_kernel(const BigRowDev* rows, T* ws) {
  const BigRowDev rw = rows[blockIdx.x];
  const int n = rw.n;
  if (n <= 0 || rw.mF <= 0) return;
  constexpr int kW = kQrThreads / 32;
  extern __shared__ __align__(16) unsigned char qr_smem[];
  T* nrm = reinterpret_cast<T*>(qr_smem);   // n: squared norms of the trailing columns
  T* tau = nrm + n;                          // n: reflector scalars
  __shared__ int s_piv;
  __shared__ T s_red[kW];
  __shared__ int s_idx[kW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* Z = ws + rw.x_off;   // column j at Z + j n (R^T)
  for (int j = warp; j < n; j += kW) {
    T sc = T(0);
    for (int i = lane; i < n; i += 32) sc += Z[(int64_t)j * n + i] * Z[(int64_t)j * n + i];
    sc = wsum(sc);
    if (lane == 0) nrm[j] = sc;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // pivot: the trailing column of largest norm
    {
      T best = T(-1);
      int bi = n;
      for (int j = k + tid; j < n; j += kQrThreads)
        if (nrm[j] > best) {
          best = nrm[j];
          bi = j;
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_red[warp] = best;
        s_idx[warp] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        T b = s_red[0];
        int ix = s_idx[0];
        for (int w = 1; w < kW; ++w)
          if (s_red[w] > b || (s_red[w] == b && s_idx[w] < ix)) {
            b = s_red[w];
            ix = s_idx[w];
          }
        s_piv = (ix < n) ? ix : k;
      }
      __syncthreads();
    }
    const int pv = s_piv;
    if (pv != k) {   // swap columns k and pv (and their norms)
      for (int i = tid; i < n; i += kQrThreads) {
        const T a = Z[(int64_t)k * n + i], b = Z[(int64_t)pv * n + i];
        Z[(int64_t)k * n + i] = b;
        Z[(int64_t)pv * n + i] = a;
      }
      if (tid == 0) {
        const T t = nrm[k];
        nrm[k] = nrm[pv];
        nrm[pv] = t;
      }
      __syncthreads();
    }
    // reflector of Z[k:, k] (warp 0): Z[k][k] <- beta, v = Z[k+1:, k] / (alpha - beta)
    if (warp == 0) {
      T x2 = T(0);
      for (int i = k + 1 + lane; i < n; i += 32) x2 += Z[(int64_t)k * n + i] * Z[(int64_t)k * n + i];
      x2 = wsum(x2);
      const T alpha = Z[(int64_t)k * n + k];
      T tk = T(0);
      if (x2 > T(0)) {
        const T beta = (alpha >= T(0)) ? -sqrt(alpha * alpha + x2) : sqrt(alpha * alpha + x2);
        tk = (beta - alpha) / beta;
        const T sc = T(1) / (alpha - beta);
        for (int i = k + 1 + lane; i < n; i += 32) Z[(int64_t)k * n + i] *= sc;
        __syncwarp();
        if (lane == 0) Z[(int64_t)k * n + k] = beta;
      }
      if (lane == 0) tau[k] = tk;
    }
    __syncthreads();
    const T tk = tau[k];
    // apply H_k = I - tau [1; v][1; v]^T to the trailing columns; their norms afresh
    for (int j = k + 1 + warp; j < n; j += kW) {
      T* zj = Z + (int64_t)j * n;
      const T* v = Z + (int64_t)k * n;
      T w = T(0);
      if (tk != T(0)) {
        for (int i = k + 1 + lane; i < n; i += 32) w += v[i] * zj[i];
        w = wsum(w) + zj[k];
        w *= tk;
      }
      T sc = T(0);
      for (int i = k + 1 + lane; i < n; i += 32) {
        const T z = zj[i] - w * v[i];
        zj[i] = z;
        sc += z * z;
      }
      sc = wsum(sc);
      if (lane == 0) {
        zj[k] -= w;
        nrm[j] = sc;
      }
    }
    __syncthreads();
  }
  // X = R3^T (column-major): X[c][r] = R3[c][r] = Z[r n + c] for c <= r
  T* X = ws + rw.t_off;
  T* V = ws + rw.v_off;
  for (int64_t e = tid; e < (int64_t)n * n; e += kQrThreads) {
    const int c = static_cast<int>(e / n), r = static_cast<int>(e % n);
    X[e] = (c <= r) ? Z[(int64_t)r * n + c] : T(0);
    V[e] = (c == r) ? T(1) : T(0);
  }
  __syncthreads();
  // V = Q3 = H_0 ... H_{n-1} (backward accumulation on the identity)
  for (int k = n - 1; k >= 0; --k) {
    const T tk = tau[k];
    if (tk != T(0)) {
      const T* v = Z + (int64_t)k * n;
      for (int j = k + warp; j < n; j += kW) {
        T* vj = V + (int64_t)j * n;
        T w = T(0);
        for (int i = k + 1 + lane; i < n; i += 32) w += v[i] * vj[i];
        w = (wsum(w) + vj[k]) * tk;
        for (int i = k + 1 + lane; i < n; i += 32) vj[i] -= w * v[i];
        if (lane == 0) vj[k] -= w;
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kJacThreads) jacobi_kernel(const BigRowDev* rows, T* ws, LevelDev L,
                                                             BigLevelArgs a, int xv_smem, SketchRes* res,
                                                             int presolved) {
  const BigRowDev rw = rows[blockIdx.x];
  const int n = rw.n, i = rw.i;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kW = kJacThreads / 32;
  __shared__ double s_red[kW];
  __shared__ T s_skip2;
  __shared__ int s_flag;
  extern __shared__ __align__(16) unsigned char big_smem[];
  T* sig = reinterpret_cast<T*>(big_smem);   // n
  int* pos = reinterpret_cast<int*>(sig + n); // n
  T* Ug = reinterpret_cast<T*>(L.U) + L.u_off[i];
  if (n <= 0) return;
  const T* D = reinterpret_cast<const T*>(L.pool) + L.diag_off[i];
  {
    double ss = 0.0;
    for (int64_t e = tid; e < (int64_t)n * n; e += kJacThreads) {
      const double v = static_cast<double>(D[e]);
      ss += v * v;
    }
    ss = wsum(ss);
    if (lane == 0) s_red[warp] = ss;
  }
  __syncthreads();
  double dn2 = 0.0;
  for (int w = 0; w < kW; ++w) dn2 += s_red[w];
  const double floor_tau = static_cast<double>(EpsB<T>::v) * sqrt(dn2);
  if (rw.mF <= 0) {
    for (int64_t e = tid; e < (int64_t)n * n; e += kJacThreads) Ug[e] = (e / n == e % n) ? T(1) : T(0);
    for (int k = tid; k < n; k += kJacThreads) L.sigma[L.vec_off[i] + k] = 0.0;
    if (tid == 0) {
      L.rank[i] = 0;
      L.tau[i] = 0.0;
    }
    return;
  }
  // columns of R contiguous; in shared memory when both n x n matrices fit
  // X and V start as the pivoted-QR preconditioner left them in the
  // workspace (presolved: block_jacobi_kernel already rotated them there)
  T* X = xv_smem ? reinterpret_cast<T*>(pos + ((n + 3) & ~3)) : ws + rw.t_off;
  T* V = xv_smem ? X + (int64_t)n * n : ws + rw.v_off;
  if (xv_smem)
    for (int64_t e = tid; e < (int64_t)n * n; e += kJacThreads) {
      X[e] = ws[rw.t_off + e];
      V[e] = ws[rw.v_off + e];
    }
  __syncthreads();
  const int nb = n + (n & 1), npairs = nb / 2;
  const T tolJ = T(n) * EpsB<T>::v, tolJ2 = tolJ * tolJ;
  bool conv = presolved != 0;
  int nsw = kBigMaxSweeps;
  for (int sweep = 0; sweep < kBigMaxSweeps && !presolved; ++sweep) {
    // pairs whose columns both stay below tau_est / (2 sqrt n) are skipped
    // (their rotation changes neither the kept subspace nor the rank)
    T cm = T(0);
    for (int j = warp; j < n; j += kW) {
      T s = T(0);
      for (int row = lane; row < n; row += 32) s += X[(int64_t)j * n + row] * X[(int64_t)j * n + row];
      s = wsum(s);
      cm = fmax(cm, s);
    }
    if (lane == 0) s_red[warp] = static_cast<double>(cm);
    __syncthreads();
    if (tid == 0) {
      double c2 = 0.0;
      for (int w = 0; w < kW; ++w) c2 = fmax(c2, s_red[w]);
      const T sm = static_cast<T>(sqrt(c2));
      T test = (a.tol == 0.0 || a.tol_mode == CE_TOL_FIXED) ? T(n) * EpsB<T>::v * sm
                                                            : ((a.tol_mode == CE_TOL_ABS) ? T(a.tol) : T(a.tol) * sm);
      test = fmax(test, static_cast<T>(floor_tau)) * T(0.5) / sqrt(T(n));
      s_skip2 = test * test;
      s_flag = 0;
    }
    __syncthreads();
    const T skip2 = s_skip2;
    const int half = lane >> 4, hl = lane & 15;
    for (int rnd = 0; rnd < nb - 1; ++rnd) {
      // half a warp per column pair of the round-robin round
      for (int tb = warp * 2; tb < npairs; tb += 2 * kW) {
        const int t = tb + half;
        int p = nb - 1, q = rnd;
        if (t != 0) {
          p = rnd + t;
          if (p >= nb - 1) p -= nb - 1;
          q = rnd - t;
          if (q < 0) q += nb - 1;
        }
        const bool valid = t < npairs && p < n && q < n;
        T* xp = X + (int64_t)(valid ? p : 0) * n;
        T* xq = X + (int64_t)(valid ? q : 0) * n;
        T al = 0, be = 0, ga = 0;
        if (valid)
          for (int row = hl; row < n; row += 16) {
            const T u = xp[row], v = xq[row];
            al += u * u;
            be += v * v;
            ga += u * v;
          }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (valid && ga != T(0) && (al >= skip2 || be >= skip2) && ga * ga > tolJ2 * al * be) {
          const T zeta = (be - al) / (T(2) * ga);
          const T az = fabs(zeta);
          const T den = (az > T(1)) ? az * (T(1) + sqrt(T(1) + T(1) / (az * az))) : az + sqrt(T(1) + az * az);
          const T tt = ((zeta >= T(0)) ? T(1) : T(-1)) / den;
          const T cs = T(1) / sqrt(T(1) + tt * tt), sn = cs * tt;
          T* vp = V + (int64_t)p * n;
          T* vq = V + (int64_t)q * n;
          for (int row = hl; row < n; row += 16) {
            const T u = xp[row], v = xq[row];
            xp[row] = cs * u - sn * v;
            xq[row] = sn * u + cs * v;
            const T u2 = vp[row], v2 = vq[row];
            vp[row] = cs * u2 - sn * v2;
            vq[row] = sn * u2 + cs * v2;
          }
          if (hl == 0) s_flag = 1;
        }
      }
      __syncthreads();
    }
    const int rotated = s_flag;
    __syncthreads();
    if (!rotated) {
      nsw = sweep + 1;
      conv = true;
      break;
    }
  }
  if (!conv && tid == 0 && a.stats && a.level < 16) atomicAdd(a.stats + 32 + a.level, 1);
  if (!presolved && tid == 0 && a.stats && a.level < 16) {
    atomicAdd(a.stats + 48 + a.level, nsw);
    atomicAdd(a.stats + 64 + a.level, 1);
  }
  __syncthreads();
  for (int j = warp; j < n; j += kW) {
    T s = T(0);
    for (int row = lane; row < n; row += 32) s += X[(int64_t)j * n + row] * X[(int64_t)j * n + row];
    s = wsum(s);
    if (lane == 0) sig[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = tid; j < n; j += kJacThreads) {
    const T sj = sig[j];
    int ps = 0;
    for (int k = 0; k < n; ++k) ps += (sig[k] > sj) || (sig[k] == sj && k < j);
    pos[j] = ps;
  }
  __syncthreads();
  // U_i[a][pos[j]] = V[:, j][a]; sigma sorted
  T* Uo = rw.mode ? ws + rw.u_out : Ug;
  for (int64_t e = tid; e < (int64_t)n * n; e += kJacThreads) {
    const int j = static_cast<int>(e / n), row = static_cast<int>(e % n);
    Uo[(int64_t)row * n + pos[j]] = V[e];
  }
  for (int j = tid; j < n; j += kJacThreads) {
    if (rw.mode)
      ws[rw.s_out + pos[j]] = sig[j];
    else
      L.sigma[L.vec_off[i] + pos[j]] = static_cast<double>(sig[j]);
  }
  __syncthreads();
  if (tid == 0) {
    // sorted singular values
    T smax = T(0);
    for (int j = 0; j < n; ++j) smax = fmax(smax, sig[j]);
    const double sm = static_cast<double>(smax);
    if (!isfinite(sm)) {
      big_status(a.status, CE_ERR_NOT_SPD, a.level, i, 2);
    } else {
      double tau;
      if (a.tol_mode == CE_TOL_FIXED) {
        const int rf = static_cast<int>(a.tol);
        tau = n * static_cast<double>(EpsB<T>::v) * sm;
        if (rf == 0) {
          tau = fmax(tau, sm);
        } else if (rf < n) {
          // sigma_rf: the rf-th largest
          double srf = 0.0;
          for (int j = 0; j < n; ++j)
            if (pos[j] == rf - 1) srf = static_cast<double>(sig[j]);
          tau = fmax(tau, (1.0 - kBigTieRel) * srf);
        }
      } else if (a.tol == 0.0) {
        tau = n * static_cast<double>(EpsB<T>::v) * sm;
      } else {
        tau = (a.tol_mode == CE_TOL_ABS) ? a.tol : a.tol * sm;
      }
      tau = fmax(tau, floor_tau);
      int rr = 0;
      for (int j = 0; j < n; ++j) rr += (static_cast<double>(sig[j]) > tau) ? 1 : 0;
      if (rw.mode) {
        res[blockIdx.x].rank = rr;
        res[blockIdx.x].tau = tau;
      } else {
        L.rank[i] = rr;
        L.tau[i] = tau;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Block one-sided Jacobi for rows whose R and V (n x n each) do not fit in
// one CTA's shared memory.  The n columns form blocks of B; each round of a
// round-robin tournament over the blocks pairs them up, and one CTA takes a
// pair of blocks: it stages their 2B columns of X (from the pivoted-QR
// preconditioner at the start) and of V in shared memory, runs one cyclic
// sweep of column rotations over them (a
// warp per column pair, the same pair test and rotation as jacobi_kernel),
// and writes them back.  All block pairs of a round, of every row of the
// colour, run at once; grid barriers (cooperative launch) separate the
// rounds.  A row has converged when one sweep over all its block pairs
// rotated nothing, the stopping rule of the one-CTA kernel; jacobi_kernel
// then reads sigma, the order, U and the rank from the rotated X and V.
// Columns move between CTAs from round to round, so they are read past L1.
// ---------------------------------------------------------------------------
struct BJRow {
  int sweeps;                // sweeps run (until converged or capped)
  double dn2;                // ||D_i||_F^2 (rounding floor of tau)
  unsigned long long cm;     // largest column norm^2 at the sweep's start (double bits)
  unsigned long long cmn;    // ... gathered during the sweep's last round
  int flag;                  // a rotation in this sweep
  int conv;                  // converged
};

template <typename T, int B>
__global__ void __launch_bounds__(32 * B) block_jacobi_kernel(const BigRowDev* rows, int nrows,
                                                              const int* item_ptr, int max_rounds, T* ws,
                                                              LevelDev L, BigLevelArgs a, BJRow* st) {
  constexpr int NT = 32 * B;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char bj_smem[];
  __shared__ double s_red[2][B];
  __shared__ int s_rot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ||D_i||_F^2 and the largest column norm of X
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const BigRowDev rw = rows[r];
    const int n = rw.n;
    if (rw.mF <= 0) {   // no far columns: nothing to rotate (U_i = I)
      if (tid == 0) {
        st[r].dn2 = 0.0;
        st[r].cm = 0ull;
        st[r].cmn = 0ull;
        st[r].flag = 0;
        st[r].conv = 1;
        st[r].sweeps = 0;
      }
      continue;
    }
    const T* X = ws + rw.t_off;   // X and V from the pivoted-QR preconditioner
    const T* D = reinterpret_cast<const T*>(L.pool) + L.diag_off[rw.i];
    double ss = 0.0;
    for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
      const double d = static_cast<double>(D[e]);
      ss += d * d;
    }
    __syncthreads();
    double cm = 0.0;
    for (int c = warp; c < n; c += B) {
      T sc = T(0);
      for (int row = lane; row < n; row += 32) sc += X[(int64_t)c * n + row] * X[(int64_t)c * n + row];
      cm = fmax(cm, static_cast<double>(wsum(sc)));
    }
    ss = wsum(ss);
    if (lane == 0) {
      s_red[0][warp] = ss;
      s_red[1][warp] = cm;
    }
    __syncthreads();
    if (tid == 0) {
      double t0 = 0.0, t1 = 0.0;
      for (int w = 0; w < B; ++w) {
        t0 += s_red[0][w];
        t1 = fmax(t1, s_red[1][w]);
      }
      st[r].dn2 = t0;
      st[r].cm = static_cast<unsigned long long>(__double_as_longlong(t1));
      st[r].cmn = 0ull;
      st[r].flag = 0;
      st[r].conv = 0;
      st[r].sweeps = 0;
    }
    __syncthreads();
  }
  grid.sync();
  const int nitems = item_ptr[nrows];
  T* Xs = reinterpret_cast<T*>(bj_smem);
  bool all_conv = false;
  for (int sweep = 0; sweep < kBigMaxSweeps && !all_conv; ++sweep) {
    for (int rnd = 0; rnd < max_rounds; ++rnd) {
      for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        int lo = 0, hi = nrows - 1;  // the row whose items hold it
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (item_ptr[mid] <= it) lo = mid; else hi = mid - 1;
        }
        const int r = lo, t = it - item_ptr[r];
        const BigRowDev rw = rows[r];
        const int n = rw.n;
        const int nbk = (n + B - 1) / B, nbp = nbk + (nbk & 1);
        if (__ldcg(&st[r].conv) || rnd >= nbp - 1) continue;   // CTA-uniform
        int I = nbp - 1, J = rnd;
        if (t != 0) {
          I = rnd + t;
          if (I >= nbp - 1) I -= nbp - 1;
          J = rnd - t;
          if (J < 0) J += nbp - 1;
        }
        // a block paired with the empty block (odd block count, or a single
        // block) sweeps over its own columns alone
        const bool vi = I < nbk, vj = J < nbk;
        if (!vi && !vj) continue;
        const int c0 = (vi ? I : J) * B, w0 = min(B, n - c0);
        const int c1 = (vi && vj) ? J * B : 0, w1 = (vi && vj) ? min(B, n - c1) : 0;
        const int nc = w0 + w1;
        T* Vs = Xs + (int64_t)2 * B * n;
        T* X = ws + rw.t_off;
        T* V = ws + rw.v_off;
        for (int64_t e = tid; e < (int64_t)nc * n; e += NT) {
          const int c = static_cast<int>(e / n), row = static_cast<int>(e % n);
          const int64_t g = (int64_t)(c < w0 ? c0 + c : c1 + c - w0) * n + row;
          Xs[e] = __ldcg(X + g);
          Vs[e] = __ldcg(V + g);
        }
        // pair-skipping threshold of the sweep (see jacobi_kernel)
        const double dn2 = __ldcg(&st[r].dn2);
        const double cmv = __longlong_as_double(static_cast<long long>(__ldcg(&st[r].cm)));
        const T sm = static_cast<T>(sqrt(cmv));
        T test = (a.tol == 0.0 || a.tol_mode == CE_TOL_FIXED) ? T(n) * EpsB<T>::v * sm
                                                              : ((a.tol_mode == CE_TOL_ABS) ? T(a.tol) : T(a.tol) * sm);
        test = fmax(test, static_cast<T>(static_cast<double>(EpsB<T>::v) * sqrt(dn2))) * T(0.5) / sqrt(T(n));
        const T skip2 = test * test;
        const T tolJ = T(n) * EpsB<T>::v, tolJ2 = tolJ * tolJ;
        if (tid == 0) s_rot = 0;
        __syncthreads();
        const int ncb = nc + (nc & 1), np = ncb / 2;
        for (int ir = 0; ir < ncb - 1; ++ir) {
          if (warp < np) {
            int p = ncb - 1, q = ir;
            if (warp != 0) {
              p = ir + warp;
              if (p >= ncb - 1) p -= ncb - 1;
              q = ir - warp;
              if (q < 0) q += ncb - 1;
            }
            if (p < nc && q < nc) {
              T* xp = Xs + (int64_t)p * n;
              T* xq = Xs + (int64_t)q * n;
              T al = 0, be = 0, ga = 0;
              for (int row = lane; row < n; row += 32) {
                const T u = xp[row], v = xq[row];
                al += u * u;
                be += v * v;
                ga += u * v;
              }
              al = wsum(al);
              be = wsum(be);
              ga = wsum(ga);
              if (ga != T(0) && (al >= skip2 || be >= skip2) && ga * ga > tolJ2 * al * be) {
                const T zeta = (be - al) / (T(2) * ga);
                const T az = fabs(zeta);
                const T den = (az > T(1)) ? az * (T(1) + sqrt(T(1) + T(1) / (az * az))) : az + sqrt(T(1) + az * az);
                const T tt = ((zeta >= T(0)) ? T(1) : T(-1)) / den;
                const T cs = T(1) / sqrt(T(1) + tt * tt), sn = cs * tt;
                T* vp = Vs + (int64_t)p * n;
                T* vq = Vs + (int64_t)q * n;
                for (int row = lane; row < n; row += 32) {
                  const T u = xp[row], v = xq[row];
                  xp[row] = cs * u - sn * v;
                  xq[row] = sn * u + cs * v;
                  const T u2 = vp[row], v2 = vq[row];
                  vp[row] = cs * u2 - sn * v2;
                  vq[row] = sn * u2 + cs * v2;
                }
                if (lane == 0) s_rot = 1;
              }
            }
          }
          __syncthreads();
        }
        for (int64_t e = tid; e < (int64_t)nc * n; e += NT) {
          const int c = static_cast<int>(e / n), row = static_cast<int>(e % n);
          const int64_t g = (int64_t)(c < w0 ? c0 + c : c1 + c - w0) * n + row;
          __stcg(X + g, Xs[e]);
          __stcg(V + g, Vs[e]);
        }
        if (rnd == nbp - 2) {   // the sweep's last round: column norms for the next sweep
          double cm = 0.0;
          for (int c = warp; c < nc; c += B) {
            T sc = T(0);
            for (int row = lane; row < n; row += 32) sc += Xs[(int64_t)c * n + row] * Xs[(int64_t)c * n + row];
            cm = fmax(cm, static_cast<double>(wsum(sc)));
          }
          if (lane == 0) atomicMax(&st[r].cmn, static_cast<unsigned long long>(__double_as_longlong(cm)));
        }
        if (tid == 0 && s_rot) atomicOr(&st[r].flag, 1);
        __syncthreads();
      }
      grid.sync();
    }
    // end of the sweep: a row without a rotation has converged
    if (blockIdx.x == 0)
      for (int r = tid; r < nrows; r += NT)
        if (!st[r].conv) {
          st[r].sweeps = sweep + 1;
          if (__ldcg(&st[r].flag) == 0) {
            st[r].conv = 1;
          } else {
            st[r].flag = 0;
            st[r].cm = __ldcg(&st[r].cmn);
            st[r].cmn = 0ull;
          }
        }
    grid.sync();
    int left = 0;
    for (int r = tid; r < nrows; r += NT) left |= __ldcg(&st[r].conv) == 0;
    all_conv = __syncthreads_or(left) == 0;
  }
  if (blockIdx.x == 0 && a.stats && a.level < 16)
    for (int r = tid; r < nrows; r += NT) {
      if (!__ldcg(&st[r].conv)) atomicAdd(a.stats + 32 + a.level, 1);
      atomicAdd(a.stats + 48 + a.level, st[r].sweeps);
      atomicAdd(a.stats + 64 + a.level, 1);
    }
}

// ---------------------------------------------------------------------------
// Randomized range finder of a large row (FP32 form): Y = F [Omega | w1 w2]
// with Gaussian Omega (mF x k) and two probe columns, Q = orth(Y[:, :k]),
// the SVD of Q^T F through the R factor of F^T Q and Jacobi on it (k x k).
// Accepted when the sketch is not saturated (r < k) and the probe estimate
// of the out-of-sketch residual ||(I - Q Q^T) F w|| is at most tau / 2, so
// the dropped part stays near tau; otherwise the exact SVD runs.
// ---------------------------------------------------------------------------
struct SketchRowDev {
  int i, n, mF, k;     // k sketch columns (+ 2 probes)
  int64_t om_off;      // Omega, mF x (k + 2)
  int64_t y_off;       // Y, n x (k + 2) (Householder vectors below the diagonal)
  int64_t q_off;       // explicit Q, n x k
  int64_t ub_off;      // U_b = Q V_B[:, :r], n x k (r columns used)
  int64_t s_out;       // sketch singular values (k), sorted
};

__device__ __forceinline__ unsigned long long big_sketch_key(unsigned long long seed, int level, int i, int g,
                                                             int c) {
  return splitmix64(seed ^ splitmix64(((unsigned long long)level << 40) ^ ((unsigned long long)i << 8) ^ 0x5EEDull) ^
                    splitmix64(((unsigned long long)g << 20) ^ (unsigned long long)c));
}

template <typename T>
__global__ void sketch_omega_kernel(const SketchRowDev* rows, T* ws, int level, unsigned long long seed) {
  const SketchRowDev rw = rows[blockIdx.y];
  const int kp = rw.k + 2;
  const int64_t tot = (int64_t)rw.mF * kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int g = static_cast<int>(e / kp), c = static_cast<int>(e - (int64_t)g * kp);
    ws[rw.om_off + e] = static_cast<T>(gauss_from_key(big_sketch_key(seed, level, rw.i, g, c)));
  }
}

// Householder QR of Y[:, :k] (n x (k + 2), row-major, global) carried along
// to the probe columns; the probe residuals; the explicit Q (n x k).
// Householder steps on a row-major matrix M (leading dimension ld): lanes run
// over columns, so every load and store of a row segment is coalesced; the
// rows below the pivot are split among warps when the columns are few.
// Reflector of column j (rows j..n-1): M[j][j] <- beta, v = M[j+1:, j] / (x0 -
// beta) stored in M and in s_v; returns tau (0: no reflection).
template <typename T>
__device__ T house_reflect_col(T* M, int ld, int n, int j, T* s_v) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ T s_t;
  __syncthreads();   // every thread is done with the previous s_t and s_v
  if (warp == 0) {
    T amax = T(0);
    for (int a = j + 1 + lane; a < n; a += 32) amax = fmax(amax, fabs(M[(int64_t)a * ld + j]));
    amax = wmax(amax);
    T tau = T(0);
    if (amax >= TinyB<T>::v) {
      T ss = T(0);
      for (int a = j + 1 + lane; a < n; a += 32) {
        const T v = M[(int64_t)a * ld + j] / amax;
        ss += v * v;
      }
      ss = wsum(ss);
      const T x0 = M[(int64_t)j * ld + j];
      const T aa = fmax(amax, fabs(x0));
      const T nrm = aa * sqrt((x0 / aa) * (x0 / aa) + ss * (amax / aa) * (amax / aa));
      const T beta = (x0 >= T(0)) ? -nrm : nrm;
      tau = (beta - x0) / beta;
      const T sc = T(1) / (x0 - beta);
      for (int a = j + 1 + lane; a < n; a += 32) {
        const T v = M[(int64_t)a * ld + j] * sc;
        M[(int64_t)a * ld + j] = v;
        s_v[a] = v;
      }
      __syncwarp();
      if (lane == 0) M[(int64_t)j * ld + j] = beta;
    }
    if (lane == 0) s_t = tau;
  }
  __syncthreads();
  return s_t;
}

// sum_{a0 <= a < a1} v[a] M[a][l]: eight independent partial sums, so eight
// row loads are in flight at a time (the rows are ld apart in memory)
template <typename T>
__device__ __forceinline__ T col_dot(const T* M, int ld, int l, const T* v, int a0, int a1) {
  T p[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  int a = a0;
  for (; a + 8 <= a1; a += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) p[u] += v[a + u] * M[(int64_t)(a + u) * ld + l];
  }
  for (; a < a1; ++a) p[0] += v[a] * M[(int64_t)a * ld + l];
  return ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
}

// M[a][l] -= d v[a] for a0 <= a < a1, eight rows at a time
template <typename T>
__device__ __forceinline__ void col_axpy(T* M, int ld, int l, const T* v, int a0, int a1, T d) {
  int a = a0;
  for (; a + 8 <= a1; a += 8) {
    T x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = M[(int64_t)(a + u) * ld + l];
#pragma unroll
    for (int u = 0; u < 8; ++u) M[(int64_t)(a + u) * ld + l] = x[u] - d * v[a + u];
  }
  for (; a < a1; ++a) M[(int64_t)a * ld + l] -= d * v[a];
}

// M[j:, c0:c1] <- (I - tau [1; v][1; v]^T) M[j:, c0:c1], v = s_v[j+1 .. n)
template <typename T, int NT>
__device__ void house_apply_cols(T* M, int ld, int n, int j, int c0, int c1, const T* s_v, T tau, T* red,
                                 T* dcol) {
  constexpr int W = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nc = c1 - c0;
  if (nc <= 0 || tau == T(0)) return;   // uniform
  const int G = (nc + 31) / 32;
  if (G >= W) {
    for (int g = warp; g < G; g += W) {
      const int l = c0 + 32 * g + lane;
      if (l < c1) {
        const T d = tau * (M[(int64_t)j * ld + l] + col_dot(M, ld, l, s_v, j + 1, n));
        M[(int64_t)j * ld + l] -= d;
        col_axpy(M, ld, l, s_v, j + 1, n, d);
      }
    }
    __syncthreads();
    return;
  }
  const int S = W / G, g = warp % G, sp = warp / G;
  const int R = n - j - 1, chunk = (R + S - 1) / S;
  const int a0 = j + 1 + sp * chunk, a1 = min(n, a0 + chunk);
  const int l = c0 + 32 * g + lane;
  const bool act = sp < S && l < c1;
  const T part = act ? col_dot(M, ld, l, s_v, a0, a1) : T(0);
  red[warp * 32 + lane] = part;
  __syncthreads();
  if (sp == 0 && l < c1) {
    T d = M[(int64_t)j * ld + l];
    for (int q = 0; q < S; ++q) d += red[(g + q * G) * 32 + lane];
    d *= tau;
    dcol[32 * g + lane] = d;
    M[(int64_t)j * ld + l] -= d;
  }
  __syncthreads();
  if (act) col_axpy(M, ld, l, s_v, a0, a1, dcol[32 * g + lane]);
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kBigThreads) sketch_qr_kernel(const SketchRowDev* rows, T* ws, SketchRes* res) {
  const SketchRowDev rw = rows[blockIdx.x];
  const int n = rw.n, k = rw.k, kp = k + 2;
  T* Y = ws + rw.y_off;
  T* Q = ws + rw.q_off;
  __shared__ T s_tau[1024], s_pr[2], s_v[kBigMaxN], red[kBigThreads], dcol[kBigThreads];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Householder QR of Y[:, :k]; the two probe columns are carried along
  for (int j = 0; j < k; ++j) {
    const T tq = house_reflect_col(Y, kp, n, j, s_v);
    if (tid == 0) s_tau[j] = tq;
    house_apply_cols<T, kBigThreads>(Y, kp, n, j, j + 1, kp, s_v, tq, red, dcol);
  }
  if (warp < 2) {  // ||(I - Q Q^T) F w|| = norm of rows k.. of H^T (F w)
    T ss = T(0);
    for (int a = k + lane; a < n; a += 32) {
      const T v = Y[(int64_t)a * kp + k + warp];
      ss += v * v;
    }
    ss = wsum(ss);
    if (lane == 0) s_pr[warp] = sqrt(ss);
  }
  // explicit Q = H_0 ... H_{k-1} [I_k; 0]
  for (int64_t e = tid; e < (int64_t)n * k; e += kBigThreads) {
    const int a = static_cast<int>(e / k), c = static_cast<int>(e - (int64_t)a * k);
    Q[e] = (a == c) ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const T tq = s_tau[j];
    if (tq != T(0)) {
      for (int a = j + 1 + tid; a < n; a += kBigThreads) s_v[a] = Y[(int64_t)a * kp + j];
      __syncthreads();
      house_apply_cols<T, kBigThreads>(Q, k, n, j, j, k, s_v, tq, red, dcol);
    }
  }
  if (tid == 0) res[blockIdx.x].probe = static_cast<double>(fmax(s_pr[0], s_pr[1]));
}

// acceptance of the sketch; an accepted row gets its rank, threshold and
// singular values (zeros beyond k) and the sketch width in kw
template <typename T>
__global__ void sketch_accept_kernel(const SketchRowDev* rows, const T* ws, SketchRes* res, LevelDev L,
                                     int* stats, int level) {
  const SketchRowDev rw = rows[blockIdx.x];
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    SketchRes& r = res[blockIdx.x];
    const bool ok = isfinite(r.tau) && r.rank < rw.k && r.probe <= 0.5 * r.tau;
    r.accepted = ok ? 1 : 0;
    s_ok = ok;
    if (ok) {
      L.rank[rw.i] = r.rank;
      L.tau[rw.i] = r.tau;
    }
    if (L.kw) L.kw[rw.i] = ok ? rw.k : -rw.k;
    if (stats && level < 16) atomicAdd(stats + 2 * level + (ok ? 0 : 1), 1);
  }
  __syncthreads();
  if (s_ok)
    for (int j = threadIdx.x; j < rw.n; j += blockDim.x)
      L.sigma[L.vec_off[rw.i] + j] = (j < rw.k) ? static_cast<double>(ws[rw.s_out + j]) : 0.0;
}

// U_i (n x n orthogonal) whose first r columns span U_b = Q V_B[:, :r]:
// Householder QR of U_b (n x r, in place), U = H_0 ... H_{r-1} into the factor
template <typename T>
__global__ void __launch_bounds__(kBigThreads) complete_u_kernel(const SketchRowDev* rows, T* ws, LevelDev L) {
  const SketchRowDev rw = rows[blockIdx.x];
  const int n = rw.n, i = rw.i, r = L.rank[i];
  T* Ub = ws + rw.ub_off;   // n x r, row-major (ld r)
  T* U = reinterpret_cast<T*>(L.U) + L.u_off[i];
  __shared__ T s_tau[1024], s_v[kBigMaxN], red[kBigThreads], dcol[kBigThreads];
  const int tid = threadIdx.x;
  for (int j = 0; j < r; ++j) {
    const T tq = house_reflect_col(Ub, r, n, j, s_v);
    if (tid == 0) s_tau[j] = tq;
    house_apply_cols<T, kBigThreads>(Ub, r, n, j, j + 1, r, s_v, tq, red, dcol);
  }
  for (int64_t e = tid; e < (int64_t)n * n; e += kBigThreads) U[e] = (e / n == e % n) ? T(1) : T(0);
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    const T tq = s_tau[j];
    if (tq != T(0)) {
      for (int a = j + 1 + tid; a < n; a += kBigThreads) s_v[a] = Ub[(int64_t)a * r + j];
      __syncthreads();
      house_apply_cols<T, kBigThreads>(U, n, n, j, j, n, s_v, tq, red, dcol);
    }
  }
}

// ---------------------------------------------------------------------------
// Cholesky of T_nn = T[r:, r:] (m x m) and its inverse: L_hat^{-1} into the
// factor (m x m row-major, zero above the diagonal).  Right-looking, 32-column
// panels: one warp factorizes the diagonal tile, the CTA solves the panel
// below it and updates the trailing lower triangle; then the inverse by
// block forward substitution, one 32-row block row at a time.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBigThreads) cholinv_kernel(const BigRowDev* rows, T* ws, LevelDev L,
                                                              BigLevelArgs a, int stage) {
  // stage: the panel's rows below the diagonal tile are copied into dynamic
  // shared memory (m x (kPW + 1)) before the trailing update reads them
  extern __shared__ __align__(16) unsigned char ci_smem[];
  T* Ps = reinterpret_cast<T*>(ci_smem);
  const BigRowDev rw = rows[blockIdx.x];
  const int n = rw.n, i = rw.i;
  const int r = L.rank[i], m = n - r;
  if (n <= 0 || m <= 0) return;
  __shared__ T Dt[kPW][kPW + 1];
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* Tg = ws + rw.t_off;
  T* Aw = ws + rw.w2_off;   // m x m work, row-major
  T* Li = reinterpret_cast<T*>(L.L) + L.l_off[i];
  for (int64_t e = tid; e < (int64_t)m * m; e += kBigThreads) {
    const int x = static_cast<int>(e / m), y = static_cast<int>(e % m);
    Aw[e] = Tg[(int64_t)(r + x) * n + r + y];
    Li[e] = T(0);
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int p0 = 0; p0 < m; p0 += kPW) {
    const int pw = min(kPW, m - p0);
    if (warp == 0) {
      for (int e = lane; e < kPW * kPW; e += 32) {
        const int x = e / kPW, y = e % kPW;
        Dt[x][y] = (x < pw && y < pw) ? Aw[(int64_t)(p0 + x) * m + p0 + y] : T(0);
      }
      __syncwarp();
      for (int k = 0; k < pw; ++k) {
        const T piv = Dt[k][k];
        if (!(piv > T(0))) {
          if (lane == 0) {
            s_bad = 1;
            big_status(a.status, CE_ERR_NOT_SPD, a.level, i, 1, p0 + k, static_cast<double>(piv));
          }
          break;
        }
        const T d = sqrt(piv);
        __syncwarp();
        if (lane == k) Dt[k][k] = d;
        if (lane > k && lane < pw) Dt[lane][k] /= d;
        __syncwarp();
        if (lane > k && lane < pw)
          for (int y = k + 1; y <= lane; ++y) Dt[lane][y] -= Dt[lane][k] * Dt[y][k];
        __syncwarp();
      }
      for (int e = lane; e < pw * pw; e += 32) {
        const int x = e / pw, y = e % pw;
        if (y <= x) Aw[(int64_t)(p0 + x) * m + p0 + y] = Dt[x][y];
      }
    }
    __syncthreads();
    if (s_bad) return;
    // panel below: A[x, p0:p0+pw] <- A[x, p0:p0+pw] L_pp^{-T}
    for (int x = p0 + pw + tid; x < m; x += kBigThreads) {
      T row[kPW];
#pragma unroll
      for (int j = 0; j < kPW; ++j) row[j] = (j < pw) ? Aw[(int64_t)x * m + p0 + j] : T(0);
#pragma unroll
      for (int j = 0; j < kPW; ++j) {
        if (j < pw) {
          T s = row[j];
          for (int k = 0; k < j; ++k) s -= row[k] * Dt[j][k];
          row[j] = s / Dt[j][j];
        }
      }
#pragma unroll
      for (int j = 0; j < kPW; ++j)
        if (j < pw) Aw[(int64_t)x * m + p0 + j] = row[j];
    }
    __syncthreads();
    // trailing lower triangle: A[x, y] -= A[x, panel] . A[y, panel], y <= x
    const int t0 = p0 + pw, nt = m - t0;
    const int64_t tri = (int64_t)nt * (nt + 1) / 2;
    if (stage && nt > 0) {
      for (int e = tid; e < nt * kPW; e += kBigThreads) {
        const int x = e / kPW, j = e % kPW;
        Ps[x * (kPW + 1) + j] = (j < pw) ? Aw[(int64_t)(t0 + x) * m + p0 + j] : T(0);
      }
      __syncthreads();
    }
    for (int64_t e = tid; e < tri; e += kBigThreads) {
      // e -> (x, y) with y <= x in the trailing block
      int x = static_cast<int>((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
      while ((int64_t)x * (x + 1) / 2 > e) --x;
      while ((int64_t)(x + 1) * (x + 2) / 2 <= e) ++x;
      const int y = static_cast<int>(e - (int64_t)x * (x + 1) / 2);
      T s = T(0);
      if (stage) {
        const T* ax = Ps + x * (kPW + 1);
        const T* ay = Ps + y * (kPW + 1);
#pragma unroll 8
        for (int j = 0; j < kPW; ++j) s += ax[j] * ay[j];
      } else {
        const T* ax = Aw + (int64_t)(t0 + x) * m + p0;
        const T* ay = Aw + (int64_t)(t0 + y) * m + p0;
        for (int j = 0; j < pw; ++j) s += ax[j] * ay[j];
      }
      Aw[(int64_t)(t0 + x) * m + t0 + y] -= s;
    }
    __syncthreads();
  }
  // inverse: X = L^{-1}, block row I: X[I, J] = L_II^{-1} (delta_IJ - sum_{J <= K < I} L[I, K] X[K, J])
  const int nbk = (m + kPW - 1) / kPW;
  for (int I = 0; I < nbk; ++I) {
    const int r0 = I * kPW, h = min(kPW, m - r0);
    // inverse of the diagonal tile by one warp: column by column forward substitution
    if (warp == 0) {
      for (int e = lane; e < kPW * kPW; e += 32) {
        const int x = e / kPW, y = e % kPW;
        Dt[x][y] = (x < h && y < h && y <= x) ? Aw[(int64_t)(r0 + x) * m + r0 + y] : T(0);
      }
    }
    __syncthreads();
    // S = -sum_{K < I} L[I, K] X[K, J] for every column c < r0 (then X[I, c] = L_II^{-1} S)
    for (int e = tid; e < h * r0; e += kBigThreads) {
      const int x = e / r0, c = e % r0;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      const T* lr = Aw + (int64_t)(r0 + x) * m;
      int k = c;
      for (; k + 4 <= r0; k += 4) {
        s0 += lr[k] * Li[(int64_t)k * m + c];
        s1 += lr[k + 1] * Li[(int64_t)(k + 1) * m + c];
        s2 += lr[k + 2] * Li[(int64_t)(k + 2) * m + c];
        s3 += lr[k + 3] * Li[(int64_t)(k + 3) * m + c];
      }
      for (; k < r0; ++k) s0 += lr[k] * Li[(int64_t)k * m + c];
      Li[(int64_t)(r0 + x) * m + c] = -((s0 + s1) + (s2 + s3));   // staged, solved below
    }
    __syncthreads();
    // columns c < r0 + h: solve L_II y = rhs (rhs = staged S, or e_c for the diagonal tile)
    for (int c = tid; c < r0 + h; c += kBigThreads) {
      T y[kPW];
#pragma unroll
      for (int x = 0; x < kPW; ++x) {
        if (x < h) {
          T s = (c < r0) ? Li[(int64_t)(r0 + x) * m + c] : ((c - r0 == x) ? T(1) : T(0));
          for (int k = 0; k < x; ++k) s -= Dt[x][k] * y[k];
          y[x] = s / Dt[x][x];
        }
      }
#pragma unroll
      for (int x = 0; x < kPW; ++x)
        if (x < h && (c < r0 || c - r0 <= x)) Li[(int64_t)(r0 + x) * m + c] = y[x];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Apply of a large-row level, one launch per colour, one CTA per row (the
// forward and backward steps of the row kernel's factor layout; vectors of
// the row in dynamic shared memory, the targets' entries read from the level
// vector).
// ---------------------------------------------------------------------------
constexpr int kBigTgt = 64;

struct BigTargets {
  int nt;
  int w[kBigTgt], pre[kBigTgt + 1];
  int64_t woff[kBigTgt], voff[kBigTgt];
};

__device__ void big_targets(const LevelDev& L, int i, int n, int r, BigTargets& T) {
  const int ci = L.colour[i];
  const int c0 = L.close_ptr[i], c1 = L.close_ptr[i + 1];
  const int nt = min(1 + (c1 - c0), kBigTgt);
  int64_t colst = 0;
  int pre = 0;
  for (int t = 0; t < nt; ++t) {
    int w, np;
    int64_t vo;
    if (t == 0) {
      w = r;
      np = n;
      vo = L.vec_off[i];
    } else {
      const int p = L.close_blk[c0 + t - 1];
      w = (L.colour[p] < ci) ? L.rank[p] : L.n[p];
      np = L.n[p];
      vo = L.vec_off[p];
    }
    T.w[t] = w;
    T.woff[t] = (int64_t)n * colst;
    T.voff[t] = vo;
    T.pre[t] = pre;
    colst += np;
    pre += w;
  }
  T.pre[nt] = pre;
  T.nt = nt;
}

template <typename T, bool kFwd>
__global__ void __launch_bounds__(kBigThreads) apply_big_kernel(LevelDev L, int q0, double* vec) {
  __shared__ BigTargets tg;
  extern __shared__ __align__(16) unsigned char big_smem[];
  const int tid = threadIdx.x;
  const int i = L.order[q0 + blockIdx.x];
  const int n = L.n[i];
  if (n == 0) return;
  const int r = L.rank[i], m = n - r;
  T* ys = reinterpret_cast<T*>(big_smem);
  T* yt = ys + n;
  T* z = yt + n;
  double* v = vec + L.vec_off[i];
  const T* U = reinterpret_cast<const T*>(L.U) + L.u_off[i];
  const T* Li = reinterpret_cast<const T*>(L.L) + L.l_off[i];
  const T* W = reinterpret_cast<const T*>(L.W) + L.w_off[i];
  if (tid == 0) big_targets(L, i, n, r, tg);
  for (int a = tid; a < n; a += kBigThreads) ys[a] = static_cast<T>(v[a]);
  __syncthreads();
  if (kFwd) {
    // yt = U^T ys
    for (int a = tid; a < n; a += kBigThreads) {
      T s = T(0);
      for (int k = 0; k < n; ++k) s += U[(int64_t)k * n + a] * ys[k];
      yt[a] = s;
    }
    __syncthreads();
    // z = L_hat^{-1} yt[r:]
    for (int a = tid; a < m; a += kBigThreads) {
      T s = T(0);
      const T* lr = Li + (int64_t)a * m;
      for (int k = 0; k <= a; ++k) s += lr[k] * yt[r + k];
      z[a] = s;
    }
    __syncthreads();
    for (int a = tid; a < m; a += kBigThreads) v[r + a] = static_cast<double>(z[a]);
    // targets: y_t[c] -= (W_t^T z)[c]; the basis of i gets yt - W_b^T z
    const int tot = tg.pre[tg.nt];
    for (int f = tid; f < tot; f += kBigThreads) {
      int t = 0;
      while (f >= tg.pre[t + 1]) ++t;
      const int c = f - tg.pre[t], w = tg.w[t];
      const T* Wt = W + tg.woff[t] + c;
      T s = T(0);
      for (int k = 0; k < m; ++k) s += Wt[(int64_t)k * w] * z[k];
      if (t == 0)
        v[c] = static_cast<double>(yt[c] - s);
      else if (L.accumulate)
        atomicAdd(&vec[tg.voff[t] + c], -static_cast<double>(s));
      else
        vec[tg.voff[t] + c] -= static_cast<double>(s);
    }
  } else {
    // rhs = z - sum_t W_t x_t (x_0 = basis of i, x_t = target values)
    for (int a = tid; a < m; a += kBigThreads) {
      T s = T(0);
      for (int t = 0; t < tg.nt; ++t) {
        const int w = tg.w[t];
        const T* Wt = W + tg.woff[t] + (int64_t)a * w;
        if (t == 0)
          for (int c = 0; c < w; ++c) s += Wt[c] * ys[c];
        else
          for (int c = 0; c < w; ++c) s += Wt[c] * static_cast<T>(vec[tg.voff[t] + c]);
      }
      yt[a] = ys[r + a] - s;
    }
    __syncthreads();
    // x_n = L_hat^{-T} rhs
    for (int a = tid; a < m; a += kBigThreads) {
      T s = T(0);
      for (int k = a; k < m; ++k) s += Li[(int64_t)k * m + a] * yt[k];
      z[a] = s;
    }
    __syncthreads();
    for (int a = tid; a < m; a += kBigThreads) ys[r + a] = z[a];
    __syncthreads();
    // y_i = U [x_b; x_n]
    for (int a = tid; a < n; a += kBigThreads) {
      T s = T(0);
      const T* ur = U + (int64_t)a * n;
      for (int k = 0; k < n; ++k) s += ur[k] * ys[k];
      v[a] = static_cast<double>(s);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct BigFail {
  cudaError_t e;
};

void bcheck(cudaError_t e) {
  if (e != cudaSuccess) throw BigFail{e};
}

template <typename T>
cudaError_t launch_gemm_t(const std::vector<GemmTask>& tasks_in, cudaStream_t s) {
  if (tasks_in.empty()) return cudaSuccess;
  std::vector<GemmTask> tasks;
  tasks.reserve(tasks_in.size());
  int tiles = 0;
  for (const GemmTask& t : tasks_in) {
    if (t.M <= 0 || t.N <= 0) continue;
    GemmTask u = t;
    u.tile0 = tiles;
    tiles += ((t.M + kGT - 1) / kGT) * ((t.N + kGT - 1) / kGT);
    tasks.push_back(u);
  }
  if (tasks.empty()) return cudaSuccess;
  GemmTask* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), tasks.size() * sizeof(GemmTask), s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d, tasks.data(), tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    gemm_tasks_kernel<T><<<tiles, kGThreads, 0, s>>>(d, static_cast<int>(tasks.size()));
    e = cudaGetLastError();
  }
  cudaFreeAsync(d, s);
  // the task array is read by the kernel before the free runs (stream order);
  // the host vector is copied before cudaMemcpyAsync from pageable memory returns
  return e;
}

// GEMM task helpers: element (x, y) of a block pair seen from block a (rows
// of a, columns of b) in the pool, where pairs are stored once as
// (min, max) row-major.
struct PairView {
  int64_t off;   // element offset in the pool
  int ld;        // leading dimension of the stored pair
  int trans;     // 1: element (x, y) at off + y * ld + x
};

PairView pair_view(const LevelPlan& P, int a, int b) {
  const int64_t off = find_pair(P, a, b);
  if (off < 0) throw BigFail{cudaErrorInvalidValue};
  if (a <= b) return {off, P.n[b], 0};
  return {off, P.n[a], 1};
}

// Block Jacobi of the rows `rv` (device copy `drv`) in the workspace `wsb`:
// the widest column block B in {32, 16, 8, 4} whose 2B columns of X and V
// fit in shared memory, one cooperative launch (a resident wave of CTAs).
template <typename T, int B>
void launch_block_jacobi_b(const std::vector<BigRowDev>& rv, const BigRowDev* drv, T* wsb, const LevelDev& D,
                           const BigLevelArgs& args, size_t smem, cudaStream_t s) {
  static size_t attr = 0;
  if (attr < smem) {
    bcheck(cudaFuncSetAttribute(block_jacobi_kernel<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  const int nr = static_cast<int>(rv.size());
  std::vector<int> ptr(nr + 1, 0);
  int max_rounds = 1;
  for (int q = 0; q < nr; ++q) {
    const int nbk = (rv[q].n + B - 1) / B, nbp = nbk + (nbk & 1);
    ptr[q + 1] = ptr[q] + nbp / 2;
    max_rounds = std::max(max_rounds, nbp - 1);
  }
  void* buf = nullptr;
  const size_t pb = (nr + 1) * sizeof(int), sb = nr * sizeof(BJRow);
  bcheck(cudaMallocAsync(&buf, sb + pb, s));
  BJRow* dst = static_cast<BJRow*>(buf);
  int* dptr = reinterpret_cast<int*>(static_cast<char*>(buf) + sb);
  bcheck(cudaMemcpyAsync(dptr, ptr.data(), pb, cudaMemcpyHostToDevice, s));
  int dev = 0, per_sm = 0;
  bcheck(cudaGetDevice(&dev));
  bcheck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_jacobi_kernel<T, B>, 32 * B, smem));
  if (per_sm < 1) throw BigFail{cudaErrorInvalidConfiguration};
  const int grid = std::max(1, std::min(std::max(ptr[nr], nr), per_sm * device_sms()));
  int nrr = nr;
  LevelDev Dv = D;
  BigLevelArgs av = args;
  void* kargs[] = {(void*)&drv, (void*)&nrr, (void*)&dptr, (void*)&max_rounds, (void*)&wsb,
                   (void*)&Dv, (void*)&av, (void*)&dst};
  g_launches.fetch_add(1, std::memory_order_relaxed);
  bcheck(cudaLaunchCooperativeKernel((const void*)block_jacobi_kernel<T, B>, dim3(grid), dim3(32 * B), kargs,
                                     smem, s));
  bcheck(cudaFreeAsync(buf, s));
}

// Column blocks of 8 by default: a colour holds few large rows, and small
// blocks give each row many block pairs (CTAs) per round; wider blocks
// (fewer rounds, fewer grid barriers) once the pairs of B = 8 would fill two
// waves of the GPU; narrower ones when 8 columns of X and V do not fit.
template <typename T>
void launch_block_jacobi(const std::vector<BigRowDev>& rv, const BigRowDev* drv, T* wsb, const LevelDev& D,
                         const BigLevelArgs& args, size_t smem_limit, cudaStream_t s) {
  int nmx = 1;
  for (const BigRowDev& r : rv) nmx = std::max(nmx, r.n);
  auto need = [&](int b) { return (size_t)4 * b * nmx * sizeof(T) + 256; };
  auto items = [&](int b) {
    int64_t t = 0;
    for (const BigRowDev& r : rv) {
      const int nbk = (r.n + b - 1) / b;
      t += (nbk + (nbk & 1)) / 2;
    }
    return t;
  };
  const int64_t wave = 2LL * device_sms();
  if (items(16) >= wave && need(32) <= smem_limit)
    return launch_block_jacobi_b<T, 32>(rv, drv, wsb, D, args, need(32), s);
  if (items(8) >= wave && need(16) <= smem_limit)
    return launch_block_jacobi_b<T, 16>(rv, drv, wsb, D, args, need(16), s);
  if (need(8) <= smem_limit) return launch_block_jacobi_b<T, 8>(rv, drv, wsb, D, args, need(8), s);
  if (need(4) <= smem_limit) return launch_block_jacobi_b<T, 4>(rv, drv, wsb, D, args, need(4), s);
  throw BigFail{cudaErrorInvalidValue};
}

template <typename T>
void run_big_level_t(LevelStore& st, cudaStream_t s, const BigLevelArgs& args, std::vector<int>& rank_h) {
  const LevelPlan& P = *st.plan;
  LevelDev& D = st.dev;
  T* pool = static_cast<T*>(D.pool);
  T* Uf = static_cast<T*>(D.U);
  T* Lf = static_cast<T*>(D.L);
  T* Wf = static_cast<T*>(D.W);
  const int es = sizeof(T);
  rank_h.assign(P.M, 0);
  std::vector<int> done(P.M, 0);
  // device time per phase (CUDA events between the phases of each colour)
  cudaEvent_t ev[9];
  for (int k = 0; k < 9; ++k) bcheck(cudaEventCreate(&ev[k]));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int k = 0; k < 9; ++k) cudaEventDestroy(e[k]);
    }
  } evg{ev};
  auto mark = [&](int k) { bcheck(cudaEventRecord(ev[k], s)); };
  auto add_phases = [&](int upto) {  // after a synchronize: phase k = ev[k] .. ev[k+1]
    for (int k = 0; k < upto; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) == cudaSuccess && args.phase_ms) args.phase_ms[k] += ms;
    }
  };
  // GEMM groups: FP32 on the tensor cores unless the CUDA cores are asked
  // for (products with K = 0 only apply beta, on the CUDA cores)
  auto run_gemm = [&](const std::vector<GemmTask>& g, int passes) {
    if (g.empty()) return;
    if (sizeof(T) == 8 || args.engine == 1) {
      bcheck(launch_gemm_t<T>(g, s));
      return;
    }
    std::vector<GemmTask> tc, cc;
    for (const GemmTask& t : g) (t.K > 0 ? tc : cc).push_back(t);
    if (!cc.empty()) bcheck(launch_gemm_t<T>(cc, s));
    if (!tc.empty()) bcheck(launch_gemm_tc(tc, passes, args.tc_err, s));
  };
  auto width = [&](int k) { return done[k] ? rank_h[k] : P.n[k]; };
  constexpr int CH = sizeof(T) == 4 ? 32 : 16;
  static size_t tsqr_dyn = 0;  // dynamic shared memory the TSQR kernel may take
  if (tsqr_dyn == 0) {
    int dev = 0, optin = 0;
    bcheck(cudaGetDevice(&dev));
    bcheck(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa, fb;
    bcheck(cudaFuncGetAttributes(&fa, tsqr_part_kernel<T, CH>));
    bcheck(cudaFuncGetAttributes(&fb, tsqr_merge_kernel<T, CH>));
    const size_t lim = static_cast<size_t>(optin) - std::max(fa.sharedSizeBytes, fb.sharedSizeBytes);
    bcheck(cudaFuncSetAttribute(tsqr_part_kernel<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim));
    bcheck(cudaFuncSetAttribute(tsqr_merge_kernel<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim));
    tsqr_dyn = lim;
  }
  static size_t jac_dyn = 0;  // dynamic shared memory the Jacobi kernel may take
  if (jac_dyn == 0) {
    int dev = 0, optin = 0;
    bcheck(cudaGetDevice(&dev));
    bcheck(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    bcheck(cudaFuncGetAttributes(&fa, jacobi_kernel<T>));
    const size_t lim = static_cast<size_t>(optin) - fa.sharedSizeBytes;
    bcheck(cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim));
    jac_dyn = lim;
  }
  // one attempt of the randomized range finder on the rows cand (indices
  // into rows) with widths kcur; sets accepted[q] and, for accepted rows,
  // U_i in the factor (rank, tau, sigma by the accept kernel)
  auto run_sketch = [&](const std::vector<int>& cand, const std::vector<int>& kcur,
                        const std::vector<BigRowDev>& rows, T* ws, std::vector<char>& accepted) {
    std::vector<SketchRowDev> sk;
    std::vector<BigRowDev> view;   // the TSQR / Jacobi of the k x k problem
    int64_t o2 = 0;
    auto take2 = [&](int64_t elems) {
      const int64_t o = o2;
      o2 += (elems + 63) & ~int64_t(63);
      return o;
    };
    int maxp = 1, kmx = 1;
    for (int q : cand) {
      const BigRowDev& r = rows[q];
      const int k = kcur[q], kp = k + 2;
      SketchRowDev d{};
      d.i = r.i;
      d.n = r.n;
      d.mF = r.mF;
      d.k = k;
      d.om_off = take2((int64_t)r.mF * kp);
      d.y_off = take2((int64_t)r.n * kp);
      d.q_off = take2((int64_t)r.n * k);
      d.ub_off = take2((int64_t)r.n * k);
      d.s_out = take2(k);
      BigRowDev v{};
      v.i = r.i;
      v.n = k;
      v.mF = r.mF;
      int parts = 1;
      while (parts < 64 && (int64_t)parts * 2 * 4 * CH <= r.mF) parts *= 2;
      v.parts = parts;
      maxp = std::max(maxp, parts);
      kmx = std::max(kmx, k);
      v.g_off = take2((int64_t)r.mF * k);      // F^T Q
      v.x_off = take2((int64_t)parts * k * k);
      v.v_off = take2((int64_t)k * k);
      v.t_off = take2((int64_t)k * k);
      v.w2_off = 0;
      v.mode = 1;
      v.u_out = take2((int64_t)k * k);
      v.s_out = d.s_out;
      sk.push_back(d);
      view.push_back(v);
    }
    const int ns = static_cast<int>(sk.size());
    T* ws2 = nullptr;
    SketchRowDev* dsk = nullptr;
    BigRowDev* dview = nullptr;
    SketchRes* dres = nullptr;
    bcheck(cudaMallocAsync(reinterpret_cast<void**>(&ws2), std::max<int64_t>(o2, 64) * es, s));
    bcheck(cudaMallocAsync(reinterpret_cast<void**>(&dsk), ns * sizeof(SketchRowDev), s));
    bcheck(cudaMallocAsync(reinterpret_cast<void**>(&dview), ns * sizeof(BigRowDev), s));
    bcheck(cudaMallocAsync(reinterpret_cast<void**>(&dres), ns * sizeof(SketchRes), s));
    bcheck(cudaMemcpyAsync(dsk, sk.data(), ns * sizeof(SketchRowDev), cudaMemcpyHostToDevice, s));
    bcheck(cudaMemcpyAsync(dview, view.data(), ns * sizeof(BigRowDev), cudaMemcpyHostToDevice, s));
    bcheck(cudaMemsetAsync(dres, 0, ns * sizeof(SketchRes), s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    sketch_omega_kernel<T><<<dim3(64, ns), 256, 0, s>>>(dsk, ws2, args.level, args.seed);
    bcheck(cudaGetLastError());
    std::vector<GemmTask> gy, gb;
    for (int t = 0; t < ns; ++t) {
      const BigRowDev& r = rows[cand[t]];
      const int k = sk[t].k, kp = k + 2, n = r.n;
      GemmTask y{};   // Y = F [Omega | probes] = (F^T)^T Omega
      y.A = ws + r.g_off; y.lda = n; y.ta = 1;
      y.B = ws2 + sk[t].om_off; y.ldb = kp; y.tb = 0;
      y.C = ws2 + sk[t].y_off; y.ldc = kp; y.Cin = y.C; y.ldcin = kp;
      y.M = n; y.N = kp; y.K = r.mF; y.alpha = 1.f; y.beta = 0.f;
      gy.push_back(y);
      GemmTask b{};   // F^T Q
      b.A = ws + r.g_off; b.lda = n; b.ta = 0;
      b.B = ws2 + sk[t].q_off; b.ldb = k; b.tb = 0;
      b.C = ws2 + view[t].g_off; b.ldc = k; b.Cin = b.C; b.ldcin = k;
      b.M = r.mF; b.N = k; b.K = n; b.alpha = 1.f; b.beta = 0.f;
      gb.push_back(b);
    }
    run_gemm(gy, 3);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    sketch_qr_kernel<T><<<ns, kBigThreads, 0, s>>>(dsk, ws2, dres);
    bcheck(cudaGetLastError());
    run_gemm(gb, 3);
    const size_t sm = (size_t)CH * kmx * es;
    if (sm > tsqr_dyn) throw BigFail{cudaErrorInvalidValue};
    g_launches.fetch_add(1, std::memory_order_relaxed);
    tsqr_part_kernel<T, CH><<<dim3(maxp, ns), kTsqrThreads, sm, s>>>(dview, ws2);
    bcheck(cudaGetLastError());
    for (int h = 1; h < maxp; h *= 2) {
      g_launches.fetch_add(1, std::memory_order_relaxed);
      tsqr_merge_kernel<T, CH><<<dim3(maxp / (2 * h), ns), kTsqrThreads, sm, s>>>(dview, ws2, h);
      bcheck(cudaGetLastError());
    }
    size_t sj = (size_t)((kmx + 3) & ~3) * (es + sizeof(int)) + 64;
    const size_t sxv = sj + (size_t)2 * kmx * kmx * es;
    const int xv = sxv <= jac_dyn ? 1 : 0;
    if (xv) sj = sxv;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    qrcp_precond_kernel<T><<<ns, kQrThreads, (size_t)2 * kmx * es, s>>>(dview, ws2);
    bcheck(cudaGetLastError());
    if (!xv) launch_block_jacobi<T>(view, dview, ws2, D, args, jac_dyn, s);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    jacobi_kernel<T><<<ns, kJacThreads, sj, s>>>(dview, ws2, D, args, xv, dres, xv ? 0 : 1);
    bcheck(cudaGetLastError());
    g_launches.fetch_add(1, std::memory_order_relaxed);
    sketch_accept_kernel<T><<<ns, 128, 0, s>>>(dsk, ws2, dres, D, args.stats, args.level);
    bcheck(cudaGetLastError());
    std::vector<SketchRes> hres(ns);
    bcheck(cudaMemcpyAsync(hres.data(), dres, ns * sizeof(SketchRes), cudaMemcpyDeviceToHost, s));
    bcheck(cudaStreamSynchronize(s));
    // accepted rows: U_b = Q V_B[:, :r], then its orthogonal completion
    std::vector<GemmTask> gu;
    std::vector<SketchRowDev> acc;
    for (int t = 0; t < ns; ++t) {
      if (!hres[t].accepted) continue;
      accepted[cand[t]] = 1;
      const int r = hres[t].rank, k = sk[t].k;
      acc.push_back(sk[t]);
      if (r == 0) continue;
      GemmTask u{};
      u.A = ws2 + sk[t].q_off; u.lda = k; u.ta = 0;
      u.B = ws2 + view[t].u_out; u.ldb = k; u.tb = 0;
      u.C = ws2 + sk[t].ub_off; u.ldc = r; u.Cin = u.C; u.ldcin = r;
      u.M = rows[cand[t]].n; u.N = r; u.K = k; u.alpha = 1.f; u.beta = 0.f;
      gu.push_back(u);
    }
    if (!acc.empty()) {
      run_gemm(gu, 3);
      SketchRowDev* dacc = nullptr;
      bcheck(cudaMallocAsync(reinterpret_cast<void**>(&dacc), acc.size() * sizeof(SketchRowDev), s));
      bcheck(cudaMemcpyAsync(dacc, acc.data(), acc.size() * sizeof(SketchRowDev), cudaMemcpyHostToDevice, s));
      g_launches.fetch_add(1, std::memory_order_relaxed);
      complete_u_kernel<T><<<static_cast<int>(acc.size()), kBigThreads, 0, s>>>(dacc, ws2, D);
      bcheck(cudaGetLastError());
      bcheck(cudaFreeAsync(dacc, s));
    }
    bcheck(cudaFreeAsync(ws2, s));
    bcheck(cudaFreeAsync(dsk, s));
    bcheck(cudaFreeAsync(dview, s));
    bcheck(cudaFreeAsync(dres, s));
  };
  for (int c = 0; c < P.ncolours; ++c) {
    const int q0 = P.colour_ptr[c], q1 = P.colour_ptr[c + 1];
    if (q1 <= q0) continue;
    // ---- layout of the colour's work space ----
    std::vector<BigRowDev> rows;
    std::vector<std::vector<int>> fpre(q1 - q0);
    int64_t off = 0;
    int nmaxc = 0, maxparts = 1;
    auto take = [&](int64_t elems) {
      const int64_t o = off;
      off += (elems + 63) & ~int64_t(63);
      return o;
    };
    std::vector<CopyTask> gather;
    for (int q = q0; q < q1; ++q) {
      const int i = P.order[q];
      BigRowDev r{};
      r.i = i;
      r.n = P.n[i];
      int mF = 0;
      std::vector<int>& fp = fpre[q - q0];
      for (int f = P.far_ptr[i]; f < P.far_ptr[i + 1]; ++f) {
        fp.push_back(mF);
        mF += width(P.far_blk[f]);
      }
      fp.push_back(mF);
      r.mF = mF;
      const int n = r.n;
      nmaxc = std::max(nmaxc, n);
      // TSQR parts: about 4 chunks of F_i^T per part, at most 64 parts
      int parts = 1;
      while (parts < 64 && (int64_t)parts * 2 * 4 * CH <= mF) parts *= 2;
      r.parts = parts;
      maxparts = std::max(maxparts, parts);
      r.g_off = take((int64_t)std::max(mF, 1) * n);
      r.x_off = take((int64_t)parts * n * n);
      r.v_off = take((int64_t)n * n);
      r.t_off = take((int64_t)n * n);
      r.w2_off = take((int64_t)n * n);
      rows.push_back(r);
      for (int f = P.far_ptr[i], ff = 0; f < P.far_ptr[i + 1]; ++f, ++ff) {
        const int k = P.far_blk[f], w = width(k);
        if (w == 0 || n == 0) continue;
        CopyTask t{};
        if (i < k) {  // stored n_i x n_k: F_ik^T = columns 0..w-1, transposed
          t.src_off = P.far_off[f];
          t.src_ld = P.n[k];
          t.rows = n;
          t.cols = w;
          t.transpose = 1;
        } else {      // stored n_k x n_i: the first w rows are F_ik^T
          t.src_off = P.far_off[f];
          t.src_ld = n;
          t.rows = w;
          t.cols = n;
          t.transpose = 0;
        }
        t.dst_off = r.g_off;
        t.dst_ld = n;
        t.r0 = fp[ff];
        t.c0 = 0;
        gather.push_back(t);
      }
    }
    // Y_p buffers (n x w_p per close target), after the fixed part
    std::vector<std::vector<int64_t>> yoff(q1 - q0);
    for (int q = q0; q < q1; ++q) {
      const int i = P.order[q];
      for (int t = P.close_ptr[i]; t < P.close_ptr[i + 1]; ++t)
        yoff[q - q0].push_back(take((int64_t)P.n[i] * std::max(width(P.close_blk[t]), 1)));
    }
    T* ws = nullptr;
    bcheck(cudaMallocAsync(reinterpret_cast<void**>(&ws), std::max<int64_t>(off, 64) * es, s));
    BigRowDev* drows = nullptr;
    bcheck(cudaMallocAsync(reinterpret_cast<void**>(&drows), rows.size() * sizeof(BigRowDev), s));
    bcheck(cudaMemcpyAsync(drows, rows.data(), rows.size() * sizeof(BigRowDev), cudaMemcpyHostToDevice, s));
    const int nr = static_cast<int>(rows.size());
    // ---- 1-3: compression ----
    mark(0);
    if (!gather.empty()) {
      CopyTask* dt = nullptr;
      bcheck(cudaMallocAsync(reinterpret_cast<void**>(&dt), gather.size() * sizeof(CopyTask), s));
      bcheck(cudaMemcpyAsync(dt, gather.data(), gather.size() * sizeof(CopyTask), cudaMemcpyHostToDevice, s));
      bcheck(launch_copy_tasks(es, es, dt, static_cast<int>(gather.size()), pool, ws, s));
      bcheck(cudaFreeAsync(dt, s));
    }
    mark(1);
    // randomized range finder (learned form in FP32): width 72, doubled for
    // the rows that saturated or failed the probe, up to min(512, 3n/4);
    // accepted rows skip the exact SVD
    std::vector<char> accepted(nr, 0);
    if (args.sketch) {
      std::vector<int> cand, kcur(nr, 0);
      for (int q = 0; q < nr; ++q) {
        const int n = rows[q].n;
        const int kmax = std::min(512, (3 * n) / 4);
        kcur[q] = std::min(kmax, 64 + 8);
        if (rows[q].mF > 0 && kcur[q] >= 8 && kcur[q] < n) cand.push_back(q);
      }
      while (!cand.empty()) {
        run_sketch(cand, kcur, rows, ws, accepted);
        std::vector<int> next;
        for (int q : cand) {
          if (accepted[q]) continue;
          const int kmax = std::min(512, (3 * rows[q].n) / 4);
          const int kn = std::min(kmax, 2 * kcur[q]);
          if (kn > kcur[q]) {
            kcur[q] = kn;
            next.push_back(q);
          }
        }
        cand.swap(next);
      }
    }
    mark(2);
    // exact SVD (TSQR of F_i^T, Jacobi on R) for every other row
    {
      std::vector<BigRowDev> ex;
      int maxp = 1, nmx = 1;
      for (int q = 0; q < nr; ++q)
        if (!accepted[q]) {
          ex.push_back(rows[q]);
          maxp = std::max(maxp, rows[q].parts);
          nmx = std::max(nmx, rows[q].n);
        }
      if (!ex.empty()) {
        const int ne = static_cast<int>(ex.size());
        BigRowDev* dex = nullptr;
        bcheck(cudaMallocAsync(reinterpret_cast<void**>(&dex), ex.size() * sizeof(BigRowDev), s));
        bcheck(cudaMemcpyAsync(dex, ex.data(), ex.size() * sizeof(BigRowDev), cudaMemcpyHostToDevice, s));
        const size_t sm = (size_t)CH * nmx * es;
        if (sm > tsqr_dyn) throw BigFail{cudaErrorInvalidValue};
        g_launches.fetch_add(1, std::memory_order_relaxed);
        tsqr_part_kernel<T, CH><<<dim3(maxp, ne), kTsqrThreads, sm, s>>>(dex, ws);
        bcheck(cudaGetLastError());
        for (int h = 1; h < maxp; h *= 2) {
          g_launches.fetch_add(1, std::memory_order_relaxed);
          tsqr_merge_kernel<T, CH><<<dim3(maxp / (2 * h), ne), kTsqrThreads, sm, s>>>(dex, ws, h);
          bcheck(cudaGetLastError());
        }
        size_t sj = (size_t)((nmx + 3) & ~3) * (es + sizeof(int)) + 64;
        const size_t sxv = sj + (size_t)2 * nmx * nmx * es;
        const int xv = sxv <= jac_dyn ? 1 : 0;
        if (xv) sj = sxv;
        g_launches.fetch_add(1, std::memory_order_relaxed);
        qrcp_precond_kernel<T><<<ne, kQrThreads, (size_t)2 * nmx * es, s>>>(dex, ws);
        bcheck(cudaGetLastError());
        // rows whose X and V do not fit in shared memory: block Jacobi over
        // many CTAs first, then jacobi_kernel only reads the result
        if (!xv) launch_block_jacobi<T>(ex, dex, ws, D, args, jac_dyn, s);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        jacobi_kernel<T><<<ne, kJacThreads, sj, s>>>(dex, ws, D, args, xv, nullptr, xv ? 0 : 1);
        bcheck(cudaGetLastError());
        bcheck(cudaFreeAsync(dex, s));
      }
    }
    mark(3);
    // ranks of the colour (the shapes of everything that follows)
    std::vector<int> rk(P.M);
    bcheck(cudaMemcpyAsync(rk.data(), D.rank, P.M * sizeof(int), cudaMemcpyDeviceToHost, s));
    int hstat = 0;
    bcheck(cudaMemcpyAsync(&hstat, args.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    bcheck(cudaStreamSynchronize(s));
    if (hstat != 0) {
      cudaFreeAsync(ws, s);
      cudaFreeAsync(drows, s);
      return;
    }
    add_phases(3);
    for (int q = q0; q < q1; ++q) rank_h[P.order[q]] = rk[P.order[q]];
    // ---- 4: X = D U, T = U^T X ----
    std::vector<GemmTask> g1, g2;
    for (int q = q0; q < q1; ++q) {
      const BigRowDev& r = rows[q - q0];
      const int i = r.i, n = r.n;
      if (n == 0) continue;
      const T* U = Uf + P.u_off[i];
      GemmTask t{};
      t.A = pool + P.diag_off[i]; t.lda = n; t.ta = 0;
      t.B = U; t.ldb = n; t.tb = 0;
      t.C = ws + r.w2_off; t.ldc = n; t.tc = 0;
      t.Cin = t.C; t.ldcin = n;
      t.M = n; t.N = n; t.K = n; t.alpha = 1.f; t.beta = 0.f;
      g1.push_back(t);
      GemmTask u{};
      u.A = U; u.lda = n; u.ta = 1;
      u.B = ws + r.w2_off; u.ldb = n; u.tb = 0;
      u.C = ws + r.t_off; u.ldc = n; u.tc = 0;
      u.Cin = u.C; u.ldcin = n;
      u.M = n; u.N = n; u.K = n; u.alpha = 1.f; u.beta = 0.f;
      g2.push_back(u);
    }
    mark(3);
    run_gemm(g1, 3);
    run_gemm(g2, 3);
    mark(4);
    // ---- 5: Cholesky of T_nn and L_hat^{-1} ----
    g_launches.fetch_add(1, std::memory_order_relaxed);
    {
      // stage the panel rows in shared memory when they fit
      static size_t ci_dyn = 0;
      if (ci_dyn == 0) {
        int dev = 0, optin = 0;
        bcheck(cudaGetDevice(&dev));
        bcheck(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cudaFuncAttributes fa;
        bcheck(cudaFuncGetAttributes(&fa, cholinv_kernel<T>));
        ci_dyn = static_cast<size_t>(optin) - fa.sharedSizeBytes;
        bcheck(cudaFuncSetAttribute(cholinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ci_dyn));
      }
      int mmax = 1;
      for (int q = 0; q < nr; ++q) mmax = std::max(mmax, rows[q].n);
      const size_t need = (size_t)mmax * (kPW + 1) * es;
      const int stage = need <= ci_dyn ? 1 : 0;
      cholinv_kernel<T><<<nr, kBigThreads, stage ? need : 0, s>>>(drows, ws, D, args, stage);
    }
    bcheck(cudaGetLastError());
    mark(5);
    // ---- 6: W_b, Y_p, far rows ----
    std::vector<GemmTask> g3, g4, g5, g6;
    for (int q = q0; q < q1; ++q) {
      const BigRowDev& rw = rows[q - q0];
      const int i = rw.i, n = rw.n, r = rank_h[i], m = n - r;
      if (n == 0) continue;
      const T* U = Uf + P.u_off[i];
      const T* Li = Lf + P.l_off[i];
      T* Wb = Wf + P.w_off[i];
      if (m > 0 && r > 0) {
        GemmTask t{};  // W_b = L_hat^{-1} T[r:, :r]
        t.A = Li; t.lda = m; t.ta = 0;
        t.B = ws + rw.t_off + (int64_t)r * n; t.ldb = n; t.tb = 0;
        t.C = Wb; t.ldc = r; t.Cin = Wb; t.ldcin = r;
        t.M = m; t.N = r; t.K = m; t.alpha = 1.f; t.beta = 0.f;
        g3.push_back(t);
      }
      // close targets: Y_p = U^T C_ip (n x w_p)
      int64_t colst = n;
      for (int tt = P.close_ptr[i], ti = 0; tt < P.close_ptr[i + 1]; ++tt, ++ti) {
        const int p = P.close_blk[tt], w = width(p);
        const int64_t ycol = colst;
        colst += P.n[p];
        (void)ycol;
        if (w == 0) continue;
        const PairView pv = pair_view(P, i, p);
        GemmTask t{};
        t.A = U; t.lda = n; t.ta = 1;
        t.B = pool + pv.off; t.ldb = pv.ld; t.tb = pv.trans;
        t.C = ws + yoff[q - q0][ti]; t.ldc = w; t.Cin = t.C; t.ldcin = w;
        t.M = n; t.N = w; t.K = n; t.alpha = 1.f; t.beta = 0.f;
        g3.push_back(t);
      }
      // far rows: F_ik <- U_b^T F_ik (the rows r.. are E_i and are dropped)
      if (r > 0) {
        const std::vector<int>& fp = fpre[q - q0];
        for (int f = P.far_ptr[i], ff = 0; f < P.far_ptr[i + 1]; ++f, ++ff) {
          const int k = P.far_blk[f], w = width(k);
          if (w == 0) continue;
          const PairView pv = pair_view(P, i, k);
          GemmTask t{};
          t.A = U; t.lda = n; t.ta = 1;
          t.B = ws + rw.g_off + (int64_t)fp[ff] * n; t.ldb = n; t.tb = 1;
          t.C = pool + pv.off; t.ldc = pv.ld; t.tc = pv.trans;
          t.Cin = t.C; t.ldcin = pv.ld; t.tcin = pv.trans;
          t.M = r; t.N = w; t.K = n; t.alpha = 1.f; t.beta = 0.f;
          g3.push_back(t);
        }
      }
    }
    run_gemm(g3, 3);
    mark(6);
    // ---- 7: D_i <- T[:r, :r] - W_b^T W_b;  W_p = L_hat^{-1} Y_p[r:] ----
    for (int q = q0; q < q1; ++q) {
      const BigRowDev& rw = rows[q - q0];
      const int i = rw.i, n = rw.n, r = rank_h[i], m = n - r;
      if (n == 0 || r == 0) continue;
      const T* Li = Lf + P.l_off[i];
      T* Wb = Wf + P.w_off[i];
      GemmTask t{};
      t.A = Wb; t.lda = r; t.ta = 1;
      t.B = Wb; t.ldb = r; t.tb = 0;
      t.Cin = ws + rw.t_off; t.ldcin = n;
      t.C = pool + P.diag_off[i]; t.ldc = n;
      t.M = r; t.N = r; t.K = m; t.alpha = -1.f; t.beta = 1.f;
      g4.push_back(t);
      (void)Li;
    }
    for (int q = q0; q < q1; ++q) {
      const BigRowDev& rw = rows[q - q0];
      const int i = rw.i, n = rw.n, r = rank_h[i], m = n - r;
      if (n == 0 || m == 0) continue;
      const T* Li = Lf + P.l_off[i];
      int64_t colst = n;
      for (int tt = P.close_ptr[i], ti = 0; tt < P.close_ptr[i + 1]; ++tt, ++ti) {
        const int p = P.close_blk[tt], w = width(p);
        T* Wp = Wf + P.w_off[i] + (int64_t)n * colst;
        colst += P.n[p];
        if (w == 0) continue;
        GemmTask t{};
        t.A = Li; t.lda = m; t.ta = 0;
        t.B = ws + yoff[q - q0][ti] + (int64_t)r * w; t.ldb = w; t.tb = 0;
        t.C = Wp; t.ldc = w; t.Cin = Wp; t.ldcin = w;
        t.M = m; t.N = w; t.K = m; t.alpha = 1.f; t.beta = 0.f;
        g4.push_back(t);
      }
    }
    // D_i with r == 0: the block is eliminated whole (nothing kept)
    run_gemm(g4, 3);
    mark(7);
    // ---- 8: kept close rows and the Schur update ----
    for (int q = q0; q < q1; ++q) {
      const BigRowDev& rw = rows[q - q0];
      const int i = rw.i, n = rw.n, r = rank_h[i], m = n - r;
      if (n == 0) continue;
      const T* Wb = Wf + P.w_off[i];
      std::vector<int> tp, tw;
      std::vector<const T*> tW;
      int64_t colst = n;
      for (int tt = P.close_ptr[i], ti = 0; tt < P.close_ptr[i + 1]; ++tt, ++ti) {
        const int p = P.close_blk[tt], w = width(p);
        const T* Wp = Wf + P.w_off[i] + (int64_t)n * colst;
        colst += P.n[p];
        if (w == 0) continue;
        if (r > 0) {  // kept rows of (i, p): Y_p[:r] - W_b^T W_p
          const PairView pv = pair_view(P, i, p);
          GemmTask t{};
          t.A = Wb; t.lda = r; t.ta = 1;
          t.B = Wp; t.ldb = w; t.tb = 0;
          t.Cin = ws + yoff[q - q0][ti]; t.ldcin = w;
          t.C = pool + pv.off; t.ldc = pv.ld; t.tc = pv.trans;
          t.M = r; t.N = w; t.K = m; t.alpha = -1.f; t.beta = 1.f;
          if (m == 0) {  // nothing eliminated: the kept rows are Y_p[:r]
            t.K = 0;
          }
          g5.push_back(t);
        }
        tp.push_back(p);
        tw.push_back(w);
        tW.push_back(Wp);
      }
      if (m == 0) continue;
      for (size_t a2 = 0; a2 < tp.size(); ++a2)
        for (size_t b2 = a2; b2 < tp.size(); ++b2) {
          const int p = tp[a2], qq = tp[b2];
          const PairView pv = pair_view(P, p, qq);
          GemmTask t{};
          t.A = tW[a2]; t.lda = tw[a2]; t.ta = 1;
          t.B = tW[b2]; t.ldb = tw[b2]; t.tb = 0;
          t.C = pool + pv.off; t.ldc = pv.ld; t.tc = pv.trans;
          t.Cin = t.C; t.ldcin = pv.ld; t.tcin = pv.trans;
          t.M = tw[a2]; t.N = tw[b2]; t.K = m; t.alpha = -1.f; t.beta = 1.f;
          t.atomic = D.accumulate;   // rows of a distance-1 colour may share (p, q)
          g6.push_back(t);
        }
    }
    run_gemm(g5, 3);
    run_gemm(g6, args.engine == 2 ? 1 : 3);
    mark(8);
    for (int q = q0; q < q1; ++q) done[P.order[q]] = 1;
    bcheck(cudaFreeAsync(ws, s));
    bcheck(cudaFreeAsync(drows, s));
    int hs2[2] = {0, 0};
    bcheck(cudaMemcpyAsync(&hs2[0], args.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    bcheck(cudaMemcpyAsync(&hs2[1], args.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    bcheck(cudaStreamSynchronize(s));
    if (hs2[1] != 0) throw BigFail{cudaErrorLaunchTimeout};
    if (hs2[0] != 0) return;
    for (int k = 3; k < 8; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) == cudaSuccess && args.phase_ms) args.phase_ms[k] += ms;
    }
  }
}

}  // namespace

cudaError_t launch_gemm_cuda(int esize, const std::vector<GemmTask>& tasks, cudaStream_t s) {
  return esize == 8 ? launch_gemm_t<double>(tasks, s) : launch_gemm_t<float>(tasks, s);
}

bool level_needs_big_rows(const LevelPlan& P) {
  if (P.nmax > kNMax) return true;
  for (int i = 0; i < P.M; ++i) {
    if (1 + P.close_ptr[i + 1] - P.close_ptr[i] > 32) return true;
    if (P.far_ptr[i + 1] - P.far_ptr[i] > 128) return true;
  }
  return false;
}

// The SVD steps of a large row on one n x n R (tests): the pivoted-QR
// preconditioner, then block Jacobi with column blocks of B; X and V copied
// out (column-major), the sweeps run into *sweeps.
template <typename T>
void debug_svd_t(int B, int n, const void* R, const void* Dm, double tol, void* X, void* V, int* sweeps,
                 cudaStream_t s) {
  const int64_t nn = (int64_t)n * n;
  T* ws = nullptr;
  void* aux = nullptr;
  struct Free {   // the buffers go back to the pool on every exit
    T*& w;
    void*& x;
    cudaStream_t st;
    ~Free() {
      if (w) cudaFreeAsync(w, st);
      if (x) cudaFreeAsync(x, st);
    }
  } guard{ws, aux, s};
  bcheck(cudaMallocAsync(reinterpret_cast<void**>(&ws), 3 * nn * sizeof(T), s));
  bcheck(cudaMallocAsync(&aux, sizeof(BigRowDev) + sizeof(int64_t) + (kStatusWords + kStatsWords) * sizeof(int), s));
  BigRowDev* drow = static_cast<BigRowDev*>(aux);
  int64_t* ddiag = reinterpret_cast<int64_t*>(static_cast<char*>(aux) + sizeof(BigRowDev));
  int* dstat = reinterpret_cast<int*>(ddiag + 1);
  BigRowDev r{};
  r.i = 0;
  r.n = n;
  r.mF = 1;
  r.parts = 1;
  r.x_off = 0;
  r.v_off = nn;
  r.t_off = 2 * nn;
  const int64_t zero = 0;
  bcheck(cudaMemcpyAsync(drow, &r, sizeof(r), cudaMemcpyHostToDevice, s));
  bcheck(cudaMemcpyAsync(ddiag, &zero, sizeof(zero), cudaMemcpyHostToDevice, s));
  bcheck(cudaMemsetAsync(dstat, 0, (kStatusWords + kStatsWords) * sizeof(int), s));
  bcheck(cudaMemcpyAsync(ws, R, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
  LevelDev D{};
  D.pool = const_cast<void*>(Dm);
  D.diag_off = ddiag;
  BigLevelArgs a{};
  a.level = 0;
  a.tol = tol;
  a.tol_mode = CE_TOL_REL;
  a.status = dstat;
  a.stats = dstat + kStatusWords;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  qrcp_precond_kernel<T><<<1, kQrThreads, (size_t)2 * n * sizeof(T), s>>>(drow, ws);
  bcheck(cudaGetLastError());
  const std::vector<BigRowDev> rv{r};
  const size_t sm = (size_t)4 * B * n * sizeof(T) + 256;
  int dev = 0, optin = 0;
  bcheck(cudaGetDevice(&dev));
  bcheck(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (sm + 2048 > (size_t)optin) throw BigFail{cudaErrorInvalidValue};
  if (B == 32) launch_block_jacobi_b<T, 32>(rv, drow, ws, D, a, sm, s);
  else if (B == 16) launch_block_jacobi_b<T, 16>(rv, drow, ws, D, a, sm, s);
  else if (B == 8) launch_block_jacobi_b<T, 8>(rv, drow, ws, D, a, sm, s);
  else launch_block_jacobi_b<T, 4>(rv, drow, ws, D, a, sm, s);
  bcheck(cudaMemcpyAsync(X, ws + 2 * nn, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
  bcheck(cudaMemcpyAsync(V, ws + nn, nn * sizeof(T), cudaMemcpyDeviceToDevice, s));
  int hs[kStatsWords];
  bcheck(cudaMemcpyAsync(hs, dstat + kStatusWords, sizeof(hs), cudaMemcpyDeviceToHost, s));
  bcheck(cudaStreamSynchronize(s));
  if (sweeps) *sweeps = hs[48];
}

cudaError_t debug_svd(int esize, int B, int n, const void* R, const void* Dm, double tol, void* X, void* V,
                      int* sweeps, cudaStream_t s) {
  try {
    if (esize == 8)
      debug_svd_t<double>(B, n, R, Dm, tol, X, V, sweeps, s);
    else
      debug_svd_t<float>(B, n, R, Dm, tol, X, V, sweeps, s);
  } catch (const BigFail& f) {
    return f.e;
  }
  return cudaSuccess;
}

cudaError_t run_big_level(int esize, LevelStore& st, int level, double tol, int tol_mode, int* status, int* stats,
                          int engine, double* phase_ms, int sketch, unsigned long long seed, cudaStream_t s) {
  int* tc_err = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tc_err), sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(tc_err, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(tc_err, s);
    return e;
  }
  BigLevelArgs a{level, tol, tol_mode, status, stats, engine, tc_err, phase_ms,
                 (esize == 4 && sketch && tol_mode != CE_TOL_FIXED) ? 1 : 0, seed};
  try {
    std::vector<int> rank_h;
    if (esize == 8)
      run_big_level_t<double>(st, s, a, rank_h);
    else
      run_big_level_t<float>(st, s, a, rank_h);
  } catch (const BigFail& f) {
    e = f.e;
  }
  cudaFreeAsync(tc_err, s);
  return e;
}

cudaError_t launch_apply_big(int esize, const LevelDev& L, const LevelPlan& P, double* vec, int forward,
                             cudaStream_t s) {
  const size_t sm = (size_t)3 * std::max(P.nmax, 1) * esize;
  for (int cc = 0; cc < P.ncolours; ++cc) {
    const int c = forward ? cc : P.ncolours - 1 - cc;
    const int q0 = P.colour_ptr[c], cnt = P.colour_ptr[c + 1] - q0;
    if (cnt <= 0) continue;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (esize == 8) {
      if (forward)
        apply_big_kernel<double, true><<<cnt, kBigThreads, sm, s>>>(L, q0, vec);
      else
        apply_big_kernel<double, false><<<cnt, kBigThreads, sm, s>>>(L, q0, vec);
    } else {
      if (forward)
        apply_big_kernel<float, true><<<cnt, kBigThreads, sm, s>>>(L, q0, vec);
      else
        apply_big_kernel<float, false><<<cnt, kBigThreads, sm, s>>>(L, q0, vec);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ce
