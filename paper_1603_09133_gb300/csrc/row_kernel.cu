// ce_row_kernel: Algorithm 2 for the block rows of one level, one CTA per
// block row at a time (one iteration of its loop per row; a persistent
// launch per level, see below).
//
//   0. ||D_i||_F (rounding floor of the truncation threshold)
//   A. compression (Section 2.2, eq. rreav): R factor of F_i^T.  Rows of F_i^T
//      are cut into chunks of 32; warp w reduces chunks w, w+QW, ... into its
//      own triangular R_w with warp-synchronous Householder steps (no CTA
//      barrier per column), then the R_w are merged pairwise (tree).  F_i F_i^T
//      = R^T R, so F_i and R^T share their left singular vectors.
//   B. one-sided (Hestenes) Jacobi on the columns of R: R V = U' S gives
//      U_i = V and sigma = S (descending); half a warp per column pair, so all
//      pairs of a round-robin round run at once; r_i = #{sigma_k > tau_i},
//      tau_i from the tolerance (CE(eps)) or just below sigma_r (CE(r), the
//      fixed-rank strategy of the Section 2.2 remark).
//   C. transform and elimination (eq. q, eq. sm_L): T = U^T D U, Cholesky of
//      the non-basis block T_nn = L_hat L_hat^T, L_hat^{-1} formed once so every
//      W = L_hat^{-1} S is a GEMM; close rows <- U^T C (kept rows minus the
//      basis Schur term), far rows <- U_b^T F (rows r.. are E_i, dropped), and
//      the Schur update A(p, q) -= W_p^T W_q between close targets.
// L. (learned ranks) an MLP-predicted width, a randomized range finder and an
//    a-posteriori check replace A-B for the rows that pass it.
// Blocks of one colour have disjoint closed neighbourhoods (distance-2
// colouring); a row waits for the lower-colour rows within distance 2, so
// rows running at the same time touch disjoint block pairs.
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>

#include "kernels.h"
#include "mlp_infer.cuh"
#include "rng.cuh"

namespace ce {

namespace {

constexpr int kMaxWarps = 16;
constexpr int kChunk = 32;       // rows of F_i^T per warp Householder pass
constexpr int kMaxSweeps = 40;   // Jacobi sweep cap (bounded loop)
constexpr int kMaxTargets = 32;
constexpr int kMaxFar = 128;
constexpr double kTieRel = 1e-3; // CE(r): singular values this close to sigma_r stay with it

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

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename T>
__device__ __forceinline__ T half_sum(T v) {  // sum over the 16 lanes of a half warp
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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

__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }

// Householder reflector of the column x = [x0; c] (c held as c_lo, c_hi by
// each lane for rows lane and lane + 32), unit-leading form H = I - tau v v^T,
// v = [1; sc c], beta = -sign(x0) ||x||.  Columns whose largest entry is
// subnormal are rounding noise and give tau = 0.  Returns false for tau = 0.
template <typename T>
__device__ __forceinline__ bool reflector(T x0, T c_lo, T c_hi, T& beta, T& tau, T& sc) {
  T amax = warp_max(fmax(fabs(c_lo), fabs(c_hi)));
  if (!(amax >= Tiny<T>::v)) return false;
  const T ia = fast_rcp(amax);
  const T xl = c_lo * ia, xh = c_hi * ia;
  const T s = warp_sum(xl * xl + xh * xh);
  const T a = fmax(amax, fabs(x0));
  const T ra = fast_rcp(a);
  const T x0a = x0 * ra, ca = amax * ra;
  const T nrm = a * sqrt(x0a * x0a + s * ca * ca);
  beta = (x0 >= T(0)) ? -nrm : nrm;
  tau = (beta - x0) * fast_rcp(beta);
  sc = fast_rcp(x0 - beta);
  return true;
}

// Warp-synchronous QR update of [R; C]: R n x n upper triangular, C rows x n
// (rows <= 32).  After the call R is the triangular factor of the stack.
template <typename T>
__device__ void warp_qr_stack(T* R, T* C, T* vb, int n, int rows, int LD) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {
    const T x = (lane < rows) ? C[lane * LD + j] : T(0);
    T beta, tau, sc;
    if (!reflector(R[j * LD + j], x, T(0), beta, tau, sc)) continue;
    vb[lane] = x * sc;
    __syncwarp();
    if (lane == 0) R[j * LD + j] = beta;
    for (int l = j + 1 + lane; l < n; l += 32) {
      T d0 = R[j * LD + l], d1 = 0, d2 = 0, d3 = 0;
      int q = 0;
#pragma unroll 2
      for (; q + 3 < rows; q += 4) {
        d0 += vb[q] * C[q * LD + l];
        d1 += vb[q + 1] * C[(q + 1) * LD + l];
        d2 += vb[q + 2] * C[(q + 2) * LD + l];
        d3 += vb[q + 3] * C[(q + 3) * LD + l];
      }
      for (; q < rows; ++q) d0 += vb[q] * C[q * LD + l];
      const T d = ((d0 + d1) + (d2 + d3)) * tau;
      R[j * LD + l] -= d;
#pragma unroll 8
      for (q = 0; q < rows; ++q) C[q * LD + l] -= d * vb[q];
    }
    __syncwarp();
  }
}

// Warp-synchronous merge of two triangular factors: Ra <- R factor of
// [Ra; Rb] (both n x n upper triangular; Rb is destroyed).
template <typename T>
__device__ void warp_qr_merge(T* Ra, T* Rb, T* vb, int n, int LD) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {
    const T xl = (lane <= j) ? Rb[lane * LD + j] : T(0);
    const T xh = (lane + 32 <= j) ? Rb[(lane + 32) * LD + j] : T(0);
    T beta, tau, sc;
    if (!reflector(Ra[j * LD + j], xl, xh, beta, tau, sc)) continue;
    vb[lane] = xl * sc;
    vb[lane + 32] = xh * sc;
    __syncwarp();
    if (lane == 0) Ra[j * LD + j] = beta;
    const int rows = j + 1;
    for (int l = j + 1 + lane; l < n; l += 32) {
      T d0 = Ra[j * LD + l], d1 = 0, d2 = 0, d3 = 0;
      int q = 0;
#pragma unroll 2
      for (; q + 3 < rows; q += 4) {
        d0 += vb[q] * Rb[q * LD + l];
        d1 += vb[q + 1] * Rb[(q + 1) * LD + l];
        d2 += vb[q + 2] * Rb[(q + 2) * LD + l];
        d3 += vb[q + 3] * Rb[(q + 3) * LD + l];
      }
      for (; q < rows; ++q) d0 += vb[q] * Rb[q * LD + l];
      const T d = ((d0 + d1) + (d2 + d3)) * tau;
      Ra[j * LD + l] -= d;
#pragma unroll 8
      for (q = 0; q < rows; ++q) Rb[q * LD + l] -= d * vb[q];
    }
    __syncwarp();
  }
}

// Rows g0 .. g0+rows-1 of F_i^T (rows <= 32) -> C (row-major, ldc) by one warp.
// Lane q first finds the far block and the offset of row g0 + q, so the
// element loads that follow are independent of each other.
template <typename T>
__device__ __forceinline__ void warp_load_far_rows(T* C, int ldc, const T* pool, const LevelDev& L, int i,
                                                   int n, int g0, int rows, int nf, const int* fpre,
                                                   const int* fk, const int64_t* foff, int* wf, int* wq) {
  const int lane = threadIdx.x & 31;
  if (lane < rows) {
    const int g = g0 + lane;
    int lo = 0, hi = nf - 1;          // last f with fpre[f] <= g (skips empty blocks)
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (fpre[mid] <= g) lo = mid; else hi = mid - 1;
    }
    wf[lane] = lo;
    wq[lane] = g - fpre[lo];
  }
  __syncwarp();
  for (int e = lane; e < rows * n; e += 32) {
    const int q = e / n, a = e - q * n;
    const int f = wf[q], k = fk[f], qq = wq[q];
    const T* Xg = pool + foff[f];
    C[q * ldc + a] = (i < k) ? Xg[(int64_t)a * L.n[k] + qq] : Xg[(int64_t)qq * n + a];
  }
  __syncwarp();
}

// out(a, b) op= sum_k A(a, k) B(k, b), a < M, b < N, k < K; 2 x 2 register
// tiles over the CTA.  store(a, b, v) receives the sum.
template <typename T, int NT, typename FA, typename FB, typename FS>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, FA A, FB B, FS store) {
  const int tm = (M + 1) >> 1, tn = (N + 1) >> 1;
  for (int t = threadIdx.x; t < tm * tn; t += NT) {
    const int a0 = (t / tn) * 2, b0 = (t % tn) * 2;
    const bool a1 = a0 + 1 < M, b1 = b0 + 1 < N;
    T c00 = 0, c01 = 0, c10 = 0, c11 = 0;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const T x0 = A(a0, k), x1 = a1 ? A(a0 + 1, k) : T(0);
      const T y0 = B(k, b0), y1 = b1 ? B(k, b0 + 1) : T(0);
      c00 += x0 * y0;
      c01 += x0 * y1;
      c10 += x1 * y0;
      c11 += x1 * y1;
    }
    store(a0, b0, c00);
    if (b1) store(a0, b0 + 1, c01);
    if (a1) store(a0 + 1, b0, c10);
    if (a1 && b1) store(a0 + 1, b0 + 1, c11);
  }
}

// ---- tensor cores (FP32 form): mma.sync m16n8k8 TF32 with FP32 accumulate.
// Each FP32 operand is split x = hi + lo into two TF32 numbers and the
// product is accumulated as lo*hi + hi*lo + hi*hi ("3xTF32"), which keeps the
// rounding error at the level of FP32 arithmetic (the dropped lo*lo term is
// about 2^-22 of the product).  Fragment layout of m16n8k8 (g = lane / 4,
// q = lane % 4): A holds (g, q), (g+8, q), (g, q+4), (g+8, q+4); B holds
// (q, g), (q+4, g); C holds (g, 2q), (g, 2q+1), (g+8, 2q), (g+8, 2q+1).
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The 16 x 8 tile of C = A B (M x N, inner K) at (r0, c0), by one warp on the
// tensor cores; store(a, b, v) is called once per element of the tile.
template <class FA, class FB, class FS>
__device__ __forceinline__ void warp_tile_tc(int M, int N, int K, FA A, FB B, FS store, int r0, int c0) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  {
    const int ra = r0 + g, rb = r0 + g + 8, cb = c0 + g;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += 8) {
      const int ka = k0 + q, kb = k0 + q + 4;
      float af[4], bf[2];
      af[0] = (ra < M && ka < K) ? A(ra, ka) : 0.f;
      af[1] = (rb < M && ka < K) ? A(rb, ka) : 0.f;
      af[2] = (ra < M && kb < K) ? A(ra, kb) : 0.f;
      af[3] = (rb < M && kb < K) ? A(rb, kb) : 0.f;
      bf[0] = (ka < K && cb < N) ? B(ka, cb) : 0.f;
      bf[1] = (kb < K && cb < N) ? B(kb, cb) : 0.f;
      uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ah[u] = to_tf32(af[u]);
        al[u] = to_tf32(af[u] - __uint_as_float(ah[u]));
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        bh[u] = to_tf32(bf[u]);
        bl[u] = to_tf32(bf[u] - __uint_as_float(bh[u]));
      }
      mma_tf32(c, al, bh);
      mma_tf32(c, ah, bl);
      mma_tf32(c, ah, bh);
    }
    const int cc = c0 + 2 * q;
    if (ra < M && cc < N) store(ra, cc, c[0]);
    if (ra < M && cc + 1 < N) store(ra, cc + 1, c[1]);
    if (rb < M && cc < N) store(rb, cc, c[2]);
    if (rb < M && cc + 1 < N) store(rb, cc + 1, c[3]);
  }
}

// C = A B (M x N, inner K) on the tensor cores, one 16 x 8 tile of C per warp
// at a time; store(a, b, v) is called once per element, like cta_gemm.
template <int NT, class FA, class FB, class FS>
__device__ __forceinline__ void cta_gemm_tc(int M, int N, int K, FA A, FB B, FS store) {
  const int warp = threadIdx.x >> 5;
  const int tn = (N + 7) >> 3, tiles = ((M + 15) >> 4) * tn;
  for (int t = warp; t < tiles; t += NT / 32) warp_tile_tc(M, N, K, A, B, store, (t / tn) * 16, (t % tn) * 8);
}

// FP32 form: tensor cores when `tc` (levels whose blocks exceed 32 rows; on
// the level-1 blocks of 32 rows the 16 x 8 x 8 tiles carry too much padding
// and the CUDA cores measured faster); FP64 form: FP64 on the CUDA cores
template <typename T, int NT, class FA, class FB, class FS>
__device__ __forceinline__ void cta_mm(bool tc, int M, int N, int K, FA A, FB B, FS store) {
  if constexpr (std::is_same<T, float>::value) {
    if (tc) {
      cta_gemm_tc<NT>(M, N, K, A, B, store);
      return;
    }
  }
  cta_gemm<T, NT>(M, N, K, A, B, store);
}

// n x w tile of the pair (i, k) seen from row i -> sm (row-major, LD); the
// pair is stored once as (min, max)
template <typename T, int NT>
__device__ void load_row_tile(T* sm, const T* X, int i, int k, int n, int nk, int w, int LD) {
  if (i < k) {  // stored n x nk
    for (int e = threadIdx.x; e < n * w; e += NT) {
      int a = e / w, b = e - a * w;
      sm[a * LD + b] = X[(int64_t)a * nk + b];
    }
  } else {      // stored nk x n, tile = X[0:w, :]^T
    for (int e = threadIdx.x; e < n * w; e += NT) {
      int b = e / n, a = e - b * n;
      sm[a * LD + b] = X[(int64_t)b * n + a];
    }
  }
}

template <typename T, int NT>
__device__ void store_row_tile(const T* sm, T* X, int i, int k, int n, int nk, int rows, int w, int LD) {
  if (i < k) {
    for (int e = threadIdx.x; e < rows * w; e += NT) {
      int a = e / w, b = e - a * w;
      X[(int64_t)a * nk + b] = sm[a * LD + b];
    }
  } else {
    for (int e = threadIdx.x; e < rows * w; e += NT) {
      int b = e / rows, a = e - b * rows;
      X[(int64_t)b * n + a] = sm[a * LD + b];
    }
  }
}

// One block row i of the level (Algorithm 2 for one i), by the whole CTA.
template <typename T, int NT>
__device__ __forceinline__ void row_block(const LevelDev& L, const int i, int level, double tol, int tol_mode,
                                          int* status, int nmax, int LD, int QW, const LearnedArgs& la,
                                          long long& t_row) {
  constexpr int kWarpsNT = NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NL = nmax * LD;
  T* U = reinterpret_cast<T*>(smem_raw);            // persistent: U_i
  T* sig = U + NL;                                   // nmax
  T* sig_tmp = sig + nmax;                           // nmax
  T* un = sig_tmp + nmax;                            // union region
  const int per_warp = NL + kChunk * LD + 64;        // phase A: R_w, C_w, v_w
  T* X = un;                                         // phase B: R (= R_0), V
  T* V = un + NL;
  T* Tm = un;                                        // phase C: T, L_hat^{-1}, Y, tile
  T* Li = un + NL;
  T* Y = un + 2 * NL;
  T* Xt = un + 3 * NL;

  __shared__ double s_red[kMaxWarps];
  __shared__ int s_flag;
  __shared__ T s_skip2;
  __shared__ int s_pos[64];
  __shared__ int s_colst[kMaxTargets], s_tgt[kMaxTargets], s_w[kMaxTargets];
  __shared__ int s_fw[kMaxFar + 1], s_fpre[kMaxFar + 1], s_fk[kMaxFar];
  __shared__ int64_t s_foff[kMaxFar];
  __shared__ float s_bn2[kMaxFar + kMaxTargets];   // block norms^2 (features)
  __shared__ float s_x[kMlpFeatures], s_h[kMlpHidden];
  __shared__ int s_k, s_rowf[kChunk], s_rowq[kChunk];
  __shared__ int s_wf[kMaxWarps][kChunk], s_wq[kMaxWarps][kChunk];
  __shared__ T s_tq[64], s_probe[2];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = L.n[i];
  const int ci = L.colour[i];
  const bool tc = nmax > 32;
  // phase timer (thread 0; the marks sit where every thread passes)
  auto mark = [&](int ph) {
    if (L.prof && tid == 0 && level < 16) {
      const long long t = clock64();
      atomicAdd(L.prof + level * kProfSlots + ph, static_cast<unsigned long long>(t - t_row));
      t_row = t;
    }
  };
  T* pool = reinterpret_cast<T*>(L.pool);
  if (n == 0) {
    if (tid == 0) {
      L.rank[i] = 0;
      L.tau[i] = 0.0;
    }
    return;
  }
  const int f0 = L.far_ptr[i], nf = L.far_ptr[i + 1] - f0;
  if (nf > kMaxFar) {
    if (tid == 0) set_status(status, CE_ERR_LIMIT, level, i, 7, nf);
    return;
  }

  // ---------------- 0. ||D_i||_F and the far-row layout -------------------
  T* Dg = pool + L.diag_off[i];
  {
    double ss = 0.0;
    for (int e = tid; e < n * n; e += NT) {
      double v = static_cast<double>(Dg[e]);
      ss += v * v;
    }
    ss = warp_sum(ss);
    if (lane == 0) s_red[warp] = ss;
  }
  for (int f = tid; f < nf; f += NT) {
    const int k = L.far_blk[f0 + f];
    s_fk[f] = k;
    s_fw[f] = width_of(L, k, ci);
    s_foff[f] = L.far_off[f0 + f];
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int f = 0; f < nf; ++f) {
      s_fpre[f] = acc;
      acc += s_fw[f];
    }
    s_fpre[nf] = acc;
  }
  __syncthreads();
  const int mF = s_fpre[nf];
  mark(1);

  int r = 0;
  double tau = 0.0;
  bool have_u = false;
  double dn2_all = 0.0;
  for (int w = 0; w < kWarpsNT; ++w) dn2_all += s_red[w];
  const double floor_all = static_cast<double>(Eps<T>::v) * sqrt(dn2_all);

  // ---------------- L. learned rank + randomized range finder --------------
  // Features -> FP16 MLP -> r_hat; sketch width k = r_hat + p.  Y = F [O | w1 w2]
  // with Gaussian O (n x k) and two probe columns; Q = orth(Y[:, :k])
  // (Householder, the probes carried along give ||(I - Q Q^T) F w||); TSQR
  // of the rows of F^T Q and Jacobi on the k x k factor give the singular
  // values and vectors of Q^T F.  Accepted when the sketch is not saturated
  // (r < k) and the probe estimate of the out-of-sketch residual is at most
  // tau / 2; otherwise the exact phases A-B run.
  if (mF > 0 && (la.model != nullptr || la.record)) {
    const int cc0 = L.close_ptr[i], nclose = L.close_ptr[i + 1] - cc0;
    for (int f = warp; f < nf + nclose; f += kWarpsNT) {
      int k, w;
      const T* Xg;
      if (f < nf) {
        k = s_fk[f];
        w = s_fw[f];
        Xg = pool + s_foff[f];
      } else {
        k = L.close_blk[cc0 + f - nf];
        w = width_of(L, k, ci);
        Xg = pool + L.close_off[cc0 + f - nf];
      }
      const int nk = L.n[k];
      float ss = 0.f;
      for (int e = lane; e < n * w; e += 32) {
        const int a = e / w, b = e - a * w;
        const float v = static_cast<float>((i < k) ? Xg[(int64_t)a * nk + b] : Xg[(int64_t)b * n + a]);
        ss += v * v;
      }
      ss = warp_sum(ss);
      if (lane == 0) s_bn2[f] = ss;
    }
    __syncthreads();
    if (tid == 0) {
      float cn2 = 0.f, fn2 = 0.f, fmax = 0.f, fsum = 0.f;
      int nfl = 0;
      for (int f = 0; f < nf; ++f)
        if (s_fw[f] > 0) {
          const float v = sqrtf(s_bn2[f]);
          fn2 += s_bn2[f];
          fmax = fmaxf(fmax, v);
          fsum += v;
          ++nfl;
        }
      for (int c = 0; c < nclose; ++c) cn2 += s_bn2[nf + c];
      const float dn = static_cast<float>(sqrt(dn2_all)), fn = sqrtf(fn2), cn = sqrtf(cn2);
      const float d = dn > 0.f ? dn : 1.f, fv = fn > 0.f ? fn : 1.f;
      auto lg = [](float x) { return log10f(fmaxf(x, 1e-30f)) / 10.f; };
      s_x[0] = level / 4.f;
      s_x[1] = n / 64.f;
      s_x[2] = lg(cn / d);
      s_x[3] = lg(fn / d);
      s_x[4] = lg(fmax / fv);
      s_x[5] = lg((nfl ? fsum / nfl : 0.f) / fv);
      s_x[6] = nclose / 8.f;
      s_x[7] = nfl / 16.f;
      s_x[8] = (level > 0 ? float(n) / la.J : 0.f) / 32.f;
      s_x[9] = mF / (16.f * n);
      s_x[10] = -log10f(fmaxf(static_cast<float>(tol), 1e-30f)) / 8.f;
    }
    __syncthreads();
    if (L.feat != nullptr && tid < kMlpFeatures) L.feat[(int64_t)i * kMlpFeatures + tid] = s_x[tid];
    if (la.model != nullptr) {
    if (warp == 0) {
      const float yh = mlp_infer_warp(la.model, s_x, s_h);
      if (lane == 0) {
        int rh = static_cast<int>(ceilf(yh * n));
        rh = max(1, min(n, rh));
        s_k = min(n, rh + la.oversample);
      }
    }
    __syncthreads();
    mark(2);
    const int k = s_k;
    const int kk = k + 2;
    const bool lvl_ok = level < 16 && la.stats != nullptr;
    const int UNE = max(QW * per_warp, 4 * NL);          // union size (elements)
    const int LK = (k & 1) ? k : k + 1;                  // leading dimension of k-wide buffers
    const int pwl = k * LK + kChunk * LD + kChunk * LK + 64;  // per warp: R, rows of F^T, projected rows
    const int qwl = min(kWarpsNT, (UNE - NL) / pwl);
    if (4 * k <= 3 * n && qwl >= 1 && kk <= LD && k <= 2 * kChunk && NL + 2 * kChunk * LD <= UNE) {
      T* Q = un;                 // n x kk (columns k, k+1: probes)
      T* Cs = un + NL;           // 32 x LD rows of F^T
      T* Om = Cs + kChunk * LD;  // 32 x kk
      for (int e = tid; e < n * LD; e += NT) Q[e] = T(0);
      __syncthreads();
      for (int g0 = 0; g0 < mF; g0 += kChunk) {
        const int rows = min(kChunk, mF - g0);
        if (tid < rows) {
          const int g = g0 + tid;
          int f = 0;
          while (f + 1 < nf && s_fpre[f + 1] <= g) ++f;
          s_rowf[tid] = f;
          s_rowq[tid] = g - s_fpre[f];
        }
        for (int e = tid; e < rows * kk; e += NT) {
          const int q = e / kk, c = e - q * kk;
          Om[q * kk + c] = static_cast<T>(gauss_from_key(sketch_key(la.seed, level, i, g0 + q, c)));
        }
        __syncthreads();
        for (int e = tid; e < rows * n; e += NT) {
          const int q = e / n, a = e - q * n;
          const int f = s_rowf[q], k2 = s_fk[f], qq = s_rowq[q];
          const T* Xg = pool + s_foff[f];
          Cs[q * LD + a] = (i < k2) ? Xg[(int64_t)a * L.n[k2] + qq] : Xg[(int64_t)qq * n + a];
        }
        __syncthreads();
        for (int e = tid; e < n * kk; e += NT) {
          const int a = e / kk, c = e - a * kk;
          T acc = Q[a * LD + c];
          for (int q = 0; q < rows; ++q) acc += Cs[q * LD + a] * Om[q * kk + c];
          Q[a * LD + c] = acc;
        }
        __syncthreads();
      }
      mark(9);
      // Householder QR of Q[:, :k], applied to the probe columns as well
      for (int j = 0; j < k; ++j) {
        if (warp == 0) {
          const T xl = (j + 1 + lane < n) ? Q[(j + 1 + lane) * LD + j] : T(0);
          const T xh = (j + 33 + lane < n) ? Q[(j + 33 + lane) * LD + j] : T(0);
          T beta, tq, sc;
          const bool ok = reflector(Q[j * LD + j], xl, xh, beta, tq, sc);
          if (ok) {
            if (j + 1 + lane < n) Q[(j + 1 + lane) * LD + j] = xl * sc;
            if (j + 33 + lane < n) Q[(j + 33 + lane) * LD + j] = xh * sc;
          }
          __syncwarp();
          if (lane == 0) {
            s_tq[j] = ok ? tq : T(0);
            if (ok) Q[j * LD + j] = beta;
          }
        }
        __syncthreads();
        const T tq = s_tq[j];
        if (tq != T(0)) {
          for (int l = j + 1 + warp; l < kk; l += kWarpsNT) {
            T d = 0;
            for (int a = j + 1 + lane; a < n; a += 32) d += Q[a * LD + j] * Q[a * LD + l];
            d = warp_sum(d);
            d = (d + Q[j * LD + l]) * tq;
            if (lane == 0) Q[j * LD + l] -= d;
            for (int a = j + 1 + lane; a < n; a += 32) Q[a * LD + l] -= d * Q[a * LD + j];
          }
        }
        __syncthreads();
      }
      if (warp < 2) {   // ||(I - Q Q^T) F w|| = norm of rows k.. of H^T (F w)
        T sres = 0;
        for (int a = k + lane; a < n; a += 32) sres += Q[a * LD + k + warp] * Q[a * LD + k + warp];
        sres = warp_sum(sres);
        if (lane == 0) s_probe[warp] = sqrt(sres);
      }
      // explicit Q (n x k) into Cs: H_0 ... H_{k-1} [I; 0]
      T* Qx = Cs;   // n x LD (uses the Cs/Om space, NL >= n * LD)
      for (int e = tid; e < n * k; e += NT) {
        const int a = e / k, c = e - a * k;
        Qx[a * LD + c] = (a == c) ? T(1) : T(0);
      }
      __syncthreads();
      for (int j = k - 1; j >= 0; --j) {
        const T tq = s_tq[j];
        if (tq != T(0)) {
          for (int l = j + warp; l < k; l += kWarpsNT) {
            T d = 0;
            for (int a = j + 1 + lane; a < n; a += 32) d += Q[a * LD + j] * Qx[a * LD + l];
            d = warp_sum(d);
            d = (d + Qx[j * LD + l]) * tq;
            if (lane == 0) Qx[j * LD + l] -= d;
            for (int a = j + 1 + lane; a < n; a += 32) Qx[a * LD + l] -= d * Q[a * LD + j];
          }
        }
        __syncthreads();
      }
      for (int e = tid; e < n * LD; e += NT) Q[e] = Qx[e];   // Q <- explicit basis
      __syncthreads();
      mark(10);
      // TSQR of the rows of F^T Q (k columns), one R per warp, tree merge
      const int nchunks = (mF + kChunk - 1) / kChunk;
      const int qw = min(qwl, nchunks);
      T* wbase = un + NL;
      if (warp < qw) {
        T* Rw = wbase + warp * pwl;
        T* Cw = Rw + k * LK;
        T* Pw = Cw + kChunk * LD;
        T* vb = Pw + kChunk * LK;
        for (int e = lane; e < k * LK; e += 32) Rw[e] = T(0);
        for (int c = warp; c < nchunks; c += qw) {
          const int g0 = c * kChunk;
          const int rows = min(kChunk, mF - g0);
          warp_load_far_rows(Cw, LD, pool, L, i, n, g0, rows, nf, s_fpre, s_fk, s_foff, s_wf[warp], s_wq[warp]);
          const int k4 = (k + 3) >> 2;
          for (int e = lane; e < rows * k4; e += 32) {
            const int q2 = e / k4, c0 = (e - q2 * k4) * 4;
            T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 4
            for (int a = 0; a < n; ++a) {
              const T cv = Cw[q2 * LD + a];
              const T* qr = Q + a * LD + c0;
              a0 += cv * qr[0];
              a1 += cv * qr[1];
              a2 += cv * qr[2];
              a3 += cv * qr[3];
            }
            Pw[q2 * LK + c0] = a0;
            if (c0 + 1 < k) Pw[q2 * LK + c0 + 1] = a1;
            if (c0 + 2 < k) Pw[q2 * LK + c0 + 2] = a2;
            if (c0 + 3 < k) Pw[q2 * LK + c0 + 3] = a3;
          }
          __syncwarp();
          warp_qr_stack(Rw, Pw, vb, k, rows, LK);
        }
      }
      __syncthreads();
      for (int step = 1; step < qw; step *= 2) {
        if (warp % (2 * step) == 0 && warp + step < qw) {
          T* Ra = wbase + warp * pwl;
          T* Rb = wbase + (warp + step) * pwl;
          warp_qr_merge(Ra, Rb, Ra + k * LK + kChunk * LD + kChunk * LK, k, LK);
        }
        __syncthreads();
      }
      mark(11);
      // one-sided Jacobi on the k x k factor R (= wbase), V in Vb
      T* Xr = wbase;                 // R (k x k, ld LK)
      T* Vb = wbase + k * LK;        // warp 0's row buffers, free now (k x k, ld LK)
      for (int e = tid; e < k * k; e += NT) {
        const int a = e / k, b = e - a * k;
        Vb[a * LK + b] = (a == b) ? T(1) : T(0);
      }
      __syncthreads();
      {
        const int nb = k + (k & 1), npairs = nb / 2;
        const int half = lane >> 4, hl = lane & 15;
        const T tolJ = T(k) * Eps<T>::v, tolJ2 = tolJ * tolJ;
        bool jconv = false;
        int nsw = kMaxSweeps;
        for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
          // same negligible-pair rule as the exact path, with k columns
          for (int j = warp; j < k; j += kWarpsNT) {
            T sv = 0;
            for (int row = lane; row < k; row += 32) sv += Xr[row * LK + j] * Xr[row * LK + j];
            sv = warp_sum(sv);
            if (lane == 0) sig_tmp[j] = sv;
          }
          __syncthreads();
          if (warp == 0) {
            T cm = fmax(lane < k ? sig_tmp[lane] : T(0), lane + 32 < k ? sig_tmp[lane + 32] : T(0));
            cm = warp_max(cm);
            if (lane == 0) {
              const T sm = sqrt(cm);
              T test = (tol == 0.0 || tol_mode == CE_TOL_FIXED) ? T(n) * Eps<T>::v * sm
                                    : ((tol_mode == CE_TOL_ABS) ? T(tol) : T(tol) * sm);
              test = fmax(test, static_cast<T>(floor_all)) * T(0.5) * fast_rsqrt(T(k));
              s_skip2 = test * test;
              s_flag = 0;
            }
          }
          __syncthreads();
          const T skip2 = s_skip2;
          for (int rnd = 0; rnd < nb - 1; ++rnd) {
            for (int tb = warp * 2; tb < npairs; tb += NT / 16) {
              const int t = tb + half;
              int p = nb - 1, q = rnd;
              if (t != 0) {
                p = rnd + t;
                if (p >= nb - 1) p -= nb - 1;
                q = rnd - t;
                if (q < 0) q += nb - 1;
              }
              const bool valid = t < npairs && p < k && q < k;
              T a = 0, b = 0, g = 0;
              if (valid) {
                for (int row = hl; row < k; row += 16) {
                  T xp = Xr[row * LK + p], xq = Xr[row * LK + q];
                  a += xp * xp;
                  b += xq * xq;
                  g += xp * xq;
                }
              }
              a = half_sum(a);
              b = half_sum(b);
              g = half_sum(g);
              if (valid && g != T(0) && (a >= skip2 || b >= skip2) && g * g > tolJ2 * a * b) {
                const T zeta = (b - a) * fast_rcp(T(2) * g);
                const T az = fabs(zeta);
                const T den = (az > T(1)) ? az * (T(1) + sqrt(T(1) + fast_rcp(az * az)))
                                          : az + sqrt(T(1) + az * az);
                const T tt = ((zeta >= T(0)) ? T(1) : T(-1)) * fast_rcp(den);
                const T cs = fast_rsqrt(T(1) + tt * tt), sn = cs * tt;
                for (int row = hl; row < k; row += 16) {
                  T xp = Xr[row * LK + p], xq = Xr[row * LK + q];
                  Xr[row * LK + p] = cs * xp - sn * xq;
                  Xr[row * LK + q] = sn * xp + cs * xq;
                  T vp = Vb[row * LK + p], vq = Vb[row * LK + q];
                  Vb[row * LK + p] = cs * vp - sn * vq;
                  Vb[row * LK + q] = sn * vp + cs * vq;
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
            jconv = true;
            break;
          }
        }
        if (!jconv && tid == 0 && lvl_ok) atomicAdd(la.stats + 32 + level, 1);
        if (L.prof && tid == 0 && level < 16) {
          atomicAdd(L.prof + level * kProfSlots + kRowPhases + 2, static_cast<unsigned long long>(nsw));
          atomicAdd(L.prof + level * kProfSlots + kRowPhases + 3, 1ull);
        }
      }
      for (int j = tid; j < k; j += NT) {
        T sv = 0;
        for (int row = 0; row < k; ++row) sv += Xr[row * LK + j] * Xr[row * LK + j];
        sig_tmp[j] = sqrt(sv);
      }
      __syncthreads();
      for (int j = tid; j < k; j += NT) {
        const T sj = sig_tmp[j];
        int pos = 0;
        for (int kq = 0; kq < k; ++kq) pos += (sig_tmp[kq] > sj) || (sig_tmp[kq] == sj && kq < j);
        s_pos[j] = pos;
        sig[pos] = sj;
      }
      __syncthreads();
      if (tid == 0) {
        const double smax = static_cast<double>(sig[0]);
        double tt = (tol == 0.0 || tol_mode == CE_TOL_FIXED) ? n * static_cast<double>(Eps<T>::v) * smax
                                 : ((tol_mode == CE_TOL_ABS) ? tol : tol * smax);
        tt = fmax(tt, floor_all);
        int rr = 0;
        for (int kq = 0; kq < k; ++kq) rr += (static_cast<double>(sig[kq]) > tt) ? 1 : 0;
        const double pr = fmax(static_cast<double>(s_probe[0]), static_cast<double>(s_probe[1]));
        const bool ok = isfinite(smax) && rr < k && pr <= 0.5 * tt;
        s_flag = ok ? rr : -1;
        sig_tmp[0] = static_cast<T>(tt);
      }
      __syncthreads();
      const int rl = s_flag;
      if (rl >= 0) {
        // U_b = Q V_B(:, sorted first rl)  ->  U[:, :rl]
        for (int e = tid; e < n * rl; e += NT) {
          const int a = e / rl, c = e - a * rl;
          int j = 0;
          while (s_pos[j] != c) ++j;
          T acc = 0;
          for (int q = 0; q < k; ++q) acc += Q[a * LD + q] * Vb[q * LK + j];
          U[a * LD + c] = acc;
        }
        __syncthreads();
        // complete U_b to an orthogonal U: Householder QR of U[:, :rl] and
        // U = H_0 ... H_{rl-1} (its first rl columns span U_b)
        for (int j = 0; j < rl; ++j) {
          if (warp == 0) {
            const T xl = (j + 1 + lane < n) ? U[(j + 1 + lane) * LD + j] : T(0);
            const T xh = (j + 33 + lane < n) ? U[(j + 33 + lane) * LD + j] : T(0);
            T beta, tq, sc;
            const bool okr = reflector(U[j * LD + j], xl, xh, beta, tq, sc);
            if (okr) {
              if (j + 1 + lane < n) U[(j + 1 + lane) * LD + j] = xl * sc;
              if (j + 33 + lane < n) U[(j + 33 + lane) * LD + j] = xh * sc;
            }
            __syncwarp();
            if (lane == 0) {
              s_tq[j] = okr ? tq : T(0);
              if (okr) U[j * LD + j] = beta;
            }
          }
          __syncthreads();
          const T tq = s_tq[j];
          if (tq != T(0)) {
            for (int l = j + 1 + warp; l < rl; l += kWarpsNT) {
              T d = 0;
              for (int a = j + 1 + lane; a < n; a += 32) d += U[a * LD + j] * U[a * LD + l];
              d = warp_sum(d);
              d = (d + U[j * LD + l]) * tq;
              if (lane == 0) U[j * LD + l] -= d;
              for (int a = j + 1 + lane; a < n; a += 32) U[a * LD + l] -= d * U[a * LD + j];
            }
          }
          __syncthreads();
        }
        T* Uf = Cs;   // n x n accumulation of the reflectors
        for (int e = tid; e < n * n; e += NT) {
          const int a = e / n, c = e - a * n;
          Uf[a * LD + c] = (a == c) ? T(1) : T(0);
        }
        __syncthreads();
        for (int j = rl - 1; j >= 0; --j) {
          const T tq = s_tq[j];
          if (tq != T(0)) {
            for (int l = j + warp; l < n; l += kWarpsNT) {
              T d = 0;
              for (int a = j + 1 + lane; a < n; a += 32) d += U[a * LD + j] * Uf[a * LD + l];
              d = warp_sum(d);
              d = (d + Uf[j * LD + l]) * tq;
              if (lane == 0) Uf[j * LD + l] -= d;
              for (int a = j + 1 + lane; a < n; a += 32) Uf[a * LD + l] -= d * U[a * LD + j];
            }
          }
          __syncthreads();
        }
        for (int e = tid; e < n * n; e += NT) {
          const int a = e / n, c = e - a * n;
          U[a * LD + c] = Uf[a * LD + c];
        }
        for (int j = k + tid; j < n; j += NT) sig[j] = T(0);
        r = rl;
        tau = static_cast<double>(sig_tmp[0]);
        have_u = true;
        if (tid == 0 && lvl_ok) atomicAdd(la.stats + 2 * level, 1);
        if (tid == 0 && L.kw) L.kw[i] = k;
      } else if (tid == 0) {
        if (lvl_ok) atomicAdd(la.stats + 2 * level + 1, 1);
        if (L.kw) L.kw[i] = -k;
      }
      __syncthreads();
    } else if (tid == 0) {
      if (lvl_ok) atomicAdd(la.stats + 2 * level + 1, 1);
      if (L.kw) L.kw[i] = 0;
    }
    }  // la.model
  }

  mark(2);
  // ---------------- A. R factor of F_i^T (warp TSQR + tree merge) ----------
  if (mF > 0 && !have_u) {
    const int nchunks = (mF + kChunk - 1) / kChunk;
    const int qw = min(QW, nchunks);
    if (warp < qw) {
      T* Rw = un + warp * per_warp;
      T* Cw = Rw + NL;
      T* vb = Cw + kChunk * LD;
      for (int e = lane; e < n * LD; e += 32) Rw[e] = T(0);
      for (int c = warp; c < nchunks; c += qw) {
        const int g0 = c * kChunk;
        const int rows = min(kChunk, mF - g0);
        warp_load_far_rows(Cw, LD, pool, L, i, n, g0, rows, nf, s_fpre, s_fk, s_foff, s_wf[warp], s_wq[warp]);
        warp_qr_stack(Rw, Cw, vb, n, rows, LD);
      }
    }
    __syncthreads();
    for (int step = 1; step < qw; step *= 2) {
      if (warp % (2 * step) == 0 && warp + step < qw) {
        T* Ra = un + warp * per_warp;
        T* Rb = un + (warp + step) * per_warp;
        warp_qr_merge(Ra, Rb, Ra + NL + kChunk * LD, n, LD);
      }
      __syncthreads();
    }

    mark(3);
    // ---------------- B. one-sided Jacobi on R (= X) ------------------------
    for (int e = tid; e < n * n; e += NT) {
      int a = e / n, b = e - a * n;
      V[a * LD + b] = (a == b) ? T(1) : T(0);
    }
    __syncthreads();
    const int nb = n + (n & 1);
    const int npairs = nb / 2;
    const int half = lane >> 4, hl = lane & 15;
    const T tolJ = T(n) * Eps<T>::v;
    const T tolJ2 = tolJ * tolJ;
    double dn2 = 0.0;
    for (int w = 0; w < kWarpsNT; ++w) dn2 += s_red[w];
    const double floor_tau = static_cast<double>(Eps<T>::v) * sqrt(dn2);
    const T floor_tau_t = static_cast<T>(floor_tau);
    bool jconv = false;
    int nsw = kMaxSweeps;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
      // Columns whose norm stays below tau_est / (2 sqrt n) form a group whose
      // singular values are all below tau / 2: rotating two of them changes
      // neither the kept subspace nor the rank, so such pairs are skipped.
      // tau_est uses the largest current column norm (<= sigma_1).
      for (int j = warp; j < n; j += kWarpsNT) {
        T s = 0;
        for (int row = lane; row < n; row += 32) s += X[row * LD + j] * X[row * LD + j];
        s = warp_sum(s);
        if (lane == 0) sig_tmp[j] = s;
      }
      __syncthreads();
      if (warp == 0) {
        T cm = fmax(lane < n ? sig_tmp[lane] : T(0), lane + 32 < n ? sig_tmp[lane + 32] : T(0));
        cm = warp_max(cm);
        if (lane == 0) {
          const T sm = sqrt(cm);
          T test = (tol == 0.0 || tol_mode == CE_TOL_FIXED) ? T(n) * Eps<T>::v * sm
                                : ((tol_mode == CE_TOL_ABS) ? T(tol) : T(tol) * sm);
          test = fmax(test, floor_tau_t) * T(0.5) * fast_rsqrt(T(n));
          s_skip2 = test * test;
          s_flag = 0;
        }
      }
      __syncthreads();
      const T skip2 = s_skip2;
      for (int rnd = 0; rnd < nb - 1; ++rnd) {
        for (int tb = warp * 2; tb < npairs; tb += NT / 16) {
          const int t = tb + half;
          int p = nb - 1, q = rnd;
          if (t != 0) {
            p = rnd + t;
            if (p >= nb - 1) p -= nb - 1;
            q = rnd - t;
            if (q < 0) q += nb - 1;
          }
          const bool valid = t < npairs && p < n && q < n;
          T a = 0, b = 0, g = 0;
          if (valid) {
            for (int row = hl; row < n; row += 16) {
              T xp = X[row * LD + p], xq = X[row * LD + q];
              a += xp * xp;
              b += xq * xq;
              g += xp * xq;
            }
          }
          a = half_sum(a);
          b = half_sum(b);
          g = half_sum(g);
          if (valid && g != T(0) && (a >= skip2 || b >= skip2) && g * g > tolJ2 * a * b) {
            // tan of the rotation angle, t = sign(z) / (|z| + sqrt(1 + z^2)),
            // z = (b - a) / (2 g); cs = 1/sqrt(1 + t^2), sn = cs t is an exact
            // rotation up to rounding whatever the accuracy of t
            const T zeta = (b - a) * fast_rcp(T(2) * g);
            const T az = fabs(zeta);
            const T den = (az > T(1)) ? az * (T(1) + sqrt(T(1) + fast_rcp(az * az)))
                                      : az + sqrt(T(1) + az * az);
            const T tt = ((zeta >= T(0)) ? T(1) : T(-1)) * fast_rcp(den);
            const T cs = fast_rsqrt(T(1) + tt * tt), sn = cs * tt;
            for (int row = hl; row < n; row += 16) {
              T xp = X[row * LD + p], xq = X[row * LD + q];
              X[row * LD + p] = cs * xp - sn * xq;
              X[row * LD + q] = sn * xp + cs * xq;
              T vp = V[row * LD + p], vq = V[row * LD + q];
              V[row * LD + p] = cs * vp - sn * vq;
              V[row * LD + q] = sn * vp + cs * vq;
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
        jconv = true;
        break;
      }
    }
    if (!jconv && tid == 0 && level < 16 && la.stats) atomicAdd(la.stats + 32 + level, 1);
    if (L.prof && tid == 0 && level < 16) {
      atomicAdd(L.prof + level * kProfSlots + kRowPhases, static_cast<unsigned long long>(nsw));
      atomicAdd(L.prof + level * kProfSlots + kRowPhases + 1, 1ull);
    }
    for (int j = tid; j < n; j += NT) {
      T s = 0;
      for (int row = 0; row < n; ++row) s += X[row * LD + j] * X[row * LD + j];
      sig_tmp[j] = sqrt(s);
    }
    __syncthreads();
    for (int j = tid; j < n; j += NT) {
      const T sj = sig_tmp[j];
      int pos = 0;
      for (int k = 0; k < n; ++k) pos += (sig_tmp[k] > sj) || (sig_tmp[k] == sj && k < j);
      s_pos[j] = pos;
      sig[pos] = sj;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += NT) {
      int a = e / n, j = e - a * n;
      U[a * LD + s_pos[j]] = V[a * LD + j];
    }
    const double smax = static_cast<double>(sig[0]);
    if (!isfinite(smax)) {
      if (tid == 0) set_status(status, CE_ERR_NOT_SPD, level, i, 2);
      return;
    }
    if (tol_mode == CE_TOL_FIXED) {
      // CE(r) (Section 2.2 remark): the r leading directions, with every
      // singular value tied with sigma_r (within kTieRel) and none that is
      // rounding noise; tol carries r
      const int rf = static_cast<int>(tol);
      tau = n * static_cast<double>(Eps<T>::v) * smax;
      if (rf == 0)
        tau = fmax(tau, smax);
      else if (rf < n)
        tau = fmax(tau, (1.0 - kTieRel) * static_cast<double>(sig[rf - 1]));
    } else if (tol == 0.0) {
      tau = n * static_cast<double>(Eps<T>::v) * smax;
    } else {
      tau = (tol_mode == CE_TOL_ABS) ? tol : tol * smax;
    }
    tau = fmax(tau, floor_tau);
    if (tid == 0) {
      int rr = 0;
      for (int k = 0; k < n; ++k) rr += (static_cast<double>(sig[k]) > tau) ? 1 : 0;
      s_flag = rr;
    }
    __syncthreads();
    r = s_flag;
  } else if (mF == 0) {
    for (int e = tid; e < n * n; e += NT) {
      int a = e / n, b = e - a * n;
      U[a * LD + b] = (a == b) ? T(1) : T(0);
    }
    for (int k = tid; k < n; k += NT) sig[k] = T(0);
  }
  __syncthreads();
  mark(4);
  const int m = n - r;
  if (tid == 0) {
    L.rank[i] = r;
    L.tau[i] = tau;
  }
  for (int k = tid; k < n; k += NT) L.sigma[L.vec_off[i] + k] = static_cast<double>(sig[k]);
  T* Ug = reinterpret_cast<T*>(L.U) + L.u_off[i];
  for (int e = tid; e < n * n; e += NT) {
    int a = e / n, b = e - a * n;
    Ug[e] = U[a * LD + b];
  }

  // ---------------- C. transform + elimination ----------------------------
  for (int e = tid; e < n * n; e += NT) {
    int a = e / n, b = e - a * n;
    Y[a * LD + b] = Dg[e];
  }
  __syncthreads();
  cta_mm<T, NT>(tc, n, n, n, [&](int a, int k) { return Y[a * LD + k]; },        // Xt = D U
              [&](int k, int b) { return U[k * LD + b]; },
              [&](int a, int b, T v) { Xt[a * LD + b] = v; });
  __syncthreads();
  cta_mm<T, NT>(tc, n, n, n, [&](int a, int k) { return U[k * LD + a]; },        // Tm = U^T D U
              [&](int k, int b) { return Xt[k * LD + b]; },
              [&](int a, int b, T v) { Tm[a * LD + b] = v; });
  __syncthreads();
  // Cholesky of Tm[r:, r:]: right-looking, unscaled updates, one barrier per
  // step; L_hat(a, k) = Tm(a, k) / sqrt(Tm(k, k)) at the end
  T* Tn = Tm + r * LD + r;
  for (int k = 0; k < m; ++k) {
    const T piv = Tn[k * LD + k];
    if (!(piv > T(0))) {
      if (tid == 0) set_status(status, CE_ERR_NOT_SPD, level, i, 1, k, static_cast<double>(piv));
      return;
    }
    const int rem = m - k - 1;
    const T ip = T(1) / piv;
    for (int e = tid; e < rem * rem; e += NT) {
      const int a = k + 1 + e / rem, b = k + 1 + e % rem;
      if (b <= a) Tn[a * LD + b] -= Tn[a * LD + k] * Tn[b * LD + k] * ip;
    }
    __syncthreads();
  }
  for (int e = tid; e < m * m; e += NT) {
    const int a = e / m, k = e - a * m;
    if (k < a) Tn[a * LD + k] /= sqrt(Tn[k * LD + k]);
  }
  __syncthreads();
  for (int k = tid; k < m; k += NT) Tn[k * LD + k] = sqrt(Tn[k * LD + k]);
  __syncthreads();
  // Li = L_hat^{-1} (lower), one column per thread; the factor keeps Li
  for (int j = tid; j < m; j += NT) {
    for (int a = 0; a < j; ++a) Li[a * LD + j] = T(0);
    for (int a = j; a < m; ++a) {
      T x = (a == j) ? T(1) : T(0);
      for (int k = j; k < a; ++k) x -= Tn[a * LD + k] * Li[k * LD + j];
      Li[a * LD + j] = x / Tn[a * LD + a];
    }
  }
  __syncthreads();
  T* Lg = reinterpret_cast<T*>(L.L) + L.l_off[i];
  for (int e = tid; e < m * m; e += NT) {
    int a = e / m, b = e - a * m;
    Lg[e] = (b <= a) ? Li[a * LD + b] : T(0);
  }
  // W_b = L_hat^{-1} Tm[r:, :r] -> Y[0:m, 0:r], then back into Tm[r:, :r]
  cta_mm<T, NT>(tc, m, r, m, [&](int a, int k) { return Li[a * LD + k]; },
              [&](int k, int b) { return Tm[(r + k) * LD + b]; },
              [&](int a, int b, T v) { Y[a * LD + b] = v; });
  __syncthreads();
  T* Wbase = reinterpret_cast<T*>(L.W) + L.w_off[i];
  for (int e = tid; e < m * r; e += NT) {
    int a = e / r, b = e - a * r;
    const T v = Y[a * LD + b];
    Tm[(r + a) * LD + b] = v;
    Wbase[e] = v;
  }
  __syncthreads();
  // basis diagonal block: Tm[:r, :r] - W_b^T W_b
  cta_mm<T, NT>(tc, r, r, m, [&](int a, int k) { return Tm[(r + k) * LD + a]; },
              [&](int k, int b) { return Tm[(r + k) * LD + b]; },
              [&](int a, int b, T v) { Dg[(int64_t)a * n + b] = Tm[a * LD + b] - v; });
  mark(5);
  // target bookkeeping
  const int c0 = L.close_ptr[i], c1 = L.close_ptr[i + 1];
  const int nt = 1 + (c1 - c0);
  if (nt > kMaxTargets) {
    if (tid == 0) set_status(status, CE_ERR_LIMIT, level, i, 4, nt);
    return;
  }
  if (warp == 0) {  // lane t: target t (loads in flight together, column starts by a scan)
    int p = i, w = r, np = n;
    if (lane > 0 && lane < nt) {
      p = L.close_blk[c0 + lane - 1];
      w = width_of(L, p, ci);
      np = L.n[p];
    }
    if (lane >= nt) np = 0;
    int cs = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, cs, o);
      if (lane >= o) cs += v;
    }
    if (lane < nt) {
      s_tgt[lane] = p;
      s_w[lane] = w;
      s_colst[lane] = lane == 0 ? 0 : cs - np;
    }
  }
  __syncthreads();
  // close rows: Y = U^T X_ip; W_p = L_hat^{-1} Y[r:]; kept rows Y[:r] - W_b^T W_p
  for (int t = 1; t < nt; ++t) {
    const int p = s_tgt[t], w = s_w[t], np = L.n[p];
    T* Xg = pool + L.close_off[c0 + t - 1];
    load_row_tile<T, NT>(Xt, Xg, i, p, n, np, w, LD);
    __syncthreads();
    cta_mm<T, NT>(tc, n, w, n, [&](int a, int k) { return U[k * LD + a]; },
                [&](int k, int b) { return Xt[k * LD + b]; },
                [&](int a, int b, T v) { Y[a * LD + b] = v; });
    __syncthreads();
    T* Wp = Wbase + (int64_t)n * s_colst[t];
    cta_mm<T, NT>(tc, m, w, m, [&](int a, int k) { return Li[a * LD + k]; },
                [&](int k, int b) { return Y[(r + k) * LD + b]; },
                [&](int a, int b, T v) {
                  Xt[a * LD + b] = v;
                  Wp[a * w + b] = v;
                });
    __syncthreads();
    cta_mm<T, NT>(tc, r, w, m, [&](int a, int k) { return Tm[(r + k) * LD + a]; },
                [&](int k, int b) { return Xt[k * LD + b]; },
                [&](int a, int b, T v) { Y[a * LD + b] -= v; });
    __syncthreads();
    store_row_tile<T, NT>(Y, Xg, i, p, n, np, r, w, LD);
    __syncthreads();
  }
  mark(6);
  // far rows: keep U_b^T F (rows r.. of U^T F are E_i and are dropped)
  for (int f = 0; f < nf; ++f) {
    const int k = s_fk[f], w = s_fw[f];
    if (w == 0 || r == 0) continue;
    T* Xg = pool + s_foff[f];
    load_row_tile<T, NT>(Xt, Xg, i, k, n, L.n[k], w, LD);
    __syncthreads();
    cta_mm<T, NT>(tc, r, w, n, [&](int a, int kk) { return U[kk * LD + a]; },
                [&](int kk, int b) { return Xt[kk * LD + b]; },
                [&](int a, int b, T v) { Y[a * LD + b] = v; });
    __syncthreads();
    store_row_tile<T, NT>(Y, Xg, i, k, n, L.n[k], r, w, LD);
    __syncthreads();
  }
  mark(7);
  // Schur update between close targets: A(p, q) -= W_p^T W_q
  if (m > 0 && std::is_same<T, float>::value && tc) {
    // tensor cores: the 16 x 8 tiles of all pairs (p, q) in one list, so the
    // warps share them evenly whatever the pair sizes
    __shared__ int s_pt[kMaxTargets * (kMaxTargets + 1) / 2 + 1];
    const int np1 = nt - 1, npairs = np1 * (np1 + 1) / 2;
    if (tid == 0) {
      int acc = 0, p = 0;
      for (int a = 1; a < nt; ++a)
        for (int b = a; b < nt; ++b, ++p) {
          s_pt[p] = acc;
          acc += ((s_w[a] + 15) >> 4) * ((s_w[b] + 7) >> 3);
        }
      s_pt[npairs] = acc;
    }
    __syncthreads();
    const int total = s_pt[npairs];
    for (int t = warp; t < total; t += kWarpsNT) {
      int lo = 0, hi = npairs - 1;  // pair p: the last one starting at or before tile t
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pt[mid] <= t) lo = mid; else hi = mid - 1;
      }
      const int p = lo;
      int a = 1, rem = p;
      while (rem >= nt - a) {
        rem -= nt - a;
        ++a;
      }
      const int b = a + rem;
      const int wa = s_w[a], wb = s_w[b];
      const T* Wa = Wbase + (int64_t)n * s_colst[a];
      const T* Wb = Wbase + (int64_t)n * s_colst[b];
      T* Xg = pool + L.schur_off[L.schur_ptr[i] + nt + p];
      const int ld = L.n[s_tgt[b]];
      const int tt = t - s_pt[p], tn = (wb + 7) >> 3;
      const bool acc = L.accumulate != 0;
      warp_tile_tc(wa, wb, m, [&](int x, int k) { return static_cast<float>(Wa[k * wa + x]); },
                   [&](int k, int y) { return static_cast<float>(Wb[k * wb + y]); },
                   [&](int x, int y, float v) {
                     if (acc)
                       atomicAdd(&Xg[(int64_t)x * ld + y], -static_cast<T>(v));
                     else
                       Xg[(int64_t)x * ld + y] -= static_cast<T>(v);
                   },
                   (tt / tn) * 16, (tt % tn) * 8);
    }
  } else if (m > 0) {
    int idx = L.schur_ptr[i] + nt;   // skip the row of the basis of i
    for (int a = 1; a < nt; ++a) {
      for (int b = a; b < nt; ++b, ++idx) {
        const int wa = s_w[a], wb = s_w[b];
        const T* Wa = Wbase + (int64_t)n * s_colst[a];
        const T* Wb = Wbase + (int64_t)n * s_colst[b];
        T* Xg = pool + L.schur_off[idx];
        const int ld = L.n[s_tgt[b]];
        const bool acc = L.accumulate != 0;
        cta_mm<T, NT>(tc, wa, wb, m, [&](int x, int k) { return Wa[k * wa + x]; },
                    [&](int k, int y) { return Wb[k * wb + y]; },
                    [&](int x, int y, T v) {
                      if (acc)
                        atomicAdd(&Xg[(int64_t)x * ld + y], -v);
                      else
                        Xg[(int64_t)x * ld + y] -= v;
                    });
      }
    }
  }
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr int kDepWaitPolls = 1 << 24;  // a dependency wait gives up after L.wait_ns or this many polls

// Persistent level kernel.  CTAs take rows in the colour-major elimination
// order from one counter; before row i starts, every row of a lower colour
// within distance 2 of i (the rows whose eliminations write the pairs row i
// reads or writes) must have finished.  Two rows of different colours that
// touch a common pair are always within distance 2, so every pair sees its
// updates in colour order, exactly as with one launch per colour, while rows
// of later colours start as soon as their own neighbourhood is done.
// A row only waits for rows taken earlier, which are held by running CTAs,
// so the waits always end; they are still bounded (time and polls), and a
// recorded error anywhere ends them.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, (NT >= 512 ? 2 : NT >= 256 ? 3 : 6))
    ce_row_kernel(LevelDev L, int count, int level, double tol, int tol_mode, int* status, int nmax, int LD,
                  int QW, LearnedArgs la) {
  __shared__ int s_q;
  const int tid = threadIdx.x, lane = tid & 31;
  const bool prof = L.prof != nullptr && tid == 0 && level < 16;
  for (;;) {
    long long t_row = prof ? clock64() : 0;
    if (tid < 32) {  // warp 0 takes the next row and waits for its neighbourhood
      int q = 0;
      if (lane == 0) {
        q = atomicAdd(L.qnext, 1);
        if (q >= count || ld_acquire(status) != 0) q = -1;
      }
      q = __shfl_sync(0xffffffffu, q, 0);
      if (q >= 0) {
        const int i = L.order[q];
        const unsigned long long t0 = globaltimer_ns();
        int polls = 0;
        for (int base = L.dep_ptr[i]; base < L.dep_ptr[i + 1] && q >= 0; base += 32) {
          const int d = base + lane;
          const int* flag = d < L.dep_ptr[i + 1] ? L.done + L.dep_idx[d] : nullptr;
          for (;;) {
            const bool ok = flag == nullptr || ld_acquire(flag) != 0;
            if (__all_sync(0xffffffffu, ok)) break;
            int bad = 0;
            if (lane == 0) {
              if (ld_acquire(status) != 0)
                bad = 1;
              else if (++polls > kDepWaitPolls || globaltimer_ns() - t0 > L.wait_ns)
                bad = 2;
              if (bad == 2) set_status(status, CE_ERR_CUDA, level, i, 5);
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) {
              q = -1;
              break;
            }
            __nanosleep(128);
          }
        }
      }
      if (lane == 0) s_q = q;
    }
    __syncthreads();
    const int q = s_q;
    if (q < 0) return;
    __threadfence();
    const int i = L.order[q];
    if (prof) {
      const long long t = clock64();
      atomicAdd(L.prof + level * kProfSlots, static_cast<unsigned long long>(t - t_row));
      t_row = t;
    }
    row_block<T, NT>(L, i, level, tol, tol_mode, status, nmax, LD, QW, la, t_row);
    __syncthreads();
    if (prof) atomicAdd(L.prof + level * kProfSlots + 8, static_cast<unsigned long long>(clock64() - t_row));
    if (tid == 0) {
      __threadfence();
      st_release(L.done + i, 1);
    }
  }
}

int choose_ld(int nmax) { return (nmax % 2 == 0) ? nmax + 1 : nmax; }

size_t smem_bytes(int es, int nmax, int LD, int QW) {  // QW <= 16
  const size_t NL = (size_t)nmax * LD;
  const size_t per_warp = NL + kChunk * LD + 64;
  const size_t un = std::max(QW * per_warp, 4 * NL);
  return es * (NL + 2 * (size_t)nmax + un);
}

// Largest dynamic shared memory a CTA of ce_row_kernel<T, NT> may request
// (the device's opt-in maximum minus the kernel's static shared memory); the
// attribute is raised to it once.
template <typename T, int NT>
cudaError_t max_dyn_smem(size_t* out) {
  static size_t limit = 0;
  if (limit == 0) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, ce_row_kernel<T, NT>);
    if (e != cudaSuccess) return e;
    const size_t lim = static_cast<size_t>(optin) - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(ce_row_kernel<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
    if (e != cudaSuccess) return e;
    limit = lim;
  }
  *out = limit;
  return cudaSuccess;
}

template <typename T, int NT>
cudaError_t launch_nt(const LevelDev& L, int count, int level, double tol, int tol_mode, int* status, int nmax,
                      size_t budget, const LearnedArgs& la, cudaStream_t s) {
  const int LD = choose_ld(nmax);
  size_t limit = 0;
  cudaError_t e = max_dyn_smem<T, NT>(&limit);
  if (e != cudaSuccess) return e;
  budget = std::min(budget, limit);
  int QW = NT / 32;
  while (QW > 1 && smem_bytes(sizeof(T), nmax, LD, QW) > budget) --QW;
  const size_t smem = smem_bytes(sizeof(T), nmax, LD, QW);
  if (smem > limit) return cudaErrorInvalidValue;
  // one resident wave of persistent CTAs
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ce_row_kernel<T, NT>, NT, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(count, std::max(per_sm, 1) * sms));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ce_row_kernel<T, NT><<<grid, NT, smem, s>>>(L, count, level, tol, tol_mode, status, nmax, LD, QW, la);
  return cudaGetLastError();
}

}  // namespace


cudaError_t launch_row_kernel(int esize, const LevelDev& L, int count, int level, double tol, int tol_mode,
                              int* status, int nmax, int shape, const LearnedArgs& la, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  nmax = std::max(nmax, 1);
  // shape 0: 256-thread CTAs, about 3 per SM (72 KB each); 1: 512-thread
  // CTAs with the whole shared memory; 2: 128-thread CTAs of 40 KB
  if (esize == 8) {
    if (shape == 0) return launch_nt<double, 256>(L, count, level, tol, tol_mode, status, nmax, 72 * 1024, la, s);
    if (shape == 2) return launch_nt<double, 128>(L, count, level, tol, tol_mode, status, nmax, 40 * 1024, la, s);
    return launch_nt<double, 512>(L, count, level, tol, tol_mode, status, nmax, ~size_t(0), la, s);
  }
  if (shape == 0) return launch_nt<float, 256>(L, count, level, tol, tol_mode, status, nmax, 72 * 1024, la, s);
  if (shape == 2) return launch_nt<float, 128>(L, count, level, tol, tol_mode, status, nmax, 40 * 1024, la, s);
  return launch_nt<float, 512>(L, count, level, tol, tol_mode, status, nmax, ~size_t(0), la, s);
}

}  // namespace ce
