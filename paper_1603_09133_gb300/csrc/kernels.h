// Launch wrappers of the CE kernels (defined in factor_kernels.cu and
// apply_kernels.cu).  All launches are asynchronous on `s`.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ce_internal.h"

#include <atomic>
#include <string>
#include <vector>

namespace ce {

// kernels launched by the library (process-wide)
extern std::atomic<int64_t> g_launches;

// text returned by ce_last_error() on this thread
void set_last_error(const std::string& msg);

// SMs of the current device (read once per host thread; 1 if unreadable, so
// a grid sized from it stays valid)
inline int device_sms() {
  thread_local int sms = 0;
  if (sms <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 1;
  }
  return sms;
}

// status word layout: [0] = ce_status code, [1] = level, [2] = block,
// [3] = reason (1 pivot <= 0, 2 non-finite sigma), [4] = pivot index,
// [6..7] = pivot value (double bits)
constexpr int kStatusWords = 8;

// row phases timed by ce_row_kernel per level (ce_info.row_phase_ms): wait
// for the neighbourhood, setup, learned sketch (features, MLP, its k x k
// Jacobi and the completion of U), R of F^T, Jacobi SVD, transform +
// Cholesky + L_hat^{-1}, close rows, far rows, Schur updates; then the
// learned sketch's Y = F Omega, its Householder QR, its TSQR of F^T Q
constexpr int kRowPhases = 12;
// per level: the kRowPhases cycle sums, then Jacobi sweeps summed over rows
// and rows that ran a Jacobi SVD (exact SVD; learned sketch's k x k factor)
constexpr int kProfSlots = kRowPhases + 4;

// learned compression (randomized range finder with an MLP-predicted width)
struct LearnedArgs {
  const __half* model = nullptr;  // FP16 rank model; null: exact SVD for every row
  int oversample = 8;             // p: sketch width k = r_hat + p
  int J = 4;                      // children per super-block (parent-rank feature)
  unsigned long long seed = 0;    // key of the counter-based sketch generator
  int* stats = nullptr;           // kStatsWords counters, see below
  bool record = false;            // compute and record the features on every row
                                  // with far columns, also without a model
};

// per-level counters of a factorization (levels 0..15): [2 l] rows whose
// sketch was accepted, [2 l + 1] rows sent to the exact SVD, [32 + l] rows
// whose Jacobi iteration reached its sweep cap before every pair was
// orthogonal (their singular values are still used); large-row levels:
// [48 + l] Jacobi sweeps summed over rows, [64 + l] rows that ran one
constexpr int kStatsWords = 80;

// All `count` rows of a level (order[0, count)) in one persistent launch;
// shape 0: 256-thread CTAs with a 72 KB budget, 1: 512-thread CTAs with the
// whole shared memory.
cudaError_t launch_row_kernel(int esize, const LevelDev& L, int count, int level, double tol, int tol_mode,
                              int* status, int nmax, int shape, const LearnedArgs& la, cudaStream_t s);
cudaError_t launch_scatter_csr(int esize, const int64_t* scatter, const double* val, int64_t nnz,
                               void* pool, cudaStream_t s);
cudaError_t launch_copy_tasks(int esize_src, int esize_dst, const CopyTask* tasks, int ntasks,
                              const void* src, void* dst, cudaStream_t s);
// Dense FP64 Cholesky of every system's coarse matrix (in place, lower);
// desc = [n(nsys), offset(nsys), ...] per system.
cudaError_t coarse_cholesky(double* A, const int64_t* desc, int nsys, int nmax, int level, int* status,
                            double* tinv, cudaStream_t s);
// bytes of the tinv scratch coarse_cholesky needs (one diagonal-tile inverse per system)
size_t coarse_tile_scratch(int nsys);

// apply (x = Q^T L^{-T} L^{-1} Q r)
// one persistent launch per level and direction (see apply_kernels.cu);
// launch_apply_prep starts an apply (next epoch, queue counters zeroed)
cudaError_t launch_apply_prep(int* q, int nq, int* epoch, cudaStream_t s);
cudaError_t launch_apply_fwd(int esize, const LevelDev& L, double* vec, int* status, cudaStream_t s);
cudaError_t launch_apply_bwd(int esize, const LevelDev& L, double* vec, int* status, cudaStream_t s);
cudaError_t launch_level_move(const LevelDev& L, double* cur, double* next, int forward,
                              cudaStream_t s);
cudaError_t launch_perm(const int32_t* perm, int64_t n, const double* in, double* out, int gather,
                        cudaStream_t s);
cudaError_t launch_coarse_dinv(const double* Lc, const int64_t* desc, int nsys, int nmax, double* Dinv,
                               cudaStream_t s);
cudaError_t launch_coarse_solve_sys(const double* Lc, const double* Dinv, const int64_t* desc, int nsys,
                                    double* y, cudaStream_t s);
cudaError_t launch_coarse_solve(const double* Lc, const double* Dinv, int n, double* y, cudaStream_t s);

// PCG building blocks (FP64)
cudaError_t launch_spmv_dot(int64_t n, const int64_t* rowptr, const int32_t* col,
                            const double* val, const double* x, double* y, double* partial,
                            int nparts, cudaStream_t s);
cudaError_t launch_dot(int64_t n, const double* a, const double* b, double* partial, int nparts,
                       cudaStream_t s);
cudaError_t launch_reduce(const double* partial, int nparts, double* out, cudaStream_t s);
// scal[0]=rz, scal[1]=pAp, ... see apply_kernels.cu
cudaError_t launch_update_xr(int64_t n, double* x, double* r, const double* p, const double* Ap,
                             const double* scal, double* partial, int nparts, cudaStream_t s);
// rank-predictor MLP (mlp.cu)
cudaError_t mlp_init(float* theta, unsigned long long seed, cudaStream_t s);
cudaError_t mlp_grad(const float* X, const float* t, int ns, const float* theta, float* partial,
                     float* grad, cudaStream_t s);
cudaError_t mlp_adam_step(const float* X, const float* t, int ns, float* theta, float* partial,
                          float* m, float* v, float lr, int step, cudaStream_t s);
int mlp_partial_blocks(int ns);
cudaError_t mlp_pack(const float* theta, void* model, cudaStream_t s);
cudaError_t mlp_predict(const float* X, int ns, const void* model, float* out, cudaStream_t s);

// Grouped GEMM task: C = alpha op(A) op(B) + beta op(Cin), M x N, inner K.
// ta: A stored K x M (element (m, k) at A[k lda + m]), else M x K;
// tb: B stored N x K (element (k, n) at B[n ldb + k]), else K x N;
// tc / tcin: C / Cin stored N x M, else M x N.  Cin may alias C.
struct GemmTask {
  const void* A;
  const void* B;
  const void* Cin;
  void* C;
  int M, N, K;
  int lda, ldb, ldcin, ldc;
  int ta, tb, tcin, tc;
  float alpha, beta;
  int tile0;   // first tile of the task in its launch (set by the launcher)
  int atomic;  // 1: C += alpha op(A) op(B) by atomic additions (Cin = C, beta = 1;
               //    for products of several tasks into one C)
};

// grouped GEMM engines: CUDA cores (FP32 or FP64 by esize, big_rows.cu) and
// the tensor cores (tc_gemm.cu: FP32 operands as BF16 hi + lo, TMA-staged,
// tcgen05.mma into TMEM; passes 3 = hi*hi + hi*lo + lo*hi, 1 = hi*hi; tasks
// with K = 0 are skipped; *err is set when a pipeline wait expires)
cudaError_t launch_gemm_cuda(int esize, const std::vector<GemmTask>& tasks, cudaStream_t s);
cudaError_t launch_gemm_tc(const std::vector<GemmTask>& tasks, int passes, int* err, cudaStream_t s);

// large-row levels (big_rows.cu): whether a level needs them, the level's
// elimination (per colour, synchronizing the stream once per colour), and the
// apply of such a level (one launch per colour)
bool level_needs_big_rows(const LevelPlan& P);
// the large-row SVD steps (pivoted-QR preconditioner + block Jacobi) on one
// n x n R, for tests (ce_debug_svd)
cudaError_t debug_svd(int esize, int B, int n, const void* R, const void* Dm, double tol, void* X, void* V,
                      int* sweeps, cudaStream_t s);
cudaError_t run_big_level(int esize, LevelStore& st, int level, double tol, int tol_mode, int* status, int* stats,
                          int engine, double* phase_ms, int sketch, unsigned long long seed, cudaStream_t s);
cudaError_t launch_apply_big(int esize, const LevelDev& L, const LevelPlan& P, double* vec, int forward,
                             cudaStream_t s);

// arithmetic peak probes (probes.cu): 0 FP32 FFMA, 1 FP64 DFMA, 2 TF32
// mma.sync m16n8k8, 3 the 3xTF32 product (three TF32 MMAs per product)
cudaError_t measure_peak(int kind, double* tflops, cudaStream_t s);

cudaError_t launch_update_p(int64_t n, double* p, const double* z, const double* scal,
                            int first, cudaStream_t s);
cudaError_t launch_pcg_scalars(double* scal, int stage, cudaStream_t s);

}  // namespace ce
