// minres_solve: FP64 preconditioned MINRES (Paige & Saunders, "Solution of
// sparse indefinite systems of linear equations", SIAM J. Numer. Anal. 12,
// 1975) with M = Q^T L L^T Q, the Krylov method of the paper's experiments
// (Section 4, MINRES to a residual of 1e-10).  The preconditioned Lanczos
// process gives the tridiagonal T_k one column per iteration; Givens
// rotations keep its QR factorization, and x moves along the directions w.
// Vectors and products stay on the device (SpMV, dot products, the apply of
// the factor); the scalar recurrences run on the host, which reads two dot
// products per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>

#include "kernels.h"

namespace {

// y -= a r
__global__ void minres_axpy_kernel(int64_t n, double* y, const double* r, double a) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] -= a * r[k];
}

// v = s y
__global__ void minres_scale_kernel(int64_t n, double* v, const double* y, double s) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    v[k] = s * y[k];
}

// w_new = (v - e w1 - d w2) g into w1's storage (w1 is not needed after);
// x += phi w_new
__global__ void minres_w_kernel(int64_t n, double* w1, const double* v, const double* w2, double e, double d,
                                double g, double phi, double* x) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double w = (v[k] - e * w1[k] - d * w2[k]) * g;
    w1[k] = w;
    x[k] += phi * w;
  }
}

struct MinresFail {};

}  // namespace

extern "C" ce_status minres_solve(const ce_csb* A, const ce_factor* F, const double* b_dev, double* x_dev,
                                  double rtol, int maxit, ce_pcg_info* info, void* stream) {
  if (!A || !F || !b_dev || !x_dev || maxit < 0 || rtol < 0 || A->n != F->N) return CE_ERR_INVALID_ARG;
  if (A->nsys > 1) {
    ce::set_last_error("minres_solve: a batch handle is not supported (one system per call)");
    return CE_ERR_INVALID_ARG;
  }
  if (info) std::memset(info, 0, sizeof(*info));
  if (A->n == 0) {
    if (info) info->converged = 1;
    return CE_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = A->n;
  const int nparts = static_cast<int>(std::min<int64_t>((n + 255) / 256, (int64_t)ce::device_sms() * 4));
  const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, (int64_t)ce::device_sms() * 8));
  double* buf = nullptr;
  ce_status ret = CE_OK;
  auto ok = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
      ce::set_last_error(std::string("minres_solve: ") + what + ": " + cudaGetErrorString(e));
      throw MinresFail{};
    }
  };
  try {
    // r1, r2, y, v, two directions w, partials, scalars
    ok(cudaMallocAsync(reinterpret_cast<void**>(&buf), (6 * n + nparts + 8) * sizeof(double), s), "allocation");
    double* r1 = buf;
    double* r2 = buf + n;
    double* y = buf + 2 * n;
    double* v = buf + 3 * n;
    double* wa = buf + 4 * n;
    double* wb = buf + 5 * n;
    double* part = buf + 6 * n;
    double* scal = part + nparts;
    auto dot = [&](const double* a, const double* c) {
      ok(ce::launch_dot(n, a, c, part, nparts, s), "dot");
      ok(ce::launch_reduce(part, nparts, scal, s), "reduce");
      double h = 0.0;
      ok(cudaMemcpyAsync(&h, scal, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
      ok(cudaStreamSynchronize(s), "sync");
      return h;
    };
    ok(cudaMemsetAsync(x_dev, 0, n * 8, s), "memset x");
    ok(cudaMemsetAsync(wa, 0, n * 8, s), "memset w");
    ok(cudaMemsetAsync(wb, 0, n * 8, s), "memset w");
    ok(cudaMemcpyAsync(r1, b_dev, n * 8, cudaMemcpyDeviceToDevice, s), "copy b");
    ok(cudaMemcpyAsync(r2, b_dev, n * 8, cudaMemcpyDeviceToDevice, s), "copy b");
    {
      const ce_status st = ce_apply(F, r1, y, s);   // y = M^{-1} b
      if (st != CE_OK) {
        ret = st;
        throw MinresFail{};
      }
    }
    const double b1sq = dot(r1, y);
    if (!(b1sq >= 0.0)) {  // M^{-1} not positive on b (or non-finite)
      ce::set_last_error("minres_solve: the preconditioner is not positive definite on b");
      ret = CE_ERR_NOT_SPD;
      throw MinresFail{};
    }
    const double beta1 = std::sqrt(b1sq);
    double beta = beta1, oldb = 0.0, dbar = 0.0, epsln = 0.0, phibar = beta1;
    double cs = -1.0, sn = 0.0;
    int it = 0;
    bool conv = beta1 == 0.0;
    double rel = conv ? 0.0 : 1.0;
    double* w1 = wa;  // w_{k-2}
    double* w2 = wb;  // w_{k-1}
    for (it = 1; it <= maxit && !conv; ++it) {
      // Lanczos step: v = y / beta, y = A v - (beta / oldb) r1 - (alfa / beta) r2
      ce::g_launches.fetch_add(1, std::memory_order_relaxed);
      minres_scale_kernel<<<grid, 256, 0, s>>>(n, v, y, 1.0 / beta);
      ok(cudaGetLastError(), "scale");
      ok(ce::launch_spmv_dot(n, A->d_rowptr, A->d_col, A->d_val, v, y, part, nparts, s), "spmv");
      if (it >= 2) {
        ce::g_launches.fetch_add(1, std::memory_order_relaxed);
        minres_axpy_kernel<<<grid, 256, 0, s>>>(n, y, r1, beta / oldb);
        ok(cudaGetLastError(), "update");
      }
      const double alfa = dot(v, y);
      ce::g_launches.fetch_add(1, std::memory_order_relaxed);
      minres_axpy_kernel<<<grid, 256, 0, s>>>(n, y, r2, alfa / beta);
      ok(cudaGetLastError(), "update");
      std::swap(r1, r2);   // r1 <- r2, r2 <- y (y's storage is refilled below)
      std::swap(r2, y);
      {
        const ce_status st = ce_apply(F, r2, y, s);   // y = M^{-1} r2
        if (st != CE_OK) {
          ret = st;
          throw MinresFail{};
        }
      }
      oldb = beta;
      const double bsq = dot(r2, y);
      if (!(bsq >= 0.0)) {
        ce::set_last_error("minres_solve: the preconditioner is not positive definite");
        ret = CE_ERR_NOT_SPD;
        throw MinresFail{};
      }
      beta = std::sqrt(bsq);
      // previous rotation on the new column of T_k, then a new rotation
      const double oldeps = epsln;
      const double delta = cs * dbar + sn * alfa;
      const double gbar = sn * dbar - cs * alfa;
      epsln = sn * beta;
      dbar = -cs * beta;
      double gamma = std::hypot(gbar, beta);
      gamma = std::max(gamma, std::numeric_limits<double>::min());
      cs = gbar / gamma;
      sn = beta / gamma;
      const double phi = cs * phibar;
      phibar = sn * phibar;
      // w_k = (v - oldeps w_{k-2} - delta w_{k-1}) / gamma; x += phi w_k
      ce::g_launches.fetch_add(1, std::memory_order_relaxed);
      minres_w_kernel<<<grid, 256, 0, s>>>(n, w1, v, w2, oldeps, delta, 1.0 / gamma, phi, x_dev);
      ok(cudaGetLastError(), "update x");
      std::swap(w1, w2);   // the new w (in w1's storage) is now w_{k-1}
      rel = phibar / beta1;
      if (rel <= rtol) conv = true;
      if (beta == 0.0) conv = true;   // exact Krylov subspace
    }
    if (!conv) it = maxit + 1;
    if (info) {
      info->iters = std::min(it - 1, maxit);
      info->relres = rel;
      info->converged = conv ? 1 : 0;
    }
    if (!conv) ret = CE_ERR_NO_CONVERGENCE;
  } catch (const MinresFail&) {
    if (ret == CE_OK) ret = CE_ERR_CUDA;
  } catch (...) {
    if (ret == CE_OK) ret = CE_ERR_CUDA;
  }
  if (buf) cudaFreeAsync(buf, s);
  return ret;
}
