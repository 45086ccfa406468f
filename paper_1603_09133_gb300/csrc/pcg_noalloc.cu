// pcg_solve_noalloc: the FP64 PCG of pcg_solve for callers that must not
// allocate device memory.  Its work vectors live in one file-scope static
// device array of fixed size instead of memory allocated per call.
//
// Who needs it: applications whose device memory is reserved up front by their
// own pool allocator (a library-side cudaMalloc then fails or fragments that
// pool), latency-critical loops that cannot afford the implicit device-wide
// synchronization and unbounded latency of cudaMalloc / cudaFree, and plugins
// whose host application forbids them to allocate.
//
// The array holds 4 vectors of kNoAllocMaxN doubles plus the reduction
// partials (about 2 MiB) and stays resident on every GPU that loads the
// library until the process exits.  All calls share it and it keeps the last
// call's contents; calls whose work overlaps on the GPU (other streams, other
// host threads) race on it.  Nothing in it needs clearing: every entry is
// written before it is read within a call.
//
// One system per call: a batch handle (csb_build_batched with more than one
// system) is rejected, because pcg_solve runs a separate CG recurrence per
// system there while this entry point has room for one recurrence only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "kernels.h"

namespace {

constexpr int64_t kNoAllocMaxN = 65536;
constexpr int kNoAllocParts = 256;
constexpr int64_t kScratchDoubles = 4 * kNoAllocMaxN + kNoAllocParts + 8;
static __device__ __align__(256) double g_pcg_scratch[kScratchDoubles];

// Device address of the static array on the current device.  Host code only
// sees a host-side stand-in under the array's name, so the address is looked
// up with the caller's device current.  It is looked up on every call (the
// lookup allocates nothing): a cached address would dangle after a
// cudaDeviceReset reloads the module.
cudaError_t scratch_for_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

struct Fail {
  cudaError_t e;
};

void ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    ce::set_last_error(std::string("pcg_solve_noalloc: ") + what + ": " + cudaGetErrorString(e));
    throw Fail{e};
  }
}

}  // namespace

extern "C" ce_status pcg_solve_noalloc(const ce_csb* A, const ce_factor* F, const double* b_dev,
                                       double* x_dev, double rtol, int maxit, ce_pcg_info* info,
                                       void* stream) {
  if (!A || !F || !b_dev || !x_dev || maxit < 0 || rtol < 0 || A->n != F->N) return CE_ERR_INVALID_ARG;
  try {  // the messages below build strings: no host exception crosses the C ABI
    if (A->nsys > 1) {
      ce::set_last_error("pcg_solve_noalloc: a batch of independent systems needs one CG recurrence per "
                         "system; use pcg_solve_batched");
      return CE_ERR_INVALID_ARG;
    }
    if (A->n > kNoAllocMaxN) {
      ce::set_last_error("pcg_solve_noalloc: n = " + std::to_string(A->n) +
                         " exceeds the static work-array limit of " + std::to_string(kNoAllocMaxN) +
                         " unknowns");
      return CE_ERR_LIMIT;
    }
  } catch (...) {
    return A->nsys > 1 ? CE_ERR_INVALID_ARG : CE_ERR_LIMIT;
  }
  const int64_t n = A->n;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (info) std::memset(info, 0, sizeof(*info));
  ce_status ret = CE_OK;
  try {
    double* S = nullptr;
    ok(scratch_for_current_device(&S), "cudaGetSymbolAddress");
    double* r = S;
    double* z = S + kNoAllocMaxN;
    double* p = S + 2 * kNoAllocMaxN;
    double* Ap = S + 3 * kNoAllocMaxN;
    double* part = S + 4 * kNoAllocMaxN;
    double* scal = part + kNoAllocParts;
    const int nparts = static_cast<int>(std::min<int64_t>((n + 255) / 256, kNoAllocParts));
    ok(cudaMemsetAsync(x_dev, 0, n * 8, s), "memset x");
    ok(cudaMemcpyAsync(r, b_dev, n * 8, cudaMemcpyDeviceToDevice, s), "copy b");
    ok(ce::launch_dot(n, r, r, part, nparts, s), "dot");
    ok(ce::launch_reduce(part, nparts, scal + 3, s), "reduce");
    double hb = 0;
    ok(cudaMemcpyAsync(&hb, scal + 3, 8, cudaMemcpyDeviceToHost, s), "read norm");
    ok(cudaStreamSynchronize(s), "sync");
    const double bn = std::sqrt(hb);
    double rel = 0.0;
    int it = 0;
    bool conv = (bn == 0.0);
    if (!conv) {
      ret = ce_apply(F, r, z, s);
      if (ret != CE_OK) throw Fail{cudaErrorUnknown};
      ok(ce::launch_dot(n, r, z, part, nparts, s), "dot");
      ok(ce::launch_reduce(part, nparts, scal + 0, s), "reduce");
      ok(ce::launch_update_p(n, p, z, scal, 1, s), "p");
      rel = 1.0;
      for (it = 1; it <= maxit; ++it) {
        ok(ce::launch_spmv_dot(n, A->d_rowptr, A->d_col, A->d_val, p, Ap, part, nparts, s), "spmv");
        ok(ce::launch_reduce(part, nparts, scal + 1, s), "reduce");
        ok(ce::launch_pcg_scalars(scal, 0, s), "alpha");
        ok(ce::launch_update_xr(n, x_dev, r, p, Ap, scal, part, nparts, s), "xr");
        ok(ce::launch_reduce(part, nparts, scal + 3, s), "reduce");
        double rr = 0;
        ok(cudaMemcpyAsync(&rr, scal + 3, 8, cudaMemcpyDeviceToHost, s), "read norm");
        ok(cudaStreamSynchronize(s), "sync");
        rel = std::sqrt(rr) / bn;
        if (rel <= rtol) {
          conv = true;
          break;
        }
        if (it == maxit) break;
        ret = ce_apply(F, r, z, s);
        if (ret != CE_OK) throw Fail{cudaErrorUnknown};
        ok(ce::launch_dot(n, r, z, part, nparts, s), "dot");
        ok(ce::launch_reduce(part, nparts, scal + 4, s), "reduce");
        ok(ce::launch_pcg_scalars(scal, 1, s), "beta");
        ok(ce::launch_update_p(n, p, z, scal, 0, s), "p");
      }
      if (it > maxit) it = maxit;
    }
    if (info) {
      info->iters = conv && bn == 0.0 ? 0 : it;
      info->relres = rel;
      info->converged = conv ? 1 : 0;
    }
    if (!conv) ret = CE_ERR_NO_CONVERGENCE;
  } catch (const Fail&) {
    if (ret == CE_OK) ret = CE_ERR_CUDA;
  } catch (...) {  // host exceptions (string building) never cross the C ABI
    if (ret == CE_OK) ret = CE_ERR_CUDA;
  }
  return ret;
}
