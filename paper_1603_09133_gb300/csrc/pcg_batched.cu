// pcg_solve_batched: FP64 PCG over the independent systems of a block-diagonal
// batch (Section 3: the CE factorization preconditions conjugate gradients),
// one CG recurrence per system -- its own alpha, beta, residual norm and
// stopping test -- with one iteration captured once in a CUDA graph and
// replayed.
//
// Dot products are segmented: the rows of every system are cut into chunks of
// kChunk rows, one CTA per chunk writes a partial sum, and one thread per
// system adds its chunks in index order, so the result does not depend on
// scheduling.  A converged system is frozen (no update of x, r, p and no
// SpMV) while the others continue; its iteration count is the one at which its
// residual first met the tolerance, exactly as in the single-system loop.
//
// The graph, the work vectors and the chunk map live in the factor (created
// on the first call for a given matrix, reused after), so a warm call makes
// no allocation and no capture.  The host checks the number of unconverged
// systems one iteration behind the GPU, so the device never idles on the
// check; the one extra iteration this launches is a no-op for frozen systems.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ce_internal.h"
#include "kernels.h"

namespace ce {

namespace {

constexpr int kChunk = 2048;  // rows per reduction chunk
constexpr int kT = 256;       // threads of the chunk kernels
constexpr int kSc = 8;        // per-system scalars

// per-system scalars sc[s * kSc + .]
enum { RZ = 0, ALPHA = 1, BETA = 2, BN = 3, RELRES = 4 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double cta_sum(double v) {
  __shared__ double red[kT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = (lane < kT / 32) ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

// Ap = A p on the chunk's rows, partial p . Ap
__global__ void __launch_bounds__(kT) seg_spmv_dot_kernel(const int64_t* rowptr, const int32_t* col,
                                                          const double* val, const double* p, double* Ap,
                                                          const int64_t* chunk_row, const int32_t* chunk_sys,
                                                          const int32_t* done, double* part) {
  const int c = blockIdx.x;
  if (done[chunk_sys[c]]) {
    if (threadIdx.x == 0) part[c] = 0.0;
    return;
  }
  double acc = 0.0;
  for (int64_t row = chunk_row[c] + threadIdx.x; row < chunk_row[c + 1]; row += kT) {
    double s = 0.0;
    for (int64_t e = rowptr[row]; e < rowptr[row + 1]; ++e) s += val[e] * p[col[e]];
    Ap[row] = s;
    acc += p[row] * s;
  }
  acc = cta_sum(acc);
  if (threadIdx.x == 0) part[c] = acc;
}

// partial a . b
__global__ void __launch_bounds__(kT) seg_dot_kernel(const double* a, const double* b, const int64_t* chunk_row,
                                                     double* part) {
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int64_t k = chunk_row[c] + threadIdx.x; k < chunk_row[c + 1]; k += kT) acc += a[k] * b[k];
  acc = cta_sum(acc);
  if (threadIdx.x == 0) part[c] = acc;
}

// x += alpha p, r -= alpha Ap (active systems), partial r . r
__global__ void __launch_bounds__(kT) seg_update_xr_kernel(double* x, double* r, const double* p,
                                                           const double* Ap, const int64_t* chunk_row,
                                                           const int32_t* chunk_sys, const int32_t* done,
                                                           const double* sc, double* part) {
  const int c = blockIdx.x, sy = chunk_sys[c];
  if (done[sy]) {
    if (threadIdx.x == 0) part[c] = 0.0;
    return;
  }
  const double alpha = sc[sy * kSc + ALPHA];
  double acc = 0.0;
  for (int64_t k = chunk_row[c] + threadIdx.x; k < chunk_row[c + 1]; k += kT) {
    x[k] += alpha * p[k];
    const double rk = r[k] - alpha * Ap[k];
    r[k] = rk;
    acc += rk * rk;
  }
  acc = cta_sum(acc);
  if (threadIdx.x == 0) part[c] = acc;
}

// p = z + beta p (active systems; beta = 0 on the first pass)
__global__ void __launch_bounds__(kT) seg_update_p_kernel(double* p, const double* z, const int64_t* chunk_row,
                                                          const int32_t* chunk_sys, const int32_t* done,
                                                          const double* sc, int first) {
  const int c = blockIdx.x, sy = chunk_sys[c];
  if (done[sy]) return;
  const double beta = first ? 0.0 : sc[sy * kSc + BETA];
  // the first pass does not read p (its memory may hold NaN patterns)
  for (int64_t k = chunk_row[c] + threadIdx.x; k < chunk_row[c + 1]; k += kT)
    p[k] = first ? z[k] : z[k] + beta * p[k];
}

// Per-system step on the reduced partials (one CTA; systems in strides):
//   0  ||b||: bn, relres, done = (b == 0), its = 0
//   1  rz of the first pass
//   2  alpha = rz / pAp
//   3  ||r||: its += 1, relres, done once relres <= rtol
//   4  rz_new: beta = rz_new / rz, rz = rz_new
// Modes 0 and 3 also write the number of unconverged systems.
__global__ void __launch_bounds__(kT) sys_step_kernel(int mode, int nsys, const int32_t* sys_chunk,
                                                      const double* part, double* sc, const double* rtol,
                                                      int32_t* done, int32_t* its, int32_t* remaining) {
  int cnt = 0;
  for (int sy = threadIdx.x; sy < nsys; sy += kT) {
    double v = 0.0;
    for (int c = sys_chunk[sy]; c < sys_chunk[sy + 1]; ++c) v += part[c];
    double* q = sc + sy * kSc;
    if (mode == 0) {
      q[BN] = sqrt(v);
      done[sy] = (v == 0.0);
      its[sy] = 0;
      q[RELRES] = (v == 0.0) ? 0.0 : 1.0;
    } else if (!done[sy]) {
      if (mode == 1) {
        q[RZ] = v;
      } else if (mode == 2) {
        q[ALPHA] = q[RZ] / v;
      } else if (mode == 3) {
        its[sy] += 1;
        q[RELRES] = sqrt(v) / q[BN];
        if (q[RELRES] <= *rtol) done[sy] = 1;
      } else {
        q[BETA] = v / q[RZ];
        q[RZ] = v;
      }
    }
    cnt += !done[sy];
  }
  if (mode == 0 || mode == 3) {
    const double tot = cta_sum(static_cast<double>(cnt));
    if (threadIdx.x == 0) *remaining = static_cast<int32_t>(tot);
  }
}

struct Fail {
  cudaError_t e;
  ce_status st;
};

void ok(cudaError_t e) {
  if (e != cudaSuccess) throw Fail{e, CE_OK};
}

void ok_ce(ce_status st) {
  if (st != CE_OK) throw Fail{cudaSuccess, st};
}

}  // namespace

// Everything one batched PCG needs, kept in the factor between calls.
struct PcgBatch {
  const ce_csb* A = nullptr;
  const double* val = nullptr;
  int64_t n = 0;
  int nsys = 0, nchunks = 0;
  void* mem = nullptr;  // one device block for all of the following
  double *x, *r, *z, *p, *Ap, *part, *sc, *rtol;
  int32_t *done, *its, *remaining, *chunk_sys, *sys_chunk;
  int64_t* chunk_row;
  int32_t* h_rem = nullptr;  // pinned, two slots
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_kernels = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

void pcg_batch_release(PcgBatch* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  for (auto& e : P->ev)
    if (e) cudaEventDestroy(e);
  if (P->mem) cudaFreeAsync(P->mem, nullptr);
  delete P;
}

namespace {

// one PCG iteration for all systems (captured into the graph)
void enqueue_iteration(const ce_csb* A, const ce_factor* F, PcgBatch& P, cudaStream_t s) {
  const int nc = P.nchunks;
  seg_spmv_dot_kernel<<<nc, kT, 0, s>>>(A->d_rowptr, A->d_col, A->d_val, P.p, P.Ap, P.chunk_row, P.chunk_sys,
                                        P.done, P.part);
  sys_step_kernel<<<1, kT, 0, s>>>(2, P.nsys, P.sys_chunk, P.part, P.sc, P.rtol, P.done, P.its, P.remaining);
  seg_update_xr_kernel<<<nc, kT, 0, s>>>(P.x, P.r, P.p, P.Ap, P.chunk_row, P.chunk_sys, P.done, P.sc, P.part);
  sys_step_kernel<<<1, kT, 0, s>>>(3, P.nsys, P.sys_chunk, P.part, P.sc, P.rtol, P.done, P.its, P.remaining);
  ok_ce(ce_apply(F, P.r, P.z, s));
  seg_dot_kernel<<<nc, kT, 0, s>>>(P.r, P.z, P.chunk_row, P.part);
  sys_step_kernel<<<1, kT, 0, s>>>(4, P.nsys, P.sys_chunk, P.part, P.sc, P.rtol, P.done, P.its, P.remaining);
  seg_update_p_kernel<<<nc, kT, 0, s>>>(P.p, P.z, P.chunk_row, P.chunk_sys, P.done, P.sc, 0);
  ok(cudaGetLastError());
}

// two pinned counters per host thread, kept for the life of the process
int32_t* pinned_counters() {
  thread_local int32_t* p = nullptr;
  if (!p) ok(cudaHostAlloc(reinterpret_cast<void**>(&p), 2 * sizeof(int32_t), cudaHostAllocDefault));
  return p;
}

PcgBatch* make_batch(const ce_csb* A, const ce_factor* F, cudaStream_t s) {
  PcgBatch* P = new PcgBatch();
  try {
    P->A = A;
    P->val = A->d_val;
    P->n = A->n;
    P->nsys = A->nsys;
    std::vector<int64_t> chunk_row;
    std::vector<int32_t> chunk_sys, sys_chunk{0};
    for (int sy = 0; sy < A->nsys; ++sy) {
      for (int64_t r0 = A->sys_row[sy]; r0 < A->sys_row[sy + 1]; r0 += kChunk) {
        chunk_row.push_back(r0);
        chunk_sys.push_back(sy);
      }
      sys_chunk.push_back(static_cast<int32_t>(chunk_row.size()));
    }
    chunk_row.push_back(A->n);
    P->nchunks = static_cast<int>(chunk_sys.size());
    const int64_t n = A->n, nc = P->nchunks, ns = P->nsys;
    const size_t bytes = (5 * n + nc + ns * kSc + 1) * 8 + (nc + 1) * 8 + (3 * ns + 1 + nc + ns + 1) * 4 + 64;
    ok(cudaMallocAsync(&P->mem, bytes, s));
    char* q = static_cast<char*>(P->mem);
    auto take = [&](size_t b) {
      char* r = q;
      q += (b + 7) / 8 * 8;
      return r;
    };
    P->x = reinterpret_cast<double*>(take(n * 8));
    P->r = reinterpret_cast<double*>(take(n * 8));
    P->z = reinterpret_cast<double*>(take(n * 8));
    P->p = reinterpret_cast<double*>(take(n * 8));
    P->Ap = reinterpret_cast<double*>(take(n * 8));
    P->part = reinterpret_cast<double*>(take(nc * 8));
    P->sc = reinterpret_cast<double*>(take(ns * kSc * 8));
    P->rtol = reinterpret_cast<double*>(take(8));
    P->chunk_row = reinterpret_cast<int64_t*>(take((nc + 1) * 8));
    P->done = reinterpret_cast<int32_t*>(take(ns * 4));
    P->its = reinterpret_cast<int32_t*>(take(ns * 4));
    P->remaining = reinterpret_cast<int32_t*>(take(4));
    P->chunk_sys = reinterpret_cast<int32_t*>(take(nc * 4));
    P->sys_chunk = reinterpret_cast<int32_t*>(take((ns + 1) * 4));
    ok(cudaMemcpyAsync(P->chunk_row, chunk_row.data(), (nc + 1) * 8, cudaMemcpyHostToDevice, s));
    ok(cudaMemcpyAsync(P->chunk_sys, chunk_sys.data(), nc * 4, cudaMemcpyHostToDevice, s));
    ok(cudaMemcpyAsync(P->sys_chunk, sys_chunk.data(), (ns + 1) * 4, cudaMemcpyHostToDevice, s));
    ok(cudaMemsetAsync(P->p, 0, n * 8, s));
    P->h_rem = pinned_counters();
    for (auto& e : P->ev) ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // capture one iteration on a private stream; the launch counter keeps
    // only real launches, so the captured ones are taken back out
    cudaStream_t cap = nullptr;
    ok(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    const int64_t before = g_launches.load();
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      try {
        enqueue_iteration(A, F, *P, cap);
      } catch (const Fail& f) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(cap, &g);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        g_launches.store(before);
        throw;
      }
      ce = cudaStreamEndCapture(cap, &P->graph);
    }
    g_launches.store(before);
    cudaStreamDestroy(cap);
    ok(ce);
    ok(cudaGraphInstantiate(&P->exec, P->graph, 0));
    size_t nn = 0;
    ok(cudaGraphGetNodes(P->graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    ok(cudaGraphGetNodes(P->graph, nodes.data(), &nn));
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      ok(cudaGraphNodeGetType(nd, &t));
      if (t == cudaGraphNodeTypeKernel) ++P->graph_kernels;
    }
  } catch (...) {
    pcg_batch_release(P);
    throw;
  }
  return P;
}

}  // namespace

}  // namespace ce

extern "C" ce_status pcg_solve_batched(const ce_csb* A, const ce_factor* F, const double* b_dev, double* x_dev,
                                       double rtol, int maxit, int32_t* iters, double* relres,
                                       int32_t* converged, ce_pcg_info* info, void* stream) {
  using namespace ce;
  if (!A || !F || !b_dev || !x_dev || maxit < 0 || !(rtol >= 0) || A->n != F->N) return CE_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    PcgBatch* P = F->pcg;
    if (P && (P->A != A || P->val != A->d_val || P->n != A->n || P->nsys != A->nsys)) {
      ok(cudaDeviceSynchronize());
      pcg_batch_release(P);
      F->pcg = P = nullptr;
    }
    if (!P) {
      ok(cudaStreamSynchronize(s));
      F->pcg = P = make_batch(A, F, s);
    }
    const int nc = P->nchunks, ns = P->nsys;
    const int64_t n = A->n;
    // x = 0, r = b, ||b|| per system, z = M r, rz, p = z
    ok(cudaMemcpyAsync(P->rtol, &rtol, 8, cudaMemcpyHostToDevice, s));
    ok(cudaMemsetAsync(P->x, 0, n * 8, s));
    ok(cudaMemcpyAsync(P->r, b_dev, n * 8, cudaMemcpyDeviceToDevice, s));
    seg_dot_kernel<<<nc, kT, 0, s>>>(P->r, P->r, P->chunk_row, P->part);
    sys_step_kernel<<<1, kT, 0, s>>>(0, ns, P->sys_chunk, P->part, P->sc, P->rtol, P->done, P->its,
                                     P->remaining);
    ok(cudaGetLastError());
    g_launches.fetch_add(2, std::memory_order_relaxed);
    ok_ce(ce_apply(F, P->r, P->z, s));
    seg_dot_kernel<<<nc, kT, 0, s>>>(P->r, P->z, P->chunk_row, P->part);
    sys_step_kernel<<<1, kT, 0, s>>>(1, ns, P->sys_chunk, P->part, P->sc, P->rtol, P->done, P->its,
                                     P->remaining);
    seg_update_p_kernel<<<nc, kT, 0, s>>>(P->p, P->z, P->chunk_row, P->chunk_sys, P->done, P->sc, 1);
    ok(cudaGetLastError());
    g_launches.fetch_add(3, std::memory_order_relaxed);
    ok(cudaMemcpyAsync(P->h_rem, P->remaining, 4, cudaMemcpyDeviceToHost, s));
    ok(cudaStreamSynchronize(s));
    if (P->h_rem[0] > 0) {
      for (int it = 1; it <= maxit; ++it) {
        const int slot = it & 1;
        ok(cudaGraphLaunch(P->exec, s));
        g_launches.fetch_add(P->graph_kernels, std::memory_order_relaxed);
        ok(cudaMemcpyAsync(P->h_rem + slot, P->remaining, 4, cudaMemcpyDeviceToHost, s));
        ok(cudaEventRecord(P->ev[slot], s));
        if (it > 1) {
          ok(cudaEventSynchronize(P->ev[slot ^ 1]));
          if (P->h_rem[slot ^ 1] == 0) break;
        }
      }
    }
    ok(cudaMemcpyAsync(x_dev, P->x, n * 8, cudaMemcpyDeviceToDevice, s));
    std::vector<double> sc(static_cast<size_t>(ns) * kSc);
    std::vector<int32_t> its(ns), done(ns);
    ok(cudaMemcpyAsync(sc.data(), P->sc, sc.size() * 8, cudaMemcpyDeviceToHost, s));
    ok(cudaMemcpyAsync(its.data(), P->its, ns * 4, cudaMemcpyDeviceToHost, s));
    ok(cudaMemcpyAsync(done.data(), P->done, ns * 4, cudaMemcpyDeviceToHost, s));
    ok(cudaStreamSynchronize(s));
    int maxits = 0, all = 1;
    double maxrel = 0.0;
    for (int sy = 0; sy < ns; ++sy) {
      const double rr = sc[static_cast<size_t>(sy) * kSc + RELRES];
      if (iters) iters[sy] = its[sy];
      if (relres) relres[sy] = rr;
      if (converged) converged[sy] = done[sy];
      maxits = std::max(maxits, its[sy]);
      maxrel = std::max(maxrel, rr);
      all &= done[sy];
    }
    if (info) {
      info->iters = maxits;
      info->relres = maxrel;
      info->converged = all;
    }
    return all ? CE_OK : CE_ERR_NO_CONVERGENCE;
  } catch (const Fail& f) {
    if (f.st != CE_OK) return f.st;
    set_last_error(std::string("pcg_solve_batched: ") + cudaGetErrorString(f.e));
    return f.e == cudaErrorMemoryAllocation ? CE_ERR_OOM : CE_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    return CE_ERR_OOM;
  } catch (const std::exception& ex) {
    set_last_error(std::string("pcg_solve_batched: ") + ex.what());
    return CE_ERR_INVALID_ARG;
  }
}
