// C ABI of the CE solver: handles, level loop (Algorithm 1), apply, PCG.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "kernels.h"
#include "mlp_infer.cuh"

using ce::CopyTask;
using ce::LevelDev;
using ce::LevelPlan;
using ce::LevelStore;

namespace ce {
std::atomic<int64_t> g_launches{0};
}

namespace {

thread_local std::string g_last_error;

struct CudaFail {
  cudaError_t e;
};

void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    throw CudaFail{e};
  }
}

}  // namespace

namespace ce {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace ce

namespace {

ce_status status_of(const CudaFail& f) {
  return f.e == cudaErrorMemoryAllocation ? CE_ERR_OOM : CE_ERR_CUDA;
}

// Status of the exception in flight (called from a catch block): no exception
// crosses the C ABI.  Host allocation failures read as CE_ERR_OOM, a rejected
// input found by a host routine as CE_ERR_INVALID_ARG.
ce_status status_of_exception() {
  try {
    throw;
  } catch (const CudaFail& f) {
    return status_of(f);
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return CE_ERR_OOM;
  } catch (const std::exception& ex) {
    g_last_error = ex.what();
    return CE_ERR_INVALID_ARG;
  } catch (...) {
    g_last_error = "unknown host exception";
    return CE_ERR_CUDA;
  }
}

void init_pool_once() {
  static bool done = false;
  if (done) return;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, dev) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  done = true;
}

void* dalloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  check(cudaMallocAsync(&p, bytes, s), "cudaMallocAsync");
  return p;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// Pinned host staging buffers for the uploads of a factorization (grow-only,
// one pair per host thread).  Slot 0 carries level metadata, slot 1 copy
// tasks; a slot is reused only after its last copy has completed.
struct Staging {
  char* p = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
  bool pending = false;
};
thread_local Staging g_stage[3];  // 2: device-to-host reads of ranks and status

char* stage_get(int slot, size_t bytes) {
  Staging& S = g_stage[slot];
  if (S.pending) {
    check(cudaEventSynchronize(S.ev), "staging wait");
    S.pending = false;
  }
  if (!S.ev) check(cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming), "event");
  if (bytes > S.cap) {
    if (S.p) cudaFreeHost(S.p);
    S.p = nullptr;
    S.cap = 0;
    const size_t cap = ((std::max(bytes, size_t(1) << 20) + (size_t(1) << 20) - 1) >> 20) << 20;
    check(cudaHostAlloc(reinterpret_cast<void**>(&S.p), cap, cudaHostAllocDefault), "cudaHostAlloc");
    S.cap = cap;
  }
  return S.p;
}

void stage_upload(int slot, void* dst, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return;
  check(cudaMemcpyAsync(dst, g_stage[slot].p, bytes, cudaMemcpyHostToDevice, s), "H2D");
  check(cudaEventRecord(g_stage[slot].ev, s), "event");
  g_stage[slot].pending = true;
}

// Lays host arrays out in one device allocation: arrays first (one H2D copy
// through the staging buffer), zero-filled regions last (one memset).
struct Packer {
  struct Item {
    size_t off;
    const void* src;
    size_t bytes;
  };
  std::vector<Item> items;
  size_t size = 0, data_end = 0;
  static size_t align(size_t x) { return (x + 255) & ~size_t(255); }
  size_t add(const void* src, size_t bytes) {
    const size_t off = align(size);
    items.push_back({off, src, bytes});
    size = data_end = off + bytes;
    return off;
  }
  template <typename V>
  size_t addv(const std::vector<V>& v) {
    return add(v.data(), v.size() * sizeof(V));
  }
  size_t zeros(size_t bytes) {  // after every add()
    const size_t off = align(size);
    size = off + bytes;
    return off;
  }
  void upload(void* dst, cudaStream_t s) {
    char* h = stage_get(0, data_end);
    // slices of at most 1 MB, copied in parallel
    constexpr size_t kSlice = size_t(1) << 20;
    std::vector<std::pair<int, size_t>> sl;
    for (size_t t = 0; t < items.size(); ++t)
      for (size_t o = 0; o < items[t].bytes; o += kSlice) sl.emplace_back(static_cast<int>(t), o);
    ce::parallel_for(static_cast<int64_t>(sl.size()), 4, [&](int64_t b, int64_t e) {
      for (int64_t q = b; q < e; ++q) {
        const Item& it = items[sl[q].first];
        const size_t o = sl[q].second, nb = std::min(kSlice, it.bytes - o);
        std::memcpy(h + it.off + o, static_cast<const char*>(it.src) + o, nb);
      }
    });
    stage_upload(0, dst, data_end, s);
    if (size > data_end)
      check(cudaMemsetAsync(static_cast<char*>(dst) + data_end, 0, size - data_end, s), "memset metadata");
  }
};

int64_t pair_offset(const LevelPlan& P, int a, int b) { return ce::find_pair(P, a, b); }

// Streams and events for the size buckets' concurrent launches (created once
// per host thread, on the current device).
struct SideStreams {
  cudaStream_t st[ce::kBuckets] = {};
  cudaEvent_t fork = nullptr, join[ce::kBuckets] = {};
};

SideStreams& side_streams() {
  thread_local SideStreams ss;
  if (!ss.fork) {
    for (int b = 0; b < ce::kBuckets; ++b) {
      check(cudaStreamCreateWithFlags(&ss.st[b], cudaStreamNonBlocking), "stream");
      check(cudaEventCreateWithFlags(&ss.join[b], cudaEventDisableTiming), "event");
    }
    check(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming), "event");
  }
  return ss;
}

// Algorithmic flops and bytes of the row-kernel launches of one level,
// counted per block from its size n, rank r (m = n - r) and the widths w of
// its close and far neighbours when it is processed:
//   flops = 2 mF n^2           (Householder R of F^T, mF far rows)
//         + 12 n^3             (SVD of the n x n R with V, if mF > 0)
//         + 4 n^3 + 2 n^2 Wc + 2 n r mF   (U^T D U, U^T C, U_b^T F)
//         + m^3/3 + m^2 (r + Wc)           (Cholesky, TRSM)
//         + m ((r + Wc)^2 + r^2 + sum w^2) (Schur W_p^T W_q, p <= q)
//   bytes = e * (n^2 + n Wc + n mF                        reads D, C, F
//              + n^2 + m^2 + m (r + Wc)                  writes U, L_hat, W
//              + r^2 + r Wc + r mF                       writes kept rows
//              + 2 sum_{p<=q close} w_p w_q)             Schur targets r+w
//   A row that ran the learned compression (sketch width k = |kw_i|, k + 2
//   columns with the probes) counts the sketch instead of the exact SVD:
//         2 n mF (k + 2)       (Y = F [Omega | probes])
//         + 4 n k^2             (Householder QR of Y, explicit Q)
//         + 2 mF n k + 2 mF k^2 (rows of F^T Q, their TSQR)
//         + 12 k^3              (SVD of the k x k factor with V)
//         + 2 n k r + 2 n r^2 + 4 n^2 r   (U_b, its orthogonal completion)
//   and a rejected row (kw_i < 0) counts both.
void level_work(const LevelPlan& P, const std::vector<int>& rank, int es, double& flops,
                double& bytes, const std::vector<int>* kw = nullptr) {
  // fixed chunks summed in chunk order: the totals do not depend on timing
  constexpr int kChunks = 64;
  double pf[kChunks] = {}, pb[kChunks] = {};
  ce::parallel_for(kChunks, 1, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      const int i0 = static_cast<int>((int64_t)P.M * c / kChunks);
      const int i1 = static_cast<int>((int64_t)P.M * (c + 1) / kChunks);
      for (int i = i0; i < i1; ++i) {
        const double n = P.n[i], r = rank[i], m = n - r;
        const int ci = P.colour[i];
        auto wid = [&](int k) { return double(P.colour[k] < ci ? rank[k] : P.n[k]); };
        double mF = 0, Wc = 0, W2 = 0;
        for (int f = P.far_ptr[i]; f < P.far_ptr[i + 1]; ++f) mF += wid(P.far_blk[f]);
        for (int t = P.close_ptr[i]; t < P.close_ptr[i + 1]; ++t) {
          const double x = wid(P.close_blk[t]);
          Wc += x;
          W2 += x * x;
        }
        const double pairs = 0.5 * (Wc * Wc + W2);
        const int kwi = kw ? (*kw)[i] : 0;
        const double k = kwi < 0 ? -kwi : kwi;
        const double sketch = 2 * n * mF * (k + 2) + 4 * n * k * k + 2 * mF * n * k + 2 * mF * k * k +
                              12 * k * k * k + 2 * n * k * r + 2 * n * r * r + 4 * n * n * r;
        const double exact = 2 * mF * n * n + (mF > 0 ? 12 * n * n * n : 0);
        const double compress = kwi > 0 ? sketch : (kwi < 0 ? sketch + exact : exact);
        pf[c] += compress + 4 * n * n * n + 2 * n * n * Wc +
                 2 * n * r * mF + m * m * m / 3 + m * m * (r + Wc) + m * ((r + Wc) * (r + Wc) + r * r + W2);
        pb[c] += es * (n * n + n * Wc + n * mF + n * n + m * m + m * (r + Wc) + r * r + r * Wc + r * mF +
                       2 * pairs);
      }
    }
  });
  flops = 0;
  bytes = 0;
  for (int c = 0; c < kChunks; ++c) {
    flops += pf[c];
    bytes += pb[c];
  }
}

// Block pairs (bi <= bk) of P A P^T with blocks [blkptr[b], blkptr[b+1]) of
// rows: each block row collects its few distinct neighbour blocks in a small
// buffer.  blk_of[r] is the block of permuted row r.
std::vector<std::pair<int, int>> block_pairs(const int64_t* rowptr, const int32_t* col,
                                             const int32_t* perm, const std::vector<int32_t>& iperm,
                                             const std::vector<int64_t>& blkptr,
                                             const std::vector<int>& blk_of) {
  const int M = static_cast<int>(blkptr.size()) - 1;
  const int nch = std::max(1, std::min(ce::host_threads() * 4, (M + 1023) / 1024));
  std::vector<std::vector<std::pair<int, int>>> part(nch);
  ce::parallel_for(nch, 1, [&](int64_t c0, int64_t c1) {
    std::vector<int> nb;
    for (int64_t c = c0; c < c1; ++c)
      for (int bi = static_cast<int>((int64_t)M * c / nch); bi < (int64_t)M * (c + 1) / nch; ++bi) {
        nb.clear();
        for (int64_t r = blkptr[bi]; r < blkptr[bi + 1]; ++r) {
          const int a = perm[r];
          for (int64_t e = rowptr[a]; e < rowptr[a + 1]; ++e) {
            const int bk = blk_of[iperm[col[e]]];
            if (bk >= bi && std::find(nb.begin(), nb.end(), bk) == nb.end()) nb.push_back(bk);
          }
        }
        std::sort(nb.begin(), nb.end());
        for (int bk : nb) part[c].emplace_back(bi, bk);
      }
  });
  std::vector<std::pair<int, int>> pairs;
  for (auto& v : part) pairs.insert(pairs.end(), v.begin(), v.end());
  return pairs;
}

// A is symmetric: every (a, b, v) has a matching (b, a, v).  Rows are sorted
// in one flat copy; lookups are binary searches.
bool csr_symmetric(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val) {
  const int64_t nnz = rowptr[n];
  // rows already in ascending column order (the usual CSR) are searched in
  // place; otherwise every row is sorted into a copy first
  std::atomic<bool> sorted{true};
  ce::parallel_for(n, 8192, [&](int64_t a0, int64_t a1) {
    for (int64_t a = a0; a < a1 && sorted.load(std::memory_order_relaxed); ++a)
      for (int64_t e = rowptr[a] + 1; e < rowptr[a + 1]; ++e)
        if (col[e] <= col[e - 1]) {
          sorted.store(false);
          break;
        }
  });
  if (sorted.load()) {
    std::atomic<bool> ok{true};
    ce::parallel_for(n, 8192, [&](int64_t a0, int64_t a1) {
      for (int64_t a = a0; a < a1 && ok.load(std::memory_order_relaxed); ++a)
        for (int64_t e = rowptr[a]; e < rowptr[a + 1]; ++e) {
          const int32_t b = col[e];
          const int32_t* lo = col + rowptr[b];
          const int32_t* hi = col + rowptr[b + 1];
          const int32_t* it = std::lower_bound(lo, hi, static_cast<int32_t>(a));
          if (it == hi || *it != a || val[it - col] != val[e]) {
            ok.store(false);
            break;
          }
        }
    });
    return ok.load();
  }
  std::vector<std::pair<int32_t, double>> cv(nnz);
  ce::parallel_for(n, 8192, [&](int64_t a0, int64_t a1) {
    for (int64_t a = a0; a < a1; ++a) {
      for (int64_t e = rowptr[a]; e < rowptr[a + 1]; ++e) cv[e] = {col[e], val[e]};
      std::sort(cv.begin() + rowptr[a], cv.begin() + rowptr[a + 1]);
    }
  });
  std::atomic<bool> ok{true};
  ce::parallel_for(n, 8192, [&](int64_t a0, int64_t a1) {
    for (int64_t a = a0; a < a1 && ok.load(std::memory_order_relaxed); ++a)
      for (int64_t e = rowptr[a]; e < rowptr[a + 1]; ++e) {
        const int32_t b = cv[e].first;
        auto lo = cv.begin() + rowptr[b], hi = cv.begin() + rowptr[b + 1];
        auto it = std::lower_bound(lo, hi, std::make_pair((int32_t)a, -1e308));
        if (it == hi || it->first != a || it->second != cv[e].second) {
          ok.store(false);
          break;
        }
      }
  });
  return ok.load();
}

int max_targets(const LevelPlan& P) {
  int t = 0;
  for (int i = 0; i < P.M; ++i) t = std::max(t, 1 + P.close_ptr[i + 1] - P.close_ptr[i]);
  return t;
}

// Device metadata of a level plan: the arrays fixed by the plan (uploaded
// once per plan; level 1's is kept in the csb and shared by every factor) and
// the per-factorization state (ranks, flags, counters; zero-filled).
using ce::StaticMeta;

void* upload_static_meta(const LevelPlan& P, StaticMeta& m, size_t& bytes, cudaStream_t s) {
  Packer pk;
  m.o_n = pk.addv(P.n);
  m.o_col = pk.addv(P.colour);
  m.o_order = pk.addv(P.order);
  m.o_cp = pk.addv(P.close_ptr);
  m.o_cb = pk.addv(P.close_blk);
  m.o_co = pk.addv(P.close_off);
  m.o_fp = pk.addv(P.far_ptr);
  m.o_fb = pk.addv(P.far_blk);
  m.o_fo = pk.addv(P.far_off);
  m.o_do = pk.addv(P.diag_off);
  m.o_sp = pk.addv(P.schur_ptr);
  m.o_so = pk.addv(P.schur_off);
  m.o_uo = pk.addv(P.u_off);
  m.o_lo = pk.addv(P.l_off);
  m.o_wo = pk.addv(P.w_off);
  m.o_vo = pk.addv(P.vec_off);
  m.o_dp = pk.addv(P.dep_ptr);
  m.o_di = pk.addv(P.dep_idx);
  m.o_rp = pk.addv(P.rdep_ptr);
  m.o_ri = pk.addv(P.rdep_idx);
  bytes = pk.size;
  void* d = dalloc(bytes, s);
  pk.upload(d, s);
  return d;
}

void set_static(LevelDev& D, const void* meta, const StaticMeta& m) {
  const char* b = static_cast<const char*>(meta);
  D.n = reinterpret_cast<const int*>(b + m.o_n);
  D.colour = reinterpret_cast<const int*>(b + m.o_col);
  D.order = reinterpret_cast<const int*>(b + m.o_order);
  D.close_ptr = reinterpret_cast<const int*>(b + m.o_cp);
  D.close_blk = reinterpret_cast<const int*>(b + m.o_cb);
  D.close_off = reinterpret_cast<const int64_t*>(b + m.o_co);
  D.far_ptr = reinterpret_cast<const int*>(b + m.o_fp);
  D.far_blk = reinterpret_cast<const int*>(b + m.o_fb);
  D.far_off = reinterpret_cast<const int64_t*>(b + m.o_fo);
  D.diag_off = reinterpret_cast<const int64_t*>(b + m.o_do);
  D.schur_ptr = reinterpret_cast<const int*>(b + m.o_sp);
  D.schur_off = reinterpret_cast<const int64_t*>(b + m.o_so);
  D.u_off = reinterpret_cast<const int64_t*>(b + m.o_uo);
  D.l_off = reinterpret_cast<const int64_t*>(b + m.o_lo);
  D.w_off = reinterpret_cast<const int64_t*>(b + m.o_wo);
  D.vec_off = reinterpret_cast<const int64_t*>(b + m.o_vo);
  D.dep_ptr = reinterpret_cast<const int*>(b + m.o_dp);
  D.dep_idx = reinterpret_cast<const int*>(b + m.o_di);
  D.rdep_ptr = reinterpret_cast<const int*>(b + m.o_rp);
  D.rdep_idx = reinterpret_cast<const int*>(b + m.o_ri);
}

// Metadata and factor storage of a level.  `shared` (level 1 of a csb) holds
// the plan's fixed arrays already on the device; otherwise they are uploaded
// into the level's own block.
void build_level_store(LevelStore& st, int esize, cudaStream_t s, const void* shared = nullptr,
                       const StaticMeta* shared_m = nullptr) {
  const LevelPlan& P = *st.plan;
  LevelDev& D = st.dev;
  D.M = P.M;
  size_t sbytes = 0;
  if (shared) {
    st.smeta = nullptr;
    set_static(D, shared, *shared_m);
  } else {
    StaticMeta m;
    st.smeta = upload_static_meta(P, m, sbytes, s);
    set_static(D, st.smeta, m);
  }
  // per-factorization state, one zero-filled block
  Packer pk;
  const size_t o_rank = pk.zeros(P.M * sizeof(int)), o_done = pk.zeros(P.M * sizeof(int)),
               o_fd = pk.zeros(P.M * sizeof(int)), o_bd = pk.zeros(P.M * sizeof(int)),
               o_q = pk.zeros(ce::kBuckets * sizeof(int)),
               o_gd = pk.zeros(P.M * sizeof(int64_t)), o_tau = pk.zeros(P.M * sizeof(double)),
               o_sig = pk.zeros(P.vec_len * sizeof(double)), o_kw = pk.zeros(P.M * sizeof(int)),
               o_feat = pk.zeros((size_t)P.M * ce::kMlpFeatures * sizeof(float));
  st.meta_bytes = pk.size + sbytes;
  st.meta = dalloc(pk.size, s);
  check(cudaMemsetAsync(st.meta, 0, pk.size, s), "memset level state");
  char* b = static_cast<char*>(st.meta);
  D.rank = reinterpret_cast<int*>(b + o_rank);
  D.gdst = reinterpret_cast<int64_t*>(b + o_gd);
  D.tau = reinterpret_cast<double*>(b + o_tau);
  D.sigma = reinterpret_cast<double*>(b + o_sig);
  D.done = reinterpret_cast<int*>(b + o_done);
  D.qnext = reinterpret_cast<int*>(b + o_q);
  D.fdone = reinterpret_cast<int*>(b + o_fd);
  D.bdone = reinterpret_cast<int*>(b + o_bd);
  D.wait_ns = 2000000000ull;  // 2 s: never reached unless a row's neighbours stall
  D.accumulate = P.coloring == 2 ? 1 : 0;
  D.kw = reinterpret_cast<int*>(b + o_kw);
  D.feat = reinterpret_cast<float*>(b + o_feat);
  D.aq = nullptr;
  D.epoch = nullptr;
  D.prof = nullptr;
  const size_t ub = P.u_elems * esize, lb = P.l_elems * esize, wb = P.w_elems * esize;
  st.fac_bytes = ub + lb + wb + 3 * 256;
  st.fac = dalloc(st.fac_bytes, s);
  char* f = static_cast<char*>(st.fac);
  D.U = f;
  D.L = f + ((ub + 255) & ~size_t(255));
  D.W = static_cast<char*>(D.L) + ((lb + 255) & ~size_t(255));
  D.pool = nullptr;
}

// copy tasks: level pairs (kept corners) -> next level pairs
std::vector<std::vector<CopyTask>> reassembly_tasks(const LevelPlan& P, const std::vector<int>& rank, int J,
                                       const ce::NextLevel& nx, const LevelPlan& Pn) {
  const int64_t np = static_cast<int64_t>(P.pair_i.size());
  const int nch = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ce::host_threads() * 4, np / 8192)));
  std::vector<std::vector<CopyTask>> part(nch);
  ce::parallel_for(nch, 1, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      std::vector<CopyTask>& tasks = part[c];
      for (int64_t p = np * c / nch; p < np * (c + 1) / nch; ++p) {
        const int i = P.pair_i[p], k = P.pair_k[p];
        if (rank[i] == 0 || rank[k] == 0) continue;
        const int I = nx.parent[i], K = nx.parent[k];
        CopyTask t;
        t.src_off = P.pair_off[p];
        t.src_ld = P.n[k];
        t.rows = rank[i];
        t.cols = rank[k];
        t.dst_off = pair_offset(Pn, I, K);
        t.dst_ld = Pn.n[K];
        t.r0 = nx.child_off[i];
        t.c0 = nx.child_off[k];
        t.transpose = 0;
        tasks.push_back(t);
        if (I == K && i != k) {
          t.r0 = nx.child_off[k];
          t.c0 = nx.child_off[i];
          t.transpose = 1;
          tasks.push_back(t);
        }
      }
    }
  });
  return part;
}

// Coarse systems of the last level: system s owns blocks [so[s], so[s+1]),
// coarse rows [voff[s], voff[s] + nc[s]) and a dense nc x nc matrix at coff[s].
struct CoarseSystems {
  std::vector<int> so, sys_of;
  std::vector<int64_t> nc, coff, voff, doff;
  int64_t dense_elems = 0, dinv_elems = 0;
  int nmax = 0;
};

CoarseSystems coarse_systems(const LevelPlan& P) {
  CoarseSystems C;
  C.so = P.sys_off.empty() ? std::vector<int>{0, P.M} : P.sys_off;
  const int ns = static_cast<int>(C.so.size()) - 1;
  C.sys_of.assign(P.M, 0);
  for (int y = 0; y < ns; ++y) {
    for (int i = C.so[y]; i < C.so[y + 1]; ++i) C.sys_of[i] = y;
    const int64_t v0 = C.so[y] < P.M ? P.vec_off[C.so[y]] : P.vec_len;
    const int64_t v1 = C.so[y + 1] < P.M ? P.vec_off[C.so[y + 1]] : P.vec_len;
    C.voff.push_back(v0);
    C.nc.push_back(v1 - v0);
    C.coff.push_back(C.dense_elems);
    C.doff.push_back(C.dinv_elems);
    C.dense_elems += (v1 - v0) * (v1 - v0);
    C.dinv_elems += (v1 - v0 + 63) / 64 * 64 * 64;
    C.nmax = std::max<int>(C.nmax, static_cast<int>(v1 - v0));
  }
  return C;
}

// copy tasks: close pairs of a level -> one dense symmetric matrix per system
std::vector<CopyTask> dense_tasks(const LevelPlan& P, const CoarseSystems& C) {
  std::vector<CopyTask> tasks;
  for (size_t p = 0; p < P.pair_i.size(); ++p) {
    if (!P.pair_close[p]) continue;
    const int i = P.pair_i[p], k = P.pair_k[p];
    if (P.n[i] == 0 || P.n[k] == 0) continue;
    const int y = C.sys_of[i];
    if (C.sys_of[k] != y) throw std::logic_error("coupling between independent systems");
    CopyTask t;
    t.src_off = P.pair_off[p];
    t.src_ld = P.n[k];
    t.rows = P.n[i];
    t.cols = P.n[k];
    t.dst_off = C.coff[y];
    t.dst_ld = static_cast<int>(C.nc[y]);
    t.r0 = static_cast<int>(P.vec_off[i] - C.voff[y]);
    t.c0 = static_cast<int>(P.vec_off[k] - C.voff[y]);
    t.transpose = 0;
    tasks.push_back(t);
    if (i != k) {
      t.r0 = static_cast<int>(P.vec_off[k] - C.voff[y]);
      t.c0 = static_cast<int>(P.vec_off[i] - C.voff[y]);
      t.transpose = 1;
      tasks.push_back(t);
    }
  }
  return tasks;
}

// copy tasks given in parts (filled by separate host threads), gathered into
// the pinned staging buffer in parallel and run by one launch
void run_copy_tasks(const std::vector<std::vector<CopyTask>>& parts, int es, int ed, const void* src, void* dst,
                    cudaStream_t s) {
  std::vector<size_t> off(parts.size() + 1, 0);
  for (size_t c = 0; c < parts.size(); ++c) off[c + 1] = off[c] + parts[c].size();
  const size_t ntasks = off.back();
  if (ntasks == 0) return;
  const size_t bytes = ntasks * sizeof(CopyTask);
  void* dt = dalloc(bytes, s);
  CopyTask* h = reinterpret_cast<CopyTask*>(stage_get(1, bytes));
  ce::parallel_for(static_cast<int64_t>(parts.size()), 1, [&](int64_t b, int64_t e) {
    for (int64_t c = b; c < e; ++c) std::copy(parts[c].begin(), parts[c].end(), h + off[c]);
  });
  stage_upload(1, dt, bytes, s);
  check(ce::launch_copy_tasks(es, ed, static_cast<const CopyTask*>(dt), (int)ntasks, src, dst, s), "copy tasks");
  dfree(dt, s);
}

void run_copy_tasks(const std::vector<CopyTask>& tasks, int es, int ed, const void* src, void* dst,
                    cudaStream_t s) {
  run_copy_tasks(std::vector<std::vector<CopyTask>>{tasks}, es, ed, src, dst, s);
}

void free_factor(ce_factor* F, cudaStream_t s) {
  if (!F) return;
  for (auto& st : F->levels) {
    dfree(st.meta, s);
    dfree(st.smeta, s);
    dfree(st.fac, s);
  }
  dfree(F->d_coarse, s);
  dfree(F->d_cdinv, s);
  dfree(F->d_csys, s);
  dfree(F->d_apply, s);
  if (F->pcg) {
    cudaDeviceSynchronize();
    ce::pcg_batch_release(F->pcg);
    F->pcg = nullptr;
  }
  dfree(F->d_work, s);
  dfree(F->d_status, s);
  if (F->owned_csb) ce_csb_destroy(F->owned_csb);
  delete F;
}

}  // namespace

extern "C" {

void ce_opts_default(ce_opts* o) {
  if (!o) return;
  o->tol = 1e-4;
  o->tol_mode = CE_TOL_REL;
  o->levels = 4;
  o->J = 4;
  o->precision = CE_PREC_FP64;
  o->coloring = 1;
  o->stream = nullptr;
  o->rank_mode = CE_RANK_SVD;
  o->rank_model = nullptr;
  o->oversample = 8;
  o->seed = 0;
  o->row_shape = -1;
  o->rank = 16;
  o->nmax = 0;
  o->record_features = 0;
  o->gemm_engine = 0;
}

const char* ce_strerror(ce_status s) {
  switch (s) {
    case CE_OK: return "ok";
    case CE_ERR_INVALID_ARG: return "invalid argument";
    case CE_ERR_NOT_SPD: return "pivot block not positive definite";
    case CE_ERR_NO_CONVERGENCE: return "PCG did not converge";
    case CE_ERR_OOM: return "device out of memory";
    case CE_ERR_CUDA: return "CUDA error";
    case CE_ERR_LIMIT: return "block size limit exceeded";
  }
  return "unknown status";
}

const char* ce_last_error(void) { return g_last_error.c_str(); }

int64_t ce_launch_count(void) { return ce::g_launches.load(); }

ce_status ce_measure_peak(int kind, double* tflops, void* stream) {
  if (kind < 0 || kind > 3 || !tflops) return CE_ERR_INVALID_ARG;
  try {
    check(ce::measure_peak(kind, tflops, static_cast<cudaStream_t>(stream)), "peak probe");
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

int ce_mlp_nparams(void) { return ce::kMlpParams; }
int ce_mlp_nfeatures(void) { return ce::kMlpFeatures; }

ce_status ce_mlp_init(float* theta_dev, uint64_t seed, void* stream) {
  if (!theta_dev) return CE_ERR_INVALID_ARG;
  try {
    check(ce::mlp_init(theta_dev, seed, static_cast<cudaStream_t>(stream)), "mlp init");
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status ce_mlp_grad(const float* X_dev, const float* t_dev, int ns, const float* theta_dev,
                      float* grad_dev, void* stream) {
  if (!X_dev || !t_dev || !theta_dev || !grad_dev || ns <= 0) return CE_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = nullptr;
  ce_status ret = CE_OK;
  try {
    part = static_cast<float*>(dalloc((size_t)ce::mlp_partial_blocks(ns) * ce::kMlpParams * 4, s));
    check(ce::mlp_grad(X_dev, t_dev, ns, theta_dev, part, grad_dev, s), "mlp grad");
  } catch (...) {
    ret = status_of_exception();
  }
  dfree(part, s);
  return ret;
}

ce_status ce_mlp_train(const float* X_dev, const float* t_dev, int ns, float* theta_dev, int steps,
                       float lr, double* loss_out, void* stream) {
  if (!X_dev || !t_dev || !theta_dev || ns <= 0 || steps < 0 || !(lr > 0.f)) return CE_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float *part = nullptr, *m = nullptr, *v = nullptr, *pred = nullptr;
  ce_status ret = CE_OK;
  try {
    part = static_cast<float*>(dalloc((size_t)ce::mlp_partial_blocks(ns) * ce::kMlpParams * 4, s));
    m = static_cast<float*>(dalloc(ce::kMlpParams * 4, s));
    v = static_cast<float*>(dalloc(ce::kMlpParams * 4, s));
    check(cudaMemsetAsync(m, 0, ce::kMlpParams * 4, s), "memset");
    check(cudaMemsetAsync(v, 0, ce::kMlpParams * 4, s), "memset");
    for (int it = 1; it <= steps; ++it)
      check(ce::mlp_adam_step(X_dev, t_dev, ns, theta_dev, part, m, v, lr, it, s), "mlp adam");
    if (loss_out) {
      // loss of the FP32 parameters through the FP16 model the row kernel uses
      void* model = dalloc((size_t)ce::kMlpParams * 2, s);
      pred = static_cast<float*>(dalloc((size_t)ns * 4, s));
      check(ce::mlp_pack(theta_dev, model, s), "mlp pack");
      check(ce::mlp_predict(X_dev, ns, model, pred, s), "mlp predict");
      std::vector<float> hp(ns), ht(ns);
      check(cudaMemcpyAsync(hp.data(), pred, ns * 4, cudaMemcpyDeviceToHost, s), "D2H");
      check(cudaMemcpyAsync(ht.data(), t_dev, ns * 4, cudaMemcpyDeviceToHost, s), "D2H");
      check(cudaStreamSynchronize(s), "sync");
      double acc = 0;
      for (int k = 0; k < ns; ++k) acc += 0.5 * double(hp[k] - ht[k]) * double(hp[k] - ht[k]);
      *loss_out = acc / ns;
      dfree(model, s);
    }
  } catch (...) {
    ret = status_of_exception();
  }
  dfree(part, s);
  dfree(m, s);
  dfree(v, s);
  dfree(pred, s);
  return ret;
}

ce_status ce_mlp_pack(const float* theta_dev, void* model_dev, void* stream) {
  if (!theta_dev || !model_dev) return CE_ERR_INVALID_ARG;
  try {
    check(ce::mlp_pack(theta_dev, model_dev, static_cast<cudaStream_t>(stream)), "mlp pack");
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status ce_mlp_predict(const float* X_dev, int ns, const void* model_dev, float* out_dev, void* stream) {
  if (!X_dev || !model_dev || !out_dev || ns < 0) return CE_ERR_INVALID_ARG;
  try {
    check(ce::mlp_predict(X_dev, ns, model_dev, out_dev, static_cast<cudaStream_t>(stream)), "mlp predict");
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

}  // extern "C"

namespace {

// CSR + permutation + block pointers (+ systems) -> device CSB and level-1 plan.
ce_status build_csb(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                    const int32_t* perm, const std::vector<int64_t>& blkptr,
                    const std::vector<int>& sys_blk, const std::vector<int64_t>& sys_row, int B0,
                    ce_csb** out) {
  const int64_t nnz = rowptr[n];
  // perm is a permutation; every column in range (read-only, in parallel)
  std::vector<int32_t> iperm(n, -1);
  for (int64_t k = 0; k < n; ++k) {
    if (perm[k] < 0 || perm[k] >= n || iperm[perm[k]] != -1) return CE_ERR_INVALID_ARG;
    iperm[perm[k]] = static_cast<int32_t>(k);
  }
  std::atomic<bool> bad{false};
  ce::parallel_for(nnz, 1 << 18, [&](int64_t b, int64_t e) {
    for (int64_t q = b; q < e && !bad.load(std::memory_order_relaxed); ++q)
      if (col[q] < 0 || col[q] >= n) bad.store(true);
  });
  if (bad.load()) return CE_ERR_INVALID_ARG;
  if (!csr_symmetric(n, rowptr, col, val)) return CE_ERR_INVALID_ARG;
  const int M = static_cast<int>(blkptr.size()) - 1;
  std::vector<int> sizes(M);
  std::vector<int> blk_of(n);
  for (int b2 = 0; b2 < M; ++b2) {
    sizes[b2] = static_cast<int>(blkptr[b2 + 1] - blkptr[b2]);
    for (int64_t r = blkptr[b2]; r < blkptr[b2 + 1]; ++r) blk_of[r] = b2;
  }
  std::vector<std::pair<int, int>> pairs = block_pairs(rowptr, col, perm, iperm, blkptr, blk_of);
  ce_csb* A = new (std::nothrow) ce_csb();
  if (!A) return CE_ERR_OOM;
  A->n = n;
  A->B = B0;
  A->nnz = nnz;
  // host copy of the pattern (csb_update_values checks new values against
  // it), filled in parallel
  A->h_rowptr.resize(n + 1);
  A->h_col.resize(nnz);
  ce::parallel_for(n + 1, 1 << 16, [&](int64_t b, int64_t e) {
    std::memcpy(A->h_rowptr.data() + b, rowptr + b, (e - b) * sizeof(int64_t));
  });
  ce::parallel_for(nnz, 1 << 17, [&](int64_t b, int64_t e) {
    std::memcpy(A->h_col.data() + b, col + b, (e - b) * sizeof(int32_t));
  });
  A->nsys = static_cast<int>(sys_row.size()) - 1;
  A->sys_row = sys_row;
  try {
    A->plan1 = std::make_shared<LevelPlan>();
    ce::plan_level(*A->plan1, sizes, pairs, true, sys_blk);
    const LevelPlan& P1 = *A->plan1;
    // every entry is written below (-1: the mirror of a stored pair), so the
    // array is not zero-filled first
    std::unique_ptr<int64_t[]> scatter(new int64_t[std::max<int64_t>(nnz, 1)]);
    ce::parallel_for(n, 8192, [&](int64_t a0, int64_t a1) {
      for (int64_t a = a0; a < a1; ++a)
        for (int64_t e = rowptr[a]; e < rowptr[a + 1]; ++e) {
          const int pa = iperm[a], pb = iperm[col[e]];
          const int bi = blk_of[pa], bk = blk_of[pb];
          if (bi > bk) {
            scatter[e] = -1;
            continue;
          }
          const int64_t po = pair_offset(P1, bi, bk);
          scatter[e] = po + (int64_t)(pa - blkptr[bi]) * P1.n[bk] + (pb - blkptr[bk]);
        }
    });
    std::vector<int32_t> sys_of_row(n);
    for (int s2 = 0; s2 < A->nsys; ++s2)
      for (int64_t r = sys_row[s2]; r < sys_row[s2 + 1]; ++r) sys_of_row[r] = s2;
    init_pool_once();
    cudaStream_t s = nullptr;
    A->d_rowptr = static_cast<int64_t*>(dalloc((n + 1) * sizeof(int64_t), s));
    A->d_col = static_cast<int32_t*>(dalloc(nnz * sizeof(int32_t), s));
    A->d_val = static_cast<double*>(dalloc(nnz * sizeof(double), s));
    A->d_perm = static_cast<int32_t*>(dalloc(n * sizeof(int32_t), s));
    A->d_scatter = static_cast<int64_t*>(dalloc(nnz * sizeof(int64_t), s));
    A->d_sys_of_row = static_cast<int32_t*>(dalloc(n * sizeof(int32_t), s));
    // all arrays through one pinned staging buffer (copied in parallel)
    struct Up {
      void* dst;
      const void* src;
      size_t bytes;
    } ups[] = {{A->d_rowptr, rowptr, (n + 1) * sizeof(int64_t)},
               {A->d_col, col, nnz * sizeof(int32_t)},
               {A->d_val, val, nnz * sizeof(double)},
               {A->d_perm, perm, n * sizeof(int32_t)},
               {A->d_scatter, scatter.get(), nnz * sizeof(int64_t)},
               {A->d_sys_of_row, sys_of_row.data(), n * sizeof(int32_t)}};
    size_t off[7] = {0};
    for (int u = 0; u < 6; ++u) off[u + 1] = off[u] + ((ups[u].bytes + 255) & ~size_t(255));
    char* h = stage_get(1, off[6]);
    ce::parallel_for(6 * 16, 1, [&](int64_t b, int64_t e) {
      for (int64_t t = b; t < e; ++t) {  // 16 slices per array
        const int u = static_cast<int>(t / 16), q = static_cast<int>(t % 16);
        const size_t lo = ups[u].bytes * q / 16, hi = ups[u].bytes * (q + 1) / 16;
        std::memcpy(h + off[u] + lo, static_cast<const char*>(ups[u].src) + lo, hi - lo);
      }
    });
    for (int u = 0; u < 6; ++u)
      check(cudaMemcpyAsync(ups[u].dst, h + off[u], ups[u].bytes, cudaMemcpyHostToDevice, s), "H2D");
    check(cudaEventRecord(g_stage[1].ev, s), "event");
    g_stage[1].pending = true;
    size_t mb = 0;
    A->d_meta1 = upload_static_meta(*A->plan1, A->meta1_off, mb, s);
    check(cudaStreamSynchronize(s), "csb_build sync");
  } catch (const CudaFail& f) {
    ce_csb_destroy(A);
    return status_of(f);
  } catch (const std::bad_alloc&) {
    ce_csb_destroy(A);
    return CE_ERR_OOM;
  } catch (const std::exception& ex) {
    g_last_error = ex.what();
    ce_csb_destroy(A);
    return CE_ERR_INVALID_ARG;
  }
  *out = A;
  return CE_OK;
}

}  // namespace

extern "C" {

ce_status csb_build(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                    const int32_t* perm, int32_t B, ce_csb** out) {
  if (!out || n <= 0 || !rowptr || !col || !val || !perm || B <= 0 || n > INT32_MAX)
    return CE_ERR_INVALID_ARG;
  *out = nullptr;
  if (rowptr[0] != 0 || rowptr[n] < 0) return CE_ERR_INVALID_ARG;
  for (int64_t a = 0; a < n; ++a)
    if (rowptr[a + 1] < rowptr[a]) return CE_ERR_INVALID_ARG;
  const int M = static_cast<int>((n + B - 1) / B);
  std::vector<int64_t> blkptr(M + 1);
  for (int b2 = 0; b2 <= M; ++b2) blkptr[b2] = std::min<int64_t>(n, (int64_t)b2 * B);
  return build_csb(n, rowptr, col, val, perm, blkptr, {0, M}, {0, n}, B, out);
}

ce_status csb_build_batched(int nsys, const int64_t* row_off, const int64_t* rowptr, const int32_t* col,
                            const double* val, const int32_t* perm, const int32_t* B, ce_csb** out) {
  if (!out || nsys <= 0 || !row_off || !rowptr || !col || !val || !perm || !B) return CE_ERR_INVALID_ARG;
  *out = nullptr;
  const int64_t n = row_off[nsys];
  if (row_off[0] != 0 || n <= 0 || n > INT32_MAX || rowptr[0] != 0) return CE_ERR_INVALID_ARG;
  for (int64_t a = 0; a < n; ++a)
    if (rowptr[a + 1] < rowptr[a]) return CE_ERR_INVALID_ARG;
  std::vector<int64_t> blkptr{0};
  std::vector<int> sys_blk{0};
  std::vector<int64_t> sys_row(row_off, row_off + nsys + 1);
  for (int s2 = 0; s2 < nsys; ++s2)
    if (row_off[s2 + 1] <= row_off[s2] || B[s2] <= 0) return CE_ERR_INVALID_ARG;
  // the batch is block diagonal: each system's permutation and columns stay
  // inside its own rows (systems checked in parallel)
  std::atomic<bool> bad{false};
  ce::parallel_for(nsys, 1, [&](int64_t s0, int64_t s1) {
    for (int64_t s2 = s0; s2 < s1 && !bad.load(std::memory_order_relaxed); ++s2) {
      const int64_t r0 = row_off[s2], r1 = row_off[s2 + 1];
      for (int64_t k = r0; k < r1; ++k) {
        if (perm[k] < r0 || perm[k] >= r1) bad.store(true);
        for (int64_t e = rowptr[k]; e < rowptr[k + 1]; ++e)
          if (col[e] < r0 || col[e] >= r1) bad.store(true);
      }
    }
  });
  if (bad.load()) return CE_ERR_INVALID_ARG;
  for (int s2 = 0; s2 < nsys; ++s2) {
    const int64_t r0 = row_off[s2], r1 = row_off[s2 + 1];
    for (int64_t r = r0 + B[s2]; r < r1; r += B[s2]) blkptr.push_back(r);
    blkptr.push_back(r1);
    sys_blk.push_back(static_cast<int>(blkptr.size()) - 1);
  }
  const ce_status st = build_csb(n, rowptr, col, val, perm, blkptr, sys_blk, sys_row, B[0], out);
  if (st == CE_OK) (*out)->batched = true;
  return st;
}

void ce_csb_destroy(ce_csb* A) {
  if (!A) return;
  cudaStream_t s = nullptr;
  dfree(A->d_rowptr, s);
  dfree(A->d_col, s);
  dfree(A->d_val, s);
  dfree(A->d_perm, s);
  dfree(A->d_scatter, s);
  dfree(A->d_sys_of_row, s);
  dfree(A->d_meta1, s);
  delete A;
}

ce_status ce_plan_groups(int M, const int32_t* rank, int J, int nmax, int32_t* first_child, int* ngroups) {
  if (M < 1 || J < 1 || nmax < 0 || !rank || !first_child || !ngroups) return CE_ERR_INVALID_ARG;
  for (int i = 0; i < M; ++i)
    if (rank[i] < 0) return CE_ERR_INVALID_ARG;
  try {
    ce::LevelPlan P;
    P.M = M;
    const std::vector<int> r(rank, rank + M);
    std::vector<int> fc;
    ce::coarsen_parents(P, J, &r, nmax, &fc, nullptr);
    std::copy(fc.begin(), fc.end(), first_child);
    *ngroups = static_cast<int>(fc.size()) - 1;
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

}  // extern "C"

namespace {

// Level-1 symbolic plan of host CSR + permutation, no CUDA call (the host
// introspection entry points below); may throw std::bad_alloc.
ce_status plan1_host(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm, int32_t B,
                     LevelPlan& P, int coloring = 1) {
  if (n <= 0 || !rowptr || !col || !perm || B <= 0 || n > INT32_MAX || rowptr[0] != 0)
    return CE_ERR_INVALID_ARG;
  std::vector<int32_t> iperm(n, -1);
  for (int64_t k = 0; k < n; ++k) {
    if (perm[k] < 0 || perm[k] >= n || iperm[perm[k]] != -1) return CE_ERR_INVALID_ARG;
    iperm[perm[k]] = static_cast<int32_t>(k);
  }
  for (int64_t e = 0; e < rowptr[n]; ++e)
    if (col[e] < 0 || col[e] >= n) return CE_ERR_INVALID_ARG;
  const int M = static_cast<int>((n + B - 1) / B);
  std::vector<int> sizes(M, B);
  sizes[M - 1] = static_cast<int>(n - (int64_t)(M - 1) * B);
  std::vector<int64_t> blkptr(M + 1);
  std::vector<int> blk_of(n);
  for (int b2 = 0; b2 <= M; ++b2) blkptr[b2] = std::min<int64_t>(n, (int64_t)b2 * B);
  for (int64_t r = 0; r < n; ++r) blk_of[r] = static_cast<int>(r / B);
  std::vector<std::pair<int, int>> pairs = block_pairs(rowptr, col, perm, iperm, blkptr, blk_of);
  ce::plan_level(P, sizes, pairs, coloring);
  return CE_OK;
}

}  // namespace

extern "C" {

ce_status ce_plan_level1(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm,
                         int32_t B, int32_t* colour, int* ncolours, int64_t* npairs, int64_t* nclose) {
  try {
    LevelPlan P;
    const ce_status st = plan1_host(n, rowptr, col, perm, B, P);
    if (st != CE_OK) return st;
    if (colour) std::copy(P.colour.begin(), P.colour.end(), colour);
    if (ncolours) *ncolours = P.ncolours;
    if (npairs) *npairs = static_cast<int64_t>(P.pair_i.size());
    if (nclose) {
      int64_t c = 0;
      for (char x : P.pair_close) c += x;
      *nclose = c;
    }
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status ce_plan_colours(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm, int32_t B,
                          int coloring, int32_t* colour, int* ncolours) {
  if (coloring < 0 || coloring > 2) return CE_ERR_INVALID_ARG;
  try {
    LevelPlan P;
    const ce_status st = plan1_host(n, rowptr, col, perm, B, P, coloring);
    if (st != CE_OK) return st;
    if (colour) std::copy(P.colour.begin(), P.colour.end(), colour);
    if (ncolours) *ncolours = P.ncolours;
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status ce_plan_level1_deps(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm,
                              int32_t B, int64_t* dep_ptr, int32_t* dep_idx, int64_t cap, int64_t* ndeps) {
  try {
    LevelPlan P;
    const ce_status st = plan1_host(n, rowptr, col, perm, B, P);
    if (st != CE_OK) return st;
    const int64_t total = P.dep_ptr[P.M];
    if (ndeps) *ndeps = total;
    if (dep_idx && cap < total) return CE_ERR_INVALID_ARG;
    if (dep_ptr) std::copy(P.dep_ptr.begin(), P.dep_ptr.end(), dep_ptr);
    if (dep_idx) std::copy(P.dep_idx.begin(), P.dep_idx.end(), dep_idx);
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status ce_plan_next_level(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm,
                             int32_t B, const int32_t* rank, int J, int nmax, int32_t* next_n,
                             int32_t* next_colour, int* next_M, int64_t* next_nclose) {
  if (!rank || J < 1 || nmax < 0 || !next_M) return CE_ERR_INVALID_ARG;
  try {
    LevelPlan P;
    const ce_status st = plan1_host(n, rowptr, col, perm, B, P);
    if (st != CE_OK) return st;
    std::vector<int> r(rank, rank + P.M);
    for (int i = 0; i < P.M; ++i)
      if (r[i] < 0 || r[i] > P.n[i]) return CE_ERR_INVALID_ARG;
    const ce::NextLevel nx = ce::coarsen(P, r, J, nmax);
    LevelPlan P2;
    ce::plan_level(P2, nx.n, nx.pairs, true);
    *next_M = P2.M;
    if (next_n) std::copy(nx.n.begin(), nx.n.end(), next_n);
    if (next_colour) std::copy(P2.colour.begin(), P2.colour.end(), next_colour);
    if (next_nclose) {
      int64_t c = 0;
      for (char x : P2.pair_close) c += x;
      *next_nclose = c;
    }
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status ce_plan_level1_work(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm,
                              int32_t B, const int32_t* rank, int esize, double* flops, double* bytes) {
  if (!rank || (esize != 4 && esize != 8) || !flops || !bytes) return CE_ERR_INVALID_ARG;
  try {
    LevelPlan P;
    const ce_status st = plan1_host(n, rowptr, col, perm, B, P);
    if (st != CE_OK) return st;
    std::vector<int> r(rank, rank + P.M);
    for (int i = 0; i < P.M; ++i)
      if (r[i] < 0 || r[i] > P.n[i]) return CE_ERR_INVALID_ARG;
    level_work(P, r, esize, *flops, *bytes);
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status csb_get_tuning(const ce_csb* A, int precision, int rank_mode, int* levels, int32_t* shape,
                         int32_t* learned) {
  if (!A || !levels || precision < 0 || precision > 1 || rank_mode < 0 || rank_mode > 1) return CE_ERR_INVALID_ARG;
  *levels = A->tuned_levels[precision][rank_mode];
  for (int l = 0; l < 16; ++l) {
    if (shape) shape[l] = A->tuned_shape[precision][rank_mode][l];
    if (learned) learned[l] = A->tuned_learned[precision][rank_mode][l];
  }
  return CE_OK;
}

ce_status csb_set_tuning(ce_csb* A, int precision, int rank_mode, int levels, const int32_t* shape,
                         const int32_t* learned) {
  if (!A || precision < 0 || precision > 1 || rank_mode < 0 || rank_mode > 1 || levels < 0 || levels > 16 ||
      (levels > 0 && (!shape || !learned)))
    return CE_ERR_INVALID_ARG;
  for (int l = 0; l < levels; ++l)
    if (shape[l] < 0 || shape[l] > 3 || (learned[l] != 0 && learned[l] != 1)) return CE_ERR_INVALID_ARG;
  for (int l = 0; l < 16; ++l) {
    A->tuned_shape[precision][rank_mode][l] = l < levels ? shape[l] : 0;
    A->tuned_learned[precision][rank_mode][l] = l < levels ? learned[l] : 0;
  }
  A->tuned_levels[precision][rank_mode] = levels;
  return CE_OK;
}

int csb_blocks(const ce_csb* A) { return A ? A->plan1->M : 0; }

ce_status csb_get_colours(const ce_csb* A, int32_t* colour, int* ncolours) {
  if (!A) return CE_ERR_INVALID_ARG;
  if (colour) std::copy(A->plan1->colour.begin(), A->plan1->colour.end(), colour);
  if (ncolours) *ncolours = A->plan1->ncolours;
  return CE_OK;
}

ce_status ce_factorize(const ce_csb* A, const ce_opts* o_in, ce_factor** out, ce_info* info) {
  if (!A || !out) return CE_ERR_INVALID_ARG;
  ce_opts o;
  ce_opts_default(&o);
  if (o_in) o = *o_in;
  if (o.levels < 0 || o.J < 1 || o.tol < 0 || (o.precision != CE_PREC_FP64 && o.precision != CE_PREC_FP32) ||
      (o.tol_mode != CE_TOL_REL && o.tol_mode != CE_TOL_ABS && o.tol_mode != CE_TOL_FIXED) ||
      (o.tol_mode == CE_TOL_FIXED && (o.rank < 0 || o.rank_mode != CE_RANK_SVD)) ||
      (o.rank_mode != CE_RANK_SVD && o.rank_mode != CE_RANK_LEARNED) ||
      (o.rank_mode == CE_RANK_LEARNED && (!o.rank_model || o.oversample < 0)) || o.row_shape < -1 ||
      o.row_shape > 3 || o.nmax < 0 || o.gemm_engine < 0 || o.gemm_engine > 2 || o.coloring < 0 ||
      o.coloring > 2)
    return CE_ERR_INVALID_ARG;
  // CE(r): the row kernel takes r in place of the tolerance
  if (o.tol_mode == CE_TOL_FIXED) o.tol = static_cast<double>(o.rank);
  *out = nullptr;
  if (info) std::memset(info, 0, sizeof(*info));
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t) {
    return std::chrono::duration<double, std::milli>(clk::now() - t).count();
  };
  const clk::time_point t_call = clk::now();
  cudaStream_t s = static_cast<cudaStream_t>(o.stream);
  init_pool_once();
  ce_factor* F = new (std::nothrow) ce_factor();
  if (!F) return CE_ERR_OOM;
  F->N = A->n;
  F->prec = o.precision;
  F->esize = (o.precision == CE_PREC_FP64) ? 8 : 4;
  F->d_perm = A->d_perm;
  const int es = F->esize;
  void* pool = nullptr;
  ce_status ret = CE_OK;
  try {
    // status words, counters, then the row-phase cycle sums (16 levels)
    const size_t status_bytes = (ce::kStatusWords + ce::kStatsWords) * sizeof(int) +
                                16 * ce::kProfSlots * sizeof(unsigned long long);
    F->d_status = static_cast<int*>(dalloc(status_bytes, s));
    check(cudaMemsetAsync(F->d_status, 0, status_bytes, s), "memset");
    unsigned long long* d_prof =
        reinterpret_cast<unsigned long long*>(F->d_status + ce::kStatusWords + ce::kStatsWords);
    ce::LearnedArgs la;
    if (o.rank_mode == CE_RANK_LEARNED) la.model = static_cast<const __half*>(o.rank_model);
    la.oversample = o.oversample;
    la.J = o.J;
    la.seed = o.seed;
    la.stats = F->d_status + ce::kStatusWords;
    la.record = o.record_features != 0;
    std::shared_ptr<const LevelPlan> curp;
    if (o.coloring == 1) {
      curp = A->plan1;
    } else {   // natural order or distance-1 colours: the same pairs, another order
      const LevelPlan& P1 = *A->plan1;
      std::vector<std::pair<int, int>> pr;
      for (size_t p = 0; p < P1.pair_i.size(); ++p)
        if (P1.pair_close[p]) pr.emplace_back(P1.pair_i[p], P1.pair_k[p]);
      auto np = std::make_shared<LevelPlan>();
      ce::plan_level(*np, P1.n, pr, o.coloring, P1.sys_off);
      curp = np;
    }
    pool = dalloc(curp->pool_elems * es, s);
    check(cudaMemsetAsync(pool, 0, curp->pool_elems * es, s), "memset pool");
    check(ce::launch_scatter_csr(es, A->d_scatter, A->d_val, A->nnz, pool, s), "scatter");
    int hstatus[ce::kStatusWords];
    for (int l = 0; l < o.levels && curp->M > 0; ++l) {
      // levels whose rows outgrow the row kernel run the large-row path (and
      // so does a level whose shape is 3, forced or autotuned)
      bool big = ce::level_needs_big_rows(*curp);
      if (big && (curp->nmax > ce::kBigMaxN || max_targets(*curp) > ce::kBigMaxTargets)) {
        ret = CE_ERR_LIMIT;
        if (info) {
          info->err_level = l;
          info->err_reason = curp->nmax > ce::kBigMaxN ? 3 : 4;
          info->err_pivot = curp->nmax > ce::kBigMaxN ? curp->nmax : max_targets(*curp);
          info->levels_done = l;
        }
        break;
      }
      clk::time_point t_host = clk::now();
      // CTA shape: forced, autotuned for this csb, or 256-thread CTAs when
      // the average colour fills two waves of them
      int shape = (curp->ncolours > 0 && curp->M / curp->ncolours >= 2 * ce::device_sms()) ? 0 : 1;
      const int tp = o.precision, tr = o.rank_mode;
      if (o.row_shape >= 0)
        shape = o.row_shape;
      else if (l < A->tuned_levels[tp][tr])
        shape = A->tuned_shape[tp][tr][l];
      if (shape == 3) big = true;
      if (big) {
        // the large-row kernels take a colour's rows in one grid dimension
        int widest = 0;
        for (int c = 0; c < curp->ncolours; ++c)
          widest = std::max(widest, curp->colour_ptr[c + 1] - curp->colour_ptr[c]);
        if (widest > 65535) {
          g_last_error = "ce_factorize: a colour of a large-row level holds " + std::to_string(widest) +
                         " rows (at most 65535)";
          ret = CE_ERR_LIMIT;
          if (info) {
            info->err_level = l;
            info->err_reason = 8;
            info->err_pivot = widest;
            info->levels_done = l;
          }
          break;
        }
      }
      if (big && curp->bucket_nmax.size() > 1) {
        // the large-row path walks the colours in order; a batch's size
        // buckets reorder the rows, so this level gets a colour-major copy
        auto cp = std::make_shared<LevelPlan>(*curp);
        std::stable_sort(cp->order.begin(), cp->order.end(),
                         [&](int a, int b) { return cp->colour[a] < cp->colour[b]; });
        cp->bucket_ptr = {0, cp->M};
        cp->bucket_nmax = {cp->nmax};
        curp = cp;
      }
      F->levels.emplace_back();
      LevelStore& st = F->levels.back();
      st.plan = curp;
      if (l == 0 && curp == A->plan1 && A->d_meta1)
        build_level_store(st, es, s, A->d_meta1, &A->meta1_off);
      else
        build_level_store(st, es, s);
      st.dev.pool = pool;
      st.dev.prof = d_prof;
      const double host_ms = ms_since(t_host);
      const LevelPlan& P = *st.plan;
      cudaEvent_t ev0, ev1;
      check(cudaEventCreate(&ev0), "event");
      check(cudaEventCreate(&ev1), "event");
      check(cudaEventRecord(ev0, s), "event");
      st.big = big;
      if (info && l < 16) info->row_shape[l] = shape;
      // learned compression on this level unless the autotuner measured the
      // exact SVD faster here
      ce::LearnedArgs la_l = la;
      if (o.row_shape < 0 && l < A->tuned_levels[tp][tr] && !A->tuned_learned[tp][tr][l]) la_l.model = nullptr;
      // the large-row path runs its own randomized range finder (learned form)
      const bool big_sketch = la_l.model != nullptr && es == 4;
      if (info && l < 16) info->row_learned[l] = big ? big_sketch : la_l.model != nullptr;
      if (big) la_l.model = nullptr;
      if (info && l < 16) info->big_rows[l] = big ? 1 : 0;
      const int nbkt = static_cast<int>(P.bucket_nmax.size());
      if (big) {
        check(ce::run_big_level(es, st, l, o.tol, o.tol_mode, F->d_status, la.stats, o.gemm_engine,
                                info ? info->big_ms : nullptr, big_sketch, o.seed, s),
              "large rows");
      } else if (nbkt <= 1) {
        check(ce::launch_row_kernel(es, st.dev, P.M, l, o.tol, o.tol_mode, F->d_status, P.nmax, shape, la_l, s),
              "row kernel");
      } else {
        // one persistent launch per size bucket, side by side on their own
        // streams (the buckets never wait for each other)
        SideStreams& ss = side_streams();
        check(cudaEventRecord(ss.fork, s), "event");
        for (int b = 0; b < nbkt; ++b) {
          LevelDev Lb = st.dev;
          Lb.order += P.bucket_ptr[b];
          Lb.qnext += b;
          check(cudaStreamWaitEvent(ss.st[b], ss.fork, 0), "stream wait");
          check(ce::launch_row_kernel(es, Lb, P.bucket_ptr[b + 1] - P.bucket_ptr[b], l, o.tol, o.tol_mode,
                                      F->d_status, P.bucket_nmax[b], shape, la_l, ss.st[b]),
                "row kernel");
          check(cudaEventRecord(ss.join[b], ss.st[b]), "event");
          check(cudaStreamWaitEvent(s, ss.join[b], 0), "stream wait");
        }
      }
      check(cudaEventRecord(ev1, s), "event");
      // ranks and status into pinned memory, so the host runs on meanwhile
      int* hread = reinterpret_cast<int*>(stage_get(2, (2 * P.M + ce::kStatusWords) * sizeof(int)));
      check(cudaMemcpyAsync(hread, st.dev.rank, P.M * sizeof(int), cudaMemcpyDeviceToHost, s), "D2H");
      check(cudaMemcpyAsync(hread + P.M, F->d_status, sizeof(hstatus), cudaMemcpyDeviceToHost, s), "D2H");
      check(cudaMemcpyAsync(hread + P.M + ce::kStatusWords, st.dev.kw, P.M * sizeof(int), cudaMemcpyDeviceToHost,
                            s),
            "D2H");
      // While the GPU eliminates this level, plan the pattern of the next one
      // from the expected set of blocks that keep a basis (those with live
      // far blocks); checked against the actual ranks below.
      // r_i > 0 expected iff row i has a far column when it is processed: a far
      // neighbour k counts when it has rows left (w_k = r_k for an earlier colour,
      // n_k otherwise), decided in the elimination order
      std::vector<char> guess(P.M, 0);
      for (int q = 0; q < P.M; ++q) {
        const int i = P.order[q];
        bool far_cols = false;
        for (int f = P.far_ptr[i]; f < P.far_ptr[i + 1] && !far_cols; ++f) {
          const int k = P.far_blk[f];
          far_cols = P.colour[k] < P.colour[i] ? guess[k] != 0 : P.n[k] > 0;
        }
        guess[i] = P.n[i] > 0 && far_cols;
      }
      ce::NextLevel nx = ce::coarsen_structure(P, guess, o.J);
      auto nxtp = std::make_shared<LevelPlan>();
      ce::plan_structure(*nxtp, nx.M, nx.pairs, o.coloring, nx.sys_off);
      check(cudaStreamSynchronize(s), "level sync");
      t_host = clk::now();
      st.rank.assign(hread, hread + P.M);
      std::memcpy(hstatus, hread + P.M, sizeof(hstatus));
      st.kw.assign(hread + P.M + ce::kStatusWords, hread + 2 * P.M + ce::kStatusWords);
      float lms = 0.f;
      cudaEventElapsedTime(&lms, ev0, ev1);
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      if (info && l < 16) {
        info->level_ms[l] = lms;
        level_work(P, st.rank, es, info->level_flops[l], info->level_bytes[l], &st.kw);
      }
      if (hstatus[0] != 0) {
        ret = static_cast<ce_status>(hstatus[0]);
        if (info) {
          info->err_level = hstatus[1];
          info->err_block = hstatus[2];
          info->err_reason = hstatus[3];
          info->err_pivot = hstatus[4];
          std::memcpy(&info->err_value, hstatus + 6, sizeof(double));
        }
        break;
      }
      // coarsen (Section 2.4) and plan the next level
      {
        std::vector<char> live(P.M);
        bool same = true;
        for (int i = 0; i < P.M; ++i) {
          live[i] = st.rank[i] != 0;
          same = same && live[i] == guess[i];
        }
        if (info && l < 16)
          for (int i = 0; i < P.M; ++i) info->spec_miss[l] += live[i] != guess[i];
        // super-blocks capped at o.nmax rows (0: plain runs of J): the
        // speculative runs of J stand only if no run passes the cap
        if (o.nmax > 0 && ce::coarsen_parents(P, o.J, &st.rank, o.nmax) != nx.parent) same = false;
        if (!same) {
          nx = ce::coarsen_structure(P, live, o.J, &st.rank, o.nmax);
          ce::plan_structure(*nxtp, nx.M, nx.pairs, o.coloring, nx.sys_off);
        }
      }
      ce::coarsen_sizes(P, st.rank, nx);
      LevelPlan& nxt = *nxtp;
      ce::plan_layout(nxt, nx.n);
      std::vector<int64_t> gd(P.M);
      for (int i = 0; i < P.M; ++i) gd[i] = nxt.vec_off[nx.parent[i]] + nx.child_off[i];
      check(cudaMemcpyAsync(st.dev.gdst, gd.data(), P.M * sizeof(int64_t), cudaMemcpyHostToDevice, s), "H2D");
      void* npool = dalloc(std::max<int64_t>(nxt.pool_elems, 1) * es, s);
      check(cudaMemsetAsync(npool, 0, nxt.pool_elems * es, s), "memset pool");
      run_copy_tasks(reassembly_tasks(P, st.rank, o.J, nx, nxt), es, es, pool, npool, s);
      dfree(pool, s);
      pool = npool;
      st.dev.pool = nullptr;
      curp = nxtp;
      if (info && l < 16) info->host_ms[l] = host_ms + ms_since(t_host);
    }
    int64_t coarse_elems = 0;
    if (ret == CE_OK) {
      // dense remainder A_K and its Cholesky factor (FP64)
      const LevelPlan& cur = *curp;
      F->nc = static_cast<int>(cur.vec_len);
      const CoarseSystems C = coarse_systems(cur);
      F->nsys = static_cast<int>(C.nc.size());
      F->sys_nc = C.nc;
      F->sys_coff = C.coff;
      coarse_elems = C.dense_elems + C.dinv_elems;
      if (C.nmax > 28000) {
        ret = CE_ERR_LIMIT;
      } else if (F->nc > 0) {
        cudaEvent_t ev0, ev1;
        check(cudaEventCreate(&ev0), "event");
        check(cudaEventCreate(&ev1), "event");
        check(cudaEventRecord(ev0, s), "event");
        std::vector<int64_t> desc;
        for (auto* v : {&C.nc, &C.coff, &C.voff, &C.doff}) desc.insert(desc.end(), v->begin(), v->end());
        F->d_csys = static_cast<int64_t*>(dalloc(desc.size() * sizeof(int64_t), s));
        check(cudaMemcpyAsync(F->d_csys, desc.data(), desc.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s),
              "H2D");
        const size_t nb = (size_t)C.dense_elems * sizeof(double);
        F->d_coarse = static_cast<double*>(dalloc(nb, s));
        check(cudaMemsetAsync(F->d_coarse, 0, nb, s), "memset coarse");
        run_copy_tasks(dense_tasks(cur, C), es, 8, pool, F->d_coarse, s);
        void* tinv = dalloc(ce::coarse_tile_scratch(F->nsys), s);
        check(ce::coarse_cholesky(F->d_coarse, F->d_csys, F->nsys, C.nmax, (int)F->levels.size(), F->d_status,
                                  static_cast<double*>(tinv), s),
              "coarse chol");
        dfree(tinv, s);
        F->d_cdinv = static_cast<double*>(dalloc((size_t)C.dinv_elems * sizeof(double), s));
        check(ce::launch_coarse_dinv(F->d_coarse, F->d_csys, F->nsys, C.nmax, F->d_cdinv, s),
              "coarse diagonal inverses");
        check(cudaEventRecord(ev1, s), "event");
        check(cudaMemcpyAsync(hstatus, F->d_status, sizeof(hstatus), cudaMemcpyDeviceToHost, s), "D2H");
        check(cudaStreamSynchronize(s), "coarse sync");
        float cms = 0.f;
        cudaEventElapsedTime(&cms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        if (info) info->coarse_ms = cms;
        if (hstatus[0] != 0) {
          ret = static_cast<ce_status>(hstatus[0]);
          if (info) {
            info->err_level = hstatus[1];
            info->err_block = hstatus[2];
            info->err_reason = hstatus[3];
            info->err_pivot = hstatus[4];
            std::memcpy(&info->err_value, hstatus + 6, sizeof(double));
          }
        }
      }
    }
    dfree(pool, s);
    pool = nullptr;
    if (ret == CE_OK) {
      int64_t tot = 0;
      for (auto& st : F->levels) {
        F->vec_base.push_back(tot);
        tot += st.plan->vec_len;
      }
      F->coarse_base = tot;
      tot += F->nc;
      const int nlv = static_cast<int>(F->levels.size());
      F->d_apply = static_cast<int*>(dalloc((2 * nlv + 1) * sizeof(int), s));
      check(cudaMemsetAsync(F->d_apply, 0, (2 * nlv + 1) * sizeof(int), s), "memset apply state");
      for (int l = 0; l < nlv; ++l) {
        F->levels[l].dev.aq = F->d_apply + 2 * l;
        F->levels[l].dev.epoch = F->d_apply + 2 * nlv;
      }
      F->d_work = static_cast<double*>(dalloc(std::max<int64_t>(tot, 1) * sizeof(double), s));
      check(cudaStreamSynchronize(s), "factor sync");
      int64_t bytes = coarse_elems * 8 + tot * 8;
      for (auto& st : F->levels) bytes += st.fac_bytes + st.meta_bytes;
      F->bytes = bytes;
      int lstat[ce::kStatsWords];
      check(cudaMemcpy(lstat, F->d_status + ce::kStatusWords, sizeof(lstat), cudaMemcpyDeviceToHost), "D2H");
      unsigned long long prof[16 * ce::kProfSlots];
      check(cudaMemcpy(prof, d_prof, sizeof(prof), cudaMemcpyDeviceToHost), "D2H");
      if (info) {
        int dev = 0, khz = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) !=
                                                      cudaSuccess || khz <= 0)
          khz = 1;
        for (int l = 0; l < 16; ++l) {
          const unsigned long long* pl = prof + l * ce::kProfSlots;
          for (int p = 0; p < ce::kRowPhases; ++p) info->row_phase_ms[l][p] = static_cast<double>(pl[p]) / khz;
          for (int k = 0; k < 2; ++k) {
            const unsigned long long sw = pl[ce::kRowPhases + 2 * k], rows = pl[ce::kRowPhases + 2 * k + 1];
            info->jacobi_sweeps[l][k] = rows ? static_cast<double>(sw) / rows : 0.0;
          }
        }
        for (int l = 0; l < 16; ++l) {
          info->learned_rows[l] = lstat[2 * l];
          info->fallback_rows[l] = lstat[2 * l + 1];
          info->jacobi_capped[l] = lstat[32 + l];
          if (l < (int)F->levels.size() && F->levels[l].big) {
            info->jacobi_sweeps[l][0] = lstat[64 + l] ? static_cast<double>(lstat[48 + l]) / lstat[64 + l] : 0.0;
            info->jacobi_sweeps[l][1] = 0.0;
          }
        }
        info->levels_done = (int)F->levels.size();
        info->coarse_n = F->nc;
        info->factor_bytes = bytes;
        for (size_t l = 0; l < F->levels.size() && l < 16; ++l) {
          info->blocks[l] = F->levels[l].plan->M;
          info->colours[l] = F->levels[l].plan->ncolours;
          info->max_block[l] = F->levels[l].plan->nmax;
        }
      }
    }
  } catch (...) {
    ret = status_of_exception();
  }
  if (ret != CE_OK) {
    dfree(pool, s);
    cudaStreamSynchronize(s);
    free_factor(F, s);
    return ret;
  }
  *out = F;
  if (info) info->total_ms = ms_since(t_call);
  return CE_OK;
}

ce_status csb_update_values(ce_csb* A, const double* val, void* stream) {
  if (!A || !val) return CE_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    if (!csr_symmetric(A->n, A->h_rowptr.data(), A->h_col.data(), val)) return CE_ERR_INVALID_ARG;
    const size_t bytes = A->nnz * sizeof(double);
    char* h = stage_get(1, bytes);
    ce::parallel_for(16, 1, [&](int64_t b, int64_t e) {
      for (int64_t q = b; q < e; ++q) {
        const size_t lo = bytes * q / 16, hi = bytes * (q + 1) / 16;
        std::memcpy(h + lo, reinterpret_cast<const char*>(val) + lo, hi - lo);
      }
    });
    stage_upload(1, A->d_val, bytes, s);
    check(cudaStreamSynchronize(s), "csb_update_values sync");
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status ce_factorize_batched(const ce_csb* A, const ce_opts* o, ce_factor** out, ce_info* info) {
  if (!A || !A->batched) return CE_ERR_INVALID_ARG;
  return ce_factorize(A, o, out, info);
}

ce_status ce_autotune(ce_csb* A, const ce_opts* o_in, double* level_ms) {
  if (!A) return CE_ERR_INVALID_ARG;
  ce_opts o;
  ce_opts_default(&o);
  if (o_in) o = *o_in;
  if ((o.precision != CE_PREC_FP64 && o.precision != CE_PREC_FP32) ||
      (o.rank_mode != CE_RANK_SVD && o.rank_mode != CE_RANK_LEARNED))
    return CE_ERR_INVALID_ARG;
  // configurations: CTA shape (3: the large-row path) x (learned compression
  // on | exact SVD), the latter only when a rank model is given
  constexpr int kShapes = 4, kReps = 3;
  const bool learned = o.rank_mode == CE_RANK_LEARNED;
  const int nmodes = learned ? 2 : 1;
  double t[2][kShapes][16];
  int heur[16] = {};
  int nl = 16;
  for (int md = 0; md < nmodes; ++md)
    for (int sh = 0; sh < kShapes; ++sh) {
      ce_opts oc = o;
      oc.row_shape = sh;
      if (md == 1) oc.rank_mode = CE_RANK_SVD;
      for (int l = 0; l < 16; ++l) t[md][sh][l] = 1e300;
      // one untimed run first (allocator pools, staging buffers), then the
      // fastest of kReps timed runs per level
      for (int rep = 0; rep <= kReps; ++rep) {
        ce_factor* F = nullptr;
        ce_info info;
        ce_status st = ce_factorize(A, &oc, &F, &info);
        if (st != CE_OK && sh == 3) {
          // the large-row path is only a candidate: where it cannot run this
          // problem (a limit of its launches), it is left out of the choice
          for (int l = 0; l < 16; ++l) t[md][sh][l] = 1e300;
          break;
        }
        if (st != CE_OK) return st;
        ce_factor_destroy(F);
        nl = std::min(nl, info.levels_done);
        if (rep > 0)
          for (int l = 0; l < info.levels_done && l < 16; ++l)
            t[md][sh][l] = std::min(t[md][sh][l], info.level_ms[l]);
      }
    }
  {
    // the heuristic's shape per level, kept unless another is clearly faster
    o.row_shape = -1;
    const int saved = A->tuned_levels[o.precision][o.rank_mode];
    A->tuned_levels[o.precision][o.rank_mode] = 0;
    ce_factor* F = nullptr;
    ce_info info;
    ce_status st = ce_factorize(A, &o, &F, &info);
    A->tuned_levels[o.precision][o.rank_mode] = saved;
    if (st != CE_OK) return st;
    ce_factor_destroy(F);
    for (int l = 0; l < 16; ++l) heur[l] = info.row_shape[l];
  }
  for (int l = 0; l < nl; ++l) {
    int bm = 0, bs = heur[l];  // the default: learned (if given) with the heuristic shape
    for (int md = 0; md < nmodes; ++md)
      for (int sh = 0; sh < kShapes; ++sh)
        if (t[md][sh][l] < 0.97 * t[bm][bs][l]) {
          bm = md;
          bs = sh;
        }
    A->tuned_shape[o.precision][o.rank_mode][l] = bs;
    A->tuned_learned[o.precision][o.rank_mode][l] = learned && bm == 0;
  }
  A->tuned_levels[o.precision][o.rank_mode] = nl;
  if (level_ms)
    for (int md = 0; md < 2; ++md)
      for (int sh = 0; sh < kShapes; ++sh)
        for (int l = 0; l < 16; ++l) level_ms[(md * kShapes + sh) * 16 + l] = md < nmodes ? t[md][sh][l] : 0.0;
  return CE_OK;
}

ce_status ce_factorize_simple(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                              const int32_t* perm, int32_t B, double tol, int levels, ce_factor** out) {
  ce_csb* A = nullptr;
  ce_status st = csb_build(n, rowptr, col, val, perm, B, &A);
  if (st != CE_OK) return st;
  ce_opts o;
  ce_opts_default(&o);
  o.tol = tol;
  o.levels = levels;
  st = ce_factorize(A, &o, out, nullptr);
  if (st != CE_OK) {
    ce_csb_destroy(A);
    return st;
  }
  (*out)->owned_csb = A;
  return CE_OK;
}

void ce_factor_destroy(ce_factor* F) {
  if (!F) return;
  free_factor(F, nullptr);
}

ce_status ce_apply(const ce_factor* F, const double* r_dev, double* z_dev, void* stream) {
  if (!F || !r_dev || !z_dev) return CE_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    const int es = F->esize;
    double* coarse = F->d_work + F->coarse_base;
    const int nl = static_cast<int>(F->levels.size());
    double* v0 = nl ? F->d_work + F->vec_base[0] : coarse;
    if (nl) check(ce::launch_apply_prep(F->d_apply, 2 * nl, F->d_apply + 2 * nl, s), "apply prep");
    check(ce::launch_perm(F->d_perm, F->N, r_dev, v0, 1, s), "perm gather");
    for (int l = 0; l < nl; ++l) {
      const LevelStore& st = F->levels[l];
      double* v = F->d_work + F->vec_base[l];
      double* vn = (l + 1 < nl) ? F->d_work + F->vec_base[l + 1] : coarse;
      if (st.big)
        check(ce::launch_apply_big(es, st.dev, *st.plan, v, 1, s), "apply fwd");
      else
        check(ce::launch_apply_fwd(es, st.dev, v, F->d_status, s), "apply fwd");
      check(ce::launch_level_move(st.dev, v, vn, 1, s), "level move");
    }
    if (F->nsys == 1)
      check(ce::launch_coarse_solve(F->d_coarse, F->d_cdinv, F->nc, coarse, s), "coarse solve");
    else if (F->nc > 0)
      check(ce::launch_coarse_solve_sys(F->d_coarse, F->d_cdinv, F->d_csys, F->nsys, coarse, s),
            "coarse solve");
    for (int l = nl - 1; l >= 0; --l) {
      const LevelStore& st = F->levels[l];
      double* v = F->d_work + F->vec_base[l];
      double* vn = (l + 1 < nl) ? F->d_work + F->vec_base[l + 1] : coarse;
      check(ce::launch_level_move(st.dev, v, vn, 0, s), "level move");
      if (st.big)
        check(ce::launch_apply_big(es, st.dev, *st.plan, v, 0, s), "apply bwd");
      else
        check(ce::launch_apply_bwd(es, st.dev, v, F->d_status, s), "apply bwd");
    }
    check(ce::launch_perm(F->d_perm, F->N, v0, z_dev, 0, s), "perm scatter");
  } catch (...) {
    return status_of_exception();
  }
  return CE_OK;
}

ce_status pcg_solve(const ce_csb* A, const ce_factor* F, const double* b_dev, double* x_dev, double rtol,
                    int maxit, ce_pcg_info* info, void* stream) {
  if (!A || !F || !b_dev || !x_dev || maxit < 0 || rtol < 0 || A->n != F->N) return CE_ERR_INVALID_ARG;
  if (A->nsys > 1) return pcg_solve_batched(A, F, b_dev, x_dev, rtol, maxit, nullptr, nullptr, nullptr, info, stream);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = A->n;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms <= 0) {
    g_last_error = "pcg_solve: cannot read the device's SM count";
    return CE_ERR_CUDA;
  }
  const int nparts = static_cast<int>(std::min<int64_t>((n + 255) / 256, (int64_t)sms * 4));
  double *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr, *part = nullptr, *scal = nullptr;
  ce_status ret = CE_OK;
  if (info) std::memset(info, 0, sizeof(*info));
  try {
    r = static_cast<double*>(dalloc(n * 8, s));
    z = static_cast<double*>(dalloc(n * 8, s));
    p = static_cast<double*>(dalloc(n * 8, s));
    Ap = static_cast<double*>(dalloc(n * 8, s));
    part = static_cast<double*>(dalloc(nparts * 8, s));
    scal = static_cast<double*>(dalloc(8 * 8, s));
    check(cudaMemsetAsync(x_dev, 0, n * 8, s), "memset x");
    check(cudaMemcpyAsync(r, b_dev, n * 8, cudaMemcpyDeviceToDevice, s), "copy b");
    check(ce::launch_dot(n, r, r, part, nparts, s), "dot");
    check(ce::launch_reduce(part, nparts, scal + 3, s), "reduce");
    double hb = 0;
    check(cudaMemcpyAsync(&hb, scal + 3, 8, cudaMemcpyDeviceToHost, s), "D2H");
    check(cudaStreamSynchronize(s), "sync");
    const double bn = std::sqrt(hb);
    double rel = 0.0;
    int it = 0;
    bool conv = (bn == 0.0);
    if (!conv) {
      ret = ce_apply(F, r, z, s);
      if (ret != CE_OK) throw CudaFail{cudaErrorUnknown};
      check(ce::launch_dot(n, r, z, part, nparts, s), "dot");
      check(ce::launch_reduce(part, nparts, scal + 0, s), "reduce");
      check(ce::launch_update_p(n, p, z, scal, 1, s), "p");
      rel = 1.0;
      for (it = 1; it <= maxit; ++it) {
        check(ce::launch_spmv_dot(n, A->d_rowptr, A->d_col, A->d_val, p, Ap, part, nparts, s), "spmv");
        check(ce::launch_reduce(part, nparts, scal + 1, s), "reduce");
        check(ce::launch_pcg_scalars(scal, 0, s), "alpha");
        check(ce::launch_update_xr(n, x_dev, r, p, Ap, scal, part, nparts, s), "xr");
        check(ce::launch_reduce(part, nparts, scal + 3, s), "reduce");
        double rr = 0;
        check(cudaMemcpyAsync(&rr, scal + 3, 8, cudaMemcpyDeviceToHost, s), "D2H");
        check(cudaStreamSynchronize(s), "sync");
        rel = std::sqrt(rr) / bn;
        if (rel <= rtol) {
          conv = true;
          break;
        }
        if (it == maxit) break;
        ret = ce_apply(F, r, z, s);
        if (ret != CE_OK) throw CudaFail{cudaErrorUnknown};
        check(ce::launch_dot(n, r, z, part, nparts, s), "dot");
        check(ce::launch_reduce(part, nparts, scal + 4, s), "reduce");
        check(ce::launch_pcg_scalars(scal, 1, s), "beta");
        check(ce::launch_update_p(n, p, z, scal, 0, s), "p");
      }
      if (it > maxit) it = maxit;
    }
    if (info) {
      info->iters = conv && bn == 0.0 ? 0 : it;
      info->relres = rel;
      info->converged = conv ? 1 : 0;
    }
    if (!conv) ret = CE_ERR_NO_CONVERGENCE;
  } catch (...) {
    if (ret == CE_OK) ret = status_of_exception();
  }
  dfree(r, s);
  dfree(z, s);
  dfree(p, s);
  dfree(Ap, s);
  dfree(part, s);
  dfree(scal, s);
  return ret;
}

int ce_factor_levels(const ce_factor* F) { return F ? static_cast<int>(F->levels.size()) : 0; }

int ce_factor_level_size(const ce_factor* F, int level) {
  if (!F || level < 0 || level >= static_cast<int>(F->levels.size())) return -1;
  return F->levels[level].plan->M;
}

ce_status ce_factor_get_level(const ce_factor* F, int level, int32_t* n, int32_t* rank, int32_t* colour,
                              double* tau) {
  if (!F || level < 0 || level >= static_cast<int>(F->levels.size())) return CE_ERR_INVALID_ARG;
  const LevelStore& st = F->levels[level];
  if (n) std::copy(st.plan->n.begin(), st.plan->n.end(), n);
  if (rank) std::copy(st.rank.begin(), st.rank.end(), rank);
  if (colour) std::copy(st.plan->colour.begin(), st.plan->colour.end(), colour);
  if (tau) {
    cudaError_t e = cudaMemcpy(tau, st.dev.tau, st.plan->M * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      g_last_error = cudaGetErrorString(e);
      return CE_ERR_CUDA;
    }
  }
  return CE_OK;
}

ce_status ce_debug_wait_expiry(int kernel, double limit_ms, int32_t* status_out, void* stream) {
  if ((kernel != 0 && kernel != 1) || !(limit_ms > 0) || limit_ms > 2000 || !status_out) return CE_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LevelStore st;
  void* pool = nullptr;
  int* status = nullptr;
  int* apply_state = nullptr;
  double* vec = nullptr;
  ce_status ret = CE_OK;
  try {
    // two blocks of 4 rows coupled by one close pair: block 1 has the higher
    // colour and waits for block 0, which is never queued
    auto P = std::make_shared<LevelPlan>();
    ce::plan_level(*P, {4, 4}, {{0, 1}}, true);
    if (P->order.size() != 2 || P->order[1] != 1 || P->dep_ptr[2] - P->dep_ptr[1] != 1)
      throw std::logic_error("unexpected two-block plan");
    st.plan = P;
    build_level_store(st, 8, s);
    std::vector<double> hp(P->pool_elems, 0.0);
    for (int i = 0; i < 2; ++i)
      for (int a = 0; a < 4; ++a) hp[P->diag_off[i] + a * 4 + a] = 4.0;
    pool = dalloc(hp.size() * sizeof(double), s);
    check(cudaMemcpyAsync(pool, hp.data(), hp.size() * sizeof(double), cudaMemcpyHostToDevice, s), "H2D");
    status = static_cast<int*>(dalloc((ce::kStatusWords + ce::kStatsWords) * sizeof(int), s));
    check(cudaMemsetAsync(status, 0, (ce::kStatusWords + ce::kStatsWords) * sizeof(int), s), "memset");
    LevelDev D = st.dev;
    D.pool = pool;
    D.order += 1;                       // only block 1 is queued
    D.wait_ns = static_cast<unsigned long long>(limit_ms * 1e6);
    if (kernel == 0) {
      ce::LearnedArgs la;
      check(ce::launch_row_kernel(8, D, 1, 0, 1e-3, CE_TOL_REL, status, P->nmax, 0, la, s), "row kernel");
    } else {
      apply_state = static_cast<int*>(dalloc(4 * sizeof(int), s));
      const int init[4] = {0, 0, 1, 0};  // queue counters, epoch 1 (block 0's flag stays 0)
      check(cudaMemcpyAsync(apply_state, init, sizeof(init), cudaMemcpyHostToDevice, s), "H2D");
      D.aq = apply_state;
      D.epoch = apply_state + 2;
      D.M = 1;
      vec = static_cast<double*>(dalloc(P->vec_len * sizeof(double), s));
      check(cudaMemsetAsync(vec, 0, P->vec_len * sizeof(double), s), "memset");
      check(ce::launch_apply_fwd(8, D, vec, status, s), "apply");
    }
    check(cudaMemcpyAsync(status_out, status, ce::kStatusWords * sizeof(int), cudaMemcpyDeviceToHost, s), "D2H");
    check(cudaStreamSynchronize(s), "sync");
  } catch (...) {
    ret = status_of_exception();
  }
  cudaStreamSynchronize(s);
  dfree(st.meta, s);
  dfree(st.smeta, s);
  dfree(st.fac, s);
  dfree(pool, s);
  dfree(status, s);
  dfree(apply_state, s);
  dfree(vec, s);
  return ret;
}

ce_status ce_debug_svd(int esize, int block, int n, const void* R_dev, const void* D_dev, double tol, void* X_dev,
                       void* V_dev, int* sweeps, void* stream) {
  if ((esize != 4 && esize != 8) || (block != 4 && block != 8 && block != 16 && block != 32) || n < 1 ||
      n > ce::kBigMaxN || !R_dev || !D_dev || !X_dev || !V_dev || tol < 0)
    return CE_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = ce::debug_svd(esize, block, n, R_dev, D_dev, tol, X_dev, V_dev, sweeps, s);
  if (e == cudaErrorInvalidValue) {
    g_last_error = "ce_debug_svd: 4 x block x n values do not fit in shared memory";
    return CE_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) {
    g_last_error = std::string("ce_debug_svd: ") + cudaGetErrorString(e);
    return CE_ERR_CUDA;
  }
  return CE_OK;
}

ce_status ce_debug_gemm(int engine, int M, int N, int K, const void* A_dev, int lda, int ta, const void* B_dev,
                        int ldb, int tb, void* C_dev, int ldc, int tc, double alpha, double beta, void* stream) {
  if (engine < 0 || engine > 3 || M < 0 || N < 0 || K < 0 || !A_dev || !B_dev || !C_dev || lda <= 0 || ldb <= 0 ||
      ldc <= 0)
    return CE_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* err = nullptr;
  try {
    ce::GemmTask t{};
    t.A = A_dev;
    t.lda = lda;
    t.ta = ta != 0;
    t.B = B_dev;
    t.ldb = ldb;
    t.tb = tb != 0;
    t.C = C_dev;
    t.ldc = ldc;
    t.tc = tc != 0;
    t.Cin = C_dev;
    t.ldcin = ldc;
    t.tcin = tc != 0;
    t.M = M;
    t.N = N;
    t.K = K;
    t.alpha = static_cast<float>(alpha);
    t.beta = static_cast<float>(beta);
    const std::vector<ce::GemmTask> tasks{t};
    if (engine == 0 || engine == 3) {
      check(ce::launch_gemm_cuda(engine == 3 ? 8 : 4, tasks, s), "gemm");
    } else {
      err = static_cast<int*>(dalloc(sizeof(int), s));
      check(cudaMemsetAsync(err, 0, sizeof(int), s), "memset");
      check(ce::launch_gemm_tc(tasks, engine == 1 ? 3 : 1, err, s), "tcgen05 gemm");
      int herr = 0;
      check(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H");
      check(cudaStreamSynchronize(s), "sync");
      dfree(err, s);
      err = nullptr;
      if (herr) {
        g_last_error = "tcgen05 gemm: a pipeline wait expired";
        return CE_ERR_CUDA;
      }
    }
    check(cudaStreamSynchronize(s), "sync");
  } catch (...) {
    dfree(err, s);
    return status_of_exception();
  }
  return CE_OK;
}

ce_status ce_factor_get_features(const ce_factor* F, int level, float* feat, int32_t* kw) {
  if (!F || level < 0 || level >= static_cast<int>(F->levels.size())) return CE_ERR_INVALID_ARG;
  const LevelStore& st = F->levels[level];
  if (kw) std::copy(st.kw.begin(), st.kw.end(), kw);
  if (feat) {
    cudaError_t e = cudaMemcpy(feat, st.dev.feat, (size_t)st.plan->M * ce::kMlpFeatures * sizeof(float),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      g_last_error = cudaGetErrorString(e);
      return CE_ERR_CUDA;
    }
  }
  return CE_OK;
}

ce_status ce_factor_get_sigma(const ce_factor* F, int level, double* sigma) {
  if (!F || !sigma || level < 0 || level >= static_cast<int>(F->levels.size())) return CE_ERR_INVALID_ARG;
  const LevelStore& st = F->levels[level];
  cudaError_t e = cudaMemcpy(sigma, st.dev.sigma, st.plan->vec_len * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    g_last_error = cudaGetErrorString(e);
    return CE_ERR_CUDA;
  }
  return CE_OK;
}

}  // extern "C"
