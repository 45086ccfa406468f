// Internal types of the CE library: host plans and device views.
#pragma once
#include <algorithm>
#include <cstdint>
#include <exception>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ce.h"

namespace ce {

constexpr int kNMax = 64;  // largest block the row kernel holds in shared memory
constexpr int kBigMaxN = 1536;       // largest block of the large-row path
constexpr int kBigMaxTargets = 64;   // most targets (1 + close blocks) of a large row
constexpr int kBuckets = 3;  // size buckets of a batch's rows (<= 16, <= 32, <= 64 rows)

// Host threads for the planning loops (hardware threads, at most 16).
int host_threads();

// Runs job(t) for t in [0, tasks) on a pool of host threads kept for the
// life of the process (and the calling thread); returns when all are done.
// While the pool serves another caller the tasks run on the calling thread.
void run_tasks(int64_t tasks, const std::function<void(int64_t)>& job);

// f(begin, end) over [0, n) cut into at most host_threads() ranges of at
// least `grain` items; the first exception thrown by a range is rethrown.
template <class F>
void parallel_for(int64_t n, int64_t grain, F&& f) {
  if (n <= 0) return;
  const int64_t T = std::min<int64_t>(host_threads(), (n + grain - 1) / std::max<int64_t>(grain, 1));
  if (T <= 1) {
    f(int64_t(0), n);
    return;
  }
  std::exception_ptr err;
  std::mutex mu;
  run_tasks(T, [&](int64_t t) {
    try {
      f(n * t / T, n * (t + 1) / T);
    } catch (...) {
      std::lock_guard<std::mutex> lk(mu);
      if (!err) err = std::current_exception();
    }
  });
  if (err) std::rethrow_exception(err);
}

// ---------------------------------------------------------------------------
// Host plan of one level (Section 2.2-2.4): block sizes, the level-start
// ("close") pattern, its square (close + far pairs, eq. bsp), a distance-2
// colouring and every offset the kernels need.  Pairs are stored once, as
// (i, k) with i <= k, row-major n_i x n_k in one value pool.
// ---------------------------------------------------------------------------
struct LevelPlan {
  int M = 0;
  int coloring = 1;              // 0 natural order, 1 distance-2, 2 distance-1 colours
  std::vector<int> n;            // block sizes
  std::vector<int> colour;
  int ncolours = 0;
  std::vector<int> order;        // colour-major elimination order
  std::vector<int> colour_ptr;   // ncolours + 1 offsets into order

  // all pairs of the squared pattern, sorted by (i, k), i <= k; the pairs
  // of row i are [pair_ptr[i], pair_ptr[i+1])
  std::vector<int> pair_ptr, pair_i, pair_k;
  std::vector<int64_t> pair_off;
  std::vector<char> pair_close;
  int64_t pool_elems = 0;

  // per block (CSR-style arrays); *_pidx are indices into the pair arrays
  // (pattern only), *_off the pool offsets of those pairs (after the sizes)
  std::vector<int> close_ptr, close_blk;   // close(i) \ {i}, ascending
  std::vector<int> close_pidx;
  std::vector<int64_t> close_off;
  std::vector<int> far_ptr, far_blk;       // far pairs live when i is processed
  std::vector<int> far_pidx;
  std::vector<int64_t> far_off;
  std::vector<int> diag_pidx;
  std::vector<int64_t> diag_off;
  std::vector<int> schur_ptr;              // t(t+1)/2 target pairs, t = 1+|close|
  std::vector<int> schur_pidx;
  std::vector<int64_t> schur_off;

  // factor and vector layout
  std::vector<int64_t> u_off, l_off, w_off, vec_off;
  int64_t u_elems = 0, l_elems = 0, w_elems = 0, vec_len = 0;
  int nmax = 0;

  // independent systems: blocks [sys_off[s], sys_off[s+1]) belong to system s
  std::vector<int> sys_off;

  // rows of a lower colour within distance 2 of row i (the rows that must
  // finish before row i starts): [dep_ptr[i], dep_ptr[i+1]) of dep_idx
  std::vector<int> dep_ptr, dep_idx;
  // the transpose: rows of a higher colour within distance 2 (backward apply)
  std::vector<int> rdep_ptr, rdep_idx;

  // size buckets of a batch (whole systems, by their largest block: <= 16,
  // <= 32, larger rows): order[bucket_ptr[b], bucket_ptr[b+1]) holds bucket
  // b's rows, colour-major; no row depends on a row of another bucket
  std::vector<int> bucket_ptr, bucket_nmax;
};

// Build the plan of a level from its sizes and level-start pattern (pairs
// with i <= k; the diagonal pairs are added if missing).  sys_off (empty =
// one system) gives the blocks of each independent system.  plan_structure
// does everything that depends on the pattern alone (colouring, squared
// pattern, lists, dependencies), plan_layout what depends on the sizes
// (pool, factor and vector offsets); plan_level is both.
// coloring: 0 natural order (each block its own step), 1 distance-2 colours
// (no two rows of a colour share a block), 2 distance-1 colours (rows of a
// colour may share Schur targets, which they then update atomically)
void plan_level(LevelPlan& P, const std::vector<int>& n,
                const std::vector<std::pair<int, int>>& close_pairs, int coloring,
                const std::vector<int>& sys_off = {});
void plan_structure(LevelPlan& P, int M, const std::vector<std::pair<int, int>>& close_pairs, int coloring,
                    const std::vector<int>& sys_off);
void plan_layout(LevelPlan& P, const std::vector<int>& n);
int find_pair_idx(const LevelPlan& P, int a, int b);

// Element offset of pair (a, b) (either order) in the level pool, -1 if the
// pair is not in the squared pattern.
int64_t find_pair(const LevelPlan& P, int a, int b);

// Reassembly of level l into level l+1 (Section 2.4): copy tasks for the
// kept r_i x r_k corner of every pair into the super-block pairs.
struct CopyTask {
  int64_t src_off;   // element offset of the source block
  int64_t dst_off;   // element offset of the destination block
  int src_ld, dst_ld;
  int rows, cols;    // rows x cols of the source corner
  int r0, c0;        // destination position
  int transpose;     // 1: dst[(r0+b), (c0+a)] = src[a, b]
};

struct NextLevel {
  int M = 0;                                     // super-blocks
  std::vector<int> n;                            // super-block sizes
  std::vector<std::pair<int, int>> pairs;        // next close pattern
  std::vector<int> child_off;                    // offset of child i in its super-block
  std::vector<int> parent;                       // super-block of child i
  std::vector<int> sys_off;                      // super-blocks of each system
};

// Super-blocks: runs of J consecutive blocks of one system; a run whose ranks
// add up to more than nmax rows (the row kernel's limit) is halved until its
// parts fit, so the parts stay aligned with the runs.
NextLevel coarsen(const LevelPlan& P, const std::vector<int>& rank, int J, int nmax);
// the same in two steps: the pattern from which blocks keep a basis
// (live[i] = r_i > 0; without ranks the groups are plain runs of J), then the
// super-block sizes and child offsets
NextLevel coarsen_structure(const LevelPlan& P, const std::vector<char>& live, int J,
                            const std::vector<int>* rank = nullptr, int nmax = 0);
// the super-block of every block under that rule (and optionally each
// super-block's first child and the super-blocks of each system)
std::vector<int> coarsen_parents(const LevelPlan& P, int J, const std::vector<int>* rank, int nmax,
                                 std::vector<int>* first_child = nullptr, std::vector<int>* sys_off = nullptr);
void coarsen_sizes(const LevelPlan& P, const std::vector<int>& rank, NextLevel& nx);

// graph, work vectors and chunk map of the batched PCG (pcg_batched.cu)
struct PcgBatch;
void pcg_batch_release(PcgBatch* P);

// ---------------------------------------------------------------------------
// Device view of a level for the kernels (all pointers device).
// ---------------------------------------------------------------------------
struct LevelDev {
  int M;
  const int* n;
  const int* colour;
  int* rank;
  const int* order;
  const int* close_ptr;
  const int* close_blk;
  const int64_t* close_off;
  const int* far_ptr;
  const int* far_blk;
  const int64_t* far_off;
  const int64_t* diag_off;
  const int* schur_ptr;
  const int64_t* schur_off;
  const int64_t* u_off;
  const int64_t* l_off;
  const int64_t* w_off;
  const int64_t* vec_off;
  int64_t* gdst;        // position of block i's basis in the next vector
  double* tau;          // per block
  double* sigma;        // sum n_i (vec layout)
  const int* dep_ptr;   // lower-colour rows within distance 2 (CSR)
  const int* dep_idx;
  int* done;            // per row: 1 once eliminated (persistent launch)
  int* qnext;           // next position of the persistent launch's queue
  const int* rdep_ptr;  // higher-colour rows within distance 2 (CSR)
  const int* rdep_idx;
  int* fdone;           // per row: epoch of the last forward apply step done
  int* bdone;           // ... and of the last backward step
  int* aq;              // queue counters of the apply launches (fwd, bwd)
  float* feat;          // per row: the rank model's features (learned levels)
  int* kw;              // per row: sketch width k of the learned compression
                        // (k accepted, -k rejected for the exact SVD, 0 none)
  const int* epoch;     // epoch of the running apply
  unsigned long long wait_ns;  // a row's wait for its neighbours gives up after this long
  int accumulate;       // 1: rows of a colour may share Schur targets (distance-1
                        // colours): their updates of shared pairs and vector
                        // entries are atomic
  unsigned long long* prof;  // SM cycles per (level, row phase), summed over
                             // rows (ce_row_kernel; null: not recorded)
  void* pool;           // pair values (T)
  void* U;              // factor (T): U_i
  void* L;              //   L_hat_i^{-1} (m_i x m_i, lower)
  void* W;
};

// Byte offsets of a plan's fixed arrays inside its device metadata block.
struct StaticMeta {
  size_t o_n, o_col, o_order, o_cp, o_cb, o_co, o_fp, o_fb, o_fo, o_do, o_sp, o_so, o_uo, o_lo, o_wo, o_vo, o_dp,
      o_di, o_rp, o_ri;
};

// One level kept in a factor.
struct LevelStore {
  std::shared_ptr<const LevelPlan> plan;  // level 1 may share the csb's plan
  std::vector<int> rank;        // host copy
  std::vector<int> kw;          // host copy of the per-row sketch widths
  bool big = false;             // eliminated by the large-row path (big_rows.cu)
  LevelDev dev{};
  void* meta = nullptr;         // device per-factorization state (ranks, flags, ...)
  void* smeta = nullptr;        // device arrays fixed by the plan (null: shared)
  void* fac = nullptr;          // device U, L, W block
  size_t fac_bytes = 0;
  size_t meta_bytes = 0;
};

}  // namespace ce

struct ce_csb {
  int64_t n = 0;
  int B = 0;                     // block size (first system's for a batch)
  int nsys = 1;                  // independent systems (block-diagonal batch)
  bool batched = false;          // built by csb_build_batched
  std::vector<int64_t> sys_row;  // rows of system s: [sys_row[s], sys_row[s+1])
  int32_t* d_sys_of_row = nullptr;  // system of every row (batched PCG)
  int64_t nnz = 0;
  // host copy of the pattern (value updates are checked against it)
  std::vector<int64_t> h_rowptr;
  std::vector<int32_t> h_col;
  // device CSR of A (original ordering) and the permutation
  int64_t* d_rowptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_val = nullptr;
  int32_t* d_perm = nullptr;
  // level-1 plan and the scatter map nnz -> element of the level-1 pool
  std::shared_ptr<ce::LevelPlan> plan1;
  // row-kernel CTA shape per level chosen by ce_autotune, one choice per
  // precision (CE_PREC_*) and rank mode (CE_RANK_*)
  int tuned_levels[2][2] = {};
  int tuned_shape[2][2][16] = {};
  int tuned_learned[2][2][16] = {};  // learned compression measured faster on level l
  int64_t* d_scatter = nullptr;
  // level-1 plan's fixed arrays on the device, shared by every factorization
  void* d_meta1 = nullptr;
  ce::StaticMeta meta1_off{};
};

struct ce_factor {
  int64_t N = 0;
  int nsys = 1;
  std::vector<int64_t> sys_nc;  // coarse size of each system
  std::vector<int64_t> sys_coff;// offset of its dense factor in d_coarse
  int64_t* d_csys = nullptr;    // device copy: [nc(nsys), coff(nsys), voff(nsys), dinv_off(nsys)]
  int prec = CE_PREC_FP64;
  int esize = 8;
  std::vector<ce::LevelStore> levels;
  int nc = 0;                   // coarse size
  double* d_coarse = nullptr;   // nc x nc lower Cholesky factor (FP64)
  double* d_cdinv = nullptr;    // inverses of its 64 x 64 diagonal blocks
  int32_t* d_perm = nullptr;    // borrowed from the csb
  double* d_work = nullptr;     // level vectors (FP64) + coarse vector
  std::vector<int64_t> vec_base;// start of each level vector in d_work
  int64_t coarse_base = 0;
  int* d_status = nullptr;
  int* d_apply = nullptr;       // apply queue counters (2 per level) + epoch
  int64_t bytes = 0;
  ce_csb* owned_csb = nullptr;
  mutable ce::PcgBatch* pcg = nullptr;  // batched PCG state, built on first use
};
