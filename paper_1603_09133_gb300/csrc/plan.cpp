// Host symbolic planning of one CE level (block graph, squared pattern,
// distance-2 colouring, offsets) and of the reassembly into super-blocks.
//
// Section 2.2: eliminating a block sub-row only creates blocks inside the
// pattern of A^2 ("far" blocks are nonzero in A^2 and zero in A), so every
// pair a level can touch is known before its numeric phase and is
// preallocated here.  Section 2.4 (eq. bsp): after a sweep, J consecutive
// blocks join into one super-block; the next level's pattern is the
// coarsened squared pattern restricted to blocks with a non-empty basis.
//
// Every structure is a flat CSR array and every per-block loop runs on a few
// host threads (blocks are independent once the adjacency is known); the
// greedy colouring is sequential within one system and runs systems in
// parallel (blocks of different systems are never adjacent).
#include <algorithm>
#include <numeric>
#include <stdexcept>
#include <thread>
#include <atomic>
#include <condition_variable>
#include <mutex>

#include <unistd.h>

#include "ce_internal.h"

namespace ce {

int host_threads() {
  static const int t = [] {
    const unsigned h = std::thread::hardware_concurrency();
    return static_cast<int>(std::min(16u, std::max(1u, h)));
  }();
  return t;
}

namespace {

// Worker threads waiting for jobs; a job is a task count and a function,
// tasks are taken from an atomic counter by the workers and the caller.
struct Pool {
  std::mutex busy;                 // one job at a time
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  const std::function<void(int64_t)>* job = nullptr;
  int64_t tasks = 0;
  std::atomic<int64_t> next{0};
  int active = 0;                  // workers still inside the current job
  uint64_t generation = 0;
  int nworkers = 0;

  explicit Pool(int n) : nworkers(n) {
    for (int w = 0; w < n; ++w) std::thread([this] { loop(); }).detach();
  }

  void drain() {
    for (int64_t t; (t = next.fetch_add(1)) < tasks;) (*job)(t);
  }

  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return generation != seen; });
        seen = generation;
      }
      drain();
      std::lock_guard<std::mutex> lk(mu);
      if (--active == 0) cv_done.notify_one();
    }
  }

  void run(int64_t n, const std::function<void(int64_t)>& f) {
    {
      std::lock_guard<std::mutex> lk(mu);
      job = &f;
      tasks = n;
      next.store(0);
      active = nworkers;
      ++generation;
    }
    cv_work.notify_all();
    drain();
    std::unique_lock<std::mutex> lk(mu);
    cv_done.wait(lk, [&] { return active == 0; });
    job = nullptr;
  }
};

std::mutex g_pool_mu;
Pool* g_pool = nullptr;   // kept for the life of the process
pid_t g_pool_pid = 0;     // a forked child starts a pool of its own

}  // namespace

void run_tasks(int64_t tasks, const std::function<void(int64_t)>& job) {
  Pool* pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool || g_pool_pid != getpid()) {
      g_pool = new Pool(host_threads() - 1);
      g_pool_pid = getpid();
    }
    pool = g_pool;
  }
  std::unique_lock<std::mutex> lk(pool->busy, std::try_to_lock);
  if (!lk.owns_lock() || pool->nworkers == 0) {
    for (int64_t t = 0; t < tasks; ++t) job(t);
    return;
  }
  pool->run(tasks, job);
}

namespace {

struct Csr {
  std::vector<int64_t> ptr;
  std::vector<int> idx;
  int deg(int i) const { return static_cast<int>(ptr[i + 1] - ptr[i]); }
  const int* row(int i) const { return idx.data() + ptr[i]; }
  bool has(int i, int k) const { return std::binary_search(row(i), row(i) + deg(i), k); }
};

// sorted adjacency (diagonal included) from a list of pairs
Csr adjacency(int M, const std::vector<std::pair<int, int>>& pairs) {
  Csr A;
  std::vector<int64_t> cnt(M + 1, 0);
  for (int i = 0; i < M; ++i) cnt[i + 1] = 1;
  for (auto& p : pairs)
    if (p.first != p.second) {
      ++cnt[p.first + 1];
      ++cnt[p.second + 1];
    }
  for (int i = 0; i < M; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> raw(cnt[M]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int i = 0; i < M; ++i) raw[fill[i]++] = i;
  for (auto& p : pairs)
    if (p.first != p.second) {
      raw[fill[p.first]++] = p.second;
      raw[fill[p.second]++] = p.first;
    }
  // sort + unique per row, then compact
  std::vector<int> len(M);
  parallel_for(M, 2048, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      int* s = raw.data() + cnt[i];
      int* t = raw.data() + cnt[i + 1];
      std::sort(s, t);
      len[i] = static_cast<int>(std::unique(s, t) - s);
    }
  });
  A.ptr.assign(M + 1, 0);
  for (int i = 0; i < M; ++i) A.ptr[i + 1] = A.ptr[i] + len[i];
  A.idx.resize(A.ptr[M]);
  parallel_for(M, 4096, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) std::copy_n(raw.data() + cnt[i], len[i], A.idx.data() + A.ptr[i]);
  });
  return A;
}

// greedy colouring of blocks [b0, b1), visited in breadth-first order: every
// component starts at its block of least degree (lowest index on ties),
// neighbours are queued in ascending index; a block takes the smallest colour
// not held within distance `dist`.  dist 2: no two blocks of a colour share a
// neighbour.  dist 1: adjacent blocks differ, and two blocks of a colour share
// only neighbours of a higher colour (an earlier common neighbour would create
// the fill block between them, which both rows would then compress).
void colour_range(const Csr& adj, int b0, int b1, std::vector<int>& colour, int dist) {
  const int nb = b1 - b0;
  std::vector<int> roots(nb);
  std::iota(roots.begin(), roots.end(), b0);
  std::stable_sort(roots.begin(), roots.end(), [&](int a, int b) { return adj.deg(a) < adj.deg(b); });
  std::vector<char> seen(nb, 0);
  std::vector<int> queue;
  queue.reserve(nb);
  std::vector<int> mark;  // mark[c] == i  <=> colour c is taken near i
  for (int root : roots) {
    if (seen[root - b0]) continue;
    seen[root - b0] = 1;
    queue.assign(1, root);
    for (size_t h = 0; h < queue.size(); ++h) {
      const int i = queue[h];
      auto take = [&](int k) {
        if (k != i && colour[k] >= 0) {
          const int c = colour[k];
          if (c >= static_cast<int>(mark.size())) mark.resize(c + 1, -1);
          mark[c] = i;
        }
      };
      int c = 0;
      if (dist == 1) {
        // colours of the neighbours; a colour held by two of them must lie
        // below i's (i would be their earlier common neighbour and create the
        // fill block between them before they compress it)
        for (const int* j = adj.row(i); j != adj.row(i) + adj.deg(i); ++j) {
          if (*j == i || colour[*j] < 0) continue;
          const int cj = colour[*j];
          if (cj < static_cast<int>(mark.size()) && mark[cj] == i) c = std::max(c, cj + 1);
          take(*j);
        }
        // a neighbour j coloured below i's colour is the earlier common
        // neighbour of i and each other neighbour k of j: k's colour is out
        // if it lies above j's
        for (const int* j = adj.row(i); j != adj.row(i) + adj.deg(i); ++j) {
          if (*j == i || colour[*j] < 0) continue;
          for (const int* k = adj.row(*j); k != adj.row(*j) + adj.deg(*j); ++k)
            if (colour[*k] > colour[*j]) take(*k);
        }
      } else {
        for (const int* j = adj.row(i); j != adj.row(i) + adj.deg(i); ++j)
          for (const int* k = adj.row(*j); k != adj.row(*j) + adj.deg(*j); ++k) take(*k);
      }
      while (c < static_cast<int>(mark.size()) && mark[c] == i) ++c;
      colour[i] = c;
      for (const int* j = adj.row(i); j != adj.row(i) + adj.deg(i); ++j)
        if (!seen[*j - b0]) {
          seen[*j - b0] = 1;
          queue.push_back(*j);
        }
    }
  }
}

// Per-block output lists filled by chunks of blocks in parallel and joined in
// block order: a CSR pointer array plus one or two value arrays.
template <typename A, typename B>
void join_chunks(int M, int nch, const std::vector<std::vector<int>>& cnt, std::vector<std::vector<A>>& va,
                 std::vector<std::vector<B>>* vb, std::vector<int>& ptr, std::vector<A>& outa,
                 std::vector<B>* outb, const std::vector<int64_t>& cb) {
  ptr.assign(M + 1, 0);
  for (int c = 0; c < nch; ++c)
    for (int64_t i = cb[c]; i < cb[c + 1]; ++i) ptr[i + 1] = cnt[c][i - cb[c]];
  for (int i = 0; i < M; ++i) ptr[i + 1] += ptr[i];
  outa.resize(ptr[M]);
  if (outb) outb->resize(ptr[M]);
  parallel_for(nch, 1, [&](int64_t b, int64_t e) {
    for (int64_t c = b; c < e; ++c) {
      std::copy(va[c].begin(), va[c].end(), outa.begin() + ptr[cb[c]]);
      if (outb) std::copy((*vb)[c].begin(), (*vb)[c].end(), outb->begin() + ptr[cb[c]]);
    }
  });
}

}  // namespace

int find_pair_idx(const LevelPlan& P, int a, int b) {
  if (a > b) std::swap(a, b);
  const int* lo = P.pair_k.data() + P.pair_ptr[a];
  const int* hi = P.pair_k.data() + P.pair_ptr[a + 1];
  const int* it = std::lower_bound(lo, hi, b);
  if (it == hi || *it != b) return -1;
  return static_cast<int>(it - P.pair_k.data());
}

int64_t find_pair(const LevelPlan& P, int a, int b) {
  const int p = find_pair_idx(P, a, b);
  return p < 0 ? -1 : P.pair_off[p];
}

void plan_structure(LevelPlan& P, int M, const std::vector<std::pair<int, int>>& close_pairs, int coloring,
                    const std::vector<int>& sys_off) {
  P = LevelPlan();
  P.M = M;
  P.sys_off = sys_off;
  P.coloring = coloring;
  const Csr adj = adjacency(M, close_pairs);

  // ---- greedy colouring (distance 2, or 1 with shared Schur targets) ------
  P.colour.assign(M, -1);
  if (coloring) {
    std::vector<int> so = sys_off.empty() ? std::vector<int>{0, M} : sys_off;
    const int ns = static_cast<int>(so.size()) - 1;
    const int dist = coloring == 2 ? 1 : 2;
    parallel_for(ns, 1, [&](int64_t b, int64_t e) {
      for (int64_t s = b; s < e; ++s) colour_range(adj, so[s], so[s + 1], P.colour, dist);
    });
  } else {
    // natural order: every block is its own step
    for (int i = 0; i < M; ++i) P.colour[i] = i;
  }
  P.ncolours = M ? *std::max_element(P.colour.begin(), P.colour.end()) + 1 : 0;
  P.order.resize(M);
  std::iota(P.order.begin(), P.order.end(), 0);
  std::stable_sort(P.order.begin(), P.order.end(),
                   [&](int a, int b) { return P.colour[a] < P.colour[b]; });
  P.colour_ptr.assign(P.ncolours + 1, 0);
  for (int i = 0; i < M; ++i) P.colour_ptr[P.colour[i] + 1]++;
  for (int c = 0; c < P.ncolours; ++c) P.colour_ptr[c + 1] += P.colour_ptr[c];

  // chunks of blocks for the parallel per-block passes
  const int nch = std::max(1, std::min(host_threads() * 4, (M + 127) / 128));
  std::vector<int64_t> cb(nch + 1);
  for (int c = 0; c <= nch; ++c) cb[c] = (int64_t)M * c / nch;

  // ---- squared pattern (close + far), rows i, columns k >= i -------------
  {
    std::vector<std::vector<int>> cnt(nch), rows(nch);
    parallel_for(nch, 1, [&](int64_t b, int64_t e) {
      std::vector<int> buf;
      for (int64_t c = b; c < e; ++c) {
        cnt[c].resize(cb[c + 1] - cb[c]);
        for (int64_t i = cb[c]; i < cb[c + 1]; ++i) {
          buf.clear();
          for (const int* j = adj.row(i); j != adj.row(i) + adj.deg(i); ++j)
            for (const int* k = adj.row(*j); k != adj.row(*j) + adj.deg(*j); ++k)
              if (*k >= i) buf.push_back(*k);
          std::sort(buf.begin(), buf.end());
          buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
          cnt[c][i - cb[c]] = static_cast<int>(buf.size());
          rows[c].insert(rows[c].end(), buf.begin(), buf.end());
        }
      }
    });
    join_chunks<int, int>(M, nch, cnt, rows, nullptr, P.pair_ptr, P.pair_k, nullptr, cb);
  }
  const int np = P.pair_ptr[M];
  P.pair_i.resize(np);
  P.pair_close.resize(np);
  parallel_for(M, 2048, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i)
      for (int p = P.pair_ptr[i]; p < P.pair_ptr[i + 1]; ++p) {
        P.pair_i[p] = static_cast<int>(i);
        P.pair_close[p] = adj.has(static_cast<int>(i), P.pair_k[p]);
      }
  });
  auto pair_idx = [&](int a, int b) -> int {
    const int p = find_pair_idx(P, a, b);
    if (p < 0) throw std::logic_error("pair outside squared pattern");
    return p;
  };

  // ---- per block lists (as pair indices) ---------------------------------
  P.diag_pidx.resize(M);
  {
    std::vector<std::vector<int>> ccnt(nch), fcnt(nch), scnt(nch), cblk(nch), fblk(nch), cpi(nch), fpi(nch),
        spi(nch);
    parallel_for(nch, 1, [&](int64_t b, int64_t e) {
      std::vector<int> cand, T;
      for (int64_t c = b; c < e; ++c) {
        const int64_t nb = cb[c + 1] - cb[c];
        ccnt[c].resize(nb);
        fcnt[c].resize(nb);
        scnt[c].resize(nb);
        for (int64_t ii = cb[c]; ii < cb[c + 1]; ++ii) {
          const int i = static_cast<int>(ii);
          const int* ai = adj.row(i);
          const int di = adj.deg(i);
          P.diag_pidx[i] = pair_idx(i, i);
          T.assign(1, i);
          for (const int* k = ai; k != ai + di; ++k)
            if (*k != i) {
              cblk[c].push_back(*k);
              cpi[c].push_back(pair_idx(i, *k));
              T.push_back(*k);
            }
          ccnt[c][i - cb[c]] = di - 1;
          // far blocks of row i that hold fill when i is processed: a close
          // neighbour j of i of an earlier colour also neighbours k, and k
          // is not close to i
          cand.clear();
          for (const int* j = ai; j != ai + di; ++j) {
            if (*j == i || P.colour[*j] >= P.colour[i]) continue;
            for (const int* k = adj.row(*j); k != adj.row(*j) + adj.deg(*j); ++k)
              if (*k != i && !std::binary_search(ai, ai + di, *k)) cand.push_back(*k);
          }
          std::sort(cand.begin(), cand.end());
          cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
          for (int k : cand) {
            fblk[c].push_back(k);
            fpi[c].push_back(pair_idx(i, k));
          }
          fcnt[c][i - cb[c]] = static_cast<int>(cand.size());
          // Schur targets T = [i] + close(i): all pairs (T[a], T[b]), a <= b.
          // T[1:] ascends, so row T[a]'s pairs are walked once for all b.
          for (size_t x = 0; x < T.size(); ++x) {
            int p = P.pair_ptr[T[x]];
            for (size_t y = x; y < T.size(); ++y) {
              if (x == 0 && y > 0 && T[y] < T[0]) {  // pair stored under row T[y]
                spi[c].push_back(pair_idx(T[0], T[y]));
                continue;
              }
              while (p < P.pair_ptr[T[x] + 1] && P.pair_k[p] < T[y]) ++p;
              if (p >= P.pair_ptr[T[x] + 1] || P.pair_k[p] != T[y]) throw std::logic_error("pair outside squared pattern");
              spi[c].push_back(p);
            }
          }
          scnt[c][i - cb[c]] = static_cast<int>(T.size() * (T.size() + 1) / 2);
        }
      }
    });
    join_chunks<int, int>(M, nch, ccnt, cblk, &cpi, P.close_ptr, P.close_blk, &P.close_pidx, cb);
    join_chunks<int, int>(M, nch, fcnt, fblk, &fpi, P.far_ptr, P.far_blk, &P.far_pidx, cb);
    join_chunks<int, int>(M, nch, scnt, spi, nullptr, P.schur_ptr, P.schur_pidx, nullptr, cb);
  }

  // ---- dependencies of the persistent launches ----------------------------
  P.dep_ptr.assign(M + 1, 0);
  for (int p = 0; p < np; ++p) {
    const int i = P.pair_i[p], k = P.pair_k[p];
    if (i == k) continue;
    if (P.colour[k] < P.colour[i]) ++P.dep_ptr[i + 1];
    else if (P.colour[i] < P.colour[k]) ++P.dep_ptr[k + 1];
  }
  for (int i = 0; i < M; ++i) P.dep_ptr[i + 1] += P.dep_ptr[i];
  P.dep_idx.resize(P.dep_ptr[M]);
  {
    std::vector<int> fill(P.dep_ptr.begin(), P.dep_ptr.end() - 1);
    for (int p = 0; p < np; ++p) {
      const int i = P.pair_i[p], k = P.pair_k[p];
      if (i == k) continue;
      if (P.colour[k] < P.colour[i]) P.dep_idx[fill[i]++] = k;
      else if (P.colour[i] < P.colour[k]) P.dep_idx[fill[k]++] = i;
    }
  }
  P.rdep_ptr.assign(M + 1, 0);
  for (int k : P.dep_idx) ++P.rdep_ptr[k + 1];
  for (int i = 0; i < M; ++i) P.rdep_ptr[i + 1] += P.rdep_ptr[i];
  P.rdep_idx.resize(P.dep_idx.size());
  {
    std::vector<int> fill(P.rdep_ptr.begin(), P.rdep_ptr.end() - 1);
    for (int i = 0; i < M; ++i)
      for (int d = P.dep_ptr[i]; d < P.dep_ptr[i + 1]; ++d) P.rdep_idx[fill[P.dep_idx[d]]++] = i;
  }
}

void plan_layout(LevelPlan& P, const std::vector<int>& n) {
  const int M = P.M;
  P.n = n;
  const int np = static_cast<int>(P.pair_k.size());
  P.pair_off.resize(np);
  int64_t off = 0;
  for (int p = 0; p < np; ++p) {
    P.pair_off[p] = off;
    off += static_cast<int64_t>(n[P.pair_i[p]]) * n[P.pair_k[p]];
  }
  P.pool_elems = off;
  auto gather = [&](const std::vector<int>& idx, std::vector<int64_t>& out) {
    out.resize(idx.size());
    parallel_for(static_cast<int64_t>(idx.size()), 65536, [&](int64_t b, int64_t e) {
      for (int64_t t = b; t < e; ++t) out[t] = P.pair_off[idx[t]];
    });
  };
  gather(P.close_pidx, P.close_off);
  gather(P.far_pidx, P.far_off);
  gather(P.schur_pidx, P.schur_off);
  gather(P.diag_pidx, P.diag_off);
  // ---- factor and vector layout ------------------------------------------
  P.u_off.resize(M);
  P.l_off.resize(M);
  P.w_off.resize(M);
  P.vec_off.resize(M);
  int64_t uo = 0, lo = 0, wo = 0, vo = 0;
  P.nmax = 0;
  for (int i = 0; i < M; ++i) {
    const int64_t ni = n[i];
    P.nmax = std::max(P.nmax, n[i]);
    P.u_off[i] = uo;
    uo += ni * ni;
    P.l_off[i] = lo;
    lo += ni * ni;
    int64_t wmax = ni;
    for (int t = P.close_ptr[i]; t < P.close_ptr[i + 1]; ++t) wmax += n[P.close_blk[t]];
    P.w_off[i] = wo;
    wo += ni * wmax;
    P.vec_off[i] = vo;
    vo += ni;
  }
  P.u_elems = uo;
  P.l_elems = lo;
  P.w_elems = wo;
  P.vec_len = vo;

  // size buckets (batches only): a system goes by its largest block; the
  // colour-major order is partitioned stably by bucket
  P.bucket_ptr.assign(1, 0);
  P.bucket_nmax.clear();
  if (P.sys_off.size() > 2) {
    std::vector<int> bkt(M, 0);
    for (size_t s = 0; s + 1 < P.sys_off.size(); ++s) {
      int mx = 0;
      for (int i = P.sys_off[s]; i < P.sys_off[s + 1]; ++i) mx = std::max(mx, n[i]);
      const int b = mx <= 16 ? 0 : (mx <= 32 ? 1 : 2);
      for (int i = P.sys_off[s]; i < P.sys_off[s + 1]; ++i) bkt[i] = b;
    }
    std::vector<int> ord;
    ord.reserve(M);
    for (int b = 0; b < kBuckets; ++b) {
      int mx = 0;
      const size_t start = ord.size();
      for (int i : P.order)
        if (bkt[i] == b) {
          ord.push_back(i);
          mx = std::max(mx, n[i]);
        }
      if (ord.size() > start) {
        P.bucket_ptr.push_back(static_cast<int>(ord.size()));
        P.bucket_nmax.push_back(mx);
      }
    }
    P.order = std::move(ord);
  } else {
    P.bucket_ptr.push_back(M);
    P.bucket_nmax.push_back(P.nmax);
  }
}

void plan_level(LevelPlan& P, const std::vector<int>& n,
                const std::vector<std::pair<int, int>>& close_pairs, int coloring,
                const std::vector<int>& sys_off) {
  plan_structure(P, static_cast<int>(n.size()), close_pairs, coloring, sys_off);
  plan_layout(P, n);
}

std::vector<int> coarsen_parents(const LevelPlan& P, int J, const std::vector<int>* rank, int nmax,
                                 std::vector<int>* first_child, std::vector<int>* sys_off) {
  const int M = P.M;
  std::vector<int> so = P.sys_off;
  if (so.empty()) so = {0, M};
  std::vector<int> parent(M, 0);
  if (first_child) first_child->assign(1, 0);
  if (sys_off) sys_off->assign(so.size(), 0);
  int next = 0;
  // emit [a, b) as one super-block, or halve it (first half ceil(len/2)) while
  // its ranks add up to more than nmax rows (nmax <= 0: no cap)
  std::vector<std::pair<int, int>> stack;
  auto emit_run = [&](int a0, int b0) {
    stack.assign(1, {a0, b0});
    while (!stack.empty()) {
      const auto [a, b] = stack.back();
      stack.pop_back();
      int tot = 0;
      if (rank)
        for (int i = a; i < b; ++i) tot += (*rank)[i];
      if (b - a == 1 || !rank || nmax <= 0 || tot <= nmax) {
        for (int i = a; i < b; ++i) parent[i] = next;
        if (first_child) first_child->push_back(b);
        ++next;
      } else {
        const int mid = a + (b - a + 1) / 2;
        stack.push_back({mid, b});  // the first half is emitted first
        stack.push_back({a, mid});
      }
    }
  };
  for (size_t s = 0; s + 1 < so.size(); ++s) {
    if (sys_off) (*sys_off)[s] = next;
    // runs of J consecutive blocks of the same system
    for (int a = so[s]; a < so[s + 1]; a += J) emit_run(a, std::min(a + J, so[s + 1]));
  }
  if (sys_off) sys_off->back() = next;
  return parent;
}

NextLevel coarsen_structure(const LevelPlan& P, const std::vector<char>& live, int J, const std::vector<int>* rank,
                            int nmax) {
  NextLevel nx;
  std::vector<int> first_child;  // children of super-block I: [first_child[I], first_child[I+1])
  nx.parent = coarsen_parents(P, J, rank, nmax, &first_child, &nx.sys_off);
  const int next = static_cast<int>(first_child.size()) - 1;
  nx.M = next;
  // super-block rows in parallel: parents of the children's pairs with a
  // non-empty basis on both sides (parent() is monotone, so K >= I)
  const int nch = std::max(1, std::min(host_threads() * 4, (next + 127) / 128));
  std::vector<std::vector<std::pair<int, int>>> part(nch);
  parallel_for(nch, 1, [&](int64_t b, int64_t e) {
    std::vector<int> buf;
    for (int64_t c = b; c < e; ++c) {
      const int I0 = static_cast<int>((int64_t)next * c / nch), I1 = static_cast<int>((int64_t)next * (c + 1) / nch);
      for (int I = I0; I < I1; ++I) {
        buf.clear();
        for (int i = first_child[I]; i < first_child[I + 1]; ++i) {
          if (!live[i]) continue;
          for (int p = P.pair_ptr[i]; p < P.pair_ptr[i + 1]; ++p)
            if (live[P.pair_k[p]]) buf.push_back(nx.parent[P.pair_k[p]]);
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        for (int K : buf) part[c].emplace_back(I, K);
      }
    }
  });
  size_t tot = 0;
  for (auto& v : part) tot += v.size();
  nx.pairs.reserve(tot);
  for (auto& v : part) nx.pairs.insert(nx.pairs.end(), v.begin(), v.end());
  return nx;
}

void coarsen_sizes(const LevelPlan& P, const std::vector<int>& rank, NextLevel& nx) {
  nx.n.assign(nx.M, 0);
  nx.child_off.assign(P.M, 0);
  for (int i = 0; i < P.M; ++i) {
    nx.child_off[i] = nx.n[nx.parent[i]];
    nx.n[nx.parent[i]] += rank[i];
  }
}

NextLevel coarsen(const LevelPlan& P, const std::vector<int>& rank, int J, int nmax) {
  std::vector<char> live(P.M);
  for (int i = 0; i < P.M; ++i) live[i] = rank[i] != 0;
  NextLevel nx = coarsen_structure(P, live, J, &rank, nmax);
  coarsen_sizes(P, rank, nx);
  return nx;
}

}  // namespace ce
