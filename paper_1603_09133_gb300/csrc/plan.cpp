// Host symbolic planning of one CE level (block graph, squared pattern,
// distance-2 colouring, offsets) and of the reassembly into super-blocks.
//
// Section 2.2: eliminating a block sub-row only creates blocks inside the
// pattern of A^2 ("far" blocks are nonzero in A^2 and zero in A), so every
// pair a level can touch is known before its numeric phase and is
// preallocated here.  Section 2.4 (eq. bsp): after a sweep, J consecutive
// blocks join into one super-block; the next level's pattern is the
// coarsened squared pattern restricted to blocks with a non-empty basis.
#include <algorithm>
#include <numeric>
#include <stdexcept>

#include "ce_internal.h"

namespace ce {

namespace {

// sorted adjacency (diagonal included) from a list of pairs
std::vector<std::vector<int>> adjacency(int M, const std::vector<std::pair<int, int>>& pairs) {
  std::vector<std::vector<int>> adj(M);
  for (int i = 0; i < M; ++i) adj[i].push_back(i);
  for (auto& p : pairs) {
    if (p.first == p.second) continue;
    adj[p.first].push_back(p.second);
    adj[p.second].push_back(p.first);
  }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  return adj;
}

bool contains(const std::vector<int>& v, int x) {
  return std::binary_search(v.begin(), v.end(), x);
}

}  // namespace

void plan_level(LevelPlan& P, const std::vector<int>& n,
                const std::vector<std::pair<int, int>>& close_pairs, bool coloring) {
  const int M = static_cast<int>(n.size());
  P = LevelPlan();
  P.M = M;
  P.n = n;
  auto adj = adjacency(M, close_pairs);

  // ---- greedy distance-2 colouring, ascending block index ----------------
  P.colour.assign(M, -1);
  if (coloring) {
    std::vector<int> mark;  // mark[c] == i  <=> colour c is taken near i
    for (int i = 0; i < M; ++i) {
      for (int j : adj[i])
        for (int k : adj[j])
          if (k != i && P.colour[k] >= 0) {
            int c = P.colour[k];
            if (c >= static_cast<int>(mark.size())) mark.resize(c + 1, -1);
            mark[c] = i;
          }
      int c = 0;
      while (c < static_cast<int>(mark.size()) && mark[c] == i) ++c;
      P.colour[i] = c;
    }
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

  // ---- squared pattern (close + far), rows i, columns k >= i -------------
  std::vector<std::vector<int>> sq(M);
  for (int j = 0; j < M; ++j)
    for (int a : adj[j])
      for (int b : adj[j])
        if (a <= b) sq[a].push_back(b);
  std::vector<int> row_ptr(M + 1, 0);
  for (int i = 0; i < M; ++i) {
    auto& v = sq[i];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    row_ptr[i + 1] = row_ptr[i] + static_cast<int>(v.size());
  }
  const int np = row_ptr[M];
  P.pair_i.resize(np);
  P.pair_k.resize(np);
  P.pair_off.resize(np);
  P.pair_close.resize(np);
  int64_t off = 0;
  for (int i = 0; i < M; ++i)
    for (int t = 0; t < static_cast<int>(sq[i].size()); ++t) {
      int p = row_ptr[i] + t, k = sq[i][t];
      P.pair_i[p] = i;
      P.pair_k[p] = k;
      P.pair_off[p] = off;
      P.pair_close[p] = contains(adj[i], k);
      off += static_cast<int64_t>(n[i]) * n[k];
    }
  P.pool_elems = off;
  auto pair_offset = [&](int a, int b) -> int64_t {
    if (a > b) std::swap(a, b);
    auto& v = sq[a];
    auto it = std::lower_bound(v.begin(), v.end(), b);
    if (it == v.end() || *it != b) throw std::logic_error("pair outside squared pattern");
    return P.pair_off[row_ptr[a] + static_cast<int>(it - v.begin())];
  };

  // ---- per block lists ----------------------------------------------------
  P.close_ptr.assign(M + 1, 0);
  P.far_ptr.assign(M + 1, 0);
  P.schur_ptr.assign(M + 1, 0);
  P.diag_off.resize(M);
  for (int i = 0; i < M; ++i) {
    P.diag_off[i] = pair_offset(i, i);
    std::vector<int> cl;
    for (int k : adj[i])
      if (k != i) cl.push_back(k);
    for (int k : cl) {
      P.close_blk.push_back(k);
      P.close_off.push_back(pair_offset(i, k));
    }
    P.close_ptr[i + 1] = static_cast<int>(P.close_blk.size());
    // far blocks of row i that hold fill when i is processed: some common
    // close neighbour j of i and k was eliminated earlier
    std::vector<int> cand;
    for (int j : adj[i])
      for (int k : adj[j])
        if (k != i && !contains(adj[i], k)) cand.push_back(k);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (int k : cand) {
      bool live = false;
      for (int j : adj[i])
        if (j != i && j != k && P.colour[j] < P.colour[i] && contains(adj[k], j)) {
          live = true;
          break;
        }
      if (live) {
        P.far_blk.push_back(k);
        P.far_off.push_back(pair_offset(i, k));
      }
    }
    P.far_ptr[i + 1] = static_cast<int>(P.far_blk.size());
    // Schur targets T = [i] + close(i): all pairs (T[a], T[b]), a <= b
    std::vector<int> T;
    T.push_back(i);
    T.insert(T.end(), cl.begin(), cl.end());
    for (size_t a = 0; a < T.size(); ++a)
      for (size_t b = a; b < T.size(); ++b) P.schur_off.push_back(pair_offset(T[a], T[b]));
    P.schur_ptr[i + 1] = static_cast<int>(P.schur_off.size());
  }

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
}

NextLevel coarsen(const LevelPlan& P, const std::vector<int>& rank, int J) {
  NextLevel nx;
  const int M = P.M;
  std::vector<int> so = P.sys_off;
  if (so.empty()) so = {0, M};
  nx.parent.assign(M, 0);
  nx.child_off.assign(M, 0);
  nx.sys_off.assign(so.size(), 0);
  int next = 0;
  for (size_t s = 0; s + 1 < so.size(); ++s) {
    nx.sys_off[s] = next;
    // J consecutive blocks of the same system form one super-block
    for (int i = so[s]; i < so[s + 1]; ++i) nx.parent[i] = next + (i - so[s]) / J;
    next += (so[s + 1] - so[s] + J - 1) / J;
  }
  nx.sys_off.back() = next;
  nx.n.assign(next, 0);
  for (int i = 0; i < M; ++i) {
    nx.child_off[i] = nx.n[nx.parent[i]];
    nx.n[nx.parent[i]] += rank[i];
  }
  std::vector<std::pair<int, int>> pr;
  for (size_t p = 0; p < P.pair_i.size(); ++p) {
    int i = P.pair_i[p], k = P.pair_k[p];
    if (rank[i] == 0 || rank[k] == 0) continue;
    pr.emplace_back(nx.parent[i], nx.parent[k]);
  }
  std::sort(pr.begin(), pr.end());
  pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
  nx.pairs = std::move(pr);
  return nx;
}

}  // namespace ce
