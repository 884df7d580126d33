// Host-side structural analysis (see analysis.h).
#include "analysis.h"

#include <algorithm>
#include <numeric>
#include <queue>
#include <set>
#include <utility>

namespace gpcg {

BusGraph build_bus_graph(int n_bus, int n_branch, const int32_t* f, const int32_t* t) {
  BusGraph g;
  g.adj.n = n_bus;
  g.adj.ptr.assign(n_bus + 1, 0);
  for (int e = 0; e < n_branch; ++e) {
    g.adj.ptr[f[e] + 1]++;
    g.adj.ptr[t[e] + 1]++;
  }
  for (int b = 0; b < n_bus; ++b) g.adj.ptr[b + 1] += g.adj.ptr[b];
  g.adj.idx.resize(g.adj.ptr[n_bus]);
  g.adj_branch.resize(g.adj.ptr[n_bus]);
  std::vector<int32_t> fill(g.adj.ptr.begin(), g.adj.ptr.end() - 1);
  for (int e = 0; e < n_branch; ++e) {
    int a = f[e], b = t[e];
    g.adj.idx[fill[a]] = b; g.adj_branch[fill[a]++] = e;
    g.adj.idx[fill[b]] = a; g.adj_branch[fill[b]++] = e;
  }
  // sort each bus's neighbours (then branch) so every later pass is deterministic
  for (int b = 0; b < n_bus; ++b) {
    int s = g.adj.ptr[b], n = g.adj.ptr[b + 1] - s;
    std::vector<std::pair<int, int>> v(n);
    for (int k = 0; k < n; ++k) v[k] = {g.adj.idx[s + k], g.adj_branch[s + k]};
    std::sort(v.begin(), v.end());
    for (int k = 0; k < n; ++k) { g.adj.idx[s + k] = v[k].first; g.adj_branch[s + k] = v[k].second; }
  }
  return g;
}

namespace {

// Minimum-degree ordering on the elimination graph, ties broken by the
// smallest vertex index.  Also returns, for every vertex, its uneliminated
// neighbours at the moment it is eliminated (= its column of the complete
// Cholesky factor).
void minimum_degree(const std::vector<std::vector<int>>& adj0, std::vector<int>& order,
                    std::vector<std::vector<int>>& elim_cols) {
  int n = (int)adj0.size();
  std::vector<std::set<int>> adj(n);
  for (int v = 0; v < n; ++v) adj[v].insert(adj0[v].begin(), adj0[v].end());
  std::set<std::pair<int, int>> pq;
  for (int v = 0; v < n; ++v) pq.insert({(int)adj[v].size(), v});
  std::vector<char> done(n, 0);
  order.clear();
  elim_cols.assign(n, {});
  while (!pq.empty()) {
    auto it = pq.begin();
    int v = it->second;
    pq.erase(it);
    done[v] = 1;
    order.push_back(v);
    std::vector<int> nb(adj[v].begin(), adj[v].end());
    elim_cols[v] = nb;
    for (int u : nb) {
      pq.erase({(int)adj[u].size(), u});
      adj[u].erase(v);
      for (int w : nb)
        if (w != u) adj[u].insert(w);
      pq.insert({(int)adj[u].size(), u});
    }
    adj[v].clear();
  }
}

Csr transpose_pattern(const Csr& M, std::vector<int32_t>* pos_map) {
  Csr T;
  T.n = M.n;
  T.ptr.assign(M.n + 1, 0);
  for (int i = 0; i < M.n; ++i)
    for (int k = M.ptr[i]; k < M.ptr[i + 1]; ++k) T.ptr[M.idx[k] + 1]++;
  for (int i = 0; i < M.n; ++i) T.ptr[i + 1] += T.ptr[i];
  T.idx.resize(T.ptr[M.n]);
  if (pos_map) pos_map->resize(M.nnz());
  std::vector<int32_t> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < M.n; ++i)  // rows in increasing order -> T's cols sorted
    for (int k = M.ptr[i]; k < M.ptr[i + 1]; ++k) {
      int j = M.idx[k];
      int p = fill[j]++;
      T.idx[p] = i;
      if (pos_map) (*pos_map)[k] = p;
    }
  return T;
}

}  // namespace

MatrixPlan plan_matrix(int n_bus, const BusGraph& g, const std::vector<uint8_t>& keep,
                       bool fill) {
  MatrixPlan P;
  std::vector<int32_t> loc(n_bus, -1), bus_of_loc;
  for (int b = 0; b < n_bus; ++b)
    if (keep[b]) { loc[b] = (int)bus_of_loc.size(); bus_of_loc.push_back(b); }
  int n = (int)bus_of_loc.size();
  P.n = n;
  std::vector<std::vector<int>> adj(n);
  for (int v = 0; v < n; ++v) {
    int b = bus_of_loc[v];
    for (int k = g.adj.ptr[b]; k < g.adj.ptr[b + 1]; ++k) {
      int c = loc[g.adj.idx[k]];
      if (c >= 0 && c != v) adj[v].push_back(c);
    }
    std::sort(adj[v].begin(), adj[v].end());
    adj[v].erase(std::unique(adj[v].begin(), adj[v].end()), adj[v].end());
  }
  std::vector<int> order;
  std::vector<std::vector<int>> elim_cols;
  minimum_degree(adj, order, elim_cols);
  std::vector<int> pos(n);  // local vertex -> position in the minimum-degree order
  for (int k = 0; k < n; ++k) pos[order[k]] = k;

  // lower pattern (in minimum-degree numbering): row i holds cols j < i
  std::vector<std::vector<int>> lrows(n);
  for (int k = 0; k < n; ++k) lrows[k].push_back(k);
  if (fill) {
    for (int v = 0; v < n; ++v)
      for (int u : elim_cols[v]) lrows[pos[u]].push_back(pos[v]);
  } else {
    for (int v = 0; v < n; ++v)
      for (int u : adj[v])
        if (pos[u] < pos[v]) lrows[pos[v]].push_back(pos[u]);
  }
  // forward levels, then a stable sort of rows by level
  std::vector<int> lev(n, 0);
  for (int i = 0; i < n; ++i) {
    int m = -1;
    for (int j : lrows[i])
      if (j != i) m = std::max(m, lev[j]);
    lev[i] = m + 1;
  }
  // final order: by level; within a level by vertex (= bus) index, so rows of
  // a level that are close in the bus numbering are close in memory
  std::vector<int> byl(n);
  std::iota(byl.begin(), byl.end(), 0);
  std::sort(byl.begin(), byl.end(), [&](int a, int b) {
    return lev[a] != lev[b] ? lev[a] < lev[b] : order[a] < order[b];
  });
  std::vector<int> fin(n);  // minimum-degree position -> final row
  for (int r = 0; r < n; ++r) fin[byl[r]] = r;

  P.bus_of_row.resize(n);
  P.row_of_bus.assign(n_bus, -1);
  P.level.resize(n);
  for (int r = 0; r < n; ++r) {
    int md = byl[r];
    int v = order[md];
    P.bus_of_row[r] = bus_of_loc[v];
    P.row_of_bus[bus_of_loc[v]] = r;
    P.level[r] = lev[md];
  }
  int nlev = n ? (*std::max_element(lev.begin(), lev.end()) + 1) : 0;
  P.lev_ptr.assign(nlev + 1, 0);
  for (int r = 0; r < n; ++r) P.lev_ptr[P.level[r] + 1]++;
  for (int k = 0; k < nlev; ++k) P.lev_ptr[k + 1] += P.lev_ptr[k];

  // L in final numbering
  P.L.n = n;
  P.L.ptr.assign(n + 1, 0);
  std::vector<std::vector<int>> fl(n);
  for (int md = 0; md < n; ++md) {
    int r = fin[md];
    for (int j : lrows[md]) fl[r].push_back(fin[j]);
    std::sort(fl[r].begin(), fl[r].end());
    fl[r].erase(std::unique(fl[r].begin(), fl[r].end()), fl[r].end());
  }
  for (int r = 0; r < n; ++r) P.L.ptr[r + 1] = P.L.ptr[r] + (int)fl[r].size();
  P.L.idx.reserve(P.L.ptr[n]);
  for (int r = 0; r < n; ++r) P.L.idx.insert(P.L.idx.end(), fl[r].begin(), fl[r].end());
  P.U = transpose_pattern(P.L, &P.l_to_u);

  // A in final numbering (symmetric, with diagonal)
  P.A.n = n;
  P.A.ptr.assign(n + 1, 0);
  std::vector<std::vector<int>> ar(n);
  for (int v = 0; v < n; ++v) {
    int r = fin[pos[v]];
    ar[r].push_back(r);
    for (int u : adj[v]) ar[r].push_back(fin[pos[u]]);
    std::sort(ar[r].begin(), ar[r].end());
  }
  for (int r = 0; r < n; ++r) P.A.ptr[r + 1] = P.A.ptr[r] + (int)ar[r].size();
  P.A.idx.reserve(P.A.ptr[n]);
  P.a_diag.resize(n);
  for (int r = 0; r < n; ++r) {
    for (size_t k = 0; k < ar[r].size(); ++k)
      if (ar[r][k] == r) P.a_diag[r] = P.A.ptr[r] + (int)k;
    P.A.idx.insert(P.A.idx.end(), ar[r].begin(), ar[r].end());
  }

  // backward levels: row i waits for the rows j > i with L_ji != 0
  std::vector<int> blev(n, 0);
  for (int i = n - 1; i >= 0; --i) {
    int m = -1;
    for (int k = P.U.ptr[i]; k < P.U.ptr[i + 1]; ++k) {
      int j = P.U.idx[k];
      if (j != i) m = std::max(m, blev[j]);
    }
    blev[i] = m + 1;
  }
  int nb = n ? (*std::max_element(blev.begin(), blev.end()) + 1) : 0;
  P.blev_ptr.assign(nb + 1, 0);
  for (int i = 0; i < n; ++i) P.blev_ptr[blev[i] + 1]++;
  for (int k = 0; k < nb; ++k) P.blev_ptr[k + 1] += P.blev_ptr[k];
  P.blev_rows.resize(n);
  std::vector<int32_t> bf(P.blev_ptr.begin(), P.blev_ptr.end() - 1);
  for (int i = 0; i < n; ++i) P.blev_rows[bf[blev[i]]++] = i;
  return P;
}

void plan_tail(MatrixPlan& P, int max_rows) {
  const int n = P.n, nlev = (int)P.lev_ptr.size() - 1;
  int tl = nlev;
  while (tl > 0 && n - P.lev_ptr[tl - 1] <= max_rows) --tl;
  if (nlev - tl < 2) tl = nlev;  // a single level gains nothing
  P.tail_lev = tl;
  P.tail_row0 = nlev > 0 ? P.lev_ptr[tl] : 0;
  const int t0 = P.tail_row0;
  // backward levels of rows < t0, waiting only for rows < t0
  std::vector<int> blev(t0, 0);
  for (int i = t0 - 1; i >= 0; --i) {
    int m = -1;
    for (int k = P.U.ptr[i]; k < P.U.ptr[i + 1]; ++k) {
      const int j = P.U.idx[k];
      if (j != i && j < t0) m = std::max(m, blev[j]);
    }
    blev[i] = m + 1;
  }
  const int nb = t0 ? (*std::max_element(blev.begin(), blev.end()) + 1) : 0;
  P.tblev_ptr.assign(nb + 1, 0);
  for (int i = 0; i < t0; ++i) P.tblev_ptr[blev[i] + 1]++;
  for (int k = 0; k < nb; ++k) P.tblev_ptr[k + 1] += P.tblev_ptr[k];
  P.tblev_rows.resize(t0);
  std::vector<int32_t> bf(P.tblev_ptr.begin(), P.tblev_ptr.end() - 1);
  for (int i = 0; i < t0; ++i) P.tblev_rows[bf[blev[i]]++] = i;
}

std::vector<int32_t> rcm_order(int n, const BusGraph& g) {
  std::vector<int32_t> deg(n), out;
  for (int v = 0; v < n; ++v) deg[v] = g.adj.ptr[v + 1] - g.adj.ptr[v];
  std::vector<char> seen(n, 0);
  out.reserve(n);
  auto bfs = [&](int s, std::vector<int32_t>& ord, std::vector<char>& mark) {
    size_t head = ord.size();
    ord.push_back(s);
    mark[s] = 1;
    std::vector<int32_t> nb;
    while (head < ord.size()) {
      const int u = ord[head++];
      nb.clear();
      for (int k = g.adj.ptr[u]; k < g.adj.ptr[u + 1]; ++k)
        if (!mark[g.adj.idx[k]]) { mark[g.adj.idx[k]] = 1; nb.push_back(g.adj.idx[k]); }
      std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
      ord.insert(ord.end(), nb.begin(), nb.end());
    }
  };
  for (int s0 = 0; s0 < n; ++s0) {
    if (seen[s0]) continue;
    // start from a pseudo-peripheral vertex: the last vertex of a BFS from s0
    std::vector<int32_t> tmp;
    std::vector<char> mark(seen);
    bfs(s0, tmp, mark);
    const int start = tmp.back();
    const size_t before = out.size();
    bfs(start, out, seen);
    std::reverse(out.begin() + before, out.end());
  }
  // within each window of 128 consecutive positions, buses of higher degree
  // first (stable): kernels that take one bus per thread in this order read
  // consecutive buses and run neighbour loops of nearly equal length in a
  // warp; the permutation stays inside the window, so neighbours stay close
  for (size_t w0 = 0; w0 < out.size(); w0 += 128)
    std::stable_sort(out.begin() + w0, out.begin() + std::min(out.size(), w0 + 128),
                     [&](int a, int b) { return deg[a] > deg[b]; });
  return out;
}

bool dfs_numbering(int n_bus, const BusGraph& g, int root, std::vector<int32_t>& pre,
                   std::vector<int32_t>& size, std::vector<uint8_t>& bridge, int n_branch) {
  pre.assign(n_bus, -1);
  size.assign(n_bus, 0);
  bridge.assign(n_branch, 0);
  std::vector<int32_t> low(n_bus, 0), parent_edge(n_bus, -1), it(n_bus, 0);
  std::vector<int> stack;
  int counter = 0;
  pre[root] = counter++;
  low[root] = pre[root];
  stack.push_back(root);
  it[root] = g.adj.ptr[root];
  while (!stack.empty()) {
    int u = stack.back();
    if (it[u] < g.adj.ptr[u + 1]) {
      int k = it[u]++;
      int v = g.adj.idx[k], e = g.adj_branch[k];
      if (e == parent_edge[u]) continue;
      if (pre[v] < 0) {
        pre[v] = counter++;
        low[v] = pre[v];
        parent_edge[v] = e;
        it[v] = g.adj.ptr[v];
        stack.push_back(v);
      } else {
        low[u] = std::min(low[u], pre[v]);
      }
    } else {
      stack.pop_back();
      size[u] += 1;
      if (!stack.empty()) {
        int p = stack.back();
        size[p] += size[u];
        low[p] = std::min(low[p], low[u]);
        if (low[u] > pre[p]) bridge[parent_edge[u]] = 1;
      }
    }
  }
  return counter == n_bus;
}

}  // namespace gpcg
