// Variable order by bandwidth reduction (Appendix A.3).  Updates of variables that share a
// subproblem should run close together in the order; a low-bandwidth permutation of the
// constraint matrix gives such an order.  This is the Cuthill-McKee heuristic run on the
// bipartite graph with one node per variable and one per row (an edge per nonzero coefficient);
// the variable order is the order in which the search reaches the variable nodes.
//
// Host code only.  Start nodes follow the pseudo-peripheral node search of Gibbs, Poole and
// Stockmeyer as simplified by George and Liu: from a node of least degree, search breadth-first,
// move to a least-degree node of the last level, and repeat while the eccentricity grows.
#include <algorithm>
#include <new>
#include <vector>

#include "bdd_dbca.h"

namespace {

struct Bipartite {
  int V = 0;                   // nodes: variables 0..n-1, then rows n..n+m-1
  std::vector<long long> ptr;  // CSR adjacency
  std::vector<int> adj;
  std::vector<int> deg;
};

// Breadth-first search from s inside s's component; marks nodes with `stamp`.  Returns the
// eccentricity of s; `last` receives the nodes of the last level, `comp` every node reached.
int bfs(const Bipartite &g, int s, int stamp, std::vector<int> &mark, std::vector<int> &comp,
        std::vector<int> &last) {
  comp.clear();
  comp.push_back(s);
  mark[s] = stamp;
  size_t head = 0, level_start = 0;
  int ecc = 0;
  while (true) {
    const size_t level_end = comp.size();
    for (head = level_start; head < level_end; ++head) {
      const int u = comp[head];
      for (long long t = g.ptr[u]; t < g.ptr[u + 1]; ++t) {
        const int v = g.adj[t];
        if (mark[v] != stamp) {
          mark[v] = stamp;
          comp.push_back(v);
        }
      }
    }
    if (comp.size() == level_end) {
      last.assign(comp.begin() + (long long)level_start, comp.begin() + (long long)level_end);
      return ecc;
    }
    level_start = level_end;
    ++ecc;
  }
}

int least_degree(const Bipartite &g, const std::vector<int> &nodes) {
  int best = nodes[0];
  for (int v : nodes)
    if (g.deg[v] < g.deg[best] || (g.deg[v] == g.deg[best] && v < best)) best = v;
  return best;
}

int order_variables(int n, int m, const long long *row_ptr, const int *col, const int *val, int *rank) {
  Bipartite g;
  g.V = n + m;
  g.deg.assign(g.V, 0);
  for (int j = 0; j < m; ++j)
    for (long long t = row_ptr[j]; t < row_ptr[j + 1]; ++t) {
      if (val && val[t] == 0) continue;
      g.deg[col[t]]++;
      g.deg[n + j]++;
    }
  g.ptr.assign((size_t)g.V + 1, 0);
  for (int v = 0; v < g.V; ++v) g.ptr[v + 1] = g.ptr[v] + g.deg[v];
  g.adj.assign((size_t)g.ptr[g.V], 0);
  std::vector<long long> fill(g.ptr.begin(), g.ptr.end() - 1);
  for (int j = 0; j < m; ++j)
    for (long long t = row_ptr[j]; t < row_ptr[j + 1]; ++t) {
      if (val && val[t] == 0) continue;
      const int i = col[t];
      g.adj[fill[i]++] = n + j;
      g.adj[fill[n + j]++] = i;
    }

  std::vector<int> mark(g.V, 0), comp, last, seq;
  std::vector<char> placed(g.V, 0);
  std::vector<int> nb;
  int stamp = 0, next_rank = 0;
  seq.reserve(g.V);
  for (int i0 = 0; i0 < n; ++i0) {
    if (placed[i0] || g.deg[i0] == 0) continue;
    // pseudo-peripheral start of i0's component
    bfs(g, i0, ++stamp, mark, comp, last);
    int r = least_degree(g, comp);
    int ecc = bfs(g, r, ++stamp, mark, comp, last);
    for (int guard = 0; guard < g.V; ++guard) {
      const int x = least_degree(g, last);
      std::vector<int> last_x;
      const int ecc_x = bfs(g, x, ++stamp, mark, comp, last_x);
      if (ecc_x <= ecc) break;
      r = x;
      ecc = ecc_x;
      last.swap(last_x);
    }
    // Cuthill-McKee: breadth-first, unvisited neighbours by ascending degree, then index
    seq.clear();
    seq.push_back(r);
    placed[r] = 1;
    for (size_t head = 0; head < seq.size(); ++head) {
      const int u = seq[head];
      nb.clear();
      for (long long t = g.ptr[u]; t < g.ptr[u + 1]; ++t) {
        const int v = g.adj[t];
        if (!placed[v]) {
          placed[v] = 1;
          nb.push_back(v);
        }
      }
      std::sort(nb.begin(), nb.end(), [&](int a, int b) {
        return g.deg[a] != g.deg[b] ? g.deg[a] < g.deg[b] : a < b;
      });
      seq.insert(seq.end(), nb.begin(), nb.end());
    }
    for (int v : seq)
      if (v < n) rank[v] = next_rank++;
  }
  for (int i = 0; i < n; ++i)
    if (g.deg[i] == 0) rank[i] = next_rank++;
  return next_rank == n ? BDD_OK : BDD_EINVAL;
}

}  // namespace

extern "C" int bdd_cuthill_mckee(int n, int m, const long long *row_ptr, const int *col, const int *val,
                                 int *rank) {
  if (n < 0 || m < 0 || (n > 0 && !rank) || (m > 0 && !row_ptr)) return BDD_EINVAL;
  if ((long long)n + m >= 2147483647LL) return BDD_EINVAL;
  if (m > 0) {
    if (row_ptr[0] != 0) return BDD_EINVAL;
    for (int j = 0; j < m; ++j)
      if (row_ptr[j + 1] < row_ptr[j]) return BDD_EINVAL;
    if (row_ptr[m] > 0 && !col) return BDD_EINVAL;
    for (long long t = 0; t < row_ptr[m]; ++t)
      if (col[t] < 0 || col[t] >= n) return BDD_EINVAL;
  }
  try {
    return order_variables(n, m, row_ptr, col, val, rank);
  } catch (const std::bad_alloc &) {
    return BDD_ENOMEM;
  }
}
