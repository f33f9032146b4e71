// Host BDD compiler and device slab layout.
//
// compile_bdds: one reduced, ordered, non-skipping BDD per constraint row (Sec. 5.1, Def. 4;
// the paper builds them with the threshold method it cites, in O(N log W), Sec. 5.2).  This
// compiler is threshold-based: with the suffix-sum set T_l = { a_l y_l + ... + a_{k-1} y_{k-1} }
// of the variables still to come, two partial sums s, s' at layer l have the same feasible
// completions iff they select the same part of T_l:
//   a.x <= b : the number of t in T_l with t <= b - s,
//   a.x >= b : the number of t in T_l with t >= b - s,
//   a.x == b : the position of b - s in T_l (if present),
// and 0 means "no completion" (the false terminal).  Nodes of layer l are the distinct nonzero
// keys among the reachable partial sums, numbered in ascending order of their smallest
// reachable partial sum (the canonical order of the library's exports).  Each node keeps one
// representative sum; its 0-/1-successors are the keys of s and s + a_l at layer l+1.
//
// build_layout: turns the canonical BDDs into the tile-grouped, layer-major slabs the sweep
// kernels read.
//
// split_bdds: sub-BDDs (Sec. 6, Def. of sub-BDDs): a BDD whose consecutive layers lie in
// different intervals of the variable order is cut there; each piece becomes a BDD of its own
// (several roots when it starts below the original root), and the arcs leaving the last layer
// before a cut go into the top terminal as copy arcs.  The pieces keep the row's occurrences, so
// the slab layout, the slots and the outputs need no change.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>

#include <unistd.h>

#include "bdd_dbca.h"
#include "internal.h"

namespace bdd {
namespace {

constexpr long long kSumCap = 1LL << 22;  // largest suffix / prefix sum set per layer

struct Scratch {
  std::vector<int> order;
  std::vector<long long> a, pos;
  std::vector<long long> tlo, thi, slo, shi;  // unit rows: the sum sets as integer ranges
  std::vector<int> cols;
  std::vector<std::vector<long long>> T, S, rep;
  std::vector<std::vector<int>> id_of_key;
};

struct Chunk {
  std::vector<int> bdd_row, bdd_depth, occ_var, occ_width, lo, hi;
  std::vector<long long> occ_csr;
  int status = BDD_OK;
  int failed_row = -1;
};

inline bool sat(long long s, int sense, long long b) {
  return sense < 0 ? s <= b : (sense > 0 ? s >= b : s == b);
}

// out = sorted distinct union of A and A + a
void merge_shift(const std::vector<long long> &A, long long a, std::vector<long long> &out) {
  out.clear();
  out.reserve(2 * A.size());
  size_t i = 0, j = 0, n = A.size();
  while (i < n || j < n) {
    long long x = i < n ? A[i] : LLONG_MAX;
    long long y = j < n ? A[j] + a : LLONG_MAX;
    long long v;
    if (x < y) {
      v = x; ++i;
    } else if (y < x) {
      v = y; ++j;
    } else {
      v = x; ++i; ++j;
    }
    if (out.empty() || out.back() != v) out.push_back(v);
  }
}

inline int key_of(const std::vector<long long> &T, long long s, long long b, int sense) {
  long long r = b - s;
  if (sense < 0) return (int)(std::upper_bound(T.begin(), T.end(), r) - T.begin());
  if (sense > 0) return (int)(T.end() - std::lower_bound(T.begin(), T.end(), r));
  auto it = std::lower_bound(T.begin(), T.end(), r);
  return (it != T.end() && *it == r) ? (int)(it - T.begin()) + 1 : 0;
}

// key_of for a set T that holds every integer of [lo, hi]: the same counts and positions without
// a search
inline int key_of_range(long long lo, long long hi, long long s, long long b, int sense) {
  const long long r = b - s, m = hi - lo + 1;
  if (sense < 0) return (int)(r < lo ? 0 : r >= hi ? m : r - lo + 1);
  if (sense > 0) return (int)(r > hi ? 0 : r <= lo ? m : hi - r + 1);
  return (r >= lo && r <= hi) ? (int)(r - lo + 1) : 0;
}

// compile_row for a row whose coefficients (in layer order, sc.a) are all +1 or -1.  Then every
// suffix-sum set T_l and every reachable prefix-sum set S_l holds all integers between its least
// and greatest element (adding 0 or +-1 to a set of consecutive integers keeps them consecutive),
// so the sets are kept as ranges and keys come from key_of_range.  The nodes, their order, the
// arcs and the checks (in the same order) are those of the general path.
int compile_unit_row(int j, long long b, int sense, int max_width, int k, Scratch &sc, Chunk &out) {
  sc.tlo.resize(k + 1);
  sc.thi.resize(k + 1);
  sc.slo.resize(k);
  sc.shi.resize(k);
  sc.tlo[k] = sc.thi[k] = 0;
  for (int l = k - 1; l >= 0; --l) {
    sc.tlo[l] = sc.tlo[l + 1] + std::min(sc.a[l], 0LL);
    sc.thi[l] = sc.thi[l + 1] + std::max(sc.a[l], 0LL);
    if (sc.thi[l] - sc.tlo[l] + 1 > kSumCap) return BDD_ETOOBIG;
  }
  sc.slo[0] = sc.shi[0] = 0;
  for (int l = 0; l + 1 < k; ++l) {
    sc.slo[l + 1] = sc.slo[l] + std::min(sc.a[l], 0LL);
    sc.shi[l + 1] = sc.shi[l] + std::max(sc.a[l], 0LL);
    if (sc.shi[l + 1] - sc.slo[l + 1] + 1 > kSumCap) return BDD_ETOOBIG;
  }
  for (int l = 0; l < k; ++l) {
    std::vector<int> &ids = sc.id_of_key[l];
    ids.assign(sc.thi[l] - sc.tlo[l] + 2, -1);
    sc.rep[l].clear();
    for (long long s = sc.slo[l]; s <= sc.shi[l]; ++s) {
      const int key = key_of_range(sc.tlo[l], sc.thi[l], s, b, sense);
      if (key == 0 || ids[key] >= 0) continue;
      ids[key] = (int)sc.rep[l].size();
      sc.rep[l].push_back(s);
    }
    if (sc.rep[l].empty()) return BDD_EINFEASIBLE;
    if ((long long)sc.rep[l].size() > max_width) return BDD_ETOOBIG;
  }
  out.bdd_row.push_back(j);
  out.bdd_depth.push_back(k);
  for (int l = 0; l < k; ++l) {
    out.occ_var.push_back(sc.cols[l]);
    out.occ_csr.push_back(sc.pos[l]);
    out.occ_width.push_back((int)sc.rep[l].size());
    for (long long s : sc.rep[l]) {
      int lo, hi;
      if (l == k - 1) {
        lo = sat(s, sense, b) ? kTop : kBot;
        hi = sat(s + sc.a[l], sense, b) ? kTop : kBot;
      } else {
        const int k0 = key_of_range(sc.tlo[l + 1], sc.thi[l + 1], s, b, sense);
        const int k1 = key_of_range(sc.tlo[l + 1], sc.thi[l + 1], s + sc.a[l], b, sense);
        lo = k0 ? sc.id_of_key[l + 1][k0] : kBot;
        hi = k1 ? sc.id_of_key[l + 1][k1] : kBot;
      }
      out.lo.push_back(lo);
      out.hi.push_back(hi);
    }
  }
  return BDD_OK;
}

int compile_row(int j, const long long *row_ptr, const int *col, const int *val, const int *rank, int n,
                long long b, int sense, int max_width, Scratch &sc, Chunk &out) {
  long long s0 = row_ptr[j], e0 = row_ptr[j + 1];
  if (e0 < s0 || sense < -1 || sense > 1) return BDD_EINVAL;
  sc.order.clear();
  for (long long t = s0; t < e0; ++t) {
    if (col[t] < 0 || col[t] >= n) return BDD_EINVAL;
    if (val[t] != 0) sc.order.push_back((int)(t - s0));
  }
  // layer order: ascending place in the variable order (Appendix A.3), index order without one
  if (rank)
    std::sort(sc.order.begin(), sc.order.end(),
              [&](int x, int y) { return rank[col[s0 + x]] < rank[col[s0 + y]]; });
  else
    std::sort(sc.order.begin(), sc.order.end(),
              [&](int x, int y) { return col[s0 + x] < col[s0 + y]; });
  const int k = (int)sc.order.size();
  sc.a.resize(k);
  sc.pos.resize(k);
  sc.cols.resize(k);
  for (int l = 0; l < k; ++l) {
    long long t = s0 + sc.order[l];
    sc.a[l] = val[t];
    sc.pos[l] = t;
    sc.cols[l] = col[t];
    if (l > 0 && sc.cols[l] == sc.cols[l - 1]) return BDD_EINVAL;  // duplicate (j, i)
  }
  if (k == 0) return sat(0, sense, b) ? BDD_OK : BDD_EINFEASIBLE;
  if ((int)sc.T.size() < k + 1) {
    sc.T.resize(k + 1);
    sc.S.resize(k + 1);
    sc.rep.resize(k + 1);
    sc.id_of_key.resize(k + 1);
  }
  bool unit = true;
  for (int l = 0; l < k && unit; ++l) unit = sc.a[l] == 1 || sc.a[l] == -1;
  if (unit) return compile_unit_row(j, b, sense, max_width, k, sc, out);
  // suffix sums T_l (l = k .. 0)
  sc.T[k].assign(1, 0);
  for (int l = k - 1; l >= 0; --l) {
    merge_shift(sc.T[l + 1], sc.a[l], sc.T[l]);
    if ((long long)sc.T[l].size() > kSumCap) return BDD_ETOOBIG;
  }
  // reachable prefix sums S_l (l = 0 .. k-1)
  sc.S[0].assign(1, 0);
  for (int l = 0; l + 1 < k; ++l) {
    merge_shift(sc.S[l], sc.a[l], sc.S[l + 1]);
    if ((long long)sc.S[l + 1].size() > kSumCap) return BDD_ETOOBIG;
  }
  // nodes: distinct nonzero keys, numbered in ascending order of their smallest sum
  for (int l = 0; l < k; ++l) {
    std::vector<int> &ids = sc.id_of_key[l];
    ids.assign(sc.T[l].size() + 1, -1);
    sc.rep[l].clear();
    for (long long s : sc.S[l]) {
      int key = key_of(sc.T[l], s, b, sense);
      if (key == 0 || ids[key] >= 0) continue;
      ids[key] = (int)sc.rep[l].size();
      sc.rep[l].push_back(s);
    }
    if (sc.rep[l].empty()) return BDD_EINFEASIBLE;  // no feasible completion of the root
    if ((long long)sc.rep[l].size() > max_width) return BDD_ETOOBIG;
  }
  // emit arcs
  out.bdd_row.push_back(j);
  out.bdd_depth.push_back(k);
  for (int l = 0; l < k; ++l) {
    out.occ_var.push_back(sc.cols[l]);
    out.occ_csr.push_back(sc.pos[l]);
    out.occ_width.push_back((int)sc.rep[l].size());
    for (long long s : sc.rep[l]) {
      int lo, hi;
      if (l == k - 1) {
        lo = sat(s, sense, b) ? kTop : kBot;
        hi = sat(s + sc.a[l], sense, b) ? kTop : kBot;
      } else {
        int k0 = key_of(sc.T[l + 1], s, b, sense);
        int k1 = key_of(sc.T[l + 1], s + sc.a[l], b, sense);
        lo = k0 ? sc.id_of_key[l + 1][k0] : kBot;
        hi = k1 ? sc.id_of_key[l + 1][k1] : kBot;
      }
      out.lo.push_back(lo);
      out.hi.push_back(hi);
    }
  }
  return BDD_OK;
}

}  // namespace

namespace {

// Host worker threads of parallel_for.  A job is published by bumping an atomic generation;
// workers spin on it for a short while after each job (the calls of one build come in quick
// succession), then sleep on a condition variable.  Each takes chunks of the job from a shared
// atomic cursor and checks out when none are left; the caller works too and returns once every
// worker has checked out, so a job's fields never change under a worker.  The pool lives until
// the process exits and is never destroyed (its idle threads end with the process).  A child
// forked after the pool was made has none of its threads, so there every job runs inline.
class HostPool {
 public:
  static HostPool &get() {
    static HostPool *pool = new HostPool();
    return *pool;
  }
  bool run(long long n, long long grain, const std::function<void(long long, long long)> &body) {
    if (getpid() != owner_) return false;  // a forked child: the workers exist only in the parent
    std::unique_lock<std::mutex> busy(job_mu_, std::try_to_lock);
    if (!busy.owns_lock() || workers_.empty()) return false;
    body_ = &body;
    n_ = n;
    grain_ = grain;
    next_.store(0, std::memory_order_relaxed);
    active_.store((int)workers_.size(), std::memory_order_relaxed);
    {
      std::lock_guard<std::mutex> lk(mu_);  // a worker about to sleep sees the new generation
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    work();
    while (active_.load(std::memory_order_acquire) != 0) std::this_thread::yield();
    body_ = nullptr;
    return true;
  }

 private:
  HostPool() {
    const unsigned hw = std::thread::hardware_concurrency();
    const int extra = (int)std::min(hw ? hw : 1u, 64u) - 1;
    for (int t = 0; t < extra; ++t) workers_.emplace_back([this] { loop(); });
  }
  void work() {
    for (;;) {
      const long long b = next_.fetch_add(grain_, std::memory_order_relaxed);
      if (b >= n_) break;
      (*body_)(b, std::min(n_, b + grain_));
    }
  }
  void loop() {
    unsigned long long seen = 0;
    for (;;) {
      const auto t0 = std::chrono::steady_clock::now();
      unsigned spins = 0;
      while (gen_.load(std::memory_order_acquire) == seen) {
        if ((++spins & 255) == 0 && std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(500)) {
          std::unique_lock<std::mutex> lk(mu_);
          cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
        }
      }
      seen = gen_.load(std::memory_order_acquire);
      work();
      active_.fetch_sub(1, std::memory_order_release);
    }
  }
  const pid_t owner_ = getpid();
  std::vector<std::thread> workers_;
  std::mutex job_mu_, mu_;
  std::condition_variable cv_;
  const std::function<void(long long, long long)> *body_ = nullptr;
  long long n_ = 0, grain_ = 1;
  std::atomic<long long> next_{0};
  std::atomic<int> active_{0};
  std::atomic<unsigned long long> gen_{0};
};

}  // namespace

void parallel_for(long long n, long long grain, const std::function<void(long long, long long)> &body) {
  if (n <= 0) return;
  grain = std::max(1LL, grain);
  if (n <= grain || !HostPool::get().run(n, grain, body)) body(0, n);
}

namespace {

template <class V, class Tp>
void copy_into(V &out, size_t off, const std::vector<Tp> &v) {
  if (!v.empty()) std::memcpy(out.data() + off, v.data(), v.size() * sizeof(Tp));
}

// out[0] = 0, out[k + 1] = out[k] + in[k] for k < n (out has n + 1 entries), in three passes:
// the sums of fixed blocks in parallel, their prefix, then every block's prefix in parallel
// (the same result as the serial loop); returns the largest in[k] through *max_in.
template <class In>
void parallel_prefix(const In *in, long long n, long long *out, In *max_in) {
  constexpr long long kBlock = 1 << 16;
  const long long nblk = (n + kBlock - 1) / kBlock;
  std::vector<long long> sum(nblk + 1, 0);
  std::vector<In> mx(nblk, In(0));
  parallel_for(nblk, 1, [&](long long b0, long long b1) {
    for (long long b = b0; b < b1; ++b) {
      long long acc = 0;
      In m = In(0);
      for (long long k = b * kBlock; k < std::min(n, (b + 1) * kBlock); ++k) {
        acc += in[k];
        m = std::max(m, in[k]);
      }
      sum[b + 1] = acc;
      mx[b] = m;
    }
  });
  for (long long b = 0; b < nblk; ++b) sum[b + 1] += sum[b];
  out[0] = 0;
  parallel_for(nblk, 1, [&](long long b0, long long b1) {
    for (long long b = b0; b < b1; ++b) {
      long long acc = sum[b];
      for (long long k = b * kBlock; k < std::min(n, (b + 1) * kBlock); ++k) {
        acc += in[k];
        out[k + 1] = acc;
      }
    }
  });
  In m = In(0);
  for (long long b = 0; b < nblk; ++b) m = std::max(m, mx[b]);
  if (max_in) *max_in = m;
}

}  // namespace

int compile_bdds(int n, int m, const long long *row_ptr, const int *col, const int *val,
                 const int *b, const signed char *sense, const int *rank, int max_width,
                 long long max_nodes, HostBDDs *H, int *failed_row) {
  *failed_row = -1;
  const int rows_per_chunk = 512;
  const int nchunks = (m + rows_per_chunk - 1) / rows_per_chunk;
  std::vector<Chunk> chunks(nchunks);
  parallel_for(nchunks, 1, [&](long long c0, long long c1) {
    Scratch sc;
    for (long long cidx = c0; cidx < c1; ++cidx) {
      Chunk &ch = chunks[cidx];
      const int r0 = (int)cidx * rows_per_chunk, r1 = std::min(m, r0 + rows_per_chunk);
      for (int j = r0; j < r1; ++j) {
        const int rc = compile_row(j, row_ptr, col, val, rank, n, b[j], sense[j], max_width, sc, ch);
        if (rc != BDD_OK) {
          ch.status = rc;
          ch.failed_row = j;
          break;
        }
      }
    }
  });
  for (auto &ch : chunks)
    if (ch.status != BDD_OK) {
      *failed_row = ch.failed_row;
      return ch.status;
    }
  // concatenate in row order (each chunk's part copied in parallel)
  size_t nb = 0, O = 0, N = 0;
  std::vector<size_t> off_b(nchunks), off_o(nchunks), off_n(nchunks);
  for (int c = 0; c < nchunks; ++c) {
    off_b[c] = nb;
    off_o[c] = O;
    off_n[c] = N;
    nb += chunks[c].bdd_row.size();
    O += chunks[c].occ_var.size();
    N += chunks[c].lo.size();
  }
  if ((long long)N > max_nodes || N >= (size_t)INT_MAX || O >= (size_t)INT_MAX) return BDD_ETOOBIG;
  H->n = n;
  H->m = m;
  H->nnz = m ? row_ptr[m] : 0;
  H->bdd_row.resize(nb);
  H->bdd_depth.resize(nb);
  H->occ_var.resize(O);
  H->occ_csr.resize(O);
  H->occ_width.resize(O);
  H->lo.resize(N);
  H->hi.resize(N);
  parallel_for(nchunks, 1, [&](long long c0, long long c1) {
    for (long long c = c0; c < c1; ++c) {
      const Chunk &ch = chunks[c];
      copy_into(H->bdd_row, off_b[c], ch.bdd_row);
      copy_into(H->bdd_depth, off_b[c], ch.bdd_depth);
      copy_into(H->occ_var, off_o[c], ch.occ_var);
      copy_into(H->occ_csr, off_o[c], ch.occ_csr);
      copy_into(H->occ_width, off_o[c], ch.occ_width);
      copy_into(H->lo, off_n[c], ch.lo);
      copy_into(H->hi, off_n[c], ch.hi);
    }
  });
  chunks.clear();
  H->bdd_occ0.resize(nb + 1);
  H->occ_node0.resize(O + 1);
  parallel_prefix(H->bdd_depth.data(), (long long)nb, H->bdd_occ0.data(), &H->max_depth);
  parallel_prefix(H->occ_width.data(), (long long)O, H->occ_node0.data(), &H->max_width);
  return BDD_OK;
}

int build_layout(const HostBDDs &H, Layout *L, bool lanes2, const int *class_of_key, const int *var_deg) {
  const long long nb = H.nb(), O = H.O(), N = H.N();
  L->lanes2 = lanes2;
  // class of each BDD: its key's entry in the table, else the default for its widest layer
  std::vector<int> cls(nb);
  std::atomic<int> bad{BDD_OK};
  parallel_for(nb, 4096, [&](long long b0, long long b1) {
    for (long long b = b0; b < b1; ++b) {
      int w = 0;
      for (long long o = H.bdd_occ0[b]; o < H.bdd_occ0[b + 1]; ++o) w = std::max(w, H.occ_width[o]);
      int c = natural_class(w);
      if (c == kWarpClasses && w > kMaxBlockTileWidth) bad.store(BDD_ETOOBIG);
      if (lanes2 && w <= 2) c = 0;  // lane tiles: one lane holds both nodes of a layer
      const int want = class_of_key ? class_of_key[layout_key(w, H.bdd_depth[b])] : -1;
      if (want >= 0) {
        const bool fits = want == kWarpClasses ? w <= kMaxBlockTileWidth
                                               : want < kWarpClasses && ((1 << want) >= w || (want == 0 && lanes2 && w <= 2));
        if (!fits) bad.store(BDD_EINVAL);
        c = want;
      }
      cls[b] = c;
    }
  });
  if (bad.load() != BDD_OK) return bad.load();
  // stable counting sort by (class, depth descending); ties keep ascending row order
  const int D = H.max_depth;
  const int nkeys = (kWarpClasses + 1) * (D + 1);
  std::vector<long long> cnt(nkeys + 1, 0);
  auto key = [&](long long b) { return cls[b] * (D + 1) + (D - H.bdd_depth[b]); };
  for (long long b = 0; b < nb; ++b) cnt[key(b) + 1]++;
  for (int t = 0; t < nkeys; ++t) cnt[t + 1] += cnt[t];
  L->bdd_perm.resize(nb);
  for (long long b = 0; b < nb; ++b) L->bdd_perm[cnt[key(b)]++] = (int)b;
  L->n_sorted = (int)nb;
  L->bdd_depth.resize(nb);
  parallel_for(nb, 1 << 14, [&](long long s0, long long s1) {
    for (long long t = s0; t < s1; ++t) L->bdd_depth[t] = H.bdd_depth[L->bdd_perm[t]];
  });
  // tiles
  L->tile_occ0.clear();
  L->tile_bdd0.clear();
  L->tile_nbdd.clear();
  long long s = 0;
  for (int c = 0; c <= kWarpClasses; ++c) {
    L->class_tile_off[c] = (int)L->tile_bdd0.size();
    const int G = c < kWarpClasses ? (32 >> c) : 1;
    while (s < nb && cls[L->bdd_perm[s]] == c) {
      long long e = s;
      while (e < nb && e - s < G && cls[L->bdd_perm[e]] == c) ++e;
      L->tile_bdd0.push_back((int)s);
      L->tile_nbdd.push_back((int)(e - s));
      s = e;
    }
  }
  L->class_tile_off[kWarpClasses + 1] = (int)L->tile_bdd0.size();
  L->n_warp_tiles = L->class_tile_off[kWarpClasses];
  L->n_block_tiles = L->class_tile_off[kWarpClasses + 1] - L->class_tile_off[kWarpClasses];
  // occurrences and nodes in tile order: per-tile counts and their prefix sums, then every tile
  // filled on its own (a tile's slab is one contiguous range)
  const long long ntiles = (long long)L->tile_bdd0.size();
  L->tile_occ0.resize(ntiles);
  // (every entry of these is written below, each tile's by one parallel task)
  L->occ_of_canon.resize(O);
  L->occ_node_off.resize(O + 1);
  L->occ_var.resize(O);
  L->occ_csr.resize(O);
  hvec<long long> node_of_canon_occ(O);  // device first node of each canonical occurrence
  std::vector<long long> tile_node0(ntiles + 1, 0);
  {
    long long o = 0, v = 0;
    for (long long t = 0; t < ntiles; ++t) {
      L->tile_occ0[t] = (int)o;
      tile_node0[t] = v;
      const int b0 = L->tile_bdd0[t], nt = L->tile_nbdd[t];
      for (int q = 0; q < nt; ++q) {
        const int cb = L->bdd_perm[b0 + q];
        o += H.bdd_depth[cb];
        v += H.occ_node0[H.bdd_occ0[cb + 1]] - H.occ_node0[H.bdd_occ0[cb]];
      }
    }
    tile_node0[ntiles] = v;
    if (o != O || v != N) return BDD_EINVAL;
  }
  // lane codes (see LaneStage): both nodes' arcs of a lane-tile layer in one byte, 0 elsewhere
  L->lane_code.resize(O + kLaneCodePad);
  const long long n_lane_tiles = lanes2 ? L->class_tile_off[1] : 0;
  auto lane_arc = [](int x) -> unsigned { return x >= 0 ? (unsigned)x : x == kTop ? kLaneTop : kLaneBot; };
  parallel_for(ntiles, 64, [&](long long t0, long long t1) {
    for (long long t = t0; t < t1; ++t) {
      long long dev_o = L->tile_occ0[t], dev_node = tile_node0[t];
      const int b0 = L->tile_bdd0[t], nt = L->tile_nbdd[t];
      const int dmax = L->bdd_depth[b0];  // first BDD of a tile is the deepest
      const bool lane_tile = t < n_lane_tiles;
      for (int l = 0; l < dmax; ++l) {
        for (int q = 0; q < nt; ++q) {
          const int cb = L->bdd_perm[b0 + q];
          if (H.bdd_depth[cb] <= l) break;  // depths are non-increasing inside the tile
          const long long co = H.bdd_occ0[cb] + l;
          L->occ_of_canon[co] = (int)dev_o;
          L->occ_node_off[dev_o] = (int)dev_node;
          L->occ_var[dev_o] = H.occ_var[co];
          L->occ_csr[dev_o] = H.occ_csr[co];
          unsigned code = 0;
          if (lane_tile) {  // widths <= 2, so a non-terminal successor is node 0 or 1
            const long long cn = H.occ_node0[co];
            code = lane_arc(H.lo[cn]) | lane_arc(H.hi[cn]) << 2;
            if (H.occ_width[co] == 2) {
              const unsigned c1 = lane_arc(H.lo[cn + 1]) | lane_arc(H.hi[cn + 1]) << 2;
              if (c1 == (kLaneNoNode1 >> 4)) bad.store(BDD_EINVAL);  // a node without a path to top
              code |= c1 << 4;
            } else {
              code |= kLaneNoNode1;
            }
          }
          L->lane_code[dev_o] = (unsigned char)code;
          node_of_canon_occ[co] = dev_node;
          dev_node += H.occ_width[co];
          ++dev_o;
        }
      }
    }
  });
  if (bad.load() != BDD_OK) return bad.load();
  for (int k = 0; k < kLaneCodePad; ++k) L->lane_code[O + k] = 0;
  L->occ_node_off[O] = (int)N;
  L->max_block_width = 0;  // widest layer of a block tile
  for (long long t = L->class_tile_off[kWarpClasses]; t < ntiles; ++t) {
    const int cb = L->bdd_perm[L->tile_bdd0[t]];
    for (long long co = H.bdd_occ0[cb]; co < H.bdd_occ0[cb + 1]; ++co)
      L->max_block_width = std::max(L->max_block_width, H.occ_width[co]);
  }
  // successors as global device node ids
  L->lohi.resize(2 * N);  // every node's pair is written below
  parallel_for(nb, 256, [&](long long b0, long long b1) {
    for (long long b = b0; b < b1; ++b) {
      for (long long co = H.bdd_occ0[b]; co < H.bdd_occ0[b + 1]; ++co) {
        const bool last = co + 1 == H.bdd_occ0[b + 1];
        const long long next0 = last ? 0 : node_of_canon_occ[co + 1];
        const long long d0 = node_of_canon_occ[co];
        for (int q = 0; q < H.occ_width[co]; ++q) {
          const long long cn = H.occ_node0[co] + q;
          const int lo = H.lo[cn], hi = H.hi[cn];
          L->lohi[2 * (d0 + q)] = lo >= 0 ? (int)(next0 + lo) : lo;
          L->lohi[2 * (d0 + q) + 1] = hi >= 0 ? (int)(next0 + hi) : hi;
        }
      }
    }
  });
  // window table of every warp tile: node offsets at layer w * kWinLayers and at layer
  // min((w + 1) * kWinLayers + 1, maxd), w = 0 .. ceil(maxd / kWinLayers); entry counts first,
  // then every tile's entries filled on their own
  L->tile_win0.assign(ntiles + 1, 0);
  for (long long t = 0; t < ntiles; ++t) {
    const int dmax = L->bdd_depth[L->tile_bdd0[t]];
    const int entries = t < L->class_tile_off[kWarpClasses] ? (dmax + kWinLayers - 1) / kWinLayers + 1 : 0;
    L->tile_win0[t + 1] = L->tile_win0[t] + entries;
  }
  L->win_node.resize(2 * (size_t)L->tile_win0[ntiles]);
  parallel_for(L->class_tile_off[kWarpClasses], 256, [&](long long t0, long long t1) {
    for (long long t = t0; t < t1; ++t) {
      const int b0 = L->tile_bdd0[t], nt = L->tile_nbdd[t];
      const int dmax = L->bdd_depth[b0];
      auto node_at = [&](int layer) {  // first node of `layer` in the tile (tile end for dmax)
        long long before = 0;
        for (int q = 0; q < nt; ++q) before += std::min(L->bdd_depth[b0 + q], layer);
        return L->occ_node_off[L->tile_occ0[t] + before];
      };
      const int nwin = (dmax + kWinLayers - 1) / kWinLayers;
      int *out = L->win_node.data() + 2 * (size_t)L->tile_win0[t];
      for (int w = 0; w <= nwin; ++w) {
        out[2 * w] = node_at(std::min(w * kWinLayers, dmax));
        out[2 * w + 1] = node_at(std::min(w * kWinLayers + kWinLayers + 1, dmax));
      }
    }
  });
  // variable -> occurrences (ascending row, i.e. canonical occurrence order): degrees (the
  // caller's, else atomic counts), slots claimed in any order, then each variable's slots sorted
  // by canonical occurrence; SRMP sets (Appendix A.4): in J_i^> unless the last layer, in J_i^<
  // unless the first
  const int n = H.n;
  std::vector<int> vcnt(n + 1, 0);
  if (!var_deg) {
    parallel_for(O, 1 << 16, [&](long long a, long long e) {
      for (long long co = a; co < e; ++co) __atomic_fetch_add(&vcnt[H.occ_var[co]], 1, __ATOMIC_RELAXED);
    });
    var_deg = vcnt.data();
  }
  std::vector<long long> ptr(n + 1);
  parallel_prefix(var_deg, (long long)n, ptr.data(), (int *)nullptr);
  L->var_ptr.resize(n + 1);
  parallel_for(n + 1, 1 << 16, [&](long long a, long long e) {
    for (long long i = a; i < e; ++i) {
      L->var_ptr[i] = (int)ptr[i];
      if (i < n) vcnt[i] = 0;
    }
  });
  hvec<unsigned char> dir_canon(O);
  parallel_for(nb, 4096, [&](long long b0, long long b1) {
    for (long long b = b0; b < b1; ++b)
      for (long long co = H.bdd_occ0[b]; co < H.bdd_occ0[b + 1]; ++co)
        dir_canon[co] = (unsigned char)((co + 1 < H.bdd_occ0[b + 1] ? kDirForward : 0) |
                                        (co > H.bdd_occ0[b] ? kDirBackward : 0));
  });
  hvec<int> slot_canon(O);
  parallel_for(O, 1 << 16, [&](long long a, long long e) {
    for (long long co = a; co < e; ++co) {
      const int i = H.occ_var[co];
      slot_canon[L->var_ptr[i] + __atomic_fetch_add(&vcnt[i], 1, __ATOMIC_RELAXED)] = (int)co;
    }
  });
  L->var_occ.resize(O);
  L->occ_slot.resize(O);
  L->slot_dir.resize(O);
  parallel_for(n, 1 << 14, [&](long long a, long long e) {
    for (long long i = a; i < e; ++i) {
      int *s0 = slot_canon.data() + L->var_ptr[i], *s1 = slot_canon.data() + L->var_ptr[i + 1];
      if (s1 - s0 <= 32) {  // insertion sort of a short list
        for (int *x = s0 + 1; x < s1; ++x)
          for (int *y = x; y > s0 && y[-1] > y[0]; --y) std::swap(y[-1], y[0]);
      } else {
        std::sort(s0, s1);
      }
      for (int k = L->var_ptr[i]; k < L->var_ptr[i + 1]; ++k) {
        const int co = slot_canon[k], o = L->occ_of_canon[co];
        L->var_occ[k] = o;
        L->occ_slot[o] = k;
        L->slot_dir[k] = dir_canon[co];
      }
    }
  });
  return BDD_OK;
}

std::vector<int> balanced_cuts(const HostBDDs &H, const int *rank, int k) {
  std::vector<int> cuts;
  const int n = H.n;
  const long long N = H.N();
  if (k < 2 || n < 2 || N == 0) return cuts;
  std::vector<long long> at(n, 0);  // nodes of the layers of the variable at each place
  for (long long o = 0; o < H.O(); ++o) {
    const int i = H.occ_var[o];
    at[rank ? rank[i] : i] += H.occ_width[o];
  }
  long long acc = 0;  // nodes at places before p
  int t = 1;          // next interval boundary to place, at about t * N / k nodes
  for (int p = 1; p < n && t < k; ++p) {
    acc += at[p - 1];
    if (acc * k >= (long long)t * N) {
      cuts.push_back(p);
      while (t < k && acc * k >= (long long)t * N) ++t;
    }
  }
  return cuts;
}

int split_bdds(HostBDDs &H, const int *rank, const std::vector<int> &cuts, int depth, CopyPairs *P) {
  const int n = H.n;
  if (depth < 0 || (depth > 0 && !cuts.empty())) return BDD_EINVAL;
  for (size_t t = 0; t < cuts.size(); ++t)
    if (cuts[t] < 1 || cuts[t] >= n || (t > 0 && cuts[t] <= cuts[t - 1])) return BDD_EINVAL;
  P->cuts = cuts;
  P->cut_ptr.assign(1, 0);
  P->tail_occ.clear();
  P->tail.clear();
  P->side.clear();
  P->head.clear();
  if (cuts.empty() && depth == 0) return BDD_OK;
  // interval of every variable: the number of cuts at or before its place
  std::vector<int> interval(depth > 0 ? 0 : n);
  for (int i = 0; i < (int)interval.size(); ++i) {
    const int place = rank ? rank[i] : i;
    interval[i] = (int)(std::upper_bound(cuts.begin(), cuts.end(), place) - cuts.begin());
  }
  std::vector<char> cut_at;  // depth split: cut before layer l of the current BDD
  hvec<int> row, pdepth;
  hvec<long long> occ0;
  const long long nb = H.nb();
  for (long long b = 0; b < nb; ++b) {
    const long long o0 = H.bdd_occ0[b];
    const int k = H.bdd_depth[b];
    if (depth > 0) {
      const int q = (k + depth - 1) / depth;
      cut_at.assign(k + 1, 0);
      for (int t = 1; t < q; ++t) cut_at[(long long)t * k / q] = 1;
    }
    int start = 0;
    for (int l = 1; l <= k; ++l) {
      if (l < k && !(depth > 0 ? cut_at[l] != 0 : interval[H.occ_var[o0 + l]] != interval[H.occ_var[o0 + l - 1]]))
        continue;
      row.push_back(H.bdd_row[b]);
      pdepth.push_back(l - start);
      occ0.push_back(o0 + start);
      if (l < k) {  // cut between layers l - 1 and l: every arc between them becomes a pair
        const long long ot = o0 + l - 1;
        P->tail_occ.push_back(ot);
        for (int u = 0; u < H.occ_width[ot]; ++u)
          for (int side = 0; side < 2; ++side) {
            int &t = side ? H.hi[H.occ_node0[ot] + u] : H.lo[H.occ_node0[ot] + u];
            if (t < 0) continue;  // an arc into bot stays one (Def. of sub-BDDs)
            const long long pk = P->npairs();
            if (pk > (long long)INT_MAX + kCopy0) return BDD_ETOOBIG;
            P->tail.push_back(u);
            P->side.push_back(side);
            P->head.push_back(t);
            t = kCopy0 - (int)pk;
          }
        P->cut_ptr.push_back(P->npairs());
      }
      start = l;
    }
  }
  occ0.push_back(H.O());
  H.bdd_row = std::move(row);
  H.bdd_depth = std::move(pdepth);
  H.bdd_occ0 = std::move(occ0);
  H.max_depth = 0;
  for (int d : H.bdd_depth) H.max_depth = std::max(H.max_depth, d);
  return BDD_OK;
}

}  // namespace bdd
