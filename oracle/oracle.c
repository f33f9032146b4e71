/*
 * Oracle for BDD-based min-marginal averaging on 0-1 ILPs (Lange & Swoboda, "Efficient
 * Message Passing for 0-1 ILPs with Binary Decision Diagrams").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded FP64 C.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg load this file's library.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's notation:
 *   - BP / ILP form (Sec. 3, Def. 1 and Ex. 1): one subproblem per constraint row j, index
 *     set I_j = { i : a_ji != 0 }, feasible set X_j = { x : a_j x (<=,=,>=) b_j }.
 *   - One reduced, ordered, non-skipping BDD per row (Sec. 5.1, Def. 4 and the remark after
 *     Prop. 2), built by reducing reachable partial coefficient sums bottom-up: the node of a
 *     partial sum s at layer l is the pair (node of s, node of s + a_l) at layer l+1; equal
 *     pairs are one node, the pair (bot, bot) is bot.  Nodes of a layer are numbered by their
 *     smallest partial sum (canonical order; the paper leaves node order open).
 *   - Arc costs theta (Sec. 5.3): 1-arc of a layer-i node costs lambda^j_i, 0-arc costs 0.
 *   - Forward / backward update steps (Alg. 2, Alg. 3) with m_fwd(root) = 0,
 *     m_bwd(top) = 0, m_bwd(bot) = +inf; arc marginals and min-marginals (eqs. arc-marginal
 *     and marginal-aggregation).
 *   - Schedule S: Alg. 1 (min-marginal averaging, forward then backward over the variables,
 *     lambda initialised to c_i/|J_i|), with min-marginals taken from a full dynamic
 *     programme over the BDD at every visit, and the Prop. 1 gain checked per update.
 *   - Schedule P: the parallel-across-BDDs form with deferred averaging: within a sweep every
 *     BDD runs its layers in order using the incremental steps of Sec. 5.4 (forward: update
 *     step then aggregate; backward: aggregate then update step); the averaging share
 *     P_i/|J_i| of the previous sweep is added to lambda when its layer is visited, lambda
 *     moves by -omega*(m1 - m0), and the pending sum P_i = sum omega*(m1 - m0) is formed
 *     after the sweep.
 *   - Lower bound: sum_j E^j(lambda^j) + sum_i min(0, c_i - sum_j lambda^j_i) (the y-slack
 *     form of the dual derivation, Appendix A.1), which equals eq. (D)'s objective when
 *     sum_j lambda^j_i = c_i.
 *   - Solution counts (Appendix C.1, Table 3, counting column).
 *   - Smoothing (Appendix A.5; Appendix C.1, Table 3, log-sum-exp column): with alpha > 0 every
 *     minimum above (forward and backward steps, min-marginal aggregation, the y-slack term)
 *     becomes the soft minimum -alpha log(sum exp(-x / alpha)), evaluated in the -alpha log
 *     domain with the smaller argument factored out; E^j becomes E^j_alpha and min-marginals
 *     become marginal log-sum-exp values.  alpha = 0 is the plain min-sum algebra.
 *   - Variable order (Appendix A.3): an optional rank per variable sets the layer order of every
 *     BDD and the visiting order of Alg. 1 (identity when absent).
 *   - SRMP averaging (Appendix A.4): optionally, the averaging share of variable i goes only to
 *     the subproblems that contain a variable after i in the order (forward pass) / before i
 *     (backward pass), evenly; when there are none, to all of J_i.
 *   - Sub-BDDs and copy arcs (Sec. 6, Def. of sub-BDDs and copy-arcs, the parallel averaging
 *     algorithm and Prop. 4): optionally the variable order is cut into intervals; every BDD is
 *     split where its variables cross an interval boundary.  The earlier piece keeps the arcs
 *     crossing the cut as copy arcs into the top terminal with cost theta + mu_bar; the later
 *     piece starts at its first layer with several roots, each with initial forward message
 *     min over its entry arcs of mu (the entry arcs carry no theta).  After every forward sweep
 *     mu_bar moves by -gamma * delta_fwd + gamma * delta_bwd (delta_fwd: arc-marginal of the copy
 *     arc minus its minimum over the cut), after every backward sweep mu moves by
 *     -gamma * delta_bwd + gamma * delta_fwd (delta_bwd: the same on the entry arcs).  Each
 *     piece is a subproblem of the decomposition (its layers are its occurrences).  A depth
 *     split (a reading for deep BDDs) cuts every BDD into pieces of at most D layers instead,
 *     with the same copy arcs and steps.
 * Threads: the tests, the package smoke check and the oracle the benchmark times as the CPU
 * baseline use the single-threaded build.  Built with -fopenmp (the benchmark's second CPU
 * baseline, all host cores), the loops of schedule P over BDDs and over variables run in
 * parallel; each BDD and each variable is still computed by the same operations in the same
 * order, so that build's results equal the single-threaded build's bit for bit.
 * Readings where the paper is silent: a min-marginal that is +inf (a row that forces x_i)
 * gives the difference 0; a variable in no row contributes min(0, c_i) to the bound; an empty
 * row is dropped when 0 (sense) b holds and is infeasible otherwise.
 */
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TOP (-1)
#define ORC_BOT (-2)
/* arc target codes below ORC_COPY0: copy arc k into the top terminal, cost mu_bar[k] */
#define ORC_COPY0 (-4)

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_EINFEASIBLE = -2, ORC_ETOOBIG = -3, ORC_ENOMEM = -4 };

/* ------------------------------------------------------------------------------------ */
/* growable arrays                                                                        */
/* ------------------------------------------------------------------------------------ */
typedef struct { int *p; long long n, cap; } ivec;
typedef struct { long long *p; long long n, cap; } lvec;

static int iv_push(ivec *v, int x) {
  if (v->n == v->cap) {
    long long nc = v->cap ? 2 * v->cap : 256;
    int *q = (int *)realloc(v->p, (size_t)nc * sizeof(int));
    if (!q) return -1;
    v->p = q; v->cap = nc;
  }
  v->p[v->n++] = x;
  return 0;
}
static int lv_push(lvec *v, long long x) {
  if (v->n == v->cap) {
    long long nc = v->cap ? 2 * v->cap : 256;
    long long *q = (long long *)realloc(v->p, (size_t)nc * sizeof(long long));
    if (!q) return -1;
    v->p = q; v->cap = nc;
  }
  v->p[v->n++] = x;
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* oracle state                                                                           */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  int n, m, nb;
  long long nnz, O, N;
  int max_depth, max_width;
  /* per BDD (in ascending row order) */
  int *bdd_row, *bdd_k;
  long long *bdd_occ0;      /* [nb+1] first occurrence; occurrence o = bdd_occ0[b] + layer */
  /* per occurrence (BDD-major, layer-minor) */
  int *occ_var, *occ_bdd, *occ_layer;
  long long *occ_csr;       /* position of the coefficient in the input CSR arrays */
  long long *occ_node0;     /* [O+1] first node of the layer; nodes are BDD-major, layer-major */
  /* per node */
  int *lo, *hi;             /* local id in the next layer of the same BDD, or TOP / BOT */
  long long *minsum;        /* smallest partial sum of the node's class */
  /* per variable */
  long long *var_ptr, *var_occ; /* occurrences of each variable in ascending row order */
  int *deg;
  double *c;
  double empty_const;       /* sum over variables in no row of min(0, c_i) (soft: of agg(0, c_i)) */
  double alpha;             /* 0: min-sum; > 0: smoothing temperature */
  int srmp;                 /* 0: eq. mma-update averaging; 1: SRMP averaging */
  int *order;               /* [n] variables in visiting order (Alg. 1) */
  double *oshare;           /* [O] share each occurrence takes in the next sweep */
  /* dual state and messages */
  double *lam, *P, *delta, *share, *fm, *bm;
  /* scratch for the definitional dynamic programmes */
  double *sfm, *sbm;
  /* sub-BDDs (Sec. 6): copy-arc pairs grouped by cut, root messages of later pieces */
  long long npairs;
  int ncuts;
  long long *cut_ptr;       /* [ncuts+1] pairs of each cut */
  long long *pair_u, *pair_w; /* global node of the copy arc's tail (earlier piece), of the
                                 entry arc's head (later piece's first layer) */
  long long *pair_occ;      /* occurrence of the tail's layer */
  int *pair_hi;             /* 1: the original arc is the 1-arc (theta = lambda) */
  double *mu_bar, *mu, *dfwd, *dbwd;  /* [npairs] */
  double *root_f;           /* [N] initial forward message of first-layer nodes of each piece */
  double gamma;
  /* worst check violations seen: [monotone drop, invariant, incremental mm, prop-1 gain,
   * negative gain] */
  double worst[5];
} oracle_t;

void orc_free(void *vh) {
  oracle_t *h = (oracle_t *)vh;
  if (!h) return;
  free(h->bdd_row); free(h->bdd_k); free(h->bdd_occ0);
  free(h->occ_var); free(h->occ_bdd); free(h->occ_layer); free(h->occ_csr); free(h->occ_node0);
  free(h->lo); free(h->hi); free(h->minsum);
  free(h->var_ptr); free(h->var_occ); free(h->deg); free(h->c);
  free(h->lam); free(h->P); free(h->delta); free(h->share); free(h->fm); free(h->bm);
  free(h->sfm); free(h->sbm); free(h->order); free(h->oshare);
  free(h->cut_ptr); free(h->pair_u); free(h->pair_w); free(h->pair_occ); free(h->pair_hi);
  free(h->mu_bar); free(h->mu); free(h->dfwd); free(h->dbwd); free(h->root_f);
  free(h);
}

/* ------------------------------------------------------------------------------------ */
/* BDD construction by reduction of reachable partial sums                                */
/* ------------------------------------------------------------------------------------ */
typedef struct { int col, val; long long pos; } entry_t;

static const int *g_rank;  /* comparator context (the oracle is single-threaded) */

static int cmp_entry(const void *a, const void *b) {
  const entry_t *x = (const entry_t *)a, *y = (const entry_t *)b;
  long long rx = g_rank ? g_rank[x->col] : x->col, ry = g_rank ? g_rank[y->col] : y->col;
  return (rx > ry) - (rx < ry);
}

static int sat(long long s, int sense, long long b) {
  if (sense < 0) return s <= b;
  if (sense > 0) return s >= b;
  return s == b;
}

/* index of s in the sorted array S[0..len) (s is known to be present) */
static long long find_sum(const long long *S, long long len, long long s) {
  long long lo = 0, hi = len - 1;
  while (lo < hi) {
    long long mid = (lo + hi) / 2;
    if (S[mid] < s) lo = mid + 1; else hi = mid;
  }
  return lo;
}

#define SUM_CAP (1LL << 24)

/* Builds the BDD of one row and appends its nodes / occurrences.  Returns ORC_OK,
 * ORC_EINFEASIBLE (no feasible point), ORC_ETOOBIG or ORC_ENOMEM. */
static int build_row(const entry_t *e, int k, long long b, int sense, int row,
                     ivec *bdd_row, ivec *bdd_k, ivec *occ_var, lvec *occ_csr, lvec *occ_node0,
                     ivec *lo, ivec *hi, lvec *minsum) {
  int rc = ORC_OK;
  long long **S = (long long **)calloc((size_t)k + 1, sizeof(long long *));
  long long *len = (long long *)calloc((size_t)k + 1, sizeof(long long));
  int **cls = (int **)calloc((size_t)k + 1, sizeof(int *));
  /* nodes of each layer, collected bottom-up, emitted top-down */
  ivec *Llo = (ivec *)calloc((size_t)k, sizeof(ivec));
  ivec *Lhi = (ivec *)calloc((size_t)k, sizeof(ivec));
  lvec *Lmin = (lvec *)calloc((size_t)k, sizeof(lvec));
  if (!S || !len || !cls || !Llo || !Lhi || !Lmin) { rc = ORC_ENOMEM; goto done; }

  /* top-down: reachable partial sums S_l (sorted, distinct) */
  S[0] = (long long *)malloc(sizeof(long long));
  if (!S[0]) { rc = ORC_ENOMEM; goto done; }
  S[0][0] = 0; len[0] = 1;
  for (int l = 0; l < k; ++l) {
    long long a = e[l].val, n0 = len[l];
    if (2 * n0 > SUM_CAP) { rc = ORC_ETOOBIG; goto done; }
    long long *out = (long long *)malloc((size_t)(2 * n0) * sizeof(long long));
    if (!out) { rc = ORC_ENOMEM; goto done; }
    long long i = 0, j = 0, t = 0;
    while (i < n0 || j < n0) {  /* merge S_l and S_l + a */
      long long x = i < n0 ? S[l][i] : LLONG_MAX;
      long long y = j < n0 ? S[l][j] + a : LLONG_MAX;
      long long v;
      if (x <= y) { v = x; ++i; if (x == y) ++j; } else { v = y; ++j; }
      if (t == 0 || out[t - 1] != v) out[t++] = v;
    }
    S[l + 1] = out; len[l + 1] = t;
  }
  /* bottom-up: classes.  Layer k holds the terminal outcome of each complete sum. */
  cls[k] = (int *)malloc((size_t)len[k] * sizeof(int));
  if (!cls[k]) { rc = ORC_ENOMEM; goto done; }
  for (long long t = 0; t < len[k]; ++t) cls[k][t] = sat(S[k][t], sense, b) ? ORC_TOP : ORC_BOT;
  for (int l = k - 1; l >= 0; --l) {
    long long a = e[l].val, nl = len[l];
    cls[l] = (int *)malloc((size_t)nl * sizeof(int));
    /* open-addressing table: (lo, hi) pair -> node id */
    long long cap = 16;
    while (cap < 2 * nl) cap <<= 1;
    unsigned long long *keys = (unsigned long long *)malloc((size_t)cap * sizeof(unsigned long long));
    int *ids = (int *)malloc((size_t)cap * sizeof(int));
    if (!cls[l] || !keys || !ids) { free(keys); free(ids); rc = ORC_ENOMEM; goto done; }
    for (long long t = 0; t < cap; ++t) keys[t] = ~0ULL;
    int next_id = 0;
    for (long long t = 0; t < nl; ++t) {   /* ascending s: ids come out in min-sum order */
      long long s = S[l][t];
      int c0 = cls[l + 1][find_sum(S[l + 1], len[l + 1], s)];
      int c1 = cls[l + 1][find_sum(S[l + 1], len[l + 1], s + a)];
      if (c0 == ORC_BOT && c1 == ORC_BOT) { cls[l][t] = ORC_BOT; continue; }
      unsigned long long key = ((unsigned long long)(unsigned)(c0 + 2) << 32) | (unsigned)(c1 + 2);
      unsigned long long hsh = key * 0x9E3779B97F4A7C15ULL;
      long long slot = (long long)(hsh >> 20) & (cap - 1);
      while (keys[slot] != ~0ULL && keys[slot] != key) slot = (slot + 1) & (cap - 1);
      if (keys[slot] == ~0ULL) {
        keys[slot] = key; ids[slot] = next_id++;
        if (iv_push(&Llo[l], c0) || iv_push(&Lhi[l], c1) || lv_push(&Lmin[l], s)) {
          free(keys); free(ids); rc = ORC_ENOMEM; goto done;
        }
      }
      cls[l][t] = ids[slot];
    }
    free(keys); free(ids);
  }
  if (cls[0][0] == ORC_BOT) { rc = ORC_EINFEASIBLE; goto done; }
  /* emit */
  if (iv_push(bdd_row, row) || iv_push(bdd_k, k)) { rc = ORC_ENOMEM; goto done; }
  for (int l = 0; l < k; ++l) {
    long long nodes_before = lo->n;
    if (iv_push(occ_var, e[l].col) || lv_push(occ_csr, e[l].pos) || lv_push(occ_node0, nodes_before)) {
      rc = ORC_ENOMEM; goto done;
    }
    for (long long t = 0; t < Llo[l].n; ++t)
      if (iv_push(lo, Llo[l].p[t]) || iv_push(hi, Lhi[l].p[t]) || lv_push(minsum, Lmin[l].p[t])) {
        rc = ORC_ENOMEM; goto done;
      }
  }
done:
  if (S) for (int l = 0; l <= k; ++l) free(S[l]);
  if (cls) for (int l = 0; l <= k; ++l) free(cls[l]);
  if (Llo) for (int l = 0; l < k; ++l) { free(Llo[l].p); free(Lhi[l].p); free(Lmin[l].p); }
  free(S); free(len); free(cls); free(Llo); free(Lhi); free(Lmin);
  return rc;
}

/* Builds all BDDs.  status: ORC_* code; failed_row: the row that made it fail (or -1). */
/* rank: NULL (identity) or a permutation of 0..n-1 giving each variable's place in the order */
void *orc_build_ordered(int n, int m, const long long *row_ptr, const int *col, const int *val,
                        const int *b, const signed char *sense, const double *c, const int *rank,
                        int *status, int *failed_row) {
  *status = ORC_OK; *failed_row = -1;
  if (n < 0 || m < 0) { *status = ORC_EINVAL; return NULL; }
  if (rank) {
    char *seen = (char *)calloc((size_t)n + 1, 1);
    int ok = seen != NULL;
    for (int i = 0; i < n && ok; ++i) {
      if (rank[i] < 0 || rank[i] >= n || seen[rank[i]]) ok = 0;
      else seen[rank[i]] = 1;
    }
    free(seen);
    if (!ok) { *status = ORC_EINVAL; return NULL; }
  }
  g_rank = rank;
  for (int i = 0; i < n; ++i)
    if (!isfinite(c[i])) { *status = ORC_EINVAL; return NULL; }
  oracle_t *h = (oracle_t *)calloc(1, sizeof(oracle_t));
  if (!h) { *status = ORC_ENOMEM; return NULL; }
  h->n = n; h->m = m; h->nnz = m ? row_ptr[m] : 0;
  ivec bdd_row = {0}, bdd_k = {0}, occ_var = {0}, lo = {0}, hi = {0};
  lvec occ_csr = {0}, occ_node0 = {0}, minsum = {0};
  int rc = ORC_OK;
  for (int j = 0; j < m && rc == ORC_OK; ++j) {
    long long s = row_ptr[j], e = row_ptr[j + 1];
    if (e < s || sense[j] < -1 || sense[j] > 1) { rc = ORC_EINVAL; *failed_row = j; break; }
    int k = 0;
    entry_t *ent = (entry_t *)malloc((size_t)(e - s + 1) * sizeof(entry_t));
    if (!ent) { rc = ORC_ENOMEM; break; }
    for (long long t = s; t < e; ++t) {
      if (col[t] < 0 || col[t] >= n) { rc = ORC_EINVAL; break; }
      if (val[t] == 0) continue;            /* zero coefficients are not in I_j */
      ent[k].col = col[t]; ent[k].val = val[t]; ent[k].pos = t; ++k;
    }
    if (rc == ORC_OK) {
      qsort(ent, (size_t)k, sizeof(entry_t), cmp_entry);
      for (int t = 1; t < k; ++t)
        if (ent[t].col == ent[t - 1].col) rc = ORC_EINVAL;   /* duplicate (j, i) */
    }
    if (rc == ORC_OK) {
      if (k == 0) {
        if (!sat(0, sense[j], b[j])) rc = ORC_EINFEASIBLE;
      } else {
        rc = build_row(ent, k, b[j], sense[j], j, &bdd_row, &bdd_k, &occ_var, &occ_csr,
                       &occ_node0, &lo, &hi, &minsum);
      }
    }
    if (rc != ORC_OK) *failed_row = j;
    free(ent);
  }
  g_rank = NULL;
  h->bdd_row = bdd_row.p; h->bdd_k = bdd_k.p; h->occ_var = occ_var.p; h->occ_csr = occ_csr.p;
  h->lo = lo.p; h->hi = hi.p; h->minsum = minsum.p;
  h->nb = (int)bdd_row.n; h->O = occ_var.n; h->N = lo.n;
  if (rc != ORC_OK) { free(occ_node0.p); orc_free(h); *status = rc; return NULL; }
  if (lv_push(&occ_node0, h->N)) { free(occ_node0.p); orc_free(h); *status = ORC_ENOMEM; return NULL; }
  h->occ_node0 = occ_node0.p;

  long long O = h->O, N = h->N;
  h->bdd_occ0 = (long long *)malloc((size_t)(h->nb + 1) * sizeof(long long));
  h->occ_bdd = (int *)malloc((size_t)(O + 1) * sizeof(int));
  h->occ_layer = (int *)malloc((size_t)(O + 1) * sizeof(int));
  h->var_ptr = (long long *)calloc((size_t)n + 1, sizeof(long long));
  h->var_occ = (long long *)malloc((size_t)(O + 1) * sizeof(long long));
  h->deg = (int *)calloc((size_t)n + 1, sizeof(int));
  h->c = (double *)malloc((size_t)(n + 1) * sizeof(double));
  h->lam = (double *)calloc((size_t)O + 1, sizeof(double));
  h->delta = (double *)calloc((size_t)O + 1, sizeof(double));
  h->P = (double *)calloc((size_t)n + 1, sizeof(double));
  h->share = (double *)calloc((size_t)n + 1, sizeof(double));
  h->fm = (double *)calloc((size_t)N + 1, sizeof(double));
  h->bm = (double *)calloc((size_t)N + 1, sizeof(double));
  h->sfm = (double *)calloc((size_t)N + 1, sizeof(double));
  h->sbm = (double *)calloc((size_t)N + 1, sizeof(double));
  h->order = (int *)malloc((size_t)(n + 1) * sizeof(int));
  h->oshare = (double *)calloc((size_t)O + 1, sizeof(double));
  if (!h->order || !h->oshare) { orc_free(h); *status = ORC_ENOMEM; return NULL; }
  for (int i = 0; i < n; ++i) h->order[rank ? rank[i] : i] = i;
  if (!h->bdd_occ0 || !h->occ_bdd || !h->occ_layer || !h->var_ptr || !h->var_occ || !h->deg ||
      !h->c || !h->lam || !h->delta || !h->P || !h->share || !h->fm || !h->bm || !h->sfm ||
      !h->sbm) {
    orc_free(h); *status = ORC_ENOMEM; return NULL;
  }
  long long o = 0;
  h->max_depth = 0; h->max_width = 0;
  for (int bb = 0; bb < h->nb; ++bb) {
    h->bdd_occ0[bb] = o;
    if (h->bdd_k[bb] > h->max_depth) h->max_depth = h->bdd_k[bb];
    for (int l = 0; l < h->bdd_k[bb]; ++l, ++o) {
      h->occ_bdd[o] = bb; h->occ_layer[o] = l;
      int w = (int)(h->occ_node0[o + 1] - h->occ_node0[o]);
      if (w > h->max_width) h->max_width = w;
    }
  }
  h->bdd_occ0[h->nb] = o;
  for (long long t = 0; t < O; ++t) h->deg[h->occ_var[t]]++;
  for (int i = 0; i < n; ++i) h->var_ptr[i + 1] = h->var_ptr[i] + h->deg[i];
  {
    long long *fill = (long long *)malloc((size_t)(n + 1) * sizeof(long long));
    if (!fill) { orc_free(h); *status = ORC_ENOMEM; return NULL; }
    memcpy(fill, h->var_ptr, (size_t)(n + 1) * sizeof(long long));
    for (long long t = 0; t < O; ++t) h->var_occ[fill[h->occ_var[t]]++] = t;  /* ascending row */
    free(fill);
  }
  h->empty_const = 0.0;
  for (int i = 0; i < n; ++i) {
    h->c[i] = c[i];
    if (h->deg[i] == 0 && c[i] < 0) h->empty_const += c[i];
  }
  return h;
}

void *orc_build(int n, int m, const long long *row_ptr, const int *col, const int *val,
                const int *b, const signed char *sense, const double *c, int *status,
                int *failed_row) {
  return orc_build_ordered(n, m, row_ptr, col, val, b, sense, c, NULL, status, failed_row);
}

/* 0: the averaging of eq. mma-update; 1: SRMP averaging (Appendix A.4) */
void orc_set_srmp(void *vh, int srmp) { ((oracle_t *)vh)->srmp = srmp ? 1 : 0; }

void orc_sizes(void *vh, long long out[8]) {
  oracle_t *h = (oracle_t *)vh;
  out[0] = h->n; out[1] = h->m; out[2] = h->nb; out[3] = h->O; out[4] = h->N;
  out[5] = h->max_depth; out[6] = h->max_width; out[7] = h->nnz;
}

/* Canonical export: BDDs in ascending row order; occurrences BDD-major, layer-minor; nodes
 * BDD-major, layer-major, canonical order inside a layer; lo/hi are next-layer local ids. */
void orc_export(void *vh, int *bdd_row, int *bdd_depth, int *occ_var, long long *occ_csr,
                int *occ_width, int *lo, int *hi, long long *minsum) {
  oracle_t *h = (oracle_t *)vh;
  for (int b = 0; b < h->nb; ++b) { bdd_row[b] = h->bdd_row[b]; bdd_depth[b] = h->bdd_k[b]; }
  for (long long o = 0; o < h->O; ++o) {
    occ_var[o] = h->occ_var[o];
    occ_csr[o] = h->occ_csr[o];
    occ_width[o] = (int)(h->occ_node0[o + 1] - h->occ_node0[o]);
  }
  for (long long v = 0; v < h->N; ++v) {
    lo[v] = h->lo[v]; hi[v] = h->hi[v];
    if (minsum) minsum[v] = h->minsum[v];
  }
}

/* ------------------------------------------------------------------------------------ */
/* dynamic programmes (Alg. 2 / Alg. 3, eqs. arc-marginal and marginal-aggregation)       */
/* ------------------------------------------------------------------------------------ */
/* The aggregation of Table 3: min(a, b) for min-sum; for alpha > 0 the log-sum-exp column in
 * the -alpha log domain, -alpha log(exp(-a/alpha) + exp(-b/alpha)), written as
 * min(a, b) - alpha log(1 + exp(-|a - b| / alpha)). */
static double agg(const oracle_t *h, double a, double b) {
  if (h->alpha <= 0.0) return a < b ? a : b;
  if (isinf(a)) return b;
  if (isinf(b)) return a;
  double m = a < b ? a : b;
  return m - h->alpha * log1p(exp(-fabs(a - b) / h->alpha));
}

/* backward message of the target t of an arc leaving layer o (t is a local id in o+1) */
static double bval(const oracle_t *h, const double *bm, long long o, int t) {
  if (t == ORC_TOP) return 0.0;
  if (t == ORC_BOT) return INFINITY;
  if (t <= ORC_COPY0) return h->mu_bar[ORC_COPY0 - t];
  return bm[h->occ_node0[o + 1] + t];
}

/* initial forward message of a first-layer node: 0 at the root of a whole BDD or first piece;
 * for a later piece, the cheapest entry arc (+inf if none enters the node) */
static double root_msg(const oracle_t *h, long long v) { return h->root_f ? h->root_f[v] : 0.0; }

/* Full forward programme of BDD b into fm: m_fwd(root) = 0, then for every layer the min
 * over in-arcs (each arc relaxed once). */
static void dp_forward(const oracle_t *h, int b, const double *lam, double *fm) {
  long long o0 = h->bdd_occ0[b];
  int k = h->bdd_k[b];
  for (long long v = h->occ_node0[o0]; v < h->occ_node0[o0 + 1]; ++v) fm[v] = root_msg(h, v);
  for (int l = 1; l < k; ++l) {
    long long o = o0 + l;
    for (long long v = h->occ_node0[o]; v < h->occ_node0[o + 1]; ++v) fm[v] = INFINITY;
    for (long long u = h->occ_node0[o - 1]; u < h->occ_node0[o]; ++u) {
      if (h->lo[u] >= 0) {
        long long v = h->occ_node0[o] + h->lo[u];
        fm[v] = agg(h, fm[v], fm[u]);
      }
      if (h->hi[u] >= 0) {
        long long v = h->occ_node0[o] + h->hi[u];
        double x = fm[u] + lam[o - 1];
        fm[v] = agg(h, fm[v], x);
      }
    }
  }
}

/* backward update step (Alg. 3) for the nodes of occurrence o */
static void bwd_step(const oracle_t *h, long long o, double lam_o, double *bm) {
  for (long long u = h->occ_node0[o]; u < h->occ_node0[o + 1]; ++u) {
    double a0 = bval(h, bm, o, h->lo[u]);
    double a1 = lam_o + bval(h, bm, o, h->hi[u]);
    if (h->hi[u] == ORC_BOT) a1 = INFINITY;
    bm[u] = agg(h, a0, a1);
  }
}

/* E^j from the backward messages of the first layer: m_bwd(root) for a whole BDD, the min over
 * roots of (initial forward message + m_bwd) for a piece */
static double piece_energy(const oracle_t *h, int b, const double *bm) {
  long long o0 = h->bdd_occ0[b];
  if (!h->root_f) return bm[h->occ_node0[o0]];
  double e = INFINITY;
  for (long long v = h->occ_node0[o0]; v < h->occ_node0[o0 + 1]; ++v) e = agg(h, e, h->root_f[v] + bm[v]);
  return e;
}

/* Full backward programme of BDD b into bm; returns E^j. */
static double dp_backward(const oracle_t *h, int b, const double *lam, double *bm) {
  long long o0 = h->bdd_occ0[b];
  for (int l = h->bdd_k[b] - 1; l >= 0; --l) bwd_step(h, o0 + l, lam[o0 + l], bm);
  return piece_energy(h, b, bm);
}

/* min-marginals of occurrence o from fm (its layer) and bm (next layer) */
static void aggregate(const oracle_t *h, long long o, double lam_o, const double *fm,
                      const double *bm, double *m0, double *m1) {
  double a = INFINITY, c1 = INFINITY;
  for (long long u = h->occ_node0[o]; u < h->occ_node0[o + 1]; ++u) {
    if (h->lo[u] != ORC_BOT) {
      double x = fm[u] + bval(h, bm, o, h->lo[u]);
      a = agg(h, a, x);
    }
    if (h->hi[u] != ORC_BOT) {
      double x = fm[u] + lam_o + bval(h, bm, o, h->hi[u]);
      c1 = agg(h, c1, x);
    }
  }
  *m0 = a; *m1 = c1;
}

/* Definitional min-marginals of occurrence o under lam: full programmes on scratch arrays. */
static void minmarg_full(oracle_t *h, long long o, const double *lam, double *m0, double *m1) {
  int b = h->occ_bdd[o];
  dp_forward(h, b, lam, h->sfm);
  dp_backward(h, b, lam, h->sbm);
  aggregate(h, o, lam[o], h->sfm, h->sbm, m0, m1);
}

static double energy(oracle_t *h, int b, const double *lam) {
  return dp_backward(h, b, lam, h->sbm);
}

/* y-slack lower bound for the current lam and pending P (fresh programmes) */
double orc_bound(void *vh) {
  oracle_t *h = (oracle_t *)vh;
  double lb = h->empty_const;
  for (int b = 0; b < h->nb; ++b) lb += energy(h, b, h->lam);
  for (int i = 0; i < h->n; ++i)
    if (h->deg[i] > 0) lb += agg(h, 0.0, h->P[i]);
  return lb;
}

static double mm_diff(double m0, double m1) {
  return (isinf(m0) || isinf(m1)) ? 0.0 : m1 - m0;
}

static double rel(double err, double scale) {
  return fabs(err) / (1.0 > fabs(scale) ? 1.0 : fabs(scale));
}

static void note(double *w, double v) { if (v > *w) *w = v; }

/* ------------------------------------------------------------------------------------ */
/* initialisation                                                                         */
/* ------------------------------------------------------------------------------------ */
/* lambda^j_i = c_i / |J_i| (Alg. 1 initialisation), P = 0, then a full backward programme
 * so that every backward message is valid (precondition of Prop. 3). */
void orc_init_dual(void *vh) {
  oracle_t *h = (oracle_t *)vh;
  for (long long o = 0; o < h->O; ++o) h->lam[o] = h->c[h->occ_var[o]] / h->deg[h->occ_var[o]];
  for (int i = 0; i < h->n; ++i) h->P[i] = 0.0;
  for (long long k = 0; k < h->npairs; ++k) h->mu_bar[k] = h->mu[k] = h->dfwd[k] = h->dbwd[k] = 0.0;
  for (long long k = 0; k < h->npairs; ++k) h->root_f[h->pair_w[k]] = 0.0;
  for (int b = 0; b < h->nb; ++b) dp_backward(h, b, h->lam, h->bm);
  for (int t = 0; t < 5; ++t) h->worst[t] = 0.0;
}

/* Sets the smoothing temperature (0 = min-sum) and restarts the dual state. */
void orc_set_alpha(void *vh, double alpha) {
  oracle_t *h = (oracle_t *)vh;
  h->alpha = alpha > 0.0 ? alpha : 0.0;
  h->empty_const = 0.0;
  for (int i = 0; i < h->n; ++i)
    if (h->deg[i] == 0) h->empty_const += agg(h, 0.0, h->c[i]);
  orc_init_dual(vh);
}

void orc_worst(void *vh, double out[5]) {
  oracle_t *h = (oracle_t *)vh;
  for (int t = 0; t < 5; ++t) out[t] = h->worst[t];
}

/* ------------------------------------------------------------------------------------ */
/* schedule P: parallel across BDDs, deferred averaging                                   */
/* ------------------------------------------------------------------------------------ */
static void check_invariant(oracle_t *h) {
  for (int i = 0; i < h->n; ++i) {
    if (h->deg[i] == 0) continue;
    double s = h->P[i], scale = fabs(h->c[i]) + fabs(h->P[i]);
    for (long long t = h->var_ptr[i]; t < h->var_ptr[i + 1]; ++t) {
      s += h->lam[h->var_occ[t]];
      scale += fabs(h->lam[h->var_occ[t]]);
    }
    note(&h->worst[1], rel(s - h->c[i], scale));
  }
}

static void form_pending(oracle_t *h) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < h->n; ++i) {
    double s = 0.0;
    for (long long t = h->var_ptr[i]; t < h->var_ptr[i + 1]; ++t) s += h->delta[h->var_occ[t]];
    h->P[i] = s;
  }
}

/* Is occurrence o among the subproblems that take i's share in a forward (backward) sweep?  For
 * SRMP: those with a variable after (before) i, i.e. o is not the last (first) layer of its BDD. */
static int srmp_takes(const oracle_t *h, long long o, int forward) {
  int l = h->occ_layer[o], k = h->bdd_k[h->occ_bdd[o]];
  return forward ? l < k - 1 : l > 0;
}

/* The share each occurrence takes in the next sweep: P_i / |J_i| (eq. mma-update), or for SRMP
 * P_i / |J_i^>| on J_i^> in a forward sweep (J_i^< backward), all of J_i when that set is empty. */
static void take_share(oracle_t *h, int forward) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < h->n; ++i) {
    long long s = h->var_ptr[i], e = h->var_ptr[i + 1];
    if (e == s) continue;
    int cnt = 0;
    if (h->srmp)
      for (long long t = s; t < e; ++t) cnt += srmp_takes(h, h->var_occ[t], forward);
    for (long long t = s; t < e; ++t) {
      long long o = h->var_occ[t];
      if (!h->srmp || cnt == 0)
        h->oshare[o] = h->P[i] / (double)(e - s);
      else
        h->oshare[o] = srmp_takes(h, o, forward) ? h->P[i] / cnt : 0.0;
    }
  }
}

static void sweep_forward(oracle_t *h, double omega, int check) {
  take_share(h, 1);
#pragma omp parallel for schedule(dynamic, 64) if (!check)
  for (int b = 0; b < h->nb; ++b) {
    long long o0 = h->bdd_occ0[b];
    int k = h->bdd_k[b];
    for (long long v = h->occ_node0[o0]; v < h->occ_node0[o0 + 1]; ++v) h->fm[v] = root_msg(h, v);
    for (int l = 0; l < k; ++l) {
      long long o = o0 + l;
      if (l > 0) {  /* Alg. 2 for the nodes of layer l */
        for (long long v = h->occ_node0[o]; v < h->occ_node0[o + 1]; ++v) h->fm[v] = INFINITY;
        for (long long u = h->occ_node0[o - 1]; u < h->occ_node0[o]; ++u) {
          if (h->lo[u] >= 0) {
            long long v = h->occ_node0[o] + h->lo[u];
            h->fm[v] = agg(h, h->fm[v], h->fm[u]);
          }
          if (h->hi[u] >= 0) {
            long long v = h->occ_node0[o] + h->hi[u];
            double x = h->fm[u] + h->lam[o - 1];
            h->fm[v] = agg(h, h->fm[v], x);
          }
        }
      }
      h->lam[o] += h->oshare[o];
      double m0, m1;
      aggregate(h, o, h->lam[o], h->fm, h->bm, &m0, &m1);
      if (check) {
        double r0, r1;
        minmarg_full(h, o, h->lam, &r0, &r1);
        if (isinf(r0) != isinf(m0) || isinf(r1) != isinf(m1)) note(&h->worst[2], INFINITY);
        if (!isinf(r0)) note(&h->worst[2], rel(r0 - m0, r0));
        if (!isinf(r1)) note(&h->worst[2], rel(r1 - m1, r1));
      }
      double d = omega * mm_diff(m0, m1);
      h->lam[o] -= d;
      h->delta[o] = d;
    }
  }
  form_pending(h);
}

static void sweep_backward(oracle_t *h, double omega, int check) {
  take_share(h, 0);
#pragma omp parallel for schedule(dynamic, 64) if (!check)
  for (int b = 0; b < h->nb; ++b) {
    long long o0 = h->bdd_occ0[b];
    for (int l = h->bdd_k[b] - 1; l >= 0; --l) {
      long long o = o0 + l;
      h->lam[o] += h->oshare[o];
      double m0, m1;
      aggregate(h, o, h->lam[o], h->fm, h->bm, &m0, &m1);
      if (check) {
        double r0, r1;
        minmarg_full(h, o, h->lam, &r0, &r1);
        if (isinf(r0) != isinf(m0) || isinf(r1) != isinf(m1)) note(&h->worst[2], INFINITY);
        if (!isinf(r0)) note(&h->worst[2], rel(r0 - m0, r0));
        if (!isinf(r1)) note(&h->worst[2], rel(r1 - m1, r1));
      }
      double d = omega * mm_diff(m0, m1);
      h->lam[o] -= d;
      h->delta[o] = d;
      bwd_step(h, o, h->lam[o], h->bm);  /* Alg. 3 with the updated lambda */
    }
  }
  form_pending(h);
}

/* Copy-arc pair updates (Sec. 6, the parallel averaging algorithm).  After a forward sweep:
 * m_bar = m_fwd(tail) + theta + mu_bar is the cost of the best path of the earlier piece through
 * the copy arc; delta_fwd = m_bar - its minimum over the cut (0 where either is infinite) and
 * mu_bar += -gamma * delta_fwd + gamma * delta_bwd.  After a backward sweep: m = mu + m_bwd(head)
 * (the entry node's forward message is 0, the entry arc carries no theta); delta_bwd likewise
 * and mu += -gamma * delta_bwd + gamma * delta_fwd; then every later piece's root message is
 * the minimum of mu over the entry arcs into it. */
static double copy_marginal(const oracle_t *h, long long k) {
  return h->fm[h->pair_u[k]] + (h->pair_hi[k] ? h->lam[h->pair_occ[k]] : 0.0) + h->mu_bar[k];
}

static double entry_marginal(const oracle_t *h, long long k) { return h->mu[k] + h->bm[h->pair_w[k]]; }

static double cut_delta(double m, double mn) { return (isinf(m) || isinf(mn)) ? 0.0 : m - mn; }

static void cut_forward(oracle_t *h) {
  for (int c = 0; c < h->ncuts; ++c) {
    long long s = h->cut_ptr[c], e = h->cut_ptr[c + 1];
    double mn = INFINITY;
    for (long long k = s; k < e; ++k) {
      double m = copy_marginal(h, k);
      if (m < mn) mn = m;
    }
    for (long long k = s; k < e; ++k) h->dfwd[k] = cut_delta(copy_marginal(h, k), mn);
    for (long long k = s; k < e; ++k) h->mu_bar[k] += -h->gamma * h->dfwd[k] + h->gamma * h->dbwd[k];
  }
}

static void cut_backward(oracle_t *h) {
  for (int c = 0; c < h->ncuts; ++c) {
    long long s = h->cut_ptr[c], e = h->cut_ptr[c + 1];
    double mn = INFINITY;
    for (long long k = s; k < e; ++k) {
      double m = entry_marginal(h, k);
      if (m < mn) mn = m;
    }
    for (long long k = s; k < e; ++k) h->dbwd[k] = cut_delta(entry_marginal(h, k), mn);
    for (long long k = s; k < e; ++k) h->mu[k] += -h->gamma * h->dbwd[k] + h->gamma * h->dfwd[k];
  }
  for (long long k = 0; k < h->npairs; ++k) h->root_f[h->pair_w[k]] = INFINITY;
  for (long long k = 0; k < h->npairs; ++k)
    if (h->mu[k] < h->root_f[h->pair_w[k]]) h->root_f[h->pair_w[k]] = h->mu[k];
}

/* bound from the current messages: valid right after a backward sweep */
static double bound_after_backward(const oracle_t *h) {
  double lb = h->empty_const;
  for (int b = 0; b < h->nb; ++b) lb += piece_energy(h, b, h->bm);
  for (int i = 0; i < h->n; ++i)
    if (h->deg[i] > 0) lb += agg(h, 0.0, h->P[i]);
  return lb;
}

/* iters iterations (forward sweep, backward sweep) of schedule P.  trace[t] = bound after
 * iteration t.  check: invariant, incremental-vs-definitional min-marginals and a fresh bound
 * after every sweep (monotonicity), recorded in orc_worst(). */
int orc_run_parallel(void *vh, int iters, double omega, int check, double *trace) {
  oracle_t *h = (oracle_t *)vh;
  double prev = check ? orc_bound(h) : 0.0;
  for (int it = 0; it < iters; ++it) {
    sweep_forward(h, omega, check);
    if (h->ncuts) cut_forward(h);
    if (check) {
      check_invariant(h);
      double lb = orc_bound(h);
      note(&h->worst[0], rel(prev - lb, lb) * (prev > lb ? 1.0 : 0.0));
      prev = lb;
    }
    sweep_backward(h, omega, check);
    double lb = bound_after_backward(h);
    if (check) {
      check_invariant(h);
      double fresh = orc_bound(h);
      note(&h->worst[2], rel(fresh - lb, fresh));
      note(&h->worst[0], rel(prev - fresh, fresh) * (prev > fresh ? 1.0 : 0.0));
      prev = fresh;
    }
    if (h->ncuts) {
      cut_backward(h);
      if (check) {
        double after = orc_bound(h);
        note(&h->worst[0], rel(prev - after, after) * (prev > after ? 1.0 : 0.0));
        prev = after;
      }
    }
    if (trace) trace[it] = lb;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* derivative of the smoothed bound after K iterations of schedule P (Appendix A.5)       */
/* ------------------------------------------------------------------------------------ */
/* With alpha > 0 every aggregation is the soft minimum z = -alpha log sum_k exp(-x_k / alpha),
 * a smooth function of its arguments with dz/dx_k = exp(-(x_k - z) / alpha) (the Gibbs weight of
 * term k; 0 for x_k = +inf).  The bound after K iterations of schedule P is then a composition
 * of smooth steps of the costs c (lambda_0 = c_i/|J_i|, the initial backward programme, 2K
 * sweeps with their pending sums, the y-slack term), so reverse-mode differentiation gives
 * d bound / d c exactly: the forward run below keeps the inputs and outputs of every sweep,
 * and each step is then reversed in the opposite order.  Plain reverse-mode, no
 * recomputation tricks: a tape of (2K + 1) (O + n) + (2K + 1) N doubles. */

static double gibbs(const oracle_t *h, double x, double z) { return isinf(x) ? 0.0 : exp(-(x - z) / h->alpha); }

/* weight of P_i in the share occurrence o takes in a forward (backward) sweep (take_share) */
static double share_weight(const oracle_t *h, long long o, int forward) {
  int i = h->occ_var[o];
  long long s = h->var_ptr[i], e = h->var_ptr[i + 1];
  if (!h->srmp) return 1.0 / (double)(e - s);
  int cnt = 0;
  for (long long t = s; t < e; ++t) cnt += srmp_takes(h, h->var_occ[t], forward);
  if (cnt == 0) return 1.0 / (double)(e - s);
  return srmp_takes(h, o, forward) ? 1.0 / (double)cnt : 0.0;
}

/* Reverse of the backward update step b(u) = agg(b(lo u), lam_o + b(hi u)) of the nodes of
 * occurrence o, given the adjoints gb of those nodes: adds to gb of the next layer and to
 * *glam.  bm holds the messages of both layers. */
static void bwd_step_adjoint(const oracle_t *h, long long o, double lam_o, const double *bm, double *gb,
                             double *glam) {
  long long n1 = h->occ_node0[o + 1];
  for (long long u = h->occ_node0[o]; u < h->occ_node0[o + 1]; ++u) {
    double g = gb[u];
    if (g == 0.0) continue;
    double a0 = bval(h, bm, o, h->lo[u]);
    double a1 = h->hi[u] == ORC_BOT ? INFINITY : lam_o + bval(h, bm, o, h->hi[u]);
    double w0 = gibbs(h, a0, bm[u]), w1 = gibbs(h, a1, bm[u]);
    if (h->lo[u] >= 0) gb[n1 + h->lo[u]] += g * w0;
    if (h->hi[u] >= 0) gb[n1 + h->hi[u]] += g * w1;
    *glam += g * w1;
  }
}

/* Reverse of eq. marginal-aggregation for occurrence o (m0, m1 from fm of its layer and bm of
 * the next) followed by d = omega (m1 - m0): given gd, adds to gfm of the layer's nodes, gbm of
 * the next layer's nodes and *gmu (the multiplier the 1-arcs carry). */
static void marginal_adjoint(const oracle_t *h, long long o, double mu, const double *fm, const double *bm,
                             double omega, double gd, double *gfm, double *gbm, double *gmu) {
  double m0, m1;
  aggregate(h, o, mu, fm, bm, &m0, &m1);
  if (isinf(m0) || isinf(m1) || gd == 0.0) return;  /* d = 0 there (reading r3): no dependence */
  double g1 = omega * gd, g0 = -omega * gd;
  long long n1 = h->occ_node0[o + 1];
  for (long long u = h->occ_node0[o]; u < h->occ_node0[o + 1]; ++u) {
    if (h->lo[u] != ORC_BOT) {
      double w = gibbs(h, fm[u] + bval(h, bm, o, h->lo[u]), m0);
      gfm[u] += g0 * w;
      if (h->lo[u] >= 0) gbm[n1 + h->lo[u]] += g0 * w;
    }
    if (h->hi[u] != ORC_BOT) {
      double w = gibbs(h, fm[u] + mu + bval(h, bm, o, h->hi[u]), m1);
      gfm[u] += g1 * w;
      *gmu += g1 * w;
      if (h->hi[u] >= 0) gbm[n1 + h->hi[u]] += g1 * w;
    }
  }
}

/* Smoothed bound after K >= 0 iterations of schedule P from lambda_0 = c_i/|J_i| (the value
 * orc_run_parallel's trace ends with), and its gradient with respect to c, both FP64.  Needs
 * alpha > 0 and no copy-arc pairs.  Leaves the dual state after K iterations.  Returns 0, or
 * ORC_EINVAL / ORC_ENOMEM. */
int orc_smooth_gradient(void *vh, int K, double omega, double *bound, double *grad_c) {
  oracle_t *h = (oracle_t *)vh;
  if (!(h->alpha > 0.0) || h->npairs > 0 || K < 0) return ORC_EINVAL;
  const long long O = h->O, N = h->N, S = 2LL * K;
  const int n = h->n;
  /* tape: multipliers and pending sums at the start of sweep s (s = 2K: the end state), the
   * messages after the initial backward programme and after every sweep */
  double *lam_t = (double *)malloc((size_t)((S + 1) * O + 1) * sizeof(double));
  double *P_t = (double *)malloc((size_t)((S + 1) * n + 1) * sizeof(double));
  double *msg_t = (double *)malloc((size_t)((S + 1) * N + 1) * sizeof(double));
  double *glam = (double *)calloc((size_t)O + 1, sizeof(double));   /* adjoint of lambda */
  double *gdel = (double *)calloc((size_t)O + 1, sizeof(double));   /* adjoint of delta */
  double *gshr = (double *)calloc((size_t)O + 1, sizeof(double));   /* adjoint of the shares */
  double *gP = (double *)calloc((size_t)n + 1, sizeof(double));     /* adjoint of P */
  double *gin = (double *)calloc((size_t)N + 1, sizeof(double));    /* adjoint of the messages a sweep reads */
  double *gout = (double *)calloc((size_t)N + 1, sizeof(double));   /* adjoint of the messages a sweep writes */
  double *wf = (double *)malloc((size_t)(O + 1) * sizeof(double));
  double *wb = (double *)malloc((size_t)(O + 1) * sizeof(double));
  if (!lam_t || !P_t || !msg_t || !glam || !gdel || !gshr || !gP || !gin || !gout || !wf || !wb) {
    free(lam_t); free(P_t); free(msg_t); free(glam); free(gdel); free(gshr); free(gP); free(gin);
    free(gout); free(wf); free(wb);
    return ORC_ENOMEM;
  }
  for (long long o = 0; o < O; ++o) { wf[o] = share_weight(h, o, 1); wb[o] = share_weight(h, o, 0); }

  /* ---- forward run (the oracle's own schedule P), taping every sweep's inputs ---- */
  orc_init_dual(h);  /* lambda_0 = c/|J_i|, P = 0, initial backward programme into bm */
  memcpy(msg_t, h->bm, (size_t)N * sizeof(double));
  for (long long s = 0; s < S; ++s) {
    memcpy(lam_t + s * O, h->lam, (size_t)O * sizeof(double));
    memcpy(P_t + s * n, h->P, (size_t)n * sizeof(double));
    if (s % 2 == 0) {
      sweep_forward(h, omega, 0);
      memcpy(msg_t + (s + 1) * N, h->fm, (size_t)N * sizeof(double));
    } else {
      sweep_backward(h, omega, 0);
      memcpy(msg_t + (s + 1) * N, h->bm, (size_t)N * sizeof(double));
    }
  }
  memcpy(lam_t + S * O, h->lam, (size_t)O * sizeof(double));
  memcpy(P_t + S * n, h->P, (size_t)n * sizeof(double));
  /* the bound: the energies from the last backward messages (the initial programme's for K =
   * 0) plus the soft y-slack terms */
  const double *bm_last = msg_t + S * N;
  double lb = h->empty_const;
  for (int b = 0; b < h->nb; ++b) lb += piece_energy(h, b, bm_last);
  for (int i = 0; i < n; ++i)
    if (h->deg[i] > 0) lb += agg(h, 0.0, P_t[S * n + i]);
  *bound = lb;

  /* ---- reverse ---- */
  for (int i = 0; i < n; ++i) grad_c[i] = 0.0;
  /* d bound: 1 on every root's backward message; the slack term's Gibbs weight on P_i; for a
   * variable in no row, the weight of c_i in agg(0, c_i) */
  for (int b = 0; b < h->nb; ++b) gout[h->occ_node0[h->bdd_occ0[b]]] += 1.0;
  for (int i = 0; i < n; ++i) {
    if (h->deg[i] > 0) {
      double P = P_t[S * n + i];
      gP[i] = gibbs(h, P, agg(h, 0.0, P));
    } else {
      grad_c[i] = gibbs(h, h->c[i], agg(h, 0.0, h->c[i]));
    }
  }
  /* gout holds the adjoint of the messages the last sweep wrote (bm); glam of the end state is 0 */
  for (long long s = S - 1; s >= 0; --s) {
    const int forward = s % 2 == 0;
    const double *lam0 = lam_t + s * O, *lam1 = lam_t + (s + 1) * O;  /* before / after the sweep */
    const double *Pin = P_t + s * n;
    const double *mout = msg_t + (s + 1) * N;   /* fm (forward) / bm (backward) written */
    const double *min = msg_t + s * N;          /* bm (forward) / fm (backward) read */
    const double *w = forward ? wf : wb;
    /* pending sums after the sweep: P_i = sum of its deltas */
    for (int i = 0; i < n; ++i)
      for (long long t = h->var_ptr[i]; t < h->var_ptr[i + 1]; ++t) gdel[h->var_occ[t]] += gP[i];
    for (int i = 0; i < n; ++i) gP[i] = 0.0;
    for (long long v = 0; v < N; ++v) gin[v] = 0.0;
    for (long long o = 0; o < O; ++o) gshr[o] = 0.0;
    /* glam: adjoint of lambda after the sweep (lam1); becomes the adjoint before it (lam0) */
    for (int b = 0; b < h->nb; ++b) {
      long long o0 = h->bdd_occ0[b];
      int k = h->bdd_k[b];
      if (forward) {
        /* layers in reverse: lam1 = mu - d, d = omega (m1 - m0) from fm (this sweep) and bm (read),
         * then fm of the layer from the previous layer (Alg. 2) */
        for (int l = k - 1; l >= 0; --l) {
          long long o = o0 + l;
          double mu = lam0[o] + w[o] * Pin[h->occ_var[o]];
          double gmu = glam[o];
          double gd = gdel[o] - glam[o];
          marginal_adjoint(h, o, mu, mout, min, omega, gd, gout, gin, &gmu);
          glam[o] = gmu;   /* lambda before the sweep enters mu with weight 1 */
          gshr[o] = gmu;
          if (l > 0) {     /* fm(v) = agg over arcs u -> v of fm(u) + theta, theta = lam1 on 1-arcs */
            long long ol = o - 1;
            long long nl = h->occ_node0[o];
            for (long long u = h->occ_node0[ol]; u < h->occ_node0[o]; ++u) {
              if (h->lo[u] >= 0) {
                long long v = nl + h->lo[u];
                gout[u] += gout[v] * gibbs(h, mout[u], mout[v]);
              }
              if (h->hi[u] >= 0) {
                long long v = nl + h->hi[u];
                double wt = gout[v] * gibbs(h, mout[u] + lam1[ol], mout[v]);
                gout[u] += wt;
                glam[ol] += wt;  /* adjoint of lam1 of the previous layer (processed next) */
              }
            }
          }
        }
      } else {
        /* layers in reverse of the backward order (first to last): bm of the layer (Alg. 3 with
         * lam1), then lam1 = mu - d, d from fm (read) and bm of the next layer (written) */
        for (int l = 0; l < k; ++l) {
          long long o = o0 + l;
          double mu = lam0[o] + w[o] * Pin[h->occ_var[o]];
          double gl1 = glam[o];
          bwd_step_adjoint(h, o, lam1[o], mout, gout, &gl1);
          double gmu = gl1;
          double gd = gdel[o] - gl1;
          marginal_adjoint(h, o, mu, min, mout, omega, gd, gin, gout, &gmu);
          glam[o] = gmu;
          gshr[o] = gmu;
        }
      }
    }
    for (long long o = 0; o < O; ++o) gdel[o] = 0.0;
    /* the shares came from the pending sums before the sweep */
    for (long long o = 0; o < O; ++o) gP[h->occ_var[o]] += w[o] * gshr[o];
    /* messages read by this sweep were written by the previous one */
    memcpy(gout, gin, (size_t)N * sizeof(double));
  }
  /* gout: adjoint of the initial backward programme's messages (with lambda_0); P_0 = 0 is a
   * constant, so gP is dropped */
  for (int b = 0; b < h->nb; ++b) {
    long long o0 = h->bdd_occ0[b];
    for (int l = 0; l < h->bdd_k[b]; ++l) {
      long long o = o0 + l;
      double g = 0.0;
      bwd_step_adjoint(h, o, lam_t[o], msg_t, gout, &g);
      glam[o] += g;
    }
  }
  /* lambda_0 = c_i / |J_i| */
  for (long long o = 0; o < O; ++o) grad_c[h->occ_var[o]] += glam[o] / (double)h->deg[h->occ_var[o]];
  free(lam_t); free(P_t); free(msg_t); free(glam); free(gdel); free(gshr); free(gP); free(gin);
  free(gout); free(wf); free(wb);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* schedule S: Alg. 1 with definitional min-marginals                                     */
/* ------------------------------------------------------------------------------------ */
static void visit_variable(oracle_t *h, int i, int forward, int check, double *m0s,
                           double *m1s) {
  long long s = h->var_ptr[i], e = h->var_ptr[i + 1];
  int J = (int)(e - s);
  if (J == 0) return;
  int Jt = 0;  /* SRMP: |J_i^>| in a forward pass, |J_i^<| in a backward pass */
  if (h->srmp)
    for (long long t = s; t < e; ++t) Jt += srmp_takes(h, h->var_occ[t], forward);
  double S = 0.0, neg = 0.0, before = 0.0;
  int finite = 1;
  for (long long t = s; t < e; ++t) {
    long long o = h->var_occ[t];
    minmarg_full(h, o, h->lam, &m0s[t - s], &m1s[t - s]);
    if (isinf(m0s[t - s]) || isinf(m1s[t - s])) finite = 0;
    double d = mm_diff(m0s[t - s], m1s[t - s]);
    S += d;
    if (d < 0) neg += d;
    if (check) before += energy(h, h->occ_bdd[o], h->lam);
  }
  for (long long t = s; t < e; ++t) {  /* eq. (mma-update), or eq. (srmp-update) */
    long long o = h->var_occ[t];
    double add = S / J;
    if (h->srmp && Jt > 0) add = srmp_takes(h, o, forward) ? S / Jt : 0.0;
    h->lam[o] += -mm_diff(m0s[t - s], m1s[t - s]) + add;
  }
  if (check) {
    double after = 0.0;
    for (long long t = s; t < e; ++t) after += energy(h, h->occ_bdd[h->var_occ[t]], h->lam);
    double gain = after - before;
    double scale = fabs(before) + fabs(S) + fabs(neg);
    if (finite) note(&h->worst[3], rel(gain - ((S < 0 ? S : 0.0) - neg), scale));
    if (gain < 0) note(&h->worst[4], rel(gain, scale));
  }
}

/* iters iterations of Alg. 1 (forward pass over i = 0..n-1, backward pass over n-1..0),
 * trace[t] = sum_j E^j after iteration t.  Requires each variable to lie in distinct rows
 * only once (true by construction). */
int orc_run_sequential(void *vh, int iters, int check, double *trace) {
  oracle_t *h = (oracle_t *)vh;
  int maxJ = 1;
  for (int i = 0; i < h->n; ++i) if (h->deg[i] > maxJ) maxJ = h->deg[i];
  double *m0s = (double *)malloc((size_t)maxJ * sizeof(double));
  double *m1s = (double *)malloc((size_t)maxJ * sizeof(double));
  if (!m0s || !m1s) { free(m0s); free(m1s); return ORC_ENOMEM; }
  for (int i = 0; i < h->n; ++i) h->P[i] = 0.0;
  double prev = orc_bound(h);
  for (int it = 0; it < iters; ++it) {
    for (int k = 0; k < h->n; ++k) visit_variable(h, h->order[k], 1, check, m0s, m1s);
    for (int k = h->n - 1; k >= 0; --k) visit_variable(h, h->order[k], 0, check, m0s, m1s);
    double lb = orc_bound(h);
    if (check) {
      check_invariant(h);
      note(&h->worst[0], rel(prev - lb, lb) * (prev > lb ? 1.0 : 0.0));
    }
    prev = lb;
    if (trace) trace[it] = lb;
  }
  /* leave messages consistent with lambda */
  for (int b = 0; b < h->nb; ++b) dp_backward(h, b, h->lam, h->bm);
  free(m0s); free(m1s);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* state access (arrays indexed by position in the input CSR; zero coefficients get 0)    */
/* ------------------------------------------------------------------------------------ */
/* Is there a cut between layers l-1 and l of a BDD with first occurrence o0 and k layers?
 * With intervals (Sec. 6): its two variables lie in different intervals.  With a depth limit D
 * (interval == NULL; a reading for deep BDDs, below): l is one of floor(t k / q), t = 1 .. q-1,
 * q = ceil(k / D). */
static int cut_before(const oracle_t *h, const int *interval, int D, long long o0, int k, int l) {
  if (interval) return interval[h->occ_var[o0 + l]] != interval[h->occ_var[o0 + l - 1]];
  int q = (k + D - 1) / D;
  for (int t = 1; t < q; ++t)
    if ((long long)t * k / q == l) return 1;
  return 0;
}

static int split_core(oracle_t *h, const int *interval, int D, double gamma);

/* Splits every BDD into pieces at the interval boundaries of the variable order (Sec. 6, Def.
 * of sub-BDDs): cuts[0 .. ncuts) are ascending positions in the order; variable i lies in
 * interval #{t : cuts[t] <= place of i}.  A BDD is cut between consecutive layers whose
 * variables lie in different intervals.  gamma: the copy-arc step size.  Call before any
 * iteration (it restarts the dual state).  Returns the number of pieces, or -1 on bad input. */
int orc_split(void *vh, int ncuts, const int *cuts, double gamma) {
  oracle_t *h = (oracle_t *)vh;
  if (ncuts < 0 || h->ncuts || !(gamma > 0.0 && gamma <= 1.0)) return -1;
  for (int t = 0; t < ncuts; ++t)
    if (cuts[t] < 1 || cuts[t] >= h->n || (t > 0 && cuts[t] <= cuts[t - 1])) return -1;
  int *place = (int *)malloc((size_t)(h->n + 1) * sizeof(int));
  int *interval = (int *)malloc((size_t)(h->n + 1) * sizeof(int));
  if (!place || !interval) { free(place); free(interval); return -1; }
  for (int k = 0; k < h->n; ++k) place[h->order[k]] = k;
  for (int i = 0; i < h->n; ++i) {
    int c = 0;
    while (c < ncuts && cuts[c] <= place[i]) ++c;
    interval[i] = c;
  }
  free(place);
  int r = split_core(h, interval, 0, gamma);
  free(interval);
  return r;
}

/* Depth split (a reading: Sec. 6 cuts a BDD wherever two consecutive layers fall into
 * different intervals of one global partition, and neither the copy-arc steps nor Prop. 4's
 * argument use the partition beyond that, so a cut may sit between any two consecutive layers
 * of any BDD): every BDD with k > D layers becomes q = ceil(k / D) pieces, cut before layers
 * floor(t k / q), t = 1 .. q-1, so that no piece has more than D layers.  Returns the number of
 * pieces, or -1 on bad input. */
int orc_split_depth(void *vh, int D, double gamma) {
  oracle_t *h = (oracle_t *)vh;
  if (D < 1 || h->ncuts || !(gamma > 0.0 && gamma <= 1.0)) return -1;
  return split_core(h, NULL, D, gamma);
}

static int split_core(oracle_t *h, const int *interval, int D, double gamma) {
  /* pieces: count, then fill */
  int npieces = 0;
  long long npairs = 0;
  for (int b = 0; b < h->nb; ++b) {
    long long o0 = h->bdd_occ0[b];
    ++npieces;
    for (int l = 1; l < h->bdd_k[b]; ++l)
      if (cut_before(h, interval, D, o0, h->bdd_k[b], l)) {
        ++npieces;
        for (long long u = h->occ_node0[o0 + l - 1]; u < h->occ_node0[o0 + l]; ++u)
          npairs += (h->lo[u] >= 0) + (h->hi[u] >= 0);
      }
  }
  int *row = (int *)malloc((size_t)npieces * sizeof(int));
  int *kk = (int *)malloc((size_t)npieces * sizeof(int));
  long long *occ0 = (long long *)malloc((size_t)(npieces + 1) * sizeof(long long));
  h->cut_ptr = (long long *)malloc((size_t)(npieces + 1) * sizeof(long long));
  h->pair_u = (long long *)malloc((size_t)(npairs + 1) * sizeof(long long));
  h->pair_w = (long long *)malloc((size_t)(npairs + 1) * sizeof(long long));
  h->pair_occ = (long long *)malloc((size_t)(npairs + 1) * sizeof(long long));
  h->pair_hi = (int *)malloc((size_t)(npairs + 1) * sizeof(int));
  h->mu_bar = (double *)calloc((size_t)npairs + 1, sizeof(double));
  h->mu = (double *)calloc((size_t)npairs + 1, sizeof(double));
  h->dfwd = (double *)calloc((size_t)npairs + 1, sizeof(double));
  h->dbwd = (double *)calloc((size_t)npairs + 1, sizeof(double));
  h->root_f = (double *)calloc((size_t)h->N + 1, sizeof(double));
  if (!row || !kk || !occ0 || !h->cut_ptr || !h->pair_u || !h->pair_w || !h->pair_occ || !h->pair_hi ||
      !h->mu_bar || !h->mu || !h->dfwd || !h->dbwd || !h->root_f) {
    free(row); free(kk); free(occ0);
    return -1;
  }
  int p = 0, c = 0;
  long long k = 0;
  h->cut_ptr[0] = 0;
  for (int b = 0; b < h->nb; ++b) {
    long long o0 = h->bdd_occ0[b];
    int start = 0;
    for (int l = 1; l <= h->bdd_k[b]; ++l) {
      int boundary = l == h->bdd_k[b] || cut_before(h, interval, D, o0, h->bdd_k[b], l);
      if (!boundary) continue;
      row[p] = h->bdd_row[b];
      kk[p] = l - start;
      occ0[p] = o0 + start;
      ++p;
      if (l < h->bdd_k[b]) {  /* cut between layers l-1 and l: their arcs become copy pairs */
        long long ot = o0 + l - 1, nw = h->occ_node0[o0 + l];
        for (long long u = h->occ_node0[ot]; u < h->occ_node0[ot + 1]; ++u)
          for (int side = 0; side < 2; ++side) {
            int *t = side ? &h->hi[u] : &h->lo[u];
            if (*t < 0) continue;
            h->pair_u[k] = u;
            h->pair_w[k] = nw + *t;
            h->pair_occ[k] = ot;
            h->pair_hi[k] = side;
            *t = (int)(ORC_COPY0 - k);
            ++k;
          }
        h->cut_ptr[++c] = k;
      }
      start = l;
    }
  }
  occ0[p] = h->O;
  h->ncuts = c;
  h->npairs = npairs;
  h->gamma = gamma;
  free(h->bdd_row); free(h->bdd_k); free(h->bdd_occ0);
  h->bdd_row = row; h->bdd_k = kk; h->bdd_occ0 = occ0;
  h->nb = npieces;
  for (int b = 0; b < h->nb; ++b)
    for (int l = 0; l < h->bdd_k[b]; ++l) {
      h->occ_bdd[h->bdd_occ0[b] + l] = b;
      h->occ_layer[h->bdd_occ0[b] + l] = l;
    }
  orc_init_dual(h);
  return npieces;
}

/* Copy-arc duals: mu_bar and mu of every pair, cuts in order (pairs of a cut: tails in node
 * order, 0-arc before 1-arc). */
void orc_get_copy_duals(void *vh, double *mu_bar, double *mu) {
  oracle_t *h = (oracle_t *)vh;
  for (long long k = 0; k < h->npairs; ++k) { mu_bar[k] = h->mu_bar[k]; mu[k] = h->mu[k]; }
}

long long orc_npairs(void *vh) { return ((oracle_t *)vh)->npairs; }

/* Sets the copy-arc duals (and the root messages they imply), then recomputes the backward
 * messages. */
void orc_set_copy_duals(void *vh, const double *mu_bar, const double *mu) {
  oracle_t *h = (oracle_t *)vh;
  for (long long k = 0; k < h->npairs; ++k) { h->mu_bar[k] = mu_bar[k]; h->mu[k] = mu[k]; }
  for (long long k = 0; k < h->npairs; ++k) h->root_f[h->pair_w[k]] = INFINITY;
  for (long long k = 0; k < h->npairs; ++k)
    if (h->mu[k] < h->root_f[h->pair_w[k]]) h->root_f[h->pair_w[k]] = h->mu[k];
  for (int b = 0; b < h->nb; ++b) dp_backward(h, b, h->lam, h->bm);
}

/* lambda per coefficient; fold != 0 adds the share the next (forward) sweep would add: P_i/|J_i|,
 * or with SRMP P_i/|J_i^>| on J_i^> (all of J_i when J_i^> is empty), so that the returned
 * multipliers satisfy sum_j lambda^j_i = c_i. */
void orc_get_lambda(void *vh, int fold, double *out) {
  oracle_t *h = (oracle_t *)vh;
  if (fold) take_share(h, 1);
  for (long long t = 0; t < h->nnz; ++t) out[t] = 0.0;
  for (long long o = 0; o < h->O; ++o) out[h->occ_csr[o]] = h->lam[o] + (fold ? h->oshare[o] : 0.0);
}

void orc_get_pending(void *vh, double *P) {
  oracle_t *h = (oracle_t *)vh;
  for (int i = 0; i < h->n; ++i) P[i] = h->P[i];
}

/* Sets lambda (per CSR position) and P (NULL = 0), then recomputes backward messages. */
void orc_set_state(void *vh, const double *lam, const double *P) {
  oracle_t *h = (oracle_t *)vh;
  for (long long o = 0; o < h->O; ++o) h->lam[o] = lam[h->occ_csr[o]];
  for (int i = 0; i < h->n; ++i) h->P[i] = P ? P[i] : 0.0;
  for (int b = 0; b < h->nb; ++b) dp_backward(h, b, h->lam, h->bm);
}

/* Definitional min-marginals (full forward and backward programmes, then eq.
 * marginal-aggregation) for the current lambda, or lambda + the forward sweep's shares (as in
 * orc_get_lambda) when fold != 0. */
void orc_min_marginals(void *vh, int fold, double *m0, double *m1) {
  oracle_t *h = (oracle_t *)vh;
  double *lam = (double *)malloc((size_t)(h->O + 1) * sizeof(double));
  if (!lam) return;
  if (fold) take_share(h, 1);
  for (long long o = 0; o < h->O; ++o) lam[o] = h->lam[o] + (fold ? h->oshare[o] : 0.0);
  for (long long t = 0; t < h->nnz; ++t) { m0[t] = 0.0; m1[t] = 0.0; }
  for (int b = 0; b < h->nb; ++b) {
    dp_forward(h, b, lam, h->sfm);
    dp_backward(h, b, lam, h->sbm);
    for (int l = 0; l < h->bdd_k[b]; ++l) {
      long long o = h->bdd_occ0[b] + l;
      aggregate(h, o, lam[o], h->sfm, h->sbm, &m0[h->occ_csr[o]], &m1[h->occ_csr[o]]);
    }
  }
  free(lam);
}

/* Per-BDD energies E^j(lambda^j) (min over X_j) and solution counts |X_j| (Table 3's counting
 * algebra: count(v) = count(v0) + count(v1), count(top) = 1, count(bot) = 0). */
void orc_energies(void *vh, double *E) {
  oracle_t *h = (oracle_t *)vh;
  for (int b = 0; b < h->nb; ++b) E[b] = energy(h, b, h->lam);
}

void orc_counts(void *vh, double *counts) {
  oracle_t *h = (oracle_t *)vh;
  for (int b = 0; b < h->nb; ++b) {
    long long o0 = h->bdd_occ0[b];
    for (int l = h->bdd_k[b] - 1; l >= 0; --l) {
      long long o = o0 + l;
      for (long long u = h->occ_node0[o]; u < h->occ_node0[o + 1]; ++u) {
        double x = 0.0;
        int t0 = h->lo[u], t1 = h->hi[u];
        x += t0 == ORC_TOP ? 1.0 : (t0 == ORC_BOT ? 0.0 : h->sfm[h->occ_node0[o + 1] + t0]);
        x += t1 == ORC_TOP ? 1.0 : (t1 == ORC_BOT ? 0.0 : h->sfm[h->occ_node0[o + 1] + t1]);
        h->sfm[u] = x;
      }
    }
    counts[b] = h->sfm[h->occ_node0[o0]];
  }
}
