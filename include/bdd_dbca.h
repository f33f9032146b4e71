/*
 * bdd_dbca.h -- C ABI of the GB300 library for BDD-based dual block coordinate ascent on
 * 0-1 integer linear programs (Lange & Swoboda, "Efficient Message Passing for 0-1 ILPs with
 * Binary Decision Diagrams").
 *
 * Problem (Sec. 3, Def. 1 and Ex. 1):  min c.x  s.t.  a_j.x (<=, =, >=) b_j for every row j,
 * x in {0,1}^n.  Each row becomes one subproblem with index set I_j = { i : a_ji != 0 } and
 * one reduced, ordered BDD (Sec. 5.1, Def. 4).  The library maximises the Lagrangean dual
 * (Sec. 3.1, eq. D) over multipliers lambda^j_i, one per nonzero coefficient ("occurrence"),
 * by min-marginal averaging (Sec. 3.2, eq. mma-update) with BDD shortest-path messages
 * (Sec. 5.3, Alg. 2 and Alg. 3; Sec. 5.4 incremental form), parallel across BDDs with the
 * averaging share of each sweep applied in the next sweep, damped by omega.
 *
 * Conventions shared by every call:
 *   - Every call returns a status (BDD_OK or a negative BDD_E* code).  No call throws.
 *   - Inputs are copied; the caller keeps ownership of every array it passes.  Outputs go to
 *     caller-allocated arrays (host arrays unless the name ends in _device).
 *   - Per-coefficient arrays (lambda, mm0, mm1) are indexed by position in the caller's CSR
 *     arrays (col/val).  Positions whose coefficient is 0 are not occurrences (Ex. 1 drops
 *     them) and receive 0.
 *   - One solver handle must not be used from two host threads at once.
 *   - Device calls run on the solver's stream unless a stream is passed; results are
 *     stream-ordered.  Host-array calls synchronise before returning.  The calls of one
 *     solver are ordered among themselves even when they use different streams (each call
 *     waits on an event recorded at the end of the previous one).
 */
#ifndef BDD_DBCA_H
#define BDD_DBCA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdd_solver bdd_solver; /* opaque; created by bdd_build, released by bdd_free */

enum {
  BDD_OK = 0,
  BDD_EINVAL = -1,      /* malformed input: bad sizes / indices, duplicate (row, column), NaN/Inf cost, bad option */
  BDD_EINFEASIBLE = -2, /* a row has no 0-1 solution (see bdd_last_failed_row) */
  BDD_ETOOBIG = -3,     /* a BDD or the instance exceeds max_width / max_nodes or 32-bit indexing */
  BDD_ENOMEM = -4,      /* host allocation failed or max_device_bytes would be exceeded */
  BDD_ECUDA = -5,       /* a CUDA runtime call failed (no device, launch failure, ...) */
  BDD_ETIMEOUT = -6,    /* reserved: a bounded device-side wait gave up */
  BDD_EDEVICE = -7,     /* a device-side check failed */
  BDD_ESTATE = -8       /* the call needs device state but the solver was built host-only, or a
                           smoothed backward has no matching forward */
};

#define BDD_SIZES_LEN 19

/* Options for bdd_build.  Fill with bdd_default_options, then change fields. */
typedef struct {
  float omega;                /* damping of the min-marginal difference, in (0, 1]; default 0.5 */
  int max_width;              /* largest allowed BDD layer width; default 1 << 20 */
  long long max_nodes;        /* largest allowed total node count; default 2^31 - 1 */
  long long max_device_bytes; /* cap on device memory of the solver, 0 = no cap */
  int host_only;              /* 0: normal.  1: compile BDDs on the host only (no GPU needed);
                                 2: also build the device slab layout, kept in host memory.  With
                                 1 or 2 only bdd_sizes, bdd_export_canonical and bdd_free may be
                                 called (others return BDD_ESTATE); with 2 the export reads the
                                 slab layout back, as it does from the device */
  int device;                 /* CUDA device ordinal; -1 = the current device (default) */
  void *stream;               /* cudaStream_t for all device work; NULL = a stream the solver owns */
  int schedule;               /* 1 (default): per-phase kernels (two sweeps, two pending-sum passes
                                 per iteration) replayed from CUDA graphs with programmatic
                                 dependent launch; 0: one persistent cooperative kernel per call
                                 runs all iterations, four grid barriers per iteration.  Both run
                                 the same arithmetic; 0 falls back to 1 on devices without
                                 cooperative launch. */
  long long spin_limit;       /* polls before a grid-barrier wait gives up (then the call's host
                                 form returns BDD_ETIMEOUT); default 1 << 26 */
  float alpha;                /* smoothing temperature (Appendix A.5): 0 (default) = min-sum;
                                 alpha > 0 replaces every minimum of the iteration and of the
                                 bound by the soft minimum -alpha log sum exp(-x / alpha), so
                                 the bound is E^j_alpha-based and differentiable.  Smoothed
                                 solvers need every BDD layer to be at most 32 nodes wide
                                 (else BDD_ETOOBIG) and run schedule 1. */
  const int *var_rank;        /* variable order (Appendix A.3): NULL (default) = index order;
                                 else a host array of n entries, a permutation of 0..n-1, where
                                 var_rank[i] is the place of variable i.  Every BDD takes its
                                 row's variables in ascending rank; all inputs and outputs stay
                                 in CSR / variable index order.  Read by bdd_build only (the
                                 caller keeps ownership); not a permutation -> BDD_EINVAL.
                                 bdd_cuthill_mckee computes the paper's choice of order. */
  int averaging;              /* 0 (default): eq. (mma-update), the pending sum P_i is shared
                                 evenly over all of J_i.  1: SRMP averaging (Appendix A.4,
                                 eq. srmp-update): a forward sweep shares P_i evenly over
                                 J_i^> (subproblems of i with a variable after i in the order,
                                 i.e. i is not the last layer of the BDD), a backward sweep over
                                 J_i^< (i not the first layer); an empty set falls back to all of
                                 J_i.  Under the deferred schedule the set of a sweep applies
                                 to the shares that sweep adds.  Folded outputs (multipliers and
                                 min-marginals) add the forward-sweep shares. */
  int fused_pending;          /* schedule 1 only.  1: the pending sums are formed inside the
                                 sweeps (each variable's last visit in a sweep sums its slots and
                                 writes the next sweep's shares; a forward sweep also reduces
                                 the previous iteration's bound), two kernels per iteration.
                                 0: separate pending-sum kernels, four per iteration.  -1
                                 (default): 0, the faster plan on every workload measured.
                                 Same arithmetic either way: multipliers and pending sums are
                                 bit-identical; bounds differ only in the FP64 summation
                                 order. */
  int staging;                /* warp-tile window staging of the update sweeps.  0: bulk-copy
                                 (TMA) ring, 4-layer windows, the next window loading while one
                                 is processed; 1: 8-layer windows, each loaded by cp.async in one
                                 round and then processed; 2: the same with two buffers per warp,
                                 the next window loading while one is processed (twice the shared
                                 memory of 1).  -1 (default): the autotuner times all three at
                                 build (schedule 1: a warm-up and six iterations each, kernel by
                                 kernel, the fastest launch of each sweep counted) and keeps the
                                 fastest per sweep direction (a higher-numbered variant must be
                                 at least 5 % faster than a lower one).  The variants compute identical
                                 values; the persistent schedule and other sweeps use 0. */
  int split_intervals;        /* sub-BDDs (Sec. 6, Def. of sub-BDDs and copy-arcs; the parallel
                                 min-marginal averaging algorithm).  0 or 1 (default): no split.
                                 k >= 2: the variable order is cut into at most k intervals
                                 holding similar node counts (a node counts for its layer's
                                 variable; the first place whose preceding places hold at least
                                 t N / k nodes starts interval t + 1).  Every BDD is cut between
                                 consecutive layers whose variables lie in different intervals;
                                 each piece is a subproblem of its own (several roots when it
                                 starts below the BDD's root), the arcs crossing a cut become
                                 copy-arc pairs: the earlier piece's copy arc into top with
                                 cost theta + mu_bar, the later piece's entry arc with cost mu
                                 (the arc's theta stays with the copy arc).  After every forward
                                 sweep each cut moves mu_bar by -gamma d_fwd + gamma d_bwd, after
                                 every backward sweep mu by -gamma d_bwd + gamma d_fwd (d: an
                                 arc-marginal minus its minimum over the cut).  Min-marginals
                                 and energies then refer to the pieces.  Split solvers run
                                 schedule 1 without fused pending sums, need alpha = 0
                                 (else BDD_EINVAL) and refuse bdd_bound_parts. */
  const int *cuts;            /* explicit cut places instead (n_cuts entries, ascending, in
                                 [1, n); variable i lies in interval #{t : cuts[t] <= place of
                                 i}); overrides split_intervals; bad cuts -> BDD_EINVAL.  Read
                                 by bdd_build only. */
  int n_cuts;                 /* entries of cuts; default 0 */
  float gamma;                /* copy-arc step size in (0, 1]; default 0.5 (the paper's choice
                                 in its experiments, Sec. 7) */
  int split_depth;            /* depth split instead of intervals: 0 (default) off; D >= 1 cuts
                                 every BDD of k > D layers into q = ceil(k / D) pieces, before
                                 layers floor(t k / q), t = 1 .. q-1, with the same copy arcs and
                                 steps.  This bounds the longest chain of dependent layers a
                                 sweep walks, which a partition of the variable order does not
                                 (a BDD over consecutive variables stays whole unless a cut falls
                                 inside it).  Overrides split_intervals and cuts. */
  int lanes;                  /* BDDs whose layers have at most two nodes: 1 = lane tiles (one
                                 lane per BDD holds both nodes of a layer, 32 BDDs per warp, no
                                 shuffles or team reductions); 0 = two-lane teams (16 BDDs per
                                 warp).  Same values bit for bit.  Lane tiles need a plain
                                 solver (alpha = 0, no split, separate pending kernels, schedule
                                 1), else BDD_EINVAL.  -1 (default): the layout tuner decides
                                 per key on plain solvers (see tune_layout); lane tiles on plain
                                 solvers when the tuner is off; teams otherwise. */
  int tune_layout;            /* layout tuner (plain solvers only, else BDD_EINVAL for 1): a BDD's
                                 key is its natural width class c (the smallest team of 2^c lanes
                                 >= its widest layer, c <= 5; 6 = wider than 32, block tiles) and
                                 its depth bucket (<= 8, <= 32, <= 128, longer), key = 4 c +
                                 bucket.  For every key holding at least 1 % of the nodes (and
                                 4096) the tuner times two tile classes on a probe of that key's
                                 BDDs (all of them, or every k-th one above 16 Mi nodes) in a
                                 throwaway device solver -- for widths <= 2 two-lane teams against
                                 lane tiles, for c = 2..5 teams of 2^c against 2^(c+1) lanes (a
                                 block tile after 32) -- and keeps the alternative only when it
                                 is at least 5 % faster (fastest forward plus fastest backward
                                 sweep of three timed iterations).  -1 (default) / 1: on, 0: off.
                                 bdd_layout_table reports the choice. */
  const int *layout_classes;  /* explicit table instead of the tuner (plain solvers only):
                                 kLayoutKeys = 28 entries, -1 = default, 0..5 a team of 2^c lanes,
                                 6 a block tile, 7 lane tiles (widths <= 2 only); a class too
                                 narrow for its key -> BDD_EINVAL.  Read by bdd_build only. */
  int smooth_messages;        /* smoothed solvers: whether bdd_smooth_forward keeps the messages
                                 every sweep wrote (and the initial backward messages), (2 K + 1)
                                 N floats, so that bdd_smooth_backward reads each sweep's
                                 starting messages instead of recomputing them with one
                                 messages-only sweep per reversed sweep.  1: keep them
                                 (BDD_ENOMEM if they cannot be allocated); 0: recompute; -1
                                 (default): keep them when they fit in a quarter of the free
                                 device memory and in max_device_bytes, else recompute.  The
                                 gradient is the same either way (the recomputation repeats
                                 the forward's arithmetic). */
} bdd_options;

#define BDD_LAYOUT_KEYS 28

void bdd_default_options(bdd_options *opt);

/* Compiles one BDD per row and, unless host_only, uploads the layer-major slabs to the GPU and
 * initialises lambda^j_i = c_i / |J_i| (Alg. 1 initialisation) followed by one backward pass
 * (Prop. 3 precondition).
 *   n, m:     number of variables and rows
 *   row_ptr:  int64[m+1] CSR row pointers; col: int32[nnz] in [0, n); val: int32[nnz]
 *   b:        int32[m] right-hand sides; sense: int8[m], -1 (<=), 0 (=), +1 (>=)
 *   c:        float32[n] objective (finite)
 *   opt:      NULL = defaults
 *   out:      receives the solver, or NULL on error
 * Rows with no nonzero are dropped when 0 (sense) b holds and are infeasible otherwise. */
int bdd_build(int n, int m, const long long *row_ptr, const int *col, const int *val,
              const int *b, const signed char *sense, const float *c, const bdd_options *opt,
              bdd_solver **out);

/* Row id that made the last failing bdd_build of this host thread fail (-1 if none). */
int bdd_last_failed_row(void);

/* Runs n_iter iterations (forward sweep, then backward sweep; Alg. 1's forward and backward
 * pass) and copies results to host arrays:
 *   lower_bound: double[1], the y-slack bound after the last iteration (Appendix A.1 dual
 *                derivation; equals eq. D's objective once the pending share is folded)
 *   lambda:      float[nnz] or NULL; multipliers with the pending share folded in, so that
 *                sum_j lambda^j_i = c_i up to rounding
 *   mm0, mm1:    float[nnz] or NULL; min-marginals (Sec. 3.2 eq. min-marginals) at those
 *                multipliers, from a full forward and backward pass
 * n_iter = 0 only evaluates the outputs.  Solver state (multipliers, pending sums) after
 * the call is the same whether outputs are requested or not.  Returns BDD_ETIMEOUT if a
 * grid-barrier wait of this or an earlier device call gave up (see spin_limit). */
int bdd_iterate(bdd_solver *h, int n_iter, double *lower_bound, float *lambda, float *mm0,
                float *mm1);

/* Device form of bdd_iterate: all pointers are device pointers, each may be NULL.
 *   d_bound_trace: double[n_iter], bound after every iteration
 *   d_lambda, d_mm0, d_mm1: float[nnz] as in bdd_iterate
 *   stream: cudaStream_t to order the work on (NULL = the solver's stream)
 * Returns after enqueueing; nothing is synchronised. */
int bdd_iterate_device(bdd_solver *h, int n_iter, double *d_bound_trace, float *d_lambda,
                       float *d_mm0, float *d_mm1, void *stream);

/* Same iterations as bdd_iterate_device, run as per-phase kernels launched one by one with CUDA
 * events between them, for measurement.  kernel_ms[4] receives the summed device time of the
 * forward sweeps, the pending-sum passes after them, the backward sweeps, and the pending-sum
 * passes with the FP64 bound after them; synchronises before returning.  kernel_ms: host
 * double[4]. */
int bdd_iterate_profiled(bdd_solver *h, int n_iter, double *kernel_ms);

/* Lower bounds of independent sub-instances packed block-diagonally into one solver (rows
 * [row_off[k], row_off[k+1]) and variables [var_off[k], var_off[k+1]) form part k, with no row
 * touching another part's variables).  The y-slack bound of the dual derivation (Appendix A.1)
 * splits over such parts: out[k] = sum of E^j over part k's rows + sum of min(0, P_i) over part
 * k's variables (min(0, c_i) for variables in no row), in FP64, in a fixed order.
 *   nparts >= 1; row_off: int64[nparts+1], var_off: int64[nparts+1] (host, ascending, from 0 to
 *   m and n); out: host double[nparts].  Synchronises. */
int bdd_bound_parts(bdd_solver *h, int nparts, const long long *row_off, const long long *var_off, double *out);

/* Smoothed bound as a differentiable function of the costs (Appendix A.5; needs alpha > 0).
 * bdd_smooth_forward sets c (device float[n]), restarts (lambda = c/|J_i|), runs K iterations
 * and writes the smoothed bound after them (the y-slack form with every minimum soft) to
 * d_bound (device double[1]); it keeps a checkpoint of the multipliers and shares of every sweep
 * (2 K O floats of device memory), and of the messages every sweep wrote unless
 * bdd_options.smooth_messages says otherwise ((2 K + 1) N floats), and stores the forward's
 * generation number in *generation (host; NULL skips it).  bdd_smooth_backward then writes
 * d_grad_c (device float[n]) = g * d bound / d c, g read from d_gbound (device double[1]), by
 * reverse-mode passes over the K iterations (hand-written adjoint kernels) that take each
 * sweep's messages from those checkpoints, or recompute them from the multipliers' checkpoint
 * when the messages were not kept.  `generation` names the forward whose gradient is wanted: it must be the value that
 * forward returned, it must be the solver's last forward, and no state-changing call may come
 * in between; otherwise BDD_ESTATE (so two forwards on one solver feeding one loss cannot take
 * the second one's checkpoints for the first one's gradient).  Both enqueue on `stream` (NULL =
 * the solver's stream) and return. */
int bdd_smooth_forward(bdd_solver *h, int K, const float *d_c, double *d_bound, long long *generation,
                       void *stream);
int bdd_smooth_backward(bdd_solver *h, long long generation, const double *d_gbound, float *d_grad_c,
                        void *stream);

/* Replaces c and restarts: lambda = c/|J_i|, pending sums 0, one backward pass.  c: float[n],
 * host. */
int bdd_set_costs(bdd_solver *h, const float *c);

/* Sizes: out[0] n, [1] m, [2] BDDs (pieces of a split solver), [3] occurrences (nonzeros
 * kept), [4] nodes, [5] max depth, [6] max width, [7] nnz, [8] device bytes held, [9] warp
 * tiles, [10] block tiles, [11] schedule in use (0 persistent, 1 per-phase graphs), [12]
 * warp-tile staging the autotuner chose for the update sweeps: bits 0-1 forward, bits 2-3 backward
 * (0 bulk-copy ring of 4-layer windows, 1 8-layer cp.async windows, 2 the same
 * double-buffered), [13] cuts of the variable order, [14] copy-arc pairs, [15] depth limit of a
 * depth split (0: none), [16] 1 if BDDs of width <= 2 run as lane tiles (bdd_options.lanes),
 * [17] occurrences and [18] nodes of the lane tiles (their sweeps read one byte of arcs per
 * occurrence instead of a node offset per occurrence and a successor pair per node). */
int bdd_sizes(const bdd_solver *h, long long out[BDD_SIZES_LEN]);

/* Status a device error word maps to (no counterpart in the paper): 0 -> BDD_OK; -7 (an index
 * check of the checked build failed) -> BDD_EDEVICE; any other value (a bounded device-side wait
 * gave up) -> BDD_ETIMEOUT.  Host only; the calls that read the word use this mapping. */
int bdd_status_of_device_word(int word);

/* Tile class of every layout key (see bdd_options.tune_layout), no counterpart in the paper:
 * nodes[k] nodes of the solver's BDDs with key k, cls[k] the class they run in (-1 none, 0..5
 * a team of 2^c lanes, 6 block tiles, 7 lane tiles), ms (NULL skips it) [2k], [2k + 1]: the
 * tuner's probe time of the default and the alternative class (-1: not probed).  Arrays of
 * BDD_LAYOUT_KEYS (2 BDD_LAYOUT_KEYS for ms), host. */
int bdd_layout_table(const bdd_solver *h, long long *nodes, int *cls, float *ms);

/* Canonical form of the BDDs, read back from the device slabs (or the host copy when built
 * host_only): BDDs in ascending row order; occurrences BDD-major, layer-minor; nodes
 * BDD-major, layer-major and, inside a layer, in ascending order of the smallest partial
 * coefficient sum that reaches them.  lo/hi are node ids inside the next layer of the same
 * BDD, or -1 (top) / -2 (bot).  Array sizes: bdd_row, bdd_depth [BDDs]; occ_var, occ_csr,
 * occ_width [occurrences]; lo, hi [nodes].  occ_csr is the CSR position of the coefficient. */
int bdd_export_canonical(const bdd_solver *h, int *bdd_row, int *bdd_depth, int *occ_var,
                         long long *occ_csr, int *occ_width, int *lo, int *hi);

/* Cut places of a split solver (Sec. 6): cuts: host int32[out[13] of bdd_sizes]. */
int bdd_get_cuts(const bdd_solver *h, int *cuts);

/* Copy-arc duals of a split solver (Sec. 6, Def. of copy-arc costs): mu_bar (the copy arc's
 * dual, earlier piece) and mu (the entry arc's dual, later piece), host float[pairs] each
 * (out[14] of bdd_sizes; NULL skips one in the get form).  Pairs are in canonical order: the
 * cuts of BDD 0 (ascending row) by ascending layer, then BDD 1, ...; inside a cut, the tails
 * in canonical node order, the 0-arc before the 1-arc.  The bound is valid while every
 * mu + mu_bar <= 0.  From the all-zero duals of bdd_build / bdd_set_costs the iteration keeps
 * that: after a forward step each pair's sum is -gamma d_fwd, after a backward step -gamma d_bwd.
 * bdd_set_copy_duals also recomputes the root messages (min of mu over a head's entry arcs) and
 * the backward messages; it leaves the last deltas of the dual steps as they are, so duals set
 * by hand need not keep the sums nonpositive.  Both synchronise. */
int bdd_get_copy_duals(const bdd_solver *h, float *mu_bar, float *mu);
int bdd_set_copy_duals(bdd_solver *h, const float *mu_bar, const float *mu);

/* Dual state: lambda without the pending share (float[nnz], CSR positions) and the pending
 * sums P_i (float[n]).  bdd_set_state also recomputes the backward messages. */
int bdd_get_state(const bdd_solver *h, float *lambda, float *pending);
int bdd_set_state(bdd_solver *h, const float *lambda, const float *pending);

/* Lower bound sum_j E_j + sum_{i: deg_i > 0} min(0, P_i) + empty_const in FP64, from caller
 * device arrays, without allocating anything.  The paper has no counterpart: it is the bound
 * reduction of bdd_iterate offered on its own for callers that cannot allocate device memory
 * (code that runs inside someone else's memory pool or arena, or inside a framework that
 * forbids cudaMalloc on its hot path), who still own their inputs and output.
 *   n, nb:  variables and BDDs; max(n, nb) <= 4,194,304, else BDD_ETOOBIG (the scratch limit)
 *   d_E:    float[nb] per-BDD energies E_j; d_P: float[n] pending sums; d_deg: int32[n] |J_i|
 *   empty_const: sum of min(0, c_i) over variables in no row
 *   d_bound: double[1] output; stream: cudaStream_t (NULL = legacy default stream)
 * Scratch: a static device array of 1025 doubles (8.2 KB) that every GPU loading this library
 * holds until the process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress), so make the first call on each device before any stream
 * capture.  All calls share the array: calls that overlap on the GPU (e.g. on two streams at
 * once) race and must be serialised by the caller.  Returns after enqueueing. */
int bdd_lower_bound_noalloc(int n, int nb, const float *d_E, const float *d_P, const int *d_deg,
                            double empty_const, double *d_bound, void *stream);

/* Variable order by bandwidth reduction (Appendix A.3): the Cuthill-McKee order of the
 * bipartite variable-constraint graph (one node per variable and per row, an edge per nonzero
 * coefficient), restricted to the variables.  Host only, no GPU needed.
 *   n, m, row_ptr, col, val: the constraint matrix in CSR form, as for bdd_build (val may be
 *     NULL: every stored entry is an edge; else entries with val == 0 are skipped)
 *   rank: int32[n] output, a permutation of 0..n-1; rank[i] is the place of variable i, ready
 *     for bdd_options.var_rank.
 * Each connected component starts at a pseudo-peripheral node of least degree (repeated
 * breadth-first search), then a breadth-first search that enqueues each node's unvisited
 * neighbours in ascending degree (ties: ascending index); components follow in the order of
 * their lowest-index variable; variables in no row come last, in index order.  Deterministic.
 * Returns BDD_OK, BDD_EINVAL (bad sizes, pointers or column index) or BDD_ENOMEM. */
int bdd_cuthill_mckee(int n, int m, const long long *row_ptr, const int *col, const int *val,
                      int *rank);

/* Text for a status code (static storage). */
const char *bdd_strerror(int code);

/* Releases the solver and its device memory; NULL is ignored. */
void bdd_free(bdd_solver *h);

#ifdef __cplusplus
}
#endif

#endif /* BDD_DBCA_H */
