// C ABI of the library (include/bdd_dbca.h): solver object, device slabs, the captured
// iteration loop, outputs and state access.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "bdd_dbca.h"
#include "internal.h"

using namespace bdd;

namespace {

thread_local int g_failed_row = -1;

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) {                   \
      cudaGetLastError();                       \
      return BDD_ECUDA;                         \
    }                                           \
  } while (0)

#define RC(x)                                   \
  do {                                          \
    int rc_ = (x);                              \
    if (rc_ != 0) return rc_;                   \
  } while (0)

constexpr int kGraphIters = 8;  // iterations per captured graph
constexpr float kTuneMargin = 0.05f;  // autotuner: required gain of a later staging variant

}  // namespace

struct bdd_solver {
  // sizes
  int n = 0, m = 0;
  long long nnz = 0, nb = 0, O = 0, N = 0;
  int max_depth = 0, max_width = 0;
  bool host_only = false;
  HostBDDs host;                 // kept only for host_only solvers
  bool host_layout = false;      // host_only == 2: the slab layout is kept in host memory
  Layout layout;
  // host metadata of the device layout
  hvec<int> bdd_perm;     // sorted position -> canonical BDD index
  hvec<int> canon_row;    // canonical BDD index -> row
  hvec<int> tile_occ0, tile_bdd0, tile_nbdd;
  int class_tile_off[kWarpClasses + 2] = {0};
  int n_warp_tiles = 0, n_block_tiles = 0, block_buf = 0;
  std::vector<int> var_deg;
  std::vector<float> c;
  double empty_const = 0.0;
  // device
  int device = -1;
  float omega = 0.5f;
  float alpha = 0.f;  // smoothing temperature (0: min-sum)
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  bool own_stream = false;
  long long max_device_bytes = 0, device_bytes = 0;
  std::vector<void *> allocs;
  int *d_occ_node_off = nullptr, *d_occ_var = nullptr;
  long long *d_occ_csr = nullptr;
  int2 *d_lohi = nullptr;
  unsigned char *d_lane_code = nullptr;  // lane tiles: arcs of a layer in one byte per occurrence
  long long lane_O = 0, lane_N = 0;      // occurrences and nodes of the lane tiles
  float *d_fm = nullptr, *d_bm = nullptr, *d_lam = nullptr, *d_delta = nullptr;
  float *d_P = nullptr, *d_c = nullptr, *d_share_occ = nullptr;
  int *d_occ_slot = nullptr;
  int *d_bdd_depth = nullptr;
  int *d_bdd_row = nullptr;        // row of each BDD in sorted order
  float *d_E_row = nullptr;        // scratch for per-part bounds (lazily allocated)
  long long *d_part_off = nullptr; // scratch: row and variable offsets of the parts
  double *d_part_out = nullptr;
  int part_cap = 0;
  float *d_bdd_E = nullptr;
  int *d_tile_occ0 = nullptr, *d_tile_bdd0 = nullptr, *d_tile_nbdd = nullptr;
  int *d_tile_win0 = nullptr;
  int2 *d_win_node = nullptr;
  int *d_var_ptr = nullptr, *d_var_occ = nullptr;
  int averaging = 0;                     // 0: eq. mma-update; 1: SRMP (Appendix A.4)
  bool lanes2 = false;                   // BDDs of width <= 2 may run as lane tiles
  // layout tuner: tile class of every key (-1: default), nodes per key, probe ms of the default
  // and the alternative candidate (-1: not probed)
  int key_class[kLayoutKeys];
  long long key_nodes[kLayoutKeys];
  float key_ms[kLayoutKeys][2];
  int stage_fwd = 0, stage_bwd = 0;      // warp-tile staging of the update sweeps (autotuned)
  int staging_opt = -1;                  // bdd_options.staging
  float tune_ms[kStagings][2] = {};      // measured ms per sweep [variant][direction]
  bool fused = false;                    // per-phase plan: pending pass fused into the sweeps
  int fused_opt = -1;                    // bdd_options.fused_pending
  int *d_cnt = nullptr;                  // [n] fused plan: visits still to come per variable
  double *d_slk = nullptr;               // [n] fused plan: slack terms of the last backward sweep
  double *d_fpartial = nullptr;          // fused plan: per-block bound partials
  unsigned *d_fticket = nullptr;
  unsigned char *d_slot_dir = nullptr;   // SRMP membership bits per slot (averaging == 1)
  int4 *d_heavy = nullptr;               // variables with more than heavy_deg occurrences: {i, s, e, 0}
  int n_heavy = 0, heavy_deg = 8;
  // persistent schedule
  int schedule = 1;
  long long spin_limit = 1LL << 26;
  int grid_persist = 0;
  double *d_part = nullptr;
  unsigned *d_barrier = nullptr;
  int *d_error = nullptr;
  int block_depth_buf = 0;
  double *d_partial = nullptr, *d_trace = nullptr;
  unsigned *d_ticket = nullptr;
  int *d_iter = nullptr;
  int trace_cap = 0;
  float *d_out_lam = nullptr, *d_out_m0 = nullptr, *d_out_m1 = nullptr;
  int grid_sweep = 0, n_warp_blocks = 0, grid_reduce = 1;
  int lane_run = 1, n_lane_warps = 0;  // lane tiles per warp; warps that take lane tiles
  bool pdl_early = true;               // kernels let their successors launch when they start
  size_t smem = 0, smem_persist = 0;
  cudaGraphExec_t g_many = nullptr, g_one = nullptr;
  // smoothed bound and its gradient: per-sweep checkpoints and scratch (allocated on first use)
  int smooth_cap = 0;           // sweeps the checkpoint buffers hold
  int smooth_K = 0;             // iterations of the recorded forward (0: none)
  long long state_gen = 0;      // bumped by every call that changes the dual state
  long long smooth_gen = -1;    // state_gen right after the recorded forward
  float *ck_lam = nullptr, *ck_shr = nullptr;
  int smooth_messages = -1;     // bdd_options.smooth_messages
  float *ck_msg = nullptr;      // messages before the first sweep and after every sweep
  int msg_cap = 0;              // message checkpoints ck_msg holds
  bool smooth_msgs = false;     // the recorded forward kept its messages in ck_msg
  float *t_nodeA = nullptr, *t_nodeB = nullptr, *t_gnode = nullptr;
  float *t_glam0 = nullptr, *t_glam1 = nullptr, *t_gshr = nullptr, *t_gdelta = nullptr;
  float *t_delta = nullptr, *t_E = nullptr;
  // sub-BDDs (Sec. 6): cuts of the variable order, copy-arc pairs and their duals
  std::vector<int> cuts;
  long long npairs = 0, ngroups = 0;
  float gamma = 0.5f;
  int split_depth = 0;
  int4 *d_cut_grp = nullptr, *d_pair = nullptr;
  int *d_head_node = nullptr, *d_head_ptr = nullptr, *d_head_pair = nullptr;
  float *d_mu_bar = nullptr, *d_mu = nullptr, *d_dfwd = nullptr, *d_dbwd = nullptr;
  cudaEvent_t ev_last = nullptr;  // end of the solver's last enqueued work, on whatever stream

  bdd_solver() {
    for (int k = 0; k < kLayoutKeys; ++k) {
      key_class[k] = -1;
      key_nodes[k] = 0;
      key_ms[k][0] = key_ms[k][1] = -1.f;
    }
  }

  ~bdd_solver() {
    if (ev_last) cudaEventDestroy(ev_last);
    if (g_many) cudaGraphExecDestroy(g_many);
    if (g_one) cudaGraphExecDestroy(g_one);
    for (void *p : allocs) cudaFree(p);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  template <class Tp>
  int alloc(Tp **p, long long count) {
    // 16 spare bytes: bulk copies into shared memory read whole 16-byte blocks, up to 15 bytes
    // past an array's last element
    size_t bytes = (size_t)std::max<long long>(count, 1) * sizeof(Tp) + 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (max_device_bytes > 0 && device_bytes + (long long)bytes > max_device_bytes) return BDD_ENOMEM;
    void *q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      cudaGetLastError();
      return BDD_ENOMEM;
    }
    allocs.push_back(q);
    device_bytes += (long long)bytes;
    *p = (Tp *)q;
    return BDD_OK;
  }

  SweepParams sweep_params(float *out_m0 = nullptr, float *out_m1 = nullptr) const {
    SweepParams p{};  // value-initialised: no fused pass unless fused_params() sets one
    p.occ_node_off = d_occ_node_off;
    p.occ_csr = d_occ_csr;
    p.lohi = d_lohi;
    p.lane_code = d_lane_code;
    p.fm = d_fm;
    p.bm = d_bm;
    p.lam = d_lam;
    p.occ_slot = d_occ_slot;
    p.delta = d_delta;
    p.share_occ = d_share_occ;
    p.bdd_depth = d_bdd_depth;
    p.bdd_E = d_bdd_E;
    p.tile_occ0 = d_tile_occ0;
    p.tile_win0 = d_tile_win0;
    p.win_node = d_win_node;
    p.tile_bdd0 = d_tile_bdd0;
    p.tile_nbdd = d_tile_nbdd;
    p.out_m0 = out_m0;
    p.out_m1 = out_m1;
    for (int c = 0; c < kWarpClasses + 2; ++c) p.class_tile_off[c] = class_tile_off[c];
    p.n_warp_blocks = n_warp_blocks;
    p.lanes2 = lanes2 ? 1 : 0;
    p.lane_run = lane_run;
    p.pdl_early = pdl_early ? 1 : 0;
    p.n_lane_warps = n_lane_warps;
    p.block_buf = block_buf;
    p.block_depth_buf = block_depth_buf;
    p.omega = omega;
    p.alpha = alpha;
    p.error = d_error;
    p.n_nodes = N;
    p.n_occ = O;
    p.n_csr = nnz;
    p.n_bdd = nb;
    p.inv_alpha = alpha > 0.f ? 1.f / alpha : 0.f;
    p.copy_val = d_mu_bar;
    p.split = npairs > 0 ? 1 : 0;
    return p;
  }

  CutParams cut_params() const {
    CutParams c{};
    c.grp = d_cut_grp;
    c.pair = d_pair;
    c.head_node = d_head_node;
    c.head_ptr = d_head_ptr;
    c.head_pair = d_head_pair;
    c.mu_bar = d_mu_bar;
    c.mu = d_mu;
    c.dfwd = d_dfwd;
    c.dbwd = d_dbwd;
    c.fm = d_fm;
    c.bm = d_bm;
    c.lam = d_lam;
    c.gamma = gamma;
    c.ngroups = npairs > 0 ? (int)ngroups : 0;
    return c;
  }

  // copy-arc dual step after a sweep (split solvers; nothing otherwise)
  int cut(bool fwd, cudaStream_t s) {
    if (npairs == 0) return BDD_OK;
    return cut_launch(fwd, cut_params(), s) ? BDD_ECUDA : BDD_OK;
  }

  // parameters of the fused plan's update sweeps (bound: reduce the previous iteration's bound at
  // the start of a forward sweep)
  SweepParams fused_params(bool bound) const {
    SweepParams p = sweep_params();
    FusedParams &z = p.fz;
    z.cnt = d_cnt;
    z.occ_var = d_occ_var;
    z.var_ptr = d_var_ptr;
    z.var_occ = d_var_occ;
    z.P = d_P;
    z.share = d_share_occ;
    z.slot_dir = d_slot_dir;
    z.slk = d_slk;
    z.bound = bound ? 1 : 0;
    z.partial = d_fpartial;
    z.ticket = d_fticket;
    z.iter_ctr = d_iter;
    z.trace = d_trace;
    z.trace_cap = trace_cap;
    z.n = n;
    z.nb = (int)nb;
    z.empty_const = empty_const;
    return p;
  }

  PendingParams pending_params(int next_dir) const {
    PendingParams r{};
    r.pdl_early = pdl_early ? 1 : 0;
    r.slot_dir = d_slot_dir;
    r.next_dir = next_dir;
    r.heavy = d_heavy;
    r.n_heavy = n_heavy;
    r.heavy_deg = heavy_deg;
    r.var_ptr = d_var_ptr;
    r.var_occ = d_var_occ;
    r.delta = d_delta;
    r.P = d_P;
    r.share_occ = d_share_occ;
    r.bdd_E = d_bdd_E;
    r.partial = d_partial;
    r.ticket = d_ticket;
    r.iter_ctr = d_iter;
    r.trace = d_trace;
    r.trace_cap = trace_cap;
    r.n = n;
    r.nb = (int)nb;
    r.empty_const = empty_const;
    r.alpha = alpha;
    return r;
  }

  // Work of one solver may be enqueued on several streams (its own, or one passed per call);
  // each call first waits for the previous call's work and then marks its own end.
  int begin(cudaStream_t s) {
    CK(cudaStreamWaitEvent(s, ev_last, 0));
    return BDD_OK;
  }
  int end(cudaStream_t s) {
    CK(cudaEventRecord(ev_last, s));
    return BDD_OK;
  }

  // finish_prev: a forward update sweep that also finishes the previous iteration's deferred bound
  int sweep(bool fwd, int mode, cudaStream_t s, float *m0 = nullptr, float *m1 = nullptr, bool finish_prev = false) {
    const int staging = mode == kUpdate ? (fwd ? stage_fwd : stage_bwd) : 0;
    SweepParams p = sweep_params(m0, m1);
    if (finish_prev) {
      p.fin_partial = d_partial;
      p.fin_nblocks = grid_reduce;
      p.fin_iter = d_iter;
      p.fin_trace = d_trace;
      p.fin_cap = trace_cap;
      p.fin_const = empty_const;
    }
    return sweep_launch(fwd, mode, p, grid_sweep, s, staging) ? BDD_ECUDA : BDD_OK;
  }

  // Autotuner: time each warp-tile staging variant of the update sweeps on this instance
  // (after a warm-up iteration, `reps` iterations launched kernel by kernel between events,
  // the fastest of each sweep kept, which is robust to a stray slow launch) and keep the faster
  // variant per direction.  Both variants compute the same values, so the
  // choice affects time only; the solver is restarted afterwards.
  int autotune(cudaStream_t s, int reps) {
    if (n_warp_tiles == 0 || reps < 1) return BDD_OK;
    // lane tiles stream their windows through the bulk-copy ring whatever the staging variant:
    // when they are all the warp tiles, every variant runs the same code and there is nothing
    // to time
    if (lanes2 && class_tile_off[1] == class_tile_off[kWarpClasses]) return BDD_OK;
    // events around each sweep of every iteration, read after one synchronisation per variant
    std::vector<cudaEvent_t> ev(4 * (reps + 1), nullptr);
    int rc = BDD_OK;
    for (auto &e : ev)
      if (rc == BDD_OK && cudaEventCreate(&e) != cudaSuccess) rc = BDD_ECUDA;
    float ms[kStagings][2] = {};  // [variant][direction]: fastest launch
    for (int v = 0; v < kStagings && rc == BDD_OK; ++v) {
      stage_fwd = stage_bwd = v;
      rc = restart(s);
      for (int it = 0; it <= reps && rc == BDD_OK; ++it) {
        cudaEvent_t *e = &ev[4 * it];
        if (cudaEventRecord(e[0], s) != cudaSuccess) rc = BDD_ECUDA;
        if (rc == BDD_OK) rc = sweep(true, kUpdate, s);
        if (rc == BDD_OK && cudaEventRecord(e[1], s) != cudaSuccess) rc = BDD_ECUDA;
        if (rc == BDD_OK) rc = pending(false, s);
        if (rc == BDD_OK && cudaEventRecord(e[2], s) != cudaSuccess) rc = BDD_ECUDA;
        if (rc == BDD_OK) rc = sweep(false, kUpdate, s);
        if (rc == BDD_OK && cudaEventRecord(e[3], s) != cudaSuccess) rc = BDD_ECUDA;
        if (rc == BDD_OK) rc = pending(true, s);
      }
      if (rc == BDD_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = BDD_ECUDA;
      for (int it = 1; it <= reps && rc == BDD_OK; ++it) {  // iteration 0 warms up
        const cudaEvent_t *e = &ev[4 * it];
        float t0 = 0.f, t1 = 0.f;
        if (cudaEventElapsedTime(&t0, e[0], e[1]) != cudaSuccess || cudaEventElapsedTime(&t1, e[2], e[3]) != cudaSuccess)
          rc = BDD_ECUDA;
        if (it == 1 || t0 < ms[v][0]) ms[v][0] = t0;
        if (it == 1 || t1 < ms[v][1]) ms[v][1] = t1;
      }
    }
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    if (rc != BDD_OK) {
      cudaGetLastError();
      stage_fwd = stage_bwd = 0;
      return rc;
    }
    // a later variant (larger shared-memory footprint, fewer resident warps) replaces the choice
    // only when it is at least kTuneMargin faster: launches timed one by one miss how a variant
    // shares the SMs with its neighbours inside the captured graphs, and near-ties flipped
    // between builds
    stage_fwd = stage_bwd = 0;
    for (int v = 1; v < kStagings; ++v) {
      if (ms[v][0] < (1.f - kTuneMargin) * ms[stage_fwd][0]) stage_fwd = v;
      if (ms[v][1] < (1.f - kTuneMargin) * ms[stage_bwd][1]) stage_bwd = v;
    }
    for (int v = 0; v < kStagings; ++v)
      for (int d = 0; d < 2; ++d) tune_ms[v][d] = ms[v][d];
    return restart(s);
  }

  // pending sums and the shares of the next sweep: a forward sweep follows a bound pass (the
  // end of an iteration), a backward sweep the pass between the sweeps; `next_dir` overrides
  int pending(bool bound, cudaStream_t s, int next_dir = 0, bool defer = false) {
    if (!next_dir) next_dir = bound ? kDirForward : kDirBackward;
    PendingParams r = pending_params(next_dir);
    r.defer = defer ? 1 : 0;
    return pending_launch(bound, r, grid_reduce, s) ? BDD_ECUDA : BDD_OK;
  }

  // one iteration: forward sweep, pending sums, backward sweep, pending sums and bound.  Fused
  // plan: forward sweep (reducing the previous iteration's bound unless `first`), backward
  // sweep, and with `last` the bound kernel.
  int enqueue_iteration(cudaStream_t s, bool first = true, bool last = true) {
    if (fused) {
      if (sweep_launch(true, kUpdateFused, fused_params(!first), grid_sweep, s)) return BDD_ECUDA;
      if (sweep_launch(false, kUpdateFused, fused_params(false), grid_sweep, s)) return BDD_ECUDA;
      if (last && bound_launch(fused_params(false), grid_reduce, s)) return BDD_ECUDA;
      return BDD_OK;
    }
    // the bound's per-block partials are summed by the next iteration's forward sweep (off the
    // chain's critical path), or after the last iteration by a one-warp kernel
    const bool defer = grid_sweep > 0;
    RC(sweep(true, kUpdate, s, nullptr, nullptr, defer && !first));
    RC(cut(true, s));
    RC(pending(false, s));
    RC(sweep(false, kUpdate, s));
    RC(pending(true, s, 0, defer));
    RC(cut(false, s));
    if (defer && last &&
        bound_finish_launch(d_partial, grid_reduce, d_iter, d_trace, trace_cap, empty_const, s))
      return BDD_ECUDA;
    return BDD_OK;
  }

  int launch_persistent(int n_iter, cudaStream_t s) {
    IterParams q{};
    q.sp = sweep_params();
    q.var_ptr = d_var_ptr;
    q.var_occ = d_var_occ;
    q.P = d_P;
    q.share_occ = d_share_occ;
    q.part = d_part;
    q.barrier = d_barrier;
    q.error = d_error;
    q.trace = d_trace;
    q.trace_cap = trace_cap;
    q.n_iter = n_iter;
    q.n = n;
    q.empty_const = empty_const;
    q.spin_limit = spin_limit;
    q.slot_dir = d_slot_dir;
    q.heavy = d_heavy;
    q.n_heavy = n_heavy;
    q.heavy_deg = heavy_deg;
    CK(cudaMemsetAsync(d_barrier, 0, 2 * sizeof(unsigned), s));
    return iterate_persistent_launch(q, grid_persist, smem_persist, s) ? BDD_ECUDA : BDD_OK;
  }

  // a device-side wait of an earlier launch gave up, or (checked build) an index check failed:
  // report once, then clear
  int take_device_error(cudaStream_t s) {
    if (!d_error) return BDD_OK;
    int err = 0;
    CK(cudaMemcpyAsync(&err, d_error, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (err != 0) {
      CK(cudaMemsetAsync(d_error, 0, sizeof(int), s));
      CK(cudaStreamSynchronize(s));
    }
    return bdd_status_of_device_word(err);
  }

  int capture(int iters, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = BDD_OK;
    for (int t = 0; t < iters && rc == BDD_OK; ++t) rc = enqueue_iteration(cap_stream, t == 0, t == iters - 1);
    cudaError_t e = cudaStreamEndCapture(cap_stream, &g);
    if (rc != BDD_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc != BDD_OK ? rc : BDD_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return BDD_OK;
  }

  void drop_graphs() {
    if (g_many) cudaGraphExecDestroy(g_many);
    if (g_one) cudaGraphExecDestroy(g_one);
    g_many = g_one = nullptr;
  }

  int ensure_trace(int need) {
    if (need <= trace_cap) return BDD_OK;
    int cap = std::max(need, std::max(1024, 2 * trace_cap));
    double *t = nullptr;
    RC(alloc(&t, cap));
    d_trace = t;  // the previous buffer stays owned by `allocs` until the solver is freed
    trace_cap = cap;
    drop_graphs();  // graphs bake in the trace pointer
    return BDD_OK;
  }

  int ensure_outputs() {
    if (!d_out_lam) RC(alloc(&d_out_lam, nnz));
    if (!d_out_m0) RC(alloc(&d_out_m0, nnz));
    if (!d_out_m1) RC(alloc(&d_out_m1, nnz));
    return BDD_OK;
  }

  // lambda^j_i = c_i/|J_i|, P = 0, then backward messages (and E^j) for that lambda.  Split
  // solvers: copy-arc duals and their last deltas 0, so every root message is 0.
  int restart(cudaStream_t s) {
    if (O > 0 && init_lambda_launch(d_occ_var, d_var_ptr, d_c, d_lam, (int)O, s)) return BDD_ECUDA;
    if (npairs > 0) {
      const size_t pb = sizeof(float) * (size_t)npairs;
      CK(cudaMemsetAsync(d_mu_bar, 0, pb, s));
      CK(cudaMemsetAsync(d_mu, 0, pb, s));
      CK(cudaMemsetAsync(d_dfwd, 0, pb, s));
      CK(cudaMemsetAsync(d_dbwd, 0, pb, s));
      CK(cudaMemsetAsync(d_fm, 0, sizeof(float) * (size_t)std::max<long long>(N, 1), s));
    }
    CK(cudaMemsetAsync(d_P, 0, sizeof(float) * std::max(n, 1), s));
    CK(cudaMemsetAsync(d_delta, 0, sizeof(float) * std::max<long long>(O, 1), s));
    CK(cudaMemsetAsync(d_share_occ, 0, sizeof(float) * std::max<long long>(O, 1), s));
    return sweep(false, kMessages, s);
  }

  // min-marginals and folded multipliers for the current state; leaves the state unchanged
  int output_pass(cudaStream_t s, float *lam_out, float *m0, float *m1) {
    const size_t bytes = sizeof(float) * (size_t)nnz;
    if (lam_out) {
      if (nnz) CK(cudaMemsetAsync(lam_out, 0, bytes, s));
      if (O && scatter_lambda_launch(d_lam, d_share_occ, d_occ_csr, lam_out, (int)O, true, s))
        return BDD_ECUDA;
    }
    if (m0 || m1) {
      if (!m0 || !m1) RC(ensure_outputs());
      float *o0 = m0 ? m0 : d_out_m0, *o1 = m1 ? m1 : d_out_m1;
      if (nnz) {
        CK(cudaMemsetAsync(o0, 0, bytes, s));
        CK(cudaMemsetAsync(o1, 0, bytes, s));
      }
      RC(sweep(true, kFolded, s));
      RC(sweep(false, kFolded, s, o0, o1));
      RC(sweep(false, kMessages, s));  // backward messages of the unfolded multipliers again
    }
    return BDD_OK;
  }
};

namespace {

// Device tables of the copy-arc pairs (CutParams), from the canonical pairs and the slab layout.
struct CutTables {
  std::vector<int4> grp, pair;
  std::vector<int> head_node, head_ptr, head_pair;
};

int build_cut_tables(const HostBDDs &H, const Layout &L, const CopyPairs &P, CutTables *T) {
  const long long G = P.ngroups();
  T->grp.resize(G);
  T->pair.resize(P.npairs());
  T->head_node.clear();
  T->head_ptr.assign(1, 0);
  T->head_pair.clear();
  std::vector<int> cnt;
  for (long long g = 0; g < G; ++g) {
    const long long ot = P.tail_occ[g];
    const int dt = L.occ_of_canon[ot], dh = L.occ_of_canon[ot + 1];
    const int tail0 = L.occ_node_off[dt], head0 = L.occ_node_off[dh], w = H.occ_width[ot + 1];
    const long long ps = P.cut_ptr[g], pe = P.cut_ptr[g + 1];
    const long long hs = (long long)T->head_node.size();
    if (hs + w > INT_MAX || pe > INT_MAX) return BDD_ETOOBIG;
    T->grp[g] = make_int4((int)ps, (int)pe, (int)hs, (int)(hs + w));
    cnt.assign(w, 0);
    for (long long k = ps; k < pe; ++k) {
      T->pair[k] = make_int4(tail0 + P.tail[k], head0 + P.head[k], dt, P.side[k]);
      cnt[P.head[k]]++;
    }
    for (int t = 0; t < w; ++t) {
      T->head_node.push_back(head0 + t);
      T->head_ptr.push_back(T->head_ptr.back() + cnt[t]);
    }
    const size_t base = T->head_pair.size();
    T->head_pair.resize(base + (size_t)(pe - ps));
    std::vector<int> fill(T->head_ptr.end() - 1 - w, T->head_ptr.end() - 1);
    for (long long k = ps; k < pe; ++k) T->head_pair[fill[P.head[k]]++] = (int)k;
  }
  return BDD_OK;
}

template <class Tp, class A>
int upload(bdd_solver *h, Tp **d, const std::vector<Tp, A> &v) {
  RC(h->alloc(d, (long long)v.size()));
  if (!v.empty()) CK(cudaMemcpy(*d, v.data(), v.size() * sizeof(Tp), cudaMemcpyHostToDevice));
  return BDD_OK;
}

int setup_device(bdd_solver *h, const Layout &L, const float *c, const CutTables &ct) {
  CK(cudaEventCreateWithFlags(&h->ev_last, cudaEventDisableTiming));
  h->bdd_perm = L.bdd_perm;
  h->tile_occ0 = L.tile_occ0;
  h->tile_bdd0 = L.tile_bdd0;
  h->tile_nbdd = L.tile_nbdd;
  for (int t = 0; t < kWarpClasses + 2; ++t) h->class_tile_off[t] = L.class_tile_off[t];
  h->n_warp_tiles = L.n_warp_tiles;
  h->n_block_tiles = L.n_block_tiles;
  h->block_buf = ((L.max_block_width + 3) / 4) * 4;
  {
    int dmax = 0;
    for (int t = L.class_tile_off[kWarpClasses]; t < L.class_tile_off[kWarpClasses + 1]; ++t)
      dmax = std::max(dmax, L.bdd_depth[L.tile_bdd0[t]]);
    h->block_depth_buf = ((dmax + 3) / 4) * 4;
  }
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BDD_ECUDA;
  nsm = std::max(1, nsm);
  // lane tiles go out in runs of kLaneRunMax consecutive tiles per warp, shorter where that
  // would leave fewer than 32 warps per SM; the other warp tiles one per warp after them
  long long warp_units = L.n_warp_tiles;
  h->lane_run = 1;
  h->n_lane_warps = 0;
  if (h->lanes2) {
    const long long nlt = L.class_tile_off[1];
    h->lane_run = (int)std::max<long long>(1, std::min<long long>(kLaneRunMax, nlt / (32LL * nsm)));
    h->n_lane_warps = (int)((nlt + h->lane_run - 1) / h->lane_run);
    warp_units = h->n_lane_warps + (L.n_warp_tiles - nlt);
  }
  h->n_warp_blocks = (int)((warp_units + kWarpsPerBlock - 1) / kWarpsPerBlock);
  h->grid_sweep = h->n_warp_blocks + L.n_block_tiles;
  const int range = std::max<long long>(h->n, h->nb) > 0 ? (int)std::max<long long>(h->n, h->nb) : 1;
  // pending passes: a thread per variable (and BDD), plus one warp per variable with more than
  // heavy_deg occurrences.  heavy_deg: the least of 8, 16, 32, ... that leaves at most 4096 such
  // variables, so that each gets its own warp (a warp's two rounds of loads beat a thread's
  // serial batches for few long variables; for many, the extra warps cost more than they save)
  // (one parallel pass: variables above 8 * 2^t occurrences, for every t)
  constexpr int kDegSteps = 18;
  long long above[kDegSteps] = {};
  {
    std::mutex mu;
    parallel_for(h->n, 1 << 16, [&](long long a, long long e) {
      long long loc[kDegSteps] = {};
      for (long long i = a; i < e; ++i) {
        const int d = L.var_ptr[i + 1] - L.var_ptr[i];
        for (int t = 0; t < kDegSteps && d > (8 << t); ++t) ++loc[t];
      }
      std::lock_guard<std::mutex> lk(mu);
      for (int t = 0; t < kDegSteps; ++t) above[t] += loc[t];
    });
  }
  int step = 0;
  while (step + 1 < kDegSteps && above[step] > 4096) ++step;
  h->heavy_deg = 8 << step;
  const int n_heavy = (int)above[step];
  const int heavy_blocks = (n_heavy + kReduceThreads / 32 - 1) / (kReduceThreads / 32);
  h->grid_reduce = std::max(1, std::min(std::max((range + kReduceThreads - 1) / kReduceThreads, heavy_blocks), 152 * 16));
  // the largest dynamic shared memory any staging variant's sweep launch asks for
  h->smem = std::max(sweep_smem_bytes(h->block_buf, h->block_depth_buf, 0, h->lanes2, h->alpha > 0.f),
                     sweep_smem_bytes(h->block_buf, h->block_depth_buf, 2, h->lanes2, h->alpha > 0.f));
  h->smem_persist = persist_smem_bytes(h->block_buf, h->block_depth_buf);
  if (h->smem > 48 * 1024 && sweep_set_smem(h->smem)) return BDD_ECUDA;
  // programmatic dependent launch: each per-phase kernel lets its successor launch as soon as it
  // starts only when a sweep's grid is at most two waves; for larger grids the early-resident
  // successor blocks measured slower (8 % per iteration on the 256-instance Potts batch, 2-20 %
  // on tomography) than letting them launch as the blocks exit, while small grids gain from it
  // (30 % on Potts 20x20, 7 % on matching)
  {
    int per_sm = 0;
    if (sweep_resident_blocks(h->smem, &per_sm)) return BDD_ECUDA;
    h->pdl_early = (long long)h->grid_sweep <= 2LL * nsm * std::max(1, per_sm);
  }
  if (h->schedule == 0) {
    int max_grid = 0;
    if (iterate_set_smem(h->smem_persist) == 0 && iterate_persistent_max_grid(h->smem_persist, &max_grid) == 0) {
      // enough blocks for one warp tile per warp and one block tile per 128-thread group
      const long long need = (L.n_warp_tiles + kPersistWarps - 1) / kPersistWarps +
                             (L.n_block_tiles + kSubBlocks - 1) / kSubBlocks;
      h->grid_persist = (int)std::max<long long>(1, std::min<long long>(max_grid, need));
    } else {
      cudaGetLastError();
      h->schedule = 1;  // no cooperative launch (or not enough shared memory) on this device
    }
  }
  // per-phase plan: the pending pass fused into the sweeps only when asked for (measured slower:
  // a variable's last visit finishes it on one lane, and a warp's tail serialises many such
  // variables, longer than the separate pending kernel takes)
  h->fused = h->schedule == 1 && h->fused_opt == 1;

  // device memory estimate against the cap, before allocating anything
  const long long O = h->O, N = h->N, nb = h->nb, n = h->n;
  const long long ntiles = (long long)L.tile_bdd0.size();
  long long need = (O + 1) * 4 + O * 4 + O * 8 + N * 8 + 2 * N * 4 + 2 * O * 4 + 3 * (long long)n * 4 +
                   nb * 8 + 3 * ntiles * 4 + (n + 1) * 4 + O * 4 + h->grid_reduce * 8 + 1024 * 8 +
                   (h->averaging == 1 ? O : 0) + (h->lanes2 ? O + kLaneCodePad : 0) + 4LL * (long long)(L.tile_win0.size() + L.win_node.size()) + (h->fused ? 12 * n + 8LL * (h->grid_sweep + h->grid_reduce) : 0) +
                   h->npairs * 36 + 16 * h->ngroups + 8LL * (long long)ct.head_node.size();
  if (h->max_device_bytes > 0 && need > h->max_device_bytes) return BDD_ENOMEM;

  RC(upload(h, &h->d_occ_node_off, L.occ_node_off));
  RC(upload(h, &h->d_occ_var, L.occ_var));
  RC(upload(h, &h->d_occ_csr, L.occ_csr));
  RC(upload(h, &h->d_occ_slot, L.occ_slot));
  {
    int *tmp = nullptr;
    RC(upload(h, &tmp, L.lohi));
    h->d_lohi = reinterpret_cast<int2 *>(tmp);
  }
  if (h->lanes2) RC(upload(h, &h->d_lane_code, L.lane_code));
  RC(h->alloc(&h->d_fm, N));
  RC(h->alloc(&h->d_bm, N));
  RC(h->alloc(&h->d_lam, O));
  RC(h->alloc(&h->d_delta, O));
  RC(h->alloc(&h->d_share_occ, O));
  RC(h->alloc(&h->d_part, 2LL * std::max(1, h->grid_persist)));
  RC(h->alloc(&h->d_barrier, 2));
  RC(h->alloc(&h->d_error, 1));
  CK(cudaMemset(h->d_error, 0, sizeof(int)));
  RC(h->alloc(&h->d_P, n));
  RC(h->alloc(&h->d_c, n));
  RC(upload(h, &h->d_bdd_depth, L.bdd_depth));
  {
    std::vector<int> rows(h->nb);
    for (long long t = 0; t < h->nb; ++t) rows[t] = h->canon_row[L.bdd_perm[t]];
    RC(upload(h, &h->d_bdd_row, rows));
  }
  RC(h->alloc(&h->d_bdd_E, nb));
  RC(upload(h, &h->d_tile_occ0, L.tile_occ0));
  RC(upload(h, &h->d_tile_win0, L.tile_win0));
  {
    int *tmp = nullptr;
    RC(upload(h, &tmp, L.win_node));
    h->d_win_node = reinterpret_cast<int2 *>(tmp);
  }
  RC(upload(h, &h->d_tile_bdd0, L.tile_bdd0));
  RC(upload(h, &h->d_tile_nbdd, L.tile_nbdd));
  RC(upload(h, &h->d_var_ptr, L.var_ptr));
  RC(upload(h, &h->d_var_occ, L.var_occ));
  if (h->averaging == 1) RC(upload(h, &h->d_slot_dir, L.slot_dir));
  {
    std::vector<int4> heavy;
    for (int i = 0; i < h->n && n_heavy > 0; ++i)
      if (L.var_ptr[i + 1] - L.var_ptr[i] > h->heavy_deg)
        heavy.push_back(make_int4(i, L.var_ptr[i], L.var_ptr[i + 1], 0));
    h->n_heavy = (int)heavy.size();
    if (!heavy.empty()) RC(upload(h, &h->d_heavy, heavy));
  }
  if (h->fused) {
    RC(upload(h, &h->d_cnt, h->var_deg));
    RC(h->alloc(&h->d_slk, n));
    if (n) CK(cudaMemset(h->d_slk, 0, sizeof(double) * n));
    RC(h->alloc(&h->d_fpartial, std::max(h->grid_sweep, h->grid_reduce)));
    RC(h->alloc(&h->d_fticket, 1));
    CK(cudaMemset(h->d_fticket, 0, sizeof(unsigned)));
  }
  if (h->npairs > 0) {
    RC(upload(h, &h->d_cut_grp, ct.grp));
    RC(upload(h, &h->d_pair, ct.pair));
    RC(upload(h, &h->d_head_node, ct.head_node));
    RC(upload(h, &h->d_head_ptr, ct.head_ptr));
    RC(upload(h, &h->d_head_pair, ct.head_pair));
    RC(h->alloc(&h->d_mu_bar, h->npairs));
    RC(h->alloc(&h->d_mu, h->npairs));
    RC(h->alloc(&h->d_dfwd, h->npairs));
    RC(h->alloc(&h->d_dbwd, h->npairs));
  }
  RC(h->alloc(&h->d_partial, h->grid_reduce));
  RC(h->alloc(&h->d_ticket, 1));
  RC(h->alloc(&h->d_iter, 1));
  CK(cudaMemset(h->d_ticket, 0, sizeof(unsigned)));
  CK(cudaMemset(h->d_iter, 0, sizeof(int)));
  RC(h->ensure_trace(1024));
  if (n) CK(cudaMemcpy(h->d_c, c, sizeof(float) * n, cudaMemcpyHostToDevice));
  RC(h->restart(h->stream));
  if (h->staging_opt >= 0) {
    h->stage_fwd = h->stage_bwd = h->staging_opt;
  } else if (h->schedule == 1 && !h->fused) {
    RC(h->autotune(h->stream, 6));
  }
  RC(h->end(h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BDD_OK;
}

// ---------------------------------------------------------------------------------------
// Layout tuner.  Each key (a BDD's natural width class and its depth bucket) has up to two tile
// classes its BDDs can run in: lane tiles or two-lane teams for widths <= 2; a team of 2^c or of
// 2^(c+1) lanes (a block tile after 32) for wider ones.  For every key holding enough nodes the
// candidates are timed on a probe: the key's BDDs alone (every k-th one when they hold more than
// kProbeCap nodes, so the probe still fills the GPU many times over), each occurrence its own
// variable, built into a throwaway device solver; the update sweeps of a warm-up iteration and
// three more are timed kernel by kernel, and the fastest forward plus the fastest backward
// launch count.  The alternative replaces the default only when it is kTuneMargin faster.
// ---------------------------------------------------------------------------------------
constexpr long long kProbeCap = 16LL << 20;  // nodes of a probe
constexpr long long kProbeMin = 4096;        // keys with fewer nodes keep the default

long long bdd_nodes(const HostBDDs &H, long long b) {
  return H.occ_node0[H.bdd_occ0[b + 1]] - H.occ_node0[H.bdd_occ0[b]];
}

int bdd_width(const HostBDDs &H, long long b) {
  int w = 0;
  for (long long o = H.bdd_occ0[b]; o < H.bdd_occ0[b + 1]; ++o) w = std::max(w, H.occ_width[o]);
  return w;
}

// layout key of every BDD, and the nodes per key (both in parallel)
std::vector<unsigned char> bdd_keys(const HostBDDs &H, long long key_nodes[kLayoutKeys]) {
  std::vector<unsigned char> key(H.nb());
  parallel_for(H.nb(), 4096, [&](long long b0, long long b1) {
    for (long long b = b0; b < b1; ++b) key[b] = (unsigned char)layout_key(bdd_width(H, b), H.bdd_depth[b]);
  });
  for (int k = 0; k < kLayoutKeys; ++k) key_nodes[k] = 0;
  for (long long b = 0; b < H.nb(); ++b) key_nodes[key[b]] += bdd_nodes(H, b);
  return key;
}

HostBDDs probe_instance(const HostBDDs &H, const std::vector<unsigned char> &keys, int key, long long key_nodes) {
  HostBDDs P;
  const long long step = std::max(1LL, (key_nodes + kProbeCap - 1) / kProbeCap);
  long long seen = 0;
  P.bdd_occ0.push_back(0);
  P.occ_node0.push_back(0);
  for (long long b = 0; b < H.nb(); ++b) {
    if (keys[b] != key) continue;
    if (seen++ % step) continue;
    P.bdd_row.push_back((int)P.bdd_row.size());
    P.bdd_depth.push_back(H.bdd_depth[b]);
    P.max_depth = std::max(P.max_depth, H.bdd_depth[b]);
    for (long long o = H.bdd_occ0[b]; o < H.bdd_occ0[b + 1]; ++o) {
      const int w = H.occ_width[o];
      P.occ_var.push_back((int)P.occ_var.size());
      P.occ_csr.push_back((long long)P.occ_csr.size());
      P.occ_width.push_back(w);
      P.max_width = std::max(P.max_width, w);
      for (long long v = H.occ_node0[o]; v < H.occ_node0[o + 1]; ++v) {
        P.lo.push_back(H.lo[v]);
        P.hi.push_back(H.hi[v]);
      }
      P.occ_node0.push_back((long long)P.lo.size());
    }
    P.bdd_occ0.push_back((long long)P.occ_var.size());
  }
  P.n = (int)P.occ_var.size();
  P.m = (int)P.bdd_row.size();
  P.nnz = P.n;
  return P;
}

// ms of one forward plus one backward update sweep of the probe in the given layout (-1: failed)
float probe_time(const HostBDDs &P, bool lanes2, const int *class_of_key) {
  bdd_solver *h = new (std::nothrow) bdd_solver();
  if (!h) return -1.f;
  h->n = P.n;
  h->m = P.m;
  h->nnz = P.nnz;
  h->nb = P.nb();
  h->O = P.O();
  h->N = P.N();
  h->max_depth = P.max_depth;
  h->max_width = P.max_width;
  h->lanes2 = lanes2;
  h->staging_opt = 0;
  h->schedule = 1;
  h->canon_row = P.bdd_row;
  h->var_deg.assign(P.n, 1);
  h->c.assign(P.n, 0.f);
  float ms = -1.f;
  Layout L;
  int rc = build_layout(P, &L, lanes2, class_of_key);
  if (rc == BDD_OK && cudaGetDevice(&h->device) != cudaSuccess) rc = BDD_ECUDA;
  if (rc == BDD_OK && cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) rc = BDD_ECUDA;
  if (rc == BDD_OK) h->own_stream = true;
  if (rc == BDD_OK && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) rc = BDD_ECUDA;
  if (rc == BDD_OK) rc = setup_device(h, L, h->c.data(), CutTables());
  cudaEvent_t ev[16] = {};
  for (auto &e : ev)
    if (rc == BDD_OK && cudaEventCreate(&e) != cudaSuccess) rc = BDD_ECUDA;
  const cudaStream_t s = h->stream;
  for (int it = 0; it < 4 && rc == BDD_OK; ++it) {
    cudaEvent_t *e = &ev[4 * it];
    if (cudaEventRecord(e[0], s) != cudaSuccess) rc = BDD_ECUDA;
    if (rc == BDD_OK) rc = h->sweep(true, kUpdate, s);
    if (rc == BDD_OK && cudaEventRecord(e[1], s) != cudaSuccess) rc = BDD_ECUDA;
    if (rc == BDD_OK) rc = h->pending(false, s);
    if (rc == BDD_OK && cudaEventRecord(e[2], s) != cudaSuccess) rc = BDD_ECUDA;
    if (rc == BDD_OK) rc = h->sweep(false, kUpdate, s);
    if (rc == BDD_OK && cudaEventRecord(e[3], s) != cudaSuccess) rc = BDD_ECUDA;
    if (rc == BDD_OK) rc = h->pending(true, s);
  }
  if (rc == BDD_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = BDD_ECUDA;
  float fwd = -1.f, bwd = -1.f;
  for (int it = 1; it < 4 && rc == BDD_OK; ++it) {  // iteration 0 warms up
    float t0 = 0.f, t1 = 0.f;
    if (cudaEventElapsedTime(&t0, ev[4 * it], ev[4 * it + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t1, ev[4 * it + 2], ev[4 * it + 3]) != cudaSuccess)
      rc = BDD_ECUDA;
    if (fwd < 0.f || t0 < fwd) fwd = t0;
    if (bwd < 0.f || t1 < bwd) bwd = t1;
  }
  if (rc == BDD_OK) ms = fwd + bwd;
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete h;
  return ms;
}

// Chooses the tile class of every key of a plain solver's BDDs (see above).  allow_lanes: lane
// tiles are a candidate for widths <= 2 (-1 tuned, 0 never, 1 always).  Fills h->key_*, sets
// h->lanes2; returns a BDD_* status.
int tune_layout(bdd_solver *h, const HostBDDs &H, int allow_lanes) {
  const std::vector<unsigned char> keys = bdd_keys(H, h->key_nodes);
  const long long min_nodes = std::max(kProbeMin, H.N() / 100);
  bool any_lane = false;
  for (int k = 0; k < kLayoutKeys; ++k) {
    if (h->key_nodes[k] == 0) continue;
    const int wc = k / kDepthBuckets;
    if (wc == kWarpClasses) continue;  // block tiles: no alternative
    // candidates: [default, alternative]; for widths <= 2 the teams of two lanes (class 1) and
    // the lane tiles (class 0 with lanes2)
    const bool narrow = wc <= 1;
    if (narrow && allow_lanes == 1) {
      h->key_class[k] = 0;
      any_lane = true;
      continue;
    }
    if (narrow && allow_lanes == 0) continue;
    const int cand[2] = {narrow ? 1 : wc, narrow ? 0 : wc + 1};
    if (h->key_nodes[k] < min_nodes) {
      h->key_class[k] = cand[0];
      continue;
    }
    HostBDDs P = probe_instance(H, keys, k, h->key_nodes[k]);
    for (int t = 0; t < 2; ++t) {
      int table[kLayoutKeys];
      for (int q = 0; q < kLayoutKeys; ++q) table[q] = -1;
      table[k] = cand[t];
      h->key_ms[k][t] = probe_time(P, narrow && t == 1, table);
      if (h->key_ms[k][t] < 0.f) return BDD_ECUDA;
    }
    const bool alt = h->key_ms[k][1] < (1.f - kTuneMargin) * h->key_ms[k][0];
    h->key_class[k] = cand[alt ? 1 : 0];
    if (narrow && alt) any_lane = true;
  }
  h->lanes2 = any_lane;
  if (!any_lane)  // no lane tiles: widths <= 2 keep their natural classes (width 1 in class 0)
    for (int k = 0; k < 2 * kDepthBuckets; ++k) h->key_class[k] = -1;
  return BDD_OK;
}

bool finite_costs(const float *c, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(c[i])) return false;
  return true;
}

// sum over variables in no row of the y-slack term min(0, c_i) (its soft minimum for alpha > 0)
double empty_constant(const std::vector<int> &deg, const float *c, int n, double alpha) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    if (deg[i] != 0) continue;
    const double x = c[i], m = x < 0.0 ? x : 0.0;
    s += alpha > 0.0 ? m - alpha * std::log1p(std::exp(-std::fabs(x) / alpha)) : m;
  }
  return s;
}

}  // namespace

extern "C" {

void bdd_default_options(bdd_options *opt) {
  if (!opt) return;
  opt->omega = 0.5f;
  opt->max_width = 1 << 20;
  opt->max_nodes = 2147483647LL;
  opt->max_device_bytes = 0;
  opt->host_only = 0;
  opt->device = -1;
  opt->stream = nullptr;
  opt->schedule = 1;
  opt->spin_limit = 1LL << 26;
  opt->alpha = 0.f;
  opt->var_rank = nullptr;
  opt->averaging = 0;
  opt->fused_pending = -1;
  opt->staging = -1;
  opt->split_intervals = 0;
  opt->cuts = nullptr;
  opt->n_cuts = 0;
  opt->gamma = 0.5f;
  opt->split_depth = 0;
  opt->lanes = -1;
  opt->tune_layout = -1;
  opt->layout_classes = nullptr;
  opt->smooth_messages = -1;
}

int bdd_last_failed_row(void) { return g_failed_row; }

int bdd_build(int n, int m, const long long *row_ptr, const int *col, const int *val, const int *b,
              const signed char *sense, const float *c, const bdd_options *opt_in, bdd_solver **out) {
  g_failed_row = -1;
  if (!out) return BDD_EINVAL;
  *out = nullptr;
  bdd_options opt;
  bdd_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (n < 0 || m < 0 || (m > 0 && (!row_ptr || !b || !sense)) || (n > 0 && !c)) return BDD_EINVAL;
  if (!(opt.omega > 0.f && opt.omega <= 1.f) || opt.max_width < 1 || opt.max_nodes < 1) return BDD_EINVAL;
  if (!(opt.alpha >= 0.f) || !std::isfinite(opt.alpha)) return BDD_EINVAL;
  if (m > 0 && row_ptr[0] != 0) return BDD_EINVAL;
  for (int j = 0; j < m; ++j)
    if (row_ptr[j + 1] < row_ptr[j]) {
      g_failed_row = j;
      return BDD_EINVAL;
    }
  const long long nnz = m ? row_ptr[m] : 0;
  if (nnz > 0 && (!col || !val)) return BDD_EINVAL;
  if (!finite_costs(c, n)) return BDD_EINVAL;
  if (opt.averaging < 0 || opt.averaging > 1) return BDD_EINVAL;
  if (opt.fused_pending < -1 || opt.fused_pending > 1) return BDD_EINVAL;
  if (opt.staging < -1 || opt.staging >= kStagings) return BDD_EINVAL;
  if (opt.split_intervals < 0 || opt.n_cuts < 0 || (opt.n_cuts > 0 && !opt.cuts) || opt.split_depth < 0)
    return BDD_EINVAL;
  if (!(opt.gamma > 0.f && opt.gamma <= 1.f)) return BDD_EINVAL;
  const bool want_split = opt.split_depth > 0 || opt.n_cuts > 0 || opt.split_intervals >= 2;
  if (want_split && opt.alpha > 0.f) return BDD_EINVAL;  // sub-BDDs run the min-sum iteration only
  if (opt.lanes < -1 || opt.lanes > 1 || opt.tune_layout < -1 || opt.tune_layout > 1) return BDD_EINVAL;
  // lane tiles and the layout tuner: the plain min-sum sweeps of the per-phase schedule only
  const bool plain = opt.alpha == 0.f && !want_split && opt.fused_pending != 1 && opt.schedule == 1;
  if ((opt.lanes == 1 || opt.tune_layout == 1 || opt.layout_classes) && !plain) return BDD_EINVAL;
  bool lanes2 = opt.lanes == 1 || (opt.lanes == -1 && plain);
  if (opt.layout_classes) {  // explicit table: 7 = lane tiles (widths <= 2), else a tile class
    lanes2 = false;
    for (int k = 0; k < kLayoutKeys; ++k) {
      const int c = opt.layout_classes[k];
      if (c < -1 || c > kWarpClasses + 1 || (c == kWarpClasses + 1 && k >= 2 * kDepthBuckets)) return BDD_EINVAL;
      if (c == kWarpClasses + 1) lanes2 = true;
    }
    if (lanes2 && opt.lanes == 0) return BDD_EINVAL;
  }
  const bool tune = plain && !opt.layout_classes && opt.tune_layout != 0 && !opt.host_only;
  if (opt.var_rank) {  // a permutation of 0..n-1
    std::vector<char> seen;
    try {
      seen.assign(n, 0);
    } catch (const std::bad_alloc &) {
      return BDD_ENOMEM;
    }
    for (int i = 0; i < n; ++i) {
      const int r = opt.var_rank[i];
      if (r < 0 || r >= n || seen[r]) return BDD_EINVAL;
      seen[r] = 1;
    }
  }

  bdd_solver *h = new (std::nothrow) bdd_solver();
  if (!h) return BDD_ENOMEM;
  h->n = n;
  h->m = m;
  h->nnz = nnz;
  h->omega = opt.omega;
  h->alpha = opt.alpha;
  h->smooth_messages = opt.smooth_messages;
  h->averaging = opt.averaging;
  h->fused_opt = want_split ? 0 : opt.fused_pending;  // the copy-arc steps follow whole sweeps
  h->staging_opt = h->fused_opt == 1 ? 0 : opt.staging;
  // the persistent kernel runs the plain min-sum iteration only
  h->schedule = opt.alpha > 0.f || want_split ? 1 : opt.schedule;
  h->gamma = opt.gamma;
  h->lanes2 = lanes2;
  h->spin_limit = opt.spin_limit;
  if (opt.schedule < 0 || opt.schedule > 1 || opt.spin_limit < 1) {
    delete h;
    return BDD_EINVAL;
  }
  if (opt.host_only < 0 || opt.host_only > 2) {
    delete h;
    return BDD_EINVAL;
  }
  h->host_only = opt.host_only != 0;
  h->host_layout = opt.host_only == 2;
  h->max_device_bytes = opt.max_device_bytes;
  int failed = -1, rc;
  try {
    rc = compile_bdds(n, m, row_ptr, col, val, b, sense, opt.var_rank, opt.max_width, opt.max_nodes, &h->host,
                      &failed);
  } catch (const std::bad_alloc &) {
    rc = BDD_ENOMEM;
  }
  if (rc != BDD_OK) {
    g_failed_row = failed;
    delete h;
    return rc;
  }
  HostBDDs &H = h->host;
  CopyPairs pairs;
  if (want_split) {
    std::vector<int> cuts;
    if (opt.split_depth > 0) {
      // depth split: no interval cuts
    } else if (opt.n_cuts > 0) {
      cuts.assign(opt.cuts, opt.cuts + opt.n_cuts);
    } else {
      cuts = balanced_cuts(H, opt.var_rank, opt.split_intervals);
    }
    h->split_depth = opt.split_depth;
    try {
      rc = split_bdds(H, opt.var_rank, cuts, opt.split_depth, &pairs);
    } catch (const std::bad_alloc &) {
      rc = BDD_ENOMEM;
    }
    if (rc != BDD_OK) {
      delete h;
      return rc;
    }
    h->cuts = pairs.cuts;
    h->npairs = pairs.npairs();
    h->ngroups = pairs.ngroups();
  }
  h->nb = H.nb();
  h->O = H.O();
  h->N = H.N();
  h->max_depth = H.max_depth;
  h->max_width = H.max_width;
  h->canon_row = H.bdd_row;
  h->var_deg.assign(n, 0);
  {
    int *deg = h->var_deg.data();
    parallel_for(H.O(), 1 << 16, [&](long long a, long long e) {
      for (long long o = a; o < e; ++o) __atomic_fetch_add(&deg[H.occ_var[o]], 1, __ATOMIC_RELAXED);
    });
  }
  h->c.assign(c, c + n);
  h->empty_const = empty_constant(h->var_deg, c, n, h->alpha);
  if (h->host_only && !h->host_layout) {
    *out = h;
    return BDD_OK;
  }
  // tile class of every layout key: explicit, tuned on the device, or the defaults
  bool keyed = false;
  if (opt.layout_classes) {
    for (int k = 0; k < kLayoutKeys; ++k) {
      const int c = opt.layout_classes[k];
      h->key_class[k] = c == kWarpClasses + 1 ? 0 : c;
    }
    bdd_keys(H, h->key_nodes);
    keyed = true;
  } else if (tune) {
    DeviceGuard dg(opt.device);
    rc = dg.ok ? BDD_OK : BDD_ECUDA;
    try {
      if (rc == BDD_OK) rc = tune_layout(h, H, opt.lanes);
    } catch (const std::bad_alloc &) {
      rc = BDD_ENOMEM;
    }
    if (rc != BDD_OK) {
      delete h;
      return rc;
    }
    keyed = true;
  } else {
    bdd_keys(H, h->key_nodes);
  }
  Layout L;
  try {
    rc = build_layout(H, &L, h->lanes2, keyed ? h->key_class : nullptr, h->var_deg.data());
  } catch (const std::bad_alloc &) {
    rc = BDD_ENOMEM;
  }
  if (rc == BDD_OK && h->lanes2) {  // lane tiles come first: their occurrences and nodes too
    const int nlt = L.class_tile_off[1];
    h->lane_O = nlt < (int)L.tile_occ0.size() ? L.tile_occ0[nlt] : H.O();
    h->lane_N = L.occ_node_off[h->lane_O];
  }
  // smoothing: warp tiles and block tiles of at most kBlockThreads nodes per layer
  if (rc == BDD_OK && h->alpha > 0.f && L.n_block_tiles > 0 && L.max_block_width > kBlockThreads) rc = BDD_ETOOBIG;
  CutTables ct;
  if (rc == BDD_OK && h->npairs > 0 && !h->host_layout) {
    try {
      rc = build_cut_tables(H, L, pairs, &ct);
    } catch (const std::bad_alloc &) {
      rc = BDD_ENOMEM;
    }
  }
  if (rc != BDD_OK) {
    delete h;
    return rc;
  }
  if (h->host_layout) {
    h->bdd_perm = L.bdd_perm;
    h->tile_occ0 = L.tile_occ0;
    h->tile_bdd0 = L.tile_bdd0;
    h->tile_nbdd = L.tile_nbdd;
    for (int t = 0; t < kWarpClasses + 2; ++t) h->class_tile_off[t] = L.class_tile_off[t];
    h->n_warp_tiles = L.n_warp_tiles;
    h->n_block_tiles = L.n_block_tiles;
    h->layout = std::move(L);
    *out = h;
    return BDD_OK;
  }
  H = HostBDDs();  // the device slabs are the only copy from here on
  {
    DeviceGuard dg(opt.device);
    if (!dg.ok) {
      delete h;
      return BDD_ECUDA;
    }
    cudaGetDevice(&h->device);
    if (opt.stream) {
      h->stream = (cudaStream_t)opt.stream;
    } else if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return BDD_ECUDA;
    } else {
      h->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return BDD_ECUDA;
    }
    rc = setup_device(h, L, c, ct);
  }
  if (rc != BDD_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return BDD_OK;
}

int bdd_iterate_device(bdd_solver *h, int n_iter, double *d_bound_trace, float *d_lambda, float *d_mm0,
                       float *d_mm1, void *stream) {
  if (!h || n_iter < 0) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  RC(h->ensure_trace(n_iter + 1));
  if (n_iter > 0 && h->schedule == 1) {
    if (!h->g_one) RC(h->capture(1, &h->g_one));
    if (!h->g_many && n_iter >= kGraphIters) RC(h->capture(kGraphIters, &h->g_many));
  }
  RC(h->begin(s));
  if (n_iter > 0) ++h->state_gen;
  if (h->schedule == 0) {
    if (n_iter > 0) RC(h->launch_persistent(n_iter, s));
  } else {
    CK(cudaMemsetAsync(h->d_iter, 0, sizeof(int), s));
    int left = n_iter;
    while (left >= kGraphIters) {
      CK(cudaGraphLaunch(h->g_many, s));
      left -= kGraphIters;
    }
    for (; left > 0; --left) CK(cudaGraphLaunch(h->g_one, s));
  }
  if (d_bound_trace && n_iter > 0)
    CK(cudaMemcpyAsync(d_bound_trace, h->d_trace, sizeof(double) * n_iter, cudaMemcpyDeviceToDevice, s));
  RC(h->output_pass(s, d_lambda, d_mm0, d_mm1));
  return h->end(s);
}

int bdd_iterate_profiled(bdd_solver *h, int n_iter, double *kernel_ms) {
  if (!h || n_iter < 0 || !kernel_ms) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = h->stream;
  for (int t = 0; t < 4; ++t) kernel_ms[t] = 0.0;
  RC(h->ensure_trace(n_iter + 1));
  RC(h->begin(s));
  ++h->state_gen;
  CK(cudaMemsetAsync(h->d_iter, 0, sizeof(int), s));
  const int kBatch = 256;  // iterations per batch of recorded events
  std::vector<cudaEvent_t> ev(5 * kBatch, nullptr);
  int rc = BDD_OK;
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = BDD_ECUDA;
  for (int done = 0; done < n_iter && rc == BDD_OK;) {
    const int cnt = std::min(kBatch, n_iter - done);
    for (int t = 0; t < cnt && rc == BDD_OK; ++t) {
      cudaEvent_t *e = &ev[5 * t];
      if (cudaEventRecord(e[0], s) != cudaSuccess) rc = BDD_ECUDA;
      if (h->fused) {  // forward sweep, (no separate pending pass), backward sweep, bound
        if (rc == BDD_OK && sweep_launch(true, kUpdateFused, h->fused_params(false), h->grid_sweep, s)) rc = BDD_ECUDA;
        if (rc == BDD_OK && cudaEventRecord(e[1], s) != cudaSuccess) rc = BDD_ECUDA;
        if (rc == BDD_OK && cudaEventRecord(e[2], s) != cudaSuccess) rc = BDD_ECUDA;
        if (rc == BDD_OK && sweep_launch(false, kUpdateFused, h->fused_params(false), h->grid_sweep, s)) rc = BDD_ECUDA;
        if (rc == BDD_OK && cudaEventRecord(e[3], s) != cudaSuccess) rc = BDD_ECUDA;
        if (rc == BDD_OK && bound_launch(h->fused_params(false), h->grid_reduce, s)) rc = BDD_ECUDA;
        if (rc == BDD_OK && cudaEventRecord(e[4], s) != cudaSuccess) rc = BDD_ECUDA;
        continue;
      }
      if (rc == BDD_OK) rc = h->sweep(true, kUpdate, s);
      if (rc == BDD_OK && cudaEventRecord(e[1], s) != cudaSuccess) rc = BDD_ECUDA;
      if (rc == BDD_OK) rc = h->cut(true, s);
      if (rc == BDD_OK) rc = h->pending(false, s);
      if (rc == BDD_OK && cudaEventRecord(e[2], s) != cudaSuccess) rc = BDD_ECUDA;
      if (rc == BDD_OK) rc = h->sweep(false, kUpdate, s);
      if (rc == BDD_OK && cudaEventRecord(e[3], s) != cudaSuccess) rc = BDD_ECUDA;
      if (rc == BDD_OK) rc = h->pending(true, s);
      if (rc == BDD_OK) rc = h->cut(false, s);
      if (rc == BDD_OK && cudaEventRecord(e[4], s) != cudaSuccess) rc = BDD_ECUDA;
    }
    if (rc == BDD_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = BDD_ECUDA;
    for (int t = 0; t < cnt && rc == BDD_OK; ++t)
      for (int k = 0; k < 4; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[5 * t + k], ev[5 * t + k + 1]) != cudaSuccess) rc = BDD_ECUDA;
        kernel_ms[k] += ms;
      }
    done += cnt;
  }
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  if (rc != BDD_OK) cudaGetLastError();
  if (rc == BDD_OK) rc = h->end(s);
  return rc;
}

int bdd_iterate(bdd_solver *h, int n_iter, double *lower_bound, float *lambda, float *mm0, float *mm1) {
  if (!h || n_iter < 0) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = h->stream;
  if (lambda || mm0 || mm1) RC(h->ensure_outputs());
  RC(bdd_iterate_device(h, n_iter, nullptr, lambda ? h->d_out_lam : nullptr, mm0 ? h->d_out_m0 : nullptr,
                        mm1 ? h->d_out_m1 : nullptr, s));
  RC(h->begin(s));
  if (lower_bound && n_iter == 0) {
    CK(cudaMemsetAsync(h->d_iter, 0, sizeof(int), s));
    RC(h->pending(true, s));
  }
  const size_t bytes = sizeof(float) * (size_t)h->nnz;
  if (lambda && bytes) CK(cudaMemcpyAsync(lambda, h->d_out_lam, bytes, cudaMemcpyDeviceToHost, s));
  if (mm0 && bytes) CK(cudaMemcpyAsync(mm0, h->d_out_m0, bytes, cudaMemcpyDeviceToHost, s));
  if (mm1 && bytes) CK(cudaMemcpyAsync(mm1, h->d_out_m1, bytes, cudaMemcpyDeviceToHost, s));
  if (lower_bound) {
    const int last = n_iter > 0 ? n_iter - 1 : 0;
    CK(cudaMemcpyAsync(lower_bound, h->d_trace + last, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  RC(h->end(s));
  CK(cudaStreamSynchronize(s));
  return h->take_device_error(s);
}

int bdd_set_costs(bdd_solver *h, const float *c) {
  if (!h || (h->n > 0 && !c)) return BDD_EINVAL;
  if (!finite_costs(c, h->n)) return BDD_EINVAL;
  h->c.assign(c, c + h->n);
  h->empty_const = empty_constant(h->var_deg, c, h->n, h->alpha);
  if (h->host_only) return BDD_OK;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  RC(h->begin(h->stream));
  ++h->state_gen;
  if (h->n) CK(cudaMemcpyAsync(h->d_c, c, sizeof(float) * h->n, cudaMemcpyHostToDevice, h->stream));
  h->drop_graphs();  // the bound constant is baked into the captured reductions
  RC(h->restart(h->stream));
  RC(h->end(h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BDD_OK;
}

int bdd_smooth_forward(bdd_solver *h, int K, const float *d_c, double *d_bound, long long *generation,
                       void *stream) {
  if (!h || K < 1 || (h->n > 0 && !d_c) || !d_bound) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  if (!(h->alpha > 0.f)) return BDD_ESTATE;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  const long long O = h->O, N = h->N;
  if (2 * K > h->smooth_cap) {  // checkpoints of every sweep; the old buffers stay owned by allocs
    RC(h->alloc(&h->ck_lam, 2LL * K * std::max<long long>(O, 1)));
    RC(h->alloc(&h->ck_shr, 2LL * K * std::max<long long>(O, 1)));
    h->smooth_cap = 2 * K;
  }
  if (!h->t_nodeA) {
    RC(h->alloc(&h->t_nodeA, N));
    RC(h->alloc(&h->t_nodeB, N));
    RC(h->alloc(&h->t_gnode, N));
    RC(h->alloc(&h->t_glam0, O));
    RC(h->alloc(&h->t_glam1, O));
    RC(h->alloc(&h->t_gshr, O));
    RC(h->alloc(&h->t_gdelta, O));
    RC(h->alloc(&h->t_delta, O));
    RC(h->alloc(&h->t_E, h->nb));
  }
  RC(h->ensure_trace(K + 1));
  // the messages before the first sweep and after every sweep, when kept: the backward then
  // reads each sweep's starting and final messages instead of recomputing the starting ones
  h->smooth_msgs = false;
  if (h->smooth_messages != 0 && N > 0) {
    const long long count = (2LL * K + 1) * N;
    if (2 * K + 1 <= h->msg_cap) {
      h->smooth_msgs = true;
    } else {
      size_t free_b = 0, total_b = 0;
      const bool fits = h->smooth_messages == 1 ||
                        (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
                         (size_t)count * sizeof(float) <= free_b / 4);
      const int arc = fits ? h->alloc(&h->ck_msg, count) : BDD_ENOMEM;
      if (arc == BDD_OK) {
        h->msg_cap = 2 * K + 1;
        h->smooth_msgs = true;
      } else if (h->smooth_messages == 1) {
        return arc;
      }
    }
  }
  RC(h->begin(s));
  // costs: on the device for the iteration, on the host for the constant of empty variables
  std::vector<float> c(h->n);
  if (h->n) {
    CK(cudaMemcpyAsync(h->d_c, d_c, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c.data(), d_c, sizeof(float) * h->n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!finite_costs(c.data(), h->n)) return BDD_EINVAL;
  }
  h->c = c;
  h->empty_const = empty_constant(h->var_deg, c.data(), h->n, h->alpha);
  h->drop_graphs();
  RC(h->restart(s));
  CK(cudaMemsetAsync(h->d_iter, 0, sizeof(int), s));
  const size_t ob = sizeof(float) * (size_t)std::max<long long>(O, 1);
  const size_t nbytes = sizeof(float) * (size_t)N;
  if (h->smooth_msgs) CK(cudaMemcpyAsync(h->ck_msg, h->d_bm, nbytes, cudaMemcpyDeviceToDevice, s));
  for (int it = 0; it < K; ++it) {
    for (int half = 0; half < 2; ++half) {
      const long long sw = 2LL * it + half;
      if (O) {
        CK(cudaMemcpyAsync(h->ck_lam + sw * O, h->d_lam, ob, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(h->ck_shr + sw * O, h->d_share_occ, ob, cudaMemcpyDeviceToDevice, s));
      }
      RC(h->sweep(half == 0, kUpdate, s));
      if (h->smooth_msgs)
        CK(cudaMemcpyAsync(h->ck_msg + (sw + 1) * N, half == 0 ? h->d_fm : h->d_bm, nbytes,
                           cudaMemcpyDeviceToDevice, s));
      RC(h->pending(half == 1, s));
    }
  }
  CK(cudaMemcpyAsync(d_bound, h->d_trace + (K - 1), sizeof(double), cudaMemcpyDeviceToDevice, s));
  ++h->state_gen;
  h->smooth_gen = h->state_gen;
  h->smooth_K = K;
  if (generation) *generation = h->smooth_gen;
  return h->end(s);
}

int bdd_smooth_backward(bdd_solver *h, long long generation, const double *d_gbound, float *d_grad_c,
                        void *stream) {
  if (!h || !d_gbound || (h->n > 0 && !d_grad_c)) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  // the checkpoints belong to the last forward, and only while nothing has changed the state since
  if (h->smooth_K < 1 || h->smooth_gen != h->state_gen || generation != h->smooth_gen) return BDD_ESTATE;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  const long long O = h->O;
  const int K = h->smooth_K;
  const size_t ob = sizeof(float) * (size_t)std::max<long long>(O, 1);
  RC(h->begin(s));
  // seeds: the slack terms of the last pending sums (and of empty variables), E^j of every BDD
  if (h->n) CK(cudaMemsetAsync(d_grad_c, 0, sizeof(float) * h->n, s));
  CK(cudaMemsetAsync(h->t_gdelta, 0, ob, s));
  CK(cudaMemsetAsync(h->t_glam1, 0, ob, s));
  if (bound_seed_launch(h->d_var_ptr, h->d_P, h->d_c, h->t_gdelta, d_grad_c, h->n, h->alpha, d_gbound, s))
    return BDD_ECUDA;
  float *g_next = h->t_glam1, *g_cur = h->t_glam0;  // adjoint of the multipliers after / before a sweep
  // Every sweep's inputs are its checkpointed multipliers and shares and its starting messages
  // (the backward messages of those multipliers for a forward sweep, the forward messages for a
  // backward sweep); its outputs are the multipliers at the next checkpoint and the messages it
  // writes, which are exactly the next sweep's starting messages.  Walking the sweeps in
  // reverse, each step therefore recomputes only its starting messages (one messages-only
  // sweep from the checkpoint into a scratch buffer) and takes its outputs from the step before:
  // the last sweep's from the solver's final state.  When the forward kept every sweep's
  // messages, nothing is recomputed: sweep sw started from message checkpoint sw and wrote
  // checkpoint sw + 1.
  float *bufs[2] = {h->t_nodeA, h->t_nodeB};
  int xb = 0;
  const long long N = h->N;
  const float *msg_new = h->d_bm, *lam2 = h->d_lam;
  for (long long sw = 2LL * K - 1; sw >= 0; --sw) {
    const bool fwd = (sw % 2) == 0;
    const float *lam_s = h->ck_lam + sw * O, *shr_s = h->ck_shr + sw * O;
    float *pre = h->smooth_msgs ? h->ck_msg + sw * N : bufs[xb];
    SweepParams p = h->sweep_params();
    p.lam = const_cast<float *>(lam_s);  // a messages-only sweep reads the multipliers, never writes them
    p.share_occ = shr_s;
    p.delta = h->t_delta;
    p.bdd_E = h->t_E;
    if (h->smooth_msgs) {
      // kept by the forward
    } else if (fwd) {  // backward messages of the checkpoint (reads fm without using it)
      p.bm = pre;
      p.fm = const_cast<float *>(msg_new);
      if (sweep_launch(false, kMessages, p, h->grid_sweep, s)) return BDD_ECUDA;
    } else {    // forward messages of the checkpoint
      p.fm = pre;
      p.bm = const_cast<float *>(msg_new);
      if (sweep_launch(true, kMessages, p, h->grid_sweep, s)) return BDD_ECUDA;
    }
    AdjParams a{};
    a.sp = h->sweep_params();
    a.lam_s = lam_s;
    a.shr_s = shr_s;
    a.lam2 = lam2;
    a.msg_pre = pre;
    a.msg_new = msg_new;
    a.g_out_lam = g_next;
    a.g_out_delta = h->t_gdelta;
    a.g_in_lam = g_cur;
    a.g_shr = h->t_gshr;
    a.g_node = h->t_gnode;
    a.gE = sw == 2LL * K - 1 ? d_gbound : nullptr;
    if (sweep_adjoint_launch(fwd, a, h->grid_sweep, s)) return BDD_ECUDA;
    // the shares of this sweep were formed from the previous sweep's differences
    if (sw > 0 && pending_adjoint_launch(h->d_var_ptr, h->d_var_occ, h->d_slot_dir,
                                         fwd ? kDirForward : kDirBackward, h->t_gshr, h->t_gdelta, h->n, s))
      return BDD_ECUDA;
    std::swap(g_cur, g_next);
    msg_new = pre;  // this sweep's starting messages are the previous sweep's outputs
    lam2 = lam_s;
    xb ^= 1;
  }
  // lambda_0 = c / |J_i|
  if (initial_adjoint_launch(h->d_var_ptr, h->d_var_occ, g_next, d_grad_c, h->n, s)) return BDD_ECUDA;
  return h->end(s);
}

int bdd_sizes(const bdd_solver *h, long long out[BDD_SIZES_LEN]) {
  if (!h || !out) return BDD_EINVAL;
  out[0] = h->n;
  out[1] = h->m;
  out[2] = h->nb;
  out[3] = h->O;
  out[4] = h->N;
  out[5] = h->max_depth;
  out[6] = h->max_width;
  out[7] = h->nnz;
  out[8] = h->device_bytes;
  out[9] = h->n_warp_tiles;
  out[10] = h->n_block_tiles;
  out[11] = h->schedule;
  out[12] = h->stage_fwd | (h->stage_bwd << 2);
  out[13] = (long long)h->cuts.size();
  out[14] = h->npairs;
  out[15] = h->split_depth;
  out[16] = h->lanes2 ? 1 : 0;
  out[17] = h->lane_O;
  out[18] = h->lane_N;
  return BDD_OK;
}

int bdd_layout_table(const bdd_solver *h, long long *nodes, int *cls, float *ms) {
  if (!h || !nodes || !cls) return BDD_EINVAL;
  for (int k = 0; k < kLayoutKeys; ++k) {
    const int wc = k / kDepthBuckets;
    nodes[k] = h->key_nodes[k];
    int c = h->key_class[k];
    if (c < 0) c = h->lanes2 && wc <= 1 ? 0 : wc;  // the default
    if (h->lanes2 && wc <= 1 && c == 0) c = kWarpClasses + 1;  // lane tiles
    cls[k] = h->key_nodes[k] > 0 ? c : -1;
    if (ms) {
      ms[2 * k] = h->key_ms[k][0];
      ms[2 * k + 1] = h->key_ms[k][1];
    }
  }
  return BDD_OK;
}

int bdd_get_cuts(const bdd_solver *h, int *cuts) {
  if (!h || (!h->cuts.empty() && !cuts)) return BDD_EINVAL;
  std::copy(h->cuts.begin(), h->cuts.end(), cuts);
  return BDD_OK;
}

int bdd_get_copy_duals(const bdd_solver *h_in, float *mu_bar, float *mu) {
  bdd_solver *h = const_cast<bdd_solver *>(h_in);
  if (!h) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  if (h->npairs == 0) return BDD_OK;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = h->stream;
  const size_t pb = sizeof(float) * (size_t)h->npairs;
  RC(h->begin(s));
  if (mu_bar) CK(cudaMemcpyAsync(mu_bar, h->d_mu_bar, pb, cudaMemcpyDeviceToHost, s));
  if (mu) CK(cudaMemcpyAsync(mu, h->d_mu, pb, cudaMemcpyDeviceToHost, s));
  RC(h->end(s));
  CK(cudaStreamSynchronize(s));
  return BDD_OK;
}

int bdd_set_copy_duals(bdd_solver *h, const float *mu_bar, const float *mu) {
  if (!h || (h->npairs > 0 && (!mu_bar || !mu))) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  if (h->npairs == 0) return BDD_OK;
  for (long long k = 0; k < h->npairs; ++k)
    if (!std::isfinite(mu_bar[k]) || !std::isfinite(mu[k])) return BDD_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = h->stream;
  const size_t pb = sizeof(float) * (size_t)h->npairs;
  RC(h->begin(s));
  ++h->state_gen;
  CK(cudaMemcpyAsync(h->d_mu_bar, mu_bar, pb, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->d_mu, mu, pb, cudaMemcpyHostToDevice, s));
  if (cut_roots_launch(h->cut_params(), s)) return BDD_ECUDA;
  RC(h->sweep(false, kMessages, s));
  RC(h->end(s));
  CK(cudaStreamSynchronize(s));
  return BDD_OK;
}

int bdd_export_canonical(const bdd_solver *h, int *bdd_row, int *bdd_depth, int *occ_var, long long *occ_csr,
                         int *occ_width, int *lo, int *hi) {
  if (!h || !bdd_row || !bdd_depth || !occ_var || !occ_csr || !occ_width || !lo || !hi) return BDD_EINVAL;
  if (h->host_only && !h->host_layout) {
    const HostBDDs &H = h->host;
    std::copy(H.bdd_row.begin(), H.bdd_row.end(), bdd_row);
    std::copy(H.bdd_depth.begin(), H.bdd_depth.end(), bdd_depth);
    std::copy(H.occ_var.begin(), H.occ_var.end(), occ_var);
    std::copy(H.occ_csr.begin(), H.occ_csr.end(), occ_csr);
    std::copy(H.occ_width.begin(), H.occ_width.end(), occ_width);
    std::copy(H.lo.begin(), H.lo.end(), lo);
    std::copy(H.hi.begin(), H.hi.end(), hi);
    return BDD_OK;
  }
  // read the slabs back (from the device, or the host copy of the layout) and undo the tiles
  const long long O = h->O, N = h->N, nb = h->nb;
  hvec<int> off(O + 1), var(O), depth(nb), lohi(2 * N);
  hvec<long long> csr(O);
  hvec<unsigned char> code(h->lanes2 ? O : 0);
  if (h->host_layout) {
    const Layout &L = h->layout;
    off = L.occ_node_off;
    var = L.occ_var;
    csr = L.occ_csr;
    depth = L.bdd_depth;
    lohi = L.lohi;
    if (h->lanes2) std::copy(L.lane_code.begin(), L.lane_code.begin() + O, code.begin());
  } else {
    DeviceGuard dg(h->device);
    if (!dg.ok) return BDD_ECUDA;
    CK(cudaEventSynchronize(h->ev_last));
    CK(cudaMemcpy(off.data(), h->d_occ_node_off, sizeof(int) * (O + 1), cudaMemcpyDeviceToHost));
    if (O) {
      CK(cudaMemcpy(var.data(), h->d_occ_var, sizeof(int) * O, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(csr.data(), h->d_occ_csr, sizeof(long long) * O, cudaMemcpyDeviceToHost));
    }
    if (nb) CK(cudaMemcpy(depth.data(), h->d_bdd_depth, sizeof(int) * nb, cudaMemcpyDeviceToHost));
    if (N) CK(cudaMemcpy(lohi.data(), h->d_lohi, sizeof(int) * 2 * N, cudaMemcpyDeviceToHost));
    if (h->lanes2 && O) CK(cudaMemcpy(code.data(), h->d_lane_code, O, cudaMemcpyDeviceToHost));
  }
  // device occurrence of (sorted BDD s, layer l), by the tile rule the kernels use
  std::vector<std::vector<int>> occ_of(nb);
  for (size_t t = 0; t < h->tile_bdd0.size(); ++t) {
    int o = h->tile_occ0[t];
    const int b0 = h->tile_bdd0[t], nt = h->tile_nbdd[t];
    for (int q = 0; q < nt; ++q) occ_of[b0 + q].assign(depth[b0 + q], -1);
    for (int l = 0; l < depth[b0]; ++l)
      for (int q = 0; q < nt && depth[b0 + q] > l; ++q) occ_of[b0 + q][l] = o++;
  }
  // lane tiles: the sweeps read only the lane codes there, so they must give the slabs' node
  // offsets (the layer's nodes BDD by BDD from the tile's running node count) and arcs
  if (h->lanes2) {
    const int n_lane_tiles = h->class_tile_off[1];
    for (int t = 0; t < n_lane_tiles; ++t) {
      const int b0 = h->tile_bdd0[t], nt = h->tile_nbdd[t];
      if (nt < 1 || nt > 32) return BDD_EDEVICE;
      long long node = off[h->tile_occ0[t]];
      for (int l = 0; l < depth[b0]; ++l)
        for (int q = 0; q < nt && depth[b0 + q] > l; ++q) {
          const int o = occ_of[b0 + q][l];
          const unsigned c = code[o];
          const int w = (c >> 4) == (kLaneNoNode1 >> 4) ? 1 : 2;
          if (off[o] != node || off[o + 1] - off[o] != w) return BDD_EDEVICE;
          const long long next0 = l + 1 < depth[b0 + q] ? off[occ_of[b0 + q][l + 1]] : 0;
          for (int k = 0; k < w; ++k)
            for (int a = 0; a < 2; ++a) {
              const int g = lohi[2 * (off[o] + k) + a];
              const unsigned want = g >= 0 ? (unsigned)(g - next0) : g == kTop ? kLaneTop : kLaneBot;
              if (want > kLaneBot || ((c >> (4 * k + 2 * a)) & 3u) != want) return BDD_EDEVICE;
            }
          node += w;
        }
    }
  }
  std::vector<int> sorted_of_canon(nb);
  for (long long s = 0; s < nb; ++s) sorted_of_canon[h->bdd_perm[s]] = (int)s;
  long long co = 0, cn = 0;
  for (long long cb = 0; cb < nb; ++cb) {
    const int s = sorted_of_canon[cb];
    bdd_row[cb] = h->canon_row[cb];
    bdd_depth[cb] = depth[s];
    for (int l = 0; l < depth[s]; ++l, ++co) {
      const int o = occ_of[s][l];
      if (o < 0 || o >= O) return BDD_EDEVICE;
      const int w = off[o + 1] - off[o];
      occ_var[co] = var[o];
      occ_csr[co] = csr[o];
      occ_width[co] = w;
      const int next0 = l + 1 < depth[s] ? off[occ_of[s][l + 1]] : 0;
      for (int q = 0; q < w; ++q, ++cn) {
        if (cn >= N) return BDD_EDEVICE;
        const int g0 = lohi[2 * (off[o] + q)], g1 = lohi[2 * (off[o] + q) + 1];
        lo[cn] = g0 >= 0 ? g0 - next0 : g0;
        hi[cn] = g1 >= 0 ? g1 - next0 : g1;
      }
    }
  }
  return BDD_OK;
}

int bdd_get_state(const bdd_solver *h_in, float *lambda, float *pending) {
  bdd_solver *h = const_cast<bdd_solver *>(h_in);
  if (!h) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = h->stream;
  RC(h->begin(s));
  if (lambda) {
    RC(h->ensure_outputs());
    if (h->nnz) CK(cudaMemsetAsync(h->d_out_lam, 0, sizeof(float) * h->nnz, s));
    if (h->O && scatter_lambda_launch(h->d_lam, h->d_share_occ, h->d_occ_csr, h->d_out_lam, (int)h->O, false,
                                      s))
      return BDD_ECUDA;
    if (h->nnz) CK(cudaMemcpyAsync(lambda, h->d_out_lam, sizeof(float) * h->nnz, cudaMemcpyDeviceToHost, s));
  }
  if (pending && h->n) CK(cudaMemcpyAsync(pending, h->d_P, sizeof(float) * h->n, cudaMemcpyDeviceToHost, s));
  RC(h->end(s));
  CK(cudaStreamSynchronize(s));
  return BDD_OK;
}

int bdd_set_state(bdd_solver *h, const float *lambda, const float *pending) {
  if (!h || !lambda) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = h->stream;
  RC(h->ensure_outputs());
  RC(h->begin(s));
  ++h->state_gen;
  if (h->nnz) CK(cudaMemcpyAsync(h->d_out_lam, lambda, sizeof(float) * h->nnz, cudaMemcpyHostToDevice, s));
  if (h->O && gather_lambda_launch(h->d_out_lam, h->d_occ_csr, h->d_lam, (int)h->O, s)) return BDD_ECUDA;
  if (h->n) {
    if (pending)
      CK(cudaMemcpyAsync(h->d_P, pending, sizeof(float) * h->n, cudaMemcpyHostToDevice, s));
    else
      CK(cudaMemsetAsync(h->d_P, 0, sizeof(float) * h->n, s));
    // slots holding P_i in the first slot of i reproduce P exactly; the pending pass then writes
    // the shares
    if (pending_to_slots_launch(h->d_var_ptr, h->d_P, h->d_delta, h->n, s)) return BDD_ECUDA;
    RC(h->pending(false, s, kDirForward));  // the shares of the next (forward) sweep
  }
  RC(h->sweep(false, kMessages, s));
  RC(h->end(s));
  CK(cudaStreamSynchronize(s));
  return BDD_OK;
}

int bdd_bound_parts(bdd_solver *h, int nparts, const long long *row_off, const long long *var_off, double *out) {
  if (!h || nparts < 1 || !row_off || !var_off || !out) return BDD_EINVAL;
  if (h->host_only) return BDD_ESTATE;
  if (h->npairs > 0) return BDD_EINVAL;  // pieces of one row would share its energy slot
  if (row_off[0] != 0 || var_off[0] != 0 || row_off[nparts] != h->m || var_off[nparts] != h->n) return BDD_EINVAL;
  for (int k = 0; k < nparts; ++k)
    if (row_off[k + 1] < row_off[k] || var_off[k + 1] < var_off[k]) return BDD_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return BDD_ECUDA;
  cudaStream_t s = h->stream;
  if (!h->d_E_row) RC(h->alloc(&h->d_E_row, std::max(h->m, 1)));
  if (nparts > h->part_cap) {
    RC(h->alloc(&h->d_part_off, 2LL * (nparts + 1)));
    RC(h->alloc(&h->d_part_out, nparts));
    h->part_cap = nparts;
  }
  RC(h->begin(s));
  CK(cudaMemcpyAsync(h->d_part_off, row_off, sizeof(long long) * (nparts + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->d_part_off + nparts + 1, var_off, sizeof(long long) * (nparts + 1), cudaMemcpyHostToDevice,
                     s));
  if (part_bounds_launch(h->d_bdd_E, h->d_bdd_row, (int)h->nb, h->d_E_row, h->m, h->d_part_off,
                         h->d_part_off + nparts + 1, nparts, h->d_var_ptr, h->d_P, h->d_c, h->d_part_out, s))
    return BDD_ECUDA;
  CK(cudaMemcpyAsync(out, h->d_part_out, sizeof(double) * nparts, cudaMemcpyDeviceToHost, s));
  RC(h->end(s));
  CK(cudaStreamSynchronize(s));
  return BDD_OK;
}

int bdd_status_of_device_word(int word) {
  if (word == 0) return BDD_OK;
  return word == BDD_EDEVICE ? BDD_EDEVICE : BDD_ETIMEOUT;
}

const char *bdd_strerror(int code) {
  switch (code) {
    case BDD_OK: return "ok";
    case BDD_EINVAL: return "invalid argument or malformed instance";
    case BDD_EINFEASIBLE: return "a constraint row has no 0-1 solution";
    case BDD_ETOOBIG: return "a BDD or the instance exceeds the size limits";
    case BDD_ENOMEM: return "out of host or device memory (or over max_device_bytes)";
    case BDD_ECUDA: return "CUDA runtime error";
    case BDD_ETIMEOUT: return "device-side wait gave up";
    case BDD_EDEVICE: return "device-side check failed";
    case BDD_ESTATE: return "call not valid in the solver's state (host-only solver, or no matching smoothed forward)";
    default: return "unknown status";
  }
}

void bdd_free(bdd_solver *h) {
  if (!h) return;
  if (h->host_only) {
    delete h;
    return;
  }
  DeviceGuard dg(h->device);
  delete h;
}

}  // extern "C"
