// Internal declarations shared by the host compiler, the layout builder, the kernels and the
// C ABI.  Not installed; the public interface is include/bdd_dbca.h.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <memory>
#include <utility>
#include <vector>

namespace bdd {

// Host arrays of the compiled BDDs and of the slab layout: std::vector with an allocator whose
// resize leaves new elements uninitialised (value-initialisation is skipped), so the multi-GB
// arrays are first written -- and their pages first touched -- by the parallel loops that fill
// them instead of being zeroed by one thread beforehand.  Code that needs a value writes it.
template <class T>
struct UninitAlloc {
  using value_type = T;
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U> &) {}
  T *allocate(std::size_t n) { return std::allocator<T>().allocate(n); }
  void deallocate(T *p, std::size_t n) { std::allocator<T>().deallocate(p, n); }
  template <class U>
  void construct(U *p) noexcept {
    ::new (static_cast<void *>(p)) U;  // default-initialisation: nothing for arithmetic types
  }
  template <class U, class... A>
  void construct(U *p, A &&...a) {
    ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
  }
  template <class U>
  bool operator==(const UninitAlloc<U> &) const { return true; }
  template <class U>
  bool operator!=(const UninitAlloc<U> &) const { return false; }
};
template <class T>
using hvec = std::vector<T, UninitAlloc<T>>;

constexpr int kTop = -1;   // arc into the true terminal
constexpr int kBot = -2;   // arc into the false terminal
constexpr int kNone = -3;  // no arc (lane without a node)
// Sub-BDDs (Sec. 6): an arc that crosses a cut ends in the top terminal as the copy arc of
// copy-arc pair k, encoded as kCopy0 - k; its backward message is the pair's dual mu_bar.
constexpr int kCopy0 = -4;

// Canonical host form of all BDDs (Sec. 5.1, Def. 4): BDDs in ascending row order;
// occurrences (row j, variable i) BDD-major, layer-minor; nodes BDD-major, layer-major,
// ascending smallest partial sum inside a layer; lo/hi are ids inside the next layer.
struct HostBDDs {
  int n = 0, m = 0;
  long long nnz = 0;
  hvec<int> bdd_row, bdd_depth;
  hvec<long long> bdd_occ0;   // [nb+1]
  hvec<int> occ_var;          // [O]
  hvec<long long> occ_csr;    // [O]
  hvec<int> occ_width;        // [O]
  hvec<long long> occ_node0;  // [O+1]
  hvec<int> lo, hi;           // [N]
  int max_depth = 0, max_width = 0;
  long long nb() const { return (long long)bdd_row.size(); }
  long long O() const { return (long long)occ_var.size(); }
  long long N() const { return (long long)lo.size(); }
};

// Copy-arc pairs of a split (Sec. 6, Def. of sub-BDDs and copy-arcs), in canonical order: cuts
// of BDD 0 by ascending layer, then BDD 1, ...; inside a cut, tails in node order, the 0-arc
// before the 1-arc.  Pair k joins the copy arc (tail node of the earlier piece's last layer, into
// top) with the arc entering the head node of the later piece's first layer.
struct CopyPairs {
  std::vector<int> cuts;            // places in the variable order where intervals 2.. start
  std::vector<long long> cut_ptr;   // [groups + 1] pairs of each cut of a BDD
  std::vector<long long> tail_occ;  // [groups] canonical occurrence of the tails' layer
  std::vector<int> tail, side;      // [pairs] tail node id inside that layer; 0-arc / 1-arc
  std::vector<int> head;            // [pairs] head node id inside the next layer
  long long npairs() const { return (long long)tail.size(); }
  long long ngroups() const { return (long long)tail_occ.size(); }
};

// k - 1 cut places that give every interval of the variable order about N / k nodes (a node
// counts for the interval of its layer's variable; Sec. 6 chooses the interval endpoints so).
std::vector<int> balanced_cuts(const HostBDDs &H, const int *rank, int k);

// Splits every BDD of H in place into its sub-BDDs: with depth == 0 at the interval boundaries
// `cuts` (ascending places in [1, n); rank: the variable order, null = index order), with
// depth D > 0 into pieces of at most D layers (a BDD of k layers is cut before layers
// floor(t k / q), t = 1 .. q-1, q = ceil(k / D)).  Each piece becomes a BDD of its own (bdd_row
// keeps the row); the arcs of the last layer before a cut become copy codes kCopy0 - k.
// Returns a BDD_* status.
int split_bdds(HostBDDs &H, const int *rank, const std::vector<int> &cuts, int depth, CopyPairs *P);

// Runs body(begin, end) over [0, n) in chunks of `grain` items, on the library's host worker
// threads (created on first use, one per hardware thread but the caller's, kept until the
// process exits) together with the calling thread.  One job runs on the workers at a time; a
// call that finds them busy (a solver being built on another host thread) runs inline.
void parallel_for(long long n, long long grain, const std::function<void(long long, long long)> &body);

// Compiles every row (threshold counting over suffix-sum sets; see compile.cpp).
// Returns a BDD_* status; *failed_row is the row that failed, or -1.
int compile_bdds(int n, int m, const long long *row_ptr, const int *col, const int *val,
                 const int *b, const signed char *sense, const int *rank, int max_width,
                 long long max_nodes, HostBDDs *out, int *failed_row);

// SRMP membership bits of a slot (Appendix A.4): the occurrence takes a share in a forward
// sweep (it is in J_i^>: not the last layer of its BDD) / a backward sweep (J_i^<: not the first).
constexpr unsigned char kDirForward = 1;
constexpr unsigned char kDirBackward = 2;

// Team classes of the sweep kernels.  Class c < kWarpClasses: a team of T = 1 << c lanes per
// BDD (lane t holds node t of the current layer), 32 / T BDDs per warp ("warp tile").
// Class kWarpClasses: one 128-thread group per BDD ("block tile").
constexpr int kWarpClasses = 6;
constexpr int kBlockThreads = 128;                  // per-phase kernels; block-tile group size
constexpr int kWarpsPerBlock = kBlockThreads / 32;
constexpr int kPersistThreads = 512;                // persistent kernel: one block per SM
constexpr int kPersistWarps = kPersistThreads / 32;
constexpr int kSubBlocks = kPersistThreads / kBlockThreads;
constexpr int kMaxBlockTileWidth = 12288;           // two float layer buffers in shared memory
constexpr int kMaxBlockTileDepth = 8192;

// Shared-memory stage of one warp: a window of kWinLayers layers of a warp tile (at most 32
// occurrences and 32 nodes per layer), plus the node offsets and backward messages of the layer
// after the window.  Each warp has kWarpStages of them (the next window loads while one is
// processed).
constexpr int kWinLayers = 4;
constexpr int kWarpStages = 2;
constexpr int kWinOcc = 32 * kWinLayers;
constexpr int kWinNodes = 32 * kWinLayers;
// Arrays are filled by bulk copies that start at the 16-byte boundary at or below the window's
// first element, hence the few spare elements; every array starts 16-byte aligned.
struct alignas(16) WarpStage {
  int2 lohi[kWinNodes + 2];
  float msg[kWinNodes + 32 + 4];
  int off[kWinOcc + 8];
  float lam[kWinOcc + 4];
  float shr[kWinOcc + 4];
  int slot[kWinOcc + 4];
};

// The 8-layer window of the cp.async staging variant (one buffer per warp).
constexpr int kWin8Layers = 8;
constexpr int kWin8Occ = 32 * kWin8Layers;
constexpr int kWin8Nodes = 32 * kWin8Layers;
struct alignas(16) WarpStage8 {
  int2 lohi[kWin8Nodes];
  float msg[kWin8Nodes + 32];
  int off[kWin8Occ + 32 + 1];
  float lam[kWin8Occ];
  float shr[kWin8Occ];
  int slot[kWin8Occ];
};
// shared memory of one warp: the larger of the bulk-copy ring and one 8-layer window (staging
// variants 0 and 1); two 8-layer windows for the double-buffered variant 2, whose launches get
// their own shared-memory size
constexpr size_t kWarpSmemBytes = (kWarpStages * sizeof(WarpStage) > sizeof(WarpStage8) ? kWarpStages * sizeof(WarpStage)
                                                                                          : sizeof(WarpStage8));
constexpr size_t kWarpSmemBytes2 = 2 * sizeof(WarpStage8);

// Lane tiles (layouts built with lanes2): BDDs whose layers have at most two nodes, one lane per
// BDD, 32 BDDs per tile (warp class 0).  A window holds kWinLayers layers of up to 64 nodes each
// (plus the layer after it for the backward messages of a forward update); two per warp, filled
// by the bulk-copy ring.  A warp takes a run of up to kLaneRunMax consecutive lane tiles and
// streams their windows through its two buffers.
//
// The arcs of a lane tile's layer are one byte per occurrence (lane code) instead of node
// offsets and an int2 per node: bits 4t..4t+1 hold the 0-arc and bits 4t+2..4t+3 the 1-arc of
// node t (t = 0, 1), each as 0 or 1 (that node of the BDD's next layer), kLaneTop or kLaneBot.  A layer with one node has node 1's arcs both kLaneBot, which no
// node of a reduced BDD has (every node has a path to the true terminal).  A layer's nodes follow
// the tile's layer-major order (BDD by BDD, the BDDs alive at the layer being a prefix of the
// tile), so the kernels find a lane's first node from the widths of the lanes before it.
constexpr int kLaneRunMax = 4;  // lane tiles per warp (longer runs measured no faster)
constexpr int kLaneWinNodes = 64 * kWinLayers;
constexpr unsigned kLaneTop = 2, kLaneBot = 3;
constexpr unsigned kLaneNoNode1 = 0xF0u;  // node 1's arcs of a one-node layer: both kLaneBot
constexpr int kLaneCodePad = 64;          // spare codes after the last occurrence (read, unused)
struct alignas(16) LaneStage {
  float msg[kLaneWinNodes + 64 + 4];
  float lam[kWinOcc + 4];
  float shr[kWinOcc + 4];
  int slot[kWinOcc + 4];
  unsigned char code[kWinOcc + 32 + 16];  // the window's occurrences and the layer after it
};
constexpr size_t kLaneSmemBytes = kWarpStages * sizeof(LaneStage);
constexpr int kStagings = 3;  // warp-tile staging variants of the update sweeps

// Device slab layout (host staging copy).  Occurrences are grouped by tile; inside a warp
// tile they are layer-major (layer l of every tile BDD still alive at l, in tile order; the
// tile's BDDs are sorted by depth, longest first, so the BDDs alive at l are a prefix).  Nodes
// follow their occurrence.  Successors are global node indices or kTop / kBot.  Recorded
// differences live in variable-major "slots": slot k in [var_ptr[i], var_ptr[i+1]) belongs to
// the occurrences of variable i in ascending row order.
struct Layout {
  int n_sorted = 0;                    // BDDs in sorted (device) order
  hvec<int> bdd_perm;           // sorted position -> canonical BDD index
  hvec<int> bdd_depth;          // [nb] sorted order
  hvec<int> occ_node_off;       // [O+1]
  hvec<int> occ_var;            // [O]
  hvec<long long> occ_csr;      // [O]
  hvec<int> occ_slot;           // [O] slot of the occurrence
  hvec<int> lohi;               // [2N] interleaved lo, hi
  hvec<unsigned char> lane_code;  // [O + kLaneCodePad] arcs of lane-tile layers (0 elsewhere)
  hvec<int> tile_occ0, tile_bdd0, tile_nbdd;  // per tile
  hvec<int> tile_win0;                        // [ntiles + 1] window table offsets (warp tiles)
  hvec<int> win_node;                         // window table, int pairs
  int class_tile_off[kWarpClasses + 2] = {0};        // tiles of class c: [off[c], off[c+1])
  bool lanes2 = false;                               // class 0 = lane tiles of width <= 2
  int n_warp_tiles = 0, n_block_tiles = 0;
  int max_block_width = 0;
  hvec<int> var_ptr;            // [n+1]
  hvec<int> var_occ;            // [O] device occurrence of each slot
  hvec<unsigned char> slot_dir; // [O] kDirForward / kDirBackward bits of each slot
  hvec<int> occ_of_canon;       // canonical occurrence -> device occurrence
};

// Keys of the layout tuner: a BDD's natural class (the smallest team of 2^c >= its widest
// layer, c < kWarpClasses; kWarpClasses for block tiles) and its depth bucket (<= 8, <= 32,
// <= 128, longer).
constexpr int kDepthBuckets = 4;
constexpr int kLayoutKeys = (kWarpClasses + 1) * kDepthBuckets;
inline int natural_class(int width) {
  if (width > 32) return kWarpClasses;
  int c = 0;
  while ((1 << c) < width) ++c;
  return c;
}
inline int depth_bucket(int depth) { return depth <= 8 ? 0 : depth <= 32 ? 1 : depth <= 128 ? 2 : 3; }
inline int layout_key(int width, int depth) { return natural_class(width) * kDepthBuckets + depth_bucket(depth); }

// lanes2: BDDs of width <= 2 may form the lane tiles of class 0 (32 BDDs per tile, one lane
// each).  class_of_key (kLayoutKeys entries, or null): the class each key's BDDs go to, -1 for
// the default (class 0 = lane tiles for width <= 2 when lanes2, else the natural class).  A
// class must fit the key: a team of 2^c >= the width, a block tile, or lane tiles (width <= 2,
// lanes2).  Returns BDD_EINVAL otherwise.  var_deg (H.n entries, or null): the number of
// occurrences of every variable in H.occ_var, if the caller has counted them already.
int build_layout(const HostBDDs &H, Layout *L, bool lanes2 = false, const int *class_of_key = nullptr,
                 const int *var_deg = nullptr);

// Fused pending pass of an update sweep (the per-phase plan without separate pending kernels).
// At the end of its tile every occurrence counts its variable down; the visit that brings the
// count to zero is the variable's last in this sweep, so all of its slots are final: it forms
// P_i, writes the shares of the next sweep and resets the count.  A forward sweep may also
// reduce the FP64 bound of the previous iteration from the backward sweep's E^j and slack terms.
struct FusedParams {
  int *cnt;                       // [n] visits of i still to come in this sweep; null: no fused pass
  const int *occ_var;             // [O]
  const int *var_ptr;             // [n + 1]
  const int *var_occ;             // [O]
  float *P;                       // [n] pending sums
  float *share;                   // [O] shares of the next sweep (the sweep's share_occ buffer)
  const unsigned char *slot_dir;  // SRMP membership bits per slot, or null
  double *slk;                    // [n] slack term of each variable's pending sum (backward sweeps)
  int bound;                      // forward sweep: reduce the previous iteration's bound first
  double *partial;                // [gridDim.x] per-block partial sums of the bound
  unsigned *ticket;
  int *iter_ctr;
  double *trace;
  int trace_cap;
  int n;
  int nb;
  double empty_const;
};

// Kernel parameter blocks (passed by value).
struct SweepParams {
  const int *occ_node_off;
  const long long *occ_csr;
  const int2 *lohi;
  const unsigned char *lane_code;  // lane tiles: one byte of arcs per occurrence (see LaneStage)
  float *fm;
  float *bm;
  float *lam;
  const int *occ_slot;      // slot of each occurrence (variable-major)
  float *delta;             // differences recorded by a sweep, by slot
  const float *share_occ;   // pending share P_i / |J_i| of each occurrence's variable
  const int *bdd_depth;
  float *bdd_E;
  const int *tile_occ0;
  const int *tile_win0;     // first window-table entry of each warp tile
  const int2 *win_node;     // window table: {node at layer w * kWinLayers, node at layer
                            // min((w + 1) * kWinLayers + 1, maxd)} for w = 0 .. windows
  const int *tile_bdd0;
  const int *tile_nbdd;
  float *out_m0;
  float *out_m1;
  int class_tile_off[kWarpClasses + 2];
  int n_warp_blocks;
  int lanes2;           // class-0 tiles are lane tiles (one lane per BDD of width <= 2)
  int lane_run;         // lane tiles per warp (consecutive, at most kLaneRunMax)
  int n_lane_warps;     // warps that take lane tiles: ceil(lane tiles / lane_run)
  int warp_smem;        // bytes of dynamic shared memory per warp of a warp block
  int block_buf;        // floats per shared-memory layer buffer of a block tile
  int block_depth_buf;  // floats for the per-layer shares of a block tile
  float omega;
  float alpha;          // smoothing temperature (0: min-sum)
  float inv_alpha;
  const float *copy_val; // sub-BDDs: mu_bar of every copy-arc pair (backward message of kCopy0 - k)
  int split;             // sub-BDDs: layer-0 forward messages are the root messages held in fm, and
                         // E^j is the minimum over the first layer of fm + bm
  // deferred bound of the previous iteration (forward update sweeps of the per-phase plan): the
  // per-block partials its pending pass left, summed in a fixed order by one warp of the
  // sweep's last warp block (its shallowest tiles) into fin_trace[*fin_iter]; null: nothing
  const double *fin_partial;
  int fin_nblocks;
  int *fin_iter;
  double *fin_trace;
  int fin_cap;
  double fin_const;
  int *error;            // set to BDD_ETIMEOUT if a bounded wait on a shared-memory copy gives up
                         // (a fixed time limit, kRingWaitNs in kernels.cu); to BDD_EDEVICE by a
                         // failed index check of the checked build
  long long n_nodes, n_occ, n_csr, n_bdd;  // array extents for the checked build's index checks
  FusedParams fz;       // fz.cnt == null outside the fused plan
  int pdl_early;        // 1: let the next kernel launch when this one starts; 0: as blocks exit
};

// Sweep modes.
enum SweepMode : int {
  kUpdate = 0,   // add the pending share, take min-marginals, move lambda, record delta
  kMessages = 1, // messages only (no share, no update); backward form also records E^j
  kFolded = 2,   // messages and min-marginals at lambda + share, nothing stored but messages
  kUpdateFused = 3,  // kUpdate plus the fused pending pass (SweepParams::fz)
};
__host__ __device__ constexpr bool is_update(int mode) { return mode == kUpdate || mode == kUpdateFused; }

// Pending pass: P_i = sum of i's slots, stored; share_i = P_i / |J_i| written to each of i's
// occurrences; optionally the FP64 y-slack bound sum_j E^j + sum_i min(0, P_i) + empty_const,
// reduced deterministically (per-block partials finished in block order by the last block)
// into trace[*iter_ctr].
struct PendingParams {
  const int *var_ptr;
  const int *var_occ;
  const float *delta;
  float *P;
  float *share_occ;
  const float *bdd_E;
  double *partial;
  unsigned *ticket;
  int *iter_ctr;
  double *trace;
  int trace_cap;
  int n;
  int nb;
  double empty_const;
  double alpha;  // smoothing temperature of the slack term (0: min-sum)
  const unsigned char *slot_dir;  // SRMP membership bits per slot, or null (eq. mma-update)
  int next_dir;                   // kDirForward / kDirBackward: the sweep the shares are for
  int defer;                      // bound: leave the per-block partials for the next forward sweep
                                  // (or bound_finish_launch) instead of finishing them here
  const int4 *heavy;              // variables with more than heavy_deg occurrences: {i, first slot,
  int n_heavy;                    // end slot, 0}, handled by one warp each
  int heavy_deg;
  int pdl_early;                  // as in SweepParams
};

// Persistent iteration kernel (one cooperative launch runs n_iter iterations).
struct IterParams {
  SweepParams sp;
  const int *var_ptr;
  const int *var_occ;
  float *P;             // pending sums (state)
  float *share_occ;     // shares written by the pending passes (sp.share_occ, writable)
  double *part;         // [2][gridDim.x] bound partials: E^j parts, slack parts
  unsigned *barrier;    // [2] arrival count, generation
  int *error;           // set to BDD_ETIMEOUT if a barrier wait gives up
  double *trace;
  int trace_cap;
  int n_iter;
  int n;
  double empty_const;
  long long spin_limit;
  const unsigned char *slot_dir;  // SRMP membership bits per slot, or null (eq. mma-update)
  const int4 *heavy;              // as in PendingParams
  int n_heavy;
  int heavy_deg;
};

// Adjoint of one smoothed update sweep (adjoint.cu): checkpointed inputs, recomputed outputs and
// messages, output adjoints in, input adjoints out.
struct AdjParams {
  SweepParams sp;
  const float *lam_s;        // multipliers at the sweep's start (checkpoint)
  const float *shr_s;        // shares the sweep added (checkpoint)
  const float *lam2;         // multipliers after the sweep (recomputed)
  const float *msg_pre;      // starting backward (forward sweep) / forward (backward sweep) messages
  const float *msg_new;      // messages the sweep computed: fm (forward) / bm (backward)
  const float *g_out_lam;    // adjoint of the multipliers after the sweep
  const float *g_out_delta;  // adjoint of the recorded differences, by slot
  float *g_in_lam;           // adjoint of the multipliers at the sweep's start
  float *g_shr;              // adjoint of the shares
  float *g_node;             // per-node scratch
  const double *gE;          // adjoint of every BDD's root message (the last backward sweep), or null
};

int sweep_adjoint_launch(bool forward, const AdjParams &a, int grid, cudaStream_t stream);
int pending_adjoint_launch(const int *var_ptr, const int *var_occ, const unsigned char *slot_dir, int dir,
                           const float *g_shr, float *g_delta, int n, cudaStream_t stream);
int bound_seed_launch(const int *var_ptr, const float *P, const float *c, float *g_delta, float *g_c, int n,
                      float alpha, const double *g_bound, cudaStream_t stream);
int initial_adjoint_launch(const int *var_ptr, const int *var_occ, const float *g_lam0, float *g_c, int n,
                           cudaStream_t stream);

// Copy-arc dual updates of a split solver (Sec. 6, parallel min-marginal averaging), one warp per
// cut of a BDD.  After a forward sweep: m_k = fm(tail) + theta(tail arc) + mu_bar_k, d_fwd =
// m_k - min over the cut, mu_bar_k += -gamma d_fwd + gamma d_bwd.  After a backward sweep:
// m_k = mu_k + bm(head), d_bwd likewise, mu_k += -gamma d_bwd + gamma d_fwd, then every head
// node's root message (in fm) = min of mu over the pairs entering it.
struct CutParams {
  const int4 *grp;        // [ngroups] {first pair, end pair, first head, end head}
  const int4 *pair;       // [npairs] {tail node, head node, tail occurrence, side}
  const int *head_node;   // [heads] device node of each head
  const int *head_ptr;    // [heads + 1] pairs entering each head ...
  const int *head_pair;   // ... listed here
  float *mu_bar, *mu, *dfwd, *dbwd;  // [npairs]
  float *fm;
  const float *bm;
  const float *lam;
  float gamma;
  int ngroups;
};
int cut_launch(bool forward, const CutParams &c, cudaStream_t stream);
// root messages only (after the duals were set): fm(head) = min of mu over its pairs
int cut_roots_launch(const CutParams &c, cudaStream_t stream);

// Launch wrappers (kernels.cu).  All enqueue on `stream` and return 0 or -5 (launch failure).
size_t sweep_smem_bytes(int block_buf, int block_depth_buf, int staging = 0, bool lanes2 = false,
                        bool smooth = false);
size_t sweep_warp_smem(int staging, bool lanes2);
int sweep_resident_blocks(size_t smem, int *blocks);  // blocks of a sweep launch per SM
size_t persist_smem_bytes(int block_buf, int block_depth_buf);
int sweep_set_smem(size_t bytes);
int iterate_set_smem(size_t bytes);
// staging: warp-tile window staging of a plain update sweep (0: bulk-copy ring, 1: 8-layer
// cp.async windows, 2: the same double-buffered); other modes always use the ring
int sweep_launch(bool forward, int mode, const SweepParams &p, int grid, cudaStream_t stream, int staging = 0);
int pending_launch(bool bound, const PendingParams &p, int grid, cudaStream_t stream);
// FP64 bound from the E^j and slack terms of the last fused backward sweep into trace[*iter_ctr]
int bound_launch(const SweepParams &p, int grid, cudaStream_t stream);
// finishes a deferred bound (partials of a pending pass with defer) into trace[*iter_ctr]
int bound_finish_launch(const double *partial, int nblocks, int *iter_ctr, double *trace, int cap,
                        double empty_const, cudaStream_t stream);
int iterate_persistent_max_grid(size_t smem, int *grid);
int iterate_persistent_launch(const IterParams &q, int grid, size_t smem, cudaStream_t stream);
int init_lambda_launch(const int *occ_var, const int *var_ptr, const float *c, float *lam, int O,
                       cudaStream_t stream);
int pending_to_slots_launch(const int *var_ptr, const float *P, float *delta_b, int n, cudaStream_t stream);
int scatter_lambda_launch(const float *lam, const float *share_occ, const long long *occ_csr, float *out,
                          int O, bool fold, cudaStream_t stream);
int gather_lambda_launch(const float *in, const long long *occ_csr, float *lam, int O,
                         cudaStream_t stream);
// per-part bounds: E scattered to rows, then one block per part sums its rows and variables
int part_bounds_launch(const float *bdd_E, const int *bdd_row, int nb, float *E_row, int m, const long long *row_off,
                       const long long *var_off, int nparts, const int *var_ptr, const float *P, const float *c,
                       double *out, cudaStream_t stream);
constexpr int kReduceThreads = 256;

}  // namespace bdd
