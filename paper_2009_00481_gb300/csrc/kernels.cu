// Sweep, bound and helper kernels for BDD min-marginal averaging on sm_103a.
//
// One iteration = forward sweep, then backward sweep (Sec. 3.2 Alg. 1's forward and backward
// pass, in the parallel-across-BDDs form: every BDD runs its layers in order, all BDDs at
// once; the averaging term of eq. mma-update is applied one sweep late).  Each occurrence
// records its damped min-marginal difference in a variable-major slot; when the next sweep
// visits the occurrence it adds share_i = (sum of the variable's slots) / |J_i|, which is the
// pending sum P_i / |J_i| of the deferred schedule.
//
// Sweeps walk each BDD's layers inside one team of threads with no grid synchronisation inside
// a sweep.  Warp tiles stage windows of their contiguous slab in shared memory and keep the
// current layer's messages in registers (lane t of a T-lane team holds node t; the forward step
// pushes along lo/hi arcs with shuffles, the backward step pulls successors' messages with one
// shuffle each).  Block tiles (layers wider than 32 nodes) keep two layer buffers in shared
// memory (forward step by shared-memory atomic minimum).  Forward messages are written for the
// backward sweep and backward messages for the next forward sweep (Prop. 3: every message
// stays valid for the layers not yet revisited).
//
// Two schedules run this arithmetic: per-phase kernels (forward sweep, backward sweep, bound)
// replayed from CUDA graphs, and one persistent cooperative kernel per call with two grid
// barriers per iteration.
#include <cuda_runtime.h>

#include "internal.h"
#include "device_common.cuh"

namespace bdd {

namespace {

// backward message of a terminal arc target t < 0: top -> 0, bot / none -> +inf; the copy arc of
// pair k (t = kCopy0 - k, sub-BDDs of Sec. 6) enters top at cost mu_bar_k
// (SPLIT: instantiated for split solvers only, so the unsplit sweeps carry no copy-arc code)
template <bool SPLIT>
__device__ __forceinline__ float terminal_bm(const float *__restrict__ copy_val, int t) {
  if (t == kTop) return 0.f;
  if (!SPLIT) return inf();
  return t > kCopy0 ? inf() : copy_val[kCopy0 - t];
}

// backward message of an arc target: node -> bm, else the terminal's
template <bool SPLIT>
__device__ __forceinline__ float target_bm(const float *__restrict__ bm, const float *__restrict__ copy_val, int t) {
  return t >= 0 ? bm[t] : terminal_bm<SPLIT>(copy_val, t);
}

// backward message of an arc target staged at msg[t - base]
template <bool SPLIT>
__device__ __forceinline__ float staged_bm(const float *msg, const float *__restrict__ copy_val, int base, int t) {
  return t >= 0 ? msg[t - base] : terminal_bm<SPLIT>(copy_val, t);
}

// atomic minimum on a float in shared memory (non-negative floats order like their int bits,
// negative ones reverse-order like their unsigned bits)
__device__ __forceinline__ void atomic_min_f(float *addr, float v) {
  if (v >= 0.f)
    atomicMin(reinterpret_cast<int *>(addr), __float_as_int(v));
  else
    atomicMax(reinterpret_cast<unsigned *>(addr), __float_as_uint(v));
}

__device__ __forceinline__ float mm_difference(float m0, float m1) {
  // a +inf min-marginal (a row forcing x_i) transfers nothing
  return (m0 < inf() && m1 < inf()) ? m1 - m0 : 0.f;
}

// Asynchronous global -> shared copies (cp.async): a warp issues all copies of a stage back to
// back and waits once, instead of one load round trip per element.  Data written by other
// blocks of a persistent launch is read only after a grid barrier, whose fences order those
// writes before these reads.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Programmatic dependent launch: the per-phase kernels are launched so that the next kernel of
// the chain may start while this one drains; each kernel waits here for its predecessor to
// complete (and its writes to be visible) before touching any data, and lets its own successor
// start launching right away.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// barrier of the 128-thread group `group` (named barrier 1 + group; the per-phase kernel's
// blocks are one such group)
__device__ __forceinline__ void group_sync(int group) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "r"(kBlockThreads) : "memory");
}

// Where a sweep records its differences (variable-major slots).
struct Phase {
  float *delta;
};

// Sum of slots [s, e) in ascending order -- the one summation every pending sum uses.  Loads
// go out eight at a time (independent, through L2: during a persistent launch the slots are
// written by other blocks); the additions stay in slot order.
__device__ __forceinline__ float slot_sum(const float *__restrict__ d, int s, int e) {
  float P = 0.f;
  for (int k = s; k < e; k += 8) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = k + j < e ? __ldcg(d + k + j) : 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k + j < e) P += v[j];
  }
  return P;
}

// y-slack term of one variable: min(0, P) for min-sum, its soft minimum for alpha > 0.  P is an
// FP32 pending sum; the soft term's log1p and exp run in FP32 (on this part an FP64 log1p/exp per
// variable costs more than the pending pass itself) and the term enters the bound's FP64 sum.
__device__ __forceinline__ double slack_term(float P, float alpha) {
  const float m = fminf(P, 0.f);
  if (alpha <= 0.f) return (double)m;
  return (double)(m - alpha * log1pf(expf(-fabsf(P) / alpha)));
}

// A thread's share of the bound: FP32 terms summed without FP64 arithmetic per term (this
// part's FP64 rate is 1/64 of its FP32 rate, and a pending pass with one FP64 add per variable
// and per BDD ran 0.2 ms longer per pass on the 256-instance Potts batch).  Terms of magnitude
// below 2^100 go into hi with Knuth's TwoSum, whose exact rounding error goes into lo; the
// others (and infinities, NaN) straight into lo, where they dwarf the rounding errors (and
// propagate as an FP64 sum would).  Otherwise hi + lo is the sum of the terms up to the
// roundings of the additions into lo: an error below k^2 * 2^-48 of the summed magnitudes for
// k terms (about 3e-10 for the few hundred terms a thread takes), far below the FP32 rounding
// of the terms themselves.  The threads' values are then summed in FP64.
struct BoundSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    if (!(fabsf(x) < 0x1p100f)) {
      lo += x;
      return;
    }
    const float t = hi + x;
    const float xv = t - hi;  // TwoSum: t + err = hi + x exactly
    const float err = (hi - (t - xv)) + (x - xv);
    hi = t;
    lo += err;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// the y-slack term of P: min(0, P) for min-sum (only a negative P adds anything), its soft
// minimum for alpha > 0, in FP32 either way
template <bool SMOOTH>
__device__ __forceinline__ void add_slack(BoundSum &acc, float P, float alpha) {
  if (SMOOTH) {
    const float m = fminf(P, 0.f);
    acc.add(m - alpha * log1pf(expf(-fabsf(P) / alpha)));
  } else if (P < 0.f) {
    acc.add(P);
  }
}

// the general path of pending_var for slots [s, e) of variable i
__device__ __forceinline__ float pending_tail_sum(const float *__restrict__ delta, const int *__restrict__ var_occ,
                                                  float *__restrict__ P, float *__restrict__ share_occ, int i, int s,
                                                  int e, const unsigned char *__restrict__ slot_dir, int dir) {
  const float Pi = slot_sum(delta, s, e);
  if (P) P[i] = Pi;
  if (slot_dir) {
    int cnt = 0;
    for (int k = s; k < e; ++k) cnt += (slot_dir[k] & dir) != 0;
    if (cnt > 0) {
      const float share = Pi / (float)cnt;
      for (int k = s; k < e; ++k) share_occ[var_occ[k]] = (slot_dir[k] & dir) ? share : 0.f;
      return Pi;
    }
  }
  const float share = Pi / (float)(e - s);
  for (int k = s; k < e; k += 8) {  // occurrence ids eight at a time, then the stores
    int o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = k + j < e ? var_occ[k + j] : -1;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (o[j] >= 0) share_occ[o[j]] = share;
  }
  return Pi;
}

// Pending sums (the sum in eq. mma-update, deferred): P_i = sum of i's slots in ascending
// order, stored (unless P is null), and share_i = P_i / |J_i| written to each of i's occurrences
// for the next sweep.
// With SRMP bits (Appendix A.4), P_i / |J_i^dir| to the slots in J_i^dir and 0 to the others,
// unless J_i^dir is empty (then P_i / |J_i| to all).
// FAST > 0: one round of loads for variables with at most FAST occurrences (slots, occurrence
// ids and SRMP bits together); FAST = 0: slot_sum, then the occurrence ids eight at a time.
// SKIP_HEAVY: variables with more than heavy_deg occurrences are left to pending_var_warp
// (has = false for them).
// (pending_var_se: the same for a variable whose slot range [s, e) the caller has loaded)
template <int FAST, bool SKIP_HEAVY = false>
__device__ __forceinline__ float pending_var_se(const float *__restrict__ delta, const int *__restrict__ var_occ,
                                                float *__restrict__ P, float *__restrict__ share_occ, int i, int s,
                                                int e, bool &has, const unsigned char *__restrict__ slot_dir, int dir,
                                                int heavy_deg = 0) {
  has = e > s && (!SKIP_HEAVY || e - s <= heavy_deg);
  if (!has) return 0.f;
  const int deg = e - s;
  if (FAST > 0 && deg <= FAST) {
    constexpr int W = FAST > 0 ? FAST : 1;
    float v[W];
    int o[W];
    unsigned char d[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const bool in = j < deg;
      v[j] = in ? __ldcg(delta + s + j) : 0.f;
      o[j] = in ? var_occ[s + j] : -1;
      d[j] = (in && slot_dir) ? slot_dir[s + j] : 0;
    }
    float Pi = 0.f;  // slot order, as slot_sum
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (j < deg) Pi += v[j];
    if (P) P[i] = Pi;
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) cnt += (d[j] & dir) != 0;
    const float share = Pi / (float)(cnt > 0 ? cnt : deg);
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (j < deg) share_occ[o[j]] = (cnt == 0 || (d[j] & dir)) ? share : 0.f;
    return Pi;
  }
  return pending_tail_sum(delta, var_occ, P, share_occ, i, s, e, slot_dir, dir);
}

template <int FAST, bool SKIP_HEAVY = false>
__device__ __forceinline__ float pending_var(const float *__restrict__ delta, const int *__restrict__ var_ptr,
                                             const int *__restrict__ var_occ, float *__restrict__ P,
                                             float *__restrict__ share_occ, int i, bool &has,
                                             const unsigned char *__restrict__ slot_dir, int dir, int heavy_deg = 0) {
  return pending_var_se<FAST, SKIP_HEAVY>(delta, var_occ, P, share_occ, i, var_ptr[i], var_ptr[i + 1], has, slot_dir,
                                          dir, heavy_deg);
}

// The same pending sum and shares for one variable with many occurrences (slots [s, e)), by a
// whole warp: slots, occurrence ids and SRMP bits arrive 32 at a time in one round of loads,
// every lane adds the 32 values in slot order (the additions of slot_sum, so every lane holds
// the same P_i), and the lanes write the shares.  Warp-uniform arguments.
__device__ __forceinline__ float pending_var_warp(const float *__restrict__ delta, const int *__restrict__ var_occ,
                                                  float *__restrict__ P, float *__restrict__ share_occ, int i, int s,
                                                  int e, const unsigned char *__restrict__ slot_dir, int dir) {
  const int lane = threadIdx.x & 31;
  float Pi = 0.f;
  int cnt = 0, o_first = -1;
  bool take_first = false;
  for (int k0 = s; k0 < e; k0 += 32) {
    const int k = k0 + lane;
    const bool in = k < e;
    const float v = in ? __ldcg(delta + k) : 0.f;
    const bool take = in && slot_dir && (slot_dir[k] & dir);
    if (k0 == s) {
      o_first = in ? var_occ[k] : -1;
      take_first = take;
    }
    const int here = e - k0 < 32 ? e - k0 : 32;
    for (int j = 0; j < here; ++j) Pi += __shfl_sync(kFull, v, j);
    cnt += __popc(__ballot_sync(kFull, take));
  }
  if (lane == 0 && P) P[i] = Pi;
  const float share = Pi / (float)(cnt > 0 ? cnt : e - s);
  if (o_first >= 0) share_occ[o_first] = (cnt == 0 || take_first) ? share : 0.f;
  for (int k = s + 32 + lane; k < e; k += 32)
    share_occ[var_occ[k]] = (cnt == 0 || (slot_dir[k] & dir)) ? share : 0.f;
  return Pi;
}

// Fused pending pass, the part after a variable's last visit: P_i and the next sweep's shares
// by pending_var (the pending kernel's own arithmetic), the count reset, the slack term.
template <bool FWD>
__device__ __forceinline__ void finish_variable(const SweepParams &p, int i) {
  const FusedParams &z = p.fz;
  bool has;
  const float Pi = pending_var<16>(p.delta, z.var_ptr, z.var_occ, z.P, z.share, i, has, z.slot_dir,
                               FWD ? kDirBackward : kDirForward);
  z.cnt[i] = z.var_ptr[i + 1] - z.var_ptr[i];
  if (!FWD) z.slk[i] = slack_term(Pi, p.alpha);
}

// Fused pending pass over the occurrences [o0, o0 + count) of a finished tile, by `nthreads`
// threads (index t) that have all passed a barrier after the tile's last difference store.
// Each occurrence counts its variable down (eight atomics in flight per thread); the visit that
// brings a count to zero is the variable's last in this sweep and finishes it.  `list`
// (warp tiles: shared memory for 8 * 32 ids) spreads the finished variables evenly over the
// warp's lanes; without it (block tiles) each thread finishes its own.
template <bool FWD>
__device__ __forceinline__ void pending_tail(const SweepParams &p, int o0, int count, int t, int nthreads,
                                             int *list) {
  const FusedParams &z = p.fz;
  __threadfence();  // the tile's difference slots are visible before its counts drop
  for (int base = 0; base < count; base += 8 * nthreads) {
    int iv[8], old[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = base + j * nthreads + t;
      iv[j] = k < count ? z.occ_var[o0 + k] : -1;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) old[j] = iv[j] >= 0 ? atomicSub(z.cnt + iv[j], 1) : 0;
    int mine = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) mine += old[j] == 1;
    if (list) {  // warp: exclusive prefix of the lanes' counts, then an even split
      int incl = mine;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(kFull, incl, off);
        if (t >= off) incl += u;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      if (total == 0) continue;
      int pos = incl - mine;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (old[j] == 1) list[pos++] = iv[j];
      __threadfence();  // every other visit's slots before reading them
      __syncwarp();
      for (int q = t; q < total; q += 32) finish_variable<FWD>(p, list[q]);
      __syncwarp();  // the list is rewritten by the next round
    } else if (mine) {
      __threadfence();
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (old[j] == 1) finish_variable<FWD>(p, iv[j]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// warp tiles: T lanes per BDD, 32 / T BDDs per warp.  A tile's slab is contiguous and
// layer-major, so a window of kWinLayers layers (<= 32 occurrences and <= 32 nodes per layer)
// is one contiguous range of every array; the tile's window table gives each window's node
// range without reading the slab first.  Windows are staged into shared memory with cp.async
// one window ahead of the one being processed (two buffers), so the layer recurrence runs on
// shared memory and registers while the next window's loads are in flight.  The static part
// of the first window (node offsets, arcs, slots: written once at build) is staged before the
// wait on the previous kernel of the chain.
// ---------------------------------------------------------------------------------------
// wait for the kernel this launch depends on (programmatic dependent launch); a no-op without one
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// mbarrier and bulk-copy (TMA) primitives.  A window's copies complete on its buffer's
// mbarrier: one lane posts the expected byte count and issues the copies; every lane waits for
// the phase with a bounded poll.
__device__ __forceinline__ unsigned smem_u32(const void *ptr) { return (unsigned)__cvta_generic_to_shared(ptr); }
__device__ __forceinline__ void bar_init(unsigned long long *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void bar_expect(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// the GPU's global nanosecond timer
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for phase `parity`; false if it did not complete within `ns` nanoseconds
__device__ __forceinline__ bool bar_wait_ns(unsigned long long *bar, unsigned parity, unsigned long long ns) {
  if (bar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!bar_try_wait(bar, parity))
    if (global_ns() - t0 > ns) return false;
  return true;
}
// Time limit of a wait on a window's bulk copies.  Copies that were issued always complete, in
// microseconds, so this limit only guards against a fault elsewhere; it is independent of
// bdd_options.spin_limit (the grid-barrier poll limit).
constexpr unsigned long long kRingWaitNs = 2000000000ull;
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// generic-proxy writes to global memory (earlier phases of a persistent launch) before bulk reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// generic-proxy writes to this block's shared memory before bulk copies (async proxy) into it
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// A contiguous element range [first, first + n) of an array, widened to whole 16-byte blocks
// for a bulk copy: the copy starts at a0 and the range's first element lands `shift` elements
// into the destination.
struct Range {
  const char *a0;
  unsigned bytes;
  int shift;
};
template <int E>
__device__ __forceinline__ Range range_of(const void *base, long long first, int n) {
  const char *a = static_cast<const char *>(base) + first * E;
  const unsigned long long lo = reinterpret_cast<unsigned long long>(a) & ~15ull;
  const unsigned long long hi = (reinterpret_cast<unsigned long long>(a) + (unsigned long long)n * E + 15ull) & ~15ull;
  Range r;
  r.a0 = reinterpret_cast<const char *>(lo);
  r.bytes = n > 0 ? (unsigned)(hi - lo) : 0u;
  r.shift = (int)((reinterpret_cast<unsigned long long>(a) - lo) / E);
  return r;
}

// Window w of a warp tile: layers [l0, l1), occurrences [ca, cb) (relative to the tile's first),
// nodes [na, nb); a forward update also reads the backward messages of layer l1, through nc.
struct Window {
  int l0, l1, ca, cb, na, nb, nc;
};

// the tile's window table: entry w = {node at layer w * kWinLayers, node at layer
// min(w * kWinLayers + kWinLayers + 1, maxd)}; lane w holds entry w for w < 32
__device__ __forceinline__ int2 win_entry(const SweepParams &p, int win0, int2 tab, int w) {
  if (w < 32) return make_int2(__shfl_sync(kFull, tab.x, w), __shfl_sync(kFull, tab.y, w));
  return p.win_node[win0 + w];
}

__device__ __forceinline__ Window window_of(const SweepParams &p, int win0, int2 tab, int lead_depth, int maxd,
                                            int w) {
  Window W;
  W.l0 = w * kWinLayers;
  W.l1 = min(W.l0 + kWinLayers, maxd);
  W.ca = occ_before(lead_depth, W.l0);
  W.cb = occ_before(lead_depth, W.l1);
  const int2 e0 = win_entry(p, win0, tab, w), e1 = win_entry(p, win0, tab, w + 1);
  W.na = e0.x;
  W.nb = e1.x;
  W.nc = e0.y;
  return W;
}

// The six ranges of a window (static: node offsets, arcs, slots; dynamic: multipliers, shares,
// messages -- fm for a backward sweep, bm through the extra layer for a forward update)
struct WindowRanges {
  Range off, lohi, slot, lam, shr, msg;
};
template <bool FWD, int MODE>
__device__ __forceinline__ WindowRanges ranges_of(const SweepParams &p, int occ0, const Window &W) {
  const long long oa = occ0 + W.ca;
  const int nob = W.cb - W.ca;
  WindowRanges r;
  r.off = range_of<4>(p.occ_node_off, oa, nob + 1);
  r.lohi = range_of<8>(p.lohi, W.na, W.nb - W.na);
  r.slot = range_of<4>(p.occ_slot, oa, is_update(MODE) ? nob : 0);
  r.lam = range_of<4>(p.lam, oa, nob);
  r.shr = range_of<4>(p.share_occ, oa, MODE != kMessages ? nob : 0);
  if (FWD)
    r.msg = range_of<4>(p.bm, W.na, is_update(MODE) ? W.nc - W.na : 0);
  else
    r.msg = range_of<4>(p.fm, W.na, W.nb - W.na);
  return r;
}

// Per-warp copy state: two stage buffers, their mbarriers, the parity each waits for next, and
// which buffers have copies issued that no wait has consumed yet.
template <class Stage>
struct StageRingT {
  Stage *S;                  // [kWarpStages]
  unsigned long long *bar;   // [kWarpStages]
  unsigned parity;           // bit b: parity of buffer b's next phase (lane-uniform)
  unsigned busy;             // bit b: a window was issued into buffer b and not yet waited for
};
using StageRing = StageRingT<WarpStage>;

// Lane 0 issues a window's bulk copies into buffer b: with `expect`, first the expected byte
// count of the whole window; then the static and/or the dynamic copies.  Warp-collective (every
// lane keeps the same ring state).
template <class Stage>
__device__ __forceinline__ void stage_window(const WindowRanges &r, StageRingT<Stage> &ring, int b, bool expect,
                                             bool stat, bool dyn) {
  if (expect) ring.busy |= 1u << b;
  if ((threadIdx.x & 31) != 0) return;
  Stage &S = ring.S[b];
  unsigned long long *bar = &ring.bar[b];
  if (expect)
    bar_expect(bar, r.off.bytes + r.lohi.bytes + r.slot.bytes + r.lam.bytes + r.shr.bytes + r.msg.bytes);
  if (stat) {
    if (r.off.bytes) bulk_copy(S.off, r.off.a0, r.off.bytes, bar);
    if (r.lohi.bytes) bulk_copy(S.lohi, r.lohi.a0, r.lohi.bytes, bar);
    if (r.slot.bytes) bulk_copy(S.slot, r.slot.a0, r.slot.bytes, bar);
  }
  if (dyn) {
    if (r.lam.bytes) bulk_copy(S.lam, r.lam.a0, r.lam.bytes, bar);
    if (r.shr.bytes) bulk_copy(S.shr, r.shr.a0, r.shr.bytes, bar);
    if (r.msg.bytes) bulk_copy(S.msg, r.msg.a0, r.msg.bytes, bar);
  }
}

// Waits (bounded) for every window still in flight in the ring, so that no copy lands in this
// warp's shared memory after it stops using the ring.
template <class Stage>
__device__ __forceinline__ void ring_drain(StageRingT<Stage> &ring) {
  for (int b = 0; b < kWarpStages; ++b) {
    if (!((ring.busy >> b) & 1u)) continue;
    const unsigned par = (ring.parity >> b) & 1u;
    if (__all_sync(kFull, bar_wait_ns(&ring.bar[b], par, kRingWaitNs))) ring.parity ^= 1u << b;
  }
  ring.busy = 0u;
}

// wait for buffer b's window; on a timeout record BDD_ETIMEOUT, drain the copies this warp
// still has in flight and report false (the caller abandons the tile, and a persistent launch
// takes no further tile)
template <class Stage>
__device__ __forceinline__ bool ring_wait(const SweepParams &p, StageRingT<Stage> &ring, int b) {
  const unsigned par = (ring.parity >> b) & 1u;
  if (__all_sync(kFull, bar_wait_ns(&ring.bar[b], par, kRingWaitNs))) {
    ring.parity ^= 1u << b;
    ring.busy &= ~(1u << b);
    return true;
  }
  if ((threadIdx.x & 31) == 0) atomicExch(p.error, -6);
  ring_drain(ring);
  return false;
}

// Tile parameters, depths and the window table (all static, read before the dependency wait).
struct TileInfo {
  int occ0, depth, lead_depth, maxd, nw, win0;
  int2 tab;
};

template <int T>
__device__ __forceinline__ TileInfo tile_info(const SweepParams &p, int tile) {
  const int lane = threadIdx.x & 31;
  const int team = lane / T, tl = lane % T;
  TileInfo ti;
  ti.occ0 = p.tile_occ0[tile];
  ti.win0 = p.tile_win0[tile];
  const int bdd = p.tile_bdd0[tile] + team;
  const bool valid = team < p.tile_nbdd[tile];
  ti.depth = valid ? p.bdd_depth[bdd] : 0;
  ti.lead_depth = tl == 0 ? ti.depth : 0;
  ti.maxd = __reduce_max_sync(kFull, ti.depth);
  ti.nw = (ti.maxd + kWinLayers - 1) / kWinLayers;
  ti.tab = lane <= ti.nw ? p.win_node[ti.win0 + lane] : make_int2(0, 0);
  return ti;
}

template <int T, int MODE, bool SMOOTH, bool SPLIT>
__device__ __forceinline__ void warp_forward(const SweepParams &p, const Phase &ph, int tile, StageRing &ring,
                                             double &bacc) {
  const int lane = threadIdx.x & 31;
  const int team = lane / T, tl = lane % T, tbase = team * T;
  const TileInfo ti = tile_info<T>(p, tile);
  const int occ0 = ti.occ0, depth = ti.depth, lead_depth = ti.lead_depth, maxd = ti.maxd, nw = ti.nw;
  fence_proxy_async();
  // window 0 into buffer 0: static part, dependency wait, dynamic part; window 1 into buffer 1
  Window Wn = window_of(p, ti.win0, ti.tab, lead_depth, maxd, 0);
  {
    const WindowRanges r = ranges_of<true, MODE>(p, occ0, Wn);
    stage_window(r, ring, 0, true, true, false);
    pdl_wait();
    stage_window(r, ring, 0, false, false, true);
  }
  if (nw > 1) {
    const Window W1 = window_of(p, ti.win0, ti.tab, lead_depth, maxd, 1);
    stage_window(ranges_of<true, MODE>(p, occ0, W1), ring, 1, true, true, true);
  }
  float f_prev = inf(), lam_prev = 0.f;
  int2 lh_prev = make_int2(kNone, kNone);
  for (int w = 0; w < nw; ++w) {
    const Window W = Wn;
    if (w + 1 < nw) Wn = window_of(p, ti.win0, ti.tab, lead_depth, maxd, w + 1);
    const int b = w & 1;
    WarpStage &S = ring.S[b];
    if (!ring_wait(p, ring, b)) return;
    const WindowRanges r = ranges_of<true, MODE>(p, occ0, W);
    const int *off = S.off + r.off.shift;
    const int2 *lohi = S.lohi + r.lohi.shift;
    const int *slot = S.slot + r.slot.shift;
    const float *lamw = S.lam + r.lam.shift, *shr = S.shr + r.shr.shift, *msg = S.msg + r.msg.shift;
    const int ca = W.ca, na = W.na, oa = occ0 + ca;
    for (int l = W.l0; l < W.l1; ++l) {
      const bool active = depth > l;
      const int oi = occ_before(lead_depth, l) - ca + team;
      int node0 = 0, w_l = 0;
      if (active) {
        node0 = off[BDD_IN(p, oi, W.cb - W.ca)];
        w_l = off[BDD_IN(p, oi + 1, W.cb - W.ca + 1)] - node0;
      }
      const bool has = active && tl < w_l;
      // Alg. 2: m_fwd(v) = min over in-arcs (u, v) of m_fwd(u) + theta_uv
      float f;
      if (l == 0) {  // the root, or a piece's roots with their root messages (sub-BDDs)
        f = SPLIT && has ? p.fm[BDD_NODE(p, node0 + tl)] : 0.f;
      } else {
        const int lo_l = lh_prev.x >= 0 ? lh_prev.x - node0 : kNone;
        const int hi_l = lh_prev.y >= 0 ? lh_prev.y - node0 : kNone;
        f = inf();
#pragma unroll
        for (int s = 0; s < T; ++s) {
          const float mf = __shfl_sync(kFull, f_prev, tbase + s);
          const int ls = __shfl_sync(kFull, lo_l, tbase + s);
          const int hs = __shfl_sync(kFull, hi_l, tbase + s);
          if (ls == tl) f = agg<SMOOTH>(f, mf, p);
          if (hs == tl) f = agg<SMOOTH>(f, mf + lam_prev, p);
        }
      }
      int2 lh = make_int2(kNone, kNone);
      if (has) {
        p.fm[BDD_NODE(p, node0 + tl)] = f;
        lh = lohi[BDD_IN(p, node0 - na + tl, W.nb - W.na)];
      }
      float lam = active ? lamw[oi] + (MODE != kMessages ? shr[oi] : 0.f) : 0.f;
      if (is_update(MODE)) {
        // eqs. arc-marginal / marginal-aggregation, then the damped eq. mma-update step
        const float a0 = has ? f + staged_bm<SPLIT>(msg, p.copy_val, na, lh.x) : inf();
        const float a1 = has ? f + lam + staged_bm<SPLIT>(msg, p.copy_val, na, lh.y) : inf();
        const float m0 = team_agg<T, SMOOTH>(a0, p), m1 = team_agg<T, SMOOTH>(a1, p);
        const float dd = p.omega * mm_difference(m0, m1);
        lam -= dd;
        if (active && tl == 0) {
          p.lam[BDD_OCC(p, oa + oi)] = lam;
          ph.delta[BDD_OCC(p, slot[oi])] = dd;
        }
      }
      f_prev = f;
      lh_prev = lh;
      lam_prev = lam;
    }
    __syncwarp();  // this buffer is free: stage the window after next into it
    if (w + 2 < nw) {
      const Window W2 = window_of(p, ti.win0, ti.tab, lead_depth, maxd, w + 2);
      stage_window(ranges_of<true, MODE>(p, occ0, W2), ring, b, true, true, true);
    }
  }
  if (MODE == kUpdateFused) {
    __syncwarp();
    pending_tail<true>(p, occ0, __reduce_add_sync(kFull, lead_depth), lane, 32,
                       reinterpret_cast<int *>(ring.S[0].lohi));
    // the list was written through the generic proxy into a buffer that bulk copies fill
    fence_proxy_async_smem();
    __syncwarp();
  }
}

template <int T, int MODE, bool SMOOTH, bool SPLIT>
__device__ __forceinline__ void warp_backward(const SweepParams &p, const Phase &ph, int tile, StageRing &ring,
                                              double &bacc) {
  const int lane = threadIdx.x & 31;
  const int team = lane / T, tl = lane % T, tbase = team * T;
  const TileInfo ti = tile_info<T>(p, tile);
  const int occ0 = ti.occ0, depth = ti.depth, lead_depth = ti.lead_depth, maxd = ti.maxd, nw = ti.nw;
  const int bdd = p.tile_bdd0[tile] + team;
  fence_proxy_async();
  // windows from the last to the first; the k-th processed window uses buffer k & 1
  Window Wn = window_of(p, ti.win0, ti.tab, lead_depth, maxd, nw - 1);
  {
    const WindowRanges r = ranges_of<false, MODE>(p, occ0, Wn);
    stage_window(r, ring, 0, true, true, false);
    pdl_wait();
    stage_window(r, ring, 0, false, false, true);
  }
  if (nw > 1) {
    const Window W1 = window_of(p, ti.win0, ti.tab, lead_depth, maxd, nw - 2);
    stage_window(ranges_of<false, MODE>(p, occ0, W1), ring, 1, true, true, true);
  }
  float b_next = inf();
  int node0_next = 0;
  for (int k = 0; k < nw; ++k) {
    const int w = nw - 1 - k;
    const Window W = Wn;
    if (w > 0) Wn = window_of(p, ti.win0, ti.tab, lead_depth, maxd, w - 1);
    const int b = k & 1;
    WarpStage &S = ring.S[b];
    if (!ring_wait(p, ring, b)) return;
    const WindowRanges r = ranges_of<false, MODE>(p, occ0, W);
    const int *off = S.off + r.off.shift;
    const int2 *lohi = S.lohi + r.lohi.shift;
    const int *slot = S.slot + r.slot.shift;
    const float *lamw = S.lam + r.lam.shift, *shr = S.shr + r.shr.shift, *msg = S.msg + r.msg.shift;
    const int ca = W.ca, na = W.na, oa = occ0 + ca;
    for (int l = W.l1 - 1; l >= W.l0; --l) {
      const bool active = depth > l;
      const int oi = occ_before(lead_depth, l) - ca + team;
      int node0 = 0, w_l = 0;
      if (active) {
        node0 = off[BDD_IN(p, oi, W.cb - W.ca)];
        w_l = off[BDD_IN(p, oi + 1, W.cb - W.ca + 1)] - node0;
      }
      const bool has = active && tl < w_l;
      int2 lh = make_int2(kNone, kNone);
      float f = inf();
      if (has) {
        lh = lohi[BDD_IN(p, node0 - na + tl, W.nb - W.na)];
        f = msg[BDD_IN(p, node0 - na + tl, W.nb - W.na)];
      }
      float lam = active ? lamw[oi] + (MODE != kMessages ? shr[oi] : 0.f) : 0.f;
      // successors' backward messages live on the lanes of this team (layer l + 1)
      const int s0 = lh.x >= 0 ? lh.x - node0_next : 0;
      const int s1 = lh.y >= 0 ? lh.y - node0_next : 0;
      const float g0 = __shfl_sync(kFull, b_next, tbase + (s0 & (T - 1)));
      const float g1 = __shfl_sync(kFull, b_next, tbase + (s1 & (T - 1)));
      const float b0 = lh.x >= 0 ? g0 : terminal_bm<SPLIT>(p.copy_val, lh.x);
      const float b1 = lh.y >= 0 ? g1 : terminal_bm<SPLIT>(p.copy_val, lh.y);
      if (MODE != kMessages) {
        const float m0 = team_agg<T, SMOOTH>(f + b0, p), m1 = team_agg<T, SMOOTH>(f + lam + b1, p);
        if (is_update(MODE)) {
          const float dd = p.omega * mm_difference(m0, m1);
          lam -= dd;
          if (active && tl == 0) {
            p.lam[BDD_OCC(p, oa + oi)] = lam;
            ph.delta[BDD_OCC(p, slot[oi])] = dd;
          }
        } else if (active && tl == 0 && p.out_m0) {
          const long long c = p.occ_csr[oa + oi];
          p.out_m0[BDD_CSR(p, c)] = m0;
          p.out_m1[BDD_CSR(p, c)] = m1;
        }
      }
      // Alg. 3: m_bwd(v) = min(m_bwd(v0) + 0, m_bwd(v1) + lambda)
      const float bcur = agg<SMOOTH>(b0, lam + b1, p);
      if (has) p.bm[BDD_NODE(p, node0 + tl)] = bcur;
      if (l == 0) {  // E^j(lambda^j) at the root; a piece: min over its roots of fm + bm
        const float e = SPLIT ? team_agg<T, SMOOTH>(has ? f + bcur : inf(), p) : bcur;
        if (active && tl == 0) {
          p.bdd_E[BDD_BDD(p, bdd)] = e;
          bacc += (double)e;
        }
      }
      b_next = bcur;
      node0_next = node0;
    }
    __syncwarp();
    if (w >= 2) {
      const Window W2 = window_of(p, ti.win0, ti.tab, lead_depth, maxd, w - 2);
      stage_window(ranges_of<false, MODE>(p, occ0, W2), ring, b, true, true, true);
    }
  }
  if (MODE == kUpdateFused) {
    __syncwarp();
    pending_tail<false>(p, occ0, __reduce_add_sync(kFull, lead_depth), lane, 32,
                        reinterpret_cast<int *>(ring.S[0].lohi));
    // the list was written through the generic proxy into a buffer that bulk copies fill
    fence_proxy_async_smem();
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------
// lane tiles: one lane per BDD whose layers have at most two nodes, 32 BDDs per warp (the slab
// of a warp tile of 32 one-lane teams).  A lane keeps both nodes of its BDD's current layer in
// registers, so the forward push, the min-marginals and the backward pull need no shuffles and
// no team reductions; windows of kWinLayers layers (up to 64 nodes each) are staged by the
// bulk-copy ring as for warp tiles.  A layer's arcs come from its lane code (one byte per
// occurrence, see LaneStage) instead of node offsets and a pair of node indices per node: the
// lane's first node is the layer's first node plus the nodes of the lanes before it (a ballot of
// the two-node layers), its successors are node 0 or 1 of its next layer or a terminal.  The
// arithmetic is that of a two-lane team, operation for operation and in the same order, so the
// results equal the team layout's bit for bit.
// ---------------------------------------------------------------------------------------
using LaneRing = StageRingT<LaneStage>;

// the arc a of node t in a lane code (a = 0: 0-arc, 1: 1-arc): 0 or 1, kLaneTop or kLaneBot
__device__ __forceinline__ unsigned lane_arc(unsigned code, int t, int a) { return (code >> (4 * t + 2 * a)) & 3u; }
__device__ __forceinline__ bool lane_two_nodes(unsigned code) { return (code >> 4) != (kLaneNoNode1 >> 4); }

// forward message of node t of a layer (Alg. 2) from the two nodes of the previous layer
// (messages pf0, pf1; their arcs in the lane code pc; 1-arc cost plam), relaxed in the order of
// the team path: node 0 before node 1, 0-arc first
__device__ __forceinline__ float lane_push(unsigned t, float pf0, float pf1, unsigned pc, float plam) {
  float f = inf();
  if (lane_arc(pc, 0, 0) == t) f = fminf(f, pf0);
  if (lane_arc(pc, 0, 1) == t) f = fminf(f, pf0 + plam);
  if (lane_arc(pc, 1, 0) == t) f = fminf(f, pf1);
  if (lane_arc(pc, 1, 1) == t) f = fminf(f, pf1 + plam);
  return f;
}

// The five ranges of a lane-tile window: the lane codes of its occurrences and of the layer after
// it (static; the code array carries kLaneCodePad spare entries), slots (static), multipliers,
// shares and messages (dynamic, as for warp tiles)
struct LaneRanges {
  Range code, slot, lam, shr, msg;
};
// A range of E-byte elements [first, first + n) of an array whose start is 16-byte aligned (every
// device array comes from cudaMalloc), widened to whole 16-byte blocks: the block boundaries
// follow from the element indices alone, in 32-bit arithmetic, and the first element lands
// first mod (16 / E) elements into the destination.
template <int E>
__device__ __forceinline__ Range aligned_range(const void *base, unsigned first, unsigned n) {
  constexpr unsigned B = 16 / E;  // elements per 16-byte block
  const unsigned lo = first & ~(B - 1), hi = (first + n + B - 1) & ~(B - 1);
  Range r;
  r.a0 = static_cast<const char *>(base) + (size_t)lo * E;
  r.bytes = n > 0 ? (hi - lo) * E : 0u;
  r.shift = (int)(first - lo);
  return r;
}
template <bool FWD, int MODE>
__device__ __forceinline__ LaneRanges lane_ranges_of(const SweepParams &p, int occ0, const Window &W) {
  const unsigned oa = (unsigned)(occ0 + W.ca), nob = (unsigned)(W.cb - W.ca);
  LaneRanges r;
  r.code = aligned_range<1>(p.lane_code, oa, nob + 32);
  r.slot = aligned_range<4>(p.occ_slot, oa, is_update(MODE) ? nob : 0u);
  r.lam = aligned_range<4>(p.lam, oa, nob);
  r.shr = aligned_range<4>(p.share_occ, oa, MODE != kMessages ? nob : 0u);
  if (FWD)
    r.msg = aligned_range<4>(p.bm, (unsigned)W.na, is_update(MODE) ? (unsigned)(W.nc - W.na) : 0u);
  else
    r.msg = aligned_range<4>(p.fm, (unsigned)W.na, (unsigned)(W.nb - W.na));
  return r;
}
// where a lane-tile window's first occurrence, code and message sit in its stage (the shifts of
// lane_ranges_of, without the ranges)
struct LaneShifts {
  int occ, code, msg;
};
__device__ __forceinline__ LaneShifts lane_shifts(int oa, int na) { return {oa & 3, oa & 15, na & 3}; }

// stage_window for a lane-tile window
__device__ __forceinline__ void stage_lane_window(const LaneRanges &r, LaneRing &ring, int b, bool expect, bool stat,
                                                  bool dyn) {
  if (expect) ring.busy |= 1u << b;
  if ((threadIdx.x & 31) != 0) return;
  LaneStage &S = ring.S[b];
  unsigned long long *bar = &ring.bar[b];
  if (expect) bar_expect(bar, r.code.bytes + r.slot.bytes + r.lam.bytes + r.shr.bytes + r.msg.bytes);
  if (stat) {
    if (r.code.bytes) bulk_copy(S.code, r.code.a0, r.code.bytes, bar);
    if (r.slot.bytes) bulk_copy(S.slot, r.slot.a0, r.slot.bytes, bar);
  }
  if (dyn) {
    if (r.lam.bytes) bulk_copy(S.lam, r.lam.a0, r.lam.bytes, bar);
    if (r.shr.bytes) bulk_copy(S.shr, r.shr.a0, r.shr.bytes, bar);
    if (r.msg.bytes) bulk_copy(S.msg, r.msg.a0, r.msg.bytes, bar);
  }
}

// A lane run: consecutive lane tiles [t0, t1) of one warp (at most kLaneRunMax), streamed through the
// ring as one sequence of windows (a tile's windows in sweep order, then the next tile's), so
// that the copies of a tile's first windows overlap the previous tile's last ones.  Lane i holds
// the scalars of tile t0 + i (loaded once); a tile's BDD depths and window table are loaded
// while the tile before it is staged, so no tile waits on its own parameters.
static_assert(kLaneRunMax <= 32, "a lane run keeps one tile's scalars per lane");
struct LaneRunScalars {
  int occ0, win0, win1, bdd0, nbdd;  // of tile t0 + lane (win1: the next tile's first entry)
};
struct LanePre {  // depth of this lane's BDD and window-table entry `lane` of one tile
  int depth;
  int2 tab;
};
struct LaneCursor {  // the next window to stage: window w of `tile` (tile == t1: none left)
  int tile, w, bdd0;
  TileInfo ti;
  LanePre pre;  // of tile + 1
};
// one staged window and what its processing needs
struct LaneJob {
  Window W;
  int occ0, depth, bdd0;
};

__device__ __forceinline__ LaneRunScalars lane_run_scalars(const SweepParams &p, int t0, int t1) {
  const int t = t0 + (threadIdx.x & 31);
  LaneRunScalars s{0, 0, 0, 0, 0};
  if (t < t1) {
    s.occ0 = p.tile_occ0[t];
    s.win0 = p.tile_win0[t];
    s.win1 = p.tile_win0[t + 1];
    s.bdd0 = p.tile_bdd0[t];
    s.nbdd = p.tile_nbdd[t];
  }
  return s;
}

// issues the loads of tile t's depths and window table (tile t of the run: i = t - t0 < 32)
__device__ __forceinline__ LanePre lane_pre(const SweepParams &p, const LaneRunScalars &s, int i, bool valid) {
  const int lane = threadIdx.x & 31;
  const int win0 = __shfl_sync(kFull, s.win0, i & 31), nent = __shfl_sync(kFull, s.win1, i & 31) - win0;
  const int bdd0 = __shfl_sync(kFull, s.bdd0, i & 31), nbdd = __shfl_sync(kFull, s.nbdd, i & 31);
  LanePre q{0, make_int2(0, 0)};
  if (valid && lane < nbdd) q.depth = p.bdd_depth[bdd0 + lane];
  if (valid && lane < nent) q.tab = p.win_node[win0 + lane];
  return q;
}

// tile_info<1> of tile t0 + i from its prefetched depths and window table
__device__ __forceinline__ TileInfo lane_info(const LaneRunScalars &s, int i, const LanePre &q) {
  TileInfo ti;
  ti.occ0 = __shfl_sync(kFull, s.occ0, i & 31);
  ti.win0 = __shfl_sync(kFull, s.win0, i & 31);
  ti.depth = q.depth;
  ti.lead_depth = q.depth;
  ti.maxd = __reduce_max_sync(kFull, q.depth);
  ti.nw = (ti.maxd + kWinLayers - 1) / kWinLayers;
  ti.tab = q.tab;
  return ti;
}

// enter tile c.tile (< t1): its parameters from the prefetch, then the next tile's prefetch
template <bool FWD>
__device__ __forceinline__ void lane_enter(const SweepParams &p, const LaneRunScalars &s, int t0, int t1,
                                           LaneCursor &c) {
  const int i = c.tile - t0;
  c.ti = lane_info(s, i, c.pre);
  c.bdd0 = __shfl_sync(kFull, s.bdd0, i & 31);
  c.w = FWD ? 0 : c.ti.nw - 1;
  c.pre = lane_pre(p, s, i + 1, c.tile + 1 < t1);
}

// the window after c's in stream order; skips tiles without layers
template <bool FWD>
__device__ __forceinline__ void lane_step(const SweepParams &p, const LaneRunScalars &s, int t0, int t1,
                                          LaneCursor &c) {
  if (FWD ? c.w + 1 < c.ti.nw : c.w > 0) {
    c.w += FWD ? 1 : -1;
    return;
  }
  while (++c.tile < t1) {
    lane_enter<FWD>(p, s, t0, t1, c);
    if (c.ti.nw > 0) break;
  }
}

template <bool FWD>
__device__ __forceinline__ void lane_start(const SweepParams &p, const LaneRunScalars &s, int t0, int t1,
                                           LaneCursor &c) {
  c.tile = t0;
  c.pre = lane_pre(p, s, 0, true);
  for (; c.tile < t1; ++c.tile) {
    lane_enter<FWD>(p, s, t0, t1, c);
    if (c.ti.nw > 0) break;
  }
}

__device__ __forceinline__ LaneJob lane_job(const SweepParams &p, const LaneCursor &c) {
  LaneJob j;
  j.W = window_of(p, c.ti.win0, c.ti.tab, c.ti.lead_depth, c.ti.maxd, c.w);
  j.occ0 = c.ti.occ0;
  j.depth = c.ti.depth;
  j.bdd0 = c.bdd0;
  return j;
}

// forward recurrence state carried from layer to layer: the previous layer's two messages, arcs
// and 1-arc cost
struct LaneFwd {
  float pf0, pf1, plam;
  unsigned pcode;  // the previous layer's lane code (no arcs for a lane without that layer)
};

template <int MODE>
__device__ __forceinline__ void lane_forward_window(const SweepParams &p, const Phase &ph, const LaneJob &j,
                                                    const LaneStage &S, LaneFwd &st) {
  const int lane = threadIdx.x & 31;
  const unsigned before = (1u << lane) - 1u;  // the lanes before this one
  const Window &W = j.W;
  const LaneShifts sh = lane_shifts(j.occ0 + W.ca, W.na);
  const unsigned char *code = S.code + sh.code;
  const int *slot = S.slot + sh.occ;
  const float *lamw = S.lam + sh.occ, *shr = S.shr + sh.occ, *msg = S.msg + sh.msg;
  const int ca = W.ca, na = W.na, oa = j.occ0 + ca;
  [[maybe_unused]] const int ncode = W.cb - W.ca + 32;  // staged codes: the window's occurrences and the next layer's
  int first = na;                      // the layer's first node (the window's first, then onwards)
  // layer l's occurrences before it in the tile (ob), this lane's code and the two-node lanes;
  // each layer's are taken from the step before, which decodes the layer after it
  int ob = ca;
  unsigned c = j.depth > W.l0 ? code[BDD_IN(p, lane, ncode)] : 0xFFu;
  unsigned twos = __ballot_sync(kFull, j.depth > W.l0 && lane_two_nodes(c));
  for (int l = W.l0; l < W.l1; ++l) {
    const bool active = j.depth > l;
    const int oi = ob - ca + lane;
    const bool two = active && lane_two_nodes(c);
    const int wl = active ? (two ? 2 : 1) : 0;
    const int node0 = first + lane + __popc(twos & before);  // the alive lanes are a prefix
    const int ob_n = occ_before(j.depth, l + 1);
    const int layer_nodes = (ob_n - ob) + __popc(twos);  // alive lanes + their second nodes
    // the next layer's codes (staged with the window)
    const bool active_n = j.depth > l + 1;
    const int oin = ob_n - ca + lane;
    const unsigned cn = active_n ? code[BDD_IN(p, oin, ncode)] : 0xFFu;
    const bool two_n = active_n && lane_two_nodes(cn);
    const unsigned twos_n = __ballot_sync(kFull, two_n);
    // Alg. 2: m_fwd(v) = min over in-arcs (u, v) of m_fwd(u) + theta_uv, for both nodes
    float f0 = 0.f, f1 = 0.f;  // the root (layer 0)
    if (l > 0) {
      f0 = lane_push(0u, st.pf0, st.pf1, st.pcode, st.plam);
      f1 = lane_push(1u, st.pf0, st.pf1, st.pcode, st.plam);
    }
    if (wl > 0) p.fm[BDD_NODE(p, node0)] = f0;
    if (wl > 1) p.fm[BDD_NODE(p, node0 + 1)] = f1;
    float lam = active ? lamw[oi] + (MODE != kMessages ? shr[oi] : 0.f) : 0.f;
    if (is_update(MODE)) {
      // the backward messages of this BDD's next layer (staged with the window): node 0 if the
      // BDD has that layer, node 1 if the layer has two nodes -- the only nodes its arcs reach
      const int next0 = first + layer_nodes + lane + __popc(twos_n & before) - na;
      const float bn0 = active_n ? msg[BDD_IN(p, next0, W.nc - na)] : inf();
      const float bn1 = two_n ? msg[BDD_IN(p, next0 + 1, W.nc - na)] : inf();
      auto bm_of = [&](unsigned a) { return a == 0u ? bn0 : a == 1u ? bn1 : a == kLaneTop ? 0.f : inf(); };
      // eqs. arc-marginal / marginal-aggregation, then the damped eq. mma-update step.  A node
      // the layer does not have (node 1 of a one-node layer, both nodes of a lane without the
      // layer) has both arcs to the false terminal, so its terms are +inf without a test.
      const float a00 = f0 + bm_of(lane_arc(c, 0, 0));
      const float a01 = f1 + bm_of(lane_arc(c, 1, 0));
      const float a10 = f0 + lam + bm_of(lane_arc(c, 0, 1));
      const float a11 = f1 + lam + bm_of(lane_arc(c, 1, 1));
      const float m0 = fminf(a00, a01), m1 = fminf(a10, a11);
      const float dd = p.omega * mm_difference(m0, m1);
      lam -= dd;
      if (active) {
        p.lam[BDD_OCC(p, oa + oi)] = lam;
        ph.delta[BDD_OCC(p, slot[oi])] = dd;
      }
    }
    st.pf0 = f0;
    st.pf1 = f1;
    st.pcode = c;  // 0xFF (all arcs to the false terminal) for a lane without this layer
    st.plam = lam;
    first += layer_nodes;
    ob = ob_n;
    c = cn;
    twos = twos_n;
  }
}

template <int MODE>
__device__ __forceinline__ void lane_backward_window(const SweepParams &p, const Phase &ph, const LaneJob &j,
                                                     const LaneStage &S, float &bn0, float &bn1, double &bacc) {
  const int lane = threadIdx.x & 31;
  const unsigned before = (1u << lane) - 1u;
  const Window &W = j.W;
  const LaneShifts sh = lane_shifts(j.occ0 + W.ca, W.na);
  const unsigned char *code = S.code + sh.code;
  const int *slot = S.slot + sh.occ;
  const float *lamw = S.lam + sh.occ, *shr = S.shr + sh.occ, *msg = S.msg + sh.msg;
  const int ca = W.ca, na = W.na, oa = j.occ0 + ca;
  [[maybe_unused]] const int ncode = W.cb - W.ca + 32;
  int end = W.nb;  // one past the layer's last node (the window's end, then downwards)
  int ob_n = W.cb;  // occurrences of the tile before layer l + 1
  for (int l = W.l1 - 1; l >= W.l0; --l) {
    const bool active = j.depth > l;
    const int ob = occ_before(j.depth, l);
    const int oi = ob - ca + lane;
    const unsigned c = active ? code[BDD_IN(p, oi, ncode)] : 0xFFu;
    const bool two = active && lane_two_nodes(c);
    const int wl = active ? (two ? 2 : 1) : 0;
    const unsigned twos = __ballot_sync(kFull, two);
    end -= (ob_n - ob) + __popc(twos);  // alive lanes + their second nodes: now the layer's first node
    ob_n = ob;
    const int node0 = end + lane + __popc(twos & before);
    float f0 = inf(), f1 = inf();
    if (wl > 0) f0 = msg[BDD_IN(p, node0 - na, W.nb - W.na)];
    if (wl > 1) f1 = msg[BDD_IN(p, node0 - na + 1, W.nb - W.na)];
    float lam = active ? lamw[oi] + (MODE != kMessages ? shr[oi] : 0.f) : 0.f;
    // successors' backward messages: the next layer's nodes, held by this lane (a BDD's last
    // layer has terminal arcs only, so nothing is read from the previous BDD of the lane)
    auto pull = [&](unsigned a) { return a == 0u ? bn0 : a == 1u ? bn1 : a == kLaneTop ? 0.f : inf(); };
    const float b00 = pull(lane_arc(c, 0, 0)), b01 = pull(lane_arc(c, 0, 1));
    const float b10 = pull(lane_arc(c, 1, 0)), b11 = pull(lane_arc(c, 1, 1));
    if (MODE != kMessages) {
      const float m0 = fminf(f0 + b00, f1 + b10), m1 = fminf(f0 + lam + b01, f1 + lam + b11);
      if (is_update(MODE)) {
        const float dd = p.omega * mm_difference(m0, m1);
        lam -= dd;
        if (active) {
          p.lam[BDD_OCC(p, oa + oi)] = lam;
          ph.delta[BDD_OCC(p, slot[oi])] = dd;
        }
      } else if (active && p.out_m0) {
        const long long csr = p.occ_csr[oa + oi];
        p.out_m0[BDD_CSR(p, csr)] = m0;
        p.out_m1[BDD_CSR(p, csr)] = m1;
      }
    }
    // Alg. 3: m_bwd(v) = min(m_bwd(v0) + 0, m_bwd(v1) + lambda)
    const float bc0 = fminf(b00, lam + b01), bc1 = fminf(b10, lam + b11);
    if (wl > 0) p.bm[BDD_NODE(p, node0)] = bc0;
    if (wl > 1) p.bm[BDD_NODE(p, node0 + 1)] = bc1;
    if (l == 0 && active) {  // E^j(lambda^j) at the root
      p.bdd_E[BDD_BDD(p, j.bdd0 + lane)] = bc0;
      bacc += (double)bc0;
    }
    bn0 = bc0;
    bn1 = bc1;
  }
}

// The run's window stream: stage the first two windows (the first one's static part before the
// dependency wait), then process window k from buffer k & 1 and stage window k + 2 into it.
template <bool FWD, int MODE>
__device__ __forceinline__ void lane_run(const SweepParams &p, const Phase &ph, int t0, int t1, LaneRing &ring,
                                         double &bacc) {
  fence_proxy_async();
  const LaneRunScalars s = lane_run_scalars(p, t0, t1);
  LaneCursor c;
  lane_start<FWD>(p, s, t0, t1, c);
  if (c.tile >= t1) return;
  LaneJob cur = lane_job(p, c);
  {
    const LaneRanges r = lane_ranges_of<FWD, MODE>(p, cur.occ0, cur.W);
    stage_lane_window(r, ring, 0, true, true, false);
    pdl_wait();
    stage_lane_window(r, ring, 0, false, false, true);
  }
  lane_step<FWD>(p, s, t0, t1, c);
  bool have_next = c.tile < t1;
  LaneJob next = cur;
  if (have_next) {
    next = lane_job(p, c);
    stage_lane_window(lane_ranges_of<FWD, MODE>(p, next.occ0, next.W), ring, 1, true, true, true);
    lane_step<FWD>(p, s, t0, t1, c);
  }
  LaneFwd st{0.f, 0.f, 0.f, 0xFFu};
  float bn0 = inf(), bn1 = inf();  // backward messages of the next layer's two nodes
  for (int k = 0;; ++k) {
    const int b = k & 1;
    if (!ring_wait(p, ring, b)) return;
    if (FWD)
      lane_forward_window<MODE>(p, ph, cur, ring.S[b], st);
    else
      lane_backward_window<MODE>(p, ph, cur, ring.S[b], bn0, bn1, bacc);
    __syncwarp();  // this buffer is free: stage the window after next into it
    const bool have_after = c.tile < t1;
    LaneJob after = next;
    if (have_after) {
      after = lane_job(p, c);
      stage_lane_window(lane_ranges_of<FWD, MODE>(p, after.occ0, after.W), ring, b, true, true, true);
      lane_step<FWD>(p, s, t0, t1, c);
    }
    if (!have_next) break;
    cur = next;
    next = after;
    have_next = have_after;
  }
}

// ---------------------------------------------------------------------------------------
// warp tiles, 8-layer windows: each window is staged in one round of cp.async (node offsets,
// slots and arcs, then multipliers, shares and messages; the tile's window table gives the
// window's node range) and processed once it has landed.  The first window's static part (node
// offsets, slots, arcs: written once at build) is issued before the wait on the previous kernel.
// Fewer instructions per layer than the bulk-copy ring, no overlap of loads with the layer
// recurrence; the autotuner picks between the two per solver and sweep direction.  Update
// sweeps only.
// ---------------------------------------------------------------------------------------
// One window: node offsets of occurrences [oa, oa + nox], slots and multipliers / shares of
// [oa, oa + nob), arcs of nodes [na, nb), messages of nodes [na, nm) (bm through the layer after
// the window for a forward update, fm for a backward sweep).  `first`: the launch's first
// window, whose static part goes out before the dependency wait.
template <int MODE>
__device__ __forceinline__ void issue_window_w8(const SweepParams &p, WarpStage8 &S, int oa, int nob, int nox,
                                                int na, int nb, const float *msg_src, int nm, bool first) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k <= nox; k += 32) cp_async4(&S.off[k], &p.occ_node_off[oa + k]);
  if (is_update(MODE))
    for (int k = lane; k < nob; k += 32) cp_async4(&S.slot[k], &p.occ_slot[oa + k]);
  for (int k = lane; k < nb - na; k += 32) cp_async8(&S.lohi[k], &p.lohi[na + k]);
  if (first) pdl_wait();
  for (int k = lane; k < nob; k += 32) {
    cp_async4(&S.lam[k], &p.lam[oa + k]);
    if (MODE != kMessages)
      cp_async4(&S.shr[k], &p.share_occ[oa + k]);
    else
      S.shr[k] = 0.f;
  }
  for (int k = lane; k < nm - na; k += 32) cp_async4(&S.msg[k], &msg_src[na + k]);
}

template <int MODE>
__device__ __forceinline__ void stage_window_w8(const SweepParams &p, WarpStage8 &S, int oa, int nob, int nox,
                                                int na, int nb, const float *msg_src, int nm, bool first) {
  issue_window_w8<MODE>(p, S, oa, nob, nox, na, nb, msg_src, nm, first);
  cp_async_wait();
}

// Geometry of 8-layer window k of a warp tile: layers [l0, l1), occurrences [ca, cb) relative to
// the tile (cx: through the layer after the window), nodes [na, nb) and, for a forward update,
// through the layer after the window, nc.  Node ranges come from the tile's 4-layer window table.
// Warp-collective (every lane calls it with the same k).
struct Win8 {
  int l0, l1, ca, oa, nob, nox, na, nb, nc;
};
__device__ __forceinline__ Win8 win8_of(const SweepParams &p, const TileInfo &ti, int lead_depth, int k) {
  Win8 g;
  g.l0 = k * kWin8Layers;
  g.l1 = min(g.l0 + kWin8Layers, ti.maxd);
  g.ca = occ_before(lead_depth, g.l0);
  const int cb = occ_before(lead_depth, g.l1);
  const int cx = g.l1 < ti.maxd ? occ_before(lead_depth, g.l1 + 1) : cb;
  g.oa = ti.occ0 + g.ca;
  g.nob = cb - g.ca;
  g.nox = cx - g.ca;
  const int w4 = g.l0 / kWinLayers;
  g.na = win_entry(p, ti.win0, ti.tab, w4).x;
  g.nb = win_entry(p, ti.win0, ti.tab, min(w4 + 2, ti.nw)).x;
  g.nc = win_entry(p, ti.win0, ti.tab, w4 + 1).y;  // node at layer min(l0 + 9, maxd)
  return g;
}

// NBUF = 1: each window is loaded, then processed (staging variant 1).  NBUF = 2: two buffers per
// warp, window k + 1's copies in flight (one cp.async group per window) while window k is
// processed (staging variant 2).
template <int T, int MODE, bool SMOOTH, bool SPLIT, int NBUF>
__device__ __forceinline__ void warp_forward_w8(const SweepParams &p, const Phase &ph, int tile, WarpStage8 *SB,
                                             double &bacc) {
  const int lane = threadIdx.x & 31;
  const int team = lane / T, tl = lane % T, tbase = team * T;
  const TileInfo ti = tile_info<T>(p, tile);
  const int depth = ti.depth, lead_depth = ti.lead_depth, maxd = ti.maxd;
  const int nwin = (maxd + kWin8Layers - 1) / kWin8Layers;
  float f_prev = inf(), lam_prev = 0.f;
  int2 lh_prev = make_int2(kNone, kNone);
  auto issue = [&](WarpStage8 &S, const Win8 &g, bool first) {
    issue_window_w8<MODE>(p, S, g.oa, g.nob, g.nox, g.na, g.nb, p.bm, is_update(MODE) ? g.nc : g.na, first);
  };
  if (NBUF == 2) {
    issue(SB[0], win8_of(p, ti, lead_depth, 0), true);
    cp_async_commit();
    if (nwin > 1) issue(SB[1], win8_of(p, ti, lead_depth, 1), false);
    cp_async_commit();  // (an empty group when there is no second window)
  }
  for (int k = 0; k < nwin; ++k) {
    const Win8 g = win8_of(p, ti, lead_depth, k);
    WarpStage8 &S = SB[NBUF == 2 ? (k & 1) : 0];
    if (NBUF == 1) {
      __syncwarp();  // the previous window is no longer read
      stage_window_w8<MODE>(p, S, g.oa, g.nob, g.nox, g.na, g.nb, p.bm, is_update(MODE) ? g.nc : g.na, k == 0);
    } else {
      cp_async_wait_group<1>();  // window k has landed (window k + 1 may still be in flight)
    }
    __syncwarp();
    const int ca = g.ca, oa = g.oa, na = g.na;
    for (int l = g.l0; l < g.l1; ++l) {
      const bool active = depth > l;
      const int oi = occ_before(lead_depth, l) - ca + team;
      int node0 = 0, w = 0;
      if (active) {
        node0 = S.off[BDD_IN(p, oi, g.nob)];
        w = S.off[BDD_IN(p, oi + 1, g.nox + 1)] - node0;
      }
      const bool has = active && tl < w;
      // Alg. 2: m_fwd(v) = min over in-arcs (u, v) of m_fwd(u) + theta_uv
      float f;
      if (l == 0) {  // the root, or a piece's roots with their root messages (sub-BDDs)
        f = SPLIT && has ? p.fm[BDD_NODE(p, node0 + tl)] : 0.f;
      } else {
        const int lo_l = lh_prev.x >= 0 ? lh_prev.x - node0 : kNone;
        const int hi_l = lh_prev.y >= 0 ? lh_prev.y - node0 : kNone;
        f = inf();
#pragma unroll
        for (int s = 0; s < T; ++s) {
          const float mf = __shfl_sync(kFull, f_prev, tbase + s);
          const int ls = __shfl_sync(kFull, lo_l, tbase + s);
          const int hs = __shfl_sync(kFull, hi_l, tbase + s);
          if (ls == tl) f = agg<SMOOTH>(f, mf, p);
          if (hs == tl) f = agg<SMOOTH>(f, mf + lam_prev, p);
        }
      }
      int2 lh = make_int2(kNone, kNone);
      if (has) {
        p.fm[BDD_NODE(p, node0 + tl)] = f;
        lh = S.lohi[BDD_IN(p, node0 - na + tl, g.nb - g.na)];
      }
      float lam = active ? S.lam[oi] + S.shr[oi] : 0.f;
      if (is_update(MODE)) {
        // eqs. arc-marginal / marginal-aggregation, then the damped eq. mma-update step
        const float a0 = has ? f + staged_bm<SPLIT>(S.msg, p.copy_val, na, lh.x) : inf();
        const float a1 = has ? f + lam + staged_bm<SPLIT>(S.msg, p.copy_val, na, lh.y) : inf();
        const float m0 = team_agg<T, SMOOTH>(a0, p), m1 = team_agg<T, SMOOTH>(a1, p);
        const float dd = p.omega * mm_difference(m0, m1);
        lam -= dd;
        if (active && tl == 0) {
          p.lam[BDD_OCC(p, oa + oi)] = lam;
          ph.delta[BDD_OCC(p, S.slot[oi])] = dd;
        }
      }
      f_prev = f;
      lh_prev = lh;
      lam_prev = lam;
    }
    if (NBUF == 2) {
      __syncwarp();  // this buffer is free: window k + 2 goes into it
      if (k + 2 < nwin) issue(S, win8_of(p, ti, lead_depth, k + 2), false);
      cp_async_commit();
    }
  }
}

template <int T, int MODE, bool SMOOTH, bool SPLIT, int NBUF>
__device__ __forceinline__ void warp_backward_w8(const SweepParams &p, const Phase &ph, int tile, WarpStage8 *SB,
                                              double &bacc) {
  const int lane = threadIdx.x & 31;
  const int team = lane / T, tl = lane % T, tbase = team * T;
  const TileInfo ti = tile_info<T>(p, tile);
  const int depth = ti.depth, lead_depth = ti.lead_depth, maxd = ti.maxd;
  const int bdd = p.tile_bdd0[tile] + team;
  const int nwin = (maxd + kWin8Layers - 1) / kWin8Layers;
  float b_next = inf();
  int node0_next = 0;
  // windows from the last to the first; the j-th processed window uses buffer j & 1
  auto issue = [&](WarpStage8 &S, const Win8 &g, bool first) {
    issue_window_w8<MODE>(p, S, g.oa, g.nob, g.nob, g.na, g.nb, p.fm, g.nb, first);
  };
  if (NBUF == 2) {
    issue(SB[0], win8_of(p, ti, lead_depth, nwin - 1), true);
    cp_async_commit();
    if (nwin > 1) issue(SB[1], win8_of(p, ti, lead_depth, nwin - 2), false);
    cp_async_commit();
  }
  for (int j = 0; j < nwin; ++j) {
    const int k = nwin - 1 - j;
    const Win8 g = win8_of(p, ti, lead_depth, k);
    WarpStage8 &S = SB[NBUF == 2 ? (j & 1) : 0];
    if (NBUF == 1) {
      __syncwarp();
      stage_window_w8<MODE>(p, S, g.oa, g.nob, g.nob, g.na, g.nb, p.fm, g.nb, j == 0);
    } else {
      cp_async_wait_group<1>();
    }
    __syncwarp();
    const int ca = g.ca, oa = g.oa, na = g.na;
    for (int l = g.l1 - 1; l >= g.l0; --l) {
      const bool active = depth > l;
      const int oi = occ_before(lead_depth, l) - ca + team;
      int node0 = 0, w = 0;
      if (active) {
        node0 = S.off[BDD_IN(p, oi, g.nob)];
        w = S.off[BDD_IN(p, oi + 1, g.nox + 1)] - node0;
      }
      const bool has = active && tl < w;
      int2 lh = make_int2(kNone, kNone);
      float f = inf();
      if (has) {
        lh = S.lohi[BDD_IN(p, node0 - na + tl, g.nb - g.na)];
        f = S.msg[BDD_IN(p, node0 - na + tl, g.nb - g.na)];
      }
      float lam = active ? S.lam[oi] + S.shr[oi] : 0.f;
      // successors' backward messages live on the lanes of this team (layer l + 1)
      const int s0 = lh.x >= 0 ? lh.x - node0_next : 0;
      const int s1 = lh.y >= 0 ? lh.y - node0_next : 0;
      const float g0 = __shfl_sync(kFull, b_next, tbase + (s0 & (T - 1)));
      const float g1 = __shfl_sync(kFull, b_next, tbase + (s1 & (T - 1)));
      const float b0 = lh.x >= 0 ? g0 : terminal_bm<SPLIT>(p.copy_val, lh.x);
      const float b1 = lh.y >= 0 ? g1 : terminal_bm<SPLIT>(p.copy_val, lh.y);
      if (MODE != kMessages) {
        const float m0 = team_agg<T, SMOOTH>(f + b0, p), m1 = team_agg<T, SMOOTH>(f + lam + b1, p);
        if (is_update(MODE)) {
          const float dd = p.omega * mm_difference(m0, m1);
          lam -= dd;
          if (active && tl == 0) {
            p.lam[BDD_OCC(p, oa + oi)] = lam;
            ph.delta[BDD_OCC(p, S.slot[oi])] = dd;
          }
        } else if (active && tl == 0 && p.out_m0) {
          const long long c = p.occ_csr[oa + oi];
          p.out_m0[BDD_CSR(p, c)] = m0;
          p.out_m1[BDD_CSR(p, c)] = m1;
        }
      }
      // Alg. 3: m_bwd(v) = min(m_bwd(v0) + 0, m_bwd(v1) + lambda)
      const float bcur = agg<SMOOTH>(b0, lam + b1, p);
      if (has) p.bm[BDD_NODE(p, node0 + tl)] = bcur;
      if (l == 0) {  // E^j(lambda^j) at the root; a piece: min over its roots of fm + bm
        const float e = SPLIT ? team_agg<T, SMOOTH>(has ? f + bcur : inf(), p) : bcur;
        if (active && tl == 0) {
          p.bdd_E[BDD_BDD(p, bdd)] = e;
          bacc += (double)e;
        }
      }
      b_next = bcur;
      node0_next = node0;
    }
    if (NBUF == 2) {
      __syncwarp();
      if (j + 2 < nwin) issue(S, win8_of(p, ti, lead_depth, k - 2), false);
      cp_async_commit();
    }
  }
}

// ---------------------------------------------------------------------------------------
// block tiles: one 128-thread group per BDD (layers wider than 32 nodes).  `group` selects the
// named barrier; `gt` is the thread's index inside its group.
// ---------------------------------------------------------------------------------------
struct GroupSmem {
  float2 *red;  // [kWarpsPerBlock]
  float *bufA, *bufB, *shr;
  int *off;     // [block_depth_buf + 4] node offsets of the tile's layers (narrow tiles)
  int2 *arcs;   // [block_buf] arcs of the current layer (smoothed narrow tiles), else null
};

// floats of shared memory of one block-tile group; `smooth` adds the arcs of a layer
__host__ __device__ __forceinline__ size_t group_floats(int block_buf, int block_depth_buf, bool smooth = false) {
  return 2 * kWarpsPerBlock + 2 * (size_t)block_buf + 2 * (size_t)block_depth_buf + 4 +
         (smooth ? 2 * (size_t)block_buf : 0);
}

__device__ __forceinline__ GroupSmem group_smem(float *base, const SweepParams &p) {
  GroupSmem g;
  g.red = reinterpret_cast<float2 *>(base);
  g.bufA = base + 2 * kWarpsPerBlock;
  g.bufB = g.bufA + p.block_buf;
  g.shr = g.bufB + p.block_buf;
  g.off = reinterpret_cast<int *>(g.shr + p.block_depth_buf);
  g.arcs = p.alpha > 0.f ? reinterpret_cast<int2 *>(g.off + p.block_depth_buf + 4) : nullptr;
  return g;
}

__device__ __forceinline__ float2 group_min2(float a, float b, float2 *red, int group, int gt) {
  const int lane = gt & 31, warp = gt >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a = fminf(a, __shfl_xor_sync(kFull, a, off));
    b = fminf(b, __shfl_xor_sync(kFull, b, off));
  }
  if (lane == 0) red[warp] = make_float2(a, b);
  group_sync(group);
  float2 r = red[0];
#pragma unroll
  for (int t = 1; t < kWarpsPerBlock; ++t) {
    r.x = fminf(r.x, red[t].x);
    r.y = fminf(r.y, red[t].y);
  }
  group_sync(group);  // red may be reused right after
  return r;
}

// the same reduction with the soft minimum (smoothed solvers): each warp's butterfly keeps its
// first lane's value, then the warps' values in warp order, so every thread gets the same bits
template <bool SMOOTH>
__device__ __forceinline__ float2 group_agg2(float a, float b, const SweepParams &p, float2 *red, int group, int gt) {
  if (!SMOOTH) return group_min2(a, b, red, group, gt);
  const int lane = gt & 31, warp = gt >> 5;
  a = team_agg<32, true>(a, p);
  b = team_agg<32, true>(b, p);
  if (lane == 0) red[warp] = make_float2(a, b);
  group_sync(group);
  float2 r = red[0];
#pragma unroll
  for (int t = 1; t < kWarpsPerBlock; ++t) {
    r.x = soft_min(r.x, red[t].x, p.alpha, p.inv_alpha);
    r.y = soft_min(r.y, red[t].y, p.alpha, p.inv_alpha);
  }
  group_sync(group);  // red may be reused right after
  return r;
}

// per-layer shares of a block tile, staged before its layers are processed
template <int MODE>
__device__ __forceinline__ void stage_group_shares(const SweepParams &p, int occ0, int depth, float *shr, int gt) {
  for (int l = gt; l < depth; l += kBlockThreads) {
    if (MODE != kMessages)
      cp_async4(&shr[l], &p.share_occ[occ0 + l]);
    else
      shr[l] = 0.f;
  }
  cp_async_wait();
}

template <int MODE, bool SPLIT>
__device__ __forceinline__ void block_forward(const SweepParams &p, const Phase &ph, int tile, const GroupSmem &g,
                                              int group, int gt, double &bacc) {
  const int bdd = p.tile_bdd0[tile];
  const int occ0 = p.tile_occ0[tile];
  const int depth = p.bdd_depth[bdd];
  float *cur = g.bufA, *nxt = g.bufB;
  stage_group_shares<MODE>(p, occ0, depth, g.shr, gt);
  if (SPLIT) {  // a piece's roots start from their root messages
    const int n0 = p.occ_node_off[occ0], w0 = p.occ_node_off[occ0 + 1] - n0;
    for (int t = gt; t < w0; t += kBlockThreads) cur[t] = p.fm[n0 + t];
  } else if (gt == 0) {
    cur[0] = 0.f;
  }
  group_sync(group);
  for (int l = 0; l < depth; ++l) {
    const int o = occ0 + l;
    const int node0 = p.occ_node_off[o], w = p.occ_node_off[o + 1] - node0;
    float lam = p.lam[o] + g.shr[l];
    float a0 = inf(), a1 = inf();
    for (int t = gt; t < w; t += kBlockThreads) {
      const float f = cur[t];
      p.fm[BDD_NODE(p, node0 + t)] = f;
      if (is_update(MODE)) {
        const int2 lh = p.lohi[BDD_NODE(p, node0 + t)];
        a0 = fminf(a0, f + target_bm<SPLIT>(p.bm, p.copy_val, lh.x));
        a1 = fminf(a1, f + lam + target_bm<SPLIT>(p.bm, p.copy_val, lh.y));
      }
    }
    if (is_update(MODE)) {
      const float2 mm = group_min2(a0, a1, g.red, group, gt);
      const float dd = p.omega * mm_difference(mm.x, mm.y);
      lam -= dd;
      if (gt == 0) {
        p.lam[BDD_OCC(p, o)] = lam;
        ph.delta[BDD_OCC(p, p.occ_slot[o])] = dd;
      }
    }
    if (l + 1 < depth) {
      const int next0 = node0 + w, wn = p.occ_node_off[o + 2] - next0;
      for (int t = gt; t < wn; t += kBlockThreads) nxt[t] = inf();
      group_sync(group);
      for (int t = gt; t < w; t += kBlockThreads) {
        const float f = cur[t];
        const int2 lh = p.lohi[BDD_NODE(p, node0 + t)];
        if (lh.x >= 0) atomic_min_f(&nxt[lh.x - next0], f);
        if (lh.y >= 0) atomic_min_f(&nxt[lh.y - next0], f + lam);
      }
      group_sync(group);
      float *tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
}

template <int MODE, bool SPLIT>
__device__ __forceinline__ void block_backward(const SweepParams &p, const Phase &ph, int tile, const GroupSmem &g,
                                               int group, int gt, double &bacc) {
  const int bdd = p.tile_bdd0[tile];
  const int occ0 = p.tile_occ0[tile];
  const int depth = p.bdd_depth[bdd];
  float *cur = g.bufA, *nxt = g.bufB;  // cur: backward messages of layer l + 1
  stage_group_shares<MODE>(p, occ0, depth, g.shr, gt);
  group_sync(group);
  for (int l = depth - 1; l >= 0; --l) {
    const int o = occ0 + l;
    const int node0 = p.occ_node_off[o], w = p.occ_node_off[o + 1] - node0;
    const int next0 = node0 + w;
    float lam = p.lam[o] + g.shr[l];
    if (MODE != kMessages) {
      float a0 = inf(), a1 = inf();
      for (int t = gt; t < w; t += kBlockThreads) {
        const int2 lh = p.lohi[BDD_NODE(p, node0 + t)];
        const float f = p.fm[BDD_NODE(p, node0 + t)];
        const float b0 = lh.x >= 0 ? cur[lh.x - next0] : terminal_bm<SPLIT>(p.copy_val, lh.x);
        const float b1 = lh.y >= 0 ? cur[lh.y - next0] : terminal_bm<SPLIT>(p.copy_val, lh.y);
        a0 = fminf(a0, f + b0);
        a1 = fminf(a1, f + lam + b1);
      }
      const float2 mm = group_min2(a0, a1, g.red, group, gt);
      if (is_update(MODE)) {
        const float dd = p.omega * mm_difference(mm.x, mm.y);
        lam -= dd;
        if (gt == 0) {
          p.lam[BDD_OCC(p, o)] = lam;
          ph.delta[BDD_OCC(p, p.occ_slot[o])] = dd;
        }
      } else if (gt == 0 && p.out_m0) {
        const long long c = p.occ_csr[o];
        p.out_m0[BDD_CSR(p, c)] = mm.x;
        p.out_m1[BDD_CSR(p, c)] = mm.y;
      }
    }
    float e = inf();  // a piece's energy: min over its roots of fm + bm
    for (int t = gt; t < w; t += kBlockThreads) {
      const int2 lh = p.lohi[BDD_NODE(p, node0 + t)];
      const float b0 = lh.x >= 0 ? cur[lh.x - next0] : terminal_bm<SPLIT>(p.copy_val, lh.x);
      const float b1 = lh.y >= 0 ? cur[lh.y - next0] : terminal_bm<SPLIT>(p.copy_val, lh.y);
      const float bcur = fminf(b0, lam + b1);
      p.bm[BDD_NODE(p, node0 + t)] = bcur;
      nxt[t] = bcur;
      if (l == 0) {
        if (SPLIT) {
          e = fminf(e, p.fm[node0 + t] + bcur);
        } else if (t == 0) {
          p.bdd_E[BDD_BDD(p, bdd)] = bcur;
          bacc += (double)bcur;
        }
      }
    }
    if (l == 0 && SPLIT) {
      e = group_min2(e, inf(), g.red, group, gt).x;
      if (gt == 0) {
        p.bdd_E[BDD_BDD(p, bdd)] = e;
        bacc += (double)e;
      }
    }
    group_sync(group);
    float *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

// ---------------------------------------------------------------------------------------
// block tiles whose layers are at most kBlockThreads nodes wide (one node per thread): the
// tile's node offsets and multipliers (with the shares the sweep adds) are staged in shared
// memory once, and each thread prefetches its node's arcs two layers ahead and, in a forward
// update, the backward messages of their targets one layer ahead, so the layer recurrence waits
// on no global load.  Same arithmetic as block_forward / block_backward.
// ---------------------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void stage_group_layers(const SweepParams &p, int occ0, int depth, const GroupSmem &g,
                                                   int gt) {
  for (int l = gt; l <= depth; l += kBlockThreads) g.off[l] = p.occ_node_off[occ0 + l];
  for (int l = gt; l < depth; l += kBlockThreads)
    g.shr[l] = p.lam[occ0 + l] + (MODE != kMessages ? p.share_occ[occ0 + l] : 0.f);
}

// arcs of this thread's node in layer l (none past the last layer or the layer's width)
__device__ __forceinline__ int2 narrow_arcs(const SweepParams &p, const int *off, int l, int depth, int gt) {
  if (l >= depth) return make_int2(kNone, kNone);
  const int node0 = off[l];
  return gt < off[l + 1] - node0 ? p.lohi[node0 + gt] : make_int2(kNone, kNone);
}

// SMOOTH: the forward step pulls instead of pushing -- node v of layer l + 1 aggregates its
// in-arcs scanning the nodes of layer l in order, 0-arc before 1-arc (the soft minimum is not
// associative in floating point, so a fixed order replaces the atomic minimum)
template <int MODE, bool SPLIT, bool SMOOTH = false>
__device__ __forceinline__ void block_forward_narrow(const SweepParams &p, const Phase &ph, int tile,
                                                     const GroupSmem &g, int group, int gt, double &bacc) {
  const int bdd = p.tile_bdd0[tile];
  const int occ0 = p.tile_occ0[tile];
  const int depth = p.bdd_depth[bdd];
  float *cur = g.bufA, *nxt = g.bufB;
  const int *off = g.off;
  stage_group_layers<MODE>(p, occ0, depth, g, gt);
  group_sync(group);
  {  // the root, or a piece's roots with their root messages (sub-BDDs)
    const int n0 = off[0];
    if (gt < off[1] - n0) cur[gt] = SPLIT ? p.fm[n0 + gt] : 0.f;
  }
  int2 lh = narrow_arcs(p, off, 0, depth, gt), lh1 = narrow_arcs(p, off, 1, depth, gt);
  float t0 = 0.f, t1 = 0.f;
  if (is_update(MODE)) {
    t0 = target_bm<SPLIT>(p.bm, p.copy_val, lh.x);
    t1 = target_bm<SPLIT>(p.bm, p.copy_val, lh.y);
  }
  group_sync(group);
  for (int l = 0; l < depth; ++l) {
    // in flight during this layer: the next layer's target messages, the arcs two layers on
    float u0 = 0.f, u1 = 0.f;
    if (is_update(MODE) && l + 1 < depth) {
      u0 = target_bm<SPLIT>(p.bm, p.copy_val, lh1.x);
      u1 = target_bm<SPLIT>(p.bm, p.copy_val, lh1.y);
    }
    const int2 lh2 = narrow_arcs(p, off, l + 2, depth, gt);
    const int o = occ0 + l;
    const int node0 = off[l], w = off[l + 1] - node0;
    const bool has = gt < w;
    const float f = has ? cur[gt] : inf();
    if (has) p.fm[BDD_NODE(p, node0 + gt)] = f;
    if (SMOOTH && gt < p.block_buf) g.arcs[gt] = lh;  // read by the pull after the next barrier
    float lam = g.shr[l];
    const bool more = l + 1 < depth;
    // nxt was last read before the previous layer's final barrier
    if (more && gt < off[l + 2] - off[l + 1]) nxt[gt] = inf();
    if (is_update(MODE)) {
      const float2 mm = group_agg2<SMOOTH>(has ? f + t0 : inf(), has ? f + lam + t1 : inf(), p, g.red, group, gt);
      const float dd = p.omega * mm_difference(mm.x, mm.y);
      lam -= dd;
      if (gt == 0) {
        p.lam[BDD_OCC(p, o)] = lam;
        ph.delta[BDD_OCC(p, p.occ_slot[o])] = dd;
      }
    } else if (more) {
      group_sync(group);  // the resets of nxt before the pushes
    }
    if (more) {
      const int next0 = off[l + 1];
      if (SMOOTH) {
        if (gt < off[l + 2] - next0) {
          const int v = next0 + gt;
          float acc = inf();
          for (int u = 0; u < w; ++u) {
            const int2 a = g.arcs[u];
            if (a.x == v) acc = soft_min(acc, cur[u], p.alpha, p.inv_alpha);
            if (a.y == v) acc = soft_min(acc, cur[u] + lam, p.alpha, p.inv_alpha);
          }
          nxt[gt] = acc;
        }
      } else {
        if (lh.x >= 0) atomic_min_f(&nxt[lh.x - next0], f);
        if (lh.y >= 0) atomic_min_f(&nxt[lh.y - next0], f + lam);
      }
      group_sync(group);
      float *tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    lh = lh1;
    lh1 = lh2;
    t0 = u0;
    t1 = u1;
  }
}

template <int MODE, bool SPLIT, bool SMOOTH = false>
__device__ __forceinline__ void block_backward_narrow(const SweepParams &p, const Phase &ph, int tile,
                                                      const GroupSmem &g, int group, int gt, double &bacc) {
  const int bdd = p.tile_bdd0[tile];
  const int occ0 = p.tile_occ0[tile];
  const int depth = p.bdd_depth[bdd];
  float *cur = g.bufA, *nxt = g.bufB;  // cur: backward messages of layer l + 1
  const int *off = g.off;
  stage_group_layers<MODE>(p, occ0, depth, g, gt);
  group_sync(group);
  // this thread's node in layer l: arcs and forward message, prefetched two layers ahead
  auto node_fm = [&](int l) {
    if (l < 0) return inf();
    const int node0 = off[l];
    return gt < off[l + 1] - node0 ? p.fm[node0 + gt] : inf();
  };
  const int last = depth - 1;
  int2 lh = narrow_arcs(p, off, last, depth, gt), lh1 = last >= 1 ? narrow_arcs(p, off, last - 1, depth, gt)
                                                                    : make_int2(kNone, kNone);
  float f = node_fm(last), f1 = node_fm(last - 1);
  for (int l = last; l >= 0; --l) {
    const int2 lh2 = l >= 2 ? narrow_arcs(p, off, l - 2, depth, gt) : make_int2(kNone, kNone);
    const float f2 = node_fm(l - 2);
    const int o = occ0 + l;
    const int node0 = off[l], w = off[l + 1] - node0, next0 = off[l + 1];
    const bool has = gt < w;
    float lam = g.shr[l];
    const float b0 = lh.x >= 0 ? cur[lh.x - next0] : terminal_bm<SPLIT>(p.copy_val, lh.x);
    const float b1 = lh.y >= 0 ? cur[lh.y - next0] : terminal_bm<SPLIT>(p.copy_val, lh.y);
    if (MODE != kMessages) {
      const float2 mm = group_agg2<SMOOTH>(has ? f + b0 : inf(), has ? f + lam + b1 : inf(), p, g.red, group, gt);
      if (is_update(MODE)) {
        const float dd = p.omega * mm_difference(mm.x, mm.y);
        lam -= dd;
        if (gt == 0) {
          p.lam[BDD_OCC(p, o)] = lam;
          ph.delta[BDD_OCC(p, p.occ_slot[o])] = dd;
        }
      } else if (gt == 0 && p.out_m0) {
        const long long c = p.occ_csr[o];
        p.out_m0[BDD_CSR(p, c)] = mm.x;
        p.out_m1[BDD_CSR(p, c)] = mm.y;
      }
    }
    // Alg. 3: m_bwd(v) = min(m_bwd(v0) + 0, m_bwd(v1) + lambda)
    const float bcur = agg<SMOOTH>(b0, lam + b1, p);
    if (has) {
      p.bm[BDD_NODE(p, node0 + gt)] = bcur;
      nxt[gt] = bcur;
    }
    if (l == 0) {  // E^j at the root; a piece: min over its roots of fm + bm
      if (SPLIT) {
        const float e = group_min2(has ? f + bcur : inf(), inf(), g.red, group, gt).x;
        if (gt == 0) {
          p.bdd_E[BDD_BDD(p, bdd)] = e;
          bacc += (double)e;
        }
      } else if (gt == 0) {
        p.bdd_E[BDD_BDD(p, bdd)] = bcur;
        bacc += (double)bcur;
      }
    }
    group_sync(group);
    float *tmp = cur;
    cur = nxt;
    nxt = tmp;
    lh = lh1;
    lh1 = lh2;
    f = f1;
    f1 = f2;
  }
}

// STAGE 0: bulk-copy ring (StageRing); STAGE 1: 8-layer cp.async windows (WarpStage8 at W8);
// STAGE 2: two 8-layer windows per warp, the next loading while one is processed (W8[0..1])
template <bool FWD, int MODE, bool SMOOTH, int STAGE = 0, bool SPLIT = false>
__device__ __forceinline__ void warp_tile(const SweepParams &p, const Phase &ph, int tile, StageRing &S,
                                          double &bacc, WarpStage8 *W8 = nullptr) {
  int c = 0;
  while (tile >= p.class_tile_off[c + 1]) ++c;
  switch (c) {
#define BDD_TEAM_CASE(C, T)                                                     \
  case C:                                                                       \
    if constexpr (STAGE >= 1) {                                                 \
      if (FWD) warp_forward_w8<T, MODE, SMOOTH, SPLIT, STAGE>(p, ph, tile, W8, bacc); \
      else warp_backward_w8<T, MODE, SMOOTH, SPLIT, STAGE>(p, ph, tile, W8, bacc);    \
    } else {                                                                    \
      if (FWD) warp_forward<T, MODE, SMOOTH, SPLIT>(p, ph, tile, S, bacc);       \
      else warp_backward<T, MODE, SMOOTH, SPLIT>(p, ph, tile, S, bacc);          \
    }                                                                           \
    break;
    BDD_TEAM_CASE(0, 1)
    BDD_TEAM_CASE(1, 2)
    BDD_TEAM_CASE(2, 4)
    BDD_TEAM_CASE(3, 8)
    BDD_TEAM_CASE(4, 16)
    BDD_TEAM_CASE(5, 32)
#undef BDD_TEAM_CASE
    default:
      break;
  }
}

// The bound from the per-block partials of a deferred pending pass, by one warp: lane k adds
// partials k, k + 32, ... in order, then a fixed shuffle tree; lane 0 stores.  The same bits on
// every run (the order does not depend on timing).
__device__ __forceinline__ void finish_bound(const double *partial, int nblocks, int *iter_ctr, double *trace,
                                             int cap, double empty_const) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int k = lane; k < nblocks; k += 32) s += __ldcg(partial + k);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  if (lane == 0) {
    const int it = *iter_ctr;
    if (it < cap) trace[it] = s + empty_const;
    *iter_ctr = it + 1;
  }
}

__device__ __forceinline__ double block_sum(double v, double *red, int nwarps) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nwarps; ++w) s += red[w];
  __syncthreads();
  return s;  // on thread 0
}

}  // namespace

// ---------------------------------------------------------------------------------------
// per-phase kernels
// ---------------------------------------------------------------------------------------
// FP64 bound of the last fused backward sweep: sum_j E^j + sum_i slack_i + empty_const, every
// thread of the grid taking a grid-stride share, per-block partials finished in block order by
// the last block to arrive (warp 0 of each block handles the ticket; the other warps go on).
// Needs every thread of the block; blockDim.x = nthreads.
__device__ __forceinline__ void fused_bound(const FusedParams &z, const float *__restrict__ bdd_E, int nthreads) {
  __shared__ double red[kReduceThreads / 32];
  const int range = z.n > z.nb ? z.n : z.nb;
  double acc = 0.0;
  for (int i = blockIdx.x * nthreads + threadIdx.x; i < range; i += gridDim.x * nthreads) {
    if (i < z.n) acc += z.slk[i];
    if (i < z.nb) acc += (double)bdd_E[i];
  }
  const double blk = block_sum(acc, red, nthreads / 32);
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  unsigned last = 0;
  if (lane == 0) {
    z.partial[blockIdx.x] = blk;
    __threadfence();
    last = atomicAdd(z.ticket, 1u) == gridDim.x - 1;
  }
  if (!__shfl_sync(kFull, last, 0)) return;
  __threadfence();
  double s = 0.0;
  for (unsigned t = lane; t < gridDim.x; t += 32) s += __ldcg(z.partial + t);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  if (lane == 0) {
    const int it = *z.iter_ctr;
    if (it < z.trace_cap) z.trace[it] = s + z.empty_const;
    *z.iter_ctr = it + 1;
    *z.ticket = 0u;
  }
}

template <bool FWD, int MODE, bool SMOOTH, int STAGE = 0, bool SPLIT = false>
__global__ void __launch_bounds__(kBlockThreads) sweep_kernel(const SweepParams p) {
  extern __shared__ __align__(16) float smem[];
  // the next kernel of the chain may launch now (small grids; else as this one's blocks exit):
  // it reads nothing this one writes before its own dependency wait.  This kernel reads static
  // data (slab offsets, arcs, slots) before its wait, and everything a previous kernel writes
  // only after it.
  if (p.pdl_early) pdl_release();
  if (FWD && MODE == kUpdateFused && p.fz.bound) {  // bound of the previous iteration (fused plan)
    pdl_wait();
    fused_bound(p.fz, p.bdd_E, kBlockThreads);
    if (threadIdx.x < 32) __syncwarp();
  }
  const Phase ph{p.delta};
  double bacc = 0.0;
  if ((int)blockIdx.x < p.n_warp_blocks) {
    const int warp = threadIdx.x >> 5;
    constexpr bool kLanes = !SMOOTH && !SPLIT && MODE != kUpdateFused;
    // with lane tiles, warps [0, n_lane_warps) take runs of lane_run consecutive lane tiles and
    // the warps after them one other warp tile each
    const int wi = blockIdx.x * kWarpsPerBlock + warp;
    const bool lanes = kLanes && p.lanes2;
    const bool lane_tile = lanes && wi < p.n_lane_warps;
    const int tile = !lanes ? wi : lane_tile ? wi * p.lane_run : wi - p.n_lane_warps + p.class_tile_off[1];
    if (tile >= p.class_tile_off[kWarpClasses]) return;  // whole warp leaves together
    char *mine = reinterpret_cast<char *>(smem) + (size_t)warp * p.warp_smem;
    __shared__ unsigned long long bars[kWarpsPerBlock * kWarpStages];
    if (lane_tile || STAGE == 0) {
      if ((threadIdx.x & 31) == 0) {
        for (int b = 0; b < kWarpStages; ++b) bar_init(&bars[warp * kWarpStages + b]);
        bar_init_fence();
      }
      __syncwarp();
    }
    if constexpr (kLanes) {
      if (lane_tile) {
        LaneRing ring{reinterpret_cast<LaneStage *>(mine), &bars[warp * kWarpStages], 0u, 0u};
        lane_run<FWD, MODE>(p, ph, tile, min(tile + p.lane_run, p.class_tile_off[1]), ring, bacc);
      }
    }
    if (!lane_tile) {
      if constexpr (STAGE >= 1) {
        StageRing none{nullptr, nullptr, 0u, 0u};
        warp_tile<FWD, MODE, SMOOTH, STAGE, SPLIT>(p, ph, tile, none, bacc, reinterpret_cast<WarpStage8 *>(mine));
      } else {
        StageRing ring{reinterpret_cast<WarpStage *>(mine), &bars[warp * kWarpStages], 0u, 0u};
        warp_tile<FWD, MODE, SMOOTH, 0, SPLIT>(p, ph, tile, ring, bacc);
      }
    }
    // the previous iteration's bound, by warp 0 of the last warp block (its tiles are the
    // shallowest, so the chain's critical path does not wait for this)
    if (FWD && p.fin_partial && (int)blockIdx.x == p.n_warp_blocks - 1 && warp == 0)
      finish_bound(p.fin_partial, p.fin_nblocks, p.fin_iter, p.fin_trace, p.fin_cap, p.fin_const);
  } else {  // block tiles (smoothed solvers: layers of at most kBlockThreads nodes only)
    const int tile = p.class_tile_off[kWarpClasses] + (blockIdx.x - p.n_warp_blocks);
    if (tile >= p.class_tile_off[kWarpClasses + 1]) return;  // uniform across the block
    pdl_wait();
    const GroupSmem g = group_smem(smem, p);
    if (p.block_buf <= kBlockThreads) {
      if (FWD)
        block_forward_narrow<MODE, SPLIT, SMOOTH>(p, ph, tile, g, 0, threadIdx.x, bacc);
      else
        block_backward_narrow<MODE, SPLIT, SMOOTH>(p, ph, tile, g, 0, threadIdx.x, bacc);
    } else if constexpr (!SMOOTH) {
      if (FWD)
        block_forward<MODE, SPLIT>(p, ph, tile, g, 0, threadIdx.x, bacc);
      else
        block_backward<MODE, SPLIT>(p, ph, tile, g, 0, threadIdx.x, bacc);
    }
    if (MODE == kUpdateFused) {
      group_sync(0);
      pending_tail<FWD>(p, p.tile_occ0[tile], p.bdd_depth[p.tile_bdd0[tile]], threadIdx.x, kBlockThreads,
                        nullptr);
    }
    // no warp tiles: the last block finishes the previous iteration's bound
    if (FWD && p.fin_partial && p.n_warp_blocks == 0 && blockIdx.x == gridDim.x - 1 && threadIdx.x < 32)
      finish_bound(p.fin_partial, p.fin_nblocks, p.fin_iter, p.fin_trace, p.fin_cap, p.fin_const);
  }
}

__global__ void __launch_bounds__(32) bound_finish_kernel(const double *partial, int nblocks, int *iter_ctr,
                                                          double *trace, int cap, double empty_const) {
  pdl_enter();
  finish_bound(partial, nblocks, iter_ctr, trace, cap, empty_const);
}

// the bound of the last iteration of a fused chain (no forward sweep follows to reduce it)
__global__ void __launch_bounds__(kReduceThreads) bound_kernel(const SweepParams p) {
  pdl_enter();
  fused_bound(p.fz, p.bdd_E, kReduceThreads);
}

// With `bound`, also the FP64 y-slack lower bound sum_j E^j + sum_i min(0, P_i) (+ the constant
// of variables in no row): per-block partials summed in a fixed order by the last block to
// finish, written to trace[*iter_ctr].
// SMOOTH: the slack term is the soft minimum of {0, P_i} (alpha > 0); the min-sum kernel carries
// no transcendental code.
template <bool BOUND, bool SMOOTH>
__global__ void __launch_bounds__(kReduceThreads, 8) pending_kernel(const PendingParams p) {
  // the first variable's slot range is static: load it before waiting for the sweep that writes
  // the slots, so its round trip overlaps that sweep's tail
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  int s = 0, e = 0;
  if (i0 < p.n) {
    s = p.var_ptr[i0];
    e = p.var_ptr[i0 + 1];
  }
  pdl_wait();
  if (p.pdl_early) pdl_release();
  const int range = BOUND ? (p.n > p.nb ? p.n : p.nb) : p.n;
  const int stride = gridDim.x * blockDim.x;
  // P_i is stored by the bound pass only: the pass between the sweeps of an iteration would
  // store values that the bound pass of the same iteration overwrites before anything reads them
  float *const P = BOUND ? p.P : nullptr;
  const float alpha = (float)p.alpha;
  BoundSum acc;
  for (int i = i0; i < range; i += stride) {
    // the next variable's slot range goes out before this variable's slots are loaded, so the
    // two round trips overlap (measured on the Potts batch: 0.93 -> 0.86 ms per pass)
    int sn = 0, en = 0;
    if (i + stride < p.n) {
      sn = p.var_ptr[i + stride];
      en = p.var_ptr[i + stride + 1];
    }
    if (i < p.n) {
      bool has;
      // the bound pass loads up to four slots, their occurrence ids and SRMP bits in one round
      // (0.94 against 1.01 ms per pass on the 256-instance Potts batch); the pass between the
      // sweeps is faster with the general path (0.79 against 0.87-0.88 ms with one round of up
      // to two or four slots).  The same additions in the same order either way.
      constexpr int kFast = BOUND ? 4 : 0;
      const float Pi = pending_var_se<kFast, true>(p.delta, p.var_occ, P, p.share_occ, i, s, e, has, p.slot_dir,
                                                   p.next_dir, p.heavy_deg);
      if (BOUND && has) add_slack<SMOOTH>(acc, Pi, alpha);
    }
    if (BOUND && i < p.nb) acc.add(p.bdd_E[i]);
    s = sn;
    e = en;
  }
  // variables with more than heavy_deg occurrences: one warp each
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < p.n_heavy; w += (gridDim.x * blockDim.x) >> 5) {
    const int4 hv = p.heavy[w];
    const float Pi = pending_var_warp(p.delta, p.var_occ, P, p.share_occ, hv.x, hv.y, hv.z, p.slot_dir, p.next_dir);
    if (BOUND && (threadIdx.x & 31) == 0) add_slack<SMOOTH>(acc, Pi, alpha);
  }
  if constexpr (BOUND) {
    __shared__ double red[kReduceThreads / 32];
    __shared__ bool last;
    const double blk = block_sum(acc.value(), red, kReduceThreads / 32);
    if (p.defer) {  // the next forward sweep (or a finishing kernel) sums the partials
      if (threadIdx.x == 0) p.partial[blockIdx.x] = blk;
      return;
    }
    if (threadIdx.x == 0) {
      p.partial[blockIdx.x] = blk;
      __threadfence();
      last = atomicAdd(p.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double s = 0.0;
      for (unsigned t = threadIdx.x; t < gridDim.x; t += blockDim.x) s += __ldcg(&p.partial[t]);
      s = block_sum(s, red, kReduceThreads / 32);
      if (threadIdx.x == 0) {
        const int it = *p.iter_ctr;
        if (it < p.trace_cap) p.trace[it] = s + p.empty_const;
        *p.iter_ctr = it + 1;
        *p.ticket = 0u;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// persistent iteration kernel: one cooperative launch runs n_iter iterations, each a forward
// phase and a backward phase separated by grid barriers; one 512-thread block per SM.  Every
// tile is owned by the same warp (or 128-thread group) in every phase, so its multipliers and
// messages never move between SMs; the only data crossing blocks within the launch are the
// recorded differences (read through L2) and the bound partials.
// ---------------------------------------------------------------------------------------
namespace {

// Grid-wide barrier (all blocks are resident: cooperative launch).  The wait is bounded: after
// spin_limit polls, or once another block has failed, the block records BDD_ETIMEOUT (-6) and
// every later barrier returns false at once, so the kernel always finishes.
__device__ bool grid_barrier(const IterParams &q, bool &failed) {
  __shared__ int s_fail;
  __syncthreads();
  if (threadIdx.x == 0) {
    int f = failed ? 1 : 0;
    if (!f) {
      volatile unsigned *gen = q.barrier + 1;
      volatile int *err = q.error;
      const unsigned g = *gen;
      __threadfence();
      if (atomicAdd(q.barrier, 1u) == gridDim.x - 1) {
        atomicExch(q.barrier, 0u);
        __threadfence();
        atomicAdd(q.barrier + 1, 1u);
      } else {
        long long spins = 0;
        while (*gen == g) {
          if (*err != 0 || ++spins > q.spin_limit) {
            f = 1;
            atomicExch(q.error, -6);
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
    }
    s_fail = f;
  }
  __syncthreads();
  failed = s_fail != 0;
  return !failed;
}

template <bool FWD>
__device__ __forceinline__ void persistent_phase(const SweepParams &p, float *smem, StageRing &ring, double &bacc) {
  const Phase ph{p.delta};
  const int warp = threadIdx.x >> 5;
  const int W = gridDim.x * kPersistWarps;
  const int nwt = p.class_tile_off[kWarpClasses];
  for (int tile = blockIdx.x * kPersistWarps + warp; tile < nwt; tile += W) {
    // a wait of this launch gave up: its ring may be out of step, so take no further tile (the
    // next grid barrier sees the error and ends the launch)
    if (*reinterpret_cast<volatile int *>(p.error) != 0) break;
    warp_tile<FWD, kUpdate, false>(p, ph, tile, ring, bacc);
  }
  const int bt0 = p.class_tile_off[kWarpClasses];
  const int nbt = p.class_tile_off[kWarpClasses + 1] - bt0;
  if (nbt > 0) {
    __syncthreads();  // the warps' stages are reused as group buffers
    const int group = threadIdx.x / kBlockThreads, gt = threadIdx.x % kBlockThreads;
    const GroupSmem g = group_smem(smem + group * group_floats(p.block_buf, p.block_depth_buf), p);
    for (int t = blockIdx.x * kSubBlocks + group; t < nbt; t += gridDim.x * kSubBlocks) {
      if (FWD)
        block_forward<kUpdate, false>(p, ph, bt0 + t, g, group, gt, bacc);
      else
        block_backward<kUpdate, false>(p, ph, bt0 + t, g, group, gt, bacc);
      group_sync(group);
    }
    // the group buffers were written through the generic proxy; the next phase's bulk copies
    // (async proxy) write the same shared memory: order the two
    fence_proxy_async_smem();
    __syncthreads();
  }
}

// pending sums and shares of a grid-stride range of variables; returns sum of min(0, P_i)
__device__ __forceinline__ double persistent_pending(const IterParams &q, int next_dir) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q.n; i += gridDim.x * blockDim.x) {
    bool has;
    const float Pi =
        pending_var<0, true>(q.sp.delta, q.var_ptr, q.var_occ, q.P, q.share_occ, i, has, q.slot_dir, next_dir,
                             q.heavy_deg);
    if (has && Pi < 0.f) acc += (double)Pi;
  }
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < q.n_heavy; w += (gridDim.x * blockDim.x) >> 5) {
    const int4 hv = q.heavy[w];
    const float Pi = pending_var_warp(q.sp.delta, q.var_occ, q.P, q.share_occ, hv.x, hv.y, hv.z, q.slot_dir, next_dir);
    if ((threadIdx.x & 31) == 0 && Pi < 0.f) acc += (double)Pi;
  }
  return acc;
}

// trace[it] = sum over blocks (in block order) of the E^j partials and the slack partials of
// iteration it, plus the constant of variables in no row (block 0)
__device__ void finalize_bound(const IterParams &q, int it, double *red) {
  const int G = gridDim.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < G; b += blockDim.x) v += __ldcg(q.part + b) + __ldcg(q.part + G + b);
  const double s = block_sum(v, red, kPersistWarps);
  if (threadIdx.x == 0 && it < q.trace_cap) q.trace[it] = s + q.empty_const;
}

}  // namespace

__global__ void __launch_bounds__(kPersistThreads, 1) iterate_kernel(const IterParams q) {
  extern __shared__ __align__(16) float smem[];
  __shared__ double red[kPersistWarps];
  const SweepParams &p = q.sp;
  const int G = gridDim.x;
  // per-warp stage buffers and their mbarriers (static shared memory: the dynamic region is
  // reused by block tiles)
  __shared__ unsigned long long bars[kPersistWarps * kWarpStages];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    for (int b = 0; b < kWarpStages; ++b) bar_init(&bars[warp * kWarpStages + b]);
    bar_init_fence();
  }
  __syncwarp();
  StageRing ring{reinterpret_cast<WarpStage *>(reinterpret_cast<char *>(smem) + (size_t)warp * kWarpSmemBytes),
                 &bars[warp * kWarpStages], 0u, 0u};
  bool failed = false;
  for (int it = 0; it < q.n_iter; ++it) {
    double bacc = 0.0;
    persistent_phase<true>(p, smem, ring, bacc);
    if (blockIdx.x == 0 && it > 0) finalize_bound(q, it - 1, red);  // partials of it-1 are final
    if (!grid_barrier(q, failed)) return;
    persistent_pending(q, kDirBackward);
    if (!grid_barrier(q, failed)) return;
    bacc = 0.0;
    persistent_phase<false>(p, smem, ring, bacc);
    double sum = block_sum(bacc, red, kPersistWarps);
    if (threadIdx.x == 0) q.part[blockIdx.x] = sum;  // E^j part
    if (!grid_barrier(q, failed)) return;
    sum = block_sum(persistent_pending(q, kDirForward), red, kPersistWarps);
    if (threadIdx.x == 0) q.part[G + blockIdx.x] = sum;  // slack part
    if (!grid_barrier(q, failed)) return;
  }
  if (blockIdx.x == 0 && q.n_iter > 0) finalize_bound(q, q.n_iter - 1, red);
}

// ---------------------------------------------------------------------------------------
// copy-arc pairs of sub-BDDs (Sec. 6, parallel min-marginal averaging)
// ---------------------------------------------------------------------------------------
// arc-marginal of pair k's copy arc after a forward sweep (the best path of the earlier piece
// through it: fm(tail) + theta + mu_bar) or of its entry arc after a backward sweep (the best path
// of the later piece entering through it: mu + bm(head); the entry arc carries no theta, which
// stays with the copy arc's layer)
template <bool FWD>
__device__ __forceinline__ float cut_marginal(const CutParams &c, int k) {
  const int4 q = c.pair[k];
  if (FWD) return c.fm[q.x] + (q.w ? c.lam[q.z] : 0.f) + c.mu_bar[k];
  return c.mu[k] + c.bm[q.y];
}

// root messages of a cut's heads: min of mu over the pairs entering each head
__device__ __forceinline__ void cut_roots(const CutParams &c, int4 G, int lane) {
  for (int h = G.z + lane; h < G.w; h += 32) {
    float r = inf();
    for (int q = c.head_ptr[h]; q < c.head_ptr[h + 1]; ++q) r = fminf(r, c.mu[c.head_pair[q]]);
    c.fm[c.head_node[h]] = r;
  }
}

// one warp per cut of a BDD: delta = marginal - its minimum over the cut (0 where either is
// +inf), then the gamma-damped dual step, each dual offsetting the other side's last delta
template <bool FWD>
__global__ void __launch_bounds__(kBlockThreads) cut_kernel(const CutParams c) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int g = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (g >= c.ngroups) return;
  const int4 G = c.grp[g];
  float mn = inf();
  for (int k = G.x + lane; k < G.y; k += 32) mn = fminf(mn, cut_marginal<FWD>(c, k));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mn = fminf(mn, __shfl_xor_sync(kFull, mn, off));
  for (int k = G.x + lane; k < G.y; k += 32) {
    const float m = cut_marginal<FWD>(c, k);
    const float d = (m < inf() && mn < inf()) ? m - mn : 0.f;
    if (FWD) {
      c.dfwd[k] = d;
      c.mu_bar[k] += -c.gamma * d + c.gamma * c.dbwd[k];
    } else {
      c.dbwd[k] = d;
      c.mu[k] += -c.gamma * d + c.gamma * c.dfwd[k];
    }
  }
  if (!FWD) {
    __syncwarp();  // the cut's new mu, written by all lanes, before the root messages read them
    cut_roots(c, G, lane);
  }
}

__global__ void __launch_bounds__(kBlockThreads) cut_roots_kernel(const CutParams c) {
  const int g = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (g < c.ngroups) cut_roots(c, c.grp[g], threadIdx.x & 31);
}

// ---------------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------------
// lambda^j_i = c_i / |J_i| (Alg. 1 initialisation)
__global__ void init_lambda_kernel(const int *__restrict__ occ_var, const int *__restrict__ var_ptr,
                                   const float *__restrict__ c, float *__restrict__ lam, int O) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < O; o += gridDim.x * blockDim.x) {
    const int i = occ_var[o];
    lam[o] = c[i] / (float)(var_ptr[i + 1] - var_ptr[i]);
  }
}

// pending sums as slot contents: P_i in the first slot of i, 0 in the others (so the slots
// sum to P_i exactly)
__global__ void pending_to_slots_kernel(const int *__restrict__ var_ptr, const float *__restrict__ P,
                                        float *__restrict__ delta_b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = var_ptr[i], e = var_ptr[i + 1];
    for (int k = s; k < e; ++k) delta_b[k] = k == s ? P[i] : 0.f;
  }
}

__global__ void scatter_lambda_kernel(const float *__restrict__ lam, const float *__restrict__ share_occ,
                                      const long long *__restrict__ occ_csr, float *__restrict__ out, int O,
                                      bool fold) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < O; o += gridDim.x * blockDim.x)
    out[occ_csr[o]] = lam[o] + (fold ? share_occ[o] : 0.f);
}

__global__ void gather_lambda_kernel(const float *__restrict__ in, const long long *__restrict__ occ_csr,
                                     float *__restrict__ lam, int O) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < O; o += gridDim.x * blockDim.x)
    lam[o] = in[occ_csr[o]];
}

__global__ void scatter_rows_kernel(const float *__restrict__ bdd_E, const int *__restrict__ bdd_row, int nb,
                                    float *__restrict__ E_row) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += gridDim.x * blockDim.x)
    E_row[bdd_row[j]] = bdd_E[j];
}

// one block per part: sum of E over the part's rows plus min(0, P_i) (min(0, c_i) for a variable
// in no row) over its variables, FP64, strided per thread then a fixed tree
__global__ void __launch_bounds__(kReduceThreads)
    part_bound_kernel(const float *__restrict__ E_row, const long long *__restrict__ row_off,
                      const long long *__restrict__ var_off, const int *__restrict__ var_ptr,
                      const float *__restrict__ P, const float *__restrict__ c, double *__restrict__ out) {
  const int k = blockIdx.x;
  double acc = 0.0;
  for (long long r = row_off[k] + threadIdx.x; r < row_off[k + 1]; r += blockDim.x) acc += (double)E_row[r];
  for (long long i = var_off[k] + threadIdx.x; i < var_off[k + 1]; i += blockDim.x) {
    const float v = var_ptr[i + 1] > var_ptr[i] ? P[i] : c[i];
    if (v < 0.f) acc += (double)v;
  }
  __shared__ double red[kReduceThreads / 32];
  const double s = block_sum(acc, red, kReduceThreads / 32);
  if (threadIdx.x == 0) out[k] = s;
}

// ---------------------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------------------
namespace {
int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}
int status() { return cudaGetLastError() == cudaSuccess ? 0 : -5; }

template <typename... Args>
int launch_pdl(void (*kernel)(Args...), int grid, int block, size_t smem, cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...) == cudaSuccess ? 0 : -5;
}
}  // namespace

size_t sweep_warp_smem(int staging, bool lanes2) {
  const size_t st = staging == 2 ? kWarpSmemBytes2 : kWarpSmemBytes;
  return lanes2 && kLaneSmemBytes > st ? kLaneSmemBytes : st;
}

int sweep_resident_blocks(size_t smem, int *blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, sweep_kernel<true, kUpdate, false, 0, false>,
                                                       kBlockThreads, smem) == cudaSuccess
             ? 0
             : -5;
}

size_t sweep_smem_bytes(int block_buf, int block_depth_buf, int staging, bool lanes2, bool smooth) {
  const size_t warp_part = kWarpsPerBlock * sweep_warp_smem(staging, lanes2);
  const size_t group_part = group_floats(block_buf, block_depth_buf, smooth) * sizeof(float);
  return warp_part > group_part ? warp_part : group_part;
}

// the same for a layout whose warp tiles are all lane tiles (min-sum sweeps)
size_t lane_only_smem_bytes(int block_buf, int block_depth_buf) {
  const size_t warp_part = kWarpsPerBlock * kLaneSmemBytes;
  const size_t group_part = group_floats(block_buf, block_depth_buf, false) * sizeof(float);
  return warp_part > group_part ? warp_part : group_part;
}

size_t persist_smem_bytes(int block_buf, int block_depth_buf) {
  const size_t warp_part = kPersistWarps * kWarpSmemBytes;
  const size_t group_part = kSubBlocks * group_floats(block_buf, block_depth_buf) * sizeof(float);
  return warp_part > group_part ? warp_part : group_part;
}

int sweep_launch(bool forward, int mode, const SweepParams &p_in, int grid, cudaStream_t stream, int staging) {
  if (grid <= 0) return 0;
  if (mode != kUpdate) staging = 0;
  SweepParams p = p_in;
  if (p.lanes2 && (p.alpha > 0.f || p.split || mode == kUpdateFused)) return -5;  // lane tiles: plain min-sum
  if (p.lanes2 && (reinterpret_cast<uintptr_t>(p.lane_code) | reinterpret_cast<uintptr_t>(p.occ_slot) |
                   reinterpret_cast<uintptr_t>(p.lam) | reinterpret_cast<uintptr_t>(p.share_occ) |
                   reinterpret_cast<uintptr_t>(p.fm) | reinterpret_cast<uintptr_t>(p.bm)) & 15u)
    return -5;  // lane-tile windows find their staged elements from 16-byte aligned array starts
  // a layout whose warp tiles are all lane tiles needs only the lane ring's shared memory, so
  // more blocks fit on an SM
  const bool lane_only = p.lanes2 && p.class_tile_off[1] == p.class_tile_off[kWarpClasses];
  p.warp_smem = lane_only ? (int)kLaneSmemBytes : (int)sweep_warp_smem(staging, p.lanes2 != 0);
  size_t smem = sweep_smem_bytes(p.block_buf, p.block_depth_buf, staging, p.lanes2 != 0, p.alpha > 0.f);
  if (lane_only) smem = lane_only_smem_bytes(p.block_buf, p.block_depth_buf);
  int rc = 0;
  if (p.split) {  // sub-BDDs: min-sum only, no fused pending pass
    if (p.alpha > 0.f || mode == kUpdateFused) return -5;
    if (staging == 1)
      rc = forward ? launch_pdl(sweep_kernel<true, kUpdate, false, 1, true>, grid, kBlockThreads, smem, stream, p)
                   : launch_pdl(sweep_kernel<false, kUpdate, false, 1, true>, grid, kBlockThreads, smem, stream, p);
    else if (staging == 2)
      rc = forward ? launch_pdl(sweep_kernel<true, kUpdate, false, 2, true>, grid, kBlockThreads, smem, stream, p)
                   : launch_pdl(sweep_kernel<false, kUpdate, false, 2, true>, grid, kBlockThreads, smem, stream, p);
#define BDD_SPLIT_SWEEP(F, M) rc = launch_pdl(sweep_kernel<F, M, false, 0, true>, grid, kBlockThreads, smem, stream, p)
    else if (forward && mode == kUpdate) BDD_SPLIT_SWEEP(true, kUpdate);
    else if (forward && mode == kMessages) BDD_SPLIT_SWEEP(true, kMessages);
    else if (forward) BDD_SPLIT_SWEEP(true, kFolded);
    else if (mode == kUpdate) BDD_SPLIT_SWEEP(false, kUpdate);
    else if (mode == kMessages) BDD_SPLIT_SWEEP(false, kMessages);
    else BDD_SPLIT_SWEEP(false, kFolded);
#undef BDD_SPLIT_SWEEP
    return rc ? rc : status();
  }
  if (mode == kUpdate && staging == 1) {
    if (p.alpha > 0.f)
      rc = forward ? launch_pdl(sweep_kernel<true, kUpdate, true, 1>, grid, kBlockThreads, smem, stream, p)
                   : launch_pdl(sweep_kernel<false, kUpdate, true, 1>, grid, kBlockThreads, smem, stream, p);
    else
      rc = forward ? launch_pdl(sweep_kernel<true, kUpdate, false, 1>, grid, kBlockThreads, smem, stream, p)
                   : launch_pdl(sweep_kernel<false, kUpdate, false, 1>, grid, kBlockThreads, smem, stream, p);
    return rc ? rc : status();
  }
  if (mode == kUpdate && staging == 2) {
    if (p.alpha > 0.f)
      rc = forward ? launch_pdl(sweep_kernel<true, kUpdate, true, 2>, grid, kBlockThreads, smem, stream, p)
                   : launch_pdl(sweep_kernel<false, kUpdate, true, 2>, grid, kBlockThreads, smem, stream, p);
    else
      rc = forward ? launch_pdl(sweep_kernel<true, kUpdate, false, 2>, grid, kBlockThreads, smem, stream, p)
                   : launch_pdl(sweep_kernel<false, kUpdate, false, 2>, grid, kBlockThreads, smem, stream, p);
    return rc ? rc : status();
  }
#define BDD_SWEEP(F, M)                                                                          \
  rc = p.alpha > 0.f ? launch_pdl(sweep_kernel<F, M, true>, grid, kBlockThreads, smem, stream, p)    \
                     : launch_pdl(sweep_kernel<F, M, false>, grid, kBlockThreads, smem, stream, p)
  if (forward) {
    if (mode == kUpdate) BDD_SWEEP(true, kUpdate);
    else if (mode == kUpdateFused) BDD_SWEEP(true, kUpdateFused);
    else if (mode == kMessages) BDD_SWEEP(true, kMessages);
    else BDD_SWEEP(true, kFolded);
  } else {
    if (mode == kUpdate) BDD_SWEEP(false, kUpdate);
    else if (mode == kUpdateFused) BDD_SWEEP(false, kUpdateFused);
    else if (mode == kMessages) BDD_SWEEP(false, kMessages);
    else BDD_SWEEP(false, kFolded);
  }
#undef BDD_SWEEP
  return rc ? rc : status();
}

int sweep_set_smem(size_t bytes) {
  const void *fns[] = {
      (const void *)sweep_kernel<true, kUpdate, false>,    (const void *)sweep_kernel<true, kMessages, false>,
      (const void *)sweep_kernel<true, kFolded, false>,    (const void *)sweep_kernel<false, kUpdate, false>,
      (const void *)sweep_kernel<false, kMessages, false>, (const void *)sweep_kernel<false, kFolded, false>,
      (const void *)sweep_kernel<true, kUpdate, true>,     (const void *)sweep_kernel<true, kMessages, true>,
      (const void *)sweep_kernel<true, kFolded, true>,     (const void *)sweep_kernel<false, kUpdate, true>,
      (const void *)sweep_kernel<false, kMessages, true>,  (const void *)sweep_kernel<false, kFolded, true>,
      (const void *)sweep_kernel<true, kUpdateFused, false>, (const void *)sweep_kernel<false, kUpdateFused, false>,
      (const void *)sweep_kernel<true, kUpdateFused, true>,  (const void *)sweep_kernel<false, kUpdateFused, true>,
      (const void *)sweep_kernel<true, kUpdate, false, 1>,   (const void *)sweep_kernel<false, kUpdate, false, 1>,
      (const void *)sweep_kernel<true, kUpdate, true, 1>,    (const void *)sweep_kernel<false, kUpdate, true, 1>,
      (const void *)sweep_kernel<true, kUpdate, false, 0, true>,   (const void *)sweep_kernel<false, kUpdate, false, 0, true>,
      (const void *)sweep_kernel<true, kMessages, false, 0, true>, (const void *)sweep_kernel<false, kMessages, false, 0, true>,
      (const void *)sweep_kernel<true, kFolded, false, 0, true>,   (const void *)sweep_kernel<false, kFolded, false, 0, true>,
      (const void *)sweep_kernel<true, kUpdate, false, 1, true>,   (const void *)sweep_kernel<false, kUpdate, false, 1, true>,
      (const void *)sweep_kernel<true, kUpdate, false, 2>,         (const void *)sweep_kernel<false, kUpdate, false, 2>,
      (const void *)sweep_kernel<true, kUpdate, true, 2>,          (const void *)sweep_kernel<false, kUpdate, true, 2>,
      (const void *)sweep_kernel<true, kUpdate, false, 2, true>,   (const void *)sweep_kernel<false, kUpdate, false, 2, true>};
  for (const void *f : fns)
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
      return -5;
  return 0;
}

int iterate_set_smem(size_t bytes) {
  return cudaFuncSetAttribute((const void *)iterate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes) == cudaSuccess ? 0 : -5;
}

int bound_launch(const SweepParams &p, int grid, cudaStream_t stream) {
  const int rc = launch_pdl(bound_kernel, grid, kReduceThreads, 0, stream, p);
  return rc ? rc : status();
}

int bound_finish_launch(const double *partial, int nblocks, int *iter_ctr, double *trace, int cap,
                        double empty_const, cudaStream_t stream) {
  const int rc = launch_pdl(bound_finish_kernel, 1, 32, 0, stream, partial, nblocks, iter_ctr, trace, cap,
                            empty_const);
  return rc ? rc : status();
}

int pending_launch(bool bound, const PendingParams &p, int grid, cudaStream_t stream) {
  int rc;
  if (p.alpha > 0.0)
    rc = bound ? launch_pdl(pending_kernel<true, true>, grid, kReduceThreads, 0, stream, p)
               : launch_pdl(pending_kernel<false, true>, grid, kReduceThreads, 0, stream, p);
  else
    rc = bound ? launch_pdl(pending_kernel<true, false>, grid, kReduceThreads, 0, stream, p)
               : launch_pdl(pending_kernel<false, false>, grid, kReduceThreads, 0, stream, p);
  return rc ? rc : status();
}

int iterate_persistent_max_grid(size_t smem, int *grid) {
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -5;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return -5;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -5;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iterate_kernel, kPersistThreads, smem) != cudaSuccess)
    return -5;
  *grid = sms * per_sm;
  return *grid > 0 ? 0 : -5;
}

int iterate_persistent_launch(const IterParams &q, int grid, size_t smem, cudaStream_t stream) {
  void *args[] = {const_cast<IterParams *>(&q)};
  if (cudaLaunchCooperativeKernel((const void *)iterate_kernel, dim3(grid), dim3(kPersistThreads), args, smem,
                                  stream) != cudaSuccess)
    return -5;
  return status();
}

int init_lambda_launch(const int *occ_var, const int *var_ptr, const float *c, float *lam, int O,
                       cudaStream_t stream) {
  if (O == 0) return 0;
  init_lambda_kernel<<<grid_for(O, 256), 256, 0, stream>>>(occ_var, var_ptr, c, lam, O);
  return status();
}

int pending_to_slots_launch(const int *var_ptr, const float *P, float *delta_b, int n, cudaStream_t stream) {
  if (n == 0) return 0;
  pending_to_slots_kernel<<<grid_for(n, 256), 256, 0, stream>>>(var_ptr, P, delta_b, n);
  return status();
}

int scatter_lambda_launch(const float *lam, const float *share_occ, const long long *occ_csr, float *out, int O,
                          bool fold, cudaStream_t stream) {
  if (O == 0) return 0;
  scatter_lambda_kernel<<<grid_for(O, 256), 256, 0, stream>>>(lam, share_occ, occ_csr, out, O, fold);
  return status();
}

int part_bounds_launch(const float *bdd_E, const int *bdd_row, int nb, float *E_row, int m, const long long *row_off,
                       const long long *var_off, int nparts, const int *var_ptr, const float *P, const float *c,
                       double *out, cudaStream_t stream) {
  if (m > 0 && cudaMemsetAsync(E_row, 0, sizeof(float) * m, stream) != cudaSuccess) return -5;
  if (nb > 0) scatter_rows_kernel<<<grid_for(nb, 256), 256, 0, stream>>>(bdd_E, bdd_row, nb, E_row);
  part_bound_kernel<<<nparts, kReduceThreads, 0, stream>>>(E_row, row_off, var_off, var_ptr, P, c, out);
  return status();
}

int gather_lambda_launch(const float *in, const long long *occ_csr, float *lam, int O, cudaStream_t stream) {
  if (O == 0) return 0;
  gather_lambda_kernel<<<grid_for(O, 256), 256, 0, stream>>>(in, occ_csr, lam, O);
  return status();
}

int cut_launch(bool forward, const CutParams &c, cudaStream_t stream) {
  if (c.ngroups <= 0) return 0;
  const int grid = (c.ngroups + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int rc = forward ? launch_pdl(cut_kernel<true>, grid, kBlockThreads, 0, stream, c)
                         : launch_pdl(cut_kernel<false>, grid, kBlockThreads, 0, stream, c);
  return rc ? rc : status();
}

int cut_roots_launch(const CutParams &c, cudaStream_t stream) {
  if (c.ngroups <= 0) return 0;
  cut_roots_kernel<<<(c.ngroups + kWarpsPerBlock - 1) / kWarpsPerBlock, kBlockThreads, 0, stream>>>(c);
  return status();
}

}  // namespace bdd
