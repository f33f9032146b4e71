// Reverse-mode adjoints of the smoothed iteration (Appendix A.5), for the gradient of the
// smoothed bound after K iterations with respect to the costs c.
//
// The forward map of one update sweep of one BDD (warp tiles: T lanes, lane t = node t; block
// tiles of at most 128 nodes per layer: thread t = node t):
//   forward sweep, layers l ascending:
//     fm_l(v)  = softmin over in-arcs (u, v) of fm_{l-1}(u) + theta_uv   (theta = lam''_{l-1} on
//                1-arcs, 0 on 0-arcs; fm_0(root) = 0)                                  (Alg. 2)
//     lam'_l   = lam_l + s_l                        (s_l: the pending share)
//     m0, m1   = softmin over v of fm_l(v) + bmp(lo v),  fm_l(v) + lam'_l + bmp(hi v)
//     lam''_l  = lam'_l - omega (m1 - m0);  delta_l = omega (m1 - m0)
//   where bmp are the backward messages of the sweep's starting multipliers (Alg. 3 recursion).
//   backward sweep, layers l descending: the mirror image, with fmp (forward messages of the
//   starting multipliers) in the marginals and the new backward messages
//     bmn_l(v) = softmin(bmn_{l+1}(lo v), lam''_l + bmn_{l+1}(hi v)).
// The derivative of softmin_k x_k with respect to x_k is exp(-(x_k - softmin)/alpha); every
// adjoint below is that weight times the adjoint of the soft minimum, pushed or pulled along
// the same arcs the forward map uses.  Messages and updated multipliers are recomputed from
// per-sweep checkpoints (multipliers and shares) by the forward kernels before each adjoint.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace bdd {
namespace {

// softmin weight of an argument x whose soft minimum is m (x >= m up to rounding)
__device__ __forceinline__ float weight(float x, float m, float inv_alpha) {
  if (x == inf() || m == inf()) return 0.f;
  return expf(-(x - m) * inv_alpha);
}

// message of an arc target: top -> 0, bot / none -> +inf, node -> msg
__device__ __forceinline__ float target_msg(const float *__restrict__ msg, int t) {
  if (t >= 0) return msg[t];
  return t == kTop ? 0.f : inf();
}

// Push: every lane, as target index tl of the next layer, sums the contributions c0 (along
// 0-arcs, target lo_rel) and c1 (along 1-arcs, target hi_rel) of the team's source lanes, in
// source order.
template <int T>
__device__ __forceinline__ float team_push(int lo_rel, int hi_rel, float c0, float c1, int tbase, int tl) {
  float acc = 0.f;
#pragma unroll
  for (int s = 0; s < T; ++s) {
    const int ls = __shfl_sync(kFull, lo_rel, tbase + s);
    const int hs = __shfl_sync(kFull, hi_rel, tbase + s);
    const float x0 = __shfl_sync(kFull, c0, tbase + s);
    const float x1 = __shfl_sync(kFull, c1, tbase + s);
    if (ls == tl) acc += x0;
    if (hs == tl) acc += x1;
  }
  return acc;
}

struct Team {
  int lane, team, tl, tbase, occ0, bdd, depth, lead_depth, maxd;
};

template <int T>
__device__ __forceinline__ Team team_of(const SweepParams &p, int tile) {
  Team m;
  m.lane = threadIdx.x & 31;
  m.team = m.lane / T;
  m.tl = m.lane % T;
  m.tbase = m.team * T;
  m.occ0 = p.tile_occ0[tile];
  m.bdd = p.tile_bdd0[tile] + m.team;
  const bool valid = m.team < p.tile_nbdd[tile];
  m.depth = valid ? p.bdd_depth[m.bdd] : 0;
  m.lead_depth = m.tl == 0 ? m.depth : 0;
  m.maxd = __reduce_max_sync(kFull, m.depth);
  return m;
}

// Per-layer values of a warp team's BDD (its occurrence, node range, multipliers and slot),
// loaded one layer ahead of their use so that a layer waits on one round of dependent loads
// (arcs and messages of its nodes) instead of three.  Warp-collective: every lane calls it with
// the same l.
struct LayerVals {
  int o, node0, w, slot;
  float lam_s, shr_s, lam2;
};

template <int T>
__device__ __forceinline__ LayerVals layer_vals(const AdjParams &a, const Team &m, int l) {
  LayerVals v{};
  v.o = m.occ0 + occ_before(m.lead_depth, l) + m.team;
  if (l >= 0 && m.depth > l) {
    v.node0 = a.sp.occ_node_off[v.o];
    v.w = a.sp.occ_node_off[v.o + 1] - v.node0;
    v.lam_s = a.lam_s[v.o];
    v.shr_s = a.shr_s[v.o];
    v.lam2 = a.lam2[v.o];
    v.slot = a.sp.occ_slot[v.o];
  }
  return v;
}

// The loads of one layer of a warp team's BDD, in three stages that a loop issues for three
// consecutive layers ahead of their use: the layer's per-occurrence values (their addresses need
// no load), the lane's node (its arcs, two per-node values, and the adjoints of the layer's
// outputs), and the messages of the node's arc targets (their addresses are the arcs).  A layer's
// step then waits on no load it issued: the arcs were loaded two layers earlier, the target
// messages one layer earlier.  Only the timing of the loads differs from loading each value where
// it is used; the arithmetic and its order are unchanged.
struct Ahead {
  LayerVals v;
  int2 lh;       // the node's arcs (kNone for a lane without a node)
  float x, y;    // two per-node values (which arrays depends on the loop); 0 without a node
  float gl, gd;  // adjoints of the updated multiplier (by occurrence) and of the difference (by slot)
  float b0, b1;  // messages of the 0- and 1-arc targets (target_msg)
};

// node stage of layer l: X and Y are read at the lane's node if Y_ok (Y may be null); with outs,
// the adjoints of the layer's outputs; with IN, g_in_lam at the layer's occurrence (into gl)
template <int T>
__device__ __forceinline__ void ahead_node(Ahead &q, const AdjParams &a, const Team &m, int l, const float *X,
                                           const float *Y, bool y_ok, bool outs, bool in = false) {
  const bool active = l >= 0 && m.depth > l;
  const bool has = active && m.tl < q.v.w;
  const int nd = q.v.node0 + m.tl;
  q.lh = make_int2(kNone, kNone);
  q.x = q.y = q.gl = q.gd = 0.f;
  if (has) {
    q.lh = a.sp.lohi[nd];
    q.x = X[nd];
    if (Y && y_ok) q.y = Y[nd];
  }
  if (active && outs) {
    q.gl = a.g_out_lam[q.v.o];
    q.gd = a.g_out_delta[q.v.slot];
  }
  if (active && in && m.tl == 0) q.gl = a.g_in_lam[q.v.o];
}

__device__ __forceinline__ void ahead_targets(Ahead &q, const float *msg) {
  q.b0 = target_msg(msg, q.lh.x);  // kNone: +inf, as for a lane without a node
  q.b1 = target_msg(msg, q.lh.y);
}

// Adjoint of a forward update sweep.  Descending layers: the node adjoint G of fm_l is pulled
// from the children (the forward step into layer l+1), the marginal terms are added, and their
// contributions to the starting backward messages of layer l+1 are pushed into g_node.  Then,
// ascending, the adjoint of those backward messages runs back through their recursion into the
// starting multipliers.
template <int T>
__device__ void fwd_adjoint_tile(const AdjParams &a, int tile) {
  const SweepParams &p = a.sp;
  const Team m = team_of<T>(p, tile);
  const float ia = p.inv_alpha;
  float G_next = 0.f, f_next = inf();
  int node0_next = 0, w_next = 0;
  // c: layer l (all stages), n1: layer l - 1 (node stage), n2: layer l - 2 (layer values)
  Ahead c, n1, n2;
  c.v = layer_vals<T>(a, m, m.maxd - 1);
  ahead_node<T>(c, a, m, m.maxd - 1, a.msg_new, nullptr, false, true);
  ahead_targets(c, a.msg_pre);
  n1.v = layer_vals<T>(a, m, m.maxd - 2);
  ahead_node<T>(n1, a, m, m.maxd - 2, a.msg_new, nullptr, false, true);
  n2.v = layer_vals<T>(a, m, m.maxd - 3);
  for (int l = m.maxd - 1; l >= 0; --l) {
    const Ahead q = c;
    c = n1;
    ahead_targets(c, a.msg_pre);
    n1 = n2;
    ahead_node<T>(n1, a, m, l - 2, a.msg_new, nullptr, false, true);
    n2.v = layer_vals<T>(a, m, l - 3);
    const LayerVals &v = q.v;
    const bool active = m.depth > l;
    const bool nxt = active && l + 1 < m.depth;
    const int o = v.o;
    const int node0 = active ? v.node0 : 0, w = active ? v.w : 0;
    const bool has = active && m.tl < w;
    const int2 lh = q.lh;
    const float f = has ? q.x : inf();
    const float lam1 = active ? v.lam_s + v.shr_s : 0.f;
    const float lam2 = active ? v.lam2 : 0.f;
    // pull the adjoint of fm_{l+1} through the forward step from layer l
    const int lo_loc = nxt && lh.x >= 0 ? lh.x - node0_next : -1;
    const int hi_loc = nxt && lh.y >= 0 ? lh.y - node0_next : -1;
    const float Gc0 = __shfl_sync(kFull, G_next, m.tbase + ((lo_loc < 0 ? 0 : lo_loc) & (T - 1)));
    const float fc0 = __shfl_sync(kFull, f_next, m.tbase + ((lo_loc < 0 ? 0 : lo_loc) & (T - 1)));
    const float Gc1 = __shfl_sync(kFull, G_next, m.tbase + ((hi_loc < 0 ? 0 : hi_loc) & (T - 1)));
    const float fc1 = __shfl_sync(kFull, f_next, m.tbase + ((hi_loc < 0 ? 0 : hi_loc) & (T - 1)));
    float G = 0.f, g_theta = 0.f;
    if (lo_loc >= 0) G += Gc0 * weight(f, fc0, ia);
    if (hi_loc >= 0) {
      g_theta = Gc1 * weight(f + lam2, fc1, ia);
      G += g_theta;
    }
    const float G_lam2 = q.gl + team_sum<T>(g_theta);
    // marginals of layer l and the update
    const float b0 = has ? q.b0 : inf();
    const float b1 = has ? q.b1 : inf();
    const float a0 = has ? f + b0 : inf(), a1 = has ? f + lam1 + b1 : inf();
    const float m0 = team_agg<T, true>(a0, p), m1 = team_agg<T, true>(a1, p);
    const bool finite = m0 < inf() && m1 < inf();
    const float gd = finite ? p.omega * (q.gd - G_lam2) : 0.f;  // adjoint of m1 - m0
    const float p0 = weight(a0, m0, ia), p1 = weight(a1, m1, ia);
    G += -gd * p0 + gd * p1;
    const float g_lam1 = G_lam2 + gd;  // d m1 / d lam' = 1
    if (active && m.tl == 0) {
      a.g_in_lam[o] = g_lam1;
      a.g_shr[o] = g_lam1;
    }
    // contributions to the starting backward messages of layer l + 1
    const int lo_rel = has && lh.x >= 0 && nxt ? lh.x - node0_next : kNone;
    const int hi_rel = has && lh.y >= 0 && nxt ? lh.y - node0_next : kNone;
    const float acc = team_push<T>(lo_rel, hi_rel, -gd * p0, gd * p1, m.tbase, m.tl);
    if (nxt && m.tl < w_next) a.g_node[node0_next + m.tl] = acc;
    G_next = has ? G : 0.f;
    f_next = f;
    node0_next = node0;
    w_next = w;
  }
  __syncwarp();
  // the starting backward messages: bmp_l(v) = softmin(bmp_{l+1}(lo), lam_l + bmp_{l+1}(hi)),
  // adjoints flowing from layer l to layer l + 1.  Node values: x = bmp (msg_pre), y = g_node
  // (written above by the same lane), gl = g_in_lam (written above).
  float carry = 0.f;
  c.v = layer_vals<T>(a, m, 0);
  ahead_node<T>(c, a, m, 0, a.msg_pre, a.g_node, false, false, true);
  ahead_targets(c, a.msg_pre);
  n1.v = layer_vals<T>(a, m, 1);
  ahead_node<T>(n1, a, m, 1, a.msg_pre, a.g_node, true, false, true);
  n2.v = layer_vals<T>(a, m, 2);
  for (int l = 0; l < m.maxd; ++l) {
    const Ahead q = c;
    c = n1;  // the next layer: its node stage arrived, its targets in flight
    ahead_targets(c, a.msg_pre);
    n1 = n2;
    ahead_node<T>(n1, a, m, l + 2, a.msg_pre, a.g_node, true, false, true);
    n2.v = layer_vals<T>(a, m, l + 3);
    const LayerVals &v = q.v;
    const bool active = m.depth > l;
    const bool nxt = active && l + 1 < m.depth;
    const int o = v.o;
    const int w = active ? v.w : 0;
    const int node0n = nxt ? c.v.node0 : 0;
    const bool has = active && m.tl < w;
    const int2 lh = q.lh;
    const float bn = has ? q.x : inf();
    const float Gb = has && l >= 1 ? q.y + carry : 0.f;
    const float lam = active ? v.lam_s : 0.f;
    const float b0 = has ? q.b0 : inf();
    const float b1 = has ? q.b1 : inf();
    const float q0 = has ? weight(b0, bn, ia) : 0.f;
    const float q1 = has ? weight(lam + b1, bn, ia) : 0.f;
    const float gl = team_sum<T>(Gb * q1);
    if (active && m.tl == 0) a.g_in_lam[o] = q.gl + gl;
    const int lo_rel = has && lh.x >= 0 && nxt ? lh.x - node0n : kNone;
    const int hi_rel = has && lh.y >= 0 && nxt ? lh.y - node0n : kNone;
    carry = team_push<T>(lo_rel, hi_rel, Gb * q0, Gb * q1, m.tbase, m.tl);
  }
}

// Adjoint of a backward update sweep.  Ascending layers (the reverse of the sweep): the adjoint of
// the new backward messages of layer l (seeded at the root with gE) runs through the backward
// step and, with the marginal terms, is pushed to layer l + 1; the marginal terms' adjoints of
// the starting forward messages go to g_node.  Then, descending, those run back through the
// forward recursion into the starting multipliers.
template <int T>
__device__ void bwd_adjoint_tile(const AdjParams &a, int tile) {
  const SweepParams &p = a.sp;
  const Team m = team_of<T>(p, tile);
  const float ia = p.inv_alpha;
  float carry = 0.f;
  const float gE = m.tl == 0 && a.gE ? (float)*a.gE : 0.f;
  // node values: x = fmp (msg_pre), y = bmn (msg_new); targets from msg_new
  Ahead c, n1, n2;
  c.v = layer_vals<T>(a, m, 0);
  ahead_node<T>(c, a, m, 0, a.msg_pre, a.msg_new, true, true);
  ahead_targets(c, a.msg_new);
  n1.v = layer_vals<T>(a, m, 1);
  ahead_node<T>(n1, a, m, 1, a.msg_pre, a.msg_new, true, true);
  n2.v = layer_vals<T>(a, m, 2);
  for (int l = 0; l < m.maxd; ++l) {
    const Ahead q = c;
    c = n1;  // the next layer: its node stage arrived, its targets in flight
    ahead_targets(c, a.msg_new);
    n1 = n2;
    ahead_node<T>(n1, a, m, l + 2, a.msg_pre, a.msg_new, true, true);
    n2.v = layer_vals<T>(a, m, l + 3);
    const LayerVals &v = q.v;
    const bool active = m.depth > l;
    const bool nxt = active && l + 1 < m.depth;
    const int o = v.o;
    const int node0 = active ? v.node0 : 0, w = active ? v.w : 0;
    const int node0n = nxt ? c.v.node0 : 0;
    const bool has = active && m.tl < w;
    const int2 lh = q.lh;
    const float fp = has ? q.x : inf(), bn = has ? q.y : inf();
    const float Gbn = has ? (l == 0 ? gE : carry) : 0.f;
    const float lam1 = active ? v.lam_s + v.shr_s : 0.f;
    const float lam2 = active ? v.lam2 : 0.f;
    const float b0 = has ? q.b0 : inf();
    const float b1 = has ? q.b1 : inf();
    // backward step bmn_l = softmin(b0, lam'' + b1)
    const float q0 = has ? weight(b0, bn, ia) : 0.f;
    const float q1 = has ? weight(lam2 + b1, bn, ia) : 0.f;
    const float G_lam2 = q.gl + team_sum<T>(Gbn * q1);
    // marginals and the update
    const float a0 = has ? fp + b0 : inf(), a1 = has ? fp + lam1 + b1 : inf();
    const float m0 = team_agg<T, true>(a0, p), m1 = team_agg<T, true>(a1, p);
    const bool finite = m0 < inf() && m1 < inf();
    const float gd = finite ? p.omega * (q.gd - G_lam2) : 0.f;
    const float p0 = weight(a0, m0, ia), p1 = weight(a1, m1, ia);
    if (has) a.g_node[node0 + m.tl] = -gd * p0 + gd * p1;  // adjoint of fmp_l(v), marginal part
    const float g_lam1 = G_lam2 + gd;
    if (active && m.tl == 0) {
      a.g_in_lam[o] = g_lam1;
      a.g_shr[o] = g_lam1;
    }
    const int lo_rel = has && lh.x >= 0 && nxt ? lh.x - node0n : kNone;
    const int hi_rel = has && lh.y >= 0 && nxt ? lh.y - node0n : kNone;
    carry = team_push<T>(lo_rel, hi_rel, Gbn * q0 - gd * p0, Gbn * q1 + gd * p1, m.tbase, m.tl);
  }
  __syncwarp();
  // the starting forward messages: fmp_l(v) = softmin over in-arcs of fmp_{l-1}(u) + theta,
  // adjoints flowing from layer l + 1 back to layer l.  Node values: x = fmp, y = g_node (written
  // above by the same lane), gl = g_in_lam (written above); no target messages.
  float G_next = 0.f, f_next = inf();
  int node0_next = 0;
  c.v = layer_vals<T>(a, m, m.maxd - 1);
  ahead_node<T>(c, a, m, m.maxd - 1, a.msg_pre, a.g_node, true, false, true);
  n1.v = layer_vals<T>(a, m, m.maxd - 2);
  for (int l = m.maxd - 1; l >= 0; --l) {
    const Ahead q = c;
    c = n1;
    ahead_node<T>(c, a, m, l - 1, a.msg_pre, a.g_node, true, false, true);
    n1.v = layer_vals<T>(a, m, l - 2);
    const LayerVals &v = q.v;
    const bool active = m.depth > l;
    const bool nxt = active && l + 1 < m.depth;
    const int o = v.o;
    const int node0 = active ? v.node0 : 0, w = active ? v.w : 0;
    const bool has = active && m.tl < w;
    const int2 lh = q.lh;
    const float f = has ? q.x : inf();
    float G = has ? q.y : 0.f;
    const float lam = active ? v.lam_s : 0.f;
    const int lo_loc = nxt && lh.x >= 0 ? lh.x - node0_next : -1;
    const int hi_loc = nxt && lh.y >= 0 ? lh.y - node0_next : -1;
    const float Gc0 = __shfl_sync(kFull, G_next, m.tbase + ((lo_loc < 0 ? 0 : lo_loc) & (T - 1)));
    const float fc0 = __shfl_sync(kFull, f_next, m.tbase + ((lo_loc < 0 ? 0 : lo_loc) & (T - 1)));
    const float Gc1 = __shfl_sync(kFull, G_next, m.tbase + ((hi_loc < 0 ? 0 : hi_loc) & (T - 1)));
    const float fc1 = __shfl_sync(kFull, f_next, m.tbase + ((hi_loc < 0 ? 0 : hi_loc) & (T - 1)));
    float g_theta = 0.f;
    if (lo_loc >= 0) G += Gc0 * weight(f, fc0, ia);
    if (hi_loc >= 0) {
      g_theta = Gc1 * weight(f + lam, fc1, ia);
      G += g_theta;
    }
    const float gl = team_sum<T>(g_theta);
    if (active && m.tl == 0) a.g_in_lam[o] = q.gl + gl;
    G_next = has ? G : 0.f;
    f_next = f;
    node0_next = node0;
  }
}

// ---------------------------------------------------------------------------------------
// block tiles (one 128-thread block per BDD of at most kBlockThreads nodes per layer, thread t =
// node t): the same adjoints as the warp tiles, with the team shuffles replaced by shared-memory
// exchanges.  A push along the arcs of layer l into layer l + 1 becomes a pull: node c of layer
// l + 1 sums the contributions of the nodes of layer l whose arcs enter it, in node order (0-arc
// before 1-arc), so the sums do not depend on timing.  Reductions over a layer go warp by warp
// and then over the warps in order; the soft minima of a layer are the forward sweep's
// group_agg2 reduction (the same order, so the same values).
// ---------------------------------------------------------------------------------------
struct BlockAdjSmem {
  float G[kBlockThreads];   // adjoints of layer l + 1's nodes (pull from children)
  float F[kBlockThreads];   // their messages
  int2 arcs[kBlockThreads]; // arcs of layer l
  float c0[kBlockThreads], c1[kBlockThreads];  // contributions along the 0- and 1-arcs
  float red[kWarpsPerBlock];
  float2 red2[kWarpsPerBlock];
};

// sum over the block, the same value on every thread (warp sums, then the warps in order)
__device__ __forceinline__ float block_sum_f(float v, float *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = team_sum<32>(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float r = red[0];
#pragma unroll
  for (int t = 1; t < kWarpsPerBlock; ++t) r += red[t];
  __syncthreads();
  return r;
}

// soft minima of a and b over the block (group_agg2 of the sweeps, the same order)
__device__ __forceinline__ float2 block_softmin2(float a, float b, const SweepParams &p, float2 *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = team_agg<32, true>(a, p);
  b = team_agg<32, true>(b, p);
  if (lane == 0) red[warp] = make_float2(a, b);
  __syncthreads();
  float2 r = red[0];
#pragma unroll
  for (int t = 1; t < kWarpsPerBlock; ++t) {
    r.x = soft_min(r.x, red[t].x, p.alpha, p.inv_alpha);
    r.y = soft_min(r.y, red[t].y, p.alpha, p.inv_alpha);
  }
  __syncthreads();
  return r;
}

// node c (< w_next) of layer l + 1, starting at node0n: the sum of the contributions along the
// arcs of layer l's w nodes that enter it (S.arcs, S.c0, S.c1 filled before a barrier)
__device__ __forceinline__ float pull_sum(const BlockAdjSmem &S, int w, int node0n, int c) {
  const int v = node0n + c;
  float acc = 0.f;
  for (int u = 0; u < w; ++u) {
    const int2 q = S.arcs[u];
    if (q.x == v) acc += S.c0[u];
    if (q.y == v) acc += S.c1[u];
  }
  return acc;
}

__device__ void fwd_adjoint_block(const AdjParams &a, int tile, BlockAdjSmem &S) {
  const SweepParams &p = a.sp;
  const float ia = p.inv_alpha;
  const int gt = threadIdx.x;
  const int bdd = p.tile_bdd0[tile], occ0 = p.tile_occ0[tile], depth = p.bdd_depth[bdd];
  // descending layers: adjoint of fm_l pulled from the children, the marginal terms, their
  // contributions to the starting backward messages of layer l + 1 (g_node)
  for (int l = depth - 1; l >= 0; --l) {
    const int o = occ0 + l;
    const int node0 = p.occ_node_off[o], w = p.occ_node_off[o + 1] - node0;
    const bool nxt = l + 1 < depth;
    const int node0n = node0 + w, wn = nxt ? p.occ_node_off[o + 2] - node0n : 0;
    const bool has = gt < w;
    int2 lh = make_int2(kNone, kNone);
    float f = inf();
    if (has) {
      lh = p.lohi[node0 + gt];
      f = a.msg_new[node0 + gt];
    }
    const float lam1 = a.lam_s[o] + a.shr_s[o], lam2 = a.lam2[o];
    float G = 0.f, g_theta = 0.f;
    if (has && nxt) {  // S.G, S.F: layer l + 1 (written at the end of the previous step)
      if (lh.x >= 0) G += S.G[lh.x - node0n] * weight(f, S.F[lh.x - node0n], ia);
      if (lh.y >= 0) {
        g_theta = S.G[lh.y - node0n] * weight(f + lam2, S.F[lh.y - node0n], ia);
        G += g_theta;
      }
    }
    const float G_lam2 = a.g_out_lam[o] + block_sum_f(g_theta, S.red);
    const float b0 = has ? target_msg(a.msg_pre, lh.x) : inf();
    const float b1 = has ? target_msg(a.msg_pre, lh.y) : inf();
    const float a0 = has ? f + b0 : inf(), a1 = has ? f + lam1 + b1 : inf();
    const float2 mm = block_softmin2(a0, a1, p, S.red2);
    const bool finite = mm.x < inf() && mm.y < inf();
    const float gd = finite ? p.omega * (a.g_out_delta[p.occ_slot[o]] - G_lam2) : 0.f;
    const float p0 = weight(a0, mm.x, ia), p1 = weight(a1, mm.y, ia);
    G += -gd * p0 + gd * p1;
    if (gt == 0) {
      a.g_in_lam[o] = G_lam2 + gd;
      a.g_shr[o] = G_lam2 + gd;
    }
    if (gt < kBlockThreads) {
      S.arcs[gt] = nxt ? lh : make_int2(kNone, kNone);
      S.c0[gt] = -gd * p0;
      S.c1[gt] = gd * p1;
    }
    __syncthreads();
    if (gt < wn) a.g_node[node0n + gt] = pull_sum(S, w, node0n, gt);
    __syncthreads();  // S.G / S.F of layer l + 1 no longer read
    S.G[gt] = has ? G : 0.f;
    S.F[gt] = f;
    __syncthreads();
  }
  // ascending layers: the starting backward messages bmp_l(v) = softmin(bmp_{l+1}(lo),
  // lam_l + bmp_{l+1}(hi)), adjoints flowing from layer l to layer l + 1
  float carry = 0.f;
  for (int l = 0; l < depth; ++l) {
    const int o = occ0 + l;
    const int node0 = p.occ_node_off[o], w = p.occ_node_off[o + 1] - node0;
    const bool nxt = l + 1 < depth;
    const int node0n = node0 + w, wn = nxt ? p.occ_node_off[o + 2] - node0n : 0;
    const bool has = gt < w;
    int2 lh = make_int2(kNone, kNone);
    float bn = inf(), Gb = 0.f;
    if (has) {
      lh = p.lohi[node0 + gt];
      bn = a.msg_pre[node0 + gt];
      if (l >= 1) Gb = a.g_node[node0 + gt] + carry;
    }
    const float lam = a.lam_s[o];
    const float b0 = has ? target_msg(a.msg_pre, lh.x) : inf();
    const float b1 = has ? target_msg(a.msg_pre, lh.y) : inf();
    const float q0 = has ? weight(b0, bn, ia) : 0.f;
    const float q1 = has ? weight(lam + b1, bn, ia) : 0.f;
    const float gl = block_sum_f(Gb * q1, S.red);
    if (gt == 0) a.g_in_lam[o] += gl;
    S.arcs[gt] = nxt ? lh : make_int2(kNone, kNone);
    S.c0[gt] = Gb * q0;
    S.c1[gt] = Gb * q1;
    __syncthreads();
    carry = gt < wn ? pull_sum(S, w, node0n, gt) : 0.f;
    __syncthreads();
  }
}

__device__ void bwd_adjoint_block(const AdjParams &a, int tile, BlockAdjSmem &S) {
  const SweepParams &p = a.sp;
  const float ia = p.inv_alpha;
  const int gt = threadIdx.x;
  const int bdd = p.tile_bdd0[tile], occ0 = p.tile_occ0[tile], depth = p.bdd_depth[bdd];
  // ascending layers (the reverse of the sweep): the adjoint of bmn_l (seeded at the root with
  // gE) through the backward step and, with the marginal terms, on to layer l + 1; the marginal
  // terms' adjoints of the starting forward messages go to g_node
  float carry = 0.f;
  for (int l = 0; l < depth; ++l) {
    const int o = occ0 + l;
    const int node0 = p.occ_node_off[o], w = p.occ_node_off[o + 1] - node0;
    const bool nxt = l + 1 < depth;
    const int node0n = node0 + w, wn = nxt ? p.occ_node_off[o + 2] - node0n : 0;
    const bool has = gt < w;
    int2 lh = make_int2(kNone, kNone);
    float fp = inf(), bn = inf(), Gbn = 0.f;
    if (has) {
      lh = p.lohi[node0 + gt];
      fp = a.msg_pre[node0 + gt];
      bn = a.msg_new[node0 + gt];
      Gbn = l == 0 ? (gt == 0 && a.gE ? (float)*a.gE : 0.f) : carry;
    }
    const float lam1 = a.lam_s[o] + a.shr_s[o], lam2 = a.lam2[o];
    const float b0 = has ? target_msg(a.msg_new, lh.x) : inf();
    const float b1 = has ? target_msg(a.msg_new, lh.y) : inf();
    const float q0 = has ? weight(b0, bn, ia) : 0.f;
    const float q1 = has ? weight(lam2 + b1, bn, ia) : 0.f;
    const float G_lam2 = a.g_out_lam[o] + block_sum_f(Gbn * q1, S.red);
    const float a0 = has ? fp + b0 : inf(), a1 = has ? fp + lam1 + b1 : inf();
    const float2 mm = block_softmin2(a0, a1, p, S.red2);
    const bool finite = mm.x < inf() && mm.y < inf();
    const float gd = finite ? p.omega * (a.g_out_delta[p.occ_slot[o]] - G_lam2) : 0.f;
    const float p0 = weight(a0, mm.x, ia), p1 = weight(a1, mm.y, ia);
    if (has) a.g_node[node0 + gt] = -gd * p0 + gd * p1;
    if (gt == 0) {
      a.g_in_lam[o] = G_lam2 + gd;
      a.g_shr[o] = G_lam2 + gd;
    }
    S.arcs[gt] = nxt ? lh : make_int2(kNone, kNone);
    S.c0[gt] = Gbn * q0 - gd * p0;
    S.c1[gt] = Gbn * q1 + gd * p1;
    __syncthreads();
    carry = gt < wn ? pull_sum(S, w, node0n, gt) : 0.f;
    __syncthreads();
  }
  // descending layers: the starting forward messages fmp_l(v) = softmin over in-arcs of
  // fmp_{l-1}(u) + theta, adjoints flowing from layer l + 1 back to layer l
  for (int l = depth - 1; l >= 0; --l) {
    const int o = occ0 + l;
    const int node0 = p.occ_node_off[o], w = p.occ_node_off[o + 1] - node0;
    const bool nxt = l + 1 < depth;
    const int node0n = node0 + w;
    const bool has = gt < w;
    int2 lh = make_int2(kNone, kNone);
    float f = inf(), G = 0.f;
    if (has) {
      lh = p.lohi[node0 + gt];
      f = a.msg_pre[node0 + gt];
      G = a.g_node[node0 + gt];
    }
    const float lam = a.lam_s[o];
    float g_theta = 0.f;
    if (has && nxt) {
      if (lh.x >= 0) G += S.G[lh.x - node0n] * weight(f, S.F[lh.x - node0n], ia);
      if (lh.y >= 0) {
        g_theta = S.G[lh.y - node0n] * weight(f + lam, S.F[lh.y - node0n], ia);
        G += g_theta;
      }
    }
    const float gl = block_sum_f(g_theta, S.red);
    if (gt == 0) a.g_in_lam[o] += gl;
    __syncthreads();  // S.G / S.F of layer l + 1 no longer read
    S.G[gt] = has ? G : 0.f;
    S.F[gt] = f;
    __syncthreads();
  }
}

template <bool FWD>
__device__ __forceinline__ void adjoint_tile(const AdjParams &a, int tile) {
  int c = 0;
  while (tile >= a.sp.class_tile_off[c + 1]) ++c;
  switch (c) {
#define BDD_ADJ_CASE(C, T)                    \
  case C:                                     \
    if (FWD) fwd_adjoint_tile<T>(a, tile);    \
    else bwd_adjoint_tile<T>(a, tile);        \
    break;
    BDD_ADJ_CASE(0, 1)
    BDD_ADJ_CASE(1, 2)
    BDD_ADJ_CASE(2, 4)
    BDD_ADJ_CASE(3, 8)
    BDD_ADJ_CASE(4, 16)
    BDD_ADJ_CASE(5, 32)
#undef BDD_ADJ_CASE
    default:
      break;
  }
}

}  // namespace

template <bool FWD>
__global__ void __launch_bounds__(kBlockThreads) sweep_adjoint_kernel(const AdjParams a) {
  if ((int)blockIdx.x < a.sp.n_warp_blocks) {
    const int tile = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (tile >= a.sp.class_tile_off[kWarpClasses]) return;  // whole warp
    adjoint_tile<FWD>(a, tile);
    return;
  }
  // block tiles: one block per BDD (smoothed solvers: layers of at most kBlockThreads nodes)
  const int tile = a.sp.class_tile_off[kWarpClasses] + ((int)blockIdx.x - a.sp.n_warp_blocks);
  if (tile >= a.sp.class_tile_off[kWarpClasses + 1]) return;  // uniform across the block
  __shared__ BlockAdjSmem S;
  if (FWD)
    fwd_adjoint_block(a, tile, S);
  else
    bwd_adjoint_block(a, tile, S);
}

// Adjoint of the pending sums: share_o = P_i / |J_i| and P_i = sum of the previous sweep's
// differences of i, so every slot of i receives (sum over i's occurrences of g_share) / |J_i|.
__global__ void pending_adjoint_kernel(const int *__restrict__ var_ptr, const int *__restrict__ var_occ,
                                       const unsigned char *__restrict__ slot_dir, int dir,
                                       const float *__restrict__ g_shr, float *__restrict__ g_delta, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = var_ptr[i], e = var_ptr[i + 1];
    if (e == s) continue;
    int cnt = 0;  // SRMP: the slots that took a share (all of them when none is in J_i^dir)
    if (slot_dir)
      for (int k = s; k < e; ++k) cnt += (slot_dir[k] & dir) != 0;
    float g = 0.f;
    if (cnt > 0) {
      for (int k = s; k < e; ++k)
        if (slot_dir[k] & dir) g += g_shr[var_occ[k]];
      g /= (float)cnt;
    } else {
      for (int k = s; k < e; ++k) g += g_shr[var_occ[k]];
      g /= (float)(e - s);
    }
    for (int k = s; k < e; ++k) g_delta[k] = g;
  }
}

// Seeds of the bound's adjoint.  The bound adds the soft slack term sl(P_i) = softmin(0, P_i)
// of every variable in a row (adjoint exp(-(P_i - sl)/alpha) on each slot of i, whose
// differences form P_i) and sl(c_i) of every variable in no row (adjoint into g_c directly).
__global__ void bound_seed_kernel(const int *__restrict__ var_ptr, const float *__restrict__ P,
                                  const float *__restrict__ c, float *__restrict__ g_delta, float *__restrict__ g_c,
                                  int n, float alpha, const double *__restrict__ g_bound) {
  const float scale = (float)*g_bound;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = var_ptr[i], e = var_ptr[i + 1];
    const float x = e > s ? P[i] : c[i];
    const float sl = fminf(x, 0.f) - alpha * log1pf(expf(-fabsf(x) / alpha));
    const float g = scale * expf(-(x - sl) / alpha);
    if (e > s) {
      for (int k = s; k < e; ++k) g_delta[k] = g;
    } else {
      g_c[i] = g;
    }
  }
}

// lambda_0 = c_i / |J_i|: g_c_i = (sum over i's occurrences of g_lambda_0) / |J_i|
__global__ void initial_adjoint_kernel(const int *__restrict__ var_ptr, const int *__restrict__ var_occ,
                                       const float *__restrict__ g_lam0, float *__restrict__ g_c, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = var_ptr[i], e = var_ptr[i + 1];
    if (e == s) continue;
    float g = 0.f;
    for (int k = s; k < e; ++k) g += g_lam0[var_occ[k]];
    g_c[i] = g / (float)(e - s);
  }
}

namespace {
int grid_of(long long work) {
  long long g = (work + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}
int launch_status() { return cudaGetLastError() == cudaSuccess ? 0 : -5; }
}  // namespace

int sweep_adjoint_launch(bool forward, const AdjParams &a, int grid, cudaStream_t stream) {
  if (grid <= 0) return 0;
  if (forward)
    sweep_adjoint_kernel<true><<<grid, kBlockThreads, 0, stream>>>(a);
  else
    sweep_adjoint_kernel<false><<<grid, kBlockThreads, 0, stream>>>(a);
  return launch_status();
}

int pending_adjoint_launch(const int *var_ptr, const int *var_occ, const unsigned char *slot_dir, int dir,
                           const float *g_shr, float *g_delta, int n, cudaStream_t stream) {
  if (n == 0) return 0;
  pending_adjoint_kernel<<<grid_of(n), 256, 0, stream>>>(var_ptr, var_occ, slot_dir, dir, g_shr, g_delta, n);
  return launch_status();
}

int bound_seed_launch(const int *var_ptr, const float *P, const float *c, float *g_delta, float *g_c, int n,
                      float alpha, const double *g_bound, cudaStream_t stream) {
  if (n == 0) return 0;
  bound_seed_kernel<<<grid_of(n), 256, 0, stream>>>(var_ptr, P, c, g_delta, g_c, n, alpha, g_bound);
  return launch_status();
}

int initial_adjoint_launch(const int *var_ptr, const int *var_occ, const float *g_lam0, float *g_c, int n,
                           cudaStream_t stream) {
  if (n == 0) return 0;
  initial_adjoint_kernel<<<grid_of(n), 256, 0, stream>>>(var_ptr, var_occ, g_lam0, g_c, n);
  return launch_status();
}

}  // namespace bdd
