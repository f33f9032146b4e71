// Sweep, reduction and helper kernels for BDD min-marginal averaging on sm_103a.
//
// One iteration = forward sweep, per-variable reduction, backward sweep, per-variable
// reduction with the FP64 lower bound (Sec. 3.2 Alg. 1's forward and backward pass, in the
// parallel-across-BDDs form: the averaging term of eq. mma-update is formed after a sweep and
// applied, as share_i = P_i / |J_i|, when the next sweep visits the layer of variable i).
//
// Sweep kernels walk each BDD's layers in order inside one team of threads; there is no grid
// synchronisation inside a sweep.  Messages of the current layer stay in registers (warp
// teams: lane t of a team of T lanes holds node t; the forward step pushes along lo/hi arcs
// with shuffles, the backward step pulls its successors' messages with one shuffle each) or in
// shared memory (one block per BDD for layers wider than 32 nodes, forward step by shared-memory
// atomic minimum).  Forward messages are written for the backward sweep and backward messages
// for the next forward sweep (Prop. 3: every message stays valid for the layers not yet
// revisited).
#include <cuda_runtime.h>

#include <cfloat>

#include "internal.h"

namespace bdd {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }

// backward message of an arc target: top -> 0, bot / none -> +inf, node -> bm
__device__ __forceinline__ float target_bm(const float *__restrict__ bm, int t) {
  if (t >= 0) return bm[t];
  return t == kTop ? 0.f : inf();
}

// atomic minimum on a float in shared memory (non-negative floats order like their int bits,
// negative ones reverse-order like their unsigned bits)
__device__ __forceinline__ void atomic_min_f(float *addr, float v) {
  if (v >= 0.f)
    atomicMin(reinterpret_cast<int *>(addr), __float_as_int(v));
  else
    atomicMax(reinterpret_cast<unsigned *>(addr), __float_as_uint(v));
}

template <int T>
__device__ __forceinline__ float team_min(float v) {
#pragma unroll
  for (int off = T / 2; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

__device__ __forceinline__ float mm_difference(float m0, float m1) {
  // a +inf min-marginal (a row forcing x_i) transfers nothing
  return (m0 < inf() && m1 < inf()) ? m1 - m0 : 0.f;
}

// ---------------------------------------------------------------------------------------
// warp tiles: T lanes per BDD, 32 / T BDDs per warp
// ---------------------------------------------------------------------------------------
template <int T, int MODE>
__device__ void warp_forward(const SweepParams &p, int tile) {
  const int lane = threadIdx.x & 31;
  const int team = lane / T, tl = lane % T, tbase = team * T;
  const int occ0 = p.tile_occ0[tile];
  const int bdd = p.tile_bdd0[tile] + team;
  const bool valid = team < p.tile_nbdd[tile];
  const int depth = valid ? p.bdd_depth[bdd] : 0;
  const int maxd = __reduce_max_sync(kFull, depth);
  int cum = 0;
  float f_prev = inf(), lam_prev = 0.f;
  int2 lh_prev = make_int2(kNone, kNone);
  for (int l = 0; l < maxd; ++l) {
    const int alive = __popc(__ballot_sync(kFull, tl == 0 && depth > l));
    const bool active = depth > l;
    const int o = occ0 + cum + team;
    int node0 = 0, w = 0;
    if (active) {
      node0 = p.occ_node_off[o];
      w = p.occ_node_off[o + 1] - node0;
    }
    const bool has = active && tl < w;
    // Alg. 2: m_fwd(v) = min over in-arcs (u, v) of m_fwd(u) + theta_uv
    float f;
    if (l == 0) {
      f = 0.f;
    } else {
      const int lo_l = lh_prev.x >= 0 ? lh_prev.x - node0 : kNone;
      const int hi_l = lh_prev.y >= 0 ? lh_prev.y - node0 : kNone;
      f = inf();
#pragma unroll
      for (int s = 0; s < T; ++s) {
        const float mf = __shfl_sync(kFull, f_prev, tbase + s);
        const int ls = __shfl_sync(kFull, lo_l, tbase + s);
        const int hs = __shfl_sync(kFull, hi_l, tbase + s);
        if (ls == tl) f = fminf(f, mf);
        if (hs == tl) f = fminf(f, mf + lam_prev);
      }
    }
    int2 lh = make_int2(kNone, kNone);
    if (has) {
      p.fm[node0 + tl] = f;
      lh = p.lohi[node0 + tl];
    }
    float lam = 0.f;
    if (active) {
      lam = p.lam[o];
      if (MODE != kMessages) lam += p.share[p.occ_var[o]];
    }
    if (MODE == kUpdate) {
      // eqs. arc-marginal / marginal-aggregation, then the damped eq. mma-update step
      const float a0 = has ? f + target_bm(p.bm, lh.x) : inf();
      const float a1 = has ? f + lam + target_bm(p.bm, lh.y) : inf();
      const float m0 = team_min<T>(a0), m1 = team_min<T>(a1);
      const float dd = p.omega * mm_difference(m0, m1);
      lam -= dd;
      if (active && tl == 0) {
        p.lam[o] = lam;
        p.delta[o] = dd;
      }
    }
    f_prev = f;
    lh_prev = lh;
    lam_prev = lam;
    cum += alive;
  }
}

template <int T, int MODE>
__device__ void warp_backward(const SweepParams &p, int tile) {
  const int lane = threadIdx.x & 31;
  const int team = lane / T, tl = lane % T, tbase = team * T;
  const int occ0 = p.tile_occ0[tile];
  const int bdd = p.tile_bdd0[tile] + team;
  const bool valid = team < p.tile_nbdd[tile];
  const int depth = valid ? p.bdd_depth[bdd] : 0;
  const int maxd = __reduce_max_sync(kFull, depth);
  const int total = __reduce_add_sync(kFull, tl == 0 ? depth : 0);
  int cum_ge = 0;
  float b_next = inf();
  int node0_next = 0;
  for (int l = maxd - 1; l >= 0; --l) {
    cum_ge += __popc(__ballot_sync(kFull, tl == 0 && depth > l));
    const bool active = depth > l;
    const int o = occ0 + total - cum_ge + team;
    int node0 = 0, w = 0;
    if (active) {
      node0 = p.occ_node_off[o];
      w = p.occ_node_off[o + 1] - node0;
    }
    const bool has = active && tl < w;
    int2 lh = make_int2(kNone, kNone);
    float f = inf();
    if (has) {
      lh = p.lohi[node0 + tl];
      f = p.fm[node0 + tl];
    }
    float lam = 0.f;
    if (active) {
      lam = p.lam[o];
      if (MODE != kMessages) lam += p.share[p.occ_var[o]];
    }
    // successors' backward messages live on the lanes of this team (layer l + 1)
    const int s0 = lh.x >= 0 ? lh.x - node0_next : 0;
    const int s1 = lh.y >= 0 ? lh.y - node0_next : 0;
    const float g0 = __shfl_sync(kFull, b_next, tbase + (s0 & (T - 1)));
    const float g1 = __shfl_sync(kFull, b_next, tbase + (s1 & (T - 1)));
    const float b0 = lh.x >= 0 ? g0 : (lh.x == kTop ? 0.f : inf());
    const float b1 = lh.y >= 0 ? g1 : (lh.y == kTop ? 0.f : inf());
    if (MODE != kMessages) {
      const float m0 = team_min<T>(f + b0), m1 = team_min<T>(f + lam + b1);
      if (MODE == kUpdate) {
        const float dd = p.omega * mm_difference(m0, m1);
        lam -= dd;
        if (active && tl == 0) {
          p.lam[o] = lam;
          p.delta[o] = dd;
        }
      } else if (active && tl == 0 && p.out_m0) {
        const long long c = p.occ_csr[o];
        p.out_m0[c] = m0;
        p.out_m1[c] = m1;
      }
    }
    // Alg. 3: m_bwd(v) = min(m_bwd(v0) + 0, m_bwd(v1) + lambda)
    const float bcur = fminf(b0, lam + b1);
    if (has) p.bm[node0 + tl] = bcur;
    if (l == 0 && active && tl == 0) p.bdd_E[bdd] = bcur;  // E^j(lambda^j) at the root
    b_next = bcur;
    node0_next = node0;
  }
}

// ---------------------------------------------------------------------------------------
// block tiles: one block per BDD (layers wider than 32 nodes)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float2 block_min2(float a, float b, float2 *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a = fminf(a, __shfl_xor_sync(kFull, a, off));
    b = fminf(b, __shfl_xor_sync(kFull, b, off));
  }
  if (lane == 0) red[warp] = make_float2(a, b);
  __syncthreads();
  float2 r = red[0];
#pragma unroll
  for (int t = 1; t < kWarpsPerBlock; ++t) {
    r.x = fminf(r.x, red[t].x);
    r.y = fminf(r.y, red[t].y);
  }
  __syncthreads();  // red may be reused right after
  return r;
}

template <int MODE>
__device__ void block_forward(const SweepParams &p, int tile, float *bufA, float *bufB,
                              float2 *red) {
  const int bdd = p.tile_bdd0[tile];
  const int occ0 = p.tile_occ0[tile];
  const int depth = p.bdd_depth[bdd];
  float *cur = bufA, *nxt = bufB;
  if (threadIdx.x == 0) cur[0] = 0.f;
  __syncthreads();
  for (int l = 0; l < depth; ++l) {
    const int o = occ0 + l;
    const int node0 = p.occ_node_off[o], w = p.occ_node_off[o + 1] - node0;
    float lam = p.lam[o];
    if (MODE != kMessages) lam += p.share[p.occ_var[o]];
    float a0 = inf(), a1 = inf();
    for (int t = threadIdx.x; t < w; t += kBlockThreads) {
      const float f = cur[t];
      p.fm[node0 + t] = f;
      if (MODE == kUpdate) {
        const int2 lh = p.lohi[node0 + t];
        a0 = fminf(a0, f + target_bm(p.bm, lh.x));
        a1 = fminf(a1, f + lam + target_bm(p.bm, lh.y));
      }
    }
    if (MODE == kUpdate) {
      const float2 mm = block_min2(a0, a1, red);
      const float dd = p.omega * mm_difference(mm.x, mm.y);
      lam -= dd;
      if (threadIdx.x == 0) {
        p.lam[o] = lam;
        p.delta[o] = dd;
      }
    }
    if (l + 1 < depth) {
      const int next0 = node0 + w, wn = p.occ_node_off[o + 2] - next0;
      for (int t = threadIdx.x; t < wn; t += kBlockThreads) nxt[t] = inf();
      __syncthreads();
      for (int t = threadIdx.x; t < w; t += kBlockThreads) {
        const float f = cur[t];
        const int2 lh = p.lohi[node0 + t];
        if (lh.x >= 0) atomic_min_f(&nxt[lh.x - next0], f);
        if (lh.y >= 0) atomic_min_f(&nxt[lh.y - next0], f + lam);
      }
      __syncthreads();
      float *tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
}

template <int MODE>
__device__ void block_backward(const SweepParams &p, int tile, float *bufA, float *bufB,
                               float2 *red) {
  const int bdd = p.tile_bdd0[tile];
  const int occ0 = p.tile_occ0[tile];
  const int depth = p.bdd_depth[bdd];
  float *cur = bufA, *nxt = bufB;  // cur: backward messages of layer l + 1
  for (int l = depth - 1; l >= 0; --l) {
    const int o = occ0 + l;
    const int node0 = p.occ_node_off[o], w = p.occ_node_off[o + 1] - node0;
    const int next0 = node0 + w;
    float lam = p.lam[o];
    if (MODE != kMessages) lam += p.share[p.occ_var[o]];
    if (MODE != kMessages) {
      float a0 = inf(), a1 = inf();
      for (int t = threadIdx.x; t < w; t += kBlockThreads) {
        const int2 lh = p.lohi[node0 + t];
        const float f = p.fm[node0 + t];
        const float b0 = lh.x >= 0 ? cur[lh.x - next0] : (lh.x == kTop ? 0.f : inf());
        const float b1 = lh.y >= 0 ? cur[lh.y - next0] : (lh.y == kTop ? 0.f : inf());
        a0 = fminf(a0, f + b0);
        a1 = fminf(a1, f + lam + b1);
      }
      const float2 mm = block_min2(a0, a1, red);
      if (MODE == kUpdate) {
        const float dd = p.omega * mm_difference(mm.x, mm.y);
        lam -= dd;
        if (threadIdx.x == 0) {
          p.lam[o] = lam;
          p.delta[o] = dd;
        }
      } else if (threadIdx.x == 0 && p.out_m0) {
        const long long c = p.occ_csr[o];
        p.out_m0[c] = mm.x;
        p.out_m1[c] = mm.y;
      }
    }
    for (int t = threadIdx.x; t < w; t += kBlockThreads) {
      const int2 lh = p.lohi[node0 + t];
      const float b0 = lh.x >= 0 ? cur[lh.x - next0] : (lh.x == kTop ? 0.f : inf());
      const float b1 = lh.y >= 0 ? cur[lh.y - next0] : (lh.y == kTop ? 0.f : inf());
      const float bcur = fminf(b0, lam + b1);
      p.bm[node0 + t] = bcur;
      nxt[t] = bcur;
      if (l == 0 && t == 0) p.bdd_E[bdd] = bcur;
    }
    __syncthreads();
    float *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------
template <bool FWD, int MODE>
__global__ void __launch_bounds__(kBlockThreads) sweep_kernel(const SweepParams p) {
  extern __shared__ float smem[];
  if ((int)blockIdx.x < p.n_warp_blocks) {
    const int tile = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (tile >= p.class_tile_off[kWarpClasses]) return;  // whole warp leaves together
    int c = 0;
    while (tile >= p.class_tile_off[c + 1]) ++c;
    switch (c) {
#define BDD_TEAM_CASE(C, T)                                   \
  case C:                                                     \
    if (FWD) warp_forward<T, MODE>(p, tile);                  \
    else warp_backward<T, MODE>(p, tile);                     \
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
  } else {
    const int tile = p.class_tile_off[kWarpClasses] + (blockIdx.x - p.n_warp_blocks);
    if (tile >= p.class_tile_off[kWarpClasses + 1]) return;  // uniform across the block
    float2 *red = reinterpret_cast<float2 *>(smem);
    float *bufA = smem + 2 * kWarpsPerBlock;
    float *bufB = bufA + p.block_buf;
    if (FWD)
      block_forward<MODE>(p, tile, bufA, bufB, red);
    else
      block_backward<MODE>(p, tile, bufA, bufB, red);
  }
}

// Per-variable reduction (the sum in eq. mma-update, deferred): P_i = sum of the recorded
// differences of i's occurrences in ascending row order, share_i = P_i / |J_i|.  With `bound`,
// also the FP64 y-slack lower bound sum_j E^j + sum_i min(0, P_i) (+ the constant of variables
// in no row), reduced deterministically: per-block partials, summed in block order by the last
// block to finish, written to trace[*iter_ctr].
template <bool RECOMPUTE, bool BOUND>
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const ReduceParams p) {
  const int range = p.n > p.nb ? p.n : p.nb;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < range; i += gridDim.x * blockDim.x) {
    if (i < p.n) {
      const int s = p.var_ptr[i], e = p.var_ptr[i + 1];
      float P;
      if (RECOMPUTE) {
        P = 0.f;
        for (int k = s; k < e; ++k) P += p.delta[p.var_occ[k]];
        p.P[i] = P;
        p.share[i] = e > s ? P / (float)(e - s) : 0.f;
      } else {
        P = p.P[i];
      }
      if (BOUND && e > s && P < 0.f) acc += (double)P;
    }
    if (BOUND && i < p.nb) acc += (double)p.bdd_E[i];
  }
  if constexpr (BOUND) {
    __shared__ double red[kReduceThreads / 32];
    __shared__ bool last;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int t = 0; t < kReduceThreads / 32; ++t) s += red[t];
      p.partial[blockIdx.x] = s;
      __threadfence();
      const unsigned ticket = atomicAdd(p.ticket, 1u);
      last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      double s = p.empty_const;
      const volatile double *part = p.partial;
      for (unsigned t = 0; t < gridDim.x; ++t) s += part[t];
      const int it = *p.iter_ctr;
      if (it < p.trace_cap) p.trace[it] = s;
      *p.iter_ctr = it + 1;
      *p.ticket = 0u;
    }
  }
}

// lambda^j_i = c_i / |J_i| (Alg. 1 initialisation)
__global__ void init_lambda_kernel(const int *__restrict__ occ_var, const int *__restrict__ var_ptr,
                                   const float *__restrict__ c, float *__restrict__ lam, int O) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < O; o += gridDim.x * blockDim.x) {
    const int i = occ_var[o];
    lam[o] = c[i] / (float)(var_ptr[i + 1] - var_ptr[i]);
  }
}

__global__ void share_kernel(const int *__restrict__ var_ptr, const float *__restrict__ P,
                             float *__restrict__ share, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int d = var_ptr[i + 1] - var_ptr[i];
    share[i] = d > 0 ? P[i] / (float)d : 0.f;
  }
}

__global__ void scatter_lambda_kernel(const float *__restrict__ lam, const float *__restrict__ share,
                                      const int *__restrict__ occ_var,
                                      const long long *__restrict__ occ_csr, float *__restrict__ out,
                                      int O, bool fold) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < O; o += gridDim.x * blockDim.x)
    out[occ_csr[o]] = lam[o] + (fold ? share[occ_var[o]] : 0.f);
}

__global__ void gather_lambda_kernel(const float *__restrict__ in, const long long *__restrict__ occ_csr,
                                     float *__restrict__ lam, int O) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < O; o += gridDim.x * blockDim.x)
    lam[o] = in[occ_csr[o]];
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
}  // namespace

int sweep_launch(bool forward, int mode, const SweepParams &p, int grid, cudaStream_t stream) {
  if (grid <= 0) return 0;
  const size_t smem = (2 * kWarpsPerBlock + 2 * (size_t)p.block_buf) * sizeof(float);
#define BDD_SWEEP(F, M) sweep_kernel<F, M><<<grid, kBlockThreads, smem, stream>>>(p)
  if (forward) {
    if (mode == kUpdate) BDD_SWEEP(true, kUpdate);
    else if (mode == kMessages) BDD_SWEEP(true, kMessages);
    else BDD_SWEEP(true, kFolded);
  } else {
    if (mode == kUpdate) BDD_SWEEP(false, kUpdate);
    else if (mode == kMessages) BDD_SWEEP(false, kMessages);
    else BDD_SWEEP(false, kFolded);
  }
#undef BDD_SWEEP
  return status();
}

int sweep_set_smem(size_t bytes) {
  const void *fns[] = {
      (const void *)sweep_kernel<true, kUpdate>,   (const void *)sweep_kernel<true, kMessages>,
      (const void *)sweep_kernel<true, kFolded>,   (const void *)sweep_kernel<false, kUpdate>,
      (const void *)sweep_kernel<false, kMessages>, (const void *)sweep_kernel<false, kFolded>};
  for (const void *f : fns)
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
      return -5;
  return 0;
}

int reduce_launch(bool recompute, bool bound, const ReduceParams &p, int grid, cudaStream_t stream) {
  if (recompute && bound) reduce_kernel<true, true><<<grid, kReduceThreads, 0, stream>>>(p);
  else if (recompute) reduce_kernel<true, false><<<grid, kReduceThreads, 0, stream>>>(p);
  else reduce_kernel<false, true><<<grid, kReduceThreads, 0, stream>>>(p);
  return status();
}

int init_lambda_launch(const int *occ_var, const int *var_ptr, const float *c, float *lam, int O,
                       cudaStream_t stream) {
  if (O == 0) return 0;
  init_lambda_kernel<<<grid_for(O, 256), 256, 0, stream>>>(occ_var, var_ptr, c, lam, O);
  return status();
}

int share_from_pending_launch(const int *var_ptr, const float *P, float *share, int n,
                              cudaStream_t stream) {
  if (n == 0) return 0;
  share_kernel<<<grid_for(n, 256), 256, 0, stream>>>(var_ptr, P, share, n);
  return status();
}

int scatter_lambda_launch(const float *lam, const float *share, const int *occ_var,
                          const long long *occ_csr, float *out, int O, bool fold,
                          cudaStream_t stream) {
  if (O == 0) return 0;
  scatter_lambda_kernel<<<grid_for(O, 256), 256, 0, stream>>>(lam, share, occ_var, occ_csr, out, O,
                                                                fold);
  return status();
}

int gather_lambda_launch(const float *in, const long long *occ_csr, float *lam, int O,
                         cudaStream_t stream) {
  if (O == 0) return 0;
  gather_lambda_kernel<<<grid_for(O, 256), 256, 0, stream>>>(in, occ_csr, lam, O);
  return status();
}

}  // namespace bdd
