// Device helpers shared by the sweep kernels and their adjoints (the same arithmetic in both).
#pragma once

#include "internal.h"

namespace bdd {

constexpr unsigned kFull = 0xffffffffu;

// Index checks of the checked build (compiled with -DBDD_CHECKED; see build.py): an index
// outside [0, n) records BDD_EDEVICE (-7) in the error word and is replaced by 0, so the access
// it guards stays inside its array and the host call reports the failure.  In the normal build
// the macros are the index itself and nothing is checked.
#ifdef BDD_CHECKED
__device__ __forceinline__ long long checked_index(int *err, long long i, long long n) {
  if (i < 0 || i >= n) {
    atomicExch(err, -7);
    return 0;
  }
  return i;
}
#define BDD_IN(p, i, n) checked_index((p).error, (i), (n))
#else
#define BDD_IN(p, i, n) (i)
#endif
#define BDD_NODE(p, i) BDD_IN(p, i, (p).n_nodes)
#define BDD_OCC(p, i) BDD_IN(p, i, (p).n_occ)
#define BDD_CSR(p, i) BDD_IN(p, i, (p).n_csr)
#define BDD_BDD(p, i) BDD_IN(p, i, (p).n_bdd)

__device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }

template <int T>
__device__ __forceinline__ float team_min(float v) {
#pragma unroll
  for (int off = T / 2; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

// The aggregation of the BDD algebra (Table 3): min for min-sum; for the smoothed variant
// (Appendix A.5) the soft minimum -alpha log(exp(-a/alpha) + exp(-b/alpha)), evaluated as
// min(a, b) - alpha log(1 + exp(-|a - b| / alpha)); +inf is its neutral element.
__device__ __forceinline__ float soft_min(float a, float b, float alpha, float inv_alpha) {
  if (a == inf()) return b;
  if (b == inf()) return a;
  return fminf(a, b) - alpha * log1pf(expf(-fabsf(a - b) * inv_alpha));
}

template <bool SMOOTH>
__device__ __forceinline__ float agg(float a, float b, const SweepParams &p) {
  if (SMOOTH) return soft_min(a, b, p.alpha, p.inv_alpha);
  return fminf(a, b);
}

// reduction over the T lanes of a team; the smoothed form is not exactly associative, so every
// lane takes the team's first lane's result
template <int T, bool SMOOTH>
__device__ __forceinline__ float team_agg(float v, const SweepParams &p) {
  if (!SMOOTH) return team_min<T>(v);
#pragma unroll
  for (int off = T / 2; off > 0; off >>= 1) v = soft_min(v, __shfl_xor_sync(kFull, v, off), p.alpha, p.inv_alpha);
  return __shfl_sync(kFull, v, (threadIdx.x & 31) & ~(T - 1));
}

// occurrences of the tile before layer l: sum over the tile's BDDs of min(depth, l)
__device__ __forceinline__ int occ_before(int lead_depth, int l) {
  return __reduce_add_sync(kFull, min(lead_depth, l));
}

// sum over the T lanes of a team, the same value on every lane of the team
template <int T>
__device__ __forceinline__ float team_sum(float v) {
#pragma unroll
  for (int off = T / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return __shfl_sync(kFull, v, (threadIdx.x & 31) & ~(T - 1));
}

}  // namespace bdd
