// A lower-bound reduction that allocates nothing, for callers that cannot allocate device
// memory: code running inside a memory pool or arena they do not own, or inside a
// framework that forbids cudaMalloc on its hot path.  Its scratch (one FP64 partial sum per
// block and a completion ticket) lives in a file-scope __device__ array that every GPU
// which loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "bdd_dbca.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItemsPerThread = 16;
constexpr int kMaxBlocks = 1024;
constexpr long long kMaxItems = (long long)kMaxBlocks * kThreads * kItemsPerThread;  // 4,194,304
constexpr int kMaxDevices = 64;

// [0, kMaxBlocks): block partial sums; slot kMaxBlocks holds the completion ticket (unsigned).
static __device__ __align__(256) double g_bound_scratch[kMaxBlocks + 1];

double *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Same arithmetic as the bound of the iteration's reduction: sum_j E_j + sum_{deg_i > 0}
// min(0, P_i) + empty_const, in FP64; per-block partials finished by the last block in block
// order, so repeated calls with the same inputs give the same bits.
__global__ void __launch_bounds__(kThreads)
    bound_noalloc_kernel(int n, int nb, const float *__restrict__ E, const float *__restrict__ P,
                         const int *__restrict__ deg, double empty_const, double *__restrict__ out,
                         double *scratch) {
  const int range = n > nb ? n : nb;
  double acc = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < range; i += gridDim.x * kThreads) {
    if (i < n && deg[i] > 0) {
      const float p = P[i];
      if (p < 0.f) acc += (double)p;
    }
    if (i < nb) acc += (double)E[i];
  }
  __shared__ double red[kThreads / 32];
  __shared__ bool last;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  unsigned *ticket = reinterpret_cast<unsigned *>(scratch + kMaxBlocks);
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int t = 0; t < kThreads / 32; ++t) s += red[t];
    scratch[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const volatile double *part = scratch;
    double s = empty_const;
    for (unsigned t = 0; t < gridDim.x; ++t) s += part[t];
    out[0] = s;
    *ticket = 0u;
  }
}

// Device address of the scratch array on the current device, looked up once per device.
int scratch_for_current_device(double **ptr) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return BDD_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bound_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return BDD_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *ptr = g_scratch_ptr[dev];
  return BDD_OK;
}

}  // namespace

extern "C" int bdd_lower_bound_noalloc(int n, int nb, const float *d_E, const float *d_P,
                                       const int *d_deg, double empty_const, double *d_bound,
                                       void *stream) {
  if (n < 0 || nb < 0 || !d_bound || (nb > 0 && !d_E) || (n > 0 && (!d_P || !d_deg)))
    return BDD_EINVAL;
  const long long range = n > nb ? n : nb;
  if (range > kMaxItems) return BDD_ETOOBIG;  // more items than the static scratch serves
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != BDD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the ticket must start at 0 (a previous call leaves it at 0, but an aborted one may not)
  if (cudaMemsetAsync(scratch + kMaxBlocks, 0, sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    return BDD_ECUDA;
  }
  long long blocks = (range + (long long)kThreads * kItemsPerThread - 1) / ((long long)kThreads * kItemsPerThread);
  if (blocks < 1) blocks = 1;
  bound_noalloc_kernel<<<(int)blocks, kThreads, 0, s>>>(n, nb, d_E, d_P, d_deg, empty_const, d_bound,
                                                          scratch);
  if (cudaGetLastError() != cudaSuccess) return BDD_ECUDA;
  return BDD_OK;
}
