// Deterministic FP64 reductions: fixed grid, fixed per-thread stride order, warp-shuffle
// butterfly inside warps, warps summed in index order, block partials summed in index order
// by the last block to arrive (integer ticket). The result does not depend on timing.
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>

#include "pfem_internal.h"

namespace pfem {

constexpr int kReduceThreads = 256;

// Sums v[k] over the block (k < N); the result is valid in thread 0.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* scratch /* >= 8*N doubles */) {
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) scratch[w * N + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double s = 0.0;
      for (int j = 0; j < nw; ++j) s += scratch[j * N + k];
      v[k] = s;
    }
}

// Publishes the N partials of (virtual) block vb of nvb and returns true in every thread of
// the block that publishes last, whose thread-0 `v` then holds the grand totals (summed over
// blocks in index order, so the result does not depend on which block comes last).
template <int N>
__device__ __forceinline__ bool grid_sum_v(double (&v)[N], double* partials, unsigned int* counter, double* scratch,
                                           int vb, int nvb) {
  __shared__ bool s_last;
  block_sum<N>(v, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) partials[vb * N + k] = v[k];
    // release: the partials before the count; acquire: the last block sees every partial
    const unsigned t =
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device>(*counter).fetch_add(1u, cuda::memory_order_acq_rel);
    s_last = (t == (unsigned)nvb - 1u);
  }
  __syncthreads();
  if (!s_last) return false;  // (thread 0's acquire + the barrier order the loads below)
  double acc[N];
#pragma unroll
  for (int k = 0; k < N; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < nvb; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] += __ldcg(partials + b * N + k);
  block_sum<N>(acc, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = acc[k];
    *counter = 0u;  // ready for the next use (stream order or a grid barrier makes this safe)
  }
  return true;
}

template <int N>
__device__ __forceinline__ bool grid_sum(double (&v)[N], double* partials, unsigned int* counter, double* scratch) {
  return grid_sum_v<N>(v, partials, counter, scratch, blockIdx.x, gridDim.x);
}

}  // namespace pfem
