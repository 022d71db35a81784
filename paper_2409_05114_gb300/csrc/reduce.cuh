// Fixed-order reductions of the conservation sums (lbm_totals, lbm_totals_noalloc): warp
// shuffle trees, so that every run adds the same numbers in the same order.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// Sum over the 32 lanes of a warp by a shuffle tree; lane 0 holds the result.  The additions
// and their order are the same on every run, so sums built from it are bitwise reproducible.
__device__ __forceinline__ double warp_sum_fixed(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sums five per-thread values over a block of kThreads threads (a multiple of 32, at most
// 1024): a shuffle tree in each warp, then one over the warps' results in warp 0.  Thread 0
// returns the five block totals in acc; every thread of the block must call it.
template <int kThreads>
__device__ __forceinline__ void block_sum5_fixed(double (&acc)[5]) {
  static_assert(kThreads % 32 == 0 && kThreads <= 1024, "block size");
  constexpr int kWarps = kThreads / 32;
  __shared__ double sh[5][kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const double v = warp_sum_fixed(acc[q]);
    if (lane == 0) sh[q][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = warp_sum_fixed(lane < kWarps ? sh[q][lane] : 0.0);
  }
}

// The five totals of nblocks partial sums (partials[b * 5 + q]) by one warp: lane l adds the
// blocks l, l + 32, ... in order, then the shuffle tree; lane 0 writes out[0..4].
__device__ __forceinline__ void warp_total5_fixed(const double* partials, int nblocks, double* out) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) v += partials[b * 5 + q];
    v = warp_sum_fixed(v);
    if (lane == 0) out[q] = v;
  }
}

}  // namespace lbm
