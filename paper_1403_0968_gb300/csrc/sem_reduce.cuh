// Deterministic block and grid reductions in FP64.
//
// A kernel that contributes to a dot product writes one FP64 partial per block; the block that
// finishes last (a ticket taken with atomicAdd after a memory fence) sums every partial in a
// fixed order and runs a small epilogue on the result.  The order of additions depends only on
// the grid size, so repeated solves give bit-identical scalars.
#pragma once

#include <cuda_runtime.h>

#include "sem_internal.h"

// Sum of v over the block (all threads must call; result valid in every thread).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *s_red /* >= 32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = (NT + 31) / 32;
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < NW ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s_red[0] = t;
  }
  __syncthreads();
  t = s_red[0];
  __syncthreads();
  return t;
}

// Writes this block's partial; returns true in every thread of the one block that arrives last.
// `nparts` = number of blocks contributing.  The ticket counter is reset by the last block.
template <int NT>
__device__ __forceinline__ bool publish_partial(double v, double *partials, unsigned int *ticket, double *s_red,
                                                int *s_flag) {
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v;
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    *s_flag = (t == gridDim.x - 1);
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// Called by every thread of the last block: fixed-order sum of partials[0..nparts).
template <int NT>
__device__ __forceinline__ double final_sum(const double *partials, int nparts, double *s_red) {
  double v = 0.0;
  for (int q = threadIdx.x; q < nparts; q += NT) v += ((volatile const double *)partials)[q];
  return block_sum<NT>(v, s_red);
}
