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

// Called by every thread of the last block: fixed-order sum of partials[0..nparts).  The loads go
// to L2 (ld.global.cg: coherent with the other blocks' fenced stores, not cached in L1) and are
// independent, so many are in flight at once; four accumulators keep the order fixed.
template <int NT>
__device__ __forceinline__ double final_sum(const double *partials, int nparts, double *s_red) {
  double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
  int q = threadIdx.x;
  for (; q + 3 * NT < nparts; q += 4 * NT) {
    v0 += __ldcg(partials + q);
    v1 += __ldcg(partials + q + NT);
    v2 += __ldcg(partials + q + 2 * NT);
    v3 += __ldcg(partials + q + 3 * NT);
  }
  for (; q < nparts; q += NT) v0 += __ldcg(partials + q);
  return block_sum<NT>((v0 + v1) + (v2 + v3), s_red);
}

// Two-level variant for grids of up to 256 * 4096 blocks: blocks are grouped by 256; the last
// block of each group (a ticket per group) sums the group's partials in order into gpartials[group];
// the block that completes the last group sums the group results in order.  Returns true in every
// thread of that final block, with the total in *total.  Deterministic for a given grid size.
// gtickets: one zeroed counter per group (reset here); ticket: the final counter (reset by caller).
template <int NT>
__device__ __forceinline__ bool publish_partial_2level(double v, double *partials, double *gpartials,
                                                       unsigned int *gtickets, unsigned int *ticket, double *s_red,
                                                       int *s_flag, double *total) {
  const unsigned int group = blockIdx.x / 256u, ngroups = (gridDim.x + 255u) / 256u;
  const unsigned int gsize = (gridDim.x - group * 256u) < 256u ? (gridDim.x - group * 256u) : 256u;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v;
    __threadfence();
    *s_flag = (atomicAdd(&gtickets[group], 1u) == gsize - 1u);
  }
  __syncthreads();
  if (*s_flag == 0) return false;
  __threadfence();
  const double gsum = final_sum<NT>(partials + group * 256u, (int)gsize, s_red);
  if (threadIdx.x == 0) {
    gtickets[group] = 0u;
    gpartials[group] = gsum;
    __threadfence();
    *s_flag = (atomicAdd(ticket, 1u) == ngroups - 1u);
  }
  __syncthreads();
  if (*s_flag == 0) return false;
  __threadfence();
  *total = final_sum<NT>(gpartials, (int)ngroups, s_red);
  return true;
}
