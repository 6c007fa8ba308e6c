// Internal interface of the fused batched CG step (sem_batch_step.cu), used by sem_batch.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sem_internal.h"

// one order group of a batch: its problems' entries, element count, factor stride
struct FusedGroupDesc {
  int N;
  bool otf;
  const BatchEntry *entries;
  int nbatch;
  int64_t total_E, gs;
  const int32_t *tile_entry;  // entry of each tile's first element (device, ceil(total_E / tile) entries)
};

struct FusedStepDesc {
  const FusedGroupDesc *groups;
  int ngroups;
  bool otf;
  int64_t nchunks;
  const int32_t *cp, *cl;
  const int64_t *cs;
  float *x32, *p32, *r32, *Ap32;
  const float *dinv;
  double *rz, *rzn, *rr, *rrn, *pAp, *tol2;
  int32_t *done, *iters, *counts;
  int nprob, max_it;
  unsigned int *bar;  // two zeroed counters: arrivals, generation
  int *err;           // set when a grid-wide wait gave up
  uint32_t wait_polls;
};

// elements per tile of the fused step kernel at order N (0: N is not compiled in)
int sem_batch_fused_tile_elems(int N);
// true if every order is one the fused step kernel is compiled for (3, 5, 7, 9, 11)
bool sem_batch_fused_orders_ok(const int *orders, int n);
// puts the derivative matrices of the compiled orders into the current device's
// constant memory (once per device; the same bytes for every batch)
sem_status sem_batch_fused_init();
// one inner CG step of every unfinished problem: one cooperative launch on st
sem_status sem_batch_fused_step(const FusedStepDesc &d, cudaStream_t st);
