// Matrix-free spectral-element operator apply y = M Q^T A_L Q M u (arXiv 1403.0968 §4.2.1,
// sum-factorised stiffness display), FP64 or FP32, one kernel launch:
//   gather      u_e = Q M u               (structured ids computed, or read from glo)
//   gradients   u_r = D u, u_s, u_t        (1-D contractions with the GLL derivative matrix D)
//   scaling     (w_r, w_s, w_t) = G (u_r, u_s, u_t) with the symmetric per-node factor G
//   transpose   y_e = D^T w_r + D^T w_s + D^T w_t  (+ w det J alpha u_e)
//   scatter     y += Q^T y_e                (direct-stiffness summation, masked)
//
// Thread layout: NP^2 threads per element (NP = N+1), several elements per block; each thread
// owns one line in each direction (details in sem_apply_kernel.cuh).  The element's factor block
// is staged into shared memory by one bulk (TMA) copy while the gradients are formed.  Interior
// nodes of an element belong to it alone and are stored; face, edge and corner nodes are summed
// with atomics into a zeroed y.
//
// Optionally (PCG) the kernel also forms p^T A p = sum_e u_e . y_e block by block and the last
// block to finish reduces the partials in a fixed order (deterministic), then sets
// alpha = (r, z) / (p, A p) in the solver scalars.
#include "sem_internal.h"

sem_status sem_launch_apply(sem_handle *h, sem_prec prec, const void *u, void *y, double *partials,
                            unsigned int *ticket, double *pAp_out, cudaStream_t s) {
  (void)ticket;
  (void)pAp_out;
  SemScalars *scal = partials ? h->scal : nullptr;
  int *err = &h->scal->error;
  if (prec == SEM_FP64) {
    if (!h->G64) return sem_fail(SEM_ERR_INVALID, "handle has no FP64 factors (SEM_FEAT_FP64)");
    return dispatch_apply<double>(h, static_cast<const double *>(u), static_cast<double *>(y), h->G64, h->wJa64,
                                  h->D64h, partials, scal, err, s);
  }
  if (prec == SEM_FP32) {
    if (!h->G32) return sem_fail(SEM_ERR_INVALID, "handle has no FP32 factors (SEM_FEAT_FP32)");
    // order 7, variant 5: the D-contractions on the tensor cores (3xTF32)
    if (h->N == 7 && h->apply_variant == 5)
      return sem_launch_apply_f32_tc(h, static_cast<const float *>(u), static_cast<float *>(y), partials, s);
    return dispatch_apply<float>(h, static_cast<const float *>(u), static_cast<float *>(y), h->G32, h->wJa32,
                                 h->D32h, partials, scal, err, s);
  }
  if (prec == SEM_BF16) {
    if (!h->G16) return sem_fail(SEM_ERR_INVALID, "handle has no BF16 factors (SEM_FEAT_BF16)");
    return dispatch_apply<float, __nv_bfloat16>(h, static_cast<const float *>(u), static_cast<float *>(y), h->G16,
                                                h->wJa32, h->D32h, partials, scal, err, s);
  }
  if (prec == SEM_FP32_OTF) {
    if (!h->Gotf) return sem_fail(SEM_ERR_INVALID, "handle has no map coefficients (SEM_FEAT_OTF)");
    return dispatch_apply<float, OtfGeo>(h, static_cast<const float *>(u), static_cast<float *>(y), h->Gotf,
                                         h->wJa32, h->D32h, partials, scal, err, s);
  }
  if (prec == SEM_FP64_EMU) {
    if (!h->Gemu) return sem_fail(SEM_ERR_INVALID, "handle has no double-float factors (SEM_FEAT_EMU)");
    return sem_launch_apply_emu(h, static_cast<const double *>(u), static_cast<double *>(y), partials, s);
  }
  return sem_fail(SEM_ERR_INVALID, "unknown precision");
}

extern "C" sem_status sem_apply(sem_handle *h, sem_prec prec, const void *d_u, void *d_y, sem_stream_t stream) {
  if (!h || !d_u || !d_y) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  if (d_u == d_y) return sem_fail(SEM_ERR_INVALID, "u and y must not alias");
  if (prec != SEM_FP64 && prec != SEM_FP64_EMU && prec != SEM_FP32 && prec != SEM_BF16 && prec != SEM_FP32_OTF)
    return sem_fail(SEM_ERR_INVALID, "unknown precision");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t es = (prec == SEM_FP64 || prec == SEM_FP64_EMU) ? 8 : 4;  // FP32 vectors otherwise
  SEM_CUDA_TRY(cudaMemsetAsync(d_y, 0, (size_t)h->G * es, s));
  return sem_launch_apply(h, prec, d_u, d_y, nullptr, nullptr, nullptr, s);
}

// Clears the handle's timeout flag and the reduction tickets a block that left early may have
// left behind, so that later applies and solves on the handle start clean.
sem_status sem_clear_timeout(sem_handle *h, cudaStream_t s) {
  SEM_CUDA_TRY(cudaMemsetAsync(&h->scal->error, 0, sizeof(int), s));
  SEM_CUDA_TRY(cudaMemsetAsync(h->scal->counter, 0, sizeof(h->scal->counter), s));
  SEM_CUDA_TRY(cudaMemsetAsync(h->gtickets, 0, (size_t)SEM_MAX_GROUPS * sizeof(unsigned int), s));
  return SEM_OK;
}

extern "C" sem_status sem_apply_status(sem_handle *h, sem_stream_t stream) {
  if (!h) return sem_fail(SEM_ERR_INVALID, "NULL handle");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int v = 0;
  SEM_CUDA_TRY(cudaMemcpyAsync(&v, &h->scal->error, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (!v) return SEM_OK;
  sem_status st = sem_clear_timeout(h, s);
  if (st != SEM_OK) return st;
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  return sem_fail(SEM_ERR_TIMEOUT, "an apply gave up waiting for a staged factor copy; its output is incomplete");
}

extern "C" sem_status sem_set_wait_limit(sem_handle *h, int64_t polls) {
  if (!h) return sem_fail(SEM_ERR_INVALID, "NULL handle");
  if (polls > 0xffffffffll) return sem_fail(SEM_ERR_INVALID, "wait limit above 2^32 - 1 polls");
  h->wait_polls = polls < 0 ? SEM_WAIT_POLLS_DEFAULT : (uint32_t)polls;
  return SEM_OK;
}

extern "C" sem_status sem_set_apply_variant(sem_handle *h, int32_t variant) {
  if (!h) return sem_fail(SEM_ERR_INVALID, "NULL handle");
  if (variant < -1 || variant >= 6) return sem_fail(SEM_ERR_INVALID, "apply variant must be -1 (automatic) or 0..5");
  h->apply_variant = variant;
  return SEM_OK;
}
