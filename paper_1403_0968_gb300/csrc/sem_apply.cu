// Matrix-free spectral-element operator apply y = M Q^T A_L Q M u (arXiv 1403.0968 §4.2.1,
// sum-factorised stiffness display), FP64 or FP32, one kernel launch:
//   gather      u_e = Q M u               (structured ids computed, or read from glo)
//   gradients   u_r = D u, u_s, u_t        (1-D contractions with the GLL derivative matrix D)
//   scaling     (w_r, w_s, w_t) = G (u_r, u_s, u_t) with the symmetric per-node factor G
//   transpose   y_e = D^T w_r + D^T w_s + D^T w_t  (+ w det J alpha u_e)
//   scatter     y += Q^T y_e                (direct-stiffness summation, masked)
//
// Thread layout: one thread per (i, j) column of an element, EB elements per block; each thread
// keeps its column u(i, j, 0..N) and its output column in registers and walks the k planes.  The
// r and s contractions read the current plane from shared memory; the t contraction runs in
// registers.  Each plane needs two barriers.  Interior nodes of an element belong to it alone and
// are stored; face, edge and corner nodes are summed with atomics into a zeroed y.
//
// Optionally (PCG) the kernel also forms p^T A p = sum_e u_e . y_e block by block and the last
// block to finish reduces the partials in a fixed order (deterministic), then sets
// alpha = (r, z) / (p, A p) in the solver scalars.
#include "sem_apply_kernel.cuh"

template <typename T>
static sem_status launch_for_type(sem_handle *h, const T *u, T *y, const T *Gf, const T *wJa, const T *D,
                                  double *partials, SemScalars *scal, cudaStream_t s) {
  ApplyParams<T> p;
  p.E = h->E;
  p.sx = h->box[0];
  p.sy = h->box[1];
  p.sz = h->box[2];
  p.gxs = (int64_t)h->box[0] * h->N + 1;
  p.gys = (int64_t)h->box[1] * h->N + 1;
  p.gzs = (int64_t)h->box[2] * h->N + 1;
  p.bc = h->bc;
  p.u = u;
  p.y = y;
  p.Gf = Gf;
  p.wJa = wJa;
  p.D = D;
  p.glo = h->structured ? nullptr : h->glo;
  p.mask = h->mask;
  p.partials = partials;
  p.scal = scal;
  return dispatch_apply<T>(h->N, p, s);
}

int sem_apply_blocks(const sem_handle *h, sem_prec prec) {
  (void)prec;
  const int eb = apply_eb(h->N);
  return (int)((h->E + eb - 1) / eb);
}

sem_status sem_launch_apply(sem_handle *h, sem_prec prec, const void *u, void *y, double *partials,
                            unsigned int *ticket, double *pAp_out, cudaStream_t s) {
  (void)ticket;
  (void)pAp_out;
  SemScalars *scal = partials ? h->scal : nullptr;
  if (prec == SEM_FP64) {
    if (!h->G64) return sem_fail(SEM_ERR_INVALID, "handle has no FP64 factors (SEM_FEAT_FP64)");
    return launch_for_type<double>(h, static_cast<const double *>(u), static_cast<double *>(y), h->G64, h->wJa64,
                                   h->D64, partials, scal, s);
  }
  if (prec == SEM_FP32) {
    if (!h->G32) return sem_fail(SEM_ERR_INVALID, "handle has no FP32 factors (SEM_FEAT_FP32)");
    return launch_for_type<float>(h, static_cast<const float *>(u), static_cast<float *>(y), h->G32, h->wJa32,
                                  h->D32, partials, scal, s);
  }
  if (prec == SEM_FP64_EMU) {
    if (!h->Gemu) return sem_fail(SEM_ERR_INVALID, "handle has no double-float factors (SEM_FEAT_EMU)");
    return sem_launch_apply_emu(h, static_cast<const double *>(u), static_cast<double *>(y), s);
  }
  return sem_fail(SEM_ERR_INVALID, "unknown precision");
}

extern "C" sem_status sem_apply(sem_handle *h, sem_prec prec, const void *d_u, void *d_y, sem_stream_t stream) {
  if (!h || !d_u || !d_y) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  if (d_u == d_y) return sem_fail(SEM_ERR_INVALID, "u and y must not alias");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t es = prec == SEM_FP32 ? 4 : 8;
  SEM_CUDA_TRY(cudaMemsetAsync(d_y, 0, (size_t)h->G * es, s));
  return sem_launch_apply(h, prec, d_u, d_y, nullptr, nullptr, nullptr, s);
}
