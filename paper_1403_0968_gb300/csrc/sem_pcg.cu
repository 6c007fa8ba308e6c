// Preconditioned conjugate gradients for the spectral-element system (arXiv 1403.0968 §4.2.2:
// the screened-Poisson problem is solved by PCG, whose cost is dominated by the operator apply).
// The paper does not name its preconditioner; this is Jacobi (the assembled diagonal).
//
// Per iteration three launches, none of which needs the host:
//   apply      Ap = M A M p, with p^T A p summed per element and alpha = rz / pAp set by the
//              block that finishes last (sem_apply_kernel.cuh)
//   update     x += alpha p, r -= alpha Ap, z = r / d, (r, z) and (r, r) -> beta, convergence flag
//   direction  p = z + beta p, Ap = 0 (ready for the next scatter-add)
// All scalars stay on the device (SemScalars); the host reads them every check_every iterations.
// Iterations after convergence or breakdown return at their first instruction, so a block of
// iterations can be launched (or replayed as a CUDA graph) without a host round trip.
//
// Mixed precision (SEM_SOLVE_IR): iterative refinement with an FP64-accurate outer residual
// r = b - A x and an FP32 inner Jacobi-PCG on A d = r / ||r|| to a loose tolerance, x += ||r|| d.
#include <math.h>

#include <algorithm>
#include <string>

#include "sem_internal.h"
#include "sem_reduce.cuh"

namespace {

constexpr int VT = 256;           // threads per block of the vector kernels
constexpr int VBLOCKS = 152 * 8;  // fixed grid: deterministic reduction order

template <typename T>
__global__ void __launch_bounds__(VT) k_cg_init(int64_t G, const double *b, double bscale, const double *Ax,
                                                const uint8_t *dir_zero_src, T *r, T *p, const T *dinv,
                                                SemScalars *S, double *partials, double rtol2) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  double rz = 0.0, rr = 0.0, bb = 0.0;
  (void)dir_zero_src;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) {
    const double di = (double)dinv[g];
    // Dirichlet rows have dinv = 0 and zero right-hand side: r = 0 there
    const double bg = di != 0.0 ? b[g] : 0.0;
    const double rg = (bg - (Ax ? Ax[g] : 0.0)) * bscale;
    const T rt = (T)rg;
    r[g] = rt;
    const T z = rt * dinv[g];
    p[g] = z;
    rz += (double)rt * (double)z;
    rr += (double)rt * (double)rt;
    bb += bg * bg;
  }
  const double a = block_sum<VT>(rz, s_red), c = block_sum<VT>(rr, s_red), d = block_sum<VT>(bb, s_red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = a;
    partials[gridDim.x + blockIdx.x] = c;
    partials[2 * gridDim.x + blockIdx.x] = d;
  }
  if (publish_partial<VT>(0.0, partials + 3 * gridDim.x, &S->counter[1], s_red, &s_flag)) {
    const double RZ = final_sum<VT>(partials, gridDim.x, s_red);
    const double RR = final_sum<VT>(partials + gridDim.x, gridDim.x, s_red);
    const double BB = final_sum<VT>(partials + 2 * gridDim.x, gridDim.x, s_red);
    if (threadIdx.x == 0) {
      S->rz = RZ;
      S->rr = RR;
      S->bb = BB;
      S->tol2 = rtol2 * RR;  // relative to the initial residual of this (inner or outer) solve
      S->converged = RR <= S->tol2 || RR == 0.0;
      S->breakdown = !isfinite(RR) || !isfinite(RZ);
      S->iter = 0;
      S->counter[1] = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(VT) k_cg_update(int64_t G, T *x, const T *p, T *r, const T *Ap, const T *dinv,
                                                  SemScalars *S, double *partials) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  if (S->converged || S->breakdown) return;
  const T alpha = (T)S->alpha;
  // per-thread partial sums in the vector precision (a thread sees about G / 311k entries; FP64
  // arithmetic per entry would cost more than the traffic on GB300), widened for the block sum
  T rz = T(0), rr = T(0);
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) {
    x[g] += alpha * p[g];
    const T rg = r[g] - alpha * Ap[g];
    r[g] = rg;
    const T z = rg * dinv[g];
    rz += rg * z;
    rr += rg * rg;
  }
  const double a = block_sum<VT>((double)rz, s_red), c = block_sum<VT>((double)rr, s_red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = a;
    partials[gridDim.x + blockIdx.x] = c;
  }
  if (publish_partial<VT>(0.0, partials + 2 * gridDim.x, &S->counter[2], s_red, &s_flag)) {
    const double RZ = final_sum<VT>(partials, gridDim.x, s_red);
    const double RR = final_sum<VT>(partials + gridDim.x, gridDim.x, s_red);
    if (threadIdx.x == 0) {
      S->beta = RZ / S->rz;
      S->rz = RZ;
      S->rr = RR;
      S->iter += 1;
      if (!isfinite(RR) || !isfinite(RZ)) S->breakdown = 1;
      if (RR <= S->tol2) S->converged = 1;
      S->counter[2] = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(VT) k_cg_direction(int64_t G, T *p, const T *r, T *Ap, const T *dinv,
                                                     const SemScalars *S) {
  if (S->converged || S->breakdown) return;
  const T beta = (T)S->beta;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) {
    p[g] = r[g] * dinv[g] + beta * p[g];
    Ap[g] = T(0);
  }
}

// r = M (b - Ax) in FP64 with (r, r) and (b, b) -> S->rr, S->bb (true residual)
__global__ void __launch_bounds__(VT) k_residual64(int64_t G, const double *b, const double *Ax, const double *dinv,
                                                   double *r, SemScalars *S, double *partials) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  double rr = 0.0, bb = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) {
    const bool free_node = dinv[g] != 0.0;
    const double bg = free_node ? b[g] : 0.0;
    const double rg = free_node ? bg - Ax[g] : 0.0;
    r[g] = rg;
    rr += rg * rg;
    bb += bg * bg;
  }
  const double a = block_sum<VT>(rr, s_red), c = block_sum<VT>(bb, s_red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = a;
    partials[gridDim.x + blockIdx.x] = c;
  }
  if (publish_partial<VT>(0.0, partials + 2 * gridDim.x, &S->counter[3], s_red, &s_flag)) {
    const double RR = final_sum<VT>(partials, gridDim.x, s_red);
    const double BB = final_sum<VT>(partials + gridDim.x, gridDim.x, s_red);
    if (threadIdx.x == 0) {
      S->rr = RR;
      S->bb = BB;
      S->scale = sqrt(RR);
      S->counter[3] = 0;
    }
  }
}

// x += scale * d (FP64 += FP32 correction)
__global__ void __launch_bounds__(VT) k_ir_correct(int64_t G, double *x, const float *d, const SemScalars *S) {
  const double s = S->scale;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT)
    x[g] += s * (double)d[g];
}

template <typename T>
__global__ void __launch_bounds__(VT) k_fill(int64_t G, T *v, T val) {
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) v[g] = val;
}

// ---- flexible CG (learned preconditioner) ----
// x += alpha p ; r -= alpha Ap ; (r, r) -> convergence
__global__ void __launch_bounds__(VT) k_fcg_update(int64_t G, double *x, const double *p, double *r, const double *Ap,
                                                   SemScalars *S, double *partials) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  if (S->converged || S->breakdown) return;
  const double alpha = S->alpha;
  double rr = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) {
    x[g] += alpha * p[g];
    const double rn = r[g] - alpha * Ap[g];
    r[g] = rn;
    rr += rn * rn;
  }
  if (publish_partial<VT>(block_sum<VT>(rr, s_red), partials, &S->counter[5], s_red, &s_flag)) {
    const double RR = final_sum<VT>(partials, gridDim.x, s_red);
    if (threadIdx.x == 0) {
      S->rr = RR;
      S->iter += 1;
      if (!isfinite(RR)) S->breakdown = 1;
      if (RR <= S->tol2) S->converged = 1;
      S->counter[5] = 0;
    }
  }
}

// (z, r) and (z, Ap): flexible (Polak-Ribiere) beta = (z, r - r_old) / (z,r)_old (0 on the first
// iteration after a start or restart, S->iter == S->restart_iter).  The residual step
// r - r_old is -alpha A p of the previous iteration, still held in Ap (it is cleared only by the
// direction update), so beta = -alpha (z, Ap) / (z,r)_old needs no copy of the old residual.
// second == 0: the learned z; a correction with (z, r) <= 0 or a non-finite value is rejected
// (fallback flag, counted).  second == 1: runs only after a
// rejection, on the Jacobi z; if that fails too the solve breaks down.  Every block reads the
// flags at entry, before the last block can change them, so all blocks agree.
__global__ void __launch_bounds__(VT) k_fcg_dots(int64_t G, const double *z, const double *r, const double *Ap,
                                                 SemScalars *S, double *partials, int second) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  if (S->converged || S->breakdown || (second && !S->fallback)) return;
  const bool first = S->iter == S->restart_iter;
  double a = 0.0, b = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) {
    a += z[g] * r[g];
    if (!first) b += z[g] * Ap[g];
  }
  const double A = block_sum<VT>(a, s_red), B = block_sum<VT>(b, s_red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = A;
    partials[gridDim.x + blockIdx.x] = B;
  }
  if (publish_partial<VT>(0.0, partials + 2 * gridDim.x, &S->counter[6], s_red, &s_flag)) {
    const double ZR = final_sum<VT>(partials, gridDim.x, s_red);
    const double ZAp = final_sum<VT>(partials + gridDim.x, gridDim.x, s_red);
    if (threadIdx.x == 0) {
      const double ZT = first ? ZR : ZR + S->alpha * ZAp;  // (z, r_old)
      S->zt = ZT;
      if (!(ZR > 0.0) || !isfinite(ZR) || !isfinite(ZT)) {
        if (second) S->breakdown = 1;  // the Jacobi step itself is not a descent direction
        else {
          S->fallback = 1;
          S->nfallback += 1;
        }
      } else {
        S->fallback = 0;
        S->beta = first ? 0.0 : -S->alpha * ZAp / S->rz;
        S->rz = ZR;
      }
      S->counter[6] = 0;
    }
  }
}

// z = D^-1 r where the learned correction was rejected
__global__ void __launch_bounds__(VT) k_jacobi_z(int64_t G, const double *r, const double *dinv, double *z,
                                                 const SemScalars *S) {
  if (S->converged || S->breakdown || !S->fallback) return;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) z[g] = r[g] * dinv[g];
}

// p = z + beta p (p = z on the first iteration after a start or restart), Ap = 0 for the next apply
__global__ void __launch_bounds__(VT) k_fcg_direction(int64_t G, double *p, const double *z, double *Ap,
                                                      const SemScalars *S) {
  if (S->converged || S->breakdown) return;
  const bool first = S->iter == S->restart_iter;
  const double beta = S->beta;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < G; g += (int64_t)gridDim.x * VT) {
    p[g] = first ? z[g] : z[g] + beta * p[g];
    Ap[g] = 0.0;
  }
}

// x . y over n entries -> *out, FP64, fixed reduction order for a given n
__global__ void __launch_bounds__(VT) k_dot(int64_t n, const double *x, const double *y, double *out,
                                            double *partials, unsigned int *ticket) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  double acc = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * VT + threadIdx.x; g < n; g += (int64_t)gridDim.x * VT) acc += x[g] * y[g];
  const double bs = block_sum<VT>(acc, s_red);
  if (publish_partial<VT>(bs, partials, ticket, s_red, &s_flag)) {
    const double tot = final_sum<VT>(partials, gridDim.x, s_red);
    if (threadIdx.x == 0) {
      *out = tot;
      *ticket = 0;
    }
  }
}

inline unsigned vgrid(int64_t G) {
  const int64_t need = (G + VT - 1) / VT;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(VBLOCKS, need));
}

// Copies the solver scalars to the host (synchronising the stream).  A bounded device wait that
// gave up since the solve started (an apply left its output incomplete) ends the solve with
// SEM_ERR_TIMEOUT; the flag and the reduction tickets are cleared for later calls.
sem_status read_scalars(sem_handle *h, SemScalars *out, cudaStream_t st) {
  SEM_CUDA_TRY(cudaMemcpyAsync(out, h->scal, sizeof(SemScalars), cudaMemcpyDeviceToHost, st));
  SEM_CUDA_TRY(cudaStreamSynchronize(st));
  if (out->error) {
    const sem_status s = sem_clear_timeout(h, st);
    if (s != SEM_OK) return s;
    SEM_CUDA_TRY(cudaStreamSynchronize(st));
    return sem_fail(SEM_ERR_TIMEOUT, "a bounded device wait gave up during the solve");
  }
  return SEM_OK;
}

// FP64-accurate operator into y (zeroed first); no fused epilogue.
sem_status apply64(sem_handle *h, int prec, const double *u, double *y, cudaStream_t st) {
  SEM_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)h->G * 8, st));
  return sem_launch_apply(h, (sem_prec)prec, u, y, nullptr, nullptr, nullptr, st);
}

// The caller's residual history (sem_pcg_opts.history): (iterations, relative residual) pairs
// appended at each host check while room is left.
struct History {
  double *buf = nullptr;
  int cap = 0, len = 0;
  void add(int iters, double rel) {
    if (buf && len < cap) {
      buf[2 * len] = (double)iters;
      buf[2 * len + 1] = rel;
      ++len;
    }
  }
};

// One block of `count` CG iterations on type T.
template <typename T>
sem_status cg_block(sem_handle *h, int prec, int count, T *x, T *p, T *r, T *Ap, const T *dinv, cudaStream_t st) {
  for (int it = 0; it < count; ++it) {
    sem_status s = sem_launch_apply(h, (sem_prec)prec, p, Ap, h->partials, nullptr, nullptr, st);
    if (s != SEM_OK) return s;
    k_cg_update<T><<<vgrid(h->G), VT, 0, st>>>(h->G, x, p, r, Ap, dinv, h->scal, h->partials);
    k_cg_direction<T><<<vgrid(h->G), VT, 0, st>>>(h->G, p, r, Ap, dinv, h->scal);
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

// Runs CG from the state set up by k_cg_init until convergence, breakdown or max_it.
// hist (may be null) gets (it0 + iterations, sqrt(rr / bb)) at each host check.
template <typename T>
sem_status cg_run(sem_handle *h, int prec, const sem_pcg_opts *o, T *x, T *p, T *r, T *Ap, const T *dinv,
                  cudaStream_t st, int *iters, double *rr_out, int budget, History *hist = nullptr, int it0 = 0,
                  double bb = 0.0) {
  SemScalars hs;
  sem_status s = read_scalars(h, &hs, st);
  if (s != SEM_OK) return s;
  if (hist && bb > 0) hist->add(it0 + hs.iter, sqrt(hs.rr / bb));
  const int every = std::max(1, o->check_every);
  cudaGraphExec_t exec = nullptr;
  bool graph = o->use_graph && st != nullptr;
  while (!hs.converged && !hs.breakdown && hs.iter < budget) {
    const int count = std::min(every, budget - hs.iter);
    if (graph && count == every) {
      if (!exec) {
        cudaGraph_t g;
        SEM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        sem_status cs = cg_block<T>(h, prec, count, x, p, r, Ap, dinv, st);
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (cs != SEM_OK) {
          if (ce == cudaSuccess) cudaGraphDestroy(g);
          return cs;
        }
        if (ce != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
      }
      cudaError_t ce = cudaGraphLaunch(exec, st);
      if (ce != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return sem_fail(SEM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
      }
    } else {
      s = cg_block<T>(h, prec, count, x, p, r, Ap, dinv, st);
      if (s != SEM_OK) break;
    }
    s = read_scalars(h, &hs, st);
    if (s != SEM_OK) break;
    if (hist && bb > 0) hist->add(it0 + hs.iter, sqrt(hs.rr / bb));
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (s != SEM_OK) return s;
  *iters = hs.iter;
  *rr_out = hs.rr;
  if (hs.breakdown) return sem_fail(SEM_ERR_BREAKDOWN, "CG breakdown: non-positive or non-finite p^T A p");
  return hs.converged ? SEM_OK : SEM_ERR_NOCONV;
}

}  // namespace

// `count` flexible-CG iterations with the learned preconditioner, no host synchronisation
sem_status fcg_block(sem_handle *h, int prec64, int count, double *x, cudaStream_t st) {
  const int64_t G = h->G;
  for (int it = 0; it < count; ++it) {
    sem_status s = sem_mlp_precond_apply(h, h->r64, h->z64, st);
    if (s != SEM_OK) return s;
    k_fcg_dots<<<vgrid(G), VT, 0, st>>>(G, h->z64, h->r64, h->Ap64, h->scal, h->partials, 0);
    // the fallback pair does work only after a rejected correction (rare): one block per SM of a
    // GB300 (152), so that the launches that find nothing to do cost little
    const unsigned fb = std::min(vgrid(G), 152u);
    k_jacobi_z<<<fb, VT, 0, st>>>(G, h->r64, h->dinv64, h->z64, h->scal);
    k_fcg_dots<<<fb, VT, 0, st>>>(G, h->z64, h->r64, h->Ap64, h->scal, h->partials, 1);
    k_fcg_direction<<<vgrid(G), VT, 0, st>>>(G, h->p64, h->z64, h->Ap64, h->scal);
    // Ap with fused p^T A p and alpha = (z, r) / (p, A p)
    s = sem_launch_apply(h, (sem_prec)prec64, h->p64, h->Ap64, h->partials, nullptr, nullptr, st);
    if (s != SEM_OK) return s;
    k_fcg_update<<<vgrid(G), VT, 0, st>>>(G, x, h->p64, h->r64, h->Ap64, h->scal, h->partials);
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_pcg(sem_handle *h, const double *d_b, double *d_x, const sem_pcg_opts *o,
                              sem_pcg_result *res, sem_stream_t stream) {
  NvtxRange nvtx_solve("sem_pcg");
  if (!h || !d_b || !d_x || !o || !res) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  memset(res, 0, sizeof(*res));
  History hist;
  auto ret = [&](sem_status v) {
    res->status = v;
    res->history_len = hist.len;
    return v;
  };
  if (o->history_cap < 0 || (o->history_cap > 0 && !o->history))
    return ret(sem_fail(SEM_ERR_INVALID, "history_cap needs a history array (and must not be negative)"));
  hist.buf = o->history_cap > 0 ? o->history : nullptr;
  hist.cap = o->history_cap;
  if (!h->r64) return ret(sem_fail(SEM_ERR_INVALID, "handle was set up without SEM_FEAT_PCG"));
  if (!(o->rtol > 0.0) || o->max_it < 1) return ret(sem_fail(SEM_ERR_INVALID, "bad rtol or max_it"));
  const int prec64 = o->apply_prec;
  if (prec64 != SEM_FP64 && prec64 != SEM_FP64_EMU)
    return ret(sem_fail(SEM_ERR_INVALID, "apply_prec must be SEM_FP64 or SEM_FP64_EMU"));
  if ((prec64 == SEM_FP64 && !h->G64) || (prec64 == SEM_FP64_EMU && !h->Gemu))
    return ret(sem_fail(SEM_ERR_INVALID, "handle lacks the factor set of apply_prec"));
  const int64_t G = h->G;
  sem_status s = SEM_OK;
  SemScalars hs;
  SEM_CUDA_TRY(cudaMemsetAsync(h->scal, 0, sizeof(SemScalars), st));

  if (o->mode == SEM_SOLVE_FP64) {
    NvtxRange nvtx_mode("jacobi-pcg");
    // r = b - A x0 ; z = r/d ; p = z.  A restart (from the current x) follows if the true residual
    // of a converged recurrence is still above rtol.
    int total = 0;
    for (int restart = 0; restart < 4; ++restart) {
      s = apply64(h, prec64, d_x, h->Ap64, st);
      if (s != SEM_OK) return ret(s);
      k_cg_init<double><<<vgrid(G), VT, 0, st>>>(G, d_b, 1.0, h->Ap64, nullptr, h->r64, h->p64, h->dinv64,
                                                 h->scal, h->partials, 0.0);
      SEM_CUDA_TRY(cudaMemsetAsync(h->Ap64, 0, (size_t)G * 8, st));
      s = read_scalars(h, &hs, st);
      if (s != SEM_OK) return ret(s);
      hs.tol2 = o->rtol * o->rtol * hs.bb;  // stop on ||r|| <= rtol ||b||
      hs.converged = hs.rr <= hs.tol2;
      SEM_CUDA_TRY(cudaMemcpyAsync(h->scal, &hs, sizeof(SemScalars), cudaMemcpyHostToDevice, st));
      const double bb = hs.bb;
      int iters = 0;
      double rr = 0.0;
      s = cg_run<double>(h, prec64, o, d_x, h->p64, h->r64, h->Ap64, h->dinv64, st, &iters, &rr,
                         std::max(1, o->max_it - total), &hist, total, bb);
      total += iters;
      res->recursive_relres = bb > 0 ? sqrt(rr / bb) : 0.0;
      if (s != SEM_OK) break;
      // true residual of this x
      s = apply64(h, prec64, d_x, h->Ap64, st);
      if (s != SEM_OK) break;
      k_residual64<<<vgrid(G), VT, 0, st>>>(G, d_b, h->Ap64, h->dinv64, h->t64, h->scal, h->partials);
      s = read_scalars(h, &hs, st);
      if (s != SEM_OK) break;
      if (!(hs.bb > 0) || sqrt(hs.rr / hs.bb) <= o->rtol || total >= o->max_it) break;
    }
    res->iterations = total;
  } else if (o->mode == SEM_SOLVE_IR) {
    NvtxRange nvtx_mode("refinement");
    // inner apply: FP32 factors (default), BF16-stored factors or factors recomputed on the fly,
    // FP32 arithmetic in each case
    const int inner_prec =
        (o->inner_prec == SEM_BF16 || o->inner_prec == SEM_FP32_OTF) ? o->inner_prec : (int)SEM_FP32;
    const bool have = inner_prec == SEM_BF16 ? h->G16 != nullptr
                      : inner_prec == SEM_FP32_OTF ? h->Gotf != nullptr : h->G32 != nullptr;
    if (!have || !h->r32)
      return ret(sem_fail(SEM_ERR_INVALID,
                          "IR needs SEM_FEAT_PCG and the inner factor set (SEM_FEAT_FP32, _BF16 or _OTF)"));
    const double inner = o->inner_rtol > 0 ? o->inner_rtol : 1e-4;
    int total = 0;
    for (int outer = 0; outer < 100; ++outer) {
      s = apply64(h, prec64, d_x, h->Ap64, st);
      if (s != SEM_OK) break;
      k_residual64<<<vgrid(G), VT, 0, st>>>(G, d_b, h->Ap64, h->dinv64, h->r64, h->scal, h->partials);
      s = read_scalars(h, &hs, st);
      if (s != SEM_OK) break;
      const double rel = hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0;
      res->outer = outer;
      res->recursive_relres = rel;
      hist.add(total, rel);
      if (rel <= o->rtol || hs.rr == 0.0) {
        s = SEM_OK;
        break;
      }
      if (total >= o->max_it) {
        s = sem_fail(SEM_ERR_NOCONV, "IR: inner iteration budget exhausted");
        break;
      }
      if (!isfinite(rel)) {
        s = sem_fail(SEM_ERR_BREAKDOWN, "IR: non-finite residual");
        break;
      }
      // inner FP32 solve of A d = r / ||r|| from d = 0
      k_fill<float><<<vgrid(G), VT, 0, st>>>(G, h->x32, 0.0f);
      k_fill<float><<<vgrid(G), VT, 0, st>>>(G, h->Ap32, 0.0f);
      k_cg_init<float><<<vgrid(G), VT, 0, st>>>(G, h->r64, 1.0 / hs.scale, nullptr, nullptr, h->r32, h->p32,
                                                h->dinv32, h->scal, h->partials, inner * inner);
      int iters = 0;
      double rr = 0.0;
      s = cg_run<float>(h, inner_prec, o, h->x32, h->p32, h->r32, h->Ap32, h->dinv32, st, &iters, &rr,
                        std::max(1, o->max_it - total));
      total += iters;
      if (s == SEM_ERR_NOCONV) s = SEM_OK;  // a partial inner solve still improves x
      if (s == SEM_ERR_BREAKDOWN && iters > 0) s = SEM_OK;
      if (s != SEM_OK) break;
      k_ir_correct<<<vgrid(G), VT, 0, st>>>(G, d_x, h->x32, h->scal);
    }
    res->iterations = total;
  } else if (o->mode == SEM_SOLVE_FCG_MLP) {
    NvtxRange nvtx_mode("flexible-cg");
    if (!h->z64 || !h->mlp_w) return ret(sem_fail(SEM_ERR_INVALID, "FCG needs SEM_FEAT_MLP | SEM_FEAT_PCG and sem_mlp_load"));
    // r = b - A x0 (FP64-accurate), tolerance relative to ||b||
    s = apply64(h, prec64, d_x, h->Ap64, st);
    if (s != SEM_OK) return ret(s);
    k_residual64<<<vgrid(G), VT, 0, st>>>(G, d_b, h->Ap64, h->dinv64, h->r64, h->scal, h->partials);
    s = read_scalars(h, &hs, st);
    if (s != SEM_OK) return ret(s);
    hs.tol2 = o->rtol * o->rtol * hs.bb;
    hs.converged = hs.rr <= hs.tol2;
    hs.iter = 0;
    SEM_CUDA_TRY(cudaMemcpyAsync(h->scal, &hs, sizeof(SemScalars), cudaMemcpyHostToDevice, st));
    hs.fallback = 0;
    hs.nfallback = 0;
    hs.restart_iter = 0;
    SEM_CUDA_TRY(cudaMemcpyAsync(h->scal, &hs, sizeof(SemScalars), cudaMemcpyHostToDevice, st));
    const double bb = hs.bb;
    if (bb > 0) hist.add(0, sqrt(hs.rr / bb));
    // blocks of check_every iterations, decided on the device (fallback, beta, alpha, convergence),
    // replayed as one CUDA graph; the host reads the scalars once per block
    const int every = std::max(1, o->check_every);
    cudaGraphExec_t exec = nullptr;
    const bool graph = o->use_graph && st != nullptr;
    bool eager_done = false;  // one eager iteration first: attributes and tables are set up before capture
    // When the recursive residual meets the tolerance but the FP64-accurate true residual does
    // not (the recurrence drifts over many iterations with a changing preconditioner), the
    // residual is replaced by the true one and flexible CG restarts from x, a few times at most.
    int restarts = 0;
    for (;;) {
      while (s == SEM_OK && !hs.converged && !hs.breakdown && hs.iter < o->max_it) {
        const int count = std::min(every, o->max_it - hs.iter);
        if (graph && eager_done && count == every) {
          if (!exec) {
            cudaGraph_t g;
            SEM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            sem_status cs = fcg_block(h, prec64, count, d_x, st);
            cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (cs != SEM_OK) {
              if (ce == cudaSuccess) cudaGraphDestroy(g);
              return ret(cs);
            }
            if (ce != cudaSuccess) return ret(sem_fail(SEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce)));
            ce = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess)
              return ret(sem_fail(SEM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce)));
          }
          const cudaError_t ce = cudaGraphLaunch(exec, st);
          if (ce != cudaSuccess) s = sem_fail(SEM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
        } else {
          s = fcg_block(h, prec64, graph && !eager_done ? 1 : count, d_x, st);
          eager_done = true;
        }
        if (s != SEM_OK) break;
        s = read_scalars(h, &hs, st);
        if (s == SEM_OK && bb > 0) hist.add(hs.iter, sqrt(hs.rr / bb));
      }
      if (s != SEM_OK || hs.breakdown || !hs.converged || restarts >= 8) break;
      s = apply64(h, prec64, d_x, h->Ap64, st);
      if (s != SEM_OK) break;
      k_residual64<<<vgrid(G), VT, 0, st>>>(G, d_b, h->Ap64, h->dinv64, h->r64, h->scal, h->partials);
      s = read_scalars(h, &hs, st);
      if (s != SEM_OK || hs.rr <= hs.tol2 || hs.iter >= o->max_it) break;
      ++restarts;
      hs.converged = 0;
      hs.restart_iter = hs.iter;
      SEM_CUDA_TRY(cudaMemcpyAsync(h->scal, &hs, sizeof(SemScalars), cudaMemcpyHostToDevice, st));
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (s == SEM_OK && hs.breakdown) s = sem_fail(SEM_ERR_BREAKDOWN, "flexible CG breakdown");
    const int fallbacks = hs.nfallback;
    if (s == SEM_OK && !hs.converged) s = sem_fail(SEM_ERR_NOCONV, "flexible CG: max_it reached");
    res->iterations = hs.iter;
    res->fallbacks = fallbacks;
    res->recursive_relres = bb > 0 ? sqrt(hs.rr / bb) : 0.0;
  } else {
    return ret(sem_fail(SEM_ERR_INVALID, "unknown solve mode"));
  }

  // true FP64 residual of the returned x
  if (s == SEM_OK || s == SEM_ERR_NOCONV || s == SEM_ERR_BREAKDOWN) {
    NvtxRange nvtx_true("true-residual");
    sem_status s2 = apply64(h, prec64, d_x, h->Ap64, st);
    if (s2 == SEM_OK) {
      k_residual64<<<vgrid(G), VT, 0, st>>>(G, d_b, h->Ap64, h->dinv64, h->t64, h->scal, h->partials);
      s2 = read_scalars(h, &hs, st);
    }
    if (s2 != SEM_OK) return ret(s2);
    res->true_relres = hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0;
    if (s == SEM_OK && res->true_relres > o->rtol)
      s = sem_fail(SEM_ERR_NOCONV, "true residual above rtol after the iteration budget");
  }
  return ret(s);
}

extern "C" sem_status sem_dot(sem_handle *h, const double *d_x, const double *d_y, double *d_out,
                              sem_stream_t stream) {
  if (!h || !d_x || !d_y || !d_out) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_dot<<<vgrid(h->G), VT, 0, st>>>(h->G, d_x, d_y, d_out, h->partials, &h->scal->counter[4]);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_residual(sem_handle *h, sem_prec prec, const double *d_b, const double *d_x, double *d_r,
                                   sem_stream_t stream) {
  if (!h || !d_b || !d_x || !d_r) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  if (prec != SEM_FP64 && prec != SEM_FP64_EMU) return sem_fail(SEM_ERR_INVALID, "residual needs an FP64-accurate apply");
  if (!h->t64) return sem_fail(SEM_ERR_INVALID, "handle was set up without SEM_FEAT_PCG");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  sem_status s = apply64(h, prec, d_x, h->t64, st);
  if (s != SEM_OK) return s;
  k_residual64<<<vgrid(h->G), VT, 0, st>>>(h->G, d_b, h->t64, h->dinv64, d_r, h->scal, h->partials);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}
