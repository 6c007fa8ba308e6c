// Training pairs of the learned element preconditioner: residual-to-error pairs of the element-local
// problem, produced by Jacobi-PCG on that problem.
//
// For a sampled element e and a global residual r (an iterate's residual of the global Jacobi-PCG
// solve), the local problem is the element's own operator with a small mass shift, no boundary
// conditions (the element is cut out of the mesh):
//     (A_e + sigma_e M_e) x_e = W_e r_e,   sigma_e = eps * trace(A_e) / sum_p (w det J)_p,
// with A_e the element stiffness (sum-factorised, §4.2.1; plus the problem's own lumped mass term
// if it has one), M_e the lumped mass diag(w det J), W_e = 1 / multiplicity of each node, and r_e
// zero on Dirichlet nodes.  x_e is the correction that removes the element's share of the
// residual (a one-level Neumann-Neumann step); the network learns r_e -> x_e so that the
// multiplicity-weighted average of the predicted corrections over all elements approximates
// sum_e Q^T W_e (A_e + sigma_e M_e)^-1 W_e Q r.
//
// One block per sample, NP^2 threads: thread (a, b) owns the nodes (a, b, c), c = 0..N, of its
// column.  The local Jacobi-PCG runs in FP64 with the search direction in shared memory; every
// iteration is one local sum-factorised apply and three block reductions.  The features X and
// scaled targets T are written for the network (targets divided by |r_e| / dbar_e, dbar_e the
// mean of diag(A_e)).
#include <cuda_bf16.h>
#include <math.h>

#include <string>

#include "sem_internal.h"
#include "sem_reduce.cuh"

namespace {

// factor f (rr, rs, rt, ss, st, tt) of node p of element e from whichever copy the handle holds
__device__ __forceinline__ double factor(const sem_handle &h, int64_t e, int f, int p) {
  if (h.G64) return h.G64[e * h.gs6 + (int64_t)f * h.n3 + p];
  if (h.Gemu) {
    const int64_t o = e * h.gs12 + (int64_t)(2 * f) * h.n3 + p;
    return (double)h.Gemu[o] + (double)h.Gemu[o + h.n3];
  }
  return (double)h.G32[e * h.gs6 + (int64_t)f * h.n3 + p];
}

// global id of local node p of element e (structured box or explicit numbering)
__device__ __forceinline__ int64_t node_gid(const sem_handle &h, int64_t e, int p) {
  if (h.glo) return h.glo[e * h.n3 + p];
  const int n = h.n, N = h.N;
  const int i = p % n, j = (p / n) % n, k = p / (n * n);
  const int64_t ex = e % h.box[0], ey = (e / h.box[0]) % h.box[1], ez = e / ((int64_t)h.box[0] * h.box[1]);
  const int64_t gxs = (int64_t)h.box[0] * N + 1, gys = (int64_t)h.box[1] * N + 1;
  return (ex * N + i) + gxs * ((ey * N + j) + gys * (ez * N + k));
}

// diagonal of the element stiffness at node (a, b, c): sum over the three directions of the
// squared derivative weights times the diagonal factors, plus the cross terms at the node itself
__device__ __forceinline__ double local_diag(const sem_handle &h, const double *sD, int64_t e, int a, int b,
                                            int c) {
  const int n = h.n;
  const int p = a + n * (b + n * c);
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    const double da = sD[m * n + a], db = sD[m * n + b], dc = sD[m * n + c];
    s += factor(h, e, 0, m + n * (b + n * c)) * da * da;
    s += factor(h, e, 3, a + n * (m + n * c)) * db * db;
    s += factor(h, e, 5, a + n * (b + n * m)) * dc * dc;
  }
  const double Da = sD[a * n + a], Db = sD[b * n + b], Dc = sD[c * n + c];
  s += 2.0 * (Da * Db * factor(h, e, 1, p) + Da * Dc * factor(h, e, 2, p) + Db * Dc * factor(h, e, 4, p));
  if (h.wJa64) s += h.wJa64[e * h.n3 + p];
  return s;
}

template <int NP>
__global__ void __launch_bounds__(NP * NP) k_local_pcg(sem_handle h, int nsamp, const int32_t *elems,
                                                       const double *r, double eps, double rtol, int maxit,
                                                       int sub_jacobi, float *X, float *T, int *iters) {
  constexpr int NT = NP * NP, N3 = NP * NP * NP;
  extern __shared__ __align__(16) double sm[];
  double *sp = sm, *swr = sp + N3, *sws = swr + N3, *swt = sws + N3, *sD = swt + N3, *s_red = sD + NP * NP;
  const int s = blockIdx.x;
  if (s >= nsamp) return;
  const int64_t e = elems[s];
  const int tid = threadIdx.x, a = tid % NP, b = tid / NP;
  if (e < 0 || e >= h.E) {  // not an element of this problem: a zero pair
    for (int q = tid; q < N3 + 6; q += NT) X[(size_t)s * (N3 + 6) + q] = 0.f;
    for (int q = tid; q < N3; q += NT) T[(size_t)s * N3 + q] = 0.f;
    return;
  }
  for (int q = tid; q < NP * NP; q += NT) sD[q] = h.D64[q];
  __syncthreads();

  double x[NP], res[NP], dS[NP], sh[NP], rin[NP];
  double tr = 0.0, vol = 0.0, rn2 = 0.0;
  uint32_t freebits = 0;
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    const int p = a + NP * (b + NP * c);
    const int64_t g = node_gid(h, e, p);
    const bool fr = h.dinv64[g] != 0.0;
    freebits |= (fr ? 1u : 0u) << c;
    rin[c] = fr ? r[g] : 0.0;
    res[c] = rin[c] * (double)h.inv_mult[g];  // W_e r_e
    x[c] = 0.0;
    dS[c] = local_diag(h, sD, e, a, b, c);
    sh[c] = h.wJ[e * N3 + p];
    tr += dS[c];
    vol += sh[c];
    rn2 += rin[c] * rin[c];
  }
  tr = block_sum<NT>(tr, s_red);
  vol = block_sum<NT>(vol, s_red);
  rn2 = block_sum<NT>(rn2, s_red);
  const double sigma = eps * tr / vol, dbar = tr / N3;
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    sh[c] *= sigma;  // shift of node c: sigma (w det J)
    dS[c] += sh[c];
  }

  double f2 = 0.0, rz = 0.0;
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    const double z = res[c] / dS[c];
    sp[a + NP * (b + NP * c)] = z;
    f2 += res[c] * res[c];
    rz += res[c] * z;
  }
  f2 = block_sum<NT>(f2, s_red);
  rz = block_sum<NT>(rz, s_red);
  int it = 0;
  if (f2 > 0.0) {
    for (it = 1; it <= maxit; ++it) {
      __syncthreads();  // sp complete
      // y = (A_e + sigma M_e) p, first the gradients and the factor scaling of the column's nodes
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          ur += sD[a * NP + m] * sp[m + NP * (b + NP * c)];
          us += sD[b * NP + m] * sp[a + NP * (m + NP * c)];
          ut += sD[c * NP + m] * sp[a + NP * (b + NP * m)];
        }
        const int p = a + NP * (b + NP * c);
        const double grr = factor(h, e, 0, p), grs = factor(h, e, 1, p), grt = factor(h, e, 2, p),
                     gss = factor(h, e, 3, p), gst = factor(h, e, 4, p), gtt = factor(h, e, 5, p);
        swr[p] = grr * ur + grs * us + grt * ut;
        sws[p] = grs * ur + gss * us + gst * ut;
        swt[p] = grt * ur + gst * us + gtt * ut;
      }
      __syncthreads();
      double y[NP], pAp = 0.0;
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        const int p = a + NP * (b + NP * c);
        double v = 0.0;
#pragma unroll
        for (int m = 0; m < NP; ++m)
          v += sD[m * NP + a] * swr[m + NP * (b + NP * c)] + sD[m * NP + b] * sws[a + NP * (m + NP * c)] +
               sD[m * NP + c] * swt[a + NP * (b + NP * m)];
        const double pc = sp[p];
        v += (sh[c] + (h.wJa64 ? h.wJa64[e * N3 + p] : 0.0)) * pc;
        y[c] = v;
        pAp += pc * v;
      }
      pAp = block_sum<NT>(pAp, s_red);
      if (!(pAp > 0.0) || !isfinite(pAp)) break;
      const double alpha = rz / pAp;
      double rr = 0.0, rzn = 0.0;
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        x[c] += alpha * sp[a + NP * (b + NP * c)];
        res[c] -= alpha * y[c];
        rr += res[c] * res[c];
        rzn += res[c] * res[c] / dS[c];
      }
      rr = block_sum<NT>(rr, s_red);
      if (rr <= rtol * rtol * f2) break;
      rzn = block_sum<NT>(rzn, s_red);
      const double beta = rzn / rz;
      rz = rzn;
      __syncthreads();  // every thread has read sp for this iteration
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        const int p = a + NP * (b + NP * c);
        sp[p] = res[c] / dS[c] + beta * sp[p];
      }
    }
  }
  if (tid == 0 && iters) atomicMax(iters, it);

  // features and scaled targets
  const double nrm = sqrt(rn2), inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  const double tscale = nrm > 0.0 ? dbar / nrm : 0.0;  // 1 / (|r_e| / dbar)
  const int nin = N3 + 6;
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    const int p = a + NP * (b + NP * c);
    const bool fr = (freebits >> c) & 1u;
    X[(size_t)s * nin + p] = (float)(rin[c] * inv);
    double t = x[c];
    if (sub_jacobi) t -= h.dinv64[node_gid(h, e, p)] * rin[c];
    T[(size_t)s * N3 + p] = fr ? (float)(t * tscale) : 0.f;
  }
  if (tid < 6) X[(size_t)s * nin + N3 + tid] = h.geo6[e * 6 + tid];
}

template <int NP>
sem_status launch_local(const sem_handle *h, int nsamp, const int32_t *elems, const double *r, double eps,
                        double rtol, int maxit, int sub_jacobi, float *X, float *T, int *iters, cudaStream_t st) {
  constexpr int N3 = NP * NP * NP;
  const size_t smem = (size_t)(4 * N3 + NP * NP + 32) * sizeof(double);
  static std::atomic<unsigned long long> attr_done;
  if (smem > 48 * 1024) SEM_CUDA_TRY(set_smem_limit_once(k_local_pcg<NP>, smem, attr_done));
  k_local_pcg<NP><<<nsamp, NP * NP, smem, st>>>(*h, nsamp, elems, r, eps, rtol, maxit, sub_jacobi, X, T, iters);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace

sem_status sem_mlp_local_pairs(const sem_handle *h, int nsamp, const int32_t *elems, const double *r, double eps,
                               double rtol, int maxit, int sub_jacobi, float *X, float *T, int *iters,
                               cudaStream_t st) {
  switch (h->n) {
#define SEM_LP(NPV) \
  case NPV:         \
    return launch_local<NPV>(h, nsamp, elems, r, eps, rtol, maxit, sub_jacobi, X, T, iters, st);
    SEM_LP(2) SEM_LP(3) SEM_LP(4) SEM_LP(5) SEM_LP(6) SEM_LP(7) SEM_LP(8) SEM_LP(9) SEM_LP(10) SEM_LP(11)
    SEM_LP(12)
#undef SEM_LP
    default:
      return sem_fail(SEM_ERR_INVALID, "learned preconditioner training supports orders N = 1..11");
  }
}

namespace {

// dbar[e] = trace(A_e) / n^3, the element's mean stiffness diagonal (scale of the network's output)
__global__ void k_elem_dbar(sem_handle h, float *dbar) {
  __shared__ double sD[SEM_MAX_NP * SEM_MAX_NP];
  __shared__ double s_red[32];
  const int64_t e = blockIdx.x;
  const int n = h.n;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) sD[q] = h.D64[q];
  __syncthreads();
  double t = 0.0;
  for (int p = threadIdx.x; p < h.n3; p += blockDim.x) t += local_diag(h, sD, e, p % n, (p / n) % n, p / (n * n));
  t = block_sum<256>(t, s_red);
  if (threadIdx.x == 0) dbar[e] = (float)(t / h.n3);
}

}  // namespace

sem_status sem_mlp_dbar_table(const sem_handle *h, float *dbar, cudaStream_t st) {
  k_elem_dbar<<<(unsigned)h->E, 256, 0, st>>>(*h, dbar);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}
