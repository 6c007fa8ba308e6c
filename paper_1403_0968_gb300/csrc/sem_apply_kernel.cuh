// Templated FP64 / FP32 apply kernel (see sem_apply.cu for the algorithm).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sem_internal.h"
#include "sem_reduce.cuh"

template <typename T>
struct ApplyParams {
  int64_t E;
  int sx, sy, sz;
  int64_t gxs, gys, gzs;  // global node counts per direction (structured box)
  int bc;
  const T *u;
  T *y;
  const T *Gf;   // [E][6][n3]
  const T *wJa;  // [E][n3] or NULL
  const T *D;    // [n][n]
  const int32_t *glo;
  const uint8_t *mask;
  double *partials;  // non-NULL: fuse p^T A p and the CG step length
  SemScalars *scal;
};

// elements per block: about 256 threads of n*n
__host__ __device__ constexpr int apply_eb(int N) {
  return (256 / ((N + 1) * (N + 1))) > 0 ? 256 / ((N + 1) * (N + 1)) : 1;
}

template <int N, typename T>
__global__ void __launch_bounds__((N + 1) * (N + 1) * apply_eb(N)) k_apply(const ApplyParams<T> P) {
  constexpr int NP = N + 1, NP2 = NP * NP, NP3 = NP2 * NP, EB = apply_eb(N), NT = NP2 * EB;
  __shared__ T sD[NP][NP + 1];
  __shared__ T s_u[EB][NP][NP + 1];
  __shared__ T s_wr[EB][NP][NP + 1];
  __shared__ T s_ws[EB][NP][NP + 1];
  __shared__ double s_red[32];
  __shared__ int s_flag;

  // inside a solve: nothing to do once the iteration has stopped (flag set by an earlier launch)
  if (P.scal && (P.scal->converged || P.scal->breakdown)) return;
  const int tid = threadIdx.x;
  const int es = tid / NP2, t2 = tid - es * NP2, i = t2 % NP, j = t2 / NP;
  for (int q = tid; q < NP2; q += NT) sD[q / NP][q % NP] = P.D[q];
  const int64_t e = (int64_t)blockIdx.x * EB + es;
  const bool active = e < P.E;

  // ---- gather u_e = Q M u (column (i, j, 0..N) of this element) ----
  int64_t gbase = 0;
  bool xb = false, yb = false;  // node on a box face in x / y (structured box Dirichlet)
  int ez = 0;
  if (active && !P.glo) {
    const int64_t ex = e % P.sx, ey = (e / P.sx) % P.sy;
    ez = (int)(e / ((int64_t)P.sx * P.sy));
    const int64_t I = ex * N + i, J = ey * N + j;
    gbase = I + P.gxs * (J + P.gys * ((int64_t)ez * N));
    xb = (I == 0) || (I == P.gxs - 1);
    yb = (J == 0) || (J == P.gys - 1);
  }
  T uc[NP];
  uint32_t dirbits = 0;  // bit k: node (i, j, k) is a Dirichlet node
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    int64_t g = 0;
    bool d = false;
    if (active) {
      g = P.glo ? (int64_t)P.glo[e * NP3 + t2 + NP2 * k] : gbase + P.gxs * P.gys * k;
      if (P.bc == SEM_BC_BOX) {
        if (P.glo) {
          const int64_t I = g % P.gxs, J = (g / P.gxs) % P.gys, KK = g / (P.gxs * P.gys);
          d = I == 0 || J == 0 || KK == 0 || I == P.gxs - 1 || J == P.gys - 1 || KK == P.gzs - 1;
        } else {
          const int64_t K = (int64_t)ez * N + k;
          d = xb || yb || K == 0 || K == P.gzs - 1;
        }
      } else if (P.bc == SEM_BC_MASK) {
        d = P.mask[g] != 0;
      }
    }
    dirbits |= (d ? 1u : 0u) << k;
    uc[k] = (active && !d) ? P.u[g] : T(0);
  }
  __syncthreads();
  // D rows/columns this thread needs, in registers for small orders
  constexpr bool DREG = NP <= 8;
  T Dri[DREG ? NP : 1], Drj[DREG ? NP : 1], Dci[DREG ? NP : 1], Dcj[DREG ? NP : 1];
  if constexpr (DREG) {
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      Dri[m] = sD[i][m];
      Drj[m] = sD[j][m];
      Dci[m] = sD[m][i];
      Dcj[m] = sD[m][j];
    }
  }
  T yc[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) yc[k] = T(0);

  const T *Ge = P.Gf + (active ? e : 0) * 6 * NP3 + t2;
  T g0n, g1n, g2n, g3n, g4n, g5n;
  g0n = active ? Ge[0 * NP3] : T(0);
  g1n = active ? Ge[1 * NP3] : T(0);
  g2n = active ? Ge[2 * NP3] : T(0);
  g3n = active ? Ge[3 * NP3] : T(0);
  g4n = active ? Ge[4 * NP3] : T(0);
  g5n = active ? Ge[5 * NP3] : T(0);

#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const T g0 = g0n, g1 = g1n, g2 = g2n, g3 = g3n, g4 = g4n, g5 = g5n;
    if (k + 1 < NP && active) {  // prefetch the next plane's factors
      const int o = NP2 * (k + 1);
      g0n = Ge[0 * NP3 + o];
      g1n = Ge[1 * NP3 + o];
      g2n = Ge[2 * NP3 + o];
      g3n = Ge[3 * NP3 + o];
      g4n = Ge[4 * NP3 + o];
      g5n = Ge[5 * NP3 + o];
    }
    s_u[es][j][i] = uc[k];
    __syncthreads();
    T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      if constexpr (DREG) {
        ur += Dri[m] * s_u[es][j][m];
        us += Drj[m] * s_u[es][m][i];
      } else {
        ur += sD[i][m] * s_u[es][j][m];
        us += sD[j][m] * s_u[es][m][i];
      }
      ut += sD[k][m] * uc[m];
    }
    const T wr = g0 * ur + g1 * us + g2 * ut;
    const T ws = g1 * ur + g3 * us + g4 * ut;
    const T wt = g2 * ur + g4 * us + g5 * ut;
    s_wr[es][j][i] = wr;
    s_ws[es][j][i] = ws;
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) yc[k2] += sD[k][k2] * wt;
    __syncthreads();
    T acc = T(0);
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      if constexpr (DREG)
        acc += Dci[m] * s_wr[es][j][m] + Dcj[m] * s_ws[es][m][i];
      else
        acc += sD[m][i] * s_wr[es][j][m] + sD[m][j] * s_ws[es][m][i];
    }
    yc[k] += acc;
  }
  if (P.wJa && active) {
#pragma unroll
    for (int k = 0; k < NP; ++k) yc[k] += P.wJa[e * NP3 + t2 + NP2 * k] * uc[k];
  }

  // ---- scatter y += M Q^T y_e ----
  double dotp = 0.0;
  if (active) {
    const bool ij_interior = (i > 0) && (i < N) && (j > 0) && (j < N) && !P.glo;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if ((dirbits >> k) & 1u) continue;
      const int64_t g = P.glo ? (int64_t)P.glo[e * NP3 + t2 + NP2 * k] : gbase + P.gxs * P.gys * k;
      dotp += (double)uc[k] * (double)yc[k];
      if (ij_interior && k > 0 && k < N)
        P.y[g] = yc[k];
      else
        atomicAdd(P.y + g, yc[k]);
    }
  }

  // ---- optional fused p^T A p and CG step length ----
  if (P.partials) {
    const double bs = block_sum<NT>(dotp, s_red);
    if (publish_partial<NT>(bs, P.partials, &P.scal->counter[0], s_red, &s_flag)) {
      const double pAp = final_sum<NT>(P.partials, gridDim.x, s_red);
      if (tid == 0) {
        SemScalars *S = P.scal;
        S->pAp = pAp;
        if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(S->rz)) {
          S->breakdown = 1;
          S->alpha = 0.0;
        } else {
          S->alpha = S->rz / pAp;
        }
        S->counter[0] = 0;
      }
    }
  }
}

template <typename T>
static sem_status dispatch_apply(int N, const ApplyParams<T> &p, cudaStream_t s) {
  const int eb = apply_eb(N);
  const unsigned grid = (unsigned)((p.E + eb - 1) / eb);
  if (p.partials && grid > SEM_MAX_PARTIALS) return sem_fail(SEM_ERR_INVALID, "too many elements for fused dot");
  const int nt = (N + 1) * (N + 1) * eb;
  switch (N) {
#define CASE(NN) \
  case NN:       \
    k_apply<NN, T><<<grid, nt, 0, s>>>(p); \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13)
    CASE(14) CASE(15)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID, "order out of range");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("apply launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}
