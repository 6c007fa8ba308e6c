// Persistent, software-pipelined variant of the FP64 / FP32 apply for structured boxes.
//
// Same element schedule as k_apply (sem_apply_kernel.cuh: five phases, one line per thread and
// direction, D in the constant bank), but each block stays resident and walks element tiles
// (EB elements each) with a stride of the grid size.  While tile t is computed:
//   * the factor block of tile t + grid has already been requested by one bulk (TMA) copy into
//     the second of two shared buffers, completed on its own mbarrier (phases alternate);
//   * the column of u for tile t + grid is loaded into registers during phases 3-4 of tile t.
// So the only global-memory latency left on the critical path is the scatter, which nobody
// waits for.  A fused p^T A p (CG) is accumulated over all tiles of the block and reduced once.
#pragma once

#include "sem_apply_kernel.cuh"

template <int NP, typename T, int EB>
__host__ __device__ constexpr size_t pipe_red_off() {
  using C = ApplyCfg<NP, EB>;
  return ((size_t)(2 * EB * C::GS + EB * 3 * C::BUF) * sizeof(T) + 15) / 16 * 16;
}

template <int NP, typename T, int EB>
__host__ __device__ constexpr size_t pipe_smem() {
  return pipe_red_off<NP, T, EB>() + 32 * 8 + 2 * 8 + 16;
}

template <int NP, typename T, int EB_>
__global__ void __launch_bounds__(ApplyCfg<NP, EB_>::NT) k_apply_pipe(const ApplyParams<T, NP> P, int64_t ntiles) {
  using C = ApplyCfg<NP, EB_>;
  constexpr int N = NP - 1, NP2 = C::NP2, NP3 = C::NP3, EB = C::EB, NT = C::NT, RS = C::RS, PS = C::PS,
                BUF = C::BUF, GS = C::GS;
  constexpr size_t RED_OFF = pipe_red_off<NP, T, EB_>();
  static_assert(RED_OFF % 16 == 0 && (EB * GS * sizeof(T)) % 16 == 0, "shared-memory alignment");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T *sG = reinterpret_cast<T *>(smem_raw);  // [2][EB * GS], TMA destinations
  T *sbuf = sG + 2 * EB * GS;
  double *s_red = reinterpret_cast<double *>(smem_raw + RED_OFF);
  uint64_t *bar = reinterpret_cast<uint64_t *>(s_red + 32);  // bar[0], bar[1]
  int *s_flag = reinterpret_cast<int *>(bar + 2);

  if (P.scal && (P.scal->converged || P.scal->breakdown)) return;
  const int tid = threadIdx.x;
  const int es = tid / NP2, t2 = tid - es * NP2, a = t2 % NP, b = t2 / NP;
  T *su = sbuf + es * 3 * BUF, *sr = su + BUF, *ss = sr + BUF;
  const T *D = P.D.v;
  const int64_t plane = P.gxs * P.gys;

  auto issue = [&](int64_t tile, int buf) {
    const int64_t e0 = tile * EB;
    const int64_t nel = (P.E - e0) < EB ? (P.E - e0) : EB;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tma_load_1d(sG + buf * EB * GS, static_cast<const T *>(P.Gf) + e0 * P.gs, (uint32_t)(nel * P.gs * sizeof(T)),
                bar + buf);
  };
  // column (a, b) of element e: global base index and Dirichlet bits (all set when inactive)
  auto column = [&](int64_t e, int64_t &gbase, uint32_t &dirbits) {
    gbase = 0;
    dirbits = (1u << NP) - 1u;
    if (e >= P.E) return;
    const int64_t ex = e % P.sx, exy = e / P.sx, ey = exy % P.sy, ez = exy / P.sy;
    const int64_t I = ex * N + a, J = ey * N + b;
    gbase = I + P.gxs * (J + P.gys * (ez * N));
    dirbits = 0;
    if (P.bc == SEM_BC_BOX) {
      if (I == 0 || I == P.gxs - 1 || J == 0 || J == P.gys - 1) dirbits = (1u << NP) - 1u;
      if (ez == 0) dirbits |= 1u;
      if (ez == P.sz - 1) dirbits |= 1u << N;
    }
  };

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
  }
  __syncthreads();
  int64_t tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) issue(tile, 0);
  int64_t gnext;
  uint32_t dnext;
  T un[NP];
  column(tile * EB + es, gnext, dnext);
#pragma unroll
  for (int k = 0; k < NP; ++k) un[k] = ((dnext >> k) & 1u) ? T(0) : P.u[gnext + k * plane];

  T dotp = T(0);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int bsel = it & 1;
    const uint32_t par = (uint32_t)((it >> 1) & 1);
    const int64_t next = tile + gridDim.x;
    if (tid == 0 && next < ntiles) issue(next, bsel ^ 1);
    const int64_t e = tile * EB + es;
    const bool active = e < P.E;
    const int64_t gbase = gnext;
    const uint32_t dirbits = dnext;

    // ---- phase 0: the prefetched column ----
    T uc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      uc[k] = un[k];
      su[k * PS + b * RS + a] = uc[k];
    }
    __syncthreads();

    // ---- phase 1: gradients ----
    T wt[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < NP; ++m) acc += D[k * NP + m] * uc[m];
      wt[k] = acc;
    }
    {
      T row[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = su[b * PS + a * RS + m];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < NP; ++m) acc += D[i * NP + m] * row[m];
        sr[b * PS + a * RS + i] = acc;
      }
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = su[b * PS + m * RS + a];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < NP; ++m) acc += D[j * NP + m] * row[m];
        ss[b * PS + j * RS + a] = acc;
      }
    }
    const bool ok = mbar_wait(bar + bsel, par, P.wait_polls);
    if (__syncthreads_or(!ok)) {
      // record the timeout; wait (bounded) for this block's own copies in flight, then leave
      if (tid == 0) {
        if (P.err) atomicOr(P.err, 1);
        mbar_wait(bar + bsel, par);
        if (next < ntiles) mbar_wait(bar + (bsel ^ 1), (uint32_t)(((it + 1) >> 1) & 1));
      }
      return;
    }

    // ---- phase 2: geometric factors ----
    const T *Ge = sG + bsel * EB * GS + es * GS + t2;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = k * PS + b * RS + a;
      const int o = k * NP2;
      const T g0 = Ge[0 * NP3 + o], g1 = Ge[1 * NP3 + o], g2 = Ge[2 * NP3 + o];
      const T g3 = Ge[3 * NP3 + o], g4 = Ge[4 * NP3 + o], g5 = Ge[5 * NP3 + o];
      const T ur = sr[q], us = ss[q], ut = wt[k];
      sr[q] = g0 * ur + g1 * us + g2 * ut;
      ss[q] = g1 * ur + g3 * us + g4 * ut;
      wt[k] = g2 * ur + g4 * us + g5 * ut;
    }
    T yc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < NP; ++m) acc += D[m * NP + k] * wt[m];
      yc[k] = acc;
    }
    __syncthreads();

    // prefetch the next tile's column while the transposed contractions run
    column(next * EB + es, gnext, dnext);
    if (next < ntiles) {
#pragma unroll
      for (int k = 0; k < NP; ++k) un[k] = ((dnext >> k) & 1u) ? T(0) : P.u[gnext + k * plane];
    }

    // ---- phase 3: transposed r and s contractions, in place ----
    {
      T row[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + a * RS + m];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < NP; ++m) acc += D[m * NP + i] * row[m];
        sr[b * PS + a * RS + i] = acc;
      }
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = ss[b * PS + m * RS + a];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < NP; ++m) acc += D[m * NP + j] * row[m];
        ss[b * PS + j * RS + a] = acc;
      }
    }
    __syncthreads();

    // ---- phase 4: assemble and scatter ----
    T *yp = P.y + gbase;
    const bool ij_interior = (a > 0) && (a < N) && (b > 0) && (b < N);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = k * PS + b * RS + a;
      T yk = yc[k] + sr[q] + ss[q];
      if (P.wJa && active) yk += P.wJa[e * NP3 + t2 + NP2 * k] * uc[k];
      if ((dirbits >> k) & 1u) continue;
      if (P.partials) dotp += uc[k] * yk;
      if (k > 0 && k < N && ij_interior)
        yp[k * plane] = yk;
      else
        atomicAdd(yp + k * plane, yk);
    }
  }

  if (P.partials) {
    const double bs = block_sum<NT>((double)dotp, s_red);
    if (publish_partial<NT>(bs, P.partials, &P.scal->counter[0], s_red, s_flag)) {
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

template <int NP, typename T, int EB>
static sem_status launch_apply_pipe(const ApplyParams<T, NP> &p, cudaStream_t s) {
  using C = ApplyCfg<NP, EB>;
  constexpr size_t smem = pipe_smem<NP, T, EB>();
  static_assert(smem <= SEM_MAX_SMEM_PER_BLOCK, "pipelined apply exceeds the shared memory of a block");
  static std::atomic<unsigned long long> attr_done;
  int blocks_per_sm = 0;
  cudaError_t e = set_smem_limit_once(k_apply_pipe<NP, T, EB>, smem, attr_done);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_apply_pipe<NP, T, EB>, C::NT, smem);
  if (e != cudaSuccess || blocks_per_sm < 1)
    return sem_fail(SEM_ERR_CUDA, std::string("pipelined apply set-up: ") + cudaGetErrorString(e));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (p.E + EB - 1) / EB;
  const int64_t grid = ntiles < (int64_t)sms * blocks_per_sm ? ntiles : (int64_t)sms * blocks_per_sm;
  k_apply_pipe<NP, T, EB><<<(unsigned)grid, C::NT, smem, s>>>(p, ntiles);
  e = cudaGetLastError();
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("pipelined apply launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}
