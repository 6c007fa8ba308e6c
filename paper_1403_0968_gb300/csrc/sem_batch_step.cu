// One persistent, fused launch per inner CG step of the batched solver (the preconditioned CG of
// arXiv 1403.0968 §4.2.2 run for many problems at once, sem_batch.cu).
//
// A cooperative launch of co-resident blocks of 256 threads runs the whole step in four phases
// separated by grid-wide barriers:
//   A  the batched FP32 apply Ap = A p of every unfinished problem (the sum-factorised operator of
//      §4.2.1: gather, D-contractions, geometric factors, transposed contractions, scatter-add):
//      the blocks walk the element tiles of all order groups, a tile of order N holding
//      floor(256 / (N+1)^2) elements with one (N+1)^2 column of threads each; threads past the
//      tile's columns form one inactive element slot, so every thread takes every barrier.
//      p^T A p is accumulated per problem;
//   B  alpha_p = (r,z)_p / (p,Ap)_p, x += alpha p, r -= alpha Ap, z = r / d, per-problem (r,z) and
//      (r,r), over the chunk table;
//   C  beta_p = (r,z)_new / (r,z)_old, p = z + beta p, Ap = 0;
//   D  (one block) the per-problem scalars: iteration count, convergence, breakdown (p^T A p <= 0
//      or non-finite: the problem keeps the iterate reached so far), the number still active.
// The barriers are bounded: a block that waits longer than the batch's poll limit sets the
// batch's error flag and leaves, and so does every block that sees the flag, so a step never
// hangs; the host reports SEM_ERR_TIMEOUT.  The launch is captured in the solver's CUDA graph
// like the multi-launch step it replaces.  Orders 3, 5, 7, 9 and 11 (the orders of the batched
// workload) with stored FP32 factors are compiled in, their derivative matrices held in constant
// memory; batches with other orders, or with factors recomputed on the fly, use the per-order-group
// launches.
#include <mutex>
#include <string>

#include "sem_apply_kernel.cuh"
#include "sem_batch_step.h"
#include "sem_reduce.cuh"

namespace {

constexpr int FT = 256;  // threads per block
constexpr int UNR = 4;   // nodes per thread and pass in the vector phases
constexpr int NSLOT = 5;
constexpr int SLOT_NP[NSLOT] = {4, 6, 8, 10, 12};  // orders 3, 5, 7, 9, 11

// elements per tile, and element slots (one more when threads are left over)
__host__ __device__ constexpr int fused_eb(int NP) { return FT / (NP * NP); }
__host__ __device__ constexpr int fused_es(int NP) { return FT > fused_eb(NP) * NP * NP ? fused_eb(NP) + 1 : fused_eb(NP); }
__host__ __device__ constexpr int fused_buf(int NP) { return NP * NP * (NP | 1); }  // one element-sized buffer
__host__ __device__ constexpr size_t fused_red_off(int NP) {
  return ((size_t)fused_es(NP) * 3 * fused_buf(NP) * sizeof(float) + 15) / 16 * 16;
}
__host__ __device__ constexpr size_t fused_smem_np(int NP) { return fused_red_off(NP) + (size_t)fused_es(NP) * 8; }
__host__ __device__ constexpr size_t fused_smem() {
  size_t m = 0;
  for (int s = 0; s < NSLOT; ++s) m = fused_smem_np(SLOT_NP[s]) > m ? fused_smem_np(SLOT_NP[s]) : m;
  return m;
}

// derivative matrices (even-odd form) of the compiled orders: they depend on the order alone, so
// every batch uploads the same bytes
struct FusedTables {
  DConst<4, float> D4;
  DConst<6, float> D6;
  DConst<8, float> D8;
  DConst<10, float> D10;
  DConst<12, float> D12;
};
__constant__ FusedTables c_tab;

template <int NP>
__device__ __forceinline__ const DConst<NP, float> &tab_D() {
  if constexpr (NP == 4) return c_tab.D4;
  else if constexpr (NP == 6) return c_tab.D6;
  else if constexpr (NP == 8) return c_tab.D8;
  else if constexpr (NP == 10) return c_tab.D10;
  else return c_tab.D12;
}

// one order group of the batch
struct SlotParams {
  const BatchEntry *batch;  // its problems (device table, ascending first elements)
  const int32_t *tile_entry;  // the entry of each tile's first element
  int nbatch;
  int64_t E;   // elements of the group (0: no problem of this order)
  int64_t gs;  // stored factors: element stride of the factor arrays
};

// The apply of tile `tile` of one order group: y += A u for its elements (u, y: the batch's
// concatenated FP32 vectors), p^T A p of each element added to its problem's pAp.  Elements of
// finished problems and slots past the group's last element gather nothing and scatter nothing.
template <int NP>
__device__ __forceinline__ void fused_apply_tile(const SlotParams &S, int64_t tile, const float *u, float *y,
                                                 double *pAp, unsigned char *smem) {
  constexpr int N = NP - 1, NP2 = NP * NP, NP3 = NP2 * NP, EB = fused_eb(NP), ES = fused_es(NP);
  constexpr int RS = NP | 1, PS = NP * RS, BUF = fused_buf(NP);
  static_assert(EB >= 1 && ES * NP2 >= FT, "tile against the block");
  const DConst<NP, float> &D = tab_D<NP>();
  float *sbuf = reinterpret_cast<float *>(smem);
  double *s_el = reinterpret_cast<double *>(smem + fused_red_off(NP));  // ES per-element sums
  const int tid = threadIdx.x;
  const int es = tid / NP2, t2 = tid - es * NP2, a = t2 % NP, b = t2 / NP;
  const int64_t e = tile * EB + es;
  const bool in_tile = es < EB && e < S.E;
  float *su = sbuf + es * 3 * BUF, *sr = su + BUF, *ss = sr + BUF;

  // the problem of this element: last entry whose first element is <= e, from the entry of the
  // tile's first element (at most EB - 1 steps on); other slots take entry 0
  int lo = 0;
  if (in_tile) {
    lo = S.tile_entry[tile];
    for (int q = 0; q < EB && lo + 1 < S.nbatch && S.batch[lo + 1].elem_off <= e; ++q) ++lo;
  }
  const BatchEntry &B = S.batch[lo];
  const bool live = in_tile && !*B.done;
  if (!__syncthreads_or(live)) return;  // nothing to do in this tile
  const int64_t el = live ? e - B.elem_off : 0;

  // ---- gather u_e (structured box numbering), column (i, j) = (a, b) ----
  const int64_t plane = B.gxs * B.gys;
  int64_t gbase = 0;
  uint32_t dirbits = (1u << NP) - 1u;  // bit k: node (a, b, k) is a Dirichlet node, or no element
  if (live) {
    const int64_t ex = el % B.sx, exy = el / B.sx, ey = exy % B.sy, ez = exy / B.sy;
    const int64_t I = ex * N + a, J = ey * N + b;
    gbase = I + B.gxs * (J + B.gys * (ez * N));
    dirbits = 0;
    if (B.bc == SEM_BC_BOX) {
      if (I == 0 || I == B.gxs - 1 || J == 0 || J == B.gys - 1) dirbits = (1u << NP) - 1u;
      if (ez == 0) dirbits |= 1u;
      if (ez == B.sz - 1) dirbits |= 1u << N;
    }
  }
  const float *up = u + B.g_off + gbase;
  float uc[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    uc[k] = ((dirbits >> k) & 1u) ? 0.f : up[k * plane];
    su[k * PS + b * RS + a] = uc[k];
  }
  __syncthreads();

  // ---- gradients: u_t along the thread's column, u_r and u_s through shared memory ----
  float wt[NP];  // u_t, then w_t
  line_apply<NP, float>(D, 0, uc, wt);
  {
    float row[NP], out[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = su[b * PS + a * RS + m];  // u(m, j = a, k = b)
    line_apply<NP, float>(D, 0, row, out);
#pragma unroll
    for (int i = 0; i < NP; ++i) sr[b * PS + a * RS + i] = out[i];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = su[b * PS + m * RS + a];  // u(i = a, m, k = b)
    line_apply<NP, float>(D, 0, row, out);
#pragma unroll
    for (int j = 0; j < NP; ++j) ss[b * PS + j * RS + a] = out[j];
  }
  __syncthreads();

  // ---- geometric factors, node by node along the column ----
  {
    // stored symmetric factors G_rr, G_rs, G_rt, G_ss, G_st, G_tt of each node
    const float *Ge = static_cast<const float *>(B.Gf) + el * S.gs + t2;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = k * PS + b * RS + a;
      const int o = k * NP2;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f, g5 = 0.f;
      if (live) {
        g0 = Ge[0 * NP3 + o];
        g1 = Ge[1 * NP3 + o];
        g2 = Ge[2 * NP3 + o];
        g3 = Ge[3 * NP3 + o];
        g4 = Ge[4 * NP3 + o];
        g5 = Ge[5 * NP3 + o];
      }
      const float ur = sr[q], us = ss[q], ut = wt[k];
      sr[q] = g0 * ur + g1 * us + g2 * ut;
      ss[q] = g1 * ur + g3 * us + g4 * ut;
      wt[k] = g2 * ur + g4 * us + g5 * ut;
    }
  }
  float yc[NP];
  line_apply<NP, float>(D, 1, wt, yc);
  __syncthreads();

  // ---- transposed r and s contractions ----
  {
    float row[NP], out[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + a * RS + m];  // w_r(m, j = a, k = b)
    line_apply<NP, float>(D, 1, row, out);
#pragma unroll
    for (int i = 0; i < NP; ++i) sr[b * PS + a * RS + i] = out[i];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = ss[b * PS + m * RS + a];  // w_s(i = a, m, k = b)
    line_apply<NP, float>(D, 1, row, out);
#pragma unroll
    for (int j = 0; j < NP; ++j) ss[b * PS + j * RS + a] = out[j];
  }
  if (tid < ES) s_el[tid] = 0.0;
  __syncthreads();

  // ---- assemble the column, scatter y += Q^T y_e, p^T A p of the element ----
  const float *wJa = static_cast<const float *>(B.wJa);
  float *yp = y + B.g_off + gbase;
  const bool ij_interior = (a > 0) && (a < N) && (b > 0) && (b < N);
  float dotp = 0.f;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if ((dirbits >> k) & 1u) continue;  // Dirichlet node, or no element in this slot
    const int q = k * PS + b * RS + a;
    float yk = yc[k] + sr[q] + ss[q];
    if (wJa) yk += wJa[el * NP3 + t2 + NP2 * k] * uc[k];
    dotp += uc[k] * yk;
    if (k > 0 && k < N && ij_interior)
      yp[k * plane] = yk;  // element-interior node: owned by this element alone
    else
      atomicAdd(yp + k * plane, yk);
  }
  atomicAdd(&s_el[es], (double)dotp);
  __syncthreads();
  if (t2 == 0 && live) atomicAdd(&pAp[B.prob], s_el[es]);
}

struct FusedParams {
  SlotParams slot[NSLOT];
  int64_t tile_end[NSLOT];  // tiles of slot s: [tile_end[s-1], tile_end[s])
  int64_t nchunks;
  const int32_t *cp, *cl;
  const int64_t *cs;
  float *x32, *p32, *r32, *Ap32;
  const float *dinv;
  double *rz, *rzn, *rr, *rrn, *pAp, *tol2;
  int32_t *done, *iters, *counts;
  int nprob, max_it;
  unsigned int *bar;  // [0] arrivals, [1] generation
  int *err;
  uint32_t wait_polls;
};

// Grid-wide barrier with a bounded wait: returns false (and sets *err) if this block gave up or
// another block already did.  Every thread of the block calls it.
__device__ __forceinline__ bool grid_barrier(const FusedParams &P) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = P.bar + 1;
    volatile int *err = P.err;
    const unsigned int g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(P.bar, 1u) == gridDim.x - 1u) {
      atomicExch(P.bar, 0u);  // reset before release: no block reaches the next barrier earlier
      __threadfence();
      atomicAdd(P.bar + 1, 1u);
    } else {
      ok = 0;
      for (uint32_t t = 0; t < P.wait_polls; ++t) {
        if (*gen != g) {
          ok = 1;
          break;
        }
        if (*err) break;
        __nanosleep(256);
      }
      if (!ok) atomicOr(P.err, 1);
    }
    __threadfence();
    s_ok = ok && !*err;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(FT, 4) k_batch_step(const FusedParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double s_red[32];
  const int tid = threadIdx.x;

  // ---- A: batched apply over the tiles of every order group ----
  const int64_t total = P.tile_end[NSLOT - 1];
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    int s = 0;  // order slot of tile t (constant indices into the parameter block)
    int64_t base = 0;
#pragma unroll
    for (int q = 0; q < NSLOT - 1; ++q) {
      if (t >= P.tile_end[q]) {
        s = q + 1;
        base = P.tile_end[q];
      }
    }
    const int64_t lt = t - base;
    switch (s) {
      case 0: fused_apply_tile<4>(P.slot[0], lt, P.p32, P.Ap32, P.pAp, smem); break;
      case 1: fused_apply_tile<6>(P.slot[1], lt, P.p32, P.Ap32, P.pAp, smem); break;
      case 2: fused_apply_tile<8>(P.slot[2], lt, P.p32, P.Ap32, P.pAp, smem); break;
      case 3: fused_apply_tile<10>(P.slot[3], lt, P.p32, P.Ap32, P.pAp, smem); break;
      default: fused_apply_tile<12>(P.slot[4], lt, P.p32, P.Ap32, P.pAp, smem); break;
    }
    __syncthreads();  // the tile's shared buffers are read before the next tile writes them
  }
  if (!grid_barrier(P)) return;

  // ---- B: x += alpha p, r -= alpha Ap, z = r / d; per-problem (r,z), (r,r) ----
  for (int64_t c = blockIdx.x; c < P.nchunks; c += gridDim.x) {
    const int p = P.cp[c];
    const double q = P.pAp[p];
    if (P.done[p] || !(q > 0.0) || !isfinite(q)) continue;  // uniform over the block
    const int64_t g0 = P.cs[c];
    const int len = P.cl[c];
    const float al = (float)(P.rz[p] / q);
    float ra = 0.f, rb = 0.f;
    // UNR independent nodes per thread and pass: their loads are in flight together
    for (int i0 = tid; i0 < len; i0 += UNR * FT) {
      float xv[UNR], pv[UNR], rv[UNR], av[UNR], dv[UNR];
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        const int i = i0 + j * FT;
        const bool in = i < len;
        const int64_t g = g0 + (in ? i : 0);
        xv[j] = in ? P.x32[g] : 0.f;
        pv[j] = in ? P.p32[g] : 0.f;
        rv[j] = in ? P.r32[g] : 0.f;
        av[j] = in ? P.Ap32[g] : 0.f;
        dv[j] = in ? P.dinv[g] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        const int i = i0 + j * FT;
        if (i >= len) continue;
        const int64_t g = g0 + i;
        P.x32[g] = xv[j] + al * pv[j];
        const float r = rv[j] - al * av[j];
        P.r32[g] = r;
        const float z = r * dv[j];
        ra += r * z;
        rb += r * r;
      }
    }
    const double A = block_sum<FT>((double)ra, s_red), Bs = block_sum<FT>((double)rb, s_red);
    if (tid == 0) {
      atomicAdd(P.rzn + p, A);
      atomicAdd(P.rrn + p, Bs);
    }
  }
  if (!grid_barrier(P)) return;

  // ---- C: p = z + beta p, Ap = 0 ----
  for (int64_t c = blockIdx.x; c < P.nchunks; c += gridDim.x) {
    const int p = P.cp[c];
    const double q = P.pAp[p];
    if (P.done[p] || !(q > 0.0) || !isfinite(q)) continue;
    const int64_t g0 = P.cs[c];
    const int len = P.cl[c];
    const float be = (float)(P.rzn[p] / P.rz[p]);
    for (int i0 = tid; i0 < len; i0 += UNR * FT) {
      float rv[UNR], dv[UNR], pv[UNR];
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        const int i = i0 + j * FT;
        const bool in = i < len;
        const int64_t g = g0 + (in ? i : 0);
        rv[j] = in ? P.r32[g] : 0.f;
        dv[j] = in ? P.dinv[g] : 0.f;
        pv[j] = in ? P.p32[g] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        const int i = i0 + j * FT;
        if (i >= len) continue;
        P.p32[g0 + i] = rv[j] * dv[j] + be * pv[j];
        P.Ap32[g0 + i] = 0.0f;
      }
    }
  }
  if (!grid_barrier(P)) return;

  // ---- D: per-problem scalars (one block) ----
  if (blockIdx.x == 0) {
    __shared__ int s_active;
    if (tid == 0) s_active = 0;
    __syncthreads();
    int active = 0;
    for (int p = tid; p < P.nprob; p += FT) {
      if (P.done[p]) continue;
      const double q = P.pAp[p];
      if (!(q > 0.0) || !isfinite(q)) {
        P.done[p] = 1;  // breakdown: keep the iterate reached so far
      } else {
        P.rz[p] = P.rzn[p];
        P.rr[p] = P.rrn[p];
        P.iters[p] += 1;
        if (P.rr[p] <= P.tol2[p] || P.iters[p] >= P.max_it || !isfinite(P.rr[p])) P.done[p] = 1;
      }
      P.pAp[p] = 0.0;
      P.rzn[p] = 0.0;
      P.rrn[p] = 0.0;
      if (!P.done[p]) ++active;
    }
    atomicAdd(&s_active, active);
    __syncthreads();
    if (tid == 0) P.counts[0] = s_active;
  }
}

int slot_of(int N) {
  for (int s = 0; s < NSLOT; ++s)
    if (SLOT_NP[s] == N + 1) return s;
  return -1;
}

template <int NP>
void fill_tables(DConst<NP, float> &D) {
  double x[NP], w[NP], Dd[NP * NP];
  sem_gll_tables(NP - 1, x, w, Dd);
  // D rounded to FP32 first, as the per-order-group launches receive it
  for (int q = 0; q < NP * NP; ++q) Dd[q] = (double)(float)Dd[q];
  fill_dconst<NP, float>(D, Dd);
}

std::mutex g_tab_mutex;
unsigned long long g_tab_devices = 0;  // bit d: the tables are in device d's constant memory

sem_status launch_fused(const FusedParams &P, int64_t work, cudaStream_t st) {
  constexpr size_t smem = fused_smem();
  static_assert(smem <= 227 * 1024, "fused step kernel exceeds the shared memory of a block");
  static std::atomic<unsigned long long> attr_done;
  cudaError_t e = set_smem_limit_once(k_batch_step, smem, attr_done);
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("fused step attributes: ") + cudaGetErrorString(e));
  int dev = 0, nsm = 0, per_sm = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  SEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  SEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step, FT, smem));
  if (per_sm < 1) return sem_fail(SEM_ERR_CUDA, "fused step kernel does not fit on an SM");
  int64_t grid = (int64_t)per_sm * nsm;  // co-resident blocks (cooperative launch)
  if (work < grid) grid = work > 0 ? work : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(FT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_batch_step, P);
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("fused step launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}

}  // namespace

int sem_batch_fused_tile_elems(int N) { return slot_of(N) >= 0 ? fused_eb(N + 1) : 0; }

bool sem_batch_fused_orders_ok(const int *orders, int n) {
  for (int i = 0; i < n; ++i)
    if (slot_of(orders[i]) < 0) return false;
  return true;
}

sem_status sem_batch_fused_init() {
  int dev = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return sem_fail(SEM_ERR_INVALID, "fused step: device index above 63");
  std::lock_guard<std::mutex> lock(g_tab_mutex);
  if (g_tab_devices & (1ull << dev)) return SEM_OK;
  static FusedTables tab;  // identical bytes on every call
  fill_tables<4>(tab.D4);
  fill_tables<6>(tab.D6);
  fill_tables<8>(tab.D8);
  fill_tables<10>(tab.D10);
  fill_tables<12>(tab.D12);
  cudaError_t e = cudaMemcpyToSymbol(c_tab, &tab, sizeof(tab));
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("fused step tables: ") + cudaGetErrorString(e));
  g_tab_devices |= 1ull << dev;
  return SEM_OK;
}

sem_status sem_batch_fused_step(const FusedStepDesc &d, cudaStream_t st) {
  FusedParams P;
  memset(&P, 0, sizeof(P));
  bool have[NSLOT] = {false, false, false, false, false};
  for (int i = 0; i < d.ngroups; ++i) {
    const FusedGroupDesc &g = d.groups[i];
    const int s = slot_of(g.N);
    if (s < 0) return sem_fail(SEM_ERR_INVALID, "fused step: order outside 3, 5, 7, 9, 11");
    if (g.otf) return sem_fail(SEM_ERR_INVALID, "fused step: stored FP32 factors only");
    if (have[s]) return sem_fail(SEM_ERR_INVALID, "fused step: two groups of one order");
    have[s] = true;
    P.slot[s].batch = g.entries;
    P.slot[s].tile_entry = g.tile_entry;
    P.slot[s].nbatch = g.nbatch;
    P.slot[s].E = g.total_E;
    P.slot[s].gs = g.gs;
  }
  int64_t acc = 0;
  for (int s = 0; s < NSLOT; ++s) {
    if (have[s]) {
      const int eb = fused_eb(SLOT_NP[s]);
      acc += (P.slot[s].E + eb - 1) / eb;
    }
    P.tile_end[s] = acc;
  }
  P.nchunks = d.nchunks;
  P.cp = d.cp;
  P.cl = d.cl;
  P.cs = d.cs;
  P.x32 = d.x32;
  P.p32 = d.p32;
  P.r32 = d.r32;
  P.Ap32 = d.Ap32;
  P.dinv = d.dinv;
  P.rz = d.rz;
  P.rzn = d.rzn;
  P.rr = d.rr;
  P.rrn = d.rrn;
  P.pAp = d.pAp;
  P.tol2 = d.tol2;
  P.done = d.done;
  P.iters = d.iters;
  P.counts = d.counts;
  P.nprob = d.nprob;
  P.max_it = d.max_it;
  P.bar = d.bar;
  P.err = d.err;
  P.wait_polls = d.wait_polls;
  const int64_t work = acc > d.nchunks ? acc : d.nchunks;
  return launch_fused(P, work, st);
}
