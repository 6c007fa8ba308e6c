// Batched solves of many independent spectral-element problems (structured boxes of uneven size
// and order) — the preconditioned CG of arXiv 1403.0968 §4.2.2 run for all problems at once.
//
// Layout: one caller-owned workspace holds a set-up sub-workspace per problem (factors, diagonal,
// numbering as for sem_setup) followed by batch-level arrays: concatenated global vectors (FP32
// inner-solve vectors, FP64 residual and scratch), a chunk table that cuts the concatenated
// vectors into 8192-node pieces each inside one problem, and per-problem CG scalars.
//
// Solve (mixed precision, as SEM_SOLVE_IR): an FP64-accurate residual r_p = b_p - A_p x_p per
// problem (one double-float or FP64 apply per problem), then an FP32 Jacobi-PCG on
// A_p d_p = r_p / ||r_p|| for every unfinished problem together, x_p += ||r_p|| d_p, repeated
// until every problem reaches rtol.  One inner CG step for all problems is: one batched FP32
// apply launch per order group (elements of all its problems in one grid; per-problem p^T A p
// accumulated by one atomic per element), one scalar kernel (alpha per problem), one update
// kernel over the chunks (x, r, per-problem (r,z), (r,r)), one scalar kernel (beta, convergence)
// and one direction kernel.  Blocks of steps are captured once as a CUDA graph and replayed;
// finished problems drop out (their chunks and elements are skipped).  Per-problem sums use
// atomics, so results agree with the single-problem solver to rounding, not bitwise.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "sem_batch_step.h"
#include "sem_internal.h"
#include "sem_reduce.cuh"

namespace {

constexpr int64_t CHUNK = 8192;
constexpr int BT = 256;

struct Group {
  int N;
  std::vector<int> probs;
  BatchEntry *d_entries = nullptr;
  int64_t total_E = 0;
  int64_t gs = 0;
  int variant = 1;
  bool otf = false;  // inner apply with the factors recomputed from each element's map
  std::vector<BatchEntry> h_entries;  // host copy of the group's entries
  // entries of the problems still iterating (rebuilt when one finishes): the inner steps launch
  // over these alone
  BatchEntry *d_act = nullptr;
  int act_n = 0;
  int64_t act_E = 0;
  // fused step: the active entry of each tile's first element (tiles of fused_eb elements)
  int32_t *d_tile_entry = nullptr;
  int fused_eb = 0;  // elements per tile of the fused step kernel (0: order not compiled in)
  float D32h[SEM_MAX_NP * SEM_MAX_NP];
  double gx[SEM_MAX_NP], gw[SEM_MAX_NP];
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct sem_batch {
  int nprob = 0;
  std::vector<sem_handle *> h;
  std::vector<int64_t> g_off;  // nprob + 1 entries
  int64_t G = 0;
  std::vector<Group> groups;
  int64_t nchunks = 0;
  // batch-level device arrays
  float *r32, *p32, *Ap32, *x32, *dinv32;
  double *r64, *t64;
  int32_t *chunk_prob, *chunk_len;
  int64_t *chunk_start;
  double *rz, *rzn, *rrn, *pAp, *alpha, *beta, *tol2, *scale, *rr, *bb;
  int32_t *done, *iters, *outer_done, *counts;  // counts[0]: active inner problems, [1]: unfinished outer
  unsigned int *bar;   // grid barrier of the fused step: arrivals, generation (in the counts block)
  int *err;            // set when a bounded grid-wide wait of the fused step gave up
  uint32_t wait_polls; // polls before such a wait gives up
  uint32_t features;
  bool fused_ok = false;   // stored FP32 factors and every order compiled into the fused step kernel
  bool use_fused = true;   // inner steps as the fused step kernel when fused_ok (sem_batch_set_fused)
  // chunk table on the host, and the chunks of the problems still iterating (device)
  std::vector<int32_t> h_cp, h_cl;
  std::vector<int64_t> h_cs;
  int32_t *act_cp = nullptr, *act_cl = nullptr;
  int64_t *act_cs = nullptr;
  int64_t act_nc = 0;
  std::vector<int32_t> act_done;  // the finished flags the active tables were built from
  // host sources of the uploads of the active tables (kept until the next rebuild)
  std::vector<BatchEntry> stage_entries;
  std::vector<int32_t> stage_tiles;
  std::vector<int32_t> stage_cp, stage_cl;
  std::vector<int64_t> stage_cs;
};

namespace {

struct BatchPlan {
  std::vector<size_t> sub_off, sub_size;
  size_t r32, p32, Ap32, x32, dinv32, r64, t64, chunk_prob, chunk_len, chunk_start, scal, ints, entries, total;
  size_t act_entries, act_cp, act_cl, act_cs, act_tiles;
  int64_t G, nchunks;
  std::vector<int64_t> g_off;
};

sem_status batch_plan(const sem_desc *d, int32_t nprob, uint32_t features, BatchPlan *P) {
  if (!d || nprob < 1) return sem_fail(SEM_ERR_INVALID, "batch needs at least one problem");
  if (!(features & (SEM_FEAT_FP32 | SEM_FEAT_OTF)))
    return sem_fail(SEM_ERR_INVALID, "batched solves need SEM_FEAT_FP32 or SEM_FEAT_OTF for the inner apply");
  if (!(features & (SEM_FEAT_FP64 | SEM_FEAT_EMU)))
    return sem_fail(SEM_ERR_INVALID, "batched solves need SEM_FEAT_FP64 or SEM_FEAT_EMU for the residual");
  size_t off = 0;
  P->g_off.assign(nprob + 1, 0);
  P->nchunks = 0;
  const uint32_t sub_feat = features & (SEM_FEAT_FP64 | SEM_FEAT_EMU | SEM_FEAT_FP32 | SEM_FEAT_OTF);
  for (int p = 0; p < nprob; ++p) {
    if (d[p].glo_num != nullptr || d[p].bc == SEM_BC_MASK)
      return sem_fail(SEM_ERR_INVALID, "batched problems must be structured boxes (no glo_num, no mask)");
    size_t b = 0;
    sem_status st = sem_workspace_size(&d[p], sub_feat, &b);
    if (st != SEM_OK) return st;
    P->sub_off.push_back(off);
    P->sub_size.push_back(b);
    off = align256(off + b);
    const int64_t G = ((int64_t)d[p].box[0] * d[p].N + 1) * ((int64_t)d[p].box[1] * d[p].N + 1) *
                      ((int64_t)d[p].box[2] * d[p].N + 1);
    P->g_off[p + 1] = P->g_off[p] + G;
    P->nchunks += (G + CHUNK - 1) / CHUNK;
  }
  P->G = P->g_off[nprob];
  const size_t G = (size_t)P->G;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  P->r32 = take(G * 4);
  P->p32 = take(G * 4);
  P->Ap32 = take(G * 4);
  P->x32 = take(G * 4);
  P->dinv32 = take(G * 4);
  P->r64 = take(G * 8);
  P->t64 = take(G * 8);
  P->chunk_prob = take((size_t)P->nchunks * 4);
  P->chunk_len = take((size_t)P->nchunks * 4);
  P->chunk_start = take((size_t)P->nchunks * 8);
  P->scal = take((size_t)nprob * 8 * 10);
  P->ints = take((size_t)nprob * 4 * 3 + 64);
  P->entries = take((size_t)nprob * sizeof(BatchEntry));
  P->act_entries = take((size_t)nprob * sizeof(BatchEntry));
  int64_t elems = 0;
  for (int p = 0; p < nprob; ++p) elems += d[p].nelem;
  P->act_tiles = take((size_t)elems * 4);  // at most one tile per element
  P->act_cp = take((size_t)P->nchunks * 4);
  P->act_cl = take((size_t)P->nchunks * 4);
  P->act_cs = take((size_t)P->nchunks * 8);
  P->total = off;
  return SEM_OK;
}

template <typename X>
X *at(void *base, size_t off) {
  return reinterpret_cast<X *>(static_cast<char *>(base) + off);
}

// ---------------------------------------------------------------------------------------------
// batch kernels: one block per chunk (grid-stride over chunks), per-problem sums by atomics
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void chunk_atomic2(double a, double b, double *pa, double *pb, double *s_red) {
  const double A = block_sum<BT>(a, s_red), B = block_sum<BT>(b, s_red);
  if (threadIdx.x == 0) {
    atomicAdd(pa, A);
    atomicAdd(pb, B);
  }
}

// copy each problem's FP32 inverse diagonal into the concatenated vector
__global__ void k_b_gather_dinv(int64_t n, const float *src, float *dst) {
  for (int64_t g = (int64_t)blockIdx.x * BT + threadIdx.x; g < n; g += (int64_t)gridDim.x * BT) dst[g] = src[g];
}

// r64 = M (b - Ax) ; rr_p += |r|^2 ; bb_p += |b|^2 for the problems not yet converged
__global__ void __launch_bounds__(BT) k_b_residual(int64_t nchunks, const int32_t *cp, const int64_t *cs,
                                                   const int32_t *cl, const double *b, const double *Ax,
                                                   const float *dinv, double *r64, double *rr, double *bb,
                                                   const int32_t *outer_done) {
  __shared__ double s_red[32];
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = cp[c];
    if (outer_done[p]) continue;  // uniform over the block
    const int64_t g0 = cs[c];
    double a = 0.0, bs = 0.0;
    for (int i = threadIdx.x; i < cl[c]; i += BT) {
      const int64_t g = g0 + i;
      const bool fr = dinv[g] != 0.0f;
      const double bg = fr ? b[g] : 0.0;
      const double rg = fr ? bg - Ax[g] : 0.0;
      r64[g] = rg;
      a += rg * rg;
      bs += bg * bg;
    }
    chunk_atomic2(a, bs, rr + p, bb + p, s_red);
  }
}

// per problem not yet converged: relative residual, outer convergence, scale = ||r||
__global__ void k_b_outer_check(int nprob, const double *rr, const double *bb, double rtol, double *scale,
                                double *relres, int32_t *outer_done, int32_t *done, int32_t *counts) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nprob; p += gridDim.x * blockDim.x) {
    if (outer_done[p]) {  // converged in an earlier round: stays out of the inner solves
      done[p] = 1;
      continue;
    }
    const double rel = bb[p] > 0.0 ? sqrt(rr[p] / bb[p]) : 0.0;
    relres[p] = rel;
    scale[p] = sqrt(rr[p]);
    const int fin = (rel <= rtol) || rr[p] == 0.0 || !isfinite(rel);
    outer_done[p] = fin;
    done[p] = fin;
    if (!fin) atomicAdd(&counts[1], 1);
  }
}

// inner start: r32 = r64 / scale, z = r / d, p = z, x = 0, Ap = 0 ; rz_p, rr_p
__global__ void __launch_bounds__(BT) k_b_inner_init(int64_t nchunks, const int32_t *cp, const int64_t *cs,
                                                     const int32_t *cl, const double *r64, const double *scale,
                                                     const float *dinv, float *r32, float *p32, float *x32,
                                                     float *Ap32, const int32_t *done, double *rz, double *rr) {
  __shared__ double s_red[32];
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = cp[c];
    const int64_t g0 = cs[c];
    const bool skip = done[p] != 0;
    const double inv = skip ? 0.0 : 1.0 / scale[p];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < cl[c]; i += BT) {
      const int64_t g = g0 + i;
      const float r = (float)(r64[g] * inv);
      const float z = r * dinv[g];
      r32[g] = r;
      p32[g] = z;
      x32[g] = 0.0f;
      Ap32[g] = 0.0f;
      a += (double)r * (double)z;
      b += (double)r * (double)r;
    }
    chunk_atomic2(a, b, rz + p, rr + p, s_red);
  }
}

__global__ void k_b_inner_tol(int nprob, const double *rr, double inner2, double *tol2, int32_t *done,
                              int32_t *iters, double *pAp, double *rzn, double *rrn, int32_t *counts) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nprob; p += gridDim.x * blockDim.x) {
    tol2[p] = inner2 * rr[p];
    if (rr[p] == 0.0 || !isfinite(rr[p])) done[p] = 1;
    iters[p] = 0;
    pAp[p] = 0.0;
    rzn[p] = 0.0;
    rrn[p] = 0.0;
    if (!done[p]) atomicAdd(&counts[0], 1);
  }
}

__global__ void k_b_alpha(int nprob, const double *rz, double *pAp, double *alpha, int32_t *done) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nprob; p += gridDim.x * blockDim.x) {
    if (done[p]) continue;
    const double q = pAp[p];
    if (!(q > 0.0) || !isfinite(q)) {
      done[p] = 1;  // breakdown: keep the iterate reached so far
      alpha[p] = 0.0;
    } else {
      alpha[p] = rz[p] / q;
    }
    pAp[p] = 0.0;
  }
}

__global__ void __launch_bounds__(BT) k_b_update(int64_t nchunks, const int32_t *cp, const int64_t *cs,
                                                 const int32_t *cl, float *x32, const float *p32, float *r32,
                                                 const float *Ap32, const float *dinv, const double *alpha,
                                                 const int32_t *done, double *rzn, double *rrn) {
  __shared__ double s_red[32];
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = cp[c];
    if (done[p]) continue;  // uniform over the block
    const int64_t g0 = cs[c];
    const float al = (float)alpha[p];
    float a = 0.f, b = 0.f;  // at most 32 entries per thread and chunk
    for (int i = threadIdx.x; i < cl[c]; i += BT) {
      const int64_t g = g0 + i;
      x32[g] += al * p32[g];
      const float r = r32[g] - al * Ap32[g];
      r32[g] = r;
      const float z = r * dinv[g];
      a += r * z;
      b += r * r;
    }
    chunk_atomic2((double)a, (double)b, rzn + p, rrn + p, s_red);
  }
}

__global__ void k_b_beta(int nprob, double *rz, double *rzn, double *rr, double *rrn, double *beta, const double *tol2,
                         int32_t *done, int32_t *iters, int max_it, int32_t *counts) {
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  int active = 0;
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    if (done[p]) continue;
    beta[p] = rzn[p] / rz[p];
    rz[p] = rzn[p];
    rr[p] = rrn[p];
    rzn[p] = 0.0;
    rrn[p] = 0.0;
    iters[p] += 1;
    if (rr[p] <= tol2[p] || iters[p] >= max_it || !isfinite(rr[p])) done[p] = 1;
    if (!done[p]) ++active;
  }
  atomicAdd(&s_active, active);
  __syncthreads();
  if (threadIdx.x == 0) counts[0] = s_active;
}

__global__ void __launch_bounds__(BT) k_b_direction(int64_t nchunks, const int32_t *cp, const int64_t *cs,
                                                    const int32_t *cl, float *p32, const float *r32, float *Ap32,
                                                    const float *dinv, const double *beta, const int32_t *done) {
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = cp[c];
    if (done[p]) continue;
    const int64_t g0 = cs[c];
    const float be = (float)beta[p];
    for (int i = threadIdx.x; i < cl[c]; i += BT) {
      const int64_t g = g0 + i;
      p32[g] = r32[g] * dinv[g] + be * p32[g];
      Ap32[g] = 0.0f;
    }
  }
}

__global__ void __launch_bounds__(BT) k_b_correct(int64_t nchunks, const int32_t *cp, const int64_t *cs,
                                                  const int32_t *cl, double *x, const float *x32,
                                                  const double *scale, const int32_t *outer_done) {
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = cp[c];
    if (outer_done[p]) continue;
    const int64_t g0 = cs[c];
    const double sc = scale[p];
    for (int i = threadIdx.x; i < cl[c]; i += BT) x[g0 + i] += sc * (double)x32[g0 + i];
  }
}

unsigned cgrid(int64_t nchunks) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(nchunks, 152 * 8)); }

// FP32 apply of every problem (all: the full entry tables) or of the problems still iterating
// (the active tables, with p^T A p per problem)
sem_status batch_apply32(sem_batch *B, const float *u, float *y, bool inner, cudaStream_t st) {
  for (auto &g : B->groups) {
    double *pAp = inner ? B->pAp : nullptr;
    const BatchEntry *tab = inner ? g.d_act : g.d_entries;
    const int np = inner ? g.act_n : (int)g.probs.size();
    const int64_t E = inner ? g.act_E : g.total_E;
    if (np == 0) continue;
    sem_status s = g.otf ? dispatch_apply_batch<float, OtfGeo>(g.N, tab, np, E, g.gs, u, y, g.D32h, g.gx, g.gw, pAp,
                                                               g.variant, st)
                         : dispatch_apply_batch<float, float>(g.N, tab, np, E, g.gs, u, y, g.D32h, g.gx, g.gw, pAp,
                                                              g.variant, st);
    if (s != SEM_OK) return s;
  }
  return SEM_OK;
}

// Rebuilds the entry tables and the chunk list of the problems still iterating when the set of
// finished problems (done, host copy) has changed since the last rebuild; *changed tells the
// caller to capture its step graph again (grid sizes follow the active tables).
sem_status update_active(sem_batch *B, const std::vector<int32_t> &done, cudaStream_t st, bool *changed) {
  *changed = false;
  if (done == B->act_done) return SEM_OK;
  *changed = true;
  B->act_done = done;
  B->stage_entries.clear();
  B->stage_tiles.clear();
  for (auto &g : B->groups) {
    const size_t first = B->stage_entries.size();
    int64_t E = 0;
    for (const BatchEntry &e : g.h_entries) {
      if (done[e.prob]) continue;
      BatchEntry a = e;
      a.elem_off = E;
      E += e.E;
      B->stage_entries.push_back(a);
    }
    g.act_n = (int)(B->stage_entries.size() - first);
    g.act_E = E;
    if (B->fused_ok && g.fused_eb > 0 && g.act_n > 0) {
      // first active entry of every tile (entries in ascending first-element order)
      const size_t t0 = B->stage_tiles.size();
      int lo = 0;
      for (int64_t e = 0; e < E; e += g.fused_eb) {
        while (lo + 1 < g.act_n && B->stage_entries[first + lo + 1].elem_off <= e) ++lo;
        B->stage_tiles.push_back(lo);
      }
      SEM_CUDA_TRY(cudaMemcpyAsync(g.d_tile_entry, B->stage_tiles.data() + t0,
                                   (B->stage_tiles.size() - t0) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    if (g.act_n > 0)
      SEM_CUDA_TRY(cudaMemcpyAsync(g.d_act, B->stage_entries.data() + first, g.act_n * sizeof(BatchEntry),
                                   cudaMemcpyHostToDevice, st));
  }
  B->stage_cp.clear();
  B->stage_cl.clear();
  B->stage_cs.clear();
  for (size_t c = 0; c < B->h_cp.size(); ++c) {
    if (done[B->h_cp[c]]) continue;
    B->stage_cp.push_back(B->h_cp[c]);
    B->stage_cl.push_back(B->h_cl[c]);
    B->stage_cs.push_back(B->h_cs[c]);
  }
  B->act_nc = (int64_t)B->stage_cp.size();
  if (B->act_nc > 0) {
    SEM_CUDA_TRY(cudaMemcpyAsync(B->act_cp, B->stage_cp.data(), B->act_nc * 4, cudaMemcpyHostToDevice, st));
    SEM_CUDA_TRY(cudaMemcpyAsync(B->act_cl, B->stage_cl.data(), B->act_nc * 4, cudaMemcpyHostToDevice, st));
    SEM_CUDA_TRY(cudaMemcpyAsync(B->act_cs, B->stage_cs.data(), B->act_nc * 8, cudaMemcpyHostToDevice, st));
  }
  return SEM_OK;
}

// one persistent cooperative launch per step (sem_batch_step.cu), over the active tables
sem_status fused_steps(sem_batch *B, int count, int max_it, cudaStream_t st) {
  std::vector<FusedGroupDesc> groups;
  for (const Group &g : B->groups) {
    if (g.act_n == 0) continue;
    FusedGroupDesc fg;
    fg.N = g.N;
    fg.otf = g.otf;
    fg.entries = g.d_act;
    fg.nbatch = g.act_n;
    fg.total_E = g.act_E;
    fg.gs = g.gs;
    fg.tile_entry = g.d_tile_entry;
    groups.push_back(fg);
  }
  FusedStepDesc d;
  d.groups = groups.data();
  d.ngroups = (int)groups.size();
  d.otf = false;
  d.nchunks = B->act_nc;
  d.cp = B->act_cp;
  d.cl = B->act_cl;
  d.cs = B->act_cs;
  d.x32 = B->x32;
  d.p32 = B->p32;
  d.r32 = B->r32;
  d.Ap32 = B->Ap32;
  d.dinv = B->dinv32;
  d.rz = B->rz;
  d.rzn = B->rzn;
  d.rr = B->rr;
  d.rrn = B->rrn;
  d.pAp = B->pAp;
  d.tol2 = B->tol2;
  d.done = B->done;
  d.iters = B->iters;
  d.counts = B->counts;
  d.nprob = B->nprob;
  d.max_it = max_it;
  d.bar = B->bar;
  d.err = B->err;
  d.wait_polls = B->wait_polls;
  for (int it = 0; it < count; ++it) {
    sem_status s = sem_batch_fused_step(d, st);
    if (s != SEM_OK) return s;
  }
  return SEM_OK;
}

sem_status inner_steps(sem_batch *B, int count, int max_it, bool fused, cudaStream_t st) {
  if (fused) return fused_steps(B, count, max_it, st);
  const int64_t nc = B->act_nc;
  const int np = B->nprob;
  const unsigned pg = (unsigned)((np + 255) / 256);
  for (int it = 0; it < count; ++it) {
    sem_status s = batch_apply32(B, B->p32, B->Ap32, true, st);
    if (s != SEM_OK) return s;
    k_b_alpha<<<pg, 256, 0, st>>>(np, B->rz, B->pAp, B->alpha, B->done);
    k_b_update<<<cgrid(nc), BT, 0, st>>>(nc, B->act_cp, B->act_cs, B->act_cl, B->x32, B->p32, B->r32, B->Ap32,
                                         B->dinv32, B->alpha, B->done, B->rzn, B->rrn);
    k_b_beta<<<1, 1024, 0, st>>>(np, B->rz, B->rzn, B->rr, B->rrn, B->beta, B->tol2, B->done, B->iters, max_it,
                                 B->counts);
    k_b_direction<<<cgrid(nc), BT, 0, st>>>(nc, B->act_cp, B->act_cs, B->act_cl, B->p32, B->r32, B->Ap32,
                                            B->dinv32, B->beta, B->done);
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------------------------
extern "C" sem_status sem_batch_workspace_size(const sem_desc *descs, int32_t nprob, uint32_t features,
                                               size_t *bytes) {
  if (!bytes) return sem_fail(SEM_ERR_INVALID, "bytes is NULL");
  BatchPlan P;
  sem_status s = batch_plan(descs, nprob, features, &P);
  if (s != SEM_OK) return s;
  *bytes = P.total;
  return SEM_OK;
}

extern "C" void sem_batch_free(sem_batch *B) {
  if (!B) return;
  for (auto *h : B->h) sem_free(h);
  delete B;
}

extern "C" sem_status sem_batch_setup(const sem_desc *descs, int32_t nprob, uint32_t features, void *ws,
                                      size_t bytes, sem_stream_t stream_, sem_batch **out) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream_);
  if (!out) return sem_fail(SEM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  BatchPlan P;
  sem_status s = batch_plan(descs, nprob, features, &P);
  if (s != SEM_OK) return s;
  if (!ws || bytes < P.total) return sem_fail(SEM_ERR_WORKSPACE, "batch workspace needs " + std::to_string(P.total) + " bytes");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return sem_fail(SEM_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  sem_batch *B = new sem_batch();
  B->nprob = nprob;
  B->features = features;
  B->g_off = P.g_off;
  B->G = P.G;
  B->nchunks = P.nchunks;
  const uint32_t sub_feat = features & (SEM_FEAT_FP64 | SEM_FEAT_EMU | SEM_FEAT_FP32 | SEM_FEAT_OTF);
  const bool otf = !(features & SEM_FEAT_FP32);  // stored FP32 factors when present, else on the fly
  for (int p = 0; p < nprob; ++p) {
    sem_handle *h = nullptr;
    s = sem_setup(&descs[p], sub_feat, at<char>(ws, P.sub_off[p]), P.sub_size[p], stream_, &h);
    if (s != SEM_OK) {
      sem_batch_free(B);
      return s;
    }
    B->h.push_back(h);
  }
  B->r32 = at<float>(ws, P.r32);
  B->p32 = at<float>(ws, P.p32);
  B->Ap32 = at<float>(ws, P.Ap32);
  B->x32 = at<float>(ws, P.x32);
  B->dinv32 = at<float>(ws, P.dinv32);
  B->r64 = at<double>(ws, P.r64);
  B->t64 = at<double>(ws, P.t64);
  B->chunk_prob = at<int32_t>(ws, P.chunk_prob);
  B->chunk_len = at<int32_t>(ws, P.chunk_len);
  B->chunk_start = at<int64_t>(ws, P.chunk_start);
  double *sc = at<double>(ws, P.scal);
  B->rz = sc;
  B->rzn = sc + nprob;
  B->rrn = sc + 2 * nprob;
  B->pAp = sc + 3 * nprob;
  B->alpha = sc + 4 * nprob;
  B->beta = sc + 5 * nprob;
  B->tol2 = sc + 6 * nprob;
  B->scale = sc + 7 * nprob;
  B->rr = sc + 8 * nprob;
  B->bb = sc + 9 * nprob;
  int32_t *iv = at<int32_t>(ws, P.ints);
  B->done = iv;
  B->iters = iv + nprob;
  B->outer_done = iv + 2 * nprob;
  B->counts = iv + 3 * nprob;
  B->bar = reinterpret_cast<unsigned int *>(B->counts + 8);
  B->err = B->counts + 10;
  B->wait_polls = SEM_WAIT_POLLS_DEFAULT;
  auto fail = [&](const std::string &m) {
    sem_batch_free(B);
    return sem_fail(SEM_ERR_CUDA, m);
  };
  // chunk table
  std::vector<int32_t> cp, cl;
  std::vector<int64_t> cs;
  for (int p = 0; p < nprob; ++p)
    for (int64_t g = P.g_off[p]; g < P.g_off[p + 1]; g += CHUNK) {
      cp.push_back(p);
      cs.push_back(g);
      cl.push_back((int32_t)std::min<int64_t>(CHUNK, P.g_off[p + 1] - g));
    }
  if (cudaMemcpyAsync(B->chunk_prob, cp.data(), cp.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(B->chunk_len, cl.data(), cl.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(B->chunk_start, cs.data(), cs.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail("chunk table copy");
  B->h_cp = cp;
  B->h_cl = cl;
  B->h_cs = cs;
  B->act_cp = at<int32_t>(ws, P.act_cp);
  B->act_cl = at<int32_t>(ws, P.act_cl);
  B->act_cs = at<int64_t>(ws, P.act_cs);
  // concatenated FP32 inverse diagonal
  for (int p = 0; p < nprob; ++p) {
    const int64_t n = P.g_off[p + 1] - P.g_off[p];
    k_b_gather_dinv<<<cgrid((n + BT - 1) / BT), BT, 0, st>>>(n, B->h[p]->dinv32, B->dinv32 + P.g_off[p]);
  }
  // order groups and their device entry tables
  std::map<int, std::vector<int>> byN;
  for (int p = 0; p < nprob; ++p) byN[descs[p].N].push_back(p);
  std::vector<BatchEntry> entries(nprob);
  int slot = 0;
  int64_t tile_slot = 0;  // tiles of the groups before this one (at most one per element)
  for (auto &kv : byN) {
    Group g;
    g.N = kv.first;
    g.probs = kv.second;
    g.d_entries = at<BatchEntry>(ws, P.entries) + slot;
    g.d_act = at<BatchEntry>(ws, P.act_entries) + slot;
    g.d_tile_entry = at<int32_t>(ws, P.act_tiles) + tile_slot;
    g.fused_eb = sem_batch_fused_tile_elems(g.N);
    int64_t eoff = 0;
    for (int p : g.probs) {
      const sem_handle *h = B->h[p];
      BatchEntry &E = entries[slot++];
      E.elem_off = eoff;
      E.E = h->E;
      E.sx = h->box[0];
      E.sy = h->box[1];
      E.sz = h->box[2];
      E.bc = h->bc;
      E.gxs = (int64_t)h->box[0] * h->N + 1;
      E.gys = (int64_t)h->box[1] * h->N + 1;
      E.gzs = (int64_t)h->box[2] * h->N + 1;
      E.g_off = P.g_off[p];
      E.prob = p;
      E.pad = 0;
      E.Gf = otf ? static_cast<const void *>(h->Gotf) : static_cast<const void *>(h->G32);
      E.wJa = h->wJa32;
      E.kap = otf ? h->kap32 : nullptr;
      E.done = B->done + p;
      g.h_entries.push_back(E);
      eoff += h->E;
      g.gs = otf ? SEM_OTF_STRIDE : h->gs6;
    }
    g.total_E = eoff;
    tile_slot += eoff;
    g.otf = otf;
    const int n = g.N + 1;
    for (int q = 0; q < n * n; ++q) g.D32h[q] = B->h[g.probs[0]]->D32h[q];
    for (int q = 0; q < n; ++q) {
      g.gx[q] = B->h[g.probs[0]]->gxh[q];
      g.gw[q] = B->h[g.probs[0]]->gwh[q];
    }
    B->groups.push_back(g);
  }
  {
    std::vector<int> orders;
    for (size_t i = 0; i < B->groups.size(); ++i) orders.push_back(B->groups[i].N);
    // the fused step reads stored FP32 factors (on-the-fly batches use the per-group launches)
    B->fused_ok = !otf && sem_batch_fused_orders_ok(orders.data(), (int)orders.size());
    if (B->fused_ok) {
      const sem_status fs = sem_batch_fused_init();
      if (fs != SEM_OK) {
        sem_batch_free(B);
        return fs;
      }
    }
  }
  if (cudaMemcpyAsync(at<BatchEntry>(ws, P.entries), entries.data(), entries.size() * sizeof(BatchEntry),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail("entry table copy");
  if (cudaMemsetAsync(B->done, 0, (size_t)nprob * 4 * 3 + 64, st) != cudaSuccess) return fail("memset");
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail("batch set-up");
  *out = B;
  return SEM_OK;
}

extern "C" sem_status sem_batch_info(const sem_batch *B, int32_t p, sem_info *info, int64_t *g_offset) {
  if (!B || p < 0 || p >= B->nprob) return sem_fail(SEM_ERR_INVALID, "bad batch or problem index");
  sem_status s = sem_get_info(B->h[p], info);
  if (s == SEM_OK && g_offset) *g_offset = B->g_off[p];
  return s;
}

extern "C" sem_status sem_batch_handle(sem_batch *B, int32_t p, sem_handle **out) {
  if (!B || !out || p < 0 || p >= B->nprob) return sem_fail(SEM_ERR_INVALID, "bad batch or problem index");
  *out = B->h[p];
  return SEM_OK;
}

extern "C" sem_status sem_batch_set_fused(sem_batch *B, int32_t fused) {
  if (!B) return sem_fail(SEM_ERR_INVALID, "NULL batch");
  if (fused && !B->fused_ok)
    return sem_fail(SEM_ERR_INVALID, "fused step needs stored FP32 factors and orders 3, 5, 7, 9, 11 only");
  B->use_fused = fused != 0;
  return SEM_OK;
}

extern "C" sem_status sem_batch_get_fused(const sem_batch *B, int32_t *available, int32_t *in_use) {
  if (!B) return sem_fail(SEM_ERR_INVALID, "NULL batch");
  if (available) *available = B->fused_ok ? 1 : 0;
  if (in_use) *in_use = (B->fused_ok && B->use_fused) ? 1 : 0;
  return SEM_OK;
}

extern "C" sem_status sem_batch_set_wait_limit(sem_batch *B, int64_t polls) {
  if (!B) return sem_fail(SEM_ERR_INVALID, "NULL batch");
  if (polls > 0xffffffffll) return sem_fail(SEM_ERR_INVALID, "wait limit above 2^32 - 1 polls");
  B->wait_polls = polls < 0 ? SEM_WAIT_POLLS_DEFAULT : (uint32_t)polls;
  return SEM_OK;
}

extern "C" sem_status sem_batch_set_variant(sem_batch *B, int32_t N, int32_t variant) {
  if (!B || (variant != 1 && variant != 2)) return sem_fail(SEM_ERR_INVALID, "batched apply variant must be 1 or 2");
  bool found = false;
  for (auto &g : B->groups)
    if (g.N == N) {
      g.variant = variant;
      found = true;
    }
  return found ? SEM_OK : sem_fail(SEM_ERR_INVALID, "no problem of that order in the batch");
}

extern "C" sem_status sem_batch_apply(sem_batch *B, sem_prec prec, const void *d_u, void *d_y, sem_stream_t stream) {
  if (!B || !d_u || !d_y || d_u == d_y) return sem_fail(SEM_ERR_INVALID, "bad arguments");
  if (prec != SEM_FP64 && prec != SEM_FP64_EMU && prec != SEM_FP32)
    return sem_fail(SEM_ERR_INVALID, "batched applies run in SEM_FP64, SEM_FP64_EMU or SEM_FP32");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t es = prec == SEM_FP32 ? 4 : 8;
  SEM_CUDA_TRY(cudaMemsetAsync(d_y, 0, (size_t)B->G * es, st));
  if (prec == SEM_FP32) return batch_apply32(B, static_cast<const float *>(d_u), static_cast<float *>(d_y), false, st);
  for (int p = 0; p < B->nprob; ++p) {
    sem_status s = sem_launch_apply(B->h[p], prec, static_cast<const double *>(d_u) + B->g_off[p],
                                    static_cast<double *>(d_y) + B->g_off[p], nullptr, nullptr, nullptr, st);
    if (s != SEM_OK) return s;
  }
  return SEM_OK;
}

extern "C" sem_status sem_batch_pcg(sem_batch *B, const double *d_b, double *d_x, const sem_pcg_opts *o,
                                    sem_pcg_result *res, sem_stream_t stream) {
  NvtxRange nvtx_solve("sem_batch_pcg");
  if (!B || !d_b || !d_x || !o || !res) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int np = B->nprob;
  const int prec64 = o->apply_prec;
  if (prec64 != SEM_FP64 && prec64 != SEM_FP64_EMU) return sem_fail(SEM_ERR_INVALID, "apply_prec must be FP64 or EMU");
  for (int p = 0; p < np; ++p) {
    if ((prec64 == SEM_FP64 && !B->h[p]->G64) || (prec64 == SEM_FP64_EMU && !B->h[p]->Gemu))
      return sem_fail(SEM_ERR_INVALID, "batch lacks the factor set of apply_prec");
    memset(&res[p], 0, sizeof(sem_pcg_result));
  }
  const double inner = o->inner_rtol > 0 ? o->inner_rtol : 1e-4;
  const int every = std::max(1, o->check_every);
  const int64_t nc = B->nchunks;
  const unsigned pg = (unsigned)((np + 255) / 256);
  std::vector<double> relres(np, 0.0);
  std::vector<int32_t> iters(np, 0), total(np, 0);
  double *d_relres = B->tol2;  // reused between phases as scratch for the outer check
  cudaGraphExec_t exec = nullptr;
  const bool graph = o->use_graph && st != nullptr;
  // one fused launch per step unless the caller asks for the per-order-group launches (or an
  // order is not compiled into the fused step kernel)
  const bool fused = B->fused_ok && B->use_fused && !(o->flags & SEM_PCG_MULTI_LAUNCH);
  sem_status s = SEM_OK;
  int outer = 0;
  int32_t counts[2] = {0, 0};
  std::vector<int32_t> odone(np, 0);  // problems whose FP64-accurate residual met rtol (host copy)
  SEM_CUDA_TRY(cudaMemsetAsync(B->outer_done, 0, (size_t)np * 4, st));
  std::vector<int32_t> prev_done(np, 0);
  std::vector<int32_t> done_h(np, 0);  // inner-finished flags (host copy, read at every check)
  B->act_done.clear();                 // the active tables are rebuilt at the first check
  for (; outer < 100; ++outer) {
    prev_done = odone;
    // FP64-accurate residual of every problem not yet converged (converged ones keep their x)
    SEM_CUDA_TRY(cudaMemsetAsync(B->t64, 0, (size_t)B->G * 8, st));
    for (int p = 0; p < np; ++p) {
      if (odone[p]) continue;
      s = sem_launch_apply(B->h[p], (sem_prec)prec64, d_x + B->g_off[p], B->t64 + B->g_off[p], nullptr, nullptr,
                           nullptr, st);
      if (s != SEM_OK) break;
    }
    if (s != SEM_OK) break;
    SEM_CUDA_TRY(cudaMemsetAsync(B->rr, 0, (size_t)np * 8, st));
    SEM_CUDA_TRY(cudaMemsetAsync(B->bb, 0, (size_t)np * 8, st));
    SEM_CUDA_TRY(cudaMemsetAsync(B->counts, 0, 64, st));
    k_b_residual<<<cgrid(nc), BT, 0, st>>>(nc, B->chunk_prob, B->chunk_start, B->chunk_len, d_b, B->t64, B->dinv32,
                                           B->r64, B->rr, B->bb, B->outer_done);
    k_b_outer_check<<<pg, 256, 0, st>>>(np, B->rr, B->bb, o->rtol, B->scale, d_relres, B->outer_done, B->done,
                                        B->counts);
    SEM_CUDA_TRY(cudaMemcpyAsync(relres.data(), d_relres, (size_t)np * 8, cudaMemcpyDeviceToHost, st));
    SEM_CUDA_TRY(cudaMemcpyAsync(odone.data(), B->outer_done, (size_t)np * 4, cudaMemcpyDeviceToHost, st));
    SEM_CUDA_TRY(cudaMemcpyAsync(counts, B->counts, 8, cudaMemcpyDeviceToHost, st));
    SEM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int p = 0; p < np; ++p)
      if (!prev_done[p]) res[p].true_relres = relres[p];  // checked in this refinement step
    if (counts[1] == 0) break;
    int maxt = 0;
    for (int p = 0; p < np; ++p) maxt = std::max(maxt, total[p]);
    if (maxt >= o->max_it) {
      s = sem_fail(SEM_ERR_NOCONV, "batched solve: inner iteration budget exhausted");
      break;
    }
    // batched FP32 inner solve of every unfinished problem
    SEM_CUDA_TRY(cudaMemsetAsync(B->rz, 0, (size_t)np * 8, st));
    SEM_CUDA_TRY(cudaMemsetAsync(B->rr, 0, (size_t)np * 8, st));
    k_b_inner_init<<<cgrid(nc), BT, 0, st>>>(nc, B->chunk_prob, B->chunk_start, B->chunk_len, B->r64, B->scale,
                                             B->dinv32, B->r32, B->p32, B->x32, B->Ap32, B->done, B->rz, B->rr);
    k_b_inner_tol<<<pg, 256, 0, st>>>(np, B->rr, inner * inner, B->tol2, B->done, B->iters, B->pAp, B->rzn, B->rrn,
                                      B->counts);
    const int budget = o->max_it - maxt;
    int done_steps = 0;
    while (true) {
      int32_t head[11];  // counts[0] (active problems) .. the fused step's error flag at [10]
      SEM_CUDA_TRY(cudaMemcpyAsync(head, B->counts, sizeof(head), cudaMemcpyDeviceToHost, st));
      SEM_CUDA_TRY(cudaMemcpyAsync(done_h.data(), B->done, (size_t)np * 4, cudaMemcpyDeviceToHost, st));
      SEM_CUDA_TRY(cudaStreamSynchronize(st));
      counts[0] = head[0];
      if (head[10]) {  // a bounded grid-wide wait gave up: clear the flag and the barrier, report
        SEM_CUDA_TRY(cudaMemsetAsync(B->counts + 8, 0, 3 * sizeof(int32_t), st));
        SEM_CUDA_TRY(cudaStreamSynchronize(st));
        s = sem_fail(SEM_ERR_TIMEOUT, "batched solve: a grid-wide wait of the fused step gave up");
        break;
      }
      if (counts[0] == 0 || done_steps >= budget) break;
      // launch over the problems still iterating only; a new active set needs a new graph
      bool changed = false;
      s = update_active(B, done_h, st, &changed);
      if (s != SEM_OK) break;
      if (changed && exec) {
        SEM_CUDA_TRY(cudaGraphExecDestroy(exec));
        exec = nullptr;
      }
      if (graph) {
        if (!exec) {
          cudaGraph_t g;
          SEM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
          sem_status cs = inner_steps(B, every, o->max_it, fused, st);
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
        SEM_CUDA_TRY(cudaGraphLaunch(exec, st));
      } else {
        s = inner_steps(B, every, o->max_it, fused, st);
        if (s != SEM_OK) break;
      }
      done_steps += every;
    }
    if (s != SEM_OK) break;
    SEM_CUDA_TRY(cudaMemcpyAsync(iters.data(), B->iters, (size_t)np * 4, cudaMemcpyDeviceToHost, st));
    k_b_correct<<<cgrid(nc), BT, 0, st>>>(nc, B->chunk_prob, B->chunk_start, B->chunk_len, d_x, B->x32, B->scale,
                                          B->outer_done);
    SEM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int p = 0; p < np; ++p) {
      if (odone[p]) continue;  // converged before this refinement step's inner solve
      total[p] += iters[p];
      res[p].outer = outer + 1;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  sem_status worst = s;
  for (int p = 0; p < np; ++p) {
    res[p].iterations = total[p];
    res[p].recursive_relres = res[p].true_relres;
    res[p].status = s != SEM_OK ? s : (res[p].true_relres <= o->rtol ? SEM_OK : SEM_ERR_NOCONV);
    if (worst == SEM_OK && res[p].status != SEM_OK) worst = (sem_status)res[p].status;
  }
  if (worst == SEM_ERR_NOCONV && s == SEM_OK) sem_fail(SEM_ERR_NOCONV, "some batched problems did not reach rtol");
  return worst;
}

extern "C" sem_status sem_batch_rhs(sem_batch *B, const double *d_fL, double *d_b, sem_stream_t stream) {
  if (!B || !d_fL || !d_b) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  int64_t loff = 0;
  for (int p = 0; p < B->nprob; ++p) {
    sem_status s = sem_rhs(B->h[p], d_fL + loff, d_b + B->g_off[p], stream);
    if (s != SEM_OK) return s;
    loff += B->h[p]->L;
  }
  return SEM_OK;
}
