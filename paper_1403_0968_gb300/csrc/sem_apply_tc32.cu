// FP32 operator apply (SEM_FP32, apply variant 5) at order N = 7 with the D-contractions on the
// tensor cores: the sum-factorised stiffness of arXiv 1403.0968 §4.2.1 (gather, D-contractions
// along r, s, t, per-node factor scaling, transposed contractions, scatter-add) in FP32, as the
// inner apply of the mixed-precision refinement (a TF32-MMA operator apply with FP32
// accumulation).
//
// One TF32 product keeps 11 significant bits of each operand: an error of about 2^-11 of
// |M||v| per line product, far too large for the inner solve of the refinement, whose operator
// must stay close to A relative to its smallest eigenvalue.  So each value is split in two
// (the "3xTF32" scheme, here with all four slice products):
//   * v = v1 + v2 with v1 = v with its 13 lowest mantissa bits cleared (exact in TF32) and
//     v2 = v - v1 (exact in FP32; the tensor cores read its top 11 bits);
//   * M = D1 + D2 likewise on the host (M = D for the forward products, D^T for the transposed);
//   * one MMA with K = 32 forms v1 D1 + v2 D1 + v1 D2 + v2 D2 in the FP32 accumulator: every
//     product is exact, the dropped parts are below 2^-22 of |M||v|, and the accumulation rounds
//     like an FP32 dot product.
// The A operand holds, for each of the 128 lines of a block (two elements x 64 lines), the row
// [v1 | v2 | v1 | v2] (K-major, no swizzle: core matrices of 8 rows x 16 bytes, 128 bytes apart
// along K and 1024 bytes apart along the rows); the B operand holds [D1 | D1 | D2 | D2] for the
// 8 outputs of a line (N = 16, the upper 8 columns zero).  Thread t owns line t in every
// direction, and tensor-memory lane t is its row, so each thread reads its 8 outputs with one
// tcgen05.ld.  The factor scaling and the scatter stay on the CUDA cores, as in the FP32 kernel.
//
// Blocks are persistent (one element pair after another) and hold 64 tensor-memory columns and
// about 62 KB of shared memory each, so at most three share an SM.  Every wait is bounded: a
// block that gives up records SEM_ERR_TIMEOUT in the handle's flag, waits (bounded) for its
// tensor-core work and leaves.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <string>

#include "sem_internal.h"
#include "sem_reduce.cuh"
#include "sem_tma.cuh"

namespace semtc32 {

constexpr int NP = 8, N = 7, NP2 = 64, NP3 = 512, EB = 2, NT = 128;
constexpr int RS = NP | 1, PS = NP * RS, BUF = NP * PS;  // value buffers as in the FP32 kernel
constexpr uint32_t TMEM_COLS = 64;                        // three directions x 16 columns, rounded up

// shared-memory layout (bytes)
constexpr int KW = 32;                 // K: slices v1, v2, v1, v2 of a line (8 values each)
constexpr int NC = 16;                 // N: the 8 outputs of a line and 8 zero columns
constexpr int SBO = (KW / 4) * 128;    // bytes between 8-row groups of a K-major operand
constexpr int A_BYTES = 128 * KW * 4;  // one direction's operand: 128 rows x 32 TF32 values
constexpr int B_BYTES = NC * KW * 4;   // 16 output columns x 32 values
constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + 3 * A_BYTES;             // forward slices of D, then of D^T
constexpr int OFF_V = OFF_B + 2 * B_BYTES;             // value buffers sr (also u), ss
constexpr int V_BYTES = EB * BUF * 4;
constexpr int OFF_RED = OFF_V + 2 * V_BYTES;           // 32 doubles for block sums
constexpr int OFF_MISC = OFF_RED + 32 * 8;             // mbarrier, TMEM address, flags
constexpr int SMEM_BYTES = OFF_MISC + 32;
constexpr int SMEM_ALLOC = SMEM_BYTES + 128;           // slack for the 128-byte alignment
constexpr int BLOCKS_PER_SM = 3;
static_assert(BLOCKS_PER_SM * (SMEM_ALLOC + 1024) <= 228 * 1024, "three blocks per SM");
static_assert(BLOCKS_PER_SM * TMEM_COLS <= 512, "tensor-memory columns of the resident blocks");
static_assert(OFF_B % 128 == 0 && OFF_V % 16 == 0 && OFF_RED % 16 == 0 && OFF_MISC % 16 == 0, "alignment");

struct Tc32Params {
  int64_t E, npairs;
  int sx, sy, sz;
  int64_t gxs, gys, gzs;
  int bc;
  const float *u;
  float *y;
  const float *Gf;  // [E][gs]: factor f of node p at f n3 + p
  int64_t gs;
  const float *wJa;  // [E][n3] or NULL
  const int32_t *glo;
  const uint8_t *mask;
  double *partials, *gpartials;
  unsigned int *gtickets;
  SemScalars *scal;
  int *err;
  uint32_t wait_polls;
  float d1[64], d2[64];  // the two TF32 slices of D (row-major D[i][m])
};

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory descriptor of a K-major operand without swizzle: core matrices of 8 rows x 16
// bytes, 128 bytes apart along K (leading byte offset) and SBO bytes apart along the rows
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((uint32_t)SBO >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}

// TF32 x TF32 -> FP32, both operands K-major, M = 128, N = 16
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NC >> 3) << 17) | ((128u >> 4) << 24);

// byte offset of element (row, k) of a K-major KW-wide operand
__host__ __device__ constexpr int kmajor_off(int row, int k) {
  return (row / 8) * SBO + (k / 4) * 128 + (row % 8) * 16 + (k % 4) * 4;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// this thread's A row of one direction: [v1 | v2 | v1 | v2] for its line of 8 values
__device__ __forceinline__ void line_prep(const float (&v)[NP], uint32_t arow) {
  float v1[NP], v2[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    v1[m] = __uint_as_float(__float_as_uint(v[m]) & 0xFFFFE000u);  // 11 significant bits
    v2[m] = __fsub_rn(v[m], v1[m]);                                 // exact
  }
  st_shared_v4(arow, v1[0], v1[1], v1[2], v1[3]);
  st_shared_v4(arow + 128, v1[4], v1[5], v1[6], v1[7]);
  st_shared_v4(arow + 256, v2[0], v2[1], v2[2], v2[3]);
  st_shared_v4(arow + 384, v2[4], v2[5], v2[6], v2[7]);
  st_shared_v4(arow + 512, v1[0], v1[1], v1[2], v1[3]);
  st_shared_v4(arow + 640, v1[4], v1[5], v1[6], v1[7]);
  st_shared_v4(arow + 768, v2[0], v2[1], v2[2], v2[3]);
  st_shared_v4(arow + 896, v2[4], v2[5], v2[6], v2[7]);
}

// this thread's 8 outputs of direction `dir` (tensor-memory columns 16 dir .. 16 dir + 7)
__device__ __forceinline__ void tmem_outputs(uint32_t tmem, int dir, float (&o)[NP]) {
  uint32_t r[8];
  const uint32_t ta = tmem + ((uint32_t)((threadIdx.x / 32) * 32) << 16) + (uint32_t)(dir * NC);
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) o[j] = __uint_as_float(r[j]);
}

// issues the three directions' products (four K-steps each) into columns 0, 16, 32 and commits
__device__ __forceinline__ void issue_mmas(uint32_t sA, uint32_t sB, uint32_t tmem, uint64_t *bar) {
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
#pragma unroll
    for (int ks = 0; ks < KW / 8; ++ks) {
      const uint64_t ad = kmajor_desc(sA + (uint32_t)(dir * A_BYTES + ks * 256));
      const uint64_t bd = kmajor_desc(sB + (uint32_t)(ks * 256));
      const uint32_t acc = ks > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)(dir * NC)),
          "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
          : "memory");
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

template <bool BOXM, bool DOT>
__global__ void __launch_bounds__(NT, BLOCKS_PER_SM) k_apply_f32_tc(const Tc32Params P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const uint32_t sA = smem_addr(smem + OFF_A), sB = smem_addr(smem + OFF_B);
  float *sr_all = reinterpret_cast<float *>(smem + OFF_V);
  float *ss_all = reinterpret_cast<float *>(smem + OFF_V + V_BYTES);
  double *s_red = reinterpret_cast<double *>(smem + OFF_RED);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + OFF_MISC);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + OFF_MISC + 8);
  int *s_flag = reinterpret_cast<int *>(smem + OFF_MISC + 12);

  if (DOT && P.partials && (P.scal->converged || P.scal->breakdown)) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int es = tid / NP2, t2 = tid - es * NP2, a = t2 % NP, b = t2 / NP;
  float *sr = sr_all + es * BUF, *ss = ss_all + es * BUF;

  // ---- once per block: tensor memory, barrier, the B operands (slices of D and of D^T) ----
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init(bar, 1);
  // B row n = output i (rows 8..15 zero), column k = 8 group + m against the A groups
  // (v1, v2, v1, v2): groups 0, 1 take D1, groups 2, 3 take D2.  Forward M = D, transposed M = D^T.
  for (int idx = tid; idx < 2 * NC * KW; idx += NT) {
    const int which = idx / (NC * KW), n = (idx / KW) % NC, k = idx % KW;
    const int g = k / 8, m = k % 8;
    const int q = which ? m * 8 + n : n * 8 + m;
    const float val = n < 8 ? (g < 2 ? P.d1[q] : P.d2[q]) : 0.f;
    *reinterpret_cast<float *>(smem + OFF_B + which * B_BYTES + kmajor_off(n, k)) = val;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t arow = sA + (uint32_t)kmajor_off(tid, 0);  // this thread's row in direction 0
  uint32_t phase = 0;
  bool ok = true;
  double dot_acc = 0.0;  // fused (u, Au) of this thread's nodes

  for (int64_t pair = blockIdx.x; pair < P.npairs && ok; pair += gridDim.x) {
    const int64_t e = pair * EB + es;
    const bool active = e < P.E;

    // ---- phase 0: gather the column of u ----
    int64_t gbase = 0;
    uint32_t dirbits = 0;
    float uc[NP];
    const int64_t plane = P.gxs * P.gys;
    if constexpr (BOXM) {
      if (active) {
        const int64_t ex = e % P.sx, exy = e / P.sx, ey = exy % P.sy, ez = exy / P.sy;
        const int64_t I = ex * N + a, J = ey * N + b;
        gbase = I + P.gxs * (J + P.gys * (ez * N));
        if (P.bc == SEM_BC_BOX) {
          if (I == 0 || I == P.gxs - 1 || J == 0 || J == P.gys - 1) dirbits = (1u << NP) - 1u;
          if (ez == 0) dirbits |= 1u;
          if (ez == P.sz - 1) dirbits |= 1u << N;
        }
      } else {
        dirbits = (1u << NP) - 1u;
      }
      const float *up = P.u + gbase;
#pragma unroll
      for (int k = 0; k < NP; ++k) uc[k] = ((dirbits >> k) & 1u) ? 0.f : up[k * plane];
    } else {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        int64_t g = 0;
        bool d = !active;
        if (active) {
          if (P.glo) {
            g = P.glo[e * NP3 + t2 + NP2 * k];
          } else {
            const int64_t ex = e % P.sx, ey = (e / P.sx) % P.sy, ez = e / ((int64_t)P.sx * P.sy);
            g = (ex * N + a) + P.gxs * ((ey * N + b) + P.gys * (ez * N + k));
          }
          if (P.bc == SEM_BC_BOX) {
            const int64_t I = g % P.gxs, J = (g / P.gxs) % P.gys, K = g / (P.gxs * P.gys);
            d = I == 0 || J == 0 || K == 0 || I == P.gxs - 1 || J == P.gys - 1 || K == P.gzs - 1;
          } else if (P.bc == SEM_BC_MASK) {
            d = P.mask[g] != 0;
          }
        }
        dirbits |= (d ? 1u : 0u) << k;
        uc[k] = d ? 0.f : P.u[g];
      }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) sr[k * PS + b * RS + a] = uc[k];  // sr holds u until the products read it
    __syncthreads();

    // ---- phase 1: forward products D along r, s, t ----
    {
      float row[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + a * RS + m];  // r-line (j = a, k = b)
      line_prep(row, arow);
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + m * RS + a];  // s-line (i = a, k = b)
      line_prep(row, arow + A_BYTES);
      line_prep(uc, arow + 2 * A_BYTES);  // t-line: the column
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue_mmas(sA, sB, tmem, bar);
    }
    ok = mbar_wait(bar, phase, P.wait_polls);
    if (__syncthreads_or(!ok)) {
      ok = false;  // `phase` is the completion still owed
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    float wt[NP];  // t-gradient of the column, then w_t
    {
      float o[NP];
      tmem_outputs(tmem, 0, o);
#pragma unroll
      for (int i = 0; i < NP; ++i) sr[b * PS + a * RS + i] = o[i];
      tmem_outputs(tmem, 1, o);
#pragma unroll
      for (int j = 0; j < NP; ++j) ss[b * PS + j * RS + a] = o[j];
      tmem_outputs(tmem, 2, wt);
    }
    tc_fence_before();
    __syncthreads();

    // ---- phase 2: geometric factors ----
    {
      const float *Ge = P.Gf + (active ? e : 0) * P.gs + t2;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int q = k * PS + b * RS + a;
        const int o = k * NP2;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f, g5 = 0.f;
        if (active) {
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
    __syncthreads();

    // ---- phase 3: transposed products D^T along r, s, t ----
    {
      float row[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + a * RS + m];
      line_prep(row, arow);
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = ss[b * PS + m * RS + a];
      line_prep(row, arow + A_BYTES);
      line_prep(wt, arow + 2 * A_BYTES);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue_mmas(sA, sB + B_BYTES, tmem, bar);
    }
    ok = mbar_wait(bar, phase, P.wait_polls);
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    float yt[NP];
    {
      float o[NP];
      tmem_outputs(tmem, 0, o);
#pragma unroll
      for (int i = 0; i < NP; ++i) sr[b * PS + a * RS + i] = o[i];
      tmem_outputs(tmem, 1, o);
#pragma unroll
      for (int j = 0; j < NP; ++j) ss[b * PS + j * RS + a] = o[j];
      tmem_outputs(tmem, 2, yt);
    }
    tc_fence_before();
    __syncthreads();

    // ---- phase 4: sum the three directions (+ mass term), scatter ----
    float dotp = 0.f;
    const bool ij_interior = (a > 0) && (a < N) && (b > 0) && (b < N) && !P.glo;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = k * PS + b * RS + a;
      float yk = yt[k] + sr[q] + ss[q];
      if (P.wJa && active) yk += P.wJa[e * NP3 + t2 + NP2 * k] * uc[k];
      if ((dirbits >> k) & 1u) continue;
      if (DOT) dotp += uc[k] * yk;
      int64_t g;
      if constexpr (BOXM) {
        g = gbase + k * plane;
      } else {
        if (P.glo) {
          g = P.glo[e * NP3 + t2 + NP2 * k];
        } else {
          const int64_t ex = e % P.sx, ey = (e / P.sx) % P.sy, ez = e / ((int64_t)P.sx * P.sy);
          g = (ex * N + a) + P.gxs * ((ey * N + b) + P.gys * (ez * N + k));
        }
      }
      if (ij_interior && k > 0 && k < N)
        P.y[g] = yk;  // element-interior node: owned by this element alone
      else
        atomicAdd(P.y + g, yk);
    }
    if (DOT) dot_acc += (double)dotp;
    __syncthreads();  // this pair's buffers are read before the next pair's gather writes them
  }

  if (!ok) {
    // a wait gave up: record it; wait (bounded) for the tensor-core work this block committed last
    if (tid == 0) {
      atomicOr(P.err, 1);
      mbar_wait(bar, phase);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");

  if (DOT && P.partials && ok) {
    const double bs = block_sum<NT>(dot_acc, s_red);
    double pAp;
    if (publish_partial_2level<NT>(bs, P.partials, P.gpartials, P.gtickets, &P.scal->counter[0], s_red, s_flag,
                                   &pAp)) {
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

template <bool BOXM, bool DOT>
sem_status launch(const Tc32Params &p, unsigned grid, cudaStream_t s) {
  static std::atomic<unsigned long long> attr_done;
  const cudaError_t e = set_smem_limit_once(k_apply_f32_tc<BOXM, DOT>, SMEM_ALLOC, attr_done);
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("tensor-core FP32 apply attributes: ") + cudaGetErrorString(e));
  k_apply_f32_tc<BOXM, DOT><<<grid, NT, SMEM_ALLOC, s>>>(p);
  return SEM_OK;
}

// the value of x kept by a TF32 operand whose low 13 mantissa bits are cleared, rounded to the
// nearest (ties away from zero) instead of truncated
float tf32_round(double x) {
  float f = (float)x;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  std::memcpy(&f, &b, 4);
  return f;
}

}  // namespace semtc32

// Launches the tensor-core FP32 apply (order 7 only; the caller checks).
sem_status sem_launch_apply_f32_tc(sem_handle *h, const float *u, float *y, double *partials, cudaStream_t s) {
  using namespace semtc32;
  if (h->N != 7) return sem_fail(SEM_ERR_INVALID, "tensor-core FP32 apply: order 7 only");
  if (!h->G32) return sem_fail(SEM_ERR_INVALID, "handle has no FP32 factors (SEM_FEAT_FP32)");
  Tc32Params p;
  std::memset(&p, 0, sizeof(p));
  p.E = h->E;
  p.npairs = (h->E + EB - 1) / EB;
  p.sx = h->box[0];
  p.sy = h->box[1];
  p.sz = h->box[2];
  p.gxs = (int64_t)h->box[0] * h->N + 1;
  p.gys = (int64_t)h->box[1] * h->N + 1;
  p.gzs = (int64_t)h->box[2] * h->N + 1;
  p.bc = h->bc;
  p.u = u;
  p.y = y;
  p.Gf = h->G32;
  p.gs = h->gs6;
  p.wJa = h->wJa32;
  p.glo = h->structured ? nullptr : h->glo;
  p.mask = h->mask;
  p.partials = partials;
  p.gpartials = h->gpartials;
  p.gtickets = h->gtickets;
  p.scal = h->scal;
  p.err = &h->scal->error;
  p.wait_polls = h->wait_polls;
  const double *D = h->D64h;
  for (int q = 0; q < 64; ++q) {
    p.d1[q] = tf32_round(D[q]);
    p.d2[q] = tf32_round(D[q] - (double)p.d1[q]);
  }
  if (partials && !h->scal) return sem_fail(SEM_ERR_INVALID, "fused dot needs the solver scalars");
  int dev = 0, nsm = 152;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  SEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t want = (int64_t)nsm * BLOCKS_PER_SM;
  const unsigned grid = (unsigned)(p.npairs < want ? p.npairs : want);
  if (grid == 0) return SEM_OK;
  const bool boxm = p.glo == nullptr && p.bc != SEM_BC_MASK;
  const bool dot = partials != nullptr;
  sem_status st = boxm ? (dot ? launch<true, true>(p, grid, s) : launch<true, false>(p, grid, s))
                       : (dot ? launch<false, true>(p, grid, s) : launch<false, false>(p, grid, s));
  if (st != SEM_OK) return st;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("tensor-core FP32 apply launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}
