// FP64-accurate operator apply (SEM_FP64_EMU) at order N = 7 with the D-contractions on the tensor
// cores: the sum-factorised stiffness of arXiv 1403.0968 §4.2.1 (gather, D-contractions along r,
// s, t, per-node factor scaling, transposed contractions, scatter-add) with FP64 inputs and
// outputs and an error of the order of 2^-44 of the magnitudes involved, like the double-float
// kernel (sem_emu.cuh), whose element schedule and value buffers it keeps.
//
// Why: GB300 runs FP64 at 1/61 of the FP32 rate, and the double-float kernel spends 354 of its
// 466 FP32-pipe instructions per node on the six line products (compensated sums).  Here every
// line product out_i = sum_m M[i][m] v_m (M = D or D^T, v a line of 8 double-float values
// (hi, lo)) is split by exact slicing (the Ozaki scheme on TF32) into a part the tensor cores
// compute without rounding and a small tail on the CUDA cores:
//   * per element, v is scaled by an exact power of two into |v| < 2 (u by its FP64 exponent,
//     the factor-scaled values w by their FP32 exponent; both undone exactly in the FP64
//     rebuild of y);
//   * v = v1 + v2 + v3 + vlow, v1, v2, v3 on the grids 2^-9, 2^-20, 2^-30 with at most 11
//     significant bits each (exact in TF32), |vlow| <= 2^-31; M = d1 + d2 + d3 + Mlow with d1,
//     d2, d3 on the grids 2^-5, 2^-16, 2^-27 (|M| < 2^5 at N = 7), |Mlow| <= 2^-28;
//   * the tensor cores (tcgen05.mma kind::tf32, FP32 accumulation in tensor memory) form the
//     level sums L2 = sum d1 v1, L3 = sum d1 v2 + d2 v1 (products of at most 22 bits on a common
//     grid, sums within 24 bits: exact), L4 = sum d1 v3 + d2 v2 + d3 v1 and L56 = sum d2 v3 +
//     d3 v2 + d3 v3 (rounded once, at 2^-24 of magnitudes 2^-22 and 2^-33 of the line's);
//   * the CUDA cores add the tail sum_m (Mlow[i][m] FP32(v_m) + (d1 + d2 + d3)[i][m] vlow_m) in
//     FP32 (even-odd form: M is centro-antisymmetric) and combine L2 + L3 + L4 + (L56 + tail) into
//     a double-float pair (two TwoSums, one Fast2Sum).  The error is about 2^-48 of
//     sum_m |M[i][m]| |v_m| (2^-45.5 for the compensated double-float line product).
// The A operand holds, for each of the 128 lines of a block (two elements x 64 lines), the row
// [v1 | v2 | v3 | v3] (K = 32: four TF32 MMAs of K = 8; K-major, no swizzle: core matrices of 8
// rows x 16 bytes, 128 bytes apart along K and 1024 bytes apart along the rows); the B operand
// holds the slices of M so that output column 8 l + i is level l of output i (N = 32; the second
// copy of v3 meets d3 in the last level).  Thread t owns line t in every direction, and
// tensor-memory lane t is its row, so each thread reads its own 32 level values with one
// tcgen05.ld.
//
// The factor scaling stays in double-float on the CUDA cores (a 3 x 3 product per node).  Blocks
// are persistent (one element pair after another) and hold 128 tensor-memory columns and about
// 74 KB of shared memory each, so at most three share an SM and their allocations always fit.
// Every wait is bounded: a block that gives up records SEM_ERR_TIMEOUT in the handle's flag, waits
// (bounded) for its tensor-core work and leaves.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

#include "sem_emu.cuh"

namespace semtc {

using namespace semu;

constexpr int NP = 8, N = 7, NP2 = 64, NP3 = 512, EB = 2, NT = 128;
constexpr int RS = NP | 1, PS = NP * RS, BUF = NP * PS;  // value buffers as in the double-float kernel
constexpr int DELTA = 5;                                  // max |D| = 18.94 at N = 7: below 2^5
constexpr uint32_t TMEM_COLS = 128;                       // three directions x 32 columns, rounded up

// shared-memory layout (bytes)
constexpr int KW = 32;                 // K: slices v1, v2, v3, v3 of a line (8 values each)
constexpr int SBO = (KW / 4) * 128;    // bytes between 8-row groups of a K-major operand
constexpr int A_BYTES = 128 * KW * 4;  // one direction's operand: 128 rows x 32 TF32 values
constexpr int B_BYTES = 32 * KW * 4;   // 32 output columns x 32 values
constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + 3 * A_BYTES;             // forward slices of D, then of D^T
constexpr int OFF_V = OFF_B + 2 * B_BYTES;             // value buffers sr (also su), ss
constexpr int V_BYTES = EB * BUF * 8;
constexpr int OFF_RED = OFF_V + 2 * V_BYTES;           // 32 doubles for block sums
constexpr int OFF_MISC = OFF_RED + 32 * 8;             // mbarrier, TMEM address, flags, maxima
constexpr int SMEM_BYTES = OFF_MISC + 64;
constexpr int SMEM_ALLOC = SMEM_BYTES + 128;           // slack for the 128-byte alignment
constexpr int BLOCKS_PER_SM = 3;
static_assert(4 * (SMEM_ALLOC + 1024) > 228 * 1024 && 3 * (SMEM_ALLOC + 1024) <= 228 * 1024,
              "exactly three blocks per SM: 3 x 128 tensor-memory columns always fit");
static_assert(OFF_V % 16 == 0 && OFF_RED % 16 == 0 && OFF_MISC % 16 == 0, "alignment");

struct TcParams {
  int64_t E, npairs;
  int sx, sy, sz;
  int64_t gxs, gys, gzs;
  int bc;
  const double *u;
  double *y;
  const float *Gf;  // [E][gs]: factor f hi at 2f n3 + p, lo at (2f+1) n3 + p
  int64_t gs;
  const float *wJa;  // [E][2][n3] or NULL
  const int32_t *glo;
  const uint8_t *mask;
  double *partials, *gpartials;
  unsigned int *gtickets;
  SemScalars *scal;
  int *err;
  uint32_t wait_polls;
  float d1[64], d2[64], d3[64];  // slices of D (row-major D[i][m])
  // even-odd coefficients of the tail, (M[i][m] +- M[N-i][m]) / 2 at [i][m], i, m < 4, for the
  // forward (M = D) and transposed (M = D^T) products: Mlow = M - d1 - d2 - d3, M123 = d1 + d2 + d3
  float flp[16], flm[16], f12p[16], f12m[16];
  float tlp[16], tlm[16], t12p[16], t12m[16];
};

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory descriptor of a K-major operand without swizzle: core matrices of 8 rows x 16
// bytes, 128 bytes apart along K (leading byte offset) and SBO bytes apart along the rows (stride
// byte offset)
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((uint32_t)SBO >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}

// TF32 x TF32 -> FP32, both operands K-major, M = 128, N = 32
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// byte offset of element (row, k) of a K-major KW-wide operand
__host__ __device__ constexpr int kmajor_off(int row, int k) {
  return (row / 8) * SBO + (k / 4) * 128 + (row % 8) * 16 + (k % 4) * 4;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// rounds x (|x| < 2^(k+22)) to the grid 2^k, ties to even, by the exact-magnitude constant C = 1.5 2^(k+23)
__device__ __forceinline__ float grid_round(float x, float C) { return __fsub_rn(__fadd_rn(x, C), C); }

// One line of 8 double-float values (|v| < 2): writes this thread's A row (v1 | v2 | v3 | v3) at
// `arow` and returns the tail of the 8 outputs, sum_m Mlow[i][m] FP32(v_m) + M123[i][m] vlow_m
// (even-odd form).  r1 = hi - v1 and r2 = r1 - v2 are exact; v3 takes the top bits of r2 + lo
// (|r2| <= 2^-21, |lo| <= 2^-24) and r2 - v3 is exact, so vlow = (r2 - v3) + lo carries one rounding
// of about 2^-55.
__device__ __forceinline__ void line_prep(const float2 (&v)[NP], uint32_t arow, const float *lp, const float *lm,
                                          const float *hp, const float *hm, float (&tail)[NP]) {
  constexpr float C1 = 24576.0f;       // 1.5 * 2^14: grid 2^-9
  constexpr float C2 = 12.0f;          // 1.5 * 2^3:  grid 2^-20
  constexpr float C3 = 0.01171875f;    // 1.5 * 2^-7: grid 2^-30
  float v1[NP], v2[NP], v3[NP], vf[NP], vl[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    vf[m] = v[m].x;
    v1[m] = grid_round(v[m].x, C1);
    const float r1 = __fsub_rn(v[m].x, v1[m]);
    v2[m] = grid_round(r1, C2);
    const float r2 = __fsub_rn(r1, v2[m]);
    v3[m] = grid_round(__fadd_rn(r2, v[m].y), C3);
    vl[m] = __fadd_rn(__fsub_rn(r2, v3[m]), v[m].y);
  }
  st_shared_v4(arow, v1[0], v1[1], v1[2], v1[3]);
  st_shared_v4(arow + 128, v1[4], v1[5], v1[6], v1[7]);
  st_shared_v4(arow + 256, v2[0], v2[1], v2[2], v2[3]);
  st_shared_v4(arow + 384, v2[4], v2[5], v2[6], v2[7]);
  st_shared_v4(arow + 512, v3[0], v3[1], v3[2], v3[3]);
  st_shared_v4(arow + 640, v3[4], v3[5], v3[6], v3[7]);
  st_shared_v4(arow + 768, v3[0], v3[1], v3[2], v3[3]);
  st_shared_v4(arow + 896, v3[4], v3[5], v3[6], v3[7]);
  float ef[4], of[4], el[4], ol[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    ef[m] = vf[m] + vf[N - m];
    of[m] = vf[m] - vf[N - m];
    el[m] = vl[m] + vl[N - m];
    ol[m] = vl[m] - vl[N - m];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float p = 0.f, q = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      p = fmaf(lp[i * 4 + m], of[m], p);
      p = fmaf(hp[i * 4 + m], ol[m], p);
      q = fmaf(lm[i * 4 + m], ef[m], q);
      q = fmaf(hm[i * 4 + m], el[m], q);
    }
    tail[i] = p + q;
    tail[N - i] = p - q;
  }
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// L2 + L3 + L4 + (L56 + tail) as a normalised double-float pair: L2 and L3 are exact and L4 is of
// the order of 2^-22 of the result, so both additions keep their rounding errors (TwoSum); the
// rest is below 2^-20 of the result and is added in FP32
__device__ __forceinline__ float2 combine(float L2, float L3, float L4, float L56, float tail) {
  float s, e, s2, e2;
  two_sum(L2, L3, s, e);
  two_sum(s, L4, s2, e2);
  const float c = __fadd_rn(__fadd_rn(e, e2), __fadd_rn(L56, tail));
  const float h = __fadd_rn(s2, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, s2)));
}

// this thread's 32 level values of direction `dir` (tensor-memory columns 32 dir .. 32 dir + 31)
__device__ __forceinline__ void tmem_levels(uint32_t tmem, int dir, float (&L)[32]) {
  uint32_t r[32];
  const uint32_t ta = tmem + ((uint32_t)((threadIdx.x / 32) * 32) << 16) + (uint32_t)(dir * 32);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) L[j] = __uint_as_float(r[j]);
}

// issues the three directions' products (four K-steps each) into columns 0, 32, 64 and commits
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
          " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)(dir * 32)),
          "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
          : "memory");
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

template <bool BOXM, bool DOT>
__global__ void __launch_bounds__(NT, BLOCKS_PER_SM) k_apply_emu_tc(const TcParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const uint32_t sA = smem_addr(smem + OFF_A), sB = smem_addr(smem + OFF_B);
  float2 *sr_all = reinterpret_cast<float2 *>(smem + OFF_V);
  float2 *ss_all = reinterpret_cast<float2 *>(smem + OFF_V + V_BYTES);
  double *s_red = reinterpret_cast<double *>(smem + OFF_RED);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + OFF_MISC);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + OFF_MISC + 8);
  int *s_flag = reinterpret_cast<int *>(smem + OFF_MISC + 12);
  int *s_fail = reinterpret_cast<int *>(smem + OFF_MISC + 16);
  int *s_emax = reinterpret_cast<int *>(smem + OFF_MISC + 20);  // [EB] u: largest FP64 exponent
  int *s_wmax = reinterpret_cast<int *>(smem + OFF_MISC + 28);  // [EB] w: largest FP32 exponent

  if (DOT && P.partials && (P.scal->converged || P.scal->breakdown)) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int es = tid / NP2, t2 = tid - es * NP2, a = t2 % NP, b = t2 / NP;
  float2 *sr = sr_all + es * BUF, *ss = ss_all + es * BUF;

  // ---- once per block: tensor memory, barrier, the B operands (slices of D and of D^T) ----
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    *s_fail = 0;
  }
  if (t2 == 0) {
    s_emax[es] = 1;
    s_wmax[es] = 1;
  }
  // B rows n = 8 level + i, columns k = 8 slice + m against the A slices (v1, v2, v3, v3):
  //   level 0 (L2) = [d1 0 0 0], level 1 (L3) = [d2 d1 0 0], level 2 (L4) = [d3 d2 d1 0],
  //   level 3 (L56) = [0 d3 d2 d3].  Forward M = D (M[i][m] = D[i][m]), transposed M = D^T.
  for (int idx = tid; idx < 2 * 32 * KW; idx += NT) {
    const int which = idx / (32 * KW), n = (idx / KW) % 32, k = idx % KW;
    const int lev = n / 8, i = n % 8, sl = k / 8, m = k % 8;
    const int q = which ? m * 8 + i : i * 8 + m;
    // slice index of M paired with A slice `sl` in level `lev` (0: none)
    const int which_d = lev < 3 ? (sl <= lev ? lev - sl + 1 : 0) : (sl == 0 ? 0 : sl == 2 ? 2 : 3);
    const float val = which_d == 1 ? P.d1[q] : which_d == 2 ? P.d2[q] : which_d == 3 ? P.d3[q] : 0.f;
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
  double dot_acc = 0.0;  // fused (u, y) of this thread's nodes, FP64

  for (int64_t pair = blockIdx.x; pair < P.npairs && ok; pair += gridDim.x) {
    const int64_t e = pair * EB + es;
    const bool active = e < P.E;
    {
      // the next pair of this block: its factor block (contiguous) and this thread's u column are
      // fetched into L2 now, so that their loads find them there
      const int64_t next = pair + gridDim.x;
      if (next < P.npairs) {
        const int64_t e1 = next * EB;
        if (tid == 0) {
          const int64_t nel = (P.E - e1) < EB ? (P.E - e1) : EB;
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(P.Gf + e1 * P.gs),
                       "r"((uint32_t)(nel * P.gs * sizeof(float)))
                       : "memory");
        }
        if (BOXM && e1 + es < P.E) {
          int64_t ex, ey, ez;
          box_coords(e1 + es, P.sx, P.sy, P.E, ex, ey, ez);
          const double *un = P.u + (ex * N + a) + P.gxs * ((ey * N + b) + P.gys * (ez * N));
#pragma unroll
          for (int k = 0; k < NP; ++k)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(un + k * P.gxs * P.gys) : "memory");
        }
      }
    }

    // ---- phase 0: gather u, element scale, split into (hi, lo), column in registers ----
    int64_t gbase = 0;
    uint32_t dirbits = 0;
    double ud[NP];
    const int64_t plane = P.gxs * P.gys;
    if constexpr (BOXM) {
      if (active) {
        int64_t ex, ey, ez;
        box_coords(e, P.sx, P.sy, P.E, ex, ey, ez);
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
      const double *up = P.u + gbase;
#pragma unroll
      for (int k = 0; k < NP; ++k) ud[k] = ((dirbits >> k) & 1u) ? 0.0 : up[k * plane];
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
        ud[k] = d ? 0.0 : P.u[g];
      }
    }
    {
      int emx = 1;
#pragma unroll
      for (int k = 0; k < NP; ++k) emx = max(emx, f64_biased_exp(ud[k]));
      element_max(&s_emax[es], emx, es);
    }
    __syncthreads();
    const int shift = 1023 - s_emax[es];  // u 2^shift has its element maximum in [1, 2)
    float2 uc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      uc[k] = split_f64(ud[k], shift);
      sr[k * PS + b * RS + a] = uc[k];  // sr holds u until the forward products have read it
    }
    __syncthreads();

    // ---- phase 1: forward products D along r, s, t ----
    float tailr[NP], tails[NP], tailt[NP];
    {
      float2 row[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + a * RS + m];  // r-line (j = a, k = b)
      line_prep(row, arow, P.flp, P.flm, P.f12p, P.f12m, tailr);
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + m * RS + a];  // s-line (i = a, k = b)
      line_prep(row, arow + A_BYTES, P.flp, P.flm, P.f12p, P.f12m, tails);
      line_prep(uc, arow + 2 * A_BYTES, P.flp, P.flm, P.f12p, P.f12m, tailt);  // t-line: the column
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
    float2 wt[NP];  // t-gradient of the column, then w_t
    {
      float L[32];
      tmem_levels(tmem, 0, L);
#pragma unroll
      for (int i = 0; i < NP; ++i)
        sr[b * PS + a * RS + i] = combine(L[i], L[8 + i], L[16 + i], L[24 + i], tailr[i]);
      tmem_levels(tmem, 1, L);
#pragma unroll
      for (int j = 0; j < NP; ++j)
        ss[b * PS + j * RS + a] = combine(L[j], L[8 + j], L[16 + j], L[24 + j], tails[j]);
      tmem_levels(tmem, 2, L);
#pragma unroll
      for (int k = 0; k < NP; ++k) wt[k] = combine(L[k], L[8 + k], L[16 + k], L[24 + k], tailt[k]);
    }
    tc_fence_before();
    __syncthreads();

    // ---- phase 2: geometric factors (double-float), element scale of w ----
    {
      const float *Ge = P.Gf + (active ? e : 0) * P.gs + t2;
      int wmx = 1;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int q = k * PS + b * RS + a;
        const int o = k * NP2;
        float gh[6], gl[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          gh[f] = active ? Ge[(2 * f) * NP3 + o] : 0.f;
          gl[f] = active ? Ge[(2 * f + 1) * NP3 + o] : 0.f;
        }
        const float2 ur = sr[q], us = ss[q], ut = wt[k];
        float s, c;
        dacc_first(s, c, gh[0], gl[0], ur);
        dacc(s, c, gh[1], gl[1], us);
        dacc(s, c, gh[2], gl[2], ut);
        const float2 wr = dnorm(s, c);
        dacc_first(s, c, gh[1], gl[1], ur);
        dacc(s, c, gh[3], gl[3], us);
        dacc(s, c, gh[4], gl[4], ut);
        const float2 ws = dnorm(s, c);
        dacc_first(s, c, gh[2], gl[2], ur);
        dacc(s, c, gh[4], gl[4], us);
        dacc(s, c, gh[5], gl[5], ut);
        wt[k] = dnorm(s, c);
        sr[q] = wr;
        ss[q] = ws;
        wmx = max(wmx, max((int)((__float_as_uint(wr.x) >> 23) & 0xFFu),
                           max((int)((__float_as_uint(ws.x) >> 23) & 0xFFu),
                               (int)((__float_as_uint(wt[k].x) >> 23) & 0xFFu))));
      }
      element_max(&s_wmax[es], min(wmx, 253), es);
    }
    __syncthreads();

    // ---- phase 3: transposed products D^T along r, s, t (w scaled into |w| < 2) ----
    const int ew = s_wmax[es];
    const float wsc = __uint_as_float((uint32_t)(254 - ew) << 23);  // 2^(127 - ew), exact scaling
    {
      float2 row[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const float2 v = sr[b * PS + a * RS + m];
        row[m] = make_float2(v.x * wsc, v.y * wsc);
      }
      line_prep(row, arow, P.tlp, P.tlm, P.t12p, P.t12m, tailr);
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const float2 v = ss[b * PS + m * RS + a];
        row[m] = make_float2(v.x * wsc, v.y * wsc);
      }
      line_prep(row, arow + A_BYTES, P.tlp, P.tlm, P.t12p, P.t12m, tails);
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = make_float2(wt[m].x * wsc, wt[m].y * wsc);
      line_prep(row, arow + 2 * A_BYTES, P.tlp, P.tlm, P.t12p, P.t12m, tailt);
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
      ok = false;  // `phase` is the completion still owed
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    float2 yt[NP];
    {
      float L[32];
      tmem_levels(tmem, 0, L);
#pragma unroll
      for (int i = 0; i < NP; ++i)
        sr[b * PS + a * RS + i] = combine(L[i], L[8 + i], L[16 + i], L[24 + i], tailr[i]);
      tmem_levels(tmem, 1, L);
#pragma unroll
      for (int j = 0; j < NP; ++j)
        ss[b * PS + j * RS + a] = combine(L[j], L[8 + j], L[16 + j], L[24 + j], tails[j]);
      tmem_levels(tmem, 2, L);
#pragma unroll
      for (int k = 0; k < NP; ++k) yt[k] = combine(L[k], L[8 + k], L[16 + k], L[24 + k], tailt[k]);
    }
    tc_fence_before();
    __syncthreads();
    if (t2 == 0) {  // maxima of the next pair; every thread has read this pair's values
      s_emax[es] = 1;
      s_wmax[es] = 1;
    }

    // ---- phase 4: sum the three directions (+ mass term), rebuild FP64, scatter ----
    const double unscale_w = exp2i(ew - 127), unscale_u = exp2i(-shift);
    float dps = 0.f, dpc = 0.f;
    const bool ij_interior = (a > 0) && (a < N) && (b > 0) && (b < N) && !P.glo;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = k * PS + b * RS + a;
      float s = yt[k].x, c = yt[k].y;
      dadd(s, c, sr[q]);
      dadd(s, c, ss[q]);
      if (P.wJa && active) {
        const int64_t o = e * 2 * NP3 + t2 + NP2 * k;
        float ms, mc;
        dacc_first(ms, mc, P.wJa[o], P.wJa[o + NP3], uc[k]);
        const float2 mass = dnorm(ms, mc);
        dadd(s, c, make_float2(mass.x * wsc, mass.y * wsc));
      }
      const float2 yk = dnorm(s, c);
      if ((dirbits >> k) & 1u) continue;
      if (DOT) dacc(dps, dpc, uc[k].x, uc[k].y, yk);
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
      const double yd = df_to_f64(yk) * unscale_w * unscale_u;
      if (ij_interior && k > 0 && k < N)
        P.y[g] = yd;
      else
        atomicAdd(P.y + g, yd);
    }
    if (DOT) dot_acc += df_to_f64(dnorm(dps, dpc)) * unscale_w * unscale_u * unscale_u;
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

// host: slices of a value on the grid 2^k (ties to even), in FP64
double slice(double x, int k) { return std::nearbyint(std::ldexp(x, -k)) * std::ldexp(1.0, k); }

template <bool BOXM, bool DOT>
sem_status launch(const TcParams &p, unsigned grid, cudaStream_t s) {
  static std::atomic<unsigned long long> attr_done;
  const cudaError_t e = set_smem_limit_once(k_apply_emu_tc<BOXM, DOT>, SMEM_ALLOC, attr_done);
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("tensor-core apply attributes: ") + cudaGetErrorString(e));
  k_apply_emu_tc<BOXM, DOT><<<grid, NT, SMEM_ALLOC, s>>>(p);
  return SEM_OK;
}

}  // namespace semtc

// Launches the tensor-core double-float apply (order 7 only; the caller checks).
sem_status sem_launch_apply_emu_tc(sem_handle *h, const double *u, double *y, double *partials, cudaStream_t s) {
  using namespace semtc;
  if (h->N != 7) return sem_fail(SEM_ERR_INVALID, "tensor-core double-float apply: order 7 only");
  TcParams p;
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
  p.Gf = h->Gemu;
  p.gs = h->gs12;
  p.wJa = h->wJaemu;
  p.glo = h->structured ? nullptr : h->glo;
  p.mask = h->mask;
  p.partials = partials;
  p.gpartials = h->gpartials;
  p.gtickets = h->gtickets;
  p.scal = h->scal;
  p.err = &h->scal->error;
  p.wait_polls = h->wait_polls;
  const double *D = h->D64h;
  double d12[64], dlow[64];  // d12 holds d1 + d2 + d3 (the part on the tensor cores)
  for (int q = 0; q < 64; ++q) {
    const double a1 = slice(D[q], DELTA - 10);
    const double a2 = slice(D[q] - a1, DELTA - 21);
    const double a3 = slice(D[q] - a1 - a2, DELTA - 32);
    p.d1[q] = (float)a1;
    p.d2[q] = (float)a2;
    p.d3[q] = (float)a3;
    d12[q] = a1 + a2 + a3;
    dlow[q] = D[q] - d12[q];
  }
  // even-odd pairs (M[i][m] +- M[N-i][m]) / 2, M = D (forward) or D^T (transposed)
  for (int i = 0; i < 4; ++i)
    for (int m = 0; m < 4; ++m) {
      const int o = i * 4 + m;
      const int im = i * 8 + m, nim = (N - i) * 8 + m;   // D[i][m], D[N-i][m]
      const int ti = m * 8 + i, tni = m * 8 + (N - i);   // D^T[i][m] = D[m][i], D^T[N-i][m] = D[m][N-i]
      p.flp[o] = (float)(0.5 * (dlow[im] + dlow[nim]));
      p.flm[o] = (float)(0.5 * (dlow[im] - dlow[nim]));
      p.f12p[o] = (float)(0.5 * (d12[im] + d12[nim]));
      p.f12m[o] = (float)(0.5 * (d12[im] - d12[nim]));
      p.tlp[o] = (float)(0.5 * (dlow[ti] + dlow[tni]));
      p.tlm[o] = (float)(0.5 * (dlow[ti] - dlow[tni]));
      p.t12p[o] = (float)(0.5 * (d12[ti] + d12[tni]));
      p.t12m[o] = (float)(0.5 * (d12[ti] - d12[tni]));
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
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("tensor-core apply launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}
