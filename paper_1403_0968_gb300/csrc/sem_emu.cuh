// FP64-accurate operator apply in double-float arithmetic (SEM_FP64_EMU).
//
// Same operator and the same five-phase element schedule as the FP64/FP32 kernel
// (sem_apply_kernel.cuh; arXiv 1403.0968 §4.2.1, sum-factorised stiffness display), but every
// value is carried as an unevaluated pair of FP32 numbers (hi, lo) with |lo| <= ulp(hi)/2, because
// GB300 executes FP64 FMAs at 1/61 of the FP32 rate.  Inputs and outputs stay FP64:
//   * u (FP64) is scaled per element by an exact power of two, 2^(1023 - e) with e the largest
//     biased FP64 exponent among the element's gathered values, so that the element's largest
//     |u| lies in [1, 2) whatever the scale of u; y_e is scaled back by the inverse power of two
//     when it is rebuilt as FP64 (exact).  The scaled value is split into (hi, lo) by bit
//     manipulation: hi keeps the top 24 significand bits, lo the next 24 (integer instructions,
//     not FP64 conversions);
//   * the factors are stored as (hi, lo) pairs by set-up, D as (hi, lo) launch parameters;
//   * each sum  sum_m a_m b_m  is formed with exact products (p = a_hi b_hi and its FMA
//     remainder, the published TwoProduct transformation) and Knuth's TwoSum on the high parts;
//     every low-order term goes into one FP32 compensation, and the pair is renormalised at the
//     end (Fast2Sum).  The error is about 2^-44 of the sum of |terms| per output (double-float
//     accuracy after Dekker 1971 / Ogita-Rump-Oishi 2005);
//   * y = hi + lo is rebuilt as FP64 (one FP64 add per node) and scatter-added with FP64 atomics.
// Accuracy: u of any FP64 magnitude (FP64 subnormals are flushed to zero).  Within an element,
// entries smaller than 2^-74 of its largest |u| keep FP32 relative accuracy and entries below
// 2^-126 of it are flushed: absolute errors below 2^-98 of the element's largest |u|.  The
// factors must lie within 2^-60 .. 2^60 (checked at set-up, which refuses SEM_FEAT_EMU otherwise),
// so that every intermediate product keeps its low word in the FP32 normal range.
//
// This header holds the kernel and its launcher; sem_emu_*.cu instantiate the launcher for ranges of
// orders (to spread the compile time over translation units) and sem_emu.cu dispatches by order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sem_internal.h"
#include "sem_reduce.cuh"
#include "sem_tma.cuh"

namespace semu {

// ---- double <-> double-float conversions (integer pipeline) ----
// biased FP64 exponent of u (0 for zeros and subnormals)
__device__ __forceinline__ int f64_biased_exp(double u) {
  return (int)(((unsigned int)(__double_as_longlong(u) >> 32) >> 20) & 0x7FFu);
}

// 2^k as a double, for -1022 <= k <= 1023
__device__ __forceinline__ double exp2i(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// atomicMax of v into *slot for the element this thread belongs to: a warp whose lanes all belong
// to one element reduces first and issues one atomic (a shared-memory atomic from every lane to
// the same address would serialise 32 ways)
__device__ __forceinline__ void element_max(int *slot, int v, int es) {
  const int es0 = __shfl_sync(0xffffffffu, es, 0), es31 = __shfl_sync(0xffffffffu, es, 31);
  if (es0 == es31) {
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) atomicMax(slot, v);
  } else {
    atomicMax(slot, v);
  }
}

// element coordinates (ex, ey, ez) of element e of an sx x sy x sz box, in 32-bit arithmetic when
// the element count allows (64-bit division costs several times more instructions)
__device__ __forceinline__ void box_coords(int64_t e, int sx, int sy, int64_t E, int64_t &ex, int64_t &ey,
                                           int64_t &ez) {
  if (E <= 0x7fffffffll) {
    const uint32_t e32 = (uint32_t)e, exy = e32 / (uint32_t)sx;
    ex = e32 - exy * (uint32_t)sx;
    ey = exy % (uint32_t)sy;
    ez = exy / (uint32_t)sy;
  } else {
    const int64_t exy = e / sx;
    ex = e - exy * sx;
    ey = exy % sy;
    ez = exy / sy;
  }
}

// (hi, lo) of u * 2^shift (exact scaling; shift chosen so that the result is below 2); FP64
// subnormals and results below 2^-126 are flushed to zero
__device__ __forceinline__ float2 split_f64(double u, int shift) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(u);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const int ex0 = (int)((hw >> 20) & 0x7FFu);
  const int ex = ex0 == 0 ? 0 : ex0 + shift;
  const unsigned int sign = hw & 0x80000000u;
  float h = 0.0f, l = 0.0f;
  if (ex >= 897 && ex <= 1150) {
    const unsigned int m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);  // significand bits 51..29
    h = __uint_as_float(sign | ((unsigned int)(ex - 896) << 23) | m23);
    const unsigned int mlo = lw & 0x1FFFFFFFu;  // significand bits 28..0, weight 2^(ex-1075)
    if (mlo != 0u && ex >= 949) {
      const float scale = __uint_as_float((unsigned int)(ex - 948) << 23);
      l = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(mlo), scale)) | sign);
    }
  } else if (ex > 1150) {
    h = __double2float_rn(u);  // overflow, inf or nan (not expected on this path)
  }
  return make_float2(h, l);
}

__device__ __forceinline__ double f32_as_f64(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int ex = (b >> 23) & 0xFFu;
  if (ex == 0u) return 0.0;
  const unsigned long long e64 = ex == 0xFFu ? 0x7FFull : (unsigned long long)(ex + 896u);
  const unsigned long long r =
      ((unsigned long long)(b & 0x80000000u) << 32) | (e64 << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)r);
}

__device__ __forceinline__ double df_to_f64(float2 v) { return f32_as_f64(v.x) + f32_as_f64(v.y); }

// ---- double-float dot-product accumulation: (s, c) += (dh + dl) * (v.x + v.y) ----
__device__ __forceinline__ void dacc_first(float &s, float &c, float dh, float dl, float2 v) {
  s = __fmul_rn(dh, v.x);
  float e = __fmaf_rn(dh, v.x, -s);
  e = __fmaf_rn(dh, v.y, e);
  c = __fmaf_rn(dl, v.x, e);
}

__device__ __forceinline__ void dacc(float &s, float &c, float dh, float dl, float2 v) {
  const float p = __fmul_rn(dh, v.x);
  float e = __fmaf_rn(dh, v.x, -p);
  e = __fmaf_rn(dh, v.y, e);
  e = __fmaf_rn(dl, v.x, e);
  const float t = __fadd_rn(s, p);  // TwoSum(s, p)
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// (s, c) += v
__device__ __forceinline__ void dadd(float &s, float &c, float2 v) {
  const float t = __fadd_rn(s, v.x);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(v.x, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, v.y));
}

__device__ __forceinline__ float2 dnorm(float s, float c) {
  const float h = __fadd_rn(s, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

// (s1 + c1) + sgn (s2 + c2), normalised
__device__ __forceinline__ float2 dcombine(float s1, float c1, float s2, float c2, bool minus) {
  if (minus) {
    s2 = -s2;
    c2 = -c2;
  }
  const float t = __fadd_rn(s1, s2);
  const float z = __fsub_rn(t, s1);
  const float err = __fadd_rn(__fsub_rn(s1, __fsub_rn(t, z)), __fsub_rn(s2, z));
  return dnorm(t, __fadd_rn(__fadd_rn(c1, c2), err));
}

// v[a] + sgn v[b] as an (unnormalised) pair: TwoSum of the high parts, low parts added
__device__ __forceinline__ float2 dpm(float2 va, float2 vb, bool minus) {
  const float bx = minus ? -vb.x : vb.x, by = minus ? -vb.y : vb.y;
  const float t = __fadd_rn(va.x, bx);
  const float z = __fsub_rn(t, va.x);
  const float err = __fadd_rn(__fsub_rn(va.x, __fsub_rn(t, z)), __fsub_rn(bx, z));
  return make_float2(t, __fadd_rn(__fadd_rn(va.y, by), err));
}

template <int NP>
struct DPair {
  float hi[NP * NP], lo[NP * NP];  // D[i][m] at i * NP + m
};

// Even-odd form of a centro-antisymmetric line operator M (M[N-i][N-m] = -M[i][m], true for the
// GLL derivative matrix and its transpose): with e_m = v_m + v_{N-m}, o_m = v_m - v_{N-m} (m < H),
//   p_i = sum_m A+[i][m] o_m,  q_i = sum_m A-[i][m] e_m,  out_i = p_i + q_i,  out_{N-i} = p_i - q_i,
// A+-[i][m] = (M[i][m] +- M[N-i][m]) / 2, H = n / 2.  Two H x H products replace one n x n
// product; for odd n the middle node adds one column and one row of H terms (see df_line).
template <int NP>
struct EvenOdd {
  static constexpr int H = NP / 2 > 0 ? NP / 2 : 1;
  float aph[H * H], apl[H * H], amh[H * H], aml[H * H];  // forward (M = D)
  float bph[H * H], bpl[H * H], bmh[H * H], bml[H * H];  // transposed (M = D^T)
};

template <int NP>
struct EmuParams {
  int64_t E;
  int sx, sy, sz;
  int64_t gxs, gys, gzs;
  int bc;
  const double *u;
  double *y;
  const float *Gf;  // [E][gs12]: factor f hi at 2f n3 + p, lo at (2f+1) n3 + p
  int64_t gs;
  const float *wJa;  // [E][2][n3] or NULL
  const int32_t *glo;
  const uint8_t *mask;
  double *partials;
  double *gpartials;
  unsigned int *gtickets;
  SemScalars *scal;
  int *err;             // set to 1 if a bounded wait gave up
  uint32_t wait_polls;  // polls of the staged copy's barrier before the wait gives up
  DPair<NP> D;
  EvenOdd<NP> EO;
};

// out = M v for one line, M = D (TRANS false) or D^T (TRANS true), in double-float
template <int NP, bool TRANS>
__device__ __forceinline__ void df_line(const EmuParams<NP> &P, const float2 (&v)[NP], float2 (&out)[NP]) {
  if constexpr (NP % 2 == 0) {
    constexpr int H = NP / 2;
    const float *aph = TRANS ? P.EO.bph : P.EO.aph, *apl = TRANS ? P.EO.bpl : P.EO.apl;
    const float *amh = TRANS ? P.EO.bmh : P.EO.amh, *aml = TRANS ? P.EO.bml : P.EO.aml;
    float2 ev[H], od[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      ev[m] = dpm(v[m], v[NP - 1 - m], false);
      od[m] = dpm(v[m], v[NP - 1 - m], true);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
      float sp, cp, sq, cq;
      dacc_first(sp, cp, aph[i * H], apl[i * H], od[0]);
      dacc_first(sq, cq, amh[i * H], aml[i * H], ev[0]);
#pragma unroll
      for (int m = 1; m < H; ++m) {
        dacc(sp, cp, aph[i * H + m], apl[i * H + m], od[m]);
        dacc(sq, cq, amh[i * H + m], aml[i * H + m], ev[m]);
      }
      out[i] = dcombine(sp, cp, sq, cq, false);
      out[NP - 1 - i] = dcombine(sp, cp, sq, cq, true);
    }
  } else if constexpr (NP >= 3) {
    // odd n: the same pairs around the middle node mid = N / 2, plus its own terms: M[i][mid] v_mid
    // joins q_i (mirrored with a sign like q), and the middle row, M[mid][mid] = 0 and
    // M[mid][N-m] = -M[mid][m], is sum_m M[mid][m] o_m
    constexpr int H = NP / 2, MID = NP / 2;
    const float *aph = TRANS ? P.EO.bph : P.EO.aph, *apl = TRANS ? P.EO.bpl : P.EO.apl;
    const float *amh = TRANS ? P.EO.bmh : P.EO.amh, *aml = TRANS ? P.EO.bml : P.EO.aml;
    const float *Dh = P.D.hi, *Dl = P.D.lo;
    float2 ev[H], od[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      ev[m] = dpm(v[m], v[NP - 1 - m], false);
      od[m] = dpm(v[m], v[NP - 1 - m], true);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
      float sp, cp, sq, cq;
      dacc_first(sp, cp, aph[i * H], apl[i * H], od[0]);
      dacc_first(sq, cq, amh[i * H], aml[i * H], ev[0]);
#pragma unroll
      for (int m = 1; m < H; ++m) {
        dacc(sp, cp, aph[i * H + m], apl[i * H + m], od[m]);
        dacc(sq, cq, amh[i * H + m], aml[i * H + m], ev[m]);
      }
      const int qm = TRANS ? MID * NP + i : i * NP + MID;  // M[i][mid]
      dacc(sq, cq, Dh[qm], Dl[qm], v[MID]);
      out[i] = dcombine(sp, cp, sq, cq, false);
      out[NP - 1 - i] = dcombine(sp, cp, sq, cq, true);
    }
    float s, c;
    dacc_first(s, c, Dh[TRANS ? MID : MID * NP], Dl[TRANS ? MID : MID * NP], od[0]);
#pragma unroll
    for (int m = 1; m < H; ++m) {
      const int q = TRANS ? m * NP + MID : MID * NP + m;  // M[mid][m]
      dacc(s, c, Dh[q], Dl[q], od[m]);
    }
    out[MID] = dnorm(s, c);
  }
}

__host__ __device__ constexpr int emu_eb(int NP) {
  return NP <= 2 ? 32 : NP == 3 ? 14 : NP == 4 ? 8 : NP == 5 ? 5 : NP == 6 ? 3 : NP <= 8 ? 2 : 1;
}

template <int NP>
struct EmuCfg {
  static constexpr int NP2 = NP * NP, NP3 = NP2 * NP, EB = emu_eb(NP), NT = NP2 * EB;
  static constexpr int RS = NP | 1, PS = NP * RS, BUF = NP * PS;
  static constexpr int GS = (12 * NP3 + 3) / 4 * 4;  // factor block of one element (floats)
  // the factor block can be staged in shared memory by one bulk (TMA) copy when it fits
  static constexpr bool STAGE_FITS = (size_t)EB * (GS * sizeof(float) + 3 * BUF * sizeof(float2)) <= 112 * 1024;
  // byte offsets: [factor block (TMA, offset 0)] [value buffers] [reduction slots, mbarrier]
  static constexpr size_t buf_off(bool stage) { return stage ? (size_t)EB * GS * sizeof(float) : 0; }
  static constexpr size_t red_off(bool stage) {
    return (buf_off(stage) + (size_t)EB * 3 * BUF * sizeof(float2) + 15) / 16 * 16;
  }
  // reduction slots (32 doubles), mbarrier, flag, per-element exponent maxima (EB ints)
  static constexpr size_t smem(bool stage) { return red_off(stage) + 32 * 8 + 16 + 16 + (size_t)EB * 4; }
};

// blocks per SM the register allocation is held to at high order (one element per block would
// otherwise leave one or two blocks on an SM); 0 = no floor (an explicit 1 lets the compiler take
// far more registers, and at N = 7 a floor of 5 or 6 blocks measured slower than none)
__host__ __device__ constexpr int emu_min_blocks(int NP) {
  return NP == 10 ? 4 : NP == 11 ? 3 : NP >= 12 ? 2 : 0;
}

// DOT: the fused (u, y) reduction of the CG step (pAp) is compiled in and runs when P.partials is
// set.  Plain applies use DOT = false (no reduction code; 5-10% faster from N = 8 on) except at
// N = 7, where the kernel that carries the code measured 6% faster (it is scheduled differently).
__host__ __device__ constexpr bool emu_plain_has_dot(int NP) { return NP == 8; }

// How the line products of phases 1 and 3 are laid out in code: 0 three inlined line products per
// phase; 2 the r- and s-lines through one loop body, the t-line (the thread's column, in
// registers) inlined; 3 all three directions through one loop body (the t-line read from shared
// memory).  The loops shorten the code (fewer instruction-fetch stalls) at some addressing cost.
// Measured on GB300 (GDOF/s; 64^3 mesh, 48^3 at N = 12..14; forms 0 / 2 / 3): N = 3 56 / 57.2 /
// 52, 5 41.1 / 42.5 / 41, 7 38.5 / 43.7 / 40.4, 8 28.5 / 33.2 / 30.0, 9 28.7 / 28.5 / 22,
// 10 31.0 / 33.6 / 26.0, 11 15.6 / 21.0 / 18.4, 12 16.7 / 20.6 / 20.4, 13 17.0 / 11.3 / 17.1,
// 14 15.1 / 10.3 / 16.9, 15 11.6 / 9.2 / 18.0.
__host__ __device__ constexpr int emu_loop_mode(int NP) {
  return (NP == 4 || NP == 6 || NP == 8 || NP == 9 || NP == 11 || NP == 12 || NP == 13) ? 2 : NP >= 14 ? 3 : 0;
}

template <int NP, bool BOXM, bool STAGE, bool DOT>
__global__ void __launch_bounds__(EmuCfg<NP>::NT, emu_min_blocks(NP)) k_apply_emu(const EmuParams<NP> P) {
  using C = EmuCfg<NP>;
  constexpr int N = NP - 1, NP2 = C::NP2, NP3 = C::NP3, EB = C::EB, NT = C::NT, RS = C::RS, PS = C::PS,
                BUF = C::BUF, GS = C::GS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  static_assert(C::buf_off(STAGE) % 16 == 0 && C::red_off(STAGE) % 16 == 0, "shared-memory alignment");
  float *sG = reinterpret_cast<float *>(smem_raw);  // TMA destination: 16-byte aligned at offset 0
  float2 *sbuf = reinterpret_cast<float2 *>(smem_raw + C::buf_off(STAGE));
  double *s_red = reinterpret_cast<double *>(smem_raw + C::red_off(STAGE));
  uint64_t *bar = reinterpret_cast<uint64_t *>(s_red + 32);
  int *s_flag = reinterpret_cast<int *>(bar + 1);
  int *s_emax = s_flag + 4;  // [EB] largest biased FP64 exponent of each element's u

  if (DOT && P.partials && (P.scal->converged || P.scal->breakdown)) return;
  const int tid = threadIdx.x;
  const int es = tid / NP2, t2 = tid - es * NP2, a = t2 % NP, b = t2 / NP;
  if (t2 == 0) s_emax[es] = 1;
  const int64_t e0 = (int64_t)blockIdx.x * EB;
  const int64_t e = e0 + es;
  const bool active = e < P.E;
  float2 *su = sbuf + es * 3 * BUF, *sr = su + BUF, *ss = sr + BUF;
  if constexpr (STAGE) {
    if (tid == 0) mbar_init(bar, 1);
  }
  __syncthreads();  // s_emax initialised (and the mbarrier)
  if constexpr (STAGE) {
    if (tid == 0) {
      const int64_t nel = (P.E - e0) < EB ? (P.E - e0) : EB;
      tma_load_1d(sG, P.Gf + e0 * P.gs, (uint32_t)(nel * P.gs * sizeof(float)), bar);
    }
  }

  // ---- phase 0: gather and split u ----
  int64_t gbase = 0;
  uint32_t dirbits = 0;
  float2 uc[NP];
  double ud[NP];
  if constexpr (BOXM) {
    const int64_t plane = P.gxs * P.gys;
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
  // element scale: the largest exponent over the element's gathered values
  {
    int emx = 1;
#pragma unroll
    for (int k = 0; k < NP; ++k) emx = max(emx, f64_biased_exp(ud[k]));
    element_max(&s_emax[es], emx, es);
  }
  __syncthreads();
  const int shift = 1023 - s_emax[es];  // u * 2^shift has its element maximum in [1, 2)
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    uc[k] = split_f64(ud[k], shift);
    su[k * PS + b * RS + a] = uc[k];
  }
  __syncthreads();

  // ---- phase 1: gradients ----
  float2 wt[NP];
  if constexpr (emu_loop_mode(NP) == 3) {
    // direction 0: the r-line (j = a, k = b) into sr, 1: the s-line (i = a, k = b) into ss, 2: the
    // t-line (the column) into registers; the same base and stride address input and output
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      const int ib = dir == 0 ? b * PS + a * RS : dir == 1 ? b * PS + a : b * RS + a;
      const int is = dir == 0 ? 1 : dir == 1 ? RS : PS;
      float2 row[NP], out[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = su[ib + m * is];
      df_line<NP, false>(P, row, out);
      if (dir == 2) {
#pragma unroll
        for (int k = 0; k < NP; ++k) wt[k] = out[k];
      } else {
        float2 *dst = dir == 0 ? sr : ss;
#pragma unroll
        for (int i = 0; i < NP; ++i) dst[ib + i * is] = out[i];
      }
    }
  } else if constexpr (emu_loop_mode(NP) == 2) {
    // the t-line (the column, in registers) inlined; the r-line (j = a, k = b) into sr and the
    // s-line (i = a, k = b) into ss through one loop body (the same base and stride address input
    // and output)
    df_line<NP, false>(P, uc, wt);  // u_t of the column
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      const int ib = dir == 0 ? b * PS + a * RS : b * PS + a;
      const int is = dir == 0 ? 1 : RS;
      float2 *dst = dir == 0 ? sr : ss;
      float2 row[NP], out[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = su[ib + m * is];
      df_line<NP, false>(P, row, out);
#pragma unroll
      for (int i = 0; i < NP; ++i) dst[ib + i * is] = out[i];
    }
  } else {
    df_line<NP, false>(P, uc, wt);  // u_t of the column
    float2 row[NP], out[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = su[b * PS + a * RS + m];
    df_line<NP, false>(P, row, out);
#pragma unroll
    for (int i = 0; i < NP; ++i) sr[b * PS + a * RS + i] = out[i];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = su[b * PS + m * RS + a];
    df_line<NP, false>(P, row, out);
#pragma unroll
    for (int j = 0; j < NP; ++j) ss[b * PS + j * RS + a] = out[j];
  }

  // ---- phase 2: geometric factors ----
  bool ok = true;
  if constexpr (STAGE) ok = mbar_wait(bar, 0, P.wait_polls);
  if (__syncthreads_or(!ok)) {
    // record the timeout, wait (bounded) for this block's own copy, leave without scattering
    if (tid == 0) {
      if (P.err) atomicOr(P.err, 1);
      mbar_wait(bar, 0);
    }
    return;
  }
  const float *Ge = STAGE ? (sG + es * GS + t2) : (P.Gf + (active ? e : 0) * P.gs + t2);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = k * PS + b * RS + a;
    const int o = k * NP2;
    float gh[6], gl[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      gh[f] = (STAGE || active) ? Ge[(2 * f) * NP3 + o] : 0.f;
      gl[f] = (STAGE || active) ? Ge[(2 * f + 1) * NP3 + o] : 0.f;
    }
    const float2 ur = sr[q], us = ss[q], ut = wt[k];
    float s, c;
    dacc_first(s, c, gh[0], gl[0], ur);
    dacc(s, c, gh[1], gl[1], us);
    dacc(s, c, gh[2], gl[2], ut);
    sr[q] = dnorm(s, c);
    dacc_first(s, c, gh[1], gl[1], ur);
    dacc(s, c, gh[3], gl[3], us);
    dacc(s, c, gh[4], gl[4], ut);
    ss[q] = dnorm(s, c);
    dacc_first(s, c, gh[2], gl[2], ur);
    dacc(s, c, gh[4], gl[4], us);
    dacc(s, c, gh[5], gl[5], ut);
    wt[k] = dnorm(s, c);
  }
  float2 yt[NP];
  if constexpr (emu_loop_mode(NP) == 3) {
    __syncthreads();
    // ---- phase 3: transposed contractions: 0 the r-line of sr, 1 the s-line of ss (in place),
    // 2 the column w_t in registers ----
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      const int ib = dir == 0 ? b * PS + a * RS : dir == 1 ? b * PS + a : 0;
      const int is = dir == 0 ? 1 : dir == 1 ? RS : 0;
      float2 *buf = dir == 1 ? ss : sr;
      float2 row[NP], out[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = dir == 2 ? wt[m] : buf[ib + m * is];
      df_line<NP, true>(P, row, out);
      if (dir == 2) {
#pragma unroll
        for (int k = 0; k < NP; ++k) yt[k] = out[k];
      } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) buf[ib + i * is] = out[i];
      }
    }
  } else if constexpr (emu_loop_mode(NP) == 2) {
    df_line<NP, true>(P, wt, yt);  // D^T w_t of the column
    __syncthreads();
    // ---- phase 3: transposed contractions: 0 the r-line of sr, 1 the s-line of ss (in place) ----
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      const int ib = dir == 0 ? b * PS + a * RS : b * PS + a;
      const int is = dir == 0 ? 1 : RS;
      float2 *buf = dir == 0 ? sr : ss;
      float2 row[NP], out[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = buf[ib + m * is];
      df_line<NP, true>(P, row, out);
#pragma unroll
      for (int i = 0; i < NP; ++i) buf[ib + i * is] = out[i];
    }
  } else {
    df_line<NP, true>(P, wt, yt);  // D^T w_t of the column
    __syncthreads();

    // ---- phase 3: transposed r and s contractions ----
    float2 row[NP], out[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + a * RS + m];
    df_line<NP, true>(P, row, out);
#pragma unroll
    for (int i = 0; i < NP; ++i) sr[b * PS + a * RS + i] = out[i];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = ss[b * PS + m * RS + a];
    df_line<NP, true>(P, row, out);
#pragma unroll
    for (int j = 0; j < NP; ++j) ss[b * PS + j * RS + a] = out[j];
  }
  __syncthreads();

  // ---- phase 4: assemble, convert to FP64, scatter ----
  float dps = 0.f, dpc = 0.f;  // (u, y) of this column, double-float
  const int64_t plane = P.gxs * P.gys;
  const bool ij_interior = (a > 0) && (a < N) && (b > 0) && (b < N) && !P.glo;
  const double unscale = exp2i(-shift);  // undoes the element's scaling of u (exact)
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = k * PS + b * RS + a;
    float s = yt[k].x, c = yt[k].y;
    dadd(s, c, sr[q]);
    dadd(s, c, ss[q]);
    if (P.wJa && active) {
      const int64_t o = e * 2 * NP3 + t2 + NP2 * k;
      dacc(s, c, P.wJa[o], P.wJa[o + NP3], uc[k]);
    }
    const float2 yk = dnorm(s, c);
    if ((dirbits >> k) & 1u) continue;
    if (DOT && P.partials) dacc(dps, dpc, uc[k].x, uc[k].y, yk);
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
    const double yd = df_to_f64(yk) * unscale;
    if (ij_interior && k > 0 && k < N)
      P.y[g] = yd;
    else
      atomicAdd(P.y + g, yd);
  }

  if (DOT && P.partials) {
    // (u, y) of the scaled values carries the element's scale twice
    const double bs = block_sum<NT>(df_to_f64(dnorm(dps, dpc)) * unscale * unscale, s_red);
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

template <int NP, bool BOXM, bool STAGE, bool DOT>
sem_status launch_k(const EmuParams<NP> &p, unsigned grid, cudaStream_t s) {
  using C = EmuCfg<NP>;
  static std::atomic<unsigned long long> attr_done;
  const cudaError_t e = set_smem_limit_once(k_apply_emu<NP, BOXM, STAGE, DOT>, C::smem(STAGE), attr_done);
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("emu attributes: ") + cudaGetErrorString(e));
  k_apply_emu<NP, BOXM, STAGE, DOT><<<grid, C::NT, C::smem(STAGE), s>>>(p);
  return SEM_OK;
}

template <int NP, bool STAGE>
sem_status launch_b(const EmuParams<NP> &p, bool boxm, bool dot, unsigned grid, cudaStream_t s) {
  if (dot || emu_plain_has_dot(NP))
    return boxm ? launch_k<NP, true, STAGE, true>(p, grid, s) : launch_k<NP, false, STAGE, true>(p, grid, s);
  return boxm ? launch_k<NP, true, STAGE, false>(p, grid, s) : launch_k<NP, false, STAGE, false>(p, grid, s);
}

template <int NP>
sem_status launch_emu(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal,
                      cudaStream_t s) {
  using C = EmuCfg<NP>;
  EmuParams<NP> p;
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
  p.Gf = h->Gemu;
  p.gs = h->gs12;
  p.wJa = h->wJaemu;
  p.glo = h->structured ? nullptr : h->glo;
  p.mask = h->mask;
  p.partials = partials;
  p.gpartials = h->gpartials;
  p.gtickets = h->gtickets;
  p.scal = scal;
  p.err = &h->scal->error;
  p.wait_polls = h->wait_polls;
  for (int q = 0; q < NP * NP; ++q) {
    p.D.hi[q] = h->Dhih[q];
    p.D.lo[q] = h->Dloh[q];
  }
  constexpr int H = EvenOdd<NP>::H;
  auto split = [](double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  };
  for (int i = 0; i < H && NP >= 2; ++i)  // pairs (i, N - i), i < H = n / 2, for even and odd n
    for (int m = 0; m < H; ++m) {
      const double *D = h->D64h;
      const int N = NP - 1;
      split(0.5 * (D[i * NP + m] + D[(N - i) * NP + m]), p.EO.aph[i * H + m], p.EO.apl[i * H + m]);
      split(0.5 * (D[i * NP + m] - D[(N - i) * NP + m]), p.EO.amh[i * H + m], p.EO.aml[i * H + m]);
      split(0.5 * (D[m * NP + i] + D[m * NP + (N - i)]), p.EO.bph[i * H + m], p.EO.bpl[i * H + m]);
      split(0.5 * (D[m * NP + i] - D[m * NP + (N - i)]), p.EO.bmh[i * H + m], p.EO.bml[i * H + m]);
    }
  const unsigned grid = (unsigned)((p.E + C::EB - 1) / C::EB);
  if (partials && grid > SEM_MAX_PARTIALS) return sem_fail(SEM_ERR_INVALID, "too many elements for fused dot");
  if (partials && !scal) return sem_fail(SEM_ERR_INVALID, "fused dot needs the solver scalars");
  const bool boxm = p.glo == nullptr && p.bc != SEM_BC_MASK;
  // variant 0: factor block staged by TMA when it fits; other variants read factors directly;
  // automatic (-1): direct reads, except at N = 5 where staging measured faster on GB300
  const int variant = h->apply_variant < 0 ? (NP == 6 ? 0 : 1) : h->apply_variant;
  const bool stage = C::STAGE_FITS && variant == 0;
  sem_status st;
  st = stage ? launch_b<NP, C::STAGE_FITS>(p, boxm, partials != nullptr, grid, s)
             : launch_b<NP, false>(p, boxm, partials != nullptr, grid, s);
  if (st != SEM_OK) return st;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("emu apply launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}

}  // namespace semu
