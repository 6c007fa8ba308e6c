// FP64-accurate operator apply in double-float arithmetic (SEM_FP64_EMU).
//
// Same operator and the same five-phase element schedule as the FP64/FP32 kernel
// (sem_apply_kernel.cuh; arXiv 1403.0968 §4.2.1, sum-factorised stiffness display), but every
// value is carried as an unevaluated pair of FP32 numbers (hi, lo) with |lo| <= ulp(hi)/2, because
// GB300 executes FP64 FMAs at 1/61 of the FP32 rate.  Inputs and outputs stay FP64:
//   * u (FP64) is split into (hi, lo) by bit manipulation: hi keeps the top 24 significand bits,
//     lo the next 24 (so the split costs integer instructions, not FP64 conversions);
//   * the factors are stored as (hi, lo) pairs by set-up, D as (hi, lo) launch parameters;
//   * each sum  sum_m a_m b_m  is formed with exact products (p = a_hi b_hi and its FMA
//     remainder, the published TwoProduct transformation) and Knuth's TwoSum on the high parts;
//     every low-order term goes into one FP32 compensation, and the pair is renormalised at the
//     end (Fast2Sum).  The error is about 2^-44 of the sum of |terms| per output (double-float
//     accuracy after Dekker 1971 / Ogita-Rump-Oishi 2005);
//   * y = hi + lo is rebuilt as FP64 (one FP64 add per node) and scatter-added with FP64 atomics.
// Values must lie in the FP32 normal range (about 1.2e-38 .. 3.4e38); smaller inputs are flushed
// to zero (absolute error below 1.2e-38).
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sem_internal.h"
#include "sem_reduce.cuh"

namespace {

// ---- double <-> double-float conversions (integer pipeline) ----
__device__ __forceinline__ float2 split_f64(double u) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(u);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const int ex = (int)((hw >> 20) & 0x7FFu);
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

template <int NP>
struct DPair {
  float hi[NP * NP], lo[NP * NP];  // D[i][m] at i * NP + m
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
  SemScalars *scal;
  DPair<NP> D;
};

__host__ __device__ constexpr int emu_eb(int NP) {
  return NP <= 2 ? 32 : NP == 3 ? 14 : NP == 4 ? 8 : NP == 5 ? 5 : NP == 6 ? 3 : NP <= 8 ? 2 : 1;
}

template <int NP>
struct EmuCfg {
  static constexpr int NP2 = NP * NP, NP3 = NP2 * NP, EB = emu_eb(NP), NT = NP2 * EB;
  static constexpr int RS = NP | 1, PS = NP * RS, BUF = NP * PS;
  static constexpr size_t SMEM = (size_t)EB * 4 * BUF * sizeof(float2) + 32 * 8 + 16;
};

template <int NP, bool BOXM>
__global__ void __launch_bounds__(EmuCfg<NP>::NT) k_apply_emu(const EmuParams<NP> P) {
  using C = EmuCfg<NP>;
  constexpr int N = NP - 1, NP2 = C::NP2, NP3 = C::NP3, EB = C::EB, NT = C::NT, RS = C::RS, PS = C::PS,
                BUF = C::BUF;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2 *sbuf = reinterpret_cast<float2 *>(smem_raw);
  double *s_red = reinterpret_cast<double *>(sbuf + EB * 4 * BUF);
  int *s_flag = reinterpret_cast<int *>(s_red + 32);

  if (P.scal && (P.scal->converged || P.scal->breakdown)) return;
  const int tid = threadIdx.x;
  const int es = tid / NP2, t2 = tid - es * NP2, a = t2 % NP, b = t2 / NP;
  const int64_t e = (int64_t)blockIdx.x * EB + es;
  const bool active = e < P.E;
  float2 *su = sbuf + es * 4 * BUF, *sr = su + BUF, *ss = sr + BUF, *s4 = ss + BUF;
  const float *Dh = P.D.hi, *Dl = P.D.lo;

  // ---- phase 0: gather and split u ----
  int64_t gbase = 0;
  uint32_t dirbits = 0;
  float2 uc[NP];
  if constexpr (BOXM) {
    const int64_t plane = P.gxs * P.gys;
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
    const double *up = P.u + gbase;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      uc[k] = ((dirbits >> k) & 1u) ? make_float2(0.f, 0.f) : split_f64(up[k * plane]);
      su[k * PS + b * RS + a] = uc[k];
    }
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
      uc[k] = d ? make_float2(0.f, 0.f) : split_f64(P.u[g]);
      su[k * PS + b * RS + a] = uc[k];
    }
  }
  __syncthreads();

  // ---- phase 1: gradients ----
  float2 wt[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    float s, c;
    dacc_first(s, c, Dh[k * NP], Dl[k * NP], uc[0]);
#pragma unroll
    for (int m = 1; m < NP; ++m) dacc(s, c, Dh[k * NP + m], Dl[k * NP + m], uc[m]);
    wt[k] = dnorm(s, c);
  }
  {
    float2 row[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = su[b * PS + a * RS + m];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      float s, c;
      dacc_first(s, c, Dh[i * NP], Dl[i * NP], row[0]);
#pragma unroll
      for (int m = 1; m < NP; ++m) dacc(s, c, Dh[i * NP + m], Dl[i * NP + m], row[m]);
      sr[b * PS + a * RS + i] = dnorm(s, c);
    }
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = su[b * PS + m * RS + a];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      float s, c;
      dacc_first(s, c, Dh[j * NP], Dl[j * NP], row[0]);
#pragma unroll
      for (int m = 1; m < NP; ++m) dacc(s, c, Dh[j * NP + m], Dl[j * NP + m], row[m]);
      ss[b * PS + j * RS + a] = dnorm(s, c);
    }
  }
  __syncthreads();

  // ---- phase 2: geometric factors ----
  const float *Ge = P.Gf + (active ? e : 0) * P.gs + t2;
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
  float ych[NP], ycl[NP];  // unnormalised (s, c) of D^T w_t
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    dacc_first(ych[k], ycl[k], Dh[k], Dl[k], wt[0]);
#pragma unroll
    for (int m = 1; m < NP; ++m) dacc(ych[k], ycl[k], Dh[m * NP + k], Dl[m * NP + k], wt[m]);
  }
  __syncthreads();

  // ---- phase 3: transposed r and s contractions ----
  {
    float2 row[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + a * RS + m];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      float s, c;
      dacc_first(s, c, Dh[i], Dl[i], row[0]);
#pragma unroll
      for (int m = 1; m < NP; ++m) dacc(s, c, Dh[m * NP + i], Dl[m * NP + i], row[m]);
      su[b * PS + a * RS + i] = dnorm(s, c);
    }
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = ss[b * PS + m * RS + a];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      float s, c;
      dacc_first(s, c, Dh[j], Dl[j], row[0]);
#pragma unroll
      for (int m = 1; m < NP; ++m) dacc(s, c, Dh[m * NP + j], Dl[m * NP + j], row[m]);
      s4[b * PS + j * RS + a] = dnorm(s, c);
    }
  }
  __syncthreads();

  // ---- phase 4: assemble, convert to FP64, scatter ----
  float dps = 0.f, dpc = 0.f;  // (u, y) of this column, double-float
  const int64_t plane = P.gxs * P.gys;
  const bool ij_interior = (a > 0) && (a < N) && (b > 0) && (b < N) && !P.glo;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = k * PS + b * RS + a;
    float s = ych[k], c = ycl[k];
    dadd(s, c, su[q]);
    dadd(s, c, s4[q]);
    if (P.wJa && active) {
      const int64_t o = e * 2 * NP3 + t2 + NP2 * k;
      dacc(s, c, P.wJa[o], P.wJa[o + NP3], uc[k]);
    }
    const float2 yk = dnorm(s, c);
    if ((dirbits >> k) & 1u) continue;
    if (P.partials) dacc(dps, dpc, uc[k].x, uc[k].y, yk);
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
    const double yd = df_to_f64(yk);
    if (ij_interior && k > 0 && k < N)
      P.y[g] = yd;
    else
      atomicAdd(P.y + g, yd);
  }

  if (P.partials) {
    const double bs = block_sum<NT>(df_to_f64(dnorm(dps, dpc)), s_red);
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
  p.scal = scal;
  for (int q = 0; q < NP * NP; ++q) {
    p.D.hi[q] = h->Dhih[q];
    p.D.lo[q] = h->Dloh[q];
  }
  const unsigned grid = (unsigned)((p.E + C::EB - 1) / C::EB);
  if (partials && grid > SEM_MAX_PARTIALS) return sem_fail(SEM_ERR_INVALID, "too many elements for fused dot");
  const bool boxm = p.glo == nullptr && p.bc != SEM_BC_MASK;
  static bool attr_set[2] = {false, false};
  if (!attr_set[boxm]) {
    cudaError_t e = boxm ? cudaFuncSetAttribute(k_apply_emu<NP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)C::SMEM)
                         : cudaFuncSetAttribute(k_apply_emu<NP, false>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("emu smem attribute: ") + cudaGetErrorString(e));
    attr_set[boxm] = true;
  }
  if (boxm)
    k_apply_emu<NP, true><<<grid, C::NT, C::SMEM, s>>>(p);
  else
    k_apply_emu<NP, false><<<grid, C::NT, C::SMEM, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("emu apply launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}

}  // namespace

sem_status sem_launch_apply_emu(sem_handle *h, const double *u, double *y, double *partials, cudaStream_t s) {
  SemScalars *scal = partials ? h->scal : nullptr;
  switch (h->N) {
#define CASE(NN) \
  case NN:       \
    return launch_emu<NN + 1>(h, u, y, partials, scal, s);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13)
    CASE(14) CASE(15)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID, "order out of range");
  }
}
