// Templated FP64 / FP32 apply kernel (see sem_apply.cu for the algorithm).
//
// Work split inside an element (n = NP nodes per direction, NP^2 threads per element): thread
// (a, b) owns
//   * the t-line (column) (i, j) = (a, b)   — gathered into registers, t-contractions in registers;
//   * the r-line (j, k) = (a, b)            — reads/writes one padded row of a plane buffer;
//   * the s-line (i, k) = (a, b)            — reads/writes one padded column of a plane buffer.
// Every contraction is a fully unrolled line product whose coefficients are launch parameters,
// i.e. constant-bank operands of the FMAs; it uses the centro-antisymmetry of D (line_eo: two
// H x H products on the even and odd parts of the line, H = NP/2) except for FP32 above NP = 12.  Five phases, four barriers per element:
//   0 gather u                        -> su                         (+ TMA of the factor block)
//   1 u_r (r-lines), u_s (s-lines)    -> sr, ss;  u_t in registers
//   2 per node: w = G (u_r, u_s, u_t) -> sr, ss;  w_t in registers, y_t = D^T w_t in registers
//   3 D^T w_r (r-lines) -> sr in place,  D^T w_s (s-lines) -> ss in place (a line is read by
//     its own thread only, so it can be overwritten once it sits in registers)
//   4 y = y_t + sr + ss (+ mass term), masked scatter-add to global y
// Shared plane buffers use an odd row stride so that row, column and plane accesses of a warp
// fall in distinct banks.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <string>

#include "sem_internal.h"
#include "sem_reduce.cuh"
#include "sem_tma.cuh"

template <int NP, typename T>
struct DConst {
  T v[NP * NP];  // D[i][m] at v[i * NP + m]
  // Even-odd form of D (index 0) and D^T (index 1), both centro-antisymmetric
  // (M[N-i][N-m] = -M[i][m]): for i, m < H = NP/2, A = (M[i][m] + M[i][N-m]) / 2,
  // B = (M[i][m] - M[i][N-m]) / 2; for odd NP the middle column C[i] = M[i][H] and the middle
  // row R[m] = M[H][m].
  T A[2][(NP / 2) * (NP / 2)], B[2][(NP / 2) * (NP / 2)], C[2][NP / 2 + 1], R[2][NP / 2 + 1];
};

// y = M v for a centro-antisymmetric NP x NP matrix M given in even-odd form (DConst, index t):
// with e_m = v_m + v_{N-m}, o_m = v_m - v_{N-m} (m < H), P_i = sum_m B_im o_m and
// Q_i = sum_m A_im e_m (+ C_i v_H for odd NP), y_i = P_i + Q_i and y_{N-i} = P_i - Q_i; the middle
// output of odd NP is sum_m R_m o_m (M[H][H] = 0).  2 H^2 products instead of NP^2.
template <int NP, typename T>
__device__ __forceinline__ void line_eo(const DConst<NP, T> &D, int t, const T (&v)[NP], T (&y)[NP]) {
  constexpr int H = NP / 2, N = NP - 1;
  T e[H], o[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    e[m] = v[m] + v[N - m];
    o[m] = v[m] - v[N - m];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T P = T(0), Q = T(0);
#pragma unroll
    for (int m = 0; m < H; ++m) {
      P += D.B[t][i * H + m] * o[m];
      Q += D.A[t][i * H + m] * e[m];
    }
    if constexpr (NP % 2 == 1) Q += D.C[t][i] * v[H];
    y[i] = P + Q;
    y[N - i] = P - Q;
  }
  if constexpr (NP % 2 == 1) {
    T c = T(0);
#pragma unroll
    for (int m = 0; m < H; ++m) c += D.R[t][m] * o[m];
    y[H] = c;
  }
}

// y = M v with M = D (t = 0) or D^T (t = 1): the even-odd form, except for FP32 above NP = 12,
// where the plain product measured faster (register pressure of the split: 64 -> 50 GDOF/s at
// N = 15, against +40% at N = 11 and +25% for FP64)
template <int NP, typename T>
__device__ __forceinline__ void line_apply(const DConst<NP, T> &D, int t, const T (&v)[NP], T (&y)[NP]) {
  if constexpr (sizeof(T) == 4 && NP > 12) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < NP; ++m) acc += (t == 0 ? D.v[i * NP + m] : D.v[m * NP + i]) * v[m];
      y[i] = acc;
    }
  } else {
    line_eo<NP, T>(D, t, v, y);
  }
}

// fills the matrix and its even-odd forms from D in FP64 (row-major, D[i][m] at i * NP + m)
template <int NP, typename T>
__host__ void fill_dconst(DConst<NP, T> &D, const double *Dd) {
  constexpr int H = NP / 2, N = NP - 1;
  for (int q = 0; q < NP * NP; ++q) D.v[q] = (T)Dd[q];
  for (int t = 0; t < 2; ++t) {
    auto M = [&](int i, int m) { return t == 0 ? Dd[i * NP + m] : Dd[m * NP + i]; };
    for (int i = 0; i < H; ++i)
      for (int m = 0; m < H; ++m) {
        D.A[t][i * H + m] = (T)(0.5 * (M(i, m) + M(i, N - m)));
        D.B[t][i * H + m] = (T)(0.5 * (M(i, m) - M(i, N - m)));
      }
    for (int i = 0; i <= H; ++i) {
      D.C[t][i] = (NP % 2 == 1 && i < H) ? (T)M(i, H) : T(0);
      D.R[t][i] = (NP % 2 == 1 && i < H) ? (T)M(H, i) : T(0);
    }
  }
}

template <int NP, typename T>
struct GllConst {
  T x[NP], w[NP];  // GLL points and weights (on-the-fly factors)
};

template <typename T, int NP>
struct ApplyParams {
  int64_t E;
  int sx, sy, sz;
  int64_t gxs, gys, gzs;  // global node counts per direction (structured box)
  int bc;
  const T *u;
  T *y;
  const void *Gf;  // [E][gs] of the factor type (T, or BF16): factor f of node p at f*n3 + p;
                   // OtfGeo: [E][SEM_OTF_STRIDE] map coefficients
  int64_t gs;
  const T *kap;    // OtfGeo: [E][n3] kappa, or NULL for kappa = 1
  const T *wJa;  // [E][n3] or NULL
  const int32_t *glo;
  const uint8_t *mask;
  double *partials;  // non-NULL: fuse p^T A p and the CG step length
  double *gpartials;
  unsigned int *gtickets;
  SemScalars *scal;
  int *err;          // set to 1 if a bounded wait gave up
  uint32_t wait_polls;  // polls of the staged copy's barrier before the wait gives up
  const BatchEntry *batch;  // non-NULL: batched launch over nbatch problems (structured boxes)
  int nbatch;
  double *pAp_batch;        // batched: per-problem p^T A p accumulators (atomic adds)
  DConst<NP, T> D;
  GllConst<NP, T> gll;
};

// default elements per block: about 128 threads
__host__ __device__ constexpr int apply_eb_default(int NP) {
  return NP <= 2 ? 32 : NP == 3 ? 14 : NP == 4 ? 8 : NP == 5 ? 5 : NP == 6 ? 3 : NP <= 8 ? 2 : 1;
}

template <int NP, int EB_ = apply_eb_default(NP)>
struct ApplyCfg {
  static constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  static constexpr int EB = EB_;
  static constexpr int NT = NP2 * EB;
  static constexpr int RS = NP | 1;    // row stride (odd)
  static constexpr int PS = NP * RS;   // plane stride
  static constexpr int BUF = NP * PS;  // one element-sized buffer
  static constexpr int GS = (6 * NP3 + 3) / 4 * 4;
};

// entries between consecutive element factor blocks, as laid out by set-up: 6 n^3 rounded up to a
// multiple of 4 (FP32, FP64: gs6) or of 8 (BF16: gs16), so every block starts on 16 bytes
template <int NP, typename TG>
__host__ __device__ constexpr int factor_stride() {
  return sizeof(TG) == 2 ? (6 * NP * NP * NP + 7) / 8 * 8 : (6 * NP * NP * NP + 3) / 4 * 4;
}

template <typename T, typename TG>
__device__ __forceinline__ T widen(TG v) {
  return (T)v;
}
template <>
__device__ __forceinline__ float widen<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename TG>
__host__ __device__ constexpr bool is_otf() {
  return std::is_same<TG, OtfGeo>::value;
}

// staging the factor block in shared memory is possible when it fits next to the work buffers
// (never for on-the-fly factors: there is no factor block)
template <int NP, typename T, int EB, typename TG = T>
__host__ __device__ constexpr bool apply_stage_fits() {
  using C = ApplyCfg<NP, EB>;
  return !is_otf<TG>() &&
         (size_t)C::EB * (factor_stride<NP, TG>() * sizeof(TG) + 3 * C::BUF * sizeof(T)) <= 112 * 1024;
}

// Per-thread part of the on-the-fly factors for the column (i, j) = (a, b) at r = x_a, s = x_b.
// Along the column only t varies; with J_r = R0 + t R1, J_s = S0 + t S1 and J_t = Tc (constant
// in t, the map being trilinear), the inverse-Jacobian rows scaled by det J are
//   a(t) = J_s x J_t = A0 + t A1,  b(t) = J_t x J_r = B0 + t B1,  c(t) = J_r x J_s = C0 + t C1 + t^2 C2,
// and det J = J_t . c(t) = d0 + t d1 + t^2 d2.  Then G_kl = w kappa (v_k . v_l) / det J with
// (v_r, v_s, v_t) = (a, b, c), so G (u_r, u_s, u_t) = (w kappa / det J) V (V^T (u_r, u_s, u_t)).
struct OtfColumn {
  float A0[3], A1[3], B0[3], B1[3], C0[3], C1[3], C2[3], d0, d1, d2;
};

__device__ __forceinline__ void cross3(const float u[3], const float v[3], float o[3]) {
  o[0] = u[1] * v[2] - u[2] * v[1];
  o[1] = u[2] * v[0] - u[0] * v[2];
  o[2] = u[0] * v[1] - u[1] * v[0];
}

__device__ __forceinline__ OtfColumn otf_column(const float *W, float r, float s) {
  // W: W_r, W_s, W_t, W_rs, W_rt, W_st, W_rst (x, y, z each), 16-byte aligned
  float w[24];
  const float4 *W4 = reinterpret_cast<const float4 *>(W);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float4 v = __ldg(W4 + q);
    w[4 * q] = v.x;
    w[4 * q + 1] = v.y;
    w[4 * q + 2] = v.z;
    w[4 * q + 3] = v.w;
  }
  float R0[3], R1[3], S0[3], S1[3], Tc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float Wr = w[d], Ws = w[3 + d], Wt = w[6 + d], Wrs = w[9 + d], Wrt = w[12 + d], Wst = w[15 + d],
                Wrst = w[18 + d];
    R0[d] = Wr + s * Wrs;
    R1[d] = Wrt + s * Wrst;
    S0[d] = Ws + r * Wrs;
    S1[d] = Wst + r * Wrst;
    Tc[d] = Wt + r * Wrt + s * (Wst + r * Wrst);
  }
  OtfColumn c;
  cross3(S0, Tc, c.A0);
  cross3(S1, Tc, c.A1);
  cross3(Tc, R0, c.B0);
  cross3(Tc, R1, c.B1);
  cross3(R0, S0, c.C0);
  cross3(R1, S1, c.C2);
  float x1[3], x2[3];
  cross3(R0, S1, x1);
  cross3(R1, S0, x2);
#pragma unroll
  for (int d = 0; d < 3; ++d) c.C1[d] = x1[d] + x2[d];
  c.d0 = Tc[0] * c.C0[0] + Tc[1] * c.C0[1] + Tc[2] * c.C0[2];
  c.d1 = Tc[0] * c.C1[0] + Tc[1] * c.C1[1] + Tc[2] * c.C1[2];
  c.d2 = Tc[0] * c.C2[0] + Tc[1] * c.C2[1] + Tc[2] * c.C2[2];
  return c;
}

// byte offset of the reduction slots / mbarrier after the value buffers, 16-byte aligned
template <int NP, typename T, int EB, bool STAGE, typename TG = T>
__host__ __device__ constexpr size_t apply_red_off() {
  using C = ApplyCfg<NP, EB>;
  return ((size_t)C::EB * ((STAGE ? factor_stride<NP, TG>() * sizeof(TG) : 0) + 3 * C::BUF * sizeof(T)) + 15) /
         16 * 16;
}

template <int NP, typename T, int EB, bool STAGE, typename TG = T>
__host__ __device__ constexpr size_t apply_smem() {
  return apply_red_off<NP, T, EB, STAGE, TG>() + 32 * 8 + 16 + 16;
}

// BOXM: structured box numbering with no mask array (bc NONE or BOX): global ids and Dirichlet
// flags follow from the element position, with no per-node branches on the numbering mode.
// Minimum resident blocks the FP32 kernel's registers are held to at high order, where one
// element per block otherwise leaves one or two blocks per SM; 0 = no floor (an explicit 1 lets the
// compiler take more registers).
template <typename T>
__host__ __device__ constexpr int apply_min_blocks(int NP, int EB) {
  return (sizeof(T) == 4 && EB == 1 && NP >= 13 && NP <= 15) ? 2 : 0;  // measured: +15-35% at N = 12..14
}

// FP32 with stored factors at N = 13 and 14 (full line products): the three directions of phases
// 1 and 3 through one loop body instead of three inlined line products (a third of the code, no
// spills).  Measured on GB300 (48^3 mesh, GDOF/s, loop against unrolled): N = 12 80.2 / 89.8,
// 13 77.1 / 47.3, 14 55.6 / 42.4, 15 42.1 / 53.5 (unrolled kept at N = 12 and 15).
template <typename T, typename TG>
__host__ __device__ constexpr bool apply_loop_dirs(int NP) {
  return !is_otf<TG>() && sizeof(T) == 4 && (NP == 14 || NP == 15);
}

// TG: storage type of the factors (T, or BF16 with T = float: half the factor traffic)
template <int NP, typename T, int EB_, bool STAGE, bool BOXM, typename TG = T>
__global__ void __launch_bounds__(ApplyCfg<NP, EB_>::NT, apply_min_blocks<T>(NP, EB_))
    k_apply(const ApplyParams<T, NP> P) {
  using C = ApplyCfg<NP, EB_>;
  constexpr int N = NP - 1, NP2 = C::NP2, NP3 = C::NP3, EB = C::EB, NT = C::NT, RS = C::RS, PS = C::PS,
                BUF = C::BUF, GS = factor_stride<NP, TG>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr size_t RED_OFF = apply_red_off<NP, T, EB_, STAGE, TG>();
  static_assert(RED_OFF % 16 == 0 && ((STAGE ? EB * GS : 0) * sizeof(TG)) % 16 == 0, "shared-memory alignment");
  TG *sG = reinterpret_cast<TG *>(smem_raw);  // TMA destination: 16-byte aligned at offset 0
  T *sbuf = reinterpret_cast<T *>(smem_raw + (STAGE ? EB * GS * sizeof(TG) : 0));
  double *s_red = reinterpret_cast<double *>(smem_raw + RED_OFF);
  uint64_t *bar = reinterpret_cast<uint64_t *>(s_red + 32);
  int *s_flag = reinterpret_cast<int *>(bar + 1);

  // inside a solve: nothing to do once the iteration has stopped (flag set by an earlier launch)
  if (P.scal && (P.scal->converged || P.scal->breakdown)) return;
  const int tid = threadIdx.x;
  const int es = tid / NP2, t2 = tid - es * NP2, a = t2 % NP, b = t2 / NP;
  const int64_t e0 = (int64_t)blockIdx.x * EB;
  const int64_t e = e0 + es;
  const bool active = e < P.E;
  T *su = sbuf + es * 3 * BUF, *sr = su + BUF, *ss = sr + BUF;


  if constexpr (STAGE) {
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    if (tid == 0) {
      const int64_t nel = (P.E - e0) < EB ? (P.E - e0) : EB;
      tma_load_1d(sG, static_cast<const TG *>(P.Gf) + e0 * P.gs, (uint32_t)(nel * P.gs * sizeof(TG)), bar);
    }
  }

  // ---- phase 0: gather u_e = Q M u, column (i, j) = (a, b) ----
  int64_t gbase = 0;
  uint32_t dirbits = 0;  // bit k: node (a, b, k) is a Dirichlet node (or the element is inactive)
  T uc[NP];
  // per-element problem context (single problem, or the problem of this element in a batch)
  int64_t el = e, c_gxs = P.gxs, c_gys = P.gys;
  int c_sx = P.sx, c_sy = P.sy, c_sz = P.sz, c_bc = P.bc, bp = -1;
  const T *c_u = P.u, *c_wJa = P.wJa, *c_kap = P.kap;
  const TG *c_Gf = static_cast<const TG *>(P.Gf);
  T *c_y = P.y;
  if constexpr (BOXM) {
    if (P.batch) {
      // the problem of this element; slots past the last element take entry 0 (valid pointers:
      // the on-the-fly factors are evaluated for every slot, and inactive ones store nothing)
      int lo = 0;
      if (active) {
        int hi = P.nbatch - 1;  // last problem whose first element is <= e
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (P.batch[mid].elem_off <= e) lo = mid; else hi = mid - 1;
        }
      }
      const BatchEntry &B = P.batch[lo];
      bp = active ? B.prob : -1;
      el = active ? e - B.elem_off : 0;
      c_gxs = B.gxs;
      c_gys = B.gys;
      c_sx = B.sx;
      c_sy = B.sy;
      c_sz = B.sz;
      c_bc = B.bc;
      c_u = P.u + B.g_off;
      c_y = P.y + B.g_off;
      c_Gf = static_cast<const TG *>(B.Gf);
      c_wJa = static_cast<const T *>(B.wJa);
      c_kap = static_cast<const T *>(B.kap);
      const bool skip = !active || (B.done && *B.done);
      if (__syncthreads_and(skip)) return;  // every element of this block is finished
    }
  }
  if constexpr (BOXM) {
    const int64_t plane = c_gxs * c_gys;
    if (active) {
      const int64_t ex = el % c_sx, exy = el / c_sx, ey = exy % c_sy, ez = exy / c_sy;
      const int64_t I = ex * N + a, J = ey * N + b;
      gbase = I + c_gxs * (J + c_gys * (ez * N));
      if (c_bc == SEM_BC_BOX) {
        if (I == 0 || I == c_gxs - 1 || J == 0 || J == c_gys - 1) dirbits = (1u << NP) - 1u;
        if (ez == 0) dirbits |= 1u;
        if (ez == c_sz - 1) dirbits |= 1u << N;
      }
    } else {
      dirbits = (1u << NP) - 1u;
    }
    const T *up = c_u + gbase;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      uc[k] = ((dirbits >> k) & 1u) ? T(0) : up[k * plane];
      su[k * PS + b * RS + a] = uc[k];
    }
  } else {
    bool xb = false, yb = false;
    int ez = 0;
    if (active && !P.glo) {
      const int64_t ex = e % P.sx, ey = (e / P.sx) % P.sy;
      ez = (int)(e / ((int64_t)P.sx * P.sy));
      const int64_t I = ex * N + a, J = ey * N + b;
      gbase = I + P.gxs * (J + P.gys * ((int64_t)ez * N));
      xb = (I == 0) || (I == P.gxs - 1);
      yb = (J == 0) || (J == P.gys - 1);
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      int64_t g = 0;
      bool d = !active;
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
      uc[k] = d ? T(0) : P.u[g];
      su[k * PS + b * RS + a] = uc[k];
    }
  }
  __syncthreads();

  // ---- phase 1: gradients ----
  T wt[NP];  // u_t now, w_t after phase 2
  if constexpr (apply_loop_dirs<T, TG>(NP)) {
    // direction 0: the r-line (j = a, k = b) into sr, 1: the s-line (i = a, k = b) into ss, 2: the
    // t-line (the column) into registers; the same base and stride address input and output
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      const int ib = dir == 0 ? b * PS + a * RS : dir == 1 ? b * PS + a : b * RS + a;
      const int is = dir == 0 ? 1 : dir == 1 ? RS : PS;
      T row[NP], out[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = su[ib + m * is];
      line_apply<NP, T>(P.D, 0, row, out);
      if (dir == 2) {
#pragma unroll
        for (int k = 0; k < NP; ++k) wt[k] = out[k];
      } else {
        T *dst = dir == 0 ? sr : ss;
#pragma unroll
        for (int i = 0; i < NP; ++i) dst[ib + i * is] = out[i];
      }
    }
  } else {
    line_apply<NP, T>(P.D, 0, uc, wt);
    T row[NP], out[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = su[b * PS + a * RS + m];  // u(m, j=a, k=b)
    line_apply<NP, T>(P.D, 0, row, out);
#pragma unroll
    for (int i = 0; i < NP; ++i) sr[b * PS + a * RS + i] = out[i];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = su[b * PS + m * RS + a];  // u(i=a, m, k=b)
    line_apply<NP, T>(P.D, 0, row, out);
#pragma unroll
    for (int j = 0; j < NP; ++j) ss[b * PS + j * RS + a] = out[j];
  }
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

  // ---- phase 2: geometric factors, node by node along the column ----
  if constexpr (is_otf<TG>()) {
    static_assert(std::is_same<T, float>::value, "on-the-fly factors are FP32");
    const int64_t eo = active ? el : 0;  // inactive slots evaluate a valid element and store nothing
    const OtfColumn oc =
        otf_column(reinterpret_cast<const float *>(c_Gf) + eo * SEM_OTF_STRIDE, P.gll.x[a], P.gll.x[b]);
    const float wab = P.gll.w[a] * P.gll.w[b];
    const float *kp = c_kap ? c_kap + eo * NP3 + t2 : nullptr;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = k * PS + b * RS + a;
      const float t = P.gll.x[k];
      float av[3], bv[3], cv[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        av[d] = oc.A0[d] + t * oc.A1[d];
        bv[d] = oc.B0[d] + t * oc.B1[d];
        cv[d] = oc.C0[d] + t * (oc.C1[d] + t * oc.C2[d]);
      }
      const float det = oc.d0 + t * (oc.d1 + t * oc.d2);
      float num = wab * P.gll.w[k];
      if (kp) num *= kp[k * NP2];
      const float sc = __fdividef(num, det);
      const float ur = sr[q], us = ss[q], ut = wt[k];
      float qv[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) qv[d] = av[d] * ur + bv[d] * us + cv[d] * ut;
      sr[q] = sc * (av[0] * qv[0] + av[1] * qv[1] + av[2] * qv[2]);
      ss[q] = sc * (bv[0] * qv[0] + bv[1] * qv[1] + bv[2] * qv[2]);
      wt[k] = sc * (cv[0] * qv[0] + cv[1] * qv[1] + cv[2] * qv[2]);
    }
  } else {
    const TG *Ge = STAGE ? (sG + es * GS + t2) : (c_Gf + (active ? el : 0) * P.gs + t2);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = k * PS + b * RS + a;
      const int o = k * NP2;
      T g0 = T(0), g1 = T(0), g2 = T(0), g3 = T(0), g4 = T(0), g5 = T(0);
      if (STAGE || active) {
        g0 = widen<T, TG>(Ge[0 * NP3 + o]);
        g1 = widen<T, TG>(Ge[1 * NP3 + o]);
        g2 = widen<T, TG>(Ge[2 * NP3 + o]);
        g3 = widen<T, TG>(Ge[3 * NP3 + o]);
        g4 = widen<T, TG>(Ge[4 * NP3 + o]);
        g5 = widen<T, TG>(Ge[5 * NP3 + o]);
      }
      const T ur = sr[q], us = ss[q], ut = wt[k];
      sr[q] = g0 * ur + g1 * us + g2 * ut;
      ss[q] = g1 * ur + g3 * us + g4 * ut;
      wt[k] = g2 * ur + g4 * us + g5 * ut;
    }
  }
  T yc[NP];
  if constexpr (apply_loop_dirs<T, TG>(NP)) {
    __syncthreads();
    // ---- phase 3: transposed contractions: 0 the r-line of sr, 1 the s-line of ss (in place),
    // 2 the column w_t in registers ----
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      const int ib = dir == 0 ? b * PS + a * RS : dir == 1 ? b * PS + a : 0;
      const int is = dir == 0 ? 1 : dir == 1 ? RS : 0;
      T *buf = dir == 1 ? ss : sr;
      T row[NP], out[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) row[m] = dir == 2 ? wt[m] : buf[ib + m * is];
      line_apply<NP, T>(P.D, 1, row, out);
      if (dir == 2) {
#pragma unroll
        for (int k = 0; k < NP; ++k) yc[k] = out[k];
      } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) buf[ib + i * is] = out[i];
      }
    }
  } else {
    line_apply<NP, T>(P.D, 1, wt, yc);
    __syncthreads();

    // ---- phase 3: transposed r and s contractions ----
    T row[NP], out[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = sr[b * PS + a * RS + m];  // w_r(m, j=a, k=b)
    line_apply<NP, T>(P.D, 1, row, out);
#pragma unroll
    for (int i = 0; i < NP; ++i) sr[b * PS + a * RS + i] = out[i];
#pragma unroll
    for (int m = 0; m < NP; ++m) row[m] = ss[b * PS + m * RS + a];  // w_s(i=a, m, k=b)
    line_apply<NP, T>(P.D, 1, row, out);
#pragma unroll
    for (int j = 0; j < NP; ++j) ss[b * PS + j * RS + a] = out[j];
  }
  __syncthreads();

  // ---- phase 4: assemble the column and scatter y += M Q^T y_e ----
  T dotp = T(0);
  if constexpr (BOXM) {
    const int64_t plane = c_gxs * c_gys;
    T *yp = c_y + gbase;
    const bool ij_interior = (a > 0) && (a < N) && (b > 0) && (b < N);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = k * PS + b * RS + a;
      T yk = yc[k] + sr[q] + ss[q];
      if (c_wJa && active) yk += c_wJa[el * NP3 + t2 + NP2 * k] * uc[k];
      if ((dirbits >> k) & 1u) continue;
      if (P.partials || P.pAp_batch) dotp += uc[k] * yk;
      if (k > 0 && k < N && ij_interior)
        yp[k * plane] = yk;  // element-interior node: owned by this element alone
      else
        atomicAdd(yp + k * plane, yk);
    }
  } else if (active) {
    const bool ij_interior = (a > 0) && (a < N) && (b > 0) && (b < N) && !P.glo;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if ((dirbits >> k) & 1u) continue;
      const int q = k * PS + b * RS + a;
      T yk = yc[k] + sr[q] + ss[q];
      if (P.wJa) yk += P.wJa[e * NP3 + t2 + NP2 * k] * uc[k];
      const int64_t g = P.glo ? (int64_t)P.glo[e * NP3 + t2 + NP2 * k] : gbase + P.gxs * P.gys * k;
      if (P.partials) dotp += uc[k] * yk;
      if (ij_interior && k > 0 && k < N)
        P.y[g] = yk;
      else
        atomicAdd(P.y + g, yk);
    }
  }

  // ---- batched: per-problem p^T A p, one atomic add per element ----
  if constexpr (BOXM) {
    if (P.pAp_batch) {
      double *s_el = s_red;  // EB <= 32 element slots
      if (tid < EB) s_el[tid] = 0.0;
      __syncthreads();
      if constexpr (NP2 % 32 == 0) {  // every warp lies inside one element
        double v = (double)dotp;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) atomicAdd(&s_el[es], v);
      } else {
        atomicAdd(&s_el[es], (double)dotp);
      }
      __syncthreads();
      if (t2 == 0 && active && bp >= 0) atomicAdd(&P.pAp_batch[bp], s_el[es]);
    }
  }

  // ---- optional fused p^T A p and CG step length ----
  if (P.partials) {
    const double bs = block_sum<NT>((double)dotp, s_red);
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

// largest dynamic shared memory a block may use on sm_103 (227 KB)
#define SEM_MAX_SMEM_PER_BLOCK (227 * 1024)

template <int NP, typename T, int EB, bool STAGE, typename TG = T>
static sem_status launch_apply_v(const ApplyParams<T, NP> &p, cudaStream_t s) {
  using C = ApplyCfg<NP, EB>;
  const unsigned grid = (unsigned)((p.E + C::EB - 1) / C::EB);
  if (p.partials && grid > SEM_MAX_PARTIALS) return sem_fail(SEM_ERR_INVALID, "too many elements for fused dot");
  constexpr size_t smem = apply_smem<NP, T, EB, STAGE, TG>();
  static_assert(smem <= SEM_MAX_SMEM_PER_BLOCK, "apply variant exceeds the shared memory of a block");
  const bool boxm = p.glo == nullptr && p.bc != SEM_BC_MASK;
  static std::atomic<unsigned long long> attr_done[2];
  {
    const cudaError_t e = boxm ? set_smem_limit_once(k_apply<NP, T, EB, STAGE, true, TG>, smem, attr_done[1])
                               : set_smem_limit_once(k_apply<NP, T, EB, STAGE, false, TG>, smem, attr_done[0]);
    if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("apply smem attribute: ") + cudaGetErrorString(e));
  }
  if (boxm)
    k_apply<NP, T, EB, STAGE, true, TG><<<grid, C::NT, smem, s>>>(p);
  else
    k_apply<NP, T, EB, STAGE, false, TG><<<grid, C::NT, smem, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("apply launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}

template <int NP, typename T, int EB>
static sem_status launch_apply_pipe(const ApplyParams<T, NP> &p, cudaStream_t s);
template <int NP, typename T, int EB>
__host__ __device__ constexpr size_t pipe_smem();

// Kernel variants an order can run (the autotuner picks one per problem):
//   0  default elements per block, factor block staged by TMA (when it fits)
//   1  default elements per block, factors read straight from global memory
//   2  twice the elements per block, factors from global memory
//   3  half the elements per block (at least 1), factors staged by TMA (when it fits)
//   4  persistent blocks, next tile's factors double-buffered by TMA and its u prefetched
//      (structured boxes, when two factor blocks fit; otherwise variant 0)
#define SEM_APPLY_VARIANTS 5

// Variant chosen when the handle asks for automatic selection (-1): measured on GB300 over the
// 64^3-element box at N = 3..15 (FP32: factor staging pays from N = 7 on, direct reads win
// below; FP64 is bound by its FMA pipe and indifferent; on-the-fly factors: one element per
// block at N = 3 and N = 6, 7, the default tile elsewhere).
__host__ __device__ constexpr int apply_auto_variant(int NP, bool fp32, bool otf = false) {
  return otf ? ((NP == 4 || NP == 7 || NP == 8) ? 3 : 1) : !fp32 ? 1 : (NP <= 6 ? 1 : NP == 16 ? 2 : 0);
}

template <int NP, typename T, typename TG = T>
static sem_status launch_apply_np(const ApplyParams<T, NP> &p, int variant, cudaStream_t s) {
  if (variant < 0) variant = apply_auto_variant(NP, sizeof(T) == 4, is_otf<TG>());
  constexpr int EB0 = apply_eb_default(NP);
  constexpr int EB2 = (EB0 * 2 * NP * NP <= 1024 &&
                       apply_smem<NP, T, EB0 * 2, false, TG>() <= SEM_MAX_SMEM_PER_BLOCK) ? EB0 * 2 : EB0;
  constexpr int EB3 = EB0 / 2 > 0 ? EB0 / 2 : 1;
  constexpr bool S0 = apply_stage_fits<NP, T, EB0, TG>();
  constexpr bool S3 = apply_stage_fits<NP, T, EB3, TG>();
  switch (variant) {
    case 4:
      if constexpr (std::is_same<T, TG>::value && pipe_smem<NP, T, EB0>() <= SEM_MAX_SMEM_PER_BLOCK) {
        if (p.glo == nullptr && p.bc != SEM_BC_MASK && p.batch == nullptr) return launch_apply_pipe<NP, T, EB0>(p, s);
      }
      return launch_apply_v<NP, T, EB0, S0, TG>(p, s);
    case 1:
      return launch_apply_v<NP, T, EB0, false, TG>(p, s);
    case 2:
      return launch_apply_v<NP, T, EB2, false, TG>(p, s);
    case 3:
      return launch_apply_v<NP, T, EB3, S3, TG>(p, s);
    default:
      return launch_apply_v<NP, T, EB0, S0, TG>(p, s);
  }
}

template <int NP, typename T, typename TG = T>
static sem_status apply_np(const sem_handle *h, const T *u, T *y, const void *Gf, const T *wJa, const T *Dh,
                           double *partials, SemScalars *scal, int *err, cudaStream_t s) {
  ApplyParams<T, NP> p;
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
  p.Gf = Gf;
  p.gs = is_otf<TG>() ? SEM_OTF_STRIDE : sizeof(TG) == 2 ? h->gs16 : h->gs6;
  p.kap = is_otf<TG>() ? reinterpret_cast<const T *>(h->kap32) : nullptr;
  p.wJa = wJa;
  p.glo = h->structured ? nullptr : h->glo;
  p.mask = h->mask;
  p.partials = partials;
  p.gpartials = h->gpartials;
  p.gtickets = h->gtickets;
  p.scal = scal;
  p.err = err;
  p.wait_polls = h->wait_polls;
  p.batch = nullptr;
  p.nbatch = 0;
  p.pAp_batch = nullptr;
  fill_dconst<NP, T>(p.D, h->D64h);
  for (int q = 0; q < NP; ++q) {
    p.gll.x[q] = (T)h->gxh[q];
    p.gll.w[q] = (T)h->gwh[q];
  }
  return launch_apply_np<NP, T, TG>(p, h->apply_variant, s);
}

// Batched launch over structured-box problems of one order: factors read directly (variant 2:
// twice the default elements per block; any other value: the default), per-problem p^T A p
// accumulated into pAp (may be NULL).
template <int NP, typename T, typename TG = T>
static sem_status apply_batch_np(const BatchEntry *d_entries, int nbatch, int64_t total_E, int64_t gs, const T *u,
                                 T *y, const T *Dh, const double *gx, const double *gw, double *pAp, int variant,
                                 cudaStream_t s) {
  ApplyParams<T, NP> p;
  memset(&p, 0, sizeof(p));
  p.E = total_E;
  p.sx = p.sy = p.sz = 1;
  p.gxs = p.gys = p.gzs = 1;
  p.bc = SEM_BC_BOX;
  p.u = u;
  p.y = y;
  p.Gf = nullptr;
  p.gs = gs;
  p.wait_polls = SEM_WAIT_POLLS_DEFAULT;
  p.batch = d_entries;
  p.nbatch = nbatch;
  p.pAp_batch = pAp;
  {
    double Dd[NP * NP];
    for (int q = 0; q < NP * NP; ++q) Dd[q] = (double)Dh[q];
    fill_dconst<NP, T>(p.D, Dd);
  }
  constexpr int EB0 = apply_eb_default(NP);
  constexpr int EB2 = (EB0 * 2 * NP * NP <= 1024 &&
                       apply_smem<NP, T, EB0 * 2, false>() <= SEM_MAX_SMEM_PER_BLOCK) ? EB0 * 2 : EB0;
  for (int q = 0; q < NP; ++q) {  // GLL points and weights (on-the-fly factors)
    p.gll.x[q] = (T)gx[q];
    p.gll.w[q] = (T)gw[q];
  }
  if (variant == 2) return launch_apply_v<NP, T, EB2, false, TG>(p, s);
  return launch_apply_v<NP, T, EB0, false, TG>(p, s);
}

template <typename T, typename TG>
sem_status dispatch_apply_batch(int N, const BatchEntry *d_entries, int nbatch, int64_t total_E, int64_t gs,
                                const T *u, T *y, const T *Dh, const double *gx, const double *gw, double *pAp,
                                int variant, cudaStream_t s) {
  switch (N) {
#define CASE(NN) \
  case NN:       \
    return apply_batch_np<NN + 1, T, TG>(d_entries, nbatch, total_E, gs, u, y, Dh, gx, gw, pAp, variant, s);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13)
    CASE(14) CASE(15)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID, "order out of range");
  }
}

// Instantiated per precision in sem_apply_f32.cu / sem_apply_f64.cu / sem_apply_bf16.cu.
template <typename T, typename TG>
sem_status dispatch_apply(const sem_handle *h, const T *u, T *y, const void *Gf, const T *wJa, const T *Dh,
                          double *partials, SemScalars *scal, int *err, cudaStream_t s) {
  switch (h->N) {
#define CASE(NN) \
  case NN:       \
    return apply_np<NN + 1, T, TG>(h, u, y, Gf, wJa, Dh, partials, scal, err, s);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13)
    CASE(14) CASE(15)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID, "order out of range");
  }
}
