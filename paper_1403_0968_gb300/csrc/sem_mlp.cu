// Learned element-local preconditioner: z = D^-1 r + c(r), where the correction c is a small
// multilayer perceptron that maps the residual restricted to one element (normalised) plus six
// normalised element-mean geometric factors to a correction on that element, assembled by a
// multiplicity-weighted average; used inside flexible CG (sem_pcg mode SEM_SOLVE_FCG_MLP, with
// plain Jacobi as fallback).  The network learns the part of the error that the Jacobi step
// misses, so an untrained (zero) network is exactly Jacobi.
// The paper's PCG (arXiv 1403.0968 §4.2.2) leaves the preconditioner open; this one is learned
// from residual / error pairs that Jacobi-PCG itself produces.
//
// Network: n_in = n^3 + 6 -> h1 -> h2 -> n^3, ReLU after the two hidden layers.  Parameters in
// one FP32 array: W1 [n_in][h1], b1 [h1], W2 [h1][h2], b2 [h2], W3 [h2][n^3], b3 [n^3].
// Training: mean-squared error, backward pass by three GEMMs per layer, Adam (Kingma & Ba), all
// in FP32 on the CUDA cores.  Inference inside the solver runs the layers on the tensor cores
// (sem_tc.cu): weights, features and hidden activations rounded to BF16, FP32 accumulation.
#include <cuda_bf16.h>
#include <math.h>

#include <string>

#include "sem_internal.h"
#include "sem_reduce.cuh"

namespace {

// GB300 runs FP64 instructions (arithmetic, comparisons and conversions) at 1/61 of the FP32
// rate, about two lanes per cycle per SM, which a kernel that converts or compares one FP64 value
// per node already saturates; these conversions and tests use the integer pipeline instead.

// FP64 -> FP32, rounded to nearest even (the result of __double2float_rn) for values in FP32's
// normal range; values below it give zero, values above it, infinities and NaNs take the FP64
// conversion (not expected on these paths)
__device__ __forceinline__ float f64_to_f32_rn(double u) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(u);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const int ex = (int)((hw >> 20) & 0x7FFu);
  if (ex >= 897 && ex <= 1150) {
    // sign | rebiased exponent | significand bits 51..29, then round on bits 28..0 (a carry out of
    // the significand steps the exponent, and past the largest finite value gives infinity)
    unsigned int f = (hw & 0x80000000u) | ((unsigned int)(ex - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const unsigned int rem = lw & 0x1FFFFFFFu, half = 0x10000000u;
    f += (rem > half || (rem == half && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
  }
  if (ex < 897) return __uint_as_float(hw & 0x80000000u);  // below FP32's normal range: signed zero
  return __double2float_rn(u);
}

// FP32 -> FP64 (exact); FP32 subnormals give zero
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int ex = (b >> 23) & 0xFFu;
  if (ex == 0u) return __longlong_as_double((long long)((unsigned long long)(b & 0x80000000u) << 32));
  const unsigned long long e64 = ex == 0xFFu ? 0x7FFull : (unsigned long long)(ex + 896u);
  return __longlong_as_double((long long)(((unsigned long long)(b & 0x80000000u) << 32) | (e64 << 52) |
                                          ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// u == 0.0 (either sign) on the bit pattern
__device__ __forceinline__ bool f64_is_zero(double u) {
  return ((unsigned long long)__double_as_longlong(u) << 1) == 0ull;
}

constexpr int GT = 256;  // threads of the tiled GEMM
constexpr int TM = 64, TN = 64, TK = 16;

// C[M][N] = act(op(A) op(B) + bias) (+ C if accumulate); op(A)[m][k] = TA ? A[k*lda+m] : A[m*lda+k],
// op(B)[k][n] = TB ? B[n*ldb+k] : B[k*ldb+n].  64x64 tile per block, 4x4 outputs per thread.
template <bool TA, bool TB>
__global__ void __launch_bounds__(GT) k_gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                                             const float *bias, float *C, int ldc, int relu, int accumulate) {
  __shared__ float sA[TK][TM + 4];
  __shared__ float sB[TK][TN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int q = threadIdx.x; q < TK * TM; q += GT) {
      const int kk = q / TM, mm = q % TM, m = m0 + mm, k = k0 + kk;
      sA[kk][mm] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
    }
    for (int q = threadIdx.x; q < TK * TN; q += GT) {
      const int kk = q / TN, nn = q % TN, n = n0 + nn, k = k0 + kk;
      sB[kk][nn] = (n < N && k < K) ? (TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      if (accumulate) v += C[(size_t)m * ldc + n];
      C[(size_t)m * ldc + n] = v;
    }
  }
}

template <bool TA, bool TB>
sem_status gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, const float *bias, float *C,
                int ldc, bool relu, bool accumulate, cudaStream_t s) {
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  k_gemm<TA, TB><<<grid, GT, 0, s>>>(M, N, K, A, lda, B, ldb, bias, C, ldc, relu ? 1 : 0, accumulate ? 1 : 0);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

struct Shape {
  int nin, h1, h2, nout;
  int64_t oW1, ob1, oW2, ob2, oW3, ob3, count;
};

Shape shape_of(int n3, int h1, int h2) {
  Shape s;
  s.nin = n3 + 6;
  s.h1 = h1;
  s.h2 = h2;
  s.nout = n3;
  s.oW1 = 0;
  s.ob1 = s.oW1 + (int64_t)s.nin * h1;
  s.oW2 = s.ob1 + h1;
  s.ob2 = s.oW2 + (int64_t)h1 * h2;
  s.oW3 = s.ob2 + h2;
  s.ob3 = s.oW3 + (int64_t)h2 * s.nout;
  s.count = s.ob3 + s.nout;
  return s;
}

// column sums: out[n] (+)= sum_m X[m][n]
__global__ void k_colsum(int M, int N, const float *X, float *out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += X[(size_t)m * N + n];
  out[n] = s;
}

// dH = dH * (H > 0)
__global__ void k_relu_back(int64_t n, float *dH, const float *H) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(H[i] > 0.f)) dH[i] = 0.f;
}

// dO = 2 (O - T) / (B nout), loss partials
__global__ void k_mse(int64_t n, float inv, const float *O, const float *T, float *dO, double *loss) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = O[i] - T[i];
    dO[i] = 2.f * d * inv;
    acc += (double)d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * (double)inv);
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; w -= lr mhat / (sqrt(vhat) + eps)
__global__ void k_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// o[i] = w[i] rounded to BF16 and widened back to FP32
__global__ void k_round_bf16(int64_t n, const float *w, float *o) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = __bfloat162float(__float2bfloat16_rn(w[i]));
}

// Wt[c][k] = W[k][c] in BF16 for k < K, zero for K <= k < ldk (W: K x C row-major FP32 values
// that are already BF16-exact)
__global__ void k_transpose_bf16(int K, int C, int ldk, const float *W, __nv_bfloat16 *Wt) {
  const int64_t n = (int64_t)C * ldk;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / ldk), k = (int)(i - (int64_t)c * ldk);
    Wt[i] = __float2bfloat16_rn(k < K ? W[(size_t)k * C + c] : 0.f);
  }
}

unsigned egrid(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

// global id of local node p of element e (structured box or explicit numbering)
__device__ __forceinline__ int64_t gid(const sem_handle &h, int64_t e, int p) {
  if (h.glo) return h.glo[e * h.n3 + p];
  const int n = h.n, N = h.N;
  const int i = p % n, j = (p / n) % n, k = p / (n * n);
  const int64_t ex = e % h.box[0], ey = (e / h.box[0]) % h.box[1], ez = e / ((int64_t)h.box[0] * h.box[1]);
  const int64_t gxs = (int64_t)h.box[0] * N + 1, gys = (int64_t)h.box[1] * N + 1;
  return (ex * N + i) + gxs * ((ey * N + j) + gys * (ez * N + k));
}

// Inference features of element e: X16[e] = BF16(r_e / |r_e|, geo_e) (rows of h.mlp_ldx with zero
// padding), scale[e] = |r_e| / dbar_e; r_e is zero on Dirichlet nodes.  One warp per element, FP32
// arithmetic (GB300 issues FP64 at 1/61 of the FP32 rate and the result is rounded to BF16 anyway):
// r is rounded to FP32, the norm is a warp reduction, and the second pass re-reads r (cached).
// NP = n is a template parameter so that the node index arithmetic is by constants.
constexpr int FW = 8;  // elements (warps) per block
// r at local node p of element e, zero on Dirichlet nodes.  bmask (structured box with the
// Dirichlet box condition): bit 0/1 the element touches x = 0 / x = 1, bits 2/3 y, bits 4/5 z;
// otherwise the flag comes from the inverse diagonal (zero on Dirichlet nodes).
template <int NP>
__device__ __forceinline__ double feature_value(const sem_handle &h, const double *r, int64_t e, int64_t base,
                                                int64_t gxs, int64_t plane, int p, int bmask) {
  const int i = p % NP, jk = p / NP, j = jk % NP, k = jk / NP;
  const int64_t g = h.glo ? (int64_t)h.glo[e * (NP * NP * NP) + p] : base + i + gxs * j + plane * k;
  if (bmask >= 0) {
    constexpr int N = NP - 1;
    const bool dir = ((bmask & 1) && i == 0) || ((bmask & 2) && i == N) || ((bmask & 4) && j == 0) ||
                     ((bmask & 8) && j == N) || ((bmask & 16) && k == 0) || ((bmask & 32) && k == N);
    return dir ? 0.0 : r[g];
  }
  return h.dinv32[g] != 0.f ? r[g] : 0.0;
}

// Two blocks per SM at least, so that the compiler may keep all of a lane's loads of r in flight
// before the first is used (the kernel waits on those loads, not on arithmetic).
template <int NP>
__global__ void __launch_bounds__(32 * FW, 2) k_mlp_features(sem_handle h, const double *r, __nv_bfloat16 *X16,
                                                             float *scale) {
  constexpr int N3 = NP * NP * NP, N = NP - 1;
  const int lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * FW + (threadIdx.x >> 5);
  if (e >= h.E) return;
  const int ldx = h.mlp_ldx;
  int64_t base = 0, gxs = 0, plane = 0;
  int bmask = -1;
  if (!h.glo) {
    gxs = (int64_t)h.box[0] * N + 1;
    plane = gxs * ((int64_t)h.box[1] * N + 1);
    const int64_t ex = e % h.box[0], exy = e / h.box[0], ey = exy % h.box[1], ez = exy / h.box[1];
    base = ex * N + gxs * (ey * N) + plane * (ez * N);
    if (h.bc == SEM_BC_BOX)
      bmask = (ex == 0 ? 1 : 0) | (ex == h.box[0] - 1 ? 2 : 0) | (ey == 0 ? 4 : 0) | (ey == h.box[1] - 1 ? 8 : 0) |
              (ez == 0 ? 16 : 0) | (ez == h.box[2] - 1 ? 32 : 0);
    else if (h.bc == SEM_BC_NONE)
      bmask = 0;
  }
  float acc = 0.f;
  __nv_bfloat16 *xe = X16 + (size_t)e * ldx;
  constexpr int VPL = (N3 + 31) / 32;  // values per lane
  if constexpr (VPL <= 32) {
    // one pass over r: all of the lane's loads first, then the values stay in registers between
    // the norm and the stores
    double d[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
      const int p = lane + 32 * k;
      d[k] = p < N3 ? feature_value<NP>(h, r, e, base, gxs, plane, p, bmask) : 0.0;
    }
    float vals[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
      vals[k] = f64_to_f32_rn(d[k]);
      acc = fmaf(vals[k], vals[k], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const float inv = acc > 0.f ? 1.f / sqrtf(acc) : 0.f;
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
      const int p = lane + 32 * k;
      if (p < N3) xe[p] = __float2bfloat16_rn(vals[k] * inv);
    }
  } else {
#pragma unroll 4
    for (int p = lane; p < N3; p += 32) {
      const float v = f64_to_f32_rn(feature_value<NP>(h, r, e, base, gxs, plane, p, bmask));
      acc = fmaf(v, v, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const float inv = acc > 0.f ? 1.f / sqrtf(acc) : 0.f;
#pragma unroll 4
    for (int p = lane; p < N3; p += 32)
      xe[p] = __float2bfloat16_rn(f64_to_f32_rn(feature_value<NP>(h, r, e, base, gxs, plane, p, bmask)) * inv);
  }
  const float nrm = sqrtf(acc);
  if (lane < ldx - N3) xe[N3 + lane] = lane < 6 ? __float2bfloat16_rn(h.geo6[e * 6 + lane]) : __float2bfloat16_rn(0.f);
  if (lane == 0) scale[e] = h.mlp_dbar[e] > 0.f ? nrm / h.mlp_dbar[e] : 0.f;
}

// explicit numbering: z[g] += scale_e O[e][p] / multiplicity(g) for every local node (z zeroed
// before; Dirichlet nodes stay zero)
__global__ void k_mlp_scatter(sem_handle h, const float *O, const float *scale, double *z) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h.L) return;
  const int64_t e = q / h.n3;
  const int p = (int)(q - e * h.n3);
  const int64_t g = gid(h, e, p);
  if (h.dinv64[g] == 0.0) return;
  atomicAdd(z + g, (double)scale[e] * (double)O[q] * (double)h.inv_mult[g]);
}

// structured box: z[g] = (1 / multiplicity) sum over the elements containing g of scale_e O[e][p]
// (FP32, fixed order: no atomics, deterministic) plus D^-1 r with the Jacobi base; zero on
// Dirichlet nodes.  One thread per global node (I, J, K) on a 3-D grid (x by blocks of threads, y
// and z by grid rows).  Along each direction a lattice index lies inside one element or, on an
// inner element face, in two: the lower element's local index N and the upper one's 0; the
// multiplicity is 2 per such direction.  J and K are the same for the whole block, so the (y, z)
// element pairs and their row offsets are worked out once per block; each thread adds its one or
// two x-neighbours per pair (order: z lower to upper, then y, then x, as the sum is defined).
template <int NP>
__global__ void __launch_bounds__(128) k_mlp_gather(sem_handle h, const float *__restrict__ O,
                                                    const float *__restrict__ scale, const double *__restrict__ r,
                                                    double *__restrict__ z) {
  constexpr int N = NP - 1, N3 = NP * NP * NP;
  const int sx = h.box[0], sy = h.box[1], sz = h.box[2];
  const int gxs = sx * N + 1, gys = sy * N + 1;
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y, K = blockIdx.z;
  // block-uniform: the (element row, local row) pairs in y and z
  const int eya = J / N < sy ? J / N : sy - 1, ja = J - eya * N;
  const int eza = K / N < sz ? K / N : sz - 1, ka = K - eza * N;
  const bool y2 = ja == 0 && eya > 0, z2 = ka == 0 && eza > 0;
  if (I >= gxs) return;
  const int64_t g = I + (int64_t)gxs * (J + (int64_t)gys * K);
  // both node values are loaded up front, independent of each other and of the element outputs
  // (r is read on Dirichlet nodes too, where it is not used), so that the loads overlap
  const double dv = __ldg(h.dinv64 + g), rv = __ldg(r + g);
  const int exa = I / N < sx ? I / N : sx - 1, ia = I - exa * N;
  const bool x2 = ia == 0 && exa > 0;
  float acc = 0.f;
  // block-uniform trip counts (1 or 2 each): the loops run over the pairs that exist only
#pragma unroll 1
  for (int zc = z2 ? 0 : 1; zc < 2; ++zc) {
    const int ez = zc == 0 ? eza - 1 : eza, iz = zc == 0 ? N : ka;
#pragma unroll 1
    for (int yc = y2 ? 0 : 1; yc < 2; ++yc) {
      const int ey = yc == 0 ? eya - 1 : eya, iy = yc == 0 ? N : ja;
      const int64_t erow = (int64_t)sx * (ey + (int64_t)sy * ez);  // first element of this x row
      const float *Orow = O + erow * N3 + NP * (iy + NP * iz);
      const float *srow = scale + erow;
      if (x2) acc = fmaf(__ldg(srow + exa - 1), __ldg(Orow + (exa - 1) * N3 + N), acc);
      acc = fmaf(__ldg(srow + exa), __ldg(Orow + exa * N3 + ia), acc);
    }
  }
  const float im = (x2 ? 0.5f : 1.f) * (y2 ? 0.5f : 1.f) * (z2 ? 0.5f : 1.f);
  const double c0 = f32_to_f64(acc * im);
  // the one FP64 instruction per node is the Jacobi base's fused multiply-add
  z[g] = f64_is_zero(dv) ? 0.0 : (h.mlp_jacobi_base ? fma(dv, rv, c0) : c0);
}

// z = D^-1 r (Jacobi base) before the scatter of the corrections
__global__ void k_jacobi_base(int64_t G, const double *r, const double *dinv, double *z) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x)
    z[g] = dinv[g] * r[g];
}

// element-mean factors normalised by their mean diagonal: six shape descriptors per element
__global__ void k_geo6(sem_handle h, const double *G64, const float *G32, const float *Gemu, float *geo) {
  __shared__ double s_red[32];
  const int64_t e = blockIdx.x;
  double m[6];
  for (int f = 0; f < 6; ++f) {
    double acc = 0.0;
    for (int p = threadIdx.x; p < h.n3; p += blockDim.x) {
      double v;
      if (G64) v = G64[e * h.gs6 + (int64_t)f * h.n3 + p];
      else if (Gemu) v = (double)Gemu[e * h.gs12 + (int64_t)(2 * f) * h.n3 + p] + Gemu[e * h.gs12 + (int64_t)(2 * f + 1) * h.n3 + p];
      else v = G32[e * h.gs6 + (int64_t)f * h.n3 + p];
      acc += v;
    }
    m[f] = block_sum<256>(acc, s_red) / h.n3;
  }
  const double tr = (m[0] + m[3] + m[5]) / 3.0;
  if (threadIdx.x < 6) geo[e * 6 + threadIdx.x] = tr > 0.0 ? (float)(m[threadIdx.x] / tr) : 0.f;
}

// 1 / (number of elements sharing global node g)
__global__ void k_inv_mult_acc(sem_handle h, float *cnt) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h.L) return;
  const int64_t e = q / h.n3;
  atomicAdd(cnt + gid(h, e, (int)(q - e * h.n3)), 1.f);
}
__global__ void k_inv_mult_fin(int64_t G, float *cnt) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x)
    cnt[g] = cnt[g] > 0.f ? 1.f / cnt[g] : 0.f;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// internal: set-up of the MLP tables (called by sem_setup when SEM_FEAT_MLP is requested)
// ---------------------------------------------------------------------------------------------
sem_status sem_mlp_setup_tables(sem_handle *h, cudaStream_t st) {
  k_geo6<<<(unsigned)h->E, 256, 0, st>>>(*h, h->G64, h->G32, h->Gemu, h->geo6);
  SEM_CUDA_TRY(cudaMemsetAsync(h->inv_mult, 0, (size_t)h->G * 4, st));
  k_inv_mult_acc<<<(unsigned)((h->L + 255) / 256), 256, 0, st>>>(*h, h->inv_mult);
  k_inv_mult_fin<<<egrid(h->G), 256, 0, st>>>(h->G, h->inv_mult);
  SEM_CUDA_TRY(cudaGetLastError());
  return sem_mlp_dbar_table(h, h->mlp_dbar, st);
}

// z = P_mlp(r): BF16 features of every element, the three layers on the tensor cores (BF16
// operands, FP32 accumulation; hidden activations rounded to BF16), weighted scatter.
sem_status sem_mlp_precond_apply(sem_handle *h, const double *r, double *z, cudaStream_t st) {
  NvtxRange nvtx_pre("sem_mlp_precond");
  if (!h->mlp_w) return sem_fail(SEM_ERR_INVALID, "handle was set up without SEM_FEAT_MLP");
  const Shape S = shape_of(h->n3, h->mlp_h1, h->mlp_h2);
  const int E = (int)h->E, ldx = h->mlp_ldx;
  switch (h->n) {
#define SEM_FT(NPV)                                                                                      \
  case NPV:                                                                                            \
    k_mlp_features<NPV><<<(unsigned)((E + FW - 1) / FW), 32 * FW, 0, st>>>(*h, r, h->mlp_X, h->mlp_scale); \
    break;
    SEM_FT(2) SEM_FT(3) SEM_FT(4) SEM_FT(5) SEM_FT(6) SEM_FT(7) SEM_FT(8) SEM_FT(9) SEM_FT(10) SEM_FT(11)
    SEM_FT(12) SEM_FT(13) SEM_FT(14) SEM_FT(15) SEM_FT(16)
#undef SEM_FT
    default:
      return sem_fail(SEM_ERR_INVALID, "unsupported order");
  }
  SEM_CUDA_TRY(cudaGetLastError());
  const __nv_bfloat16 *W1t = h->mlp_w, *W2t = W1t + (size_t)S.h1 * ldx, *W3t = W2t + (size_t)S.h2 * S.h1;
  int *err = &h->scal->error;
  sem_status s;
  if (h->mlp_fused && S.h1 == 256 && S.h2 == 256 && S.nout <= 512 && S.nout % 8 == 0) {
    // one launch: the hidden activations stay in shared memory (same BF16 rounding, same sums)
    if ((s = sem_mlp3_tc(E, S.nin, ldx, S.nout, h->mlp_X, W1t, W2t, W3t, h->mlp_b32 + S.ob1, h->mlp_b32 + S.ob2,
                         h->mlp_b32 + S.ob3, h->mlp_O, err, st)) != SEM_OK)
      return s;
  } else {
    if ((s = sem_gemm_tc(E, S.h1, S.nin, h->mlp_X, ldx, W1t, ldx, h->mlp_b32 + S.ob1, nullptr, h->mlp_H1, S.h1,
                         true, err, st)) != SEM_OK)
      return s;
    if ((s = sem_gemm_tc(E, S.h2, S.h1, h->mlp_H1, S.h1, W2t, S.h1, h->mlp_b32 + S.ob2, nullptr, h->mlp_H2, S.h2,
                         true, err, st)) != SEM_OK)
      return s;
    if ((s = sem_gemm_tc(E, S.nout, S.h2, h->mlp_H2, S.h2, W3t, S.h2, h->mlp_b32 + S.ob3, h->mlp_O, nullptr,
                         S.nout, false, err, st)) != SEM_OK)
      return s;
  }
  if (h->glo) {
    if (h->mlp_jacobi_base)
      k_jacobi_base<<<egrid(h->G), 256, 0, st>>>(h->G, r, h->dinv64, z);
    else
      SEM_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)h->G * sizeof(double), st));
    k_mlp_scatter<<<(unsigned)((h->L + 255) / 256), 256, 0, st>>>(*h, h->mlp_O, h->mlp_scale, z);
  } else {
    const int64_t gx3 = (int64_t)h->box[0] * h->N + 1, gy3 = (int64_t)h->box[1] * h->N + 1,
                  gz3 = (int64_t)h->box[2] * h->N + 1;
    if (gy3 > 65535 || gz3 > 65535) return sem_fail(SEM_ERR_INVALID, "box too large for the gather grid");
    switch (h->n) {
#define SEM_GT(NPV)                                                                                   \
  case NPV:                                                                                         \
    k_mlp_gather<NPV><<<dim3((unsigned)((gx3 + 127) / 128), (unsigned)gy3, (unsigned)gz3), 128, 0, st>>>( \
        *h, h->mlp_O, h->mlp_scale, r, z);                                                          \
    break;
      SEM_GT(2) SEM_GT(3) SEM_GT(4) SEM_GT(5) SEM_GT(6) SEM_GT(7) SEM_GT(8) SEM_GT(9) SEM_GT(10) SEM_GT(11)
      SEM_GT(12) SEM_GT(13) SEM_GT(14) SEM_GT(15) SEM_GT(16)
#undef SEM_GT
      default:
        return sem_fail(SEM_ERR_INVALID, "unsupported order");
    }
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

// ---------------------------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------------------------
extern "C" sem_status sem_mlp_param_count(int32_t N, int32_t h1, int32_t h2, int64_t *count) {
  if (N < 1 || N > SEM_MAX_N || h1 < 1 || h2 < 1 || !count) return sem_fail(SEM_ERR_INVALID, "bad MLP shape");
  const int n = N + 1;
  *count = shape_of(n * n * n, h1, h2).count;
  return SEM_OK;
}

extern "C" sem_status sem_mlp_samples(sem_handle *h, const double *d_r, int32_t nsamp, const int32_t *d_elems,
                                      double eps, int32_t jacobi_base, float *d_X, float *d_T, int32_t *d_iters,
                                      sem_stream_t stream) {
  if (!h || !d_r || !d_elems || !d_X || !d_T || nsamp < 1 || !(eps > 0.0))
    return sem_fail(SEM_ERR_INVALID, "bad arguments");
  if (!h->geo6) return sem_fail(SEM_ERR_INVALID, "handle was set up without SEM_FEAT_MLP");
  return sem_mlp_local_pairs(h, nsamp, d_elems, d_r, eps, SEM_MLP_LOCAL_RTOL, SEM_MLP_LOCAL_MAXIT,
                             jacobi_base ? 1 : 0, d_X, d_T, d_iters, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" sem_status sem_mlp_train_scratch(int32_t N, int32_t h1, int32_t h2, int32_t batch, size_t *bytes) {
  int64_t P;
  sem_status s = sem_mlp_param_count(N, h1, h2, &P);
  if (s != SEM_OK) return s;
  if (batch < 1 || !bytes) return sem_fail(SEM_ERR_INVALID, "bad batch");
  const int n = N + 1, n3 = n * n * n;
  // H1, H2, O, dO, dH2, dH1 activations + gradient + loss
  *bytes = ((size_t)batch * (2 * h1 + 2 * h2 + 2 * n3) + (size_t)P) * 4 + 64;
  return SEM_OK;
}

extern "C" sem_status sem_mlp_forward(int32_t N, int32_t h1, int32_t h2, const float *d_params, const float *d_X,
                                      int32_t batch, float *d_H1, float *d_H2, float *d_O, sem_stream_t stream) {
  int64_t P;
  sem_status s = sem_mlp_param_count(N, h1, h2, &P);
  if (s != SEM_OK) return s;
  if (!d_params || !d_X || !d_H1 || !d_H2 || !d_O || batch < 1) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = N + 1;
  const Shape S = shape_of(n * n * n, h1, h2);
  const float *W = d_params;
  if ((s = gemm<false, false>(batch, S.h1, S.nin, d_X, S.nin, W + S.oW1, S.h1, W + S.ob1, d_H1, S.h1, true,
                                     false, st)) != SEM_OK)
    return s;
  if ((s = gemm<false, false>(batch, S.h2, S.h1, d_H1, S.h1, W + S.oW2, S.h2, W + S.ob2, d_H2, S.h2, true,
                                     false, st)) != SEM_OK)
    return s;
  return gemm<false, false>(batch, S.nout, S.h2, d_H2, S.h2, W + S.oW3, S.nout, W + S.ob3, d_O, S.nout, false,
                                   false, st);
}

extern "C" sem_status sem_mlp_train_step(int32_t N, int32_t h1, int32_t h2, float *d_params, float *d_m, float *d_v,
                                         int32_t step, float lr, const float *d_X, const float *d_T, int32_t batch,
                                         void *d_scratch, size_t scratch_bytes, double *d_loss, float *d_grad_out,
                                         sem_stream_t stream) {
  size_t need = 0;
  sem_status s = sem_mlp_train_scratch(N, h1, h2, batch, &need);
  if (s != SEM_OK) return s;
  if (!d_params || !d_m || !d_v || !d_X || !d_T || !d_loss || step < 1) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  if (!d_scratch || scratch_bytes < need) return sem_fail(SEM_ERR_WORKSPACE, "training scratch too small");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = N + 1;
  const Shape S = shape_of(n * n * n, h1, h2);
  float *H1 = static_cast<float *>(d_scratch), *H2 = H1 + (size_t)batch * h1, *O = H2 + (size_t)batch * h2;
  float *dO = O + (size_t)batch * S.nout, *dH2 = dO + (size_t)batch * S.nout, *dH1 = dH2 + (size_t)batch * h2;
  float *g = d_grad_out ? d_grad_out : dH1 + (size_t)batch * h1;
  if ((s = sem_mlp_forward(N, h1, h2, d_params, d_X, batch, H1, H2, O, stream)) != SEM_OK) return s;
  SEM_CUDA_TRY(cudaMemsetAsync(d_loss, 0, 8, st));
  const int64_t no = (int64_t)batch * S.nout;
  k_mse<<<egrid(no), 256, 0, st>>>(no, 1.f / (float)no, O, d_T, dO, d_loss);
  const float *W = d_params;
  // layer 3: dW3 = H2^T dO, db3 = colsum dO, dH2 = dO W3^T * (H2 > 0)
  if ((s = gemm<true, false>(S.h2, S.nout, batch, H2, S.h2, dO, S.nout, nullptr, g + S.oW3, S.nout, false, false,
                                    st)) != SEM_OK)
    return s;
  k_colsum<<<(S.nout + 255) / 256, 256, 0, st>>>(batch, S.nout, dO, g + S.ob3);
  if ((s = gemm<false, true>(batch, S.h2, S.nout, dO, S.nout, W + S.oW3, S.nout, nullptr, dH2, S.h2, false,
                                    false, st)) != SEM_OK)
    return s;
  k_relu_back<<<egrid((int64_t)batch * h2), 256, 0, st>>>((int64_t)batch * h2, dH2, H2);
  // layer 2
  if ((s = gemm<true, false>(S.h1, S.h2, batch, H1, S.h1, dH2, S.h2, nullptr, g + S.oW2, S.h2, false, false,
                                    st)) != SEM_OK)
    return s;
  k_colsum<<<(S.h2 + 255) / 256, 256, 0, st>>>(batch, S.h2, dH2, g + S.ob2);
  if ((s = gemm<false, true>(batch, S.h1, S.h2, dH2, S.h2, W + S.oW2, S.h2, nullptr, dH1, S.h1, false, false,
                                    st)) != SEM_OK)
    return s;
  k_relu_back<<<egrid((int64_t)batch * h1), 256, 0, st>>>((int64_t)batch * h1, dH1, H1);
  // layer 1
  if ((s = gemm<true, false>(S.nin, S.h1, batch, d_X, S.nin, dH1, S.h1, nullptr, g + S.oW1, S.h1, false, false,
                                    st)) != SEM_OK)
    return s;
  k_colsum<<<(S.h1 + 255) / 256, 256, 0, st>>>(batch, S.h1, dH1, g + S.ob1);
  if (lr > 0.f) {
    const float b1 = 0.9f, b2 = 0.999f;
    k_adam<<<egrid(S.count), 256, 0, st>>>(S.count, d_params, g, d_m, d_v, lr, b1, b2, 1e-8f,
                                            1.f - powf(b1, (float)step), 1.f - powf(b2, (float)step));
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_mlp_load(sem_handle *h, const float *d_params, int32_t jacobi_base, sem_stream_t stream) {
  if (!h || !d_params) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  if (!h->mlp_w) return sem_fail(SEM_ERR_INVALID, "handle was set up without SEM_FEAT_MLP");
  h->mlp_jacobi_base = jacobi_base ? 1 : 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Shape S = shape_of(h->n3, h->mlp_h1, h->mlp_h2);
  const int ldx = h->mlp_ldx;
  float *b = h->mlp_b32;
  __nv_bfloat16 *W1t = h->mlp_w, *W2t = W1t + (size_t)S.h1 * ldx, *W3t = W2t + (size_t)S.h2 * S.h1;
  k_round_bf16<<<egrid(S.count), 256, 0, st>>>(S.count, d_params, b);
  k_transpose_bf16<<<egrid((int64_t)S.h1 * ldx), 256, 0, st>>>(S.nin, S.h1, ldx, b + S.oW1, W1t);
  k_transpose_bf16<<<egrid((int64_t)S.h2 * S.h1), 256, 0, st>>>(S.h1, S.h2, S.h1, b + S.oW2, W2t);
  k_transpose_bf16<<<egrid((int64_t)S.nout * S.h2), 256, 0, st>>>(S.h2, S.nout, S.h2, b + S.oW3, W3t);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_mlp_set_fused(sem_handle *h, int32_t on) {
  if (!h) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  h->mlp_fused = on ? 1 : 0;
  return SEM_OK;
}

extern "C" sem_status sem_mlp_precond(sem_handle *h, const double *d_r, double *d_z, sem_stream_t stream) {
  if (!h || !d_r || !d_z) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  return sem_mlp_precond_apply(h, d_r, d_z, reinterpret_cast<cudaStream_t>(stream));
}
