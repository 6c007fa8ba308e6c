// Discontinuous-Galerkin shallow-water volume kernel of arXiv 1403.0968 §4.3 (include/sem_dg.h).
//
// Per element and node the kernel forms the fluxes F, G of the conservative shallow-water system
// from the nodal fields, combines them with the element's affine-map factors into
// Xr = rx F + ry G and Xs = sx F + sy G, and applies the weak derivative matrices:
// rhs = Drw Xr + Dsw Xs + S.  A block of 256 threads takes batches of floor(256 / Np) elements,
// one thread per element node, and stays resident over many batches (one block per free slot of
// the device), so that it loads the operators once; the two Np x Np operators (rows zero padded to an odd number of 16-byte
// vectors, so that threads on consecutive rows hit distinct banks) and the block's Xr, Xs sit in
// shared memory and are read 16 bytes at a time; every thread of an element reads the same X
// vector (a broadcast).  Per element the kernel reads 5 Np field
// values and 4 factors and writes 3 Np values; it performs 12 Np^2 flops in the products.
//
// The operators are built on the host in FP64 from the orthonormal (Dubiner) basis of the
// triangle: psi_ij = P_i(a) ((1-s)/2)^i P_j^(2i+1,0)(s) / sqrt(2 / ((2i+1)(i+j+1))) with the
// collapsed coordinate a = 2(1+r)/(1-s) - 1; the product P_i(a) ((1-s)/2)^i is evaluated by the
// Legendre three-term recurrence multiplied through by ((1-s)/2)^(k+1), which has no division and
// so no singularity at the vertex s = 1.
#include <cmath>
#include <vector>

#include "../../include/sem_dg.h"
#include "sem_internal.h"

__device__ int g_dg_bad;  // zero-area / clockwise triangle flag of sem_dg_geometry

namespace {

constexpr int DG_NT = 256;

__host__ __device__ constexpr int dg_np(int N) { return (N + 1) * (N + 2) / 2; }
// Row stride of the operators and of the X rows in shared memory, in elements of a type of `es`
// bytes: a whole number of 16-byte vectors (zero padded), and an odd number of them so that the
// 16-byte row loads of eight consecutive rows fall in distinct bank groups.
__host__ __device__ constexpr int dg_vw(int es) { return 16 / es; }
__host__ __device__ constexpr int dg_ld(int N, int es) {
  return ((dg_np(N) + dg_vw(es) - 1) / dg_vw(es)) % 2 ? (dg_np(N) + dg_vw(es) - 1) / dg_vw(es) * dg_vw(es)
                                                        : ((dg_np(N) + dg_vw(es) - 1) / dg_vw(es) + 1) * dg_vw(es);
}
__host__ __device__ constexpr int dg_xw(int N, int es) {  // X row length: Np rounded up to whole vectors
  return (dg_np(N) + dg_vw(es) - 1) / dg_vw(es) * dg_vw(es);
}

// ---------------------------------------------------------------------------------------------
// host: operators
// ---------------------------------------------------------------------------------------------

// P_k^(alpha,0)(x) and its derivative, k = 0..n (three-term recurrence and its derivative)
void jacobi_p(int n, double alpha, double x, double *P, double *dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n >= 1) {
    P[1] = ((alpha + 2.0) * x + alpha) / 2.0;
    dP[1] = (alpha + 2.0) / 2.0;
  }
  for (int k = 2; k <= n; ++k) {
    const double a1 = 2.0 * k * (k + alpha) * (2.0 * k + alpha - 2.0);
    const double b = 2.0 * k + alpha - 1.0;
    const double c2 = (2.0 * k + alpha) * (2.0 * k + alpha - 2.0);
    const double d = 2.0 * (k + alpha - 1.0) * (k - 1.0) * (2.0 * k + alpha);
    P[k] = (b * (c2 * x + alpha * alpha) * P[k - 1] - d * P[k - 2]) / a1;
    dP[k] = (b * (c2 * P[k - 1] + (c2 * x + alpha * alpha) * dP[k - 1]) - d * dP[k - 2]) / a1;
  }
}

// In-place Gauss-Jordan inverse with partial pivoting (n x n, row-major); false if singular.
bool invert(std::vector<double> &A, int n) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[p * n + k], A[c * n + k]);
        std::swap(I[p * n + k], I[c * n + k]);
      }
    const double inv = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] *= inv;
      I[c * n + k] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        I[r * n + k] -= f * I[c * n + k];
      }
    }
  }
  A.swap(I);
  return true;
}

std::vector<double> matmul(const std::vector<double> &A, const std::vector<double> &B, int n) {
  std::vector<double> C(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double a = A[i * n + k];
      for (int j = 0; j < n; ++j) C[i * n + j] += a * B[k * n + j];
    }
  return C;
}

std::vector<double> transpose(const std::vector<double> &A, int n) {
  std::vector<double> T(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) T[j * n + i] = A[i * n + j];
  return T;
}

// Vandermonde matrices of the orthonormal basis at the equispaced nodes: V, d/dr, d/ds
void vandermonde(int N, std::vector<double> &V, std::vector<double> &Vr, std::vector<double> &Vs) {
  const int np = dg_np(N);
  V.assign(np * np, 0.0);
  Vr.assign(np * np, 0.0);
  Vs.assign(np * np, 0.0);
  std::vector<double> Q(N + 2), Qr(N + 2), Qs(N + 2), P(N + 1), dP(N + 1);
  int n = 0;
  for (int b = 0; b <= N; ++b)
    for (int a = 0; a + b <= N; ++a, ++n) {
      const double r = -1.0 + 2.0 * a / N, s = -1.0 + 2.0 * b / N;
      // Q_k = P_k(a) q^k, q = (1-s)/2:  (k+1) Q_{k+1} = (2k+1) (a q) Q_k - k q^2 Q_{k-1}, a q = r + (1+s)/2
      const double aq = r + 0.5 * (1.0 + s), q = 0.5 * (1.0 - s), q2 = q * q, dq2s = -q;
      Q[0] = 1.0, Qr[0] = 0.0, Qs[0] = 0.0;
      Q[1] = aq, Qr[1] = 1.0, Qs[1] = 0.5;
      for (int k = 1; k < N; ++k) {
        Q[k + 1] = ((2.0 * k + 1.0) * aq * Q[k] - k * q2 * Q[k - 1]) / (k + 1.0);
        Qr[k + 1] = ((2.0 * k + 1.0) * (Q[k] + aq * Qr[k]) - k * q2 * Qr[k - 1]) / (k + 1.0);
        Qs[k + 1] = ((2.0 * k + 1.0) * (0.5 * Q[k] + aq * Qs[k]) - k * (dq2s * Q[k - 1] + q2 * Qs[k - 1])) / (k + 1.0);
      }
      int m = 0;
      for (int i = 0; i <= N; ++i) {
        jacobi_p(N - i, 2.0 * i + 1.0, s, P.data(), dP.data());
        for (int j = 0; i + j <= N; ++j, ++m) {
          const double w = 1.0 / std::sqrt(2.0 / ((2.0 * i + 1.0) * (i + j + 1.0)));
          V[n * np + m] = w * Q[i] * P[j];
          Vr[n * np + m] = w * Qr[i] * P[j];
          Vs[n * np + m] = w * (Qs[i] * P[j] + Q[i] * dP[j]);
        }
      }
    }
}

// ---------------------------------------------------------------------------------------------
// device: volume kernel
// ---------------------------------------------------------------------------------------------

template <typename T>
struct alignas(16) DgVec {
  T v[16 / sizeof(T)];
};

// Elements per thread: with ET > 1 every operator vector a thread loads serves ET elements (fewer
// shared-memory wavefronts per output); FP64 keeps 1 (its FMA pipe is the bound, and its shared
// memory would not fit).  Measured on 212,800 triangles: ET = 2 1.2x over 1 at N = 6..8, slower at
// N = 2; ET = 3 (73 registers, 3 blocks per SM) a further 5% at N = 7 and 8.5% at N = 8, level at
// N = 6; ET = 4 (90 registers) slower.
__host__ __device__ constexpr int dg_et(int N, int es) { return es == 4 && N >= 7 ? 3 : es == 4 && N >= 3 ? 2 : 1; }

template <typename T, int N>
__global__ void __launch_bounds__(DG_NT) k_dg_volume(int64_t E, T g, const T *__restrict__ ops,
                                                     const T *__restrict__ Q, const T *__restrict__ Bxy,
                                                     const T *__restrict__ geo, T *__restrict__ rhs) {
  constexpr int NP = dg_np(N), LD = dg_ld(N, sizeof(T)), XW = dg_xw(N, sizeof(T));
  constexpr int ET = dg_et(N, sizeof(T)), EG = DG_NT / NP, EB = EG * ET;  // groups, elements per batch
  constexpr int VW = dg_vw(sizeof(T)), NV = XW / VW;  // 16-byte vectors per row
  __shared__ alignas(16) T sD[2 * NP * LD];
  __shared__ alignas(16) T sX[EB][6][XW];
  const int tid = threadIdx.x;
  for (int q = tid; q < 2 * NP * LD; q += DG_NT) sD[q] = ops[q];
  // zero the padding of the X rows (it meets the zero padding of the operator rows)
  for (int q = tid; q < EB * 6 * (XW - NP); q += DG_NT) {
    const int row = q / (XW - NP);
    sX[row / 6][row % 6][NP + q % (XW - NP)] = T(0);
  }
  const int el = tid / NP, i = tid - el * NP;  // group (ET consecutive elements of a batch), node
  const bool grp = el < EG;
  const DgVec<T> *dr = reinterpret_cast<const DgVec<T> *>(sD + i * LD);
  const DgVec<T> *ds = reinterpret_cast<const DgVec<T> *>(sD + NP * LD + i * LD);
  const DgVec<T> *x0 = reinterpret_cast<const DgVec<T> *>(&sX[grp ? el * ET : 0][0][0]);
  constexpr int XS = 6 * NV;  // vectors per element in sX
  // persistent blocks: the operators are loaded once per block, batches of EB elements follow
  const int64_t nbatch = (E + EB - 1) / EB;
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int64_t e0 = batch * EB + (int64_t)el * ET;
    T h[ET], bx[ET], by[ET];
#pragma unroll
    for (int t = 0; t < ET; ++t) {
      const int64_t e = e0 + t;
      h[t] = T(1), bx[t] = T(0), by[t] = T(0);
      if (grp && e < E) {
        const T *q = Q + e * 3 * NP + i;
        h[t] = q[0];
        const T hu = q[NP], hv = q[2 * NP];
        bx[t] = Bxy[e * 2 * NP + i];
        by[t] = Bxy[e * 2 * NP + NP + i];
        const T rx = geo[e * 4 + 0], ry = geo[e * 4 + 1], sx = geo[e * 4 + 2], sy = geo[e * 4 + 3];
        const T ih = T(1) / h[t], u = hu * ih, v = hv * ih, p = T(0.5) * g * h[t] * h[t];
        const T F0 = hu, F1 = hu * u + p, F2 = hu * v;
        const T G0 = hv, G1 = hv * u, G2 = hv * v + p;
        T(*X)[XW] = sX[el * ET + t];
        X[0][i] = rx * F0 + ry * G0;
        X[1][i] = rx * F1 + ry * G1;
        X[2][i] = rx * F2 + ry * G2;
        X[3][i] = sx * F0 + sy * G0;
        X[4][i] = sx * F1 + sy * G1;
        X[5][i] = sx * F2 + sy * G2;
      }
    }
    __syncthreads();
    if (grp && e0 < E) {
      // 16-byte loads: one operator vector serves three fields of ET elements; each X vector is the
      // same for every thread of the element (a broadcast)
      T a[ET][3];
#pragma unroll
      for (int t = 0; t < ET; ++t) a[t][0] = a[t][1] = a[t][2] = T(0);
#pragma unroll
      for (int jv = 0; jv < NV; ++jv) {
        const DgVec<T> wr = dr[jv], ws = ds[jv];
#pragma unroll
        for (int t = 0; t < ET; ++t) {
          const DgVec<T> *xt = x0 + t * XS;
          const DgVec<T> r0 = xt[0 * NV + jv], r1 = xt[1 * NV + jv], r2 = xt[2 * NV + jv];
          const DgVec<T> s0 = xt[3 * NV + jv], s1 = xt[4 * NV + jv], s2 = xt[5 * NV + jv];
#pragma unroll
          for (int k = 0; k < VW; ++k) {
            a[t][0] += wr.v[k] * r0.v[k] + ws.v[k] * s0.v[k];
            a[t][1] += wr.v[k] * r1.v[k] + ws.v[k] * s1.v[k];
            a[t][2] += wr.v[k] * r2.v[k] + ws.v[k] * s2.v[k];
          }
        }
      }
#pragma unroll
      for (int t = 0; t < ET; ++t) {
        const int64_t e = e0 + t;
        if (e < E) {
          T *o = rhs + e * 3 * NP + i;
          o[0] = a[t][0];
          o[NP] = a[t][1] - g * h[t] * bx[t];
          o[2 * NP] = a[t][2] - g * h[t] * by[t];
        }
      }
    }
    __syncthreads();  // the next batch overwrites sX
  }
}

// rx, ry, sx, sy of each triangle: the inverse of [[x_r, x_s], [y_r, y_s]] with x_r = (x2 - x1)/2,
// x_s = (x3 - x1)/2 (and y alike); bad is set when the Jacobian is not positive
template <typename T>
__global__ void k_dg_geometry(int64_t E, const double *__restrict__ v, T *__restrict__ geo, int *bad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double *p = v + e * 6;
  const double xr = 0.5 * (p[2] - p[0]), xs = 0.5 * (p[4] - p[0]);
  const double yr = 0.5 * (p[3] - p[1]), ys = 0.5 * (p[5] - p[1]);
  const double J = xr * ys - xs * yr;
  if (!(J > 0.0)) atomicOr(bad, 1);
  geo[e * 4 + 0] = (T)(ys / J);
  geo[e * 4 + 1] = (T)(-xs / J);
  geo[e * 4 + 2] = (T)(-yr / J);
  geo[e * 4 + 3] = (T)(xr / J);
}

template <typename T, int N>
sem_status launch_dg(int64_t E, double g, const void *ops, const void *Q, const void *Bxy, const void *geo,
                     void *rhs, cudaStream_t s) {
  constexpr int EB = DG_NT / dg_np(N) * dg_et(N, sizeof(T));
  const int64_t batches = (E + EB - 1) / EB;
  // persistent grid: as many blocks as fit on the device at once (each loads the operators once)
  int dev = 0, sms = 0, per_sm = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  SEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dg_volume<T, N>, DG_NT, 0));
  const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  const int64_t blocks = batches < resident ? batches : resident;
  k_dg_volume<T, N><<<(unsigned)blocks, DG_NT, 0, s>>>(
      E, (T)g, static_cast<const T *>(ops), static_cast<const T *>(Q), static_cast<const T *>(Bxy),
      static_cast<const T *>(geo), static_cast<T *>(rhs));
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

template <typename T>
sem_status dg_dispatch(int N, int64_t E, double g, const void *ops, const void *Q, const void *Bxy, const void *geo,
                       void *rhs, cudaStream_t s) {
  switch (N) {
    case 1: return launch_dg<T, 1>(E, g, ops, Q, Bxy, geo, rhs, s);
    case 2: return launch_dg<T, 2>(E, g, ops, Q, Bxy, geo, rhs, s);
    case 3: return launch_dg<T, 3>(E, g, ops, Q, Bxy, geo, rhs, s);
    case 4: return launch_dg<T, 4>(E, g, ops, Q, Bxy, geo, rhs, s);
    case 5: return launch_dg<T, 5>(E, g, ops, Q, Bxy, geo, rhs, s);
    case 6: return launch_dg<T, 6>(E, g, ops, Q, Bxy, geo, rhs, s);
    case 7: return launch_dg<T, 7>(E, g, ops, Q, Bxy, geo, rhs, s);
    case 8: return launch_dg<T, 8>(E, g, ops, Q, Bxy, geo, rhs, s);
    default: return sem_fail(SEM_ERR_INVALID, "DG order must be 1..8");
  }
}

}  // namespace

extern "C" sem_status sem_dg_operators(int32_t N, double *Drw, double *Dsw) {
  if (N < 1 || N > SEM_DG_MAX_ORDER) return sem_fail(SEM_ERR_INVALID, "DG order must be 1..8");
  if (!Drw || !Dsw) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  const int np = dg_np(N);
  std::vector<double> V, Vr, Vs;
  vandermonde(N, V, Vr, Vs);
  std::vector<double> Vinv = V;
  if (!invert(Vinv, np)) return sem_fail(SEM_ERR_INVALID, "singular Vandermonde matrix");
  const std::vector<double> Dr = matmul(Vr, Vinv, np), Ds = matmul(Vs, Vinv, np);
  const std::vector<double> A = matmul(V, transpose(V, np), np);             // Mhat^-1
  const std::vector<double> Ainv = matmul(transpose(Vinv, np), Vinv, np);    // Mhat
  const std::vector<double> Wr = matmul(matmul(A, transpose(Dr, np), np), Ainv, np);
  const std::vector<double> Ws = matmul(matmul(A, transpose(Ds, np), np), Ainv, np);
  for (int q = 0; q < np * np; ++q) {
    Drw[q] = Wr[q];
    Dsw[q] = Ws[q];
  }
  return SEM_OK;
}

extern "C" sem_status sem_dg_operator_bytes(int32_t N, sem_prec prec, size_t *bytes) {
  if (N < 1 || N > SEM_DG_MAX_ORDER) return sem_fail(SEM_ERR_INVALID, "DG order must be 1..8");
  if (prec != SEM_FP64 && prec != SEM_FP32) return sem_fail(SEM_ERR_INVALID, "DG precision must be FP64 or FP32");
  if (!bytes) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  const int es = prec == SEM_FP64 ? 8 : 4;
  *bytes = (size_t)2 * dg_np(N) * dg_ld(N, es) * es;
  return SEM_OK;
}

extern "C" sem_status sem_dg_load_operators(int32_t N, sem_prec prec, void *d_ops, size_t bytes, sem_stream_t stream) {
  size_t need = 0;
  sem_status st = sem_dg_operator_bytes(N, prec, &need);
  if (st != SEM_OK) return st;
  if (!d_ops || bytes < need) return sem_fail(SEM_ERR_INVALID, "operator buffer missing or too small");
  const int np = dg_np(N), ld = dg_ld(N, prec == SEM_FP64 ? 8 : 4);
  std::vector<double> Wr(np * np), Ws(np * np);
  st = sem_dg_operators(N, Wr.data(), Ws.data());
  if (st != SEM_OK) return st;
  std::vector<double> d64(2 * np * ld, 0.0);
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j) {
      d64[i * ld + j] = Wr[i * np + j];
      d64[np * ld + i * ld + j] = Ws[i * np + j];
    }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prec == SEM_FP64) {
    SEM_CUDA_TRY(cudaMemcpyAsync(d_ops, d64.data(), need, cudaMemcpyHostToDevice, s));
  } else {
    std::vector<float> d32(d64.size());
    for (size_t q = 0; q < d64.size(); ++q) d32[q] = (float)d64[q];
    SEM_CUDA_TRY(cudaMemcpyAsync(d_ops, d32.data(), need, cudaMemcpyHostToDevice, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));  // the host copy goes out of scope
    return SEM_OK;
  }
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  return SEM_OK;
}

extern "C" sem_status sem_dg_volume(sem_prec prec, int32_t N, int64_t E, double g, const void *d_ops, const void *d_Q,
                                    const void *d_Bxy, const void *d_geo, void *d_rhs, sem_stream_t stream) {
  if (!d_ops || !d_Q || !d_Bxy || !d_geo || !d_rhs) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  if (E < 1) return sem_fail(SEM_ERR_INVALID, "element count must be positive");
  if (N < 1 || N > SEM_DG_MAX_ORDER) return sem_fail(SEM_ERR_INVALID, "DG order must be 1..8");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prec == SEM_FP64) return dg_dispatch<double>(N, E, g, d_ops, d_Q, d_Bxy, d_geo, d_rhs, s);
  if (prec == SEM_FP32) return dg_dispatch<float>(N, E, g, d_ops, d_Q, d_Bxy, d_geo, d_rhs, s);
  return sem_fail(SEM_ERR_INVALID, "DG precision must be SEM_FP64 or SEM_FP32");
}

extern "C" sem_status sem_dg_geometry(sem_prec prec, int64_t E, const double *d_verts, void *d_geo,
                                      sem_stream_t stream) {
  if (!d_verts || !d_geo) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  if (E < 1) return sem_fail(SEM_ERR_INVALID, "element count must be positive");
  if (prec != SEM_FP64 && prec != SEM_FP32) return sem_fail(SEM_ERR_INVALID, "DG precision must be FP64 or FP32");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int *bad = nullptr;  // a static device word (calls on one device must not run concurrently)
  SEM_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&bad), g_dg_bad));
  SEM_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  const unsigned blocks = (unsigned)((E + 255) / 256);
  if (prec == SEM_FP64)
    k_dg_geometry<double><<<blocks, 256, 0, s>>>(E, d_verts, static_cast<double *>(d_geo), bad);
  else
    k_dg_geometry<float><<<blocks, 256, 0, s>>>(E, d_verts, static_cast<float *>(d_geo), bad);
  SEM_CUDA_TRY(cudaGetLastError());
  int bad_h = 0;
  SEM_CUDA_TRY(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (bad_h) return sem_fail(SEM_ERR_INVALID, "triangle with non-positive Jacobian (clockwise or degenerate)");
  return SEM_OK;
}
