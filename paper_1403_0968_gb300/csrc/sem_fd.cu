// Finite-difference wave step of arXiv 1403.0968 §4.1 (Algorithm 1): one leapfrog step of
// u_tt = u_xx + u_yy with central (2r+1)-point second-derivative stencils in x and y on a periodic
// grid, neighbour indices wrapped as the §4.1 kernel listing does (include/sem_fd.h).
//
// The step reads u_n and u_{n-1} once and writes u_{n+1} once per node (12 bytes in FP32, 24 in
// FP64): an HBM-bound stencil.  A block of 256 threads owns a 64 x 32 output tile (64 x 64 for the
// FP32 kernel with column pairs); it copies the tile of u_n with its halo (r nodes on each side,
// wrapped around the grid at its edges) into shared memory, then each thread produces 8
// consecutive outputs of one column (of two adjacent columns in the FP32 pair kernel): the y
// stencil from a register window of 8 + 2r values of its column, the x stencil from its row in
// shared memory (consecutive threads read consecutive words: no bank conflicts).  The halo
// overlap of neighbouring tiles is read from L2, not from HBM.  u_{n+1} overwrites u_{n-1} in
// place: each node of that grid is read and written by the thread that owns it only.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched from the driver at run time)
#include <cudaTypedefs.h>

#include <mutex>

#include "../../include/sem_fd.h"
#include "sem_internal.h"
#include "sem_tma.cuh"

__device__ int g_fd_timeout;  // set when a bounded wait of the TMA-staged step gave up

namespace {

constexpr int FD_TX = 64;  // threads (outputs) per tile row
constexpr int FD_TY = 4;   // thread rows per block
constexpr int FD_RY = 8;   // outputs per thread along y
constexpr int FD_TILE_Y = FD_TY * FD_RY;

// x mod n in [0, n) for a coordinate of a halo tile (|x| < n + 2 r); the division only runs for
// coordinates outside the grid, i.e. in the tiles at the grid's edges
__device__ __forceinline__ int64_t fd_wrap(int64_t x, int64_t n) {
  if (x >= 0 && x < n) return x;
  x %= n;
  return x < 0 ? x + n : x;
}

// Fills the [TH][TW] tile whose entry (row, col) is u_n at grid node (x0 - XOFF + col, y0 - R + row),
// indices wrapped around the grid (periodic boundary): the path of the tiles at the grid's edges.
template <typename T, int R, int XOFF, int TH, int TW>
__device__ __forceinline__ void fd_load_wrapped(const T *__restrict__ u, int64_t w, int64_t h, int64_t x0, int64_t y0,
                                                int tid, T (*s)[TW]) {
  constexpr int NT = FD_TX * FD_TY;
  for (int idx = tid; idx < TH * TW; idx += NT) {
    const int row = idx / TW, col = idx - row * TW;
    const int64_t gxl = fd_wrap(x0 - XOFF + col, w), gyl = fd_wrap(y0 - R + row, h);
    s[row][col] = u[gyl * w + gxl];
  }
}

// Stencil coefficients with dt^2 and the spacings folded in:
//   u_{n+1} = center u_n + sum_{k>=1} cx[k] (u(i+k) + u(i-k)) + cy[k] (u(j+k) + u(j-k)) - u_{n-1}
template <typename T>
struct FdCoef {
  T cx[SEM_FD_MAX_RADIUS + 1], cy[SEM_FD_MAX_RADIUS + 1];
  T center;
};

template <typename T, int R>
__global__ void __launch_bounds__(FD_TX *FD_TY) k_fd_step(const T *__restrict__ u, T *__restrict__ up, int64_t w,
                                                          int64_t h, const FdCoef<T> c) {
  constexpr int TW = FD_TX + 2 * R, TH = FD_TILE_Y + 2 * R, NT = FD_TX * FD_TY;
  constexpr int NLD = (TH * TW + NT - 1) / NT;  // tile entries per thread
  __shared__ T s[TH][TW];
  const int64_t x0 = (int64_t)blockIdx.x * FD_TX, y0 = (int64_t)blockIdx.y * FD_TILE_Y;
  const int tid = threadIdx.y * FD_TX + threadIdx.x;
  const int tx = threadIdx.x, r0 = threadIdx.y * FD_RY;  // first output row of this thread in the tile
  const int64_t gx = x0 + tx;
  // Offsets inside a tile fit 32 bits when (32 + 2r) rows of the grid do (checked by the host);
  // the 64-bit part is formed once per thread.
  const int w32 = (int)w;
  // every load of the tile is issued before the first shared-memory store, and this thread's
  // u_{n-1} values are fetched at the same time, so their latencies overlap
  T v[NLD];
  const bool inside = x0 >= R && y0 >= R && x0 + FD_TX + R <= w && y0 + FD_TILE_Y + R <= h;
  if (inside) {  // the whole tile and its halo lie in the grid: no bounds checks
    const T *ub = u + ((y0 - R) * w + (x0 - R));  // tile origin
#pragma unroll
    for (int it = 0; it < NLD; ++it) {
      const int idx = tid + it * NT;
      const int row = idx / TW, col = idx - row * TW;
      v[it] = (idx < TH * TW) ? ub[row * w32 + col] : T(0);
    }
  } else {  // a tile at the grid's edge: halo indices wrap around (periodic boundary)
#pragma unroll
    for (int it = 0; it < NLD; ++it) {
      const int idx = tid + it * NT;
      const int row = idx / TW, col = idx - row * TW;
      v[it] = (idx < TH * TW) ? u[fd_wrap(y0 - R + row, h) * w + fd_wrap(x0 - R + col, w)] : T(0);
    }
  }
  const bool col_ok = gx < w;
  const int rows_left = (int)((h - (y0 + r0)) < FD_RY ? (h - (y0 + r0)) : FD_RY);  // may be <= 0
  // this thread's first output; dereferenced only for nodes in the grid
  T *pb = up + ((col_ok && rows_left > 0) ? ((y0 + r0) * w + gx) : 0);
  T pv[FD_RY];
#pragma unroll
  for (int j = 0; j < FD_RY; ++j) pv[j] = (col_ok && j < rows_left) ? pb[j * w32] : T(0);
#pragma unroll
  for (int it = 0; it < NLD; ++it) {
    const int idx = tid + it * NT;
    if (idx < TH * TW) {
      const int row = idx / TW;
      s[row][idx - row * TW] = v[it];
    }
  }
  __syncthreads();
  if (!col_ok) return;
  T col[FD_RY + 2 * R];
#pragma unroll
  for (int q = 0; q < FD_RY + 2 * R; ++q) col[q] = s[r0 + q][tx + R];
#pragma unroll
  for (int j = 0; j < FD_RY; ++j) {
    if (j < rows_left) {
      const T *row = &s[r0 + j + R][tx + R];
      T acc = c.center * col[j + R];
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        acc += c.cy[k] * (col[j + R - k] + col[j + R + k]);
        acc += c.cx[k] * (row[-k] + row[k]);
      }
      pb[j * w32] = acc - pv[j];
    }
  }
}

// TMA-staged variant: one 2-D tensor copy brings the tile of u_n with its halo into shared memory
// while the threads fetch their u_{n-1} values; no per-element index arithmetic or bounds checks
// for the tile.  The tile starts RA >= r columns left of the outputs, RA a multiple of 16 bytes,
// so every copy starts on a 16-byte boundary.  Needs rows of a multiple of 16 bytes (the tensor
// map's stride).  A tile whose halo crosses the grid's edge cannot take the copy (the copy fills
// outside the grid with zeros, the periodic boundary wants the wrapped nodes): those tiles, a
// thin frame of the grid, load the halo with plain wrapped loads instead.
template <typename T, int R>
__host__ __device__ constexpr int fd_ra() {
  return (R * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
}

template <typename T, int R>
__global__ void __launch_bounds__(FD_TX *FD_TY) k_fd_step_tma(const __grid_constant__ CUtensorMap tmap,
                                                              const T *__restrict__ u, T *__restrict__ up,
                                                              int64_t w, int64_t h, const FdCoef<T> c) {
  constexpr int RA = fd_ra<T, R>(), TW = FD_TX + 2 * RA, TH = FD_TILE_Y + 2 * R;
  __shared__ alignas(128) T s[TH][TW];
  __shared__ uint64_t bar;
  const int64_t x0 = (int64_t)blockIdx.x * FD_TX, y0 = (int64_t)blockIdx.y * FD_TILE_Y;
  const int tid = threadIdx.y * FD_TX + threadIdx.x;
  const int tx = threadIdx.x, r0 = threadIdx.y * FD_RY;
  const int64_t gx = x0 + tx;
  const int w32 = (int)w;
  // block-uniform: does the halo tile lie inside the grid?
  const bool inside = x0 >= R && y0 >= R && x0 + FD_TX + R <= w && y0 + FD_TILE_Y + R <= h;
  if (!inside) fd_load_wrapped<T, R, RA, TH, TW>(u, w, h, x0, y0, tid, s);
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (inside && tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)),
                 "r"((uint32_t)(TH * TW * sizeof(T)))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(&s[0][0])),
        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"((int)(x0 - RA)), "r"((int)(y0 - R)), "r"(smem_addr(&bar))
        : "memory");
  }
  const bool col_ok = gx < w;
  const int rows_left = (int)((h - (y0 + r0)) < FD_RY ? (h - (y0 + r0)) : FD_RY);
  T *pb = up + ((col_ok && rows_left > 0) ? ((y0 + r0) * w + gx) : 0);
  T pv[FD_RY];
#pragma unroll
  for (int j = 0; j < FD_RY; ++j) pv[j] = (col_ok && j < rows_left) ? pb[j * w32] : T(0);
  const bool ok = inside ? mbar_wait(&bar, 0) : true;
  if (__syncthreads_or(!ok)) {
    // the copy did not complete in time: record it, wait once more (bounded) for the copy this
    // block issued, and leave without writing
    if (tid == 0) {
      atomicOr(&g_fd_timeout, 1);
      mbar_wait(&bar, 0);
    }
    return;
  }
  if (!col_ok) return;
  T col[FD_RY + 2 * R];
#pragma unroll
  for (int q = 0; q < FD_RY + 2 * R; ++q) col[q] = s[r0 + q][tx + RA];
#pragma unroll
  for (int j = 0; j < FD_RY; ++j) {
    if (j < rows_left) {
      const T *row = &s[r0 + j + R][tx + RA];
      T acc = c.center * col[j + R];
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        acc += c.cy[k] * (col[j + R - k] + col[j + R + k]);
        acc += c.cx[k] * (row[-k] + row[k]);
      }
      pb[j * w32] = acc - pv[j];
    }
  }
}

// FP32 TMA-staged variant on a 64 x 64 tile: the block's 256 threads as 32 column pairs x 8 row
// groups, each forming 2 adjacent columns x 8 rows.  The column windows stay 8 + 2r long (read as
// pairs), and the x stencil of a row is 2r + 2 values shared by both columns (read as pairs from
// an even column): about half the shared-memory loads per output of the kernel above.
constexpr int FD_TILE_Y2 = 64;
static_assert(FD_TX * FD_TY == 32 * 8 && 8 * FD_RY == FD_TILE_Y2, "thread layout of the pair kernel");

template <int R>
__global__ void __launch_bounds__(FD_TX *FD_TY, 4) k_fd_step_tma2(const __grid_constant__ CUtensorMap tmap,
                                                               const float *__restrict__ u, float *__restrict__ up,
                                                               int64_t w, int64_t h, const FdCoef<float> c) {
  constexpr int RA = fd_ra<float, R>(), TW = FD_TX + 2 * RA, TH = FD_TILE_Y2 + 2 * R;
  constexpr int RE = (R + 1) / 2 * 2;  // R rounded up to even: the x stencil's pairs start at an even column
  static_assert(RA >= RE && RA % 2 == 0 && TW % 2 == 0, "halo of the tile against the pair loads");
  __shared__ alignas(128) float s[TH][TW];
  __shared__ uint64_t bar;
  const int64_t x0 = (int64_t)blockIdx.x * FD_TX, y0 = (int64_t)blockIdx.y * FD_TILE_Y2;
  const int tid = threadIdx.y * FD_TX + threadIdx.x;
  const int w32 = (int)w;
  // block-uniform: does the halo tile lie inside the grid?
  const bool inside = x0 >= R && y0 >= R && x0 + FD_TX + R <= w && y0 + FD_TILE_Y2 + R <= h;
  if (!inside) fd_load_wrapped<float, R, RA, TH, TW>(u, w, h, x0, y0, tid, s);
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (inside && tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)),
                 "r"((uint32_t)(TH * TW * sizeof(float)))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(&s[0][0])),
        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"((int)(x0 - RA)), "r"((int)(y0 - R)), "r"(smem_addr(&bar))
        : "memory");
  }
  // this thread's outputs: columns x0 + cx2, cx2 + 1 (cx2 even) of rows y0 + ry .. ry + 7
  const int cx2 = 2 * (tid & 31), ry = (tid >> 5) * FD_RY;
  const int64_t gx2 = x0 + cx2;
  const bool col_ok = gx2 < w;  // rows are a multiple of 16 bytes, so column gx2 + 1 is in the grid too
  const int rows_left = (int)((h - (y0 + ry)) < FD_RY ? (h - (y0 + ry)) : FD_RY);
  float *pb = up + ((col_ok && rows_left > 0) ? ((y0 + ry) * w + gx2) : 0);
  float2 pv[FD_RY];
#pragma unroll
  for (int j = 0; j < FD_RY; ++j)
    pv[j] = (col_ok && j < rows_left) ? *reinterpret_cast<const float2 *>(pb + j * w32) : make_float2(0.f, 0.f);
  const bool ok = inside ? mbar_wait(&bar, 0) : true;
  if (__syncthreads_or(!ok)) {
    // the copy did not complete in time: record it, wait once more (bounded) for the copy this
    // block issued, and leave without writing
    if (tid == 0) {
      atomicOr(&g_fd_timeout, 1);
      mbar_wait(&bar, 0);
    }
    return;
  }
  if (!col_ok) return;
  float2 col[FD_RY + 2 * R];  // the two columns as a register window along y
#pragma unroll
  for (int q = 0; q < FD_RY + 2 * R; ++q) col[q] = *reinterpret_cast<const float2 *>(&s[ry + q][cx2 + RA]);
#pragma unroll
  for (int j = 0; j < FD_RY; ++j) {
    if (j < rows_left) {
      float xr[2 * RE + 2];  // columns cx2 - RE .. cx2 + 1 + RE of the row; xr[RE] is column cx2
#pragma unroll
      for (int q = 0; q <= RE; ++q) {
        const float2 v = *reinterpret_cast<const float2 *>(&s[ry + j + R][cx2 + RA - RE + 2 * q]);
        xr[2 * q] = v.x;
        xr[2 * q + 1] = v.y;
      }
      float a0 = c.center * col[j + R].x, a1 = c.center * col[j + R].y;
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        a0 += c.cy[k] * (col[j + R - k].x + col[j + R + k].x);
        a1 += c.cy[k] * (col[j + R - k].y + col[j + R + k].y);
        a0 += c.cx[k] * (xr[RE - k] + xr[RE + k]);
        a1 += c.cx[k] * (xr[RE + 1 - k] + xr[RE + 1 + k]);
      }
      *reinterpret_cast<float2 *>(pb + j * w32) = make_float2(a0 - pv[j].x, a1 - pv[j].y);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 fd_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <typename T, int R>
sem_status launch_fd(int64_t w, int64_t h, const T *u, T *up, const FdCoef<T> &c, cudaStream_t s) {
  const int64_t gxb = (w + FD_TX - 1) / FD_TX, gyb = (h + FD_TILE_Y - 1) / FD_TILE_Y;
  if (gxb > 0x7fffffff || gyb > 65535) return sem_fail(SEM_ERR_INVALID, "grid too large for one launch");
  if (w * (int64_t)(FD_TILE_Y + 2 * R + 1) >= ((int64_t)1 << 31))
    return sem_fail(SEM_ERR_INVALID, "grid rows too long for 32-bit tile offsets");
  // TMA path when the grid's rows are whole 16-byte units and u starts on a 16-byte boundary
  const bool tma_ok = (w * (int64_t)sizeof(T)) % 16 == 0 && (reinterpret_cast<uintptr_t>(u) & 15u) == 0 &&
                      w <= 0x7fffffff && h <= 0x7fffffff;
  if (tma_ok) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = fd_map_encoder();
    constexpr int RA = fd_ra<T, R>();
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[1] = {(cuuint64_t)w * sizeof(T)};
    if constexpr (sizeof(T) == 4) {
      // FP32: the 64 x 64 tile with column pairs, when u_{n-1} / u_{n+1} start on an 8-byte boundary
      if ((reinterpret_cast<uintptr_t>(up) & 7u) == 0 && w * (int64_t)(FD_TILE_Y2 + 2 * R + 1) < ((int64_t)1 << 31)) {
        const cuuint32_t box2[2] = {(cuuint32_t)(FD_TX + 2 * RA), (cuuint32_t)(FD_TILE_Y2 + 2 * R)};
        const cuuint32_t estr2[2] = {1, 1};
        if (enc && enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<T *>(u), dims, strides, box2, estr2,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
          const int64_t gyb2 = (h + FD_TILE_Y2 - 1) / FD_TILE_Y2;
          k_fd_step_tma2<R><<<dim3((unsigned)gxb, (unsigned)gyb2), dim3(FD_TX, FD_TY), 0, s>>>(
              tm, reinterpret_cast<const float *>(u), reinterpret_cast<float *>(up), w, h,
              reinterpret_cast<const FdCoef<float> &>(c));
          SEM_CUDA_TRY(cudaGetLastError());
          return SEM_OK;
        }
      }
    }
    const cuuint32_t box[2] = {(cuuint32_t)(FD_TX + 2 * RA), (cuuint32_t)(FD_TILE_Y + 2 * R)};
    const cuuint32_t estr[2] = {1, 1};
    if (enc && enc(&tm, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<T *>(u), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
      k_fd_step_tma<T, R><<<dim3((unsigned)gxb, (unsigned)gyb), dim3(FD_TX, FD_TY), 0, s>>>(tm, u, up, w, h, c);
      SEM_CUDA_TRY(cudaGetLastError());
      return SEM_OK;
    }
  }
  k_fd_step<T, R><<<dim3((unsigned)gxb, (unsigned)gyb), dim3(FD_TX, FD_TY), 0, s>>>(u, up, w, h, c);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

template <typename T>
sem_status fd_dispatch(int r, int64_t w, int64_t h, double dt, double dx, double dy, const void *u, void *up,
                       cudaStream_t s) {
  double cw[2 * SEM_FD_MAX_RADIUS + 1];
  sem_status st = sem_fd_weights(r, cw);
  if (st != SEM_OK) return st;
  FdCoef<T> c;
  for (int k = 0; k <= SEM_FD_MAX_RADIUS; ++k) c.cx[k] = c.cy[k] = T(0);
  const double ax = dt * dt / (dx * dx), ay = dt * dt / (dy * dy);
  for (int k = 1; k <= r; ++k) {
    c.cx[k] = (T)(ax * cw[r + k]);
    c.cy[k] = (T)(ay * cw[r + k]);
  }
  c.center = (T)(2.0 + (ax + ay) * cw[r]);
  const T *uu = static_cast<const T *>(u);
  T *pp = static_cast<T *>(up);
  switch (r) {
    case 1: return launch_fd<T, 1>(w, h, uu, pp, c, s);
    case 2: return launch_fd<T, 2>(w, h, uu, pp, c, s);
    case 3: return launch_fd<T, 3>(w, h, uu, pp, c, s);
    case 4: return launch_fd<T, 4>(w, h, uu, pp, c, s);
    case 5: return launch_fd<T, 5>(w, h, uu, pp, c, s);
    case 6: return launch_fd<T, 6>(w, h, uu, pp, c, s);
    case 7: return launch_fd<T, 7>(w, h, uu, pp, c, s);
    default: return sem_fail(SEM_ERR_INVALID, "stencil radius must be 1..7");
  }
}

}  // namespace

// c_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!) for k >= 1 and c_0 = -2 sum_{k>=1} c_k: the
// closed form of the central weights of order 2r (Fornberg, Math. Comp. 51, 1988).
extern "C" sem_status sem_fd_weights(int32_t r, double *c) {
  if (r < 1 || r > SEM_FD_MAX_RADIUS) return sem_fail(SEM_ERR_INVALID, "stencil radius must be 1..7");
  if (!c) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  auto fact = [](int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
  };
  const double rf2 = fact(r) * fact(r);
  double sum = 0.0;
  for (int k = 1; k <= r; ++k) {
    const double ck = ((k % 2) ? 2.0 : -2.0) * rf2 / ((double)k * k * fact(r - k) * fact(r + k));
    c[r + k] = c[r - k] = ck;
    sum += ck;
  }
  c[r] = -2.0 * sum;
  return SEM_OK;
}

extern "C" sem_status sem_fd_step(sem_prec prec, int32_t r, int64_t w, int64_t h, double dt, double dx, double dy,
                                  const void *d_u, void *d_uprev_next, sem_stream_t stream) {
  if (!d_u || !d_uprev_next) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  if (d_u == d_uprev_next) return sem_fail(SEM_ERR_INVALID, "u and uprev_next must not alias");
  if (w < 1 || h < 1) return sem_fail(SEM_ERR_INVALID, "grid sizes must be positive");
  if (!(dt > 0.0) || !(dx > 0.0) || !(dy > 0.0)) return sem_fail(SEM_ERR_INVALID, "dt, dx, dy must be positive");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prec == SEM_FP64) return fd_dispatch<double>(r, w, h, dt, dx, dy, d_u, d_uprev_next, s);
  if (prec == SEM_FP32) return fd_dispatch<float>(r, w, h, dt, dx, dy, d_u, d_uprev_next, s);
  return sem_fail(SEM_ERR_INVALID, "finite-difference step precision must be SEM_FP64 or SEM_FP32");
}

extern "C" sem_status sem_fd_status(sem_stream_t stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int *flag = nullptr;
  SEM_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&flag), g_fd_timeout));
  int v = 0;
  SEM_CUDA_TRY(cudaMemcpyAsync(&v, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (!v) return SEM_OK;
  SEM_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  return sem_fail(SEM_ERR_TIMEOUT, "a finite-difference step gave up waiting for its tile copy");
}
