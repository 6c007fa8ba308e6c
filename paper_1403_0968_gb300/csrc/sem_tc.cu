// Tensor-core (tcgen05) BF16 GEMM with FP32 accumulation in tensor memory, for the dense layers of
// the learned element preconditioner:  C[M][N] = act(A[M][K] B[K][N] + bias), with A the BF16
// activations (row-major, K contiguous) and B given as its transpose Bt[N][K] (BF16, K
// contiguous), i.e. both operands K-major.
//
// One block of 128 threads computes a 128 x 256 tile of C, walking K in slices of 64:
//   * the four warps copy the 128 x 64 slice of A and the 256 x 64 slice of Bt into shared memory
//     with cp.async (16 bytes per copy, zero fill past M, N or K), in the canonical no-swizzle
//     K-major layout of 8-row x 16-byte core matrices (K-adjacent core matrices 128 bytes apart,
//     8-row groups 1024 bytes apart); two stages, so the copy of slice i+1 overlaps the MMAs of
//     slice i;
//   * one thread issues four tcgen05.mma (kind::f16, M = 128, N = 256, K = 16) per slice into a
//     128-lane x 256-column FP32 accumulator in tensor memory and commits them to the stage's
//     mbarrier; a stage is refilled only after the MMAs that read it have completed (bounded wait);
//   * the epilogue moves the accumulator to registers with tcgen05.ld (warp w reads lanes
//     32w..32w+31, one row per thread), adds the bias, applies ReLU and stores FP32 or BF16.
// Tensor memory (256 columns) is allocated by warp 0 at the start and released by it at the end on
// every path; 96 KB of shared memory per block keeps at most two blocks (512 columns) on an SM, so
// the allocation never waits.
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "sem_internal.h"
#include "sem_tma.cuh"

namespace {

constexpr int TC_M = 128, TC_N = 256, TC_K = 64, TC_THREADS = 128;
constexpr int TC_LBO = 128;                   // bytes between K-adjacent core matrices
constexpr int TC_SBO = (TC_K / 8) * 128;      // bytes between 8-row groups
constexpr int TC_A_BYTES = TC_M * TC_K * 2;   // 16 KB
constexpr int TC_B_BYTES = TC_N * TC_K * 2;   // 32 KB
constexpr int TC_STAGE = TC_A_BYTES + TC_B_BYTES;
constexpr size_t TC_SMEM = 2 * TC_STAGE + 64;
static_assert(TC_SMEM * 3 > 228 * 1024, "at most two blocks per SM, so two tensor-memory allocations fit");

// shared-memory matrix descriptor of a K-major operand without swizzling
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);         // start address / 16
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;  // leading (K) byte offset / 16
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;  // stride (M or N) byte offset / 16
  d |= (uint64_t)1 << 46;                          // descriptor version
  return d;                                        // base offset 0, no swizzle
}

// instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M = 128, N = 256
__host__ __device__ constexpr uint32_t mma_idesc() {
  return (1u << 4)                         // accumulator FP32
         | (1u << 7)                       // A is BF16
         | (1u << 10)                      // B is BF16
         | ((uint32_t)(TC_N >> 3) << 17)   // N / 8
         | ((uint32_t)(TC_M >> 4) << 24);  // M / 16
}

// byte offset of element (row, k) of a K-major tile in the canonical layout
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * TC_SBO + (k >> 3) * TC_LBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// copies rows [r0, r0 + ROWS) x k [k0, k0 + 64) of a K-major BF16 matrix (nrows x K, leading
// dimension ld) into the canonical layout at sdst; out-of-range parts are zero-filled
template <int ROWS>
__device__ __forceinline__ void load_slice(uint32_t sdst, const __nv_bfloat16 *X, int nrows, int K, int ld, int r0,
                                           int k0) {
#pragma unroll 4
  for (int q = threadIdx.x; q < ROWS * (TC_K / 8); q += TC_THREADS) {
    const int row = q / (TC_K / 8), kc = (q % (TC_K / 8)) * 8;
    const int r = r0 + row, k = k0 + kc;
    const int valid = (r < nrows && k < K) ? min(8, K - k) : 0;
    const __nv_bfloat16 *src = valid ? X + (size_t)r * ld + k : X;
    cp_async16(sdst + core_off(row, kc), src, (uint32_t)valid * 2u);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt, int ldb,
              const float *bias, float *C32, __nv_bfloat16 *C16, int ldc, int relu, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * TC_STAGE);  // one per stage
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  const uint32_t s0 = smem_addr(smem);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(TC_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  const int nsl = (K + TC_K - 1) / TC_K;
  load_slice<TC_M>(s0, A, M, K, lda, m0, 0);
  load_slice<TC_N>(s0 + TC_A_BYTES, Bt, N, K, ldb, n0, 0);
  bool ok = true;
  for (int i = 0; i < nsl; ++i) {
    const uint32_t st = (uint32_t)(i & 1), sa = s0 + st * TC_STAGE, sb = sa + TC_A_BYTES;
    asm volatile("cp.async.wait_all;" ::: "memory");
    // this thread's copies are complete; make them visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t idesc = mma_idesc();
#pragma unroll
      for (int kk = 0; kk < TC_K / 16; ++kk) {
        const uint64_t ad = smem_desc(sa + kk * 2 * TC_LBO), bd = smem_desc(sb + kk * 2 * TC_LBO);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&bar[st]))
                   : "memory");
    }
    if (i + 1 < nsl) {
      if (i >= 1) {  // the other stage was read by the MMAs of slice i - 1
        const bool done = mbar_wait(&bar[st ^ 1u], (uint32_t)((i - 1) >> 1) & 1u);
        if (__syncthreads_or(!done)) {
          ok = false;
          break;
        }
      }
      const uint32_t na = s0 + (st ^ 1u) * TC_STAGE;
      load_slice<TC_M>(na, A, M, K, lda, m0, (i + 1) * TC_K);
      load_slice<TC_N>(na + TC_A_BYTES, Bt, N, K, ldb, n0, (i + 1) * TC_K);
    }
  }
  if (ok) {
    const int last = nsl - 1;
    const bool done = mbar_wait(&bar[last & 1], (uint32_t)(last >> 1) & 1u);
    if (__syncthreads_or(!done)) ok = false;
  }
  tc_fence_after();

  if (ok) {
    const int row = m0 + warp * 32 + lane;  // accumulator lane = row of the tile
#pragma unroll 1
    for (int c0 = 0; c0 < TC_N && n0 + c0 < N; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
            "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row >= M) continue;
      const int nb = n0 + c0;
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = nb + j < N ? nb + j : N - 1;
        v[j] = __uint_as_float(r[j]) + (bias ? __ldg(bias + n) : 0.f);
        if (relu) v[j] = fmaxf(v[j], 0.f);
      }
      if (nb + 32 <= N) {  // whole chunk: 16-byte stores (ldc % 8 == 0, 16-byte aligned base)
        if (C32) {
          float4 *o = reinterpret_cast<float4 *>(C32 + (size_t)row * ldc + nb);
#pragma unroll
          for (int j = 0; j < 8; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
          uint4 *o = reinterpret_cast<uint4 *>(C16 + (size_t)row * ldc + nb);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t w[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * j + 2 * t], v[8 * j + 2 * t + 1]);
              w[t] = *reinterpret_cast<const uint32_t *>(&b2);
            }
            o[j] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (nb + j >= N) break;
          if (C32) C32[(size_t)row * ldc + nb + j] = v[j];
          else C16[(size_t)row * ldc + nb + j] = __float2bfloat16_rn(v[j]);
        }
      }
    }
  } else if (tid == 0 && err) {
    atomicOr(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// C = act(A Bt^T + bias) on the tensor cores (layouts in the file comment).  A holds M rows of
// leading dimension lda >= K, Bt N rows of leading dimension ldb >= K; exactly one of C32 / C16.
sem_status sem_gemm_tc(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt, int ldb,
                       const float *bias, float *C32, __nv_bfloat16 *C16, int ldc, bool relu, int *err,
                       cudaStream_t s) {
  if (M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N || (lda % 8) || (ldb % 8) || (ldc % 8) || !A ||
      !Bt || (!C32 == !C16) || !aligned16(A) || !aligned16(Bt) || !aligned16(C32) || !aligned16(C16))
    return sem_fail(SEM_ERR_INVALID,
                    "tensor-core GEMM: needs 16-byte aligned operands, leading dimensions >= extents and % 8 == 0, "
                    "exactly one output");
  if (M > 65535 * TC_M) return sem_fail(SEM_ERR_INVALID, "tensor-core GEMM: M above 65535 tiles");
  int dev = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  static bool attr[64] = {};
  if (dev < 0 || dev >= 64) return sem_fail(SEM_ERR_INVALID, "device index out of range");
  if (!attr[dev]) {
    SEM_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    attr[dev] = true;
  }
  dim3 grid((N + TC_N - 1) / TC_N, (M + TC_M - 1) / TC_M);
  k_gemm_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(M, N, K, A, lda, Bt, ldb, bias, C32, C16, ldc, relu ? 1 : 0, err);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *d_A, int32_t lda, const void *d_Bt,
                                    int32_t ldb, const float *d_bias, float *d_C, int32_t ldc, int32_t relu,
                                    int32_t *d_err, sem_stream_t stream) {
  if (!d_A || !d_Bt || !d_C) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  return sem_gemm_tc(M, N, K, static_cast<const __nv_bfloat16 *>(d_A), lda, static_cast<const __nv_bfloat16 *>(d_Bt),
                     ldb, d_bias, d_C, nullptr, ldc, relu != 0, d_err, reinterpret_cast<cudaStream_t>(stream));
}
