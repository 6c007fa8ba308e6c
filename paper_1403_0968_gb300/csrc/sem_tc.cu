// Tensor-core (tcgen05) BF16 GEMM with FP32 accumulation in tensor memory, for the dense layers of
// the learned element preconditioner:  C[M][N] = act(A[M][K] B[K][N] + bias), with A the BF16
// activations (row-major, K contiguous) and B given as its transpose Bt[N][K] (BF16, K
// contiguous), i.e. both operands K-major.
//
// One block of 128 threads computes a 128 x 128 tile of C, walking K in slices of 64, with the
// roles split by warp:
//   * producer (one thread of warp 0): per slice, two tensor copies (cp.async.bulk.tensor, TMA)
//     bring the 128 x 64 slice of A and the 128 x 64 slice of Bt into a shared-memory stage in
//     the 128-byte-swizzled K-major layout (each row's 64 values fill one 128-byte line, the
//     16-byte chunk j of line r sits at chunk j ^ (r mod 8)); rows past M or N and columns past K
//     read as zero.  Three stages; a stage is refilled once the MMAs that read it have committed.
//   * MMA issuer (one thread of warp 1): per slice, waits for the stage's copies (mbarrier
//     transaction count), issues four tcgen05.mma (kind::f16, M = 128, N = 128, K = 16) into a
//     128-lane x 128-column FP32 accumulator in tensor memory and commits them to the stage's
//     "empty" mbarrier; after the last slice it commits once more to the "done" mbarrier.
//   * epilogue (all four warps): waits for "done", moves the accumulator to registers with
//     tcgen05.ld (warp w reads lanes 32w..32w+31, one row per thread), adds the bias, applies
//     ReLU and stores FP32 or BF16.
// Every wait is bounded; a block that gives up skips its epilogue and reports it in *err.  Tensor
// memory (128 columns) is allocated by warp 0 at the start and released by it at the end on every
// path; 97 KB of shared memory per block allows two blocks on an SM (one's epilogue overlaps the
// other's main loop) and no third, so the allocations never wait.
//
// The second kernel here, k_mlp3_tc, runs all three layers of the preconditioner's network in one
// launch with the hidden activations kept in shared memory (its comment gives the design).
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched from the driver at run time)
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include <string>

#include "sem_internal.h"
#include "sem_tma.cuh"

namespace {

constexpr int TC_M = 128, TC_N = 128, TC_K = 64, TC_THREADS = 128, TC_S = 3;
constexpr int TC_SBO = 1024;                  // bytes between 8-row groups (8 lines of 128 bytes)
constexpr int TC_A_BYTES = TC_M * TC_K * 2;   // 16 KB
constexpr int TC_B_BYTES = TC_N * TC_K * 2;   // 16 KB
constexpr int TC_STAGE = TC_A_BYTES + TC_B_BYTES;
constexpr size_t TC_SMEM = TC_S * TC_STAGE + 1024 + 128;  // + alignment slack, barriers, TMEM address
static_assert(TC_SMEM * 3 > 228 * 1024 && 2 * TC_N <= 512,
              "at most two blocks per SM, so both tensor-memory allocations always fit");
static_assert(TC_M * TC_N * 4 <= TC_S * TC_STAGE, "the FP32 output tile fits in the operand stages");
static_assert(TC_SMEM <= 227 * 1024, "shared memory per block");
static_assert(TC_K * 2 == 128, "one 128-byte swizzle line per row and slice");

// shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled layout; the start
// address may step by 32 bytes (16 values of K) inside a 1024-byte-aligned swizzle atom
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);         // start address / 16
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;  // stride (M or N) byte offset / 16
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // layout: 128-byte swizzle; base offset 0
  return d;
}

// instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M = 128, N = TC_N
__host__ __device__ constexpr uint32_t mma_idesc() {
  return (1u << 4)                         // accumulator FP32
         | (1u << 7)                       // A is BF16
         | (1u << 10)                      // B is BF16
         | ((uint32_t)(TC_N >> 3) << 17)   // N / 8
         | ((uint32_t)(TC_M >> 4) << 24);  // M / 16
}

// 2-D tensor copy global -> shared (128-byte swizzle per the tensor map), completing on bar
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmC, int M, int N, int K, const float *bias, float *C32,
              __nv_bfloat16 *C16, int relu, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // barriers: full[TC_S] (copies landed), empty[TC_S] (MMAs done with the stage), done
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + TC_S * TC_STAGE + 1024);
  uint64_t *empty = full + TC_S, *done = empty + TC_S;
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(done + 1);
  __shared__ int s_fail, s_issued, s_consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  const uint32_t s0 = (smem_addr(smem) + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(TC_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int j = 0; j < TC_S; ++j) {
      mbar_init(&full[j], 1);
      mbar_init(&empty[j], 1);
    }
    mbar_init(done, 1);
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  const int nsl = (K + TC_K - 1) / TC_K;
  if (tid == 0) {  // producer
    for (int j = 0; j < nsl; ++j) {
      const int st = j % TC_S;
      if (j >= TC_S && !mbar_wait(&empty[st], (uint32_t)((j / TC_S) - 1) & 1u)) {
        atomicOr(&s_fail, 1);
        break;
      }
      const uint32_t sa = s0 + (uint32_t)st * TC_STAGE;
      mbar_expect_tx(&full[st], (uint32_t)TC_STAGE);
      tma_load_2d(sa, &tmA, j * TC_K, m0, &full[st]);
      tma_load_2d(sa + TC_A_BYTES, &tmB, j * TC_K, n0, &full[st]);
      s_issued = j + 1;
    }
  } else if (tid == 32) {  // MMA issuer
    const uint32_t idesc = mma_idesc();
    for (int i = 0; i < nsl; ++i) {
      const int st = i % TC_S;
      if (!mbar_wait(&full[st], (uint32_t)(i / TC_S) & 1u)) {
        atomicOr(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const uint32_t sa = s0 + (uint32_t)st * TC_STAGE, sb = sa + TC_A_BYTES;
#pragma unroll
      for (int kk = 0; kk < TC_K / 16; ++kk) {
        const uint64_t ad = smem_desc(sa + kk * 32), bd = smem_desc(sb + kk * 32);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&empty[st]))
                   : "memory");
      s_consumed = i + 1;
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(done))
                 : "memory");
  }
  __syncwarp();
  // the accumulator is complete once "done" flips (bounded wait; a failed role skips it)
  bool ok = mbar_wait(done, 0u);
  __syncthreads();  // the producer and MMA threads have left their loops: s_fail is final
  ok = !__syncthreads_or(!ok || s_fail != 0);
  tc_fence_after();

  if (ok) {
    // The output tile goes through shared memory (the operand stages are free now) in the 128-byte
    // swizzled layout, one 16 KB block per 128 bytes of columns, and leaves by tensor stores, so that
    // every global write is a full coalesced line; rows past M and columns past N are clipped by
    // the tensor map.  es = element size of C.
    const int es = C32 ? 4 : 2, cols_per_block = 128 / es;
    const int r = warp * 32 + lane;  // accumulator lane = row of the tile
    const uint32_t rbase = s0 + (uint32_t)r * 128u;
#pragma unroll 1
    for (int c0 = 0; c0 < TC_N && n0 + c0 < N; c0 += 32) {
      uint32_t acc[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(acc[0]), "=r"(acc[1]), "=r"(acc[2]), "=r"(acc[3]), "=r"(acc[4]), "=r"(acc[5]), "=r"(acc[6]),
            "=r"(acc[7]), "=r"(acc[8]), "=r"(acc[9]), "=r"(acc[10]), "=r"(acc[11]), "=r"(acc[12]), "=r"(acc[13]),
            "=r"(acc[14]), "=r"(acc[15]), "=r"(acc[16]), "=r"(acc[17]), "=r"(acc[18]), "=r"(acc[19]),
            "=r"(acc[20]), "=r"(acc[21]), "=r"(acc[22]), "=r"(acc[23]), "=r"(acc[24]), "=r"(acc[25]),
            "=r"(acc[26]), "=r"(acc[27]), "=r"(acc[28]), "=r"(acc[29]), "=r"(acc[30]), "=r"(acc[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = n0 + c0 + j < N ? n0 + c0 + j : N - 1;
        v[j] = __uint_as_float(acc[j]) + (bias ? __ldg(bias + n) : 0.f);
        if (relu) v[j] = fmaxf(v[j], 0.f);
      }
      // 16-byte chunks of this row's 32 values: 8 (FP32) or 4 (BF16)
      const int byte0 = c0 * es, blk = byte0 / 128, off = byte0 % 128;
      const uint32_t line = rbase + (uint32_t)blk * (TC_M * 128u);
      if (C32) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const uint32_t ch = (uint32_t)(((off >> 4) + t) ^ (r & 7));
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(line + ch * 16u), "f"(v[4 * t]),
                       "f"(v[4 * t + 1]), "f"(v[4 * t + 2]), "f"(v[4 * t + 3])
                       : "memory");
        }
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          uint32_t w[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * t + 2 * q], v[8 * t + 2 * q + 1]);
            w[q] = *reinterpret_cast<const uint32_t *>(&b2);
          }
          const uint32_t ch = (uint32_t)(((off >> 4) + t) ^ (r & 7));
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(line + ch * 16u), "r"(w[0]), "r"(w[1]),
                       "r"(w[2]), "r"(w[3])
                       : "memory");
        }
      }
    }
    // generic-proxy writes -> visible to the tensor (async) proxy, then one thread stores the blocks
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      const int nblk = (min(TC_N, N - n0) * es + 127) / 128;
      for (int b = 0; b < nblk; ++b)
        asm volatile(
            "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                reinterpret_cast<uint64_t>(&tmC)),
            "r"(n0 + b * cols_per_block), "r"(m0), "r"(s0 + (uint32_t)b * (TC_M * 128u))
            : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // shared memory read before exit
    }
  } else if (tid == 0) {
    if (err) atomicOr(err, 1);
    // a role gave up: wait (bounded) for the tensor copies that were issued but never consumed, so
    // that none is still writing this block's shared memory when it exits
    for (int j = s_consumed; j < s_issued; ++j) mbar_wait(&full[j % TC_S], (uint32_t)(j / TC_S) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
}

// ---------------------------------------------------------------------------------------------
// The three layers in one kernel: O = (relu(relu(X W1 + b1) W2 + b2)) W3 + b3, hidden widths 256,
// the hidden activations rounded to BF16 exactly as the layer-by-layer path rounds them, but kept
// in shared memory instead of going out to global memory and back.  One block per tile of 128
// element rows (1 block per SM: all 512 tensor-memory columns, 209 KB of shared memory); roles by
// warp:
//   * warp 0 (one thread), producer: stage loads by tensor copy, per K slice of 64: layer 1 the
//     128 x 64 slice of X and the 256 x 64 slice of W1^T, layer 2 a 256 x 64 slice of W2^T,
//     layer 3 a 256 x 64 slice of W3^T per half of the outputs (rows past n_out read as zero).
//     Three 48 KB stages; it runs ahead into the next layer's weights while an epilogue works.
//   * warp 1 (one thread), MMA issuer: layer 1 into tensor-memory columns 0..255, layer 2 (A =
//     the BF16 activations in shared memory) into columns 256..511, layer 3 into columns
//     0..n_out-1 (two MMAs of N <= 256 per K step when n_out > 256).
//   * warps 2..5, epilogue: accumulator rows to registers (warp w reads lanes 32 (w mod 4) ..),
//     bias, ReLU and BF16 into the 64 KB activation buffer in the 128-byte swizzled K-major
//     layout the MMA reads (K block c / 64, row r at r * 128 bytes, 16-byte chunk j at
//     j ^ (r mod 8)); after layer 3, bias and FP32 output by tensor stores through four 16 KB
//     slots of the same buffer.
// Hand-over by mbarriers: full/empty per stage, acc1/acc2/acc3 (tcgen05.commit after a layer's
// MMAs), h1/h2 (128 epilogue arrivals once the activations are written and fenced for the async
// proxy).  Every wait is bounded; a role that gives up records it, the waits of the others then
// run out, and tensor memory is released only after the MMAs and copies in flight have completed.
constexpr int F_M = 128, F_H = 256, F_K = 64, F_S = 3, F_THREADS = 192;
constexpr int F_H_BYTES = F_M * F_H * 2;         // 64 KB: four K blocks of 16 KB
constexpr int F_KBLK = F_M * 128;                // one K block (64 values) of a 128-row operand
constexpr int F_A_BYTES = F_M * F_K * 2;         // 16 KB
constexpr int F_B_BYTES = F_H * F_K * 2;         // 32 KB
constexpr int F_STAGE = F_A_BYTES + F_B_BYTES;   // 48 KB
constexpr size_t F_SMEM = F_H_BYTES + F_S * F_STAGE + 1024 + 256;
static_assert(F_SMEM + 4 * 256 * 4 + 1024 <= 227 * 1024, "shared memory per block (with the static biases)");
static_assert(F_SMEM * 2 > 228 * 1024, "one block per SM, so the 512-column allocation never waits");
static_assert(F_KBLK == 16384 && F_STAGE % 1024 == 0, "swizzle atoms stay 1024-byte aligned");

__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(F_M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t a[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
        "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]),
        "=r"(a[16]), "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]),
        "=r"(a[24]), "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(a[j]);
}

// OR of v over the 128 epilogue threads (named barrier 1): every one of them takes the same branch
__device__ __forceinline__ bool epi_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, 128, q;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// a 256-wide accumulator (columns col0..col0+255 of this thread's lane) -> relu(acc + bias) in BF16,
// row r of the activation buffer (bias in shared memory)
__device__ __forceinline__ void hidden_to_smem(uint32_t taddr, uint32_t sH, int r, const float *bias) {
#pragma unroll 1
  for (int c0 = 0; c0 < F_H; c0 += 32) {
    float v[32];
    tmem_ld32(taddr + (uint32_t)c0, v);
    const uint32_t line = sH + (uint32_t)(c0 / F_K) * F_KBLK + (uint32_t)r * 128u;
    const int ch0 = (c0 % F_K) * 2 / 16;  // first 16-byte chunk of these 32 values in the line
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = 8 * t + 2 * q;
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(fmaxf(v[j] + bias[c0 + j], 0.f),
                                                        fmaxf(v[j + 1] + bias[c0 + j + 1], 0.f));
        w[q] = *reinterpret_cast<const uint32_t *>(&b2);
      }
      const uint32_t ch = (uint32_t)((ch0 + t) ^ (r & 7));
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(line + ch * 16u), "r"(w[0]), "r"(w[1]),
                   "r"(w[2]), "r"(w[3])
                   : "memory");
    }
  }
}

__global__ void __launch_bounds__(F_THREADS, 1)
    k_mlp3_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
              const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmW3,
              const __grid_constant__ CUtensorMap tmO, int nin, int nout, const float *b1, const float *b2,
              const float *b3, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + F_H_BYTES + F_S * F_STAGE + 1024);
  uint64_t *empty = full + F_S, *acc1 = empty + F_S, *acc2 = acc1 + 1, *acc3 = acc1 + 2, *h1 = acc1 + 3,
           *h2 = acc1 + 4, *fin = acc1 + 5;
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(fin + 1);
  __shared__ int s_fail, s_issued, s_consumed;
  __shared__ float s_bias[4 * F_H];  // b1 | b2 | b3 (zero past n_out)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * F_M;
  const uint32_t s0 = (smem_addr(smem) + 1023u) & ~1023u;
  const uint32_t sH = s0, sSt = s0 + F_H_BYTES;
  const int nsl1 = (nin + F_K - 1) / F_K, nh3 = nout > F_H ? 2 : 1;
  const int nq = nsl1 + F_H / F_K + nh3 * (F_H / F_K);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(2 * F_H)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int j = 0; j < F_S; ++j) {
      mbar_init(&full[j], 1);
      mbar_init(&empty[j], 1);
    }
    mbar_init(acc1, 1);
    mbar_init(acc2, 1);
    mbar_init(acc3, 1);
    mbar_init(h1, 128);
    mbar_init(h2, 128);
    mbar_init(fin, 1);
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (tid == 0) {  // producer
    for (int q = 0; q < nq; ++q) {
      const int st = q % F_S;
      if (q >= F_S && !mbar_wait(&empty[st], (uint32_t)((q / F_S) - 1) & 1u)) {
        atomicOr(&s_fail, 1);
        break;
      }
      const uint32_t sa = sSt + (uint32_t)st * F_STAGE, sb = sa + F_A_BYTES;
      if (q < nsl1) {
        mbar_expect_tx(&full[st], (uint32_t)F_STAGE);
        tma_load_2d(sa, &tmX, q * F_K, m0, &full[st]);
        tma_load_2d(sb, &tmW1, q * F_K, 0, &full[st]);
      } else if (q < nsl1 + F_H / F_K) {
        mbar_expect_tx(&full[st], (uint32_t)F_B_BYTES);
        tma_load_2d(sb, &tmW2, (q - nsl1) * F_K, 0, &full[st]);
      } else {
        const int t = q - nsl1 - F_H / F_K;
        mbar_expect_tx(&full[st], (uint32_t)F_B_BYTES);
        tma_load_2d(sb, &tmW3, (t % 4) * F_K, (t / 4) * F_H, &full[st]);
      }
      s_issued = q + 1;
    }
  } else if (tid == 32) {  // MMA issuer
    const uint32_t id_h = idesc_bf16(F_H);
    const int na = nout < F_H ? nout : F_H;
    const uint32_t id_a = idesc_bf16((na + 15) & ~15), id_b = idesc_bf16(nh3 == 2 ? ((nout - F_H + 15) & ~15) : 16);
    bool ok = true;
    for (int q = 0; q < nq; ++q) {
      const int st = q % F_S;
      if (q == nsl1 || q == nsl1 + F_H / F_K) {  // a layer is issued: its accumulator to the epilogue
        mma_commit(q == nsl1 ? acc1 : acc2);
        if (!mbar_wait(q == nsl1 ? h1 : h2, 0u)) {  // the activations it reads next
          ok = false;
          break;
        }
        tc_fence_after();
      }
      if (!mbar_wait(&full[st], (uint32_t)(q / F_S) & 1u)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = sSt + (uint32_t)st * F_STAGE, sb = sa + F_A_BYTES;
      uint32_t abase, d, id;
      int j;
      if (q < nsl1) {
        j = q;
        abase = sa;
        d = tmem;
        id = id_h;
      } else if (q < nsl1 + F_H / F_K) {
        j = q - nsl1;
        abase = sH + (uint32_t)j * F_KBLK;
        d = tmem + F_H;
        id = id_h;
      } else {
        const int t = q - nsl1 - F_H / F_K;
        j = t % 4;
        abase = sH + (uint32_t)j * F_KBLK;
        d = tmem + (uint32_t)((t / 4) * F_H);
        id = t / 4 ? id_b : id_a;
      }
#pragma unroll
      for (int kk = 0; kk < F_K / 16; ++kk)
        mma_bf16(d, smem_desc(abase + kk * 32), smem_desc(sb + kk * 32), id, (j > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[st]);
      s_consumed = q + 1;
    }
    if (ok) mma_commit(acc3);
    else atomicOr(&s_fail, 1);
    mma_commit(fin);  // arrives once every MMA issued above has completed
  } else if (warp >= 2) {  // epilogue
    const int qd = warp & 3, r = qd * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(qd * 32) << 16);
    const bool issuer = tid == 64;
    for (int i = tid - 64; i < 4 * F_H; i += 128)  // published to the other epilogue warps by epi_any
      s_bias[i] = i < F_H ? b1[i] : i < 2 * F_H ? b2[i - F_H] : (i - 2 * F_H < nout ? b3[i - 2 * F_H] : 0.f);
    bool bad = epi_any(!mbar_wait(acc1, 0u));
    if (!bad) {
      tc_fence_after();
      hidden_to_smem(tl, sH, r, s_bias);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      mbar_arrive(h1);
      bad = epi_any(!mbar_wait(acc2, 0u));
    }
    if (!bad) {
      tc_fence_after();
      hidden_to_smem(tl + F_H, sH, r, s_bias + F_H);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      mbar_arrive(h2);
      bad = epi_any(!mbar_wait(acc3, 0u));
    }
    if (!bad) {
      tc_fence_after();
      const int nch = (nout + 31) / 32;
#pragma unroll 1
      for (int c = 0; c < nch; ++c) {
        const uint32_t slot = sH + (uint32_t)(c % 4) * F_KBLK;
        if (c >= 4) {  // the store that read this slot four chunks ago has finished reading it
          if (issuer) asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory");
          epi_sync();
        }
        float v[32];
        tmem_ld32(tl + (uint32_t)(c * 32), v);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          float o[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            o[q] = v[4 * t + q] + s_bias[2 * F_H + c * 32 + 4 * t + q];
          }
          const uint32_t ch = (uint32_t)(t ^ (r & 7));
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(slot + (uint32_t)r * 128u + ch * 16u),
                       "f"(o[0]), "f"(o[1]), "f"(o[2]), "f"(o[3])
                       : "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_sync();
        if (issuer) {
          asm volatile(
              "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                  reinterpret_cast<uint64_t>(&tmO)),
              "r"(c * 32), "r"(m0), "r"(slot)
              : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      if (issuer) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    if (bad && lane == 0) atomicOr(&s_fail, 1);
  }
  __syncwarp();
  __syncthreads();  // every role has left its loop (all waits are bounded)
  if (tid == 0) {
    if (s_fail) {
      if (err) atomicOr(err, 1);
      // copies issued but never consumed must land before this block's shared memory goes away
      for (int j = s_consumed; j < s_issued; ++j) mbar_wait(&full[j % F_S], (uint32_t)(j / F_S) & 1u);
    }
    mbar_wait(fin, 0u);  // the MMAs have completed before their tensor memory is released
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * F_H) : "memory");
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// cuTensorMapEncodeTiled from the driver (through the runtime, so nothing links libcuda directly)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

// a row-major matrix (rows x cols of es-byte elements, leading dimension ld elements) as a 2-D
// tensor map whose box is box_cols x box_rows, 128-byte swizzled in shared memory; loads outside
// the matrix return zeros, stores outside it are dropped
bool make_map(CUtensorMap *m, CUtensorMapDataType type, int es, const void *base, int rows, int cols, int ld,
              int box_cols, int box_rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * es};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, type, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

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
  static std::atomic<unsigned long long> attr_done;
  SEM_CUDA_TRY(set_smem_limit_once(k_gemm_tc, TC_SMEM, attr_done));
  CUtensorMap tmA, tmB, tmC;
  const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const bool okmap = make_map(&tmA, bf, 2, A, M, K, lda, TC_K, TC_M) && make_map(&tmB, bf, 2, Bt, N, K, ldb, TC_K, TC_N) &&
                     (C32 ? make_map(&tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, C32, M, N, ldc, 32, TC_M)
                          : make_map(&tmC, bf, 2, C16, M, N, ldc, 64, TC_M));
  if (!okmap) return sem_fail(SEM_ERR_CUDA, "tensor-core GEMM: tensor map encoding failed");
  dim3 grid((N + TC_N - 1) / TC_N, (M + TC_M - 1) / TC_M);
  k_gemm_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(tmA, tmB, tmC, M, N, K, bias, C32, C16, relu ? 1 : 0, err);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

// O = (relu(relu(X W1t^T + b1) W2t^T + b2)) W3t^T + b3 in one launch (k_mlp3_tc): X [M][ldx] with
// nin features, W1t [256][ldx], W2t [256][256], W3t [nout][256] (BF16, K contiguous), O [M][nout]
// FP32; hidden widths 256, 8 <= nout <= 512 and a multiple of 8.
sem_status sem_mlp3_tc(int M, int nin, int ldx, int nout, const __nv_bfloat16 *X, const __nv_bfloat16 *W1t,
                       const __nv_bfloat16 *W2t, const __nv_bfloat16 *W3t, const float *b1, const float *b2,
                       const float *b3, float *O, int *err, cudaStream_t s) {
  if (M < 1 || nin < 1 || ldx < nin || (ldx % 8) || nout < 8 || nout > 2 * F_H || (nout % 8) || !X || !W1t ||
      !W2t || !W3t || !b1 || !b2 || !b3 || !O || !aligned16(X) || !aligned16(W1t) || !aligned16(W2t) ||
      !aligned16(W3t) || !aligned16(O))
    return sem_fail(SEM_ERR_INVALID,
                    "fused tensor-core layers: needs 16-byte aligned operands, ldx >= nin and % 8 == 0, "
                    "8 <= nout <= 512 and % 8 == 0");
  static std::atomic<unsigned long long> attr_done;
  SEM_CUDA_TRY(set_smem_limit_once(k_mlp3_tc, F_SMEM, attr_done));
  CUtensorMap tmX, tmW1, tmW2, tmW3, tmO;
  const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const bool okmap = make_map(&tmX, bf, 2, X, M, nin, ldx, F_K, F_M) &&
                     make_map(&tmW1, bf, 2, W1t, F_H, nin, ldx, F_K, F_H) &&
                     make_map(&tmW2, bf, 2, W2t, F_H, F_H, F_H, F_K, F_H) &&
                     make_map(&tmW3, bf, 2, W3t, nout, F_H, F_H, F_K, F_H) &&
                     make_map(&tmO, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, O, M, nout, nout, 32, F_M);
  if (!okmap) return sem_fail(SEM_ERR_CUDA, "fused tensor-core layers: tensor map encoding failed");
  k_mlp3_tc<<<(unsigned)((M + F_M - 1) / F_M), F_THREADS, F_SMEM, s>>>(tmX, tmW1, tmW2, tmW3, tmO, nin, nout, b1,
                                                                     b2, b3, err);
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

extern "C" sem_status sem_mlp_layers_bf16(int32_t M, int32_t nin, int32_t ldx, int32_t nout, const void *d_X,
                                          const void *d_W1t, const void *d_W2t, const void *d_W3t, const float *d_b1,
                                          const float *d_b2, const float *d_b3, float *d_O, int32_t *d_err,
                                          sem_stream_t stream) {
  if (!d_X || !d_W1t || !d_W2t || !d_W3t || !d_b1 || !d_b2 || !d_b3 || !d_O)
    return sem_fail(SEM_ERR_INVALID, "NULL argument");
  using B = const __nv_bfloat16 *;
  return sem_mlp3_tc(M, nin, ldx, nout, static_cast<B>(d_X), static_cast<B>(d_W1t), static_cast<B>(d_W2t),
                     static_cast<B>(d_W3t), d_b1, d_b2, d_b3, d_O, d_err, reinterpret_cast<cudaStream_t>(stream));
}
