// Internal declarations of libsem: the host-side handle, the device workspace layout and the
// launch helpers shared by the .cu files.  Not part of the ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/sem.h"
#include <nvtx3/nvToolsExt.h>

// A named NVTX range for the lifetime of the object (solve phases show up in ncu's NVTX filters
// and in any NVTX-aware tracer; without one attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

#define SEM_MAX_N 15
#define SEM_MAX_NP (SEM_MAX_N + 1)

// Polls of an mbarrier before a bounded wait gives up (about 10 ms at the SM clock): the default
// of every handle; sem_set_wait_limit changes it per handle.
#define SEM_WAIT_POLLS_DEFAULT (1u << 22)

// Number of partial-sum slots a solver reduction may use, and groups of 256 of them.
#define SEM_MAX_PARTIALS (1 << 20)
#define SEM_MAX_GROUPS (SEM_MAX_PARTIALS / 256)

// Device-resident solver scalars.  Every CG scalar lives here so that no iteration needs the
// host; the host reads `rr`, `converged` and `breakdown` only at check points.
struct SemScalars {
  double rz;        // (r, z) of the current iterate
  double pAp;       // (p, A p)
  double rr;        // (r, r)
  double bb;        // (b, b)
  double alpha;     // CG step length
  double beta;      // CG direction update
  double tol2;      // rtol^2 (b, b): convergence threshold on (r, r)
  double scale;     // IR: norm of the current outer residual (inner RHS is r / scale)
  int32_t converged;
  int32_t breakdown;
  int32_t iter;
  int32_t error;    // 1 if a bounded device-side wait gave up (SEM_ERR_TIMEOUT)
  unsigned int counter[8];  // last-block-done tickets, one per reduction site
  double zt;        // flexible CG: (z_new, r_old)
  int32_t fallback; // flexible CG: 1 if the learned correction was rejected this iteration
  int32_t nfallback;  // flexible CG: iterations that fell back to Jacobi
  int32_t restart_iter;  // flexible CG: iteration count at the last restart (its first iteration)
  int32_t pad2;
};

// Tag for the factor type of the on-the-fly apply (SEM_FP32_OTF): no factor stream; each element
// carries the seven non-constant coefficient vectors of its trilinear map
//   x(r,s,t) = c + r W_r + s W_s + t W_t + rs W_rs + rt W_rt + st W_st + rst W_rst
// (W_m = sum_v X_v prod_{d in m} sigma_d(v) / 8 over the vertices v with sign sigma_d(v) = +-1),
// stored as W_r, W_s, W_t, W_rs, W_rt, W_st, W_rst (x, y, z each) and three zeros of padding.
struct OtfGeo {};
#define SEM_OTF_STRIDE 24

// hidden widths of the learned element preconditioner
#define SEM_MLP_H1 256
// element-local solves of the training pairs: relative residual and iteration cap
#define SEM_MLP_LOCAL_RTOL 1e-10
#define SEM_MLP_LOCAL_MAXIT 2000
#define SEM_MLP_H2 256

struct sem_handle {
  int N, n, n3;
  int64_t E, G, L;
  int64_t gs6;   // per-element stride of G64 / G32 (6 n^3 rounded up to 4 entries: 16-byte blocks)
  int64_t gs12;  // per-element stride of Gemu (12 n^3 rounded up to 4)
  int64_t gs16;  // per-element stride of G16 (6 n^3 rounded up to 8: 16-byte blocks of BF16)
  int box[3];
  bool structured;  // box numbering computed on the fly (no glo array)
  int bc;           // sem_bc
  bool has_alpha;
  uint32_t features;
  int device;
  int apply_variant;  // kernel variant of the FP64/FP32 apply (see sem_apply_kernel.cuh), 0 = default
  uint32_t wait_polls;  // polls before a staged copy's bounded wait gives up (SEM_WAIT_POLLS_DEFAULT)

  // host copies of the derivative matrix: passed to kernels as launch parameters, so that the
  // contractions read D from the constant bank
  double D64h[SEM_MAX_NP * SEM_MAX_NP];
  double gxh[SEM_MAX_NP], gwh[SEM_MAX_NP];  // GLL points and weights (host copies)
  float D32h[SEM_MAX_NP * SEM_MAX_NP], Dhih[SEM_MAX_NP * SEM_MAX_NP], Dloh[SEM_MAX_NP * SEM_MAX_NP];

  // ---- device pointers into the caller's workspace ----
  double *D64;          // [n][n] D[i][m] = l_m'(x_i)
  float *D32;           // [n][n] FP32 copy
  float *Dhi, *Dlo;     // [n][n] double-float split of D64
  double *gll_x, *gll_w;
  double *verts;        // [E][8][3]
  double *G64;          // [E][gs6]: factor f of node p at f*n3 + p (rr, rs, rt, ss, st, tt)
  float *G32;           // [E][gs6]
  __nv_bfloat16 *G16;   // [E][gs16] BF16 copy (SEM_FEAT_BF16), gs16 = 6 n3 rounded up to 8
  float *Gemu;          // [E][gs12]: factor f hi at 2f*n3 + p, lo at (2f+1)*n3 + p
  float *Gotf;          // [E][SEM_OTF_STRIDE] trilinear-map coefficients (SEM_FEAT_OTF), see OtfGeo
  float *kap32;         // [E][n3] FP32 kappa for SEM_FP32_OTF, NULL when kappa is 1
  double *wJ;           // [E][n3] lumped mass w det J
  double *wJa64;        // [E][n3] w det J alpha (has_alpha)
  float *wJa32;         // [E][n3]
  float *wJaemu;        // [E][2][n3] hi, lo
  int32_t *glo;         // [E][n3] global ids (unstructured only)
  uint8_t *mask;        // [G] Dirichlet flags (SEM_BC_MASK only)
  double *dinv64;       // [G] 1 / diag (0 on Dirichlet nodes)
  float *dinv32;        // [G]
  // solver storage (SEM_FEAT_PCG)
  double *r64, *p64, *Ap64, *t64;       // [G]
  float *r32, *p32, *Ap32, *x32;        // [G] (IR inner solve; needs SEM_FEAT_FP32)
  double *partials;                     // [SEM_MAX_PARTIALS]
  double *gpartials;                    // [SEM_MAX_GROUPS] group sums of two-level reductions
  unsigned int *gtickets;               // [SEM_MAX_GROUPS] zeroed group counters
  SemScalars *scal;
  // learned preconditioner (SEM_FEAT_MLP)
  float *geo6;        // [E][6] normalised element-mean factors
  float *inv_mult;    // [G] 1 / number of elements sharing the node
  __nv_bfloat16 *mlp_w;  // BF16 weights transposed for the tensor cores: W1^T [h1][mlp_ldx], W2^T [h2][h1],
                         // W3^T [n3][h2], one after the other
  float *mlp_b32;        // the parameters rounded to BF16 and widened back to FP32 (biases read here)
  __nv_bfloat16 *mlp_X;  // [E][mlp_ldx] features (n3 + 6 values, zero padding)
  __nv_bfloat16 *mlp_H1, *mlp_H2;  // [E][h1], [E][h2] hidden activations
  float *mlp_scale, *mlp_O;        // [E] output scales |r_e| / dbar_e, [E][n3] outputs
  float *mlp_dbar;                 // [E] mean of the element stiffness diagonal, trace(A_e) / n3
  int mlp_h1, mlp_h2, mlp_ldx;     // mlp_ldx = n3 + 6 rounded up to a multiple of 8
  int mlp_jacobi_base;             // 1: z = D^-1 r + averaged corrections; 0: averaged corrections only
  int mlp_fused;                   // 1 (default): the three layers in one launch where the shapes allow
  double *z64;        // [G] preconditioned residual of flexible CG
};

// ----- kernel attributes -----
// Raises the dynamic shared-memory limit of `kernel` to `bytes` once per device (the attribute is
// per device; `done` is the caller's static bit set, one bit per device index < 64).
template <typename K>
cudaError_t set_smem_limit_once(K *kernel, size_t bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// GLL points x, weights w (N + 1 each) and derivative matrix D[i][j] = l_j'(x_i) (row-major) of
// order N, in FP64 on the host
void sem_gll_tables(int N, double *x, double *w, double *D);

// ----- error reporting -----
sem_status sem_fail(sem_status st, const std::string &msg);
#define SEM_CUDA_TRY(call)                                                                    \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return sem_fail(SEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e));      \
  } while (0)

// ----- shared launch entry points (defined in the .cu files) -----
// sem_apply_f32.cu / sem_apply_f64.cu / sem_apply_bf16.cu (TG: factor storage type)
template <typename T, typename TG = T>
sem_status dispatch_apply(const sem_handle *h, const T *u, T *y, const void *Gf, const T *wJa, const T *Dh,
                          double *partials, SemScalars *scal, int *err, cudaStream_t s);
// One structured-box problem inside a batched apply launch (all problems of a launch share the
// order).  Elements [elem_off, elem_off + E) of the launch belong to it; its global vectors start
// at g_off in the concatenated vectors.
struct BatchEntry {
  int64_t elem_off, E;
  int64_t gxs, gys, gzs, g_off;
  int32_t sx, sy, sz, bc;
  int32_t prob, pad;     // index of the problem in the batch (per-problem accumulators)
  const void *Gf;        // this problem's factor array (element stride gs), or its map coefficients
                         // (on-the-fly factors)
  const void *wJa;       // this problem's w det J alpha, or NULL
  const void *kap;       // on-the-fly factors: this problem's FP32 nodal kappa, or NULL for kappa = 1
  const int32_t *done;   // non-NULL: the problem's solve has stopped, skip its elements
};

// Dh: the order's derivative matrix; gx, gw: its GLL points and weights (host arrays, used by the
// on-the-fly factors)
template <typename T, typename TG = T>
sem_status dispatch_apply_batch(int N, const BatchEntry *d_entries, int nbatch, int64_t total_E, int64_t gs,
                                const T *u, T *y, const T *Dh, const double *gx, const double *gw, double *pAp,
                                int variant, cudaStream_t s);
// sem_apply.cu
sem_status sem_clear_timeout(sem_handle *h, cudaStream_t s);
sem_status sem_launch_apply(sem_handle *h, sem_prec prec, const void *u, void *y, double *pAp_partials,
                            unsigned int *ticket, double *pAp_out, cudaStream_t s);
// sem_mlp.cu
sem_status sem_mlp_setup_tables(sem_handle *h, cudaStream_t st);
sem_status sem_mlp_precond_apply(sem_handle *h, const double *r, double *z, cudaStream_t st);
// sem_mlp_targets.cu: training pairs from element-local shifted Neumann solves (Jacobi-PCG per
// element), and the per-element table dbar_e = trace(A_e) / n3
sem_status sem_mlp_local_pairs(const sem_handle *h, int nsamp, const int32_t *elems, const double *r, double eps,
                               double rtol, int maxit, int sub_jacobi, float *X, float *T, int *iters,
                               cudaStream_t st);
sem_status sem_mlp_dbar_table(const sem_handle *h, float *dbar, cudaStream_t st);
// sem_tc.cu: C = act(A Bt^T + bias) on the tensor cores (BF16 operands, K contiguous; FP32 or BF16 C)
sem_status sem_gemm_tc(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt, int ldb,
                       const float *bias, float *C32, __nv_bfloat16 *C16, int ldc, bool relu, int *err,
                       cudaStream_t s);
// sem_tc.cu: the preconditioner's three layers in one launch (hidden widths 256, nout <= 512)
sem_status sem_mlp3_tc(int M, int nin, int ldx, int nout, const __nv_bfloat16 *X, const __nv_bfloat16 *W1t,
                       const __nv_bfloat16 *W2t, const __nv_bfloat16 *W3t, const float *b1, const float *b2,
                       const float *b3, float *O, int *err, cudaStream_t s);
// sem_emu.cu
sem_status sem_launch_apply_emu(sem_handle *h, const double *u, double *y, double *partials, cudaStream_t s);
// sem_emu_tc.cu: the double-float apply with the D-contractions on the tensor cores (order 7)
sem_status sem_launch_apply_emu_tc(sem_handle *h, const double *u, double *y, double *partials, cudaStream_t s);
// sem_apply_tc32.cu: the FP32 apply with the D-contractions on the tensor cores (order 7)
sem_status sem_launch_apply_f32_tc(sem_handle *h, const float *u, float *y, double *partials, cudaStream_t s);
