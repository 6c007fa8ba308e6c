/*
 * sem.h — C ABI of the GB300 spectral-element operator library (libsem.so).
 *
 * The library applies and inverts the spectral-element discretisation of the screened-Poisson
 * problem of arXiv 1403.0968 §4.2:
 *     -div(kappa grad u) + alpha u = f   in Omega subset R^3                  (§4.2, Eq. 1)
 *     <kappa grad u, grad v> + <alpha u, v> = <f, v>,  u, v in V              (§4.2.1, Eq. 2)
 * on hexahedral elements with tensor-product Lagrange bases on the N+1 Gauss-Lobatto-Legendre
 * nodes, GLL quadrature, a lumped mass matrix, per-node geometric factors G-hat = G^T G scaled by
 * J w kappa (§4.2.1, sum-factorised stiffness display) and distinct global/local numbering with
 * direct-stiffness summation (§4.2.1, last paragraph).  The linear solver is preconditioned CG
 * (§4.2.2).
 *
 * Conventions shared by every call:
 *   n = N+1; element-local node (i,j,k) has index i + n*(j + n*k) (i along r);
 *   vertex v = a + 2b + 4c of an element sits at reference corner (2a-1, 2b-1, 2c-1);
 *   a structured box of sx*sy*sz elements numbers element (ex,ey,ez) as ex + sx*(ey + sy*ez) and
 *   global node (I,J,K) (I = ex*N + i, ...) as I + (sx*N+1)*(J + (sy*N+1)*K);
 *   "global vectors" have one entry per global node, "local arrays" are [nelem][n^3].
 *   Device pointers (prefix d_) must be valid CUDA device memory of the current device; every
 *   call is asynchronous on the given stream unless stated otherwise.
 * Errors are returned as sem_status; nothing aborts or exits.  sem_last_error() gives a message
 * (thread-local, valid until the next call on the same thread).
 * The library never allocates device memory after sem_setup: all device storage lives in the
 * caller-owned workspace.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-identical to cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *sem_stream_t;

typedef enum {
  SEM_OK = 0,
  SEM_ERR_INVALID = 1,    /* bad argument, unsupported order or size */
  SEM_ERR_CUDA = 2,       /* a CUDA runtime call or kernel launch failed */
  SEM_ERR_NOCONV = 3,     /* solver hit max_it before reaching rtol */
  SEM_ERR_BREAKDOWN = 4,  /* non-finite or non-positive CG scalar */
  SEM_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up (sem_apply_status, sem_pcg) */
  SEM_ERR_WORKSPACE = 6   /* workspace too small or misaligned */
} sem_status;

/* Arithmetic of an operator apply. */
typedef enum {
  SEM_FP64 = 0,      /* FP64 vectors, FP64 factors, FP64 arithmetic */
  SEM_FP64_EMU = 1,  /* FP64 vectors and factors, arithmetic in pairs of FP32 (double-float), with each
                        element's u scaled by an exact power of two so that any FP64 magnitude of u
                        keeps FP64-level accuracy (FP64 subnormals are flushed to zero) */
  SEM_FP32 = 2,      /* FP32 vectors, FP32 factors, FP32 arithmetic */
  /* 3 is not used: a TF32 tensor-core apply would not beat the HBM-bound FP32 kernel */
  SEM_BF16 = 4,      /* FP32 vectors, factors stored in BF16 (rounded to nearest from FP64 at set-up),
                        FP32 arithmetic: half the factor traffic, about 2^-9 relative error per factor */
  SEM_FP32_OTF = 5   /* FP32 vectors and arithmetic, the six factors recomputed at every node from the
                        element's trilinear map (21 coefficients per element) instead of read: no
                        factor stream (kappa, when not 1, is read as one FP32 value per local node) */
} sem_prec;

/* Boundary condition. */
typedef enum {
  SEM_BC_NONE = 0,  /* pure Neumann: the operator is the full assembled A */
  SEM_BC_BOX = 1,   /* homogeneous Dirichlet on every boundary node of the structured box */
  SEM_BC_MASK = 2   /* homogeneous Dirichlet where dirichlet[g] != 0 */
} sem_bc;

/* Feature bits for sem_workspace_size / sem_setup: which factor sets and solver storage exist. */
enum {
  SEM_FEAT_FP64 = 1u << 0,  /* FP64 factors (SEM_FP64 apply, FP64 Jacobi-PCG) */
  SEM_FEAT_EMU = 1u << 1,   /* factors as FP32 hi/lo pairs (SEM_FP64_EMU apply); set-up refuses it
                               (SEM_ERR_INVALID) when a factor exceeds 2^60 or a diagonal factor
                               (rr, ss, tt) falls below 2^-60 in magnitude */
  SEM_FEAT_FP32 = 1u << 2,  /* FP32 factors (SEM_FP32 apply, FP32 inner solves) */
  SEM_FEAT_PCG = 1u << 3,   /* solver vectors for sem_pcg */
  SEM_FEAT_MLP = 1u << 4,   /* learned element preconditioner: tables, activations, weights */
  SEM_FEAT_BF16 = 1u << 5,  /* BF16 factors (SEM_BF16 apply, BF16 inner solves of refinement); needs
                               one of the other factor sets as well */
  SEM_FEAT_OTF = 1u << 6    /* per-element map coefficients for SEM_FP32_OTF (and OTF inner solves of
                               refinement): 96 bytes per element, plus FP32 kappa per local node when
                               kappa is not 1.  May be the only factor set. */
};

/*
 * One problem.  All arrays are HOST pointers read only during sem_setup.
 *   N          polynomial order, 1..15.
 *   box        element counts (sx, sy, sz) of a structured box; used for numbering when
 *              glo_num == NULL and for SEM_BC_BOX.
 *   nelem      number of elements (= sx*sy*sz for a box).
 *   vertices   [nelem][8][3] trilinear element vertices.
 *   glo_num    [nelem][n^3] global ids in [0, nglobal), or NULL for box numbering.
 *   nglobal    number of global nodes (ignored, and computed, for box numbering).
 *   kappa_modes, kappa_nmodes   kappa(x) = exp(sum_m a_m cos(2 pi k_m.x + phi_m)), rows
 *              (kx, ky, kz, phi, a); nmodes = 0 means kappa = 1.
 *   kappa      [nelem][n^3] nodal kappa; overrides kappa_modes when non-NULL.
 *   alpha      [nelem][n^3] nodal screening coefficient alpha, or NULL for alpha = 0.
 *   bc         sem_bc; dirichlet [nglobal] flags for SEM_BC_MASK.
 */
typedef struct {
  int32_t N;
  int32_t box[3];
  int64_t nelem;
  const double *vertices;
  const int64_t *glo_num;
  int64_t nglobal;
  int32_t kappa_nmodes;
  const double *kappa_modes;
  const double *kappa;
  const double *alpha;
  int32_t bc;
  const uint8_t *dirichlet;
} sem_desc;

typedef struct sem_handle sem_handle;

/*
 * Bytes of device workspace sem_setup needs for this problem and feature set (features: OR of
 * SEM_FEAT_*).  Pure host computation.  Returns SEM_ERR_INVALID for an unsupported order, an
 * empty or inconsistent description.
 */
sem_status sem_workspace_size(const sem_desc *desc, uint32_t features, size_t *bytes);

/*
 * Builds everything the applies and solves need inside d_workspace (caller-owned device memory
 * of at least sem_workspace_size bytes, 256-byte aligned): GLL nodes, derivative matrix,
 * per-node geometric factors (§4.2.1: w_i w_j w_k det J kappa (d r/d x)(d r/d x)^T, six per node),
 * lumped mass w det J, numbering, Dirichlet mask and the assembled Jacobi diagonal.  Copies the
 * host arrays to the device (synchronously) and runs the set-up kernels on `stream`; returns
 * after the stream has finished.  *out receives a host-side handle; the workspace must outlive it.
 * Errors: SEM_ERR_INVALID (description), SEM_ERR_WORKSPACE (size or alignment), SEM_ERR_CUDA;
 * SEM_ERR_INVALID also when an element is tangled (det J <= 0 at some node).
 */
sem_status sem_setup(const sem_desc *desc, uint32_t features, void *d_workspace, size_t bytes,
                     sem_stream_t stream, sem_handle **out);

/* Releases the host handle (not the workspace).  NULL is allowed. */
void sem_free(sem_handle *h);

/*
 * y = M A M u: the assembled spectral-element operator (stiffness plus lumped mass term when
 * alpha was given) with M the Dirichlet mask, by sum factorisation (§4.2.1, sum-factorised
 * stiffness display): gather Q, D-contractions along r, s, t, per-node 6-factor scaling,
 * transposed contractions, direct-stiffness scatter-add Q^T.
 *   prec   SEM_FP64 / SEM_FP64_EMU: d_u, d_y are double[nglobal];  SEM_FP32, SEM_BF16,
 *          SEM_FP32_OTF: float[nglobal].
 *   d_u and d_y must not alias.  d_y is overwritten (entries on Dirichlet nodes become 0).
 * Asynchronous: a staged factor copy whose bounded wait gave up is reported later by
 * sem_apply_status (SEM_ERR_TIMEOUT).
 * Errors: SEM_ERR_INVALID if the handle lacks the factor set for prec, SEM_ERR_CUDA.
 */
sem_status sem_apply(sem_handle *h, sem_prec prec, const void *d_u, void *d_y, sem_stream_t stream);

/*
 * Synchronises `stream` and reports whether an apply on this handle (sem_apply, or one inside a
 * solve) gave up waiting for its staged factor copy since the last check: SEM_ERR_TIMEOUT, and
 * the flag is cleared (together with the handle's reduction tickets); that apply's output is
 * incomplete.  SEM_OK otherwise.  sem_pcg checks the same flag at every host check point and
 * returns SEM_ERR_TIMEOUT.  Errors: SEM_ERR_INVALID, SEM_ERR_CUDA.
 */
sem_status sem_apply_status(sem_handle *h, sem_stream_t stream);

/*
 * Number of polls after which the bounded wait of a staged factor copy gives up, for the applies
 * of this handle: polls < 0 restores the default (2^22 polls, about 10 ms), 0 makes every staged
 * wait give up at once.  A block whose wait gave up records the timeout, waits (with the default
 * bound) for its own copy and leaves without scattering, so the error path runs without a fault
 * or a hang: this is how the timeout status is tested.  Errors: SEM_ERR_INVALID.
 */
sem_status sem_set_wait_limit(sem_handle *h, int64_t polls);

/*
 * Selects the kernel variant of the apply for this handle (tile shape: elements per thread block
 * and whether the per-element factor block is staged in shared memory by a bulk TMA copy):
 *   -1 automatic (the default after sem_setup): a per-order choice measured on GB300;
 *   0 default elements per block, factors staged (when they fit); 1 default, factors read from
 *   global memory; 2 twice the elements per block, factors from global; 3 half the elements per
 *   block, staged; 4 persistent blocks that double-buffer the next tile's factors by TMA and
 *   prefetch its u (structured boxes; otherwise as 0); 5 (order 7 only: the D-contractions on
 *   the tensor cores — SEM_FP64_EMU by exact TF32 slicing to its FP64 accuracy, SEM_FP32 by
 *   two-slice TF32 ("3xTF32") with FP32 accumulation, about 2^-22 of |D||v| per line product;
 *   at other orders SEM_FP64_EMU treats 5 as 1 and the other precisions as 0; on GB300 both
 *   measured slower than their CUDA-core kernels, which stay the automatic choice).
 *   SEM_FP64_EMU distinguishes 0 (staged) from 1..4 (direct reads); SEM_FP32_OTF has no factor
 *   block, so 0, 1 and 4 coincide.
 * All variants compute the same operator (results differ by the order of the atomic scatter-add
 * and, for variant 5 of SEM_FP32, by the TF32 slicing).  Used by autotuning.  Errors:
 * SEM_ERR_INVALID.
 */
sem_status sem_set_apply_variant(sem_handle *h, int32_t variant);

/*
 * b = M Q^T (w det J f): the lumped-mass load vector of the right-hand side <f, v> (§4.2.1,
 * Eq. 2 and the lumped-mass display) from nodal values d_fL[nelem][n^3] (double).  d_b is
 * double[nglobal], overwritten.
 */
sem_status sem_rhs(sem_handle *h, const double *d_fL, double *d_b, sem_stream_t stream);

/* Physical coordinates of every element-local node, d_xyz[nelem][n^3][3] (double). */
sem_status sem_node_coords(sem_handle *h, double *d_xyz, sem_stream_t stream);

/* Global id of every element-local node, d_glo[nelem][n^3] (int64) — for bit-exact checks. */
sem_status sem_glo_num(sem_handle *h, int64_t *d_glo, sem_stream_t stream);

/* Assembled diagonal of M A M (1 on Dirichlet nodes), d_diag double[nglobal]. */
sem_status sem_diag(sem_handle *h, double *d_diag, sem_stream_t stream);

/* Sizes of a set-up problem: N, nelem, nglobal, number of local nodes. */
typedef struct {
  int32_t N;
  int64_t nelem;
  int64_t nglobal;
  int64_t nlocal;
} sem_info;
sem_status sem_get_info(const sem_handle *h, sem_info *info);

/* Solver choice for sem_pcg. */
typedef enum {
  SEM_SOLVE_FP64 = 0,    /* Jacobi-PCG, FP64 vectors and scalars, apply in opts->apply_prec */
  SEM_SOLVE_IR = 1,      /* FP64 iterative refinement around an FP32 inner Jacobi-PCG */
  SEM_SOLVE_FCG_MLP = 2  /* flexible CG with the learned element preconditioner (sem_mlp_load),
                            Jacobi where the learned correction fails (z.r <= 0 or non-finite) */
} sem_solve_mode;

typedef struct {
  double rtol;          /* stop when the true ||b - A x||_2 <= rtol ||b||_2 (FP64 residual) */
  int32_t max_it;       /* cap on total CG iterations (inner iterations for IR) */
  int32_t mode;         /* sem_solve_mode */
  int32_t apply_prec;   /* SEM_FP64 or SEM_FP64_EMU: the FP64-accurate apply used for the outer
                           residual (IR) or inside CG (SEM_SOLVE_FP64) */
  double inner_rtol;    /* IR only: relative tolerance of each inner FP32 solve (e.g. 1e-4) */
  int32_t check_every;  /* iterations between host convergence checks (>= 1) */
  int32_t use_graph;    /* 1: launch each block of check_every iterations as one CUDA graph */
  int32_t inner_prec;   /* IR only: SEM_BF16 for BF16-stored factors in the inner apply,
                           SEM_FP32_OTF for factors recomputed on the fly, anything else (0 by
                           default) for stored FP32 factors */
  int32_t flags;        /* OR of SEM_PCG_* below (0 by default) */
  int32_t history_cap;  /* sem_pcg: capacity of history in (iteration, residual) pairs; 0: none */
  double *history;      /* sem_pcg: HOST array of 2 * history_cap doubles owned by the caller, or
                           NULL: at every host check the pair (iterations so far, relative
                           residual) is appended while room is left — the recursive residual
                           of CG and flexible CG, the true FP64 residual of each refinement step
                           for IR; sem_batch_pcg ignores it */
} sem_pcg_opts;

/* sem_pcg_opts.flags */
enum {
  SEM_PCG_MULTI_LAUNCH = 1u << 0  /* sem_batch_pcg: run each inner step as one launch per order group
                                     plus four vector kernels instead of the fused step kernel */
};

typedef struct {
  int32_t status;          /* sem_status of the solve */
  int32_t iterations;      /* total CG iterations (inner iterations summed for IR) */
  int32_t outer;           /* IR refinement steps (0 for SEM_SOLVE_FP64) */
  double true_relres;      /* ||b - A x||_2 / ||b||_2 recomputed with the FP64-accurate apply */
  double recursive_relres; /* last recursive residual estimate of the CG recurrence */
  int32_t fallbacks;       /* SEM_SOLVE_FCG_MLP: iterations that fell back to Jacobi */
  int32_t history_len;     /* pairs written to opts->history (0 without one) */
} sem_pcg_result;

/*
 * Solves M A M x = b (b zero on Dirichlet nodes) by Jacobi-preconditioned CG (§4.2.2) from the
 * initial guess in d_x (double[nglobal]); on return d_x holds the solution.  Needs SEM_FEAT_PCG
 * and the factor sets of the chosen mode (FP64 or EMU for the FP64 apply, FP32 for IR).
 * Synchronises `stream` every check_every iterations to test convergence.  The result (and
 * the status it carries) is written to *res; the return value is the same status.
 * Errors: SEM_ERR_NOCONV, SEM_ERR_BREAKDOWN (p^T A p <= 0 or non-finite), SEM_ERR_TIMEOUT
 * (a bounded device wait gave up: an apply left its output incomplete), SEM_ERR_INVALID,
 * SEM_ERR_CUDA.
 */
sem_status sem_pcg(sem_handle *h, const double *d_b, double *d_x, const sem_pcg_opts *opts,
                   sem_pcg_result *res, sem_stream_t stream);

/*
 * *d_out = sum_g x[g] y[g] over the nglobal entries of two global vectors (double), in FP64.
 * The two-stage reduction adds in an order fixed by nglobal alone, so repeated calls give
 * bit-identical results.  This is the inner product of the CG iteration (§4.2.2) exposed for
 * callers that build their own Krylov loop on sem_apply.  Uses the handle's workspace as
 * scratch: calls on one handle (and a running sem_pcg) must not overlap.  d_out is a device
 * pointer to one double, written asynchronously on `stream`.
 */
sem_status sem_dot(sem_handle *h, const double *d_x, const double *d_y, double *d_out, sem_stream_t stream);

/*
 * Allocation-free variant of sem_dot (the paper has no counterpart; this is a library service):
 * *d_out = sum_g x[g] y[g] over n doubles, FP64, for callers that must not allocate device
 * memory where they need the product (a step inside a host framework that owns all device memory
 * through its own pool, or a real-time loop that forbids cudaMalloc after start-up, since
 * cudaMalloc may synchronise the device and can fail under memory pressure).  Needs no handle and
 * no workspace: the reduction scratch (1024 FP64 partials and a ticket, about 8 KB) is a static
 * device array that every GPU loading the library keeps until exit.  The first call on a device,
 * with that device current, looks up the array's device address, clears the ticket and
 * synchronises the device: make it before any stream capture.  All calls share the array and it
 * keeps the last call's partials: calls whose kernels overlap on the GPU race and must be
 * serialised by the caller.  The looked-up address is kept for the life of the process, so the
 * function must not be used on a device after cudaDeviceReset (the address would be stale).
 * Allocates nothing (no cudaMalloc/cudaFree).
 *   n       number of entries, 0 <= n <= 2^30 (larger n: SEM_ERR_INVALID, nothing launched).
 *   d_x, d_y device vectors of n doubles; d_out device pointer to one double, written on stream.
 */
sem_status sem_dot_static(int64_t n, const double *d_x, const double *d_y, double *d_out, sem_stream_t stream);

/*
 * ---- Batched solves: many independent structured-box problems at once ----
 * A batch holds nprob problems (sem_desc entries with glo_num == NULL and bc NONE or BOX), of any
 * mix of sizes and orders.  Their global vectors are concatenated in problem order; problem p
 * starts at the offset sem_batch_info reports.  The solve is the mixed-precision refinement of
 * SEM_SOLVE_IR (§4.2.2 PCG with Jacobi) run for every problem together: per-problem FP64-accurate
 * residuals, then one FP32 Jacobi-PCG iteration of all unfinished problems per step, with
 * per-problem scalars, until each problem reaches rtol.  A step is one persistent cooperative
 * launch (the batched apply of all orders, the x/r update and the direction update separated by
 * bounded grid-wide barriers) when the batch stores FP32 factors and every order is 3, 5, 7, 9
 * or 11; otherwise (factors recomputed on the fly, other orders, or SEM_PCG_MULTI_LAUNCH) one
 * batched apply launch per order group plus four short kernels.  Blocks of steps are replayed
 * as a CUDA graph.
 */
typedef struct sem_batch sem_batch;

/* Workspace bytes for a batch (features must include SEM_FEAT_FP32 or SEM_FEAT_OTF for the FP32
   inner apply, stored factors being used when both are given, and SEM_FEAT_FP64 or SEM_FEAT_EMU
   for the residual; SEM_FEAT_PCG is implied).  Host-only. */
sem_status sem_batch_workspace_size(const sem_desc *descs, int32_t nprob, uint32_t features, size_t *bytes);

/* Sets up every problem (as sem_setup) inside one caller-owned workspace; returns after the
   stream has finished.  Errors as sem_setup, plus SEM_ERR_INVALID for unstructured problems. */
sem_status sem_batch_setup(const sem_desc *descs, int32_t nprob, uint32_t features, void *d_workspace,
                           size_t bytes, sem_stream_t stream, sem_batch **out);

/* Sizes of problem p and the offset of its global nodes in the concatenated vectors. */
sem_status sem_batch_info(const sem_batch *b, int32_t p, sem_info *info, int64_t *g_offset);

/* The single-problem handle of problem p (owned by the batch; valid until sem_batch_free). */
sem_status sem_batch_handle(sem_batch *b, int32_t p, sem_handle **out);

/* Tile variant of the batched FP32 apply for the problems of order N: 1 default elements per
   block, 2 twice as many (factors are read directly in batched launches).  Used by autotuning
   of the per-order-group launches (SEM_PCG_MULTI_LAUNCH); the fused step kernel uses tiles of
   floor(256 / (N+1)^2) elements. */
sem_status sem_batch_set_variant(sem_batch *b, int32_t N, int32_t variant);

/* y = M A M u for every problem of the batch on concatenated vectors: SEM_FP32 (the batch's inner
   apply: stored FP32 factors, or factors recomputed on the fly when the batch has only
   SEM_FEAT_OTF) in one launch per order group, SEM_FP64 / SEM_FP64_EMU one launch per problem. */
sem_status sem_batch_apply(sem_batch *b, sem_prec prec, const void *d_u, void *d_y, sem_stream_t stream);

/* Lumped-mass right-hand sides of every problem from concatenated nodal values (problem order,
   [nelem_p][n_p^3] each) into the concatenated d_b. */
sem_status sem_batch_rhs(sem_batch *b, const double *d_fL, double *d_b, sem_stream_t stream);

/* Solves every problem from the initial guesses in d_x (concatenated, double); res[p] receives
   problem p's result.  opts: rtol, max_it (inner iterations per problem), apply_prec (SEM_FP64 or
   SEM_FP64_EMU, the residual apply), inner_rtol, check_every (steps per graph replay), use_graph;
   mode is ignored.  Returns SEM_OK if every problem converged, else the first failing status. */
sem_status sem_batch_pcg(sem_batch *b, const double *d_b, double *d_x, const sem_pcg_opts *opts,
                         sem_pcg_result *res, sem_stream_t stream);

/* Inner-step form of sem_batch_pcg for this batch: fused != 0 the fused step kernel (the default
   whenever it is available: stored FP32 factors and every order 3, 5, 7, 9 or 11), 0 one launch
   per order group plus four vector kernels.  Either form gives the same iterates to rounding; the
   autotuner times both.  Errors: SEM_ERR_INVALID (NULL batch, or fused asked where unavailable). */
sem_status sem_batch_set_fused(sem_batch *b, int32_t fused);

/* Whether the fused step kernel is available to this batch, and whether sem_batch_pcg uses it
   (either pointer may be NULL).  Errors: SEM_ERR_INVALID for a NULL batch. */
sem_status sem_batch_get_fused(const sem_batch *b, int32_t *available, int32_t *in_use);

/* Polls after which a grid-wide wait of the fused step kernel gives up (polls < 0: the default,
   2^22 polls of about 256 ns; 0: every wait but the last block's gives up at once).  A step whose
   wait gave up leaves its blocks without finishing the step and sem_batch_pcg returns
   SEM_ERR_TIMEOUT (the flag and the barrier are cleared for later solves): this is how the
   timeout path is tested, with no fault and no hang.  Errors: SEM_ERR_INVALID. */
sem_status sem_batch_set_wait_limit(sem_batch *b, int64_t polls);

/* Releases the batch and its problem handles (not the workspace).  NULL is allowed. */
void sem_batch_free(sem_batch *b);

/*
 * ---- Learned element-local preconditioner (flexible CG, SEM_SOLVE_FCG_MLP) ----
 * z = B r + sum_e Q^T W_e (s_e c(r_e)), zero on Dirichlet nodes: a multilayer perceptron c maps the
 * residual on one element, normalised to unit norm, plus six normalised element-mean geometric
 * factors (input n^3 + 6) through two ReLU layers of 256 to a correction on the element's n^3
 * nodes; each correction is scaled by s_e = |r_e| / dbar_e (dbar_e = trace(A_e) / n^3) and the
 * corrections are averaged over the elements sharing each node (W_e = 1 / multiplicity).  The
 * base B is D^-1 (Jacobi base, the network learns the correction to a Jacobi step) or 0 (the
 * network alone: a learned one-level Neumann-Neumann step), chosen by jacobi_base at training
 * (sem_mlp_samples) and at loading (sem_mlp_load).  The paper's PCG (§4.2.2) leaves the
 * preconditioner open; plain Jacobi is the fallback wherever a correction is rejected.
 * Parameters: one FP32 array, W1 [n^3+6][256], b1 [256], W2 [256][256], b2 [256], W3 [256][n^3],
 * b3 [n^3] (row-major; sem_mlp_param_count gives the length).  Training and inference run on the
 * device; inference runs the layers on the tensor cores with BF16 weights and activations, FP32
 * accumulation.
 */
sem_status sem_mlp_param_count(int32_t N, int32_t h1, int32_t h2, int64_t *count);

/* Training pairs from one global residual d_r (double[nglobal], typically a Jacobi-PCG iterate's
   residual): for the elements d_elems[0..nsamp) (int32, device), features
   X [nsamp][n^3+6] = (r_e / |r_e|, geometric factors) and targets
   T [nsamp][n^3] = (x_e - jacobi_base (D^-1 r)_e) dbar_e / |r_e|, where x_e solves the element's
   own shifted Neumann problem
   (A_e + sigma_e M_e) x_e = W_e r_e, sigma_e = eps trace(A_e) / sum_p (w det J)_p (eps > 0,
   e.g. 1e-2), by Jacobi-PCG on the element to relative residual 1e-10 (at most 2000 steps);
   r_e and T are zero on Dirichlet nodes; an index outside [0, nelem) gives a zero row in X and
   T.  d_iters (int32, may be NULL) receives the maximum
   number of local steps taken (atomic max; zero it first).  Orders N = 1..11.  Needs a handle
   set up with SEM_FEAT_MLP. */
sem_status sem_mlp_samples(sem_handle *h, const double *d_r, int32_t nsamp, const int32_t *d_elems, double eps,
                           int32_t jacobi_base, float *d_X, float *d_T, int32_t *d_iters, sem_stream_t stream);

/* Bytes of device scratch sem_mlp_train_step needs for a minibatch. */
sem_status sem_mlp_train_scratch(int32_t N, int32_t h1, int32_t h2, int32_t batch, size_t *bytes);

/* Forward pass on a minibatch: H1 = relu(X W1 + b1), H2 = relu(H1 W2 + b2), O = H2 W3 + b3
   (FP32 parameters, FP32 arithmetic). */
sem_status sem_mlp_forward(int32_t N, int32_t h1, int32_t h2, const float *d_params, const float *d_X, int32_t batch,
                           float *d_H1, float *d_H2, float *d_O, sem_stream_t stream);

/* One training step on a minibatch: forward, mean-squared-error loss (written to *d_loss),
   backward, and (if lr > 0) one Adam update (beta1 0.9, beta2 0.999, eps 1e-8; step >= 1 is the
   update count for bias correction) of d_params with moments d_m, d_v.  The gradient is also
   written to d_grad_out when non-NULL (same layout as the parameters). */
sem_status sem_mlp_train_step(int32_t N, int32_t h1, int32_t h2, float *d_params, float *d_m, float *d_v, int32_t step,
                              float lr, const float *d_X, const float *d_T, int32_t batch, void *d_scratch,
                              size_t scratch_bytes, double *d_loss, float *d_grad_out, sem_stream_t stream);

/* Loads trained FP32 parameters into the handle (rounded to BF16 for inference) and selects the
   base of the preconditioner (jacobi_base != 0: D^-1 r plus the corrections; the default of a
   new handle). */
sem_status sem_mlp_load(sem_handle *h, const float *d_params, int32_t jacobi_base, sem_stream_t stream);

/* z = B r + sum_e Q^T W_e (s_e c(r_e)): the learned preconditioner applied to a global residual
   (double[nglobal]). */
sem_status sem_mlp_precond(sem_handle *h, const double *d_r, double *d_z, sem_stream_t stream);

/* Inference layout: on != 0 (the default of a new handle) runs the three layers as one launch
   (hidden activations kept in shared memory) wherever the hidden widths are 256 and n^3 <= 512
   is a multiple of 8, otherwise three launches of sem_gemm_bf16's kernel; both round the hidden
   activations to BF16 and sum in the same order, so z is the same.  Errors: SEM_ERR_INVALID. */
sem_status sem_mlp_set_fused(sem_handle *h, int32_t on);

/* One dense layer of the preconditioner's inference on the tensor cores (the paper has no
   counterpart): C = act(A Bt^T + bias), C[m][n] = sum_k A[m][k] Bt[n][k] + bias[n], act = ReLU if
   relu != 0 else identity.  d_A: BF16 [M][lda], d_Bt: BF16 [N][ldb] (the weight matrix
   transposed, so both operands have K contiguous), d_bias: float[N] or NULL, d_C: float [M][ldc],
   all device memory owned by the caller.  Products are exact in FP32, sums in FP32 (order of the
   tensor core).  Requires lda, ldb >= K, ldc >= N, all three multiples of 8, 16-byte aligned
   pointers, M <= 65535 * 128; otherwise SEM_ERR_INVALID and nothing is launched.  d_err (int32,
   may be NULL) is OR-ed with 1 if a block gave up waiting for its tensor-core operations (its tile
   of C is then left unwritten). */
sem_status sem_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *d_A, int32_t lda, const void *d_Bt, int32_t ldb,
                         const float *d_bias, float *d_C, int32_t ldc, int32_t relu, int32_t *d_err,
                         sem_stream_t stream);

/* The preconditioner's three layers in one launch (the paper has no counterpart):
   O = (relu(relu(X W1t^T + b1) W2t^T + b2)) W3t^T + b3 with the two hidden activations (width
   256) rounded to BF16 and kept on chip.  d_X: BF16 [M][ldx] (nin values per row), d_W1t: BF16
   [256][ldx], d_W2t: BF16 [256][256], d_W3t: BF16 [nout][256], d_b1, d_b2: float[256], d_b3:
   float[nout], d_O: float [M][nout]; all device memory owned by the caller.  The same roundings
   and sums as three sem_gemm_bf16 calls (BF16 hidden outputs between them).  Requires ldx >= nin
   and a multiple of 8, 8 <= nout <= 512 and a multiple of 8, 16-byte aligned pointers; otherwise
   SEM_ERR_INVALID and nothing is launched.  d_err (int32, may be NULL) is OR-ed with 1 if a block
   gave up waiting for its copies or tensor-core operations (its rows of O are then unwritten). */
sem_status sem_mlp_layers_bf16(int32_t M, int32_t nin, int32_t ldx, int32_t nout, const void *d_X, const void *d_W1t,
                               const void *d_W2t, const void *d_W3t, const float *d_b1, const float *d_b2,
                               const float *d_b3, float *d_O, int32_t *d_err, sem_stream_t stream);

/* r = M (b - A x) with an FP64-accurate apply (SEM_FP64 or SEM_FP64_EMU); needs SEM_FEAT_PCG
   (its scratch vector holds A x).  All three vectors are double[nglobal]. */
sem_status sem_residual(sem_handle *h, sem_prec prec, const double *d_b, const double *d_x, double *d_r,
                        sem_stream_t stream);

/* Message describing the last error on this thread ("" if none). */
const char *sem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
