// Set-up of a spectral-element problem inside the caller's device workspace: GLL nodes and the
// derivative matrix (host, FP64), per-node geometric factors and lumped mass (device),
// numbering, Dirichlet mask and the assembled Jacobi diagonal.  Also the small helper entry
// points (coordinates, numbering copy-out, right-hand side, diagonal, info, errors).
//
// Discretisation (arXiv 1403.0968 §4.2.1): tensor-product Lagrange basis on the N+1
// Gauss-Lobatto-Legendre nodes; lumped mass J w_abc; stiffness through the per-node matrix
// J G^T G (six unique entries) evaluated at every elemental node; kappa scales the flux.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "sem_internal.h"

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

sem_status sem_fail(sem_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

extern "C" const char *sem_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------------------------------
// 1-D GLL rule and derivative matrix (host, double)
// ------------------------------------------------------------------------------------------
// Legendre P_N and P'_N at x by the three-term recurrence; P'_N from the derivative recurrence
// P'_{k+1} = P'_{k-1} + (2k+1) P_k.
static void legendre_with_derivative(int N, double x, double *P, double *dP) {
  double pm1 = 1.0, p = x, dpm1 = 0.0, dp = 1.0;
  if (N == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 1; k < N; ++k) {
    double pn = ((2 * k + 1) * x * p - k * pm1) / (k + 1);
    double dpn = dpm1 + (2 * k + 1) * p;
    pm1 = p;
    p = pn;
    dpm1 = dp;
    dp = dpn;
  }
  *P = p;
  *dP = dp;
}

// Interior GLL nodes are the zeros of P'_N.  Newton on P'_N with P''_N from Legendre's equation
// (1 - x^2) P''_N = 2 x P'_N - N (N+1) P_N, started at the Chebyshev-Gauss-Lobatto points;
// the rule is symmetric, so only the left half is iterated and mirrored.
static void gll_rule(int N, double *x, double *w) {
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i <= N / 2; ++i) {
    double xi = -cos(M_PI * i / N);
    for (int it = 0; it < 60; ++it) {
      double P, dP;
      legendre_with_derivative(N, xi, &P, &dP);
      double d2P = (2.0 * xi * dP - N * (N + 1.0) * P) / (1.0 - xi * xi);
      double dx = dP / d2P;
      xi -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    x[i] = xi;
    x[N - i] = -xi;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int i = 0; i <= N; ++i) {
    double P, dP;
    legendre_with_derivative(N, x[i], &P, &dP);
    w[i] = 2.0 / (N * (N + 1.0) * P * P);
  }
}

// D[i][j] = l_j'(x_i) in the Legendre form: P_N(x_i) / (P_N(x_j) (x_i - x_j)) off the diagonal,
// -N(N+1)/4 and +N(N+1)/4 at the two corners, 0 on the rest of the diagonal.
static void gll_derivative(int N, const double *x, double *D) {
  int n = N + 1;
  std::vector<double> P(n);
  for (int i = 0; i < n; ++i) {
    double dP;
    legendre_with_derivative(N, x[i], &P[i], &dP);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      D[i * n + j] = (i == j) ? 0.0 : P[i] / (P[j] * (x[i] - x[j]));
  D[0] = -N * (N + 1.0) / 4.0;
  D[N * n + N] = N * (N + 1.0) / 4.0;
}

void sem_gll_tables(int N, double *x, double *w, double *D) {
  gll_rule(N, x, w);
  gll_derivative(N, x, D);
}

// ------------------------------------------------------------------------------------------
// workspace layout
// ------------------------------------------------------------------------------------------
namespace {
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

struct Plan {
  size_t D64, D32, Dhi, Dlo, gx, gw, verts, modes, G64, G32, Gemu, wJ, wJa64, wJa32, wJaemu, glo, mask,
      dinv64, dinv32, r64, p64, Ap64, t64, r32, p32, Ap32, x32, partials, scal, kap_tmp, alpha_tmp, total,
      Gotf, kap32;
  size_t G16, geo6, inv_mult, mlp_w, mlp_b32, mlp_X, mlp_scale, mlp_H1, mlp_H2, mlp_O, mlp_dbar, z64, gpartials,
      gtickets;
  bool need64, needEmu, need32, needPcg, needMlp, need16, needOtf;
};

const size_t NONE = ~(size_t)0;

sem_status validate(const sem_desc *d, uint32_t feat, int64_t *G_out) {
  if (!d) return sem_fail(SEM_ERR_INVALID, "desc is NULL");
  if (d->N < 1 || d->N > SEM_MAX_N) return sem_fail(SEM_ERR_INVALID, "order N must be in 1..15");
  if (d->nelem <= 0) return sem_fail(SEM_ERR_INVALID, "nelem must be positive");
  if (!d->vertices) return sem_fail(SEM_ERR_INVALID, "vertices is NULL");
  if ((feat & (SEM_FEAT_FP64 | SEM_FEAT_EMU | SEM_FEAT_FP32 | SEM_FEAT_OTF)) == 0)
    return sem_fail(SEM_ERR_INVALID, "features must request at least one factor set");
  if ((feat & SEM_FEAT_MLP) && (feat & (SEM_FEAT_FP64 | SEM_FEAT_EMU | SEM_FEAT_FP32)) == 0)
    return sem_fail(SEM_ERR_INVALID, "SEM_FEAT_MLP needs stored FP64, EMU or FP32 factors");
  if (d->kappa_nmodes < 0 || (d->kappa_nmodes > 0 && !d->kappa_modes))
    return sem_fail(SEM_ERR_INVALID, "kappa_modes missing");
  if (d->kappa_nmodes > 64) return sem_fail(SEM_ERR_INVALID, "at most 64 kappa modes");
  if (d->bc < SEM_BC_NONE || d->bc > SEM_BC_MASK) return sem_fail(SEM_ERR_INVALID, "bad bc");
  if (d->glo_num == nullptr || d->bc == SEM_BC_BOX) {
    if (d->box[0] < 1 || d->box[1] < 1 || d->box[2] < 1)
      return sem_fail(SEM_ERR_INVALID, "box element counts must be positive");
    if ((int64_t)d->box[0] * d->box[1] * d->box[2] != d->nelem)
      return sem_fail(SEM_ERR_INVALID, "nelem != box[0]*box[1]*box[2]");
  }
  int64_t G;
  if (d->glo_num == nullptr) {
    G = ((int64_t)d->box[0] * d->N + 1) * ((int64_t)d->box[1] * d->N + 1) * ((int64_t)d->box[2] * d->N + 1);
  } else {
    G = d->nglobal;
    if (G <= 0 || G >= ((int64_t)1 << 31))
      return sem_fail(SEM_ERR_INVALID, "explicit numbering needs 0 < nglobal < 2^31");
  }
  if (d->bc == SEM_BC_MASK && !d->dirichlet) return sem_fail(SEM_ERR_INVALID, "dirichlet flags missing");
  *G_out = G;
  return SEM_OK;
}

Plan make_plan(const sem_desc *d, uint32_t feat, int64_t G) {
  Plan p;
  Layout L;
  int n = d->N + 1;
  size_t n3 = (size_t)n * n * n, E = (size_t)d->nelem, Ln = E * n3;
  p.needPcg = feat & SEM_FEAT_PCG;
  p.need64 = feat & SEM_FEAT_FP64;
  p.needEmu = feat & SEM_FEAT_EMU;
  p.need32 = feat & SEM_FEAT_FP32;
  p.need16 = feat & SEM_FEAT_BF16;
  p.needOtf = feat & SEM_FEAT_OTF;
  bool alpha = d->alpha != nullptr;
  p.D64 = L.take(n * n * 8);
  p.D32 = L.take(n * n * 4);
  p.Dhi = L.take(n * n * 4);
  p.Dlo = L.take(n * n * 4);
  p.gx = L.take(n * 8);
  p.gw = L.take(n * 8);
  p.verts = L.take(E * 24 * 8);
  p.modes = L.take(64 * 5 * 8);
  const size_t gs6 = (6 * n3 + 3) / 4 * 4, gs12 = (12 * n3 + 3) / 4 * 4;
  p.G64 = p.need64 ? L.take(E * gs6 * 8) : NONE;
  p.G32 = p.need32 ? L.take(E * gs6 * 4) : NONE;
  p.Gemu = p.needEmu ? L.take(E * gs12 * 4) : NONE;
  const size_t gs16 = (6 * n3 + 7) / 8 * 8;
  p.G16 = p.need16 ? L.take(E * gs16 * 2) : NONE;
  p.Gotf = p.needOtf ? L.take(E * SEM_OTF_STRIDE * 4) : NONE;
  p.kap32 = (p.needOtf && (d->kappa || d->kappa_nmodes > 0)) ? L.take(Ln * 4) : NONE;
  p.wJ = L.take(Ln * 8);
  p.wJa64 = (alpha && p.need64) ? L.take(Ln * 8) : NONE;
  p.wJa32 = (alpha && (p.need32 || p.need16 || p.needOtf)) ? L.take(Ln * 4) : NONE;
  p.wJaemu = (alpha && p.needEmu) ? L.take(Ln * 8) : NONE;
  p.glo = d->glo_num ? L.take(Ln * 4) : NONE;
  p.mask = d->bc == SEM_BC_MASK ? L.take((size_t)G) : NONE;
  p.dinv64 = L.take((size_t)G * 8);
  p.dinv32 = L.take((size_t)G * 4);
  p.r64 = p.needPcg ? L.take((size_t)G * 8) : NONE;
  p.p64 = p.needPcg ? L.take((size_t)G * 8) : NONE;
  p.Ap64 = p.needPcg ? L.take((size_t)G * 8) : NONE;
  p.t64 = p.needPcg ? L.take((size_t)G * 8) : NONE;
  bool ir = p.needPcg && (p.need32 || p.need16 || p.needOtf);
  p.r32 = ir ? L.take((size_t)G * 4) : NONE;
  p.p32 = ir ? L.take((size_t)G * 4) : NONE;
  p.Ap32 = ir ? L.take((size_t)G * 4) : NONE;
  p.x32 = ir ? L.take((size_t)G * 4) : NONE;
  p.partials = L.take((size_t)SEM_MAX_PARTIALS * 8);
  p.gpartials = L.take((size_t)SEM_MAX_GROUPS * 8);
  p.gtickets = L.take((size_t)SEM_MAX_GROUPS * 4);
  p.scal = L.take(sizeof(SemScalars));
  p.kap_tmp = d->kappa ? L.take(Ln * 8) : NONE;
  p.alpha_tmp = alpha ? L.take(Ln * 8) : NONE;
  p.needMlp = feat & SEM_FEAT_MLP;
  const size_t nin = n3 + 6, np = nin * SEM_MLP_H1 + SEM_MLP_H1 + (size_t)SEM_MLP_H1 * SEM_MLP_H2 + SEM_MLP_H2 +
                                  (size_t)SEM_MLP_H2 * n3 + n3;
  p.geo6 = p.needMlp ? L.take(E * 6 * 4) : NONE;
  p.inv_mult = p.needMlp ? L.take((size_t)G * 4) : NONE;
  const size_t ldx = (nin + 7) / 8 * 8;  // BF16 rows of 16-byte multiples for the tensor cores
  p.mlp_w = p.needMlp ? L.take((ldx * SEM_MLP_H1 + (size_t)SEM_MLP_H1 * SEM_MLP_H2 + (size_t)SEM_MLP_H2 * n3) * 2)
                      : NONE;
  p.mlp_b32 = p.needMlp ? L.take(np * 4) : NONE;
  p.mlp_X = p.needMlp ? L.take(E * ldx * 2) : NONE;
  p.mlp_scale = p.needMlp ? L.take(E * 4) : NONE;
  p.mlp_H1 = p.needMlp ? L.take(E * SEM_MLP_H1 * 2) : NONE;
  p.mlp_H2 = p.needMlp ? L.take(E * SEM_MLP_H2 * 2) : NONE;
  p.mlp_O = p.needMlp ? L.take(E * n3 * 4) : NONE;
  p.mlp_dbar = p.needMlp ? L.take(E * 4) : NONE;
  p.z64 = (p.needMlp && p.needPcg) ? L.take((size_t)G * 8) : NONE;
  p.total = L.off;
  return p;
}

template <typename T>
T *at(void *base, size_t off) {
  return off == NONE ? nullptr : reinterpret_cast<T *>(static_cast<char *>(base) + off);
}
}  // namespace

extern "C" sem_status sem_workspace_size(const sem_desc *desc, uint32_t features, size_t *bytes) {
  int64_t G;
  sem_status st = validate(desc, features, &G);
  if (st != SEM_OK) return st;
  if (!bytes) return sem_fail(SEM_ERR_INVALID, "bytes is NULL");
  *bytes = make_plan(desc, features, G).total;
  return SEM_OK;
}

// ------------------------------------------------------------------------------------------
// device geometry
// ------------------------------------------------------------------------------------------
struct SetupArgs {
  int N, n, n3;
  int64_t E, gs6, gs12, gs16;
  const double *verts, *gx, *gw, *modes, *kap, *alpha;
  int nmodes;
  double *G64, *wJ, *wJa64;
  float *G32, *Gemu, *wJa32, *wJaemu;
  __nv_bfloat16 *G16;
  float *kap32;     // FP32 kappa per local node (SEM_FEAT_OTF with kappa not 1), or NULL
  double *wJa_tmp;  // FP64 w det J alpha for the diagonal (overwrites the alpha copy in place)
  int *tangled;
  int *emu_range;   // [0] largest biased FP64 exponent of any factor or w det J alpha, [1] smallest
                    // of the diagonal factors (rr, ss, tt): the double-float range check
};

__device__ static int biased_exp(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FFull);
}

// x(r,s,t) = sum_v X_v (1 + r_v r)(1 + s_v s)(1 + t_v t)/8 with analytic derivatives;
// jac[d][c] = d x_d / d r_c.
__device__ static void map_point(const double *X, double r, double s, double t, double xyz[3], double jac[3][3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    xyz[d] = 0.0;
    jac[d][0] = jac[d][1] = jac[d][2] = 0.0;
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double sr = (v & 1) ? 1.0 : -1.0, ss = (v & 2) ? 1.0 : -1.0, st = (v & 4) ? 1.0 : -1.0;
    const double a = 1.0 + sr * r, b = 1.0 + ss * s, c = 1.0 + st * t;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double X8 = 0.125 * X[3 * v + d];
      xyz[d] += X8 * a * b * c;
      jac[d][0] += X8 * sr * b * c;
      jac[d][1] += X8 * a * ss * c;
      jac[d][2] += X8 * a * b * st;
    }
  }
}

__device__ static double kappa_at(const double *modes, int nmodes, const double xyz[3]) {
  double g = 0.0;
  for (int m = 0; m < nmodes; ++m) {
    const double *q = modes + 5 * m;
    g += q[4] * cos(2.0 * M_PI * (q[0] * xyz[0] + q[1] * xyz[1] + q[2] * xyz[2]) + q[3]);
  }
  return exp(g);
}

// The six factors G_kl = w det J kappa (grad r_k . grad r_l) of node (i, j, k) of element e, with
// det J and kappa; returns false if det J <= 0 (a tangled element).
__device__ static bool node_factors(const SetupArgs &a, int64_t e, int i, int j, int k, double g[6], double *wdet_out,
                                    double *kap_out) {
  double xyz[3], J[3][3];
  map_point(a.verts + 24 * e, a.gx[i], a.gx[j], a.gx[k], xyz, J);
  // cofactors: inverse Jacobian rows are d r_c / d x_d = cof^T / det
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  double R[3][3];  // R[c][d] = d r_c / d x_d
  R[0][0] = c00 / det;
  R[1][0] = c01 / det;
  R[2][0] = c02 / det;
  R[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  R[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  R[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  R[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  R[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  R[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  const int64_t q = e * a.n3 + i + a.n * (j + a.n * k);
  const double kap = a.kap ? a.kap[q] : kappa_at(a.modes, a.nmodes, xyz);
  const double wdet = a.gw[i] * a.gw[j] * a.gw[k] * det;
  int f = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int c2 = c; c2 < 3; ++c2) {
      g[f++] = wdet * kap * (R[c][0] * R[c2][0] + R[c][1] * R[c2][1] + R[c][2] * R[c2][2]);
    }
  *wdet_out = wdet;
  *kap_out = kap;
  return det > 0.0;
}

__global__ void k_setup_factors(SetupArgs a) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.E * a.n3) return;
  const int64_t e = q / a.n3;
  const int p = (int)(q - e * a.n3);
  const int i = p % a.n, j = (p / a.n) % a.n, k = p / (a.n * a.n);
  double g[6], wdet, kap;
  if (!node_factors(a, e, i, j, k, g, &wdet, &kap)) atomicOr(a.tangled, 1);
  if (a.kap32) a.kap32[q] = (float)kap;
  if (a.Gemu) {
    int mx = 0;
#pragma unroll
    for (int ff = 0; ff < 6; ++ff) mx = max(mx, biased_exp(g[ff]));
    if (a.alpha) mx = max(mx, biased_exp(wdet * a.alpha[q]));
    atomicMax(&a.emu_range[0], mx);
    atomicMin(&a.emu_range[1], min(biased_exp(g[0]), min(biased_exp(g[3]), biased_exp(g[5]))));
  }
  const int64_t base = e * a.gs6 + p;
#pragma unroll
  for (int ff = 0; ff < 6; ++ff) {
    if (a.G64) a.G64[base + (int64_t)ff * a.n3] = g[ff];
    if (a.G32) a.G32[base + (int64_t)ff * a.n3] = (float)g[ff];
    if (a.G16) a.G16[e * a.gs16 + (int64_t)ff * a.n3 + p] = __double2bfloat16(g[ff]);
    if (a.Gemu) {
      const float hi = (float)g[ff];
      const float lo = (float)(g[ff] - (double)hi);
      a.Gemu[e * a.gs12 + (int64_t)(2 * ff) * a.n3 + p] = hi;
      a.Gemu[e * a.gs12 + (int64_t)(2 * ff + 1) * a.n3 + p] = lo;
    }
  }
  a.wJ[q] = wdet;
  if (a.alpha) {
    const double wa = wdet * a.alpha[q];
    a.wJa_tmp[q] = wa;
    if (a.wJa64) a.wJa64[q] = wa;
    if (a.wJa32) a.wJa32[q] = (float)wa;
    if (a.wJaemu) {
      const float hi = (float)wa;
      a.wJaemu[e * 2 * a.n3 + p] = hi;
      a.wJaemu[e * 2 * a.n3 + a.n3 + p] = (float)(wa - (double)hi);
    }
  }
}

// Coefficient vectors of the trilinear map of each element (the OtfGeo layout): for a subset m of
// the directions {r, s, t}, W_m = sum_v X_v prod_{d in m} sigma_d(v) / 8, formed in FP64 and
// rounded once to FP32.
__global__ void k_setup_otf(const double *verts, int64_t E, float *out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int masks[7] = {1, 2, 4, 3, 5, 6, 7};  // r, s, t, rs, rt, st, rst (bit 0 = r)
  const double *X = verts + 24 * e;
  float *o = out + e * SEM_OTF_STRIDE;
  for (int c = 0; c < 7; ++c)
    for (int d = 0; d < 3; ++d) {
      double acc = 0.0;
      for (int v = 0; v < 8; ++v) {
        double sg = 1.0;
        for (int b = 0; b < 3; ++b)
          if ((masks[c] >> b) & 1) sg *= ((v >> b) & 1) ? 1.0 : -1.0;
        acc += sg * X[3 * v + d];
      }
      o[3 * c + d] = (float)(0.125 * acc);
    }
  o[21] = o[22] = o[23] = 0.0f;
}

// global id of local node p of element e
__device__ __forceinline__ static int64_t node_id(const sem_handle &h, const int *glo, int64_t e, int p,
                                                   int64_t gxs, int64_t gys) {
  if (glo) return glo[e * h.n3 + p];
  const int n = h.n, N = h.N;
  const int i = p % n, j = (p / n) % n, k = p / (n * n);
  const int64_t ex = e % h.box[0], ey = (e / h.box[0]) % h.box[1], ez = e / ((int64_t)h.box[0] * h.box[1]);
  return (ex * N + i) + gxs * ((ey * N + j) + gys * (ez * N + k));
}

__device__ __forceinline__ static bool is_dirichlet(const sem_handle &h, const uint8_t *mask, int64_t g,
                                                    int64_t gxs, int64_t gys, int64_t gzs) {
  if (h.bc == SEM_BC_MASK) return mask[g] != 0;
  if (h.bc == SEM_BC_BOX) {
    const int64_t I = g % gxs, J = (g / gxs) % gys, K = g / (gxs * gys);
    return I == 0 || J == 0 || K == 0 || I == gxs - 1 || J == gys - 1 || K == gzs - 1;
  }
  return false;
}

// Diagonal of the element operator at node p = (a,b,c), from the sparsity of the reference
// derivatives (§4.2.1): d phi_abc / dr at node (m,b,c) is D[m][a] and vanishes off that line.
// G(f, m) returns factor f at node m of the element.
template <typename GF>
__device__ static double diag_entry(const sem_handle &h, int p, GF G) {
  const int n = h.n;
  const int a = p % n, b = (p / n) % n, c = p / (n * n);
  const double *D = h.D64;
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    const double dra = D[m * n + a], dsb = D[m * n + b], dtc = D[m * n + c];
    s += G(0, m + n * (b + n * c)) * dra * dra;
    s += G(3, a + n * (m + n * c)) * dsb * dsb;
    s += G(5, a + n * (b + n * m)) * dtc * dtc;
  }
  const double Da = D[a * n + a], Db = D[b * n + b], Dc = D[c * n + c];
  s += 2.0 * (Da * Db * G(1, p) + Da * Dc * G(2, p) + Db * Dc * G(4, p));
  return s;
}

// assembled diagonal from a stored factor set; Glo (if any) holds the low halves of double-float pairs
template <typename TG>
__global__ void k_setup_diag(sem_handle h, const TG *Gf, const TG *Glo, int64_t estride, int fstride,
                             const double *wJa, double *diag) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h.L) return;
  const int64_t e = q / h.n3;
  const int p = (int)(q - e * h.n3);
  const int n3 = h.n3;
  double s = diag_entry(h, p, [&](int f, int m) -> double {
    const int64_t idx = e * estride + (int64_t)f * fstride * n3 + m;
    double v = (double)Gf[idx];
    if (Glo) v += (double)Glo[idx];
    return v;
  });
  if (wJa) s += wJa[q];
  const int64_t gxs = (int64_t)h.box[0] * h.N + 1, gys = (int64_t)h.box[1] * h.N + 1;
  atomicAdd(diag + node_id(h, h.glo, e, p, gxs, gys), s);
}

// assembled diagonal with the factors evaluated in FP64 from the map (no stored factor set)
__global__ void k_setup_diag_geo(sem_handle h, SetupArgs a, const double *wJa, double *diag) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h.L) return;
  const int64_t e = q / h.n3;
  const int p = (int)(q - e * h.n3);
  const int n = h.n;
  double s = diag_entry(h, p, [&](int f, int m) -> double {
    double g[6], wdet, kap;
    node_factors(a, e, m % n, (m / n) % n, m / (n * n), g, &wdet, &kap);
    return g[f];
  });
  if (wJa) s += wJa[q];
  const int64_t gxs = (int64_t)h.box[0] * h.N + 1, gys = (int64_t)h.box[1] * h.N + 1;
  atomicAdd(diag + node_id(h, h.glo, e, p, gxs, gys), s);
}

__global__ void k_setup_dinv(sem_handle h, const double *diag, double *dinv64, float *dinv32) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= h.G) return;
  const int64_t gxs = (int64_t)h.box[0] * h.N + 1, gys = (int64_t)h.box[1] * h.N + 1,
                gzs = (int64_t)h.box[2] * h.N + 1;
  const bool dir = is_dirichlet(h, h.mask, g, gxs, gys, gzs);
  const double v = dir ? 0.0 : 1.0 / diag[g];
  dinv64[g] = v;
  dinv32[g] = (float)v;
}

__global__ void k_node_coords(sem_handle h, double *xyz) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h.L) return;
  const int64_t e = q / h.n3;
  const int p = (int)(q - e * h.n3);
  const int n = h.n, i = p % n, j = (p / n) % n, k = p / (n * n);
  double x[3], J[3][3];
  map_point(h.verts + 24 * e, h.gll_x[i], h.gll_x[j], h.gll_x[k], x, J);
  xyz[3 * q + 0] = x[0];
  xyz[3 * q + 1] = x[1];
  xyz[3 * q + 2] = x[2];
}

__global__ void k_glo_num(sem_handle h, int64_t *out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h.L) return;
  const int64_t e = q / h.n3;
  const int p = (int)(q - e * h.n3);
  const int64_t gxs = (int64_t)h.box[0] * h.N + 1, gys = (int64_t)h.box[1] * h.N + 1;
  out[q] = node_id(h, h.glo, e, p, gxs, gys);
}

__global__ void k_rhs_scatter(sem_handle h, const double *fL, double *b) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h.L) return;
  const int64_t e = q / h.n3;
  const int p = (int)(q - e * h.n3);
  const int64_t gxs = (int64_t)h.box[0] * h.N + 1, gys = (int64_t)h.box[1] * h.N + 1,
                gzs = (int64_t)h.box[2] * h.N + 1;
  const int64_t g = node_id(h, h.glo, e, p, gxs, gys);
  if (!is_dirichlet(h, h.mask, g, gxs, gys, gzs)) atomicAdd(b + g, h.wJ[q] * fL[q]);
}

__global__ void k_diag_out(sem_handle h, double *out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= h.G) return;
  const double v = h.dinv64[g];
  out[g] = v == 0.0 ? 1.0 : 1.0 / v;
}

static inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// ------------------------------------------------------------------------------------------
// entry points
// ------------------------------------------------------------------------------------------
extern "C" sem_status sem_setup(const sem_desc *d, uint32_t features, void *ws, size_t bytes, sem_stream_t stream_,
                                sem_handle **out) {
  NvtxRange nvtx_setup("sem_setup");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  int64_t G;
  sem_status st = validate(d, features, &G);
  if (st != SEM_OK) return st;
  if (!out) return sem_fail(SEM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  Plan P = make_plan(d, features, G);
  if (!ws || bytes < P.total)
    return sem_fail(SEM_ERR_WORKSPACE, "workspace needs " + std::to_string(P.total) + " bytes");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return sem_fail(SEM_ERR_WORKSPACE, "workspace must be 256-byte aligned");

  sem_handle *h = new sem_handle();
  memset(h, 0, sizeof(*h));
  h->N = d->N;
  h->n = d->N + 1;
  h->n3 = h->n * h->n * h->n;
  h->E = d->nelem;
  h->G = G;
  h->L = h->E * h->n3;
  h->gs6 = (6 * (int64_t)h->n3 + 3) / 4 * 4;
  h->gs12 = (12 * (int64_t)h->n3 + 3) / 4 * 4;
  h->gs16 = (6 * (int64_t)h->n3 + 7) / 8 * 8;
  h->box[0] = d->box[0];
  h->box[1] = d->box[1];
  h->box[2] = d->box[2];
  h->structured = d->glo_num == nullptr;
  h->bc = d->bc;
  h->has_alpha = d->alpha != nullptr;
  h->features = features;
  h->apply_variant = -1;  // automatic tile choice
  h->wait_polls = SEM_WAIT_POLLS_DEFAULT;
  cudaGetDevice(&h->device);
  h->D64 = at<double>(ws, P.D64);
  h->D32 = at<float>(ws, P.D32);
  h->Dhi = at<float>(ws, P.Dhi);
  h->Dlo = at<float>(ws, P.Dlo);
  h->gll_x = at<double>(ws, P.gx);
  h->gll_w = at<double>(ws, P.gw);
  h->verts = at<double>(ws, P.verts);
  h->G64 = at<double>(ws, P.G64);
  h->G32 = at<float>(ws, P.G32);
  h->G16 = at<__nv_bfloat16>(ws, P.G16);
  h->Gemu = at<float>(ws, P.Gemu);
  h->Gotf = at<float>(ws, P.Gotf);
  h->kap32 = at<float>(ws, P.kap32);
  h->wJ = at<double>(ws, P.wJ);
  h->wJa64 = at<double>(ws, P.wJa64);
  h->wJa32 = at<float>(ws, P.wJa32);
  h->wJaemu = at<float>(ws, P.wJaemu);
  h->glo = at<int32_t>(ws, P.glo);
  h->mask = at<uint8_t>(ws, P.mask);
  h->dinv64 = at<double>(ws, P.dinv64);
  h->dinv32 = at<float>(ws, P.dinv32);
  h->r64 = at<double>(ws, P.r64);
  h->p64 = at<double>(ws, P.p64);
  h->Ap64 = at<double>(ws, P.Ap64);
  h->t64 = at<double>(ws, P.t64);
  h->r32 = at<float>(ws, P.r32);
  h->p32 = at<float>(ws, P.p32);
  h->Ap32 = at<float>(ws, P.Ap32);
  h->x32 = at<float>(ws, P.x32);
  h->partials = at<double>(ws, P.partials);
  h->gpartials = at<double>(ws, P.gpartials);
  h->gtickets = at<unsigned int>(ws, P.gtickets);
  h->scal = at<SemScalars>(ws, P.scal);
  h->geo6 = at<float>(ws, P.geo6);
  h->inv_mult = at<float>(ws, P.inv_mult);
  h->mlp_w = at<__nv_bfloat16>(ws, P.mlp_w);
  h->mlp_b32 = at<float>(ws, P.mlp_b32);
  h->mlp_X = at<__nv_bfloat16>(ws, P.mlp_X);
  h->mlp_scale = at<float>(ws, P.mlp_scale);
  h->mlp_H1 = at<__nv_bfloat16>(ws, P.mlp_H1);
  h->mlp_H2 = at<__nv_bfloat16>(ws, P.mlp_H2);
  h->mlp_O = at<float>(ws, P.mlp_O);
  h->mlp_dbar = at<float>(ws, P.mlp_dbar);
  h->mlp_h1 = SEM_MLP_H1;
  h->mlp_h2 = SEM_MLP_H2;
  h->mlp_ldx = (h->n3 + 6 + 7) / 8 * 8;
  h->mlp_jacobi_base = 1;
  h->mlp_fused = 1;
  h->z64 = at<double>(ws, P.z64);

  auto fail = [&](sem_status s) {
    delete h;
    return s;
  };

  // 1-D rule and derivative matrix (host) and their single/double-float copies
  const int n = h->n;
  std::vector<double> x(n), w(n), D(n * n);
  gll_rule(h->N, x.data(), w.data());
  gll_derivative(h->N, x.data(), D.data());
  std::vector<float> D32(n * n), Dhi(n * n), Dlo(n * n);
  for (int q = 0; q < n * n; ++q) {
    D32[q] = (float)D[q];
    Dhi[q] = (float)D[q];
    Dlo[q] = (float)(D[q] - (double)Dhi[q]);
    h->D64h[q] = D[q];
    if (q < n) {
      h->gxh[q] = x[q];
      h->gwh[q] = w[q];
    }
    h->D32h[q] = D32[q];
    h->Dhih[q] = Dhi[q];
    h->Dloh[q] = Dlo[q];
  }
#define COPY(dst, src, nbytes)                                                                 \
  do {                                                                                         \
    cudaError_t _e = cudaMemcpyAsync((dst), (src), (nbytes), cudaMemcpyHostToDevice, stream);  \
    if (_e != cudaSuccess) return fail(sem_fail(SEM_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(_e))); \
  } while (0)
  COPY(h->D64, D.data(), n * n * 8);
  COPY(h->D32, D32.data(), n * n * 4);
  COPY(h->Dhi, Dhi.data(), n * n * 4);
  COPY(h->Dlo, Dlo.data(), n * n * 4);
  COPY(h->gll_x, x.data(), n * 8);
  COPY(h->gll_w, w.data(), n * 8);
  COPY(h->verts, d->vertices, (size_t)h->E * 24 * 8);
  double *modes = at<double>(ws, P.modes);
  if (d->kappa_nmodes > 0) COPY(modes, d->kappa_modes, (size_t)d->kappa_nmodes * 5 * 8);
  double *kap = at<double>(ws, P.kap_tmp);
  if (d->kappa) COPY(kap, d->kappa, (size_t)h->L * 8);
  double *alpha = at<double>(ws, P.alpha_tmp);
  if (d->alpha) COPY(alpha, d->alpha, (size_t)h->L * 8);
  std::vector<int32_t> glo32;
  if (d->glo_num) {
    glo32.resize(h->L);
    for (int64_t q = 0; q < h->L; ++q) {
      const int64_t g = d->glo_num[q];
      if (g < 0 || g >= G) return fail(sem_fail(SEM_ERR_INVALID, "glo_num entry out of range"));
      glo32[q] = (int32_t)g;
    }
    COPY(h->glo, glo32.data(), (size_t)h->L * 4);
  }
  if (d->bc == SEM_BC_MASK) COPY(h->mask, d->dirichlet, (size_t)G);
#undef COPY

  int *tangled = reinterpret_cast<int *>(h->partials);
  int *emu_range = tangled + 2;  // [max exponent, min diagonal exponent], see SetupArgs
  if (cudaMemsetAsync(tangled, 0, 3 * sizeof(int), stream) != cudaSuccess ||
      cudaMemsetAsync(emu_range + 1, 0x7F, sizeof(int), stream) != cudaSuccess)
    return fail(sem_fail(SEM_ERR_CUDA, "memset"));
  // solver scalars and group counters hold the reduction tickets, which must start at zero
  if (cudaMemsetAsync(h->scal, 0, sizeof(SemScalars), stream) != cudaSuccess ||
      cudaMemsetAsync(h->gtickets, 0, (size_t)SEM_MAX_GROUPS * 4, stream) != cudaSuccess)
    return fail(sem_fail(SEM_ERR_CUDA, "memset"));
  SetupArgs sa;
  sa.N = h->N;
  sa.n = n;
  sa.n3 = h->n3;
  sa.E = h->E;
  sa.gs6 = h->gs6;
  sa.gs12 = h->gs12;
  sa.gs16 = h->gs16;
  sa.verts = h->verts;
  sa.gx = h->gll_x;
  sa.gw = h->gll_w;
  sa.modes = modes;
  sa.nmodes = d->kappa_nmodes;
  sa.kap = d->kappa ? kap : nullptr;
  sa.alpha = d->alpha ? alpha : nullptr;
  sa.wJa_tmp = d->alpha ? alpha : nullptr;
  sa.G64 = h->G64;
  sa.G32 = h->G32;
  sa.G16 = h->G16;
  sa.kap32 = h->kap32;
  sa.Gemu = h->Gemu;
  sa.wJ = h->wJ;
  sa.wJa64 = h->wJa64;
  sa.wJa32 = h->wJa32;
  sa.wJaemu = h->wJaemu;
  sa.tangled = tangled;
  sa.emu_range = emu_range;
  k_setup_factors<<<grid_for(h->L, 256), 256, 0, stream>>>(sa);
  if (h->Gotf) k_setup_otf<<<grid_for(h->E, 128), 128, 0, stream>>>(h->verts, h->E, h->Gotf);

  // assembled diagonal: accumulate into dinv64, then invert it in place with the mask
  sem_handle hd = *h;  // by-value copy for kernels
  if (cudaMemsetAsync(h->dinv64, 0, (size_t)G * 8, stream) != cudaSuccess)
    return fail(sem_fail(SEM_ERR_CUDA, "memset"));
  const double *wJa_diag = d->alpha ? alpha : nullptr;  // holds w det J alpha after the factor kernel
  if (h->G64)
    k_setup_diag<double><<<grid_for(h->L, 256), 256, 0, stream>>>(hd, h->G64, nullptr, h->gs6, 1, wJa_diag,
                                                                   h->dinv64);
  else if (h->Gemu)
    k_setup_diag<float><<<grid_for(h->L, 256), 256, 0, stream>>>(hd, h->Gemu, h->Gemu + h->n3, h->gs12, 2,
                                                                  wJa_diag, h->dinv64);
  else if (h->G32)
    k_setup_diag<float><<<grid_for(h->L, 256), 256, 0, stream>>>(hd, h->G32, nullptr, h->gs6, 1, wJa_diag,
                                                                  h->dinv64);
  else
    k_setup_diag_geo<<<grid_for(h->L, 256), 256, 0, stream>>>(hd, sa, wJa_diag, h->dinv64);
  k_setup_dinv<<<grid_for(G, 256), 256, 0, stream>>>(hd, h->dinv64, h->dinv64, h->dinv32);
  if (h->geo6) {
    sem_handle hm = *h;
    sem_status ms = sem_mlp_setup_tables(&hm, stream);
    if (ms != SEM_OK) return fail(ms);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(sem_fail(SEM_ERR_CUDA, std::string("setup kernels: ") + cudaGetErrorString(e)));
  int flags_h[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(flags_h, tangled, 4 * sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(sem_fail(SEM_ERR_CUDA, std::string("setup: ") + cudaGetErrorString(e)));
  if (flags_h[0]) return fail(sem_fail(SEM_ERR_INVALID, "tangled element: det J <= 0 at some node"));
  // double-float factors: every intermediate product must keep its low word in the FP32 normal
  // range, which holds for factors within 2^-60 .. 2^60 (biased FP64 exponents 963 .. 1083)
  if (h->Gemu && (flags_h[2] > 1023 + 60 || flags_h[3] < 1023 - 60))
    return fail(sem_fail(SEM_ERR_INVALID,
                         "SEM_FEAT_EMU: geometric factors outside 2^-60 .. 2^60 (rescale the mesh or kappa)"));
  *out = h;
  return SEM_OK;
}

extern "C" void sem_free(sem_handle *h) { delete h; }

extern "C" sem_status sem_get_info(const sem_handle *h, sem_info *info) {
  if (!h || !info) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  info->N = h->N;
  info->nelem = h->E;
  info->nglobal = h->G;
  info->nlocal = h->L;
  return SEM_OK;
}

extern "C" sem_status sem_node_coords(sem_handle *h, double *d_xyz, sem_stream_t s) {
  if (!h || !d_xyz) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  k_node_coords<<<grid_for(h->L, 256), 256, 0, reinterpret_cast<cudaStream_t>(s)>>>(*h, d_xyz);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_glo_num(sem_handle *h, int64_t *d_glo, sem_stream_t s) {
  if (!h || !d_glo) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  k_glo_num<<<grid_for(h->L, 256), 256, 0, reinterpret_cast<cudaStream_t>(s)>>>(*h, d_glo);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_rhs(sem_handle *h, const double *d_fL, double *d_b, sem_stream_t s_) {
  if (!h || !d_fL || !d_b) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(s_);
  SEM_CUDA_TRY(cudaMemsetAsync(d_b, 0, (size_t)h->G * 8, s));
  k_rhs_scatter<<<grid_for(h->L, 256), 256, 0, s>>>(*h, d_fL, d_b);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_diag(sem_handle *h, double *d_diag, sem_stream_t s) {
  if (!h || !d_diag) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  k_diag_out<<<grid_for(h->G, 256), 256, 0, reinterpret_cast<cudaStream_t>(s)>>>(*h, d_diag);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}
