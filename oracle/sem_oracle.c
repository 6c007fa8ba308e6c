/*
 * Plain, slow FP64 CPU oracle for the spectral-element screened-Poisson operator of
 * arXiv 1403.0968, §4.2 ("Spectral Element Methods"), and for the solvers built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes (each function names the passage it follows):
 *   PDE        -div(kappa grad u) + alpha u = f            §4.2, Eq. 1
 *   weak form  <kappa grad u, grad v> + <alpha u, v> = <f, v>, V = continuous piecewise Q_N
 *                                                           §4.2.1, Eq. 2
 *   basis      tensor-product Lagrange polynomials on the 1-D Gauss-Lobatto-Legendre nodes
 *                                                           §4.2.1 (basis display)
 *   quadrature the same GLL nodes; the mass matrix is lumped to J w_abc (§4.2.1, lumped-mass
 *              display); the stiffness operator is the chain-rule / G^T G form of the
 *              sum-factorised display at the end of §4.2.1, with the geometric factors kept
 *              per elemental node.
 *   numbering  distinct global and local node numbering (§4.2.1, last paragraph, after
 *              Fischer 1991) with direct-stiffness summation Q^T.
 *   solver     preconditioned conjugate gradients (§4.2.2, first paragraph); the paper does not
 *              name the preconditioner, the Jacobi (diagonal) one is used.
 *
 * Parity pins: every function here is checked by tests/test_oracle_pins.py against closed forms,
 * invariants or brute force (GLL tables, quadrature exactness, A*1 = 0, symmetry, u^T A u against
 * the exact integral of |grad u|^2, dense element matrices, direct solves).
 *
 * Conventions (readings of the paper where it is silent):
 *   node (i,j,k) of an element has local index i + n*(j + n*k), n = N+1, i runs along r;
 *   vertex v = a + 2b + 4c sits at reference corner (r,s,t) = (2a-1, 2b-1, 2c-1);
 *   the six geometric factors per node are stored (rr, rs, rt, ss, st, tt) as
 *   G[e][f][node] and already include w_i w_j w_k, det J and kappa;
 *   kappa multiplies G at each node (the paper's u-hat = kappa u is read as kappa scaling
 *   the flux, which is what -div(kappa grad u) requires).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288L

/* ------------------------------------------------------------------------------------------
 * Legendre polynomial P_N and its derivative at x, by the three-term recurrence
 * (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}; P'_N from (1-x^2) P'_N = N (P_{N-1} - x P_N).
 * ---------------------------------------------------------------------------------------- */
static void legendre(int N, long double x, long double *pN, long double *pNm1) {
  long double p0 = 1.0L, p1 = x;
  if (N == 0) { *pN = 1.0L; *pNm1 = 0.0L; return; }
  for (int k = 1; k < N; ++k) {
    long double p2 = ((2.0L * k + 1.0L) * x * p1 - k * p0) / (k + 1.0L);
    p0 = p1;
    p1 = p2;
  }
  *pN = p1;
  *pNm1 = p0;
}

/*
 * GLL nodes and weights of order N (N+1 points) on [-1,1] — the 1-D Gauss-Lobatto-Legendre
 * nodes of §4.2.1.  x_0 = -1, x_N = 1, interior nodes are the roots of P'_N, found by Newton's
 * method in long double on q(x) = (1-x^2) P'_N(x) / N = P_{N-1} - x P_N, started from the
 * Chebyshev-Gauss-Lobatto points.  Weights w_i = 2 / (N (N+1) P_N(x_i)^2).
 * Returns 0 on success, -1 for N < 1.
 */
int orc_gll(int N, double *x, double *w) {
  if (N < 1) return -1;
  for (int i = 0; i <= N; ++i) {
    long double xi = -cosl(ORC_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 100; ++it) {
        long double pN, pNm1;
        legendre(N, xi, &pN, &pNm1);
        /* q = (1-x^2) P'_N / N; by Legendre's equation d/dx[(1-x^2) P'_N] = -N(N+1) P_N,
           so q' = -(N+1) P_N. */
        long double q = pNm1 - xi * pN;
        long double dq = -(N + 1.0L) * pN;
        long double step = q / dq;
        xi -= step;
        if (fabsl(step) < 1e-30L) break;
      }
    }
    long double pN, pNm1;
    legendre(N, xi, &pN, &pNm1);
    x[i] = (double)xi;
    w[i] = (double)(2.0L / ((long double)N * (N + 1.0L) * pN * pN));
  }
  return 0;
}

/*
 * Derivative matrix D[i*n + j] = l_j'(x_i) of the Lagrange basis on the nodes x (n = N+1),
 * straight from the product definition l_j(x) = prod_{b != j} (x - x_b) / (x_j - x_b):
 *   l_j'(x) = sum_{c != j} [ 1/(x_j - x_c) * prod_{b != j, c} (x - x_b)/(x_j - x_b) ].
 * This is the one-dimensional phi-hat' of §4.2.1 (derivative-sparsity display).
 */
void orc_lagrange_deriv(int N, const double *x, double *D) {
  int n = N + 1;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      long double sum = 0.0L;
      for (int c = 0; c < n; ++c) {
        if (c == j) continue;
        long double prod = 1.0L / ((long double)x[j] - x[c]);
        for (int b = 0; b < n; ++b) {
          if (b == j || b == c) continue;
          prod *= ((long double)x[i] - x[b]) / ((long double)x[j] - x[b]);
        }
        sum += prod;
      }
      D[i * n + j] = (double)sum;
    }
  }
}

/* Lagrange basis value l_j(y) on nodes x, product definition. */
static long double lagrange_val(int N, const double *x, int j, long double y) {
  long double p = 1.0L;
  for (int b = 0; b <= N; ++b)
    if (b != j) p *= (y - x[b]) / ((long double)x[j] - x[b]);
  return p;
}

/* ------------------------------------------------------------------------------------------
 * Trilinear element map x(r,s,t) = sum_v X_v (1 + r_v r)(1 + s_v s)(1 + t_v t) / 8 and its
 * analytic Jacobian d x_d / d r_k, for the hexahedra D^e mapped from [-1,1]^3 (§4.2.1).
 * ---------------------------------------------------------------------------------------- */
static void trilinear(const double *X /* [8][3] */, double r, double s, double t, double xyz[3],
                      double jac[3][3] /* jac[d][k] = d x_d / d r_k */) {
  for (int d = 0; d < 3; ++d) {
    xyz[d] = 0.0;
    for (int k = 0; k < 3; ++k) jac[d][k] = 0.0;
  }
  for (int v = 0; v < 8; ++v) {
    double rv = (v & 1) ? 1.0 : -1.0, sv = (v & 2) ? 1.0 : -1.0, tv = (v & 4) ? 1.0 : -1.0;
    double fr = 1.0 + rv * r, fs = 1.0 + sv * s, ft = 1.0 + tv * t;
    for (int d = 0; d < 3; ++d) {
      double Xd = X[v * 3 + d];
      xyz[d] += Xd * fr * fs * ft / 8.0;
      jac[d][0] += Xd * rv * fs * ft / 8.0;
      jac[d][1] += Xd * fr * sv * ft / 8.0;
      jac[d][2] += Xd * fr * fs * tv / 8.0;
    }
  }
}

static double det3(double a[3][3]) {
  return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
         a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
         a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

/* inverse of a 3x3 matrix by cofactors: inv[k][d] = d r_k / d x_d when a = dx/dr */
static void inv3(double a[3][3], double inv[3][3]) {
  double det = det3(a);
  inv[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / det;
  inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
  inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
  inv[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / det;
  inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
  inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
  inv[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / det;
  inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
  inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
}

/*
 * kappa(x) = exp( sum_m a_m cos(2 pi k_m . x + phi_m) ), modes[m] = (kx, ky, kz, phi, a).
 * With nmodes == 0 this is kappa = 1.  (The material coefficient kappa(x) of §4.2, Eq. 1; the
 * Fourier-mode form is the synthetic workload's choice.)
 */
double orc_kappa(int nmodes, const double *modes, double x, double y, double z) {
  double g = 0.0;
  for (int m = 0; m < nmodes; ++m) {
    const double *md = modes + 5 * m;
    g += md[4] * cos(2.0 * (double)ORC_PI * (md[0] * x + md[1] * y + md[2] * z) + md[3]);
  }
  return exp(g);
}

/* physical coordinates of every elemental node: xyz[(e*n3 + p)*3 + d] */
int orc_node_coords(int N, int64_t nelem, const double *vert, double *xyz) {
  int n = N + 1, n3 = n * n * n;
  double *x = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
  if (orc_gll(N, x, w)) { free(x); free(w); return -1; }
  for (int64_t e = 0; e < nelem; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          double p[3], jac[3][3];
          trilinear(vert + e * 24, x[i], x[j], x[k], p, jac);
          int64_t q = e * n3 + i + n * (j + n * k);
          for (int d = 0; d < 3; ++d) xyz[q * 3 + d] = p[d];
        }
  free(x);
  free(w);
  return 0;
}

/*
 * Per-node geometric factors of the sum-factorised stiffness display of §4.2.1:
 *   G_kl = w_i w_j w_k * det(J) * kappa * sum_d (d r_k / d x_d)(d r_l / d x_d),
 * i.e. J^e * G-hat with G-hat = G^T G, stored as G[(e*6 + f)*n3 + p] for f = rr, rs, rt, ss, st, tt.
 * Also the lumped mass w_i w_j w_k det(J) (§4.2.1 lumped-mass display) in wJ[e*n3 + p].
 * kappa_nodal (may be NULL) overrides the Fourier-mode kappa; NULL and nmodes == 0 means kappa = 1.
 * Returns -2 if some det(J) <= 0 (tangled element).
 */
int orc_factors(int N, int64_t nelem, const double *vert, const double *kappa_nodal, int nmodes,
                const double *modes, double *G, double *wJ) {
  int n = N + 1, n3 = n * n * n;
  double *x = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
  if (orc_gll(N, x, w)) { free(x); free(w); return -1; }
  int bad = 0;
  for (int64_t e = 0; e < nelem; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int p = i + n * (j + n * k);
          double xyz[3], jac[3][3], rx[3][3];
          trilinear(vert + e * 24, x[i], x[j], x[k], xyz, jac);
          double det = det3(jac);
          if (!(det > 0.0)) bad = 1;
          inv3(jac, rx); /* rx[k][d] = d r_k / d x_d */
          double kap = kappa_nodal ? kappa_nodal[e * n3 + p]
                                   : orc_kappa(nmodes, modes, xyz[0], xyz[1], xyz[2]);
          double wd = w[i] * w[j] * w[k] * det;
          int f = 0;
          for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b) {
              double g = 0.0;
              for (int d = 0; d < 3; ++d) g += rx[a][d] * rx[b][d];
              G[(e * 6 + f) * n3 + p] = wd * kap * g;
              ++f;
            }
          if (wJ) wJ[e * n3 + p] = wd;
        }
  free(x);
  free(w);
  return bad ? -2 : 0;
}

/*
 * O1: dense element matrix by brute force, straight from the weak form (§4.2.1, Eq. 2) with
 * GLL quadrature and the chain rule u_x = r_x u_r + s_x u_s + t_x u_t:
 *   A_pq = sum_m w_m det J_m kappa_m  (J^-T grad_r phi_p)(xi_m) . (J^-T grad_r phi_q)(xi_m)
 *          + delta_pq w_p det J_p alpha_p .
 * grad_r phi_p at node m is evaluated from the Lagrange product formula at the node
 * coordinates (no D matrix), so this is independent of the sum-factorised path.
 * O(n^9) work: for 1-8 elements only.  A is n3 x n3 row-major.
 */
int orc_element_matrix(int N, const double *vert_e, const double *kappa_e, const double *alpha_e,
                       double *A) {
  int n = N + 1, n3 = n * n * n;
  double *x = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
  if (orc_gll(N, x, w)) { free(x); free(w); return -1; }
  /* dl[a*n + m] = l_a'(x_m) and lv[a*n + m] = l_a(x_m), both from the product formula */
  long double *dl = malloc(sizeof(long double) * n * n), *lv = malloc(sizeof(long double) * n * n);
  for (int a = 0; a < n; ++a)
    for (int m = 0; m < n; ++m) {
      long double s = 0.0L;
      for (int c = 0; c < n; ++c) {
        if (c == a) continue;
        long double prod = 1.0L / ((long double)x[a] - x[c]);
        for (int b = 0; b < n; ++b)
          if (b != a && b != c) prod *= ((long double)x[m] - x[b]) / ((long double)x[a] - x[b]);
        s += prod;
      }
      dl[a * n + m] = s;
      lv[a * n + m] = lagrange_val(N, x, a, x[m]);
    }
  /* physical gradients of every basis function at every quadrature node */
  double *grad = malloc(sizeof(double) * (size_t)n3 * n3 * 3); /* [p][m][3] */
  double *wq = malloc(sizeof(double) * n3);
  for (int mk = 0; mk < n; ++mk)
    for (int mj = 0; mj < n; ++mj)
      for (int mi = 0; mi < n; ++mi) {
        int m = mi + n * (mj + n * mk);
        double xyz[3], jac[3][3], rx[3][3];
        trilinear(vert_e, x[mi], x[mj], x[mk], xyz, jac);
        double det = det3(jac);
        inv3(jac, rx);
        double kap = kappa_e ? kappa_e[m] : 1.0;
        wq[m] = w[mi] * w[mj] * w[mk] * det * kap;
        for (int pk = 0; pk < n; ++pk)
          for (int pj = 0; pj < n; ++pj)
            for (int pi = 0; pi < n; ++pi) {
              int p = pi + n * (pj + n * pk);
              long double gr = dl[pi * n + mi] * lv[pj * n + mj] * lv[pk * n + mk];
              long double gs = lv[pi * n + mi] * dl[pj * n + mj] * lv[pk * n + mk];
              long double gt = lv[pi * n + mi] * lv[pj * n + mj] * dl[pk * n + mk];
              for (int d = 0; d < 3; ++d)
                grad[((size_t)p * n3 + m) * 3 + d] =
                    (double)(gr * rx[0][d] + gs * rx[1][d] + gt * rx[2][d]);
            }
      }
  for (int p = 0; p < n3; ++p)
    for (int q = 0; q < n3; ++q) {
      long double s = 0.0L;
      for (int m = 0; m < n3; ++m) {
        const double *gp = grad + ((size_t)p * n3 + m) * 3, *gq = grad + ((size_t)q * n3 + m) * 3;
        s += (long double)wq[m] * ((long double)gp[0] * gq[0] + (long double)gp[1] * gq[1] +
                                   (long double)gp[2] * gq[2]);
      }
      A[(size_t)p * n3 + q] = (double)s;
    }
  if (alpha_e) {
    for (int pk = 0; pk < n; ++pk)
      for (int pj = 0; pj < n; ++pj)
        for (int pi = 0; pi < n; ++pi) {
          int p = pi + n * (pj + n * pk);
          double xyz[3], jac[3][3];
          trilinear(vert_e, x[pi], x[pj], x[pk], xyz, jac);
          A[(size_t)p * n3 + p] += w[pi] * w[pj] * w[pk] * det3(jac) * alpha_e[p];
        }
  }
  free(grad);
  free(wq);
  free(dl);
  free(lv);
  free(x);
  free(w);
  return 0;
}

/*
 * O2: local (unassembled) operator by plain sum factorisation — the sum-factorised stiffness
 * display at the end of §4.2.1, written out step by step for every element:
 *   u_r = sum_m D_im u_mjk,  u_s = sum_m D_jm u_imk,  u_t = sum_m D_km u_ijm      (gradients)
 *   (w_r, w_s, w_t) = G (u_r, u_s, u_t)   with the symmetric 6-factor G at node ijk (scaling)
 *   y_ijk = sum_m D_mi w_r,mjk + D_mj w_s,imk + D_mk w_t,ijm                      (transpose)
 *   y_ijk += wJalpha_ijk u_ijk                                          (lumped mass term)
 * D here is built from the Lagrange product formula (orc_lagrange_deriv).  Elements are
 * independent, so the element loop runs under OpenMP.  uL, yL are [E][n3].
 */
void orc_apply_local(int N, int64_t nelem, const double *G, const double *wJalpha,
                     const double *uL, double *yL) {
  int n = N + 1, n3 = n * n * n;
  double x[32], w[32], D[32 * 32];
  orc_gll(N, x, w);
  orc_lagrange_deriv(N, x, D);
#pragma omp parallel
  {
    double *ur = malloc(sizeof(double) * n3), *us = malloc(sizeof(double) * n3),
           *ut = malloc(sizeof(double) * n3);
#pragma omp for schedule(static)
    for (int64_t e = 0; e < nelem; ++e) {
      const double *u = uL + e * n3;
      const double *g = G + e * 6 * n3;
      double *y = yL + e * n3;
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            double a = 0.0, b = 0.0, c = 0.0;
            for (int m = 0; m < n; ++m) {
              a += D[i * n + m] * u[m + n * (j + n * k)];
              b += D[j * n + m] * u[i + n * (m + n * k)];
              c += D[k * n + m] * u[i + n * (j + n * m)];
            }
            int p = i + n * (j + n * k);
            ur[p] = g[0 * n3 + p] * a + g[1 * n3 + p] * b + g[2 * n3 + p] * c;
            us[p] = g[1 * n3 + p] * a + g[3 * n3 + p] * b + g[4 * n3 + p] * c;
            ut[p] = g[2 * n3 + p] * a + g[4 * n3 + p] * b + g[5 * n3 + p] * c;
          }
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int m = 0; m < n; ++m) {
              s += D[m * n + i] * ur[m + n * (j + n * k)];
              s += D[m * n + j] * us[i + n * (m + n * k)];
              s += D[m * n + k] * ut[i + n * (j + n * m)];
            }
            int p = i + n * (j + n * k);
            if (wJalpha) s += wJalpha[e * n3 + p] * u[p];
            y[p] = s;
          }
    }
    free(ur);
    free(us);
    free(ut);
  }
}

/*
 * Global numbering of a structured sx*sy*sz box of elements (element (ex,ey,ez) has index
 * ex + sx*(ey + sy*ez)): global id of local node (i,j,k) is I + (sx N + 1)(J + (sy N + 1) K)
 * with I = ex N + i etc.  Nodes shared by neighbouring elements get one id (distinct
 * global/local numbering, §4.2.1 after Fischer 1991).
 */
void orc_box_numbering(int sx, int sy, int sz, int N, int64_t *glo) {
  int n = N + 1, n3 = n * n * n;
  int64_t gx = (int64_t)sx * N + 1, gy = (int64_t)sy * N + 1;
  for (int ez = 0; ez < sz; ++ez)
    for (int ey = 0; ey < sy; ++ey)
      for (int ex = 0; ex < sx; ++ex) {
        int64_t e = ex + (int64_t)sx * (ey + (int64_t)sy * ez);
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              int64_t I = (int64_t)ex * N + i, J = (int64_t)ey * N + j, K = (int64_t)ez * N + k;
              glo[e * n3 + i + n * (j + n * k)] = I + gx * (J + gy * K);
            }
      }
}

/* 1 on global nodes of the box boundary (homogeneous Dirichlet), 0 elsewhere */
void orc_box_dirichlet(int sx, int sy, int sz, int N, uint8_t *mask) {
  int64_t gx = (int64_t)sx * N + 1, gy = (int64_t)sy * N + 1, gz = (int64_t)sz * N + 1;
  for (int64_t K = 0; K < gz; ++K)
    for (int64_t J = 0; J < gy; ++J)
      for (int64_t I = 0; I < gx; ++I)
        mask[I + gx * (J + gy * K)] =
            (I == 0 || J == 0 || K == 0 || I == gx - 1 || J == gy - 1 || K == gz - 1) ? 1 : 0;
}

/*
 * Assembled operator y = M Q^T A_L Q M u on global nodes (M zeroes Dirichlet nodes; mask may be
 * NULL).  Q gathers by glo, Q^T sums local results into their global node in ascending (e,p)
 * order — the direct-stiffness summation of §4.2.1.
 */
void orc_apply(int N, int64_t nelem, const int64_t *glo, const double *G, const double *wJalpha,
               int64_t nglobal, const uint8_t *mask, const double *u, double *y) {
  int n = N + 1, n3 = n * n * n;
  int64_t L = nelem * n3;
  double *uL = malloc(sizeof(double) * L), *yL = malloc(sizeof(double) * L);
  for (int64_t q = 0; q < L; ++q) {
    int64_t g = glo[q];
    uL[q] = (mask && mask[g]) ? 0.0 : u[g];
  }
  orc_apply_local(N, nelem, G, wJalpha, uL, yL);
  for (int64_t g = 0; g < nglobal; ++g) y[g] = 0.0;
  for (int64_t q = 0; q < L; ++q) y[glo[q]] += yL[q];
  if (mask)
    for (int64_t g = 0; g < nglobal; ++g)
      if (mask[g]) y[g] = 0.0;
  free(uL);
  free(yL);
}

/*
 * Assembled diagonal of M A M (Jacobi preconditioner).  The diagonal entry of the element
 * operator at node p = (a,b,c) follows from the derivative-sparsity display of §4.2.1
 * (d/dr phi_abc at node (m1,m2,m3) is D[m1][a] when (m2,m3) = (b,c), else 0):
 *   A_pp = sum_m1 G_rr(m1,b,c) D[m1][a]^2 + sum_m2 G_ss(a,m2,c) D[m2][b]^2
 *        + sum_m3 G_tt(a,b,m3) D[m3][c]^2
 *        + 2 D[a][a] D[b][b] G_rs(p) + 2 D[a][a] D[c][c] G_rt(p) + 2 D[b][b] D[c][c] G_st(p)
 *        + wJalpha(p).
 * Dirichlet nodes get 1.
 */
void orc_diag(int N, int64_t nelem, const int64_t *glo, const double *G, const double *wJalpha,
              int64_t nglobal, const uint8_t *mask, double *diag) {
  int n = N + 1, n3 = n * n * n;
  double x[32], w[32], D[32 * 32];
  orc_gll(N, x, w);
  orc_lagrange_deriv(N, x, D);
  for (int64_t g = 0; g < nglobal; ++g) diag[g] = 0.0;
  for (int64_t e = 0; e < nelem; ++e) {
    const double *g = G + e * 6 * n3;
    for (int c = 0; c < n; ++c)
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          int p = a + n * (b + n * c);
          double s = 0.0;
          for (int m = 0; m < n; ++m) {
            s += g[0 * n3 + m + n * (b + n * c)] * D[m * n + a] * D[m * n + a];
            s += g[3 * n3 + a + n * (m + n * c)] * D[m * n + b] * D[m * n + b];
            s += g[5 * n3 + a + n * (b + n * m)] * D[m * n + c] * D[m * n + c];
          }
          s += 2.0 * D[a * n + a] * D[b * n + b] * g[1 * n3 + p];
          s += 2.0 * D[a * n + a] * D[c * n + c] * g[2 * n3 + p];
          s += 2.0 * D[b * n + b] * D[c * n + c] * g[4 * n3 + p];
          if (wJalpha) s += wJalpha[e * n3 + p];
          diag[glo[e * n3 + p]] += s;
        }
  }
  if (mask)
    for (int64_t gi = 0; gi < nglobal; ++gi)
      if (mask[gi]) diag[gi] = 1.0;
}

/* Right-hand side b = M Q^T (w J f) from nodal f (lumped mass, §4.2.1). */
void orc_rhs(int N, int64_t nelem, const int64_t *glo, const double *wJ, const double *fL,
             int64_t nglobal, const uint8_t *mask, double *b) {
  int n3 = (N + 1) * (N + 1) * (N + 1);
  for (int64_t g = 0; g < nglobal; ++g) b[g] = 0.0;
  for (int64_t q = 0; q < nelem * n3; ++q) b[glo[q]] += wJ[q] * fL[q];
  if (mask)
    for (int64_t g = 0; g < nglobal; ++g)
      if (mask[g]) b[g] = 0.0;
}

static double dot(int64_t n, const double *a, const double *b) {
  long double s = 0.0L;
  for (int64_t i = 0; i < n; ++i) s += (long double)a[i] * b[i];
  return (double)s;
}

/*
 * Jacobi-preconditioned conjugate gradients (the PCG of §4.2.2; preconditioned CG as in Saad,
 * Iterative Methods, Algorithm 9.1), on the masked global system, from the initial guess in x.
 *   r = b - A x; z = r / d; p = z
 *   loop: alpha = (r,z)/(p,Ap); x += alpha p; r -= alpha Ap;
 *         stop when ||r||_2 <= rtol ||b||_2; z = r/d; beta = (r,z)_new/(r,z)_old; p = z + beta p
 * Returns the iteration count, or -1 without convergence in max_it.  res_out gets the final
 * recursive relative residual.
 */
int orc_pcg(int N, int64_t nelem, const int64_t *glo, const double *G, const double *wJalpha,
            int64_t nglobal, const uint8_t *mask, const double *diag, const double *b, double *x,
            double rtol, int max_it, double *res_out) {
  double *r = malloc(sizeof(double) * nglobal), *z = malloc(sizeof(double) * nglobal),
         *p = malloc(sizeof(double) * nglobal), *Ap = malloc(sizeof(double) * nglobal);
  orc_apply(N, nelem, glo, G, wJalpha, nglobal, mask, x, Ap);
  for (int64_t i = 0; i < nglobal; ++i) {
    r[i] = ((mask && mask[i]) ? 0.0 : b[i]) - Ap[i];
    z[i] = r[i] / diag[i];
    p[i] = z[i];
  }
  double bnorm = sqrt(dot(nglobal, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
  double rz = dot(nglobal, r, z);
  int it = 0, conv = 0;
  double rel = sqrt(dot(nglobal, r, r)) / bnorm;
  if (rel <= rtol) conv = 1;
  while (!conv && it < max_it) {
    orc_apply(N, nelem, glo, G, wJalpha, nglobal, mask, p, Ap);
    double alpha = rz / dot(nglobal, p, Ap);
    for (int64_t i = 0; i < nglobal; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    ++it;
    rel = sqrt(dot(nglobal, r, r)) / bnorm;
    if (rel <= rtol) { conv = 1; break; }
    for (int64_t i = 0; i < nglobal; ++i) z[i] = r[i] / diag[i];
    double rz_new = dot(nglobal, r, z);
    double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t i = 0; i < nglobal; ++i) p[i] = z[i] + beta * p[i];
  }
  if (res_out) *res_out = rel;
  free(r);
  free(z);
  free(p);
  free(Ap);
  return conv ? it : -1;
}

/* Thread count of the OpenMP loops (the timed CPU baseline reports it and also runs on one core):
   sets it when n > 0 and returns the count that was in effect before. */
int orc_threads(int n) {
#ifdef _OPENMP
  const int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
#else
  (void)n;
  return 1;
#endif
}
