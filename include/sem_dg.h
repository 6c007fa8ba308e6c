/*
 * libsem — discontinuous-Galerkin shallow-water volume kernel (arXiv 1403.0968 §4.3).
 *
 * The 2-D shallow-water equations in conservative form (§4.3, governing equations):
 * Q = (h, hu, hv), F = (hu, hu^2/h + g h^2/2, hu hv/h), G = (hv, hu hv/h, hv^2/h + g h^2/2),
 * S = (0, -g h dB/dx, -g h dB/dy), discretised by nodal DG of degree N on affine triangles
 * (§4.3, the weak form).  The volume kernel returns, per element and node, the volume term of the
 * weak form with the element mass matrix applied inverted:
 *
 *   rhs_i = sum_j Drw_ij (rx F_j + ry G_j) + Dsw_ij (sx F_j + sy G_j) + S_i,
 *
 * Drw = Mhat^-1 Shat_r^T, Dsw = Mhat^-1 Shat_s^T on the reference triangle
 * T = {r, s >= -1, r + s <= 0} with Mhat_ij = int_T l_i l_j and (Shat_r)_ij = int_T l_i dl_j/dr,
 * l_i the Lagrange basis on the equispaced nodes r = -1 + 2a/N, s = -1 + 2b/N (a + b <= N,
 * a fastest), Np = (N+1)(N+2)/2 nodes.  Element arrays are [E][field][Np] in device memory the
 * caller owns.  Errors are returned, never raised; nothing is allocated.
 */
#pragma once

#include "sem.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_DG_MAX_ORDER 8 /* the orders the paper measures */

/* Host only.  Drw, Dsw (row-major Np x Np, FP64) of order N, from the orthonormal (Dubiner)
   basis: Drw = (V V^T) Dr^T (V V^T)^-1 with Dr = V_r V^-1.  Errors: SEM_ERR_INVALID. */
sem_status sem_dg_operators(int32_t N, double *Drw, double *Dsw);

/* Host only.  Bytes of the device operator block of order N in precision prec (SEM_FP64 or
   SEM_FP32): Drw then Dsw, each row zero padded to an odd number of 16-byte vectors. */
sem_status sem_dg_operator_bytes(int32_t N, sem_prec prec, size_t *bytes);

/* Writes the operator block of order N into d_ops (device, sem_dg_operator_bytes long), on
   stream.  Errors: SEM_ERR_INVALID, SEM_ERR_CUDA. */
sem_status sem_dg_load_operators(int32_t N, sem_prec prec, void *d_ops, size_t bytes, sem_stream_t stream);

/* d_geo[E][4] = (rx, ry, sx, sy) of each triangle's affine map x = -(r+s)/2 v1 + (1+r)/2 v2 +
   (1+s)/2 v3, from d_verts[E][3][2] (FP64, counter-clockwise), formed in FP64 and stored in prec
   (SEM_FP64 or SEM_FP32).  Errors: SEM_ERR_INVALID (also for a zero-area triangle, reported by
   a flag the call reads back), SEM_ERR_CUDA.  Synchronises the stream. */
sem_status sem_dg_geometry(sem_prec prec, int64_t E, const double *d_verts, void *d_geo, sem_stream_t stream);

/*
 * The volume right-hand side.
 *   prec    SEM_FP64 (double arrays) or SEM_FP32 (float arrays); arithmetic in that type.
 *   N       order 1..SEM_DG_MAX_ORDER;  E elements (>= 1);  g gravitational acceleration.
 *   d_ops   operator block from sem_dg_load_operators (same N and prec).
 *   d_Q     [E][3][Np] nodal h, hu, hv (h > 0).
 *   d_Bxy   [E][2][Np] nodal dB/dx, dB/dy.
 *   d_geo   [E][4] rx, ry, sx, sy of each element's affine map.
 *   d_rhs   [E][3][Np] output; must not overlap the inputs.
 * One kernel launch.  Errors: SEM_ERR_INVALID, SEM_ERR_CUDA.
 */
sem_status sem_dg_volume(sem_prec prec, int32_t N, int64_t E, double g, const void *d_ops, const void *d_Q,
                         const void *d_Bxy, const void *d_geo, void *d_rhs, sem_stream_t stream);

#ifdef __cplusplus
}
#endif
