/*
 * libsem — finite-difference wave step (arXiv 1403.0968 §4.1).
 *
 * The 2-D acoustic wave equation u_tt = u_xx + u_yy (§4.1, governing equation) on a structured
 * grid of w x h nodes, stepped by the central second difference in time with central
 * (2r+1)-point second-derivative stencils of order 2r in each direction (§4.1, the discrete
 * stencil operator display, and Algorithm 1):
 *
 *   u_{n+1}(i,j) = 2 u_n(i,j) - u_{n-1}(i,j)
 *                  + dt^2 ( sum_k c_k u_n(i+k,j) / dx^2 + sum_k c_k u_n(i,j+k) / dy^2 ),  k = -r..r.
 *
 * The boundary is periodic, as in the §4.1 kernel listing: neighbour indices wrap around the grid,
 * i+k modulo w and j+k modulo h (the listing's (i + k + w) % w for w >= r; grids narrower than the
 * stencil wrap more than once).  Every grid node is updated.  Grids are row-major [h][w]
 * (x fastest), in device memory the caller owns.  Errors are returned, never raised; nothing is
 * allocated.
 */
#pragma once

#include "sem.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_FD_MAX_RADIUS 7 /* stencil sizes 3..15, the range the paper measures */

/* Host only.  c[0..2r] = c_{-r..r}, the central second-derivative weights of order 2r (exact for
   polynomials of degree <= 2r+1), in FP64.  Errors: SEM_ERR_INVALID (r outside 1..7, c NULL). */
sem_status sem_fd_weights(int32_t r, double *c);

/*
 * One leapfrog step.
 *   prec          SEM_FP64 (double grids) or SEM_FP32 (float grids); arithmetic in that type.
 *   r             stencil radius, 1..SEM_FD_MAX_RADIUS.
 *   w, h          grid nodes in x and y (>= 1 each).
 *   dt, dx, dy    time step and node spacings (> 0).
 *   d_u           u_n, [h][w], read only.
 *   d_uprev_next  in: u_{n-1}; out: u_{n+1} (each node is read before it is overwritten by the
 *                 thread that owns it).  Must not alias d_u.
 * One kernel launch on `stream`.  When the rows are a multiple of 16 bytes and d_u is 16-byte
 * aligned, the tile of u_n with its halo is staged in shared memory by one 2-D tensor (TMA) copy per
 * block, with a bounded wait (see sem_fd_status); otherwise, and for the tiles whose halo wraps
 * around the grid's edge, by plain loads.
 * Errors: SEM_ERR_INVALID (bad argument), SEM_ERR_CUDA.
 */
sem_status sem_fd_step(sem_prec prec, int32_t r, int64_t w, int64_t h, double dt, double dx, double dy,
                       const void *d_u, void *d_uprev_next, sem_stream_t stream);

/* Synchronises `stream` and reports whether a step since the last call gave up waiting for its
   tile copy (SEM_ERR_TIMEOUT; the flag is then cleared, that step's output is incomplete);
   SEM_OK otherwise.  The flag is one per device, shared by all streams. */
sem_status sem_fd_status(sem_stream_t stream);

#ifdef __cplusplus
}
#endif
