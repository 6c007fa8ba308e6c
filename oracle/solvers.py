"""Plainly written solvers around the oracle's operator: mixed-precision iterative refinement and
flexible CG (test infrastructure only: the tests, the smoke check and the benchmark's CPU-baseline
leg may use it; the product library never does, and this module imports nothing from the CUDA
package).

The paper solves the screened-Poisson system by preconditioned CG (§4.2.2) and names neither a
preconditioner nor a precision scheme; the two variants here are the ones the GPU library builds on
that statement, written out step by step in numpy with the oracle's FP64 operator (``apply``) as
the only library primitive:

  ir   iterative refinement (Wilkinson): the outer residual r = b - A x in FP64; an inner
       Jacobi-PCG on A d = r / ||r|| run in FP32 arithmetic (every vector FP32, the operator's
       result rounded to FP32) to a relative tolerance; x += ||r|| d; repeat until the FP64
       residual meets rtol.
  fcg  flexible CG (Notay 2000, FCG(1) with the Polak-Ribiere direction update) with an arbitrary,
       possibly iteration-dependent preconditioner z = P(r): beta = (z_k, r_k - r_{k-1}) /
       (z_{k-1}, r_{k-1}), p = z + beta p, alpha = (z_k, r_k) / (p, A p).  A correction with
       (z, r) <= 0 or a non-finite entry is replaced by the Jacobi step D^-1 r for that iteration.

Parity status (pins in tests/test_oracle_pins.py): both against a dense direct solve of the
assembled brute-force matrix; fcg with the fixed Jacobi preconditioner against the oracle's
Jacobi-PCG (same iterates in exact arithmetic); fcg with a randomly varying SPD preconditioner and
with a rejected (negative) correction; ir's outer residual contraction against its inner tolerance.
"""
from __future__ import annotations

import numpy as np

from . import apply


def _free(mask, n):
    return np.ones(n, dtype=bool) if mask is None else (np.asarray(mask) == 0)


def jacobi_pcg(op, b, dinv, rtol, max_it, dtype=np.float64):
    """Saad Alg. 9.1 with z = dinv * r, in the arithmetic of `dtype` (vectors and scalars), from
    x0 = 0; stops when ||r|| <= rtol ||b||.  op(p) returns A p in that dtype.
    Returns (x, iterations)."""
    b = b.astype(dtype)
    dinv = dinv.astype(dtype)
    x = np.zeros_like(b)
    r = b.copy()
    z = r * dinv
    p = z.copy()
    rz = np.dot(r, z)
    tol2 = dtype(rtol) ** 2 * np.dot(b, b)
    it = 0
    while it < max_it and np.dot(r, r) > tol2:
        q = op(p)
        alpha = rz / np.dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        z = r * dinv
        rz_new = np.dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


def ir(N, glo, G, b, dg, mask=None, rtol=1e-10, inner_rtol=1e-3, max_outer=50, inner_max_it=100000):
    """Iterative refinement: FP64 outer residual, FP32 inner Jacobi-PCG.  dg is the assembled
    diagonal (1 on Dirichlet nodes).  Returns (x, outer steps, inner iterations, residual history)."""
    b = np.asarray(b, dtype=np.float64)
    free = _free(mask, b.shape[0])
    dinv = np.where(free, 1.0 / np.asarray(dg, dtype=np.float64), 0.0)

    def op32(p):  # the operator in FP32: FP32 input, result rounded to FP32
        return apply(N, glo, G, p.astype(np.float64), mask=mask).astype(np.float32)

    x = np.zeros_like(b)
    nb = np.linalg.norm(np.where(free, b, 0.0))
    hist = []
    inner_total = 0
    for outer in range(max_outer + 1):
        r = np.where(free, b - apply(N, glo, G, x, mask=mask), 0.0)
        nr = np.linalg.norm(r)
        hist.append(nr / nb if nb > 0 else 0.0)
        if nr <= rtol * nb or outer == max_outer:
            return x, outer, inner_total, hist
        d, its = jacobi_pcg(op32, r / nr, dinv, inner_rtol, inner_max_it, dtype=np.float32)
        inner_total += its
        x = x + nr * d.astype(np.float64)
    return x, max_outer, inner_total, hist


def fcg(N, glo, G, b, dg, precond, mask=None, rtol=1e-10, max_it=100000):
    """Flexible CG with z = precond(r, k) (k = iteration index) and the Jacobi fallback.
    Returns (x, iterations, number of fallbacks)."""
    b = np.asarray(b, dtype=np.float64)
    free = _free(mask, b.shape[0])
    dinv = np.where(free, 1.0 / np.asarray(dg, dtype=np.float64), 0.0)
    x = np.zeros_like(b)
    r = np.where(free, b, 0.0)
    tol2 = rtol * rtol * np.dot(r, r)
    p = None
    z_old_r_old = None
    r_old = None
    fallbacks = 0
    k = 0
    while k < max_it and np.dot(r, r) > tol2:
        z = np.where(free, precond(r, k), 0.0)
        zr = np.dot(z, r)
        if not (zr > 0.0) or not np.all(np.isfinite(z)):
            z = r * dinv
            zr = np.dot(z, r)
            fallbacks += 1
        if p is None:
            p = z.copy()
        else:
            beta = np.dot(z, r - r_old) / z_old_r_old
            p = z + beta * p
        q = apply(N, glo, G, p, mask=mask)
        alpha = zr / np.dot(p, q)
        x = x + alpha * p
        r_old = r
        z_old_r_old = zr
        r = r - alpha * q
        k += 1
    return x, k, fallbacks
