"""FP64 reference of the finite-difference wave example of arXiv 1403.0968 §4.1 (test
infrastructure only: the tests, the smoke check and the benchmark's CPU-baseline leg may use it;
the product library never does, and this module imports nothing from the CUDA package).

What it computes (§4.1, the discrete stencil operator display and Algorithm 1): the 2-D wave
equation u_tt = u_xx + u_yy on a structured grid of w x h nodes (x fastest, spacing dx, dy),
stepped by the central second difference in time (leapfrog) with central (2r+1)-point
second-derivative stencils of order 2r in x and in y:

    u_{n+1}(i, j) = 2 u_n(i, j) - u_{n-1}(i, j)
                    + dt^2 ( sum_k c_k u_n(i+k, j) / dx^2 + sum_k c_k u_n(i, j+k) / dy^2 ),
    k = -r..r,

with periodic boundaries: the neighbour indices wrap around the grid, i+k taken modulo w and j+k
modulo h, as the paper's fd2d kernel listing does (§4.1), and every grid node is updated.  The
listing wraps with (i + k + w) % w, which equals (i + k) mod w whenever w >= r; for grids narrower
than the stencil the mathematical modulo is taken (the stencil then visits a node more than once).
The sign of the time terms follows the wave equation; the paper's display prints them with the
opposite sign (a reading, recorded with the others in the design notes).

The weights c_k are the unique symmetric weights that make the stencil exact for every polynomial
of degree <= 2r: sum_k c_k k^m = m! [m == 2] for m = 0..2r, solved here in exact rational
arithmetic (Gauss-Jordan over fractions).

Parity status (pins in tests/test_fd_oracle_pins.py): weights against the published tables for
r = 1..4 and against exactness on monomials; the step on a grid-periodic Fourier mode against its
closed-form leapfrog amplitude recurrence (every node, including the wrapped edges); commutation
with cyclic shifts of the grid; the step against a cubic exact solution of the wave equation away
from the wrap seam; the order of accuracy of the stencils on a smooth function; the time-reversal
symmetry of leapfrog.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def weights_exact(r: int):
    """Central second-derivative weights c_{-r..r} as Fractions (moment conditions, exact)."""
    if r < 1:
        raise ValueError("radius must be >= 1")
    # unknowns c_0, c_1..c_r (c_{-k} = c_k); odd moments vanish by symmetry, so the conditions are
    # m = 0, 2, 4, .., 2r:  c_0 [m == 0] + 2 sum_{k>=1} c_k k^m = m! [m == 2]
    n = r + 1
    A = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    for row, m in enumerate(range(0, 2 * r + 1, 2)):
        A[row][0] = Fraction(1 if m == 0 else 0)
        for k in range(1, r + 1):
            A[row][k] = Fraction(2 * k ** m)
        b[row] = Fraction(2 if m == 2 else 0)
    # Gauss-Jordan elimination, exact
    for col in range(n):
        piv = next(i for i in range(col, n) if A[i][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        p = A[col][col]
        A[col] = [a / p for a in A[col]]
        b[col] = b[col] / p
        for i in range(n):
            if i != col and A[i][col] != 0:
                f = A[i][col]
                A[i] = [a - f * c for a, c in zip(A[i], A[col])]
                b[i] = b[i] - f * b[col]
    half = b  # c_0, c_1, .., c_r
    return [half[abs(k)] for k in range(-r, r + 1)]


def weights(r: int) -> np.ndarray:
    """The same weights as FP64 numbers, c_{-r..r}."""
    return np.array([float(c) for c in weights_exact(r)])


def laplacian(u: np.ndarray, r: int, dx: float, dy: float) -> np.ndarray:
    """sum_k c_k u(i+k, j) / dx^2 + sum_k c_k u(i, j+k) / dy^2 on an [h][w] grid, indices periodic."""
    h, w = u.shape
    c = weights(r)
    lap = np.zeros_like(u)
    for k in range(-r, r + 1):
        xi = (np.arange(w) + k) % w  # i + k wrapped into [0, w)
        yj = (np.arange(h) + k) % h  # j + k wrapped into [0, h)
        lap += c[k + r] * u[:, xi] / (dx * dx)
        lap += c[k + r] * u[yj, :] / (dy * dy)
    return lap


def step(u: np.ndarray, uprev: np.ndarray, r: int, dt: float, dx: float, dy: float) -> np.ndarray:
    """u_{n+1} from u_n = u and u_{n-1} = uprev (both [h][w], FP64)."""
    u = np.asarray(u, dtype=np.float64)
    uprev = np.asarray(uprev, dtype=np.float64)
    return 2.0 * u - uprev + dt * dt * laplacian(u, r, dx, dy)


def run(u1: np.ndarray, u0: np.ndarray, nsteps: int, r: int, dt: float, dx: float, dy: float):
    """nsteps leapfrog steps from (u_n, u_{n-1}) = (u1, u0); returns (u_{n+nsteps}, u_{n+nsteps-1})."""
    cur, prev = np.asarray(u1, dtype=np.float64), np.asarray(u0, dtype=np.float64)
    for _ in range(nsteps):
        cur, prev = step(cur, prev, r, dt, dx, dy), cur
    return cur, prev


def step_at(u: np.ndarray, uprev: np.ndarray, r: int, dt: float, dx: float, dy: float, nodes):
    """u_{n+1} at a few nodes (i, j) = (x index, y index) only, for full-size sampled checks."""
    h, w = u.shape
    c = weights(r)
    out = []
    for (i, j) in nodes:
        lap = 0.0
        for k in range(-r, r + 1):
            lap += c[k + r] * u[j, (i + k) % w] / (dx * dx)
            lap += c[k + r] * u[(j + k) % h, i] / (dy * dy)
        out.append(2.0 * u[j, i] - uprev[j, i] + dt * dt * lap)
    return np.array(out)
