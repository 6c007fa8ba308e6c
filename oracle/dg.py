"""FP64 reference of the discontinuous-Galerkin shallow-water volume kernel of arXiv 1403.0968
§4.3 (test infrastructure only: the tests, the smoke check and the benchmark's CPU-baseline leg
may use it; the product library never does, and this module imports nothing from the CUDA
package).

What it computes (§4.3, the conservative shallow-water system and the weak form's volume term):
on each affine triangle D^e with nodal (Lagrange) basis l_i of degree N, the volume term of the
semi-discrete weak form, with the element mass matrix applied inverted as nodal DG does,

    rhs_i = (M^e)^-1 [ <F, dl_i/dx> + <G, dl_i/dy> ] + S_i
          = sum_j Drw_ij (rx F_j + ry G_j) + Dsw_ij (sx F_j + sy G_j) + S_i,

for the fields Q = (h, hu, hv), fluxes F = (hu, hu^2/h + g h^2/2, hu hv/h), G = (hv, hu hv/h,
hv^2/h + g h^2/2) and source S = (0, -g h B_x, -g h B_y), with F, G, S interpolated at the nodes.
On the reference triangle T = {r, s >= -1, r + s <= 0}: Mhat_ij = int_T l_i l_j,
(Shat_r)_ij = int_T l_i dl_j/dr, Drw = Mhat^-1 Shat_r^T (and s alike); the element map
x = -(r+s)/2 v1 + (1+r)/2 v2 + (1+s)/2 v3 gives rx, ry, sx, sy and J (M^e = J Mhat).

Nodes (the paper does not fix them): the equispaced nodes r = -1 + 2i/N, s = -1 + 2j/N,
i + j <= N, numbered with i fastest.  The reference matrices are computed exactly in rational
arithmetic: Lagrange coefficients from the monomial Vandermonde matrix, monomial integrals over T
in closed form, Gauss-Jordan elimination over fractions.

Parity status (pins in tests/test_dg_oracle_pins.py): monomial integrals against numerical
cubature; Mhat and Shat against symbolic integration of polynomial pairs (sympy); the
integration-by-parts identity Shat_r + Shat_r^T = edge integral of l_i l_j n_r; the geometric
factors against the vertex map; the whole volume term against symbolic integration on a physical
triangle for fluxes of degree <= N.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import comb, factorial

import numpy as np


def nodes(N: int):
    """Equispaced nodes (r, s) of the reference triangle as Fractions, i fastest."""
    return [(Fraction(-1) + Fraction(2 * i, N), Fraction(-1) + Fraction(2 * j, N))
            for j in range(N + 1) for i in range(N + 1 - j)]


def monomials(N: int):
    """Exponents (a, b) of r^a s^b, total degree <= N."""
    return [(a, d - a) for d in range(N + 1) for a in range(d, -1, -1)]


def tri_integral(a: int, b: int) -> Fraction:
    """int_T r^a s^b dr ds over T = {r, s >= -1, r + s <= 0}, exact.

    With r = 2x - 1, s = 2y - 1 the triangle becomes {x, y >= 0, x + y <= 1}, dr ds = 4 dx dy, and
    int x^p y^q = p! q! / (p + q + 2)!."""
    tot = Fraction(0)
    for p in range(a + 1):
        for q in range(b + 1):
            c = comb(a, p) * comb(b, q) * (2 ** p) * (2 ** q) * (-1) ** (a - p + b - q)
            tot += Fraction(c * factorial(p) * factorial(q), factorial(p + q + 2))
    return 4 * tot


def _inverse(A):
    """Gauss-Jordan inverse over Fractions."""
    n = len(A)
    M = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(i for i in range(col, n) if M[i][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        p = M[col][col]
        M[col] = [v / p for v in M[col]]
        for i in range(n):
            if i != col and M[i][col] != 0:
                f = M[i][col]
                M[i] = [v - f * w for v, w in zip(M[i], M[col])]
    return [row[n:] for row in M]


def _matmul(A, B):
    Bt = list(zip(*B))
    return [[sum((x * y for x, y in zip(row, col)), Fraction(0)) for col in Bt] for row in A]


def _transpose(A):
    return [list(r) for r in zip(*A)]


@lru_cache(maxsize=None)
def operators_exact(N: int):
    """(Mhat, Shat_r, Shat_s, Drw, Dsw) as lists of Fractions, Np x Np."""
    nd, mono = nodes(N), monomials(N)
    Np = len(nd)
    V = [[r ** a * s ** b for (a, b) in mono] for (r, s) in nd]  # V[i][p] = m_p(node_i)
    C = _inverse(V)  # l_i = sum_p C[p][i] m_p
    # monomial Gram and derivative integrals
    Mm = [[tri_integral(a1 + a2, b1 + b2) for (a2, b2) in mono] for (a1, b1) in mono]
    Smr = [[(a2 * tri_integral(a1 + a2 - 1, b1 + b2) if a2 > 0 else Fraction(0)) for (a2, b2) in mono]
           for (a1, b1) in mono]
    Sms = [[(b2 * tri_integral(a1 + a2, b1 + b2 - 1) if b2 > 0 else Fraction(0)) for (a2, b2) in mono]
           for (a1, b1) in mono]
    Ct = _transpose(C)
    Mhat = _matmul(Ct, _matmul(Mm, C))
    Sr = _matmul(Ct, _matmul(Smr, C))
    Ss = _matmul(Ct, _matmul(Sms, C))
    Minv = _inverse(Mhat)
    Drw = _matmul(Minv, _transpose(Sr))
    Dsw = _matmul(Minv, _transpose(Ss))
    assert all(len(r) == Np for r in Drw)
    return Mhat, Sr, Ss, Drw, Dsw


def operators(N: int):
    """The same matrices as FP64 arrays: dict with Mhat, Sr, Ss, Drw, Dsw."""
    names = ("Mhat", "Sr", "Ss", "Drw", "Dsw")
    return {k: np.array([[float(x) for x in row] for row in m]) for k, m in zip(names, operators_exact(N))}


def geometry(verts: np.ndarray):
    """rx, ry, sx, sy, J per triangle from vertices [E][3][2] (affine map, counter-clockwise)."""
    v = np.asarray(verts, dtype=np.float64)
    xr = 0.5 * (v[:, 1, 0] - v[:, 0, 0])
    xs = 0.5 * (v[:, 2, 0] - v[:, 0, 0])
    yr = 0.5 * (v[:, 1, 1] - v[:, 0, 1])
    ys = 0.5 * (v[:, 2, 1] - v[:, 0, 1])
    J = xr * ys - xs * yr
    return ys / J, -xs / J, -yr / J, xr / J, J


def fluxes(Q: np.ndarray, g: float):
    """F, G ([E][3][Np]) of the conservative shallow-water system from Q = (h, hu, hv)."""
    h, hu, hv = Q[:, 0], Q[:, 1], Q[:, 2]
    F = np.stack([hu, hu * hu / h + 0.5 * g * h * h, hu * hv / h], axis=1)
    G = np.stack([hv, hu * hv / h, hv * hv / h + 0.5 * g * h * h], axis=1)
    return F, G


def volume(N: int, Q: np.ndarray, Bxy: np.ndarray, geo, g: float) -> np.ndarray:
    """The volume right-hand side [E][3][Np] for nodal fields Q [E][3][Np], bathymetry gradients
    Bxy [E][2][Np] and geo = (rx, ry, sx, sy) per element, in FP64."""
    ops = operators(N)
    Drw, Dsw = ops["Drw"], ops["Dsw"]
    rx, ry, sx, sy = (np.asarray(a, dtype=np.float64)[:, None, None] for a in geo[:4])
    F, G = fluxes(np.asarray(Q, dtype=np.float64), g)
    Xr = rx * F + ry * G
    Xs = sx * F + sy * G
    out = np.einsum("ij,efj->efi", Drw, Xr) + np.einsum("ij,efj->efi", Dsw, Xs)
    h = Q[:, 0]
    out[:, 1] += -g * h * Bxy[:, 0]
    out[:, 2] += -g * h * Bxy[:, 1]
    return out
