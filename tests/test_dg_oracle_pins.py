"""Pins of the DG shallow-water volume oracle (oracle/dg.py, arXiv 1403.0968 §4.3) against facts
fixed by mathematics: numerical cubature, symbolic integration of polynomials (sympy), the
integration-by-parts identity of the reference stiffness matrices, and the affine vertex map.
CPU only."""
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import dg


@pytest.mark.parametrize("a,b", [(0, 0), (1, 0), (0, 1), (2, 3), (4, 1), (3, 3)])
def test_monomial_integrals_against_cubature(a, b):
    integrate = pytest.importorskip("scipy.integrate")
    val, _ = integrate.dblquad(lambda s, r: r ** a * s ** b, -1, 1, lambda r: -1, lambda r: -r, epsabs=1e-13)
    assert abs(float(dg.tri_integral(a, b)) - val) < 1e-12


def _poly_values(sp, expr, N):
    r, s = sp.symbols("r s")
    return [F(str(sp.nsimplify(expr.subs({r: sp.Rational(nr.numerator, nr.denominator),
                                           s: sp.Rational(ns.numerator, ns.denominator)}))))
            for (nr, ns) in dg.nodes(N)]


def _tri(sp, expr):
    r, s = sp.symbols("r s")
    return F(str(sp.integrate(sp.integrate(expr, (s, -1, -r)), (r, -1, 1))))


@pytest.mark.parametrize("N", [1, 2, 3])
def test_mass_and_stiffness_against_symbolic_integrals(N):
    # f^T Mhat g = int f g and f^T Shat_r g = int f dg/dr for polynomials of degree <= N, exactly
    sp = pytest.importorskip("sympy")
    r, s = sp.symbols("r s")
    f = sum(sp.Integer((3 * a + 5 * b) % 7 - 3) * r ** a * s ** b for (a, b) in dg.monomials(N))
    g = sum(sp.Integer((2 * a + 3 * b + 1) % 5 - 2) * r ** a * s ** b for (a, b) in dg.monomials(N))
    fv, gv = _poly_values(sp, f, N), _poly_values(sp, g, N)
    Mhat, Sr, Ss, Drw, Dsw = dg.operators_exact(N)

    def quad(A):
        return sum(fv[i] * A[i][j] * gv[j] for i in range(len(fv)) for j in range(len(gv)))

    assert quad(Mhat) == _tri(sp, f * g)
    assert quad(Sr) == _tri(sp, f * sp.diff(g, r))
    assert quad(Ss) == _tri(sp, f * sp.diff(g, s))


@pytest.mark.parametrize("N", [2, 4])
def test_stiffness_integration_by_parts(N):
    # Shat_r + Shat_r^T is the edge integral of l_i l_j n_r: the hypotenuse r + s = 0 (n_r = 1/sqrt2,
    # length 2 sqrt2) and the edge r = -1 (n_r = -1); the edge s = -1 has n_r = 0
    sp = pytest.importorskip("sympy")
    r, s, t = sp.symbols("r s t")
    f = 1 + 2 * r - s + r * s
    g = 3 - r + 2 * s * s if N >= 2 else 3 - r
    fv, gv = _poly_values(sp, f, N), _poly_values(sp, g, N)
    Mhat, Sr, Ss, Drw, Dsw = dg.operators_exact(N)
    lhs = sum(fv[i] * (Sr[i][j] + Sr[j][i]) * gv[j] for i in range(len(fv)) for j in range(len(gv)))
    fg = f * g
    rhs = sp.integrate(fg.subs({r: t, s: -t}), (t, -1, 1)) - sp.integrate(fg.subs(r, -1), (s, -1, 1))
    assert lhs == F(str(rhs))


def test_weak_derivative_matrices_definition():
    Mhat, Sr, Ss, Drw, Dsw = (np.array([[float(x) for x in row] for row in m]) for m in dg.operators_exact(3))
    np.testing.assert_allclose(Mhat @ Drw, Sr.T, atol=1e-14)
    np.testing.assert_allclose(Mhat @ Dsw, Ss.T, atol=1e-14)
    assert abs(Mhat.sum() - 2.0) < 1e-14  # area of the reference triangle


def test_geometry_of_affine_triangles():
    v = np.array([[[0.1, 0.2], [1.3, 0.4], [0.5, 1.6]], [[2.0, 1.0], [2.5, 3.0], [-1.0, 2.0]]])
    rx, ry, sx, sy, J = dg.geometry(v)
    for e in range(2):
        (x1, y1), (x2, y2), (x3, y3) = v[e]
        area = 0.5 * ((x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1))
        assert abs(2 * J[e] - area) < 1e-14  # reference area 2
        dxdr = np.array([[x2 - x1, x3 - x1], [y2 - y1, y3 - y1]]) / 2
        np.testing.assert_allclose(np.array([[rx[e], ry[e]], [sx[e], sy[e]]]) @ dxdr, np.eye(2), atol=1e-14)


def test_volume_term_against_symbolic_weak_form():
    # one physical triangle, N = 3, h = 1 and linear momenta: F and G are quadratic, so the nodal
    # interpolation is exact and J Mhat (rhs - S) must equal <F, dl_i/dx> + <G, dl_i/dy> exactly
    sp = pytest.importorskip("sympy")
    N, g = 3, 9.81
    x, y, r, s = sp.symbols("x y r s")
    V = [(sp.Rational(1, 10), sp.Rational(1, 5)), (sp.Rational(13, 10), sp.Rational(2, 5)),
         (sp.Rational(1, 2), sp.Rational(8, 5))]
    X = -(r + s) / 2 * V[0][0] + (1 + r) / 2 * V[1][0] + (1 + s) / 2 * V[2][0]
    Y = -(r + s) / 2 * V[0][1] + (1 + r) / 2 * V[1][1] + (1 + s) / 2 * V[2][1]
    hu = sp.Rational(1, 3) + x - 2 * y
    hv = sp.Rational(-1, 2) + 2 * x + y
    Fx = [hu, hu * hu + sp.Rational(981, 200), hu * hv]
    Gy = [hv, hu * hv, hv * hv + sp.Rational(981, 200)]
    verts = np.array([[[float(a), float(b)] for (a, b) in V]])
    rx, ry, sx, sy, J = dg.geometry(verts)
    nd = dg.nodes(N)
    xy = [(X.subs({r: sp.Rational(a.numerator, a.denominator), s: sp.Rational(b.numerator, b.denominator)}),
           Y.subs({r: sp.Rational(a.numerator, a.denominator), s: sp.Rational(b.numerator, b.denominator)}))
          for (a, b) in nd]
    Q = np.zeros((1, 3, len(nd)))
    Q[0, 0] = 1.0
    Q[0, 1] = [float(hu.subs({x: px, y: py})) for (px, py) in xy]
    Q[0, 2] = [float(hv.subs({x: px, y: py})) for (px, py) in xy]
    out = dg.volume(N, Q, np.zeros((1, 2, len(nd))), (rx, ry, sx, sy), g)
    Mhat = dg.operators(N)["Mhat"]
    got = J[0] * (out[0] @ Mhat.T)  # J Mhat rhs, per field
    # exact: int_T (F dl/dx + G dl/dy) J dr ds with dl/dx = rx dl/dr + sx dl/ds (rx.. exact rationals)
    Jx = sp.Matrix([[sp.diff(X, r), sp.diff(X, s)], [sp.diff(Y, r), sp.diff(Y, s)]])
    Jd = Jx.det()
    inv = Jx.inv()  # [[rx, ry], [sx, sy]]
    mono = dg.monomials(N)
    Vm = sp.Matrix([[sp.Rational(a.numerator, a.denominator) ** p * sp.Rational(b.numerator, b.denominator) ** q
                     for (p, q) in mono] for (a, b) in nd])
    C = Vm.inv()
    for i in range(len(nd)):
        li = sum(C[k, i] * r ** p * s ** q for k, (p, q) in enumerate(mono))
        dlx = inv[0, 0] * sp.diff(li, r) + inv[1, 0] * sp.diff(li, s)
        dly = inv[0, 1] * sp.diff(li, r) + inv[1, 1] * sp.diff(li, s)
        for f in range(3):
            integrand = (Fx[f].subs({x: X, y: Y}) * dlx + Gy[f].subs({x: X, y: Y}) * dly) * Jd
            exact = float(sp.integrate(sp.integrate(sp.expand(integrand), (s, -1, -r)), (r, -1, 1)))
            assert abs(got[f, i] - exact) < 1e-11 * max(1.0, abs(exact)), (i, f, got[f, i], exact)


def test_triangle_mesh_generator():
    # the stand-in DG mesh: 2 nx ny counter-clockwise triangles covering the unit square exactly
    import workloads as W

    v = W.tri_mesh(7, 5, perturb=0.2, seed=3)
    assert v.shape == (70, 3, 2)
    rx, ry, sx, sy, J = dg.geometry(v)
    assert np.all(J > 0)
    assert abs(2.0 * J.sum() - 1.0) < 1e-14
    assert W.tri_mesh(280, 380).shape[0] == 212800
