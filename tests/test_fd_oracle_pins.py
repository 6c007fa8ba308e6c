"""Pins of the finite-difference wave oracle (oracle/fd.py, arXiv 1403.0968 §4.1) against facts
fixed by mathematics, not by the oracle itself: published stencil tables, polynomial exactness,
order of accuracy, the closed-form leapfrog recurrence of a grid-periodic Fourier mode (the
periodic boundary of the §4.1 kernel listing), commutation with cyclic shifts, an exact polynomial
solution of the wave equation and leapfrog's time symmetry.  CPU only."""
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import fd

# central second-derivative weights c_0..c_r of order 2r (Fornberg's tables)
PUBLISHED = {
    1: [F(-2), F(1)],
    2: [F(-5, 2), F(4, 3), F(-1, 12)],
    3: [F(-49, 18), F(3, 2), F(-3, 20), F(1, 90)],
    4: [F(-205, 72), F(8, 5), F(-1, 5), F(8, 315), F(-1, 560)],
}


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_weights_match_published_tables(r):
    c = fd.weights_exact(r)
    assert len(c) == 2 * r + 1
    for k in range(r + 1):
        assert c[r + k] == PUBLISHED[r][k] and c[r - k] == PUBLISHED[r][k]


@pytest.mark.parametrize("r", range(1, 8))
def test_weights_exact_on_shifted_monomials(r):
    # sum_k c_k f(x0 + k) = f''(x0) for f = x^m, m <= 2r + 1 (symmetry adds one degree), exactly;
    # degree 2r + 2 is not reproduced
    c = fd.weights_exact(r)
    x0 = F(3, 7)
    for m in range(0, 2 * r + 3):
        lhs = sum(ck * (x0 + k) ** m for ck, k in zip(c, range(-r, r + 1)))
        rhs = m * (m - 1) * x0 ** (m - 2) if m >= 2 else F(0)
        if m <= 2 * r + 1:
            assert lhs == rhs, (r, m)
        else:
            assert lhs != rhs, (r, m)
    assert sum(c) == 0


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_order_of_accuracy(r):
    # error of the stencil on sin at a point scales as h^(2r)
    c = fd.weights(r)

    def err(h):
        x0 = 0.3
        approx = sum(ck * np.sin(x0 + k * h) for ck, k in zip(c, range(-r, r + 1))) / (h * h)
        return abs(approx + np.sin(x0))

    h = 0.4
    ratio = err(h) / err(h / 2)
    assert abs(np.log2(ratio) - 2 * r) < 0.3, (r, ratio)


def _exact(x, y, t):
    # u_tt = u_xx + u_yy: x^3 + 3 x t^2 (6x = 6x), t^3 + 3 t x^2 (6t = 6t), y^2 + t^2 (2 = 2)
    return x ** 3 + 3 * x * t ** 2 + t ** 3 + 3 * t * x ** 2 + y ** 2 + t ** 2


@pytest.mark.parametrize("r", [1, 2, 3, 5, 7])
def test_step_reproduces_polynomial_solution(r):
    # the solution is cubic in x and t, quadratic in y: the stencils (exact to degree 2r+1) and
    # leapfrog (exact to degree 3 in t) reproduce it except within r nodes of the wrap seam (the
    # polynomial is not periodic); dx != dy, so exchanging the directions fails
    w, h = 40, 33
    dx, dy, dt = 0.05, 0.07, 0.02
    X = -1.0 + dx * np.arange(w)[None, :] + 0.0 * np.arange(h)[:, None]
    Y = -1.0 + dy * np.arange(h)[:, None] + 0.0 * np.arange(w)[None, :]
    t1 = 0.3
    u1, u0 = _exact(X, Y, t1), _exact(X, Y, t1 - dt)
    u2 = fd.step(u1, u0, r, dt, dx, dy)
    ref = _exact(X, Y, t1 + dt)
    inner = (slice(r, h - r), slice(r, w - r))
    assert np.max(np.abs(u2[inner] - ref[inner])) < 1e-11 * np.max(np.abs(ref))
    # near the seam the wrapped neighbours make a visible difference
    assert np.max(np.abs(u2 - ref)) > 1e-3


def test_leapfrog_is_time_reversible():
    g = np.random.default_rng(3)
    u, up = g.uniform(-1, 1, (20, 25)), g.uniform(-1, 1, (20, 25))
    un = fd.step(u, up, 3, 0.01, 0.03, 0.04)
    back = fd.step(u, un, 3, 0.01, 0.03, 0.04)
    assert np.max(np.abs(back - up)) < 1e-13


def test_sampled_nodes_match_full_step():
    g = np.random.default_rng(4)
    u, up = g.uniform(-1, 1, (17, 23)), g.uniform(-1, 1, (17, 23))
    full = fd.step(u, up, 4, 0.01, 0.05, 0.06)
    nodes = [(0, 0), (22, 16), (3, 9), (21, 1), (11, 8)]
    np.testing.assert_allclose(fd.step_at(u, up, 4, 0.01, 0.05, 0.06, nodes),
                               [full[j, i] for (i, j) in nodes], rtol=1e-14, atol=1e-14)


def _fornberg(r):
    # closed form of the central second-derivative weights of order 2r (Fornberg, Math. Comp. 51,
    # 1988): c_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!), c_0 = -2 sum_{k>=1} c_k
    from math import factorial
    ck = [F(0)] + [F(2 * (-1) ** (k + 1) * factorial(r) ** 2, k * k * factorial(r - k) * factorial(r + k))
                   for k in range(1, r + 1)]
    ck[0] = -2 * sum(ck[1:])
    return ck


@pytest.mark.parametrize("r", range(1, 8))
def test_closed_form_weights(r):
    # the oracle's Gauss-Jordan moment solve against Fornberg's closed form (and the tables, r <= 4)
    ck = _fornberg(r)
    if r in PUBLISHED:
        assert ck == PUBLISHED[r]
    c = fd.weights_exact(r)
    assert [c[r + k] for k in range(r + 1)] == ck


def _symbol(r, theta):
    # Fourier symbol of the stencil: sum_k c_k e^{i k theta} = c_0 + 2 sum_{k>=1} c_k cos(k theta)
    ck = [float(v) for v in _fornberg(r)]
    return ck[0] + 2.0 * sum(ck[k] * np.cos(k * theta) for k in range(1, r + 1))


@pytest.mark.parametrize("r,h,w,m,q", [(1, 16, 24, 1, 2), (2, 33, 20, 3, 1), (4, 40, 29, 5, 7),
                                       (7, 21, 50, 2, 4), (7, 3, 5, 1, 1), (5, 1, 9, 2, 0)])
def test_periodic_fourier_mode_recurrence(r, h, w, m, q):
    # A grid-periodic mode f(i, j) = cos(2 pi (m i / w + q j / h) + phi) is an eigenvector of both
    # periodic stencils, with eigenvalues symbol(2 pi m / w) / dx^2 and symbol(2 pi q / h) / dy^2.
    # Leapfrog then maps (A1 f, A0 f) to A2 f with A2 = (2 + dt^2 (lx + ly)) A1 - A0 at EVERY node,
    # the wrapped edges included: a zero ghost layer, a missing wrap in one direction, exchanged
    # spacings or a dropped y term each break it.  Grids narrower than the stencil (w = 5, h = 3 at
    # r = 7) wrap more than once.
    dx, dy, dt = 0.05, 0.07, 0.01
    i = np.arange(w)[None, :]
    j = np.arange(h)[:, None]
    f = np.cos(2 * np.pi * (m * i / w + q * j / h) + 0.4)
    a1, a0 = 1.3, 0.9
    lx = _symbol(r, 2 * np.pi * m / w) / dx ** 2
    ly = _symbol(r, 2 * np.pi * q / h) / dy ** 2
    a2 = (2.0 + dt * dt * (lx + ly)) * a1 - a0
    got = fd.step(a1 * f, a0 * f, r, dt, dx, dy)
    assert np.max(np.abs(got - a2 * f)) < 1e-12 * max(abs(a2), 1.0)
    # the sampled-node form agrees at the corners and edges
    nodes = [(0, 0), (w - 1, h - 1), (0, h - 1), (w - 1, 0), (w // 2, 0)]
    np.testing.assert_allclose(fd.step_at(a1 * f, a0 * f, r, dt, dx, dy, nodes), [a2 * f[jj, ii] for ii, jj in nodes],
                               rtol=0, atol=1e-12 * max(abs(a2), 1.0))


def test_step_commutes_with_cyclic_shifts():
    # periodic boundaries make the step translation invariant on the torus
    g = np.random.default_rng(5)
    u, up = g.uniform(-1, 1, (19, 26)), g.uniform(-1, 1, (19, 26))
    base = fd.step(u, up, 5, 0.01, 0.03, 0.04)
    for sh in [(3, 0), (0, 7), (-4, 11)]:
        got = fd.step(np.roll(u, sh, axis=(0, 1)), np.roll(up, sh, axis=(0, 1)), 5, 0.01, 0.03, 0.04)
        np.testing.assert_allclose(got, np.roll(base, sh, axis=(0, 1)), rtol=0, atol=1e-13)
