"""Pins of the finite-difference wave oracle (oracle/fd.py, arXiv 1403.0968 §4.1) against facts
fixed by mathematics, not by the oracle itself: published stencil tables, polynomial exactness,
order of accuracy, an exact polynomial solution of the wave equation and leapfrog's time
symmetry.  CPU only."""
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
    # leapfrog (exact to degree 3 in t) reproduce it except within r nodes of the ghost layer;
    # dx != dy, so exchanging the directions fails
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
    # near the boundary the zero ghost nodes make a visible difference
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
