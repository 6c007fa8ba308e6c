"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix (no GPU).

Each test pins one oracle function to something other than itself: closed-form GLL tables, exact
quadrature, exactness of D on polynomials, the Legendre form of D, u^T A u against the exact
integral of |grad u|^2 (§4.2.1, Eq. 2), A 1 = 0, symmetry, positive (semi)definiteness, dense
brute-force element matrices, direct dense solves and manufactured-solution convergence.
"""
import itertools
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------
# 1-D: GLL nodes, weights, derivative matrix
# ------------------------------------------------------------------------------------------
def _golden_gll():
    rows = {}
    for line in open(os.path.join(GOLDEN, "gll_closed_forms.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        left, right = line.split("|")
        parts = left.split()
        rows[int(parts[0])] = (np.array([float(v) for v in parts[1:]]), np.array([float(v) for v in right.split()]))
    return rows


def test_gll_closed_forms(orc):
    for N, (xg, wg) in _golden_gll().items():
        x, w = orc.gll(N)
        np.testing.assert_allclose(x, xg, atol=1e-15)
        np.testing.assert_allclose(w, wg, atol=1e-15)


@pytest.mark.parametrize("N", list(range(1, 16)))
def test_gll_quadrature_exact_to_2N_minus_1(orc, N):
    x, w = orc.gll(N)
    assert x[0] == -1.0 and x[-1] == 1.0 and np.all(np.diff(x) > 0)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14, (N, k)
    # degree 2N is not integrated exactly (Lobatto rule has degree 2N-1)
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-10


@pytest.mark.parametrize("N", list(range(1, 16)))
def test_D_exact_on_polynomials_and_corners(orc, N):
    x, _ = orc.gll(N)
    D = orc.lagrange_deriv(N, x)
    for k in range(N + 1):
        d = D @ (x ** k)
        exact = k * x ** (k - 1) if k else np.zeros_like(x)
        assert np.max(np.abs(d - exact)) < 1e-12 * max(1.0, N * N * k), (N, k)
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-12 * N * N
    assert abs(D[N, N] - N * (N + 1) / 4.0) < 1e-12 * N * N
    for i in range(1, N):
        assert abs(D[i, i]) < 1e-12 * N * N


@pytest.mark.parametrize("N", [2, 3, 5, 7, 9, 11, 15])
def test_D_matches_legendre_form(orc, N):
    # off-diagonal D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) (Legendre form of the GLL derivative
    # matrix); P_N from numpy's Legendre series evaluation, independent of the oracle.
    x, _ = orc.gll(N)
    D = orc.lagrange_deriv(N, x)
    c = np.zeros(N + 1)
    c[N] = 1.0
    P = np.polynomial.legendre.legval(x, c)
    for i in range(N + 1):
        for j in range(N + 1):
            if i != j:
                assert abs(D[i, j] - P[i] / (P[j] * (x[i] - x[j]))) < 1e-12 * N * N


def test_gll_weights_match_legendre_form(orc):
    for N in range(1, 16):
        x, w = orc.gll(N)
        c = np.zeros(N + 1)
        c[N] = 1.0
        P = np.polynomial.legendre.legval(x, c)
        np.testing.assert_allclose(w, 2.0 / (N * (N + 1) * P ** 2), rtol=1e-13)
        # interior nodes are roots of P_N'
        if N > 1:
            dP = np.polynomial.legendre.legval(x[1:-1], np.polynomial.legendre.legder(c))
            assert np.max(np.abs(dP)) < 1e-11 * N ** 3


def test_kappa_special_cases(orc):
    assert orc.kappa(None, np.array([[0.3, 0.2, 0.1]]))[0] == 1.0
    modes = np.array([[1.0, 0.0, 0.0, 0.0, math.log(2.0)]])
    np.testing.assert_allclose(orc.kappa(modes, np.array([[0.0, 0.7, 0.1], [0.5, 0.0, 0.0], [0.25, 0.0, 0.0]])),
                               [2.0, 0.5, 1.0], rtol=1e-15)


# ------------------------------------------------------------------------------------------
# geometry
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 3, 7])
def test_lumped_mass_sums_to_volume(orc, N):
    # det J of a trilinear map has per-variable degree <= 2 <= 2N-1, so GLL integrates it exactly:
    # the lumped mass (§4.2.1) of the perturbed unit-cube mesh sums to its volume, 1.
    v = W.box_vertices(3, 2, 4, seed=11)
    _, wJ = orc.factors(N, v)
    assert abs(wJ.sum() - 1.0) < 1e-13


def test_affine_box_factors_closed_form(orc):
    N = 4
    hx, hy, hz = 0.5, 0.25, 2.0
    # vertex v = a + 2b + 4c at (a hx, b hy, c hz)
    v = np.array([[[(q & 1) * hx, ((q >> 1) & 1) * hy, ((q >> 2) & 1) * hz] for q in range(8)]])
    G, wJ = orc.factors(N, v)
    x, w = orc.gll(N)
    n = N + 1
    J = hx * hy * hz / 8.0
    for k, j, i in itertools.product(range(n), repeat=3):
        p = i + n * (j + n * k)
        ww = w[i] * w[j] * w[k] * J
        assert abs(wJ[0, p] - ww) < 1e-15
        np.testing.assert_allclose(G[0, :, p], [ww * (2 / hx) ** 2, 0, 0, ww * (2 / hy) ** 2, 0, ww * (2 / hz) ** 2],
                                   rtol=1e-14, atol=1e-15 * ww * (2 / hy) ** 2)


def test_box_numbering_matches_coordinate_brute_force(orc):
    # On an unperturbed mesh, two local nodes are the same global node iff they have the same
    # coordinates; the lexicographic (x fastest) order of the distinct points fixes the ids.
    for (sx, sy, sz, N) in [(1, 1, 1, 1), (2, 3, 2, 2), (3, 2, 2, 3), (2, 2, 2, 5)]:
        v = W.box_vertices(sx, sy, sz, perturb=0.0)
        xyz = orc.node_coords(N, v).reshape(-1, 3)
        key = np.round(xyz * (sx * sy * sz * N * 64), 0).astype(np.int64)
        uniq, inv = np.unique(key[:, [2, 1, 0]], axis=0, return_inverse=True)
        glo = orc.box_numbering(sx, sy, sz, N).reshape(-1)
        assert len(uniq) == orc.box_nglobal(sx, sy, sz, N)
        assert np.array_equal(glo, inv.reshape(-1))
        mask = orc.box_dirichlet(sx, sy, sz, N)
        on_bnd = np.zeros(len(uniq), dtype=np.uint8)
        pts = uniq[:, [2, 1, 0]] / (sx * sy * sz * N * 64)
        on_bnd[np.any((np.abs(pts) < 1e-12) | (np.abs(pts - 1.0) < 1e-12), axis=1)] = 1
        assert np.array_equal(mask, on_bnd)


# ------------------------------------------------------------------------------------------
# operator: energy identity, invariants, brute force
# ------------------------------------------------------------------------------------------
def _tensor_box_vertices(xs, ys, zs):
    """Axis-aligned, non-uniform tensor mesh (affine elements) from breakpoint lists."""
    verts = []
    for ez in range(len(zs) - 1):
        for ey in range(len(ys) - 1):
            for ex in range(len(xs) - 1):
                verts.append([[xs[ex + (q & 1)], ys[ey + ((q >> 1) & 1)], zs[ez + ((q >> 2) & 1)]] for q in range(8)])
    return np.array(verts, dtype=float)


def _poly_eval(coef, xyz):
    out = np.zeros(xyz.shape[:-1])
    for (a, b, c), cf in coef.items():
        out += cf * xyz[..., 0] ** a * xyz[..., 1] ** b * xyz[..., 2] ** c
    return out


def _grad_energy_exact(coef, lo, hi):
    """int over the box [lo,hi] of |grad u|^2 for u = sum c_abc x^a y^b z^c (exact antiderivatives)."""
    def mono_int(p, q, r):
        return ((hi[0] ** (p + 1) - lo[0] ** (p + 1)) / (p + 1) * (hi[1] ** (q + 1) - lo[1] ** (q + 1)) / (q + 1)
                * (hi[2] ** (r + 1) - lo[2] ** (r + 1)) / (r + 1))

    tot = 0.0
    items = list(coef.items())
    for d in range(3):
        for (m1, c1), (m2, c2) in itertools.product(items, items):
            if m1[d] == 0 or m2[d] == 0:
                continue
            e = [m1[0] + m2[0], m1[1] + m2[1], m1[2] + m2[2]]
            e[d] -= 2
            tot += c1 * c2 * m1[d] * m2[d] * mono_int(*e)
    return tot


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_energy_equals_exact_integral(orc, N):
    # For u of total degree <= N, every monomial of |grad u|^2 has per-variable degree <= 2N-2,
    # which GLL integrates exactly: u^T A u = int |grad u|^2 on any affine box mesh (§4.2.1, Eq. 2).
    g = W.rng(100 + N)
    coef = {}
    for a in range(N + 1):
        for b in range(N + 1 - a):
            for c in range(N + 1 - a - b):
                coef[(a, b, c)] = g.uniform(-1, 1)
    xs, ys, zs = [0.0, 0.3, 1.0], [0.0, 0.55, 0.8, 1.0], [0.0, 0.45, 1.0]
    v = _tensor_box_vertices(xs, ys, zs)
    G, _ = orc.factors(N, v)
    xyz = orc.node_coords(N, v)
    uL = _poly_eval(coef, xyz)
    yL = orc.apply_local(N, G, uL)
    energy = float(np.sum(uL * yL))
    exact = _grad_energy_exact(coef, (0, 0, 0), (1, 1, 1))
    assert abs(energy - exact) < 1e-12 * max(1.0, abs(exact))


@pytest.mark.parametrize("N", [2, 4])
def test_mass_term_energy(orc, N):
    # with constant alpha the lumped mass term adds alpha * int u^2, exact for per-variable degree <= N-1
    g = W.rng(7)
    coef = {(a, b, c): g.uniform(-1, 1) for a in range(N) for b in range(N) for c in range(N) if a + b + c <= N - 1}
    v = _tensor_box_vertices([0.0, 0.4, 1.0], [0.0, 1.0], [0.0, 0.7, 1.0])
    G, wJ = orc.factors(N, v)
    xyz = orc.node_coords(N, v)
    uL = _poly_eval(coef, xyz)
    alpha = 2.5
    y0 = orc.apply_local(N, G, uL)
    y1 = orc.apply_local(N, G, uL, wJalpha=alpha * wJ)
    # int u^2 on [0,1]^3 by a high-order tensor Gauss rule (numpy's leggauss), independent of GLL
    gx, gw = np.polynomial.legendre.leggauss(N + 2)
    gx = 0.5 * (gx + 1)
    gw = 0.5 * gw
    P = np.stack(np.meshgrid(gx, gx, gx, indexing="ij"), axis=-1)
    Wt = gw[:, None, None] * gw[None, :, None] * gw[None, None, :]
    exact = alpha * float(np.sum(Wt * _poly_eval(coef, P) ** 2))
    assert abs(float(np.sum(uL * (y1 - y0))) - exact) < 1e-13 * max(1.0, exact)


def _mesh(sx, sy, sz, N, seed=5, modes=None):
    orc = __import__("oracle")
    v = W.box_vertices(sx, sy, sz, seed=seed)
    G, wJ = orc.factors(N, v, modes=modes)
    glo = orc.box_numbering(sx, sy, sz, N)
    return v, G, wJ, glo


@pytest.mark.parametrize("N", [1, 3, 7])
def test_constant_in_nullspace(orc, N):
    v, G, wJ, glo = _mesh(3, 2, 2, N, modes=W.kappa_modes(4, seed=3))
    ng = orc.box_nglobal(3, 2, 2, N)
    y1 = orc.apply(N, glo, G, np.ones(ng))
    yr = orc.apply(N, glo, G, W.uniform(ng, seed=9))
    assert np.max(np.abs(y1)) < 1e-13 * np.max(np.abs(yr)) * N * N


def test_symmetry_with_kappa_alpha_mask(orc):
    N = 5
    v, G, wJ, glo = _mesh(2, 3, 2, N, modes=W.kappa_modes(16, seed=4))
    ng = orc.box_nglobal(2, 3, 2, N)
    mask = orc.box_dirichlet(2, 3, 2, N)
    wJa = 0.7 * wJ
    u, w = W.uniform(ng, seed=1), W.uniform(ng, seed=2)
    a = np.dot(w, orc.apply(N, glo, G, u, mask=mask, wJalpha=wJa))
    b = np.dot(u, orc.apply(N, glo, G, w, mask=mask, wJalpha=wJa))
    assert abs(a - b) < 1e-13 * max(abs(a), 1e-30)


def _dense_assembled_O1(orc, v, N, glo, ng, kappa_nodal=None, alpha=None):
    n3 = (N + 1) ** 3
    A = np.zeros((ng, ng))
    for e in range(v.shape[0]):
        Ae = orc.element_matrix(N, v[e], None if kappa_nodal is None else kappa_nodal[e],
                                None if alpha is None else alpha[e])
        idx = glo[e]
        A[np.ix_(idx, idx)] += Ae
    return A


@pytest.mark.parametrize("N,box", [(1, (2, 2, 2)), (3, (2, 2, 2)), (4, (2, 1, 1)), (7, (1, 1, 1))])
def test_sum_factorised_equals_dense_brute_force(orc, N, box):
    # O2 (sum factorisation + gather/scatter) against O1 (weak form by brute-force quadrature,
    # assembled densely) on 1-8 perturbed elements with variable kappa and alpha.
    sx, sy, sz = box
    modes = W.kappa_modes(16, seed=21)
    v = W.box_vertices(sx, sy, sz, seed=13, perturb=0.2)
    xyz = orc.node_coords(N, v)
    kap = orc.kappa(modes, xyz)
    G, wJ = orc.factors(N, v, kappa_nodal=kap)
    G2, _ = orc.factors(N, v, modes=modes)
    np.testing.assert_allclose(G, G2, rtol=1e-15, atol=0)
    glo = orc.box_numbering(sx, sy, sz, N)
    ng = orc.box_nglobal(sx, sy, sz, N)
    alpha = 0.3 + W.uniform(v.shape[0] * (N + 1) ** 3, seed=3, lo=0, hi=1).reshape(v.shape[0], -1)
    A = _dense_assembled_O1(orc, v, N, glo, ng, kappa_nodal=kap, alpha=alpha)
    cols = np.stack([orc.apply(N, glo, G, np.eye(ng)[q], wJalpha=alpha * wJ) for q in range(ng)], axis=1)
    assert np.max(np.abs(cols - A)) < 1e-12 * np.max(np.abs(A))
    assert np.max(np.abs(A - A.T)) < 1e-13 * np.max(np.abs(A))
    # diagonal (Jacobi) against the dense matrix
    d = orc.diag(N, glo, G, ng, wJalpha=alpha * wJ)
    np.testing.assert_allclose(d, np.diag(A), rtol=1e-12)


def test_psd_and_spd_after_mask(orc):
    N, box = 3, (2, 2, 1)
    v = W.box_vertices(*box, seed=17, perturb=0.2)
    glo = orc.box_numbering(*box, N)
    ng = orc.box_nglobal(*box, N)
    A = _dense_assembled_O1(orc, v, N, glo, ng)
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-12 * ev.max()
    assert abs(ev.min()) < 1e-12 * ev.max()  # exactly one zero mode (constants)
    assert ev[1] > 1e-6 * ev.max()
    mask = orc.box_dirichlet(*box, N).astype(bool)
    Ai = A[np.ix_(~mask, ~mask)]
    np.linalg.cholesky(Ai)  # raises if not SPD


def test_patch_test_affine(orc):
    # on an affine (unperturbed) mesh, A applied to a linear function vanishes at interior nodes
    N, box = 4, (3, 2, 2)
    v = W.box_vertices(*box, perturb=0.0)
    G, _ = orc.factors(N, v)
    glo = orc.box_numbering(*box, N)
    ng = orc.box_nglobal(*box, N)
    xyz = np.zeros((ng, 3))
    xyz[glo.reshape(-1)] = orc.node_coords(N, v).reshape(-1, 3)
    u = 0.3 + 1.2 * xyz[:, 0] - 0.7 * xyz[:, 1] + 2.0 * xyz[:, 2]
    y = orc.apply(N, glo, G, u)
    interior = orc.box_dirichlet(*box, N) == 0
    ref = np.max(np.abs(orc.apply(N, glo, G, W.uniform(ng, seed=1))))
    assert np.max(np.abs(y[interior])) < 1e-13 * ref


# general affine meshes: a dense, non-symmetric map x = M y + c of a tensor box mesh, so that
# J^-1 is a full matrix at every node and its off-diagonal terms (and its orientation: J^-1 J^-T
# against J^-T J^-1) enter the factors
_M_AFFINE = np.array([[1.0, 0.35, -0.2], [0.15, 0.9, 0.4], [-0.3, 0.1, 1.1]])
_C_AFFINE = np.array([0.2, -0.1, 0.3])


def _affine_mesh():
    xs, ys, zs = [0.0, 0.35, 1.0], [0.0, 0.6, 1.0], [0.0, 0.5, 0.75, 1.0]
    vy = _tensor_box_vertices(xs, ys, zs)
    return vy @ _M_AFFINE.T + _C_AFFINE, (xs, ys, zs)


def _poly_grad(coef, xyz):
    """Analytic gradient of u = sum c_abc x^a y^b z^c at points xyz [..., 3]."""
    g = np.zeros(xyz.shape)
    for (a, b, c), cf in coef.items():
        x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
        if a:
            g[..., 0] += cf * a * x ** (a - 1) * y ** b * z ** c
        if b:
            g[..., 1] += cf * b * x ** a * y ** (b - 1) * z ** c
        if c:
            g[..., 2] += cf * c * x ** a * y ** b * z ** (c - 1)
    return g


def test_affine_factors_closed_form(orc):
    # on an element that is the image of an axis-aligned box under x = M y + c, dx/dr = M diag(h/2)
    # is constant, so G = w_i w_j w_k det J J^-1 J^-T with numpy's inverse of that constant matrix
    N = 3
    v, (xs, ys, zs) = _affine_mesh()
    G, wJ = orc.factors(N, v)
    xg, wg = orc.gll(N)
    w3 = (wg[:, None, None] * wg[None, :, None] * wg[None, None, :]).reshape(-1)  # index k, j, i -> p
    e = 0
    for ez in range(len(zs) - 1):
        for ey in range(len(ys) - 1):
            for ex in range(len(xs) - 1):
                h = np.array([xs[ex + 1] - xs[ex], ys[ey + 1] - ys[ey], zs[ez + 1] - zs[ez]])
                J = _M_AFFINE @ np.diag(h / 2)
                Ji = np.linalg.inv(J)
                Gh = Ji @ Ji.T  # sum_d (dr_k/dx_d)(dr_l/dx_d)
                dj = np.linalg.det(J)
                ref = np.array([Gh[0, 0], Gh[0, 1], Gh[0, 2], Gh[1, 1], Gh[1, 2], Gh[2, 2]])
                got = G[e].reshape(6, -1)
                np.testing.assert_allclose(got, (w3 * dj)[None, :] * ref[:, None], rtol=1e-13, atol=1e-15)
                np.testing.assert_allclose(wJ[e], w3 * dj, rtol=1e-14)
                e += 1
    assert abs(Gh[0, 1]) > 0.05 and abs(Gh[1, 2]) > 0.05  # the off-diagonal terms are exercised


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_energy_exact_on_general_affine_mesh(orc, N):
    # u of total degree <= N in x stays of total degree <= N in the reference coordinates of an
    # affine element and |grad u|^2 of degree <= 2N-2, integrated exactly by GLL: u^T A u equals
    # int_Omega |grad u|^2 (§4.2.1, Eq. 2, the chain rule display and G-hat = G^T G).  The exact
    # integral is |det M| times numpy's Gauss-Legendre rule on [0,1]^3 of |grad u(M y + c)|^2.
    g = W.rng(300 + N)
    coef = {}
    for a in range(N + 1):
        for b in range(N + 1 - a):
            for c in range(N + 1 - a - b):
                coef[(a, b, c)] = g.uniform(-1, 1)
    v, _ = _affine_mesh()
    G, _ = orc.factors(N, v)
    xyz = orc.node_coords(N, v)
    uL = _poly_eval(coef, xyz)
    energy = float(np.sum(uL * orc.apply_local(N, G, uL)))
    gx, gw = np.polynomial.legendre.leggauss(N + 2)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    Y = np.stack(np.meshgrid(gx, gx, gx, indexing="ij"), axis=-1)
    Wt = gw[:, None, None] * gw[None, :, None] * gw[None, None, :]
    X = Y @ _M_AFFINE.T + _C_AFFINE
    exact = abs(np.linalg.det(_M_AFFINE)) * float(np.sum(Wt * np.sum(_poly_grad(coef, X) ** 2, axis=-1)))
    assert abs(energy - exact) < 1e-12 * max(1.0, abs(exact))
    # the dense brute-force element matrices (O1) give the same energy
    e1 = sum(float(uL[e] @ orc.element_matrix(N, v[e]) @ uL[e]) for e in range(v.shape[0]))
    assert abs(e1 - exact) < 1e-12 * max(1.0, abs(exact))


def test_patch_test_general_affine(orc):
    # A applied to a linear function vanishes at the interior nodes of a general affine mesh
    N = 4
    v, (xs, ys, zs) = _affine_mesh()
    box = (len(xs) - 1, len(ys) - 1, len(zs) - 1)
    G, _ = orc.factors(N, v)
    glo = orc.box_numbering(*box, N)
    ng = orc.box_nglobal(*box, N)
    xyz = np.zeros((ng, 3))
    xyz[glo.reshape(-1)] = orc.node_coords(N, v).reshape(-1, 3)
    u = 0.3 + 1.2 * xyz[:, 0] - 0.7 * xyz[:, 1] + 2.0 * xyz[:, 2]
    y = orc.apply(N, glo, G, u)
    interior = orc.box_dirichlet(*box, N) == 0
    ref = np.max(np.abs(orc.apply(N, glo, G, W.uniform(ng, seed=1))))
    assert np.max(np.abs(y[interior])) < 1e-13 * ref


# ------------------------------------------------------------------------------------------
# solver
# ------------------------------------------------------------------------------------------
def test_pcg_matches_direct_solve(orc):
    N, box = 3, (2, 2, 2)
    modes = W.kappa_modes(16, seed=8)
    v = W.box_vertices(*box, seed=4)
    xyz = orc.node_coords(N, v)
    kap = orc.kappa(modes, xyz)
    G, wJ = orc.factors(N, v, kappa_nodal=kap)
    glo = orc.box_numbering(*box, N)
    ng = orc.box_nglobal(*box, N)
    mask = orc.box_dirichlet(*box, N)
    A = _dense_assembled_O1(orc, v, N, glo, ng, kappa_nodal=kap)
    f = W.sine_forcing(xyz, modes)
    b = orc.rhs(N, glo, wJ, f, ng, mask=mask)
    dg = orc.diag(N, glo, G, ng, mask=mask)
    x, it, res = orc.pcg(N, glo, G, b, dg, mask=mask, rtol=1e-12)
    assert it > 0 and res <= 1e-12
    free = mask == 0
    xd = np.zeros(ng)
    xd[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    assert np.max(np.abs(x - xd)) < 1e-10 * np.max(np.abs(xd))
    assert orc.true_relres(N, glo, G, b, x, mask=mask) < 1e-11


def _solver_case(orc):
    N, box = 3, (2, 2, 2)
    modes = W.kappa_modes(16, seed=8)
    v = W.box_vertices(*box, seed=4)
    xyz = orc.node_coords(N, v)
    kap = orc.kappa(modes, xyz)
    G, wJ = orc.factors(N, v, kappa_nodal=kap)
    glo = orc.box_numbering(*box, N)
    ng = orc.box_nglobal(*box, N)
    mask = orc.box_dirichlet(*box, N)
    A = _dense_assembled_O1(orc, v, N, glo, ng, kappa_nodal=kap)
    b = orc.rhs(N, glo, wJ, W.sine_forcing(xyz, modes), ng, mask=mask)
    dg = orc.diag(N, glo, G, ng, mask=mask)
    free = mask == 0
    xd = np.zeros(ng)
    xd[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    return N, G, glo, mask, b, dg, xd


def test_ir_matches_direct_solve(orc):
    # FP64-residual refinement around an FP32 inner Jacobi-PCG reaches the dense direct solution;
    # each refinement step shrinks the FP64 residual by about the inner tolerance
    from oracle import solvers

    N, G, glo, mask, b, dg, xd = _solver_case(orc)
    x, outer, inner, hist = solvers.ir(N, glo, G, b, dg, mask=mask, rtol=1e-10, inner_rtol=1e-3)
    assert orc.true_relres(N, glo, G, b, x, mask=mask) <= 1e-10
    assert np.max(np.abs(x - xd)) < 1e-9 * np.max(np.abs(xd))
    assert 3 <= outer <= 6 and inner > 0
    assert all(h1 < 2e-2 * h0 for h0, h1 in zip(hist[:-1], hist[1:])), hist


def test_fcg_with_fixed_jacobi_equals_pcg(orc):
    # with a fixed SPD preconditioner the Polak-Ribiere beta equals the Fletcher-Reeves one in
    # exact arithmetic ((z_k, r_{k-1}) = 0), so flexible CG reproduces Jacobi-PCG
    from oracle import solvers

    N, G, glo, mask, b, dg, xd = _solver_case(orc)
    dinv = np.where(mask == 0, 1.0 / dg, 0.0)
    x, k, fb = solvers.fcg(N, glo, G, b, dg, lambda r, it: dinv * r, mask=mask, rtol=1e-10)
    xp, kp, _ = orc.pcg(N, glo, G, b, dg, mask=mask, rtol=1e-10)
    assert fb == 0 and abs(k - kp) <= 1, (k, kp)
    assert np.max(np.abs(x - xp)) < 1e-8 * np.max(np.abs(xp))
    assert np.max(np.abs(x - xd)) < 1e-8 * np.max(np.abs(xd))


def test_fcg_with_varying_preconditioner(orc):
    # a different random SPD (diagonal) preconditioner at every iteration: flexible CG still
    # reaches the direct solution
    from oracle import solvers

    N, G, glo, mask, b, dg, xd = _solver_case(orc)
    dinv = np.where(mask == 0, 1.0 / dg, 0.0)
    g = W.rng(17)

    def prec(r, it):
        return dinv * (0.5 + g.uniform(size=r.shape[0])) * r

    x, k, fb = solvers.fcg(N, glo, G, b, dg, prec, mask=mask, rtol=1e-10)
    assert fb == 0 and orc.true_relres(N, glo, G, b, x, mask=mask) <= 1e-9
    assert np.max(np.abs(x - xd)) < 1e-8 * np.max(np.abs(xd))


def test_fcg_rejects_non_descent_corrections(orc):
    # z = -D^-1 r has (z, r) < 0 on every iteration: each is replaced by the Jacobi step, so the
    # solve becomes Jacobi-PCG, iteration for iteration
    from oracle import solvers

    N, G, glo, mask, b, dg, xd = _solver_case(orc)
    dinv = np.where(mask == 0, 1.0 / dg, 0.0)
    x, k, fb = solvers.fcg(N, glo, G, b, dg, lambda r, it: -dinv * r, mask=mask, rtol=1e-10)
    _, kp, _ = orc.pcg(N, glo, G, b, dg, mask=mask, rtol=1e-10)
    assert fb == k and abs(k - kp) <= 1
    assert np.max(np.abs(x - xd)) < 1e-8 * np.max(np.abs(xd))


def test_manufactured_solution_converges_spectrally(orc):
    # nodal error against u* = sin sin sin must shrink monotonically as N grows (spectral accuracy)
    box = (2, 2, 2)
    errs = []
    for N in (3, 5, 7, 9):
        v = W.box_vertices(*box, seed=6)
        G, wJ = orc.factors(N, v)
        glo = orc.box_numbering(*box, N)
        ng = orc.box_nglobal(*box, N)
        mask = orc.box_dirichlet(*box, N)
        xyzL = orc.node_coords(N, v)
        b = orc.rhs(N, glo, wJ, W.sine_forcing(xyzL), ng, mask=mask)
        dg = orc.diag(N, glo, G, ng, mask=mask)
        x, it, _ = orc.pcg(N, glo, G, b, dg, mask=mask, rtol=1e-13)
        xyz = np.zeros((ng, 3))
        xyz[glo.reshape(-1)] = xyzL.reshape(-1, 3)
        errs.append(np.max(np.abs(x - W.sine_solution(xyz))))
    assert all(errs[i + 1] < 0.5 * errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-6, errs


# ------------------------------------------------------------------------------------------
# learned preconditioner reference (oracle/mlp.py)
# ------------------------------------------------------------------------------------------
def test_mlp_backward_matches_finite_differences():
    from oracle import mlp

    g = W.rng(5)
    lay = mlp.layout(8, 6, 5)  # n3 = 8 (N = 1), tiny hidden layers
    p = g.normal(0, 0.5, size=lay["count"])
    X = g.normal(size=(7, 14))
    T = g.normal(size=(7, 8))
    loss, grad = mlp.loss_and_grad(p, X, T, lay)
    for idx in g.integers(0, lay["count"], size=40):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (mlp.loss_and_grad(pp, X, T, lay)[0] - mlp.loss_and_grad(pm, X, T, lay)[0]) / (2 * h)
        assert abs(fd - grad[idx]) < 1e-7 * max(1.0, abs(fd)), idx


def test_adam_first_step_closed_form():
    from oracle import mlp

    g = W.rng(6).normal(size=50)
    p0 = W.rng(7).normal(size=50)
    p1, m, v = mlp.adam(p0, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    # after one step mhat = g, vhat = g^2: every parameter moves by lr sign(g) (up to eps)
    np.testing.assert_allclose(p1 - p0, -1e-3 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)


def test_geo_features_of_affine_cube(orc):
    from oracle import mlp

    N = 3
    v = np.array([[[(q & 1) * 0.5, ((q >> 1) & 1) * 0.5, ((q >> 2) & 1) * 0.5] for q in range(8)]])
    G, _ = orc.factors(N, v)
    np.testing.assert_allclose(mlp.geo6(G)[0], [1, 0, 0, 1, 0, 1], atol=1e-14)
    v2 = np.array([[[(q & 1) * 1.0, ((q >> 1) & 1) * 0.5, ((q >> 2) & 1) * 0.25] for q in range(8)]])
    G2, _ = orc.factors(N, v2)
    # diagonal factors scale as 1/h_d^2: (1, 4, 16) / 7
    np.testing.assert_allclose(mlp.geo6(G2)[0], np.array([1, 0, 0, 4, 0, 16]) / 7.0, rtol=1e-13, atol=1e-14)


def test_bf16_rounding_against_torch_and_ties():
    import torch

    from oracle import mlp

    g = W.rng(8)
    x = np.concatenate([g.normal(size=5000) * 10.0 ** g.uniform(-6, 6, size=5000), [0.0, -0.0, 1.0, -3.5]])
    x32 = x.astype(np.float32)  # FP32 inputs: torch's FP32 -> BF16 conversion rounds once, to nearest even
    ref = torch.from_numpy(x32).to(torch.bfloat16).float().double().numpy()
    np.testing.assert_array_equal(mlp.bf16(x32.astype(np.float64)), ref)
    # hand-worked ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 -> even mantissa 1;
    # 1 + 3 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6 -> even mantissa 1 + 2^-6;
    # 255 has 8 significant bits (exact); 257 lies halfway between 256 and 258 -> 256
    np.testing.assert_array_equal(mlp.bf16([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 255.0, 257.0]),
                                  [1.0, 1 + 2.0 ** -6, -1.0, 255.0, 256.0])


def test_forward_with_bf16_activations_rounds_every_layer_input():
    from oracle import mlp

    g = W.rng(9)
    lay = mlp.layout(8, 6, 5)
    p = mlp.bf16(g.normal(0, 0.5, size=lay["count"]))
    X = g.normal(size=(7, 14))
    H1, H2, O = mlp.forward(p, X, lay, act_bf16=True)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, lay)
    import torch

    r = lambda a: torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).double().numpy()
    h1 = np.maximum(mlp.bf16(X) @ W1 + b1, 0.0)
    np.testing.assert_array_equal(H1, mlp.bf16(h1))
    h2 = np.maximum(H1 @ W2 + b2, 0.0)
    np.testing.assert_array_equal(H2, mlp.bf16(h2))
    np.testing.assert_allclose(O, H2 @ W3 + b3, rtol=0, atol=0)
    # every activation is representable in BF16 (8 significant bits): torch's rounding leaves it unchanged
    for A in (H1, H2):
        np.testing.assert_array_equal(r(A), A)


def test_local_solve_closed_form_for_constant_load(orc):
    # A_e 1 = 0 for the stiffness, so (A_e + sigma M_e) x = M_e 1 has x = 1 / sigma exactly
    from oracle import mlp

    N = 3
    v = W.box_vertices(1, 1, 1, seed=12)
    modes = W.kappa_modes(8, seed=13)
    xyz = orc.node_coords(N, v)
    A = orc.element_matrix(N, v[0], kappa_e=orc.kappa(modes, xyz[0]))
    _, wJ = orc.factors(N, v, modes=modes)
    eps = 1e-2
    sigma = eps * np.trace(A) / np.sum(wJ[0])
    x = mlp.local_solve(A, wJ[0], wJ[0], eps)
    np.testing.assert_allclose(x, np.full(x.shape, 1.0 / sigma), rtol=1e-9)


def test_exact_element_corrections_beat_jacobi(orc):
    # the preconditioner the network is trained to reproduce (exact element targets, averaged)
    # needs fewer PCG iterations than Jacobi: the reading of the training targets is useful
    from oracle import mlp

    box, N = (3, 3, 3), 4
    v = W.box_vertices(*box, seed=14)
    modes = W.contrast_modes(100.0, seed=15)
    G, wJ = orc.factors(N, v, modes=modes)
    glo, mask = orc.box_numbering(*box, N), orc.box_dirichlet(*box, N)
    ng = orc.box_nglobal(*box, N)
    # element matrices column by column from the sum-factorised local operator (equal to the
    # brute-force weak form, pinned above)
    E, n3 = glo.shape
    A = np.zeros((E, n3, n3))
    for q in range(n3):
        u = np.zeros((E, n3))
        u[:, q] = 1.0
        A[:, :, q] = orc.apply_local(N, G, u)
    mult = np.zeros(ng)
    np.add.at(mult, glo.ravel(), 1.0)
    free = mask == 0
    dg = orc.diag(N, glo, G, ng, mask=mask)
    dinv = np.where(free, 1.0 / dg, 0.0)

    def nn(r):
        z = np.zeros(ng)
        for e in range(glo.shape[0]):
            ids = glo[e]
            x = mlp.local_solve(A[e], wJ[e], np.where(free[ids], r[ids], 0.0) / mult[ids], 1e-2)
            np.add.at(z, ids, x / mult[ids])
        return np.where(free, z, 0.0)

    b = np.where(free, W.uniform(ng, seed=16), 0.0)

    def pcg(prec):
        x, r = np.zeros(ng), b.copy()
        z = prec(r)
        p, rz = z.copy(), r @ z
        for it in range(1, 2000):
            Ap = orc.apply(N, glo, G, p, mask=mask)
            al = rz / (p @ Ap)
            x += al * p
            r -= al * Ap
            if np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b):
                return it
            z = prec(r)
            rz, rz0 = r @ z, rz
            p = z + (rz / rz0) * p
        return 2000

    it_j, it_nn = pcg(lambda r: dinv * r), pcg(nn)
    assert it_nn < 0.7 * it_j, (it_nn, it_j)
