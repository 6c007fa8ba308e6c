"""FP64 reference of the learned element-local preconditioner (test infrastructure only).

The network (n^3 + 6 -> h1 -> h2 -> n^3, ReLU after the hidden layers), its mean-squared-error
loss, the backward pass, Adam (Kingma & Ba, 2015: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
w -= lr mhat / (sqrt(vhat) + eps) with bias-corrected mhat, vhat), the per-element features
(residual on the element divided by its norm, plus six element-mean geometric factors divided by
their mean diagonal) and the assembled preconditioner (scaled element outputs averaged over the
elements sharing a node), written plainly in numpy.  Parameter layout: W1 [n_in][h1], b1, W2
[h1][h2], b2, W3 [h2][n_out], b3, row-major in one vector.

Pins (tests/test_oracle_pins.py): central finite differences of the loss against the backward
pass; Adam against its closed form after one step (|update| = lr for every component); features of
an affine cube element against their closed form; BF16 rounding against torch's FP32 -> BF16
conversion and hand-worked ties.  The preconditioner is z = D^-1 r + c(r): the
network learns the error a Jacobi step leaves, so a zero network is Jacobi.  The gain of the learned preconditioner over
Jacobi has no value in the paper to pin against ("parity unpinned"; it is measured).
"""
from __future__ import annotations

import numpy as np


def layout(n3: int, h1: int, h2: int):
    nin, nout = n3 + 6, n3
    sizes = [("W1", nin * h1), ("b1", h1), ("W2", h1 * h2), ("b2", h2), ("W3", h2 * nout), ("b3", nout)]
    out, off = {}, 0
    for name, sz in sizes:
        out[name] = (off, sz)
        off += sz
    out["count"] = off
    out["shape"] = (nin, h1, h2, nout)
    return out


def unpack(params, lay):
    nin, h1, h2, nout = lay["shape"]
    get = lambda k: np.asarray(params[lay[k][0]:lay[k][0] + lay[k][1]], dtype=np.float64)
    return (get("W1").reshape(nin, h1), get("b1"), get("W2").reshape(h1, h2), get("b2"),
            get("W3").reshape(h2, nout), get("b3"))


def bf16(x):
    """x rounded to the nearest BF16 value (8 significant bits), ties to even; no overflow or
    subnormal handling (the network's values are far inside the range)."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))  # x = m 2^e, 1/2 <= |m| < 1
    return np.ldexp(np.round(m * 256.0), e - 8)       # np.round rounds halves to even


def forward(params, X, lay, act_bf16=False):
    """Layer outputs H1, H2, O; with act_bf16 the input of every layer (features, H1, H2) is
    rounded to BF16 first, as in the tensor-core inference."""
    W1, b1, W2, b2, W3, b3 = unpack(params, lay)
    rnd = bf16 if act_bf16 else (lambda a: a)
    X = rnd(np.asarray(X, dtype=np.float64))
    H1 = rnd(np.maximum(X @ W1 + b1, 0.0))
    H2 = rnd(np.maximum(H1 @ W2 + b2, 0.0))
    O = H2 @ W3 + b3
    return H1, H2, O


def loss_and_grad(params, X, T, lay):
    """Mean over all B * n_out entries of (O - T)^2 and its gradient (same layout as params)."""
    W1, b1, W2, b2, W3, b3 = unpack(params, lay)
    X = np.asarray(X, dtype=np.float64)
    H1, H2, O = forward(params, X, lay)
    D = O - np.asarray(T, dtype=np.float64)
    n = D.size
    loss = float(np.sum(D * D) / n)
    dO = 2.0 * D / n
    gW3 = H2.T @ dO
    gb3 = dO.sum(axis=0)
    dH2 = (dO @ W3.T) * (H2 > 0)
    gW2 = H1.T @ dH2
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2.T) * (H1 > 0)
    gW1 = X.T @ dH1
    gb1 = dH1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam(params, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def geo6(G):
    """Element means of the six factors divided by the mean of their diagonal (G: [E, 6, n3])."""
    m = np.asarray(G, dtype=np.float64).mean(axis=2)
    tr = (m[:, 0] + m[:, 3] + m[:, 5]) / 3.0
    return np.where(tr[:, None] > 0, m / np.where(tr > 0, tr, 1.0)[:, None], 0.0)


def features(glo, mask, r, geo, elems, xstar=None, xk=None, dinv=None):
    """X [s, n3+6], T [s, n3] (if xstar, xk given) and scale [s] for the elements ``elems``.

    Targets are the error left after a Jacobi step, (x* - x_k - D^-1 r) on the element, divided by
    the element's residual norm (dinv: inverse assembled diagonal, zero on Dirichlet nodes).
    """
    r = np.asarray(r, dtype=np.float64)
    free = np.asarray(mask) == 0 if mask is not None else np.ones(r.shape[0], dtype=bool)
    ids = np.asarray(glo)[np.asarray(elems)]
    re = np.where(free[ids], r[ids], 0.0)
    nrm = np.sqrt(np.sum(re * re, axis=1))
    inv = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)
    X = np.concatenate([re * inv[:, None], np.asarray(geo)[np.asarray(elems)]], axis=1)
    T = None
    if xstar is not None:
        e = np.asarray(xstar, dtype=np.float64) - np.asarray(xk, dtype=np.float64) - np.asarray(dinv) * r
        T = np.where(free[ids], e[ids], 0.0) * inv[:, None]
    return X, T, nrm


def precond(params, lay, glo, mask, r, geo, nglobal, dinv, act_bf16=False):
    """z = D^-1 r + sum_e Q^T (|r_e| MLP(features_e)) / multiplicity, zero on Dirichlet nodes."""
    glo = np.asarray(glo)
    E = glo.shape[0]
    X, _, nrm = features(glo, mask, r, geo, np.arange(E))
    _, _, O = forward(params, X, lay, act_bf16=act_bf16)
    mult = np.zeros(nglobal)
    np.add.at(mult, glo.ravel(), 1.0)
    z = np.zeros(nglobal)
    np.add.at(z, glo.ravel(), (O * nrm[:, None]).ravel())
    z = np.where(mult > 0, z / np.where(mult > 0, mult, 1.0), 0.0) + np.asarray(dinv) * np.asarray(r)
    if mask is not None:
        z[np.asarray(mask) != 0] = 0.0
    return z
