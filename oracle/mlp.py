"""FP64 reference of the learned element-local preconditioner (test infrastructure only).

The network (n^3 + 6 -> h1 -> h2 -> n^3, ReLU after the hidden layers), its mean-squared-error
loss, the backward pass, Adam (Kingma & Ba, 2015: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
w -= lr mhat / (sqrt(vhat) + eps) with bias-corrected mhat, vhat), the per-element features
(residual on the element divided by its norm, plus six element-mean geometric factors divided by
their mean diagonal), the training pairs and the assembled preconditioner, written plainly in
numpy.  Parameter layout: W1 [n_in][h1], b1, W2 [h1][h2], b2, W3 [h2][n_out], b3, row-major in
one vector.

Training pair of element e for a global residual r (zero on Dirichlet nodes): the input is the
feature vector, the target the solution x_e of the element's own shifted Neumann problem
(A_e + sigma_e M_e) x_e = W_e r_e, sigma_e = eps trace(A_e) / sum_p (w det J)_p, W_e = 1 /
multiplicity, zero on Dirichlet nodes, divided by |r_e| / dbar_e, dbar_e = trace(A_e) / n^3.
The preconditioner is z = B r + sum_e Q^T W_e (scale_e MLP(features_e)), scale_e = |r_e| /
dbar_e, zero on Dirichlet nodes: the multiplicity-weighted average of the predicted element
corrections (a learned one-level Neumann-Neumann step), on a Jacobi base B = D^-1 (targets
x_e - (D^-1 r)_e) or none (B = 0).

Pins (tests/test_oracle_pins.py): central finite differences of the loss against the backward
pass; Adam against its closed form after one step (|update| = lr for every component); features of
an affine cube element against their closed form; BF16 rounding against torch's FP32 -> BF16
conversion and hand-worked ties; the local solve against its closed form for a constant load
(A_e 1 = 0, so (A_e + sigma M_e)^-1 M_e 1 = 1 / sigma); the exact element corrections in PCG
against Jacobi (fewer iterations).
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


def local_solve(Ae, wJe, rhs, eps):
    """x = (A_e + sigma M_e)^-1 rhs with M_e = diag(wJe), sigma = eps trace(A_e) / sum(wJe)."""
    Ae = np.asarray(Ae, dtype=np.float64)
    wJe = np.asarray(wJe, dtype=np.float64)
    sigma = eps * np.trace(Ae) / np.sum(wJe)
    return np.linalg.solve(Ae + sigma * np.diag(wJe), np.asarray(rhs, dtype=np.float64))


def features(glo, mask, r, geo, elems, dbar):
    """X [s, n3+6] and scale [s] = |r_e| / dbar_e for the elements ``elems`` (dbar per element)."""
    r = np.asarray(r, dtype=np.float64)
    free = np.asarray(mask) == 0 if mask is not None else np.ones(r.shape[0], dtype=bool)
    ids = np.asarray(glo)[np.asarray(elems)]
    re = np.where(free[ids], r[ids], 0.0)
    nrm = np.sqrt(np.sum(re * re, axis=1))
    inv = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)
    X = np.concatenate([re * inv[:, None], np.asarray(geo)[np.asarray(elems)]], axis=1)
    return X, nrm / np.asarray(dbar, dtype=np.float64)[np.asarray(elems)]


def pairs(Aelems, wJ, glo, mask, r, geo, elems, eps, nglobal, dinv=None):
    """Training pairs X [s, n3+6], T [s, n3] of the sampled elements (Aelems[s]: dense A_e of
    element elems[s]; wJ [E, n3] lumped mass).  With dinv (the inverse assembled diagonal, zero on
    Dirichlet nodes) the targets are the corrections to a Jacobi step, x_e - (D^-1 r)_e."""
    glo = np.asarray(glo)
    r = np.asarray(r, dtype=np.float64)
    free = np.asarray(mask) == 0 if mask is not None else np.ones(r.shape[0], dtype=bool)
    mult = np.zeros(nglobal)
    np.add.at(mult, glo.ravel(), 1.0)
    dbar = np.zeros(glo.shape[0])
    for s, e in enumerate(elems):
        dbar[e] = np.trace(Aelems[s]) / glo.shape[1]
    X, scale = features(glo, mask, r, geo, elems, dbar)
    T = np.zeros((len(elems), glo.shape[1]))
    for s, e in enumerate(elems):
        ids = glo[e]
        re = np.where(free[ids], r[ids], 0.0)
        x = local_solve(Aelems[s], np.asarray(wJ)[e], re / mult[ids], eps)
        if dinv is not None:
            x = x - np.asarray(dinv)[ids] * re
        T[s] = np.where(free[ids], x, 0.0) / scale[s] if scale[s] > 0 else 0.0
    return X, T


def precond(params, lay, glo, mask, r, geo, dbar, nglobal, act_bf16=False, dinv=None):
    """z = [D^-1 r +] sum_e Q^T W_e (scale_e MLP(features_e)), zero on Dirichlet nodes (the
    Jacobi base D^-1 r when dinv is given)."""
    glo = np.asarray(glo)
    E = glo.shape[0]
    X, scale = features(glo, mask, r, geo, np.arange(E), dbar)
    _, _, O = forward(params, X, lay, act_bf16=act_bf16)
    mult = np.zeros(nglobal)
    np.add.at(mult, glo.ravel(), 1.0)
    z = np.zeros(nglobal)
    np.add.at(z, glo.ravel(), (O * scale[:, None]).ravel())
    z = np.where(mult > 0, z / np.where(mult > 0, mult, 1.0), 0.0)
    if dinv is not None:
        z = z + np.asarray(dinv) * np.asarray(r, dtype=np.float64)
    if mask is not None:
        z[np.asarray(mask) != 0] = 0.0
    return z
