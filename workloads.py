"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds random draws and the closed-form manufactured problem only; it contains none
of the spectral-element method's arithmetic (no GLL nodes, no geometric factors, no operator).
Every generator uses numpy's PCG64 with an explicit seed and draws in a fixed lexicographic order,
so both sides of a parity test see identical inputs.

Workloads (the paper measures SEM kernels on hexahedral meshes at orders 1..8, §4.2.2; it gives
no mesh, so these stand in for it):
  * ``box_vertices``   structured s_x*s_y*s_z hex mesh of [0,1]^3 with interior lattice vertices
                       perturbed per coordinate by U(-p h, p h) (h = 1/s per direction, p = 0.1);
  * ``uniform``        nodal fields u ~ U(-1, 1);
  * ``kappa_modes``    random Fourier modes for kappa(x) = exp(sum_m a_m cos(2 pi k_m.x + phi_m));
  * ``batch_problems`` a list of independent box problems of uneven size and order;
  * ``sine_solution`` / ``sine_forcing``  the manufactured solution u* = sin(pi x) sin(pi y) sin(pi z)
                       and its forcing f = -div(kappa grad u*) (closed form, works on numpy or torch).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 1403


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def box_vertices(sx: int, sy: int, sz: int, perturb: float = 0.1, seed: int = BASE_SEED) -> np.ndarray:
    """Vertices [E, 8, 3] of a structured box mesh of [0,1]^3.

    Element (ex, ey, ez) has index ex + sx*(ey + sy*ez); its vertex v = a + 2b + 4c is lattice point
    (ex+a, ey+b, ez+c).  Every lattice point draws three U(-1,1) numbers in lexicographic order
    (x fastest); only interior points use them (scaled by perturb*h), so boundary faces stay planar.
    """
    gx, gy, gz = sx + 1, sy + 1, sz + 1
    h = np.array([1.0 / sx, 1.0 / sy, 1.0 / sz])
    I, J, K = np.meshgrid(np.arange(gx), np.arange(gy), np.arange(gz), indexing="ij")
    lat = np.stack([I * h[0], J * h[1], K * h[2]], axis=-1)  # [gx, gy, gz, 3]
    lat = np.transpose(lat, (2, 1, 0, 3)).copy()  # [gz, gy, gx, 3], x fastest
    d = rng(seed).uniform(-1.0, 1.0, size=(gz, gy, gx, 3))
    interior = np.zeros((gz, gy, gx), dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    lat[interior] += perturb * d[interior] * h
    E = sx * sy * sz
    ex, ey, ez = np.meshgrid(np.arange(sx), np.arange(sy), np.arange(sz), indexing="ij")
    ex, ey, ez = (np.transpose(a, (2, 1, 0)).reshape(-1) for a in (ex, ey, ez))
    verts = np.empty((E, 8, 3))
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
        verts[:, v, :] = lat[ez + c, ey + b, ex + a]
    return verts


def box_nglobal(sx: int, sy: int, sz: int, N: int) -> int:
    return (sx * N + 1) * (sy * N + 1) * (sz * N + 1)


def uniform(n: int, seed: int = BASE_SEED, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=n)


def kappa_modes(nmodes: int = 16, amplitude: float = 0.25, seed: int = BASE_SEED) -> np.ndarray:
    """[nmodes, 5] rows (kx, ky, kz, phi, a): k uniform on {-4..4}^3 without 0, phi ~ U(0, 2pi)."""
    g = rng(seed)
    out = np.zeros((nmodes, 5))
    for m in range(nmodes):
        while True:
            k = g.integers(-4, 5, size=3)
            if np.any(k != 0):
                break
        out[m, :3] = k
        out[m, 3] = g.uniform(0.0, 2.0 * math.pi)
        out[m, 4] = amplitude
    return out


def contrast_modes(contrast: float, nmodes: int = 16, seed: int = BASE_SEED) -> np.ndarray:
    """Fourier modes whose exp(g) has max/min ratio at most ``contrast`` (|g| <= ln(contrast)/2)."""
    return kappa_modes(nmodes, amplitude=math.log(contrast) / (2.0 * nmodes), seed=seed)


@dataclass
class BoxProblem:
    sx: int
    sy: int
    sz: int
    N: int
    seed: int

    @property
    def nelem(self) -> int:
        return self.sx * self.sy * self.sz

    @property
    def nglobal(self) -> int:
        return box_nglobal(self.sx, self.sy, self.sz, self.N)


def batch_problems(nprob: int = 256, smin: int = 8, smax: int = 32, orders=(3, 5, 7, 9, 11),
                   seed: int = BASE_SEED + 3) -> list[BoxProblem]:
    """Independent cube problems: side s ~ U{smin..smax}, order N ~ U(orders), own seed each."""
    g = rng(seed)
    out = []
    for k in range(nprob):
        s = int(g.integers(smin, smax + 1))
        N = int(orders[int(g.integers(0, len(orders)))])
        out.append(BoxProblem(s, s, s, N, seed + 1000 + k))
    return out


def _xp(a):
    try:
        import torch

        if isinstance(a, torch.Tensor):
            return torch
    except ImportError:  # pragma: no cover
        pass
    return np


def sine_solution(xyz):
    """u*(x) = sin(pi x) sin(pi y) sin(pi z) on [..., 3] points (numpy or torch)."""
    xp = _xp(xyz)
    s = xp.sin(math.pi * xyz)
    return s[..., 0] * s[..., 1] * s[..., 2]


def sine_forcing(xyz, modes=None):
    """f = -div(kappa grad u*) for u* = sine_solution and kappa = exp(g), g from ``modes``.

    f = kappa (3 pi^2 u* - grad g . grad u*),  grad g = -sum_m a_m 2 pi k_m sin(2 pi k_m.x + phi_m).
    """
    xp = _xp(xyz)
    s = xp.sin(math.pi * xyz)
    c = xp.cos(math.pi * xyz)
    u = s[..., 0] * s[..., 1] * s[..., 2]
    du = [math.pi * c[..., 0] * s[..., 1] * s[..., 2],
          math.pi * s[..., 0] * c[..., 1] * s[..., 2],
          math.pi * s[..., 0] * s[..., 1] * c[..., 2]]
    g = xp.zeros_like(u)
    dg = [xp.zeros_like(u) for _ in range(3)]
    if modes is not None:
        for kx, ky, kz, phi, a in np.asarray(modes, dtype=np.float64):
            arg = 2.0 * math.pi * (kx * xyz[..., 0] + ky * xyz[..., 1] + kz * xyz[..., 2]) + phi
            g = g + a * xp.cos(arg)
            sn = xp.sin(arg)
            for d, kd in enumerate((kx, ky, kz)):
                dg[d] = dg[d] - a * 2.0 * math.pi * kd * sn
    kap = xp.exp(g)
    return kap * (3.0 * math.pi ** 2 * u - (dg[0] * du[0] + dg[1] * du[1] + dg[2] * du[2]))


def tri_mesh(nx: int, ny: int, perturb: float = 0.1, seed: int = BASE_SEED) -> np.ndarray:
    """Vertices [E][3][2] (counter-clockwise) of a triangulated nx x ny grid of [0,1]^2: each cell
    split along its lower-left to upper-right diagonal into two triangles, E = 2 nx ny; interior
    lattice points moved per coordinate by U(-p h, p h) (h = 1/nx, 1/ny), boundary straight."""
    gx, gy = nx + 1, ny + 1
    h = np.array([1.0 / nx, 1.0 / ny])
    J, I = np.meshgrid(np.arange(gy), np.arange(gx), indexing="ij")
    lat = np.stack([I * h[0], J * h[1]], axis=-1).astype(np.float64)  # [gy, gx, 2], x fastest
    d = rng(seed).uniform(-1.0, 1.0, size=(gy, gx, 2))
    interior = np.zeros((gy, gx), dtype=bool)
    interior[1:-1, 1:-1] = True
    lat[interior] += perturb * d[interior] * h
    cj, ci = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ci, cj = ci.reshape(-1), cj.reshape(-1)
    p00, p10, p01, p11 = lat[cj, ci], lat[cj, ci + 1], lat[cj + 1, ci], lat[cj + 1, ci + 1]
    lower = np.stack([p00, p10, p11], axis=1)  # counter-clockwise
    upper = np.stack([p00, p11, p01], axis=1)
    return np.stack([lower, upper], axis=1).reshape(-1, 3, 2)


def swe_fields(E: int, Np: int, seed: int = BASE_SEED):
    """Nodal shallow-water fields Q [E][3][Np] (h ~ U(0.5, 1.5), hu, hv ~ U(-0.5, 0.5)) and bathymetry
    gradients Bxy [E][2][Np] ~ U(-1, 1)."""
    g = rng(seed)
    Q = np.empty((E, 3, Np))
    Q[:, 0] = g.uniform(0.5, 1.5, size=(E, Np))
    Q[:, 1:] = g.uniform(-0.5, 0.5, size=(E, 2, Np))
    return Q, g.uniform(-1.0, 1.0, size=(E, 2, Np))
