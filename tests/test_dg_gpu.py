"""Parity of the CUDA DG shallow-water volume kernel (sem_dg_volume, arXiv 1403.0968 §4.3) against
the FP64 oracle (oracle/dg.py).  Tolerances (relative max-norm over the output): FP64 1e-12 (the
two sides build the derivative matrices by different routes, agreeing to ~2e-14 relative), FP32
1e-5."""
import numpy as np
import pytest

import workloads as W
from oracle import dg

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
G = 9.81


@pytest.fixture(scope="module")
def sem():
    from paper_1403_0968_gb300 import build

    build.build()
    import paper_1403_0968_gb300 as sem

    sem.lib()
    return sem


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _run(sem, N, verts, Q, Bxy, prec):
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    ops = sem.dg_load_operators(N, dt)
    geo = sem.dg_geometry(verts, dt)
    out = sem.dg_volume(N, torch.from_numpy(Q).to(dt).cuda(), torch.from_numpy(Bxy).to(dt).cuda(), geo, G, ops)
    return out.double().cpu().numpy(), geo.double().cpu().numpy()


@pytest.mark.parametrize("N", range(1, 9))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny", [(5, 4), (9, 7)])
def test_volume_matches_oracle(sem, N, prec, nx, ny):
    # 40 and 126 perturbed triangles: several blocks and a ragged last block at every order
    verts = W.tri_mesh(nx, ny, perturb=0.2, seed=N + nx)
    E, Np = verts.shape[0], (N + 1) * (N + 2) // 2
    Q, Bxy = W.swe_fields(E, Np, seed=N + 100)
    got, geo = _run(sem, N, verts, Q, Bxy, prec)
    rx, ry, sx, sy, J = dg.geometry(verts)
    assert relerr(geo, np.stack([rx, ry, sx, sy], axis=1)) < (1e-15 if prec == "fp64" else 1e-7)
    ref = dg.volume(N, Q, Bxy, (rx, ry, sx, sy), G)
    assert relerr(got, ref) < TOL[prec]


def test_single_element_resting_layer(sem):
    # one element, a resting layer (h = 2, hu = hv = 0, flat bottom): the mass equation has no
    # volume flux at all, the momentum equations only the pressure term g h^2 / 2
    verts = np.array([[[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]]])
    N, Np = 4, 15
    Q = np.zeros((1, 3, Np))
    Q[0, 0] = 2.0
    Bxy = np.zeros((1, 2, Np))
    got, _ = _run(sem, N, verts, Q, Bxy, "fp64")
    rx, ry, sx, sy, J = dg.geometry(verts)
    ref = dg.volume(N, Q, Bxy, (rx, ry, sx, sy), G)
    assert relerr(got, ref) < TOL["fp64"]
    assert np.all(got[0, 0] == 0.0)  # no mass flux without momentum


def test_clockwise_triangle_rejected(sem):
    import torch

    verts = np.array([[[0.0, 0.0], [0.0, 1.0], [1.0, 0.0]]])
    with pytest.raises(sem.SemError):
        sem.dg_geometry(verts, torch.float64)


@pytest.mark.parametrize("N", [1, 4, 8])
def test_full_size_sampled(sem, N):
    # the 212,800-element bench mesh (280 x 380 cells, two triangles each), FP32: sampled elements
    # against the oracle
    import torch

    verts = W.tri_mesh(280, 380, perturb=0.1, seed=W.BASE_SEED + 900)
    E, Np = verts.shape[0], (N + 1) * (N + 2) // 2
    assert E == 212800
    Q, Bxy = W.swe_fields(E, Np, seed=W.BASE_SEED + 901)
    got, _ = _run(sem, N, verts, Q, Bxy, "fp32")
    idx = np.unique(np.concatenate([W.rng(N).integers(0, E, size=64), [0, 1, E - 2, E - 1]]))
    rx, ry, sx, sy, J = dg.geometry(verts[idx])
    ref = dg.volume(N, Q[idx], Bxy[idx], (rx, ry, sx, sy), G)
    assert relerr(got[idx], ref) < TOL["fp32"]
    torch.cuda.empty_cache()
