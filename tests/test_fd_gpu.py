"""Parity of the CUDA finite-difference wave step (sem_fd_step, arXiv 1403.0968 §4.1, periodic
boundary as in the §4.1 kernel listing) against the FP64 oracle (oracle/fd.py).  Tolerances
(relative max-norm): FP64 1e-12 per step, FP32 1e-5 per step; several steps 1e-11 / 1e-4."""
import numpy as np
import pytest

from oracle import fd

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def sem():
    from paper_1403_0968_gb300 import build

    build.build()
    import paper_1403_0968_gb300 as sem

    sem.lib()
    return sem


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _grids(h, w, seed):
    g = np.random.default_rng(seed)
    return g.uniform(-1, 1, (h, w)), g.uniform(-1, 1, (h, w))


def _dev(a, prec):
    import torch

    return torch.from_numpy(a).to(torch.float64 if prec == "fp64" else torch.float32).cuda().contiguous()


@pytest.mark.parametrize("r", range(1, 8))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("h,w", [(37, 101), (70, 65), (33, 200), (45, 132), (70, 256)])
def test_step_matches_oracle(sem, r, prec, h, w):
    # several tiles of 64 x 32 outputs with ragged last tiles in both directions; rows of a multiple
    # of 16 bytes (w = 200, 132, 256) take the TMA-staged kernel, the others the plain-load one
    u, up = _grids(h, w, seed=10 * r + h)
    dt, dx, dy = 0.004, 0.011, 0.013
    ref = fd.step(u, up, r, dt, dx, dy)
    ud, upd = _dev(u, prec), _dev(up, prec)
    sem.fd_step(ud, upd, r, dt, dx, dy)
    sem.fd_status()
    assert relerr(upd.double().cpu().numpy(), ref) < TOL[prec]
    # u_n is left untouched
    assert np.array_equal(ud.double().cpu().numpy(), u.astype(np.float32 if prec == "fp32" else np.float64))


@pytest.mark.parametrize("w", [130, 128])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-4)])
def test_many_steps_match_oracle(sem, prec, tol, w):
    # a smooth pulse stepped 40 times at a stable time step (w = 128: the TMA-staged kernel)
    h, r = 96, 4
    dx = dy = 2.0 / (w - 1)
    dt = 0.3 * dx
    y, x = np.mgrid[0:h, 0:w]
    u1 = np.exp(-((x - 60) ** 2 + (y - 50) ** 2) / 60.0)
    u0 = u1.copy()
    ref, _ = fd.run(u1, u0, 40, r, dt, dx, dy)
    a, b = sem.fd_run(_dev(u1, prec), _dev(u0, prec), 40, r, dt, dx, dy)
    sem.fd_status()
    assert relerr(a.double().cpu().numpy(), ref) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("h,w,r", [(1, 1, 1), (1, 1, 7), (2, 3, 7), (5, 1, 3), (1, 64, 2), (32, 64, 5), (33, 65, 7),
                                   (3, 4, 7), (40, 8, 5), (7, 16, 7), (100, 192, 7)])
def test_degenerate_and_exact_tile_grids(sem, h, w, r, prec):
    # grids narrower than the stencil (the halo wraps more than once), single rows and columns,
    # exactly one tile, one node past it; w = 4, 8, 16 (FP32) and 192 have 16-byte rows: their
    # edge tiles take the wrapped plain loads inside the TMA-staged kernel
    u, up = _grids(h, w, seed=h * 100 + w)
    ref = fd.step(u, up, r, 0.01, 0.02, 0.03)
    ud, upd = _dev(u, prec), _dev(up, prec)
    sem.fd_step(ud, upd, r, 0.01, 0.02, 0.03)
    sem.fd_status()
    assert relerr(upd.double().cpu().numpy(), ref) < TOL[prec]


@pytest.mark.parametrize("w", [256, 250])
@pytest.mark.parametrize("r", [1, 7])
def test_periodic_mode_on_gpu(sem, r, w):
    # a grid-periodic Fourier mode stays a mode: the step multiplies it by the closed-form leapfrog
    # amplitude at every node, the wrapped edges included (w = 256: TMA-staged interior tiles)
    h = 96
    dx, dy, dt = 0.05, 0.07, 0.01
    i, j = np.arange(w)[None, :], np.arange(h)[:, None]
    f = np.cos(2 * np.pi * (3 * i / w + 2 * j / h) + 0.4)
    ref = fd.step(1.3 * f, 0.9 * f, r, dt, dx, dy)
    ud, upd = _dev(1.3 * f, "fp64"), _dev(0.9 * f, "fp64")
    sem.fd_step(ud, upd, r, dt, dx, dy)
    sem.fd_status()
    out = upd.cpu().numpy()
    assert relerr(out, ref) < TOL["fp64"]
    # proportional to the mode everywhere
    amp = out[f != 0] / f[f != 0]
    big = np.abs(f[f != 0]) > 0.1
    assert np.max(np.abs(amp[big] - amp[big][0])) < 1e-9 * abs(amp[big][0])


def test_polynomial_solution_on_gpu(sem):
    # the exact cubic solution of the wave equation is reproduced away from the wrap seam
    h, w, r = 50, 70, 3
    dx, dy, dt = 0.03, 0.04, 0.01
    X = -1.0 + dx * np.arange(w)[None, :] + 0.0 * np.arange(h)[:, None]
    Y = -1.0 + dy * np.arange(h)[:, None] + 0.0 * np.arange(w)[None, :]

    def ex(t):
        return X ** 3 + 3 * X * t ** 2 + t ** 3 + 3 * t * X ** 2 + Y ** 2 + t ** 2

    ud, upd = _dev(ex(0.5), "fp64"), _dev(ex(0.5 - dt), "fp64")
    sem.fd_step(ud, upd, r, dt, dx, dy)
    out, ref = upd.cpu().numpy()[r:h - r, r:w - r], ex(0.5 + dt)[r:h - r, r:w - r]
    assert np.max(np.abs(out - ref)) < 1e-11 * np.max(np.abs(ref))


def test_invalid_arguments_rejected(sem):
    import torch

    u = torch.zeros(8, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):
        sem.fd_step(u, u, 1, 0.1, 0.1, 0.1)  # aliasing
    v = torch.zeros_like(u)
    with pytest.raises(sem.SemError):
        sem.fd_step(u, v, 8, 0.1, 0.1, 0.1)  # radius
    with pytest.raises(sem.SemError):
        sem.fd_step(u, v, 2, 0.0, 0.1, 0.1)  # time step


@pytest.mark.parametrize("r", [1, 4, 7])
def test_full_size_sampled(sem, r):
    # the 16384 x 16384 benchmark grid, FP32, one step: sampled nodes against the oracle node by node
    import torch

    n = 16384
    g = torch.Generator(device="cuda").manual_seed(1403 + r)
    ud = torch.rand(n, n, device="cuda", generator=g) * 2 - 1
    upd = torch.rand(n, n, device="cuda", generator=g) * 2 - 1
    dx = dy = 2.0 / (n - 1)
    dt = 0.4 * dx
    rng = np.random.default_rng(r)
    nodes = [tuple(int(v) for v in rng.integers(0, n, size=2)) for _ in range(40)]
    nodes += [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (63, 31), (64, 32), (5, n - 3)]
    # each sampled node's stencil cross (rows j-r..j+r and columns i-r..i+r, wrapped around the
    # grid) and its u_{n-1}, copied to the host before the step overwrites u_{n-1}; the oracle
    # steps the (2r+1) x (2r+1) patch at its centre, where no index wraps inside the patch
    patches = []
    for (i, j) in nodes:
        rows = torch.tensor([(j + k) % n for k in range(-r, r + 1)], device="cuda")
        cols = torch.tensor([(i + k) % n for k in range(-r, r + 1)], device="cuda")
        pu = ud[rows][:, cols].double().cpu().numpy()
        pup = upd[rows][:, cols].double().cpu().numpy()
        patches.append((pu, pup))
    sem.fd_step(ud, upd, r, dt, dx, dy)
    torch.cuda.synchronize()
    got = np.array([float(upd[j, i]) for (i, j) in nodes])
    ref = np.array([fd.step_at(pu, pup, r, dt, dx, dy, [(r, r)])[0] for (pu, pup) in patches])
    assert np.max(np.abs(got - ref)) < TOL["fp32"] * max(np.max(np.abs(ref)), 1.0)
