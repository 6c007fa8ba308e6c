"""Failure paths on the GPU, made on the host, with no fault and no hang (arXiv 1403.0968 §4.2.2
solver; the statuses are the library's own): a staged copy whose bounded wait is told to give up
at once (SEM_ERR_TIMEOUT from sem_apply_status and sem_pcg, and recovery afterwards), an
indefinite operator from a negative screening coefficient (SEM_ERR_BREAKDOWN), NaN network
weights (flexible CG falls back to Jacobi on every iteration), and Dirichlet flag arrays with
arbitrary non-zero bytes or every node flagged."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sem():
    from paper_1403_0968_gb300 import build

    build.build()
    import paper_1403_0968_gb300 as sem

    sem.lib()
    return sem


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _box_problem(sem, box=(3, 3, 2), N=5, features=None, alpha=None, seed=W.BASE_SEED):
    v = W.box_vertices(*box, seed=seed)
    feats = features or (sem.SEM_FEAT_FP64 | sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG)
    return sem.Problem(N, v, box=box, bc="box", alpha=alpha, features=feats), v


@pytest.mark.parametrize("prec,variant", [("fp64_emu", 0), ("fp64", 0), ("fp32", 0), ("fp64", 4), ("fp32", 4)])
def test_staged_copy_timeout_is_reported_and_cleared(sem, orc, prec, variant):
    box, N = (3, 3, 2), 5
    prob, v = _box_problem(sem, box, N)
    prob.set_apply_variant(variant)  # 0: factor block staged by a bulk copy; 4: persistent, double-buffered
    u = torch.from_numpy(W.uniform(prob.nglobal, seed=7)).cuda()
    uu = u.float() if prec == "fp32" else u
    prob.apply_status()  # nothing pending
    prob.set_wait_limit(0)  # every staged wait gives up at once; each block still waits for its own copy
    prob.apply(uu, prec=prec)
    with pytest.raises(sem.SemError) as ei:
        prob.apply_status()
    assert ei.value.status == sem.SEM_ERR_TIMEOUT
    prob.apply_status()  # the flag was cleared
    # the default limit again: the handle works and the result is right
    prob.set_wait_limit(-1)
    y = prob.apply(uu, prec=prec).double().cpu().numpy()
    prob.apply_status()
    G, _ = orc.factors(N, v)
    yo = orc.apply(N, orc.box_numbering(*box, N), G, u.cpu().numpy(), mask=orc.box_dirichlet(*box, N))
    assert _relerr(y, yo) < (1e-12 if prec.startswith("fp64") else 1e-5)


@pytest.mark.parametrize("mode,apply_prec", [("fp64", "fp64_emu"), ("fp64", "fp64"), ("ir", "fp64_emu")])
def test_pcg_returns_timeout_and_recovers(sem, orc, mode, apply_prec):
    box, N = (3, 3, 2), 5
    prob, v = _box_problem(sem, box, N)
    prob.set_apply_variant(0)
    b = prob.rhs(W.sine_forcing(prob.node_coords(), None))
    prob.set_wait_limit(0)
    _, info = prob.pcg(b, rtol=1e-10, mode=mode, apply_prec=apply_prec, raise_on_error=False)
    assert info["status"] == "SEM_ERR_TIMEOUT", info
    prob.set_wait_limit(-1)
    x, info = prob.pcg(b, rtol=1e-10, mode=mode, apply_prec=apply_prec)
    assert info["status"] == "SEM_OK"
    G, _ = orc.factors(N, v)
    rel = orc.true_relres(N, orc.box_numbering(*box, N), G, b.cpu().numpy(), x.cpu().numpy(),
                          mask=orc.box_dirichlet(*box, N))
    assert rel <= 1e-10


def test_indefinite_operator_breaks_down(sem):
    # alpha = -1e4 (host input) makes M A M indefinite: the first p^T A p is negative and the solve
    # stops with SEM_ERR_BREAKDOWN instead of iterating on garbage
    box, N = (2, 2, 2), 3
    E, n3 = 8, (N + 1) ** 3
    prob, _ = _box_problem(sem, box, N, alpha=np.full((E, n3), -1e4),
                           features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_PCG)
    b = prob.rhs(W.sine_forcing(prob.node_coords(), None))
    _, info = prob.pcg(b, rtol=1e-10, mode="fp64", apply_prec="fp64", raise_on_error=False)
    assert info["status"] == "SEM_ERR_BREAKDOWN", info


def test_nan_weights_fall_back_to_jacobi(sem, orc):
    # NaN parameters loaded on the host make every learned correction non-finite: flexible CG
    # must take the Jacobi step on every iteration and still reach the true 1e-10
    from paper_1403_0968_gb300 import learn

    box, N = (3, 3, 3), 3
    prob, v = _box_problem(sem, box, N, features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_PCG | sem.SEM_FEAT_MLP)
    p = learn.he_init(N, seed=0)
    p[::97] = np.nan
    prob.mlp_load(torch.from_numpy(p).cuda(), jacobi_base=True)
    b = prob.rhs(W.sine_forcing(prob.node_coords(), None))
    x, info = prob.pcg(b, rtol=1e-10, mode="fcg_mlp", apply_prec="fp64_emu")
    assert info["status"] == "SEM_OK" and info["fallbacks"] == info["iterations"] > 0, info
    G, _ = orc.factors(N, v)
    rel = orc.true_relres(N, orc.box_numbering(*box, N), G, b.cpu().numpy(), x.cpu().numpy(),
                          mask=orc.box_dirichlet(*box, N))
    assert rel <= 1e-10


def _mask_problem(sem, flags, box=(2, 3, 2), N=4):
    v = W.box_vertices(*box, seed=11)
    return sem.Problem(N, v, box=box, bc="mask", dirichlet=flags,
                       features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_PCG)


def test_dirichlet_flags_any_nonzero_byte(sem, orc):
    # a flag array holding arbitrary non-zero bytes marks the same nodes as a 0/1 array: the
    # operator and the assembled diagonal agree
    box, N = (2, 3, 2), 4
    ng = orc.box_nglobal(*box, N)
    g = np.random.default_rng(3)
    m01 = (g.uniform(size=ng) < 0.3).astype(np.uint8)
    junk = m01 * g.integers(1, 256, size=ng).astype(np.uint8)
    p01, pj = _mask_problem(sem, m01, box, N), _mask_problem(sem, junk, box, N)
    u = torch.from_numpy(W.uniform(ng, seed=5)).cuda()
    y01, yj = p01.apply(u).cpu().numpy(), pj.apply(u).cpu().numpy()
    assert _relerr(yj, y01) < 1e-14
    assert np.all(yj[m01 != 0] == 0.0)
    # the diagonal is assembled with atomics: equal to the last bit of the summation order
    np.testing.assert_allclose(pj.diag().cpu().numpy(), p01.diag().cpu().numpy(), rtol=2e-15, atol=0)


def test_every_node_dirichlet(sem):
    # the degenerate mask: the operator is zero and the solve returns x = 0 at once
    box, N = (2, 2, 1), 3
    ng = (2 * N + 1) * (2 * N + 1) * (N + 1)
    prob = _mask_problem(sem, np.ones(ng, dtype=np.uint8), box, N)
    u = torch.from_numpy(W.uniform(ng, seed=2)).cuda()
    assert float(prob.apply(u).abs().max()) == 0.0
    b = torch.zeros(ng, dtype=torch.float64, device="cuda")
    x, info = prob.pcg(b, rtol=1e-10, mode="fp64", apply_prec="fp64")
    assert info["status"] == "SEM_OK" and info["iterations"] == 0 and float(x.abs().max()) == 0.0
