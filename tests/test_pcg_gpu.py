"""Jacobi-PCG and mixed-precision refinement on the GPU, checked by the FP64 oracle.

The oracle recomputes the true relative residual ||b - A x|| / ||b|| of the GPU's x; the
iteration count of the FP64 solve must match the oracle's Jacobi-PCG within 2.
"""
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


def _problem(sem, orc, box, N, modes=None, seed=W.BASE_SEED, features=None):
    v = W.box_vertices(*box, seed=seed)
    feats = features or (sem.SEM_FEAT_FP64 | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG)
    prob = sem.Problem(N, v, box=box, kappa_modes=modes, bc="box", features=feats)
    b = prob.rhs(W.sine_forcing(prob.node_coords(), modes))
    G, wJ = orc.factors(N, v, modes=modes)
    glo = orc.box_numbering(*box, N)
    mask = orc.box_dirichlet(*box, N)
    return prob, b, G, glo, mask, v


def test_c1_fp64_pcg_matches_oracle(sem, orc):
    # 4^3 elements, N=7, manufactured u = sin sin sin, homogeneous Dirichlet, rtol 1e-10
    box, N = (4, 4, 4), 7
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N)
    x, info = prob.pcg(b, rtol=1e-10, mode="fp64", apply_prec="fp64")
    bh = b.cpu().numpy()
    rel = orc.true_relres(N, glo, G, bh, x.cpu().numpy(), mask=mask)
    assert rel <= 1e-10, info
    dg = orc.diag(N, glo, G, prob.nglobal, mask=mask)
    xo, it_o, _ = orc.pcg(N, glo, G, bh, dg, mask=mask, rtol=1e-10)
    assert abs(info["iterations"] - it_o) <= 2, (info, it_o)
    assert np.max(np.abs(x.cpu().numpy() - xo)) < 1e-8 * np.max(np.abs(xo))
    # discretisation error against the manufactured solution
    xyz = np.zeros((prob.nglobal, 3))
    xyz[glo.reshape(-1)] = orc.node_coords(N, v).reshape(-1, 3)
    assert np.max(np.abs(x.cpu().numpy() - W.sine_solution(xyz))) < 1e-4


def test_graph_and_eager_agree(sem, orc):
    # CUDA-graph replay and eager launches run the same kernels; the dot products reduce in a
    # fixed order, but the scatter-add uses atomics, so iterates agree to rounding, not bitwise.
    box, N = (3, 3, 2), 5
    prob, b, *_ = _problem(sem, orc, box, N, modes=W.kappa_modes(16, seed=3))
    x1, i1 = prob.pcg(b, rtol=1e-10, use_graph=True, check_every=7)
    x2, i2 = prob.pcg(b, rtol=1e-10, use_graph=False, check_every=3)
    assert abs(i1["iterations"] - i2["iterations"]) <= 1
    assert float((x1 - x2).abs().max()) < 1e-9 * float(x2.abs().max())
    assert i1["true_relres"] <= 1e-10 and i2["true_relres"] <= 1e-10


def test_ir_reaches_fp64_accuracy(sem, orc):
    box, N = (4, 3, 3), 7
    modes = W.kappa_modes(16, amplitude=0.25, seed=W.BASE_SEED + 2)
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N, modes=modes)
    x, info = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64", inner_rtol=1e-4)
    rel = orc.true_relres(N, glo, G, b.cpu().numpy(), x.cpu().numpy(), mask=mask)
    assert rel <= 1e-10, info
    assert info["outer"] >= 2


def test_ir_outer_steps_match_oracle_ir(sem, orc):
    # the GPU refinement (FP32 factors and arithmetic inside) against the oracle's plainly written
    # refinement (FP32 inner Jacobi-PCG around the FP64 operator): same number of outer steps
    from oracle import solvers

    box, N = (3, 3, 2), 5
    modes = W.kappa_modes(16, amplitude=0.25, seed=W.BASE_SEED + 5)
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N, modes=modes)
    x, info = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64", inner_rtol=1e-3)
    dg = orc.diag(N, glo, G, prob.nglobal, mask=mask)
    xo, outer, inner, hist = solvers.ir(N, glo, G, b.cpu().numpy(), dg, mask=mask, rtol=1e-10, inner_rtol=1e-3)
    assert abs(info["outer"] - outer) <= 1, (info, outer, hist)
    assert orc.true_relres(N, glo, G, b.cpu().numpy(), x.cpu().numpy(), mask=mask) <= 1e-10
    assert np.max(np.abs(x.cpu().numpy() - xo)) < 1e-8 * np.max(np.abs(xo))


def test_fcg_with_untrained_network_matches_oracle_fcg(sem, orc):
    # a network with zero parameters adds nothing to the Jacobi base, so the GPU's flexible CG is
    # flexible CG with z = D^-1 r: its iteration count matches the oracle's flexible CG
    from oracle import solvers
    from paper_1403_0968_gb300 import learn

    box, N = (3, 3, 3), 3
    feats = sem.SEM_FEAT_EMU | sem.SEM_FEAT_PCG | sem.SEM_FEAT_MLP
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N, modes=W.kappa_modes(8, seed=12), features=feats)
    prob.mlp_load(torch.zeros(learn.he_init(N, seed=0).shape, dtype=torch.float32, device="cuda"), jacobi_base=True)
    x, info = prob.pcg(b, rtol=1e-10, mode="fcg_mlp", apply_prec="fp64_emu")
    dg = orc.diag(N, glo, G, prob.nglobal, mask=mask)
    dinv = np.where(mask == 0, 1.0 / dg, 0.0)
    xo, k, fb = solvers.fcg(N, glo, G, b.cpu().numpy(), dg, lambda r, it: dinv * r, mask=mask, rtol=1e-10)
    assert info["fallbacks"] == 0 and fb == 0
    assert abs(info["iterations"] - k) <= 2, (info, k)
    assert np.max(np.abs(x.cpu().numpy() - xo)) < 1e-8 * np.max(np.abs(xo))


def test_noconv_reported(sem, orc):
    prob, b, *_ = _problem(sem, orc, (3, 3, 3), 5)
    x, info = prob.pcg(b, rtol=1e-10, max_it=3, raise_on_error=False)
    assert info["status"] == "SEM_ERR_NOCONV"
    assert info["iterations"] == 3


def test_zero_rhs_returns_zero(sem, orc):
    prob, b, *_ = _problem(sem, orc, (2, 2, 2), 3)
    x, info = prob.pcg(torch.zeros_like(b), rtol=1e-10)
    assert info["iterations"] == 0 and float(x.abs().max()) == 0.0


def test_dot_deterministic_and_accurate(sem, orc):
    prob, *_ = _problem(sem, orc, (5, 4, 3), 6, features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_PCG)
    x = torch.from_numpy(W.uniform(prob.nglobal, seed=1)).cuda()
    y = torch.from_numpy(W.uniform(prob.nglobal, seed=2)).cuda()
    d1 = prob.dot(x, y)
    d2 = prob.dot(x, y)
    assert torch.equal(d1, d2)
    ref = float(np.dot(x.cpu().numpy().astype(np.longdouble), y.cpu().numpy().astype(np.longdouble)))
    assert abs(float(d1.item()) - ref) < 1e-13 * float(np.sum(np.abs(x.cpu().numpy() * y.cpu().numpy())))


def test_fp64_pcg_with_emulated_apply(sem, orc):
    box, N = (4, 4, 4), 7
    feats = sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N, features=feats)
    x, info = prob.pcg(b, rtol=1e-10, mode="fp64", apply_prec="fp64_emu")
    assert orc.true_relres(N, glo, G, b.cpu().numpy(), x.cpu().numpy(), mask=mask) <= 1e-10, info
    x2, info2 = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64_emu")
    assert orc.true_relres(N, glo, G, b.cpu().numpy(), x2.cpu().numpy(), mask=mask) <= 1e-10, info2


def test_fp64_pcg_with_tensor_core_apply(sem, orc):
    # Jacobi-PCG whose FP64-accurate apply runs the D-contractions on the tensor cores (variant 5,
    # order 7) with the fused p^T A p of that kernel: same iterations as the oracle's PCG
    box, N = (4, 4, 4), 7
    feats = sem.SEM_FEAT_EMU | sem.SEM_FEAT_PCG
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N, features=feats)
    prob.set_apply_variant(5)
    x, info = prob.pcg(b, rtol=1e-10, mode="fp64", apply_prec="fp64_emu")
    bh = b.cpu().numpy()
    assert orc.true_relres(N, glo, G, bh, x.cpu().numpy(), mask=mask) <= 1e-10, info
    dg = orc.diag(N, glo, G, prob.nglobal, mask=mask)
    _, it_o, _ = orc.pcg(N, glo, G, bh, dg, mask=mask, rtol=1e-10)
    assert abs(info["iterations"] - it_o) <= 2, (info, it_o)


def test_ir_with_tensor_core_inner_apply_reaches_fp64_accuracy(sem, orc):
    # refinement whose inner FP32 Jacobi-PCG applies the operator on the tensor cores (3xTF32,
    # variant 5 at order 7; the outer FP64-accurate residual then also runs on the tensor cores):
    # the true residual reaches 1e-10 with about as many inner iterations as the CUDA-core inner
    # apply
    box, N = (4, 4, 4), 7
    feats = sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N, features=feats)
    x1, i1 = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64_emu", inner_rtol=1e-3)
    prob.set_apply_variant(5)
    x5, i5 = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64_emu", inner_rtol=1e-3)
    bh = b.cpu().numpy()
    assert orc.true_relres(N, glo, G, bh, x5.cpu().numpy(), mask=mask) <= 1e-10, i5
    assert i5["iterations"] <= 1.1 * i1["iterations"] + 5, (i5, i1)


def test_ir_with_bf16_inner_apply_reaches_fp64_accuracy(sem, orc):
    # refinement around an inner solve whose operator has BF16-rounded factors: the FP64-accurate
    # outer residual still drives the true residual to 1e-10
    box, N = (4, 4, 4), 7
    feats = sem.SEM_FEAT_EMU | sem.SEM_FEAT_BF16 | sem.SEM_FEAT_PCG
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N, features=feats)
    x, info = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64_emu", inner_rtol=1e-3, inner_prec="bf16")
    assert orc.true_relres(N, glo, G, b.cpu().numpy(), x.cpu().numpy(), mask=mask) <= 1e-10, info


def test_ir_with_on_the_fly_inner_apply_reaches_fp64_accuracy(sem, orc):
    # refinement whose inner FP32 solve recomputes the factors from the element map at every
    # apply (no stored FP32 factors): same FP64-accurate result, iteration count close to the
    # stored-factor inner solve
    box, N = (4, 4, 4), 7
    feats = sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_OTF | sem.SEM_FEAT_PCG
    prob, b, G, glo, mask, v = _problem(sem, orc, box, N, features=feats)
    x, info = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64_emu", inner_rtol=1e-3, inner_prec="fp32_otf")
    assert orc.true_relres(N, glo, G, b.cpu().numpy(), x.cpu().numpy(), mask=mask) <= 1e-10, info
    x2, info2 = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64_emu", inner_rtol=1e-3)
    assert abs(info["iterations"] - info2["iterations"]) <= max(4, info2["iterations"] // 20), (info, info2)


def test_full_size_mixed_precision_solve(sem, orc):
    # the 48^3-element, N = 7 variable-kappa solve of the benchmark: FP32-inner refinement with the
    # FP64-accurate outer residual, checked by the oracle's own FP64 residual on the full mesh
    box, N = (48, 48, 48), 7
    v = W.box_vertices(*box, seed=W.BASE_SEED + 3)
    modes = W.kappa_modes(16, amplitude=0.25, seed=W.BASE_SEED + 3)
    prob = sem.Problem(N, v, box=box, kappa_modes=modes, bc="box",
                       features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG)
    b = prob.rhs(W.sine_forcing(prob.node_coords(), modes))
    x, info = prob.pcg(b, rtol=1e-10, mode="ir", apply_prec="fp64_emu", inner_rtol=1e-3)
    assert info["status"] == "SEM_OK", info
    G, _ = orc.factors(N, v, modes=modes)
    glo, mask = orc.box_numbering(*box, N), orc.box_dirichlet(*box, N)
    assert orc.true_relres(N, glo, G, b.cpu().numpy(), x.cpu().numpy(), mask=mask) <= 1e-10, info
    del prob
    torch.cuda.empty_cache()


def test_residual_history(sem, orc):
    # the solve's residual history (sem_pcg_opts.history): one (iterations, relative residual) pair
    # per host check, from the initial residual (b itself from x0 = 0, relative residual 1) down to
    # the recursive residual the result reports; IR records the true residual of each refinement
    # step; a short array keeps the first pairs; a capacity without an array is refused
    from paper_1403_0968_gb300 import learn

    box, N = (3, 3, 3), 3
    feats = sem.SEM_FEAT_FP64 | sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG | sem.SEM_FEAT_MLP
    prob, b, *_ = _problem(sem, orc, box, N, modes=W.kappa_modes(8, seed=13), features=feats)
    prob.mlp_load(torch.zeros(learn.he_init(N, seed=0).shape, dtype=torch.float32, device="cuda"))
    for mode, prec in (("fp64", "fp64"), ("fcg_mlp", "fp64_emu"), ("ir", "fp64_emu")):
        x, info = prob.pcg(b, rtol=1e-10, mode=mode, apply_prec=prec, check_every=5, history=1000)
        h = info["history"]
        assert info["status"] == "SEM_OK" and len(h) >= 2, (mode, info)
        its = [k for k, _ in h]
        assert its[0] == 0 and abs(h[0][1] - 1.0) < 1e-12, (mode, h[0])
        assert all(a <= c for a, c in zip(its, its[1:])) and its[-1] == info["iterations"], (mode, its)
        assert h[-1][1] <= 1e-10, (mode, h[-1])
        if mode == "ir":
            assert len(h) == info["outer"] + 1 and h[-1][1] == info["recursive_relres"]
        elif mode == "fp64":
            assert h[-1][1] == info["recursive_relres"]
    x, info = prob.pcg(b, rtol=1e-10, mode="fp64", check_every=5, history=2)
    assert len(info["history"]) == 2 and info["status"] == "SEM_OK"
    o = sem.SemPcgOpts()
    o.rtol, o.max_it, o.mode, o.apply_prec, o.check_every = 1e-10, 100, sem.SEM_SOLVE_FP64, 0, 5
    o.history_cap = 3  # and no array
    with pytest.raises(sem.SemError):
        sem.sem_pcg(prob.handle, b, torch.zeros_like(b), o)
