"""Batched solves of independent problems of uneven size and order, checked by the FP64 oracle."""
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


def _problems(n=10, seed=11, smin=2, smax=4, orders=(2, 3, 5, 7)):
    g = W.rng(seed)
    out = []
    for k in range(n):
        s = int(g.integers(smin, smax + 1))
        N = int(orders[int(g.integers(0, len(orders)))])
        box = (s, s + (k % 2), s)
        modes = W.kappa_modes(8, amplitude=0.2, seed=seed + k) if k % 3 == 0 else None
        out.append({"N": N, "box": box, "vertices": W.box_vertices(*box, seed=seed + 100 + k), "kappa_modes": modes})
    return out


def _oracle(orc, pr):
    N, box = pr["N"], pr["box"]
    G, wJ = orc.factors(N, pr["vertices"], modes=pr["kappa_modes"])
    return G, wJ, orc.box_numbering(*box, N), orc.box_dirichlet(*box, N)


@pytest.mark.parametrize("inner,orders", [("fp32", (2, 3, 5, 7)), ("otf", (2, 3, 5, 7)), ("otf", (9, 11)),
                                          ("fp32", (9, 11))])
def test_batched_apply_matches_oracle(sem, orc, inner, orders):
    # the FP32 batched apply with stored factors, or recomputed from each element's map when the
    # batch holds only the map coefficients (SEM_FEAT_OTF)
    probs = _problems(orders=orders)
    feats = sem.SEM_FEAT_EMU | (sem.SEM_FEAT_FP32 if inner == "fp32" else sem.SEM_FEAT_OTF)
    B = sem.Batch(probs, features=feats)
    u = torch.from_numpy(W.uniform(B.nglobal, seed=3)).cuda()
    y32 = B.apply(u.float(), torch.empty(B.nglobal, dtype=torch.float32, device="cuda"), prec="fp32")
    yem = B.apply(u, torch.empty_like(u), prec="fp64_emu")
    uh, y32h, yemh = u.cpu().numpy(), y32.double().cpu().numpy(), yem.cpu().numpy()
    for p, pr in enumerate(probs):
        G, wJ, glo, mask = _oracle(orc, pr)
        sl = slice(B.offsets[p], B.offsets[p] + B.sizes[p])
        yo = orc.apply(pr["N"], glo, G, uh[sl], mask=mask)
        sc = np.max(np.abs(yo))
        assert np.max(np.abs(y32h[sl] - yo)) < 1e-5 * sc, p
        assert np.max(np.abs(yemh[sl] - yo)) < 1e-12 * sc, p


@pytest.mark.parametrize("variant,inner", [(1, "fp32"), (2, "fp32"), (1, "otf")])
def test_batched_solve_reaches_fp64_accuracy(sem, orc, variant, inner):
    probs = _problems(n=12, seed=21)
    feats = sem.SEM_FEAT_EMU | (sem.SEM_FEAT_FP32 if inner == "fp32" else sem.SEM_FEAT_OTF)
    B = sem.Batch(probs, features=feats)
    for N in B.orders:
        B.set_variant(N, variant)
    fL = torch.cat([W.sine_forcing(B.node_coords(p), probs[p]["kappa_modes"]) for p in range(B.nprob)])
    b = B.rhs(fL)
    x, res, status = B.pcg(b, rtol=1e-10, check_every=8)
    assert status == "SEM_OK", res
    bh, xh = b.cpu().numpy(), x.cpu().numpy()
    for p, pr in enumerate(probs):
        G, wJ, glo, mask = _oracle(orc, pr)
        sl = slice(B.offsets[p], B.offsets[p] + B.sizes[p])
        rel = orc.true_relres(pr["N"], glo, G, bh[sl], xh[sl], mask=mask)
        assert rel <= 1e-10, (p, rel, res[p])
        assert res[p]["outer"] >= 1 and res[p]["true_relres"] <= 1e-10


def test_fused_step_matches_multi_launch(sem, orc):
    # orders 3, 5, 7, 9, 11 with stored FP32 factors: each inner step is one persistent cooperative
    # launch (batched apply of all orders, updates, per-problem scalars, separated by bounded
    # grid-wide barriers); the same solve with one launch per order group and four vector kernels
    # per step gives the same iterates to rounding, and both meet the oracle's FP64 residual
    probs = _problems(n=10, seed=51, smin=2, smax=3, orders=(3, 5, 7, 9, 11))
    B = sem.Batch(probs, features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32)
    fL = torch.cat([W.sine_forcing(B.node_coords(p), probs[p]["kappa_modes"]) for p in range(B.nprob)])
    b = B.rhs(fL)
    xf, rf, sf = B.pcg(b, rtol=1e-11, check_every=8)
    xm, rm, sm = B.pcg(b, rtol=1e-11, check_every=8, multi_launch=True)
    assert sf == "SEM_OK" and sm == "SEM_OK", (rf, rm)
    bh, xfh = b.cpu().numpy(), xf.cpu().numpy()
    for p, pr in enumerate(probs):
        # FP32 inner solves stopped at inner_rtol: a different summation order moves each inner
        # solve's stopping step by a few iterations
        assert abs(rf[p]["iterations"] - rm[p]["iterations"]) <= max(3 * rm[p]["outer"], rm[p]["iterations"] // 20), \
            (p, rf[p], rm[p])
        G, wJ, glo, mask = _oracle(orc, pr)
        sl = slice(B.offsets[p], B.offsets[p] + B.sizes[p])
        assert orc.true_relres(pr["N"], glo, G, bh[sl], xfh[sl], mask=mask) <= 1e-11, (p, rf[p])
    # both residuals are below 1e-11 ||b||: the two solutions agree to the condition number times that
    assert float((xf - xm).abs().max()) < 1e-7 * float(xm.abs().max())


@pytest.mark.parametrize("multi_launch", [False, True])
def test_problem_finished_before_the_first_step(sem, orc, multi_launch):
    # one problem with a zero right-hand side is finished at the first residual check: the inner
    # steps launch over the other problems only (entry tables and chunk list rebuilt), its x stays
    # exactly zero, and the others reach the oracle's 1e-10
    probs = _problems(n=5, seed=81, smin=2, smax=3, orders=(3, 5, 7))
    B = sem.Batch(probs, features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32)
    fL = torch.cat([W.sine_forcing(B.node_coords(p), probs[p]["kappa_modes"]) for p in range(B.nprob)])
    b = B.rhs(fL)
    z = 2
    b[B.offsets[z]:B.offsets[z] + B.sizes[z]] = 0.0
    x, res, status = B.pcg(b, rtol=1e-10, check_every=4, multi_launch=multi_launch)
    assert status == "SEM_OK", res
    assert res[z]["iterations"] == 0 and float(x[B.offsets[z]:B.offsets[z] + B.sizes[z]].abs().max()) == 0.0
    bh, xh = b.cpu().numpy(), x.cpu().numpy()
    for p, pr in enumerate(probs):
        if p == z:
            continue
        G, wJ, glo, mask = _oracle(orc, pr)
        sl = slice(B.offsets[p], B.offsets[p] + B.sizes[p])
        assert orc.true_relres(pr["N"], glo, G, bh[sl], xh[sl], mask=mask) <= 1e-10, (p, res[p])


def test_fused_step_timeout_reported_and_cleared(sem, orc):
    # a grid-wide wait told to give up at once: the fused step's blocks leave, the solve returns
    # SEM_ERR_TIMEOUT with no hang; with the default limit the same batch then solves normally
    probs = _problems(n=6, seed=61, smin=2, smax=3, orders=(3, 5, 7))
    B = sem.Batch(probs, features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32)
    fL = torch.cat([W.sine_forcing(B.node_coords(p), probs[p]["kappa_modes"]) for p in range(B.nprob)])
    b = B.rhs(fL)
    B.set_wait_limit(0)
    _, _, status = B.pcg(b, rtol=1e-10, check_every=4)
    assert status == "SEM_ERR_TIMEOUT"
    B.set_wait_limit(-1)
    x, res, status = B.pcg(b, rtol=1e-10, check_every=4)
    assert status == "SEM_OK", res
    assert max(r["true_relres"] for r in res) <= 1e-10


def test_batched_solve_matches_single_problem_solves(sem, orc):
    # the same problems solved one by one with the single-problem refinement give the same x
    probs = _problems(n=4, seed=31, orders=(3, 5))
    B = sem.Batch(probs)
    fL = torch.cat([W.sine_forcing(B.node_coords(p), probs[p]["kappa_modes"]) for p in range(B.nprob)])
    b = B.rhs(fL)
    xb, res, status = B.pcg(b, rtol=1e-11, use_graph=False)
    assert status == "SEM_OK"
    for p, pr in enumerate(probs):
        single = sem.Problem(pr["N"], pr["vertices"], box=pr["box"], kappa_modes=pr["kappa_modes"], bc="box",
                             features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG)
        sl = slice(B.offsets[p], B.offsets[p] + B.sizes[p])
        xs, info = single.pcg(b[sl].contiguous(), rtol=1e-11, mode="ir", apply_prec="fp64_emu")
        assert float((xs - xb[sl]).abs().max()) < 1e-8 * float(xs.abs().max())


def test_autotuner_persists_choices(sem, tmp_path, monkeypatch):
    from paper_1403_0968_gb300 import autotune

    monkeypatch.setenv("SEM_AUTOTUNE_TABLE", str(tmp_path / "tune.json"))
    probs = _problems(n=6, seed=41)
    B = sem.Batch(probs)
    chosen = autotune.tune_batch(B, reps=2)
    assert set(chosen) == set(B.orders) and all(v in (1, 2) for v in chosen.values())
    again = autotune.tune_batch(B, reps=2)  # served from the table
    assert again == chosen
    box = (4, 4, 4)
    P = sem.Problem(5, W.box_vertices(*box), box=box, features=sem.SEM_FEAT_FP32)
    v = autotune.tune_problem(P, "fp32", reps=2)
    assert v in (0, 1, 2, 3)
    import json

    tab = json.load(open(tmp_path / "tune.json"))
    assert any(k.startswith("problem/fp32/N5") for k in tab) and any(k.startswith("batch/fp32") for k in tab)


def test_step_form_choice(sem, tmp_path, monkeypatch):
    # the fused step exists for stored FP32 factors at orders 3..11 only; the autotuner times both
    # step forms, keeps the faster, and serves it from its table afterwards
    from paper_1403_0968_gb300 import autotune

    monkeypatch.setenv("SEM_AUTOTUNE_TABLE", str(tmp_path / "tune.json"))
    B = sem.Batch(_problems(n=6, seed=71, orders=(3, 5, 7)))
    assert B.fused_state() == (True, True)
    chosen = autotune.tune_batch(B, reps=2)
    assert chosen["fused"] in (True, False) and B.fused_state() == (True, chosen["fused"])
    B.set_fused(not chosen["fused"])
    assert autotune.tune_batch(B, reps=2) == chosen and B.fused_state()[1] == chosen["fused"]
    otf = sem.Batch(_problems(n=3, seed=72, orders=(3, 5)), features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_OTF)
    assert otf.fused_state() == (False, False)
    with pytest.raises(sem.SemError) as ei:
        otf.set_fused(True)
    assert ei.value.status == sem.SEM_ERR_INVALID
    otf.set_fused(False)  # the per-order-group launches are always available


def test_c4_full_size_sampled(sem, orc):
    # the batched workload at its stated size (256 problems, sides 8..32 elements, orders 3..11:
    # 2.34e9 local DOFs, the inner factors recomputed on the fly so that it fits in HBM), in the
    # launch configuration of the batched solve: the FP32 inner apply and the FP64 residual apply
    # on random u, checked against the oracle on sampled problems (the smallest of each order and
    # one of median size)
    plist = W.batch_problems(nprob=256, smin=8, smax=32)
    probs = [{"N": q.N, "box": (q.sx, q.sy, q.sz), "vertices": W.box_vertices(q.sx, q.sy, q.sz, seed=q.seed)}
             for q in plist]
    B = sem.Batch(probs, features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_OTF)
    assert sum(B.nlocal) == sum(q.sx * q.sy * q.sz * (q.N + 1) ** 3 for q in plist)
    g = torch.Generator(device="cuda").manual_seed(W.BASE_SEED + 44)
    u = torch.rand(B.nglobal, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
    y64 = B.apply(u, torch.empty_like(u), prec="fp64")
    u32 = u.float()
    y32 = B.apply(u32, torch.empty_like(u32), prec="fp32")
    picks = {}
    for p, q in enumerate(plist):
        if q.N not in picks or q.sx < plist[picks[q.N]].sx:
            picks[q.N] = p
    by_size = sorted(range(len(plist)), key=lambda p: plist[p].sx)
    for p in sorted(set(picks.values()) | {by_size[len(by_size) // 2]}):
        pr = probs[p]
        G, wJ, glo, mask = _oracle(orc, {"N": pr["N"], "box": pr["box"], "vertices": pr["vertices"],
                                         "kappa_modes": None})
        sl = slice(B.offsets[p], B.offsets[p] + B.sizes[p])
        uh = u[sl].cpu().numpy()
        yo = orc.apply(pr["N"], glo, G, uh, mask=mask)
        sc = np.max(np.abs(yo))
        assert np.max(np.abs(y64[sl].cpu().numpy() - yo)) < 1e-12 * sc, (p, pr["N"], pr["box"])
        yo32 = orc.apply(pr["N"], glo, G, u32[sl].double().cpu().numpy(), mask=mask)
        assert np.max(np.abs(y32[sl].double().cpu().numpy() - yo32)) < 1e-5 * sc, (p, pr["N"], pr["box"])
    del B, u, y64, u32, y32
    torch.cuda.empty_cache()
