"""The learned element preconditioner on the GPU against the FP64 reference (oracle/mlp.py)."""
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


def _bf16_round(x):
    """Round-to-nearest-even FP32 -> BF16 -> FP32, written out on the bit pattern."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def test_forward_and_gradients_match_oracle(sem):
    from oracle import mlp

    from paper_1403_0968_gb300 import learn

    N = 3
    n3 = 64
    lay = mlp.layout(n3, sem.MLP_H1, sem.MLP_H2)
    p = learn.he_init(N, seed=3)
    g = W.rng(4)
    X = g.normal(size=(300, n3 + 6)).astype(np.float32)
    T = g.normal(size=(300, n3)).astype(np.float32)
    pd, Xd, Td = (torch.from_numpy(a).cuda() for a in (p, X, T))
    _, _, O = sem.mlp_forward(N, pd, Xd)
    _, _, Oo = mlp.forward(p, X, lay)
    assert np.max(np.abs(O.cpu().numpy() - Oo)) < 1e-5 * np.max(np.abs(Oo))
    tr = sem.MlpTrainer(N, pd.clone(), 300)
    grad = torch.empty_like(pd)
    loss = tr.step(Xd, Td, lr=0.0, grad_out=grad)
    lo, go = mlp.loss_and_grad(p, X, T, lay)
    assert abs(float(loss.item()) - lo) < 1e-5 * lo
    assert np.max(np.abs(grad.cpu().numpy() - go)) < 1e-4 * np.max(np.abs(go))
    # one Adam step
    tr2 = sem.MlpTrainer(N, pd.clone(), 300, lr=1e-3)
    tr2.step(Xd, Td)
    p1, _, _ = mlp.adam(p.astype(np.float64), go, np.zeros_like(go), np.zeros_like(go), 1, 1e-3)
    got = tr2.params.cpu().numpy().astype(np.float64)
    # where the gradient is resolved in FP32 the update matches; a first Adam step never moves a
    # parameter by more than lr (components with |g| near eps amplify FP32 gradient rounding)
    big = np.abs(go) > 1e-4 * np.max(np.abs(go))
    assert np.max(np.abs(got - p1)[big]) < 2e-6
    assert np.max(np.abs(got - p)) <= 1e-3 * (1 + 1e-5)


def _elem_mats(orc, N, v, modes, elems):
    """Dense element operators A_e (the oracle's brute-force weak form) of the given elements."""
    xyz = orc.node_coords(N, v)
    return [orc.element_matrix(N, v[e], kappa_e=orc.kappa(modes, xyz[e])) for e in elems]


def _precond_case(sem, orc, explicit):
    from oracle import mlp

    from paper_1403_0968_gb300 import learn

    box, N = (3, 3, 2), 3
    modes = W.kappa_modes(8, seed=5)
    v = W.box_vertices(*box, seed=6)
    glo, mask = orc.box_numbering(*box, N), orc.box_dirichlet(*box, N)
    ng = orc.box_nglobal(*box, N)
    if explicit:  # the box under a permutation of global ids, Dirichlet set as flags: scatter path
        perm = W.rng(11).permutation(ng)
        glo_p, mask_p = perm[glo], np.zeros(ng, dtype=np.uint8)
        mask_p[perm] = mask
        glo, mask = glo_p, mask_p
        P = sem.Problem(N, v, box=box, glo_num=glo, nglobal=ng, kappa_modes=modes, bc="mask", dirichlet=mask,
                        features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_PCG | sem.SEM_FEAT_MLP)
    else:
        P = sem.Problem(N, v, box=box, kappa_modes=modes, bc="box",
                        features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_PCG | sem.SEM_FEAT_MLP)
    G, wJ = orc.factors(N, v, modes=modes)
    geo = mlp.geo6(G)
    r = W.uniform(ng, seed=7)
    A = _elem_mats(orc, N, v, modes, range(glo.shape[0]))
    return P, N, glo, mask, ng, G, wJ, geo, r, A, learn


@pytest.mark.parametrize("explicit,jacobi_base", [(False, True), (True, True), (False, False), (True, False)])
def test_samples_and_precond_match_oracle(sem, orc, explicit, jacobi_base):
    from oracle import mlp

    P, N, glo, mask, ng, G, wJ, geo, r, A, learn = _precond_case(sem, orc, explicit)
    dinv = np.where(mask != 0, 0.0, 1.0 / orc.diag(N, glo, G, ng, mask=mask)) if jacobi_base else None
    elems = np.array([0, 5, 17, 3], dtype=np.int32)
    X, T, its = P.mlp_samples(torch.from_numpy(r).cuda(), torch.from_numpy(elems).cuda(), eps=1e-2,
                              jacobi_base=jacobi_base)
    Xo, To = mlp.pairs([A[e] for e in elems], wJ, glo, mask, r, geo, elems, 1e-2, ng, dinv=dinv)
    np.testing.assert_allclose(X.cpu().numpy(), Xo, atol=2e-7 * np.max(np.abs(Xo)) + 1e-7)
    # the element solves run to 1e-10 in FP64 and are stored in FP32
    assert np.max(np.abs(T.cpu().numpy() - To)) <= 1e-6 * np.max(np.abs(To))
    assert 0 < int(its.item()) < 2000
    p = learn.he_init(N, seed=10)
    P.mlp_load(torch.from_numpy(p).cuda(), jacobi_base=jacobi_base)
    z = P.mlp_precond(torch.from_numpy(r).cuda()).cpu().numpy()
    dbar = np.array([np.trace(Ae) / Ae.shape[0] for Ae in A])
    zo = mlp.precond(_bf16_round(p).astype(np.float64), mlp.layout(64, 256, 256), glo, mask, r, geo, dbar, ng,
                     act_bf16=True, dinv=dinv)
    # The tensor cores sum in FP32, the oracle in FP64; both round every layer input to BF16.  An
    # activation whose FP32 and FP64 values round to neighbouring BF16 numbers (a few in 1e5 here)
    # moves the outputs it feeds by about one BF16 ulp (2^-8) of one term; elsewhere the two agree
    # to FP32 round-off.  A wrong layout or layer moves every output by the size of the outputs.
    err = np.abs(z - zo) / np.max(np.abs(zo))
    assert err.max() < 2e-3 and np.median(err) < 1e-5, (err.max(), np.median(err))
    assert np.all(z[mask != 0] == 0.0)


@pytest.mark.parametrize("N,box", [(3, (5, 5, 5)), (5, (4, 4, 9)), (7, (5, 5, 6)), (7, (16, 16, 16))])
def test_fused_layers_match_layer_by_layer(sem, N, box):
    # the three layers in one launch (activations kept in shared memory) against one launch per
    # layer: the same BF16 roundings and FP32 sums, so the same z; ragged last tiles of 128
    # elements (125, 144, 150 elements), one and two output halves (n^3 = 64, 216, 512), biases
    # nonzero so that every bias is read
    from paper_1403_0968_gb300 import learn

    n3 = (N + 1) ** 3
    P = sem.Problem(N, W.box_vertices(*box, seed=31), box=box, kappa_modes=W.kappa_modes(8, seed=32), bc="box",
                    features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_PCG | sem.SEM_FEAT_MLP)
    p = learn.he_init(N, seed=33)
    h = sem.MLP_H1
    nin = n3 + 6
    o1 = nin * h
    o2 = o1 + h + h * h
    o3 = o2 + h + h * n3
    g = W.rng(34)
    p[o1:o1 + h] = g.uniform(-0.2, 0.2, h)
    p[o2:o2 + h] = g.uniform(-0.2, 0.2, h)
    p[o3:o3 + n3] = g.uniform(-0.2, 0.2, n3)
    assert o3 + n3 == p.shape[0]
    P.mlp_load(torch.from_numpy(p).cuda())
    r = torch.from_numpy(W.uniform(P.nglobal, seed=35)).cuda()
    P.mlp_set_fused(True)
    zf = P.mlp_precond(r).cpu().numpy()
    P.mlp_set_fused(False)
    zu = P.mlp_precond(r).cpu().numpy()
    P.mlp_set_fused(True)
    assert np.all(np.isfinite(zf)) and np.max(np.abs(zu)) > 0
    # equal unless the tensor core's FP32 sums differ with the tile width, which can move one
    # hidden activation across a BF16 rounding boundary (one BF16 ulp of one term)
    err = np.abs(zf - zu) / np.max(np.abs(zu))
    assert np.array_equal(zf, zu) or (err.max() < 2e-3 and np.median(err) == 0.0), (err.max(), np.median(err))


def _field(k, N=5, s=5, contrast=30.0):
    box = (s, s, s)
    modes = W.contrast_modes(contrast, seed=W.BASE_SEED + 50 + k)
    return {"N": N, "box": box, "vertices": W.box_vertices(*box, seed=W.BASE_SEED + 60 + k), "kappa_modes": modes,
            "forcing": (lambda m: (lambda xyz: W.sine_forcing(xyz, m)))(modes)}


@pytest.mark.parametrize("jacobi_base", [True, False])
def test_trained_preconditioner_in_flexible_cg(sem, orc, jacobi_base):
    # what the trained network gains over the method without it: flexible CG with the learned
    # preconditioner against Jacobi-PCG on a held-out kappa field, both to the true 1e-10
    from paper_1403_0968_gb300 import learn

    train_fields = [_field(k) for k in range(32)]
    X, T = learn.generate_pairs(train_fields, per_field=2000, rhs_per_field=16, seed=1, jacobi_base=jacobi_base)
    params, hist = learn.train(5, X, T, epochs=20, batch=128, lr=1e-3, seed=2)
    assert hist[-1] < hist[0]  # the network learns
    test = _field(99)
    P = sem.Problem(test["N"], test["vertices"], box=test["box"], kappa_modes=test["kappa_modes"], bc="box",
                    features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG | sem.SEM_FEAT_MLP)
    b = P.rhs(test["forcing"](P.node_coords()))
    P.mlp_load(params, jacobi_base=jacobi_base)
    xf, info_f = P.pcg(b, rtol=1e-10, mode="fcg_mlp", apply_prec="fp64_emu")
    xj, info_j = P.pcg(b, rtol=1e-10, mode="fp64", apply_prec="fp64_emu")
    G, _ = orc.factors(test["N"], test["vertices"], modes=test["kappa_modes"])
    glo, mask = orc.box_numbering(*test["box"], test["N"]), orc.box_dirichlet(*test["box"], test["N"])
    assert orc.true_relres(test["N"], glo, G, b.cpu().numpy(), xf.cpu().numpy(), mask=mask) <= 1e-10, info_f
    print(f"\nlearned FCG (Jacobi base {jacobi_base}): {info_f['iterations']} its ({info_f['fallbacks']} fallbacks); "
          f"Jacobi-PCG: {info_j['iterations']} its; training loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    if jacobi_base:  # the default form must gain
        assert info_f["iterations"] < info_j["iterations"], (info_f, info_j)


def test_rejected_corrections_fall_back_to_jacobi(sem, orc):
    # a network whose correction is a large negative multiple of the residual makes z.r < 0:
    # every iteration must fall back to Jacobi and the solve must still converge
    from paper_1403_0968_gb300 import learn

    N = 3
    test = _field(7, N=N, s=4)
    P = sem.Problem(N, test["vertices"], box=test["box"], kappa_modes=test["kappa_modes"], bc="box",
                    features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_PCG | sem.SEM_FEAT_MLP)
    p = np.zeros_like(learn.he_init(N, seed=0))
    n3 = 64
    from oracle import mlp

    lay = mlp.layout(n3, 256, 256)
    W1 = np.zeros((n3 + 6, 256), dtype=np.float32)
    W1[np.arange(n3), np.arange(n3)] = 1.0          # H1[:n3] = relu(r_hat)
    W1[np.arange(n3), 64 + np.arange(n3)] = -1.0    # H1[64:128] = relu(-r_hat)
    W2 = np.zeros((256, 256), dtype=np.float32)
    W2[np.arange(128), np.arange(128)] = 1.0
    W3 = np.zeros((256, n3), dtype=np.float32)
    W3[np.arange(n3), np.arange(n3)] = -1e4         # O = 1e4 (-relu(r) + relu(-r)) = -1e4 r_hat,
    W3[64 + np.arange(n3), np.arange(n3)] = 1e4     # so z is a negative multiple of r: z.r < 0
    for name, arr in (("W1", W1), ("W2", W2), ("W3", W3)):
        off, sz = lay[name]
        p[off:off + sz] = arr.ravel()
    P.mlp_load(torch.from_numpy(p).cuda(), jacobi_base=False)
    b = P.rhs(test["forcing"](P.node_coords()))
    x, info = P.pcg(b, rtol=1e-10, mode="fcg_mlp", apply_prec="fp64_emu")
    assert info["status"] == "SEM_OK" and info["fallbacks"] == info["iterations"], info


def test_resume_from_checkpoint_continues_adam(sem, tmp_path):
    # training resumed from a checkpoint (weights, Adam moments, step count) takes the same next
    # step as training that never stopped; a checkpoint of the weights alone restarts Adam and
    # takes a different one
    from paper_1403_0968_gb300 import learn

    N, batch = 3, 128
    n3, nin = (N + 1) ** 3, (N + 1) ** 3 + 6
    g = np.random.default_rng(7)
    X = torch.from_numpy(g.standard_normal((4 * batch, nin)).astype(np.float32)).cuda()
    T = torch.from_numpy((0.1 * g.standard_normal((4 * batch, n3))).astype(np.float32)).cuda()
    a = sem.MlpTrainer(N, torch.from_numpy(learn.he_init(N, seed=8)).cuda(), batch, lr=1e-3)
    for i in range(3):
        a.step(X[i * batch:(i + 1) * batch], T[i * batch:(i + 1) * batch])
    f = tmp_path / "ck.npz"
    learn.save_checkpoint(f, N, a.params, trainer=a)
    ck = learn.load_checkpoint(f)
    b = learn.resume_trainer(ck, batch)
    c = learn.resume_trainer({k: v for k, v in ck.items() if k not in ("m", "v", "step", "lr")}, batch)
    assert b.step_count == 3 and c.step_count == 0
    for tr in (a, b, c):
        tr.step(X[3 * batch:], T[3 * batch:])
    torch.cuda.synchronize()
    scale = float(a.params.abs().max())
    assert float((a.params - b.params).abs().max()) <= 1e-7 * scale
    assert float((a.m - b.m).abs().max()) <= 1e-7 * float(a.m.abs().max())
    assert float((a.params - c.params).abs().max()) > 1e-5 * scale
