"""Parity of the CUDA operator apply (through the C ABI) against the FP64 oracle.

Tolerances (relative max-norm ||y - y*||_inf / ||y*||_inf): FP64 1e-12, FP32 1e-5 (stored FP32
factors, or factors recomputed in FP32 from the element map: SEM_FP32_OTF).
Integer outputs (numbering) are compared bit for bit.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp64_emu": 1e-12, "fp32_otf": 1e-5}
F32 = ("fp32", "bf16", "fp32_otf")  # precisions that apply to float32 vectors


@pytest.fixture(scope="module")
def sem():
    from paper_1403_0968_gb300 import build

    build.build()
    import paper_1403_0968_gb300 as sem

    sem.lib()
    return sem


def relerr(y, yo):
    return float(np.max(np.abs(y - yo)) / max(np.max(np.abs(yo)), 1e-300))


def _setup(sem, orc, box, N, seed=1, modes=None, alpha=False, bc="box", perturb=0.1, features=None):
    v = W.box_vertices(*box, seed=seed, perturb=perturb)
    E = v.shape[0]
    n3 = (N + 1) ** 3
    al = (0.5 + W.uniform(E * n3, seed=seed + 7, lo=0, hi=1)).reshape(E, n3) if alpha else None
    feats = features if features is not None else (sem.SEM_FEAT_FP64 | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_EMU |
                                                   sem.SEM_FEAT_OTF)
    prob = sem.Problem(N, v, box=box, kappa_modes=modes, alpha=al, bc=bc, features=feats)
    G, wJ = orc.factors(N, v, modes=modes)
    glo = orc.box_numbering(*box, N)
    mask = orc.box_dirichlet(*box, N) if bc == "box" else None
    return prob, v, G, wJ, glo, mask, (None if al is None else al * wJ)


def _apply(prob, u, prec):
    import torch

    dt = torch.float32 if prec in F32 else torch.float64
    y = prob.apply(torch.from_numpy(u).to(dt).cuda(), prec=prec)
    return y.double().cpu().numpy()


CASES = [((1, 1, 1), 1), ((2, 2, 2), 1), ((3, 2, 2), 2), ((3, 2, 1), 3), ((2, 3, 2), 4), ((3, 3, 2), 5),
         ((2, 2, 3), 6), ((4, 4, 4), 7), ((3, 1, 2), 8), ((2, 2, 2), 9), ((1, 2, 2), 11), ((2, 1, 2), 12),
         ((1, 2, 1), 13), ((2, 1, 1), 14), ((2, 1, 1), 15)]


@pytest.mark.parametrize("box,N", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp64_emu", "fp32_otf"])
def test_apply_matches_oracle(sem, orc, box, N, prec):
    modes = W.kappa_modes(16, seed=N + 40)
    prob, v, G, wJ, glo, mask, wJa = _setup(sem, orc, box, N, seed=N, modes=modes, alpha=True)
    u = W.uniform(prob.nglobal, seed=100 + N)
    y = _apply(prob, u, prec)
    yo = orc.apply(N, glo, G, u, mask=mask, wJalpha=wJa)
    assert relerr(y, yo) < TOL[prec]
    assert np.all(y[mask.astype(bool)] == 0.0)


@pytest.mark.parametrize("N", [1, 3, 7])
def test_neumann_constant_nullspace(sem, orc, N):
    prob, *_ = _setup(sem, orc, (3, 2, 2), N, bc="none")
    ones = np.ones(prob.nglobal)
    y1 = _apply(prob, ones, "fp64")
    yr = _apply(prob, W.uniform(prob.nglobal, seed=3), "fp64")
    assert np.max(np.abs(y1)) < 1e-13 * N * N * np.max(np.abs(yr))


def test_symmetry_on_gpu(sem, orc):
    prob, *_ = _setup(sem, orc, (3, 2, 2), 6, modes=W.kappa_modes(8, seed=2), alpha=True)
    u, w = W.uniform(prob.nglobal, seed=1), W.uniform(prob.nglobal, seed=2)
    a = np.dot(w, _apply(prob, u, "fp64"))
    b = np.dot(u, _apply(prob, w, "fp64"))
    assert abs(a - b) < 1e-13 * abs(a)


@pytest.mark.parametrize("box,N", [((3, 2, 2), 4), ((2, 1, 2), 7), ((2, 1, 1), 13)])
def test_explicit_numbering_and_mask(sem, orc, box, N):
    # unstructured path: the box numbering under a random permutation of global ids, given as
    # glo_num, with the Dirichlet set given as a flag array (N = 7 and 13 take the kernels' loop
    # over the three directions)
    v = W.box_vertices(*box, seed=3)
    glo = orc.box_numbering(*box, N)
    ng = orc.box_nglobal(*box, N)
    perm = W.rng(5).permutation(ng)
    glo_p = perm[glo]
    mask_p = np.zeros(ng, dtype=np.uint8)
    mask_p[perm] = orc.box_dirichlet(*box, N)
    modes = W.kappa_modes(16, seed=9)
    prob = sem.Problem(N, v, box=box, glo_num=glo_p, nglobal=ng, kappa_modes=modes, bc="mask", dirichlet=mask_p,
                       features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_EMU | sem.SEM_FEAT_OTF)
    assert np.array_equal(prob.glo_num().cpu().numpy(), glo_p)
    G, _ = orc.factors(N, v, modes=modes)
    u = W.uniform(ng, seed=4)
    for prec in ("fp64", "fp32", "fp64_emu", "fp32_otf"):
        assert relerr(_apply(prob, u, prec), orc.apply(N, glo_p, G, u, mask=mask_p)) < TOL[prec]


def test_numbering_coords_diag_rhs(sem, orc):
    box, N = (3, 2, 4), 5
    modes = W.kappa_modes(16, seed=11)
    prob, v, G, wJ, glo, mask, _ = _setup(sem, orc, box, N, modes=modes, features=sem.SEM_FEAT_FP64)
    assert np.array_equal(prob.glo_num().cpu().numpy(), glo)
    xyz = prob.node_coords()
    np.testing.assert_allclose(xyz.cpu().numpy(), orc.node_coords(N, v), rtol=0, atol=1e-15)
    d = prob.diag().cpu().numpy()
    do = orc.diag(N, glo, G, prob.nglobal, mask=mask)
    assert relerr(d, do) < 1e-13
    fL = W.sine_forcing(xyz, modes)
    b = prob.rhs(fL).cpu().numpy()
    bo = orc.rhs(N, glo, wJ, W.sine_forcing(orc.node_coords(N, v), modes), prob.nglobal, mask=mask)
    assert relerr(b, bo) < 1e-13


def test_c1_workload(sem, orc):
    # 4x4x4 hex mesh of [0,1]^3, N=7, interior vertices perturbed U(-0.1h, 0.1h), u ~ U(-1,1)
    box, N = (4, 4, 4), 7
    prob, v, G, wJ, glo, mask, _ = _setup(sem, orc, box, N, seed=W.BASE_SEED + 1)
    assert prob.nlocal == 32768 and prob.nglobal == 24389
    u = W.uniform(prob.nglobal, seed=W.BASE_SEED + 1)
    yo = orc.apply(N, glo, G, u, mask=mask)
    for prec in ("fp64", "fp32", "fp64_emu", "fp32_otf"):
        assert relerr(_apply(prob, u, prec), yo) < TOL[prec]


def _sampled_oracle(orc, N, v, box, u, nodes_ijk, modes=None, round_bf16=False):
    """Exact y at a few global nodes (I, J, K) of a structured box: sum of the element-local
    oracle applies of every element that contains the node (Dirichlet box); with round_bf16 the
    factors are first rounded to BF16 (the operator the BF16-factor apply computes)."""
    from oracle import mlp

    sx, sy, sz = box
    gx, gy, gz = sx * N + 1, sy * N + 1, sz * N + 1
    n = N + 1
    out = []
    for (I, J, K) in nodes_ijk:
        if I in (0, gx - 1) or J in (0, gy - 1) or K in (0, gz - 1):
            out.append(0.0)
            continue
        tot = 0.0
        for ex in {min(I // N, sx - 1), (I - 1) // N} if I % N == 0 else {I // N}:
            for ey in {min(J // N, sy - 1), (J - 1) // N} if J % N == 0 else {J // N}:
                for ez in {min(K // N, sz - 1), (K - 1) // N} if K % N == 0 else {K // N}:
                    e = ex + sx * (ey + sy * ez)
                    G, _ = orc.factors(N, v[e:e + 1], modes=modes)
                    if round_bf16:
                        G = mlp.bf16(G)
                    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
                    ii, jj, kk = (np.transpose(a, (2, 1, 0)).reshape(-1) for a in (ii, jj, kk))
                    Ig, Jg, Kg = ex * N + ii, ey * N + jj, ez * N + kk
                    ids = Ig + gx * (Jg + gy * Kg)
                    dirl = (Ig == 0) | (Jg == 0) | (Kg == 0) | (Ig == gx - 1) | (Jg == gy - 1) | (Kg == gz - 1)
                    ue = np.where(dirl, 0.0, u[ids])
                    ye = orc.apply_local(N, G, ue[None, :])[0]
                    p = (I - ex * N) + n * ((J - ey * N) + n * (K - ez * N))
                    tot += ye[p]
        out.append(tot)
    return np.array(out)


@pytest.mark.parametrize("N", [3, 7, 11, 15])
def test_full_size_sampled(sem, orc, N):
    # the 64^3-element benchmark mesh: compare sampled outputs with the oracle computed node by node
    import torch

    box = (64, 64, 64)
    v = W.box_vertices(*box, seed=W.BASE_SEED + 2)
    prob = sem.Problem(N, v, box=box, bc="box",
                       features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_EMU | sem.SEM_FEAT_BF16 |
                       sem.SEM_FEAT_OTF)
    u = W.uniform(prob.nglobal, seed=W.BASE_SEED + 2)
    ud = torch.from_numpy(u).cuda()
    y64 = prob.apply(ud, prec="fp64").cpu().numpy()
    yem = prob.apply(ud, prec="fp64_emu").cpu().numpy()
    y32 = prob.apply(ud.float(), prec="fp32").double().cpu().numpy()
    y16 = prob.apply(ud.float(), prec="bf16").double().cpu().numpy()
    yotf = prob.apply(ud.float(), prec="fp32_otf").double().cpu().numpy()
    gx = 64 * N + 1
    g = W.rng(77)
    pts = [tuple(int(c) for c in g.integers(0, gx, size=3)) for _ in range(24)]
    pts += [(N, N, N), (N, 5, 2 * N), (1, 1, 1), (gx - 2, gx - 2, gx - 2), (3 * N, 3 * N, 3 * N)]
    yo = _sampled_oracle(orc, N, v, box, u, pts)
    idx = [I + gx * (J + gx * K) for (I, J, K) in pts]
    scale = np.max(np.abs(y64))
    assert np.max(np.abs(y64[idx] - yo)) < 1e-12 * scale
    assert np.max(np.abs(yem[idx] - yo)) < 1e-12 * scale
    assert np.max(np.abs(y32[idx] - yo)) < 1e-5 * scale
    assert np.max(np.abs(yotf[idx] - yo)) < 1e-5 * scale
    # every node: factors recomputed on the fly against stored FP32 factors
    assert np.max(np.abs(yotf - y32)) < 2e-5 * scale
    yo16 = _sampled_oracle(orc, N, v, box, u, pts, round_bf16=True)
    assert np.max(np.abs(y16[idx] - yo16)) < 1e-5 * scale
    # every node: the FP64-accurate double-float apply against the FP64 apply
    assert np.max(np.abs(yem - y64)) < 1e-12 * scale
    del prob
    torch.cuda.empty_cache()


@pytest.mark.parametrize("variant", [-1, 0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("N", [2, 5, 7, 10])
def test_apply_variants_agree(sem, orc, variant, N):
    box = (3, 2, 3)
    modes = W.kappa_modes(16, seed=N)
    prob, v, G, wJ, glo, mask, wJa = _setup(sem, orc, box, N, seed=N, modes=modes, alpha=True)
    prob.set_apply_variant(variant)
    u = W.uniform(prob.nglobal, seed=200 + N)
    yo = orc.apply(N, glo, G, u, mask=mask, wJalpha=wJa)
    for prec in ("fp64", "fp32", "fp64_emu", "fp32_otf"):
        assert relerr(_apply(prob, u, prec), yo) < TOL[prec]


@pytest.mark.parametrize("box,explicit", [((3, 2, 3), False), ((3, 3, 1), False), ((1, 1, 1), False),
                                          ((2, 3, 2), True)])
def test_tensor_core_fp32_apply(sem, orc, box, explicit):
    # order 7, FP32 apply with the D-contractions on the tensor cores (variant 5: two TF32 slices of
    # each operand, FP32 accumulation) against the oracle with the FP32 bound, and against the
    # CUDA-core FP32 kernel; odd element counts leave half a block's pair empty; the explicit
    # numbering with a flag-array mask takes the unstructured gather and scatter
    N = 7
    modes = W.kappa_modes(16, seed=31)
    v = W.box_vertices(*box, seed=32)
    E, n3 = v.shape[0], (N + 1) ** 3
    al = (0.5 + W.uniform(E * n3, seed=33, lo=0, hi=1)).reshape(E, n3)
    glo = orc.box_numbering(*box, N)
    ng = orc.box_nglobal(*box, N)
    mask = orc.box_dirichlet(*box, N)
    feats = sem.SEM_FEAT_FP32
    if explicit:
        perm = W.rng(34).permutation(ng)
        glo, mask_p = perm[glo], np.zeros(ng, dtype=np.uint8)
        mask_p[perm] = mask
        mask = mask_p
        prob = sem.Problem(N, v, box=box, glo_num=glo, nglobal=ng, kappa_modes=modes, alpha=al, bc="mask",
                           dirichlet=mask, features=feats)
    else:
        prob = sem.Problem(N, v, box=box, kappa_modes=modes, alpha=al, bc="box", features=feats)
    G, wJ = orc.factors(N, v, modes=modes)
    u = W.uniform(ng, seed=35)
    yo = orc.apply(N, glo, G, u, mask=mask, wJalpha=al * wJ)
    prob.set_apply_variant(5)
    y_tc = _apply(prob, u, "fp32")
    prob.apply_status()
    prob.set_apply_variant(1)
    y_cc = _apply(prob, u, "fp32")
    e_tc, e_cc = relerr(y_tc, yo), relerr(y_cc, yo)
    print(f"\ntensor-core FP32 error {e_tc:.2e}, CUDA-core FP32 {e_cc:.2e}")
    assert e_tc < TOL["fp32"] and e_cc < TOL["fp32"]
    assert np.all(y_tc[mask != 0] == 0.0)


@pytest.mark.parametrize("box,explicit", [((3, 2, 3), False), ((3, 3, 1), False), ((1, 1, 1), False),
                                          ((2, 3, 2), True)])
def test_tensor_core_double_float_apply(sem, orc, box, explicit):
    # order 7, FP64-accurate apply with the D-contractions on the tensor cores (variant 5) against
    # the oracle and against the CUDA-core double-float kernel (variant 1, also the automatic
    # choice): odd element counts leave half a block's pair empty; the explicit numbering with a
    # flag-array mask takes the unstructured gather and scatter
    N = 7
    modes = W.kappa_modes(16, seed=21)
    v = W.box_vertices(*box, seed=22)
    E, n3 = v.shape[0], (N + 1) ** 3
    al = (0.5 + W.uniform(E * n3, seed=23, lo=0, hi=1)).reshape(E, n3)
    glo = orc.box_numbering(*box, N)
    ng = orc.box_nglobal(*box, N)
    mask = orc.box_dirichlet(*box, N)
    if explicit:
        perm = W.rng(24).permutation(ng)
        glo, mask_p = perm[glo], np.zeros(ng, dtype=np.uint8)
        mask_p[perm] = mask
        mask = mask_p
        prob = sem.Problem(N, v, box=box, glo_num=glo, nglobal=ng, kappa_modes=modes, alpha=al, bc="mask",
                           dirichlet=mask, features=sem.SEM_FEAT_EMU)
    else:
        prob = sem.Problem(N, v, box=box, kappa_modes=modes, alpha=al, bc="box", features=sem.SEM_FEAT_EMU)
    G, wJ = orc.factors(N, v, modes=modes)
    u = W.uniform(ng, seed=25)
    yo = orc.apply(N, glo, G, u, mask=mask, wJalpha=al * wJ)
    prob.set_apply_variant(5)
    y_tc = _apply(prob, u, "fp64_emu")
    prob.set_apply_variant(1)
    y_df = _apply(prob, u, "fp64_emu")
    prob.set_apply_variant(-1)
    y_auto = _apply(prob, u, "fp64_emu")
    e_tc, e_df = relerr(y_tc, yo), relerr(y_df, yo)
    print(f"\ntensor-core double-float error {e_tc:.2e}, CUDA-core double-float {e_df:.2e}")
    assert e_tc < 1e-12 and e_df < 1e-12
    assert relerr(y_auto, y_df) < 1e-15 and relerr(y_tc, y_df) < 1e-13


def test_emu_on_wide_dynamic_range(sem, orc):
    # entries spanning 1e-30 .. 1e+30 exercise the bit-level FP64 <-> double-float split
    box, N = (3, 2, 2), 5
    prob, v, G, wJ, glo, mask, _ = _setup(sem, orc, box, N, seed=8)
    g = W.rng(9)
    u = W.uniform(prob.nglobal, seed=9) * 10.0 ** g.integers(-30, 31, size=prob.nglobal)
    yo = orc.apply(N, glo, G, u, mask=mask)
    assert relerr(_apply(prob, u, "fp64_emu"), yo) < 1e-12


@pytest.mark.parametrize("scale_exp", [-80, -120, 100, -1000, 1000])
@pytest.mark.parametrize("N", [3, 7])
def test_emu_on_uniformly_scaled_u(sem, orc, scale_exp, N):
    # u scaled uniformly by 2^k far outside the FP32 range: each element's u is brought to [1, 2)
    # by an exact power of two inside the kernel, so the error relative to the max-norm of that
    # scaled case stays at FP64 level
    box = (3, 2, 2)
    prob, v, G, wJ, glo, mask, _ = _setup(sem, orc, box, N, seed=12, modes=W.kappa_modes(8, seed=3))
    u = np.ldexp(W.uniform(prob.nglobal, seed=13), scale_exp)
    yo = orc.apply(N, glo, G, u, mask=mask)
    assert np.isfinite(yo).all() and np.max(np.abs(yo)) > 0
    assert relerr(_apply(prob, u, "fp64_emu"), yo) < 1e-12


@pytest.mark.parametrize("N", [3, 7])
def test_emu_on_scaled_mesh(sem, orc, N):
    # a mesh of size 1e-9: the factors shrink with it (w det J |grad r|^2 ~ h), well inside the
    # checked 2^-60 .. 2^60 range, and the apply keeps FP64 accuracy
    box = (3, 2, 2)
    v = W.box_vertices(*box, seed=14) * 1e-9
    prob = sem.Problem(N, v, box=box, bc="box", features=sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP64)
    G, _ = orc.factors(N, v)
    u = W.uniform(prob.nglobal, seed=15)
    yo = orc.apply(N, orc.box_numbering(*box, N), G, u, mask=orc.box_dirichlet(*box, N))
    assert relerr(_apply(prob, u, "fp64_emu"), yo) < 1e-12


def test_emu_refuses_factors_outside_its_range(sem, orc):
    # a mesh of size 1e-30 puts the factors near 1e-32, below 2^-60: set-up refuses the
    # double-float factor set instead of returning silently inaccurate applies
    box, N = (2, 2, 2), 3
    v = W.box_vertices(*box, seed=16) * 1e-30
    with pytest.raises(sem.SemError) as ei:
        sem.Problem(N, v, box=box, bc="box", features=sem.SEM_FEAT_EMU)
    assert ei.value.status == sem.SEM_ERR_INVALID and "2^-60" in str(ei.value)
    sem.Problem(N, v, box=box, bc="box", features=sem.SEM_FEAT_FP64)  # plain FP64 is unaffected


@pytest.mark.parametrize("box,N", [((3, 2, 2), 2), ((3, 3, 2), 5), ((4, 4, 4), 7), ((2, 2, 2), 9), ((2, 1, 1), 14)])
def test_bf16_factor_apply_matches_oracle_with_rounded_factors(sem, orc, box, N):
    # SEM_BF16: factors stored in BF16 (nearest from FP64), FP32 arithmetic.  Against the oracle's
    # apply with the same BF16-rounded factors the bound is the FP32 one; against the unrounded
    # operator the error is of the order of the BF16 rounding (2^-9 relative per factor).
    from oracle import mlp

    modes = W.kappa_modes(16, seed=N + 60)
    feats = sem.SEM_FEAT_FP32 | sem.SEM_FEAT_BF16
    prob, v, G, wJ, glo, mask, wJa = _setup(sem, orc, box, N, seed=N + 3, modes=modes, alpha=True, features=feats)
    u = W.uniform(prob.nglobal, seed=N + 5)
    y = _apply(prob, u, "bf16")
    y_rounded = orc.apply(N, glo, mlp.bf16(G), u, mask=mask, wJalpha=wJa)
    assert relerr(y, y_rounded) < TOL["fp32"]
    e = relerr(y, orc.apply(N, glo, G, u, mask=mask, wJalpha=wJa))
    assert 1e-6 < e < 2e-2, e


def test_bf16_factors_need_their_feature(sem, orc):
    prob, *_ = _setup(sem, orc, (2, 2, 2), 3, features=sem.SEM_FEAT_FP32)
    with pytest.raises(sem.SemError):
        _apply(prob, W.uniform(prob.nglobal, seed=1), "bf16")


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64", "fp64_emu", "fp32_otf"])
def test_apply_writes_only_its_output(sem, orc, prec):
    # y is a view into a larger buffer whose tail holds a sentinel: zeroing and scatter-add must
    # stay inside the nglobal entries of y, whatever the precision's element size
    import torch

    feats = sem.SEM_FEAT_FP64 | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_EMU | sem.SEM_FEAT_BF16 | sem.SEM_FEAT_OTF
    prob, *_ = _setup(sem, orc, (2, 2, 2), 3, features=feats)
    dt = torch.float32 if prec in F32 else torch.float64
    u = torch.from_numpy(W.uniform(prob.nglobal, seed=3)).to(dt).cuda()
    buf = torch.full((prob.nglobal + 4096,), 7.0, dtype=dt, device="cuda")
    prob.apply(u, buf[:prob.nglobal], prec=prec)
    torch.cuda.synchronize()
    assert bool((buf[prob.nglobal:] == 7.0).all())


@pytest.mark.parametrize("box,N,kind", [((3, 2, 2), 2, "modes"), ((3, 3, 2), 5, "nodal"), ((4, 4, 4), 7, "one"),
                                        ((2, 2, 2), 9, "nodal"), ((2, 1, 1), 15, "modes")])
def test_otf_only_handle(sem, orc, box, N, kind):
    # SEM_FEAT_OTF as the only factor set: the Jacobi diagonal comes from factors evaluated in FP64
    # from the map at set-up, the apply recomputes them in FP32 at every node; kappa from Fourier
    # modes, from a nodal array (read in FP32 by the apply) or 1; screened term included
    import torch

    v = W.box_vertices(*box, seed=N + 11, perturb=0.15)
    E, n3 = v.shape[0], (N + 1) ** 3
    modes = W.kappa_modes(16, seed=N + 70) if kind == "modes" else None
    kap = np.exp(0.5 * W.uniform(E * n3, seed=N + 71)).reshape(E, n3) if kind == "nodal" else None
    al = (0.5 + W.uniform(E * n3, seed=N + 72, lo=0, hi=1)).reshape(E, n3)
    prob = sem.Problem(N, v, box=box, kappa_modes=modes, kappa=kap, alpha=al, bc="box", features=sem.SEM_FEAT_OTF)
    G, wJ = orc.factors(N, v, kappa_nodal=kap, modes=modes)
    glo = orc.box_numbering(*box, N)
    mask = orc.box_dirichlet(*box, N)
    d = prob.diag().cpu().numpy()
    assert relerr(d, orc.diag(N, glo, G, prob.nglobal, mask=mask, wJalpha=al * wJ)) < 1e-13
    u = W.uniform(prob.nglobal, seed=N + 73)
    y = prob.apply(torch.from_numpy(u).float().cuda(), prec="fp32_otf").double().cpu().numpy()
    assert relerr(y, orc.apply(N, glo, G, u, mask=mask, wJalpha=al * wJ)) < TOL["fp32_otf"]
    with pytest.raises(sem.SemError):
        prob.apply(torch.from_numpy(u).float().cuda(), prec="fp32")


def test_otf_on_strongly_distorted_elements(sem, orc):
    # vertices moved by up to 30% of the spacing: the Jacobian varies strongly inside each element,
    # so every term of the trilinear map matters
    box, N = (3, 3, 3), 6
    v = W.box_vertices(*box, seed=5, perturb=0.3)
    prob = sem.Problem(N, v, box=box, bc="none", features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_OTF)
    G, _ = orc.factors(N, v)
    glo = orc.box_numbering(*box, N)
    u = W.uniform(prob.nglobal, seed=6)
    assert relerr(_apply(prob, u, "fp32_otf"), orc.apply(N, glo, G, u)) < TOL["fp32_otf"]
