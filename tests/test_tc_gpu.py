"""Tensor-core BF16 GEMM (sem_gemm_bf16, the dense layers of the learned preconditioner) against
the exact product of the same BF16 values in FP64.

Bound: the products of two BF16 values are exact in FP32; the K-term sums are FP32 (the tensor
core's internal additions may truncate rather than round, so unit 2^-22 instead of 2^-24), so
|C - C_exact| <= K * 2^-22 * sum_k |a_k b_k|, plus one FP32 rounding of the bias add.  A
transposed operand, a dropped or repeated K slice, a wrong row or column tile gives an error of
the order of the entries themselves."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sem():
    from paper_1403_0968_gb300 import build

    build.build()
    import paper_1403_0968_gb300 as sem

    sem.lib()
    return sem


def _bf16(rng, shape, scale=1.0):
    return torch.from_numpy((rng.standard_normal(shape) * scale).astype(np.float32)).to(torch.bfloat16)


def _check(sem, M, N, K, lda, ldb, relu, seed, bias=True):
    rng = np.random.default_rng(seed)
    A, Bt = _bf16(rng, (M, lda)), _bf16(rng, (N, ldb), 0.1)
    b = torch.from_numpy(rng.standard_normal(N).astype(np.float32)) if bias else None
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = sem.gemm_bf16(A.cuda(), Bt.cuda(), None if b is None else b.cuda(), relu=relu, K=K, err=err)
    torch.cuda.synchronize()
    a = A.float().double().numpy()[:, :K]
    bt = Bt.float().double().numpy()[:, :K]
    ref = a @ bt.T + (b.double().numpy() if b is not None else 0.0)
    if relu:
        ref = np.maximum(ref, 0.0)
    bound = K * 2.0 ** -22 * (np.abs(a) @ np.abs(bt).T) + 2.0 ** -23 * np.abs(ref) + 1e-30
    got = C.cpu().numpy()[:, :N].astype(np.float64)
    assert int(err.item()) == 0
    viol = np.abs(got - ref) / bound
    assert viol.max() <= 1.0, (M, N, K, float(viol.max()))
    assert np.all(C.cpu().numpy()[:, N:] == 0.0)  # columns past N untouched


def test_ragged_tiles_and_k_slices(sem):
    # 3 row tiles (last 44 rows), 2 column tiles (last 44 columns), 4 K slices (last 8)
    _check(sem, 300, 300, 200, 200, 200, relu=False, seed=1)


def test_relu_and_partial_k_chunk(sem):
    # K = 518 inside leading dimension 520: the last 16-byte chunk holds 6 values, rest zero-filled
    _check(sem, 257, 512, 518, 520, 520, relu=True, seed=2)


def test_single_row_column_and_product(sem):
    _check(sem, 1, 8, 1, 8, 8, relu=False, seed=3)
    _check(sem, 1, 1, 5, 8, 8, relu=False, seed=4, bias=False)


def test_network_layer_shapes(sem):
    # the three inference layers at N = 7 (n^3 = 512, n_in = 518 padded to 520, hidden 256)
    _check(sem, 1000, 256, 518, 520, 520, relu=True, seed=5)
    _check(sem, 1000, 256, 256, 256, 256, relu=True, seed=6)
    _check(sem, 1000, 512, 256, 256, 256, relu=False, seed=7)


def test_rejects_bad_layouts(sem):
    A = torch.zeros((16, 20), dtype=torch.bfloat16, device="cuda")
    Bt = torch.zeros((8, 24), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(sem.SemError):
        sem.gemm_bf16(A, Bt)  # lda = 20 is not a multiple of 8


def test_full_size_layer_sampled_rows(sem):
    # the first inference layer at 32^3 elements, N = 7 (M = 32768 rows, K = 518 in rows of 520),
    # in the launch configuration of the preconditioner: sampled rows against the exact product
    M, N, K, ld = 32768, 256, 518, 520
    rng = np.random.default_rng(8)
    A = _bf16(rng, (M, ld))
    Bt = _bf16(rng, (N, ld), 0.1)
    b = torch.from_numpy(rng.standard_normal(N).astype(np.float32))
    C = sem.gemm_bf16(A.cuda(), Bt.cuda(), b.cuda(), relu=True, K=K)
    rows = np.concatenate([rng.integers(0, M, size=200), [0, 127, 128, M - 129, M - 1]])
    a = A.float().double().numpy()[rows, :K]
    bt = Bt.float().double().numpy()[:, :K]
    ref = np.maximum(a @ bt.T + b.double().numpy(), 0.0)
    bound = K * 2.0 ** -22 * (np.abs(a) @ np.abs(bt).T) + 2.0 ** -23 * np.abs(ref) + 1e-30
    got = C.cpu().numpy()[rows, :N].astype(np.float64)
    assert (np.abs(got - ref) / bound).max() <= 1.0


def _layers_case(sem, M, nin, nout, seed):
    """The three layers in one launch against three sem_gemm_bf16 launches with the hidden outputs
    rounded to BF16 in between (round to nearest even, as the fused epilogue rounds them)."""
    rng = np.random.default_rng(seed)
    ldx = (nin + 7) // 8 * 8
    X = _bf16(rng, (M, ldx)).cuda()
    W1t, W2t, W3t = _bf16(rng, (256, ldx), 0.1).cuda(), _bf16(rng, (256, 256), 0.1).cuda(), _bf16(rng, (nout, 256), 0.1).cuda()
    b1, b2, b3 = (torch.from_numpy(rng.uniform(-0.5, 0.5, n).astype(np.float32)).cuda() for n in (256, 256, nout))
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    O = sem.mlp_layers_bf16(X, nin, W1t, W2t, W3t, b1, b2, b3, err=err)
    H1 = sem.gemm_bf16(X, W1t, b1, relu=True, K=nin).to(torch.bfloat16)
    H2 = sem.gemm_bf16(H1, W2t, b2, relu=True).to(torch.bfloat16)
    ref = sem.gemm_bf16(H2, W3t, b3)[:, :nout]
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    o, r = O.cpu().numpy(), ref.cpu().numpy()
    # equal unless the tensor core's FP32 sums differ with the tile width (128 columns per launch
    # against 256 in the fused kernel), which can move a hidden activation across a BF16 rounding
    # boundary: one BF16 ulp of one term in the outputs it feeds
    d = np.abs(o - r) / np.max(np.abs(r))
    assert np.array_equal(o, r) or (d.max() < 2e-3 and np.median(d) == 0.0), (M, nin, nout, d.max(), np.median(d))


@pytest.mark.parametrize("M,nin,nout", [(1, 70, 64), (200, 70, 64), (200, 222, 216), (1000, 518, 512),
                                        (300, 518, 264), (129, 40, 8), (257, 100, 296)])
def test_fused_layers_match_three_launches(sem, M, nin, nout):
    # ragged tiles of 128 rows, K slices of 64 with a partial last slice, one output half (n_out
    # <= 256) and two (the second as narrow as 8 outputs, rounded up to an MMA width of 16)
    _layers_case(sem, M, nin, nout, seed=M + nin + nout)


def test_fused_layers_full_size(sem):
    # the preconditioner's layers at 32^3 elements, N = 7: 32768 rows, 518 -> 256 -> 256 -> 512
    _layers_case(sem, 32768, 518, 512, seed=21)


def test_fused_layers_reject_bad_shapes(sem):
    X = torch.zeros((16, 72), dtype=torch.bfloat16, device="cuda")
    W = torch.zeros((256, 72), dtype=torch.bfloat16, device="cuda")
    W2 = torch.zeros((256, 256), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(520, dtype=torch.float32, device="cuda")
    for nout in (12, 520):  # not a multiple of 8; above two output halves
        W3 = torch.zeros((nout, 256), dtype=torch.bfloat16, device="cuda")
        with pytest.raises(sem.SemError):
            sem.mlp_layers_bf16(X, 70, W, W2, W3, b, b, b)
