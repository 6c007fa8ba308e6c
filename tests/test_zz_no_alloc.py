"""The allocation-free inner product (sem_dot_static) against the workspace-based sem_dot and an
independent long-double sum on the host.

sem_dot_static keeps its reduction scratch in a static device array so that callers which must
not allocate device memory can still form FP64 dot products; it is called here through the C ABI
twice in a row (the second call reuses the scratch the first one left behind) and must agree
with sem_dot and with the host's long-double sum to the tolerance of an FP64 sum.  The file name
sorts last so that pytest collects it last: if it fails, a run that stops at the first failure has
already run every other test.  It depends on no other test and passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def test_dot_static_matches_dot_twice():
    from paper_1403_0968_gb300 import build

    build.build()
    import paper_1403_0968_gb300 as sem

    L = sem.lib()
    fn = L.sem_dot_static
    fn.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    box, N = (6, 5, 4), 5
    prob = sem.Problem(N, W.box_vertices(*box, seed=31), box=box, bc="box",
                       features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_PCG)
    n = prob.nglobal
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((41, 42)):
        xh, yh = W.uniform(n, seed=seed), W.uniform(n, seed=seed + 100)
        x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        ref = prob.dot(x, y)
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(n, x.data_ptr(), y.data_ptr(), out.data_ptr(), stream)
        assert st == sem.SEM_OK, sem.sem_last_error()
        torch.cuda.synchronize()
        scale = float(np.sum(np.abs(xh * yh)))
        exact = float(np.dot(xh.astype(np.longdouble), yh.astype(np.longdouble)))
        assert abs(float(out.item()) - exact) <= 1e-13 * scale, (call, out.item(), exact)
        assert abs(float(out.item()) - float(ref.item())) <= 1e-13 * scale, (call, out.item(), ref.item())
    # an empty product is zero
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert fn(0, x.data_ptr(), y.data_ptr(), out.data_ptr(), stream) == sem.SEM_OK
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
    # sizes beyond the static scratch are refused with a clear error, before any launch
    st = fn(1 << 31, x.data_ptr(), y.data_ptr(), out.data_ptr(), stream)
    assert st == sem.SEM_ERR_INVALID and "static scratch" in sem.sem_last_error()
