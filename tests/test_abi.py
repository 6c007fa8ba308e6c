"""Host-side checks of the C ABI (no GPU): the library builds, loads, exports every function that
include/*.h declares, and validates descriptions before touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sem():
    from paper_1403_0968_gb300 import build

    build.build()
    import paper_1403_0968_gb300 as sem

    sem.lib()
    return sem


def _declared_functions():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(sem_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(sem):
    names = _declared_functions()
    assert "sem_apply" in names and "sem_pcg" in names and "sem_setup" in names
    L = ctypes.CDLL(sem.build.LIB)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def _desc(sem, N=3, box=(2, 2, 1)):
    v = W.box_vertices(*box)
    d = sem.SemDesc()
    d.N = N
    d.box[0], d.box[1], d.box[2] = box
    d.nelem = v.shape[0]
    d.vertices = v.ctypes.data
    d.bc = sem.SEM_BC_BOX
    return d, v


def test_workspace_size_is_host_logic(sem):
    d, v = _desc(sem)
    n = sem.sem_workspace_size(d, sem.SEM_FEAT_FP64)
    n2 = sem.sem_workspace_size(d, sem.SEM_FEAT_FP64 | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_PCG)
    assert 0 < n < n2
    assert n % 256 == 0


@pytest.mark.parametrize("field,value", [("N", 0), ("N", 16), ("nelem", 0), ("bc", 7)])
def test_invalid_descriptions_rejected(sem, field, value):
    d, v = _desc(sem)
    setattr(d, field, value)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_workspace_size(d, sem.SEM_FEAT_FP64)
    assert ei.value.status == sem.SEM_ERR_INVALID


def test_inconsistent_box_rejected(sem):
    d, v = _desc(sem)
    d.box[0] = 5
    with pytest.raises(sem.SemError):
        sem.sem_workspace_size(d, sem.SEM_FEAT_FP64)


def test_setup_rejects_small_workspace_without_touching_device(sem):
    d, v = _desc(sem)
    h = ctypes.c_void_p(None)
    st = sem.lib().sem_setup(ctypes.byref(d), sem.SEM_FEAT_FP64, None, 0, None, ctypes.byref(h))
    assert st == sem.SEM_ERR_WORKSPACE
    assert "workspace" in sem.sem_last_error()


def test_otf_workspace_is_per_element(sem):
    # SEM_FEAT_OTF alone stores 96 bytes of map coefficients per element and no factor stream:
    # far less than the FP32 factors (24 bytes per local node)
    d, v = _desc(sem)
    n_otf = sem.sem_workspace_size(d, sem.SEM_FEAT_OTF)
    n_32 = sem.sem_workspace_size(d, sem.SEM_FEAT_FP32)
    L = d.nelem * (d.N + 1) ** 3
    assert n_32 - n_otf >= 24 * L - 96 * d.nelem - 256
    assert sem.sem_workspace_size(d, sem.SEM_FEAT_OTF | sem.SEM_FEAT_FP32) > n_32


def test_learned_preconditioner_needs_stored_factors(sem):
    d, v = _desc(sem)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_workspace_size(d, sem.SEM_FEAT_OTF | sem.SEM_FEAT_MLP)
    assert ei.value.status == sem.SEM_ERR_INVALID


@pytest.mark.parametrize("r", range(1, 8))
def test_fd_weights_host_closed_form_matches_oracle(sem, r):
    # the library's closed-form weights (host logic) against the oracle's exact rational solve
    from oracle import fd

    exact = [float(c) for c in fd.weights_exact(r)]
    got = sem.fd_weights(r)
    assert np.max(np.abs(got - np.array(exact))) <= 4 * np.finfo(float).eps * np.max(np.abs(exact))


@pytest.mark.parametrize("r", [0, 8, -1])
def test_fd_weights_reject_bad_radius(sem, r):
    with pytest.raises(sem.SemError) as ei:
        sem.fd_weights(r)
    assert ei.value.status == sem.SEM_ERR_INVALID


@pytest.mark.parametrize("N", range(1, 9))
def test_dg_operators_host_match_oracle(sem, N):
    # the library's weak derivative matrices (orthonormal-basis route, FP64, host logic) against the
    # oracle's exact rational construction
    from oracle import dg

    Drw, Dsw = sem.dg_operators(N)
    o = dg.operators(N)
    for a, b in ((Drw, o["Drw"]), (Dsw, o["Dsw"])):
        assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


def test_dg_rejects_bad_order(sem):
    with pytest.raises(sem.SemError):
        sem.dg_operators(9)


def test_fd_and_dg_argument_checks_are_host_logic(sem):
    # invalid arguments are rejected before any device work (runs without a GPU)
    L = sem.lib()
    buf = ctypes.c_void_p(16)  # never dereferenced: every call below fails its argument checks first
    other = ctypes.c_void_p(32)
    assert L.sem_fd_step(sem.SEM_FP32, 1, 8, 8, 0.1, 0.1, 0.1, buf, buf, None) == sem.SEM_ERR_INVALID  # aliasing
    assert L.sem_fd_step(sem.SEM_FP32, 8, 8, 8, 0.1, 0.1, 0.1, buf, other, None) == sem.SEM_ERR_INVALID  # radius
    assert L.sem_fd_step(sem.SEM_FP32, 2, 0, 8, 0.1, 0.1, 0.1, buf, other, None) == sem.SEM_ERR_INVALID  # width
    assert L.sem_fd_step(sem.SEM_FP32, 2, 8, 8, -1.0, 0.1, 0.1, buf, other, None) == sem.SEM_ERR_INVALID  # dt
    assert L.sem_fd_step(sem.SEM_BF16, 2, 8, 8, 0.1, 0.1, 0.1, buf, other, None) == sem.SEM_ERR_INVALID  # precision
    assert L.sem_dg_volume(sem.SEM_FP32, 9, 10, 9.81, buf, buf, buf, buf, other, None) == sem.SEM_ERR_INVALID
    assert L.sem_dg_volume(sem.SEM_FP32, 3, 0, 9.81, buf, buf, buf, buf, other, None) == sem.SEM_ERR_INVALID
    assert L.sem_dg_volume(sem.SEM_BF16, 3, 10, 9.81, buf, buf, buf, buf, other, None) == sem.SEM_ERR_INVALID
    assert L.sem_dg_volume(sem.SEM_FP32, 3, 10, 9.81, None, buf, buf, buf, other, None) == sem.SEM_ERR_INVALID
    n = ctypes.c_size_t(0)
    assert L.sem_dg_operator_bytes(8, sem.SEM_FP32, ctypes.byref(n)) == sem.SEM_OK
    assert n.value == 2 * 45 * 52 * 4  # rows padded to 13 vectors of 4 floats (an odd count)
    assert L.sem_dg_operator_bytes(8, sem.SEM_FP64, ctypes.byref(n)) == sem.SEM_OK
    assert n.value == 2 * 45 * 46 * 8  # 23 vectors of 2 doubles
    assert L.sem_dg_load_operators(8, sem.SEM_FP32, buf, 16, None) == sem.SEM_ERR_INVALID  # too small


def test_batch_host_checks(sem):
    # batched solves: the feature mask needs an inner (FP32 or on-the-fly) and a residual (FP64 or
    # double-float) factor set, problems must be structured boxes, and the entry points reject a
    # NULL batch before touching the device
    L = sem.lib()
    d1, v1 = _desc(sem)
    d2, v2 = _desc(sem, N=5, box=(2, 1, 1))
    descs = (sem.SemDesc * 2)(d1, d2)
    nb = ctypes.c_size_t(0)
    ok = sem.SEM_FEAT_EMU | sem.SEM_FEAT_FP32
    assert L.sem_batch_workspace_size(descs, 2, ok, ctypes.byref(nb)) == sem.SEM_OK and nb.value > 0
    one = ctypes.c_size_t(0)
    assert L.sem_batch_workspace_size(descs, 1, ok, ctypes.byref(one)) == sem.SEM_OK and one.value < nb.value
    for feats in (sem.SEM_FEAT_EMU, sem.SEM_FEAT_FP32, sem.SEM_FEAT_BF16 | sem.SEM_FEAT_EMU):
        assert L.sem_batch_workspace_size(descs, 2, feats, ctypes.byref(nb)) == sem.SEM_ERR_INVALID, feats
    assert L.sem_batch_workspace_size(descs, 0, ok, ctypes.byref(nb)) == sem.SEM_ERR_INVALID
    glo = np.zeros(d1.nelem * (d1.N + 1) ** 3, dtype=np.int32)
    d1.glo_num = glo.ctypes.data
    descs = (sem.SemDesc * 2)(d1, d2)
    assert L.sem_batch_workspace_size(descs, 2, ok, ctypes.byref(nb)) == sem.SEM_ERR_INVALID  # unstructured
    a, u = ctypes.c_int32(0), ctypes.c_int32(0)
    assert L.sem_batch_set_fused(None, 1) == sem.SEM_ERR_INVALID
    assert L.sem_batch_get_fused(None, ctypes.byref(a), ctypes.byref(u)) == sem.SEM_ERR_INVALID
    assert L.sem_batch_set_wait_limit(None, 5) == sem.SEM_ERR_INVALID
    assert L.sem_batch_set_variant(None, 3, 1) == sem.SEM_ERR_INVALID
    assert L.sem_batch_apply(None, sem.SEM_FP32, None, None, None) == sem.SEM_ERR_INVALID
    res = (sem.SemPcgResult * 1)()
    assert L.sem_batch_pcg(None, None, None, None, res, None) == sem.SEM_ERR_INVALID


def test_mlp_layer_entry_points_check_arguments_on_the_host(sem):
    # the fused layer kernel's entry point and the inference-layout switch reject bad arguments
    # before any device work (runs without a GPU); the pointers are never dereferenced
    L = sem.lib()
    a = ctypes.c_void_p(256)  # 16-byte aligned
    mis = ctypes.c_void_p(264)  # 8 bytes off
    ok = (1000, 518, 520, 512, a, a, a, a, a, a, a, a, None, None)
    bad = [
        (1000, 518, 520, 512, None, a, a, a, a, a, a, a, None, None),  # NULL operand
        (0, 518, 520, 512, a, a, a, a, a, a, a, a, None, None),  # no rows
        (1000, 518, 512, 512, a, a, a, a, a, a, a, a, None, None),  # ldx < nin
        (1000, 518, 524, 512, a, a, a, a, a, a, a, a, None, None),  # ldx not a multiple of 8
        (1000, 518, 520, 520, a, a, a, a, a, a, a, a, None, None),  # above two output halves
        (1000, 518, 520, 12, a, a, a, a, a, a, a, a, None, None),  # outputs not a multiple of 8
        (1000, 518, 520, 512, mis, a, a, a, a, a, a, a, None, None),  # misaligned X
        (1000, 518, 520, 512, a, a, a, a, a, a, a, mis, None, None),  # misaligned O
    ]
    assert len(ok) == len(bad[0])
    for args in bad:
        assert L.sem_mlp_layers_bf16(*args) == sem.SEM_ERR_INVALID, args
    assert L.sem_mlp_set_fused(None, 1) == sem.SEM_ERR_INVALID
