"""GB300-native spectral-element operator apply and PCG solver (arXiv 1403.0968 §4.2).

Thin Python binding over the C ABI in include/sem.h (libsem.so, built by ``build.py``): argument
marshalling only, every step of the operator and the solvers runs in the library's CUDA kernels.
PyTorch provides device memory (the workspace and the vectors) and the CUDA stream.

There is no CPU fallback: if libsem.so is missing or fails to load, ``lib()`` raises.

Low-level functions keep the C names (``sem_workspace_size``, ``sem_setup``, ``sem_apply``,
``sem_rhs``, ``sem_pcg``, ``sem_free`` ...); ``Problem`` bundles a handle with its workspace.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["lib", "Problem", "SEM_FP64", "SEM_FP64_EMU", "SEM_FP32", "SEM_BF16", "SEM_FP32_OTF", "SEM_BC_NONE", "SEM_BC_BOX", "SEM_BC_MASK",
           "SEM_FEAT_FP64", "SEM_FEAT_EMU", "SEM_FEAT_FP32", "SEM_FEAT_BF16", "SEM_FEAT_OTF", "SEM_FEAT_PCG", "SEM_SOLVE_FP64", "SEM_SOLVE_IR",
           "SemError", "sem_workspace_size", "sem_setup", "sem_apply", "sem_rhs", "sem_pcg", "sem_free",
           "sem_node_coords", "sem_glo_num", "sem_diag", "sem_get_info", "sem_last_error", "sem_set_apply_variant", "sem_dot", "Batch",
           "sem_apply_status", "sem_set_wait_limit",
           "fd_weights", "fd_step", "fd_run", "fd_status", "dg_operators", "dg_load_operators", "dg_volume",
           "dg_geometry"]

SEM_OK, SEM_ERR_INVALID, SEM_ERR_CUDA, SEM_ERR_NOCONV, SEM_ERR_BREAKDOWN, SEM_ERR_TIMEOUT, SEM_ERR_WORKSPACE = range(7)
SEM_FP64, SEM_FP64_EMU, SEM_FP32, SEM_BF16, SEM_FP32_OTF = 0, 1, 2, 4, 5
SEM_BC_NONE, SEM_BC_BOX, SEM_BC_MASK = 0, 1, 2
SEM_FEAT_FP64, SEM_FEAT_EMU, SEM_FEAT_FP32, SEM_FEAT_PCG, SEM_FEAT_MLP, SEM_FEAT_BF16, SEM_FEAT_OTF = \
    1, 2, 4, 8, 16, 32, 64
SEM_SOLVE_FP64, SEM_SOLVE_IR, SEM_SOLVE_FCG_MLP = 0, 1, 2
SEM_PCG_MULTI_LAUNCH = 1
MLP_H1 = MLP_H2 = 256
MLP_EPS = 1e-2  # mass shift of the element-local problems that define the training targets
STATUS_NAMES = {0: "SEM_OK", 1: "SEM_ERR_INVALID", 2: "SEM_ERR_CUDA", 3: "SEM_ERR_NOCONV", 4: "SEM_ERR_BREAKDOWN",
                5: "SEM_ERR_TIMEOUT", 6: "SEM_ERR_WORKSPACE"}
PREC = {"fp64": SEM_FP64, "fp64_emu": SEM_FP64_EMU, "emu": SEM_FP64_EMU, "fp32": SEM_FP32, "bf16": SEM_BF16,
        "fp32_otf": SEM_FP32_OTF}
FP32_VECTOR_PRECS = (SEM_FP32, SEM_BF16, SEM_FP32_OTF)  # applies on float32 vectors


class SemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SemDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("box", ctypes.c_int32 * 3), ("nelem", ctypes.c_int64),
                ("vertices", ctypes.c_void_p), ("glo_num", ctypes.c_void_p), ("nglobal", ctypes.c_int64),
                ("kappa_nmodes", ctypes.c_int32), ("kappa_modes", ctypes.c_void_p), ("kappa", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("bc", ctypes.c_int32), ("dirichlet", ctypes.c_void_p)]


class SemInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("nelem", ctypes.c_int64), ("nglobal", ctypes.c_int64),
                ("nlocal", ctypes.c_int64)]


class SemPcgOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_it", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("apply_prec", ctypes.c_int32), ("inner_rtol", ctypes.c_double), ("check_every", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("inner_prec", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("history_cap", ctypes.c_int32), ("history", ctypes.POINTER(ctypes.c_double))]


class SemPcgResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("outer", ctypes.c_int32),
                ("true_relres", ctypes.c_double), ("recursive_relres", ctypes.c_double),
                ("fallbacks", ctypes.c_int32), ("history_len", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libsem.so (raises if it was not built: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libsem.so not found at {path}; build it with paper_1403_0968_gb300.build.build()")
            L = ctypes.CDLL(path)
            L.sem_workspace_size.argtypes = [ctypes.POINTER(SemDesc), ctypes.c_uint32, ctypes.POINTER(ctypes.c_size_t)]
            L.sem_setup.argtypes = [ctypes.POINTER(SemDesc), ctypes.c_uint32, _P, ctypes.c_size_t, _P,
                                    ctypes.POINTER(_P)]
            L.sem_free.argtypes = [_P]
            L.sem_free.restype = None
            L.sem_apply.argtypes = [_P, ctypes.c_int, _P, _P, _P]
            L.sem_rhs.argtypes = [_P, _P, _P, _P]
            L.sem_node_coords.argtypes = [_P, _P, _P]
            L.sem_glo_num.argtypes = [_P, _P, _P]
            L.sem_diag.argtypes = [_P, _P, _P]
            L.sem_get_info.argtypes = [_P, ctypes.POINTER(SemInfo)]
            L.sem_pcg.argtypes = [_P, _P, _P, ctypes.POINTER(SemPcgOpts), ctypes.POINTER(SemPcgResult), _P]
            L.sem_dot.argtypes = [_P, _P, _P, _P, _P]
            L.sem_dot.restype = ctypes.c_int
            L.sem_set_apply_variant.argtypes = [_P, ctypes.c_int32]
            L.sem_apply_status.argtypes = [_P, _P]
            L.sem_apply_status.restype = ctypes.c_int
            L.sem_set_wait_limit.argtypes = [_P, ctypes.c_int64]
            L.sem_set_wait_limit.restype = ctypes.c_int
            L.sem_set_apply_variant.restype = ctypes.c_int
            L.sem_batch_workspace_size.argtypes = [ctypes.POINTER(SemDesc), ctypes.c_int32, ctypes.c_uint32,
                                                   ctypes.POINTER(ctypes.c_size_t)]
            L.sem_batch_setup.argtypes = [ctypes.POINTER(SemDesc), ctypes.c_int32, ctypes.c_uint32, _P,
                                          ctypes.c_size_t, _P, ctypes.POINTER(_P)]
            L.sem_batch_info.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(SemInfo), ctypes.POINTER(ctypes.c_int64)]
            L.sem_batch_handle.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(_P)]
            L.sem_batch_set_variant.argtypes = [_P, ctypes.c_int32, ctypes.c_int32]
            L.sem_batch_set_wait_limit.argtypes = [_P, ctypes.c_int64]
            L.sem_batch_set_wait_limit.restype = ctypes.c_int
            L.sem_batch_set_fused.argtypes = [_P, ctypes.c_int32]
            L.sem_batch_set_fused.restype = ctypes.c_int
            L.sem_batch_get_fused.argtypes = [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
            L.sem_batch_get_fused.restype = ctypes.c_int
            L.sem_batch_apply.argtypes = [_P, ctypes.c_int, _P, _P, _P]
            L.sem_batch_rhs.argtypes = [_P, _P, _P, _P]
            L.sem_batch_pcg.argtypes = [_P, _P, _P, ctypes.POINTER(SemPcgOpts), ctypes.POINTER(SemPcgResult), _P]
            L.sem_batch_free.argtypes = [_P]
            L.sem_batch_free.restype = None
            for name in ("sem_batch_workspace_size", "sem_batch_setup", "sem_batch_info", "sem_batch_handle",
                         "sem_batch_set_variant", "sem_batch_apply", "sem_batch_rhs", "sem_batch_pcg"):
                getattr(L, name).restype = ctypes.c_int
            L.sem_residual.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
            L.sem_mlp_param_count.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int64)]
            L.sem_mlp_samples.argtypes = [_P, _P, ctypes.c_int32, _P, ctypes.c_double, ctypes.c_int32, _P, _P, _P,
                                          _P]
            L.sem_mlp_train_scratch.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_size_t)]
            L.sem_mlp_forward.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P,
                                          _P, _P]
            L.sem_mlp_train_step.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, ctypes.c_int32,
                                             ctypes.c_float, _P, _P, ctypes.c_int32, _P, ctypes.c_size_t, _P, _P, _P]
            L.sem_mlp_load.argtypes = [_P, _P, ctypes.c_int32, _P]
            L.sem_mlp_precond.argtypes = [_P, _P, _P, _P]
            L.sem_mlp_set_fused.argtypes = [_P, ctypes.c_int32]
            L.sem_mlp_layers_bf16.argtypes = [ctypes.c_int32] * 4 + [_P] * 8 + [_P, _P]
            L.sem_gemm_bf16.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, _P,
                                        ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]
            for name in ("sem_residual", "sem_mlp_param_count", "sem_mlp_samples", "sem_mlp_train_scratch",
                         "sem_mlp_forward", "sem_mlp_train_step", "sem_mlp_load", "sem_mlp_precond",
                         "sem_mlp_set_fused", "sem_mlp_layers_bf16", "sem_gemm_bf16"):
                getattr(L, name).restype = ctypes.c_int
            L.sem_fd_weights.argtypes = [ctypes.c_int32, _P]
            L.sem_fd_step.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, _P, _P, _P]
            L.sem_fd_weights.restype = ctypes.c_int
            L.sem_dg_operators.argtypes = [ctypes.c_int32, _P, _P]
            L.sem_dg_operator_bytes.argtypes = [ctypes.c_int32, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
            L.sem_dg_load_operators.argtypes = [ctypes.c_int32, ctypes.c_int, _P, ctypes.c_size_t, _P]
            L.sem_dg_volume.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, _P, _P, _P, _P,
                                        _P, _P]
            L.sem_dg_geometry.argtypes = [ctypes.c_int, ctypes.c_int64, _P, _P, _P]
            for name in ("sem_dg_operators", "sem_dg_operator_bytes", "sem_dg_load_operators", "sem_dg_volume",
                         "sem_dg_geometry"):
                getattr(L, name).restype = ctypes.c_int
            L.sem_fd_step.restype = ctypes.c_int
            L.sem_fd_status.argtypes = [_P]
            L.sem_fd_status.restype = ctypes.c_int
            L.sem_last_error.argtypes = []
            L.sem_last_error.restype = ctypes.c_char_p
            for name in ("sem_workspace_size", "sem_setup", "sem_apply", "sem_rhs", "sem_node_coords", "sem_glo_num",
                         "sem_diag", "sem_get_info", "sem_pcg"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def sem_last_error() -> str:
    return lib().sem_last_error().decode()


def _check(status):
    if status != SEM_OK:
        raise SemError(status, sem_last_error())


def _ptr(t):
    """Device/host pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------------------------------
# C-named functions (pointers are torch tensors / numpy arrays; streams are torch streams)
# ------------------------------------------------------------------------------------------
def sem_workspace_size(desc: SemDesc, features: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().sem_workspace_size(ctypes.byref(desc), features, ctypes.byref(n)))
    return n.value


def sem_setup(desc: SemDesc, features: int, workspace, stream=None):
    h = ctypes.c_void_p(None)
    _check(lib().sem_setup(ctypes.byref(desc), features, _ptr(workspace), workspace.numel(), _stream(stream),
                           ctypes.byref(h)))
    return h


def sem_free(h):
    lib().sem_free(h)


def sem_apply(h, prec, u, y, stream=None):
    _check(lib().sem_apply(h, PREC.get(prec, prec), _ptr(u), _ptr(y), _stream(stream)))


def sem_set_apply_variant(h, variant: int):
    _check(lib().sem_set_apply_variant(h, int(variant)))


def sem_apply_status(h, stream=None):
    _check(lib().sem_apply_status(h, _stream(stream)))


def sem_set_wait_limit(h, polls: int):
    _check(lib().sem_set_wait_limit(h, int(polls)))


def sem_rhs(h, fL, b, stream=None):
    _check(lib().sem_rhs(h, _ptr(fL), _ptr(b), _stream(stream)))


def sem_node_coords(h, xyz, stream=None):
    _check(lib().sem_node_coords(h, _ptr(xyz), _stream(stream)))


def sem_glo_num(h, glo, stream=None):
    _check(lib().sem_glo_num(h, _ptr(glo), _stream(stream)))


def sem_diag(h, d, stream=None):
    _check(lib().sem_diag(h, _ptr(d), _stream(stream)))


def sem_dot(h, x, y, out, stream=None):
    _check(lib().sem_dot(h, _ptr(x), _ptr(y), _ptr(out), _stream(stream)))


def sem_get_info(h) -> SemInfo:
    info = SemInfo()
    _check(lib().sem_get_info(h, ctypes.byref(info)))
    return info


def sem_pcg(h, b, x, opts: SemPcgOpts, stream=None, raise_on_error=True) -> SemPcgResult:
    res = SemPcgResult()
    st = lib().sem_pcg(h, _ptr(b), _ptr(x), ctypes.byref(opts), ctypes.byref(res), _stream(stream))
    if raise_on_error:
        _check(st)
    return res


# ------------------------------------------------------------------------------------------
# convenience wrapper
# ------------------------------------------------------------------------------------------
class Problem:
    """One spectral-element problem set up on the current CUDA device.

    Host inputs (numpy): ``vertices`` [E, 8, 3]; optional ``glo_num`` [E, n^3] int64 with ``nglobal``;
    ``kappa_modes`` [m, 5] or nodal ``kappa`` [E, n^3]; nodal ``alpha``; ``bc`` one of "none", "box",
    "mask" (with ``dirichlet`` flags [nglobal]).  ``features`` picks the factor sets to build.
    """

    def __init__(self, N, vertices, box=None, glo_num=None, nglobal=0, kappa_modes=None, kappa=None, alpha=None,
                 bc="box", dirichlet=None, features=SEM_FEAT_FP64 | SEM_FEAT_FP32 | SEM_FEAT_PCG, stream=None):
        import torch

        self._keep = []

        def host(a, dtype):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dtype)
            self._keep.append(a)
            return a

        v = host(vertices, np.float64)
        E = v.shape[0]
        d = SemDesc()
        d.N = int(N)
        bx = box if box is not None else (E, 1, 1)
        d.box[0], d.box[1], d.box[2] = (int(b) for b in bx)
        d.nelem = E
        d.vertices = _ptr(v)
        g = host(glo_num, np.int64)
        d.glo_num = _ptr(g)
        d.nglobal = int(nglobal)
        km = host(kappa_modes, np.float64)
        d.kappa_nmodes = 0 if km is None else int(km.shape[0])
        d.kappa_modes = _ptr(km)
        d.kappa = _ptr(host(kappa, np.float64))
        d.alpha = _ptr(host(alpha, np.float64))
        d.bc = {"none": SEM_BC_NONE, "box": SEM_BC_BOX, "mask": SEM_BC_MASK}[bc] if isinstance(bc, str) else int(bc)
        d.dirichlet = _ptr(host(dirichlet, np.uint8))
        self.desc = d
        self.features = features
        nbytes = sem_workspace_size(d, features)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.handle = sem_setup(d, features, self.workspace, stream)
        info = sem_get_info(self.handle)
        self.N, self.nelem, self.nglobal, self.nlocal = info.N, info.nelem, info.nglobal, info.nlocal
        self._keep = []  # host arrays are only read during set-up

    def close(self):
        if getattr(self, "handle", None):
            sem_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_apply_variant(self, variant: int):
        sem_set_apply_variant(self.handle, variant)

    def apply_status(self, stream=None):
        """Raises SemError(SEM_ERR_TIMEOUT) if an apply gave up waiting for a staged copy."""
        sem_apply_status(self.handle, stream)

    def set_wait_limit(self, polls: int):
        """Polls before a staged copy's bounded wait gives up (negative: the default)."""
        sem_set_wait_limit(self.handle, polls)

    # ---- operator and helpers ----
    def apply(self, u, y=None, prec="fp64", stream=None):
        import torch

        p = PREC.get(prec, prec)
        dt = torch.float32 if p in FP32_VECTOR_PRECS else torch.float64
        if u.dtype != dt or not u.is_cuda or not u.is_contiguous() or u.numel() != self.nglobal:
            raise ValueError(f"u must be a contiguous CUDA {dt} vector of length {self.nglobal}")
        if y is None:
            y = torch.empty_like(u)
        sem_apply(self.handle, p, u, y, stream)
        return y

    def rhs(self, fL, stream=None):
        import torch

        fL = fL.contiguous()
        b = torch.empty(self.nglobal, dtype=torch.float64, device="cuda")
        sem_rhs(self.handle, fL, b, stream)
        return b

    def node_coords(self, stream=None):
        import torch

        xyz = torch.empty((self.nelem, (self.N + 1) ** 3, 3), dtype=torch.float64, device="cuda")
        sem_node_coords(self.handle, xyz, stream)
        return xyz

    def glo_num(self, stream=None):
        import torch

        g = torch.empty((self.nelem, (self.N + 1) ** 3), dtype=torch.int64, device="cuda")
        sem_glo_num(self.handle, g, stream)
        return g

    def dot(self, x, y, stream=None):
        """FP64 inner product of two global vectors (deterministic order); returns a 1-element tensor."""
        import torch

        out = torch.empty(1, dtype=torch.float64, device="cuda")
        sem_dot(self.handle, x, y, out, stream)
        return out

    def diag(self, stream=None):
        import torch

        d = torch.empty(self.nglobal, dtype=torch.float64, device="cuda")
        sem_diag(self.handle, d, stream)
        return d

    def residual(self, b, x, prec="fp64_emu", stream=None):
        """r = M (b - A x) with an FP64-accurate apply."""
        import torch

        r = torch.empty_like(b)
        _check(lib().sem_residual(self.handle, PREC[prec], _ptr(b), _ptr(x), _ptr(r), _stream(stream)))
        return r

    def mlp_samples(self, r, elems, eps=MLP_EPS, jacobi_base=True, stream=None):
        """Training pairs of elements ``elems`` for the global residual r (sem_mlp_samples):
        features X [s, n^3+6], targets T [s, n^3] and the most local solver steps any sample took."""
        import torch

        n3 = (self.N + 1) ** 3
        elems = elems.to(torch.int32).contiguous()
        X = torch.empty((elems.numel(), n3 + 6), dtype=torch.float32, device="cuda")
        T = torch.empty((elems.numel(), n3), dtype=torch.float32, device="cuda")
        its = torch.zeros(1, dtype=torch.int32, device="cuda")
        _check(lib().sem_mlp_samples(self.handle, _ptr(r), elems.numel(), _ptr(elems), float(eps),
                                     1 if jacobi_base else 0, _ptr(X), _ptr(T), _ptr(its), _stream(stream)))
        return X, T, its

    def mlp_load(self, params, jacobi_base=True, stream=None):
        _check(lib().sem_mlp_load(self.handle, _ptr(params.contiguous()), 1 if jacobi_base else 0, _stream(stream)))

    def mlp_set_fused(self, on=True):
        """Three layers in one launch (True, the default) or one launch per layer."""
        _check(lib().sem_mlp_set_fused(self.handle, 1 if on else 0))

    def mlp_precond(self, r, stream=None):
        import torch

        z = torch.empty_like(r)
        _check(lib().sem_mlp_precond(self.handle, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def pcg(self, b, x0=None, rtol=1e-10, max_it=20000, mode="fp64", apply_prec="fp64", inner_rtol=1e-4,
            check_every=25, use_graph=True, stream=None, raise_on_error=True, inner_prec="fp32", history=0):
        """history > 0: info["history"] holds up to that many (iterations, relative residual) pairs, one
        per host check (sem_pcg_opts.history)."""
        import torch

        x = torch.zeros_like(b) if x0 is None else x0.clone()
        o = SemPcgOpts()
        o.rtol = rtol
        o.max_it = max_it
        o.mode = {"fp64": SEM_SOLVE_FP64, "ir": SEM_SOLVE_IR, "fcg_mlp": SEM_SOLVE_FCG_MLP}[mode]
        o.apply_prec = PREC[apply_prec]
        o.inner_rtol = inner_rtol
        o.check_every = check_every
        o.use_graph = 1 if use_graph else 0
        o.inner_prec = PREC[inner_prec]
        hbuf = None
        if history > 0:
            hbuf = (ctypes.c_double * (2 * int(history)))()
            o.history_cap = int(history)
            o.history = ctypes.cast(hbuf, ctypes.POINTER(ctypes.c_double))
        res = sem_pcg(self.handle, b, x, o, stream, raise_on_error=raise_on_error)
        info = {"status": STATUS_NAMES[res.status], "iterations": res.iterations, "outer": res.outer,
                "true_relres": res.true_relres, "recursive_relres": res.recursive_relres,
                "fallbacks": res.fallbacks}
        if hbuf is not None:
            info["history"] = [(int(hbuf[2 * i]), float(hbuf[2 * i + 1])) for i in range(res.history_len)]
        return x, info


class Batch:
    """Many independent structured-box problems solved together (see sem_batch_* in include/sem.h).

    ``problems``: list of dicts with keys N, vertices, box and optionally kappa_modes, bc.
    """

    def __init__(self, problems, features=SEM_FEAT_EMU | SEM_FEAT_FP32, stream=None):
        import torch

        self._keep = []
        n = len(problems)
        descs = (SemDesc * n)()
        for i, pr in enumerate(problems):
            v = np.ascontiguousarray(pr["vertices"], dtype=np.float64)
            self._keep.append(v)
            d = descs[i]
            d.N = int(pr["N"])
            d.box[0], d.box[1], d.box[2] = (int(b) for b in pr["box"])
            d.nelem = v.shape[0]
            d.vertices = v.ctypes.data
            km = pr.get("kappa_modes")
            if km is not None:
                km = np.ascontiguousarray(km, dtype=np.float64)
                self._keep.append(km)
                d.kappa_nmodes = km.shape[0]
                d.kappa_modes = km.ctypes.data
            d.bc = {"none": SEM_BC_NONE, "box": SEM_BC_BOX}[pr.get("bc", "box")]
        nbytes = ctypes.c_size_t(0)
        _check(lib().sem_batch_workspace_size(descs, n, features, ctypes.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p(None)
        _check(lib().sem_batch_setup(descs, n, features, _ptr(self.workspace), nbytes.value, _stream(stream),
                                     ctypes.byref(h)))
        self.handle = h
        self._keep = []
        self.nprob = n
        self.offsets, self.sizes, self.nlocal = [], [], []
        for i in range(n):
            info, off = SemInfo(), ctypes.c_int64(0)
            _check(lib().sem_batch_info(h, i, ctypes.byref(info), ctypes.byref(off)))
            self.offsets.append(off.value)
            self.sizes.append(info.nglobal)
            self.nlocal.append(info.nlocal)
        self.nglobal = self.offsets[-1] + self.sizes[-1]
        self.orders = sorted({int(pr["N"]) for pr in problems})

    def close(self):
        if getattr(self, "handle", None):
            lib().sem_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def problem(self, p):
        """(handle, global offset, nglobal) of problem p; the handle stays owned by the batch."""
        h = ctypes.c_void_p(None)
        _check(lib().sem_batch_handle(self.handle, p, ctypes.byref(h)))
        return h, self.offsets[p], self.sizes[p]

    def set_variant(self, N, variant):
        _check(lib().sem_batch_set_variant(self.handle, int(N), int(variant)))

    def set_wait_limit(self, polls: int):
        """Polls before a grid-wide wait of the fused step gives up (negative: the default)."""
        _check(lib().sem_batch_set_wait_limit(self.handle, int(polls)))

    def set_fused(self, fused: bool):
        """Inner steps of pcg as the fused step kernel (True) or as per-order-group launches."""
        _check(lib().sem_batch_set_fused(self.handle, 1 if fused else 0))

    def fused_state(self):
        """(available, in_use) of the fused step kernel for this batch."""
        a, u = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(lib().sem_batch_get_fused(self.handle, ctypes.byref(a), ctypes.byref(u)))
        return bool(a.value), bool(u.value)

    def apply(self, u, y, prec="fp32", stream=None):
        _check(lib().sem_batch_apply(self.handle, PREC.get(prec, prec), _ptr(u), _ptr(y), _stream(stream)))
        return y

    def rhs(self, fL, stream=None):
        import torch

        b = torch.empty(self.nglobal, dtype=torch.float64, device="cuda")
        _check(lib().sem_batch_rhs(self.handle, _ptr(fL.contiguous()), _ptr(b), _stream(stream)))
        return b

    def rhs_problem(self, p, fL, b, stream=None):
        """Problem p's lumped-mass right-hand side from its nodal values fL [nelem_p, n_p^3] into its
        slice of the concatenated b (one problem at a time: no concatenated nodal array)."""
        h, off, n = self.problem(p)
        sem_rhs(h, fL.contiguous(), b[off:off + n], stream)
        return b

    def node_coords(self, p, stream=None):
        import torch

        h, _, _ = self.problem(p)
        xyz = torch.empty((self.nlocal[p], 3), dtype=torch.float64, device="cuda")
        sem_node_coords(h, xyz, stream)
        return xyz

    def pcg(self, b, x0=None, rtol=1e-10, max_it=20000, apply_prec="fp64_emu", inner_rtol=1e-4, check_every=16,
            use_graph=True, stream=None, multi_launch=False):
        """multi_launch: one launch per order group and four vector kernels per inner step instead of
        the fused step kernel."""
        import torch

        x = torch.zeros_like(b) if x0 is None else x0.clone()
        o = SemPcgOpts()
        o.rtol, o.max_it, o.mode, o.apply_prec = rtol, max_it, SEM_SOLVE_IR, PREC[apply_prec]
        o.inner_rtol, o.check_every, o.use_graph = inner_rtol, check_every, 1 if use_graph else 0
        o.flags = SEM_PCG_MULTI_LAUNCH if multi_launch else 0
        res = (SemPcgResult * self.nprob)()
        st = lib().sem_batch_pcg(self.handle, _ptr(b), _ptr(x), ctypes.byref(o), res, _stream(stream))
        out = [{"status": STATUS_NAMES[r.status], "iterations": r.iterations, "outer": r.outer,
                "true_relres": r.true_relres} for r in res]
        return x, out, STATUS_NAMES.get(st, st)


# ------------------------------------------------------------------------------------------
# learned preconditioner: network shape, forward pass and training steps on the device
# ------------------------------------------------------------------------------------------
def mlp_param_count(N: int, h1: int = MLP_H1, h2: int = MLP_H2) -> int:
    c = ctypes.c_int64(0)
    _check(lib().sem_mlp_param_count(N, h1, h2, ctypes.byref(c)))
    return c.value


def mlp_forward(N, params, X, h1=MLP_H1, h2=MLP_H2, stream=None):
    import torch

    B = X.shape[0]
    n3 = (N + 1) ** 3
    H1 = torch.empty((B, h1), dtype=torch.float32, device="cuda")
    H2 = torch.empty((B, h2), dtype=torch.float32, device="cuda")
    O = torch.empty((B, n3), dtype=torch.float32, device="cuda")
    _check(lib().sem_mlp_forward(N, h1, h2, _ptr(params), _ptr(X.contiguous()), B, _ptr(H1), _ptr(H2), _ptr(O),
                                 _stream(stream)))
    return H1, H2, O


def gemm_bf16(A, Bt, bias=None, relu=False, K=None, err=None, stream=None):
    """C = act(A[:, :K] Bt[:, :K]^T + bias) on the tensor cores (sem_gemm_bf16).

    A: bfloat16 [M][lda], Bt: bfloat16 [N][ldb] on the device (leading dimensions multiples of 8);
    K defaults to A.shape[1].  Returns float32 [M][N'] with N' = N rounded up to a multiple of 8
    (columns beyond N untouched zeros)."""
    import torch

    M, lda = A.shape
    N, ldb = Bt.shape
    K = lda if K is None else K
    ldc = (N + 7) // 8 * 8
    C = torch.zeros((M, ldc), dtype=torch.float32, device=A.device)
    _check(lib().sem_gemm_bf16(M, N, K, _ptr(A), lda, _ptr(Bt), ldb, _ptr(bias), _ptr(C), ldc, 1 if relu else 0,
                               _ptr(err), _stream(stream)))
    return C


def mlp_layers_bf16(X, nin, W1t, W2t, W3t, b1, b2, b3, err=None, stream=None, out=None):
    """The three layers in one launch (sem_mlp_layers_bf16): X bfloat16 [M][ldx] (nin features),
    W1t [256][ldx], W2t [256][256], W3t [nout][256] bfloat16, b1, b2, b3 float32; returns float32
    [M][nout] (written into out when given)."""
    import torch

    M, ldx = X.shape
    nout = W3t.shape[0]
    O = torch.zeros((M, nout), dtype=torch.float32, device=X.device) if out is None else out
    if O.shape != (M, nout) or O.dtype != torch.float32 or not O.is_contiguous():
        raise ValueError("out must be a contiguous float32 [M][nout] tensor")
    _check(lib().sem_mlp_layers_bf16(M, nin, ldx, nout, _ptr(X), _ptr(W1t), _ptr(W2t), _ptr(W3t), _ptr(b1), _ptr(b2),
                                     _ptr(b3), _ptr(O), _ptr(err), _stream(stream)))
    return O


class MlpTrainer:
    """Adam training of the element network on the device (sem_mlp_train_step)."""

    def __init__(self, N, params, batch, h1=MLP_H1, h2=MLP_H2, lr=1e-3):
        import torch

        self.N, self.h1, self.h2, self.batch, self.lr = N, h1, h2, batch, lr
        self.params = params.contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        nb = ctypes.c_size_t(0)
        _check(lib().sem_mlp_train_scratch(N, h1, h2, batch, ctypes.byref(nb)))
        self.scratch = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.step_count = 0

    def step(self, X, T, lr=None, grad_out=None, stream=None):
        self.step_count += 1
        _check(lib().sem_mlp_train_step(self.N, self.h1, self.h2, _ptr(self.params), _ptr(self.m), _ptr(self.v),
                                        self.step_count, float(self.lr if lr is None else lr), _ptr(X.contiguous()),
                                        _ptr(T.contiguous()), X.shape[0], _ptr(self.scratch), self.scratch.numel(),
                                        _ptr(self.loss), _ptr(grad_out), _stream(stream)))
        return self.loss


# ---- finite-difference wave step (include/sem_fd.h) ----
FD_MAX_RADIUS = 7


def fd_weights(r: int) -> np.ndarray:
    """c_{-r..r}: central second-derivative weights of order 2r (sem_fd_weights, host only)."""
    c = np.zeros(2 * r + 1) if 1 <= r <= FD_MAX_RADIUS else np.zeros(1)
    _check(lib().sem_fd_weights(int(r), c.ctypes.data))
    return c


def fd_step(u, uprev_next, r: int, dt: float, dx: float, dy: float, stream=None):
    """One leapfrog step of u_tt = u_xx + u_yy (sem_fd_step): u is u_n ([h][w] CUDA tensor, float32
    or float64); uprev_next holds u_{n-1} and is overwritten with u_{n+1}.  Returns uprev_next."""
    import torch

    if u.dtype not in (torch.float32, torch.float64) or uprev_next.dtype != u.dtype:
        raise ValueError("u and uprev_next must both be float32 or both float64")
    if (u.dim() != 2 or u.shape != uprev_next.shape or not u.is_cuda or not uprev_next.is_cuda
            or not u.is_contiguous() or not uprev_next.is_contiguous()):
        raise ValueError("u and uprev_next must be contiguous CUDA grids [h][w] of the same shape")
    prec = SEM_FP64 if u.dtype == torch.float64 else SEM_FP32
    h, w = u.shape
    _check(lib().sem_fd_step(prec, int(r), int(w), int(h), float(dt), float(dx), float(dy), _ptr(u),
                             _ptr(uprev_next), _stream(stream)))
    return uprev_next


def fd_status(stream=None):
    """Raises SemError (SEM_ERR_TIMEOUT) if a step since the last call gave up waiting for its tile
    copy (sem_fd_status; synchronises the stream)."""
    _check(lib().sem_fd_status(_stream(stream)))


def fd_run(u, uprev, nsteps: int, r: int, dt: float, dx: float, dy: float, stream=None):
    """nsteps leapfrog steps from (u_n, u_{n-1}) = (u, uprev), alternating the two buffers; returns
    the tensors holding (u_{n+nsteps}, u_{n+nsteps-1})."""
    cur, prev = u, uprev
    for _ in range(nsteps):
        fd_step(cur, prev, r, dt, dx, dy, stream)
        cur, prev = prev, cur
    return cur, prev


# ---- DG shallow-water volume kernel (include/sem_dg.h) ----
DG_MAX_ORDER = 8


def dg_np(N: int) -> int:
    return (N + 1) * (N + 2) // 2


def dg_operators(N: int):
    """(Drw, Dsw) of order N as FP64 numpy arrays (sem_dg_operators, host only)."""
    n = dg_np(N) if 1 <= N <= DG_MAX_ORDER else 1
    Drw, Dsw = np.zeros((n, n)), np.zeros((n, n))
    _check(lib().sem_dg_operators(int(N), Drw.ctypes.data, Dsw.ctypes.data))
    return Drw, Dsw


def dg_load_operators(N: int, dtype, stream=None):
    """Device operator block of order N (sem_dg_load_operators) as a uint8 CUDA tensor."""
    import torch

    prec = SEM_FP64 if dtype == torch.float64 else SEM_FP32
    nb = ctypes.c_size_t(0)
    _check(lib().sem_dg_operator_bytes(int(N), prec, ctypes.byref(nb)))
    ops = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    _check(lib().sem_dg_load_operators(int(N), prec, _ptr(ops), nb.value, _stream(stream)))
    return ops


def dg_volume(N: int, Q, Bxy, geo, g: float, ops, out=None, stream=None):
    """Volume right-hand side [E][3][Np] (sem_dg_volume) for CUDA tensors Q [E][3][Np], Bxy [E][2][Np],
    geo [E][4] of one dtype (float32 or float64) and the operator block from dg_load_operators."""
    import torch

    if Q.dtype not in (torch.float32, torch.float64) or any(t.dtype != Q.dtype for t in (Bxy, geo)):
        raise ValueError("Q, Bxy and geo must share one dtype, float32 or float64")
    E, n = Q.shape[0], dg_np(N)
    if tuple(Q.shape) != (E, 3, n) or tuple(Bxy.shape) != (E, 2, n) or tuple(geo.shape) != (E, 4):
        raise ValueError("shapes must be Q [E][3][Np], Bxy [E][2][Np], geo [E][4]")
    if not all(t.is_cuda and t.is_contiguous() for t in (Q, Bxy, geo, ops)):
        raise ValueError("inputs must be contiguous CUDA tensors")
    if out is None:
        out = torch.empty_like(Q)
    prec = SEM_FP64 if Q.dtype == torch.float64 else SEM_FP32
    _check(lib().sem_dg_volume(prec, int(N), int(E), float(g), _ptr(ops), _ptr(Q), _ptr(Bxy), _ptr(geo), _ptr(out),
                               _stream(stream)))
    return out


def dg_geometry(verts, dtype, stream=None):
    """geo [E][4] = (rx, ry, sx, sy) on the device (sem_dg_geometry) from vertices [E][3][2] (numpy or
    CUDA tensor, float64, counter-clockwise)."""
    import torch

    v = torch.as_tensor(verts, dtype=torch.float64).cuda().contiguous()
    E = v.shape[0]
    geo = torch.empty(E, 4, dtype=dtype, device="cuda")
    prec = SEM_FP64 if dtype == torch.float64 else SEM_FP32
    _check(lib().sem_dg_geometry(prec, int(E), _ptr(v), _ptr(geo), _stream(stream)))
    return geo
