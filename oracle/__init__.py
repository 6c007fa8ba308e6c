"""Plain FP64 CPU oracle for the SEM screened-Poisson operator of arXiv 1403.0968 §4.2.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; the product library never does.  The arithmetic lives in ``sem_oracle.c``
(plain C, FP64, OpenMP over elements); this module compiles it with gcc and wraps it with
ctypes and numpy.  It imports nothing from the CUDA package and shares no code with it.

Parity status of each function (pins in tests/test_oracle_pins.py):
  gll, lagrange_deriv        pinned: closed-form GLL tables N=1..4, quadrature exactness,
                             D exact on polynomials, corner values -N(N+1)/4, Legendre form of D
  factors, node_coords       pinned: sum of wJ = domain volume; affine-element closed forms
  element_matrix (O1)        pinned: u^T A u = integral |grad u|^2, A 1 = 0, symmetry, PSD
  apply_local / apply (O2)   pinned: equals O1 columns on 1-8 perturbed elements
  diag                       pinned: equals the diagonal of the dense assembled O1 matrix
  rhs, pcg                   pinned: dense direct solve; manufactured-solution convergence
  solvers.ir, solvers.fcg    pinned: dense direct solve; fcg with fixed Jacobi equals pcg; varying
                             and rejected preconditioners; ir residual contraction (oracle/solvers.py)
  mlp (oracle/mlp.py)        see its docstring; fd (oracle/fd.py), dg (oracle/dg.py) likewise
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsem_oracle.so")
_lock = threading.Lock()
_lib = None

_i32, _i64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile sem_oracle.c into oracle/_build/libsem_oracle.so (gcc, -O2, OpenMP, IEEE math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_gll.argtypes = [_i32, _p, _p]
            L.orc_gll.restype = _i32
            L.orc_threads.argtypes = [_i32]
            L.orc_threads.restype = _i32
            L.orc_lagrange_deriv.argtypes = [_i32, _p, _p]
            L.orc_kappa.argtypes = [_i32, _p, _f64, _f64, _f64]
            L.orc_kappa.restype = _f64
            L.orc_node_coords.argtypes = [_i32, _i64, _p, _p]
            L.orc_node_coords.restype = _i32
            L.orc_factors.argtypes = [_i32, _i64, _p, _p, _i32, _p, _p, _p]
            L.orc_factors.restype = _i32
            L.orc_element_matrix.argtypes = [_i32, _p, _p, _p, _p]
            L.orc_element_matrix.restype = _i32
            L.orc_apply_local.argtypes = [_i32, _i64, _p, _p, _p, _p]
            L.orc_box_numbering.argtypes = [_i32, _i32, _i32, _i32, _p]
            L.orc_box_dirichlet.argtypes = [_i32, _i32, _i32, _i32, _p]
            L.orc_apply.argtypes = [_i32, _i64, _p, _p, _p, _i64, _p, _p, _p]
            L.orc_diag.argtypes = [_i32, _i64, _p, _p, _p, _i64, _p, _p]
            L.orc_rhs.argtypes = [_i32, _i64, _p, _p, _p, _i64, _p, _p]
            L.orc_pcg.argtypes = [_i32, _i64, _p, _p, _p, _i64, _p, _p, _p, _p, _f64, _i32, _p]
            L.orc_pcg.restype = _i32
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------------------------------
# 1-D ingredients
# ------------------------------------------------------------------------------------------
def threads() -> int:
    """OpenMP threads the oracle's loops use."""
    return lib().orc_threads(0)


def set_threads(n: int) -> int:
    """Sets the oracle's OpenMP thread count; returns the previous one."""
    return lib().orc_threads(int(n))


def gll(N: int):
    """GLL nodes and weights of order N (§4.2.1); returns (x, w) of length N+1."""
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().orc_gll(N, _ptr(x), _ptr(w)) != 0:
        raise ValueError("N must be >= 1")
    return x, w


def lagrange_deriv(N: int, x=None):
    """D[i, j] = l_j'(x_i) from the Lagrange product formula (§4.2.1)."""
    if x is None:
        x, _ = gll(N)
    x = _c(x, np.float64)
    D = np.zeros((N + 1, N + 1))
    lib().orc_lagrange_deriv(N, _ptr(x), _ptr(D))
    return D


def kappa(modes, xyz):
    """kappa(x) = exp(sum_m a_m cos(2 pi k_m.x + phi_m)) at points xyz[..., 3]."""
    modes = _c(modes if modes is not None else np.zeros((0, 5)), np.float64)
    pts = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    out = np.array([lib().orc_kappa(len(modes), _ptr(modes), *p) for p in pts])
    return out.reshape(np.asarray(xyz).shape[:-1])


# ------------------------------------------------------------------------------------------
# geometry and numbering
# ------------------------------------------------------------------------------------------
def node_coords(N: int, vertices):
    v = _c(vertices, np.float64)
    E = v.shape[0]
    n3 = (N + 1) ** 3
    xyz = np.zeros((E, n3, 3))
    if lib().orc_node_coords(N, E, _ptr(v), _ptr(xyz)) != 0:
        raise ValueError("bad order")
    return xyz


def factors(N: int, vertices, kappa_nodal=None, modes=None):
    """Per-node factors G[E, 6, n3] (rr, rs, rt, ss, st, tt; with w, det J, kappa) and wJ[E, n3]."""
    v = _c(vertices, np.float64)
    E = v.shape[0]
    n3 = (N + 1) ** 3
    G = np.zeros((E, 6, n3))
    wJ = np.zeros((E, n3))
    modes = _c(modes, np.float64)
    nm = 0 if modes is None else modes.shape[0]
    rc = lib().orc_factors(N, E, _ptr(v), _ptr(_c(kappa_nodal, np.float64)), nm, _ptr(modes), _ptr(G), _ptr(wJ))
    if rc == -2:
        raise ValueError("tangled element: det J <= 0")
    if rc != 0:
        raise ValueError("bad order")
    return G, wJ


def box_numbering(sx: int, sy: int, sz: int, N: int):
    n3 = (N + 1) ** 3
    glo = np.zeros((sx * sy * sz, n3), dtype=np.int64)
    lib().orc_box_numbering(sx, sy, sz, N, _ptr(glo))
    return glo


def box_nglobal(sx, sy, sz, N):
    return (sx * N + 1) * (sy * N + 1) * (sz * N + 1)


def box_dirichlet(sx: int, sy: int, sz: int, N: int):
    m = np.zeros(box_nglobal(sx, sy, sz, N), dtype=np.uint8)
    lib().orc_box_dirichlet(sx, sy, sz, N, _ptr(m))
    return m


# ------------------------------------------------------------------------------------------
# operators
# ------------------------------------------------------------------------------------------
def element_matrix(N: int, vert_e, kappa_e=None, alpha_e=None):
    """O1: dense element matrix from the weak form by quadrature (O(n^9); small N only)."""
    n3 = (N + 1) ** 3
    A = np.zeros((n3, n3))
    rc = lib().orc_element_matrix(N, _ptr(_c(vert_e, np.float64)), _ptr(_c(kappa_e, np.float64)),
                                  _ptr(_c(alpha_e, np.float64)), _ptr(A))
    if rc != 0:
        raise ValueError("bad order")
    return A


def apply_local(N: int, G, uL, wJalpha=None):
    """O2: unassembled sum-factorised operator y_L = A_L u_L on [E, n3] arrays."""
    G = _c(G, np.float64)
    uL = _c(uL, np.float64)
    E = G.shape[0]
    yL = np.zeros_like(uL)
    lib().orc_apply_local(N, E, _ptr(G), _ptr(_c(wJalpha, np.float64)), _ptr(uL), _ptr(yL))
    return yL


def apply(N: int, glo, G, u, mask=None, wJalpha=None):
    """Assembled y = M Q^T A_L Q M u on global nodes."""
    glo = _c(glo, np.int64)
    G = _c(G, np.float64)
    u = _c(u, np.float64)
    y = np.zeros_like(u)
    lib().orc_apply(N, glo.shape[0], _ptr(glo), _ptr(G), _ptr(_c(wJalpha, np.float64)), u.shape[0],
                    _ptr(_c(mask, np.uint8)), _ptr(u), _ptr(y))
    return y


def diag(N: int, glo, G, nglobal: int, mask=None, wJalpha=None):
    glo = _c(glo, np.int64)
    G = _c(G, np.float64)
    d = np.zeros(nglobal)
    lib().orc_diag(N, glo.shape[0], _ptr(glo), _ptr(G), _ptr(_c(wJalpha, np.float64)), nglobal,
                   _ptr(_c(mask, np.uint8)), _ptr(d))
    return d


def rhs(N: int, glo, wJ, fL, nglobal: int, mask=None):
    """b = M Q^T (w J f) from nodal f on [E, n3]."""
    glo = _c(glo, np.int64)
    b = np.zeros(nglobal)
    lib().orc_rhs(N, glo.shape[0], _ptr(glo), _ptr(_c(wJ, np.float64)), _ptr(_c(fL, np.float64)), nglobal,
                  _ptr(_c(mask, np.uint8)), _ptr(b))
    return b


def pcg(N: int, glo, G, b, dg, mask=None, wJalpha=None, x0=None, rtol=1e-10, max_it=10000):
    """Jacobi-PCG (§4.2.2; Saad Alg. 9.1).  Returns (x, iterations, recursive rel. residual)."""
    glo = _c(glo, np.int64)
    G = _c(G, np.float64)
    b = _c(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    res = ctypes.c_double(0.0)
    it = lib().orc_pcg(N, glo.shape[0], _ptr(glo), _ptr(G), _ptr(_c(wJalpha, np.float64)), b.shape[0],
                       _ptr(_c(mask, np.uint8)), _ptr(_c(dg, np.float64)), _ptr(b), _ptr(x), rtol, max_it,
                       ctypes.byref(res))
    return x, it, res.value


def true_relres(N: int, glo, G, b, x, mask=None, wJalpha=None):
    """||b - A x||_2 / ||b||_2 recomputed in FP64 by the oracle (the check of solve accuracy)."""
    r = np.asarray(b, dtype=np.float64) - apply(N, glo, G, x, mask=mask, wJalpha=wJalpha)
    if mask is not None:
        r[np.asarray(mask, dtype=bool)] = 0.0
    return float(np.linalg.norm(r) / np.linalg.norm(b))
