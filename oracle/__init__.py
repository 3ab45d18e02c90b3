"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never imports it and
shares no code with it.  Every routine here is plain, slow and meant to be
checked by eye against the passages it cites:

* ``svdvals``        -- Householder bidiagonalisation + implicit-shift
                        Golub-Kahan QR (svdvals.c); the reference result for
                        the whole pipeline of the paper's Section 5.1.1.
* ``bidiag``         -- the one-stage bidiagonalisation on its own.
* ``bdsvd``          -- bidiagonal singular values by Golub-Kahan QR.
* ``jacobi_svdvals`` -- second, independent oracle (one-sided Jacobi).
* ``mlp`` / ``tuner`` submodules -- the learned cost model and the tuner's
                        search-space / argmin definitions (Eq. 1).

Parity status of each function is stated in the module that defines it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "svdvals.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile svdvals.c with gcc + OpenMP into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of svdvals.c (used by the mutation tests)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    src, "-o", out_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_svdvals.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, dp, ctypes.c_int]
    lib.oracle_bidiag.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, dp, dp, ctypes.c_int]
    lib.oracle_bdsvd.argtypes = [ctypes.c_int, dp, dp, dp]
    lib.oracle_jacobi_svdvals.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, dp]
    for f in (lib.oracle_svdvals, lib.oracle_bidiag, lib.oracle_bdsvd, lib.oracle_jacobi_svdvals):
        f.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load the oracle library (building it first if needed)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st: int, what: str):
    if st < 0:
        raise ValueError(f"{what}: bad argument (status {st})")
    if st > 0:
        raise RuntimeError(f"{what}: no convergence ({st} values unconverged)")


def svdvals(A, nthreads: int = 0, lib=None) -> np.ndarray:
    """Singular values (descending) of a dense real matrix, FP64."""
    lib = lib or load()
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    m, n = A.shape
    S = np.zeros(min(m, n), dtype=np.float64)
    if m == 0 or n == 0:
        return S
    _check(lib.oracle_svdvals(m, n, _dp(A), max(m, 1), _dp(S), int(nthreads)), "oracle_svdvals")
    return S


def bidiag(A, nthreads: int = 0, lib=None):
    """One-stage Householder bidiagonalisation of A (m >= n): returns (d, e)."""
    lib = lib or load()
    W = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = W.shape
    if m < n:
        raise ValueError("bidiag expects m >= n")
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 0) + 1)
    _check(lib.oracle_bidiag(m, n, _dp(W), max(m, 1), _dp(d), _dp(e), int(nthreads)), "oracle_bidiag")
    return d, e[: max(n - 1, 0)]


def bdsvd(d, e, lib=None) -> np.ndarray:
    """Singular values of the upper bidiagonal matrix (d, e), descending."""
    lib = lib or load()
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.shape[0]
    e = np.ascontiguousarray(e, dtype=np.float64)
    if e.shape[0] != max(n - 1, 0):
        raise ValueError("e must have n-1 entries")
    e1 = np.zeros(max(n, 1))
    e1[: e.shape[0]] = e
    S = np.zeros(n)
    if n:
        _check(lib.oracle_bdsvd(n, _dp(d), _dp(e1), _dp(S)), "oracle_bdsvd")
    return S


def jacobi_svdvals(A, lib=None) -> np.ndarray:
    """Second oracle: one-sided Jacobi singular values (small matrices)."""
    lib = lib or load()
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    m, n = A.shape
    S = np.zeros(min(m, n))
    if m and n:
        _check(lib.oracle_jacobi_svdvals(m, n, _dp(A), max(m, 1), _dp(S)), "oracle_jacobi_svdvals")
    return S


def bidiagonal_dense(d, e) -> np.ndarray:
    """The dense upper bidiagonal matrix with diagonal d and superdiagonal e."""
    n = len(d)
    B = np.diag(np.asarray(d, dtype=np.float64))
    if n > 1:
        B[np.arange(n - 1), np.arange(1, n)] = e
    return B
