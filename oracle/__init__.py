"""Plain CPU FP64 oracle for the shared-LHS batched tri/pentadiagonal solvers
(arXiv:1909.04539, Sec. 3.1 and Sec. 4.1).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may.  The arithmetic lives in ``bsolve_oracle.c`` (plain loops,
true divisions, the paper's step order); this module only marshals numpy
arrays into it.  It shares no code with the CUDA library.

Layouts: an interleaved batch is a C-contiguous array of shape (N, M) holding
row i of system j at [i, j] (the paper's ``B[i*M + j]``); a system-contiguous
("strided") batch has shape (M, N).  Bands are (width, N) arrays, width 3
(a, b, c; diagonal b) or 5 (a, b, c, d, e; diagonal c), as in the paper.

Parity status of every function here is pinned by ``tests/test_oracle.py``.
"""
from __future__ import annotations

import contextlib
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def _load(path: str) -> ctypes.CDLL:
    L = ctypes.CDLL(path)
    i64, dp, i32 = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.oracle_tri_factor.argtypes = [i64, dp, dp, dp]
    L.oracle_penta_factor.argtypes = [i64, dp, dp]
    L.oracle_solve.argtypes = [i32, i64, dp, dp, i64, i64, i64]
    L.oracle_transpose_bands.argtypes = [i32, i64, dp, dp]
    L.oracle_transpose_bands.restype = None
    L.oracle_band_matvec.argtypes = [i32, i64, dp, dp, dp, i64, i64, i64]
    L.oracle_band_matvec.restype = None
    L.oracle_residual.argtypes = [i32, i64, dp, dp, dp, dp, i64, i64, i64]
    L.oracle_residual.restype = None
    L.oracle_band_grad.argtypes = [i32, i64, dp, dp, i64, i64, i64, dp]
    L.oracle_band_grad.restype = None
    L.oracle_periodic_tri_solve.argtypes = [i64, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, dp, i64, i64, i64]
    L.oracle_periodic_tri_solve_bands.argtypes = [i64, dp, dp, i64, i64, i64]
    L.oracle_band_grad_periodic.argtypes = [i64, dp, dp, i64, i64, i64, dp]
    L.oracle_band_grad_periodic.restype = None
    L.oracle_adi_halfstep.argtypes = [i64, i64, ctypes.c_double, dp, dp, i32]
    L.oracle_adi_halfstep_bands.argtypes = [i64, i64, ctypes.c_double, i32, dp, dp, dp, i32, i32]
    L.oracle_cn_steps.argtypes = [i32, i64, dp, i32, dp, i64, i64, i64, i32]
    L.oracle_num_threads.argtypes = []
    L.oracle_set_threads.argtypes = [i32]
    L.oracle_set_threads.restype = None
    return L


def lib() -> ctypes.CDLL:
    """Load (building if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        _LIB = _load(_build.build())
    return _LIB


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every call to another build of the oracle source
    (the mutation tests use this to show that the pins catch planted bugs)."""
    global _LIB
    saved = _LIB
    _LIB = _load(path)
    try:
        yield
    finally:
        _LIB = saved


def _p(x: np.ndarray):
    assert x.dtype == np.float64 and x.flags.c_contiguous
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _strides(X: np.ndarray, layout: str):
    if layout == "interleaved":
        N, M = X.shape
        return N, M, M, 1
    if layout == "strided":
        M, N = X.shape
        return N, M, 1, N
    raise ValueError(layout)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


class OracleError(RuntimeError):
    pass


def _bands(bands) -> np.ndarray:
    b = np.ascontiguousarray(bands, dtype=np.float64)
    if b.ndim != 2 or b.shape[0] not in (3, 5):
        raise ValueError("bands must have shape (3, N) or (5, N)")
    return b


def tri_factor(bands):
    """Thomas pre-factorisation (Sec. 3.1): returns (chat, pivots)."""
    b = _bands(bands)
    N = b.shape[1]
    chat, piv = np.zeros(N), np.zeros(N)
    st = lib().oracle_tri_factor(N, _p(b), _p(chat), _p(piv))
    if st != 0:
        raise OracleError(f"zero or non-finite pivot at row {st}")
    return chat, piv


def penta_factor(bands):
    """A = L R (Sec. 4.1): returns (alpha, beta, gamma, delta, eps)."""
    b = _bands(bands)
    N = b.shape[1]
    f = np.zeros((5, N))
    st = lib().oracle_penta_factor(N, _p(b), _p(f))
    if st != 0:
        raise OracleError(f"penta factorisation failed (status {st})")
    return tuple(f[k].copy() for k in range(5))


def solve(bands, B, layout: str = "interleaved") -> np.ndarray:
    """X = A^{-1} B for every system of the batch (copy; B is untouched)."""
    b = _bands(bands)
    X = np.array(B, dtype=np.float64, order="C", copy=True)
    N, M, rs, ss = _strides(X, layout)
    if N != b.shape[1]:
        raise ValueError("band length and row count differ")
    st = lib().oracle_solve(b.shape[0], N, _p(b), _p(X), M, rs, ss)
    if st != 0:
        raise OracleError(f"solve failed (status {st})")
    return X


def transpose_bands(bands) -> np.ndarray:
    b = _bands(bands)
    out = np.zeros_like(b)
    lib().oracle_transpose_bands(b.shape[0], b.shape[1], _p(b), _p(out))
    return out


def solve_adjoint(bands, G, layout: str = "interleaved") -> np.ndarray:
    """A^{-T} G: the definition written out, a solve with the bands of A^T."""
    return solve(transpose_bands(bands), G, layout)


def matvec(bands, X, layout: str = "interleaved") -> np.ndarray:
    b = _bands(bands)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.zeros_like(X)
    N, M, rs, ss = _strides(X, layout)
    lib().oracle_band_matvec(b.shape[0], N, _p(b), _p(X), _p(Y), M, rs, ss)
    return Y


def residual(bands, B, X, layout: str = "interleaved") -> np.ndarray:
    b = _bands(bands)
    B = np.ascontiguousarray(B, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    R = np.zeros_like(X)
    N, M, rs, ss = _strides(X, layout)
    lib().oracle_residual(b.shape[0], N, _p(b), _p(B), _p(X), _p(R), M, rs, ss)
    return R


def band_grad(width: int, GB, X, layout: str = "interleaved") -> np.ndarray:
    """dL/d(bands) = -(A^{-T} G) X^T restricted to the bands; shape (width, N)."""
    GB = np.ascontiguousarray(GB, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, M, rs, ss = _strides(X, layout)
    out = np.zeros((width, N))
    lib().oracle_band_grad(width, N, _p(GB), _p(X), M, rs, ss, _p(out))
    return out


def periodic_tri_solve(a: float, b: float, c: float, B, layout: str = "interleaved"):
    """Constant periodic tridiagonal solve via Sherman-Morrison (Sec. 3.3)."""
    X = np.array(B, dtype=np.float64, order="C", copy=True)
    N, M, rs, ss = _strides(X, layout)
    st = lib().oracle_periodic_tri_solve(N, a, b, c, _p(X), M, rs, ss)
    if st != 0:
        raise OracleError(f"periodic solve failed (status {st})")
    return X


def periodic_tri_solve_bands(bands, B, layout: str = "interleaved"):
    """Periodic tridiagonal solve via Sherman-Morrison (Sec. 3.3), general
    bands: row i has a_i at column i-1 and c_i at column i+1 modulo N."""
    b = _bands(bands)
    X = np.array(B, dtype=np.float64, order="C", copy=True)
    N, M, rs, ss = _strides(X, layout)
    st = lib().oracle_periodic_tri_solve_bands(N, _p(b), _p(X), M, rs, ss)
    if st != 0:
        raise OracleError(f"periodic solve failed (status {st})")
    return X


def periodic_transpose_bands(bands) -> np.ndarray:
    """Bands of A^T for a periodic tridiagonal A: row i of A^T has c_{i-1}
    at column i-1 and a_{i+1} at column i+1 (indices modulo N)."""
    b = np.asarray(bands, dtype=np.float64)
    return np.stack([np.roll(b[2], 1), b[1], np.roll(b[0], -1)])


def periodic_solve_adjoint(bands, G, layout: str = "interleaved"):
    """A^{-T} G for a periodic tridiagonal A: the periodic solve of A^T."""
    return periodic_tri_solve_bands(periodic_transpose_bands(bands), G, layout)


def band_grad_periodic(GB, X, layout: str = "interleaved") -> np.ndarray:
    """-(GB) X^T on the 3N entries of a periodic tridiagonal matrix."""
    GB = np.ascontiguousarray(GB, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, M, rs, ss = _strides(X, layout)
    out = np.zeros((3, N))
    lib().oracle_band_grad_periodic(N, _p(GB), _p(X), M, rs, ss, _p(out))
    return out


def cn_steps(bands, C, steps: int = 1, periodic: bool = False, layout: str = "interleaved") -> np.ndarray:
    """``steps`` Crank-Nicolson steps C <- A^{-1} (2I - A) C (the paper's
    diffusion and hyperdiffusion benchmarks); ``periodic``: A is the periodic
    tridiagonal matrix of ``bands``."""
    b = _bands(bands)
    X = np.array(C, dtype=np.float64, order="C", copy=True)
    N, M, rs, ss = _strides(X, layout)
    st = lib().oracle_cn_steps(b.shape[0], N, _p(b), int(bool(periodic)), _p(X), M, rs, ss, int(steps))
    if st != 0:
        raise OracleError(f"CN step failed (status {st})")
    return X


def adi_halfstep(u, r: float, implicit_axis: int) -> np.ndarray:
    """One Peaceman-Rachford half-step on u[y, x] (Dirichlet 0 outside)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    ny, nx = u.shape
    out = np.zeros_like(u)
    st = lib().oracle_adi_halfstep(ny, nx, float(r), _p(u), _p(out), int(implicit_axis))
    if st != 0:
        raise OracleError(f"ADI solve failed (status {st})")
    return out


def adi_halfstep_bands(u, r: float, bands, implicit_axis: int, transpose: bool = False) -> np.ndarray:
    """ADI half-step with the implicit operator S given by its bands (width 3
    or 5): out = S^{-1} (I + r d2) u, or with transpose=True the transposed
    map out = S^{-T} (I + r d2) u (the adjoint half-step); the explicit second
    difference acts along the other axis, Dirichlet 0 outside the grid."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    b = _bands(bands)
    ny, nx = u.shape
    n_row = nx if implicit_axis == 0 else ny
    if b.shape[1] != n_row:
        raise ValueError("bands must have as many rows as the implicit axis")
    out = np.zeros_like(u)
    st = lib().oracle_adi_halfstep_bands(ny, nx, float(r), b.shape[0], _p(b), _p(u), _p(out), int(implicit_axis),
                                         int(bool(transpose)))
    if st != 0:
        raise OracleError(f"ADI solve failed (status {st})")
    return out


def lib_path() -> str:
    return os.path.abspath(_build.lib_path())
