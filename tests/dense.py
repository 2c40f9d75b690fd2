"""Dense-matrix helpers for the tests: build full matrices from bands with
numpy only, so that library routines (LAPACK through numpy/scipy) can check
the oracle independently of its own code."""
import numpy as np


def dense_from_bands(bands: np.ndarray) -> np.ndarray:
    """Full N x N matrix with band k of row i at column i + k - width//2."""
    w, N = bands.shape
    h = w // 2
    A = np.zeros((N, N))
    for i in range(N):
        for k in range(w):
            col = i + k - h
            if 0 <= col < N:
                A[i, col] = bands[k, i]
    return A


def second_difference(n: int) -> np.ndarray:
    """tridiag(1, -2, 1), homogeneous Dirichlet."""
    return np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)


def periodic_tri(N: int, a: float, b: float, c: float) -> np.ndarray:
    """Periodic tridiagonal matrix with a in the top-right and c in the
    bottom-left corner (the constant periodic matrix of Sec. 3.3)."""
    A = np.diag(b * np.ones(N)) + np.diag(a * np.ones(N - 1), -1) + np.diag(c * np.ones(N - 1), 1)
    A[0, N - 1] = a
    A[N - 1, 0] = c
    return A


def periodic_from_bands(bands: np.ndarray) -> np.ndarray:
    """Full cyclic tridiagonal matrix: band k of row i at column
    (i + k - 1) mod N (N >= 3)."""
    _, N = bands.shape
    A = np.zeros((N, N))
    for i in range(N):
        for k in range(3):
            A[i, (i + k - 1) % N] = bands[k, i]
    return A


def to_layout(X_nm: np.ndarray, layout: str) -> np.ndarray:
    """(N, M) interleaved block to the requested storage."""
    return np.ascontiguousarray(X_nm if layout == "interleaved" else X_nm.T)


def from_layout(X: np.ndarray, layout: str) -> np.ndarray:
    return X if layout == "interleaved" else X.T


def rel_l2(x, ref) -> float:
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def sys_rel_err(x, ref, layout: str = "interleaved") -> float:
    """Largest relative L2 error of one system, max_j |x_j - ref_j| / |ref_j|
    over the systems j (columns of an interleaved (N, M) block, rows of a
    strided (M, N) one); a system whose reference is zero must be exactly
    zero."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if layout != "interleaved":
        x, ref = x.T, ref.T
    # scaled by each system's largest entry, so that norms of systems near
    # the ends of the FP64 range neither overflow nor underflow
    sc = np.max(np.abs(ref), axis=0)
    sc = np.where(sc > 0, sc, 1.0)
    num = np.linalg.norm((x - ref) / sc, axis=0)
    den = np.linalg.norm(ref / sc, axis=0)
    zero = den == 0
    if np.any(num[zero] != 0):
        return float("inf")
    return float(np.max(num[~zero] / den[~zero])) if np.any(~zero) else 0.0
