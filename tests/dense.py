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
    """||x - ref||_2 / ||ref||_2 over the whole array (both scaled by the
    largest |ref| first, so that values near the ends of the FP64 range
    neither overflow nor underflow the norms)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    sc = float(np.max(np.abs(ref))) if ref.size else 0.0
    if not np.isfinite(sc) or sc == 0.0:
        sc = 1.0
    return float(np.linalg.norm((x - ref) / sc) / np.linalg.norm(ref / sc))


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


U32 = 2.0 ** -24  # unit roundoff of FP32
_KAPPA: dict = {}


def _inv_norm_inf_banded(b: np.ndarray, chunk: int = 1024) -> float:
    """||A^{-1}||_inf of a non-cyclic banded matrix from LAPACK banded solves
    of the identity, a block of columns at a time (the row sums of |A^{-1}|
    accumulate across blocks)."""
    from scipy.linalg import solve_banded
    w, N = b.shape
    h = w // 2
    ab = np.zeros((w, N))  # LAPACK band storage: ab[h + i - j, j] = A[i, j]
    for k in range(w):
        off = k - h  # column = row + off
        for i in range(max(0, -off), min(N, N - off)):
            ab[h - off, i + off] = b[k, i]
    rows = np.zeros(N)
    for j0 in range(0, N, chunk):
        E = np.zeros((N, min(chunk, N - j0)))
        E[np.arange(j0, j0 + E.shape[1]), np.arange(E.shape[1])] = 1.0
        rows += np.abs(solve_banded((h, h), ab, E)).sum(axis=1)
    return float(rows.max())


def cond_inf(bands: np.ndarray, periodic: bool = False) -> float:
    """kappa_inf(A) = ||A||_inf ||A^{-1}||_inf of the (cyclic) banded matrix:
    the dense inverse (LAPACK through numpy) up to N = 4096; beyond
    (non-cyclic), Varah's upper bound for a strictly diagonally dominant
    matrix, else banded solves of the identity; cached per matrix."""
    import hashlib
    b = np.ascontiguousarray(bands, dtype=np.float64)
    key = (b.shape, periodic, hashlib.sha1(b.tobytes()).hexdigest())
    if key not in _KAPPA:
        N = b.shape[1]
        if N <= 4096 or periodic:
            A = periodic_from_bands(b) if periodic else dense_from_bands(b)
            _KAPPA[key] = float(np.abs(A).sum(axis=1).max() * np.abs(np.linalg.inv(A)).sum(axis=1).max())
        else:
            h = b.shape[0] // 2
            absA = np.zeros(N)
            for k in range(b.shape[0]):
                off = k - h
                lo, hi = max(0, -off), min(N, N - off)
                absA[lo:hi] += np.abs(b[k, lo:hi])
            diag = np.abs(b[h])
            margin = float(np.min(2.0 * diag - absA))  # |a_ii| - sum_{j != i} |a_ij|
            # strictly row diagonally dominant: Varah's bound
            # ||A^{-1}||_inf <= 1 / min_i (|a_ii| - sum_{j != i} |a_ij|)
            inv = 1.0 / margin if margin > 0 else _inv_norm_inf_banded(b)
            _KAPPA[key] = float(absA.max() * inv)
    return _KAPPA[key]


def tol32(bands: np.ndarray, periodic: bool = False, ops: int = 1) -> float:
    """Tolerance of a solve in FP32 arithmetic against the FP64 oracle on the
    same (FP32- or BF16-representable) input: ops * width * kappa_inf(A) * u,
    u = 2^-24, for the error of every system in the max norm and of the batch
    in L2.  Each row of a banded LU sweep combines `width` terms, so the
    computed solution solves (A + dA) x = b with |dA| <= ~width u |L||U|; for
    the diagonally dominant matrices of these tests |L||U| stays within a
    small factor of |A|, and the relative forward error is at most kappa_inf
    times the relative backward error.  ops counts chained solves and
    explicit operators (time steps) whose errors add."""
    return ops * bands.shape[0] * cond_inf(bands, periodic) * U32


def sys_max_err(x, ref, layout: str = "interleaved") -> float:
    """Largest relative error of one system in the max norm,
    max_j ||x_j - ref_j||_inf / ||ref_j||_inf over the systems j (columns of
    an interleaved (N, M) block, rows of a strided (M, N) one); a system whose
    reference is zero must be exactly zero."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if layout != "interleaved":
        x, ref = x.T, ref.T
    num = np.max(np.abs(x - ref), axis=0)
    den = np.max(np.abs(ref), axis=0)
    zero = den == 0
    if np.any(num[zero] != 0):
        return float("inf")
    return float(np.max(num[~zero] / den[~zero])) if np.any(~zero) else 0.0


def parity(x, ref, tol: float, layout: str = "interleaved") -> None:
    """Asserts that the batch's relative L2 error and every system's relative
    max-norm error are below tol."""
    e_batch = rel_l2(x, ref)
    e_sys = sys_max_err(x, ref, layout)
    assert e_batch < tol and e_sys < tol, f"batch {e_batch:.3e}, worst system {e_sys:.3e}, tolerance {tol:.3e}"
