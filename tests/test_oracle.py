"""Pins for the CPU FP64 oracle: it is checked against things that do not
come from itself -- LAPACK dense and banded solves, manufactured solutions,
closed-form eigenpairs of Toeplitz bands, the factorisation identities
A = L U and A = L R of Sec. 3.1 / Sec. 4.1, the adjoint dot-product identity,
central finite differences of the loss, and a dense periodic matrix.

Every ``pin_*`` function is also run against deliberately broken builds of
the oracle source in ``test_oracle_mutations.py``.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from tests.dense import (dense_from_bands, from_layout, periodic_from_bands, periodic_tri, rel_l2,
                         second_difference, to_layout)

LAYOUTS = ("interleaved", "strided")


def _case(width, N, M, seed):
    rng = np.random.default_rng(seed)
    bands = synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)
    B = rng.uniform(-1.0, 1.0, (N, M))
    return bands, B


# ---------------------------------------------------------------- pins


def pin_dense_lu(width, N, layout, M=3, seed=1):
    """Oracle solve == LAPACK dense LU (numpy.linalg.solve)."""
    bands, B = _case(width, N, M, seed)
    X = from_layout(oracle.solve(bands, to_layout(B, layout), layout), layout)
    ref = np.linalg.solve(dense_from_bands(bands), B)
    assert rel_l2(X, ref) < 1e-14, rel_l2(X, ref)


def pin_solve_banded(width, N, seed=2):
    """Oracle solve == LAPACK gbsv through scipy.linalg.solve_banded."""
    bands, B = _case(width, N, 4, seed)
    h = width // 2
    ab = np.zeros((width, N))  # scipy's upper-form band storage
    A = dense_from_bands(bands)
    for r in range(width):
        off = h - r
        for j in range(N):
            i = j - off
            if 0 <= i < N:
                ab[r, j] = A[i, j]
    ref = scipy.linalg.solve_banded((h, h), ab, B)
    X = oracle.solve(bands, B)
    assert rel_l2(X, ref) < 1e-14


def pin_manufactured(width, N, M=5, seed=3):
    """Pick X, form B = A X densely, solve: recover X to ~kappa N u."""
    rng = np.random.default_rng(seed)
    bands, _ = _case(width, N, 1, seed)
    Xt = rng.uniform(-1.0, 1.0, (N, M))
    B = dense_from_bands(bands) @ Xt
    X = oracle.solve(bands, B)
    assert rel_l2(X, Xt) < 1e-13


def pin_toeplitz_tri(N, a, b, c):
    """Tridiagonal Toeplitz (a, b, c), ac > 0: eigenpairs
    lambda_k = b + 2 sgn(a) sqrt(ac) cos(k pi/(N+1)),
    v_k(i) = (a/c)^{i/2} sin(i k pi/(N+1)); the solve of A x = v_k is v_k/lambda_k."""
    bands = synth.toeplitz_bands(N, (a, b, c))
    i = np.arange(1, N + 1)
    ks = np.arange(1, N + 1)
    th = ks * math.pi / (N + 1)
    V = (a / c) ** (i[:, None] / 2.0) * np.sin(np.outer(i, th))
    lam = b + 2.0 * np.sign(a) * math.sqrt(a * c) * np.cos(th)
    X = oracle.solve(bands, V)
    assert rel_l2(X, V / lam[None, :]) < 1e-12


def pin_toeplitz_penta(N, s):
    """A = I + s D2^2 (interior [s, -4s, 1+6s, -4s, s], corner diagonals 1+5s):
    sine eigenvectors with lambda_k = 1 + s (2 - 2 cos(k pi/(N+1)))^2."""
    bands = synth.toeplitz_bands(N, (s, -4 * s, 1 + 6 * s, -4 * s, s))
    bands[2, 0] = bands[2, N - 1] = 1 + 5 * s
    i = np.arange(1, N + 1)
    th = np.arange(1, N + 1) * math.pi / (N + 1)
    V = np.sin(np.outer(i, th))
    lam = 1.0 + s * (2.0 - 2.0 * np.cos(th)) ** 2
    X = oracle.solve(bands, V)
    assert rel_l2(X, V / lam[None, :]) < 1e-12


def pin_tri_factor_identity(N, seed=4):
    """Rebuild A = L U from the Thomas factors: L = diag(pivots) + sub(a),
    U = I + super(chat)."""
    bands, _ = _case(3, N, 1, seed)
    chat, piv = oracle.tri_factor(bands)
    L = np.diag(piv) + np.diag(bands[0, 1:], -1)
    U = np.eye(N) + np.diag(chat[:-1], 1)
    A = dense_from_bands(bands)
    assert np.max(np.abs(L @ U - A)) < 1e-14 * np.max(np.abs(A)) * 8


def pin_penta_factor_identity(N, seed=5):
    """Rebuild A = L R from (alpha, beta, gamma, delta, eps) (Sec. 4.1)."""
    bands, _ = _case(5, N, 1, seed)
    al, be, ga, de, ep = oracle.penta_factor(bands)
    L = np.diag(al) + np.diag(be[1:], -1) + np.diag(ep[2:], -2)
    R = np.eye(N) + np.diag(ga[:-1], 1) + np.diag(de[:-2], 2)
    A = dense_from_bands(bands)
    assert np.max(np.abs(L @ R - A)) < 1e-14 * np.max(np.abs(A)) * 8
    # values the factorisation leaves undefined are zero
    assert be[0] == 0 and ga[N - 1] == 0 and de[N - 2] == 0 and de[N - 1] == 0


def pin_adjoint(width, N, layout, M=4, seed=6):
    """A^{-T} G == dense solve with A^T, and <A^{-T} g, b> == <g, A^{-1} b>."""
    bands, G = _case(width, N, M, seed)
    rng = np.random.default_rng(seed + 100)
    Bm = rng.uniform(-1, 1, (N, M))
    Y = from_layout(oracle.solve_adjoint(bands, to_layout(G, layout), layout), layout)
    A = dense_from_bands(bands)
    assert rel_l2(Y, np.linalg.solve(A.T, G)) < 1e-14
    X = oracle.solve(bands, Bm)
    lhs = np.sum(Y * Bm, axis=0)
    rhs = np.sum(G * X, axis=0)
    assert np.allclose(lhs, rhs, rtol=1e-13, atol=1e-13)


def pin_band_grad_fd(width, N=7, M=3, seed=7):
    """Band gradient of L(A) = sum(G * A^{-1} B) against central differences
    of L itself, entry by entry, and against -(A^{-T}G) X^T densely."""
    bands, B = _case(width, N, M, seed)
    rng = np.random.default_rng(seed + 1)
    G = rng.uniform(-1, 1, (N, M))
    X = oracle.solve(bands, B)
    GB = oracle.solve_adjoint(bands, G)
    dbands = oracle.band_grad(width, GB, X)
    A = dense_from_bands(bands)
    Xd = np.linalg.solve(A, B)
    dA = -np.linalg.solve(A.T, G) @ Xd.T
    h = width // 2
    for k in range(width):
        for i in range(N):
            col = i + k - h
            if not (0 <= col < N):
                assert dbands[k, i] == 0.0
                continue
            assert abs(dbands[k, i] - dA[i, col]) < 1e-12 * (1 + abs(dA[i, col]))
            eps = 1e-6
            Ap, Am = A.copy(), A.copy()
            Ap[i, col] += eps
            Am[i, col] -= eps
            fd = (np.sum(G * np.linalg.solve(Ap, B)) - np.sum(G * np.linalg.solve(Am, B))) / (2 * eps)
            assert abs(dbands[k, i] - fd) < 1e-7 * (1 + abs(fd)), (k, i, dbands[k, i], fd)


def pin_residual(width, N, layout, seed=8):
    """R = B - A X and Y = A X against dense products."""
    bands, B = _case(width, N, 3, seed)
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, B.shape)
    A = dense_from_bands(bands)
    R = from_layout(oracle.residual(bands, to_layout(B, layout), to_layout(X, layout), layout), layout)
    Y = from_layout(oracle.matvec(bands, to_layout(X, layout), layout), layout)
    assert np.max(np.abs(R - (B - A @ X))) < 1e-14
    assert np.max(np.abs(Y - A @ X)) < 1e-14


def pin_periodic(N, a, b, c, seed=9):
    """Sherman-Morrison periodic solve == dense solve of the periodic matrix;
    for a == c the cosine Fourier modes are eigenvectors with
    lambda_k = b + 2a cos(2 pi k / N)."""
    rng = np.random.default_rng(seed)
    B = rng.uniform(-1, 1, (N, 3))
    X = oracle.periodic_tri_solve(a, b, c, B)
    assert rel_l2(X, np.linalg.solve(periodic_tri(N, a, b, c), B)) < 1e-13
    if a == c:
        m = np.arange(N)
        k = 3
        v = np.cos(2 * math.pi * k * m / N)[:, None]
        x = oracle.periodic_tri_solve(a, b, c, v)
        assert rel_l2(x, v / (b + 2 * a * math.cos(2 * math.pi * k / N))) < 1e-13


def pin_periodic_bands(N, seed=13):
    """General periodic bands (a_1 and c_N in the corners) against a dense
    solve of the periodic matrix."""
    rng = np.random.default_rng(seed)
    a, c = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    b = np.abs(a) + np.abs(c) + rng.uniform(1, 2, N)
    A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    A[0, N - 1] = a[0]
    A[N - 1, 0] = c[N - 1]
    B = rng.uniform(-1, 1, (N, 3))
    X = oracle.periodic_tri_solve_bands(np.stack([a, b, c]), B)
    assert rel_l2(X, np.linalg.solve(A, B)) < 1e-13


def pin_periodic_adjoint(N, layout, seed=15):
    """Periodic A^{-T} G against a dense solve with the transposed cyclic
    matrix, and the dot-product identity <A^{-T} g, b> = <g, A^{-1} b>."""
    rng = np.random.default_rng(seed)
    bands = synth.random_periodic_bands(N, rng)
    G = rng.uniform(-1, 1, (N, 4))
    Bm = rng.uniform(-1, 1, (N, 4))
    A = periodic_from_bands(bands)
    Y = from_layout(oracle.periodic_solve_adjoint(bands, to_layout(G, layout), layout), layout)
    assert rel_l2(Y, np.linalg.solve(A.T, G)) < 1e-13
    X = oracle.periodic_tri_solve_bands(bands, Bm)
    assert np.allclose(np.sum(Y * Bm, axis=0), np.sum(G * X, axis=0), rtol=1e-13, atol=1e-13)


def pin_periodic_band_grad(N=5, M=3, seed=16):
    """Band gradient of L = sum(G * A^{-1} B) for a cyclic A, every entry
    (corners included) against -(A^{-T} G) X^T and central differences."""
    rng = np.random.default_rng(seed)
    bands = synth.random_periodic_bands(N, rng)
    B = rng.uniform(-1, 1, (N, M))
    G = rng.uniform(-1, 1, (N, M))
    A = periodic_from_bands(bands)
    X = oracle.periodic_tri_solve_bands(bands, B)
    GB = oracle.periodic_solve_adjoint(bands, G)
    db = oracle.band_grad_periodic(GB, X)
    dA = -np.linalg.solve(A.T, G) @ np.linalg.solve(A, B).T
    eps = 1e-6
    for k in range(3):
        for i in range(N):
            col = (i + k - 1) % N
            assert abs(db[k, i] - dA[i, col]) < 1e-12 * (1 + abs(dA[i, col]))
            Ap, Am = A.copy(), A.copy()
            Ap[i, col] += eps
            Am[i, col] -= eps
            fd = (np.sum(G * np.linalg.solve(Ap, B)) - np.sum(G * np.linalg.solve(Am, B))) / (2 * eps)
            assert abs(db[k, i] - fd) < 1e-7 * (1 + abs(fd)), (k, i)


def pin_cn_tri(N, s, K):
    """K Crank-Nicolson steps of the diffusion benchmark matrix
    A = (-s, 1 + 2s, -s) with zero boundary values: sine modes
    sin(i k pi/(N+1)) are multiplied by g^K, g = (1 - 2s(1 - cos t))/(1 + 2s(1 - cos t)),
    t = k pi/(N+1)."""
    bands = synth.toeplitz_bands(N, (-s, 1 + 2 * s, -s))
    i = np.arange(1, N + 1)
    th = np.array([1, 2, 7, N // 2, N]) * math.pi / (N + 1)
    V = np.sin(np.outer(i, th))
    g = (1 - 2 * s * (1 - np.cos(th))) / (1 + 2 * s * (1 - np.cos(th)))
    assert rel_l2(oracle.cn_steps(bands, V, K), V * g[None, :] ** K) < 1e-12


def pin_cn_penta(N, s, K):
    """K CN steps with A = I + s D2^2 (interior (s, -4s, 1 + 6s, -4s, s) as in
    the hyperdiffusion benchmark, corner diagonals 1 + 5s): sine modes are
    multiplied by g^K, g = (1 - s m^2)/(1 + s m^2), m = 2 - 2 cos t."""
    bands = synth.toeplitz_bands(N, (s, -4 * s, 1 + 6 * s, -4 * s, s))
    bands[2, 0] = bands[2, N - 1] = 1 + 5 * s
    i = np.arange(1, N + 1)
    th = np.array([1, 3, N // 3, N]) * math.pi / (N + 1)
    V = np.sin(np.outer(i, th))
    m2 = (2 - 2 * np.cos(th)) ** 2
    g = (1 - s * m2) / (1 + s * m2)
    assert rel_l2(oracle.cn_steps(bands, V, K), V * g[None, :] ** K) < 1e-12


def pin_cn_periodic(N, s, K, layout="interleaved"):
    """K CN steps of the periodic diffusion benchmark (Sec. 3.2 scheme on a
    periodic domain): Fourier modes cos/sin(2 pi k i / N) are multiplied by
    g^K, g = (1 - 2s(1 - cos t))/(1 + 2s(1 - cos t)), t = 2 pi k / N."""
    bands = synth.periodic_toeplitz_bands(N, (-s, 1 + 2 * s, -s))
    i = np.arange(N)
    ks = np.array([0, 1, 3, N // 2])
    th = 2 * math.pi * ks / N
    V = np.concatenate([np.cos(np.outer(i, th)), np.sin(np.outer(i, th[1:3]))], axis=1)
    g = (1 - 2 * s * (1 - np.cos(th))) / (1 + 2 * s * (1 - np.cos(th)))
    gg = np.concatenate([g, g[1:3]])
    X = from_layout(oracle.cn_steps(bands, to_layout(V, layout), K, periodic=True, layout=layout), layout)
    assert rel_l2(X, V * gg[None, :] ** K) < 1e-12


def pin_adi(ny, nx, r, seed=10):
    """ADI half-steps against the dense Kronecker operators:
    axis 0: (I - r Dxx) out = (I + r Dyy) u; axis 1: (I - r Dyy) out = (I + r Dxx) u."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (ny, nx))
    Dx, Dy = second_difference(nx), second_difference(ny)
    Ix, Iy = np.eye(nx), np.eye(ny)
    # vec(u) row-major: index y*nx + x  ->  kron(Y-op, X-op)
    Kxx = np.kron(Iy, Dx)
    Kyy = np.kron(Dy, Ix)
    I = np.eye(nx * ny)
    ref0 = np.linalg.solve(I - r * Kxx, (I + r * Kyy) @ u.ravel()).reshape(ny, nx)
    ref1 = np.linalg.solve(I - r * Kyy, (I + r * Kxx) @ u.ravel()).reshape(ny, nx)
    assert rel_l2(oracle.adi_halfstep(u, r, 0), ref0) < 1e-14
    assert rel_l2(oracle.adi_halfstep(u, r, 1), ref1) < 1e-14


def pin_adi_bands(ny, nx, r, width, seed=11):
    """ADI half-steps with a non-symmetric implicit operator S and their
    transposes against dense Kronecker operators: S^{-1} E u and S^{-T} E u
    (E = I + r d2 along the other axis), and the adjoint identity
    <v, F(u)> = <F^T(v), u> between the forward and transposed half-steps."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (ny, nx))
    v = rng.uniform(-1, 1, (ny, nx))
    Dx, Dy = second_difference(nx), second_difference(ny)
    Ix, Iy = np.eye(nx), np.eye(ny)
    for axis in (0, 1):
        n = nx if axis == 0 else ny
        bands = synth.random_tri_bands(n, rng) if width == 3 else synth.random_penta_bands(n, rng)
        S = dense_from_bands(bands)
        if axis == 0:
            Sk, Ek = np.kron(Iy, S), np.kron(np.eye(ny) + r * Dy, Ix)
        else:
            Sk, Ek = np.kron(S, Ix), np.kron(Iy, np.eye(nx) + r * Dx)
        fwd = oracle.adi_halfstep_bands(u, r, bands, axis)
        adj = oracle.adi_halfstep_bands(v, r, bands, axis, transpose=True)
        assert rel_l2(fwd.ravel(), np.linalg.solve(Sk, Ek @ u.ravel())) < 1e-13
        assert rel_l2(adj.ravel(), np.linalg.solve(Sk.T, Ek @ v.ravel())) < 1e-13
        assert rel_l2(adj.ravel(), (np.linalg.solve(Sk, Ek)).T @ v.ravel()) < 1e-12
        lhs, rhs = float(np.sum(v * fwd)), float(np.sum(adj * u))
        assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1)


def all_pins():
    """Every pin with a set of arguments, as (name, thunk) pairs."""
    out = []
    for width, Ns in ((3, (2, 3, 5, 17, 64)), (5, (4, 5, 6, 7, 16, 64))):
        for N in Ns:
            for layout in LAYOUTS:
                out.append((f"dense_lu_w{width}_N{N}_{layout}", lambda w=width, n=N, l=layout: pin_dense_lu(w, n, l)))
        out.append((f"solve_banded_w{width}", lambda w=width: pin_solve_banded(w, 33)))
        out.append((f"manufactured_w{width}", lambda w=width: pin_manufactured(w, 129)))
        for layout in LAYOUTS:
            out.append((f"adjoint_w{width}_{layout}", lambda w=width, l=layout: pin_adjoint(w, 23, l)))
            out.append((f"residual_w{width}_{layout}", lambda w=width, l=layout: pin_residual(w, 19, l)))
        out.append((f"band_grad_fd_w{width}", lambda w=width: pin_band_grad_fd(w)))
    out += [
        ("toeplitz_adi", lambda: pin_toeplitz_tri(50, -0.5, 2.0, -0.5)),
        ("toeplitz_spline", lambda: pin_toeplitz_tri(64, 1 / 6, 4 / 6, 1 / 6)),
        ("toeplitz_cn_diffusion", lambda: pin_toeplitz_tri(40, -3.2, 7.4, -3.2)),
        ("toeplitz_nonsym_pos", lambda: pin_toeplitz_tri(30, 0.2, 1.5, 0.5)),
        ("toeplitz_nonsym_neg", lambda: pin_toeplitz_tri(30, -0.3, 1.9, -0.7)),
        ("toeplitz_penta", lambda: pin_toeplitz_penta(48, 0.1)),
        ("toeplitz_penta_stiff", lambda: pin_toeplitz_penta(33, 2.5)),
        ("tri_factor_identity", lambda: pin_tri_factor_identity(40)),
        ("penta_factor_identity", lambda: pin_penta_factor_identity(40)),
        ("penta_factor_identity_min", lambda: pin_penta_factor_identity(4)),
        ("periodic_sym", lambda: pin_periodic(32, -0.4, 1.8, -0.4)),
        ("periodic_nonsym", lambda: pin_periodic(17, 0.3, 2.0, -0.6)),
        ("periodic_bands", lambda: pin_periodic_bands(23)),
        ("periodic_bands_min", lambda: pin_periodic_bands(3, 14)),
        ("periodic_adjoint_il", lambda: pin_periodic_adjoint(19, "interleaved")),
        ("periodic_adjoint_st", lambda: pin_periodic_adjoint(3, "strided", 17)),
        ("periodic_band_grad", lambda: pin_periodic_band_grad()),
        ("periodic_band_grad_min", lambda: pin_periodic_band_grad(3, 2, 18)),
        ("adi_rect", lambda: pin_adi(5, 7, 0.5)),
        ("adi_bands_tri", lambda: pin_adi_bands(6, 9, 0.5, 3)),
        ("adi_bands_penta", lambda: pin_adi_bands(7, 8, 0.3, 5)),
        ("cn_tri", lambda: pin_cn_tri(40, 0.7, 5)),
        ("cn_penta", lambda: pin_cn_penta(30, 0.3, 4)),
        ("cn_periodic", lambda: pin_cn_periodic(24, 0.9, 6)),
        ("cn_periodic_strided", lambda: pin_cn_periodic(9, 0.4, 3, "strided")),
    ]
    return out


@pytest.mark.parametrize("name,thunk", all_pins(), ids=[n for n, _ in all_pins()])
def test_pin(name, thunk):
    thunk()


# ---------------------------------------------------------------- edge cases


def test_singular_pivot_detected():
    bands = synth.toeplitz_bands(6, (1.0, 0.0, 1.0))  # b_1 = 0
    with pytest.raises(oracle.OracleError):
        oracle.solve(bands, np.ones((6, 2)))
    pb = synth.toeplitz_bands(6, (0.1, 0.2, 0.0, 0.2, 0.1))  # alpha_1 = c_1 = 0
    with pytest.raises(oracle.OracleError):
        oracle.solve(pb, np.ones((6, 2)))


def test_single_system_and_min_sizes():
    for width, N in ((3, 2), (5, 4)):
        bands, B = _case(width, N, 1, 11)
        X = oracle.solve(bands, B)
        assert rel_l2(X, np.linalg.solve(dense_from_bands(bands), B)) < 1e-15


def test_penta_too_small_rejected():
    bands, B = _case(5, 4, 1, 12)
    with pytest.raises(oracle.OracleError):
        oracle.solve(bands[:, :3], B[:3])


def test_clamped_hyperdiffusion_matrix():
    """The clamped I + 0.1 D4 matrix: identity first/last two rows,
    interior [0.1, -0.4, 1.6, -0.4, 0.1]; solvable without pivoting."""
    A = dense_from_bands(synth.clamped_hyperdiffusion_bands(16, 0.1))
    assert np.allclose(A[:2, :], np.eye(16)[:2, :]) and np.allclose(A[-2:, :], np.eye(16)[-2:, :])
    assert np.allclose(A[5, 3:8], [0.1, -0.4, 1.6, -0.4, 0.1])
    pin_penta_clamped = np.random.default_rng(0).uniform(-1, 1, (16, 3))
    X = oracle.solve(synth.clamped_hyperdiffusion_bands(16, 0.1), pin_penta_clamped)
    assert rel_l2(X, np.linalg.solve(A, pin_penta_clamped)) < 1e-14
