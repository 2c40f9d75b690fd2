"""The parity checks themselves (tests.dense.parity, tol32), on the CPU: an
error planted in one system of an oracle solution must fail them even where
the batch's relative L2 error stays below the tolerance, and the derived
FP32 bound must sit above what FP32 arithmetic actually gives (an FP32
emulation of the oracle's sweeps is out of scope here; the rounding of the
solution to FP32 is the floor every FP32 path meets)."""
import numpy as np
import pytest

import oracle
import synth
from tests.dense import cond_inf, parity, rel_l2, sys_max_err, tol32


def _penta_case(M=256):
    bands = synth.clamped_hyperdiffusion_bands(512, 0.1)
    B = np.random.default_rng(0).standard_normal((512, M))
    return bands, oracle.solve(bands, B)


def test_planted_fp32_error_in_one_system_fails():
    """A 1e-6 relative error in one system's column (the FP32 bound of the
    penta N = 512 benchmark matrix is ~9e-7) fails the check, while the
    batch L2 error alone would have passed."""
    bands, X = _penta_case()
    tol = tol32(bands)
    assert 5e-7 < tol < 1e-6
    bad = X.copy()
    j = 17
    bad[200, j] += 1e-6 * np.max(np.abs(X[:, j]))
    assert rel_l2(bad, X) < tol  # invisible to the batch norm
    with pytest.raises(AssertionError):
        parity(bad, X, tol)
    parity(X, X, tol)


def test_planted_fp64_error_in_one_system_fails():
    bands, X = _penta_case()
    bad = X.copy()
    bad[3, 100] += 1e-11 * np.max(np.abs(X[:, 100]))
    assert rel_l2(bad, X) < 1e-12
    with pytest.raises(AssertionError):
        parity(bad, X, 1e-12)


def test_planted_error_strided_layout():
    """The strided layout's systems are rows."""
    bands, X = _penta_case(64)
    Xs = np.ascontiguousarray(X.T)
    bad = Xs.copy()
    bad[5, 7] += 1e-5 * np.max(np.abs(Xs[5]))
    with pytest.raises(AssertionError):
        parity(bad, Xs, tol32(bands), "strided")
    assert sys_max_err(bad, Xs, "interleaved") < 1e-5  # as columns the error would be diluted


def test_fp32_bound_above_rounding_floor():
    """Rounding the exact solution to FP32 stays well inside the bound."""
    bands, X = _penta_case()
    X32 = X.astype(np.float32).astype(np.float64)
    assert sys_max_err(X32, X) < tol32(bands) / 5


@pytest.mark.parametrize("N", [64, 300])
def test_cond_inf_against_dense_and_closed_form(N):
    """kappa_inf from the dense inverse against the banded-solve path, and for
    tridiag(-1, 4, -1) against its closed-form bounds (Varah: ||A^{-1}|| <=
    1/2; row sums 6)."""
    from tests import dense
    rng = np.random.default_rng(N)
    b = synth.random_penta_bands(N, rng)
    A = dense.dense_from_bands(b)
    k = np.abs(A).sum(1).max() * dense._inv_norm_inf_banded(b, chunk=32)
    assert abs(cond_inf(b) - k) < 1e-12 * k
    t = synth.toeplitz_bands(N, (-1.0, 4.0, -1.0))
    assert 6.0 * 0.25 < cond_inf(t) <= 6.0 * 0.5 + 1e-12
