"""GPU tests of the windowed sweeps (BS_OPT_WINDOW, csrc/sweep_win.cu): the
forward values stay on chip and each block's backward sweep starts from zero
at the block's end, writing only the rows whose distance from that start is
past the handle's window (2^-50 for pair arithmetic on FP64 data, 2^-28 for
FP32).

Checks against the FP64 oracle, on the batch's relative L2 error and every
system's relative max-norm error (tests.dense.parity):
- FP64 data (pairs): 1e-12, the FP64 target;
- FP32 and BF16 storage: against the oracle's solve of the stored (rounded)
  input, the per-matrix bound of the FP32 sweeps plus the window (fp32_tol);
- windowed against two-sweep results: FP64 within 1e-13 per system (the
  2^-50 window plus the pairs' rounding, which the windowed sweep's second
  pass over a block's last rows changes), FP32 within 2^-20;
- block edges: N from 2 to a few blocks around the window and block sizes,
  N = 1024 with M = 2^16 + 2 (ragged groups), both layouts' fallbacks;
- a matrix whose backward responses do not decay within reach has no window
  and takes the two-sweep kernels.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, sys_max_err, tol32

pytestmark = pytest.mark.gpu



def fp32_tol(bands):
    """The FP32 bound of the matrix (tests.dense.tol32) plus the window's
    2^-28 (relative to the system's largest value)."""
    return tol32(bands) + 2.0 ** -28


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    return m


@pytest.fixture
def one_thread(bs):
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 1)
    yield
    bs.set_option(bs.OPT_PARTITION, 0)
    bs.set_option(bs.OPT_TWISTED, 0)
    bs.set_option(bs.OPT_WINDOW, 0)


def _bands(kind, N, seed):
    rng = np.random.default_rng(seed)
    if kind == "tri":
        return synth.random_tri_bands(N, rng)
    if kind == "penta":
        return synth.random_penta_bands(N, rng)
    if kind == "spline":
        return synth.spline_bands(N)
    if kind == "hyper":
        return synth.clamped_hyperdiffusion_bands(N, 0.1)
    if kind == "adi":
        return synth.adi_bands(N, 0.5)
    raise ValueError(kind)


def _run(bs, f, Bh, dtype, adjoint=False, window=0):
    bs.set_option(bs.OPT_WINDOW, window)
    B = torch.tensor(Bh, dtype=dtype, device="cuda")
    if adjoint:
        bs.solve_adjoint(f, B)
    else:
        bs.solve(f, B)
    torch.cuda.synchronize()
    return B.double().cpu().numpy()


NS = [2, 3, 5, 8, 27, 28, 29, 31, 33, 47, 57, 60, 61, 100, 257, 513]


@pytest.mark.parametrize("kind", ["tri", "penta", "spline", "hyper"])
@pytest.mark.parametrize("N", NS)
def test_fp64_window_block_edges(bs, one_thread, kind, N):
    if kind == "penta" and N < 4 or kind == "hyper" and N < 8:
        pytest.skip("pentadiagonal needs N >= 4 (clamped rows: N >= 8)")
    bands = _bands(kind, N, N)
    rng = np.random.default_rng(N + 1)
    M = 515
    Bh = rng.standard_normal((N, M))
    f = bs.Factor(bands)
    for adjoint, ref in ((False, oracle.solve(bands, Bh)), (True, oracle.solve_adjoint(bands, Bh))):
        Xw = _run(bs, f, Bh, torch.float64, adjoint, 2)
        Xs = _run(bs, f, Bh, torch.float64, adjoint, 1)
        parity(Xw, ref, 1e-12)
        assert sys_max_err(Xw, Xs) < 1e-13


@pytest.mark.parametrize("kind", ["tri", "penta", "spline", "hyper"])
@pytest.mark.parametrize("N", NS)
def test_fp32_window_block_edges(bs, one_thread, kind, N):
    if kind == "penta" and N < 4 or kind == "hyper" and N < 8:
        pytest.skip("pentadiagonal needs N >= 4 (clamped rows: N >= 8)")
    bands = _bands(kind, N, N + 5)
    rng = np.random.default_rng(N + 2)
    for M in (513, 20000):
        Bh = rng.standard_normal((N, M)).astype(np.float32).astype(np.float64)
        f = bs.Factor(bands)
        for adjoint, ref in ((False, oracle.solve(bands, Bh)), (True, oracle.solve_adjoint(bands, Bh))):
            Xw = _run(bs, f, Bh, torch.float32, adjoint, 0)
            Xs = _run(bs, f, Bh, torch.float32, adjoint, 1)
            parity(Xw, ref, fp32_tol(bands))
            assert sys_max_err(Xw, Xs) < 2.0 ** -20


@pytest.mark.parametrize("kind,N", [("tri", 64), ("penta", 37), ("spline", 1024), ("hyper", 512)])
def test_bf16_window(bs, one_thread, kind, N):
    bands = _bands(kind, N, 3)
    M = 4098
    B = torch.tensor(np.random.default_rng(4).uniform(-1, 1, (N, M)), dtype=torch.bfloat16, device="cuda")
    f = bs.Factor(bands)
    ref = oracle.solve(bands, B.double().cpu().numpy())
    for window in (0, 1):
        bs.set_option(bs.OPT_WINDOW, window)
        X = bs.solve_bf16(f, B)
        torch.cuda.synchronize()
        parity(X.double().cpu().numpy(), ref, fp32_tol(bands))


def test_large_ragged_batch(bs):
    """Default options: N = 1024 spline, M = 2^16 + 2 and M = 2^16 + 1 (odd:
    one system per thread), FP64 data in pairs, sampled per system."""
    N = 1024
    bands = synth.spline_bands(N)
    f = bs.Factor(bands)
    for M in (65538, 65537):
        B = synth.uniform_rhs(N, M, M, "cuda")
        X = B.clone()
        bs.solve(f, X)
        torch.cuda.synchronize()
        cols = np.r_[np.arange(8), M - 1 - np.arange(8), np.random.default_rng(M).choice(M, 240, replace=False)]
        Bs = B[:, cols].cpu().numpy()
        parity(X[:, cols].cpu().numpy(), oracle.solve(bands, Bs), 1e-12)


def test_slow_decay_has_no_window_and_stays_correct(bs, one_thread):
    """(-0.5, 1.05, -0.5): the backward responses decay by ~0.73 per row, so
    2^-50 takes ~110 rows and 2^-28 ~60, past both windows' reach; the solves
    take the two-sweep kernels (condition number ~40)."""
    N, M = 300, 2000
    bands = np.zeros((3, N))
    bands[0, 1:] = -0.5
    bands[1] = 1.05
    bands[2, :-1] = -0.5
    f = bs.Factor(bands)
    Bh = np.random.default_rng(5).uniform(-1, 1, (N, M))
    ref = oracle.solve(bands, Bh)
    X0 = _run(bs, f, Bh, torch.float64, False, 2)
    X1 = _run(bs, f, Bh, torch.float64, False, 1)
    assert np.array_equal(X0, X1)
    parity(X0, ref, 1e-12)
