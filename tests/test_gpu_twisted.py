"""GPU parity of the two-ended tridiagonal and pentadiagonal solves (two
threads per system meeting in the middle; used for small batches) against
the CPU FP64 oracle, through the C ABI.  Tolerances as for the one-thread
sweeps, on the batch's relative L2 error and every system's relative
max-norm error (tests.dense.parity): FP64 1e-12, FP32 the FP32 bound of the
matrix (tests.dense.tol32); the two-ended and one-thread FP64 results agree
to 1e-13 (same arithmetic per row, another elimination order)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, rel_l2, tol32

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    yield m
    m.set_option(m.OPT_TWISTED, 0)
    m.set_option(m.OPT_PARTITION, 0)


def _solve(bs, f, Bh, dtype, twisted, layout="interleaved"):
    bs.set_option(bs.OPT_TWISTED, twisted)
    bs.set_option(bs.OPT_PARTITION, 1)
    try:
        B = torch.tensor(Bh, dtype=dtype, device="cuda")
        bs.solve(f, B, layout)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_TWISTED, 0)
        bs.set_option(bs.OPT_PARTITION, 0)
    return B.double().cpu().numpy()


def _bands(width, N, rng):
    return synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)


@pytest.mark.parametrize("width,N", [(3, 2), (3, 3), (3, 4), (3, 5), (3, 16), (3, 17), (3, 64), (3, 257),
                                     (3, 1000), (5, 4), (5, 5), (5, 6), (5, 7), (5, 16), (5, 33), (5, 64),
                                     (5, 255), (5, 1000)])
@pytest.mark.parametrize("M", [1, 2, 7, 33, 1024])
def test_twisted_fp64(bs, width, N, M):
    rng = np.random.default_rng(N * 7919 + M + width)
    bands = _bands(width, N, rng)
    Bh = rng.uniform(-1, 1, (N, M))
    f = bs.Factor(bands)
    Xt = _solve(bs, f, Bh, torch.float64, 2)
    X1 = _solve(bs, f, Bh, torch.float64, 1)
    ref = oracle.solve(bands, Bh)
    parity(Xt, ref, TOL64)
    assert rel_l2(Xt, X1) < 1e-13


@pytest.mark.parametrize("width,N,M", [(3, 2, 3), (3, 5, 1), (3, 64, 1024), (3, 333, 130), (3, 1024, 4099),
                                       (5, 4, 3), (5, 9, 1), (5, 64, 1024), (5, 333, 130), (5, 1024, 4099)])
def test_twisted_fp32(bs, width, N, M):
    rng = np.random.default_rng(N + 31 * M + width)
    bands = _bands(width, N, rng)
    Bh = rng.uniform(-1, 1, (N, M)).astype(np.float32).astype(np.float64)
    f = bs.Factor(bands)
    X = _solve(bs, f, Bh, torch.float32, 2)
    parity(X, oracle.solve(bands, Bh), tol32(bands))


@pytest.mark.parametrize("name", ["adi", "spline", "toeplitz_weak", "clamped_hyper", "hyper"])
def test_twisted_structured_bands(bs, name):
    """Toeplitz-like matrices (ADI I - 0.5 d2, the [1,4,1]/6 spline, a barely
    dominant (-1, 2.01, -1), the clamped I + 0.1 D4 and I + 0.4 D4) at
    N = 512, 1000 systems."""
    N, M = 512, 1000
    bands = {"adi": synth.adi_bands(N, 0.5), "spline": synth.spline_bands(N),
             "toeplitz_weak": synth.toeplitz_bands(N, (-1.0, 2.01, -1.0)),
             "clamped_hyper": synth.clamped_hyperdiffusion_bands(N, 0.1),
             "hyper": synth.toeplitz_bands(N, (0.4, -1.6, 3.4, -1.6, 0.4))}[name]
    rng = np.random.default_rng(17)
    Bh = rng.uniform(-1, 1, (N, M))
    f = bs.Factor(bands)
    Xt = _solve(bs, f, Bh, torch.float64, 2)
    X1 = _solve(bs, f, Bh, torch.float64, 1)
    ref = oracle.solve(bands, Bh)
    tol = 1e-11 if name == "toeplitz_weak" else TOL64  # condition number ~4e3
    parity(Xt, ref, tol)
    assert rel_l2(Xt, X1) < 1e-12


@pytest.mark.parametrize("width", [3, 5])
def test_default_choice(bs, width):
    """Small batches take the two-ended sweep by default (not bitwise the
    one-thread result, right against the oracle); large ones and the strided
    layout do not."""
    rng = np.random.default_rng(5)
    bands = _bands(width, 64, rng)
    f = bs.Factor(bands)
    Bh = rng.uniform(-1, 1, (64, 1024))
    X0 = _solve(bs, f, Bh, torch.float64, 0)
    X1 = _solve(bs, f, Bh, torch.float64, 1)
    assert not np.array_equal(X0, X1)
    parity(X0, oracle.solve(bands, Bh), TOL64)
    Bs = np.ascontiguousarray(Bh.T)
    assert np.array_equal(_solve(bs, f, Bs, torch.float64, 0, "strided"),
                          _solve(bs, f, Bs, torch.float64, 1, "strided"))
    Bl = rng.uniform(-1, 1, (64, 65536))
    assert np.array_equal(_solve(bs, f, Bl, torch.float64, 0), _solve(bs, f, Bl, torch.float64, 1))


def test_periodic_handle_not_twisted(bs):
    pb = synth.random_periodic_bands(40, np.random.default_rng(8))
    f = bs.Factor(pb, periodic=True)
    Bh = np.random.default_rng(9).uniform(-1, 1, (40, 64))
    X2 = _solve(bs, f, Bh, torch.float64, 2)
    X1 = _solve(bs, f, Bh, torch.float64, 1)
    assert np.array_equal(X2, X1)
    parity(X2, oracle.periodic_tri_solve_bands(pb, Bh), TOL64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("width,N,M", [(3, 2, 5), (3, 3, 1), (3, 64, 1024), (3, 333, 77), (3, 1000, 130),
                                       (5, 4, 5), (5, 7, 1), (5, 64, 1024), (5, 333, 77), (5, 1000, 130)])
def test_twisted_adjoint_and_band_grad(bs, width, N, M, dtype):
    """A^{-T} G by the two-ended sweep of A^T (non-symmetric bands, so A^T's
    plans differ from A's), then the band gradient."""
    rng = np.random.default_rng(3 * N + M + width)
    bands = _bands(width, N, rng)
    Bh = rng.uniform(-1, 1, (N, M))
    Gh = rng.uniform(-1, 1, (N, M))
    if dtype == torch.float32:
        Bh = Bh.astype(np.float32).astype(np.float64)
        Gh = Gh.astype(np.float32).astype(np.float64)
    f = bs.Factor(bands)
    res = {}
    for tw in (2, 1):
        bs.set_option(bs.OPT_TWISTED, tw)
        bs.set_option(bs.OPT_PARTITION, 1)
        try:
            X = torch.tensor(Bh, dtype=dtype, device="cuda")
            bs.solve(f, X)
            G = torch.tensor(Gh, dtype=dtype, device="cuda")
            G, db = bs.solve_adjoint(f, G, X=X)
            torch.cuda.synchronize()
        finally:
            bs.set_option(bs.OPT_TWISTED, 0)
            bs.set_option(bs.OPT_PARTITION, 0)
        res[tw] = (X.double().cpu().numpy(), G.double().cpu().numpy(), db.cpu().numpy())
    X, GB, db = res[2]
    GB_ref = oracle.solve_adjoint(bands, Gh)
    tol = TOL64 if dtype == torch.float64 else tol32(bands)
    parity(GB, GB_ref, tol)
    parity(X, oracle.solve(bands, Bh), tol)
    db_ref = oracle.band_grad(width, GB, X)
    assert np.max(np.abs(db - db_ref)) / np.max(np.abs(db_ref)) < (1e-13 if dtype == torch.float64 else 1e-6)
    if dtype == torch.float64:
        assert rel_l2(GB, res[1][1]) < 1e-13


@pytest.mark.parametrize("width,N,M", [(3, 64, 1024), (3, 5, 3), (5, 64, 1000), (5, 300, 77)])
def test_twisted_bf16_storage(bs, width, N, M):
    """BF16-stored right-hand sides, FP32 arithmetic and output: two-ended
    against the oracle on the BF16 values and against the one-thread sweep."""
    rng = np.random.default_rng(N + M + width)
    bands = _bands(width, N, rng)
    f = bs.Factor(bands)
    B = torch.tensor(rng.uniform(-1, 1, (N, M)), dtype=torch.bfloat16, device="cuda")
    out = {}
    for tw in (2, 1):
        bs.set_option(bs.OPT_TWISTED, tw)
        bs.set_option(bs.OPT_PARTITION, 1)
        try:
            out[tw] = bs.solve_bf16(f, B).double().cpu().numpy()
        finally:
            bs.set_option(bs.OPT_TWISTED, 0)
            bs.set_option(bs.OPT_PARTITION, 0)
    ref = oracle.solve(bands, B.double().cpu().numpy())
    parity(out[2], ref, tol32(bands))
    parity(out[2], out[1], tol32(bands))
