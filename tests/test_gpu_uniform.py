"""GPU parity of uniform pentadiagonal matrices (Sec. 4.1,
cuPentUniformBatch: the outermost sub-diagonal a_i = eps for every in-range
row) against the CPU FP64 oracle, through the C ABI.  With BS_OPT_UNIFORM = 2
the FP32-arithmetic sweeps read eps as one scalar; FP64 solves keep the
general sweeps (bitwise equal with the option on and off).  Tolerances as
for the general sweeps, on the batch's relative L2 error and every system's
relative max-norm error (tests.dense.parity): FP64 1e-12, FP32 and
BF16-stored the FP32 bound of the matrix (tests.dense.tol32); the scalar and
general FP32 sweeps differ in operation order only (agree to 1e-6).  A matrix with
one differing a_i takes the general sweeps in every precision."""
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
    m.set_option(m.OPT_UNIFORM, 0)
    m.set_option(m.OPT_PARTITION, 0)
    m.set_option(m.OPT_TWISTED, 0)


def _bands(kind, N, rng):
    if kind == "hyper":
        s = 0.4
        return synth.toeplitz_bands(N, (s, -4 * s, 1 + 6 * s, -4 * s, s))
    return synth.uniform_penta_bands(N, rng)


def _solve(bs, f, Bh, dtype, layout, uniform_opt):
    """The one-thread sweeps (no partition, no two-ended sweep), with the
    scalar-eps form requested (2) or not (1)."""
    bs.set_option(bs.OPT_UNIFORM, uniform_opt)
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 1)
    try:
        B = torch.tensor(Bh, dtype=dtype, device="cuda")
        bs.solve(f, B, layout)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_UNIFORM, 0)
        bs.set_option(bs.OPT_PARTITION, 0)
        bs.set_option(bs.OPT_TWISTED, 0)
    return B.double().cpu().numpy()


SHAPES = [(4, 1), (5, 6), (7, 33), (37, 130), (512, 4096), (1000, 515)]


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("kind", ["hyper", "random"])
@pytest.mark.parametrize("N,M", SHAPES)
def test_uniform_fp64(bs, N, M, kind, layout):
    rng = np.random.default_rng(7 * N + M)
    bands = _bands(kind, N, rng)
    B = rng.uniform(-1, 1, (N, M))
    Bh = B if layout == "interleaved" else np.ascontiguousarray(B.T)
    f = bs.Factor(bands)
    Xu = _solve(bs, f, Bh, torch.float64, layout, 2)
    Xg = _solve(bs, f, Bh, torch.float64, layout, 1)
    parity(Xu, oracle.solve(bands, Bh, layout), TOL64, layout)
    assert np.array_equal(Xu, Xg)  # FP64: the general sweeps either way


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("N,M", [(5, 7), (130, 1031), (130, 1030), (512, 4096)])
def test_uniform_fp32(bs, N, M, layout):
    rng = np.random.default_rng(11 * N + M)
    bands = _bands("random", N, rng)
    B = rng.uniform(-1, 1, (N, M)).astype(np.float32).astype(np.float64)
    Bh = B if layout == "interleaved" else np.ascontiguousarray(B.T)
    f = bs.Factor(bands)
    X = _solve(bs, f, Bh, torch.float32, layout, 2)
    Xg = _solve(bs, f, Bh, torch.float32, layout, 1)
    parity(X, oracle.solve(bands, Bh, layout), tol32(bands), layout)
    assert rel_l2(X, Xg) < 1e-6
    if N * M >= 4096:
        assert not np.array_equal(X, Xg)  # the scalar form really ran


def test_uniform_bf16(bs):
    N, M = 512, 4096
    rng = np.random.default_rng(5)
    bands = _bands("hyper", N, rng)
    f = bs.Factor(bands)
    B = torch.tensor(rng.uniform(-1, 1, (N, M)), dtype=torch.bfloat16, device="cuda")
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 1)
    bs.set_option(bs.OPT_UNIFORM, 2)
    try:
        X = bs.solve_bf16(f, B)
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
        bs.set_option(bs.OPT_TWISTED, 0)
        bs.set_option(bs.OPT_UNIFORM, 0)
    ref = oracle.solve(bands, B.double().cpu().numpy())
    parity(X.double().cpu().numpy(), ref, tol32(bands))


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_uniform_adjoint_and_band_grad(bs, layout, dtype):
    N, M = 300, 2050
    rng = np.random.default_rng(9)
    bands = _bands("random", N, rng)
    B = rng.uniform(-1, 1, (N, M))
    Gm = rng.uniform(-1, 1, (N, M))
    if dtype == torch.float32:
        B = B.astype(np.float32).astype(np.float64)
        Gm = Gm.astype(np.float32).astype(np.float64)
    tr = (lambda A: A) if layout == "interleaved" else (lambda A: np.ascontiguousarray(A.T))
    f = bs.Factor(bands)
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 1)
    bs.set_option(bs.OPT_UNIFORM, 2)
    try:
        X = torch.tensor(tr(B), dtype=dtype, device="cuda")
        bs.solve(f, X, layout)
        G = torch.tensor(tr(Gm), dtype=dtype, device="cuda")
        G, db = bs.solve_adjoint(f, G, layout, X=X)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
        bs.set_option(bs.OPT_TWISTED, 0)
        bs.set_option(bs.OPT_UNIFORM, 0)
    GB_ref = oracle.solve_adjoint(bands, tr(Gm), layout)
    parity(G.double().cpu().numpy(), GB_ref, TOL64 if dtype == torch.float64 else tol32(bands), layout)
    db_ref = oracle.band_grad(5, G.double().cpu().numpy(), X.double().cpu().numpy(), layout)
    err = np.max(np.abs(db.cpu().numpy() - db_ref)) / np.max(np.abs(db_ref))
    assert err < (1e-13 if dtype == torch.float64 else 1e-6)


def test_non_uniform_takes_general_sweeps(bs):
    """One differing a_i: the handle is not uniform, so requesting the scalar
    form changes nothing."""
    N, M = 256, 1024
    rng = np.random.default_rng(3)
    bands = synth.uniform_penta_bands(N, rng)
    bands[0, 100] += 0.125
    bands[2, 100] += 0.125
    Bh = rng.uniform(-1, 1, (N, M))
    f = bs.Factor(bands)
    X0 = _solve(bs, f, Bh, torch.float32, "interleaved", 2)
    X1 = _solve(bs, f, Bh, torch.float32, "interleaved", 1)
    assert np.array_equal(X0, X1)
    # FP32 rounding of the input (kappa u) and the FP32 sweeps
    parity(X0, oracle.solve(bands, Bh), tol32(bands, ops=2))


def test_uniform_partitioned_small_batch(bs):
    """A small batch of a uniform matrix runs row-partitioned (the block plans
    use the general sweeps) and still matches the oracle."""
    N, M = 2000, 77
    rng = np.random.default_rng(13)
    bands = _bands("random", N, rng)
    Bh = rng.uniform(-1, 1, (N, M))
    f = bs.Factor(bands)
    bs.set_option(bs.OPT_PARTITION, 2)
    try:
        B = torch.tensor(Bh, device="cuda")
        bs.solve(f, B)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
    parity(B.cpu().numpy(), oracle.solve(bands, Bh), TOL64)
