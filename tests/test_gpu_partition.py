"""GPU parity of the row-partitioned solves, tridiagonal and pentadiagonal
(blocks of rows per thread, a banded reduced system for the block-edge
values, a correction near the edges) against the CPU FP64 oracle, through the
C ABI.  The partition is
forced with OPT_PARTITION = 2 (it is otherwise used automatically for small
batches).  Every check bounds the batch's relative L2 error and every
system's relative max-norm error (tests.dense.parity): FP64 1e-12; FP32 and
BF16-stored twice the FP32 bound of one solve (tests.dense.tol32: the block
solves, then the reduced system and the edge correction).  The partitioned
and unpartitioned FP64 results must also agree to 1e-13."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, rel_l2, tol32

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _tol(dtype, bands):
    return TOL64 if dtype == torch.float64 else tol32(bands, ops=2)


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    yield m
    m.set_option(m.OPT_PARTITION, 0)


def _run(bs, f, Bh, dtype, layout, mode):
    bs.set_option(bs.OPT_PARTITION, mode)
    try:
        B = torch.tensor(Bh, dtype=dtype, device="cuda")
        bs.solve(f, B, layout)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
    return B.double().cpu().numpy()


SHAPES = [(3, 400, 3), (3, 768, 1), (3, 768, 7), (3, 1000, 64), (3, 4096, 130), (3, 5000, 33), (3, 4096, 2048),
          (5, 384, 5), (5, 512, 64), (5, 777, 33), (5, 4096, 300)]


def _bands(width, N, rng):
    return synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width,N,M", SHAPES)
def test_partitioned_fp64(bs, width, N, M, layout):
    rng = np.random.default_rng(N + 3 * M)
    bands = _bands(width, N, rng)
    B = rng.uniform(-1, 1, (N, M))
    Bh = B if layout == "interleaved" else np.ascontiguousarray(B.T)
    f = bs.Factor(bands)
    Xp = _run(bs, f, Bh, torch.float64, layout, 2)
    Xu = _run(bs, f, Bh, torch.float64, layout, 1)
    ref = oracle.solve(bands, Bh, layout)
    parity(Xp, ref, TOL64, layout)
    assert rel_l2(Xp, Xu) < 1e-13


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width,N,M", [(3, 768, 5), (3, 4096, 130), (3, 5000, 1024), (5, 512, 4096), (5, 2000, 77)])
def test_partitioned_fp32(bs, width, N, M, layout):
    rng = np.random.default_rng(N + 5 * M)
    bands = _bands(width, N, rng)
    B = rng.uniform(-1, 1, (N, M)).astype(np.float32).astype(np.float64)
    Bh = B if layout == "interleaved" else np.ascontiguousarray(B.T)
    f = bs.Factor(bands)
    X = _run(bs, f, Bh, torch.float32, layout, 2)
    parity(X, oracle.solve(bands, Bh, layout), _tol(torch.float32, bands), layout)


def test_partitioned_bf16(bs):
    N, M = 4096, 260
    rng = np.random.default_rng(21)
    bands = synth.random_tri_bands(N, rng)
    f = bs.Factor(bands)
    B = torch.tensor(rng.uniform(-1, 1, (N, M)), dtype=torch.bfloat16, device="cuda")
    bs.set_option(bs.OPT_PARTITION, 2)
    try:
        X = bs.solve_bf16(f, B)
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
    ref = oracle.solve(bands, B.double().cpu().numpy())
    parity(X.double().cpu().numpy(), ref, _tol(torch.float32, bands))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width", [3, 5])
def test_partitioned_adjoint_and_band_grad(bs, width, layout, dtype):
    """Non-symmetric bands, so A^T's partition differs from A's."""
    N, M = 2000, 300
    rng = np.random.default_rng(31)
    bands = _bands(width, N, rng)
    B = rng.uniform(-1, 1, (N, M))
    Gm = rng.uniform(-1, 1, (N, M))
    if dtype == torch.float32:
        B = B.astype(np.float32).astype(np.float64)
        Gm = Gm.astype(np.float32).astype(np.float64)
    tr = (lambda A: A) if layout == "interleaved" else (lambda A: np.ascontiguousarray(A.T))
    f = bs.Factor(bands)
    bs.set_option(bs.OPT_PARTITION, 2)
    try:
        X = torch.tensor(tr(B), dtype=dtype, device="cuda")
        bs.solve(f, X, layout)
        G = torch.tensor(tr(Gm), dtype=dtype, device="cuda")
        G, db = bs.solve_adjoint(f, G, layout, X=X)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
    tol = _tol(dtype, bands)
    parity(X.double().cpu().numpy(), oracle.solve(bands, tr(B), layout), tol, layout)
    GB_ref = oracle.solve_adjoint(bands, tr(Gm), layout)
    parity(G.double().cpu().numpy(), GB_ref, tol, layout)
    db_ref = oracle.band_grad(width, G.double().cpu().numpy(), X.double().cpu().numpy(), layout)
    err = np.max(np.abs(db.cpu().numpy() - db_ref)) / np.max(np.abs(db_ref))
    assert err < (1e-13 if dtype == torch.float64 else 1e-6)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_partitioned_adi(bs, axis, adjoint, dtype):
    """ADI half-steps on a 1024 x 1024 grid (the implicit axis splits into 4
    blocks of 256 rows), forward and adjoint, against the oracle's half-step
    and its transpose (oracle.adi_halfstep_bands), and partitioned against
    unpartitioned."""
    n, r = 1024, 0.5
    u = synth.adi_field(n, 5, "cpu", torch.float64).numpy()
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
    f = bs.Factor(synth.adi_bands(n, r))
    ut = torch.tensor(u, dtype=dtype, device="cuda")
    outs = {}
    for mode in (2, 1):
        bs.set_option(bs.OPT_PARTITION, mode)
        try:
            outs[mode] = bs.adi_halfstep(f, ut, r, axis, adjoint=adjoint).double().cpu().numpy()
        finally:
            bs.set_option(bs.OPT_PARTITION, 0)
    bands = synth.adi_bands(n, r)
    ref = oracle.adi_halfstep_bands(u, r, bands, axis, transpose=adjoint)
    # the explicit operator, then the partitioned solve
    tol = TOL64 if dtype == torch.float64 else tol32(bands, ops=3)
    parity(outs[2], ref, tol, "strided" if axis == 0 else "interleaved")
    assert rel_l2(outs[2], outs[1]) < (1e-13 if dtype == torch.float64 else tol)


def test_no_partition_without_decay(bs):
    """A tridiagonal matrix whose spikes do not decay within a block gets no
    partition; forcing the option then falls back to the plain solve."""
    N, M = 4096, 64
    bands = synth.toeplitz_bands(N, (-1.0, 2.0001, -1.0))
    rng = np.random.default_rng(41)
    Bh = rng.uniform(-1, 1, (N, M))
    f = bs.Factor(bands)
    X = _run(bs, f, Bh, torch.float64, "interleaved", 2)
    Xu = _run(bs, f, Bh, torch.float64, "interleaved", 1)
    assert np.array_equal(X, Xu)
    assert rel_l2(X, oracle.solve(bands, Bh)) < 1e-9  # condition number ~1e7


def test_partitioned_clamped_hyperdiffusion_fp32(bs):
    """The clamped I + 0.1 D4 matrix at N = 512 splits into two blocks; the
    partitioned FP32 solve of 65536 systems against the oracle (sampled) and
    the unpartitioned one."""
    N, M = 512, 65536
    bands = synth.clamped_hyperdiffusion_bands(N, 0.1)
    f = bs.Factor(bands)
    B = synth.normal_rhs(N, M, 3, "cuda").float().cpu().numpy()
    cols = np.random.default_rng(2).choice(M, 128, replace=False)
    X = _run(bs, f, B, torch.float32, "interleaved", 2)
    Xu = _run(bs, f, B, torch.float32, "interleaved", 1)
    ref = oracle.solve(bands, B[:, cols].astype(np.float64))
    parity(X[:, cols], ref, _tol(torch.float32, bands))
    assert rel_l2(X, Xu) < 1e-6


def test_partitioned_penta_adi(bs):
    """An ADI half-step whose implicit operator is pentadiagonal (I + s D2^2
    along the implicit axis) runs partitioned; same result as unpartitioned."""
    n = 1024
    s = 0.3
    bands = synth.toeplitz_bands(n, (s, -4 * s, 1 + 6 * s, -4 * s, s))
    f = bs.Factor(bands)
    u = synth.adi_field(n, 7, "cuda", torch.float64)
    outs = {}
    for mode in (2, 1):
        bs.set_option(bs.OPT_PARTITION, mode)
        try:
            outs[mode] = bs.adi_halfstep(f, u, 0.5, 1).cpu().numpy()
        finally:
            bs.set_option(bs.OPT_PARTITION, 0)
    assert rel_l2(outs[2], outs[1]) < 1e-13
