"""GPU parity of the mixed-precision solve (FP32 storage, FP32 sweeps, one
refinement step with an FP64-accurate residual, FP64 result) against the
oracle's FP64 solve of the same FP32-rounded B.

Tolerances, on the batch's relative L2 error and every system's relative
max-norm error (tests.dense.parity): 1e-12 with one refinement step (the
stated FP64 target); the unrefined FP32 solution (refine_steps=0) within the
FP32 bound of the matrix (tests.dense.tol32)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, rel_l2, tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    return m


def _bands(width, N, seed):
    rng = np.random.default_rng(seed)
    return synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)


@pytest.mark.parametrize("mode", [0, 1], ids=["factor", "system"])
@pytest.mark.parametrize("width,N,M", [(3, 2, 1), (3, 3, 5), (3, 64, 1024), (3, 100, 333), (3, 1024, 257),
                                       (5, 4, 1), (5, 5, 7), (5, 37, 33), (5, 512, 1000), (5, 130, 4099)])
def test_refine_random(bs, width, N, M, mode):
    bands = _bands(width, N, N + M)
    B = torch.tensor(np.random.default_rng(M).uniform(-1, 1, (N, M)), dtype=torch.float32, device="cuda")
    f = bs.Factor(bands)
    X = bs.solve_refine(f, B, refine_steps=1, mode=mode)
    X0 = bs.solve_refine(f, B, refine_steps=0)
    torch.cuda.synchronize()
    ref = oracle.solve(bands, B.double().cpu().numpy())
    parity(X.cpu().numpy(), ref, 1e-12)
    parity(X0.cpu().numpy(), ref, tol32(bands))


@pytest.mark.parametrize("mode", [0, 1], ids=["factor", "system"])
def test_refine_clamped_hyperdiffusion_full_size(bs, mode):
    """Penta I + 0.1 D4 clamped, N=512, M=65536, RHS ~ N(0,1) stored in FP32:
    512 sampled systems against the oracle, every system via the residual."""
    N, M = 512, 65536
    bands = synth.clamped_hyperdiffusion_bands(N, 0.1)
    f = bs.Factor(bands)
    B = synth.normal_rhs(N, M, 0, "cuda").float()
    X = bs.solve_refine(f, B, mode=mode)
    torch.cuda.synchronize()
    cols = np.union1d(np.random.default_rng(4).choice(M, 512, replace=False), [0, M - 1])
    ref = oracle.solve(bands, B[:, cols].double().cpu().numpy())
    assert rel_l2(X[:, cols].cpu().numpy(), ref) < 1e-12
    b = torch.tensor(bands, device="cuda")
    R = B.double()
    for k, off in enumerate(range(-2, 3)):
        lo, hi = max(0, -off), N - max(0, off)
        R[lo:hi] -= b[k, lo:hi, None] * X[lo + off:hi + off]
    assert (torch.linalg.norm(R) / torch.linalg.norm(B.double())).item() < 1e-13


@pytest.mark.parametrize("mode", [0, 1], ids=["factor", "system"])
def test_refine_spline_sampled(bs, mode):
    """Tri [1,4,1]/6 natural spline, N=1024, spline RHS stored in FP32 (a
    2^16-system slice of the 2^20-system workload; the full size runs in the
    benchmark of that workload)."""
    N, M = 1024, 1 << 16
    bands = synth.spline_bands(N)
    f = bs.Factor(bands)
    B = synth.spline_rhs(N, M, 0, "cuda")
    X = bs.solve_refine(f, B, mode=mode)
    torch.cuda.synchronize()
    cols = np.random.default_rng(5).choice(M, 256, replace=False)
    ref = oracle.solve(bands, B[:, cols].double().cpu().numpy())
    assert rel_l2(X[:, cols].cpu().numpy(), ref) < 1e-12


def test_refine_rejects_bad_arguments(bs):
    f = bs.Factor(_bands(3, 16, 0))
    B = torch.zeros(16, 8, dtype=torch.float32, device="cuda")
    with pytest.raises(bs.BsolveError):
        bs.solve_refine(f, B, refine_steps=9)
    with pytest.raises(bs.BsolveError):
        bs.solve_refine(f, B, refine_steps=-1)
    with pytest.raises(bs.BsolveError):
        bs.solve_refine(f, B, mode=7)
    with pytest.raises(ValueError):
        bs.solve_refine(f, B.double())


@pytest.mark.parametrize("mode", [0, 1], ids=["factor", "system"])
def test_refine_zero_tiny_and_huge_columns(bs, mode):
    """Columns that are all zero must come back as exact (signed) zeros; a
    column scaled to 1e-20 and one scaled to 1e30 keep the relative accuracy
    (the FP64 result is assembled from FP32 parts by exact integer widening,
    whose zero and special-value cases run behind a rare branch)."""
    N, M = 300, 64
    bands = _bands(3, N, 4)
    rng = np.random.default_rng(9)
    Bh = rng.uniform(-1, 1, (N, M)).astype(np.float32)
    Bh[:, 3] = 0.0
    Bh[:, 5] = -0.0
    Bh[:, 7] *= np.float32(1e-20)
    Bh[:, 9] *= np.float32(1e30)
    f = bs.Factor(bands)
    X = bs.solve_refine(f, torch.tensor(Bh, device="cuda"), mode=mode).cpu().numpy()
    assert np.all(X[:, 3] == 0.0) and np.all(X[:, 5] == 0.0)
    ref = oracle.solve(bands, Bh.astype(np.float64))
    for j in (0, 7, 9):
        assert rel_l2(X[:, j], ref[:, j]) < 1e-12, j


@pytest.mark.parametrize("width,N,M", [(3, 64, 1024), (5, 512, 1000), (3, 1024, 4096), (5, 37, 9)])
def test_refine_auto_small_batch_is_fp64_solve(bs, width, N, M):
    """REFINE_AUTO on a small batch: B widened exactly to FP64 and solved in
    FP64 (bitwise the FP64 solve of the widened input), right against the
    oracle to FP64 rounding."""
    rng = np.random.default_rng(N + M)
    bands = synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)
    f = bs.Factor(bands)
    B = torch.tensor(rng.uniform(-1, 1, (N, M)), dtype=torch.float32, device="cuda")
    X = bs.solve_refine(f, B, mode=bs.REFINE_AUTO)
    X64 = B.double()
    bs.solve(f, X64)
    torch.cuda.synchronize()
    assert torch.equal(X, X64)
    ref = oracle.solve(bands, B.double().cpu().numpy())
    assert rel_l2(X.cpu().numpy(), ref) < 1e-12


def test_refine_auto_large_batch_is_factor_mode(bs):
    """Above the small-batch threshold REFINE_AUTO is the factor-wise
    refinement, bit for bit."""
    N, M = 64, 65536
    rng = np.random.default_rng(3)
    bands = synth.random_tri_bands(N, rng)
    f = bs.Factor(bands)
    B = torch.tensor(rng.uniform(-1, 1, (N, M)), dtype=torch.float32, device="cuda")
    Xa = bs.solve_refine(f, B, mode=bs.REFINE_AUTO)
    Xf = bs.solve_refine(f, B, mode=bs.REFINE_FACTOR)
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xf)
