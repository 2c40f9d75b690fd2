"""GPU parity of the plain sweeps against the CPU FP64 oracle, through the C
ABI.  Every check bounds both the relative L2 error of the batch and the
relative max-norm error of every system (tests.dense.parity):
  FP64: 1e-12 (the stated target for every FP64 path);
  FP32 storage and arithmetic: width * kappa_inf(A) * 2^-24 per matrix
    (tests.dense.tol32; ~1e-6 for the matrices here);
  BF16 storage, FP32 arithmetic: compared with the oracle's solve of the
    BF16-rounded B, so only the FP32 arithmetic differs: the same bound.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, tol32

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    return m


def _bands(width, N, seed):
    rng = np.random.default_rng(seed)
    return synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)


def _rhs(N, M, seed, layout):
    rng = np.random.default_rng(seed + 7)
    B = rng.uniform(-1, 1, (N, M))
    return B if layout == "interleaved" else np.ascontiguousarray(B.T)


def _gpu_solve(bs, f, Bh, dtype, layout):
    B = torch.tensor(Bh, dtype=dtype, device="cuda")
    bs.solve(f, B, layout)
    torch.cuda.synchronize()
    return B.double().cpu().numpy()


def test_config0_random_tri_fp64(bs):
    """Tridiagonal, N=64, M=1024, a,c ~ U(-1,1), b = |a|+|c|+U(1,2), RHS ~
    U(-1,1), seed 0 -- the full workload against the oracle."""
    bands, Bh = synth.random_tri_case(64, 1024, 0)
    f = bs.Factor(bands)
    for layout in ("interleaved", "strided"):
        B_in = Bh if layout == "interleaved" else np.ascontiguousarray(Bh.T)
        X = _gpu_solve(bs, f, B_in, torch.float64, layout)
        ref = oracle.solve(bands, B_in, layout)
        parity(X, ref, TOL64, layout)


SHAPES = [(3, 2, 1), (3, 2, 5), (3, 3, 7), (3, 33, 31), (3, 100, 1000), (3, 257, 1027), (3, 64, 4096),
          (5, 4, 1), (5, 5, 6), (5, 37, 33), (5, 130, 515), (5, 512, 2048)]


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width,N,M", SHAPES)
def test_fp64_ragged(bs, width, N, M, layout):
    bands = _bands(width, N, N * 7 + M)
    Bh = _rhs(N, M, M, layout)
    f = bs.Factor(bands)
    X = _gpu_solve(bs, f, Bh, torch.float64, layout)
    parity(X, oracle.solve(bands, Bh, layout), TOL64, layout)


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width,N,M", SHAPES)
def test_fp32_ragged(bs, width, N, M, layout):
    bands = _bands(width, N, N * 11 + M)
    Bh = _rhs(N, M, M + 1, layout).astype(np.float32).astype(np.float64)
    f = bs.Factor(bands)
    X = _gpu_solve(bs, f, Bh, torch.float32, layout)
    parity(X, oracle.solve(bands, Bh, layout), tol32(bands), layout)


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width,N,M", [(3, 64, 1024), (5, 37, 33), (3, 257, 1027), (5, 512, 4096)])
def test_bf16_storage(bs, width, N, M, layout):
    bands = _bands(width, N, N + M)
    Bh = _rhs(N, M, M + 2, layout)
    B = torch.tensor(Bh, dtype=torch.bfloat16, device="cuda")
    f = bs.Factor(bands)
    X = bs.solve_bf16(f, B, layout=layout)
    torch.cuda.synchronize()
    ref = oracle.solve(bands, B.double().cpu().numpy(), layout)
    parity(X.double().cpu().numpy(), ref, tol32(bands), layout)


def test_misaligned_pointer_uses_scalar_path(bs):
    """A view starting one element into a buffer cannot take 128-bit loads."""
    N, M = 40, 64
    bands = _bands(3, N, 5)
    Bh = _rhs(N, M, 9, "interleaved")
    buf = torch.zeros(N * M + 1, dtype=torch.float64, device="cuda")
    B = buf[1:].view(N, M)
    B.copy_(torch.tensor(Bh, device="cuda"))
    f = bs.Factor(bands)
    bs.solve(f, B)
    torch.cuda.synchronize()
    parity(B.cpu().numpy(), oracle.solve(bands, Bh), TOL64)
    assert buf[0].item() == 0.0


def test_solve_leaves_other_memory_alone(bs):
    """Canaries on both sides of the batch stay untouched."""
    N, M = 77, 333
    bands = _bands(5, N, 8)
    Bh = _rhs(N, M, 10, "interleaved")
    pad = 4096
    buf = torch.full((pad + N * M + pad,), 12345.0, dtype=torch.float64, device="cuda")
    B = buf[pad:pad + N * M].view(N, M)
    B.copy_(torch.tensor(Bh, device="cuda"))
    f = bs.Factor(bands)
    bs.solve(f, B)
    torch.cuda.synchronize()
    assert torch.all(buf[:pad] == 12345.0) and torch.all(buf[pad + N * M:] == 12345.0)
    parity(B.cpu().numpy(), oracle.solve(bands, Bh), TOL64)


def test_deterministic(bs):
    bands = _bands(5, 300, 1)
    Bh = _rhs(300, 5000, 2, "interleaved")
    f = bs.Factor(bands)
    a = _gpu_solve(bs, f, Bh, torch.float64, "interleaved")
    b = _gpu_solve(bs, f, Bh, torch.float64, "interleaved")
    assert np.array_equal(a, b)


def test_singular_rejected(bs):
    bands = synth.toeplitz_bands(6, (1.0, 0.0, 1.0))
    with pytest.raises(bs.BsolveError) as ei:
        bs.Factor(bands)
    assert ei.value.status == 2


def test_wrong_shape_rejected(bs):
    f = bs.Factor(_bands(3, 10, 0))
    with pytest.raises(ValueError):
        bs.solve(f, torch.zeros(11, 4, dtype=torch.float64, device="cuda"))


def test_config1_penta_full_size_sampled(bs):
    """A = I + 0.1 D4 clamped, N=512, M=65536, RHS ~ N(0,1) (seed 0) at full
    size in the launch configuration the benchmark times; 512 sampled systems
    are checked against the oracle one by one, the rest via the residual."""
    N, M = 512, 65536
    bands = synth.clamped_hyperdiffusion_bands(N, 0.1)
    f = bs.Factor(bands)
    B0 = synth.normal_rhs(N, M, 0, "cuda")
    X = B0.clone()
    bs.solve(f, X)
    torch.cuda.synchronize()
    cols = np.random.default_rng(3).choice(M, 512, replace=False)
    cols = np.union1d(cols, [0, 1, M - 2, M - 1])
    Bs = B0[:, cols].cpu().numpy()
    ref = oracle.solve(bands, Bs)
    parity(X[:, cols].cpu().numpy(), ref, TOL64)
    # every system: relative residual with the banded product on the GPU in FP64
    b = torch.tensor(bands, device="cuda")
    R = B0.clone()
    for k, off in enumerate(range(-2, 3)):
        lo, hi = max(0, -off), N - max(0, off)
        R[lo:hi] -= b[k, lo:hi, None] * X[lo + off:hi + off]
    assert (torch.linalg.norm(R) / torch.linalg.norm(B0)).item() < 1e-13
    # FP32 on the same data: error stated against the oracle
    X32 = B0.float()
    bs.solve(f, X32)
    torch.cuda.synchronize()
    ref32 = oracle.solve(bands, B0[:, cols].float().double().cpu().numpy())
    parity(X32[:, cols].double().cpu().numpy(), ref32, tol32(bands))


@pytest.mark.parametrize("width,N,M", [(3, 64, 1024), (3, 1000, 4100), (3, 1024, 8192), (5, 512, 4096),
                                       (5, 37, 36), (5, 4, 8), (3, 2, 4), (5, 2000, 1028), (3, 4096, 64)])
def test_onchip_kernel_matches_streaming_and_oracle(bs, width, N, M):
    """FP32 and BF16-input solves and FP32 adjoints through the on-chip TMA
    kernel (option 2) and the streaming kernels (option 1) give the oracle's
    answer within the FP32 bound, and the device status stays clean."""
    from paper_1909_04539_gb300 import api
    bands = _bands(width, N, 3 * N + M)
    Bh = np.random.default_rng(M).uniform(-1, 1, (N, M))
    f = bs.Factor(bands)
    outs = {}
    bs.set_option(api.OPT_TWISTED, 1)  # small tridiagonal batches: not the two-ended sweep
    for kern in (2, 1):
        bs.set_option(api.OPT_SWEEP_KERNEL, kern)
        X = torch.tensor(Bh, dtype=torch.float32, device="cuda")
        bs.solve(f, X)
        Y = torch.tensor(Bh, dtype=torch.float32, device="cuda")
        bs.solve_adjoint(f, Y)
        Xb = bs.solve_bf16(f, torch.tensor(Bh, dtype=torch.bfloat16, device="cuda"))
        torch.cuda.synchronize()
        outs[kern] = (X.double().cpu().numpy(), Y.double().cpu().numpy(), Xb.double().cpu().numpy())
    bs.set_option(api.OPT_SWEEP_KERNEL, 0)
    bs.set_option(api.OPT_TWISTED, 0)
    B32 = Bh.astype(np.float32).astype(np.float64)
    Bb = torch.tensor(Bh, dtype=torch.bfloat16).double().numpy()
    ref, refa, refb = oracle.solve(bands, B32), oracle.solve_adjoint(bands, B32), oracle.solve(bands, Bb)
    tol = tol32(bands)
    for kern in (2, 1):
        X, Y, Xb = outs[kern]
        parity(X, ref, tol)
        parity(Y, refa, tol)
        parity(Xb, refb, tol)
    assert bs.device_status() == 0


@pytest.mark.parametrize("cta", [32, 64, 128, 256, 448])
@pytest.mark.parametrize("width,N,M,dtype", [(5, 512, 4100, torch.float64), (3, 257, 1027, torch.float32),
                                              (3, 1000, 3000, torch.float64)])
def test_cta_threads_option(bs, width, N, M, dtype, cta):
    """Every CTA size of BS_OPT_CTA_THREADS gives the oracle's solution (the
    last shape is row-partitioned; sizes above 128 reach the windowed sweeps
    only)."""
    bands = _bands(width, N, 11)
    Bh = _rhs(N, M, 11, "interleaved")
    if dtype == torch.float32:
        Bh = Bh.astype(np.float32).astype(np.float64)
    f = bs.Factor(bands)
    bs.set_option(bs.OPT_CTA_THREADS, cta)
    try:
        X = torch.tensor(Bh, dtype=dtype, device="cuda")
        bs.solve(f, X)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_CTA_THREADS, 0)
    parity(X.double().cpu().numpy(), oracle.solve(bands, Bh), TOL64 if dtype == torch.float64 else tol32(bands))
