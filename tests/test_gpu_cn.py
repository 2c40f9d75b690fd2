"""GPU parity of the fused Crank-Nicolson steps C <- A^{-1} (2I - A) C (the
explicit side formed inside the forward sweep) against the oracle's
definition (explicit product, then solve), through the C ABI.  Tolerances,
on the batch's relative L2 error and every system's relative max-norm error
after the stated number of steps (tests.dense.parity): FP64 1e-12; FP32, for
the oracle run on the FP32-rounded start, the FP32 bound of one solve
(tests.dense.tol32) for each explicit product and each solve (the schemes
are stable, so the rounding errors of the steps add but do not grow)."""
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


def _run(bs, f, C0, dtype, steps):
    C = torch.tensor(C0, dtype=dtype, device="cuda")
    bs.cn_steps(f, C, steps)
    torch.cuda.synchronize()
    return C.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,M,sigma,steps", [(3, 1, 0.3, 2), (5, 6, 2.0, 3), (64, 1000, 0.25, 5),
                                             (257, 1030, 5.0, 3), (1024, 4096, 1.0, 2)])
def test_periodic_diffusion(bs, N, M, sigma, steps, dtype):
    """The paper's benchmark (Sec. 3.2-3.3): periodic (-s, 1 + 2s, -s)."""
    bands = synth.periodic_toeplitz_bands(N, (-sigma, 1 + 2 * sigma, -sigma))
    rng = np.random.default_rng(N + M)
    C0 = rng.uniform(-1, 1, (N, M))
    if dtype == torch.float32:
        C0 = C0.astype(np.float32).astype(np.float64)
    f = bs.Factor(bands, periodic=True)
    X = _run(bs, f, C0, dtype, steps)
    tol = TOL64 if dtype == torch.float64 else tol32(bands, periodic=True, ops=2 * steps)
    parity(X, oracle.cn_steps(bands, C0, steps, periodic=True), tol)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,M,steps", [(4, 1, 1), (5, 7, 2), (64, 512, 3), (513, 2050, 2), (3000, 40, 1)])
def test_hyperdiffusion_penta(bs, N, M, steps, dtype):
    """The paper's second benchmark (Sec. 4.2) with zero boundary values:
    (s, -4s, 1 + 6s, -4s, s)."""
    s = 0.4
    bands = synth.toeplitz_bands(N, (s, -4 * s, 1 + 6 * s, -4 * s, s))
    rng = np.random.default_rng(3 * N + M)
    C0 = rng.uniform(-1, 1, (N, M))
    if dtype == torch.float32:
        C0 = C0.astype(np.float32).astype(np.float64)
    f = bs.Factor(bands)
    X = _run(bs, f, C0, dtype, steps)
    tol = TOL64 if dtype == torch.float64 else tol32(bands, ops=2 * steps)
    parity(X, oracle.cn_steps(bands, C0, steps), tol)


@pytest.mark.parametrize("N,M", [(2, 3), (100, 33), (1000, 64)])
def test_diffusion_tri_random_bands(bs, N, M):
    """Non-constant tridiagonal bands (any handle defines a step)."""
    rng = np.random.default_rng(N * M)
    bands = synth.random_tri_bands(N, rng)
    C0 = rng.uniform(-1, 1, (N, M))
    f = bs.Factor(bands)
    X = _run(bs, f, C0, torch.float64, 3)
    parity(X, oracle.cn_steps(bands, C0, 3), TOL64)


def test_clamped_hyperdiffusion_matrix(bs):
    bands = synth.clamped_hyperdiffusion_bands(512, 0.1)
    rng = np.random.default_rng(5)
    C0 = rng.uniform(-1, 1, (512, 2048))
    f = bs.Factor(bands)
    X = _run(bs, f, C0, torch.float64, 4)
    parity(X, oracle.cn_steps(bands, C0, 4), TOL64)


def test_zero_steps_and_errors(bs):
    bands = synth.periodic_toeplitz_bands(16, (-0.5, 2.0, -0.5))
    f = bs.Factor(bands, periodic=True)
    C0 = np.random.default_rng(1).uniform(-1, 1, (16, 8))
    assert np.array_equal(_run(bs, f, C0, torch.float64, 0), C0)
    C = torch.zeros(8, 16, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="interleaved"):
        bs.cn_steps(f, C, 1, layout="strided")


@pytest.mark.parametrize("kind", ["penta", "periodic"])
@pytest.mark.parametrize("pairs", [0, 1])
def test_fp64_steps_pairs_and_native_with_edge_values(bs, pairs, kind):
    """FP64 steps run the explicit side and the solve in FP32 pairs by
    default (option 0) and natively on request (1); for a periodic handle
    the explicit side wraps around and the Sherman-Morrison sum and
    correction are carried in pairs too.  The batch mixes ordinary systems
    with ones the pairs' range cannot hold (values near 2^300 and 2^-300, a
    subnormal entry; 2^80 for the periodic handle, 2^100 for the banded one,
    in the last or the first row, the rows the periodic explicit side wraps
    to) and a zero system;
    those lanes compute in FP64.  Every system against the oracle."""
    N, M = 37, 70
    per = kind == "periodic"
    bands = (synth.periodic_toeplitz_bands(N, (-0.7, 2.4, -0.7)) if per
             else synth.clamped_hyperdiffusion_bands(N, 0.3))
    rng = np.random.default_rng(11)
    C0 = rng.uniform(-1, 1, (N, M))
    C0[:, 3] *= 2.0 ** 300
    C0[:, 4] *= 2.0 ** -300
    C0[:, 5] = 0.0
    C0[5, 6] = 5e-324
    C0[:, 40] *= 2.0 ** (70 if per else 90)  # inside the pairs' range, near its top
    C0[N - 1, 41] = 2.0 ** (80 if per else 100)  # above it, in the last row
    C0[0, 42] = -(2.0 ** (80 if per else 100))   # above it, in the first row
    f = bs.Factor(bands, periodic=per)
    bs.set_option(bs.OPT_F64_PAIRS, pairs)
    try:
        X = _run(bs, f, C0, torch.float64, 3)
    finally:
        bs.set_option(bs.OPT_F64_PAIRS, 0)
    ref = oracle.cn_steps(bands, C0, 3, periodic=per)
    for j in range(M):
        scale = np.abs(ref[:, j]).max()
        if scale == 0.0:
            assert np.all(X[:, j] == 0.0), j
        else:
            assert np.abs(X[:, j] - ref[:, j]).max() <= 1e-12 * scale, j


@pytest.mark.parametrize("N,M,sigma", [(3, 2, 0.3), (4, 1, 1.0), (5, 33, 2.0), (64, 1000, 0.25), (600, 513, 1.0)])
def test_periodic_pairs_against_native(bs, N, M, sigma):
    """Periodic diffusion steps in FP32 pairs (the default) and native FP64
    (BS_OPT_F64_PAIRS = 1): both within the FP64 tolerance of the oracle,
    and different in their rounding (the pair kernel ran)."""
    bands = synth.periodic_toeplitz_bands(N, (-sigma, 1 + 2 * sigma, -sigma))
    C0 = np.random.default_rng(N * M).uniform(-1, 1, (N, M))
    f = bs.Factor(bands, periodic=True)
    Xp = _run(bs, f, C0, torch.float64, 3)
    bs.set_option(bs.OPT_F64_PAIRS, 1)
    try:
        Xn = _run(bs, f, C0, torch.float64, 3)
    finally:
        bs.set_option(bs.OPT_F64_PAIRS, 0)
    ref = oracle.cn_steps(bands, C0, 3, periodic=True)
    parity(Xp, ref, TOL64)
    parity(Xn, ref, 1e-14)
    if N * M > 1000:
        assert not np.array_equal(Xp, Xn)
