"""GPU parity at large N, where a CTA's coefficients no longer fit in shared
memory and the sweeps read them from global memory (one thread per system,
partition and two-ended sweep off), and on the default (row-partitioned)
path; sampled systems against the CPU FP64 oracle, through the C ABI.
Every check bounds the relative L2 error of the sampled systems and the
relative max-norm error of each (tests.dense.parity): FP64 1e-12, FP32 /
BF16-stored the FP32 bound of the matrix (tests.dense.tol32; against the
oracle on the rounded inputs)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    yield m
    m.set_option(m.OPT_PARTITION, 0)
    m.set_option(m.OPT_TWISTED, 0)


def _bands(width, N, rng):
    return synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)


@pytest.mark.parametrize("one_thread", [True, False])
@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width", [3, 5])
def test_large_n_solve(bs, width, layout, one_thread):
    N, M = 20000, 1500
    rng = np.random.default_rng(width * 7 + (layout == "strided"))
    bands = _bands(width, N, rng)
    f = bs.Factor(bands)
    B = rng.uniform(-1, 1, (N, M))
    cols = rng.choice(M, 24, replace=False)
    ref = oracle.solve(bands, B[:, cols])
    tr = (lambda A: A) if layout == "interleaved" else (lambda A: np.ascontiguousarray(A.T))
    bs.set_option(bs.OPT_PARTITION, 1 if one_thread else 0)
    bs.set_option(bs.OPT_TWISTED, 1 if one_thread else 0)
    try:
        for dtype, tol in ((torch.float64, 1e-12), (torch.float32, tol32(bands))):
            X = torch.tensor(tr(B), dtype=dtype, device="cuda")
            bs.solve(f, X, layout)
            torch.cuda.synchronize()
            Xh = X.double().cpu().numpy()
            Xh = Xh if layout == "interleaved" else Xh.T
            r = ref if dtype == torch.float64 else oracle.solve(bands, B[:, cols].astype(np.float32).astype(np.float64))
            parity(Xh[:, cols], r, tol)
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
        bs.set_option(bs.OPT_TWISTED, 0)


@pytest.mark.parametrize("width", [3, 5])
def test_large_n_bf16_adjoint_band_grad(bs, width):
    N, M = 16384, 1024
    rng = np.random.default_rng(50 + width)
    bands = _bands(width, N, rng)
    f = bs.Factor(bands)
    B = rng.uniform(-1, 1, (N, M))
    cols = rng.choice(M, 16, replace=False)
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 1)
    try:
        Bb = torch.tensor(B, dtype=torch.bfloat16, device="cuda")
        Xb = bs.solve_bf16(f, Bb)
        X = torch.tensor(B, device="cuda")
        bs.solve(f, X)
        G = torch.tensor(rng.uniform(-1, 1, (N, M)), device="cuda")
        Gh = G.cpu().numpy()
        G, db = bs.solve_adjoint(f, G, X=X)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
        bs.set_option(bs.OPT_TWISTED, 0)
    Bbh = Bb.double().cpu().numpy()
    parity(Xb.double().cpu().numpy()[:, cols], oracle.solve(bands, Bbh[:, cols]), tol32(bands))
    GBr = oracle.solve_adjoint(bands, Gh[:, cols])
    parity(G.cpu().numpy()[:, cols], GBr, 1e-12)
    db_ref = oracle.band_grad(width, G.cpu().numpy(), X.cpu().numpy())
    assert np.max(np.abs(db.cpu().numpy() - db_ref)) / np.max(np.abs(db_ref)) < 1e-13


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_large_n_cn_steps(bs, dtype):
    """Crank-Nicolson steps with the coefficients and explicit bands read from
    global memory (N = 20000)."""
    N, M = 20000, 64
    s = 0.3
    bands = synth.toeplitz_bands(N, (s, -4 * s, 1 + 6 * s, -4 * s, s))
    rng = np.random.default_rng(77)
    C0 = rng.uniform(-1, 1, (N, M))
    if dtype == torch.float32:
        C0 = C0.astype(np.float32).astype(np.float64)
    f = bs.Factor(bands)
    C = torch.tensor(C0, dtype=dtype, device="cuda")
    bs.cn_steps(f, C, 2)
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == torch.float64 else tol32(bands, ops=4)
    parity(C.double().cpu().numpy(), oracle.cn_steps(bands, C0, 2), tol)
