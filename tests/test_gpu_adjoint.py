"""GPU parity of the adjoint solve A^{-T} G and of the band-gradient
reduction against the oracle, and of the autograd wrapper against finite
differences of the loss."""
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


def _to(X, layout):
    return X if layout == "interleaved" else np.ascontiguousarray(X.T)


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width,N,M", [(3, 2, 3), (3, 64, 1024), (3, 129, 77), (5, 4, 2), (5, 37, 33),
                                       (5, 512, 1000)])
def test_adjoint_and_band_grad_fp64(bs, width, N, M, layout):
    rng = np.random.default_rng(N + M + width)
    bands = _bands(width, N, N + 3)
    Bh = rng.uniform(-1, 1, (N, M))
    Gh = rng.uniform(-1, 1, (N, M))
    Xref = oracle.solve(bands, Bh)
    GBref = oracle.solve_adjoint(bands, Gh)
    dref = oracle.band_grad(width, GBref, Xref)
    f = bs.Factor(bands)
    X = torch.tensor(_to(Xref, layout), device="cuda")
    G = torch.tensor(_to(Gh, layout), device="cuda")
    G, db = bs.solve_adjoint(f, G, layout, X=X)
    torch.cuda.synchronize()
    GB = G.cpu().numpy()
    parity(GB, _to(GBref, layout), 1e-12, layout)
    assert rel_l2(db.cpu().numpy(), dref) < 1e-12


@pytest.mark.parametrize("width", [3, 5])
def test_adjoint_fp32(bs, width):
    N, M = 200, 999
    rng = np.random.default_rng(width)
    bands = _bands(width, N, 5)
    Gh = rng.uniform(-1, 1, (N, M)).astype(np.float32).astype(np.float64)
    f = bs.Factor(bands)
    G = torch.tensor(Gh, dtype=torch.float32, device="cuda")
    bs.solve_adjoint(f, G)
    torch.cuda.synchronize()
    parity(G.double().cpu().numpy(), oracle.solve_adjoint(bands, Gh), tol32(bands))


def test_band_grad_deterministic(bs):
    N, M = 300, 20000
    rng = np.random.default_rng(1)
    bands = _bands(5, N, 2)
    f = bs.Factor(bands)
    X = torch.tensor(rng.uniform(-1, 1, (N, M)), device="cuda")
    G0 = torch.tensor(rng.uniform(-1, 1, (N, M)), device="cuda")
    _, d1 = bs.solve_adjoint(f, G0.clone(), X=X)
    _, d2 = bs.solve_adjoint(f, G0.clone(), X=X)
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)


@pytest.mark.parametrize("width", [3, 5])
def test_autograd_against_finite_differences(bs, width):
    """Directional central differences of L = sum(W * A^{-1} B) in FP64, for a
    random direction in the bands and in B at once."""
    N, M = 24, 6
    rng = np.random.default_rng(10 + width)
    bands0 = _bands(width, N, 7)
    B0 = rng.uniform(-1, 1, (N, M))
    W = rng.uniform(-1, 1, (N, M))
    dirb = rng.uniform(-1, 1, bands0.shape)
    dirB = rng.uniform(-1, 1, B0.shape)
    h = width // 2
    for k in range(width):  # entries outside the matrix do not exist
        for i in range(N):
            if not (0 <= i + k - h < N):
                dirb[k, i] = 0.0
    bands = torch.tensor(bands0, requires_grad=True)
    B = torch.tensor(B0, device="cuda", requires_grad=True)
    X = bs.SolveFn.apply(bands, B)
    loss = (X * torch.tensor(W, device="cuda")).sum()
    loss.backward()
    analytic = float((bands.grad.numpy() * dirb).sum() + (B.grad.cpu().numpy() * dirB).sum())

    def L(t):
        return float(np.sum(W * oracle.solve(bands0 + t * dirb, B0 + t * dirB)))

    eps = 1e-6
    fd = (L(eps) - L(-eps)) / (2 * eps)
    assert abs(analytic - fd) < 1e-7 * (1 + abs(fd)), (analytic, fd)
    # and exactly against the oracle's gradient
    GB = oracle.solve_adjoint(bands0, W)
    assert rel_l2(B.grad.cpu().numpy(), GB) < 1e-12
    assert rel_l2(bands.grad.numpy(), oracle.band_grad(width, GB, oracle.solve(bands0, B0))) < 1e-12


def _band_abs_bound(width, GB, X):
    """sum_j |GB[i, j]| |X[i + k - h, j]| per band entry: the scale a rounding
    error of the reduction is measured against."""
    return oracle.band_grad(width, np.abs(GB), np.abs(X)) * -1.0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("width", [3, 5])
@pytest.mark.parametrize("case", ["in_range", "huge", "tiny", "zeros"])
def test_band_grad_pair_sums(bs, width, layout, case, dtype):
    """Band gradient with pair sums (FP32 data: every band; FP64 data: the
    top band) over runs of systems, FP64 sums of the runs, against the oracle
    on the same values in FP64: within 1e-12 of the absolute-value sums per
    entry.  'huge' and 'tiny' put one value outside [2^-32, 2^48), which
    sends the CTAs that meet it to FP64 FMAs; 'zeros' zeroes whole rows and
    systems."""
    N, M = 301, 5003
    rng = np.random.default_rng(width + 17)
    GB = rng.uniform(-1, 1, (N, M)).astype(dtype)
    X = rng.uniform(-1, 1, (N, M)).astype(dtype)
    if case == "huge":
        GB[7, 123] = 2.0 ** 60
    elif case == "tiny":
        X[150, 4000] = 2.0 ** -40
    elif case == "zeros":
        GB[10:20, :] = 0.0
        X[:, 100:300] = 0.0
    ref = oracle.band_grad(width, GB.astype(np.float64), X.astype(np.float64))
    scale = _band_abs_bound(width, GB.astype(np.float64), X.astype(np.float64))
    f = bs.Factor(_bands(width, N, 3))
    db = bs.band_grad(f, torch.tensor(_to(GB, layout), device="cuda"), torch.tensor(_to(X, layout), device="cuda"),
                      layout)
    got = db.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300)
    assert rel_l2(got, ref) < 1e-12
