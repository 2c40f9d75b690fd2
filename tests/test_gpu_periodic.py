"""GPU parity of the periodic (cyclic) tridiagonal path -- Sherman-Morrison,
Sec. 3.3, with the rank-one correction fused into the two sweeps -- against
the CPU FP64 oracle, through the C ABI.

Every check bounds the batch's relative L2 error and every system's relative
max-norm error (tests.dense.parity): FP64 1e-12; FP32 storage and arithmetic
twice the FP32 bound of one solve of the cyclic matrix (tests.dense.tol32:
the sweeps, then the rank-one correction with its dot product per system);
BF16 storage with FP32 arithmetic is compared with the oracle's solve of the
BF16-rounded input at the same bound.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, rel_l2, tol32

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _tol32(bands):
    return tol32(bands, periodic=True, ops=2)


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    return m


def _case(N, M, seed, layout):
    rng = np.random.default_rng(seed)
    bands = synth.random_periodic_bands(N, rng)
    B = rng.uniform(-1, 1, (N, M))
    return bands, (B if layout == "interleaved" else np.ascontiguousarray(B.T))


SHAPES = [(3, 1), (3, 7), (4, 2), (5, 33), (17, 31), (64, 1024), (100, 1000), (257, 1027), (513, 4096),
          (1030, 130)]


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("N,M", SHAPES)
def test_periodic_fp64(bs, N, M, layout):
    bands, Bh = _case(N, M, N * 13 + M, layout)
    f = bs.Factor(bands, periodic=True)
    B = torch.tensor(Bh, device="cuda")
    bs.solve(f, B, layout)
    ref = oracle.periodic_tri_solve_bands(bands, Bh, layout)
    parity(B.cpu().numpy(), ref, TOL64, layout)


@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("N,M", SHAPES)
def test_periodic_fp32(bs, N, M, layout):
    bands, Bh = _case(N, M, N * 17 + M, layout)
    Bh = Bh.astype(np.float32).astype(np.float64)
    f = bs.Factor(bands, periodic=True)
    B = torch.tensor(Bh, dtype=torch.float32, device="cuda")
    bs.solve(f, B, layout)
    ref = oracle.periodic_tri_solve_bands(bands, Bh, layout)
    parity(B.double().cpu().numpy(), ref, _tol32(bands), layout)


@pytest.mark.parametrize("N,M", [(3, 4), (64, 1024), (257, 1030)])
def test_periodic_bf16(bs, N, M):
    bands, Bh = _case(N, M, N + 5 * M, "interleaved")
    f = bs.Factor(bands, periodic=True)
    B = torch.tensor(Bh, dtype=torch.bfloat16, device="cuda")
    X = bs.solve_bf16(f, B)
    ref = oracle.periodic_tri_solve_bands(bands, B.double().cpu().numpy())
    parity(X.double().cpu().numpy(), ref, _tol32(bands))


@pytest.mark.parametrize("N,M", [(64, 1), (256, 512)])
def test_paper_constant_case(bs, N, M):
    """The constant periodic matrix of Sec. 3.3 (a, b, c) = (-r, 1 + 2r, -r)
    with r = 0.5 -- the implicit diffusion operator on a periodic grid --
    and a non-symmetric constant case."""
    rng = np.random.default_rng(N + M)
    for a, b, c in ((-0.5, 2.0, -0.5), (0.3, 2.0, -0.6)):
        Bh = rng.uniform(-1, 1, (N, M))
        f = bs.Factor(synth.periodic_toeplitz_bands(N, (a, b, c)), periodic=True)
        B = torch.tensor(Bh, device="cuda")
        bs.solve(f, B)
        parity(B.cpu().numpy(), oracle.periodic_tri_solve(a, b, c, Bh), TOL64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("layout", ["interleaved", "strided"])
@pytest.mark.parametrize("N,M", [(3, 5), (37, 130), (300, 2050)])
def test_periodic_adjoint_and_band_grad(bs, N, M, layout, dtype):
    bands, Bh = _case(N, M, 3 * N + M, layout)
    rng = np.random.default_rng(N * M + 1)
    Gh = rng.uniform(-1, 1, Bh.shape)
    if dtype == torch.float32:
        Bh = Bh.astype(np.float32).astype(np.float64)
        Gh = Gh.astype(np.float32).astype(np.float64)
    f = bs.Factor(bands, periodic=True)
    X = torch.tensor(Bh, dtype=dtype, device="cuda")
    bs.solve(f, X, layout)
    G = torch.tensor(Gh, dtype=dtype, device="cuda")
    G, db = bs.solve_adjoint(f, G, layout, X=X)
    GB_ref = oracle.periodic_solve_adjoint(bands, Gh, layout)
    parity(G.double().cpu().numpy(), GB_ref, TOL64 if dtype == torch.float64 else _tol32(bands), layout)
    # band gradient of the GPU's own GB and X, against the oracle's reduction
    db_ref = oracle.band_grad_periodic(G.double().cpu().numpy(), X.double().cpu().numpy(), layout)
    err = np.max(np.abs(db.cpu().numpy() - db_ref)) / np.max(np.abs(db_ref))
    assert err < (1e-13 if dtype == torch.float64 else 1e-6), err
    # the corner entries are defined (non-zero for random data)
    d = db.cpu().numpy()
    assert d[0, 0] != 0.0 and d[2, N - 1] != 0.0


def test_periodic_solvefn_gradients(bs):
    """SolveFn with periodic=True: d/dB and d/d(bands) of sum(W * X) against
    the oracle's adjoint and periodic band gradient."""
    N, M = 40, 300
    bands, Bh = _case(N, M, 99, "interleaved")
    Wh = np.random.default_rng(100).uniform(-1, 1, (N, M))
    tb = torch.tensor(bands, requires_grad=True)
    B = torch.tensor(Bh, device="cuda", requires_grad=True)
    X = bs.SolveFn.apply(tb, B, None, "interleaved", True)
    (X * torch.tensor(Wh, device="cuda")).sum().backward()
    GB = oracle.periodic_solve_adjoint(bands, Wh)
    Xr = oracle.periodic_tri_solve_bands(bands, Bh)
    parity(B.grad.cpu().numpy(), GB, TOL64)
    assert rel_l2(tb.grad.numpy(), oracle.band_grad_periodic(GB, Xr)) < 1e-12


def test_periodic_sampled_large(bs):
    """N=1024, M=2^18 FP64 in the launch configuration of a large batch;
    64 sampled systems against the oracle."""
    N, M = 1024, 1 << 18
    rng = np.random.default_rng(7)
    bands = synth.random_periodic_bands(N, rng)
    f = bs.Factor(bands, periodic=True)
    B = synth.uniform_rhs(N, M, 7, "cuda")
    cols = np.sort(rng.choice(M, 64, replace=False))
    B_s = B[:, cols].cpu().numpy()
    bs.solve(f, B)
    ref = oracle.periodic_tri_solve_bands(bands, B_s)
    parity(B[:, cols].cpu().numpy(), ref, TOL64)


def test_periodic_unsupported_paths(bs):
    bands, _ = _case(16, 4, 1, "interleaved")
    f = bs.Factor(bands, periodic=True)
    B = torch.rand(16, 8, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="periodic"):
        bs.solve_refine(f, B)
    u = torch.rand(16, 16, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="periodic"):
        bs.adi_halfstep(f, u, 0.5, 0)


def test_periodic_factor_errors(bs):
    with pytest.raises(ValueError):
        bs.Factor(np.ones((5, 8)), periodic=True)
    bands = synth.random_periodic_bands(8, np.random.default_rng(3))
    bad = bands.copy()
    bad[1, 0] = 0.0  # b_1 = 0: the split gamma = -b_1 is undefined
    with pytest.raises(RuntimeError, match="b_1"):
        bs.Factor(bad, periodic=True)
    with pytest.raises(RuntimeError, match="N must be"):
        bs.Factor(bands[:, :2], periodic=True)
    # a singular cyclic matrix: every row sums to zero (a + b + c = 0)
    sing = synth.periodic_toeplitz_bands(8, (-1.0, 2.0, -1.0))
    with pytest.raises(RuntimeError, match="singular|pivot"):
        bs.Factor(sing, periodic=True)


@pytest.mark.parametrize("b", [2.05, 2.6])
def test_periodic_weak_dominance(bs, b):
    """Cyclic (-1, b, -1) with N = 4096: the correction vectors decay slowly
    (ratio ~0.8 for b = 2.05), so hundreds of rows at each end carry
    correction terms and the rest skip them; FP64 parity with the oracle."""
    N, M = 4096, 130
    rng = np.random.default_rng(int(b * 100))
    Bh = rng.uniform(-1, 1, (N, M))
    f = bs.Factor(synth.periodic_toeplitz_bands(N, (-1.0, b, -1.0)), periodic=True)
    for layout in ("interleaved", "strided"):
        B_in = Bh if layout == "interleaved" else np.ascontiguousarray(Bh.T)
        B = torch.tensor(B_in, device="cuda")
        bs.solve(f, B, layout)
        ref = oracle.periodic_tri_solve(-1.0, b, -1.0, B_in, layout)
        parity(B.cpu().numpy(), ref, TOL64, layout)


@pytest.fixture
def pair_mode(bs):
    yield lambda m: bs.set_option(bs.OPT_F64_PAIRS, m)
    bs.set_option(bs.OPT_F64_PAIRS, 0)


def _solve_both(bs, f, Bh):
    X = torch.tensor(Bh, device="cuda")
    bs.solve(f, X)
    G = torch.tensor(Bh, device="cuda")
    bs.solve_adjoint(f, G)
    return X.cpu().numpy(), G.cpu().numpy()


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("N,M", [(3, 2), (4, 1), (5, 34), (64, 1024), (257, 1030), (1030, 4096)])
def test_periodic_fp64_pairs(bs, pair_mode, N, M, mode):
    """FP64 periodic solves carried in FP32 pairs (BS_OPT_F64_PAIRS 2: one
    system per thread, 3: two): the Sherman-Morrison sum sigma and the
    correction x_i = y_i - sigma pc_i (Sec. 3.3) in pair arithmetic, primal
    and adjoint, against the oracle at the FP64 tolerance; they differ from
    the native FP64 solve (option 1) by the pairs' rounding only."""
    bands, Bh = _case(N, M, 5 * N + M, "interleaved")
    Bh = Bh * np.ldexp(1.0, np.random.default_rng(N).integers(-20, 20, M))
    f = bs.Factor(bands, periodic=True)
    pair_mode(mode)
    Xp, Gp = _solve_both(bs, f, Bh)
    pair_mode(1)
    Xn, Gn = _solve_both(bs, f, Bh)
    ref_x = oracle.periodic_tri_solve_bands(bands, Bh)
    ref_g = oracle.periodic_solve_adjoint(bands, Bh)
    parity(Xp, ref_x, TOL64)
    parity(Gp, ref_g, TOL64)
    parity(Xn, ref_x, 1e-14)
    parity(Gn, ref_g, 1e-14)
    if N * M > 1000:  # the pair path ran: its rounding differs from FP64's
        assert not np.array_equal(Xp, Xn)


@pytest.mark.parametrize("mode", [2, 3])
def test_periodic_pairs_out_of_range_inputs(bs, pair_mode, mode):
    """Inputs the periodic pair sweeps do not hold (|x| >= 2^80, so that the
    correction stays inside FP32; 1e200; 1e-200; an FP64 subnormal) send
    their warp to native FP64 from that row on, sigma carried over; NaN and
    inf poison only their own system; a zero system stays zero."""
    pair_mode(mode)
    N, M = 300, 4096
    bands = synth.random_periodic_bands(N, np.random.default_rng(21))
    Bh = np.random.default_rng(22).uniform(-1, 1, (N, M))
    specials = {70: ("scale", 1e200), 200: ("scale", 1e-200), 333: ("one", 5e-324), 501: ("one", 2.0 ** 85),
                502: ("one", 2.0 ** 80), 640: ("one", 1e-25), 900: ("nan", np.nan), 1300: ("inf", np.inf),
                2000: ("zero", 0.0)}
    for j, (kind, v) in specials.items():
        row = (j * 7) % N
        if kind == "scale":
            Bh[:, j] *= v
        elif kind == "zero":
            Bh[:, j] = 0.0
        else:
            Bh[row, j] = v
    f = bs.Factor(bands, periodic=True)
    X, G = _solve_both(bs, f, Bh)
    finite = [j for j in range(M) if np.all(np.isfinite(Bh[:, j]))]
    bad = [j for j in range(M) if j not in finite]
    refs = (oracle.periodic_tri_solve_bands(bands, Bh[:, finite]), oracle.periodic_solve_adjoint(bands, Bh[:, finite]))
    for got, ref in zip((X, G), refs):
        parity(got[:, finite], ref, TOL64)
        for j in bad:
            assert not np.all(np.isfinite(got[:, j]))
    assert np.all(X[:, 2000] == 0) and np.all(G[:, 2000] == 0)
