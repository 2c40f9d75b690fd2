"""GPU parity of the FP64 solves carried in FP32 pairs (BS_OPT_F64_PAIRS,
csrc/sweep_df.cu, csrc/sweep_win.cu) against the FP64 oracle, through the C
ABI, with and without the windowed sweeps (BS_OPT_WINDOW).

Tolerance: 1e-12 relative L2 per system (the largest over the batch), the
stated FP64 target; the arithmetic carries ~48 significant bits, so errors
are ~1e-14 on these well-conditioned bands.  Also: the same numbers from one
and two systems per thread, ragged batches (odd M, M = 1, N = 2..4), inputs
outside the pairs' range (huge, tiny, subnormal, inf, NaN: those warps
continue in native FP64), a matrix whose sweep gains exceed the admitted
bound (native FP64 throughout), zero systems, and the band gradient on the
adjoint the pairs produce.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    return m


@pytest.fixture(params=[2, 1], ids=["windowed", "two-sweep"])
def one_thread_paths(bs, request):
    """Every FP64 solve one thread per system (no partition, no two-ended
    sweep), so that small batches also take the pair sweeps; run once with
    the windowed sweeps (forward values on chip) and once with the two-sweep
    kernel (forward values in the output buffer)."""
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 1)
    bs.set_option(bs.OPT_WINDOW, request.param)
    yield
    bs.set_option(bs.OPT_PARTITION, 0)
    bs.set_option(bs.OPT_TWISTED, 0)
    bs.set_option(bs.OPT_F64_PAIRS, 0)
    bs.set_option(bs.OPT_WINDOW, 0)


def _bands(width, N, seed):
    rng = np.random.default_rng(seed)
    return synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)


def _solve(bs, f, Bh, adjoint=False):
    B = torch.tensor(Bh, device="cuda")
    if adjoint:
        bs.solve_adjoint(f, B)
    else:
        bs.solve(f, B)
    torch.cuda.synchronize()
    return B.cpu().numpy()


SHAPES = [(3, 2, 1), (3, 3, 7), (3, 33, 31), (3, 64, 1024), (3, 257, 1027), (3, 1024, 4096),
          (5, 4, 1), (5, 5, 6), (5, 37, 33), (5, 130, 515), (5, 512, 2048), (5, 600, 4097)]


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("width,N,M", SHAPES)
def test_pairs_primal_and_adjoint(bs, one_thread_paths, width, N, M, mode):
    bs.set_option(bs.OPT_F64_PAIRS, mode)
    bands = _bands(width, N, N * 13 + M)
    rng = np.random.default_rng(N + M)
    Bh = rng.standard_normal((N, M)) * np.ldexp(1.0, rng.integers(-20, 20, M))
    f = bs.Factor(bands)
    X = _solve(bs, f, Bh)
    G = _solve(bs, f, Bh, adjoint=True)
    parity(X, oracle.solve(bands, Bh), TOL)
    parity(G, oracle.solve_adjoint(bands, Bh), TOL)


@pytest.mark.parametrize("width,N,M", [(3, 257, 1030), (5, 512, 4096)])
def test_one_and_two_systems_per_thread_agree(bs, one_thread_paths, width, N, M):
    """Per system the arithmetic does not depend on how many systems a
    thread carries: bitwise equal results."""
    bands = _bands(width, N, 3)
    Bh = np.random.default_rng(4).uniform(-1, 1, (N, M))
    f = bs.Factor(bands)
    bs.set_option(bs.OPT_F64_PAIRS, 2)
    X1 = _solve(bs, f, Bh)
    bs.set_option(bs.OPT_F64_PAIRS, 3)
    X2 = _solve(bs, f, Bh)
    assert np.array_equal(X1, X2)


def test_pairs_closer_to_oracle_than_native_needs(bs, one_thread_paths):
    """The clamped I + 0.1 D4 benchmark matrix (N = 512): pairs and native
    FP64 both match the oracle per system; the pairs within 1e-13, native
    FP64 within 1e-14 (max norm per system)."""
    bands = synth.clamped_hyperdiffusion_bands(512, 0.1)
    Bh = np.random.default_rng(0).standard_normal((512, 8192))
    f = bs.Factor(bands)
    ref = oracle.solve(bands, Bh)
    bs.set_option(bs.OPT_F64_PAIRS, 0)
    Xp = _solve(bs, f, Bh)
    bs.set_option(bs.OPT_F64_PAIRS, 1)
    Xn = _solve(bs, f, Bh)
    parity(Xp, ref, 1e-13)
    parity(Xn, ref, 1e-14)


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("width", [3, 5])
def test_out_of_range_inputs_fall_back_per_warp(bs, one_thread_paths, width, mode):
    """Systems with inputs the pairs cannot hold (1e200, 1e-200, an FP64
    subnormal, 2^101) are computed in native FP64 by their warp; a NaN or inf
    input poisons only its own system; the other systems of the same warps
    stay within tolerance.  Each special system sits in a different warp, at a
    different row (the switch happens mid-sweep)."""
    bs.set_option(bs.OPT_F64_PAIRS, mode)
    N, M = 300, 4096
    bands = _bands(width, N, 11)
    rng = np.random.default_rng(12)
    Bh = rng.uniform(-1, 1, (N, M))
    specials = {70: ("scale", 1e200), 200: ("scale", 1e-200), 333: ("one", 5e-324), 501: ("one", 2.0 ** 101),
                640: ("one", 1e-25), 900: ("nan", np.nan), 1300: ("inf", np.inf), 2000: ("zero", 0.0)}
    for j, (kind, v) in specials.items():
        row = (j * 7) % N
        if kind == "scale":
            Bh[:, j] *= v
        elif kind == "zero":
            Bh[:, j] = 0.0
        else:
            Bh[row, j] = v
    f = bs.Factor(bands)
    X = _solve(bs, f, Bh)
    G = _solve(bs, f, Bh, adjoint=True)
    finite = [j for j in range(M) if np.all(np.isfinite(Bh[:, j]))]
    bad = [j for j in range(M) if j not in finite]
    for got, ref in ((X, oracle.solve(bands, Bh[:, finite])), (G, oracle.solve_adjoint(bands, Bh[:, finite]))):
        parity(got[:, finite], ref, TOL)
        for j in bad:
            assert not np.all(np.isfinite(got[:, j]))
    assert np.all(X[:, 2000] == 0) and np.all(G[:, 2000] == 0)


def test_unadmitted_matrices_stay_native(bs, one_thread_paths):
    """Handles the pairs do not admit still solve correctly (native FP64):
    a well-conditioned matrix scaled by 1e-35 (its sweep coefficients 1/p
    ~1e35 lie above the pairs' coefficient range 2^100), and a diagonally
    dominant tridiagonal matrix whose rows are scaled by 2^0 .. 2^-30 (its
    forward sweep scales 1/p_i reach 2^30, a gain above 2^24)."""
    bs.set_option(bs.OPT_F64_PAIRS, 2)
    rng = np.random.default_rng(1)
    N, M = 40, 640
    scaled = _bands(5, N, 7) * 1e-35
    steep = _bands(3, N, 8) * np.ldexp(1.0, -np.round(np.arange(N) * 30 / (N - 1)).astype(int))
    for bands in (scaled, steep):
        Bh = rng.uniform(-1, 1, (N, M))
        f = bs.Factor(bands)
        X = _solve(bs, f, Bh)
        parity(X, oracle.solve(bands, Bh), TOL)


@pytest.mark.parametrize("width,N,M", [(3, 129, 777), (5, 512, 4096)])
def test_band_gradient_of_pair_adjoint(bs, one_thread_paths, width, N, M):
    bs.set_option(bs.OPT_F64_PAIRS, 0)
    bands = _bands(width, N, 21)
    rng = np.random.default_rng(22)
    Bh = rng.uniform(-1, 1, (N, M))
    Gh = rng.uniform(-1, 1, (N, M))
    Xref = oracle.solve(bands, Bh)
    GBref = oracle.solve_adjoint(bands, Gh)
    f = bs.Factor(bands)
    X = torch.tensor(Bh, device="cuda")
    bs.solve(f, X)
    G = torch.tensor(Gh, device="cuda")
    G, db = bs.solve_adjoint(f, G, X=X)
    torch.cuda.synchronize()
    parity(G.cpu().numpy(), GBref, TOL)
    dref = oracle.band_grad(width, GBref, Xref)
    assert np.linalg.norm(db.cpu().numpy() - dref) / np.linalg.norm(dref) < TOL


def test_default_path_full_size_benchmark_batch(bs):
    """The benchmark's penta N = 512, M = 65536 batch through the default
    path (pairs, two systems per thread): a 2048-system sample per system
    against the oracle, and every system through the FP64 residual."""
    N, M = 512, 65536
    bands = synth.clamped_hyperdiffusion_bands(N, 0.1)
    B = synth.normal_rhs(N, M, 0, "cuda")
    f = bs.Factor(bands)
    X = B.clone()
    bs.solve(f, X)
    torch.cuda.synchronize()
    cols = np.random.default_rng(3).choice(M, 2048, replace=False)
    Bs = B[:, cols].cpu().numpy()
    parity(X[:, cols].cpu().numpy(), oracle.solve(bands, Bs), TOL)
    # every system: the relative FP64 residual |B - A X| / |B| per system
    b = torch.tensor(bands, device="cuda")
    R = B.clone()
    for k in range(5):
        off = k - 2
        lo, hi = max(0, -off), N - max(0, off)
        R[lo:hi] -= b[k, lo:hi, None] * X[lo + off:hi + off]
    rel = torch.linalg.norm(R, dim=0) / torch.linalg.norm(B, dim=0)
    assert float(rel.max()) < 1e-13
