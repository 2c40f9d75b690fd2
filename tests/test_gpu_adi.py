"""GPU parity of the fused ADI half-steps (explicit second difference across
systems + shared tridiagonal solve) against the oracle, both axes, forward
and adjoint; the autograd wrapper against finite differences.  Every check
bounds the grid's relative L2 error and the relative max-norm error of every
grid line solved as one system (tests.dense.parity): FP64 1e-12, FP32 the
bound of one FP32 solve (tests.dense.tol32) for the explicit operator and
for the solve of each half-step.  The adjoint half-step S^{-T} (I + r d2) u
is checked against the oracle's transposed half-step
(oracle.adi_halfstep_bands) with a non-symmetric S, where it differs from
the forward map, on grids whose lines run row-partitioned, and on the full
4096^2 grid."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, rel_l2, second_difference, tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    return m


def _lines(axis):
    """The systems of a half-step as a layout of the (ny, nx) grid: grid rows
    for axis 0 (solved along x), grid columns for axis 1."""
    return "strided" if axis == 0 else "interleaved"


def _factor(bs, n, r):
    return bs.Factor(synth.adi_bands(n, r))


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("ny,nx", [(1, 1), (3, 5), (33, 17), (100, 64), (70, 257), (1000, 777), (777, 1000)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_adi_halfstep(bs, axis, ny, nx, dtype):
    r = 0.5
    n = nx if axis == 0 else ny
    if n < 2:
        pytest.skip("a tridiagonal handle needs N >= 2")
    rng = np.random.default_rng(ny * 1000 + nx)
    u = rng.uniform(-1, 1, (ny, nx))
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
    f = _factor(bs, n, r)
    out = bs.adi_halfstep(f, torch.tensor(u, dtype=dtype, device="cuda"), r, axis)
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == torch.float64 else tol32(synth.adi_bands(n, r), ops=2)
    parity(out.double().cpu().numpy(), oracle.adi_halfstep(u, r, axis), tol, _lines(axis))


@pytest.mark.parametrize("axis", [0, 1])
def test_adi_adjoint_is_transpose(bs, axis):
    """<out(u), g> == <u, adjoint(g)> and the adjoint against the dense
    transpose on a small rectangular grid."""
    ny, nx, r = 9, 13, 0.5
    n = nx if axis == 0 else ny
    f = _factor(bs, n, r)
    rng = np.random.default_rng(axis)
    u = rng.uniform(-1, 1, (ny, nx))
    g = rng.uniform(-1, 1, (ny, nx))
    out = bs.adi_halfstep(f, torch.tensor(u, device="cuda"), r, axis).cpu().numpy()
    adj = bs.adi_halfstep(f, torch.tensor(g, device="cuda"), r, axis, adjoint=True).cpu().numpy()
    assert abs(np.sum(out * g) - np.sum(u * adj)) < 1e-12 * (1 + abs(np.sum(out * g)))
    Dx, Dy = second_difference(nx), second_difference(ny)
    I = np.eye(nx * ny)
    Kxx, Kyy = np.kron(np.eye(ny), Dx), np.kron(Dy, np.eye(nx))
    T = np.linalg.solve(I - r * Kxx, I + r * Kyy) if axis == 0 else np.linalg.solve(I - r * Kyy, I + r * Kxx)
    parity(adj, (T.T @ g.ravel()).reshape(ny, nx), 1e-12, _lines(axis))


def test_adi_full_grid_4096(bs):
    """The 4096 x 4096 heat-equation grid, r = 0.5, u ~ U(-1,1) (seed 0): one
    full Peaceman-Rachford step (x-implicit then y-implicit) in FP64 against
    the oracle on the whole grid, and in FP32 within the bound of four FP32
    operations (two explicit operators, two solves)."""
    n, r = 4096, 0.5
    f = _factor(bs, n, r)
    u = synth.adi_field(n, 0, "cuda")
    half = bs.adi_halfstep(f, u, r, 0)
    full = bs.adi_halfstep(f, half, r, 1)
    u32 = u.float()
    full32 = bs.adi_halfstep(f, bs.adi_halfstep(f, u32, r, 0), r, 1)
    torch.cuda.synchronize()
    uh = u.cpu().numpy()
    ref = oracle.adi_halfstep(oracle.adi_halfstep(uh, r, 0), r, 1)
    parity(full.cpu().numpy(), ref, 1e-12, _lines(1))
    ref32 = oracle.adi_halfstep(oracle.adi_halfstep(u32.double().cpu().numpy(), r, 0), r, 1)
    parity(full32.double().cpu().numpy(), ref32, tol32(synth.adi_bands(n, r), ops=4), _lines(1))


def test_adi_autograd_finite_differences(bs):
    """Gradient of L = sum(W * step(u)) for a full ADI step (both half-steps)
    against central differences in FP64, along a random direction."""
    ny, nx, r = 12, 10, 0.5
    fx, fy = _factor(bs, nx, r), _factor(bs, ny, r)
    rng = np.random.default_rng(3)
    u0 = rng.uniform(-1, 1, (ny, nx))
    W = rng.uniform(-1, 1, (ny, nx))
    du = rng.uniform(-1, 1, (ny, nx))
    u = torch.tensor(u0, device="cuda", requires_grad=True)
    out = bs.ADIHalfStepFn.apply(bs.ADIHalfStepFn.apply(u, fx, r, 0), fy, r, 1)
    (out * torch.tensor(W, device="cuda")).sum().backward()
    analytic = float((u.grad.cpu().numpy() * du).sum())

    def L(t):
        v = oracle.adi_halfstep(oracle.adi_halfstep(u0 + t * du, r, 0), r, 1)
        return float(np.sum(W * v))

    eps = 1e-6
    fd = (L(eps) - L(-eps)) / (2 * eps)
    assert abs(analytic - fd) < 1e-7 * (1 + abs(fd))


@pytest.mark.parametrize("partition", [2, 1])
@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_adi_nonsymmetric_operator_vs_oracle(bs, axis, adjoint, partition, dtype):
    """A non-symmetric diagonally dominant implicit operator S on a 400 x 1024
    grid (lines of 1024 or 400 rows: row-partitioned with partition = 2),
    forward S^{-1} E u and adjoint S^{-T} E u against the oracle per line."""
    ny, nx, r = 400, 1024, 0.5
    n = nx if axis == 0 else ny
    rng = np.random.default_rng(n + axis)
    bands = synth.random_tri_bands(n, rng)
    u = rng.uniform(-1, 1, (ny, nx))
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
    f = bs.Factor(bands)
    bs.set_option(bs.OPT_PARTITION, partition)
    try:
        out = bs.adi_halfstep(f, torch.tensor(u, dtype=dtype, device="cuda"), r, axis, adjoint=adjoint)
        torch.cuda.synchronize()
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
    ref = oracle.adi_halfstep_bands(u, r, bands, axis, transpose=adjoint)
    out = out.double().cpu().numpy()
    parity(out, ref, 1e-12 if dtype == torch.float64 else tol32(bands, ops=2), _lines(axis))
    if adjoint:  # really the transpose: the forward map differs
        assert rel_l2(oracle.adi_halfstep_bands(u, r, bands, axis), ref) > 1e-3


@pytest.mark.parametrize("axis", [0, 1])
def test_adi_adjoint_full_grid_4096(bs, axis):
    """The 4096 x 4096 heat-equation grid, r = 0.5: the adjoint half-step
    (row-partitioned, as every 4096-line launch runs) in FP64 against the
    oracle's transposed half-step on the whole grid, per line."""
    n, r = 4096, 0.5
    bands = synth.adi_bands(n, r)
    f = bs.Factor(bands)
    u = synth.adi_field(n, 1, "cuda")
    adj = bs.adi_halfstep(f, u, r, axis, adjoint=True)
    torch.cuda.synchronize()
    ref = oracle.adi_halfstep_bands(u.cpu().numpy(), r, bands, axis, transpose=True)
    parity(adj.cpu().numpy(), ref, 1e-12, _lines(axis))



@pytest.mark.parametrize("case", ["huge", "tiny", "zeros"])
def test_adi_pair_kernel_redo(bs, case):
    """The FP64 y-implicit half-step runs in FP32 pairs; a warp whose columns
    hold an input outside the pairs' range ([2^-72, 2^91), zero allowed)
    redoes them in FP64.  Columns with 2^95, 2^-80 or zeros beside ordinary
    ones, row-partitioned (1024 rows: 4 blocks) and not (400 rows), against
    the oracle per line.  (r = 0.3: with r = 0.5 the stencil's centre weight
    1 - 2r is zero, and the oracle's unfused u + r (left - 2u + right) loses
    a huge column's neighbour terms to cancellation, which the fused form
    keeps.)"""
    for ny, nx in ((1024, 300), (400, 300)):
        r = 0.3
        rng = np.random.default_rng(ny + len(case))
        u = rng.uniform(-1, 1, (ny, nx))
        if case == "huge":
            u[:, 37] *= 2.0 ** 95
        elif case == "tiny":
            u[100:200, 70] = 2.0 ** -80
        else:
            u[:, 5:40] = 0.0
            u[10:20, :] = 0.0
        f = _factor(bs, ny, r)
        out = bs.adi_halfstep(f, torch.tensor(u, device="cuda"), r, 1)
        torch.cuda.synchronize()
        parity(out.cpu().numpy(), oracle.adi_halfstep(u, r, 1), 1e-12, _lines(1))
