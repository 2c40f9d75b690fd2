"""CPU model of the arithmetic of the mixed-precision solve's factor mode
(paper_1909_04539_gb300/csrc/refine_math.cuh, frefine_pass1/2): FP32 data,
FP32 sweeps, one refinement of each triangular sweep with a residual taken to
FP64 accuracy in FP32 arithmetic, FP64 result.  The kernel forms each sweep
as ((p - q2) - q1) with q_k the rounded products and both differences as
TwoSums, so the residual is the sum of the errors the sweep already holds:

  forward  rho   = cc + e1 + e2 - eq1 - eq2 - l1_lo w1 - l2_lo w2,
           cc    = s b - fl(s_hi b) to FP64 accuracy;
  backward sigma = g1 + g2 + g3 - eq1 - eq2 - u1_lo x1 - u2_lo x2
           (x = ((w - q2) - q1) + delta, three TwoSums).

This model runs those operations in numpy FP32 (one system per column; an
FMA is the exact FP64 product plus one rounding to FP32) and checks the
result against the FP64 oracle per system.  It pins the method: one step
reaches FP64 accuracy on the benchmark matrices, a stiff matrix's single
step does not (so more steps are needed there, as the library's
refine_steps provide); the GPU parity tests check the kernel itself.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.dense import sys_rel_err
from tests.test_df_host import _plans

f32 = np.float32


def _fma(a, b, c):
    return (a.astype(np.float64) * b + c).astype(f32)


def _two_diff(a, b):
    """a - b = s + e exactly (Knuth's TwoSum on -b)."""
    s = a - b
    bv = s - a
    return s, (a - (s - bv)) + (-b - bv)


def _split(c):
    h = c.astype(f32)
    return h, (c - h.astype(np.float64)).astype(f32)


def _model_solve(prim, bw, B32):
    """Both passes for every column of B32 (N x M, float32); returns X."""
    s, l1, l2, _, u1, u2 = (np.asarray(c, dtype=np.float64) for c in prim)
    N, M = B32.shape
    (sh, sl), (l1h, l1l), (l2h, l2l) = _split(s), _split(l1), _split(l2)
    (u1h, u1l), (u2h, u2l) = _split(u1), _split(u2)
    z = np.zeros(M, f32)
    w, dl = np.zeros((N, M), f32), np.zeros((N, M), f32)
    w1 = w2 = d1 = d2 = z
    for i in range(N):
        b = B32[i]
        p = b * sh[i]
        r = _fma(np.full(M, sl[i]), b, _fma(np.full(M, sh[i]), b, -p))
        x = p
        if bw == 2:
            q2 = l2h[i] * w2
            r = r - _fma(np.full(M, l2h[i]), w2, -q2)
            r = _fma(np.full(M, -l2l[i]), w2, r)
            x, e = _two_diff(p, q2)
            r = r + e
        q1 = l1h[i] * w1
        r = r - _fma(np.full(M, l1h[i]), w1, -q1)
        r = _fma(np.full(M, -l1l[i]), w1, r)
        y, e = _two_diff(x, q1)
        rho = r + e
        w[i] = y
        w2, w1 = w1, y
        d = rho
        if bw == 2:
            d = _fma(np.full(M, -l2h[i]), d2, d)
        d = _fma(np.full(M, -l1h[i]), d1, d)
        dl[i] = d
        d2, d1 = d1, d
    X = np.zeros((N, M))
    x1 = x2 = e1 = e2 = z
    for i in range(N - 1, -1, -1):
        a, r = w[i], np.zeros(M, f32)
        if bw == 2:
            q2 = u2h[i] * x2
            r = _fma(np.full(M, -u2l[i]), x2, -_fma(np.full(M, u2h[i]), x2, -q2))
            a, g = _two_diff(w[i], q2)
            r = r + g
        q1 = u1h[i] * x1
        r = r - _fma(np.full(M, u1h[i]), x1, -q1)
        r = _fma(np.full(M, -u1l[i]), x1, r)
        a2, g = _two_diff(a, q1)
        r = r + g
        v, g = _two_diff(a2, -dl[i])
        sig = r + g
        x2, x1 = x1, v
        ev = sig
        if bw == 2:
            ev = _fma(np.full(M, -u2h[i]), e2, ev)
        ev = _fma(np.full(M, -u1h[i]), e1, ev)
        e2, e1 = e1, ev
        X[i] = v.astype(np.float64) + ev.astype(np.float64)
    return X


def _fp32_plain(prim, bw, B32):
    """The FP32 solve alone (no refinement), for contrast."""
    s, l1, l2, _, u1, u2 = (np.asarray(c, dtype=np.float64).astype(f32) for c in prim)
    N, M = B32.shape
    w = np.zeros((N, M), f32)
    for i in range(N):
        v = B32[i] * s[i]
        if bw == 2 and i >= 2:
            v = _fma(np.full(M, -l2[i]), w[i - 2], v)
        if i >= 1:
            v = _fma(np.full(M, -l1[i]), w[i - 1], v)
        w[i] = v
    x = np.zeros((N, M), f32)
    for i in range(N - 1, -1, -1):
        v = w[i]
        if bw == 2 and i + 2 < N:
            v = _fma(np.full(M, -u2[i]), x[i + 2], v)
        if i + 1 < N:
            v = _fma(np.full(M, -u1[i]), x[i + 1], v)
        x[i] = v
    return x.astype(np.float64)


CASES = {
    "penta_benchmark": lambda: synth.clamped_hyperdiffusion_bands(512, 0.1),
    "tri_spline": lambda: synth.spline_bands(1024),
    "tri_random": lambda: synth.random_tri_bands(257, np.random.default_rng(3)),
    "penta_random": lambda: synth.random_penta_bands(130, np.random.default_rng(4)),
    "tri_adi": lambda: synth.adi_bands(600, 0.5),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_one_refinement_step_reaches_fp64_accuracy(case):
    bands = CASES[case]()
    N = bands.shape[1]
    B32 = np.random.default_rng(N).uniform(-1, 1, (N, 48)).astype(f32)
    B = B32.astype(np.float64)
    prim, _ = _plans(bands)
    ref = oracle.solve(bands, B)
    err = sys_rel_err(_model_solve(prim, bands.shape[0] // 2, B32), ref)
    assert err < 5e-14, err
    # the FP32 solve it refines is ~1e8 times less accurate
    assert sys_rel_err(_fp32_plain(prim, bands.shape[0] // 2, B32), ref) > 1e-9


def test_stiff_matrix_needs_more_than_one_step():
    """I + 4000 D4 (condition number ~6e4): one step leaves an error well
    above the FP64 target (the library's refine_steps take it below)."""
    bands = synth.toeplitz_bands(256, (4e3, -1.6e4, 1 + 2.4e4, -1.6e4, 4e3))
    N = bands.shape[1]
    B32 = np.random.default_rng(9).uniform(-1, 1, (N, 32)).astype(f32)
    prim, _ = _plans(bands)
    err = sys_rel_err(_model_solve(prim, 2, B32), oracle.solve(bands, B32.astype(np.float64)))
    assert 1e-12 < err < 1e-8, err


def test_zero_and_scaled_systems():
    """A zero system stays exactly zero; scaling a system by a power of two
    scales the result exactly (the model's FP32 operations stay normal)."""
    bands = synth.clamped_hyperdiffusion_bands(64, 0.1)
    rng = np.random.default_rng(5)
    B32 = rng.uniform(-1, 1, (64, 3)).astype(f32)
    B32[:, 0] = 0
    B32[:, 2] = B32[:, 1] * f32(2.0 ** 20)
    prim, _ = _plans(bands)
    X = _model_solve(prim, 2, B32)
    assert np.all(X[:, 0] == 0.0)
    assert np.array_equal(X[:, 2], X[:, 1] * 2.0 ** 20)
