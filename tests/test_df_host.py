"""CPU tests of the FP32-pair arithmetic of the FP64-accurate pair sweeps
(paper_1909_04539_gb300/csrc/df_math.cuh), built for the host with g++ (IEEE
single precision, no FMA contraction) through tests/host/df_host.cpp:

- split: h is the FP64 value truncated to 24 significant bits, l the FP32
  rounding of the rest (|x - h - l| <= 2^-48 |x|), the range flag exactly on
  zero and 2^-72 <= |x| < 2^101;
- combine: within one FP64 ulp of h + l, including a power-of-two h with l
  of the other sign (the binade below) and signed zeros;
- TwoSum: exact for arbitrary operands (checked in exact rational arithmetic);
- the two sweeps run as the kernel runs them, on tridiagonal and
  pentadiagonal systems, primal and adjoint, against the FP64 oracle per
  system at 1e-13 (the library's tolerance for this path is 1e-12);
- the periodic (cyclic) tridiagonal solve as the periodic pair sweeps run
  it -- the Sherman-Morrison sum and correction (Sec. 3.3) in pairs with the
  weights scaled by a power of two -- primal and adjoint, against the
  oracle's periodic solve per system at 1e-13;
- Crank-Nicolson steps as the fused pair kernel runs them (the explicit
  side 2I - A formed in pairs from the rows, then the pair solve; periodic:
  wrapped and with the Sherman-Morrison terms), banded tri / penta and
  cyclic tri, against the oracle's steps per system at 1e-13.
"""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests.dense import sys_rel_err

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host", "df_host.cpp")
OUT = os.path.join(HERE, "host", "_build", "libdfhost.so")


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    hdr = os.path.join(HERE, "..", "paper_1909_04539_gb300", "csrc", "df_math.cuh")
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(SRC), os.path.getmtime(hdr)):
        tmp = OUT + f".{os.getpid()}.tmp"
        subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC", "-o", tmp, SRC],
                       check=True)
        os.replace(tmp, OUT)
    L = ctypes.CDLL(OUT)
    P = np.ctypeslib.ndpointer
    L.df_split.argtypes = [P(np.float64), P(np.float32), P(np.float32), P(np.int32), ctypes.c_long]
    L.df_combine.argtypes = [P(np.float32), P(np.float32), P(np.float64), ctypes.c_long]
    L.df_two_sum.argtypes = [P(np.float32), P(np.float32), P(np.float32), P(np.float32), ctypes.c_long]
    L.df_split_fast.argtypes = [P(np.float64), P(np.float32), P(np.float32), P(np.int32), ctypes.c_long]
    L.df_combine_fast.argtypes = [P(np.float32), P(np.float32), P(np.float64), P(np.int32), ctypes.c_long]
    d = P(np.float64)
    L.df_sweep.argtypes = [d, d, d, d, d, d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long, d, d]
    L.df_sweep_periodic.argtypes = [d, d, d, d, ctypes.c_int, ctypes.c_int, P(np.float32), ctypes.c_long,
                                    ctypes.c_long, ctypes.c_long, d, d]
    L.df_cn_step.argtypes = [d, ctypes.c_int, ctypes.c_int, d, d, d, d, d, P(np.float32), ctypes.c_long,
                             ctypes.c_long, ctypes.c_long, d, d]
    return L


def _split(L, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = np.empty(x.size, np.float32)
    lo = np.empty(x.size, np.float32)
    ok = np.empty(x.size, np.int32)
    L.df_split(x, h, lo, ok, x.size)
    return h, lo, ok.astype(bool)


def test_split_truncates_and_flags_range(lib):
    rng = np.random.default_rng(0)
    x = rng.uniform(1, 2, 200000) * np.ldexp(1.0, rng.integers(-72, 101, 200000)) * rng.choice([-1, 1], 200000)
    h, lo, ok = _split(lib, x)
    assert ok.all()
    # h: x with its low 29 mantissa bits cleared (truncation to 24 bits)
    trunc = (x.view(np.uint64) & ~np.uint64((1 << 29) - 1)).view(np.float64)
    assert np.array_equal(h.astype(np.float64), trunc)
    rest = x - trunc  # exact (Sterbenz)
    assert np.all(np.abs(lo.astype(np.float64) - rest) <= np.abs(rest) * 2.0 ** -24)
    assert np.all(np.abs(h.astype(np.float64) + lo.astype(np.float64) - x) <= np.abs(x) * 2.0 ** -48)
    nz = lo != 0
    assert np.all(np.abs(lo[nz]) >= np.finfo(np.float32).tiny)  # l is a normal number


def test_split_range_edges(lib):
    lo_edge, hi_edge = np.ldexp(1.0, -72), np.ldexp(1.0, 101)
    vals = np.array([0.0, -0.0, lo_edge, -lo_edge, np.nextafter(lo_edge, 0), hi_edge, np.nextafter(hi_edge, 0),
                     -np.nextafter(hi_edge, 0), np.inf, -np.inf, np.nan, 5e-324, 1e-300, 1e300, 1.0])
    h, lo, ok = _split(lib, vals)
    assert ok.tolist() == [True, True, True, True, False, False, True, True, False, False, False, False, False,
                           False, True]
    assert h[0] == 0 and not np.signbit(h[0]) and lo[0] == 0
    assert h[1] == 0 and np.signbit(h[1]) and lo[1] == 0
    for i in (2, 3, 6, 7, 14):
        assert float(h[i]) + float(lo[i]) == pytest.approx(vals[i], rel=2.0 ** -47)


def _combine(L, h, lo):
    h = np.ascontiguousarray(h, np.float32)
    lo = np.ascontiguousarray(lo, np.float32)
    out = np.empty(h.size, np.float64)
    L.df_combine(h, lo, out, h.size)
    return out


def test_combine_within_one_ulp(lib):
    rng = np.random.default_rng(1)
    n = 100000
    h = (rng.uniform(1, 2, n) * np.ldexp(1.0, rng.integers(-70, 100, n)) * rng.choice([-1, 1], n)).astype(np.float32)
    ulp = np.spacing(np.abs(h)).astype(np.float64)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    # powers of two with the low part pointing either way
    p2 = np.ldexp(np.float32(1), rng.integers(-70, 100, 2000)).astype(np.float32) * rng.choice([-1, 1], 2000)
    lp = (rng.uniform(-0.5, 0.5, 2000) * np.spacing(np.abs(p2)).astype(np.float64)).astype(np.float32)
    h = np.concatenate([h, p2.astype(np.float32)])
    lo = np.concatenate([lo, lp])
    c = _combine(lib, h, lo)
    err = np.abs((c - h.astype(np.float64)) - lo.astype(np.float64))
    assert np.all(err <= np.spacing(np.abs(c)))


def test_combine_zero_and_exact_cases(lib):
    h = np.array([0.0, -0.0, 1.0, -1.0, 1.5, 2.0 ** -100], np.float32)
    lo = np.array([0.0, 0.0, -2.0 ** -30, 2.0 ** -30, 2.0 ** -26, 0.0], np.float32)
    c = _combine(lib, h, lo)
    assert c[0] == 0 and not np.signbit(c[0])
    assert c[1] == 0 and np.signbit(c[1])
    assert c[2] == 1.0 - 2.0 ** -30 and c[3] == -(1.0 - 2.0 ** -30)
    assert c[4] == 1.5 + 2.0 ** -26 and c[5] == 2.0 ** -100


def test_fast_split_agrees_and_refuses_edges(lib):
    """split_fast gives split()'s pair wherever it accepts, accepts exactly
    2^-72 <= |x| < 2^101, and refuses zeros (handled by split())."""
    rng = np.random.default_rng(7)
    n = 200000
    x = rng.uniform(1, 2, n) * np.ldexp(1.0, rng.integers(-80, 110, n)) * rng.choice([-1, 1], n)
    x = np.concatenate([x, [0.0, -0.0, np.ldexp(1.0, -72), np.nextafter(np.ldexp(1.0, -72), 0),
                            np.ldexp(1.0, 101), np.nextafter(np.ldexp(1.0, 101), 0), np.inf, np.nan, 5e-324]])
    h = np.empty(x.size, np.float32)
    lo = np.empty(x.size, np.float32)
    ok = np.empty(x.size, np.int32)
    lib.df_split_fast(x, h, lo, ok, x.size)
    ax = np.abs(x)
    want = (ax >= np.ldexp(1.0, -72)) & (ax < np.ldexp(1.0, 101))
    assert np.array_equal(ok.astype(bool), want)
    h2, lo2, ok2 = _split(lib, x)
    assert np.array_equal(h[want], h2[want]) and np.array_equal(lo[want], lo2[want])


def test_combine_fast_rounds_once(lib):
    """combine_fast is h + l rounded once to FP64 wherever combine_ok (|h| >=
    2^-70), including zero and subnormal low parts."""
    rng = np.random.default_rng(8)
    n = 100000
    h = (rng.uniform(1, 2, n) * np.ldexp(1.0, rng.integers(-75, 100, n)) * rng.choice([-1, 1], n)).astype(np.float32)
    lo = (rng.uniform(-0.5, 0.5, n) * np.spacing(np.abs(h)).astype(np.float64)).astype(np.float32)
    lo[::7] = 0.0
    lo[1::7] = np.float32(1e-40)
    out = np.empty(n)
    ok = np.empty(n, np.int32)
    lib.df_combine_fast(h, lo, out, ok, n)
    okb = ok.astype(bool)
    assert np.array_equal(okb, np.abs(h) >= np.float32(2.0 ** -70))
    exact = [Fraction(float(a)) + Fraction(float(b)) for a, b in zip(h[okb][::53], lo[okb][::53])]
    got = out[okb][::53]
    for g, e in zip(got, exact):
        assert g == float(e)  # Python rounds the exact rational once, to nearest


def test_two_sum_exact(lib):
    rng = np.random.default_rng(2)
    n = 20000
    a = (rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-40, 40, n))).astype(np.float32)
    b = (rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-40, 40, n))).astype(np.float32)
    s = np.empty(n, np.float32)
    t = np.empty(n, np.float32)
    lib.df_two_sum(a, b, s, t, n)
    for i in range(0, n, 97):
        assert Fraction(float(a[i])) + Fraction(float(b[i])) == Fraction(float(s[i])) + Fraction(float(t[i]))
    assert np.array_equal(s, (a + b).astype(np.float32))


def _plans(bands):
    """The recurrence coefficients of the primal and adjoint solves (the
    paper's Thomas / A = L R factors, Sec. 3.1 / Sec. 4.1), computed here in
    plain numpy for the test."""
    w, N = bands.shape
    z = np.zeros(N)
    if w == 3:
        a, b, c = bands
        p, ch = np.zeros(N), np.zeros(N)
        for i in range(N):
            p[i] = b[i] - (a[i] * ch[i - 1] if i else 0.0)
            ch[i] = c[i] / p[i] if i + 1 < N else 0.0
        r = 1 / p
        l1 = np.where(np.arange(N) > 0, a * r, 0.0)
        prim = (r, l1, z, np.ones(N), ch, z)
        al1 = np.concatenate([[0.0], ch[:-1]])
        au1 = np.concatenate([a[1:] * r[:-1], [0.0]])
        adj = (np.ones(N), al1, z, r, au1, z)
        return prim, adj
    a, b, c, d, e = bands
    al, be, ga, de, ep = (np.zeros(N) for _ in range(5))
    for i in range(N):
        A = a[i] if i >= 2 else 0.0
        B = b[i] if i >= 1 else 0.0
        D = d[i] if i + 1 < N else 0.0
        E = e[i] if i + 2 < N else 0.0
        ep[i] = A
        be[i] = B - A * (ga[i - 2] if i >= 2 else 0.0)
        al[i] = c[i] - A * (de[i - 2] if i >= 2 else 0.0) - be[i] * (ga[i - 1] if i >= 1 else 0.0)
        ga[i] = (D - be[i] * (de[i - 1] if i >= 1 else 0.0)) / al[i]
        de[i] = E / al[i]
    ia = 1 / al
    idx = np.arange(N)
    prim = (ia, np.where(idx >= 1, be * ia, 0.0), np.where(idx >= 2, ep * ia, 0.0), np.ones(N), ga, de)
    adj = (np.ones(N), np.concatenate([[0.0], ga[:-1]]), np.concatenate([[0.0, 0.0], de[:-2]]), ia,
           np.concatenate([be[1:] * ia[:-1], [0.0]]), np.concatenate([ep[2:] * ia[:-2], [0.0, 0.0]]))
    return prim, adj


def _sweep(L, coefs, has_s, has_t, bw, f):
    N = f.size
    x = np.empty(N)
    cs = [np.ascontiguousarray(c, np.float64) for c in coefs]
    L.df_sweep(*cs, int(has_s), int(has_t), bw, N, np.ascontiguousarray(f), x)
    return x


@pytest.mark.parametrize("width,N", [(3, 2), (3, 65), (3, 1024), (5, 4), (5, 37), (5, 512)])
def test_pair_sweeps_match_oracle(lib, width, N):
    rng = np.random.default_rng(N + width)
    bands = synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)
    M = 24
    B = rng.standard_normal((N, M)) * np.ldexp(1.0, rng.integers(-30, 30, M))
    prim, adj = _plans(bands)
    bw = width // 2
    X = np.stack([_sweep(lib, prim, True, False, bw, B[:, j]) for j in range(M)], axis=1)
    G = np.stack([_sweep(lib, adj, False, True, bw, B[:, j]) for j in range(M)], axis=1)
    assert sys_rel_err(X, oracle.solve(bands, B)) < 1e-13
    assert sys_rel_err(G, oracle.solve_adjoint(bands, B)) < 1e-13


@pytest.mark.parametrize("kind", ["hyper", "spline", "adi", "stiff"])
def test_pair_sweep_structured_matrices(lib, kind):
    """The benchmark matrix I + 0.1 D4 clamped (N = 512), the spline and ADI
    tridiagonal matrices (N = 1024) and stiff hyperdiffusion I + 1000 D4
    (N = 512, condition number ~1.6e4: the pairs' error grows with it, as
    FP64's does)."""
    bands = {"hyper": lambda: synth.clamped_hyperdiffusion_bands(512, 0.1), "spline": lambda: synth.spline_bands(1024),
             "adi": lambda: synth.adi_bands(1024, 0.5),
             "stiff": lambda: synth.toeplitz_bands(512, (1e3, -4e3, 1 + 6e3, -4e3, 1e3))}[kind]()
    rng = np.random.default_rng(5)
    N = bands.shape[1]
    B = rng.standard_normal((N, 16))
    prim, adj = _plans(bands)
    bw = bands.shape[0] // 2
    X = np.stack([_sweep(lib, prim, True, False, bw, B[:, j]) for j in range(16)], axis=1)
    G = np.stack([_sweep(lib, adj, False, True, bw, B[:, j]) for j in range(16)], axis=1)
    tol = 1e-12 if kind == "stiff" else 1e-13
    assert sys_rel_err(X, oracle.solve(bands, B)) < tol
    assert sys_rel_err(G, oracle.solve_adjoint(bands, B)) < tol


def _periodic_setup(bands):
    """The corner-free matrix A' = A - u v^T of a cyclic tridiagonal A
    (gamma = -b_1, u = (gamma, 0, .., 0, c_N), v = (1, 0, .., 0, a_1 /
    gamma), Sec. 3.3), its recurrence coefficients, and the Sherman-Morrison
    weights of the primal and adjoint solves: z = A'^{-1} u, q = A'^{-T} v,
    primal (pw, pc) = (q, z / (1 + v.z)), adjoint (z, q / (1 + v.z));
    entries below 2^-60 max / N dropped, the middle rows where both vanish
    recorded as [lo, hi)."""
    a, b, c = (np.asarray(r, dtype=np.float64) for r in bands)
    N = a.size
    gam = -b[0]
    v_last = a[0] / gam
    mod = np.stack([np.where(np.arange(N) > 0, a, 0.0), b.copy(), np.where(np.arange(N) < N - 1, c, 0.0)])
    mod[1, 0] = b[0] - gam
    mod[1, N - 1] = b[N - 1] - c[N - 1] * v_last
    u = np.zeros(N)
    u[0], u[N - 1] = gam, c[N - 1]
    v = np.zeros(N)
    v[0], v[N - 1] = 1.0, v_last
    z = oracle.solve(mod, u[:, None])[:, 0]
    q = oracle.solve_adjoint(mod, v[:, None])[:, 0]
    den = 1.0 + z[0] + v_last * z[N - 1]
    tq, tz = np.abs(q).max() * 2.0 ** -60 / N, np.abs(z).max() * 2.0 ** -60 / N
    keep = (np.abs(q) > tq) | (np.abs(z) > tz)
    q, z = np.where(keep, q, 0.0), np.where(keep, z, 0.0)
    lo = max([i + 1 for i in range(N // 2) if keep[i]], default=0)
    hi = min([i for i in range(N // 2, N) if keep[i]], default=N)
    lo = min(lo, hi)
    prim, adj = _plans(mod)
    return (prim, (q, z / den)), (adj, (z, q / den)), lo, hi


def _scaled_pairs(pw, pc):
    """(pw', pc') = (2^k pw, 2^-k pc), max |pw'| in [1, 2), as (hi, lo) float
    pairs per row: 4 N floats."""
    k = 1 - int(np.frexp(np.abs(pw).max())[1])
    w, cc = np.ldexp(pw, k), np.ldexp(pc, -k)
    wh, ch = w.astype(np.float32), cc.astype(np.float32)
    wl, cl = (w - wh).astype(np.float32), (cc - ch).astype(np.float32)
    return np.ascontiguousarray(np.stack([wh, wl, ch, cl], axis=1).ravel())


def _periodic_sweep(L, coefs, weights, lo, hi, has_s, has_t, f):
    s, l1, _, t, u1, _ = (np.ascontiguousarray(c, np.float64) for c in coefs)
    x = np.empty(f.size)
    L.df_sweep_periodic(s, l1, t, u1, int(has_s), int(has_t), _scaled_pairs(*weights), lo, hi, f.size,
                        np.ascontiguousarray(f), x)
    return x


PERIODIC = {
    "random_N3": lambda: synth.random_periodic_bands(3, np.random.default_rng(1)),
    "random_N5": lambda: synth.random_periodic_bands(5, np.random.default_rng(2)),
    "random_N37": lambda: synth.random_periodic_bands(37, np.random.default_rng(3)),
    "random_N300": lambda: synth.random_periodic_bands(300, np.random.default_rng(4)),
    "diffusion_N1024": lambda: synth.periodic_toeplitz_bands(1024, (-0.5, 2.0, -0.5)),
    "spline_N1024": lambda: synth.periodic_toeplitz_bands(1024, (1 / 6, 4 / 6, 1 / 6)),
    "weak_N512": lambda: synth.periodic_toeplitz_bands(512, (-1.0, 2.05, -1.0)),
    "nonsymmetric_N64": lambda: synth.periodic_toeplitz_bands(64, (0.3, 2.0, -0.6)),
}


@pytest.mark.parametrize("case", sorted(PERIODIC))
def test_periodic_pair_sweeps_match_oracle(lib, case):
    bands = PERIODIC[case]()
    N = bands.shape[1]
    rng = np.random.default_rng(N)
    M = 16
    B = rng.standard_normal((N, M)) * np.ldexp(1.0, rng.integers(-30, 30, M))
    (prim, pw), (adj, aw), lo, hi = _periodic_setup(bands)
    X = np.stack([_periodic_sweep(lib, prim, pw, lo, hi, True, False, B[:, j]) for j in range(M)], axis=1)
    G = np.stack([_periodic_sweep(lib, adj, aw, lo, hi, False, True, B[:, j]) for j in range(M)], axis=1)
    assert sys_rel_err(X, oracle.periodic_tri_solve_bands(bands, B)) < 1e-13
    assert sys_rel_err(G, oracle.periodic_solve_adjoint(bands, B)) < 1e-13


def _cn_pairs(L, bands, periodic, C0, steps):
    """`steps` Crank-Nicolson steps of every column of C0 in pair arithmetic."""
    width, N = bands.shape
    b = np.ascontiguousarray(bands, dtype=np.float64)
    if periodic:
        (prim, pw), _, lo, hi = _periodic_setup(bands)
        pq = _scaled_pairs(*pw)
    else:
        prim, _ = _plans(bands)
        pq, lo, hi = np.zeros(4 * N, np.float32), 0, N
    s, l1, l2, _, u1, u2 = (np.ascontiguousarray(c, np.float64) for c in prim)
    C = np.array(C0, dtype=np.float64)
    for _ in range(steps):
        for j in range(C.shape[1]):
            x = np.empty(N)
            L.df_cn_step(b, width, int(periodic), s, l1, l2, u1, u2, pq, lo, hi, N, np.ascontiguousarray(C[:, j]), x)
            C[:, j] = x
    return C


CN = {
    "hyperdiffusion_N512": (lambda: synth.toeplitz_bands(512, (0.1, -0.4, 1.6, -0.4, 0.1)), False),
    "clamped_hyper_N64": (lambda: synth.clamped_hyperdiffusion_bands(64, 0.3), False),
    "random_tri_N100": (lambda: synth.random_tri_bands(100, np.random.default_rng(7)), False),
    "periodic_diffusion_N1024": (lambda: synth.periodic_toeplitz_bands(1024, (-0.5, 2.0, -0.5)), True),
    "periodic_diffusion_N3": (lambda: synth.periodic_toeplitz_bands(3, (-0.3, 1.6, -0.3)), True),
    "periodic_random_N40": (lambda: synth.random_periodic_bands(40, np.random.default_rng(8)), True),
}


@pytest.mark.parametrize("case", sorted(CN))
def test_cn_pair_steps_match_oracle(lib, case):
    make, periodic = CN[case]
    bands = make()
    N = bands.shape[1]
    C0 = np.random.default_rng(N + 1).uniform(-1, 1, (N, 6))
    got = _cn_pairs(lib, bands, periodic, C0, 3)
    ref = oracle.cn_steps(bands, C0, 3, periodic=periodic)
    # per system, relative to its starting values: the steps damp most
    # modes (the cyclic N = 3 case keeps only the mean), so the result can
    # be far smaller than the values whose rounding it carries
    err = np.abs(got - ref).max(axis=0) / np.abs(C0).max(axis=0)
    assert err.max() < 1e-13, err.max()
