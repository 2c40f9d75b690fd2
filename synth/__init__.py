"""Seeded synthetic inputs shared by the tests, the benchmark, the smoke check
and the oracle.  This module holds none of the solver arithmetic: it only
draws band coefficients and right-hand sides with the shapes, value
distributions and structure of the workloads below, so that both the CUDA
path and the oracle can be fed the very same numbers.

Workloads (sizes as stated; the paper used cuSten-generated Crank-Nicolson
right-hand sides on unspecified data, which these stand in for):

* ``random_tri``: tridiagonal, a, c ~ U(-1, 1), b = |a| + |c| + U(1, 2)
  (strictly diagonally dominant); default N = 64, M = 1024.
* ``clamped_hyperdiffusion_penta``: A = I + s D4 with the [1, -4, 6, -4, 1]
  stencil, s = 0.1, first and last two rows identity; N = 512, M = 65536,
  RHS ~ N(0, 1).
* ``spline_tri``: natural cubic-spline matrix [1, 4, 1]/6, N = 1024,
  M = 2**20, RHS = second differences of sums of 8 random sinusoids.
* ``adi``: 4096 x 4096 heat-equation field u ~ U(-1, 1), r = 0.5.
* ``serving``: 256 resident LHS and a Poisson request stream.

Host draws use ``numpy.random.default_rng(seed)`` (PCG64) in the order the
docstrings give.  Large right-hand sides are drawn with
``torch.Generator(device).manual_seed(seed)`` directly on the target device;
a CPU and a CUDA generator give different (equally valid) streams, so every
comparison copies the very tensor the GPU used back to the host.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# Band matrices (host, FP64).  Bands are (width, N): tri (a, b, c) with b the
# diagonal; penta (a, b, c, d, e) with c the diagonal.  Entries outside the
# matrix are stored as 0.
# --------------------------------------------------------------------------


def random_tri_bands(N: int, rng: np.random.Generator) -> np.ndarray:
    """Draw a, c ~ U(-1,1) then u ~ U(1,2) for all N rows (in that order), zero
    a_1 and c_N, and set b = |a| + |c| + u."""
    a = rng.uniform(-1.0, 1.0, N)
    c = rng.uniform(-1.0, 1.0, N)
    u = rng.uniform(1.0, 2.0, N)
    a[0] = 0.0
    c[N - 1] = 0.0
    b = np.abs(a) + np.abs(c) + u
    return np.stack([a, b, c])


def random_periodic_bands(N: int, rng: np.random.Generator) -> np.ndarray:
    """Periodic tridiagonal bands: a, c ~ U(-1,1) then u ~ U(1,2) for all N
    rows, b = |a| + |c| + u; a_1 and c_N are kept (they are the corner
    entries of the cyclic matrix)."""
    a = rng.uniform(-1.0, 1.0, N)
    c = rng.uniform(-1.0, 1.0, N)
    u = rng.uniform(1.0, 2.0, N)
    b = np.abs(a) + np.abs(c) + u
    return np.stack([a, b, c])


def random_penta_bands(N: int, rng: np.random.Generator) -> np.ndarray:
    """Off-diagonals a, b, d, e ~ U(-1,1), then u ~ U(1,2); outside entries
    zeroed; diagonal c = sum of |off-diagonals| + u (strictly dominant)."""
    a = rng.uniform(-1.0, 1.0, N)
    b = rng.uniform(-1.0, 1.0, N)
    d = rng.uniform(-1.0, 1.0, N)
    e = rng.uniform(-1.0, 1.0, N)
    u = rng.uniform(1.0, 2.0, N)
    a[:2] = 0.0
    b[0] = 0.0
    d[N - 1] = 0.0
    e[N - 2:] = 0.0
    c = np.abs(a) + np.abs(b) + np.abs(d) + np.abs(e) + u
    return np.stack([a, b, c, d, e])


def uniform_penta_bands(N: int, rng: np.random.Generator, a: float = 0.25) -> np.ndarray:
    """Pentadiagonal bands whose outermost sub-diagonal is the constant a (the
    uniform case of Sec. 4.1); b, d, e ~ U(-1,1) and u ~ U(1,2) per row in that
    order, outside entries zeroed, diagonal c = sum of |off-diagonals| + u."""
    b = rng.uniform(-1.0, 1.0, N)
    d = rng.uniform(-1.0, 1.0, N)
    e = rng.uniform(-1.0, 1.0, N)
    u = rng.uniform(1.0, 2.0, N)
    av = np.full(N, float(a))
    av[:2] = 0.0
    b[0] = 0.0
    d[N - 1] = 0.0
    e[N - 2:] = 0.0
    c = np.abs(av) + np.abs(b) + np.abs(d) + np.abs(e) + u
    return np.stack([av, b, c, d, e])


def toeplitz_bands(N: int, diagonals) -> np.ndarray:
    """Constant bands (e.g. (-r, 1+2r, -r)), outside entries zeroed."""
    w = len(diagonals)
    h = w // 2
    out = np.zeros((w, N))
    for k, v in enumerate(diagonals):
        out[k, :] = v
        off = k - h
        if off < 0:
            out[k, : -off] = 0.0
        elif off > 0:
            out[k, N - off:] = 0.0
    return out


def periodic_toeplitz_bands(N: int, diagonals) -> np.ndarray:
    """Constant cyclic tridiagonal bands (a, b, c) on every row, a_1 and c_N
    included (they are the corner entries of the periodic matrix)."""
    a, b, c = diagonals
    return np.stack([np.full(N, float(a)), np.full(N, float(b)), np.full(N, float(c))])


def clamped_hyperdiffusion_bands(N: int = 512, s: float = 0.1, clamped: bool = True) -> np.ndarray:
    """A = I + s D4, D4 the [1, -4, 6, -4, 1] stencil.  With ``clamped`` the
    first and last two rows are identity rows (Dirichlet-clamped values);
    otherwise the stencil is truncated at the ends."""
    bands = toeplitz_bands(N, (s, -4 * s, 1 + 6 * s, -4 * s, s))
    if clamped:
        for i in (0, 1, N - 2, N - 1):
            bands[:, i] = 0.0
            bands[2, i] = 1.0
    return bands


def spline_bands(N: int = 1024) -> np.ndarray:
    """Natural cubic-spline second-derivative matrix [1, 4, 1]/6 (unit
    spacing); rows 1 and N have two entries."""
    return toeplitz_bands(N, (1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0))


def adi_bands(N: int = 4096, r: float = 0.5) -> np.ndarray:
    """I - r delta^2 with homogeneous Dirichlet ends: (-r, 1 + 2r, -r)."""
    return toeplitz_bands(N, (-r, 1 + 2 * r, -r))


# --------------------------------------------------------------------------
# Right-hand sides
# --------------------------------------------------------------------------


def uniform_rhs_host(N: int, M: int, rng: np.random.Generator) -> np.ndarray:
    """(N, M) interleaved block ~ U(-1, 1)."""
    return rng.uniform(-1.0, 1.0, (N, M))


def random_tri_case(N: int = 64, M: int = 1024, seed: int = 0):
    """Bands then RHS from one generator, in that order."""
    rng = np.random.default_rng(seed)
    bands = random_tri_bands(N, rng)
    B = uniform_rhs_host(N, M, rng)
    return bands, B


def random_penta_case(N: int, M: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    bands = random_penta_bands(N, rng)
    B = uniform_rhs_host(N, M, rng)
    return bands, B


def normal_rhs(N: int, M: int, seed: int, device, dtype=None):
    """(N, M) block ~ N(0, 1) drawn on ``device`` (torch)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn((N, M), generator=g, device=device, dtype=dtype or torch.float64)


def uniform_rhs(N: int, M: int, seed: int, device, dtype=None):
    """(N, M) block ~ U(-1, 1) drawn on ``device`` (torch)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.rand((N, M), generator=g, device=device, dtype=dtype or torch.float64)
    return x.mul_(2.0).sub_(1.0)


def spline_rhs(N: int, M: int, seed: int, device, n_modes: int = 8, chunk: int = 1 << 16):
    """Second differences of random smooth signals, one signal per system.

    For system j: y(t) = sum_k A_k sin(2 pi f_k t / N + phi_k), t = 0..N+1,
    A_k ~ U(-1,1), f_k ~ U(0, N/8) (continuous), phi_k ~ U(0, 2 pi), the three
    (M, n_modes) parameter blocks drawn in that order.  Row i (1..N) of the
    RHS is y(i-1) - 2 y(i) + y(i+1), built in FP64 and returned as FP32 (the
    storage precision of the mixed-precision path) with shape (N, M)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = torch.float64
    A = torch.rand((M, n_modes), generator=g, device=device, dtype=f64) * 2 - 1
    f = torch.rand((M, n_modes), generator=g, device=device, dtype=f64) * (N / 8.0)
    phi = torch.rand((M, n_modes), generator=g, device=device, dtype=f64) * (2 * math.pi)
    out = torch.empty((N, M), device=device, dtype=torch.float32)
    t = torch.arange(N + 2, device=device, dtype=f64).unsqueeze(1)  # (N+2, 1)
    for j0 in range(0, M, chunk):
        j1 = min(M, j0 + chunk)
        y = torch.zeros((N + 2, j1 - j0), device=device, dtype=f64)
        for k in range(n_modes):
            w = (2 * math.pi / N) * f[j0:j1, k]
            y += A[j0:j1, k] * torch.sin(t * w + phi[j0:j1, k])
        out[:, j0:j1] = (y[:-2] - 2 * y[1:-1] + y[2:]).to(torch.float32)
    return out


def adi_field(n: int = 4096, seed: int = 0, device="cpu", dtype=None):
    """(n, n) field u[y, x] ~ U(-1, 1)."""
    return uniform_rhs(n, n, seed, device, dtype)


# --------------------------------------------------------------------------
# Serving workload
# --------------------------------------------------------------------------


@dataclass
class LhsSpec:
    lhs_id: int
    width: int          # 3 or 5
    N: int
    bands: np.ndarray   # (width, N)


def serving_lhs(lhs_id: int, n_min: int = 64, n_max: int = 4096) -> LhsSpec:
    """LHS number ``lhs_id`` of the resident pool, seeded 1000 + lhs_id:
    width tri/penta Bernoulli(0.5), N = round(exp U(ln n_min, ln n_max)),
    bands diagonally dominant as in ``random_tri_bands``/``random_penta_bands``."""
    rng = np.random.default_rng(1000 + lhs_id)
    width = 3 if rng.uniform() < 0.5 else 5
    N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
    N = max(N, 4)
    bands = random_tri_bands(N, rng) if width == 3 else random_penta_bands(N, rng)
    return LhsSpec(lhs_id, width, N, bands)


@dataclass
class Request:
    rid: int
    arrival_s: float
    lhs_id: int
    M: int
    refine: bool        # FP32 storage + FP64 refinement if True, else FP64
    seed: int


def serving_requests(n: int, rate_hz: float, n_lhs: int = 256, m_max: int = 65536,
                     seed: int = 0):
    """Poisson arrivals at ``rate_hz``; LHS uniform over the pool; M =
    round(exp U(0, ln m_max)); precision Bernoulli(0.5).  Draw order per
    request: inter-arrival gap, LHS id, M, precision."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n):
        t += rng.exponential(1.0 / rate_hz) if rate_hz > 0 else 0.0
        lhs = int(rng.integers(0, n_lhs))
        M = int(round(math.exp(rng.uniform(0.0, math.log(m_max)))))
        refine = bool(rng.uniform() < 0.5)
        out.append(Request(r, t, lhs, max(M, 1), refine, seed * 1_000_003 + r))
    return out
