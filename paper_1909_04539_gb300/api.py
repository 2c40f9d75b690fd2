"""Torch-facing wrappers of the C ABI (argument marshalling only).

Layouts: an interleaved batch is a contiguous tensor of shape (N, M) (row i
of system j at [i, j], the paper's B[i*M + j]); a strided batch has shape
(M, N) (system-contiguous).  Every call is enqueued on the current torch
CUDA stream unless ``stream`` is given.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import check, lib

_DTYPE = {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2}
_LAYOUT = {"interleaved": 0, "strided": 1}

OPT_INFLIGHT_BYTES = 0
OPT_BLOCKS_PER_SM = 1
OPT_SWEEP_KERNEL = 2
OPT_TMA_AHEAD = 3
OPT_PARTITION = 4
OPT_UNIFORM = 5
OPT_TWISTED = 6
OPT_CTA_THREADS = 7
OPT_F64_PAIRS = 8
OPT_WINDOW = 9


def device_status(reset: bool = False) -> int:
    """Sticky device status of the bounded-wait kernels (0 = fine)."""
    v = ctypes.c_int()
    check(lib().bs_device_status(ctypes.byref(v), int(bool(reset))), "bs_device_status")
    return int(v.value)


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def set_option(opt: int, value: int) -> None:
    check(lib().bs_set_option(int(opt), int(value)), "bs_set_option")


def measure_fp64_rate(stream=None) -> float:
    """FP64 FMA instructions per second of the current device (blocking)."""
    v = ctypes.c_double()
    check(lib().bs_measure_fp64_rate(ctypes.byref(v), _stream(stream)), "bs_measure_fp64_rate")
    return float(v.value)


def lhs_bytes(width: int, N: int, elem_bytes: int) -> int:
    return int(lib().bs_lhs_bytes(width, N, elem_bytes))


class Factor:
    """One factorised shared LHS resident on a device (``bs_factor``).

    ``bands``: (width, N) float64 array-like, width 3 (a, b, c) or 5
    (a, b, c, d, e), row-aligned as in the paper.  ``periodic=True`` (width 3
    only, ``bs_factor_periodic``): cyclic tridiagonal, a_1 is the top-right
    corner entry and c_N the bottom-left one."""

    def __init__(self, bands, device=None, periodic: bool = False):
        if isinstance(bands, torch.Tensor):
            bands = bands.detach().to("cpu", torch.float64).numpy()
        b = np.ascontiguousarray(np.asarray(bands, dtype=np.float64))
        if b.ndim != 2:
            raise ValueError("bands must be a (width, N) array")
        self.width, self.N = int(b.shape[0]), int(b.shape[1])
        self.periodic = bool(periodic)
        if self.periodic and self.width != 3:
            raise ValueError("a periodic factor is tridiagonal (width 3)")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("Factor lives on a CUDA device")
        self.device = dev
        h = ctypes.c_void_p()
        bp = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        with torch.cuda.device(dev):
            if self.periodic:
                check(lib().bs_factor_periodic(bp, self.N, ctypes.byref(h)), "bs_factor_periodic")
            else:
                check(lib().bs_factor(bp, self.width, self.N, ctypes.byref(h)), "bs_factor")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("Factor has been closed")
        return self._h

    @property
    def device_bytes(self) -> int:
        n = ctypes.c_size_t()
        check(lib().bs_handle_info(self.handle, None, None, ctypes.byref(n)), "bs_handle_info")
        return int(n.value)

    def close(self) -> None:
        """Release the device copy (bs_destroy); raises and keeps the handle
        while server requests that name it have not finished."""
        if getattr(self, "_h", None) is not None:
            check(lib().bs_destroy(self._h), "bs_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch(f: Factor, T: torch.Tensor, layout: str, what: str) -> int:
    if layout not in _LAYOUT:
        raise ValueError(f"layout must be one of {list(_LAYOUT)}")
    if not T.is_cuda or T.device != f.device:
        raise ValueError(f"{what} must be a CUDA tensor on {f.device}")
    if not T.is_contiguous() or T.dim() != 2:
        raise ValueError(f"{what} must be a contiguous 2-D tensor")
    N, M = (T.shape[0], T.shape[1]) if layout == "interleaved" else (T.shape[1], T.shape[0])
    if N != f.N:
        raise ValueError(f"{what} has {N} rows, the factor has N={f.N}")
    return int(M)


def solve(f: Factor, B: torch.Tensor, layout: str = "interleaved", stream=None) -> torch.Tensor:
    """In-place solve A X = B (float64: FP64 arithmetic; float32: FP32)."""
    M = _batch(f, B, layout, "B")
    if B.dtype not in (torch.float64, torch.float32):
        raise ValueError("B must be float64 or float32 (bfloat16: solve_bf16)")
    check(lib().bs_solve(f.handle, ctypes.c_void_p(B.data_ptr()), _DTYPE[B.dtype], _LAYOUT[layout], M,
                         _stream(stream)), "bs_solve")
    return B


def solve_bf16(f: Factor, B: torch.Tensor, X: torch.Tensor | None = None, layout: str = "interleaved",
               stream=None) -> torch.Tensor:
    """BF16-stored B, FP32 arithmetic, FP32 solution X (returned)."""
    M = _batch(f, B, layout, "B")
    if B.dtype != torch.bfloat16:
        raise ValueError("B must be bfloat16")
    if X is None:
        X = torch.empty(B.shape, dtype=torch.float32, device=B.device)
    _batch(f, X, layout, "X")
    if X.dtype != torch.float32 or X.shape != B.shape:
        raise ValueError("X must be float32 with B's shape")
    check(lib().bs_solve_bf16(f.handle, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                              _LAYOUT[layout], M, _stream(stream)), "bs_solve_bf16")
    return X


REFINE_FACTOR = 0
REFINE_SYSTEM = 1
REFINE_AUTO = 2


def solve_refine(f: Factor, B: torch.Tensor, X: torch.Tensor | None = None, refine_steps: int = 1,
                 layout: str = "interleaved", stream=None, mode: int = REFINE_AUTO) -> torch.Tensor:
    """FP32-stored (float32) or BF16-stored (bfloat16) B, FP32 sweeps plus
    ``refine_steps`` (0..8) steps of iterative refinement with FP64-accurate
    residuals (``mode`` for the first step: REFINE_FACTOR per triangular
    factor, two passes; REFINE_SYSTEM on r = B - A X0, three passes;
    REFINE_AUTO as REFINE_FACTOR, but small batches solved in FP64 from the
    widened input; further steps on the whole system); returns the FP64
    solution X (also used as workspace), in ``layout``."""
    M = _batch(f, B, layout, "B")
    if B.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("B must be float32 or bfloat16")
    if X is None:
        X = torch.empty(B.shape, dtype=torch.float64, device=B.device)
    _batch(f, X, layout, "X")
    if X.dtype != torch.float64 or X.shape != B.shape:
        raise ValueError("X must be float64 with B's shape")
    check(lib().bs_solve_refine(f.handle, ctypes.c_void_p(B.data_ptr()), _DTYPE[B.dtype],
                                ctypes.c_void_p(X.data_ptr()), _LAYOUT[layout], M, int(refine_steps),
                                int(mode), _stream(stream)), "bs_solve_refine")
    return X


def solve_adjoint(f: Factor, G: torch.Tensor, layout: str = "interleaved", X: torch.Tensor | None = None,
                  dbands: torch.Tensor | None = None, stream=None):
    """In-place G <- A^{-T} G.  With X (the primal solution) also returns the
    band gradient -(A^{-T} G) X^T on the bands, shape (width, N) float64."""
    M = _batch(f, G, layout, "G")
    if G.dtype not in (torch.float64, torch.float32):
        raise ValueError("G must be float64 or float32")
    xp = dp = None
    if X is not None:
        _batch(f, X, layout, "X")
        if X.dtype != G.dtype or X.shape != G.shape:
            raise ValueError("X must match G in dtype and shape")
        if dbands is None:
            dbands = torch.empty((f.width, f.N), dtype=torch.float64, device=G.device)
        if dbands.dtype != torch.float64 or not dbands.is_contiguous() or dbands.numel() != f.width * f.N:
            raise ValueError("dbands must be a contiguous float64 (width, N) tensor")
        xp, dp = ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(dbands.data_ptr())
    check(lib().bs_solve_adjoint(f.handle, ctypes.c_void_p(G.data_ptr()), _DTYPE[G.dtype], _LAYOUT[layout], M,
                                 xp, dp, _stream(stream)), "bs_solve_adjoint")
    return (G, dbands) if X is not None else G


def band_grad(f: Factor, GB: torch.Tensor, X: torch.Tensor, layout: str = "interleaved",
              dbands: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """-(GB) X^T on the bands, given GB = A^{-T} dL/dX; (width, N) float64."""
    M = _batch(f, GB, layout, "GB")
    _batch(f, X, layout, "X")
    if X.dtype != GB.dtype or X.shape != GB.shape or GB.dtype not in (torch.float64, torch.float32):
        raise ValueError("GB and X must be float64 or float32 tensors of one shape")
    if dbands is None:
        dbands = torch.empty((f.width, f.N), dtype=torch.float64, device=GB.device)
    if dbands.dtype != torch.float64 or not dbands.is_contiguous() or dbands.numel() != f.width * f.N:
        raise ValueError("dbands must be a contiguous float64 (width, N) tensor")
    check(lib().bs_band_grad(f.handle, ctypes.c_void_p(GB.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                             _DTYPE[GB.dtype], _LAYOUT[layout], M, ctypes.c_void_p(dbands.data_ptr()),
                             _stream(stream)), "bs_band_grad")
    return dbands


def cn_steps(f: Factor, C: torch.Tensor, steps: int = 1, layout: str = "interleaved", stream=None) -> torch.Tensor:
    """``steps`` Crank-Nicolson steps in place, C <- A^{-1} (2I - A) C (A the
    factor's matrix: the scheme's LHS I - (dt/2) L); float64 or float32."""
    M = _batch(f, C, layout, "C")
    if C.dtype not in (torch.float64, torch.float32):
        raise ValueError("C must be float64 or float32")
    check(lib().bs_cn_steps(f.handle, ctypes.c_void_p(C.data_ptr()), _DTYPE[C.dtype], _LAYOUT[layout], M,
                            int(steps), _stream(stream)), "bs_cn_steps")
    return C


def adi_halfstep(f: Factor, u: torch.Tensor, r: float, implicit_axis: int, out: torch.Tensor | None = None,
                 adjoint: bool = False, stream=None) -> torch.Tensor:
    """One Peaceman-Rachford half-step on the (ny, nx) field u (row-major,
    Dirichlet 0 outside): axis 0 solves along x with the explicit operator
    along y, axis 1 the other way round.  ``f`` factorises the implicit LHS
    (e.g. I - r d2 of the grid length along that axis).  ``adjoint`` applies
    the transposed map."""
    if u.dim() != 2 or not u.is_contiguous() or not u.is_cuda or u.device != f.device:
        raise ValueError("u must be a contiguous 2-D CUDA tensor on the factor's device")
    if u.dtype not in (torch.float64, torch.float32):
        raise ValueError("u must be float64 or float32")
    ny, nx = u.shape
    if out is None:
        out = torch.empty_like(u)
    if out.shape != u.shape or out.dtype != u.dtype or not out.is_contiguous() or out.device != u.device:
        raise ValueError("out must match u")
    check(lib().bs_adi_halfstep(f.handle, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                _DTYPE[u.dtype], ny, nx, float(r), int(implicit_axis), int(bool(adjoint)),
                                _stream(stream)), "bs_adi_halfstep")
    return out


class ADIHalfStepFn(torch.autograd.Function):
    """out = S^{-1} E u for one ADI half-step, differentiable in u; the
    backward pass is the transposed half-step (adjoint sweeps)."""

    @staticmethod
    def forward(ctx, u, factor, r, implicit_axis):
        ctx.factor, ctx.r, ctx.axis = factor, r, implicit_axis
        return adi_halfstep(factor, u.detach().contiguous(), r, implicit_axis)

    @staticmethod
    def backward(ctx, g):
        gu = adi_halfstep(ctx.factor, g.detach().contiguous(), ctx.r, ctx.axis, adjoint=True)
        return gu, None, None, None


class SolveFn(torch.autograd.Function):
    """X = A^{-1} B with gradients for B and for the band entries of A.

    ``SolveFn.apply(bands, B, factor=None, layout="interleaved", periodic=False)``:
    bands is a (width, N) float64 tensor (its values define A; pass ``factor``
    to reuse an existing factorisation of the same bands; ``periodic`` makes A
    cyclic tridiagonal, whose band gradient includes the two corners).  The
    backward pass is the hand-written adjoint: one transposed solve with the
    same factors plus the band-gradient reduction over the batch."""

    @staticmethod
    def forward(ctx, bands, B, factor=None, layout="interleaved", periodic=False):
        f = factor if factor is not None else Factor(bands.detach(), device=B.device, periodic=periodic)
        X = solve(f, B.detach().clone().contiguous(), layout)
        ctx.factor = f
        ctx.layout = layout
        ctx.bands_device = bands.device
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, gX):
        (X,) = ctx.saved_tensors
        GB = gX.detach().to(X.dtype).contiguous().clone()
        need_bands = ctx.needs_input_grad[0]
        if need_bands:
            GB, db = solve_adjoint(ctx.factor, GB, ctx.layout, X=X)
            db = db.to(ctx.bands_device)
        else:
            solve_adjoint(ctx.factor, GB, ctx.layout)
            db = None
        return db, (GB if ctx.needs_input_grad[1] else None), None, None, None
