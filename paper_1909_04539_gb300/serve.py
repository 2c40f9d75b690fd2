"""Python handle on the request server of libbsolve (``bs_server_*``):
continuous batching of shared-LHS solves with an HBM budget.  Marshalling
only -- admission, batching, graph replay and completion tracking run in the
library's worker thread."""
from __future__ import annotations

import ctypes

import torch

from ._lib import BsolveError, check, lib
from .api import Factor

F64 = 0
F32_REFINE = 1
STATES = {0: "queued", 1: "running", 2: "done", 3: "cancelled", 4: "failed"}
STAT_NAMES = ["batches", "completed", "failed", "queued", "running", "arena_used", "arena_peak", "arena_size",
              "max_batch_requests", "max_concurrent_batches"]


class Server:
    """``Server(hbm_budget_bytes, n_streams)`` on the current CUDA device."""

    def __init__(self, hbm_budget_bytes: int, n_streams: int = 4):
        h = ctypes.c_void_p()
        check(lib().bs_server_create(int(hbm_budget_bytes), int(n_streams), ctypes.byref(h)), "bs_server_create")
        self._h = h
        self._keep = {}  # request id -> host tensors kept alive until release

    def submit(self, f: Factor, B: torch.Tensor, X: torch.Tensor, mode: int) -> int:
        """Queue a solve of the interleaved (N, M) host batch B into host X
        (float64 for F64, float32 B + float64 X for F32_REFINE)."""
        for T, what in ((B, "B"), (X, "X")):
            if T.is_cuda or not T.is_contiguous() or T.dim() != 2 or T.shape[0] != f.N:
                raise ValueError(f"{what} must be a contiguous host (N, M) tensor")
        if X.dtype != torch.float64 or B.shape != X.shape:
            raise ValueError("X must be float64 with B's shape")
        want = torch.float64 if mode == F64 else torch.float32
        if B.dtype != want:
            raise ValueError(f"B must be {want} for this mode")
        rid = ctypes.c_int64()
        check(lib().bs_server_submit(self._h, f.handle, ctypes.c_void_p(B.data_ptr()),
                                     ctypes.c_void_p(X.data_ptr()), int(mode), int(B.shape[1]),
                                     ctypes.byref(rid)), "bs_server_submit")
        self._keep[rid.value] = (B, X, f)
        return rid.value

    def poll(self, rid: int):
        st, lat = ctypes.c_int(), ctypes.c_double()
        check(lib().bs_server_poll(self._h, rid, ctypes.byref(st), ctypes.byref(lat)), "bs_server_poll")
        return STATES[st.value], (lat.value if lat.value >= 0 else None)

    def wait(self, rid: int, timeout_s: float = 60.0) -> str:
        st = ctypes.c_int()
        check(lib().bs_server_wait(self._h, rid, float(timeout_s), ctypes.byref(st)), "bs_server_wait")
        return STATES[st.value]

    def cancel(self, rid: int) -> None:
        check(lib().bs_server_cancel(self._h, rid), "bs_server_cancel")

    def release(self, rid: int) -> None:
        check(lib().bs_server_release(self._h, rid), "bs_server_release")
        self._keep.pop(rid, None)

    def pause(self, paused: bool = True) -> None:
        check(lib().bs_server_pause(self._h, int(bool(paused))), "bs_server_pause")

    def fail_on_admit(self, rid: int) -> None:
        check(lib().bs_server_fail_on_admit(self._h, rid), "bs_server_fail_on_admit")

    def stats(self) -> dict:
        out = (ctypes.c_int64 * len(STAT_NAMES))()
        check(lib().bs_server_stats(self._h, out, len(STAT_NAMES)), "bs_server_stats")
        return dict(zip(STAT_NAMES, list(out)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            h, self._h = self._h, None
            lib().bs_server_destroy(h)
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Server", "F64", "F32_REFINE", "BsolveError"]
