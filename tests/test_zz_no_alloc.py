"""bs_band_grad_noalloc: the band-gradient reduction for callers that cannot
allocate device memory while they run (its scratch is a fixed array inside
the library).  Called through the C ABI twice in a row, it must agree with
bs_band_grad (which allocates its scratch per call): within the 1e-12
relative tolerance used for every FP64 result, and in fact bitwise, since
both run the same kernels in the same reduction order -- for FP64 and FP32
data, both layouts, and a periodic handle (column index wrapped); sizes
beyond its fixed array are refused.  Kept in a file of its own, collected
last."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1909_04539_gb300 import build
    build.build()
    from paper_1909_04539_gb300 import _lib
    return _lib.lib()


def _call(L, name, f, GB, X, db, layout=0):
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dtype = 0 if GB.dtype == torch.float64 else 1
    return getattr(L, name)(f.handle, ctypes.c_void_p(GB.data_ptr()), ctypes.c_void_p(X.data_ptr()), dtype, layout,
                            GB.shape[1] if layout == 0 else GB.shape[0], ctypes.c_void_p(db.data_ptr()), st)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("width,N,M,layout,periodic", [(5, 512, 20000, 0, False), (3, 77, 1003, 0, False),
                                                       (5, 64, 300, 1, False), (3, 129, 2049, 0, True),
                                                       (3, 40, 333, 1, True)])
def test_noalloc_matches_allocating_entry_point(lib, width, N, M, layout, periodic, dtype):
    import paper_1909_04539_gb300 as bs
    rng = np.random.default_rng(N + M)
    if periodic:
        bands = synth.random_periodic_bands(N, rng)
    else:
        bands = synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)
    f = bs.Factor(bands, periodic=periodic)
    shape = (N, M) if layout == 0 else (M, N)
    GB = torch.tensor(rng.uniform(-1, 1, shape), device="cuda", dtype=dtype)
    X = torch.tensor(rng.uniform(-1, 1, shape), device="cuda", dtype=dtype)
    ref = torch.empty((width, N), dtype=torch.float64, device="cuda")
    assert _call(lib, "bs_band_grad", f, GB, X, ref, layout) == 0
    for _ in range(2):  # two calls in a row share the fixed scratch
        out = torch.full((width, N), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, "bs_band_grad_noalloc", f, GB, X, out, layout) == 0
        torch.cuda.synchronize()
        err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-12, err
        assert torch.equal(out, ref)


def test_noalloc_refuses_sizes_beyond_its_array(lib):
    import paper_1909_04539_gb300 as bs
    N = 60000  # needs 5 x 60000 doubles of partial sums, more than the 262144 held
    f = bs.Factor(synth.random_penta_bands(N, np.random.default_rng(0)))
    GB = torch.zeros((N, 4), dtype=torch.float64, device="cuda")
    db = torch.zeros((5, N), dtype=torch.float64, device="cuda")
    assert _call(lib, "bs_band_grad_noalloc", f, GB, GB, db) == 1
    assert b"fixed array" in lib.bs_last_error()


def test_noalloc_refuses_n_times_m_overflow(lib):
    """The same N*M bound as the allocating entry point."""
    import paper_1909_04539_gb300 as bs
    f = bs.Factor(synth.random_tri_bands(8, np.random.default_rng(1)))
    GB = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    db = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    huge = (1 << 62) // 8
    p = ctypes.c_void_p(GB.data_ptr())
    assert lib.bs_band_grad_noalloc(f.handle, p, p, 0, 0, huge, ctypes.c_void_p(db.data_ptr()), st) == 1
    assert b"too large" in lib.bs_last_error()
