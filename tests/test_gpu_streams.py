"""Concurrent use of one handle from several CUDA streams (the handle is
immutable after factorisation, so solves on different streams may overlap):
an FP64 solve, an FP32 solve, a mixed-precision solve, an adjoint solve with
its band gradient and a row-partitioned small batch, all enqueued on four
streams before any is waited for, each compared bitwise with the same call
run alone and with the CPU FP64 oracle (tolerances as in the single-call
parity tests)."""
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


def _work(bs, f, inputs, streams):
    """Enqueues every job, job k on streams[k % len(streams)]; returns the
    output tensors (not yet synchronised)."""
    B64, B32, Br, G, X0, Bp = inputs
    outs = []
    jobs = [
        lambda s: (bs.solve(f, B64, stream=s),),
        lambda s: (bs.solve(f, B32, stream=s),),
        lambda s: (bs.solve_refine(f, Br, stream=s),),
        lambda s: bs.solve_adjoint(f, G, X=X0, stream=s),
        lambda s: (bs.solve(f, Bp, stream=s),),
    ]
    for k, job in enumerate(jobs):
        s = streams[k % len(streams)]
        with torch.cuda.stream(s):
            outs.append(job(s))
    return outs


def _inputs(bands, N, M, Mp, rng):
    B = rng.uniform(-1, 1, (N, M))
    Gh = rng.uniform(-1, 1, (N, M))
    X0h = oracle.solve(bands, B)
    Bph = rng.uniform(-1, 1, (N, Mp))
    return B, Gh, X0h, Bph


def _fresh(B, Gh, X0h, Bph):
    dev = "cuda"
    return (torch.tensor(B, device=dev), torch.tensor(B, dtype=torch.float32, device=dev),
            torch.tensor(B, dtype=torch.float32, device=dev), torch.tensor(Gh, device=dev),
            torch.tensor(X0h, device=dev), torch.tensor(Bph, device=dev))


@pytest.mark.parametrize("width", [3, 5])
def test_concurrent_streams_one_handle(bs, width):
    N, M, Mp = 1024, 8192, 96
    rng = np.random.default_rng(width)
    bands = synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)
    f = bs.Factor(bands)
    B, Gh, X0h, Bph = _inputs(bands, N, M, Mp, rng)
    # alone, one call at a time on the default stream
    ins = _fresh(B, Gh, X0h, Bph)
    alone = _work(bs, f, ins, [torch.cuda.current_stream()])
    torch.cuda.synchronize()
    # the same calls overlapping on four streams
    streams = [torch.cuda.Stream() for _ in range(4)]
    ins2 = _fresh(B, Gh, X0h, Bph)
    torch.cuda.synchronize()
    conc = _work(bs, f, ins2, streams)
    torch.cuda.synchronize()
    for a, c in zip(alone, conc):
        for ta, tc in zip(a, c):
            assert torch.equal(ta, tc)
    X64, X32, XR, (GB, db), Xp = conc[0][0], conc[1][0], conc[2][0], conc[3], conc[4][0]
    ref = oracle.solve(bands, B)
    parity(X64.cpu().numpy(), ref, 1e-12)
    ref_r = oracle.solve(bands, B.astype(np.float32).astype(np.float64))
    parity(X32.double().cpu().numpy(), ref_r, tol32(bands))
    parity(XR.cpu().numpy(), ref_r, 1e-12)
    GB_ref = oracle.solve_adjoint(bands, Gh)
    parity(GB.cpu().numpy(), GB_ref, 1e-12)
    db_ref = oracle.band_grad(width, GB_ref, X0h)
    assert np.max(np.abs(db.cpu().numpy() - db_ref)) / np.max(np.abs(db_ref)) < 1e-12
    assert rel_l2(Xp.cpu().numpy(), oracle.solve(bands, Bph)) < 1e-12
