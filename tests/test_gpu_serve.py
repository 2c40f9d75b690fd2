"""Request server: results against the oracle and bitwise against the direct
(unpartitioned) solves, the same whether a request runs alone or in a mix,
admission under a small HBM budget, and host-side failure handling
(oversized request, cancellation, a request that fails at admission, wait
time-outs)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    return m


@pytest.fixture(scope="module")
def serve(bs):
    from paper_1909_04539_gb300 import serve as sv
    return sv


def _lhs_pool(bs, n=6):
    specs = [synth.serving_lhs(i, 16, 600) for i in range(n)]
    return specs, [bs.Factor(s.bands) for s in specs]


def _request(spec, M, mode, seed):
    rng = np.random.default_rng(seed)
    B = torch.tensor(rng.uniform(-1, 1, (spec.N, M)), dtype=torch.float64 if mode == 0 else torch.float32)
    return B.pin_memory(), torch.empty((spec.N, M), dtype=torch.float64).pin_memory()


def test_mix_equals_alone_and_direct(bs, serve):
    specs, facs = _lhs_pool(bs)
    rng = np.random.default_rng(0)
    reqs = []
    for r in range(24):
        k = int(rng.integers(len(specs)))
        M = int(rng.integers(1, 3000))
        mode = int(rng.integers(2))
        reqs.append((k, M, mode, 100 + r))
    srv = serve.Server(1 << 30, n_streams=3)
    # the mix: everything submitted at once
    mix = []
    for k, M, mode, seed in reqs:
        B, X = _request(specs[k], M, mode, seed)
        mix.append((srv.submit(facs[k], B, X, mode), B, X))
    for rid, _, _ in mix:
        assert srv.wait(rid, 60) == "done"
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    # alone: one at a time
    for (k, M, mode, seed), (rid, B, X) in zip(reqs, mix):
        B2, X2 = _request(specs[k], M, mode, seed)
        r2 = srv.submit(facs[k], B2, X2, mode)
        assert srv.wait(r2, 60) == "done"
        assert torch.equal(X, X2), "result depends on the batch"
        # bitwise equal to the direct API's one-thread-per-system solve (a
        # small direct batch may otherwise run row-partitioned or two-ended,
        # equal to rounding), and right against the oracle
        bs.set_option(bs.OPT_PARTITION, 1)
        bs.set_option(bs.OPT_TWISTED, 1)
        try:
            if mode == 0:
                D = bs.solve(facs[k], B.cuda())
            else:
                D = bs.solve_refine(facs[k], B.cuda(), mode=bs.REFINE_FACTOR)
            torch.cuda.synchronize()
        finally:
            bs.set_option(bs.OPT_PARTITION, 0)
            bs.set_option(bs.OPT_TWISTED, 0)
        assert torch.equal(D.cpu(), X)  # same per-system arithmetic as the direct solves
        ref = oracle.solve(specs[k].bands, B.double().numpy())
        assert rel_l2(X.numpy(), ref) < 1e-12
    srv.close()


def test_admission_under_small_budget(bs, serve):
    """Requests totalling ~8x the budget all complete; the arena never holds
    more than the budget."""
    specs, facs = _lhs_pool(bs, 3)
    budget = 4 << 20
    srv = serve.Server(budget, n_streams=2)
    ids = []
    total = 0
    for r in range(40):
        k = r % 3
        M = 300 + 17 * r
        B, X = _request(specs[k], M, r % 2, r)
        total += specs[k].N * M * (8 if r % 2 == 0 else 12)
        ids.append((srv.submit(facs[k], B, X, r % 2), k, B, X))
    for rid, k, B, X in ids:
        assert srv.wait(rid, 120) == "done"
        assert rel_l2(X.numpy(), oracle.solve(specs[k].bands, B.double().numpy())) < 1e-12
    st = srv.stats()
    assert total > 4 * budget
    assert st["arena_peak"] <= budget and st["arena_used"] == 0
    srv.close()


def test_oversized_request_rejected(bs, serve):
    specs, facs = _lhs_pool(bs, 1)
    srv = serve.Server(1 << 20, n_streams=1)
    B, X = _request(specs[0], 20000, 0, 1)
    with pytest.raises(bs.BsolveError) as ei:
        srv.submit(facs[0], B, X, 0)
    assert ei.value.status == 3
    srv.close()


def test_cancel_failure_and_timeout(bs, serve):
    specs, facs = _lhs_pool(bs, 2)
    srv = serve.Server(64 << 20, n_streams=2)
    srv.pause(True)
    subs = []
    for r in range(6):
        B, X = _request(specs[r % 2], 500 + r, r % 2, 50 + r)
        subs.append((srv.submit(facs[r % 2], B, X, r % 2), r % 2, B, X))
    # nothing is admitted while paused: a bounded wait times out
    with pytest.raises(bs.BsolveError) as ei:
        srv.wait(subs[0][0], 0.2)
    assert ei.value.status == 5
    srv.cancel(subs[1][0])
    srv.fail_on_admit(subs[2][0])
    srv.pause(False)
    states = [srv.wait(rid, 60) for rid, _, _, _ in subs]
    assert states[1] == "cancelled" and states[2] == "failed"
    for (rid, k, B, X), s in zip(subs, states):
        if s == "done":
            assert rel_l2(X.numpy(), oracle.solve(specs[k].bands, B.double().numpy())) < 1e-12
    assert states.count("done") == 4
    with pytest.raises(bs.BsolveError):
        srv.cancel(subs[0][0])  # already finished
    st = srv.stats()
    assert st["failed"] == 1 and st["arena_used"] == 0
    srv.release(subs[0][0])
    with pytest.raises(bs.BsolveError):
        srv.poll(subs[0][0])
    srv.close()


def test_handle_pinned_while_requests_pending(bs, serve):
    """bs_destroy refuses a handle that queued server requests name (the
    worker would read its plans); once they finish or are cancelled it is
    released normally."""
    specs, facs = _lhs_pool(bs, 1)
    srv = serve.Server(1 << 28, n_streams=2)
    srv.pause(True)
    B, X = _request(specs[0], 64, 0, 1)
    rid = srv.submit(facs[0], B, X, 0)
    with pytest.raises(bs.BsolveError, match="have not finished"):
        facs[0].close()
    # the failed close left the handle usable: still registered
    assert facs[0].device_bytes > 0
    srv.cancel(rid)
    facs[0].close()
    srv.close()


def test_pageable_host_buffers_rejected(bs, serve):
    specs, facs = _lhs_pool(bs, 1)
    srv = serve.Server(1 << 26, n_streams=1)
    B = torch.zeros((specs[0].N, 8), dtype=torch.float64)  # not pinned
    X = torch.zeros((specs[0].N, 8), dtype=torch.float64).pin_memory()
    with pytest.raises(bs.BsolveError, match="page-locked"):
        srv.submit(facs[0], B, X, 0)
    srv.close()



@pytest.mark.parametrize("mode", [0, 1])
def test_large_request_paced_copies(bs, serve, mode):
    """A request larger than the copy window (four 8 MiB pieces) with small
    ones beside it: the copies are paced, every result still equals the
    direct solve bitwise."""
    specs, facs = _lhs_pool(bs, 3)
    k = max(range(3), key=lambda q: specs[q].N)
    M = (80 << 20) // (specs[k].N * 8) + 7
    srv = serve.Server(1 << 30, n_streams=3)
    subs = [(k, M, mode, 7)] + [(q % 3, 50 + q, q % 2, 20 + q) for q in range(6)]
    out = []
    for kk, MM, md, seed in subs:
        B, X = _request(specs[kk], MM, md, seed)
        out.append((srv.submit(facs[kk], B, X, md), kk, md, B, X))
    for rid, *_ in out:
        assert srv.wait(rid, 120) == "done"
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 1)
    try:
        for rid, kk, md, B, X in out:
            if md == 0:
                D = bs.solve(facs[kk], B.cuda())
            else:
                D = bs.solve_refine(facs[kk], B.cuda(), mode=bs.REFINE_FACTOR)
            torch.cuda.synchronize()
            assert torch.equal(D.cpu(), X)
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
        bs.set_option(bs.OPT_TWISTED, 0)
    srv.close()


@pytest.mark.parametrize("width", [3, 5])
def test_short_systems_through_the_rings(bs, serve, width):
    """Requests whose N is below, at and just above the grouped kernel's ring
    depth (16 rows) and not a multiple of its 4-row blocks: each result equals
    the direct solve bitwise and the oracle's to 1e-12."""
    Ns = [2, 3, 5, 7, 12, 15, 16, 17, 19, 21, 34] if width == 3 else [4, 5, 7, 12, 15, 16, 17, 19, 21, 34]
    rng = np.random.default_rng(width)
    facs = []
    for N in Ns:
        bands = synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)
        facs.append((bands, bs.Factor(bands)))
    srv = serve.Server(1 << 30, n_streams=2)
    out = []
    for q, (bands, f) in enumerate(facs):
        for mode in (0, 1):
            M = 1 + 37 * q + 5 * mode
            g = np.random.default_rng(1000 + 10 * q + mode)
            B = torch.tensor(g.uniform(-1, 1, (f.N, M)), dtype=torch.float64 if mode == 0 else torch.float32)
            B = B.pin_memory()
            X = torch.empty((f.N, M), dtype=torch.float64).pin_memory()
            out.append((srv.submit(f, B, X, mode), bands, f, mode, B, X))
    for rid, *_ in out:
        assert srv.wait(rid, 60) == "done"
    bs.set_option(bs.OPT_PARTITION, 1)
    bs.set_option(bs.OPT_TWISTED, 1)
    try:
        for rid, bands, f, mode, B, X in out:
            if mode == 0:
                D = bs.solve(f, B.cuda())
            else:
                D = bs.solve_refine(f, B.cuda(), mode=bs.REFINE_FACTOR)
            torch.cuda.synchronize()
            assert torch.equal(D.cpu(), X), (f.N, mode)
            ref = oracle.solve(bands, B.double().numpy())
            assert rel_l2(X.numpy(), ref) < 1e-12, (f.N, mode)
    finally:
        bs.set_option(bs.OPT_PARTITION, 0)
        bs.set_option(bs.OPT_TWISTED, 0)
    srv.close()
