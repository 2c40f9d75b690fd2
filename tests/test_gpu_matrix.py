"""Randomised GPU parity over the dispatch space: band width, N, M, storage
type, layout and the launch options (row partition, two-ended sweep,
uniform-scalar sweeps, on-chip TMA kernel) drawn from a fixed seed, each case
checked on sampled systems against the CPU FP64 oracle through the C ABI,
on the relative L2 error of the samples and the relative max-norm error of
each (tests.dense.parity): FP64 1e-12; FP32 / BF16-stored the FP32 bound of
the matrix (tests.dense.tol32) against the oracle on the rounded inputs;
refined FP32-stored 1e-12."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.dense import parity, tol32

pytestmark = pytest.mark.gpu

N_CASES = 200


def _cases():
    rng = np.random.default_rng(20260101)
    out = []
    for c in range(N_CASES):
        width = int(rng.choice([3, 5]))
        n_min = 2 if width == 3 else 4
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(6000)))))
        m_max = max(1, min(70000, 3_000_000 // N))
        M = int(round(math.exp(rng.uniform(0.0, math.log(m_max)))))
        op = str(rng.choice(["solve", "solve", "adjoint", "refine"]))
        dtype = str(rng.choice(["f64", "f32", "bf16"])) if op == "solve" else str(rng.choice(["f64", "f32"]))
        layout = "interleaved" if dtype == "bf16" or op == "refine" else str(rng.choice(["interleaved", "strided"]))
        opts = {"partition": int(rng.choice([0, 1, 2])), "twisted": int(rng.choice([0, 1, 2])),
                "uniform": int(rng.choice([0, 2])), "kernel": int(rng.choice([0, 0, 2])),
                "refine_mode": int(rng.choice([0, 1, 2])), "uniform_bands": bool(rng.uniform() < 0.3)}
        out.append((c, width, N, M, op, dtype, layout, opts))
    return out


@pytest.fixture(scope="module")
def bs():
    from paper_1909_04539_gb300 import build
    build.build()
    import paper_1909_04539_gb300 as m
    yield m
    for o in (m.OPT_PARTITION, m.OPT_TWISTED, m.OPT_UNIFORM, m.OPT_SWEEP_KERNEL):
        m.set_option(o, 0)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: f"c{c[0]}-w{c[1]}-N{c[2]}-M{c[3]}-{c[4]}-{c[5]}-{c[6]}")
def test_dispatch_matrix(bs, case):
    c, width, N, M, op, dtype, layout, opts = case
    rng = np.random.default_rng(1000 + c)
    if width == 5 and opts["uniform_bands"]:
        bands = synth.uniform_penta_bands(N, rng)
    else:
        bands = synth.random_tri_bands(N, rng) if width == 3 else synth.random_penta_bands(N, rng)
    f = bs.Factor(bands)
    B = rng.uniform(-1, 1, (N, M))
    cols = np.sort(rng.choice(M, min(M, 16), replace=False))
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    to_dev = (lambda A: A) if layout == "interleaved" else (lambda A: np.ascontiguousarray(A.T))
    from_dev = (lambda A: A) if layout == "interleaved" else (lambda A: A.T)
    bs.set_option(bs.OPT_PARTITION, opts["partition"])
    bs.set_option(bs.OPT_TWISTED, opts["twisted"])
    bs.set_option(bs.OPT_UNIFORM, opts["uniform"])
    bs.set_option(bs.OPT_SWEEP_KERNEL, opts["kernel"])
    try:
        Bd = torch.tensor(to_dev(B), device="cuda").to(tdt)
        Bin = from_dev(Bd.double().cpu().numpy())  # the values the GPU sees
        tol = 1e-12 if dtype == "f64" else tol32(bands)
        if op == "solve":
            if dtype == "bf16":
                X = bs.solve_bf16(f, Bd, layout=layout)
            else:
                X = bs.solve(f, Bd, layout)
            torch.cuda.synchronize()
            got = from_dev(X.double().cpu().numpy())[:, cols]
            parity(got, oracle.solve(bands, Bin[:, cols]), tol)
        elif op == "adjoint":
            X = bs.solve(f, Bd.clone(), layout)
            G = torch.tensor(to_dev(rng.uniform(-1, 1, (N, M))), device="cuda").to(tdt)
            Gin = from_dev(G.double().cpu().numpy())
            G, db = bs.solve_adjoint(f, G, layout, X=X)
            torch.cuda.synchronize()
            GB = from_dev(G.double().cpu().numpy())
            parity(GB[:, cols], oracle.solve_adjoint(bands, Gin[:, cols]), tol)
            db_ref = oracle.band_grad(width, GB, from_dev(X.double().cpu().numpy()))
            scale = max(np.max(np.abs(db_ref)), 1e-300)
            assert np.max(np.abs(db.cpu().numpy() - db_ref)) / scale < (1e-13 if dtype == "f64" else 1e-6)
        else:
            B32 = torch.tensor(B, dtype=torch.float32, device="cuda")
            X = bs.solve_refine(f, B32, mode=opts["refine_mode"])
            torch.cuda.synchronize()
            ref = oracle.solve(bands, B32.double().cpu().numpy()[:, cols])
            parity(X.cpu().numpy()[:, cols], ref, 1e-12)
    finally:
        for o in (bs.OPT_PARTITION, bs.OPT_TWISTED, bs.OPT_UNIFORM, bs.OPT_SWEEP_KERNEL):
            bs.set_option(o, 0)
    assert bs.device_status() == 0
