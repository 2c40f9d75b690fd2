"""Golden fixtures: the paper's printed coefficients (Sec. 3.2, Sec. 4.2),
its storage formulas (Sec. 3.1, Sec. 4.1), and a small oracle regression
fixture written by tests/golden/make_golden.py."""
import json
import os

import numpy as np

import oracle
import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_cn_hyperdiffusion_bands_match_paper():
    g = _load("paper_values.json")["cn_hyperdiffusion_penta"]["bands_in_sigma"]
    s = 0.1
    bands = synth.clamped_hyperdiffusion_bands(16, s, clamped=False)
    for k, name in enumerate("abcde"):
        p0, p1 = g[name]
        assert np.isclose(bands[k, 8], p0 + p1 * s)


def test_cn_diffusion_bands_match_paper():
    g = _load("paper_values.json")["cn_diffusion_tri"]["bands_in_sigma"]
    sigma = 0.7
    bands = synth.toeplitz_bands(9, (-sigma, 1 + 2 * sigma, -sigma))
    for k, name in enumerate("abc"):
        p0, p1 = g[name]
        assert np.isclose(bands[k, 4], p0 + p1 * sigma)


def test_storage_reductions_match_paper():
    g = _load("paper_values.json")["storage"]
    N, M = 512, 65536
    tri = 1 - (3 * N + M * N) / (4 * M * N)
    penta = 1 - (5 * N + M * N) / (6 * M * N)
    assert abs(tri - g["tri_reduction_approx"]) < 0.005
    assert abs(penta - g["penta_reduction_approx"]) < 0.005


def test_oracle_regression_fixture():
    doc = _load("oracle_small.json")
    for name, case in doc.items():
        X = oracle.solve(np.array(case["bands"]), np.array(case["B"]))
        ref = np.array(case["X"])
        assert np.max(np.abs(X - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref))), name
